// div B norms of caller-owned face fields without any allocation.
//
// grmhd_diagnostics needs a context, and a context needs caller-allocated scratch
// for its reduction rows.  Some callers cannot allocate device memory at the point
// where they want this check: a host that has handed all device memory to its own
// pool or arena, a real-time loop that forbids allocation after start-up, or code
// running inside a framework that owns the allocator.  For them this file provides
// one entry point whose only scratch is a fixed array in the library's own device
// memory.  The paper has no counterpart to this call.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/grmhd.h"
#include "grmhd_device.cuh"

namespace grmhd {
void set_last_error(const char* msg);  // message for grmhd_last_error (capi.cu)
}

namespace {

using grmhd::CP3;
using grmhd::Dims;

constexpr int kThreads = 256;                  // one interior cell per thread
constexpr int kMaxRows = 8192;                 // one row of partial sums per block
constexpr int kRowWidth = 3;                   // sum |div|, sum div^2, max |div|
constexpr int kMaxDevices = 64;

// Library-owned scratch: kMaxRows x 3 doubles = 192 KiB, held on every GPU that loads
// the library until the process exits.  In host code the name is only a stand-in for
// the device object; kernels receive the address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_divb_rows[kMaxRows * kRowWidth];

double* g_rows_addr[kMaxDevices] = {nullptr};
std::mutex g_rows_mu;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// each block writes its whole row, so no part of the array needs clearing
__global__ void __launch_bounds__(kThreads) k_divb_rows(Dims g, CP3 bf, double* __restrict__ rows)
{
    __shared__ double sh[3][kThreads / 32];
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long t = blockIdx.x * (long long)kThreads + threadIdx.x;
    double a = 0.0, s = 0.0, m = 0.0;
    if (t < tot) {
        int c[3];
        grmhd::interior_coords(g, t, c);
        const long long o = grmhd::lin(g, c[0], c[1], c[2]);
        const double dv = grmhd::cell_divb(g, bf.p, c, o);
        a = fabs(dv);
        s = dv * dv;
        m = fabs(dv);
    }
    a = warp_sum(a);
    s = warp_sum(s);
    m = warp_max(m);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[0][w] = a;
        sh[1][w] = s;
        sh[2][w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ra = 0.0, rs = 0.0, rm = 0.0;
        for (int k = 0; k < kThreads / 32; k++) {
            ra += sh[0][k];
            rs += sh[1][k];
            rm = fmax(rm, sh[2][k]);
        }
        rows[blockIdx.x * kRowWidth + 0] = ra;
        rows[blockIdx.x * kRowWidth + 1] = rs;
        rows[blockIdx.x * kRowWidth + 2] = rm;
    }
}

__global__ void __launch_bounds__(kThreads) k_divb_fold(const double* __restrict__ rows, int nrows, double ncell,
                                                      double* __restrict__ out)
{
    __shared__ double sh[3][kThreads / 32];
    double a = 0.0, s = 0.0, m = 0.0;
    for (int r = threadIdx.x; r < nrows; r += kThreads) {
        a += rows[r * kRowWidth + 0];
        s += rows[r * kRowWidth + 1];
        m = fmax(m, rows[r * kRowWidth + 2]);
    }
    a = warp_sum(a);
    s = warp_sum(s);
    m = warp_max(m);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[0][w] = a;
        sh[1][w] = s;
        sh[2][w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ra = 0.0, rs = 0.0, rm = 0.0;
        for (int k = 0; k < kThreads / 32; k++) {
            ra += sh[0][k];
            rs += sh[1][k];
            rm = fmax(rm, sh[2][k]);
        }
        out[0] = ra / ncell;
        out[1] = sqrt(rs / ncell);
        out[2] = rm;
    }
}

grmhd_status err(grmhd_status s, const char* msg)
{
    grmhd::set_last_error(msg);
    return s;
}

// address of g_divb_rows on the current device, looked up once per device (on the
// first call with that device current) and kept until the process exits.  A device
// reset unloads the module, so the kept address is stale afterwards: a process that
// resets a device must not call grmhd_divb_noalloc on it again.
grmhd_status rows_address(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(GRMHD_ERR_CUDA, "grmhd_divb_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return err(GRMHD_ERR_ARG, "grmhd_divb_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_rows_mu);
    if (!g_rows_addr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_divb_rows);
        if (e != cudaSuccess || !p) return err(GRMHD_ERR_CUDA, "grmhd_divb_noalloc: cudaGetSymbolAddress failed");
        g_rows_addr[dev] = p;
    }
    *out = g_rows_addr[dev];
    return GRMHD_OK;
}

}  // namespace

extern "C" grmhd_status grmhd_divb_noalloc(const grmhd_grid* grid, const double* const* bface, double* out,
                                           grmhd_stream_t stream)
{
    if (!grid || !bface || !out) return err(GRMHD_ERR_ARG, "grmhd_divb_noalloc: NULL argument");
    if (grid->ndim < 1 || grid->ndim > 3) return err(GRMHD_ERR_ARG, "grmhd_divb_noalloc: ndim must be 1, 2 or 3");
    Dims g;
    g.ncell = 1;
    long long cells = 1;
    for (int d = 0; d < 3; d++) {
        g.act[d] = d < grid->ndim;
        if (g.act[d]) {
            if (grid->n[d] < 1 || !std::isfinite(grid->lo[d]) || !std::isfinite(grid->hi[d]) ||
                !(grid->hi[d] > grid->lo[d]) || !std::isfinite(grid->n[d] / (grid->hi[d] - grid->lo[d])) ||
                grid->bc[d] < 0 || grid->bc[d] > 2)
                return err(GRMHD_ERR_ARG,
                           "grmhd_divb_noalloc: invalid grid (n >= 1, finite lo < hi with finite n/(hi-lo), bc 0..2)");
            if (grid->bc[d] == GRMHD_BC_PERIODIC && grid->n[d] < 2)
                return err(GRMHD_ERR_ARG, "grmhd_divb_noalloc: a periodic direction needs at least 2 cells");
        }
        g.n[d] = g.act[d] ? grid->n[d] : 1;
        g.ng[d] = g.act[d] ? 2 : 0;
        g.N[d] = g.n[d] + 2 * g.ng[d];
        g.bc[d] = g.act[d] ? grid->bc[d] : GRMHD_BC_PERIODIC;
        g.idx[d] = g.act[d] ? g.n[d] / (grid->hi[d] - grid->lo[d]) : 0.0;
        g.ncell *= g.N[d];
        cells *= g.n[d];
    }
    g.st[0] = 1;
    g.st[1] = g.N[0];
    g.st[2] = (long long)g.N[0] * g.N[1];
    g.gh = g.igh = 0.0;
    grmhd::set_divisors(g);
    const long long rows = (cells + kThreads - 1) / kThreads;
    if (rows > kMaxRows)
        return err(GRMHD_ERR_ARG,
                   "grmhd_divb_noalloc: grid too large: at most 8192 * 256 = 2097152 interior cells");
    double* scratch = nullptr;
    grmhd_status s = rows_address(&scratch);
    if (s != GRMHD_OK) return s;
    CP3 bf;
    for (int d = 0; d < 3; d++) {
        // an inactive direction's array is never read and may be NULL
        if (g.act[d] && !bface[d]) return err(GRMHD_ERR_ARG, "grmhd_divb_noalloc: bface[d] is NULL for an active d");
        bf.p[d] = g.act[d] ? bface[d] : nullptr;
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_divb_rows<<<(unsigned)rows, kThreads, 0, st>>>(g, bf, scratch);
    k_divb_fold<<<1, kThreads, 0, st>>>(scratch, (int)rows, (double)cells, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(GRMHD_ERR_CUDA, "grmhd_divb_noalloc: kernel launch failed");
    return GRMHD_OK;
}

namespace grmhd {
GRMHD_OOB_READER(oob_noalloc)
}  // namespace grmhd
