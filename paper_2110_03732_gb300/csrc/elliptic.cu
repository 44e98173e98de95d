// Elliptic divergence cleaning (arXiv 2110.03732 Sec. 3.3) by geometric multigrid,
// sm_103a, FP64: solve lap(Phi) = div q_B and set q_B <- q_B - grad(Phi).
//
// Operators (Cartesian reference metric, so flat):
//   staggered fields (CT): div on cells from face differences, grad on faces from the
//     two adjacent cells; lap = div(grad) is the compact (2 ndim + 1)-point stencil and
//     the cleaned field is divergence-free to the solver's accuracy;
//   cell-centred fields (GLM): div and grad by central differences with the same
//     compact lap (an approximate projection).
//   Periodic directions wrap; in the others Phi has zero normal gradient (no flux
//   through the boundary face, which is not corrected).  The right-hand side is made
//   mean-free (the constants are the null space).
//
// Multigrid: cell-centred levels, each halving every active extent while all of them
// are even and at least 4.  V(2,2) cycles: red-black Gauss-Seidel smoothing (valid,
// hence deterministic, because every level but the coarsest has even extents), the
// residual of the 2^ndim children averaged to the coarse cell, tensor-product linear
// interpolation (weights 3/4, 1/4) back.  The coarsest level (at most 4096 cells) is
// solved by conjugate gradients in one thread block with fixed-order reductions and
// a bounded iteration count.  Every launch is deterministic; the cycle count is fixed
// by the caller, so a cleaning is launches only (no host synchronisation).
#include <cuda_runtime.h>

#include "elliptic.h"
#include "grmhd_device.cuh"

namespace grmhd {

namespace {

// cell (i, j, k) of a level, x fastest; returns the neighbour's index along d (side s =
// +-1), or -1 past a non-periodic boundary
__device__ __forceinline__ long long mg_nb(const MgLevel& L, const int* bc, int i, int j, int k, int d, int s)
{
    int c[3] = {i, j, k};
    c[d] += s;
    if (c[d] < 0 || c[d] >= L.n[d]) {
        if (bc[d] != BC_PERIODIC) return -1;
        c[d] = (c[d] + L.n[d]) % L.n[d];
    }
    return c[0] + (long long)L.n[0] * (c[1] + (long long)L.n[1] * c[2]);
}

struct MgArgs {
    int bc[3];
    int act[3];
};

// cell (i, j, k) of level item t (levels hold fewer than 2^31 cells: mg_plan)
__device__ __forceinline__ void mg_coords(const MgLevel& L, long long t, int& i, int& j, int& k)
{
    const int u = (int)t;
    const int r = u / L.n[0];
    i = u - r * L.n[0];
    j = r % L.n[1];
    k = r / L.n[1];
}

// (L Phi)_c split as sum_nb Phi_nb / h^2 - diag Phi_c; returns the neighbour sum, the
// diagonal and the number of neighbours missing past non-periodic boundaries (0: the
// full stencil, whose diagonal is the level's dfull)
__device__ __forceinline__ void mg_stencil(const MgLevel& L, const MgArgs& m, const double* __restrict__ phi, int i,
                                           int j, int k, double& nbsum, double& diag, int& miss)
{
    nbsum = 0.0;
    miss = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!m.act[d]) continue;
        const long long lo = mg_nb(L, m.bc, i, j, k, d, -1), hi = mg_nb(L, m.bc, i, j, k, d, 1);
        double s2;
        if (lo >= 0 && hi >= 0) {
            s2 = phi[lo] + phi[hi];
        } else {
            s2 = lo >= 0 ? phi[lo] : (hi >= 0 ? phi[hi] : 0.0);
            miss += (lo < 0) + (hi < 0);
        }
        nbsum += s2 * L.ih2[d];
    }
    diag = L.dfull;
    if (miss) {
        diag = 0.0;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (!m.act[d]) continue;
            if (mg_nb(L, m.bc, i, j, k, d, -1) >= 0) diag += L.ih2[d];
            if (mg_nb(L, m.bc, i, j, k, d, 1) >= 0) diag += L.ih2[d];
        }
    }
}

// cells of colour `color` ((i + j + k) & 1) of a level, enumerated x fastest: item t
// is the u-th such cell of row (j, k), u = t mod ceil(n_x / 2)
__device__ __forceinline__ long long mg_half_items(const MgLevel& L)
{
    return (long long)((L.n[0] + 1) >> 1) * L.n[1] * L.n[2];
}

// red-black Gauss-Seidel update of item t of colour `color`.  The full stencil's
// diagonal reciprocal is the level's; a boundary cell (fewer neighbours) divides.
__device__ __forceinline__ void mg_smooth_cell(const MgLevel& L, const MgArgs& m, int color, long long t)
{
    const int h0 = (L.n[0] + 1) >> 1;
    const int u = (int)t, row = u / h0;
    const int j = row % L.n[1], k = row / L.n[1];
    const int i = 2 * (u - row * h0) + ((color + j + k) & 1);
    if (i >= L.n[0]) return;
    const int c = i + L.n[0] * row;
    double nbsum, diag;
    int miss;
    mg_stencil(L, m, L.phi, i, j, k, nbsum, diag, miss);
    if (!miss) L.phi[c] = (nbsum - L.rhs[c]) * L.idiag;
    else if (diag > 0.0) L.phi[c] = (nbsum - L.rhs[c]) / diag;
}

__global__ void __launch_bounds__(256) k_mg_smooth(MgLevel L, MgArgs m, int color)
{
    const long long items = mg_half_items(L);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < items;
         t += (long long)gridDim.x * blockDim.x)
        mg_smooth_cell(L, m, color, t);
}

// coarse rhs of cell t = mean of its children's residuals rhs - L Phi; coarse Phi = 0
__device__ __forceinline__ void mg_restrict_cell(const MgLevel& F, const MgLevel& C, const MgArgs& m, long long t)
{
    {
        int I, J, K;
        mg_coords(C, t, I, J, K);
        double sum = 0.0;
        for (int dk = 0; dk <= m.act[2]; dk++)
            for (int dj = 0; dj <= m.act[1]; dj++)
                for (int di = 0; di <= m.act[0]; di++) {
                    const int i = 2 * I * m.act[0] + di, j = 2 * J * m.act[1] + dj, k = 2 * K * m.act[2] + dk;
                    const long long f = i + (long long)F.n[0] * (j + (long long)F.n[1] * k);
                    double nbsum, diag;
                    int miss;
                    mg_stencil(F, m, F.phi, i, j, k, nbsum, diag, miss);
                    sum += F.rhs[f] - (nbsum - diag * F.phi[f]);
                }
        // 1 / (number of children), a power of two
        C.rhs[t] = sum * ((m.act[0] ? 0.5 : 1.0) * (m.act[1] ? 0.5 : 1.0) * (m.act[2] ? 0.5 : 1.0));
        C.phi[t] = 0.0;
    }
}

__global__ void __launch_bounds__(256) k_mg_restrict(MgLevel F, MgLevel C, MgArgs m)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < C.cells;
         t += (long long)gridDim.x * blockDim.x)
        mg_restrict_cell(F, C, m, t);
}

// Phi_fine += linear interpolation of the coarse correction: along each active
// direction the child takes 3/4 of its parent and 1/4 of the parent's neighbour on its
// side (the parent itself past a non-periodic boundary)
__device__ __forceinline__ void mg_prolong_cell(const MgLevel& F, const MgLevel& C, const MgArgs& m, long long t)
{
    {
        int c[3];
        mg_coords(F, t, c[0], c[1], c[2]);
        int P[3], S[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            P[d] = m.act[d] ? c[d] >> 1 : c[d];
            S[d] = m.act[d] ? ((c[d] & 1) ? 1 : -1) : 0;
        }
        double v = 0.0;
        for (int ok = 0; ok <= m.act[2]; ok++)
            for (int oj = 0; oj <= m.act[1]; oj++)
                for (int oi = 0; oi <= m.act[0]; oi++) {
                    const int off[3] = {oi, oj, ok};
                    int q[3];
                    double w = 1.0;
                    for (int d = 0; d < 3; d++) {
                        if (!m.act[d]) { q[d] = P[d]; continue; }
                        q[d] = P[d] + off[d] * S[d];
                        w *= off[d] ? 0.25 : 0.75;
                        if (q[d] < 0 || q[d] >= C.n[d]) {
                            if (m.bc[d] == BC_PERIODIC) q[d] = (q[d] + C.n[d]) % C.n[d];
                            else q[d] = P[d];
                        }
                    }
                    v += w * C.phi[q[0] + (long long)C.n[0] * (q[1] + (long long)C.n[1] * q[2])];
                }
        F.phi[t] += v;
    }
}

__global__ void __launch_bounds__(256) k_mg_prolong(MgLevel F, MgLevel C, MgArgs m)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < F.cells;
         t += (long long)gridDim.x * blockDim.x)
        mg_prolong_cell(F, C, m, t);
}

// fixed-order block sum (blockDim.x a multiple of 32, at most 1024)
__device__ __forceinline__ double mg_block_sum(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) sh[32] = v;
    }
    __syncthreads();
    return sh[32];
}

// coarsest level: conjugate gradients on -lap (symmetric positive semi-definite) with
// a mean-free right-hand side, in one block.  r, p and q are scratch vectors of the
// level's size; iterations end at ||r|| <= 1e-15 ||b|| or after max_it.
__device__ __forceinline__ void mg_cg_block(const MgLevel& L, const MgArgs& m, double* __restrict__ res,
                                            double* __restrict__ p, double* __restrict__ q, int max_it, double* sh)
{
    const long long n = L.cells;
    // b = -(rhs - mean rhs); x = 0, r = b, p = r
    double s = 0.0;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) s += L.rhs[t];
    const double mean = mg_block_sum(s, sh) / (double)n;
    double rr = 0.0;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) {
        const double b = -(L.rhs[t] - mean);
        res[t] = b;
        p[t] = b;
        L.phi[t] = 0.0;
        rr += b * b;
    }
    rr = mg_block_sum(rr, sh);
    const double stop = 1e-30 * rr;
    for (int it = 0; it < max_it && rr > stop && rr > 0.0; it++) {
        // q = -lap p
        double pq = 0.0;
        for (long long t = threadIdx.x; t < n; t += blockDim.x) {
            int i, j, k;
            mg_coords(L, t, i, j, k);
            double nbsum, diag;
            int miss;
            mg_stencil(L, m, p, i, j, k, nbsum, diag, miss);
            const double v = diag * p[t] - nbsum;
            q[t] = v;
            pq += p[t] * v;
        }
        pq = mg_block_sum(pq, sh);
        if (!(pq > 0.0)) break;
        const double alpha = rr / pq;
        double rn = 0.0;
        for (long long t = threadIdx.x; t < n; t += blockDim.x) {
            L.phi[t] += alpha * p[t];
            const double r = res[t] - alpha * q[t];
            res[t] = r;
            rn += r * r;
        }
        rn = mg_block_sum(rn, sh);
        const double beta = rn / rr;
        rr = rn;
        for (long long t = threadIdx.x; t < n; t += blockDim.x) p[t] = res[t] + beta * p[t];
        __syncthreads();
    }
    __syncthreads();
}

// the levels first..nlev-1 (each at most kMgBlockCells cells) of one V-cycle in a
// single block: down-leg smoothing and restriction, conjugate gradients on the
// coarsest, up-leg interpolation and smoothing -- the same updates in the same order
// as the one-launch-per-step form, with block barriers in place of launches.  With
// smem set the block moves these levels and the CG vectors into dynamic shared memory
// (level `first` in from its global arrays at the start, its Phi back at the end).
struct MgTail {
    MgLevel lev[kMgMaxLevels];
    long long soff[kMgMaxLevels];   // with smem: offset (doubles) of each tail level's
                                    // Phi (its rhs follows) in the shared block
    long long scg;                  // with smem: offset of the CG vectors r, p, q
    int first, nlev;
    int smem;
};

// level l of the tail with its arrays where the block keeps them (a register copy: the
// kernel's parameter block itself is never written, which would move it to local memory)
__device__ __forceinline__ MgLevel tail_level(const MgTail& T, int l, double* sm)
{
    MgLevel L = T.lev[l];
    if (T.smem) {
        L.phi = sm + T.soff[l];
        L.rhs = L.phi + L.cells;
    }
    return L;
}

__global__ void __launch_bounds__(1024) k_mg_tail(MgTail T, MgArgs m, double* __restrict__ res,
                                                   double* __restrict__ p, double* __restrict__ q, int max_it)
{
    extern __shared__ double tail_sm[];
    __shared__ double sh[33];
    if (T.smem) {
        const MgLevel G = T.lev[T.first];
        const MgLevel L = tail_level(T, T.first, tail_sm);
        for (long long t = threadIdx.x; t < L.cells; t += blockDim.x) {
            L.phi[t] = G.phi[t];
            L.rhs[t] = G.rhs[t];
        }
        const long long nc = T.lev[T.nlev - 1].cells;
        res = tail_sm + T.scg;
        p = res + nc;
        q = p + nc;
        __syncthreads();
    }
    for (int l = T.first; l + 1 < T.nlev; l++) {
        const MgLevel L = tail_level(T, l, tail_sm), C = tail_level(T, l + 1, tail_sm);
        const long long items = mg_half_items(L);
        for (int s = 0; s < 2; s++)
            for (int color = 0; color < 2; color++) {
                for (long long t = threadIdx.x; t < items; t += blockDim.x) mg_smooth_cell(L, m, color, t);
                __syncthreads();
            }
        for (long long t = threadIdx.x; t < C.cells; t += blockDim.x) mg_restrict_cell(L, C, m, t);
        __syncthreads();
    }
    mg_cg_block(tail_level(T, T.nlev - 1, tail_sm), m, res, p, q, max_it, sh);
    for (int l = T.nlev - 2; l >= T.first; l--) {
        const MgLevel L = tail_level(T, l, tail_sm), C = tail_level(T, l + 1, tail_sm);
        for (long long t = threadIdx.x; t < L.cells; t += blockDim.x) mg_prolong_cell(L, C, m, t);
        __syncthreads();
        const long long items = mg_half_items(L);
        for (int s = 0; s < 2; s++)
            for (int color = 0; color < 2; color++) {
                for (long long t = threadIdx.x; t < items; t += blockDim.x) mg_smooth_cell(L, m, color, t);
                __syncthreads();
            }
    }
    if (T.smem) {
        const MgLevel G = T.lev[T.first];
        const MgLevel L = tail_level(T, T.first, tail_sm);
        for (long long t = threadIdx.x; t < L.cells; t += blockDim.x) G.phi[t] = L.phi[t];
    }
}

// fine right-hand side: div q_B on the interior cells (faces or central), and block
// partial sums for its mean
__global__ void __launch_bounds__(256) k_mg_div(Dims g, CP3 bq, int cc, MgLevel L, MgArgs m, double* __restrict__ part)
{
    __shared__ double sh[33];
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L.cells;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        mg_coords(L, t, c[0], c[1], c[2]);
        int p[3] = {c[0] + g.ng[0], c[1] + g.ng[1], c[2] + g.ng[2]};
        const long long o = lin(g, p[0], p[1], p[2]);
        double dv = 0.0;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (!g.act[d]) continue;
            if (cc) {
                // central difference; past a non-periodic boundary the cell itself (zero
                // gradient, whatever the boundary kind)
                const long long hi = mg_nb(L, m.bc, c[0], c[1], c[2], d, 1);
                const long long lo = mg_nb(L, m.bc, c[0], c[1], c[2], d, -1);
                int ch[3] = {c[0], c[1], c[2]}, cl[3] = {c[0], c[1], c[2]};
                if (hi >= 0) ch[d] = (c[d] + 1) % L.n[d];
                if (lo >= 0) cl[d] = (c[d] - 1 + L.n[d]) % L.n[d];
                const double vh = bq.p[d][lin(g, ch[0] + g.ng[0], ch[1] + g.ng[1], ch[2] + g.ng[2])];
                const double vl = bq.p[d][lin(g, cl[0] + g.ng[0], cl[1] + g.ng[1], cl[2] + g.ng[2])];
                dv += (vh - vl) * (0.5 * g.idx[d]);
            } else {
                int up[3] = {p[0], p[1], p[2]};
                up[d] += 1;
                dv += (bq.p[d][face_at(g, d, up)] - bq.p[d][o]) * g.idx[d];
            }
        }
        L.rhs[t] = dv;
        L.phi[t] = 0.0;
        s += dv;
    }
    s = mg_block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// mean of the partial sums (one block), subtracted from the fine right-hand side
__global__ void __launch_bounds__(256) k_mg_mean(const double* __restrict__ part, int nb, double* __restrict__ mean,
                                                 long long cells)
{
    __shared__ double sh[33];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    s = mg_block_sum(s, sh);
    if (threadIdx.x == 0) *mean = s / (double)cells;
}

__global__ void __launch_bounds__(256) k_mg_sub_mean(MgLevel L, const double* __restrict__ mean)
{
    const double mu = *mean;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L.cells;
         t += (long long)gridDim.x * blockDim.x)
        L.rhs[t] -= mu;
}

// q_B -= grad Phi: staggered (lower face of each interior cell; the lower boundary face
// of a non-periodic direction is kept) or central (cell-centred)
__global__ void __launch_bounds__(256) k_mg_correct(Dims g, P3 bq, int cc, MgLevel L, MgArgs m)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L.cells;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        mg_coords(L, t, c[0], c[1], c[2]);
        const long long o = lin(g, c[0] + g.ng[0], c[1] + g.ng[1], c[2] + g.ng[2]);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (!g.act[d]) continue;
            const long long lo = mg_nb(L, m.bc, c[0], c[1], c[2], d, -1);
            if (cc) {
                const long long hi = mg_nb(L, m.bc, c[0], c[1], c[2], d, 1);
                const double pl = lo < 0 ? L.phi[t] : L.phi[lo];
                const double ph = hi < 0 ? L.phi[t] : L.phi[hi];
                bq.p[d][o] -= (ph - pl) * (0.5 * g.idx[d]);
            } else if (lo >= 0) {
                bq.p[d][o] -= (L.phi[t] - L.phi[lo]) * g.idx[d];
            }
        }
    }
}

// items of one colour of a level (mg_half_items on the host)
long long half_items(const MgLevel& L)
{
    return (long long)((L.n[0] + 1) / 2) * L.n[1] * L.n[2];
}

int mg_grid(long long work, int nsm)
{
    long long b = (work + 255) / 256;
    const long long cap = (long long)nsm * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int mg_plan(const Dims& g, MgPlan* plan)
{
    MgPlan p;
    p.nlev = 0;
    int n[3] = {g.n[0], g.n[1], g.n[2]};
    long long total = 0;
    for (;;) {
        if (p.nlev >= kMgMaxLevels) return -1;
        MgLevel& L = p.lev[p.nlev];
        long long cells = 1;
        for (int d = 0; d < 3; d++) {
            L.n[d] = n[d];
            const double h = g.act[d] ? (1.0 / g.idx[d]) * (double)(g.n[d] / n[d]) : 1.0;
            L.ih2[d] = g.act[d] ? 1.0 / (h * h) : 0.0;
            cells *= n[d];
        }
        // the device's summation order: per active direction, its two neighbours
        L.dfull = 0.0;
        for (int d = 0; d < 3; d++)
            if (g.act[d]) {
                L.dfull += L.ih2[d];
                L.dfull += L.ih2[d];
            }
        L.idiag = L.dfull > 0.0 ? 1.0 / L.dfull : 0.0;
        if (cells >= (1LL << 31)) return -3;
        L.cells = cells;
        L.offset = total;
        total += cells;
        p.nlev++;
        bool can = true;
        for (int d = 0; d < 3; d++)
            if (g.act[d] && (n[d] % 2 != 0 || n[d] < 4)) can = false;
        if (!can) break;
        for (int d = 0; d < 3; d++)
            if (g.act[d]) n[d] /= 2;
    }
    if (p.lev[p.nlev - 1].cells > kMgMaxCoarse) return -2;
    p.total = total;
    *plan = p;
    return 0;
}

size_t mg_scratch_bytes(const MgPlan& p)
{
    // phi and rhs of every level; CG vectors r, p, q of the coarsest; partial sums; mean
    const size_t coarse = (size_t)p.lev[p.nlev - 1].cells;
    return sizeof(double) * (2 * (size_t)p.total + 3 * coarse + kMgParts + 1);
}

cudaError_t mg_clean(const Dims& g, const MgPlan& plan0, double* scratch, double* const* bq, bool cc, int cycles,
                     int nsm, cudaStream_t st, long long* launches)
{
    long long nl = 0;
    MgPlan plan = plan0;
    const long long T = plan.total;
    const long long nc = plan.lev[plan.nlev - 1].cells;
    for (int l = 0; l < plan.nlev; l++) {
        MgLevel& L = plan.lev[l];
        L.phi = scratch + L.offset;
        L.rhs = scratch + T + L.offset;
    }
    double* cg_r = scratch + 2 * T;
    double* cg_p = cg_r + nc;
    double* cg_q = cg_p + nc;
    double* part = cg_q + nc;
    double* mean = part + kMgParts;
    MgArgs m;
    for (int d = 0; d < 3; d++) {
        m.bc[d] = g.bc[d];
        m.act[d] = g.act[d];
    }
    const MgLevel& F = plan.lev[0];
    CP3 cq;
    P3 pq;
    for (int d = 0; d < 3; d++) {
        cq.p[d] = bq[d];
        pq.p[d] = bq[d];
    }
    const int nb = (int)((F.cells + 255) / 256 < kMgParts ? (F.cells + 255) / 256 : kMgParts);
    nl++;
    k_mg_div<<<nb, 256, 0, st>>>(g, cq, cc ? 1 : 0, F, m, part);
    nl++;
    k_mg_mean<<<1, 256, 0, st>>>(part, nb, mean, F.cells);
    nl++;
    k_mg_sub_mean<<<mg_grid(F.cells, nsm), 256, 0, st>>>(F, mean);
    const int cg_it = (int)(2 * nc + 20);
    // levels of at most kMgBlockCells cells run inside one block (k_mg_tail)
    MgTail tail;
    for (int l = 0; l < plan.nlev; l++) tail.lev[l] = plan.lev[l];
    tail.nlev = plan.nlev;
    tail.first = plan.nlev - 1;
    while (tail.first > 0 && plan.lev[tail.first - 1].cells <= kMgBlockCells) tail.first--;
    long long soff = 0;
    for (int l = tail.first; l < plan.nlev; l++) {
        tail.soff[l] = soff;
        soff += 2 * plan.lev[l].cells;
    }
    tail.scg = soff;
    const size_t tail_bytes = sizeof(double) * (size_t)(soff + 3 * nc);
    tail.smem = tail_bytes <= kMgTailSmem ? 1 : 0;
    const size_t tail_dyn = tail.smem ? tail_bytes : 0;
    for (int cyc = 0; cyc < cycles; cyc++) {
        for (int l = 0; l < tail.first; l++) {
            const MgLevel& L = plan.lev[l];
            const int bs = mg_grid(half_items(L), nsm);
            for (int s = 0; s < 2; s++) {
                nl++;
                k_mg_smooth<<<bs, 256, 0, st>>>(L, m, 0);
                nl++;
                k_mg_smooth<<<bs, 256, 0, st>>>(L, m, 1);
            }
            nl++;
            k_mg_restrict<<<mg_grid(plan.lev[l + 1].cells, nsm), 256, 0, st>>>(L, plan.lev[l + 1], m);
        }
        // the small levels and the coarsest solve (from zero); with a single level this
        // is the whole solve, and further cycles would repeat it
        nl++;
        k_mg_tail<<<1, 1024, tail_dyn, st>>>(tail, m, cg_r, cg_p, cg_q, cg_it);
        if (plan.nlev == 1) break;
        for (int l = tail.first - 1; l >= 0; l--) {
            const MgLevel& L = plan.lev[l];
            const int b = mg_grid(L.cells, nsm), bs = mg_grid(half_items(L), nsm);
            nl++;
            k_mg_prolong<<<b, 256, 0, st>>>(L, plan.lev[l + 1], m);
            for (int s = 0; s < 2; s++) {
                nl++;
                k_mg_smooth<<<bs, 256, 0, st>>>(L, m, 0);
                nl++;
                k_mg_smooth<<<bs, 256, 0, st>>>(L, m, 1);
            }
        }
    }
    nl++;
    k_mg_correct<<<mg_grid(F.cells, nsm), 256, 0, st>>>(g, pq, cc ? 1 : 0, F, m);
    if (launches) *launches += nl;
    return cudaGetLastError();
}

GRMHD_OOB_READER(oob_elliptic)

}  // namespace grmhd
