// CUDA kernels of one IMEX-RK stage of resistive (GR)MHD with staggered
// constrained transport (arXiv 2110.03732), sm_103a, FP64 and mixed precision.
//
//   k_implicit   Sec. 2.4: per-cell Newton on u coupled to the implicit E update;
//                writes stage primitives and the stiff rate R = (q_E - q_E,base)/(a_ii dt)
//   k_stencil<M, T, P>  one launch per stage of
//                - the flux tasks, Sec. 2.1 + Sec. 5 defaults: MC (or PPM)
//                  reconstruction to the D-faces, marched along D, and the HLL flux with
//                  the maximal-diffusivity speeds of Sec. 2.5 (on flat 1-D / 2-D grids
//                  also the degenerate edge EMFs), and
//                - the edge-EMF tasks, Sec. 3.2 steps (i)-(vii): the upwind (UCT-HLL)
//                  edge EMF hat{E}_C, marched along C + 2 when both transverse
//                  directions are active
//                in FP64 or (T = float) mixed precision
//   k_flux_march<D>, k_emf_ideal<C>  the fluxes and App. A edge EMF of the ideal-limit
//                variant (separate launches: the flux writes the transport velocities)
//   k_update<M>  flux divergence + non-stiff sources (Sec. 2.1) and the CT face update
//                (Sec. 3.2); writes L, or folds it straight into the IMEX stage bases and
//                the final combination (Sec. 2.3)
//   k_prim2con, k_curlA (Sec. 4), k_dt (Sec. 2.5), k_divb, k_totals: set-up and
//   diagnostics; k_implicit_cc, k_curlA_cc, k_prim2con_cc, k_diag_cc: the same for the
//   cell-centred fields of the GLM variant (its flux and update kernels: glm.cu)
#include <cstring>

#include "grmhd_device.cuh"
#include "items.cuh"
#include "kernels.h"
#include "launch.cuh"

namespace grmhd {

thread_local bool launch_overlap = false;

// ---------------------------------------------------------------------------
// implicit step
// ---------------------------------------------------------------------------

// Five blocks per SM (96 registers, about 1 KB of spills): against four (128 registers)
// the mixed-precision and metric instances ran 1.5-4 % faster (512^2 vortex mixed 58.1 ->
// 57.3 us, 128^3 star mixed 398 -> 381 us, FP64 455 -> 442 us per launch); the flat FP64
// instance is unchanged (79.3 us).
template <bool M, bool ACC>
__global__ void __launch_bounds__(128, 5) k_implicit(Dims g, ImpArgs a)
{
    grid_dep_sync();
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        implicit_item<M, false, ACC>(g, a, t);
}

// the same solve with cell-centred q_B (GLM variant, Sec. 3.1)
template <bool M>
__global__ void __launch_bounds__(128, 4) k_implicit_cc(Dims g, ImpArgs a)
{
    grid_dep_sync();
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        implicit_item<M, true>(g, a, t);
}

// ---------------------------------------------------------------------------
// face fluxes
// ---------------------------------------------------------------------------

// MC (or PPM) fluxes, K consecutive D-faces per thread (flux_march_item)
template <int D, bool M, typename T, bool P = false>
__global__ void __launch_bounds__(128) k_flux_march(Dims g, FluxArgs<T> a)
{
    grid_dep_sync();
    const long long nq = g.dq[D].d;   // chunks of g.mk[D] faces per line
    const long long tot = nq * (D == 0 ? (long long)g.n[1] * g.n[2]
                                       : (D == 1 ? (long long)g.n[0] * g.n[2] : (long long)g.n[0] * g.n[1]));
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        flux_march_item<D, M, T, P>(g, a.prim, a.bf, a.psi, a.alp, a.F, a.vbar, a.Eh, t);
}

// ---------------------------------------------------------------------------
// the explicit stencil of a stage: face fluxes and upwind constrained transport
// (hat{E}_C on the edges along C, stored at the corner index that is lower in
// a = C+1 and b = C+2)
// ---------------------------------------------------------------------------

// The face fluxes of every active direction and the edge EMFs the flux tasks do not
// write, in one launch (resistive UCT, FP64 or mixed precision).  Block ranges select
// the task (the same items, march lengths and grid copies as separate launches would
// take, so every face and edge is bitwise the same); one launch keeps the SMs filled
// across what would be three to six single-wave kernels with their tails.
template <typename T>
struct StencilTasks {
    int b0[7];                 // first block of task s (flux x, y, z; EMF x, y, z); b0[6] = grid
    int emarch[3];             // EMF task C marches along C + 2 (both transverse directions active)
    Dims g[6];                 // each task's copy of the grid, with its march length
    FluxArgs<T> fa[3];
    EmfArgs<T> ea[3];
};

template <int D, bool M, typename T, bool P>
__device__ __forceinline__ void stencil_flux(const Dims& g, const FluxArgs<T>& a, long long t0, long long nt)
{
    const long long tot = g.dq[D].d * (D == 0 ? (long long)g.n[1] * g.n[2]
                                              : (D == 1 ? (long long)g.n[0] * g.n[2] : (long long)g.n[0] * g.n[1]));
    for (long long t = t0; t < tot; t += nt)
        flux_march_item<D, M, T, P>(g, a.prim, a.bf, a.psi, a.alp, a.F, nullptr, a.Eh, t);
}

template <int C, bool M, typename T, bool P>
__device__ __forceinline__ void stencil_emf(const Dims& g, const EmfArgs<T>& a, int march, long long t0,
                                            long long nt)
{
    constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
    if (march) {
        const long long tot = (long long)g.dq[B].d * g.n[C] * (g.n[A] + 1);
        for (long long t = t0; t < tot; t += nt) emf_march_item<C, M, T, P>(g, a.prim, a.bf, a.psi, a.alp, a.Eh, t);
    } else {
        long long tot = 1;
#pragma unroll
        for (int d = 0; d < 3; d++) tot *= (d == C) ? g.n[d] : (g.act[d] ? g.n[d] + 1 : 1);
        for (long long t = t0; t < tot; t += nt) emf_item<C, M, T, P>(g, a.prim, a.bf, a.psi, a.alp, a.Eh, t);
    }
}

// The FP32 PPM instance is held to 96 registers (five blocks per SM, 160 B of spills):
// at its natural 128 it ran 2 % slower.  The others keep the compiler's choice.
template <bool M, typename T, bool P>
__global__ void __launch_bounds__(128, (sizeof(T) == 4 && P) ? 5 : 0) k_stencil(StencilTasks<T> L)
{
    grid_dep_sync();
    const int b = blockIdx.x;
    int s = 0;
#pragma unroll
    for (int i = 1; i < 6; i++)
        if (b >= L.b0[i]) s = i;   // empty tasks have b0[i] == b0[i + 1]
    switch (s) {
#define GRMHD_STENCIL_CASE(S, CALL)                                                   \
    case S: {                                                                         \
        const long long nt = (long long)(L.b0[S + 1] - L.b0[S]) * blockDim.x;        \
        const long long t0 = (long long)(b - L.b0[S]) * blockDim.x + threadIdx.x;    \
        CALL;                                                                         \
        break;                                                                        \
    }
        GRMHD_STENCIL_CASE(0, (stencil_flux<0, M, T, P>(L.g[0], L.fa[0], t0, nt)))
        GRMHD_STENCIL_CASE(1, (stencil_flux<1, M, T, P>(L.g[1], L.fa[1], t0, nt)))
        GRMHD_STENCIL_CASE(2, (stencil_flux<2, M, T, P>(L.g[2], L.fa[2], t0, nt)))
        GRMHD_STENCIL_CASE(3, (stencil_emf<0, M, T, P>(L.g[3], L.ea[0], L.emarch[0], t0, nt)))
        GRMHD_STENCIL_CASE(4, (stencil_emf<1, M, T, P>(L.g[4], L.ea[1], L.emarch[1], t0, nt)))
        GRMHD_STENCIL_CASE(5, (stencil_emf<2, M, T, P>(L.g[5], L.ea[2], L.emarch[2], t0, nt)))
#undef GRMHD_STENCIL_CASE
    default: break;
    }
}

// ideal-limit edge EMF (App. A) from the stored transport velocities
struct VbarArgs {
    const double* p[3][2];
};

template <int C, bool M>
__global__ void __launch_bounds__(128) k_emf_ideal(Dims g, EmfArgs<double> a, VbarArgs vb)
{
    grid_dep_sync();
    long long tot = 1;
#pragma unroll
    for (int d = 0; d < 3; d++) tot *= (d == C) ? g.n[d] : (g.act[d] ? g.n[d] + 1 : 1);
    CP8 prim;
#pragma unroll
    for (int v = 0; v < 8; v++) prim.p[v] = a.prim.p[v];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        emf_ideal_item<C, M>(g, prim, a.bf, a.psi, a.alp, vb.p, a.Eh, t);
}

// ---------------------------------------------------------------------------
// update: cell-centred L (flux divergence + non-stiff sources) and face L_B (CT)
// ---------------------------------------------------------------------------

// The FP32-flux instances are held to 32 registers (16 blocks per SM, 300-570 B of
// spills): the 513^2 items of a 512^2 stage then fit one wave instead of 1.5 and the
// 128^3 star's mixed update ran 454 -> 421 us per launch (512^2: 42.8 -> 41.7 us).  The
// FP64 instances keep the compiler's choice (64-78 registers): bound by the FP64 pipe,
// they only lost from more blocks.
template <bool M, bool F32>
__global__ void __launch_bounds__(128, F32 ? 16 : 0) k_update(Dims g, UpdateArgs a)
{
    grid_dep_sync();
    long long tot = 1;
#pragma unroll
    for (int d = 0; d < 3; d++) tot *= g.act[d] ? g.n[d] + 1 : 1;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        update_item<M, F32>(g, a, t);
}

// ---------------------------------------------------------------------------
// set-up: face q_B = curl of the edge potential (Sec. 4), prim -> cons (Sec. 2.1)
// ---------------------------------------------------------------------------

__global__ void k_curlA(Dims g, CP3 A, P3 bf)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.ncell;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[0] = (int)(t % g.N[0]);
        c[1] = (int)((t / g.N[0]) % g.N[1]);
        c[2] = (int)(t / ((long long)g.N[0] * g.N[1]));
#pragma unroll
        for (int fa = 0; fa < 3; fa++) {
            const int fb = (fa + 1) % 3, fc = (fa + 2) % 3;
            if ((g.act[fb] && c[fb] + 1 >= g.N[fb]) || (g.act[fc] && c[fc] + 1 >= g.N[fc])) continue;
            double r = 0.0;
            if (g.act[fb]) r += (A.p[fc][chk(g, t + g.st[fb])] - A.p[fc][t]) * g.idx[fb];
            if (g.act[fc]) r -= (A.p[fb][chk(g, t + g.st[fc])] - A.p[fb][t]) * g.idx[fc];
            bf.p[fa][t] = r;
        }
    }
}

__global__ void k_prim2con(Dims g, CP8 prim, CP3 bf, const double* __restrict__ psi, P8 q)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.ncell;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[0] = (int)(t % g.N[0]);
        c[1] = (int)((t / g.N[0]) % g.N[1]);
        c[2] = (int)(t / ((long long)g.N[0] * g.N[1]));
        const double ps = psi ? psi[t] : 1.0;
        const double p2 = ps * ps, p6 = p2 * p2 * p2;
        double pr[8], B[3];
#pragma unroll
        for (int v = 0; v < 8; v++) pr[v] = prim.p[v][t];
#pragma unroll
        for (int e = 0; e < 3; e++) B[e] = cell_qB(g, bf.p[e], e, c) / p6;
        FaceState s;
        face_state(pr, B, 0, ps, 1.0, g.gh, s);
#pragma unroll
        for (int v = 0; v < 8; v++) q.p[v][t] = s.q[v];
    }
}

// cell-centred q_B^i = eta^{ijk} d_j A_k from a cell-centred potential by central
// differences (Sec. 4, cell-centred fields), interior cells; the potential is read
// as given on the whole padded grid
__global__ void k_curlA_cc(Dims g, CP3 A, P3 qB)
{
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = g.ng[0] + (int)(t % g.n[0]);
        const int j = g.ng[1] + (int)((t / g.n[0]) % g.n[1]);
        const int k = g.ng[2] + (int)(t / ((long long)g.n[0] * g.n[1]));
        const long long o = lin(g, i, j, k);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            double r = 0.0;
            if (g.act[b]) r += (A.p[c][chk(g, o + g.st[b])] - A.p[c][chk(g, o - g.st[b])]) * (0.5 * g.idx[b]);
            if (g.act[c]) r -= (A.p[b][chk(g, o + g.st[c])] - A.p[b][chk(g, o - g.st[c])]) * (0.5 * g.idx[c]);
            qB.p[a][o] = r;
        }
    }
}

// prim -> cons with cell-centred q_B, every padded cell; q_Phi = psi^6 Phi (Sec. 3.1)
// from the primitive Phi (NULL: zero)
__global__ void k_prim2con_cc(Dims g, CP8 prim, CP3 qB, const double* __restrict__ psi,
                              const double* __restrict__ phi, double* __restrict__ qphi, P8 q)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const double ps = psi ? psi[t] : 1.0;
        const double p2 = ps * ps, p6 = p2 * p2 * p2;
        double pr[8], B[3];
#pragma unroll
        for (int v = 0; v < 8; v++) pr[v] = prim.p[v][t];
#pragma unroll
        for (int e = 0; e < 3; e++) B[e] = qB.p[e][t] / p6;
        FaceState s;
        face_state(pr, B, 0, ps, 1.0, g.gh, s);
#pragma unroll
        for (int v = 0; v < 8; v++) q.p[v][t] = s.q[v];
        qphi[t] = phi ? p6 * phi[t] : 0.0;
    }
}

// FP32 copy of caller primitives at every padded cell (fixed-boundary ghosts
// included) with the densitised cell-centred q_B, for the mixed-precision path
__global__ void k_prim_to32(Dims g, CP8 prim, CP3 bf, F11 p32)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.ncell;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[0] = (int)(t % g.N[0]);
        c[1] = (int)((t / g.N[0]) % g.N[1]);
        c[2] = (int)(t / ((long long)g.N[0] * g.N[1]));
#pragma unroll
        for (int v = 0; v < 8; v++) p32.p[v][t] = (float)prim.p[v][t];
#pragma unroll
        for (int e = 0; e < 3; e++) p32.p[8 + e][t] = (float)cell_qB(g, bf.p[e], e, c);
    }
}

// ---------------------------------------------------------------------------
// reductions (fixed-order block trees: deterministic for a given launch shape)
// ---------------------------------------------------------------------------

template <typename Op>
__device__ __forceinline__ double block_reduce(double v, Op op, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (w == 0) {
        v = l < nw ? sh[l] : 0.0;   // identity of sum, and of max over non-negative values
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

struct OpSum { __device__ double operator()(double a, double b) const { return a + b; } };
struct OpMax { __device__ double operator()(double a, double b) const { return fmax(a, b); } };

// per block: [max over cells of sum_d alpha sqrt(gamma^dd)/dx_d]
__global__ void __launch_bounds__(256) k_dt(Dims g, const double* __restrict__ psi, const double* __restrict__ alp,
                                            double* __restrict__ part)
{
    __shared__ double sh[32];
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    double m = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = g.ng[0] + (int)(t % g.n[0]);
        const int j = g.ng[1] + (int)((t / g.n[0]) % g.n[1]);
        const int k = g.ng[2] + (int)(t / ((long long)g.n[0] * g.n[1]));
        const long long o = lin(g, i, j, k);
        const double ps = psi ? psi[o] : 1.0;
        const double sp = (alp ? alp[o] : 1.0) / (ps * ps);
        m = fmax(m, sp * (g.idx[0] + g.idx[1] + g.idx[2]));
    }
    m = block_reduce(m, OpMax(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

// per block: [sum |div q_B|, sum div^2, max |div|, sum q_0..q_7 (times dV)]
__global__ void __launch_bounds__(256) k_diag(Dims g, CP3 bf, CP8 q, double dV, double* __restrict__ part)
{
    __shared__ double sh[32];
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    double s1 = 0.0, s2 = 0.0, mx = 0.0, tq[8];
#pragma unroll
    for (int v = 0; v < 8; v++) tq[v] = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[0] = g.ng[0] + (int)(t % g.n[0]);
        c[1] = g.ng[1] + (int)((t / g.n[0]) % g.n[1]);
        c[2] = g.ng[2] + (int)(t / ((long long)g.n[0] * g.n[1]));
        const long long o = lin(g, c[0], c[1], c[2]);
        const double dv = cell_divb(g, bf.p, c, o);
        s1 += fabs(dv);
        s2 += dv * dv;
        mx = fmax(mx, fabs(dv));
#pragma unroll
        for (int v = 0; v < 8; v++) tq[v] += q.p[v][o] * dV;
    }
    double r = block_reduce(s1, OpSum(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 11 + 0] = r;
    r = block_reduce(s2, OpSum(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 11 + 1] = r;
    r = block_reduce(mx, OpMax(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 11 + 2] = r;
#pragma unroll
    for (int v = 0; v < 8; v++) {
        r = block_reduce(tq[v], OpSum(), sh);
        if (threadIdx.x == 0) part[blockIdx.x * 11 + 3 + v] = r;
    }
}

// the same with cell-centred q_B: div by central differences (GLM variant)
__global__ void __launch_bounds__(256) k_diag_cc(Dims g, CP3 qB, CP8 q, double dV, double* __restrict__ part)
{
    __shared__ double sh[32];
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    double s1 = 0.0, s2 = 0.0, mx = 0.0, tq[8];
#pragma unroll
    for (int v = 0; v < 8; v++) tq[v] = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[0] = g.ng[0] + (int)(t % g.n[0]);
        c[1] = g.ng[1] + (int)((t / g.n[0]) % g.n[1]);
        c[2] = g.ng[2] + (int)(t / ((long long)g.n[0] * g.n[1]));
        const long long o = lin(g, c[0], c[1], c[2]);
        double dv = 0.0;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (!g.act[d]) continue;
            int cu[3] = {c[0], c[1], c[2]}, cl[3] = {c[0], c[1], c[2]};
            cu[d] += 1;
            cl[d] -= 1;
            dv += (qB.p[d][cell_at(g, cu)] - qB.p[d][cell_at(g, cl)]) * (0.5 * g.idx[d]);
        }
        s1 += fabs(dv);
        s2 += dv * dv;
        mx = fmax(mx, fabs(dv));
#pragma unroll
        for (int v = 0; v < 8; v++) tq[v] += q.p[v][o] * dV;
    }
    double r = block_reduce(s1, OpSum(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 11 + 0] = r;
    r = block_reduce(s2, OpSum(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 11 + 1] = r;
    r = block_reduce(mx, OpMax(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 11 + 2] = r;
#pragma unroll
    for (int v = 0; v < 8; v++) {
        r = block_reduce(tq[v], OpSum(), sh);
        if (threadIdx.x == 0) part[blockIdx.x * 11 + 3 + v] = r;
    }
}

// second pass: one block folds `nb` partial rows of width `w`; column kinds: 0 sum, 1 max
__global__ void __launch_bounds__(256) k_fold(const double* __restrict__ part, int nb, int w,
                                              const int* __restrict__ kinds_unused, unsigned kinds_mask,
                                              double* __restrict__ out)
{
    __shared__ double sh[32];
    (void)kinds_unused;
    for (int col = 0; col < w; col++) {
        const bool is_max = (kinds_mask >> col) & 1u;
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const double x = part[(long long)b * w + col];
            v = is_max ? fmax(v, x) : v + x;
        }
        v = is_max ? block_reduce(v, OpMax(), sh) : block_reduce(v, OpSum(), sh);
        if (threadIdx.x == 0) out[col] = v;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static int grid_for(long long work, int threads, int nsm)
{
    long long b = (work + threads - 1) / threads;
    const long long cap = (long long)nsm * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_implicit(const Dims& g, const ImpArgs& a, int nsm, cudaStream_t st)
{
    const long long work = (long long)g.n[0] * g.n[1] * g.n[2];
    const bool m = a.psi || a.alp;
    if (a.dwacc) launch_k(m ? k_implicit<true, true> : k_implicit<false, true>, grid_for(work, 128, nsm), 128, st, g, a);
    else launch_k(m ? k_implicit<true, false> : k_implicit<false, false>, grid_for(work, 128, nsm), 128, st, g, a);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_hist_init(long long n, const double* __restrict__ u1,
                                                   const double* __restrict__ u2, const double* __restrict__ u3,
                                                   const double* __restrict__ psi, P3f hs, P3f hd)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double p2 = psi ? psi[t] * psi[t] : 1.0;
        hs.p[0][t] = (float)(p2 * u1[t]);
        hs.p[1][t] = (float)(p2 * u2[t]);
        hs.p[2][t] = (float)(p2 * u3[t]);
        hd.p[0][t] = hd.p[1][t] = hd.p[2][t] = 0.0f;
    }
}

cudaError_t launch_hist_init(const Dims& g, const double* u1, const double* u2, const double* u3, const double* psi,
                             P3f hs, P3f hd, int nsm, cudaStream_t st)
{
    k_hist_init<<<grid_for(g.ncell, 256, nsm), 256, 0, st>>>(g.ncell, u1, u2, u3, psi, hs, hd);
    return cudaGetLastError();
}

cudaError_t launch_implicit_cc(const Dims& g, const ImpArgs& a, int nsm, cudaStream_t st)
{
    const long long work = (long long)g.n[0] * g.n[1] * g.n[2];
    // GLM contexts are FP64 only: the FP64 residual accepts the root
    launch_k(a.psi || a.alp ? k_implicit_cc<true> : k_implicit_cc<false>, grid_for(work, 128, nsm), 128, st, g,
             a);
    return cudaGetLastError();
}


// resident 128-thread blocks per SM of a marching flux kernel (its register count
// decides: about 2 for FP64, 4 for FP32), queried once
template <int D, bool M, typename T, bool P>
static int march_blocks_per_sm()
{
    static int nb = 0;
    if (nb < 1) {
        int q = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k_flux_march<D, M, T, P>, 128, 0) != cudaSuccess ||
            q < 1)
            q = 1;
        nb = q;
    }
    return nb;
}

// faces per thread by march_len (start-up: 3 cells for MC, 5 for PPM, each about a
// fifth of a face's work).  For FP64, waves are counted at no more than two resident
// blocks per SM.  At 8 warps the FP64 flux already keeps the FP64 pipe ~75-80 % busy, and
// a third block (where the registers allow it) adds no throughput.  A shorter march to
// fill that block would only add start-ups: 5 faces at three blocks per SM took 123 us
// per 512^2 launch, against 117 us for 7 faces at two.
template <int D, bool M, typename T, bool P>
static void flux_march_launch(const Dims& g, int nsm, cudaStream_t st, const FluxArgs<T>& a)
{
    const long long other = D == 0 ? (long long)g.n[1] * g.n[2]
                                   : (D == 1 ? (long long)g.n[0] * g.n[2] : (long long)g.n[0] * g.n[1]);
    const int bps = march_blocks_per_sm<D, M, T, P>();
    const int K = march_len(g.n[D], other, nsm, sizeof(T) == 8 && bps > 2 ? 2 : bps, P ? 1.0 : 0.6);
    Dims gl = g;
    set_march(gl, D, K);
    const int b = grid_for((long long)gl.dq[D].d * other, 128, nsm);
    launch_k(k_flux_march<D, M, T, P>, b, 128, st, gl, a);
}

template <typename T, bool P>
static void flux_dispatch(const Dims& g, int d, bool m, int nsm, cudaStream_t st, const FluxArgs<T>& a)
{
    if (d == 0) m ? flux_march_launch<0, true, T, P>(g, nsm, st, a) : flux_march_launch<0, false, T, P>(g, nsm, st, a);
    else if (d == 1) m ? flux_march_launch<1, true, T, P>(g, nsm, st, a) : flux_march_launch<1, false, T, P>(g, nsm, st, a);
    else m ? flux_march_launch<2, true, T, P>(g, nsm, st, a) : flux_march_launch<2, false, T, P>(g, nsm, st, a);
}

// edges of direction C (one per thread when A or B is inactive)
static long long emf_work(const Dims& g, int c)
{
    long long work = 1;
    for (int d = 0; d < 3; d++) work *= (d == c) ? g.n[d] : (g.act[d] ? g.n[d] + 1 : 1);
    return work;
}

cudaError_t launch_flux(const Dims& g, int d, CP8 prim, CP3 bf, const double* psi, const double* alp, P8 F, int nsm,
                        cudaStream_t st, double* const* vbar, bool ppm, double* const* Eh)
{
    FluxArgs<double> a;
    for (int k = 0; k < 3; k++) a.Eh[k] = Eh && !(psi || alp) ? Eh[k] : nullptr;
    for (int v = 0; v < 8; v++) {
        a.prim.p[v] = prim.p[v];
        a.F.p[v] = F.p[v];
    }
    a.vbar[0] = vbar ? vbar[0] : nullptr;
    a.vbar[1] = vbar ? vbar[1] : nullptr;
    a.bf = bf;
    a.psi = psi;
    a.alp = alp;
    if (ppm) flux_dispatch<double, true>(g, d, psi || alp, nsm, st, a);
    else flux_dispatch<double, false>(g, d, psi || alp, nsm, st, a);
    return cudaGetLastError();
}

template <bool M, typename T, bool P>
static int stencil_blocks_per_sm()
{
    static int nb = 0;
    if (nb < 1) {
        int q = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k_stencil<M, T, P>, 128, 0) != cudaSuccess || q < 1)
            q = 1;
        nb = q;
    }
    return nb;
}

template <typename T>
static cudaError_t stencil_launch(const Dims& g, const PrimIn<T>& prim, CP3 bf, const double* psi, const double* alp,
                                  const FluxOut<T>* F, double* const (*fe)[3], double* const* Eh, int nsm,
                                  cudaStream_t st, bool ppm)
{
    const bool m = psi || alp;
    const int bps = ppm ? (m ? stencil_blocks_per_sm<true, T, true>() : stencil_blocks_per_sm<false, T, true>())
                        : (m ? stencil_blocks_per_sm<true, T, false>() : stencil_blocks_per_sm<false, T, false>());
    const double c0 = ppm ? 1.0 : 0.6;
    StencilTasks<T> L;
    memset(&L, 0, sizeof L);
    int nb = 0;
    for (int d = 0; d < 3; d++) {
        L.b0[d] = nb;
        L.g[d] = g;
        FluxArgs<T>& a = L.fa[d];
        a.prim = prim;
        a.bf = bf;
        a.psi = psi;
        a.alp = alp;
        if (!g.act[d]) continue;
        a.F = F[d];
        for (int k = 0; k < 3; k++) a.Eh[k] = fe && !m ? fe[d][k] : nullptr;
        const long long other = d == 0 ? (long long)g.n[1] * g.n[2]
                                       : (d == 1 ? (long long)g.n[0] * g.n[2] : (long long)g.n[0] * g.n[1]);
        set_march(L.g[d], d, march_len(g.n[d], other, nsm, bps, c0));
        nb += grid_for((long long)L.g[d].dq[d].d * other, 128, nsm);
    }
    for (int c = 0; c < 3; c++) {
        L.b0[3 + c] = nb;
        L.g[3 + c] = g;
        EmfArgs<T>& a = L.ea[c];
        a.prim = prim;
        a.bf = bf;
        a.psi = psi;
        a.alp = alp;
        if (!Eh || !Eh[c]) continue;
        a.Eh = Eh[c];
        const int A = (c + 1) % 3, B = (c + 2) % 3;
        if (g.act[A] && g.act[B]) {
            const long long other = (long long)g.n[c] * (g.n[A] + 1);
            set_march(L.g[3 + c], B, march_len(g.n[B], other, nsm, bps, c0));
            L.emarch[c] = 1;
            nb += grid_for((long long)L.g[3 + c].dq[B].d * other, 128, nsm);
        } else {
            nb += grid_for(emf_work(g, c), 128, nsm);
        }
    }
    L.b0[6] = nb;
    if (nb == 0) return cudaSuccess;
    if (ppm) launch_k(m ? k_stencil<true, T, true> : k_stencil<false, T, true>, nb, 128, st, L);
    else launch_k(m ? k_stencil<true, T, false> : k_stencil<false, T, false>, nb, 128, st, L);
    return cudaGetLastError();
}

cudaError_t launch_stencil32(const Dims& g, const PrimIn<float>& prim, CP3 bf, const double* psi, const double* alp,
                             const FluxOut<float>* F, double* const (*fe)[3], double* const* Eh, int nsm,
                             cudaStream_t st, bool ppm)
{
    return stencil_launch<float>(g, prim, bf, psi, alp, F, fe, Eh, nsm, st, ppm);
}

cudaError_t launch_stencil64(const Dims& g, CP8 prim, CP3 bf, const double* psi, const double* alp, const P8* F,
                             double* const (*fe)[3], double* const* Eh, int nsm, cudaStream_t st, bool ppm)
{
    PrimIn<double> p;
    FluxOut<double> fo[3];
    for (int v = 0; v < 8; v++) p.p[v] = prim.p[v];
    for (int d = 0; d < 3; d++)
        for (int v = 0; v < 8; v++) fo[d].p[v] = F[d].p[v];
    return stencil_launch<double>(g, p, bf, psi, alp, fo, fe, Eh, nsm, st, ppm);
}

cudaError_t launch_emf_ideal(const Dims& g, int c, CP8 prim, CP3 bf, const double* psi, const double* alp,
                             const double* const (*vb)[2], double* Eh, int nsm, cudaStream_t st)
{
    EmfArgs<double> a;
    for (int v = 0; v < 8; v++) a.prim.p[v] = prim.p[v];
    a.bf = bf;
    a.psi = psi;
    a.alp = alp;
    a.Eh = Eh;
    VbarArgs v;
    for (int d = 0; d < 3; d++)
        for (int k = 0; k < 2; k++) v.p[d][k] = vb[d][k];
    const int b = grid_for(emf_work(g, c), 128, nsm);
    const bool m = psi || alp;
    if (c == 0) launch_k(m ? k_emf_ideal<0, true> : k_emf_ideal<0, false>, b, 128, st, g, a, v);
    else if (c == 1) launch_k(m ? k_emf_ideal<1, true> : k_emf_ideal<1, false>, b, 128, st, g, a, v);
    else launch_k(m ? k_emf_ideal<2, true> : k_emf_ideal<2, false>, b, 128, st, g, a, v);
    return cudaGetLastError();
}

cudaError_t launch_update(const Dims& g, const UpdateArgs& a, int nsm, cudaStream_t st)
{
    long long work = 1;
    for (int d = 0; d < 3; d++) work *= g.act[d] ? g.n[d] + 1 : 1;
    const int b = grid_for(work, 128, nsm);
    const bool m = a.psi || a.alp;
    if (a.f32) launch_k(m ? k_update<true, true> : k_update<false, true>, b, 128, st, g, a);
    else launch_k(m ? k_update<true, false> : k_update<false, false>, b, 128, st, g, a);
    return cudaGetLastError();
}

cudaError_t launch_curlA(const Dims& g, CP3 A, P3 bf, int nsm, cudaStream_t st)
{
    k_curlA<<<grid_for(g.ncell, 256, nsm), 256, 0, st>>>(g, A, bf);
    return cudaGetLastError();
}

cudaError_t launch_prim2con(const Dims& g, CP8 prim, CP3 bf, const double* psi, P8 q, int nsm, cudaStream_t st)
{
    k_prim2con<<<grid_for(g.ncell, 256, nsm), 256, 0, st>>>(g, prim, bf, psi, q);
    return cudaGetLastError();
}

cudaError_t launch_prim_to32(const Dims& g, CP8 prim, CP3 bf, F11 p32, int nsm, cudaStream_t st)
{
    k_prim_to32<<<grid_for(g.ncell, 256, nsm), 256, 0, st>>>(g, prim, bf, p32);
    return cudaGetLastError();
}

cudaError_t launch_dt(const Dims& g, const double* psi, const double* alp, double* part, int nblk, double* out,
                      cudaStream_t st)
{
    k_dt<<<nblk, 256, 0, st>>>(g, psi, alp, part);
    k_fold<<<1, 256, 0, st>>>(part, nblk, 1, nullptr, 1u, out);
    return cudaGetLastError();
}

cudaError_t launch_diag(const Dims& g, CP3 bf, CP8 q, double dV, double* part, int nblk, double* out,
                        cudaStream_t st)
{
    k_diag<<<nblk, 256, 0, st>>>(g, bf, q, dV, part);
    k_fold<<<1, 256, 0, st>>>(part, nblk, 11, nullptr, 1u << 2, out);
    return cudaGetLastError();
}

cudaError_t launch_curlA_cc(const Dims& g, CP3 A, P3 qB, int nsm, cudaStream_t st)
{
    k_curlA_cc<<<grid_for((long long)g.n[0] * g.n[1] * g.n[2], 256, nsm), 256, 0, st>>>(g, A, qB);
    return cudaGetLastError();
}

cudaError_t launch_prim2con_cc(const Dims& g, CP8 prim, CP3 qB, const double* psi, const double* phi, double* qphi,
                               P8 q, int nsm, cudaStream_t st)
{
    k_prim2con_cc<<<grid_for(g.ncell, 256, nsm), 256, 0, st>>>(g, prim, qB, psi, phi, qphi, q);
    return cudaGetLastError();
}

cudaError_t launch_diag_cc(const Dims& g, CP3 qB, CP8 q, double dV, double* part, int nblk, double* out,
                           cudaStream_t st)
{
    k_diag_cc<<<nblk, 256, 0, st>>>(g, qB, q, dV, part);
    k_fold<<<1, 256, 0, st>>>(part, nblk, 11, nullptr, 1u << 2, out);
    return cudaGetLastError();
}

GRMHD_OOB_READER(oob_kernels)

}  // namespace grmhd
