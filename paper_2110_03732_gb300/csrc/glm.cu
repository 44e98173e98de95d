// GLM hyperbolic divergence cleaning (arXiv 2110.03732 Sec. 3.1) with cell-centred
// magnetic fields: the explicit part of an IMEX stage for 12 cell-centred variables
// (D, S_1..3, tau, E^1..3, q_B^1..3, q_Phi), sm_103a, FP64.
//
//   k_glm_flux<D>  MC reconstruction of the 8 primitives, B^i = q_B^i/psi^6 and
//                  Phi = q_Phi/psi^6 to the D-faces; HLL flux of all 12 with the
//                  maximal-diffusivity speeds of Sec. 2.5.  With beta = 0:
//                    (f_B^j)^D = eta^{jDk} alpha E_k,   (f_Phi)^D = alpha q_B^D
//   k_glm_update   flux divergence + sources: the Gauss-law charge term of s_E and the
//                  metric terms of s_S, s_tau (Sec. 2.1), and for the new fields
//                    s_B^i  = -psi^6 alpha gamma^{ij} d_j Phi = -alpha psi^2 d_i Phi
//                    s_Phi  = -alpha kappa_B q_Phi + q_B^i d_i alpha
//                  (central differences of cell values); writes L, or folds it into the
//                  IMEX stage bases and the final combination (Sec. 2.3)
//
// Phi's flux divergence enters with the sign of the conservative form of Sec. 2.1
// (d_t q + d_i f^i = s with the f_Phi and s_Phi of Sec. 3.1), which makes (B, Phi) a
// damped wave system.  The charge field Psi is not evolved; rho_e comes from Gauss's
// law as in the staggered scheme.  The implicit solve is the one of Sec. 2.4 with the
// cell-centred field (k_implicit_cc in kernels.cu).
#include "grmhd_device.cuh"
#include "items.cuh"
#include "kernels.h"
#include "launch.cuh"

namespace grmhd {

// HLL fluxes of the 12 variables at the D-face with padded coordinates c (between the
// cells of linear indices rm and r0 = c - e_D, c) from the reconstructed states:
// prL / prR the 8 primitives, BL / BR the coordinate B = q_B / psi^6, phL / phR
// Phi = q_Phi / psi^6.  Writes twice the flux (the update folds the 1/2).
template <int D, bool M>
__device__ __forceinline__ void glm_face_flux(const Dims& g, const GlmFluxArgs& a, long long rm, long long r0,
                                              const double* prL, const double* prR, const double* BL,
                                              const double* BR, double phL, double phR)
{
    const double* __restrict__ psi = M ? a.psi : nullptr;
    const double* __restrict__ alp = M ? a.alp : nullptr;
    constexpr int D1 = (D + 1) % 3, D2 = (D + 2) % 3;
    const double psf = psi ? 0.5 * (psi[rm] + psi[r0]) : 1.0;
    const double alf = alp ? 0.5 * (alp[rm] + alp[r0]) : 1.0;
    const double pf2 = psf * psf, pf4 = pf2 * pf2, pf6 = pf4 * pf2;
    FaceState sL, sR;
    face_state<double>(prL, BL, D, psf, alf, g.gh, sL);
    face_state<double>(prR, BR, D, psf, alf, g.gh, sR);
    // HLL with c+ = c- = alpha sqrt(gamma^DD) (Sec. 2.5, maximal diffusivity); with equal
    // speeds (c f_L + c f_R - c^2 (q_R - q_L)) / 2c = (f_L + f_R - c (q_R - q_L)) / 2
    const double cs = psi ? alf * rcp_pos(pf2) : alf;
    const long long o = r0;
#pragma unroll
    for (int v = 0; v < 8; v++) a.F[v][o] = sL.f[v] + sR.f[v] - cs * (sR.q[v] - sL.q[v]);
    // q_B^j = psi^6 B^j with (f_B^j)^D = eta^{jDk} alpha psi^4 E^k: 0, -alpha psi^4 E^D2,
    // +alpha psi^4 E^D1 for j = D, D1, D2; q_Phi = psi^6 Phi with (f_Phi)^D = alpha q_B^D
    const double ap4 = alf * pf4;
    double qL[4], qR[4], fL[4], fR[4];
    qL[D] = pf6 * BL[D];
    qR[D] = pf6 * BR[D];
    fL[D] = 0.0;
    fR[D] = 0.0;
    qL[D1] = pf6 * BL[D1];
    qR[D1] = pf6 * BR[D1];
    fL[D1] = -ap4 * prL[5 + D2];
    fR[D1] = -ap4 * prR[5 + D2];
    qL[D2] = pf6 * BL[D2];
    qR[D2] = pf6 * BR[D2];
    fL[D2] = ap4 * prL[5 + D1];
    fR[D2] = ap4 * prR[5 + D1];
    qL[3] = pf6 * phL;
    qR[3] = pf6 * phR;
    fL[3] = alf * qL[D];
    fR[3] = alf * qR[D];
#pragma unroll
    for (int v = 0; v < 4; v++) a.F[8 + v][o] = fL[v] + fR[v] - cs * (qR[v] - qL[v]);
}

// MC (or PPM when P) reconstruction of the 8 primitives, B^i = q_B^i / psi^6 and
// Phi = q_Phi / psi^6 to K consecutive D-faces per thread, marched along D with one
// LineRec per quantity (as flux_march_item)
template <int D, bool M, bool P>
__device__ __forceinline__ void glm_flux_march_item(const Dims& g, const GlmFluxArgs& a, long long t)
{
    using Rec = LineRec<double, P>;
    const double* __restrict__ psi = M ? a.psi : nullptr;
    constexpr int NV = 12;
    int c[3], f0, f1;
    march_coords<D>(g, t, c, f0, f1);
    auto load = [&](int m, double* x) {
        int cs[3] = {c[0], c[1], c[2]};
        cs[D] = P ? ext_cell(g, D, m) : m;
        const long long mi = cell_at(g, cs);
#pragma unroll
        for (int v = 0; v < 8; v++) x[v] = a.prim[v][mi];
        double ip6 = 1.0;
        if (psi) {
            const double ps = psi[lin(g, cs[0], cs[1], cs[2])], p2 = ps * ps;
            ip6 = rcp_pos(p2 * p2 * p2);
        }
#pragma unroll
        for (int e = 0; e < 3; e++) x[8 + e] = a.qB[e][mi] * ip6;
        x[11] = a.qphi[mi] * ip6;
    };
    Rec rec[NV];
    {
        double w[Rec::NINIT][NV];
#pragma unroll
        for (int k = 0; k < Rec::NINIT; k++) load(f0 - Rec::NINIT + Rec::AHEAD + k, w[k]);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            double x[Rec::NINIT];
#pragma unroll
            for (int k = 0; k < Rec::NINIT; k++) x[k] = w[k][v];
            rec[v].init(x);
        }
    }
    int cm[3] = {c[0], c[1], c[2]};
    cm[D] = f0 - 1;
    long long rm = lin(g, cm[0], cm[1], cm[2]);
    for (int f = f0; f < f1; f++) {
        double x[NV];
        load(f + Rec::AHEAD, x);
        double prL[8], prR[8], BL[3], BR[3], phL, phR;
#pragma unroll
        for (int v = 0; v < 8; v++) rec[v].step(x[v], prL[v], prR[v]);
#pragma unroll
        for (int e = 0; e < 3; e++) rec[8 + e].step(x[8 + e], BL[e], BR[e]);
        rec[11].step(x[11], phL, phR);
        c[D] = f;
        const long long r0 = lin(g, c[0], c[1], c[2]);
        glm_face_flux<D, M>(g, a, rm, r0, prL, prR, BL, BR, phL, phR);
        rm = r0;
    }
}

template <int D, bool M, bool P = false>
__global__ void __launch_bounds__(128) k_glm_flux(Dims g, GlmFluxArgs a)
{
    grid_dep_sync();
    const long long nq = g.dq[D].d;   // chunks of g.mk[D] faces per line
    const long long tot = nq * (D == 0 ? (long long)g.n[1] * g.n[2]
                                       : (D == 1 ? (long long)g.n[0] * g.n[2] : (long long)g.n[0] * g.n[1]));
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        glm_flux_march_item<D, M, P>(g, a, t);
}

__device__ __forceinline__ void glm_out(const GlmUpdateArgs& a, int v, long long o, double L, bool has_r)
{
    if (a.mode == UPD_WRITE_L) {
        a.L[v][o] = L;
        return;
    }
    // as out_value: host-formed dt products, q^n read at stage 0 only
    const double r = has_r ? a.R[v - 5][o] : 0.0;
    const double qn = a.stage == 0 ? a.qn[v][o] : 0.0;
    for (int k = a.stage + 1; k < a.s; k++) {
        const double prev = a.stage == 0 ? qn : a.base[k][v][o];
        double nb = prev + a.cL[k] * L;
        if (has_r) nb += a.cR[k] * r;
        a.base[k][v][o] = nb;
    }
    const double prev = a.stage == 0 ? qn : a.acc[v][o];
    double nv = prev + a.cwL * L;
    if (has_r) nv += a.cwR * r;
    if (a.stage == a.s - 1) a.qn[v][o] = nv;
    else a.acc[v][o] = nv;
}

template <bool M>
__device__ __forceinline__ void glm_update_item(const Dims& g, const GlmUpdateArgs& a, long long t)
{
    const double* __restrict__ psi = M ? a.psi : nullptr;
    const double* __restrict__ alp = M ? a.alp : nullptr;
    int c[3];
    interior_coords(g, t, c);
    const long long o = lin(g, c[0], c[1], c[2]);
    double Lc[12];
#pragma unroll
    for (int v = 0; v < 12; v++) Lc[v] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!g.act[d]) continue;
        const long long o1 = chk(g, o + g.st[d]);
        const double hidx = 0.5 * g.idx[d];   // F holds twice the flux
#pragma unroll
        for (int v = 0; v < 12; v++) {
            const double* __restrict__ Fv = a.F[d][v];
            Lc[v] -= (Fv[o1] - Fv[o]) * hidx;
        }
    }
    cell_sources<true>(g, a.prim, a.qB, psi, alp, c, o, Lc);
    const double ps = psi ? psi[o] : 1.0;
    const double al = alp ? alp[o] : 1.0;
    const double p2 = ps * ps;
    Lc[11] -= al * a.kappa * a.qphi[o];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!g.act[d]) continue;
        int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
        cp[d] += 1;
        cm[d] -= 1;
        double sp = psi ? psi[chk(g, o + g.st[d])] : 1.0, sm = psi ? psi[chk(g, o - g.st[d])] : 1.0;
        sp = sp * sp;
        sm = sm * sm;
        const double sp3 = sp * sp * sp, sm3 = sm * sm * sm, r = rcp_pos(sp3 * sm3);
        const double php = a.qphi[cell_at(g, cp)] * (sm3 * r);   // q_Phi / psi^6
        const double phm = a.qphi[cell_at(g, cm)] * (sp3 * r);
        Lc[8 + d] -= al * p2 * ((php - phm) * (0.5 * g.idx[d]));
        if (alp) Lc[11] += a.qB[d][o] * ((alp[chk(g, o + g.st[d])] - alp[chk(g, o - g.st[d])]) * (0.5 * g.idx[d]));
    }
#pragma unroll
    for (int v = 0; v < 12; v++) glm_out(a, v, o, Lc[v], v >= 5 && v < 8);
}

__global__ void __launch_bounds__(128) k_glm_update_flat(Dims g, GlmUpdateArgs a)
{
    grid_dep_sync();
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        glm_update_item<false>(g, a, t);
}

__global__ void __launch_bounds__(128) k_glm_update_metric(Dims g, GlmUpdateArgs a)
{
    grid_dep_sync();
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        glm_update_item<true>(g, a, t);
}

static int glm_grid(long long work, int threads, int nsm)
{
    long long b = (work + threads - 1) / threads;
    const long long cap = (long long)nsm * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

template <int D, bool M, bool P>
static int glm_blocks_per_sm()
{
    static int nb = 0;
    if (nb < 1) {
        int q = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k_glm_flux<D, M, P>, 128, 0) != cudaSuccess || q < 1)
            q = 1;
        nb = q;
    }
    return nb;
}

// faces per thread as for the staggered-field flux kernels
template <int D, bool M, bool P>
static void glm_flux_launch(const Dims& g, const GlmFluxArgs& a, int nsm, cudaStream_t st)
{
    const long long other = D == 0 ? (long long)g.n[1] * g.n[2]
                                   : (D == 1 ? (long long)g.n[0] * g.n[2] : (long long)g.n[0] * g.n[1]);
    const int K = march_len(g.n[D], other, nsm, glm_blocks_per_sm<D, M, P>(), P ? 1.0 : 0.6);
    Dims gl = g;
    set_march(gl, D, K);
    launch_k(k_glm_flux<D, M, P>, glm_grid((long long)gl.dq[D].d * other, 128, nsm), 128, st, gl, a);
}

template <bool P>
static void glm_flux_dispatch(const Dims& g, int d, bool m, const GlmFluxArgs& a, int nsm, cudaStream_t st)
{
    if (d == 0) m ? glm_flux_launch<0, true, P>(g, a, nsm, st) : glm_flux_launch<0, false, P>(g, a, nsm, st);
    else if (d == 1) m ? glm_flux_launch<1, true, P>(g, a, nsm, st) : glm_flux_launch<1, false, P>(g, a, nsm, st);
    else m ? glm_flux_launch<2, true, P>(g, a, nsm, st) : glm_flux_launch<2, false, P>(g, a, nsm, st);
}

cudaError_t launch_glm_flux(const Dims& g, int d, const GlmFluxArgs& a, int nsm, cudaStream_t st, bool ppm)
{
    const bool m = a.psi || a.alp;
    if (ppm) glm_flux_dispatch<true>(g, d, m, a, nsm, st);
    else glm_flux_dispatch<false>(g, d, m, a, nsm, st);
    return cudaGetLastError();
}

cudaError_t launch_glm_update(const Dims& g, const GlmUpdateArgs& a, int nsm, cudaStream_t st)
{
    const int b = glm_grid((long long)g.n[0] * g.n[1] * g.n[2], 128, nsm);
    launch_k(a.psi || a.alp ? k_glm_update_metric : k_glm_update_flat, b, 128, st, g, a);
    return cudaGetLastError();
}

GRMHD_OOB_READER(oob_glm)

}  // namespace grmhd
