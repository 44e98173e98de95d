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

namespace grmhd {

// P: PPM reconstruction (cells c-3..c+2) instead of MC (c-2..c+1)
template <int D, bool M, bool P = false>
__device__ __forceinline__ void glm_flux_item(const Dims& g, const GlmFluxArgs& a, long long t)
{
    constexpr int NS = P ? 6 : 4, OFF = P ? 3 : 2;
    const double* __restrict__ psi = M ? a.psi : nullptr;
    const double* __restrict__ alp = M ? a.alp : nullptr;
    constexpr int D1 = (D + 1) % 3, D2 = (D + 2) % 3;
    const int e0 = g.n[0] + (D == 0), e1 = g.n[1] + (D == 1);
    int c[3];
    c[0] = g.ng[0] + (int)(t % e0);
    c[1] = g.ng[1] + (int)((t / e0) % e1);
    c[2] = g.ng[2] + (int)(t / ((long long)e0 * e1));
    long long mi[NS], ri[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        int cs[3] = {c[0], c[1], c[2]};
        cs[D] = P ? ext_cell(g, D, c[D] + s - OFF) : c[D] + s - OFF;
        mi[s] = cell_at(g, cs);
        ri[s] = lin(g, cs[0], cs[1], cs[2]);
    }
    double ip6[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        const double ps = psi ? psi[ri[s]] : 1.0;
        const double p2 = ps * ps;
        ip6[s] = 1.0 / (p2 * p2 * p2);
    }
    // MC or PPM face states of w[0..NS-1]
    auto rec = [&](const double* w, double& L, double& R) {
        if (P) ppm_face<double>(w, L, R);
        else mc_face<double>(w[0], w[1], w[2], w[NS - 1], L, R);
    };
    double prL[8], prR[8], BL[3], BR[3], phL, phR;
#pragma unroll
    for (int v = 0; v < 8; v++) {
        const double* __restrict__ x = a.prim[v];
        double w[NS];
#pragma unroll
        for (int s = 0; s < NS; s++) w[s] = x[mi[s]];
        rec(w, prL[v], prR[v]);
    }
#pragma unroll
    for (int e = 0; e < 3; e++) {
        const double* __restrict__ x = a.qB[e];
        double w[NS];
#pragma unroll
        for (int s = 0; s < NS; s++) w[s] = x[mi[s]] * ip6[s];
        rec(w, BL[e], BR[e]);
    }
    {
        const double* __restrict__ x = a.qphi;
        double w[NS];
#pragma unroll
        for (int s = 0; s < NS; s++) w[s] = x[mi[s]] * ip6[s];
        rec(w, phL, phR);
    }
    const double psf = psi ? 0.5 * (psi[ri[OFF - 1]] + psi[ri[OFF]]) : 1.0;
    const double alf = alp ? 0.5 * (alp[ri[OFF - 1]] + alp[ri[OFF]]) : 1.0;
    const double pf2 = psf * psf, pf4 = pf2 * pf2, pf6 = pf4 * pf2;
    FaceState sL, sR;
    face_state<double>(prL, BL, D, psf, alf, g.gh, sL);
    face_state<double>(prR, BR, D, psf, alf, g.gh, sR);
    // HLL with c+ = c- = alpha sqrt(gamma^DD) (Sec. 2.5, maximal diffusivity); with equal
    // speeds (c f_L + c f_R - c^2 (q_R - q_L)) / 2c = (f_L + f_R - c (q_R - q_L)) / 2
    const double cs = alf / pf2;
    const long long o = lin(g, c[0], c[1], c[2]);
#pragma unroll
    for (int v = 0; v < 8; v++)
        a.F[v][o] = (sL.f[v] + sR.f[v] - cs * (sR.q[v] - sL.q[v])) * 0.5;
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
    for (int v = 0; v < 4; v++)
        a.F[8 + v][o] = (fL[v] + fR[v] - cs * (qR[v] - qL[v])) * 0.5;
}

template <int D, bool M, bool P = false>
__global__ void __launch_bounds__(128) k_glm_flux(Dims g, GlmFluxArgs a)
{
    const long long tot = (long long)(g.n[0] + (D == 0)) * (g.n[1] + (D == 1)) * (g.n[2] + (D == 2));
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        glm_flux_item<D, M, P>(g, a, t);
}

__device__ __forceinline__ void glm_out(const GlmUpdateArgs& a, int v, long long o, double L, bool has_r)
{
    if (a.mode == UPD_WRITE_L) {
        a.L[v][o] = L;
        return;
    }
    const double r = has_r ? a.R[v - 5][o] : 0.0;
    const double qn = a.qn[v][o];
    for (int k = a.stage + 1; k < a.s; k++) {
        const double prev = a.stage == 0 ? qn : a.base[k][v][o];
        a.base[k][v][o] = prev + a.dt * (a.At[k][a.stage] * L + a.A[k][a.stage] * r);
    }
    const double prev = a.stage == 0 ? qn : a.acc[v][o];
    const double nv = prev + a.dt * (a.wt[a.stage] * L + a.w[a.stage] * r);
    if (a.stage == a.s - 1) a.qn[v][o] = nv;
    else a.acc[v][o] = nv;
}

template <bool M>
__device__ __forceinline__ void glm_update_item(const Dims& g, const GlmUpdateArgs& a, long long t)
{
    const double* __restrict__ psi = M ? a.psi : nullptr;
    const double* __restrict__ alp = M ? a.alp : nullptr;
    int c[3];
    c[0] = g.ng[0] + (int)(t % g.n[0]);
    c[1] = g.ng[1] + (int)((t / g.n[0]) % g.n[1]);
    c[2] = g.ng[2] + (int)(t / ((long long)g.n[0] * g.n[1]));
    const long long o = lin(g, c[0], c[1], c[2]);
    double Lc[12];
#pragma unroll
    for (int v = 0; v < 12; v++) Lc[v] = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!g.act[d]) continue;
        const long long o1 = o + g.st[d];
#pragma unroll
        for (int v = 0; v < 12; v++) {
            const double* __restrict__ Fv = a.F[d][v];
            Lc[v] -= (Fv[o1] - Fv[o]) * g.idx[d];
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
        double sp = psi ? psi[o + g.st[d]] : 1.0, sm = psi ? psi[o - g.st[d]] : 1.0;
        sp = sp * sp;
        sm = sm * sm;
        const double sp3 = sp * sp * sp, sm3 = sm * sm * sm, r = 1.0 / (sp3 * sm3);
        const double php = a.qphi[cell_at(g, cp)] * (sm3 * r);   // q_Phi / psi^6
        const double phm = a.qphi[cell_at(g, cm)] * (sp3 * r);
        Lc[8 + d] -= al * p2 * ((php - phm) * (0.5 * g.idx[d]));
        if (alp) Lc[11] += a.qB[d][o] * ((alp[o + g.st[d]] - alp[o - g.st[d]]) * (0.5 * g.idx[d]));
    }
#pragma unroll
    for (int v = 0; v < 12; v++) glm_out(a, v, o, Lc[v], v >= 5 && v < 8);
}

__global__ void __launch_bounds__(128) k_glm_update_flat(Dims g, GlmUpdateArgs a)
{
    const long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        glm_update_item<false>(g, a, t);
}

__global__ void __launch_bounds__(128) k_glm_update_metric(Dims g, GlmUpdateArgs a)
{
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

cudaError_t launch_glm_flux(const Dims& g, int d, const GlmFluxArgs& a, int nsm, cudaStream_t st, bool ppm)
{
    const long long work = (long long)(g.n[0] + (d == 0)) * (g.n[1] + (d == 1)) * (g.n[2] + (d == 2));
    const int b = glm_grid(work, 128, nsm);
    const bool m = a.psi || a.alp;
    if (ppm) {
        if (d == 0) m ? k_glm_flux<0, true, true><<<b, 128, 0, st>>>(g, a) : k_glm_flux<0, false, true><<<b, 128, 0, st>>>(g, a);
        else if (d == 1) m ? k_glm_flux<1, true, true><<<b, 128, 0, st>>>(g, a) : k_glm_flux<1, false, true><<<b, 128, 0, st>>>(g, a);
        else m ? k_glm_flux<2, true, true><<<b, 128, 0, st>>>(g, a) : k_glm_flux<2, false, true><<<b, 128, 0, st>>>(g, a);
        return cudaGetLastError();
    }
    if (d == 0) m ? k_glm_flux<0, true><<<b, 128, 0, st>>>(g, a) : k_glm_flux<0, false><<<b, 128, 0, st>>>(g, a);
    else if (d == 1) m ? k_glm_flux<1, true><<<b, 128, 0, st>>>(g, a) : k_glm_flux<1, false><<<b, 128, 0, st>>>(g, a);
    else m ? k_glm_flux<2, true><<<b, 128, 0, st>>>(g, a) : k_glm_flux<2, false><<<b, 128, 0, st>>>(g, a);
    return cudaGetLastError();
}

cudaError_t launch_glm_update(const Dims& g, const GlmUpdateArgs& a, int nsm, cudaStream_t st)
{
    const int b = glm_grid((long long)g.n[0] * g.n[1] * g.n[2], 128, nsm);
    if (a.psi || a.alp) k_glm_update_metric<<<b, 128, 0, st>>>(g, a);
    else k_glm_update_flat<<<b, 128, 0, st>>>(g, a);
    return cudaGetLastError();
}

}  // namespace grmhd
