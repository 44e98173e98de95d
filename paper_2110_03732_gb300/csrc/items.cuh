// Per-item bodies of the stage kernels (one cell, face or edge each), shared by
// the single-problem kernels (kernels.cu) and the batched multi-problem kernels
// (batch.cu), so that a problem advanced alone or inside a batch runs exactly the
// same arithmetic.  See kernels.cu for the paper passages each body follows.
#pragma once

#include "grmhd_device.cuh"
#include "kernels.h"

namespace grmhd {

// ---------------------------------------------------------------------------
// implicit step (Sec. 2.4): item t = interior cell t (x fastest)
// ---------------------------------------------------------------------------

// CC: the magnetic field is cell-centred (a.bf holds cell q_B, GLM variant) instead of
// staggered on faces.  ACC: the mixed-precision path, whose double-word residual
// accepts the root (newton_refine_dw)
template <bool M, bool CC = false, bool ACC = false>
__device__ __forceinline__ void implicit_item(const Dims& g, const ImpArgs& a, long long t)
{
    // flat metric: alpha = psi = 1 known at compile time
    const double* __restrict__ psi = M ? a.psi : nullptr;
    const double* __restrict__ alp = M ? a.alp : nullptr;
    const CP8& qb = a.qb;
    const CP3& bf = a.bf;
    const double* __restrict__ eta = a.eta;
    const double eta_u = a.eta_u, a_dt = a.a_dt, tol = a.tol, rho_atm = a.rho_atm, p_atm = a.p_atm;
    const int kmax = a.kmax;
    const P8& prim = a.prim;
    const P3& R = a.R;
    const P3& qE_out = a.qE_out;
    const F11& p32 = a.p32;
    unsigned long long* nfail = a.nfail;
    int c[3];
    interior_coords(g, t, c);
    const long long id = lin(g, c[0], c[1], c[2]);
    const double ps = psi ? psi[id] : 1.0;
    const double al = alp ? alp[id] : 1.0;
    const double p2 = ps * ps, p4 = p2 * p2, ip2 = M ? rcp_pos(p2) : 1.0, ip4 = ip2 * ip2, ip6 = ip4 * ip2;
    CellIn ci;
    ci.gh = g.gh;
    ci.igh = g.igh;
    ci.xi = a.xi;
    ci.ighf = a.ighf;
    ci.xif = a.xif;
    ci.D = qb.p[0][id] * ip6;
    ci.S[0] = qb.p[1][id] * ip6 * ip2;
    ci.S[1] = qb.p[2][id] * ip6 * ip2;
    ci.S[2] = qb.p[3][id] * ip6 * ip2;
    ci.tau = qb.p[4][id] * ip6;
    double qEs[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        qEs[i] = qb.p[5 + i][id];
        ci.Es[i] = qEs[i] * ip4;
        ci.B[i] = (CC ? bf.p[i][id] : cell_qB(g, bf.p[i], i, c)) * ip4;
    }
    const double et = eta ? eta[id] : eta_u;
    // flat: eta / (a_ii dt) with the host's reciprocal, no division
    ci.etat = a.stiff ? (M ? et * rcp_pos(al) * a.ia_dt : et * a.ia_dt) : -1.0;
    cell_derive(ci);
    double u[3];
    Eval e;
    bool atmo = false;
    // Newton start: this stage's last root plus its last change (a linear extrapolation
    // over steps, kept in FP32: it is only a start) when the history is kept, else the
    // latest primitives
    const bool hist = a.hs[0] != nullptr;
    float hsv[3] = {0.0f, 0.0f, 0.0f};
    F3 ust = {{0.0f, 0.0f, 0.0f}};
    if (a.atm && ci.D < a.d_atm) {
        atmo = true;   // (its history is left as it is)
    } else {
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            if (hist) {
                hsv[i] = a.hs[i][id];
                ust.x[i] = hsv[i] + a.hd[i][id];
                u[i] = f2d_int(ust.x[i]);
            } else {
                u[i] = p2 * prim.p[1 + i][id];
            }
            if (!mag_below_int(u[i], kHi1e30)) fin = false;   // also NaN
        }
        if (!fin) u[0] = u[1] = u[2] = 0.0;
        int it = newton_solve<ACC>(ci, u, e, kmax, tol, a.tolf, hist && fin, ust);
        if (it < 0 && fin) {
            u[0] = u[1] = u[2] = 0.0;
            it = newton_solve<ACC>(ci, u, e, kmax, tol, a.tolf, false, ust);
        }
        if (it < 0) {
            atomicAdd(nfail, 1ull);
            if (!a.atm) {
                // no atmosphere: leave the cell's primitives as they were, no stiff update
                if (R.p[0])
#pragma unroll
                    for (int i = 0; i < 3; i++) R.p[i][id] = 0.0;
                return;
            }
            atmo = true;
        }
    }
    double rho, pres;
    if (atmo) {
        // atmosphere: rest state at the floor density and pressure, E kept
        rho = rho_atm;
        pres = p_atm;
        u[0] = u[1] = u[2] = 0.0;
        e.E[0] = ci.Es[0];
        e.E[1] = ci.Es[1];
        e.E[2] = ci.Es[2];
    } else {
        const double iW = e.iW;
        rho = ci.D * iW;
        pres = (e.wt * iW - rho) * g.igh;
    }
    prim.p[0][id] = rho;
    prim.p[4][id] = pres;
    if (p32.p[0]) {
        // FP32 copy for the mixed-precision explicit kernels, with the densitised
        // cell-centred q_B of the stage
        // (converted on the integer pipe: a hardware conversion issues on the FP64 pipe)
        p32.p[0][id] = d2f_int(rho);
        p32.p[4][id] = d2f_int(pres);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            p32.p[1 + i][id] = d2f_int(u[i] * ip2);
            p32.p[5 + i][id] = d2f_int(e.E[i] * ip2);
            p32.p[8 + i][id] = d2f_int(ci.B[i] * p4);
        }
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        prim.p[1 + i][id] = u[i] * ip2;
        prim.p[5 + i][id] = e.E[i] * ip2;
        const double qEn = p4 * e.E[i];
        if (R.p[0]) R.p[i][id] = a.stiff ? (qEn - qEs[i]) * a.ia_dt : 0.0;
        if (qE_out.p[0]) qE_out.p[i][id] = qEn;
        if (hist && !atmo) {
            const float un = d2f_int(u[i]);
            a.hd[i][id] = un - hsv[i];
            a.hs[i][id] = un;
        }
    }
}

// ---------------------------------------------------------------------------
// face fluxes (Sec. 2.1, Sec. 2.5, Sec. 5 defaults): item t = D-face t
// ---------------------------------------------------------------------------

// cell-centred densitised q_B^e of the (mapped) cell: from the staggered faces on
// the FP64 path, from the stage's FP32 copy on the mixed path
__device__ __forceinline__ double cell_qB_in(const Dims& g, const PrimIn<double>&, const CP3& bf, int e, const int* cs,
                                             long long)
{
    return cell_qB(g, bf.p[e], e, cs);
}
__device__ __forceinline__ float cell_qB_in(const Dims&, const PrimIn<float>& pa, const CP3&, int e, const int*,
                                            long long mi)
{
    return pa.p[8 + e][mi];
}

// the upwind edge EMF of Sec. 3.2 (Londrillo & Del Zanna 2004) with c+ = c- in each
// direction, where the four-state weights are all 1/4 and the diffusive coefficients
// c^2/2c are c/2: h_XY = alpha E_C^XY (X the A side, Y the B side), q_B^B reconstructed
// along A, q_B^A along B
template <typename T>
__device__ __forceinline__ T uct_edge(T hLL, T hLR, T hRL, T hRR, T ca, T cb, T qBbL, T qBbR, T qBaL, T qBaR)
{
    return scale_pow2<T, -2>(hLL + hLR + hRL + hRR) + (T(0.5) * ca) * (qBbR - qBbL) - (T(0.5) * cb) * (qBaR - qBaL);
}

// HLL flux at the D-face with padded coordinates c (between the cells of linear
// indices rm = c - e_D and r0 = c) from the reconstructed states: prL / prR the 8
// primitives (coordinate u^i and E^i), BL / BR the coordinate B with the two transverse
// components set (the normal one is the face's own).  Writes twice the flux at r0, and
// the ideal-limit transport velocities when vbar is set.  prL, prR, BL, BR are
// overwritten.
//
// Eh (flat metric only, else NULL): Eh[C] set for an edge direction C != D whose
// third direction is inactive (a 1-D or 2-D grid).  Its edges then coincide with the
// D-faces, and the UCT EMF there needs only reconstructions along D of E_C and of the
// transverse q_B, which are this face's states: the face writes hat{E}_C, what emf_item
// computes from the same MC or PPM values (to round-off: the edge formula here is
// reduced for the coinciding states).
template <int D, bool M, typename T>
__device__ __forceinline__ void face_flux(const Dims& g, const CP3& bf, const double* psi_in, const double* alp_in,
                                          const int* c, long long rm, long long r0, T* prL, T* prR, T* BL, T* BR,
                                          const FluxOut<T>& F, double* const* vbar, double* const* Eh = nullptr)
{
    const double* __restrict__ psi = M ? psi_in : nullptr;
    const double* __restrict__ alp = M ? alp_in : nullptr;
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    const T psf = psi ? mean2<T>(psi[rm], psi[r0]) : T(1);
    const T alf = alp ? mean2<T>(alp[rm], alp[r0]) : T(1);
    const T pf2 = psf * psf, ipf2 = psi ? rcp_t(pf2) : T(1);
    // orthonormal-frame states at the face: u_hat = psi^2 u, E_hat = psi^2 E,
    // B_hat = psi^2 B (normal: q_B / psi^4)
    BL[D] = BR[D] = (T)bf.p[D][face_at(g, D, c)] * (ipf2 * ipf2);
    if (!M && Eh) {
        // C = D + 1: A = D + 2 (inactive), B = D; C = D + 2: A = D, B = D + 1 (inactive)
        // uct_edge with the inactive side's two states equal: the four-state mean is
        // the mean of the two D states, the normal field's jump across the inactive
        // side is zero, and the unit speeds leave (E_L + E_R -/+ jump of the transverse
        // q_B along D) / 2
        if (Eh[T1]) Eh[T1][r0] = to_f64(scale_pow2<T, -1>((prL[5 + T1] + prR[5 + T1]) - (BR[T2] - BL[T2])));
        if (Eh[T2]) Eh[T2][r0] = to_f64(scale_pow2<T, -1>((prL[5 + T2] + prR[5 + T2]) + (BR[T1] - BL[T1])));
    }
    if (psi) {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            prL[1 + i] *= pf2;
            prR[1 + i] *= pf2;
            prL[5 + i] *= pf2;
            prR[5 + i] *= pf2;
            if (i != D) {
                BL[i] *= pf2;
                BR[i] *= pf2;
            }
        }
    }
    // HLL with c+ = c- = c = alpha sqrt(gamma^DD) = alpha / psi^2 (Sec. 2.5, maximal
    // diffusivity): (c f_L + c f_R - c^2 (q_R - q_L)) / 2c = (f_L + f_R - c (q_R - q_L)) / 2.
    // Each densitised q_v is psi^k_v times its flat-space (psi = alpha = 1) value and its
    // flux alpha psi^(k_v - 2) times, k = 6, 8, 8, 8, 6, 4, 4, 4: the HLL flux is then
    // alpha psi^(k_v - 2) times the flat-space HLL flux (unit speed) of the
    // orthonormal states.  F stores twice the flux (no 1/2 here: the update folds it).
    T gL[8], gR[8], iWL, iWR;
    face_hll_half<T, 1>(prL, BL, D, (T)g.gh, gL, iWL);
    face_hll_half<T, -1>(prR, BR, D, (T)g.gh, gR, iWR);
    const T h2 = alf * pf2, h4 = h2 * pf2, h6 = h4 * pf2;
    const long long o = r0;
#pragma unroll
    for (int v = 0; v < 8; v++) {
        const T hv = v == 0 || v == 4 ? h4 : (v < 4 ? h6 : h2);
        F.p[v][o] = (gL[v] + gR[v]) * hv;
    }
    if (vbar && vbar[0]) {
        // App. A steps (i)-(ii): vhat^j = alpha v^j (beta = 0) of the L and R states,
        // vbar^j = (c- vhat^j_R + c+ vhat^j_L)/(c- + c+), their mean for c+ = c-;
        // v^j = u_hat^j / (psi^2 W)
        const double al = (double)(alf * ipf2);
        const double iL = (double)iWL, iR = (double)iWR;
        const double vL1 = al * (double)prL[1 + T1] * iL, vR1 = al * (double)prR[1 + T1] * iR;
        const double vL2 = al * (double)prL[1 + T2] * iL, vR2 = al * (double)prR[1 + T2] * iR;
        vbar[0][o] = (vR1 + vL1) * 0.5;
        vbar[1][o] = (vR2 + vL2) * 0.5;
    }
}

// Marching reconstruction along a line of cells, one quantity: the face states of the
// faces f0, f0+1, ... from one new cell per face.  MC keeps the last two cell values,
// their difference and the older cell's right-face state; PPM keeps the last two cell
// values, the newer one's MC slope, the interface value below it and the limited right
// edge of the cell before.  Each step returns the states of face f (between cells f-1
// and f): bitwise those of mc_face / ppm_face, whose slopes and interface values are
// the same expressions, each now evaluated once.
template <typename T, bool P>
struct LineRec;

template <typename T>
struct LineRec<T, false> {
    static constexpr int NINIT = 3, AHEAD = 1;   // cells f0-2..f0 first; step f loads f+1
    T a, b, d, l;
    __device__ __forceinline__ void init(const T* x)
    {
        a = x[1];
        b = x[2];
        d = b - a;
        l = a + minmod3<T>(a - x[0], scale_pow2<T, -2>(b - x[0]), d);
    }
    __device__ __forceinline__ void step(T x, T& L, T& R)
    {
        const T dn = x - b;
        const T hs = minmod3<T>(d, scale_pow2<T, -2>(x - a), dn);
        L = l;
        R = b - hs;
        l = b + hs;
        a = b;
        b = x;
        d = dn;
    }
};

template <typename T>
struct LineRec<T, true> {
    static constexpr int NINIT = 5, AHEAD = 2;   // cells f0-3..f0+1 first; step f loads f+2
    T a0, a1, s0, ip, lr;                        // a_f, a_f+1, slope_f, I_f-1/2, right edge_f-1
    __device__ __forceinline__ void init(const T* x)
    {
        const T sm2 = ppm_slope<T>(x[0], x[1], x[2]);
        const T sm1 = ppm_slope<T>(x[1], x[2], x[3]);
        s0 = ppm_slope<T>(x[2], x[3], x[4]);
        T lL = ppm_iface_s<T>(x[1], x[2], sm2, sm1);
        ip = ppm_iface_s<T>(x[2], x[3], sm1, s0);
        T lR = ip;
        ppm_limit<T>(x[2], lL, lR);
        lr = lR;
        a0 = x[3];
        a1 = x[4];
    }
    __device__ __forceinline__ void step(T x, T& L, T& R)
    {
        const T s1 = ppm_slope<T>(a0, a1, x);
        const T in = ppm_iface_s<T>(a0, a1, s0, s1);
        T rL = ip, rR = in;
        ppm_limit<T>(a0, rL, rR);
        L = lr;
        R = rL;
        lr = rR;
        ip = in;
        s0 = s1;
        a0 = a1;
        a1 = x;
    }
};

// item t of a face march along D in chunks of K: the padded coordinates c of the
// line (c[D] unset) and its faces f0 .. f1-1 (padded indices).  Chunks along D,
// x-fastest over the other directions; for D = 0 the chunks themselves run along x.
template <int D>
__device__ __forceinline__ void march_coords(const Dims& g, long long t, int* c, int& f0, int& f1)
{
    const int K = g.mk[D];
    int idx[3];
    // the chunk index along D takes the place of the D coordinate in an x-fastest box
    box_coords(t, D == 0 ? g.dq[0] : g.dv[0], D == 1 ? g.dq[1] : g.dv[1], idx);
    const int q = idx[D];
#pragma unroll
    for (int d = 0; d < 3; d++) c[d] = d == D ? 0 : g.ng[d] + idx[d];
    f0 = g.ng[D] + q * K;
    f1 = min(f0 + K, g.ng[D] + g.n[D] + 1);
}

// The same fluxes for K consecutive D-faces per thread (MC, or PPM when P): the thread
// marches along D with one LineRec per reconstructed quantity, so each new face loads
// one cell and reconstructs once (the per-face forms load four or six cells and
// compute two MC slopes, or three interface values and two parabola limits).  Items:
// chunks of K faces along D, x-fastest over the other directions (for D = 0 the chunks
// themselves run along x).
template <int D, bool M, typename T, bool P = false>
__device__ __forceinline__ void flux_march_item(const Dims& g, const PrimIn<T>& prim, const CP3& bf,
                                                const double* psi_in, const double* alp_in, const FluxOut<T>& F,
                                                double* const* vbar, double* const* Eh, long long t)
{
    using Rec = LineRec<T, P>;
    const double* __restrict__ psi = M ? psi_in : nullptr;
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    constexpr int NV = 10;   // 8 primitives and the two transverse B
    int c[3], f0, f1;
    march_coords<D>(g, t, c, f0, f1);
    // the 10 reconstructed values of the cell at padded coordinate m along D (PPM's
    // stencil reaches a third ghost: ext_cell maps it)
    auto load = [&](int m, T* x) {
        int cs[3] = {c[0], c[1], c[2]};
        cs[D] = P ? ext_cell(g, D, m) : m;
        const long long mi = cell_at(g, cs);
#pragma unroll
        for (int v = 0; v < 8; v++) x[v] = prim.p[v][mi];
        T ip6 = T(1);
        if (psi) {
            const T ps = met_t<T>(psi[lin(g, cs[0], cs[1], cs[2])]), p2 = ps * ps;
            ip6 = rcp_t(p2 * p2 * p2);
        }
        x[8] = (T)cell_qB_in(g, prim, bf, T1, cs, mi) * ip6;
        x[9] = (T)cell_qB_in(g, prim, bf, T2, cs, mi) * ip6;
    };
    Rec rec[NV];
    {
        T w[Rec::NINIT][NV];
#pragma unroll
        for (int k = 0; k < Rec::NINIT; k++) load(f0 - Rec::NINIT + Rec::AHEAD + k, w[k]);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            T x[Rec::NINIT];
#pragma unroll
            for (int k = 0; k < Rec::NINIT; k++) x[k] = w[k][v];
            rec[v].init(x);
        }
    }
    int cm[3] = {c[0], c[1], c[2]};
    cm[D] = f0 - 1;
    long long rm = lin(g, cm[0], cm[1], cm[2]);
    for (int f = f0; f < f1; f++) {
        T x[NV];
        load(f + Rec::AHEAD, x);
        T prL[8], prR[8], BL[3], BR[3];
#pragma unroll
        for (int v = 0; v < 8; v++) rec[v].step(x[v], prL[v], prR[v]);
        rec[8].step(x[8], BL[T1], BR[T1]);
        rec[9].step(x[9], BL[T2], BR[T2]);
        c[D] = f;
        const long long r0 = lin(g, c[0], c[1], c[2]);
        face_flux<D, M, T>(g, bf, psi_in, alp_in, c, rm, r0, prL, prR, BL, BR, F, vbar, Eh);
        rm = r0;
    }
}

// ---------------------------------------------------------------------------
// upwind constrained transport (Sec. 3.2): item t = C-edge t
// ---------------------------------------------------------------------------

// Face speeds at a C-edge (Sec. 2.5: c = alpha sqrt(gamma^dd) = alpha / psi^2 at a face,
// whose alpha and psi are the means of the two cells beside it): cab[0] the larger of
// the (up to two) A-faces touching the edge, cab[1] likewise for the B-faces; 1 in an
// inactive direction.  The larger of a0/q0 and a1/q1 is picked by comparing a0 q1 with
// a1 q0, and both quotients come from one reciprocal.
template <typename T>
__device__ __forceinline__ void edge_speeds(const Dims& g, const double* __restrict__ psi,
                                            const double* __restrict__ alp, long long i0, bool aa, bool ba,
                                            long long sA, long long sB, T* cab)
{
    T num[2] = {T(1), T(1)}, den[2] = {T(1), T(1)};
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const bool act = k == 0 ? aa : ba, oth = k == 0 ? ba : aa;
        if (!act) continue;
        const long long sn = k == 0 ? sA : sB, so = k == 0 ? sB : sA;
        for (int tt = 0; tt < (oth ? 2 : 1); tt++) {
            const long long cf = chk(g, i0 - tt * so), cfm = chk(g, cf - sn);
            const T psf = psi ? mean2<T>(psi[cfm], psi[cf]) : T(1);
            const T alf = alp ? mean2<T>(alp[cfm], alp[cf]) : T(1);
            const T q = psf * psf;
            if (tt == 0 || alf * den[k] > num[k] * q) {
                num[k] = alf;
                den[k] = q;
            }
        }
    }
    const T r = rcp_t(den[0] * den[1]);
    cab[0] = num[0] * den[1] * r;
    cab[1] = num[1] * den[0] * r;
}

// P: PPM reconstruction (six cells or faces per pass) instead of MC (four)
template <int C, bool M, typename T, bool P = false>
__device__ __forceinline__ void emf_item(const Dims& g, const PrimIn<T>& prim, const CP3& bf, const double* psi_in,
                                         const double* alp_in, double* __restrict__ Eh, long long t)
{
    constexpr int NS = P ? 6 : 4, OFF = P ? 3 : 2;
    const double* __restrict__ psi = M ? psi_in : nullptr;
    const double* __restrict__ alp = M ? alp_in : nullptr;
    constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
    const bool aa = g.act[A], ba = g.act[B];
    const T* __restrict__ Ec = prim.p[5 + C];
    // edges: n[d] along C, n[d] + 1 along an active transverse d (1 if inactive)
    int c[3];
    box_coords(t, C == 0 ? g.dv[0] : g.dvp[0], C == 1 ? g.dv[1] : g.dvp[1], c);
#pragma unroll
    for (int d = 0; d < 3; d++) c[d] += g.ng[d];
    // steps (ii)-(iii): covariant E_C = psi^4 E^C, to A-faces then along B
    T s[2][NS];   // [X = A-side L/R][B offset -OFF..+OFF-1]
    const int nb = ba ? NS : 1;
    for (int ob = 0; ob < nb; ob++) {
        int cb[3] = {c[0], c[1], c[2]};
        if (ba) cb[B] = P ? ext_cell(g, B, c[B] + ob - OFF) : c[B] + ob - OFF;
        if (aa) {
            T v[NS];
#pragma unroll
            for (int sa = 0; sa < NS; sa++) {
                int cs[3] = {cb[0], cb[1], cb[2]};
                cs[A] = P ? ext_cell(g, A, cb[A] + sa - OFF) : cb[A] + sa - OFF;
                const T ps = psi ? met_t<T>(psi[lin(g, cs[0], cs[1], cs[2])]) : T(1);
                const T p2 = ps * ps;
                v[sa] = p2 * p2 * Ec[cell_at(g, cs)];
            }
            if (P) ppm_face<T>(v, s[0][ob], s[1][ob]);
            else mc_face<T>(v[0], v[1], v[2], v[NS - 1], s[0][ob], s[1][ob]);
        } else {
            const T ps = psi ? met_t<T>(psi[lin(g, cb[0], cb[1], cb[2])]) : T(1);
            const T p2 = ps * ps;
            s[0][ob] = s[1][ob] = p2 * p2 * Ec[cell_at(g, cb)];
        }
    }
    T EXY[2][2];
#pragma unroll
    for (int X = 0; X < 2; X++) {
        if (!ba) EXY[X][0] = EXY[X][1] = s[X][0];
        else if (P) ppm_face<T>(s[X], EXY[X][0], EXY[X][1]);
        else mc_face<T>(s[X][0], s[X][1], s[X][2], s[X][NS - 1], EXY[X][0], EXY[X][1]);
    }
    // step (iv): q_B^B (B-faces) along A, q_B^A (A-faces) along B
    T qBbL, qBbR, qBaL, qBaR;
    if (aa) {
        T v[NS];
#pragma unroll
        for (int sa = 0; sa < NS; sa++) {
            int cs[3] = {c[0], c[1], c[2]};
            cs[A] = P ? ext_cell(g, A, c[A] + sa - OFF) : c[A] + sa - OFF;
            v[sa] = (T)bf.p[B][face_at(g, B, cs)];
        }
        if (P) ppm_face<T>(v, qBbL, qBbR);
        else mc_face<T>(v[0], v[1], v[2], v[NS - 1], qBbL, qBbR);
    } else {
        qBbL = qBbR = (T)bf.p[B][face_at(g, B, c)];
    }
    if (ba) {
        T v[NS];
#pragma unroll
        for (int sb = 0; sb < NS; sb++) {
            int cs[3] = {c[0], c[1], c[2]};
            cs[B] = P ? ext_cell(g, B, c[B] + sb - OFF) : c[B] + sb - OFF;
            v[sb] = (T)bf.p[A][face_at(g, A, cs)];
        }
        if (P) ppm_face<T>(v, qBaL, qBaR);
        else mc_face<T>(v[0], v[1], v[2], v[NS - 1], qBaL, qBaR);
    } else {
        qBaL = qBaR = (T)bf.p[A][face_at(g, A, c)];
    }
    // lapse at the edge (mean of the adjacent cells) and the face speeds
    const long long i0 = lin(g, c[0], c[1], c[2]);
    const long long sA = aa ? g.st[A] : 0, sB = ba ? g.st[B] : 0;
    T ale = T(1), ca = T(1), cb = T(1);
    if (alp || psi) {
        // mean of the 1, 2 or 4 cells around the edge
        T sum = alp ? met_t<T>(alp[i0]) : T(1), w = T(1);
        if (aa) { sum += alp ? met_t<T>(alp[chk(g, i0 - sA)]) : T(1); w = T(0.5); }
        if (ba) {
            sum += alp ? met_t<T>(alp[chk(g, i0 - sB)]) : T(1);
            if (aa) sum += alp ? met_t<T>(alp[chk(g, i0 - sA - sB)]) : T(1);
            w *= T(0.5);
        }
        ale = sum * w;
        T cab[2];
        edge_speeds<T>(g, psi, alp, i0, aa, ba, sA, sB, cab);
        ca = cab[0];
        cb = cab[1];
    }
    // steps (v)-(vii): hat{E}^{XY} = alpha E_C^{XY}; Londrillo & Del Zanna (2004) with
    // c+ = c- in each direction, where the four-state weights are all 1/4 and the
    // diffusive coefficients c^2/2c are c/2
    const T hLL = ale * EXY[0][0], hLR = ale * EXY[0][1], hRL = ale * EXY[1][0], hRR = ale * EXY[1][1];
    Eh[i0] = to_f64(uct_edge<T>(hLL, hLR, hRL, hRR, ca, cb, qBbL, qBbR, qBaL, qBaR));
}

// The same EMFs for K consecutive C-edges along B per thread (MC, or PPM when P; A and
// B both active): the A-direction reconstruction of E_C on each row of cells along B,
// and q_B^A, are marched along B with LineRec (one new row per edge instead of four or
// six), so each edge computes one A-row, three one-cell B steps and its own q_B^B
// reconstruction.  The results are bitwise those of emf_item.  Items: chunks of K edges
// along B, x-fastest over the other two directions (the chunks run along x when B = 0).
template <int C, bool M, typename T, bool P = false>
__device__ __forceinline__ void emf_march_item(const Dims& g, const PrimIn<T>& prim, const CP3& bf,
                                               const double* psi_in, const double* alp_in, double* __restrict__ Eh,
                                               long long t)
{
    using Rec = LineRec<T, P>;
    constexpr int NS = P ? 6 : 4, OFF = P ? 3 : 2;
    const double* __restrict__ psi = M ? psi_in : nullptr;
    const double* __restrict__ alp = M ? alp_in : nullptr;
    constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
    const T* __restrict__ Ec = prim.p[5 + C];
    const int K = g.mk[B];
    // x-fastest box: the chunks along B, n[C] edges along C, n[A] + 1 along A
    int c[3], idx[3];
    box_coords(t, B == 0 ? g.dq[0] : (C == 0 ? g.dv[0] : g.dvp[0]),
               B == 1 ? g.dq[1] : (C == 1 ? g.dv[1] : g.dvp[1]), idx);
#pragma unroll
    for (int d = 0; d < 3; d++) c[d] = g.ng[d] + (d == B ? 0 : idx[d]);
    const int f0 = g.ng[B] + idx[B] * K;
    const int f1 = min(f0 + K, g.ng[B] + g.n[B] + 1);
    // a face state along A from the NS values v (cells or faces c[A]-OFF..)
    auto recA = [&](const T* v, T& L, T& R) {
        if (P) ppm_face<T>(v, L, R);
        else mc_face<T>(v[0], v[1], v[2], v[NS - 1], L, R);
    };
    // row m along B: covariant E_C = psi^4 E^C reconstructed along A to the A-face c[A],
    // and q_B^A at that A-face
    auto row = [&](int m, T* x) {
        const int mb = P ? ext_cell(g, B, m) : m;
        T v[NS];
#pragma unroll
        for (int sa = 0; sa < NS; sa++) {
            int cs[3] = {c[0], c[1], c[2]};
            cs[B] = mb;
            cs[A] = P ? ext_cell(g, A, c[A] + sa - OFF) : c[A] + sa - OFF;
            const T ps = psi ? met_t<T>(psi[lin(g, cs[0], cs[1], cs[2])]) : T(1);
            const T p2 = ps * ps;
            v[sa] = p2 * p2 * Ec[cell_at(g, cs)];
        }
        recA(v, x[0], x[1]);
        int cs[3] = {c[0], c[1], c[2]};
        cs[B] = mb;
        x[2] = (T)bf.p[A][face_at(g, A, cs)];
    };
    Rec rec[3];
    {
        T w[Rec::NINIT][3];
#pragma unroll
        for (int k = 0; k < Rec::NINIT; k++) row(f0 - Rec::NINIT + Rec::AHEAD + k, w[k]);
#pragma unroll
        for (int v = 0; v < 3; v++) {
            T x[Rec::NINIT];
#pragma unroll
            for (int k = 0; k < Rec::NINIT; k++) x[k] = w[k][v];
            rec[v].init(x);
        }
    }
    for (int f = f0; f < f1; f++) {
        T x3[3];
        row(f + Rec::AHEAD, x3);
        T L[3], R[3];
#pragma unroll
        for (int v = 0; v < 3; v++) rec[v].step(x3[v], L[v], R[v]);
        c[B] = f;
        // q_B^B (B-faces) along A
        T qBbL, qBbR;
        {
            T v[NS];
#pragma unroll
            for (int sa = 0; sa < NS; sa++) {
                int cs[3] = {c[0], c[1], c[2]};
                cs[A] = P ? ext_cell(g, A, c[A] + sa - OFF) : c[A] + sa - OFF;
                v[sa] = (T)bf.p[B][face_at(g, B, cs)];
            }
            recA(v, qBbL, qBbR);
        }
        const long long i0 = lin(g, c[0], c[1], c[2]);
        const long long sA = g.st[A], sB = g.st[B];
        T ale = T(1), ca = T(1), cb = T(1);
        if (alp || psi) {
            T sum = alp ? met_t<T>(alp[i0]) : T(1);
            sum += alp ? met_t<T>(alp[chk(g, i0 - sA)]) : T(1);
            sum += alp ? met_t<T>(alp[chk(g, i0 - sB)]) : T(1);
            sum += alp ? met_t<T>(alp[chk(g, i0 - sA - sB)]) : T(1);
            ale = sum * T(0.25);
            T cab[2];
            edge_speeds<T>(g, psi, alp, i0, true, true, sA, sB, cab);
            ca = cab[0];
            cb = cab[1];
        }
        // EXY[X][Y]: X the A side (the row's L / R), Y the B side (L = this edge's
        // lower-B state)
        Eh[i0] = to_f64(uct_edge<T>(ale * L[0], ale * R[0], ale * L[1], ale * R[1], ca, cb, qBbL, qBbR, L[2],
                                     R[2]));
    }
}

// ---------------------------------------------------------------------------
// ideal-limit edge EMF (App. A), FP64: item t = C-edge t (as emf_item)
// ---------------------------------------------------------------------------

// transport velocity vhat^j = alpha v^j of the cell at padded coordinates cs (the
// "face" value in an inactive direction)
__device__ __forceinline__ double cell_vhat(const Dims& g, const CP8& prim, const double* __restrict__ psi,
                                            const double* __restrict__ alp, int j, const int* cs)
{
    const long long mi = cell_at(g, cs), ri = lin(g, cs[0], cs[1], cs[2]);
    const double ps = psi ? psi[ri] : 1.0;
    const double p4 = ps * ps * ps * ps;
    const double u0 = prim.p[1][mi], u1 = prim.p[2][mi], u2 = prim.p[3][mi];
    return (alp ? alp[ri] : 1.0) * prim.p[1 + j][mi] * rsqrt(1.0 + p4 * (u0 * u0 + u1 * u1 + u2 * u2));
}

// vb[d][k]: transport velocities at the d-faces, component (d + 1 + k) % 3
template <int C, bool M>
__device__ __forceinline__ void emf_ideal_item(const Dims& g, const CP8& prim, const CP3& bf, const double* psi_in,
                                               const double* alp_in, const double* const (*vb)[2],
                                               double* __restrict__ Eh, long long t)
{
    const double* __restrict__ psi = M ? psi_in : nullptr;
    const double* __restrict__ alp = M ? alp_in : nullptr;
    constexpr int A = (C + 1) % 3, B = (C + 2) % 3;
    const bool aa = g.act[A], ba = g.act[B];
    // edges: n[d] along C, n[d] + 1 along an active transverse d (1 if inactive)
    int c[3];
    box_coords(t, C == 0 ? g.dv[0] : g.dvp[0], C == 1 ? g.dv[1] : g.dvp[1], c);
#pragma unroll
    for (int d = 0; d < 3; d++) c[d] += g.ng[d];
    // step (iii): q_B^B and vbar^A (both at B-faces) along A; q_B^A and vbar^B (A-faces)
    // along B.  vbar^A is component A = B + 2 of the B-faces, vbar^B component B = A + 1
    // of the A-faces.
    double qBbL, qBbR, qBaL, qBaR, vaL, vaR, vbL, vbR;
    {
        double q[4], v[4];
        const int ns = aa ? 4 : 1;
        for (int sa = 0; sa < ns; sa++) {
            int cs[3] = {c[0], c[1], c[2]};
            if (aa) cs[A] += sa - 2;
            const long long fi = face_at(g, B, cs);
            q[sa] = bf.p[B][fi];
            v[sa] = ba ? vb[B][1][fi] : cell_vhat(g, prim, psi, alp, A, cs);
        }
        if (aa) {
            mc_face<double>(q[0], q[1], q[2], q[3], qBbL, qBbR);
            mc_face<double>(v[0], v[1], v[2], v[3], vaL, vaR);
        } else {
            qBbL = qBbR = q[0];
            vaL = vaR = v[0];
        }
    }
    {
        double q[4], v[4];
        const int ns = ba ? 4 : 1;
        for (int sb = 0; sb < ns; sb++) {
            int cs[3] = {c[0], c[1], c[2]};
            if (ba) cs[B] += sb - 2;
            const long long fi = face_at(g, A, cs);
            q[sb] = bf.p[A][fi];
            v[sb] = aa ? vb[A][0][fi] : cell_vhat(g, prim, psi, alp, B, cs);
        }
        if (ba) {
            mc_face<double>(q[0], q[1], q[2], q[3], qBaL, qBaR);
            mc_face<double>(v[0], v[1], v[2], v[3], vbL, vbR);
        } else {
            qBaL = qBaR = q[0];
            vbL = vbR = v[0];
        }
    }
    // speeds: each direction takes the larger alpha sqrt(gamma^dd) of its two faces at
    // the edge (1 in an inactive direction)
    const long long i0 = lin(g, c[0], c[1], c[2]);
    const long long sA = aa ? g.st[A] : 0, sB = ba ? g.st[B] : 0;
    double ca = 1.0, cb = 1.0;
    if (alp || psi) {
        double cab[2];
        edge_speeds(g, psi, alp, i0, aa, ba, sA, sB, cab);
        ca = cab[0];
        cb = cab[1];
    }
    // step (iv), the upwind formula of App. A (sqrt(gamma_hat) = 1); with c+ = c- each
    // term (c v_R q_R + c v_L q_L - c^2 (q_R - q_L)) / 2c is
    // (v_R q_R + v_L q_L - c (q_R - q_L)) / 2
    Eh[i0] = -(vaR * qBbR + vaL * qBbL - ca * (qBbR - qBbL)) * 0.5 +
             (vbR * qBaR + vbL * qBaL - cb * (qBaR - qBaL)) * 0.5;
}

// ---------------------------------------------------------------------------
// update (Sec. 2.1 sources, Sec. 3.2 CT, Sec. 2.3 stage folds): item t = cell/face t
// ---------------------------------------------------------------------------

__device__ __forceinline__ void out_value(const UpdateArgs& a, int v, long long o, double L, bool has_r)
{
    if (a.mode == UPD_WRITE_L) {
        a.L[v][o] = L;
        return;
    }
    // base_k += dt (At[k][i] L + A[k][i] R), acc += dt (wt[i] L + w[i] R), with the
    // dt products formed on the host; q^n is read at stage 0 only
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

// non-stiff sources of the 8 cell-centred variables at interior cell c (linear index
// o), added to Lc (Sec. 2.1, beta = 0, K_ij = 0): the Gauss-law charge term of s_E
// and, with a metric, s_S and s_tau.  bsrc: staggered face q_B, or cell q_B if CC.
template <bool CC>
__device__ __forceinline__ void cell_sources(const Dims& g, const double* const* prim, const double* const* bsrc,
                                             const double* __restrict__ psi, const double* __restrict__ alp,
                                             const int* c, long long o, double* Lc)
{
    const double ps = psi ? psi[o] : 1.0;
    const double al = alp ? alp[o] : 1.0;
    const double p2 = ps * ps, p4 = p2 * p2, p6 = p4 * p2;
    double u[3];
#pragma unroll
    for (int i = 0; i < 3; i++) u[i] = prim[1 + i][o];
    const double xw = 1.0 + p4 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double iW = rsqrt(xw);
    const double W = xw * iW;
    // Gauss law: sqrt(gamma) rho_e = div q_E by central differences
    double divqE = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!g.act[d]) continue;
        int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
        cp[d] += 1;
        cm[d] -= 1;
        double sp = psi ? psi[chk(g, o + g.st[d])] : 1.0, sm = psi ? psi[chk(g, o - g.st[d])] : 1.0;
        sp = sp * sp;
        sm = sm * sm;
        const double qp = sp * sp * sp * prim[5 + d][cell_at(g, cp)];
        const double qm = sm * sm * sm * prim[5 + d][cell_at(g, cm)];
        divqE += (qp - qm) * (0.5 * g.idx[d]);
    }
    // s_E (non-stiff part) = -alpha sqrt(gamma) rho_e v^i
#pragma unroll
    for (int i = 0; i < 3; i++) Lc[5 + i] -= al * divqE * (u[i] * iW);
    if (psi || alp) {
        // s_S and s_tau for beta = 0, K_ij = 0 (Sec. 2.1) in the orthonormal frame:
        //   s_S_i = psi^6 [-(tau + D) d_i alpha + 2 alpha (d_i psi / psi)(rho h W^2 v^2 + 3p + U)]
        //   s_tau = -psi^4 S_hat_i d_i alpha
        const double rho = prim[0][o], p = prim[4][o];
        const double ip4 = rcp_pos(p4), ips = ps * p2 * ip4;   // psi^-4, psi^-1
        double uh[3], Eh[3], Bh[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            uh[i] = p2 * u[i];
            Eh[i] = p2 * prim[5 + i][o];
            Bh[i] = (CC ? bsrc[i][o] : cell_qB(g, bsrc[i], i, c)) * ip4;   // psi^2 q_B / psi^6
        }
        const double rhoh = rho + g.gh * p;
        const double U = 0.5 * (Eh[0] * Eh[0] + Eh[1] * Eh[1] + Eh[2] * Eh[2] + Bh[0] * Bh[0] +
                                Bh[1] * Bh[1] + Bh[2] * Bh[2]);
        const double D = rho * W;
        const double tauD = rhoh * W * W - p + U;  // tau + D
        double S[3];
        S[0] = rhoh * W * uh[0] + (Eh[1] * Bh[2] - Eh[2] * Bh[1]);
        S[1] = rhoh * W * uh[1] + (Eh[2] * Bh[0] - Eh[0] * Bh[2]);
        S[2] = rhoh * W * uh[2] + (Eh[0] * Bh[1] - Eh[1] * Bh[0]);
        const double tr = rhoh * (uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2]) + 3.0 * p + U;
        (void)D;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            if (!g.act[i]) continue;
            const double ap = alp ? alp[chk(g, o + g.st[i])] : 1.0, am = alp ? alp[chk(g, o - g.st[i])] : 1.0;
            const double pp = psi ? psi[chk(g, o + g.st[i])] : 1.0, pm = psi ? psi[chk(g, o - g.st[i])] : 1.0;
            const double dal = (ap - am) * (0.5 * g.idx[i]);
            const double dps = (pp - pm) * (0.5 * g.idx[i]);
            Lc[1 + i] += p6 * (-tauD * dal + 2.0 * al * (dps * ips) * tr);
            Lc[4] -= p4 * S[i] * dal;
        }
    }
}

// F32: the fluxes are FP32 arrays (mixed precision).  Each difference of two FP32
// values is then exact as a double-word, and the divergence sum_d (F[o + e_d] - F[o])
// / (2 dx_d) is formed in double-word arithmetic on the FP32 pipe (about 2^-46 of its
// terms, far below the FP32 fluxes' own error) and widened by one FP64 add, in place
// of two FP64 instructions per flux.
// The same sources on the mixed-precision path, in FP32 from the stage's FP32
// primitives and cell q_B (the values its FP32 fluxes were built from), each term
// widened and added to Lc in FP64.  The metric differences d_i alpha, d_i psi are
// taken in FP64 before rounding (a slowly varying alpha would otherwise lose digits to
// cancellation); the rest carries FP32 rounding, below the FP32 fluxes' own error.
__device__ __forceinline__ void cell_sources_f32(const Dims& g, const float* const* p32,
                                                 const double* __restrict__ psi, const double* __restrict__ alp,
                                                 const int* c, long long o, double* Lc)
{
    const float ps = psi ? d2f_int(psi[o]) : 1.0f;
    const float al = alp ? d2f_int(alp[o]) : 1.0f;
    const float p2 = ps * ps, p4 = p2 * p2, p6 = p4 * p2;
    float u[3];
#pragma unroll
    for (int i = 0; i < 3; i++) u[i] = p32[1 + i][o];
    const float xw = 1.0f + p4 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const float iW = rsqrtf(xw);
    const float W = xw * iW;
    float divqE = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!g.act[d]) continue;
        int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
        cp[d] += 1;
        cm[d] -= 1;
        float sp = psi ? d2f_int(psi[chk(g, o + g.st[d])]) : 1.0f, sm = psi ? d2f_int(psi[chk(g, o - g.st[d])]) : 1.0f;
        sp = sp * sp;
        sm = sm * sm;
        const float qp = sp * sp * sp * p32[5 + d][cell_at(g, cp)];
        const float qm = sm * sm * sm * p32[5 + d][cell_at(g, cm)];
        divqE += (qp - qm) * (0.5f * d2f_int(g.idx[d]));
    }
#pragma unroll
    for (int i = 0; i < 3; i++) Lc[5 + i] -= f2d_int(al * divqE * (u[i] * iW));
    if (psi || alp) {
        const float rho = p32[0][o], p = p32[4][o];
        const float ip4 = 1.0f / p4, ips = ps * p2 * ip4;   // psi^-4, psi^-1
        float uh[3], Eh[3], Bh[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            uh[i] = p2 * u[i];
            Eh[i] = p2 * p32[5 + i][o];
            Bh[i] = p32[8 + i][o] * ip4;   // psi^2 q_B / psi^6
        }
        const float rhoh = rho + d2f_int(g.gh) * p;
        const float U = 0.5f * (Eh[0] * Eh[0] + Eh[1] * Eh[1] + Eh[2] * Eh[2] + Bh[0] * Bh[0] + Bh[1] * Bh[1] +
                                Bh[2] * Bh[2]);
        const float tauD = rhoh * W * W - p + U;   // tau + D
        float S[3];
        S[0] = rhoh * W * uh[0] + (Eh[1] * Bh[2] - Eh[2] * Bh[1]);
        S[1] = rhoh * W * uh[1] + (Eh[2] * Bh[0] - Eh[0] * Bh[2]);
        S[2] = rhoh * W * uh[2] + (Eh[0] * Bh[1] - Eh[1] * Bh[0]);
        const float tr = rhoh * (uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2]) + 3.0f * p + U;
        float s4 = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            if (!g.act[i]) continue;
            const long long op = chk(g, o + g.st[i]), om = chk(g, o - g.st[i]);
            const float hi = 0.5f * d2f_int(g.idx[i]);
            const float dal = alp ? d2f_int(alp[op] - alp[om]) * hi : 0.0f;
            const float dps = psi ? d2f_int(psi[op] - psi[om]) * hi : 0.0f;
            Lc[1 + i] += f2d_int(p6 * (-tauD * dal + 2.0f * al * (dps * ips) * tr));
            s4 += S[i] * dal;
        }
        Lc[4] -= f2d_int(p4 * s4);
    }
}

template <bool M, bool F32 = false>
__device__ __forceinline__ void update_item(const Dims& g, const UpdateArgs& a, long long t)
{
    // flat metric: alpha = psi = 1 known at compile time
    const double* __restrict__ psi = M ? a.psi : nullptr;
    const double* __restrict__ alp = M ? a.alp : nullptr;
    // cells and their upper faces: n[d] + 1 along an active d
    int c[3];
    box_coords(t, g.dvp[0], g.dvp[1], c);
#pragma unroll
    for (int d = 0; d < 3; d++) c[d] += g.ng[d];
    bool interior = true;
#pragma unroll
    for (int d = 0; d < 3; d++)
        if (c[d] >= g.ng[d] + g.n[d]) interior = false;
    const long long o = lin(g, c[0], c[1], c[2]);
    if (interior) {
        double Lc[8];
        if (F32) {
            dw acc[8];
            bool first = true;
#pragma unroll
            for (int v = 0; v < 8; v++) acc[v] = dw_make(0.0f);
#pragma unroll
            for (int d = 0; d < 3; d++) {
                if (!g.act[d]) continue;
                const long long o1 = chk(g, o + g.st[d]);
                const dw h = {g.hix[d][0], g.hix[d][1]};   // F holds twice the flux
#pragma unroll
                for (int v = 0; v < 8; v++) {
                    const float* __restrict__ Fv = reinterpret_cast<const float*>(a.F[d][v]);
                    const dw term = dw_mul(two_sum(Fv[o1], -Fv[o]), h);
                    acc[v] = first ? term : dw_add(acc[v], term);
                }
                first = false;
            }
#pragma unroll
            for (int v = 0; v < 8; v++) Lc[v] = -dw_to_double(acc[v]);
        } else {
#pragma unroll
            for (int v = 0; v < 8; v++) Lc[v] = 0.0;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                if (!g.act[d]) continue;
                const long long o1 = chk(g, o + g.st[d]);
                const double hidx = 0.5 * g.idx[d];   // F holds twice the flux
#pragma unroll
                for (int v = 0; v < 8; v++) {
                    const double* __restrict__ Fv = a.F[d][v];
                    Lc[v] -= (Fv[o1] - Fv[o]) * hidx;
                }
            }
        }
        if (F32) cell_sources_f32(g, a.p32, psi, alp, c, o, Lc);
        else cell_sources<false>(g, a.prim, a.bf, psi, alp, c, o, Lc);
#pragma unroll
        for (int v = 0; v < 8; v++) out_value(a, v, o, Lc[v], v >= 5);
    }
    // CT: d q_B^fa / dt = -d_fb hat{E}_fc + d_fc hat{E}_fb  (fa, fb, fc cyclic)
#pragma unroll
    for (int fa = 0; fa < 3; fa++) {
        const int fb = (fa + 1) % 3, fc = (fa + 2) % 3;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            int hi = g.ng[d] + g.n[d] - 1;
            if (d == fa && g.act[d] && g.bc[d] != BC_PERIODIC) hi += 1;
            if (c[d] > hi) ok = false;
        }
        if (!ok) continue;
        double r = 0.0;
        const double* __restrict__ Ec = a.Eh[fc];
        const double* __restrict__ Eb = a.Eh[fb];
        if (g.act[fb]) r -= (Ec[chk(g, o + g.st[fb])] - Ec[o]) * g.idx[fb];
        if (g.act[fc]) r += (Eb[chk(g, o + g.st[fc])] - Eb[o]) * g.idx[fc];
        out_value(a, 8 + fa, o, r, false);
    }
}

}  // namespace grmhd
