// Device-side building blocks of the resistive-MHD IMEX stage (arXiv 2110.03732).
//
// Everything here is evaluated in the local orthonormal frame of the conformally
// flat metric gamma_ij = psi^4 delta_ij (beta^i = 0): a vector X^i has orthonormal
// components X_hat = psi^2 X^i, a covector X_hat = psi^-2 X_i, so that every dot and
// cross product is the flat-space one.  Densitised conserved variables are
// q_D = psi^6 D, q_S = psi^8 S_hat, q_tau = psi^6 tau, q_E = psi^4 E_hat,
// q_B = psi^4 B_hat (Sec. 2.1 with sqrt(gamma) = psi^6 and sqrt(gamma_hat) = 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace grmhd {

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_FIXED = 2 };

// Padded grid, passed by value to every kernel.  Active directions have ng = 2 ghost
// cells per side; inactive ones have one cell and no ghosts.  Arrays are x-fastest.
struct Dims {
    int n[3], ng[3], N[3], bc[3], act[3];
    long long st[3];       // strides of x, y, z
    double idx[3];         // 1/dx (0 where inactive)
    double gh;             // Gamma_hat_1 = Gamma/(Gamma - 1)
    double igh;            // 1/Gamma_hat_1
    long long ncell;       // padded cells
};

struct P8 { double* p[8]; };          // rho, u^1..3, p, E^1..3  (or 8 conserved)
struct P3 { double* p[3]; };          // three face / edge / R arrays
struct CP8 { const double* p[8]; };
struct CP3 { const double* p[3]; };

// ---------------------------------------------------------------------------
// boundary conditions applied on read: periodic wraps, outflow clamps to the last
// interior cell (last real face for a face along its own direction), fixed reads
// the stored ghost value
// ---------------------------------------------------------------------------

__device__ __forceinline__ int map_cell(const Dims& g, int d, int m)
{
    if (!g.act[d]) return 0;
    const int lo = g.ng[d], n = g.n[d];
    if (g.bc[d] == BC_PERIODIC) {
        int r = (m - lo) % n;
        return lo + (r < 0 ? r + n : r);
    }
    if (g.bc[d] == BC_OUTFLOW) return m < lo ? lo : (m > lo + n - 1 ? lo + n - 1 : m);
    return m;
}

__device__ __forceinline__ int map_face(const Dims& g, int d, int m)
{
    if (!g.act[d]) return 0;
    const int lo = g.ng[d], n = g.n[d];
    if (g.bc[d] == BC_PERIODIC) {
        int r = (m - lo) % n;
        return lo + (r < 0 ? r + n : r);
    }
    if (g.bc[d] == BC_OUTFLOW) return m < lo ? lo : (m > lo + n ? lo + n : m);
    return m;
}

__device__ __forceinline__ long long lin(const Dims& g, int i, int j, int k)
{
    return (long long)i + g.st[1] * j + g.st[2] * k;
}

// mapped cell index of padded coordinates c[3]
__device__ __forceinline__ long long cell_at(const Dims& g, const int* c)
{
    return lin(g, map_cell(g, 0, c[0]), map_cell(g, 1, c[1]), map_cell(g, 2, c[2]));
}

// mapped index of the face array of direction fd at padded coordinates c[3]
__device__ __forceinline__ long long face_at(const Dims& g, int fd, const int* c)
{
    int m[3];
#pragma unroll
    for (int d = 0; d < 3; d++) m[d] = (d == fd) ? map_face(g, d, c[d]) : map_cell(g, d, c[d]);
    return lin(g, m[0], m[1], m[2]);
}

// cell-centred q_B^e of the cell at padded coordinates c: the cell is mapped first,
// then the mean of its two e-faces (the lower face alone where the upper one lies
// outside a fixed-boundary array); an inactive e stores the cell value itself
__device__ __forceinline__ double cell_qB(const Dims& g, const double* __restrict__ bf, int e, const int* c)
{
    int m[3];
#pragma unroll
    for (int d = 0; d < 3; d++) m[d] = map_cell(g, d, c[d]);
    const long long i0 = lin(g, m[0], m[1], m[2]);
    if (!g.act[e]) return bf[i0];
    int h = m[e] + 1;
    if (g.bc[e] == BC_PERIODIC && h == g.ng[e] + g.n[e]) h = g.ng[e];
    if (h >= g.N[e]) return bf[i0];
    const long long i1 = i0 + (long long)(h - m[e]) * g.st[e];
    return 0.5 * (bf[i0] + bf[i1]);
}

// ---------------------------------------------------------------------------
// MC limiter (monotonised central, van Leer 1974)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double minmod3(double a, double b, double c)
{
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

__device__ __forceinline__ double mc_slope(double um, double u0, double up)
{
    return minmod3(2.0 * (u0 - um), 0.5 * (up - um), 2.0 * (up - u0));
}

// left/right states at the face between a1 and a2 from the four cells a0 a1 a2 a3
__device__ __forceinline__ void mc_face(double a0, double a1, double a2, double a3, double& L, double& R)
{
    L = a1 + 0.5 * mc_slope(a0, a1, a2);
    R = a2 - 0.5 * mc_slope(a1, a2, a3);
}

// ---------------------------------------------------------------------------
// physical state at a face in the orthonormal frame (Sec. 2.1)
// ---------------------------------------------------------------------------

struct FaceState {
    double q[8];    // densitised conserved: D, S_1..3, tau, E^1..3
    double f[8];    // flux of the same along the face normal
};

// prim: rho, u^1..3, p, E^1..3 (coordinate components) and B^1..3 (coordinate);
// psi, alpha at the face; d = normal direction
__device__ __forceinline__ void face_state(const double* pr, const double* B, int d, double psi, double alp,
                                           double gh, FaceState& s)
{
    const double p2 = psi * psi, p4 = p2 * p2, p6 = p4 * p2;
    const double rho = pr[0], p = pr[4];
    double u[3], E[3], Bh[3];
#pragma unroll
    for (int i = 0; i < 3; i++) { u[i] = p2 * pr[1 + i]; E[i] = p2 * pr[5 + i]; Bh[i] = p2 * B[i]; }
    const double W = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double iW = 1.0 / W;
    const double rhoh = rho + gh * p;
    const double D = rho * W;
    const double U = 0.5 * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + Bh[0] * Bh[0] + Bh[1] * Bh[1] + Bh[2] * Bh[2]);
    double S[3];
    S[0] = rhoh * W * u[0] + (E[1] * Bh[2] - E[2] * Bh[1]);
    S[1] = rhoh * W * u[1] + (E[2] * Bh[0] - E[0] * Bh[2]);
    S[2] = rhoh * W * u[2] + (E[0] * Bh[1] - E[1] * Bh[0]);
    const double tau = rhoh * W * W - p + U - D;
    s.q[0] = p6 * D;
#pragma unroll
    for (int j = 0; j < 3; j++) s.q[1 + j] = p6 * p2 * S[j];
    s.q[4] = p6 * tau;
#pragma unroll
    for (int j = 0; j < 3; j++) s.q[5 + j] = p4 * E[j];
    // fluxes along d (beta = 0)
    const double vd = u[d] * iW;
    const double rhw2 = rhoh * W * W;
    s.f[0] = p4 * alp * D * vd;
#pragma unroll
    for (int j = 0; j < 3; j++)
        s.f[1 + j] = p6 * alp * ((j == d ? p + U : 0.0) + rhw2 * vd * (u[j] * iW) - E[d] * E[j] - Bh[d] * Bh[j]);
    s.f[4] = p4 * alp * (S[d] - vd * D);
    // (f_E^j)^d = alpha psi^2 eta^{djk} B_hat_k
    const double ap2 = alp * p2;
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    s.f[5 + d] = 0.0;
    s.f[5 + d1] = ap2 * Bh[d2];
    s.f[5 + d2] = -ap2 * Bh[d1];
}

// ---------------------------------------------------------------------------
// implicit electric field + velocity solve (Sec. 2.4), xi = 0, orthonormal frame
// ---------------------------------------------------------------------------

struct CellIn {
    double D, S[3], tau, Es[3], B[3];   // undensitised orthonormal components
    double etat;                        // eta / (alpha a_ii dt); < 0: E held fixed
    double gh, igh;
};

struct Eval {
    double W, E[3], wt, U, A1, iWe, iden, Esu, f[3], g;
    double fm;   // max |f_i|
    double M;    // momentum scale of f: max(|S_i|, |(E x B)_i|, |w_t u_i|)
};

// E(u) from A_0 E = eta_t E* + A_1 (E*.u) u - u x B with A_0 = W + eta_t,
// A_1 = eta_t/(1 + eta_t W); then w_tilde and f = w_tilde u - S + E x B
__device__ __forceinline__ void evaluate(const CellIn& c, const double* u, Eval& e)
{
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    e.W = sqrt(1.0 + uu);
    if (c.etat >= 0.0) {
        e.iWe = 1.0 / (e.W + c.etat);
        e.A1 = c.etat / (1.0 + c.etat * e.W);
        e.Esu = c.Es[0] * u[0] + c.Es[1] * u[1] + c.Es[2] * u[2];
        const double a = e.A1 * e.Esu;
        e.E[0] = (c.etat * c.Es[0] + a * u[0] - (u[1] * c.B[2] - u[2] * c.B[1])) * e.iWe;
        e.E[1] = (c.etat * c.Es[1] + a * u[1] - (u[2] * c.B[0] - u[0] * c.B[2])) * e.iWe;
        e.E[2] = (c.etat * c.Es[2] + a * u[2] - (u[0] * c.B[1] - u[1] * c.B[0])) * e.iWe;
    } else {
        e.iWe = 0.0; e.A1 = 0.0; e.Esu = 0.0;
        e.E[0] = c.Es[0]; e.E[1] = c.Es[1]; e.E[2] = c.Es[2];
    }
    e.U = 0.5 * (e.E[0] * e.E[0] + e.E[1] * e.E[1] + e.E[2] * e.E[2] + c.B[0] * c.B[0] + c.B[1] * c.B[1] +
                 c.B[2] * c.B[2]);
    e.iden = 1.0 / (uu + 1.0 - c.igh);
    e.wt = (e.W * (c.tau + c.D - e.U) - c.D * c.igh) * e.iden;
    const double x0 = e.E[1] * c.B[2] - e.E[2] * c.B[1];
    const double x1 = e.E[2] * c.B[0] - e.E[0] * c.B[2];
    const double x2 = e.E[0] * c.B[1] - e.E[1] * c.B[0];
    const double w0 = e.wt * u[0], w1 = e.wt * u[1], w2 = e.wt * u[2];
    e.f[0] = w0 - c.S[0] + x0;
    e.f[1] = w1 - c.S[1] + x1;
    e.f[2] = w2 - c.S[2] + x2;
    e.g = e.f[0] * e.f[0] + e.f[1] * e.f[1] + e.f[2] * e.f[2];
    e.fm = fmax(fabs(e.f[0]), fmax(fabs(e.f[1]), fabs(e.f[2])));
    e.M = fmax(fmax(fmax(fabs(c.S[0]), fabs(c.S[1])), fmax(fabs(c.S[2]), fabs(x0))),
               fmax(fmax(fabs(x1), fabs(x2)), fmax(fabs(w0), fmax(fabs(w1), fabs(w2)))));
}

// Jacobian J_ij = w_t delta_ij + u_i dw_t/du_j + (dE/du_j x B)_i
__device__ __forceinline__ void jacobian(const CellIn& c, const double* u, const Eval& e, double J[3][3])
{
    const double iW = 1.0 / e.W;
    double dE[3][3];   // dE_i / du_j
    if (c.etat >= 0.0) {
        // W (W + eta_t) dE_i/du_j = -E_i u_j + A_1 W u_i E*_j + (A_1 W delta_ij - A_1^2 u_i u_j)(E*.u)
        //                          - W eps_ijl B_l
        const double A1 = e.A1, a2 = A1 * A1 * e.Esu * iW;
        const double s = e.iWe;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                dE[i][j] = (-e.E[i] * u[j] * iW + A1 * u[i] * c.Es[j] - a2 * u[i] * u[j] +
                            (i == j ? A1 * e.Esu : 0.0)) * s;
        // - eps_ijl B_l / (W + eta_t)
        dE[0][1] -= c.B[2] * s; dE[0][2] += c.B[1] * s;
        dE[1][2] -= c.B[0] * s; dE[1][0] += c.B[2] * s;
        dE[2][0] -= c.B[1] * s; dE[2][1] += c.B[0] * s;
    } else {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) dE[i][j] = 0.0;
    }
    const double base = c.tau + c.D - e.U;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const double dU = e.E[0] * dE[0][j] + e.E[1] * dE[1][j] + e.E[2] * dE[2][j];
        const double dwt = (base * u[j] * iW - e.W * dU - 2.0 * e.wt * u[j]) * e.iden;
        // (dE/du_j x B)
        const double cx = dE[1][j] * c.B[2] - dE[2][j] * c.B[1];
        const double cy = dE[2][j] * c.B[0] - dE[0][j] * c.B[2];
        const double cz = dE[0][j] * c.B[1] - dE[1][j] * c.B[0];
        J[0][j] = u[0] * dwt + cx;
        J[1][j] = u[1] * dwt + cy;
        J[2][j] = u[2] * dwt + cz;
    }
    J[0][0] += e.wt; J[1][1] += e.wt; J[2][2] += e.wt;
}

// x = -J^{-1} f by the adjugate; returns false for a singular J
__device__ __forceinline__ bool newton_dir(const double J[3][3], const double* f, double* x)
{
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(fabs(det) > 0.0)) return false;
    const double id = -1.0 / det;
    const double c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    const double c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    const double c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    const double c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    const double c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    const double c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    x[0] = (c00 * f[0] + c10 * f[1] + c20 * f[2]) * id;
    x[1] = (c01 * f[0] + c11 * f[1] + c21 * f[2]) * id;
    x[2] = (c02 * f[0] + c12 * f[1] + c22 * f[2]) * id;
    return true;
}

// Globally convergent Newton (backtracking on |f|^2 with the Armijo condition and a
// bounded step).  u: in = initial guess, out = solution.  Converged when |f| is at
// `tol` against its own momentum scale M, or when the step no longer moves u.
// Returns iterations, or -1.
__device__ __forceinline__ int newton_solve(const CellIn& c, double* u, Eval& e, int kmax, double tol)
{
    evaluate(c, u, e);
    for (int it = 1; it <= kmax; it++) {
        double J[3][3], dx[3];
        jacobian(c, u, e, J);
        if (!newton_dir(J, e.f, dx)) return -1;
        const double nu = fmax(1.0, sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
        const double nx = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
        if (nx > 100.0 * nu) {
            const double s = 100.0 * nu / nx;
            dx[0] *= s; dx[1] *= s; dx[2] *= s;
        }
        // slope of |f|^2 along the Newton direction is -2|f|^2
        const double g0 = e.g;
        double lam = 1.0, ut[3];
        Eval et;
        for (int ls = 0; ls < 30; ls++) {
            ut[0] = u[0] + lam * dx[0]; ut[1] = u[1] + lam * dx[1]; ut[2] = u[2] + lam * dx[2];
            evaluate(c, ut, et);
            if (et.g <= g0 * (1.0 - 2e-4 * lam) || !(g0 > 0.0)) break;
            double lq = g0 * lam * lam / (et.g - g0 + 2.0 * g0 * lam);
            if (!(lq == lq)) lq = 0.5 * lam;
            lam = fmin(fmax(lq, 0.1 * lam), 0.5 * lam);
        }
        const double step = lam * fmax(fabs(dx[0]), fmax(fabs(dx[1]), fabs(dx[2])));
        u[0] = ut[0]; u[1] = ut[1]; u[2] = ut[2];
        e = et;
        const double umax = fmax(fabs(u[0]), fmax(fabs(u[1]), fabs(u[2])));
        if (e.fm <= tol * e.M || step <= 1e-15 * umax) {
            if (!(e.wt > 0.0) || !(e.W < 1e10)) return -1;
            return it;
        }
    }
    return -1;
}

}  // namespace grmhd
