/*
 * grmhd_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU statement of one IMEX Runge-Kutta step of
 * resistive (general-relativistic) MHD on a uniform Cartesian grid with a fixed,
 * conformally flat background metric (gamma_ij = psi^4 delta_ij, beta^i = 0),
 * staggered face magnetic fields and upwind constrained transport (or, as a
 * variant, cell-centred magnetic fields with GLM hyperbolic cleaning), following
 * arXiv 2110.03732 (Cheong et al., "Gmunu: ... resistive GRMHD").
 *
 * Only tests, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use this
 * file.  It shares no code with the CUDA path: it has its own structs, its own
 * index arithmetic and its own statement of every formula, written in the
 * paper's coordinate-component notation (indices raised/lowered with
 * gamma_ij = psi^4 delta_ij explicitly), with every intermediate stored in full
 * arrays and no fusion.
 *
 * Paper passages followed (section / equation):
 *   conserved variables, fluxes, sources          Sec. 2.1 (q, f^i, s; Gauss law for rho_e)
 *   Ohm's law with the mean-field dynamo xi       Sec. 2.2
 *   IMEX-RK stages, SSP2(2,2,2) tableau           Sec. 2.3 (Table "IMEX-SSP2(2,2,2)")
 *   implicit E + velocity Newton, A_k, Jacobian   Sec. 2.4 (eq. im_E, f_i, J_ij)
 *   characteristic speeds (maximal diffusivity)   Sec. 2.5
 *   constrained transport, UCT-HLL edge EMF       Sec. 3.2 (steps i-vii)
 *   GLM hyperbolic cleaning (cell-centred B, Phi) Sec. 3.1 (q_Phi, f_Phi, s_Phi, s_B)
 *   B from an edge vector potential               Sec. 4
 *   MC limiter + HLL defaults                     Sec. 5 (opening paragraph)
 *   ideal-limit HLL UCT (transport velocities)    App. A (steps i-iv)
 *   PPM reconstruction (named for the star runs)  Sec. 5; Colella & Woodward (1984)
 *
 * Readings where the paper is silent or garbled:
 *   - IMEX sum limits: q(i) = q^n + dt sum_{j<i} at_ij L(j) + dt sum_{j<=i} a_ij R(j),
 *     q^{n+1} = q^n + dt sum_i (wt_i L(i) + w_i R(i))  (Pareschi-Russo form).
 *   - eta_tilde = eta / (alpha a_ii dt) inside stage i.
 *   - the implicit E equation carries a minus sign in front of W/eta_tilde; the
 *     A_k printed in Sec. 2.4 are consistent with that sign.
 *   - d(U_EM)/du^j = E_i dE^i/du^j in the derivative of w_tilde.
 *   - HLL speeds c+ = max(0, lambda+), c- = max(0, -lambda-) with lambda from Sec. 2.5,
 *     the metric averaged linearly to faces; at an edge each direction takes the
 *     larger speed of its two adjacent faces.
 *   - reconstructed: rho, u^i (= W v^i), p, E^i and the two transverse cell-centred B^i;
 *     the normal B at a face is the staggered value.  For the edge EMF the covariant
 *     E_c = psi^4 E^c is reconstructed (face, then edge) and multiplied by the lapse
 *     averaged to the edge.
 *   - cell-centred B = mean of the two staggered faces.
 *   - rho_e from a central difference of cell-centred q_E (Gauss law).
 *   - ghost cells: periodic, outflow (copy of the nearest interior cell) or fixed
 *     (left as given).
 *   - Newton: analytic Jacobian, backtracking line search on 0.5|f|^2 with the Armijo
 *     condition and a bounded step (Press et al., "globally convergent Newton");
 *     initial guess = the previous stage's velocity, from rest as the fallback;
 *     converged when |f| is at round-off against the momentum terms it balances.
 *   - atmosphere (not described in the paper): with rho_atm > 0, a cell whose
 *     D < 10 rho_atm, or whose solve fails, is set to rest at (rho_atm, p_atm) with E
 *     kept and no stiff update.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NQ 8         /* cell-centred conserved: D, S_1..3, tau, E^1..3 */
#define NPR 8        /* cell-centred primitives: rho, u^1..3, p, E^1..3 */
#define NREC 11      /* reconstructed: the 8 primitives + B^1..3 (normal one unused) */
#define MAXS 4

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_FIXED = 2 };

typedef struct {
    int ndim;
    int n[3], ng[3], N[3], act[3], bc[3];
    double dx[3];
    double Gam;        /* ideal-gas adiabatic index Gamma */
    double rho_atm;    /* atmosphere density (0: no atmosphere treatment) */
    double p_atm;      /* atmosphere pressure */
    double xi;         /* mean-field dynamo parameter (uniform) */
    int emf;           /* edge EMF: 0 = resistive UCT (Sec. 3.2), 1 = ideal-limit UCT (App. A) */
    int rec;           /* reconstruction: 0 = MC (Sec. 5 default), 1 = PPM (Sec. 5, star runs) */
    long ncell;        /* padded cells */
} OGrid;

static void grid_setup(OGrid* g, const int* gi, const double* gd)
{
    g->ndim = gi[0];
    for (int d = 0; d < 3; d++) {
        g->n[d] = gi[1 + d];
        g->bc[d] = gi[4 + d];
        g->act[d] = (d < g->ndim) ? 1 : 0;
        g->ng[d] = g->act[d] ? 2 : 0;
        g->N[d] = g->n[d] + 2 * g->ng[d];
        g->dx[d] = gd[d];
    }
    g->Gam = gd[3];
    g->rho_atm = gd[4];
    g->p_atm = gd[5];
    g->xi = gd[6];
    g->emf = (int)gd[7];
    g->rec = (int)gd[8];
    g->ncell = (long)g->N[0] * g->N[1] * g->N[2];
}

static long at(const OGrid* g, int i, int j, int k) { return i + (long)g->N[0] * (j + (long)g->N[1] * k); }

static long shift(const OGrid* g, long c, int d, int s)
{
    long st = (d == 0) ? 1 : (d == 1) ? g->N[0] : (long)g->N[0] * g->N[1];
    return c + s * st;
}

static void coords(const OGrid* g, long c, int* ijk)
{
    ijk[0] = (int)(c % g->N[0]);
    ijk[1] = (int)((c / g->N[0]) % g->N[1]);
    ijk[2] = (int)(c / ((long)g->N[0] * g->N[1]));
}

static int is_interior(const OGrid* g, const int* ijk)
{
    for (int d = 0; d < 3; d++)
        if (ijk[d] < g->ng[d] || ijk[d] >= g->ng[d] + g->n[d]) return 0;
    return 1;
}

static double* dalloc(long n) { return (double*)calloc((size_t)n, sizeof(double)); }

/* ------------------------------------------------------------------ */
/* ghost cells                                                          */
/* ------------------------------------------------------------------ */

/* cell-centred array: fill the ghost layers of each active direction in turn */
static void fill_cell_ghosts(const OGrid* g, double* a)
{
    for (int d = 0; d < 3; d++) {
        if (!g->act[d] || g->bc[d] == BC_FIXED) continue;
        int ijk[3];
        for (long c = 0; c < g->ncell; c++) {
            coords(g, c, ijk);
            int m = ijk[d], lo = g->ng[d], hi = g->ng[d] + g->n[d] - 1;
            if (m >= lo && m <= hi) continue;
            int src;
            if (g->bc[d] == BC_PERIODIC) {
                src = lo + (((m - lo) % g->n[d]) + g->n[d]) % g->n[d];
            } else {
                src = m < lo ? lo : hi;
            }
            int s3[3] = {ijk[0], ijk[1], ijk[2]};
            s3[d] = src;
            a[c] = a[at(g, s3[0], s3[1], s3[2])];
        }
    }
}

/* face array of direction fd: along fd the faces ng..ng+n are real (ng+n is a copy
 * of ng when periodic); across fd it behaves like a cell array */
static void fill_face_ghosts(const OGrid* g, double* a, int fd)
{
    for (int d = 0; d < 3; d++) {
        if (!g->act[d] || g->bc[d] == BC_FIXED) continue;
        int ijk[3];
        for (long c = 0; c < g->ncell; c++) {
            coords(g, c, ijk);
            int m = ijk[d], lo = g->ng[d];
            int hi = (d == fd) ? g->ng[d] + g->n[d] : g->ng[d] + g->n[d] - 1;
            int src;
            if (g->bc[d] == BC_PERIODIC) {
                if (d == fd) {
                    if (m >= lo && m < lo + g->n[d]) continue;
                } else if (m >= lo && m <= hi) {
                    continue;
                }
                src = lo + (((m - lo) % g->n[d]) + g->n[d]) % g->n[d];
            } else {
                if (m >= lo && m <= hi) continue;
                src = m < lo ? lo : hi;
            }
            int s3[3] = {ijk[0], ijk[1], ijk[2]};
            s3[d] = src;
            a[c] = a[at(g, s3[0], s3[1], s3[2])];
        }
    }
}

/* cell-centred conserved q_B from the staggered faces: mean of the two faces of the
 * cell in each active direction (the upper face taken alone where it is outside the
 * padded array), the face value itself in an inactive direction; then ghost fill */
static void cell_qB(const OGrid* g, double* const* bf, double** qBc)
{
    int ijk[3];
    for (int d = 0; d < 3; d++) {
        for (long c = 0; c < g->ncell; c++) {
            if (!g->act[d]) { qBc[d][c] = bf[d][c]; continue; }
            coords(g, c, ijk);
            if (ijk[d] + 1 < g->N[d])
                qBc[d][c] = 0.5 * (bf[d][c] + bf[d][shift(g, c, d, 1)]);
            else
                qBc[d][c] = bf[d][c];
        }
        fill_cell_ghosts(g, qBc[d]);
    }
}

/* ------------------------------------------------------------------ */
/* metric helpers: gamma_ij = psi^4 delta_ij, sqrt(gamma) = psi^6        */
/* ------------------------------------------------------------------ */

static double psi_at(const double* psi, long c) { return psi ? psi[c] : 1.0; }
static double alp_at(const double* alp, long c) { return alp ? alp[c] : 1.0; }

/* Levi-Civita symbol eta^{ijk} */
static double levi(int i, int j, int k)
{
    if (i == j || j == k || i == k) return 0.0;
    if ((i == 0 && j == 1 && k == 2) || (i == 1 && j == 2 && k == 0) || (i == 2 && j == 0 && k == 1)) return 1.0;
    return -1.0;
}

/* ------------------------------------------------------------------ */
/* prim -> cons (Sec. 2.1 definitions of q)                              */
/* ------------------------------------------------------------------ */

/* prim: rho, u^i (=W v^i, contravariant), p, E^i; B^i contravariant; out: densitised q */
static void prim2con_point(const double* pr, const double* B, double psi, double Gam, double* q)
{
    double g = psi * psi * psi * psi, sg = g * psi * psi;
    double rho = pr[0], p = pr[4];
    double uu = 0, E2 = 0, B2 = 0;
    for (int i = 0; i < 3; i++) {
        uu += g * pr[1 + i] * pr[1 + i];
        E2 += g * pr[5 + i] * pr[5 + i];
        B2 += g * B[i] * B[i];
    }
    double W = sqrt(1.0 + uu);
    double h = 1.0 + Gam / (Gam - 1.0) * p / rho;
    double D = rho * W;
    double v_lo[3], E_lo[3], B_lo[3];
    for (int i = 0; i < 3; i++) { v_lo[i] = g * pr[1 + i] / W; E_lo[i] = g * pr[5 + i]; B_lo[i] = g * B[i]; }
    (void)E_lo; (void)B_lo;
    double S[3];
    for (int j = 0; j < 3; j++) {
        double exb = 0;
        for (int k = 0; k < 3; k++)
            for (int l = 0; l < 3; l++) exb += levi(j, k, l) * pr[5 + k] * B[l];
        S[j] = rho * h * W * W * v_lo[j] + sg * exb;     /* S_j = rho h W^2 v_j + sqrt(gamma) eta_jkl E^k B^l */
    }
    double tau = rho * h * W * W - p + 0.5 * (E2 + B2) - D;
    q[0] = sg * D;
    for (int j = 0; j < 3; j++) q[1 + j] = sg * S[j];
    q[4] = sg * tau;
    for (int j = 0; j < 3; j++) q[5 + j] = sg * pr[5 + j];
}

/* ------------------------------------------------------------------ */
/* implicit step (Sec. 2.4), xi = 0                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    double D, S[3], tau, Es[3], B[3];  /* undensitised; S covariant, Es, B contravariant */
    double g;                          /* psi^4 */
    double sg;                         /* psi^6 */
    double etat;                       /* eta_tilde; < 0 means E held fixed (E = E*) */
    double xi;                         /* mean-field dynamo parameter (Sec. 2.2) */
    double Gh;                         /* Gamma_hat_1 = Gamma/(Gamma-1) */
} OCell;

/* E(u) from eq. im_E:
 *   A_0 E^i = eta_t E*^i + A_1 (E*_k u^k) u^i + A_2 eps^{ijk} u_j E*_k + A_3 B^i
 *             + A_4 (B_k u^k) u^i + A_5 eps^{ijk} u_j B_k
 * with the A_k(W) of Sec. 2.4, and its derivative dE^i/du^j from the Sec. 2.4
 * expression (with the A_k' printed there).  Returns W. */
static double efield(const OCell* c, const double* u, double* E, double dE[3][3])
{
    double g = c->g, sg = c->sg;
    double uu = 0;
    for (int i = 0; i < 3; i++) uu += g * u[i] * u[i];
    double W = sqrt(1.0 + uu);
    double u_lo[3], B_lo[3], Es_lo[3];
    for (int i = 0; i < 3; i++) { u_lo[i] = g * u[i]; B_lo[i] = g * c->B[i]; Es_lo[i] = g * c->Es[i]; }
    if (c->etat < 0) {
        for (int i = 0; i < 3; i++) {
            E[i] = c->Es[i];
            if (dE) for (int j = 0; j < 3; j++) dE[i][j] = 0.0;
        }
        return W;
    }
    double et = c->etat, xi = c->xi, x2 = xi * xi;
    double p = W + et, q = 1.0 + et * W;
    double A0 = W + et + x2 * (W * W - 1.0) / p;
    double A1 = et / q + x2 * et * W / (p * q);
    double A2 = -xi * et / p;
    double A3 = xi * q / p;
    double A4 = xi * (1.0 - et * et + x2) / (p * q);
    double A5 = -1.0 - x2 * W / p;
    double A0d = 1.0 + x2 * (1.0 + W * W + 2.0 * W * et) / (p * p);
    double A1d = -et * et / (q * q) - x2 * et * et * (W * W - 1.0) / (q * q * p * p);
    double A2d = xi * et / (p * p);
    double A3d = xi * (et * et - 1.0) / (p * p);
    double A4d = -xi * (1.0 - et * et + x2) * (1.0 + et * et + 2.0 * W * et) / (q * q * p * p);
    double A5d = -x2 * et / (p * p);
    double Esu = 0, Bu = 0, eps_uEs[3], eps_uB[3];
    for (int k = 0; k < 3; k++) { Esu += Es_lo[k] * u[k]; Bu += B_lo[k] * u[k]; }
    for (int i = 0; i < 3; i++) {
        double s1 = 0, s2 = 0;
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) {
                s1 += levi(i, j, k) / sg * u_lo[j] * Es_lo[k];
                s2 += levi(i, j, k) / sg * u_lo[j] * B_lo[k];
            }
        eps_uEs[i] = s1;
        eps_uB[i] = s2;
    }
    for (int i = 0; i < 3; i++)
        E[i] = (et * c->Es[i] + A1 * Esu * u[i] + A2 * eps_uEs[i] + A3 * c->B[i] + A4 * Bu * u[i] + A5 * eps_uB[i]) / A0;
    if (dE) {
        /* A_0 W dE^i/du^j = -A0' E^i u_j + A_1 W u^i E*_j + A3' B^i u_j + A_4 W u^i B_j
         *   + (A_1 W delta^i_j + A1' u^i u_j)(E*_k u^k) + eps^{ilm}(A_2 W gamma_lj + A2' u_l u_j) E*_m
         *   + (A_4 W delta^i_j + A4' u^i u_j)(B_k u^k) + eps^{ilm}(A_5 W gamma_lj + A5' u_l u_j) B_m */
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double dl = (i == j ? 1.0 : 0.0);
                double t = -A0d * E[i] * u_lo[j] + A1 * W * u[i] * Es_lo[j] + A3d * c->B[i] * u_lo[j]
                           + A4 * W * u[i] * B_lo[j]
                           + (A1 * W * dl + A1d * u[i] * u_lo[j]) * Esu
                           + (A4 * W * dl + A4d * u[i] * u_lo[j]) * Bu;
                double s = 0;
                for (int l = 0; l < 3; l++)
                    for (int m = 0; m < 3; m++) {
                        double glj = (l == j ? g : 0.0);
                        s += levi(i, l, m) / sg * ((A2 * W * glj + A2d * u_lo[l] * u_lo[j]) * Es_lo[m]
                                                   + (A5 * W * glj + A5d * u_lo[l] * u_lo[j]) * B_lo[m]);
                    }
                dE[i][j] = (t + s) / (A0 * W);
            }
    }
    return W;
}

/* residual f_i(u) = w_t gamma_ij u^j - (S_i - eps_ilm E^l B^m) and, if J != NULL, J_ij */
static void residual(const OCell* c, const double* u, double* f, double J[3][3], double* E, double* W_out, double* wt_out)
{
    double g = c->g, sg = c->sg, Gh = c->Gh;
    double dE[3][3];
    double W = efield(c, u, E, J ? dE : NULL);
    double E2 = 0, B2 = 0;
    for (int i = 0; i < 3; i++) { E2 += g * E[i] * E[i]; B2 += g * c->B[i] * c->B[i]; }
    double U = 0.5 * (E2 + B2);
    double den = W * W - 1.0 / Gh;
    double wt = (W * (c->tau + c->D - U) - c->D / Gh) / den;
    double u_lo[3];
    for (int i = 0; i < 3; i++) u_lo[i] = g * u[i];
    double eEB[3];
    for (int i = 0; i < 3; i++) {
        double s = 0;
        for (int l = 0; l < 3; l++)
            for (int m = 0; m < 3; m++) s += sg * levi(i, l, m) * E[l] * c->B[m];
        eEB[i] = s;
        f[i] = wt * u_lo[i] - (c->S[i] - eEB[i]);
    }
    if (J) {
        double dwt[3];
        for (int j = 0; j < 3; j++) {
            double dU = 0;
            for (int i = 0; i < 3; i++) dU += g * E[i] * dE[i][j];
            dwt[j] = ((c->tau + c->D - U) * u_lo[j] / W - 2.0 * wt * u_lo[j] - W * dU) / den;
        }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double s = 0;
                for (int l = 0; l < 3; l++)
                    for (int m = 0; m < 3; m++) s += sg * levi(i, l, m) * dE[l][j] * c->B[m];
                J[i][j] = wt * (i == j ? g : 0.0) + u_lo[i] * dwt[j] + s;
            }
    }
    if (W_out) *W_out = W;
    if (wt_out) *wt_out = wt;
}

/* Gaussian elimination with partial pivoting: solves M x = b (M, b copied) */
static int solve3(double M[3][3], const double* b, double* x)
{
    double a[3][4];
    for (int i = 0; i < 3; i++) { for (int j = 0; j < 3; j++) a[i][j] = M[i][j]; a[i][3] = b[i]; }
    for (int col = 0; col < 3; col++) {
        int piv = col;
        for (int r = col + 1; r < 3; r++) if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col) for (int j = 0; j < 4; j++) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
        for (int r = col + 1; r < 3; r++) {
            double fct = a[r][col] / a[col][col];
            for (int j = col; j < 4; j++) a[r][j] -= fct * a[col][j];
        }
    }
    for (int i = 2; i >= 0; i--) {
        double s = a[i][3];
        for (int j = i + 1; j < 3; j++) s -= a[i][j] * x[j];
        x[i] = s / a[i][i];
    }
    return 0;
}

static double half_norm2(const double* f) { return 0.5 * (f[0] * f[0] + f[1] * f[1] + f[2] * f[2]); }

/* globally convergent Newton on f(u) = 0; returns iterations (>0) or -1 on failure.
 * in: u = initial guess; out: u (contravariant), E (contravariant), rho, p */
static int newton_cell(const OCell* c, double* u, double* E, double* rho, double* p, int kmax, double tol)
{
    double f[3], J[3][3], W, wt;
    /* u holds the initial guess on entry (the caller's previous-stage velocity, or
     * rest: at u = 0, E(0) = eta_t E_star / (1 + eta_t) stays finite in both the
     * stiff and the non-stiff limits) */
    int it;
    for (it = 1; it <= kmax; it++) {
        residual(c, u, f, J, E, &W, &wt);
        double g0 = half_norm2(f);
        double dx[3], mf[3] = {-f[0], -f[1], -f[2]};
        if (solve3(J, mf, dx) != 0) return -1;
        /* step bound (Press et al.): |dx| <= 100 max(|u|, 1) */
        {
            double nx = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
            double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            double mx = 100.0 * (nu > 1.0 ? nu : 1.0);
            if (nx > mx) for (int i = 0; i < 3; i++) dx[i] *= mx / nx;
        }
        /* backtracking: Armijo condition with slope grad(g).dx = -|f|^2 */
        double slope = -2.0 * g0, lam = 1.0, un[3], fn[3], En[3];
        for (int ls = 0; ls < 40; ls++) {
            for (int i = 0; i < 3; i++) un[i] = u[i] + lam * dx[i];
            residual(c, un, fn, NULL, En, NULL, NULL);
            double g1 = half_norm2(fn);
            if (g1 <= g0 + 1e-4 * lam * slope || !(g0 > 0)) break;
            double lq = -slope * lam * lam / (2.0 * (g1 - g0 - slope * lam));
            if (!(lq == lq)) lq = 0.5 * lam;
            if (lq < 0.1 * lam) lq = 0.1 * lam;
            if (lq > 0.5 * lam) lq = 0.5 * lam;
            lam = lq;
        }
        double dn = 0;
        for (int i = 0; i < 3; i++) {
            double s = lam * dx[i];
            dn += s * s;
            u[i] = un[i];
        }
        /* f_i has momentum units: it is converged when it is at round-off against the
         * momentum terms it balances (|S_i|, |eps_ilm E^l B^m|, |w_t u_i|); a step that
         * no longer moves u also ends the iteration */
        residual(c, u, f, NULL, E, &W, &wt);
        double M = 0, fm = 0, um = 0;
        for (int i = 0; i < 3; i++) {
            double exb = 0;
            for (int l = 0; l < 3; l++)
                for (int m = 0; m < 3; m++) exb += c->sg * levi(i, l, m) * E[l] * c->B[m];
            M = fmax(M, fmax(fabs(c->S[i]), fmax(fabs(exb), fabs(wt * c->g * u[i]))));
            fm = fmax(fm, fabs(f[i]));
            um = fmax(um, fabs(u[i]));
        }
        if (fm <= tol * M) break;
        if (sqrt(dn) <= 1e-15 * um) break;
    }
    if (it > kmax) return -1;
    residual(c, u, f, NULL, E, &W, &wt);
    if (!(wt > 0) || !(W < 1e10)) return -1;
    *rho = c->D / W;
    *p = (wt / W - *rho) / c->Gh;
    return it;
}

/* ------------------------------------------------------------------ */
/* MC limited reconstruction (Sec. 5: "2nd order MC limiter")            */
/* ------------------------------------------------------------------ */

static double minmod3(double a, double b, double c)
{
    if (a > 0 && b > 0 && c > 0) return fmin(a, fmin(b, c));
    if (a < 0 && b < 0 && c < 0) return fmax(a, fmax(b, c));
    return 0.0;
}

static double mc_slope(double um, double u0, double up)
{
    return minmod3(2.0 * (u0 - um), 0.5 * (up - um), 2.0 * (up - u0));
}

/* index of the cell s steps from c along d; beyond the two stored ghost layers (the PPM
 * stencil reaches three) periodic wraps, outflow takes the boundary cell, fixed the
 * outermost stored ghost */
static long nb_cell(const OGrid* g, long c, int d, int s)
{
    int ijk[3];
    coords(g, c, ijk);
    int m = ijk[d] + s;
    if (m < 0 || m >= g->N[d]) {
        int lo = g->ng[d], hi = g->ng[d] + g->n[d] - 1;
        if (g->bc[d] == BC_PERIODIC) m = lo + (((m - lo) % g->n[d]) + g->n[d]) % g->n[d];
        else if (g->bc[d] == BC_OUTFLOW) m = m < lo ? lo : hi;
        else m = m < 0 ? 0 : g->N[d] - 1;
    }
    ijk[d] = m;
    return at(g, ijk[0], ijk[1], ijk[2]);
}

/* PPM (Colella & Woodward 1984, their interface interpolation and monotonicity
 * constraints, no steepening or flattening): the interface value between cells j and
 * j+1 from cells j-1..j+2, with the monotone slope delta_m a = the MC slope */
static double ppm_iface(double am, double a0, double ap, double app)
{
    return a0 + 0.5 * (ap - a0) - (mc_slope(a0, ap, app) - mc_slope(am, a0, ap)) / 6.0;
}

/* the parabola in cell a0 with edge values (*aL, *aR), limited to be monotone */
static void ppm_limit(double a0, double* aL, double* aR)
{
    if ((*aR - a0) * (a0 - *aL) <= 0.0) {
        *aL = a0;
        *aR = a0;
        return;
    }
    double dd = *aR - *aL, m6 = 6.0 * (a0 - 0.5 * (*aL + *aR));
    if (dd * m6 > dd * dd) *aL = 3.0 * a0 - 2.0 * *aR;
    else if (-dd * dd > dd * m6) *aR = 3.0 * a0 - 2.0 * *aL;
}

/* left and right states at the lower d-face of cell c of the array a (values of the
 * cells around, or of the faces of another direction, which are cells along d) */
static void face_lr(const OGrid* g, const double* a, long c, int d, double* L, double* R)
{
    if (g->rec == 1) {
        double v[6];
        for (int s = 0; s < 6; s++) v[s] = a[nb_cell(g, c, d, s - 3)];
        /* cells c-3..c+2 = v[0..5]; interfaces c-3/2, c-1/2, c+1/2 */
        double im = ppm_iface(v[0], v[1], v[2], v[3]);
        double i0 = ppm_iface(v[1], v[2], v[3], v[4]);
        double ip = ppm_iface(v[2], v[3], v[4], v[5]);
        double lL = im, lR = i0;       /* cell c-1 */
        ppm_limit(v[2], &lL, &lR);
        double rL = i0, rR = ip;       /* cell c */
        ppm_limit(v[3], &rL, &rR);
        *L = lR;
        *R = rL;
        return;
    }
    long m2 = shift(g, c, d, -2), m1 = shift(g, c, d, -1), p1 = shift(g, c, d, 1);
    *L = a[m1] + 0.5 * mc_slope(a[m2], a[m1], a[c]);
    *R = a[c] - 0.5 * mc_slope(a[m1], a[c], a[p1]);
}

/* ------------------------------------------------------------------ */
/* physical flux and conserved state at a face (Sec. 2.1)                */
/* ------------------------------------------------------------------ */

/* pr: rho, u^1..3, p, E^1..3 ; B^1..3 ; direction d; metric psi, alpha at the face.
 * q: densitised conserved D, S_j, tau, E^j ;  F: flux of the same, in direction d */
static void face_flux(const double* pr, const double* B, int d, double psi, double alp, double Gam, double* q, double* F)
{
    double g = psi * psi * psi * psi, sg = g * psi * psi, ginv = 1.0 / g;
    prim2con_point(pr, B, psi, Gam, q);
    double rho = pr[0], p = pr[4];
    double uu = 0, E2 = 0, B2 = 0;
    for (int i = 0; i < 3; i++) { uu += g * pr[1 + i] * pr[1 + i]; E2 += g * pr[5 + i] * pr[5 + i]; B2 += g * B[i] * B[i]; }
    double W = sqrt(1.0 + uu), h = 1.0 + Gam / (Gam - 1.0) * p / rho;
    double v[3], v_lo[3], E_lo[3], B_lo[3];
    for (int i = 0; i < 3; i++) { v[i] = pr[1 + i] / W; v_lo[i] = g * v[i]; E_lo[i] = g * pr[5 + i]; B_lo[i] = g * B[i]; }
    double D = q[0] / sg, tau = q[4] / sg, S_lo[3];
    for (int j = 0; j < 3; j++) S_lo[j] = q[1 + j] / sg;
    /* (f_D)^d = sqrt(gamma) D vhat^d, vhat^d = alpha v^d - beta^d */
    F[0] = sg * D * alp * v[d];
    /* (f_S_j)^d = sqrt(gamma) alpha S^d_j */
    for (int j = 0; j < 3; j++)
        F[1 + j] = sg * alp * ((p + 0.5 * (E2 + B2)) * (d == j ? 1.0 : 0.0) + rho * h * W * W * v[d] * v_lo[j]
                               - pr[5 + d] * E_lo[j] - B[d] * B_lo[j]);
    /* (f_tau)^d = sqrt(gamma) alpha (S^d - v^d D) */
    F[4] = sg * alp * (ginv * S_lo[d] - v[d] * D);
    /* (f_E^j)^d = sqrt(gamma) (1/sqrt(gamma)) eta^{djk} alpha B_k */
    for (int j = 0; j < 3; j++) {
        double s = 0;
        for (int k = 0; k < 3; k++) s += levi(d, j, k) * alp * B_lo[k];
        F[5 + j] = s;
    }
    (void)tau;
}

/* ------------------------------------------------------------------ */
/* the explicit operator L (cell-centred fluxes + sources, CT for faces)  */
/* ------------------------------------------------------------------ */

typedef struct {
    const OGrid* g;
    const double* alp;
    const double* psi;
} OCtx;

/* non-stiff sources of the 8 cell-centred variables at interior cell c (Sec. 2.1,
 * beta = 0, K_ij = 0), added to Lc: the Gauss-law charge term of s_E and, with a
 * metric, s_S and s_tau.  Bc: cell-centred contravariant B^i (ghosts filled). */
static void cell_sources(const OCtx* X, double* const* prim, double* const* Bc, long c, double* Lc)
{
    const OGrid* g = X->g;
    double ps = psi_at(X->psi, c), al = alp_at(X->alp, c);
    double gg = ps * ps * ps * ps, sg = gg * ps * ps;
    double uu = 0;
    for (int i = 0; i < 3; i++) uu += gg * prim[1 + i][c] * prim[1 + i][c];
    double W = sqrt(1.0 + uu);
    double v_up[3];
    for (int i = 0; i < 3; i++) v_up[i] = prim[1 + i][c] / W;
    /* Gauss law: sqrt(gamma) rho_e = div q_E (central difference) */
    double divqE = 0;
    for (int d = 0; d < 3; d++) {
        if (!g->act[d]) continue;
        long cp1 = shift(g, c, d, 1), cm1 = shift(g, c, d, -1);
        double qEp = pow(psi_at(X->psi, cp1), 6) * prim[5 + d][cp1];
        double qEm = pow(psi_at(X->psi, cm1), 6) * prim[5 + d][cm1];
        divqE += (qEp - qEm) / (2.0 * g->dx[d]);
    }
    double rhoe = divqE / sg;
    /* s_E non-stiff part: sqrt(gamma) (rho_e beta^i - alpha rho_e v^i), beta = 0 */
    for (int i = 0; i < 3; i++) Lc[5 + i] += -sg * al * rhoe * v_up[i];
    if (X->alp || X->psi) {
        /* s_S_i and s_tau with beta = 0, K_ij = 0 (Sec. 2.1):
         *   s_S_i = alpha sqrt(gamma) { -T^00 alpha d_i alpha + 1/2 T^jk d_i gamma_jk }
         *   s_tau = alpha sqrt(gamma) { -T^0j d_j alpha }
         * T^00 = (tau + D)/alpha^2, alpha T^0j = S^j, T^jk = stress (spatial) */
        double rho = prim[0][c], p = prim[4][c], h = 1.0 + g->Gam / (g->Gam - 1.0) * p / rho;
        double E2 = 0, B2 = 0;
        for (int i = 0; i < 3; i++) { E2 += gg * prim[5 + i][c] * prim[5 + i][c]; B2 += gg * Bc[i][c] * Bc[i][c]; }
        double pr8[NPR], q8[NQ], Bp[3];
        for (int v = 0; v < NPR; v++) pr8[v] = prim[v][c];
        for (int k = 0; k < 3; k++) Bp[k] = Bc[k][c];
        prim2con_point(pr8, Bp, ps, g->Gam, q8);
        double D = q8[0] / sg, tau = q8[4] / sg, S_lo[3];
        for (int j = 0; j < 3; j++) S_lo[j] = q8[1 + j] / sg;
        double T00 = (tau + D) / (al * al);
        double Tjk[3][3];
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                Tjk[j][k] = rho * h * W * W * v_up[j] * v_up[k] + p * (j == k ? 1.0 / gg : 0.0)
                            + 0.5 * (E2 + B2) * (j == k ? 1.0 / gg : 0.0)
                            - prim[5 + j][c] * prim[5 + k][c] - Bc[j][c] * Bc[k][c];
        for (int i = 0; i < 3; i++) {
            if (!g->act[i]) continue;
            long cp1 = shift(g, c, i, 1), cm1 = shift(g, c, i, -1);
            double dal = (alp_at(X->alp, cp1) - alp_at(X->alp, cm1)) / (2.0 * g->dx[i]);
            double dps = (psi_at(X->psi, cp1) - psi_at(X->psi, cm1)) / (2.0 * g->dx[i]);
            double dgam = 4.0 * ps * ps * ps * dps;     /* d_i gamma_jj (j = k) */
            double tr = 0;
            for (int j = 0; j < 3; j++) tr += Tjk[j][j] * dgam;
            Lc[1 + i] += al * sg * (-T00 * al * dal + 0.5 * tr);
            Lc[4] += al * sg * (-(S_lo[i] / gg) / al * dal);
        }
    }
}

/* prim: 8 padded arrays with ghosts filled; qBc: cell-centred q_B (3, filled);
 * bf: face q_B (3, ghosts filled); out L: 8 cell-centred + 3 face (interior) */
static void explicit_L(const OCtx* X, double* const* prim, double* const* qBc, double* const* bf, double** L)
{
    const OGrid* g = X->g;
    long nc = g->ncell;
    int ijk[3];
    /* cell-centred primitive B and covariant E_c for the EMF */
    double* Bc[3];
    double* Ecov[3];
    for (int d = 0; d < 3; d++) {
        Bc[d] = dalloc(nc); Ecov[d] = dalloc(nc);
        for (long c = 0; c < nc; c++) {
            double ps = psi_at(X->psi, c), gg = ps * ps * ps * ps;
            Bc[d][c] = qBc[d][c] / (gg * ps * ps);
            Ecov[d][c] = gg * prim[5 + d][c];
        }
    }
    /* face states and HLL fluxes, direction by direction; the flux for the 8
     * cell-centred variables lives at face index f (between cells f-1 and f) */
    double* F[3][NQ];
    /* App. A step (ii): HLL-weighted transverse transport velocities vbar^j at the
     * d-faces (ideal EMF only); in an inactive direction d the "face" is the cell and
     * vbar^j is the cell's vhat^j = alpha v^j (beta = 0) */
    double* vbar[3][3];
    for (int d = 0; d < 3; d++) for (int v = 0; v < NQ; v++) F[d][v] = NULL;
    for (int d = 0; d < 3; d++)
        for (int j = 0; j < 3; j++) {
            vbar[d][j] = NULL;
            if (g->emf != 1 || j == d) continue;
            vbar[d][j] = dalloc(nc);
            if (g->act[d]) continue;
            for (long c = 0; c < nc; c++) {
                double gg = pow(psi_at(X->psi, c), 4), uu = 0;
                for (int k = 0; k < 3; k++) uu += gg * prim[1 + k][c] * prim[1 + k][c];
                vbar[d][j][c] = alp_at(X->alp, c) * prim[1 + j][c] / sqrt(1.0 + uu);
            }
        }
    for (int d = 0; d < 3; d++) {
        if (!g->act[d]) continue;
        for (int v = 0; v < NQ; v++) F[d][v] = dalloc(nc);
        for (long c = 0; c < nc; c++) {
            coords(g, c, ijk);
            int f = ijk[d];
            if (f < 2 || f > g->N[d] - 2) continue;
            long cm2 = shift(g, c, d, -2), cm1 = shift(g, c, d, -1), cp1 = shift(g, c, d, 1);
            double recL[NREC], recR[NREC];
            (void)cm2; (void)cp1;
            for (int v = 0; v < NREC; v++) face_lr(g, v < NPR ? prim[v] : Bc[v - NPR], c, d, &recL[v], &recR[v]);
            double psf = 0.5 * (psi_at(X->psi, cm1) + psi_at(X->psi, c));
            double alf = 0.5 * (alp_at(X->alp, cm1) + alp_at(X->alp, c));
            double gf = psf * psf * psf * psf;
            double BL[3], BR[3];
            for (int k = 0; k < 3; k++) { BL[k] = recL[NPR + k]; BR[k] = recR[NPR + k]; }
            BL[d] = BR[d] = bf[d][c] / (gf * psf * psf);   /* normal B: the staggered face value */
            double qL[NQ], qR[NQ], FL[NQ], FR[NQ];
            face_flux(recL, BL, d, psf, alf, g->Gam, qL, FL);
            face_flux(recR, BR, d, psf, alf, g->Gam, qR, FR);
            /* Sec. 2.5: lambda_pm = alpha (pm sqrt(gamma^dd)) - beta^d, beta = 0 */
            double lp = alf * sqrt(1.0 / gf), lm = -alf * sqrt(1.0 / gf);
            double cp = fmax(0.0, lp), cm = fmax(0.0, -lm);
            for (int v = 0; v < NQ; v++)
                F[d][v][c] = (cp * FL[v] + cm * FR[v] - cp * cm * (qR[v] - qL[v])) / (cp + cm);
            if (g->emf == 1) {
                /* App. A steps (i)-(ii): vhat^j = alpha v^j of the L and R states,
                 * vbar^j = (c- vhat^j_R + c+ vhat^j_L)/(c- + c+) */
                double uuL = 0, uuR = 0;
                for (int k = 0; k < 3; k++) { uuL += gf * recL[1 + k] * recL[1 + k]; uuR += gf * recR[1 + k] * recR[1 + k]; }
                double WL = sqrt(1.0 + uuL), WR = sqrt(1.0 + uuR);
                for (int j = 0; j < 3; j++) {
                    if (j == d) continue;
                    double vL = alf * recL[1 + j] / WL, vR = alf * recR[1 + j] / WR;
                    vbar[d][j][c] = (cm * vR + cp * vL) / (cm + cp);
                }
            }
        }
    }
    /* transport velocities of faces outside the interior (in the transverse directions)
     * follow the grid's boundary rule, like every other quantity read there */
    if (g->emf == 1)
        for (int d = 0; d < 3; d++)
            for (int j = 0; j < 3; j++)
                if (g->act[d] && j != d) fill_face_ghosts(g, vbar[d][j], d);
    /* cell-centred L: flux divergence + non-stiff sources */
    for (long c = 0; c < nc; c++) {
        coords(g, c, ijk);
        if (!is_interior(g, ijk)) continue;
        double Lc[NQ];
        for (int v = 0; v < NQ; v++) Lc[v] = 0.0;
        for (int d = 0; d < 3; d++) {
            if (!g->act[d]) continue;
            long cp1 = shift(g, c, d, 1);
            for (int v = 0; v < NQ; v++) Lc[v] -= (F[d][v][cp1] - F[d][v][c]) / g->dx[d];
        }
        cell_sources(X, prim, Bc, c, Lc);
        for (int v = 0; v < NQ; v++) L[v][c] = Lc[v];
    }
    /* upwind constrained transport: edge EMF hat{E}_c for c = 0,1,2 with the pair
     * (a, b) = (c+1, c+2) mod 3; stored at the lower-a, lower-b corner index */
    double* Eh[3];
    for (int cc = 0; cc < 3; cc++) {
        Eh[cc] = dalloc(nc);
        int a = (cc + 1) % 3, b = (cc + 2) % 3;
        /* step (ii): E_c to a-faces, L/R (cell values where a is inactive) */
        double* EaL = dalloc(nc);
        double* EaR = dalloc(nc);
        for (long c = 0; c < nc; c++) {
            coords(g, c, ijk);
            if (!g->act[a]) { EaL[c] = EaR[c] = Ecov[cc][c]; continue; }
            int f = ijk[a];
            if (f < 2 || f > g->N[a] - 2) continue;
            face_lr(g, Ecov[cc], c, a, &EaL[c], &EaR[c]);
        }
        for (long c = 0; c < nc; c++) {
            coords(g, c, ijk);
            /* the edge must be reachable by both stencils */
            if (g->act[a] && (ijk[a] < 2 || ijk[a] > g->N[a] - 2)) continue;
            if (g->act[b] && (ijk[b] < 2 || ijk[b] > g->N[b] - 2)) continue;
            if (!g->act[a] && !g->act[b]) {
                Eh[cc][c] = alp_at(X->alp, c) * Ecov[cc][c];
                continue;
            }
            /* step (iii): along b to the edge: E_c^{XY}, X = a-side, Y = b-side */
            double EXY[2][2];
            const double* src[2] = {EaL, EaR};
            for (int X2 = 0; X2 < 2; X2++) {
                if (!g->act[b]) { EXY[X2][0] = EXY[X2][1] = src[X2][c]; continue; }
                face_lr(g, src[X2], c, b, &EXY[X2][0], &EXY[X2][1]);
            }
            /* step (iv): q_B^b (b-faces) along a -> L/R in a; q_B^a (a-faces) along b -> L/R in b */
            double qBbL, qBbR, qBaL, qBaR;
            if (g->act[a]) {
                face_lr(g, bf[b], c, a, &qBbL, &qBbR);
            } else {
                qBbL = qBbR = bf[b][c];
            }
            if (g->act[b]) {
                face_lr(g, bf[a], c, b, &qBaL, &qBaR);
            } else {
                qBaL = qBaR = bf[a][c];
            }
            /* lapse at the edge: mean of the cells around it; speeds of the faces */
            long cells[4];
            int nce = 0;
            long am = g->act[a] ? shift(g, c, a, -1) : c;
            cells[nce++] = c;
            if (g->act[a]) cells[nce++] = am;
            if (g->act[b]) {
                cells[nce++] = shift(g, c, b, -1);
                if (g->act[a]) cells[nce++] = shift(g, am, b, -1);
            }
            double ale = 0;
            for (int t = 0; t < nce; t++) ale += alp_at(X->alp, cells[t]);
            ale /= nce;
            double ca = 1.0, cb = 1.0;
            if (g->act[a]) {
                /* a-faces adjacent to the edge: at b-cells e-1 and e */
                ca = 0.0;
                for (int t = 0; t < (g->act[b] ? 2 : 1); t++) {
                    long cf = t == 0 ? c : shift(g, c, b, -1);
                    long cfm = shift(g, cf, a, -1);
                    double psf = 0.5 * (psi_at(X->psi, cfm) + psi_at(X->psi, cf));
                    double alf = 0.5 * (alp_at(X->alp, cfm) + alp_at(X->alp, cf));
                    double sp = alf / (psf * psf);
                    if (sp > ca) ca = sp;
                }
            }
            if (g->act[b]) {
                cb = 0.0;
                for (int t = 0; t < (g->act[a] ? 2 : 1); t++) {
                    long cf = t == 0 ? c : shift(g, c, a, -1);
                    long cfm = shift(g, cf, b, -1);
                    double psf = 0.5 * (psi_at(X->psi, cfm) + psi_at(X->psi, cf));
                    double alf = 0.5 * (alp_at(X->alp, cfm) + alp_at(X->alp, cf));
                    double sp = alf / (psf * psf);
                    if (sp > cb) cb = sp;
                }
            }
            double cap = ca, cam = ca, cbp = cb, cbm = cb;
            if (g->emf == 1) {
                /* App. A steps (iii)-(iv): vbar^a of the b-faces reconstructed along a,
                 * vbar^b of the a-faces along b (with q_B^b along a, q_B^a along b) */
                double vaL, vaR, vbL, vbR;
                const double* va = vbar[b][a];
                const double* vb = vbar[a][b];
                if (g->act[a]) {
                    face_lr(g, va, c, a, &vaL, &vaR);
                } else {
                    vaL = vaR = va[c];
                }
                if (g->act[b]) {
                    face_lr(g, vb, c, b, &vbL, &vbR);
                } else {
                    vbL = vbR = vb[c];
                }
                Eh[cc][c] = -(cam * vaR * qBbR + cap * vaL * qBbL - cam * cap * (qBbR - qBbL)) / (cam + cap)
                            + (cbm * vbR * qBaR + cbp * vbL * qBaL - cbm * cbp * (qBaR - qBaL)) / (cbm + cbp);
                continue;
            }
            /* step (v): hat{E}^{XY} = alpha E_c^{XY} (beta = 0) */
            double hLL = ale * EXY[0][0], hLR = ale * EXY[0][1], hRL = ale * EXY[1][0], hRR = ale * EXY[1][1];
            /* step (vii): Londrillo & Del Zanna (2004) */
            Eh[cc][c] = (cap * cbp * hLL + cap * cbm * hLR + cam * cbp * hRL + cam * cbm * hRR) / ((cap + cam) * (cbp + cbm))
                        + cap * cam / (cap + cam) * (qBbR - qBbL)
                        - cbp * cbm / (cbp + cbm) * (qBaR - qBaL);
        }
        free(EaL); free(EaR);
    }
    /* CT (Sec. 3.2): d(q_B^a)/dt on a-faces, Delta A = product of the two transverse
     * widths: -d_b hat{E}_c + d_c hat{E}_b with (a, b, c) cyclic */
    for (int fa = 0; fa < 3; fa++) {
        int fb = (fa + 1) % 3, fc = (fa + 2) % 3;
        for (long c = 0; c < nc; c++) {
            coords(g, c, ijk);
            int ok = 1;
            for (int d = 0; d < 3; d++) {
                int lo = g->ng[d], hi = g->ng[d] + g->n[d] - 1;
                if (d == fa && g->act[d] && g->bc[d] != BC_PERIODIC) hi += 1;
                if (ijk[d] < lo || ijk[d] > hi) ok = 0;
            }
            if (!ok) continue;
            double r = 0;
            /* hat{E}_c lives on edges along c, i.e. varies in a and b */
            if (g->act[fb]) r -= (Eh[fc][shift(g, c, fb, 1)] - Eh[fc][c]) / g->dx[fb];
            if (g->act[fc]) r += (Eh[fb][shift(g, c, fc, 1)] - Eh[fb][c]) / g->dx[fc];
            L[NQ + fa][c] = r;
        }
    }
    for (int d = 0; d < 3; d++) {
        free(Bc[d]); free(Ecov[d]); free(Eh[d]);
        for (int v = 0; v < NQ; v++) free(F[d][v]);
        for (int j = 0; j < 3; j++) free(vbar[d][j]);
    }
}

/* ------------------------------------------------------------------ */
/* exported API                                                         */
/* ------------------------------------------------------------------ */

/* gi: ndim, n0, n1, n2, bc0, bc1, bc2 ; gd: dx0, dx1, dx2, Gamma, rho_atm, p_atm, xi.
 * All arrays padded. */

/* staggered q_B from an edge vector potential (Sec. 4, q_B^i = eta^{ijk} d_j A_k with
 * sqrt(gamma_hat) = 1).  A[c] lives on edges along c (lower corner index). Faces whose
 * stencil leaves the array are left untouched. */
void orc_curl_A(const int* gi, const double* gd, double* const* A, double** bf)
{
    OGrid G; grid_setup(&G, gi, gd);
    int ijk[3];
    for (int fa = 0; fa < 3; fa++) {
        int fb = (fa + 1) % 3, fc = (fa + 2) % 3;
        for (long c = 0; c < G.ncell; c++) {
            coords(&G, c, ijk);
            if ((G.act[fb] && ijk[fb] + 1 >= G.N[fb]) || (G.act[fc] && ijk[fc] + 1 >= G.N[fc])) continue;
            double r = 0;
            if (G.act[fb]) r += (A[fc][shift(&G, c, fb, 1)] - A[fc][c]) / G.dx[fb];
            if (G.act[fc]) r -= (A[fb][shift(&G, c, fc, 1)] - A[fb][c]) / G.dx[fc];
            bf[fa][c] = r;
        }
    }
}

/* prim (8 padded) + face q_B (3 padded) -> densitised conserved q (8 padded, all cells) */
void orc_prim2con(const int* gi, const double* gd, double* const* prim, double* const* bf, const double* psi, double** q)
{
    OGrid G; grid_setup(&G, gi, gd);
    double* qBc[3];
    double* bfc[3];
    for (int d = 0; d < 3; d++) {
        qBc[d] = dalloc(G.ncell);
        bfc[d] = dalloc(G.ncell);
        memcpy(bfc[d], bf[d], sizeof(double) * G.ncell);
        fill_face_ghosts(&G, bfc[d], d);
    }
    cell_qB(&G, bfc, qBc);
    for (long c = 0; c < G.ncell; c++) {
        double pr[NPR], B[3], qq[NQ];
        double ps = psi_at(psi, c), sg = pow(ps, 6);
        for (int v = 0; v < NPR; v++) pr[v] = prim[v][c];
        for (int d = 0; d < 3; d++) B[d] = qBc[d][c] / sg;
        prim2con_point(pr, B, ps, G.Gam, qq);
        for (int v = 0; v < NQ; v++) q[v][c] = qq[v];
    }
    for (int d = 0; d < 3; d++) { free(qBc[d]); free(bfc[d]); }
}

/* single-cell implicit solve, exposed for the pins.  in: D, S_i, tau, E*^i, B^i
 * (undensitised), xi; psi, eta_tilde (< 0: E fixed), Gamma, initial guess (NULL: rest).
 * out: u^i, E^i, rho, p.  returns Newton iterations or -1 */
int orc_solve_cell(const double* in, double psi, double etat, double Gam, const double* guess, double* u, double* E,
                   double* rho_p)
{
    OCell c;
    c.D = in[0];
    for (int i = 0; i < 3; i++) { c.S[i] = in[1 + i]; c.Es[i] = in[5 + i]; c.B[i] = in[8 + i]; }
    c.tau = in[4];
    c.g = pow(psi, 4); c.sg = pow(psi, 6);
    c.etat = etat; c.Gh = Gam / (Gam - 1.0);
    c.xi = in[11];
    for (int i = 0; i < 3; i++) u[i] = guess ? guess[i] : 0.0;
    return newton_cell(&c, u, E, &rho_p[0], &rho_p[1], 100, 1e-14);
}

/* residual + analytic Jacobian at a given u (for the finite-difference pin) */
void orc_residual_cell(const double* in, double psi, double etat, double Gam, const double* u, double* f, double* J9, double* E)
{
    OCell c;
    c.D = in[0];
    for (int i = 0; i < 3; i++) { c.S[i] = in[1 + i]; c.Es[i] = in[5 + i]; c.B[i] = in[8 + i]; }
    c.tau = in[4];
    c.g = pow(psi, 4); c.sg = pow(psi, 6);
    c.etat = etat; c.Gh = Gam / (Gam - 1.0);
    c.xi = in[11];
    double J[3][3];
    residual(&c, u, f, J, E, NULL, NULL);
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) J9[3 * i + j] = J[i][j];
}

/* implicit stage solve over interior cells (Sec. 2.4): base q (8 padded) and face
 * q_B (3) in; q_E of the base replaced by the solution; prims out (8, interior);
 * R = (q_E - q_E,base)/(a_ii dt) (3, interior).  eta: per-cell or NULL -> eta_u.
 * a_dt = a_ii * dt; a_dt <= 0 means E held fixed (plain con2prim).
 * stats[0] += failures, stats[1] = max iterations.  Returns failures. */
static int implicit_cells(const OGrid* Gp, double a_dt, double** q, double* const* qBc,
                          const double* alp, const double* psi, const double* eta, double eta_u,
                          double** prim, double** R, int* stats)
{
    const OGrid G = *Gp;
    int fails = 0, maxit = 0, ijk[3];
    for (long c = 0; c < G.ncell; c++) {
        coords(&G, c, ijk);
        if (!is_interior(&G, ijk)) continue;
        double ps = psi_at(psi, c), sg = pow(ps, 6);
        OCell cl;
        cl.g = pow(ps, 4); cl.sg = sg; cl.Gh = G.Gam / (G.Gam - 1.0);
        cl.xi = G.xi;
        cl.D = q[0][c] / sg; cl.tau = q[4][c] / sg;
        for (int i = 0; i < 3; i++) { cl.S[i] = q[1 + i][c] / sg; cl.Es[i] = q[5 + i][c] / sg; cl.B[i] = qBc[i][c] / sg; }
        double et = eta ? eta[c] : eta_u;
        cl.etat = a_dt > 0 ? et / (alp_at(alp, c) * a_dt) : -1.0;
        /* initial guess: the velocity of the previous stage held in prim (the paper
         * does not fix one); from rest if that is not finite or does not converge */
        double u[3], E[3], rho, p;
        int it = 0, atmo = 0;
        if (G.rho_atm > 0 && cl.D < 10.0 * G.rho_atm) {
            atmo = 1;
        } else {
            int fin = 1;
            for (int i = 0; i < 3; i++) { u[i] = prim[1 + i][c]; if (!(fabs(u[i]) < 1e30)) fin = 0; }
            if (!fin) for (int i = 0; i < 3; i++) u[i] = 0.0;
            it = newton_cell(&cl, u, E, &rho, &p, 100, 1e-14);
            if (it < 0 && fin) {
                for (int i = 0; i < 3; i++) u[i] = 0.0;
                it = newton_cell(&cl, u, E, &rho, &p, 100, 1e-14);
            }
            if (it < 0) {
                fails++;
                if (!(G.rho_atm > 0)) continue;
                atmo = 1;
            }
        }
        if (atmo) {
            /* atmosphere: rest state at the floor density and pressure, E kept (no stiff
             * update) */
            rho = G.rho_atm;
            p = G.p_atm;
            for (int i = 0; i < 3; i++) { u[i] = 0.0; E[i] = cl.Es[i]; }
            it = 0;
        }
        if (it > maxit) maxit = it;
        prim[0][c] = rho;
        for (int i = 0; i < 3; i++) prim[1 + i][c] = u[i];
        prim[4][c] = p;
        for (int i = 0; i < 3; i++) prim[5 + i][c] = E[i];
        for (int i = 0; i < 3; i++) {
            double qEn = sg * E[i];
            if (R) R[i][c] = a_dt > 0 ? (qEn - q[5 + i][c]) / a_dt : 0.0;
            q[5 + i][c] = qEn;
        }
    }
    if (stats) { stats[0] += fails; if (maxit > stats[1]) stats[1] = maxit; }
    return fails;
}

int orc_implicit(const int* gi, const double* gd, double a_dt, double** q, double* const* bf,
                 const double* alp, const double* psi, const double* eta, double eta_u,
                 double** prim, double** R, int* stats)
{
    OGrid G; grid_setup(&G, gi, gd);
    double* qBc[3];
    double* bfc[3];
    for (int d = 0; d < 3; d++) {
        qBc[d] = dalloc(G.ncell);
        bfc[d] = dalloc(G.ncell);
        memcpy(bfc[d], bf[d], sizeof(double) * G.ncell);
        fill_face_ghosts(&G, bfc[d], d);
    }
    cell_qB(&G, bfc, qBc);
    int fails = implicit_cells(&G, a_dt, q, qBc, alp, psi, eta, eta_u, prim, R, stats);
    for (int d = 0; d < 3; d++) { free(qBc[d]); free(bfc[d]); }
    return fails;
}

/* explicit operator L for given stage prims (8 padded; interior set, ghosts: fixed-BC
 * values) and face q_B (3 padded).  L out: 8 cell-centred + 3 face arrays. */
void orc_explicit_L(const int* gi, const double* gd, double* const* prim_in, double* const* bf_in,
                    const double* alp, const double* psi, double** L)
{
    OGrid G; grid_setup(&G, gi, gd);
    OCtx X = {&G, alp, psi};
    double* prim[NPR];
    double* bf[3];
    double* qBc[3];
    for (int v = 0; v < NPR; v++) {
        prim[v] = dalloc(G.ncell);
        memcpy(prim[v], prim_in[v], sizeof(double) * G.ncell);
        fill_cell_ghosts(&G, prim[v]);
    }
    for (int d = 0; d < 3; d++) {
        bf[d] = dalloc(G.ncell);
        qBc[d] = dalloc(G.ncell);
        memcpy(bf[d], bf_in[d], sizeof(double) * G.ncell);
        fill_face_ghosts(&G, bf[d], d);
    }
    cell_qB(&G, bf, qBc);
    explicit_L(&X, prim, qBc, bf, L);
    for (int v = 0; v < NPR; v++) free(prim[v]);
    for (int d = 0; d < 3; d++) { free(bf[d]); free(qBc[d]); }
}

/* one IMEX step with a DIRK-type tableau (a_ii > 0 for every stage).
 * At, A: s*s row-major; wt, w: s.  q (8) and bf (3) updated in place (interior).
 * prim (8 padded): in = fixed-BC ghost values, out = last stage primitives.
 * stats: [0] failures, [1] max Newton iterations. Returns 0 or -1 (bad tableau). */
int orc_step(const int* gi, const double* gd, int s, const double* At, const double* A,
             const double* wt, const double* w, double dt, double** q, double** bf,
             const double* alp, const double* psi, const double* eta, double eta_u,
             double** prim, int* stats)
{
    OGrid G; grid_setup(&G, gi, gd);
    if (s < 1 || s > MAXS) return -1;
    for (int i = 0; i < s; i++) if (!(A[i * s + i] > 0)) return -1;
    long nc = G.ncell;
    double* Ls[MAXS][NQ + 3];
    double* Rs[MAXS][3];
    double* qs[NQ];
    double* bs[3];
    for (int i = 0; i < s; i++) {
        for (int v = 0; v < NQ + 3; v++) Ls[i][v] = dalloc(nc);
        for (int v = 0; v < 3; v++) Rs[i][v] = dalloc(nc);
    }
    for (int v = 0; v < NQ; v++) qs[v] = dalloc(nc);
    for (int d = 0; d < 3; d++) bs[d] = dalloc(nc);
    int ijk[3];
    for (int i = 0; i < s; i++) {
        /* stage base: q^n + dt sum_{j<i} (at_ij L(j) + a_ij R(j)) -- ghosts keep q^n */
        for (int v = 0; v < NQ; v++) memcpy(qs[v], q[v], sizeof(double) * nc);
        for (int d = 0; d < 3; d++) memcpy(bs[d], bf[d], sizeof(double) * nc);
        for (int j = 0; j < i; j++) {
            double at_ = At[i * s + j], a_ = A[i * s + j];
            for (long c = 0; c < nc; c++) {
                coords(&G, c, ijk);
                for (int v = 0; v < NQ; v++) {
                    if (!is_interior(&G, ijk)) continue;
                    qs[v][c] += dt * at_ * Ls[j][v][c];
                    if (v >= 5) qs[v][c] += dt * a_ * Rs[j][v - 5][c];
                }
                for (int d = 0; d < 3; d++) bs[d][c] += dt * at_ * Ls[j][NQ + d][c];
            }
        }
        orc_implicit(gi, gd, A[i * s + i] * dt, qs, bs, alp, psi, eta, eta_u, prim, Rs[i], stats);
        orc_explicit_L(gi, gd, prim, bs, alp, psi, Ls[i]);
    }
    for (long c = 0; c < nc; c++) {
        coords(&G, c, ijk);
        int inter = is_interior(&G, ijk);
        for (int i = 0; i < s; i++) {
            if (inter) {
                for (int v = 0; v < NQ; v++) {
                    q[v][c] += dt * wt[i] * Ls[i][v][c];
                    if (v >= 5) q[v][c] += dt * w[i] * Rs[i][v - 5][c];
                }
            }
            for (int d = 0; d < 3; d++) bf[d][c] += dt * wt[i] * Ls[i][NQ + d][c];
        }
    }
    for (int i = 0; i < s; i++) {
        for (int v = 0; v < NQ + 3; v++) free(Ls[i][v]);
        for (int v = 0; v < 3; v++) free(Rs[i][v]);
    }
    for (int v = 0; v < NQ; v++) free(qs[v]);
    for (int d = 0; d < 3; d++) free(bs[d]);
    return 0;
}

/* Delta t = CFL / max_cells sum_d (alpha sqrt(gamma^dd) + |beta^d|)/dx_d  (Sec. 2.5) */
double orc_dt(const int* gi, const double* gd, const double* alp, const double* psi, double cfl)
{
    OGrid G; grid_setup(&G, gi, gd);
    int ijk[3];
    double mx = 0;
    for (long c = 0; c < G.ncell; c++) {
        coords(&G, c, ijk);
        if (!is_interior(&G, ijk)) continue;
        double ps = psi_at(psi, c), s = 0;
        for (int d = 0; d < 3; d++)
            if (G.act[d]) s += alp_at(alp, c) * sqrt(1.0 / pow(ps, 4)) / G.dx[d];
        if (s > mx) mx = s;
    }
    return cfl / mx;
}

/* discrete div q_B per interior cell (Sec. 3.2 / Eq. divb_0 with sqrt(gamma_hat) = 1):
 * out[0] = mean |div|, out[1] = sqrt(mean div^2), out[2] = max |div| */
void orc_divb(const int* gi, const double* gd, double* const* bf_in, double* out)
{
    OGrid G; grid_setup(&G, gi, gd);
    double* bf[3];
    for (int d = 0; d < 3; d++) {
        bf[d] = dalloc(G.ncell);
        memcpy(bf[d], bf_in[d], sizeof(double) * G.ncell);
        fill_face_ghosts(&G, bf[d], d);
    }
    int ijk[3];
    double s1 = 0, s2 = 0, mx = 0;
    long n = 0;
    for (long c = 0; c < G.ncell; c++) {
        coords(&G, c, ijk);
        if (!is_interior(&G, ijk)) continue;
        double dv = 0;
        for (int d = 0; d < 3; d++)
            if (G.act[d]) dv += (bf[d][shift(&G, c, d, 1)] - bf[d][c]) / G.dx[d];
        s1 += fabs(dv); s2 += dv * dv; if (fabs(dv) > mx) mx = fabs(dv);
        n++;
    }
    out[0] = s1 / n; out[1] = sqrt(s2 / n); out[2] = mx;
    for (int d = 0; d < 3; d++) free(bf[d]);
}

/* volume totals of the 8 cell-centred conserved variables over the interior */
void orc_totals(const int* gi, const double* gd, double* const* q, double* out)
{
    OGrid G; grid_setup(&G, gi, gd);
    int ijk[3];
    double dV = 1;
    for (int d = 0; d < 3; d++) if (G.act[d]) dV *= G.dx[d];
    for (int v = 0; v < NQ; v++) out[v] = 0;
    for (long c = 0; c < G.ncell; c++) {
        coords(&G, c, ijk);
        if (!is_interior(&G, ijk)) continue;
        for (int v = 0; v < NQ; v++) out[v] += q[v][c] * dV;
    }
}

/* ------------------------------------------------------------------ */
/* GLM hyperbolic divergence cleaning with cell-centred B (Sec. 3.1)     */
/* ------------------------------------------------------------------ */
/*
 * The variant evolves 12 cell-centred variables: the 8 above, q_B^1..3 at cell
 * centres, and q_Phi = sqrt(gamma) Phi.  All 12 are reconstructed (as primitives:
 * rho, u, p, E, B = q_B/sqrt(gamma), Phi = q_Phi/sqrt(gamma)) and advanced by HLL
 * fluxes in the conservative form of Sec. 2.1, with beta = 0:
 *     (f_B^j)^i = -(1/sqrt(gamma)) sqrt(gamma) eta^{ijk} alpha E_k = eta^{jik} alpha E_k
 *     (f_Phi)^i = alpha q_B^i
 * and the sources of Sec. 3.1 with K_ij = 0:
 *     s_B^i  = -sqrt(gamma) alpha gamma^{ij} d_j Phi
 *     s_Phi  =  sqrt(gamma) [ -alpha kappa_B Phi + B^i d_i alpha ]
 * Readings: the flux and source of Phi are taken from their reference-metric
 * definitions (Sec. 3.1) in the conservative form d_t q + d_i f^i = s of Sec. 2.1
 * (the projected Phi equation printed before them has the opposite sign on the
 * divergence, which would make the (B, Phi) system anti-diffusive); d_j Phi and
 * d_i alpha are central differences of the cell values; the charge field Psi is
 * not evolved (charge conservation is not handled by default, Sec. 5), so rho_e
 * still comes from Gauss's law.  The kappa_B damping belongs to the explicit part.
 */
#define NGLM 12   /* 8 + q_B^1..3 + q_Phi */

/* face state and flux of the 12 GLM variables; pr: 8 primitives, B: B^1..3, Phi */
static void face_flux_glm(const double* pr, const double* B, double Phi, int d, double psi, double alp, double Gam,
                          double* q, double* F)
{
    double g = psi * psi * psi * psi, sg = g * psi * psi;
    face_flux(pr, B, d, psi, alp, Gam, q, F);
    for (int j = 0; j < 3; j++) {
        q[NQ + j] = sg * B[j];
        double s = 0;
        for (int k = 0; k < 3; k++) s += levi(j, d, k) * alp * g * pr[5 + k];   /* eta^{jdk} alpha E_k */
        F[NQ + j] = s;
    }
    q[NQ + 3] = sg * Phi;
    F[NQ + 3] = alp * sg * B[d];
}

/* prim (8), qB (3) and qPhi with ghosts filled; L out: 12 cell-centred arrays (interior) */
static void explicit_L_glm(const OCtx* X, double kappa, double* const* prim, double* const* qB, const double* qPhi,
                           double** L)
{
    const OGrid* g = X->g;
    long nc = g->ncell;
    int ijk[3];
    double* rec[NGLM];           /* reconstructed: 8 primitives, B^1..3, Phi */
    double* Bc[3];
    for (int v = 0; v < NPR; v++) rec[v] = prim[v];
    for (int v = NPR; v < NGLM; v++) rec[v] = dalloc(nc);
    for (long c = 0; c < nc; c++) {
        double sg = pow(psi_at(X->psi, c), 6);
        for (int d = 0; d < 3; d++) rec[NPR + d][c] = qB[d][c] / sg;
        rec[NPR + 3][c] = qPhi[c] / sg;
    }
    for (int d = 0; d < 3; d++) Bc[d] = rec[NPR + d];
    double* F[3][NGLM];
    for (int d = 0; d < 3; d++) for (int v = 0; v < NGLM; v++) F[d][v] = NULL;
    for (int d = 0; d < 3; d++) {
        if (!g->act[d]) continue;
        for (int v = 0; v < NGLM; v++) F[d][v] = dalloc(nc);
        for (long c = 0; c < nc; c++) {
            coords(g, c, ijk);
            int f = ijk[d];
            if (f < 2 || f > g->N[d] - 2) continue;
            long cm1 = shift(g, c, d, -1);
            double rL[NGLM], rR[NGLM];
            for (int v = 0; v < NGLM; v++) face_lr(g, rec[v], c, d, &rL[v], &rR[v]);
            double psf = 0.5 * (psi_at(X->psi, cm1) + psi_at(X->psi, c));
            double alf = 0.5 * (alp_at(X->alp, cm1) + alp_at(X->alp, c));
            double gf = psf * psf * psf * psf;
            double qL[NGLM], qR[NGLM], FL[NGLM], FR[NGLM];
            face_flux_glm(rL, rL + NPR, rL[NPR + 3], d, psf, alf, g->Gam, qL, FL);
            face_flux_glm(rR, rR + NPR, rR[NPR + 3], d, psf, alf, g->Gam, qR, FR);
            double lp = alf * sqrt(1.0 / gf), lm = -alf * sqrt(1.0 / gf);
            double cp = fmax(0.0, lp), cm = fmax(0.0, -lm);
            for (int v = 0; v < NGLM; v++)
                F[d][v][c] = (cp * FL[v] + cm * FR[v] - cp * cm * (qR[v] - qL[v])) / (cp + cm);
        }
    }
    for (long c = 0; c < nc; c++) {
        coords(g, c, ijk);
        if (!is_interior(g, ijk)) continue;
        double Lc[NGLM];
        for (int v = 0; v < NGLM; v++) Lc[v] = 0.0;
        for (int d = 0; d < 3; d++) {
            if (!g->act[d]) continue;
            long cp1 = shift(g, c, d, 1);
            for (int v = 0; v < NGLM; v++) Lc[v] -= (F[d][v][cp1] - F[d][v][c]) / g->dx[d];
        }
        cell_sources(X, prim, Bc, c, Lc);
        double ps = psi_at(X->psi, c), al = alp_at(X->alp, c);
        double gg = ps * ps * ps * ps, sg = gg * ps * ps;
        /* s_B^i = -sqrt(gamma) alpha gamma^{ij} d_j Phi ; s_Phi = -alpha kappa q_Phi + q_B^i d_i alpha */
        Lc[NQ + 3] += -al * kappa * qPhi[c];
        for (int i = 0; i < 3; i++) {
            if (!g->act[i]) continue;
            long cp1 = shift(g, c, i, 1), cm1 = shift(g, c, i, -1);
            double dPhi = (rec[NPR + 3][cp1] - rec[NPR + 3][cm1]) / (2.0 * g->dx[i]);
            double dal = (alp_at(X->alp, cp1) - alp_at(X->alp, cm1)) / (2.0 * g->dx[i]);
            Lc[NQ + i] += -sg * al * (1.0 / gg) * dPhi;
            Lc[NQ + 3] += qB[i][c] * dal;
        }
        for (int v = 0; v < NGLM; v++) L[v][c] = Lc[v];
    }
    for (int v = NPR; v < NGLM; v++) free(rec[v]);
    for (int d = 0; d < 3; d++)
        for (int v = 0; v < NGLM; v++) free(F[d][v]);
}

/* cell-centred q_B^i = eta^{ijk} d_j A_k from a cell-centred potential by central
 * differences (Sec. 4, the cell-centred case), on interior cells; the potential is
 * used as given on the whole padded grid (as for the edge potential); ghosts of q_B
 * untouched */
void orc_curl_A_cc(const int* gi, const double* gd, double* const* A, double** qB)
{
    OGrid G; grid_setup(&G, gi, gd);
    int ijk[3];
    for (long c = 0; c < G.ncell; c++) {
        coords(&G, c, ijk);
        if (!is_interior(&G, ijk)) continue;
        for (int i = 0; i < 3; i++) {
            double r = 0;
            for (int j = 0; j < 3; j++) {
                if (!G.act[j]) continue;
                for (int k = 0; k < 3; k++) {
                    double e = levi(i, j, k);
                    if (e == 0.0) continue;
                    r += e * (A[k][shift(&G, c, j, 1)] - A[k][shift(&G, c, j, -1)]) / (2.0 * G.dx[j]);
                }
            }
            qB[i][c] = r;
        }
    }
}

/* prim (8) + cell-centred q_B (3) -> q (8), all cells (q_B ghosts filled first) */
void orc_prim2con_cc(const int* gi, const double* gd, double* const* prim, double* const* qB_in, const double* psi,
                     double** q)
{
    OGrid G; grid_setup(&G, gi, gd);
    double* qB[3];
    for (int d = 0; d < 3; d++) {
        qB[d] = dalloc(G.ncell);
        memcpy(qB[d], qB_in[d], sizeof(double) * G.ncell);
        fill_cell_ghosts(&G, qB[d]);
    }
    for (long c = 0; c < G.ncell; c++) {
        double pr[NPR], B[3], qq[NQ];
        double ps = psi_at(psi, c), sg = pow(ps, 6);
        for (int v = 0; v < NPR; v++) pr[v] = prim[v][c];
        for (int d = 0; d < 3; d++) B[d] = qB[d][c] / sg;
        prim2con_point(pr, B, ps, G.Gam, qq);
        for (int v = 0; v < NQ; v++) q[v][c] = qq[v];
    }
    for (int d = 0; d < 3; d++) free(qB[d]);
}

/* the implicit solve with the cell-centred q_B given directly (interior read) */
int orc_implicit_cc(const int* gi, const double* gd, double a_dt, double** q, double* const* qB,
                    const double* alp, const double* psi, const double* eta, double eta_u,
                    double** prim, double** R, int* stats)
{
    OGrid G; grid_setup(&G, gi, gd);
    return implicit_cells(&G, a_dt, q, qB, alp, psi, eta, eta_u, prim, R, stats);
}

/* GLM explicit operator: prim (8), qB (3), qPhi; L out: 12 arrays */
void orc_explicit_L_glm(const int* gi, const double* gd, double kappa, double* const* prim_in, double* const* qB_in,
                        const double* qPhi_in, const double* alp, const double* psi, double** L)
{
    OGrid G; grid_setup(&G, gi, gd);
    OCtx X = {&G, alp, psi};
    double* prim[NPR];
    double* qB[3];
    double* qPhi = dalloc(G.ncell);
    for (int v = 0; v < NPR; v++) {
        prim[v] = dalloc(G.ncell);
        memcpy(prim[v], prim_in[v], sizeof(double) * G.ncell);
        fill_cell_ghosts(&G, prim[v]);
    }
    for (int d = 0; d < 3; d++) {
        qB[d] = dalloc(G.ncell);
        memcpy(qB[d], qB_in[d], sizeof(double) * G.ncell);
        fill_cell_ghosts(&G, qB[d]);
    }
    memcpy(qPhi, qPhi_in, sizeof(double) * G.ncell);
    fill_cell_ghosts(&G, qPhi);
    explicit_L_glm(&X, kappa, prim, qB, qPhi, L);
    for (int v = 0; v < NPR; v++) free(prim[v]);
    for (int d = 0; d < 3; d++) free(qB[d]);
    free(qPhi);
}

/* one IMEX step of the GLM variant: q (8), qB (3 cell-centred), qPhi updated in place
 * (interior); otherwise as orc_step */
int orc_step_glm(const int* gi, const double* gd, int s, const double* At, const double* A,
                 const double* wt, const double* w, double dt, double kappa, double** q, double** qB, double* qPhi,
                 const double* alp, const double* psi, const double* eta, double eta_u,
                 double** prim, int* stats)
{
    OGrid G; grid_setup(&G, gi, gd);
    if (s < 1 || s > MAXS) return -1;
    for (int i = 0; i < s; i++) if (!(A[i * s + i] > 0)) return -1;
    long nc = G.ncell;
    double* Ls[MAXS][NGLM];
    double* Rs[MAXS][3];
    double* qs[NGLM];
    double* qn[NGLM];
    for (int v = 0; v < NQ; v++) qn[v] = q[v];
    for (int d = 0; d < 3; d++) qn[NQ + d] = qB[d];
    qn[NQ + 3] = qPhi;
    for (int i = 0; i < s; i++) {
        for (int v = 0; v < NGLM; v++) Ls[i][v] = dalloc(nc);
        for (int v = 0; v < 3; v++) Rs[i][v] = dalloc(nc);
    }
    for (int v = 0; v < NGLM; v++) qs[v] = dalloc(nc);
    int ijk[3];
    for (int i = 0; i < s; i++) {
        for (int v = 0; v < NGLM; v++) memcpy(qs[v], qn[v], sizeof(double) * nc);
        for (int j = 0; j < i; j++) {
            double at_ = At[i * s + j], a_ = A[i * s + j];
            for (long c = 0; c < nc; c++) {
                coords(&G, c, ijk);
                if (!is_interior(&G, ijk)) continue;
                for (int v = 0; v < NGLM; v++) {
                    qs[v][c] += dt * at_ * Ls[j][v][c];
                    if (v >= 5 && v < NQ) qs[v][c] += dt * a_ * Rs[j][v - 5][c];
                }
            }
        }
        orc_implicit_cc(gi, gd, A[i * s + i] * dt, qs, qs + NQ, alp, psi, eta, eta_u, prim, Rs[i], stats);
        orc_explicit_L_glm(gi, gd, kappa, prim, qs + NQ, qs[NQ + 3], alp, psi, Ls[i]);
    }
    for (long c = 0; c < nc; c++) {
        coords(&G, c, ijk);
        if (!is_interior(&G, ijk)) continue;
        for (int i = 0; i < s; i++)
            for (int v = 0; v < NGLM; v++) {
                qn[v][c] += dt * wt[i] * Ls[i][v][c];
                if (v >= 5 && v < NQ) qn[v][c] += dt * w[i] * Rs[i][v - 5][c];
            }
    }
    for (int i = 0; i < s; i++) {
        for (int v = 0; v < NGLM; v++) free(Ls[i][v]);
        for (int v = 0; v < 3; v++) free(Rs[i][v]);
    }
    for (int v = 0; v < NGLM; v++) free(qs[v]);
    return 0;
}

/* div q_B of cell-centred fields by central differences over interior cells
 * (Eq. divb_0 with sqrt(gamma_hat) = 1): mean |div|, rms, max */
void orc_divb_cc(const int* gi, const double* gd, double* const* qB_in, double* out)
{
    OGrid G; grid_setup(&G, gi, gd);
    double* qB[3];
    for (int d = 0; d < 3; d++) {
        qB[d] = dalloc(G.ncell);
        memcpy(qB[d], qB_in[d], sizeof(double) * G.ncell);
        fill_cell_ghosts(&G, qB[d]);
    }
    int ijk[3];
    double s1 = 0, s2 = 0, mx = 0;
    long n = 0;
    for (long c = 0; c < G.ncell; c++) {
        coords(&G, c, ijk);
        if (!is_interior(&G, ijk)) continue;
        double dv = 0;
        for (int d = 0; d < 3; d++)
            if (G.act[d]) dv += (qB[d][shift(&G, c, d, 1)] - qB[d][shift(&G, c, d, -1)]) / (2.0 * G.dx[d]);
        s1 += fabs(dv); s2 += dv * dv; if (fabs(dv) > mx) mx = fabs(dv);
        n++;
    }
    out[0] = s1 / n; out[1] = sqrt(s2 / n); out[2] = mx;
    for (int d = 0; d < 3; d++) free(qB[d]);
}

/* face states of one array along d at every face whose stencil fits (TEST export of
 * face_lr): L, R padded arrays, the lower d-face of each cell */
void orc_face_states(const int* gi, const double* gd, const double* a, int d, double* L, double* R)
{
    OGrid G; grid_setup(&G, gi, gd);
    int ijk[3];
    for (long c = 0; c < G.ncell; c++) {
        coords(&G, c, ijk);
        if (ijk[d] < 2 || ijk[d] > G.N[d] - 2) continue;
        face_lr(&G, a, c, d, &L[c], &R[c]);
    }
}
