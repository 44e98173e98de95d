// C-ABI of the GB300 resistive-MHD IMEX stage: context, scratch carving, launch
// sequencing.  See include/grmhd.h for the contract of every call.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/grmhd.h"
#include "capi_internal.h"
#include "elliptic.h"
#include "kernels.h"
#include "launch.cuh"

using namespace grmhd;

namespace {

thread_local char g_err[512] = "";

grmhd_status fail(grmhd_status s, const char* fmt, const char* a = "")
{
    snprintf(g_err, sizeof g_err, fmt, a);
    return s;
}

grmhd_status cuda_fail(cudaError_t e, const char* where)
{
    snprintf(g_err, sizeof g_err, "%s: %s", where, cudaGetErrorString(e));
    return GRMHD_ERR_CUDA;
}

constexpr int kRedBlocks = 1024;   // partial rows of the reductions
constexpr size_t kAlign = 256;

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

namespace grmhd {
// lets other translation units of the library report through grmhd_last_error
void set_last_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace grmhd

struct grmhd_ctx_s {
    Dims g;
    grmhd_grid grid;
    grmhd_params par;
    grmhd_tableau tab;
    double dV;
    int nsm;
    bool bound, any_fixed;
    double* q[8];
    double* bf[3];
    double* prim[8];
    double* R[3];
    double* base[4][12];   // later stages' bases: 8 cell-centred + 3 B (+ q_Phi for GLM)
    double* acc[12];
    double* F[3][12];      // FP64 face fluxes (8; 12 for GLM)
    double* Eh[3];
    float* p32[11];      // mixed precision: FP32 stage primitives + cell-centred q_B
    double* vblk[3][2];  // per active direction, two FP64 arrays (the ideal-limit EMF's
                         // transport velocities)
    float* hs[4][3];     // per stage: its last Newton root u (orthonormal, FP32) ...
    float* hd[4][3];     // ... and that root minus the one before (the start guess is
                         // their sum: a linear extrapolation over steps)
    bool hist;           // hs / hd hold valid history (set by grmhd_init_from_prims)
    bool mixed;
    double* red_part;
    double* red_out;
    unsigned long long* nfail;
    const double* psi;
    const double* alp;
    const double* eta;
    double eta_u;
    double xi;           // mean-field dynamo parameter (0: none)
    bool glm;            // GLM cleaning with cell-centred B (Sec. 3.1) instead of CT
    bool ideal;          // ideal-limit edge EMF (App. A)
    bool ppm;            // PPM reconstruction instead of MC
    double* vbar[3][2];  // its transport velocities at the d-faces (vblk, or NULL)
    double kappa;        // GLM damping kappa_B
    double* qphi;        // GLM: bound q_Phi
    long long launches;
    // programmatic dependent launch of the stage kernels (launch.cuh)
    bool overlap;
    // optional per-kernel timing: events around each launch, folded on request
    bool timing;
    bool ev_made;
    int npend;
    cudaEvent_t ev[64][2];
    int ev_kind[64];
    double t_ms[4];
    long long t_n[4];
};

namespace {

grmhd_status check_grid(const grmhd_grid* g)
{
    if (!g) return fail(GRMHD_ERR_ARG, "grid is NULL");
    if (g->ndim < 1 || g->ndim > 3) return fail(GRMHD_ERR_ARG, "ndim must be 1, 2 or 3");
    for (int d = 0; d < g->ndim; d++) {
        if (g->n[d] < 1) return fail(GRMHD_ERR_ARG, "n[d] must be >= 1 in every active direction");
        if (!std::isfinite(g->lo[d]) || !std::isfinite(g->hi[d]) || !(g->hi[d] > g->lo[d]) ||
            !std::isfinite(g->n[d] / (g->hi[d] - g->lo[d])))
            return fail(GRMHD_ERR_ARG, "lo and hi must be finite with hi > lo (and n/(hi - lo) finite) in every "
                                       "active direction");
        if (g->bc[d] < 0 || g->bc[d] > 2) return fail(GRMHD_ERR_ARG, "bc must be PERIODIC, OUTFLOW or FIXED");
        if (g->bc[d] == GRMHD_BC_PERIODIC && g->n[d] < 2)
            return fail(GRMHD_ERR_ARG, "a periodic direction needs at least 2 cells");
    }
    long long cells = 1;
    for (int d = 0; d < g->ndim; d++) cells *= g->n[d];
    if (cells >= (1ll << 32)) return fail(GRMHD_ERR_ARG, "grids of 2^32 or more interior cells are not supported");
    return GRMHD_OK;
}

grmhd_status check_tab(const grmhd_tableau* t)
{
    if (!t) return fail(GRMHD_ERR_ARG, "tableau is NULL");
    if (t->s < 1 || t->s > 4) return fail(GRMHD_ERR_ARG, "tableau must have 1..4 stages");
    for (int i = 0; i < t->s; i++) {
        if (!(t->A[i * t->s + i] > 0.0)) return fail(GRMHD_ERR_ARG, "implicit tableau needs a_ii > 0");
        for (int j = i; j < t->s; j++)
            if (t->At[i * t->s + j] != 0.0) return fail(GRMHD_ERR_ARG, "explicit tableau must be strictly lower");
        for (int j = i + 1; j < t->s; j++)
            if (t->A[i * t->s + j] != 0.0) return fail(GRMHD_ERR_ARG, "implicit tableau must be lower triangular");
    }
    return GRMHD_OK;
}

Dims make_dims(const grmhd_grid* gr, double gam)
{
    Dims g;
    g.ncell = 1;
    for (int d = 0; d < 3; d++) {
        g.act[d] = d < gr->ndim;
        g.n[d] = g.act[d] ? gr->n[d] : 1;
        g.ng[d] = g.act[d] ? 2 : 0;
        g.N[d] = g.n[d] + 2 * g.ng[d];
        g.bc[d] = g.act[d] ? gr->bc[d] : GRMHD_BC_PERIODIC;
        g.idx[d] = g.act[d] ? g.n[d] / (gr->hi[d] - gr->lo[d]) : 0.0;
        g.ncell *= g.N[d];
    }
    g.st[0] = 1;
    g.st[1] = g.N[0];
    g.st[2] = (long long)g.N[0] * g.N[1];
    g.gh = gam / (gam - 1.0);
    g.igh = (gam - 1.0) / gam;
    set_divisors(g);
    return g;
}

// scratch carve: returns the byte count; with base != NULL assigns the pointers
size_t carve(grmhd_ctx* c, const Dims& g, int s, int ndim, char* base, bool glm = false)
{
    const size_t arr = round_up(sizeof(double) * (size_t)g.ncell);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += round_up(bytes);
        return p;
    };
    if (glm) {
        // GLM: 12 cell-centred variables per stage base and flux direction, no EMFs
        for (int v = 0; v < 8; v++) { char* p = take(arr); if (c) c->prim[v] = (double*)p; }
        for (int v = 0; v < 3; v++) { char* p = take(arr); if (c) c->R[v] = (double*)p; }
        for (int k = 1; k < s; k++)
            for (int v = 0; v < 12; v++) { char* p = take(arr); if (c) c->base[k][v] = (double*)p; }
        for (int v = 0; v < 12; v++) { char* p = take(arr); if (c) c->acc[v] = (double*)p; }
        for (int d = 0; d < ndim; d++)
            for (int v = 0; v < 12; v++) { char* p = take(arr); if (c) c->F[d][v] = (double*)p; }
        const size_t arr32 = round_up(sizeof(float) * (size_t)g.ncell);
        for (int k = 0; k < s; k++)
            for (int v = 0; v < 3; v++) {
                char* p = take(arr32);
                char* q = take(arr32);
                if (c) { c->hs[k][v] = (float*)p; c->hd[k][v] = (float*)q; }
            }
        { char* p = take(sizeof(double) * kRedBlocks * 11); if (c) c->red_part = (double*)p; }
        { char* p = take(sizeof(double) * 16); if (c) c->red_out = (double*)p; }
        { char* p = take(sizeof(unsigned long long)); if (c) c->nfail = (unsigned long long*)p; }
        return off;
    }
    for (int v = 0; v < 8; v++) { char* p = take(arr); if (c) c->prim[v] = (double*)p; }
    for (int v = 0; v < 3; v++) { char* p = take(arr); if (c) c->R[v] = (double*)p; }
    for (int k = 1; k < s; k++)
        for (int v = 0; v < 11; v++) { char* p = take(arr); if (c) c->base[k][v] = (double*)p; }
    for (int v = 0; v < 11; v++) { char* p = take(arr); if (c) c->acc[v] = (double*)p; }
    for (int d = 0; d < ndim; d++)
        for (int v = 0; v < 8; v++) { char* p = take(arr); if (c) c->F[d][v] = (double*)p; }
    for (int v = 0; v < 3; v++) { char* p = take(arr); if (c) c->Eh[v] = (double*)p; }
    for (int d = 0; d < ndim; d++)
        for (int k = 0; k < 2; k++) { char* p = take(arr); if (c) c->vblk[d][k] = (double*)p; }
    const size_t arr32 = round_up(sizeof(float) * (size_t)g.ncell);
    for (int v = 0; v < 11; v++) { char* p = take(arr32); if (c) c->p32[v] = (float*)p; }
    for (int k = 0; k < s; k++)
        for (int v = 0; v < 3; v++) {
            char* p = take(arr32);
            char* q = take(arr32);
            if (c) { c->hs[k][v] = (float*)p; c->hd[k][v] = (float*)q; }
        }
    { char* p = take(sizeof(double) * kRedBlocks * 11); if (c) c->red_part = (double*)p; }
    { char* p = take(sizeof(double) * 16); if (c) c->red_out = (double*)p; }
    { char* p = take(sizeof(unsigned long long)); if (c) c->nfail = (unsigned long long*)p; }
    return off;
}

CP8 cp8(double* const* p)
{
    CP8 r;
    for (int v = 0; v < 8; v++) r.p[v] = p[v];
    return r;
}
CP8 cp8c(const double* const* p)
{
    CP8 r;
    for (int v = 0; v < 8; v++) r.p[v] = p[v];
    return r;
}
CP3 cp3(double* const* p)
{
    CP3 r;
    for (int v = 0; v < 3; v++) r.p[v] = p[v];
    return r;
}
CP3 cp3c(const double* const* p)
{
    CP3 r;
    for (int v = 0; v < 3; v++) r.p[v] = p[v];
    return r;
}
P8 p8(double* const* p)
{
    P8 r;
    for (int v = 0; v < 8; v++) r.p[v] = p[v];
    return r;
}
P3 p3(double* const* p)
{
    P3 r;
    for (int v = 0; v < 3; v++) r.p[v] = p ? p[v] : nullptr;
    return r;
}

bool emf_needed(const Dims& g, int c) { return g.act[(c + 1) % 3] || g.act[(c + 2) % 3]; }

// the flux direction whose kernel writes the edge EMF of direction c (flat metric,
// resistive UCT, exactly one of the two directions transverse to c active: the edges
// then coincide with that direction's faces, and the MC or PPM face states the flux
// kernel holds are the reconstructions the EMF needs), else -1
int fused_emf_dir(const grmhd_ctx* c, int k)
{
    const Dims& g = c->g;
    if (c->psi || c->alp || c->ideal) return -1;
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    if (g.act[a] == g.act[b]) return -1;
    return g.act[a] ? a : b;
}

ImpArgs imp_args(grmhd_ctx* c, CP8 qb, CP3 bf, double a_dt, P8 prim, P3 R, P3 qE_out, F11 p32)
{
    ImpArgs a;
    a.qb = qb;
    a.bf = bf;
    a.psi = c->psi;
    a.alp = c->alp;
    a.eta = c->eta;
    a.eta_u = c->eta_u;
    a.a_dt = a_dt;
    a.ia_dt = a_dt > 0.0 ? 1.0 / a_dt : 0.0;
    a.ighf = (float)c->g.igh;
    a.xif = (float)c->xi;
    a.prim = prim;
    a.R = R;
    a.qE_out = qE_out;
    a.kmax = c->par.newton_kmax;
    a.tol = c->par.newton_tol;
    a.tolf = (float)c->par.newton_tol;
    a.dwacc = c->mixed ? 1 : 0;
    a.stiff = a_dt > 0.0;
    a.rho_atm = c->par.rho_atm;
    a.p_atm = c->par.p_atm;
    a.atm = c->par.rho_atm > 0.0;
    a.d_atm = 10.0 * c->par.rho_atm;
    a.xi = c->xi;
    a.p32 = p32;
    a.nfail = c->nfail;
    for (int v = 0; v < 3; v++) a.hs[v] = a.hd[v] = nullptr;
    return a;
}

F11 f11(grmhd_ctx* c)
{
    F11 r;
    for (int v = 0; v < 11; v++) r.p[v] = c->mixed ? c->p32[v] : nullptr;
    return r;
}

// programmatic dependent launch for the kernels launched while it lives (the stage
// kernels open with grid_dep_sync, launch.cuh); restores the previous setting
struct OverlapScope {
    bool prev;
    explicit OverlapScope(bool on) : prev(grmhd::launch_overlap) { grmhd::launch_overlap = on; }
    ~OverlapScope() { grmhd::launch_overlap = prev; }
    OverlapScope(const OverlapScope&) = delete;
    OverlapScope& operator=(const OverlapScope&) = delete;
};

// kernel kinds for the timing hooks
enum { KIND_IMPLICIT = 0, KIND_FLUX = 1, KIND_EMF = 2, KIND_UPDATE = 3 };

int tbegin(grmhd_ctx* c, int kind, cudaStream_t st)
{
    if (!c->timing || c->npend >= 64) return -1;
    const int i = c->npend++;
    c->ev_kind[i] = kind;
    cudaEventRecord(c->ev[i][0], st);
    return i;
}

void tend(grmhd_ctx* c, int i, cudaStream_t st)
{
    if (i >= 0) cudaEventRecord(c->ev[i][1], st);
}

// fluxes, EMFs and the update for the given stage primitives / faces
grmhd_status explicit_part(grmhd_ctx* c, CP8 prim, CP3 bfs, UpdateArgs& a, cudaStream_t st)
{
    const Dims& g = c->g;
    cudaError_t e;
    // mixed precision: reconstruction, HLL and the edge EMF in FP32 from the stage's
    // FP32 primitives; the update (sources, CT, stage folds) stays FP64
    PrimIn<float> p32;
    for (int v = 0; v < 11; v++) p32.p[v] = c->p32[v];
    if (c->mixed) {
        // FP32 arithmetic and FP32 fluxes (in the first half of each flux array): the
        // fluxes of every direction and the edge EMFs in one launch
        FluxOut<float> fo[3];
        double* fe[3][3];
        double* eh[3];
        for (int d = 0; d < 3; d++)
            for (int v = 0; v < 8; v++) fo[d].p[v] = reinterpret_cast<float*>(c->F[d][v]);
        for (int d = 0; d < 3; d++)
            for (int k = 0; k < 3; k++) fe[d][k] = fused_emf_dir(c, k) == d ? c->Eh[k] : nullptr;
        for (int k = 0; k < 3; k++) eh[k] = emf_needed(g, k) && fused_emf_dir(c, k) < 0 ? c->Eh[k] : nullptr;
        const int tk = tbegin(c, KIND_FLUX, st);
        e = launch_stencil32(g, p32, bfs, c->psi, c->alp, fo, fe, eh, c->nsm, st, c->ppm);
        tend(c, tk, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "stencil kernel");
    }
    // FP64, resistive UCT: likewise one launch, unless the flux of a single direction is
    // the only task (a flat 1-D grid), where the plain flux kernel launches faster
    int ntask = 0;
    for (int d = 0; d < 3; d++) ntask += g.act[d] ? 1 : 0;
    for (int k = 0; k < 3; k++) ntask += emf_needed(g, k) && fused_emf_dir(c, k) < 0 ? 1 : 0;
    const bool fused = c->mixed || (!c->ideal && ntask > 1);
    if (!c->mixed && fused) {
        P8 fo[3];
        double* fe[3][3];
        double* eh[3];
        for (int d = 0; d < 3; d++) fo[d] = p8(c->F[d]);
        for (int d = 0; d < 3; d++)
            for (int k = 0; k < 3; k++) fe[d][k] = fused_emf_dir(c, k) == d ? c->Eh[k] : nullptr;
        for (int k = 0; k < 3; k++) eh[k] = emf_needed(g, k) && fused_emf_dir(c, k) < 0 ? c->Eh[k] : nullptr;
        const int tk = tbegin(c, KIND_FLUX, st);
        e = launch_stencil64(g, prim, bfs, c->psi, c->alp, fo, fe, eh, c->nsm, st, c->ppm);
        tend(c, tk, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "stencil kernel");
    }
    // the ideal-limit EMF: the flux launches (which also write the transport velocities),
    // then one EMF launch per edge direction; or the one flux launch of a flat 1-D grid
    for (int d = 0; d < 3 && !fused; d++) {
        if (!g.act[d]) continue;
        const int tk = tbegin(c, KIND_FLUX, st);
        double* eh64[3] = {nullptr, nullptr, nullptr};
        for (int k = 0; k < 3; k++)
            if (fused_emf_dir(c, k) == d) eh64[k] = c->Eh[k];
        e = launch_flux(g, d, prim, bfs, c->psi, c->alp, p8(c->F[d]), c->nsm, st, c->ideal ? c->vbar[d] : nullptr,
                        c->ppm, eh64);
        tend(c, tk, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "flux kernel");
    }
    for (int k = 0; k < 3 && !fused; k++) {
        if (!emf_needed(g, k) || fused_emf_dir(c, k) >= 0) continue;
        const int tk = tbegin(c, KIND_EMF, st);
        e = launch_emf_ideal(g, k, prim, bfs, c->psi, c->alp, c->vbar, c->Eh[k], c->nsm, st);
        tend(c, tk, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "emf kernel");
    }
    for (int d = 0; d < 3; d++)
        for (int v = 0; v < 8; v++) a.F[d][v] = !g.act[d] ? nullptr : c->F[d][v];
    a.f32 = c->mixed ? 1 : 0;
    for (int k = 0; k < 3; k++) a.Eh[k] = c->Eh[k];
    for (int v = 0; v < 8; v++) a.prim[v] = prim.p[v];
    for (int v = 0; v < 11; v++) a.p32[v] = c->mixed ? c->p32[v] : nullptr;
    for (int k = 0; k < 3; k++) a.bf[k] = bfs.p[k];
    a.psi = c->psi;
    a.alp = c->alp;
    const int tk = tbegin(c, KIND_UPDATE, st);
    e = launch_update(g, a, c->nsm, st);
    tend(c, tk, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "update kernel");
    return GRMHD_OK;
}

// GLM (Sec. 3.1): fluxes of the 12 cell-centred variables per direction, then the
// update; qB / qphi are the stage's cell fields
grmhd_status explicit_part_glm(grmhd_ctx* c, CP8 prim, CP3 qB, const double* qphi, GlmUpdateArgs& a,
                               cudaStream_t st)
{
    const Dims& g = c->g;
    cudaError_t e;
    GlmFluxArgs fa;
    for (int v = 0; v < 8; v++) fa.prim[v] = prim.p[v];
    for (int v = 0; v < 3; v++) fa.qB[v] = qB.p[v];
    fa.qphi = qphi;
    fa.psi = c->psi;
    fa.alp = c->alp;
    for (int d = 0; d < 3; d++) {
        if (!g.act[d]) continue;
        for (int v = 0; v < 12; v++) fa.F[v] = c->F[d][v];
        const int tk = tbegin(c, KIND_FLUX, st);
        e = launch_glm_flux(g, d, fa, c->nsm, st, c->ppm);
        tend(c, tk, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "GLM flux kernel");
    }
    for (int d = 0; d < 3; d++)
        for (int v = 0; v < 12; v++) a.F[d][v] = g.act[d] ? c->F[d][v] : nullptr;
    for (int v = 0; v < 8; v++) a.prim[v] = prim.p[v];
    for (int v = 0; v < 3; v++) a.qB[v] = qB.p[v];
    a.qphi = qphi;
    a.psi = c->psi;
    a.alp = c->alp;
    a.kappa = c->kappa;
    const int tk = tbegin(c, KIND_UPDATE, st);
    e = launch_glm_update(g, a, c->nsm, st);
    tend(c, tk, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "GLM update kernel");
    return GRMHD_OK;
}

// GLM stage update arguments (the stage folds of UpdateArgs over 12 variables)
void glm_stage_args(grmhd_ctx* c, int i, double dt, GlmUpdateArgs* a)
{
    const int S = c->tab.s;
    memset(a, 0, sizeof *a);
    a->mode = UPD_STAGE;
    a->stage = i;
    a->s = S;
    a->dt = dt;
    for (int r = 0; r < S; r++) {
        for (int k = 0; k < S; k++) {
            a->At[r][k] = c->tab.At[r * S + k];
            a->A[r][k] = c->tab.A[r * S + k];
        }
        a->wt[r] = c->tab.wt[r];
        a->w[r] = c->tab.w[r];
        a->cL[r] = dt * c->tab.At[r * S + i];
        a->cR[r] = dt * c->tab.A[r * S + i];
    }
    a->cwL = dt * c->tab.wt[i];
    a->cwR = dt * c->tab.w[i];
    for (int v = 0; v < 3; v++) a->R[v] = c->R[v];
    for (int v = 0; v < 8; v++) a->qn[v] = c->q[v];
    for (int v = 0; v < 3; v++) a->qn[8 + v] = c->bf[v];
    a->qn[11] = c->qphi;
    for (int k = 1; k < S; k++)
        for (int v = 0; v < 12; v++) a->base[k][v] = c->base[k][v];
    for (int v = 0; v < 12; v++) a->acc[v] = c->acc[v];
}

grmhd_status need_bound(const grmhd_ctx* c)
{
    if (!c) return fail(GRMHD_ERR_ARG, "context is NULL");
    if (!c->bound) return fail(GRMHD_ERR_STATE, "call grmhd_bind first");
    return GRMHD_OK;
}


}  // namespace

extern "C" {

grmhd_status grmhd_tableau_ssp2(grmhd_tableau* t)
{
    if (!t) return fail(GRMHD_ERR_ARG, "tableau is NULL");
    memset(t, 0, sizeof *t);
    const double gm = 1.0 - 1.0 / std::sqrt(2.0);
    t->s = 2;
    t->At[2] = 1.0;  // At[1][0]
    t->A[0] = gm;
    t->A[2] = 1.0 - 2.0 * gm;
    t->A[3] = gm;
    t->wt[0] = t->wt[1] = 0.5;
    t->w[0] = t->w[1] = 0.5;
    return GRMHD_OK;
}

grmhd_status grmhd_scratch_bytes(const grmhd_grid* grid, const grmhd_tableau* tab, size_t* bytes)
{
    grmhd_status s = check_grid(grid);
    if (s != GRMHD_OK) return s;
    if ((s = check_tab(tab)) != GRMHD_OK) return s;
    if (!bytes) return fail(GRMHD_ERR_ARG, "bytes is NULL");
    Dims g = make_dims(grid, 2.0);
    // enough for either divergence scheme
    *bytes = std::max(carve(nullptr, g, tab->s, grid->ndim, nullptr, false),
                      carve(nullptr, g, tab->s, grid->ndim, nullptr, true));
    return GRMHD_OK;
}

grmhd_status grmhd_create(const grmhd_grid* grid, const grmhd_params* par, const grmhd_tableau* tab,
                          grmhd_ctx** out)
{
    grmhd_status s = check_grid(grid);
    if (s != GRMHD_OK) return s;
    if ((s = check_tab(tab)) != GRMHD_OK) return s;
    if (!par || !out) return fail(GRMHD_ERR_ARG, "params/out is NULL");
    if (!(par->gamma_eos > 1.0)) return fail(GRMHD_ERR_ARG, "gamma_eos must exceed 1");
    if (par->rho_atm < 0.0 || par->p_atm < 0.0) return fail(GRMHD_ERR_ARG, "atmosphere floor must be >= 0");
    if (par->precision != GRMHD_PREC_FP64 && par->precision != GRMHD_PREC_MIXED)
        return fail(GRMHD_ERR_ARG, "precision must be GRMHD_PREC_FP64 or GRMHD_PREC_MIXED");
    if (par->divb != GRMHD_DIVB_CT && par->divb != GRMHD_DIVB_GLM)
        return fail(GRMHD_ERR_ARG, "divb must be GRMHD_DIVB_CT or GRMHD_DIVB_GLM");
    // the mixed path accepts the root by its double-word residual (~1e-14 of the
    // momentum scale), which bounds the exact residual for tolerances from 1e-11 up
    if (par->precision == GRMHD_PREC_MIXED && par->newton_tol > 0.0 && par->newton_tol < 1e-11)
        return fail(GRMHD_ERR_ARG, "mixed precision needs newton_tol >= 1e-11 (or 0 for the default 1e-10)");
    if (par->divb == GRMHD_DIVB_GLM && par->precision != GRMHD_PREC_FP64)
        return fail(GRMHD_ERR_ARG, "GLM cleaning runs in FP64 only");
    if (par->divb == GRMHD_DIVB_GLM && !(par->kappa_b >= 0.0))
        return fail(GRMHD_ERR_ARG, "kappa_b must be >= 0");
    if (par->emf != GRMHD_EMF_RESISTIVE && par->emf != GRMHD_EMF_IDEAL)
        return fail(GRMHD_ERR_ARG, "emf must be GRMHD_EMF_RESISTIVE or GRMHD_EMF_IDEAL");
    if (par->rec != GRMHD_REC_MC && par->rec != GRMHD_REC_PPM)
        return fail(GRMHD_ERR_ARG, "rec must be GRMHD_REC_MC or GRMHD_REC_PPM");
    if (par->rec == GRMHD_REC_PPM && par->emf == GRMHD_EMF_IDEAL)
        return fail(GRMHD_ERR_ARG, "PPM takes the resistive EMF or GLM");
    if (par->emf == GRMHD_EMF_IDEAL) {
        if (par->divb != GRMHD_DIVB_CT || par->precision != GRMHD_PREC_FP64)
            return fail(GRMHD_ERR_ARG, "the ideal-limit EMF needs constrained transport in FP64");
        for (int d = 0; d < grid->ndim; d++)
            if (grid->bc[d] == GRMHD_BC_FIXED)
                return fail(GRMHD_ERR_ARG, "the ideal-limit EMF does not take FIXED boundaries");
    }
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    grmhd_ctx* c = new (std::nothrow) grmhd_ctx_s();
    if (!c) return fail(GRMHD_ERR_ARG, "out of host memory");
    c->g = make_dims(grid, par->gamma_eos);
    c->grid = *grid;
    c->par = *par;
    // the mixed path's FP32 fluxes carry relative errors near 1e-7: a residual below
    // 1e-10 changes none of its results and saves Newton iterations
    if (c->par.newton_tol <= 0.0) c->par.newton_tol = c->par.precision == GRMHD_PREC_MIXED ? 1e-10 : 1e-13;
    if (c->par.newton_kmax <= 0) c->par.newton_kmax = 50;
    c->tab = *tab;
    c->dV = 1.0;
    c->any_fixed = false;
    for (int d = 0; d < grid->ndim; d++) {
        c->dV *= (grid->hi[d] - grid->lo[d]) / grid->n[d];
        if (grid->bc[d] == GRMHD_BC_FIXED) c->any_fixed = true;
    }
    c->nsm = nsm;
    c->mixed = par->precision == GRMHD_PREC_MIXED;
    c->glm = par->divb == GRMHD_DIVB_GLM;
    c->ideal = par->emf == GRMHD_EMF_IDEAL;
    c->ppm = par->rec == GRMHD_REC_PPM;
    c->kappa = c->glm ? par->kappa_b : 0.0;
    *out = c;
    return GRMHD_OK;
}

grmhd_status grmhd_destroy(grmhd_ctx* ctx)
{
    if (ctx && ctx->ev_made)
        for (int i = 0; i < 64; i++) {
            cudaEventDestroy(ctx->ev[i][0]);
            cudaEventDestroy(ctx->ev[i][1]);
        }
    delete ctx;
    return GRMHD_OK;
}

grmhd_status grmhd_set_timing(grmhd_ctx* c, int enable)
{
    if (!c) return fail(GRMHD_ERR_ARG, "context is NULL");
    if (enable && !c->timing) {
        if (!c->ev_made) {
            for (int i = 0; i < 64; i++)
                for (int k = 0; k < 2; k++) {
                    cudaError_t e = cudaEventCreate(&c->ev[i][k]);
                    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
                }
            c->ev_made = true;
        }
        c->timing = true;
        c->npend = 0;
        for (int k = 0; k < 4; k++) { c->t_ms[k] = 0.0; c->t_n[k] = 0; }
    } else if (!enable && c->timing) {
        // events already recorded stay readable until the next grmhd_set_timing(1)
        c->timing = false;
    }
    return GRMHD_OK;
}

grmhd_status grmhd_set_launch_overlap(grmhd_ctx* c, int enable)
{
    if (!c) return fail(GRMHD_ERR_ARG, "context is NULL");
    c->overlap = enable != 0;
    return GRMHD_OK;
}

grmhd_status grmhd_kernel_times(grmhd_ctx* c, double* ms, long long* launches)
{
    if (!c) return fail(GRMHD_ERR_ARG, "context is NULL");
    if (!c->ev_made) return fail(GRMHD_ERR_STATE, "timing is off: call grmhd_set_timing first");
    for (int i = 0; i < c->npend; i++) {
        cudaError_t e = cudaEventSynchronize(c->ev[i][1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, c->ev[i][0], c->ev[i][1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        c->t_ms[c->ev_kind[i]] += t;
        c->t_n[c->ev_kind[i]] += 1;
    }
    c->npend = 0;
    for (int k = 0; k < 4; k++) {
        if (ms) ms[k] = c->t_ms[k];
        if (launches) launches[k] = c->t_n[k];
    }
    return GRMHD_OK;
}

grmhd_status grmhd_bind(grmhd_ctx* c, double* const* q, double* const* bface, void* scratch, size_t scratch_bytes)
{
    if (!c || !q || !bface || !scratch) return fail(GRMHD_ERR_ARG, "NULL argument to grmhd_bind");
    for (int v = 0; v < 8; v++)
        if (!q[v]) return fail(GRMHD_ERR_ARG, "q[v] is NULL");
    for (int v = 0; v < 3; v++)
        if (!bface[v]) return fail(GRMHD_ERR_ARG, "bface[v] is NULL");
    if ((uintptr_t)scratch % kAlign) return fail(GRMHD_ERR_SCRATCH, "scratch must be 256-byte aligned");
    const size_t need = carve(nullptr, c->g, c->tab.s, c->grid.ndim, nullptr, c->glm);
    if (scratch_bytes < need) return fail(GRMHD_ERR_SCRATCH, "scratch smaller than grmhd_scratch_bytes");
    carve(c, c->g, c->tab.s, c->grid.ndim, (char*)scratch, c->glm);
    // ideal-limit EMF: its two transport-velocity arrays per direction
    for (int d = 0; d < 3; d++)
        for (int k = 0; k < 2; k++) c->vbar[d][k] = (c->ideal && d < c->grid.ndim) ? c->vblk[d][k] : nullptr;
    for (int v = 0; v < 8; v++) c->q[v] = q[v];
    for (int v = 0; v < 3; v++) c->bf[v] = bface[v];
    c->bound = true;
    cudaError_t e = cudaMemsetAsync(c->nfail, 0, sizeof(unsigned long long), 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return GRMHD_OK;
}

grmhd_status grmhd_bind_phi(grmhd_ctx* c, double* q_phi)
{
    if (!c || !q_phi) return fail(GRMHD_ERR_ARG, "NULL argument to grmhd_bind_phi");
    if (!c->glm) return fail(GRMHD_ERR_STATE, "grmhd_bind_phi needs a GLM context");
    c->qphi = q_phi;
    return GRMHD_OK;
}

grmhd_status grmhd_set_metric(grmhd_ctx* c, const double* alpha, const double* psi)
{
    if (!c) return fail(GRMHD_ERR_ARG, "context is NULL");
    if ((alpha || psi) && c->tab.s == 1)
        return fail(GRMHD_ERR_ARG, "a curved metric needs a tableau with at least two stages");
    c->alp = alpha;
    c->psi = psi;
    return GRMHD_OK;
}

grmhd_status grmhd_set_eta(grmhd_ctx* c, const double* eta_cc, double eta_uniform)
{
    if (!c) return fail(GRMHD_ERR_ARG, "context is NULL");
    if (!eta_cc && !(eta_uniform > 0.0)) return fail(GRMHD_ERR_ARG, "uniform eta must be positive");
    c->eta = eta_cc;
    c->eta_u = eta_uniform;
    return GRMHD_OK;
}

grmhd_status grmhd_set_dynamo(grmhd_ctx* c, double xi)
{
    if (!c) return fail(GRMHD_ERR_ARG, "context is NULL");
    if (!(xi == xi)) return fail(GRMHD_ERR_ARG, "xi must be a number");
    c->xi = xi;
    return GRMHD_OK;
}

// Newton start history of every stage: the initial velocity, no trend
static grmhd_status init_history(grmhd_ctx* c, const double* const* prim, cudaStream_t st)
{
    for (int k = 0; k < c->tab.s; k++) {
        P3f hs, hd;
        for (int v = 0; v < 3; v++) {
            hs.p[v] = c->hs[k][v];
            hd.p[v] = c->hd[k][v];
        }
        cudaError_t e = launch_hist_init(c->g, prim[1], prim[2], prim[3], c->psi, hs, hd, c->nsm, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "history kernel");
    }
    c->hist = true;
    return GRMHD_OK;
}

grmhd_status grmhd_init_from_prims(grmhd_ctx* c, const double* const* prim, const double* const* A_edge,
                                   grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (!prim) return fail(GRMHD_ERR_ARG, "prim is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const Dims& g = c->g;
    const size_t bytes = sizeof(double) * (size_t)g.ncell;
    cudaError_t e;
    if (c->glm) {
        if (!c->qphi) return fail(GRMHD_ERR_STATE, "call grmhd_bind_phi first");
        if (A_edge) {
            e = launch_curlA_cc(g, cp3c(A_edge), p3(c->bf), c->nsm, st);
            c->launches++;
            if (e != cudaSuccess) return cuda_fail(e, "curl kernel");
        }
        for (int v = 0; v < 8; v++) {
            e = cudaMemcpyAsync(c->prim[v], prim[v], bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        }
        // prim[8] is the primitive Phi (NULL: zero); the kernel densitises it
        e = launch_prim2con_cc(g, cp8c(prim), cp3(c->bf), c->psi, prim[8], c->qphi, p8(c->q), c->nsm, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "prim2con kernel");
        return init_history(c, prim, st);
    }
    if (A_edge) {
        for (int v = 0; v < 3; v++) {
            e = cudaMemsetAsync(c->bf[v], 0, bytes, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        }
        e = launch_curlA(g, cp3c(A_edge), p3(c->bf), c->nsm, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "curl kernel");
    }
    for (int v = 0; v < 8; v++) {
        e = cudaMemcpyAsync(c->prim[v], prim[v], bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
    e = launch_prim2con(g, cp8c(prim), cp3(c->bf), c->psi, p8(c->q), c->nsm, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "prim2con kernel");
    if (c->mixed) {
        e = launch_prim_to32(g, cp8c(prim), cp3(c->bf), f11(c), c->nsm, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "prim_to32 kernel");
    }
    return init_history(c, prim, st);
}

grmhd_status grmhd_compute_dt(grmhd_ctx* c, double* dt, grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (!dt) return fail(GRMHD_ERR_ARG, "dt is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_dt(c->g, c->psi, c->alp, c->red_part, kRedBlocks, c->red_out, st);
    c->launches += 2;
    if (e != cudaSuccess) return cuda_fail(e, "dt kernel");
    double mx = 0.0;
    e = cudaMemcpyAsync(&mx, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "dt readback");
    if (!(mx > 0.0)) return fail(GRMHD_ERR_ARG, "characteristic speeds vanish");
    *dt = c->par.cfl / mx;
    return GRMHD_OK;
}

grmhd_status grmhd_stage(grmhd_ctx* c, int i, double dt, grmhd_stream_t stream)
{
    NvtxRange nv("grmhd_stage");
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (i < 0 || i >= c->tab.s) return fail(GRMHD_ERR_ARG, "stage index out of range");
    if (!(dt > 0.0)) return fail(GRMHD_ERR_ARG, "dt must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (c->glm && !c->qphi) return fail(GRMHD_ERR_STATE, "call grmhd_bind_phi first");
    // events recorded between the launches would serialise them anyway
    const OverlapScope ov(c->overlap && !c->timing);
    if (i == 0 && c->any_fixed) {
        e = ctx_copy_fixed_faces(c, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
    ImpArgs ia;
    UpdateArgs a;
    ctx_stage_args(c, i, dt, &ia, &a);
    if (c->glm) {
        // GLM: the stage's cell q_B (ia.bf) and q_Phi are the bound state at stage 0 and
        // the stage base afterwards
        const int tk = tbegin(c, KIND_IMPLICIT, st);
        e = launch_implicit_cc(c->g, ia, c->nsm, st);
        tend(c, tk, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "implicit kernel");
        GlmUpdateArgs ga;
        glm_stage_args(c, i, dt, &ga);
        CP8 pr;
        for (int v = 0; v < 8; v++) pr.p[v] = c->prim[v];
        return explicit_part_glm(c, pr, ia.bf, i == 0 ? c->qphi : c->base[i][11], ga, st);
    }
    const int tk = tbegin(c, KIND_IMPLICIT, st);
    e = launch_implicit(c->g, ia, c->nsm, st);
    tend(c, tk, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "implicit kernel");
    CP8 pr;
    for (int v = 0; v < 8; v++) pr.p[v] = c->prim[v];
    return explicit_part(c, pr, ia.bf, a, st);
}

grmhd_status grmhd_step(grmhd_ctx* c, double dt, grmhd_stream_t stream)
{
    NvtxRange nv("grmhd_step");
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    for (int i = 0; i < c->tab.s; i++) {
        s = grmhd_stage(c, i, dt, stream);
        if (s != GRMHD_OK) return s;
    }
    return GRMHD_OK;
}

grmhd_status grmhd_get_prims(grmhd_ctx* c, double* const* prim_out, grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (!prim_out) return fail(GRMHD_ERR_ARG, "prim_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    for (int v = 0; v < 8; v++) {
        e = cudaMemcpyAsync(prim_out[v], c->prim[v], sizeof(double) * (size_t)c->g.ncell, cudaMemcpyDeviceToDevice,
                            st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
    const ImpArgs ia = imp_args(c, cp8(c->q), cp3(c->bf), 0.0, p8(prim_out), p3(nullptr), p3(nullptr), F11{});
    e = c->glm ? launch_implicit_cc(c->g, ia, c->nsm, st) : launch_implicit(c->g, ia, c->nsm, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "con2prim kernel");
    return GRMHD_OK;
}

grmhd_status grmhd_implicit(grmhd_ctx* c, double a_dt, double* const* q, const double* const* bface,
                            double* const* prim, double* const* R, grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (!q || !bface || !prim || !R) return fail(GRMHD_ERR_ARG, "NULL argument to grmhd_implicit");
    const ImpArgs ia = imp_args(c, cp8(q), cp3c(bface), a_dt, p8(prim), p3(R), p3(q + 5), F11{});
    cudaError_t e = c->glm ? launch_implicit_cc(c->g, ia, c->nsm, (cudaStream_t)stream)
                           : launch_implicit(c->g, ia, c->nsm, (cudaStream_t)stream);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(e, "implicit kernel");
    return GRMHD_OK;
}

grmhd_status grmhd_explicit_L(grmhd_ctx* c, const double* const* prim, const double* const* bface, double* const* L,
                              grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (!prim || !bface || !L) return fail(GRMHD_ERR_ARG, "NULL argument to grmhd_explicit_L");
    if (c->glm) return fail(GRMHD_ERR_STATE, "GLM context: use grmhd_explicit_L_glm");
    if (c->mixed) {
        cudaError_t e = launch_prim_to32(c->g, cp8c(prim), cp3c(bface), f11(c), c->nsm, (cudaStream_t)stream);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(e, "prim_to32 kernel");
    }
    UpdateArgs a;
    memset(&a, 0, sizeof a);
    a.mode = UPD_WRITE_L;
    for (int v = 0; v < 11; v++) a.L[v] = L[v];
    return explicit_part(c, cp8c(prim), cp3c(bface), a, (cudaStream_t)stream);
}

grmhd_status grmhd_explicit_L_glm(grmhd_ctx* c, const double* const* prim, const double* const* qB,
                                  const double* q_phi, double* const* L, grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (!prim || !qB || !q_phi || !L) return fail(GRMHD_ERR_ARG, "NULL argument to grmhd_explicit_L_glm");
    if (!c->glm) return fail(GRMHD_ERR_STATE, "grmhd_explicit_L_glm needs a GLM context");
    GlmUpdateArgs a;
    memset(&a, 0, sizeof a);
    a.mode = UPD_WRITE_L;
    for (int v = 0; v < 12; v++) a.L[v] = L[v];
    return explicit_part_glm(c, cp8c(prim), cp3c(qB), q_phi, a, (cudaStream_t)stream);
}

grmhd_status grmhd_diagnostics(grmhd_ctx* c, double* divb, double* totals, long long* nfail, grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = c->glm ? launch_diag_cc(c->g, cp3(c->bf), cp8(c->q), c->dV, c->red_part, kRedBlocks, c->red_out, st)
                           : launch_diag(c->g, cp3(c->bf), cp8(c->q), c->dV, c->red_part, kRedBlocks, c->red_out, st);
    c->launches += 2;
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics kernel");
    double out[11];
    unsigned long long nf = 0;
    e = cudaMemcpyAsync(out, c->red_out, sizeof out, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nf, c->nfail, sizeof nf, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics readback");
    const double ncell = (double)c->g.n[0] * c->g.n[1] * c->g.n[2];
    if (divb) {
        divb[0] = out[0] / ncell;
        divb[1] = std::sqrt(out[1] / ncell);
        divb[2] = out[2];
    }
    if (totals)
        for (int v = 0; v < 8; v++) totals[v] = out[3 + v];
    if (nfail) *nfail = (long long)nf;
    return nf ? GRMHD_WARN_C2P_FAILED : GRMHD_OK;
}

grmhd_status grmhd_bounds_violations(long long* count, int reset)
{
    if (!count) return fail(GRMHD_ERR_ARG, "count is NULL");
#ifdef GRMHD_CHECK_BOUNDS
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before reading the bounds counters");
    unsigned long long (*const readers[])(bool) = {oob_kernels, oob_glm, oob_elliptic, oob_batch, oob_noalloc};
    unsigned long long total = 0;
    for (auto rd : readers) {
        const unsigned long long v = rd(reset != 0);
        if (v == ~0ull) return fail(GRMHD_ERR_CUDA, "reading a bounds counter failed");
        total += v;
    }
    *count = (long long)total;
#else
    (void)reset;
    *count = -1;   // not a checked build
#endif
    return GRMHD_OK;
}

grmhd_status grmhd_clean_scratch_bytes(const grmhd_grid* grid, size_t* bytes)
{
    grmhd_status s = check_grid(grid);
    if (s != GRMHD_OK) return s;
    if (!bytes) return fail(GRMHD_ERR_ARG, "bytes is NULL");
    MgPlan plan;
    const int r = mg_plan(make_dims(grid, 2.0), &plan);
    if (r == -1) return fail(GRMHD_ERR_ARG, "multigrid: too many levels");
    if (r == -2)
        return fail(GRMHD_ERR_ARG,
                    "multigrid: the coarsest level (every active extent halved while all are even and >= 4) "
                    "has more than 4096 cells");
    if (r == -3) return fail(GRMHD_ERR_ARG, "multigrid: the grid has 2^31 cells or more");
    *bytes = round_up(mg_scratch_bytes(plan));
    return GRMHD_OK;
}

grmhd_status grmhd_clean_divb(grmhd_ctx* c, int cycles, void* scratch, size_t scratch_bytes, grmhd_stream_t stream)
{
    NvtxRange nv("grmhd_clean_divb");
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (cycles < 1 || cycles > 1000) return fail(GRMHD_ERR_ARG, "cycles must be in 1..1000");
    if (!scratch) return fail(GRMHD_ERR_ARG, "scratch is NULL");
    if ((uintptr_t)scratch % kAlign) return fail(GRMHD_ERR_SCRATCH, "scratch must be 256-byte aligned");
    MgPlan plan;
    if (mg_plan(c->g, &plan) != 0) return grmhd_clean_scratch_bytes(&c->grid, &scratch_bytes);
    if (scratch_bytes < mg_scratch_bytes(plan))
        return fail(GRMHD_ERR_SCRATCH, "scratch smaller than grmhd_clean_scratch_bytes");
    cudaError_t e = mg_clean(c->g, plan, (double*)scratch, c->bf, c->glm, cycles, c->nsm, (cudaStream_t)stream,
                             &c->launches);
    if (e != cudaSuccess) return cuda_fail(e, "multigrid kernels");
    return GRMHD_OK;
}

long long grmhd_launch_count(const grmhd_ctx* c) { return c ? c->launches : 0; }

// the start blob: 8 FP64 primitive arrays, then per stage 3 + 3 FP32 history arrays
static size_t start_bytes(const grmhd_ctx* c)
{
    const size_t n = (size_t)c->g.ncell;
    return 8 * n * sizeof(double) + (size_t)c->tab.s * 6 * n * sizeof(float);
}

// copy the start arrays to (save) or from (load) the blob p, in blob order
static cudaError_t start_copy(grmhd_ctx* c, char* p, bool save, cudaStream_t st)
{
    const size_t n = (size_t)c->g.ncell;
    auto cp = [&](void* arr, size_t bytes) -> cudaError_t {
        cudaError_t e = save ? cudaMemcpyAsync(p, arr, bytes, cudaMemcpyDefault, st)
                             : cudaMemcpyAsync(arr, p, bytes, cudaMemcpyDefault, st);
        p += bytes;
        return e;
    };
    for (int v = 0; v < 8; v++) {
        const cudaError_t e = cp(c->prim[v], n * sizeof(double));
        if (e != cudaSuccess) return e;
    }
    for (int k = 0; k < c->tab.s; k++)
        for (int v = 0; v < 3; v++) {
            cudaError_t e = cp(c->hs[k][v], n * sizeof(float));
            if (e == cudaSuccess) e = cp(c->hd[k][v], n * sizeof(float));
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

grmhd_status grmhd_start_bytes(const grmhd_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(GRMHD_ERR_ARG, "grmhd_start_bytes: context or bytes is NULL");
    *bytes = start_bytes(c);
    return GRMHD_OK;
}

grmhd_status grmhd_save_start(grmhd_ctx* c, void* dst, size_t bytes, grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (!dst || (uintptr_t)dst % 8) return fail(GRMHD_ERR_ARG, "dst must be non-NULL and 8-byte aligned");
    if (bytes < start_bytes(c)) return fail(GRMHD_ERR_ARG, "dst is smaller than grmhd_start_bytes");
    if (!c->hist) return fail(GRMHD_ERR_STATE, "call grmhd_init_from_prims first");
    const cudaError_t e = start_copy(c, (char*)dst, true, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    return GRMHD_OK;
}

grmhd_status grmhd_load_start(grmhd_ctx* c, const void* src, size_t bytes, grmhd_stream_t stream)
{
    grmhd_status s = need_bound(c);
    if (s != GRMHD_OK) return s;
    if (!src || (uintptr_t)src % 8) return fail(GRMHD_ERR_ARG, "src must be non-NULL and 8-byte aligned");
    if (bytes != start_bytes(c)) return fail(GRMHD_ERR_ARG, "src is not a start blob of this grid and tableau");
    const cudaError_t e = start_copy(c, (char*)src, false, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    c->hist = true;
    return GRMHD_OK;
}

const char* grmhd_last_error(void) { return g_err; }

}  // extern "C"

// ---------------------------------------------------------------------------
// accessors for the batched executor (capi_internal.h)
// ---------------------------------------------------------------------------

const Dims& ctx_dims(const grmhd_ctx* c) { return c->g; }
bool ctx_metric(const grmhd_ctx* c) { return c->psi || c->alp; }
bool ctx_bound(const grmhd_ctx* c) { return c->bound; }
bool ctx_mixed(const grmhd_ctx* c) { return c->mixed; }
bool ctx_any_fixed(const grmhd_ctx* c) { return c->any_fixed; }
bool ctx_glm(const grmhd_ctx* c) { return c->glm; }
bool ctx_ideal(const grmhd_ctx* c) { return c->ideal; }
bool ctx_ppm(const grmhd_ctx* c) { return c->ppm; }
int ctx_stages(const grmhd_ctx* c) { return c->tab.s; }
int ctx_nsm(const grmhd_ctx* c) { return c->nsm; }

bool ctx_same_scheme(const grmhd_ctx* a, const grmhd_ctx* b)
{
    if (a->mixed != b->mixed || a->tab.s != b->tab.s) return false;
    const int n = a->tab.s * a->tab.s;
    for (int k = 0; k < n; k++)
        if (a->tab.At[k] != b->tab.At[k] || a->tab.A[k] != b->tab.A[k]) return false;
    for (int k = 0; k < a->tab.s; k++)
        if (a->tab.wt[k] != b->tab.wt[k] || a->tab.w[k] != b->tab.w[k]) return false;
    return true;
}

void ctx_stage_args(grmhd_ctx* c, int i, double dt, ImpArgs* ia, UpdateArgs* a)
{
    const int S = c->tab.s;
    double* const* qb = i == 0 ? c->q : c->base[i];
    double* const* fb = i == 0 ? c->bf : c->base[i] + 8;
    const double a_dt = c->tab.A[i * S + i] * dt;
    *ia = imp_args(c, cp8(qb), cp3(fb), a_dt, p8(c->prim), p3(c->R), p3(nullptr), f11(c));
    if (c->hist)
        for (int v = 0; v < 3; v++) {
            ia->hs[v] = c->hs[i][v];
            ia->hd[v] = c->hd[i][v];
        }
    memset(a, 0, sizeof *a);
    a->mode = UPD_STAGE;
    a->stage = i;
    a->s = S;
    a->dt = dt;
    for (int r = 0; r < S; r++) {
        for (int k = 0; k < S; k++) {
            a->At[r][k] = c->tab.At[r * S + k];
            a->A[r][k] = c->tab.A[r * S + k];
        }
        a->wt[r] = c->tab.wt[r];
        a->w[r] = c->tab.w[r];
        a->cL[r] = dt * c->tab.At[r * S + i];
        a->cR[r] = dt * c->tab.A[r * S + i];
    }
    a->cwL = dt * c->tab.wt[i];
    a->cwR = dt * c->tab.w[i];
    for (int v = 0; v < 3; v++) a->R[v] = c->R[v];
    for (int v = 0; v < 8; v++) a->qn[v] = c->q[v];
    for (int v = 0; v < 3; v++) a->qn[8 + v] = c->bf[v];
    for (int k = 1; k < S; k++)
        for (int v = 0; v < 11; v++) a->base[k][v] = c->base[k][v];
    for (int v = 0; v < 11; v++) a->acc[v] = c->acc[v];
}

float* ctx_p32(grmhd_ctx* c, int v) { return c->p32[v]; }
double* ctx_flux64(grmhd_ctx* c, int d, int v) { return d < c->grid.ndim ? c->F[d][v] : nullptr; }
double* ctx_emf64(grmhd_ctx* c, int k) { return c->Eh[k]; }
int ctx_fused_emf_dir(const grmhd_ctx* c, int k) { return fused_emf_dir(c, k); }

cudaError_t ctx_copy_fixed_faces(grmhd_ctx* c, cudaStream_t st)
{
    for (int k = 1; k < c->tab.s; k++)
        for (int v = 0; v < (c->glm ? 4 : 3); v++) {
            const double* src = v < 3 ? c->bf[v] : c->qphi;
            cudaError_t e = cudaMemcpyAsync(c->base[k][8 + v], src, sizeof(double) * (size_t)c->g.ncell,
                                            cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

grmhd_status batch_fail(grmhd_status s, const char* msg)
{
    grmhd::set_last_error(msg);
    return s;
}

// the Newton starting points (primitives and the FP32 start history) and the failure
// count, to host memory and back
cudaError_t ctx_save_guess(grmhd_ctx* c, std::vector<double>& host, cudaStream_t st)
{
    const size_t n = (size_t)c->g.ncell, nh = (size_t)c->tab.s * 6 * ((n + 1) / 2);
    host.resize(8 * n + 1 + nh);
    for (int v = 0; v < 8; v++) {
        cudaError_t e = cudaMemcpyAsync(host.data() + v * n, c->prim[v], n * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(host.data() + 8 * n, c->nfail, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    float* h = (float*)(host.data() + 8 * n + 1);
    for (int k = 0; k < c->tab.s; k++)
        for (int v = 0; v < 3; v++) {
            e = cudaMemcpyAsync(h, c->hs[k][v], n * sizeof(float), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h + n, c->hd[k][v], n * sizeof(float), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return e;
            h += 2 * n;
        }
    return cudaStreamSynchronize(st);
}

cudaError_t ctx_restore_guess(grmhd_ctx* c, const std::vector<double>& host, cudaStream_t st)
{
    const size_t n = (size_t)c->g.ncell;
    for (int v = 0; v < 8; v++) {
        cudaError_t e = cudaMemcpyAsync(c->prim[v], host.data() + v * n, n * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(c->nfail, host.data() + 8 * n, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const float* h = (const float*)(host.data() + 8 * n + 1);
    for (int k = 0; k < c->tab.s; k++)
        for (int v = 0; v < 3; v++) {
            e = cudaMemcpyAsync(c->hs[k][v], h, n * sizeof(float), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c->hd[k][v], h + n, n * sizeof(float), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
            h += 2 * n;
        }
    return cudaStreamSynchronize(st);
}
