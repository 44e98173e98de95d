// Launch interface between the C-ABI layer (capi.cu) and the kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "grmhd_device.cuh"

namespace grmhd {

enum { UPD_WRITE_L = 0, UPD_STAGE = 1 };

// stage primitives as the explicit kernels read them: FP64 (rho, u^1..3, p, E^1..3),
// or FP32 on the mixed-precision path with the densitised cell-centred q_B^1..3 added
template <typename T> struct PrimIn;
template <> struct PrimIn<double> { const double* p[8]; };
template <> struct PrimIn<float> { const float* p[11]; };
// face fluxes of the 8 cell-centred variables, stored as twice the HLL flux (the
// update kernel folds the 1/2 into its 1/dx): FP64, or FP32 on the mixed path
template <typename T> struct FluxOut { T* p[8]; };
struct F11 { float* p[11]; };

// arguments of the implicit solve of one problem and stage
struct ImpArgs {
    CP8 qb;                 // stage base q (8)
    CP3 bf;                 // stage face fields
    const double* psi;
    const double* alp;
    const double* eta;      // per-cell resistivity or NULL
    double eta_u;
    double a_dt;            // a_ii dt (<= 0: E held fixed)
    double ia_dt;           // 1 / (a_ii dt) (0 when a_dt <= 0)
    float ighf, xif;        // FP32 1/Gamma_hat and xi
    P8 prim;                // in: Newton start; out: stage primitives
    P3 R;                   // stiff rates (or NULL)
    P3 qE_out;              // solved q_E (or NULL)
    int kmax;
    double tol, rho_atm, p_atm;
    float tolf;             // tol in FP32 (for the double-word corrections)
    int dwacc;              // mixed precision (tol >= 1e-11): the double-word residual
                            // accepts the root (the ACC instantiations)
    int stiff;              // a_dt > 0 (else E is held fixed)
    int atm;                // rho_atm > 0 (an atmosphere is set)
    double d_atm;           // 10 rho_atm: cells with D below it are atmosphere
    double xi;              // mean-field dynamo parameter
    F11 p32;                // FP32 copy for the mixed path (or NULL)
    unsigned long long* nfail;
    float* hs[3];           // this stage's last Newton root u (orthonormal), or NULL ...
    float* hd[3];           // ... and its change from the one before: start at hs + hd
};

struct P3f { float* p[3]; };

template <typename T>
struct FluxArgs {
    PrimIn<T> prim;
    CP3 bf;
    const double* psi;
    const double* alp;
    FluxOut<T> F;           // twice the face fluxes (FP32 values in mixed precision)
    double* vbar[2];        // ideal-limit EMF: transverse transport velocities (or NULL)
    double* Eh[3];          // edge EMFs written by the flux kernel (flat 1-D / 2-D grids,
                            // see face_flux), NULL for those the EMF kernels compute
};

template <typename T>
struct EmfArgs {
    PrimIn<T> prim;
    CP3 bf;
    const double* psi;
    const double* alp;
    double* Eh;             // edge EMFs (FP64 also on the mixed path)
};

// Arguments of the update kernel.  Variables 0..7 are cell-centred (D, S_1..3, tau,
// E^1..3), 8..10 are the face fields.
struct UpdateArgs {
    int mode;               // UPD_WRITE_L: L -> L[]; UPD_STAGE: fold into base/acc/qn
    int stage, s;
    double dt;
    double At[4][4], A[4][4], wt[4], w[4];
    double cL[4], cR[4];    // dt At[k][stage], dt A[k][stage]: this stage's terms in base k
    double cwL, cwR;        // dt wt[stage], dt w[stage]: its terms in the final combination
    const double* F[3][8];  // twice the face fluxes per active direction (float arrays when f32)
    int f32;                // the fluxes are FP32 (the mixed-precision flux kernels)
    const double* Eh[3];    // edge EMFs
    const double* prim[8];  // stage primitives (padded)
    const float* p32[11];   // their FP32 copy with the cell q_B (mixed precision: the sources)
    const double* bf[3];    // stage face fields
    const double* psi;
    const double* alp;
    const double* R[3];     // stiff rates of this stage (E components)
    double* L[11];
    double* qn[11];         // bound state: read at stage 0, written by the last stage
    double* base[4][11];    // bases of later stages (index k >= 1)
    double* acc[11];        // running final combination
};

cudaError_t launch_implicit(const Dims& g, const ImpArgs& a, int nsm, cudaStream_t st);
// Newton start history at initialisation: hs = psi^2 u (the orthonormal velocity of the
// coordinate u1..u3), hd = 0, on every cell
cudaError_t launch_hist_init(const Dims& g, const double* u1, const double* u2, const double* u3, const double* psi,
                             P3f hs, P3f hd, int nsm, cudaStream_t st);
// mixed precision: the fluxes of every active direction (F[d]; fe[d][k]: the edge EMFs
// the d-flux writes on a flat 1-D / 2-D grid, or NULL) and the edge EMFs Eh[c] (NULL
// for those not computed here) in one launch of k_stencil32
cudaError_t launch_stencil32(const Dims& g, const PrimIn<float>& prim, CP3 bf, const double* psi, const double* alp,
                             const FluxOut<float>* F, double* const (*fe)[3], double* const* Eh, int nsm,
                             cudaStream_t st, bool ppm = false);
// the same for the FP64 path (resistive UCT; the ideal-limit EMF keeps its own launches)
cudaError_t launch_stencil64(const Dims& g, CP8 prim, CP3 bf, const double* psi, const double* alp, const P8* F,
                             double* const (*fe)[3], double* const* Eh, int nsm, cudaStream_t st, bool ppm = false);
cudaError_t launch_prim_to32(const Dims& g, CP8 prim, CP3 bf, F11 p32, int nsm, cudaStream_t st);
// ppm: PPM reconstruction instead of MC (FP64 only)
cudaError_t launch_flux(const Dims& g, int d, CP8 prim, CP3 bf, const double* psi, const double* alp, P8 F, int nsm,
                        cudaStream_t st, double* const* vbar = nullptr, bool ppm = false,
                        double* const* Eh = nullptr);
// Eh (flat metric only; ignored otherwise): the edge EMF arrays the flux kernel of
// direction d writes itself (fused_emf_dir), NULL entries for the others
// ideal-limit edge EMF (App. A): vb[d][k] are the transport velocities of the d-faces,
// component (d + 1 + k) % 3 (NULL for inactive directions)
cudaError_t launch_emf_ideal(const Dims& g, int c, CP8 prim, CP3 bf, const double* psi, const double* alp,
                             const double* const (*vb)[2], double* Eh, int nsm, cudaStream_t st);
cudaError_t launch_update(const Dims& g, const UpdateArgs& a, int nsm, cudaStream_t st);
cudaError_t launch_curlA(const Dims& g, CP3 A, P3 bf, int nsm, cudaStream_t st);
cudaError_t launch_prim2con(const Dims& g, CP8 prim, CP3 bf, const double* psi, P8 q, int nsm, cudaStream_t st);
cudaError_t launch_dt(const Dims& g, const double* psi, const double* alp, double* part, int nblk, double* out,
                      cudaStream_t st);
cudaError_t launch_diag(const Dims& g, CP3 bf, CP8 q, double dV, double* part, int nblk, double* out,
                        cudaStream_t st);

// ---------------------------------------------------------------------------
// GLM hyperbolic cleaning variant (Sec. 3.1): cell-centred q_B^1..3 and q_Phi are
// evolved with the 8 cell-centred variables; variables 8..10 are q_B^1..3 and 11 is
// q_Phi in the arrays below.  Kernels in glm.cu.
// ---------------------------------------------------------------------------

struct GlmFluxArgs {
    const double* prim[8];  // stage primitives (padded)
    const double* qB[3];    // stage cell-centred q_B
    const double* qphi;     // stage q_Phi
    const double* psi;
    const double* alp;
    double* F[12];          // twice the face fluxes of the 12 variables along the launch direction
};

struct GlmUpdateArgs {
    int mode;               // UPD_WRITE_L or UPD_STAGE (as UpdateArgs)
    int stage, s;
    double dt;
    double kappa;           // kappa_B, the damping of Phi
    double At[4][4], A[4][4], wt[4], w[4];
    double cL[4], cR[4], cwL, cwR;   // the dt products of UpdateArgs
    const double* F[3][12];  // twice the face fluxes
    const double* prim[8];
    const double* qB[3];
    const double* qphi;
    const double* psi;
    const double* alp;
    const double* R[3];
    double* L[12];
    double* qn[12];
    double* base[4][12];
    double* acc[12];
};

cudaError_t launch_implicit_cc(const Dims& g, const ImpArgs& a, int nsm, cudaStream_t st);
cudaError_t launch_glm_flux(const Dims& g, int d, const GlmFluxArgs& a, int nsm, cudaStream_t st, bool ppm = false);
cudaError_t launch_glm_update(const Dims& g, const GlmUpdateArgs& a, int nsm, cudaStream_t st);
cudaError_t launch_curlA_cc(const Dims& g, CP3 A, P3 qB, int nsm, cudaStream_t st);
cudaError_t launch_prim2con_cc(const Dims& g, CP8 prim, CP3 qB, const double* psi, const double* phi, double* qphi,
                               P8 q, int nsm, cudaStream_t st);
cudaError_t launch_diag_cc(const Dims& g, CP3 qB, CP8 q, double dV, double* part, int nblk, double* out,
                           cudaStream_t st);

// index-bounds violations counted by each translation unit's kernels in a checked
// build (GRMHD_CHECK_BOUNDS; 0 otherwise, ~0 if the counter could not be read)
unsigned long long oob_kernels(bool reset);
unsigned long long oob_glm(bool reset);
unsigned long long oob_elliptic(bool reset);
unsigned long long oob_batch(bool reset);
unsigned long long oob_noalloc(bool reset);

}  // namespace grmhd
