// Internal accessors of a context (capi.cu) used by the batched executor (batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/grmhd.h"
#include "kernels.h"

// NVTX range around a host call (visible to nsys / ncu range filters; a no-op when no
// tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

const grmhd::Dims& ctx_dims(const grmhd_ctx* c);
bool ctx_metric(const grmhd_ctx* c);
bool ctx_bound(const grmhd_ctx* c);
bool ctx_mixed(const grmhd_ctx* c);
bool ctx_any_fixed(const grmhd_ctx* c);
bool ctx_glm(const grmhd_ctx* c);
bool ctx_ideal(const grmhd_ctx* c);
bool ctx_ppm(const grmhd_ctx* c);
int ctx_stages(const grmhd_ctx* c);
int ctx_nsm(const grmhd_ctx* c);
bool ctx_same_scheme(const grmhd_ctx* a, const grmhd_ctx* b);
// implicit-solve and update arguments of stage i with time step dt (the same values
// grmhd_stage uses)
void ctx_stage_args(grmhd_ctx* c, int i, double dt, grmhd::ImpArgs* imp, grmhd::UpdateArgs* upd);
float* ctx_p32(grmhd_ctx* c, int v);
double* ctx_flux64(grmhd_ctx* c, int d, int v);
double* ctx_emf64(grmhd_ctx* c, int k);
// the flux direction whose kernel writes the edge EMF of direction k, or -1
int ctx_fused_emf_dir(const grmhd_ctx* c, int k);
// FIXED boundaries: copy the bound face fields into the later stages' face arrays
cudaError_t ctx_copy_fixed_faces(grmhd_ctx* c, cudaStream_t st);
grmhd_status batch_fail(grmhd_status s, const char* msg);
// save / restore the Newton starting point (stage primitives) and the failure count
cudaError_t ctx_save_guess(grmhd_ctx* c, std::vector<double>& host, cudaStream_t st);
cudaError_t ctx_restore_guess(grmhd_ctx* c, const std::vector<double>& host, cudaStream_t st);
