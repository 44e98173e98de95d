// Multigrid elliptic cleaning (elliptic.cu): level plan and entry point.
#pragma once

#include <cuda_runtime.h>

#include "grmhd_device.cuh"

namespace grmhd {

constexpr int kMgMaxLevels = 16;
constexpr long long kMgMaxCoarse = 4096;   // cells of the coarsest level (one thread block)
constexpr long long kMgBlockCells = 1024;  // levels this small run inside one thread block
                                           // (one SM does 2 FP64 FMA per cycle: larger
                                           // levels are faster as grid-wide launches)
constexpr size_t kMgTailSmem = 48 * 1024;  // the block keeps its levels in shared memory
                                           // when they fit in this many bytes
constexpr int kMgParts = 1024;             // partial sums of the mean

// one cell-centred level (no ghosts, x fastest)
struct MgLevel {
    int n[3];
    double ih2[3];        // 1/h^2 per active direction, 0 otherwise
    double dfull, idiag;  // diagonal of the full (2 ndim + 1)-point stencil (summed in
                          // the device's order) and its reciprocal
    long long cells;
    long long offset;     // of this level's arrays in the phi / rhs blocks
    double* phi;
    double* rhs;
};

struct MgPlan {
    int nlev;
    long long total;      // cells over all levels
    MgLevel lev[kMgMaxLevels];
};

// levels for grid g: 0 on success, -1 too many levels, -2 coarsest level above
// kMgMaxCoarse cells, -3 a grid of 2^31 cells or more
int mg_plan(const Dims& g, MgPlan* plan);
size_t mg_scratch_bytes(const MgPlan& plan);
// clean the three q_B arrays bq in place (staggered faces, or cell-centred if cc) with
// `cycles` V-cycles; scratch of mg_scratch_bytes(plan) bytes (8-byte aligned)
cudaError_t mg_clean(const Dims& g, const MgPlan& plan, double* scratch, double* const* bq, bool cc, int cycles,
                     int nsm, cudaStream_t st, long long* launches);

}  // namespace grmhd
