// Launch of the stage kernels with programmatic dependent launch (sm_90 and later).
//
// The kernels of one IMEX stage run back to back on one stream, each reading what the
// one before wrote.  Launched with the programmatic-stream-serialisation attribute, a
// kernel may be scheduled before its predecessor has completed and flushed.  Every
// stage kernel opens with grid_dep_sync() (griddepcontrol.wait): it waits until the
// preceding grid has completed and its memory is visible.  No kernel triggers its
// dependents explicitly, so each block triggers when it exits.  A kernel's blocks are
// therefore placed only once every block of its predecessor has finished its work, and
// what is hidden is the launch latency and the completion and flush of the grid before.
// An early trigger (griddepcontrol.launch_dependents at the top of each kernel) was
// slower: the next kernel's waiting blocks then sat on SMs beside running ones for the
// whole of a launch.  Since no kernel touches memory before its predecessor has
// finished, the results are bitwise those of plain launches.  Kernels launched without
// the attribute (every launch while launch_overlap is off) see the wait as a no-op.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace grmhd {

// set by the C API for the duration of a stage (one context per thread)
extern thread_local bool launch_overlap;

__device__ __forceinline__ void grid_dep_sync()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// k<<<grid, block, 0, st>>>(args...), with the programmatic attribute when
// launch_overlap is set.  k must open with grid_dep_sync().
template <typename... P, typename... A>
inline cudaError_t launch_k(void (*k)(P...), int grid, int block, cudaStream_t st, A&&... args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = launch_overlap ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Items (faces or edges) per thread of a march over `other` lines of n + 1 items, with
// 128-thread blocks of which bps are resident per SM: the K in 8..1 that minimises
// (waves of resident blocks) x (K + c0), c0 being a march's start-up in items (the
// cells reconstructed before the first item).  The kernels keep about two blocks per
// SM and are latency- rather than throughput-limited at that occupancy, so an SM given
// fewer blocks does not finish sooner: what counts is how many waves there are and how
// long each thread's march is.  Ties go to the larger K (fewer loads and slopes).
inline int march_len(int n, long long other, int nsm, int bps, double c0)
{
    int best = 8;
    double best_v = 0.0;
    for (int K = 8; K >= 1; K--) {
        const long long blocks = (((long long)(n + K) / K) * other + 127) / 128;
        const long long slots = (long long)nsm * (bps > 0 ? bps : 1);
        const double v = (double)((blocks + slots - 1) / slots) * (K + c0);
        if (K == 8 || v < best_v * (1.0 - 1e-9)) {
            best = K;
            best_v = v;
        }
    }
    return best;
}

}  // namespace grmhd
