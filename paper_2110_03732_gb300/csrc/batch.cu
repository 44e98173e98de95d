// Batched execution of many independent resistive-MHD problems (uneven grids,
// different resistivities, flat or fixed-metric) on one GPU: each stage issues one
// launch per kernel kind for all problems together.  A launch walks a work list of
// (problem, item range) chunks and runs, for each item, the same per-item body as the
// single-problem kernels (items.cuh).  A problem's results do not depend on which
// other problems share its batch or how the work is chunked: it gets bit for bit what
// it gets in a batch of its own (no cross-problem reduction or atomic on the result
// path).  Problems keep their own contexts (state, scratch, metric, eta, Newton
// parameters); the batch adds a descriptor table and the work lists, both in
// caller-provided device memory.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/grmhd.h"
#include "capi_internal.h"
#include "items.cuh"

using namespace grmhd;

namespace {

// one problem at one stage: everything its kernels read
struct ProbStage {
    Dims g;
    ImpArgs imp;
    PrimIn<double> p64;
    PrimIn<float> p32;
    CP3 bfs;
    const double* psi;
    const double* alp;
    FluxOut<double> F64[3];   // fluxes: FP64, or FP32 in the same arrays (mixed precision)
    double* Eh64[3];
    double* fe64[3][3];   // [D][C]: edge EMFs written by the D-flux kernel (flat 1-D / 2-D)
    UpdateArgs upd;
    int fixed;            // FIXED boundaries: the later bases take the face fields each step
};

// grid-wide barrier of the persistent launch (device memory in the batch scratch):
// arrivals, generation, and the error flag a wait that ran out sets
struct BarrierState {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

// faces (edges) per item of the batched flux (EMF) kernels: each item marches K of them
constexpr int kMarch = 4;

struct Chunk {
    int prob;
    int pad;
    long long begin, end;
};

// work-list kinds: implicit, flux D, emf C, update; each split flat / metric
enum { WL_IMP = 0, WL_FLUX = 1, WL_EMF = 4, WL_UPD = 7, WL_KINDS = 8 };

constexpr int kAlign = 256;
size_t rup(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// autotuner candidates: threads per block, items per chunk
struct Cfg {
    int threads, items;
};
const Cfg kCands[] = {{128, 128}, {128, 512}, {256, 256}, {256, 1024}, {64, 256}};
constexpr int kNCand = sizeof(kCands) / sizeof(kCands[0]);
constexpr int kMinItems = 128;   // smallest chunk of any candidate (scratch sizing)

// ---------------------------------------------------------------------------
// batched kernels
// ---------------------------------------------------------------------------

template <bool M, bool ACC>
__global__ void __launch_bounds__(256) kb_implicit(const ProbStage* __restrict__ P, int s, int stage,
                                                  const Chunk* __restrict__ ch, int nch)
{
    for (int i = blockIdx.x; i < nch; i += gridDim.x) {
        const Chunk k = ch[i];
        const ProbStage& ps = P[k.prob * s + stage];
        for (long long t = k.begin + threadIdx.x; t < k.end; t += blockDim.x)
            implicit_item<M, false, ACC>(ps.g, ps.imp, t);
    }
}

template <typename T> __device__ __forceinline__ const PrimIn<T>& prim_of(const ProbStage& ps);
template <> __device__ __forceinline__ const PrimIn<double>& prim_of<double>(const ProbStage& ps) { return ps.p64; }
template <> __device__ __forceinline__ const PrimIn<float>& prim_of<float>(const ProbStage& ps) { return ps.p32; }
// the D-fluxes in the stencil precision: the FP32 fluxes of the mixed path occupy the
// first half of the same arrays
template <typename T> __device__ __forceinline__ FluxOut<T> flux_of(const ProbStage& ps, int d);
template <> __device__ __forceinline__ FluxOut<double> flux_of<double>(const ProbStage& ps, int d) { return ps.F64[d]; }
template <> __device__ __forceinline__ FluxOut<float> flux_of<float>(const ProbStage& ps, int d)
{
    FluxOut<float> f;
#pragma unroll
    for (int v = 0; v < 8; v++) f.p[v] = reinterpret_cast<float*>(ps.F64[d].p[v]);
    return f;
}
// item t: kMarch consecutive D-faces (flux_march_item)
template <int D, bool M, typename T>
__global__ void __launch_bounds__(256) kb_flux(const ProbStage* __restrict__ P, int s, int stage,
                                              const Chunk* __restrict__ ch, int nch)
{
    for (int i = blockIdx.x; i < nch; i += gridDim.x) {
        const Chunk k = ch[i];
        const ProbStage& ps = P[k.prob * s + stage];
        for (long long t = k.begin + threadIdx.x; t < k.end; t += blockDim.x)
            flux_march_item<D, M, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp, flux_of<T>(ps, D), nullptr,
                                     ps.fe64[D], t);
    }
}

// item t: kMarch consecutive C-edges along C + 2 when both transverse directions are
// active (emf_march_item), else one edge (emf_item)
template <int C, bool M, typename T>
__global__ void __launch_bounds__(256) kb_emf(const ProbStage* __restrict__ P, int s, int stage,
                                             const Chunk* __restrict__ ch, int nch)
{
    for (int i = blockIdx.x; i < nch; i += gridDim.x) {
        const Chunk k = ch[i];
        const ProbStage& ps = P[k.prob * s + stage];
        const bool march = ps.g.act[(C + 1) % 3] && ps.g.act[(C + 2) % 3];
        for (long long t = k.begin + threadIdx.x; t < k.end; t += blockDim.x) {
            if (march) emf_march_item<C, M, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp, ps.Eh64[C], t);
            else emf_item<C, M, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp, ps.Eh64[C], t);
        }
    }
}

template <bool M, bool F32>
__global__ void __launch_bounds__(256) kb_update(const ProbStage* __restrict__ P, int s, int stage,
                                                const Chunk* __restrict__ ch, int nch)
{
    for (int i = blockIdx.x; i < nch; i += gridDim.x) {
        const Chunk k = ch[i];
        const ProbStage& ps = P[k.prob * s + stage];
        for (long long t = k.begin + threadIdx.x; t < k.end; t += blockDim.x) update_item<M, F32>(ps.g, ps.upd, t);
    }
}

// ---------------------------------------------------------------------------
// persistent launch: every phase of nsteps steps in one cooperative launch
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier (all blocks are co-resident: cooperative launch).  Each block's
// writes are fenced before it arrives; the last arrival resets the count and advances
// the generation; the others wait for the generation to change, for at most limit_ns
// of the global timer.  A wait that runs out sets the batch's error flag; every block
// that sees the flag (waiting, or at its next barrier) returns false and leaves the
// kernel, so the launch ends within about one limit and the host reads the flag.
__device__ bool grid_barrier(BarrierState* bs, unsigned nblocks, unsigned long long limit_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &bs->gen;
        volatile int* err = &bs->err;
        int good = *err == 0;
        if (good) {
            const unsigned g = *gen;
            __threadfence();
            if (atomicAdd(&bs->count, 1u) == nblocks - 1) {
                atomicExch(&bs->count, 0u);
                __threadfence();
                atomicAdd(&bs->gen, 1u);
            } else {
                const unsigned long long t0 = global_ns();
                while (*gen == g) {
                    if (*err) {
                        good = 0;
                        break;
                    }
                    if (global_ns() - t0 > limit_ns) {
                        atomicExch(&bs->err, 1);
                        good = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
            if (*err) good = 0;
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

struct PersistLists {
    const Chunk* ch;
    int off[WL_KINDS][2], cnt[WL_KINDS][2];
};

// the items of one work-list kind and metric flag, chunks spread over the blocks
#define PERSIST_ITEMS(KIND, MM, BODY)                                                   \
    {                                                                                   \
        const Chunk* ch_ = L.ch + L.off[KIND][MM];                                      \
        const int n_ = L.cnt[KIND][MM];                                                 \
        for (int i_ = blockIdx.x; i_ < n_; i_ += gridDim.x) {                           \
            const Chunk k_ = ch_[i_];                                                   \
            const ProbStage& ps = P[k_.prob * s + stage];                               \
            for (long long t = k_.begin + threadIdx.x; t < k_.end; t += blockDim.x) {   \
                BODY;                                                                   \
            }                                                                           \
        }                                                                               \
    }

template <int C, bool M, typename T>
__device__ __forceinline__ void emf_any_item(const ProbStage& ps, long long t)
{
    if (ps.g.act[(C + 1) % 3] && ps.g.act[(C + 2) % 3])
        emf_march_item<C, M, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp, ps.Eh64[C], t);
    else
        emf_item<C, M, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp, ps.Eh64[C], t);
}

// nsteps IMEX steps of every problem: per stage the implicit solves, then the face
// fluxes and edge EMFs (which read the same stage primitives and write separate
// arrays), then the update, with a grid barrier after each phase; FIXED-boundary
// problems first copy their face fields into the later-stage bases, as
// grmhd_batch_step does.  The per-item bodies are those of the per-kind kernels.
//
// Registers: the fused kernel takes the largest need of its phases (255 unbounded).
// The mixed-precision instantiation is bounded to four 128-thread blocks per SM: on
// the 256-box batch that ran 38.4 ms per step against 50.7 ms at two blocks (spills of
// ~1.7 KB cost less than the lost occupancy); the FP64 one stays at two (four would
// spill 4.6 KB).
template <typename T>
__global__ void __launch_bounds__(128, (sizeof(T) == 4 ? 4 : 2)) kb_persistent(const ProbStage* __restrict__ P, int n, int s, PersistLists L,
                                                     BarrierState* bs, int nsteps, unsigned long long limit_ns,
                                                     int any_fixed)
{
    const unsigned nb = gridDim.x;
    for (int step = 0; step < nsteps; step++) {
        if (any_fixed) {
            for (int p = 0; p < n; p++) {
                const ProbStage& ps = P[p * s];
                if (!ps.fixed) continue;
                const long long nc = ps.g.ncell;
                for (int k = 1; k < s; k++)
                    for (int v = 0; v < 3; v++) {
                        const double* __restrict__ src = ps.upd.qn[8 + v];
                        double* __restrict__ dst = ps.upd.base[k][8 + v];
                        for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc;
                             t += (long long)gridDim.x * blockDim.x)
                            dst[t] = src[t];
                    }
            }
            if (!grid_barrier(bs, nb, limit_ns)) return;
        }
        for (int stage = 0; stage < s; stage++) {
            PERSIST_ITEMS(WL_IMP, 0, (implicit_item<false, false, sizeof(T) == 4>(ps.g, ps.imp, t)))
            PERSIST_ITEMS(WL_IMP, 1, (implicit_item<true, false, sizeof(T) == 4>(ps.g, ps.imp, t)))
            if (!grid_barrier(bs, nb, limit_ns)) return;
            PERSIST_ITEMS(WL_FLUX + 0, 0, (flux_march_item<0, false, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp,
                                                                       flux_of<T>(ps, 0), nullptr, ps.fe64[0], t)))
            PERSIST_ITEMS(WL_FLUX + 0, 1, (flux_march_item<0, true, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp,
                                                                      flux_of<T>(ps, 0), nullptr, ps.fe64[0], t)))
            PERSIST_ITEMS(WL_FLUX + 1, 0, (flux_march_item<1, false, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp,
                                                                       flux_of<T>(ps, 1), nullptr, ps.fe64[1], t)))
            PERSIST_ITEMS(WL_FLUX + 1, 1, (flux_march_item<1, true, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp,
                                                                      flux_of<T>(ps, 1), nullptr, ps.fe64[1], t)))
            PERSIST_ITEMS(WL_FLUX + 2, 0, (flux_march_item<2, false, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp,
                                                                       flux_of<T>(ps, 2), nullptr, ps.fe64[2], t)))
            PERSIST_ITEMS(WL_FLUX + 2, 1, (flux_march_item<2, true, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp,
                                                                      flux_of<T>(ps, 2), nullptr, ps.fe64[2], t)))
            PERSIST_ITEMS(WL_EMF + 0, 0, (emf_any_item<0, false, T>(ps, t)))
            PERSIST_ITEMS(WL_EMF + 0, 1, (emf_any_item<0, true, T>(ps, t)))
            PERSIST_ITEMS(WL_EMF + 1, 0, (emf_any_item<1, false, T>(ps, t)))
            PERSIST_ITEMS(WL_EMF + 1, 1, (emf_any_item<1, true, T>(ps, t)))
            PERSIST_ITEMS(WL_EMF + 2, 0, (emf_any_item<2, false, T>(ps, t)))
            PERSIST_ITEMS(WL_EMF + 2, 1, (emf_any_item<2, true, T>(ps, t)))
            if (!grid_barrier(bs, nb, limit_ns)) return;
            PERSIST_ITEMS(WL_UPD, 0, (update_item<false, sizeof(T) == 4>(ps.g, ps.upd, t)))
            PERSIST_ITEMS(WL_UPD, 1, (update_item<true, sizeof(T) == 4>(ps.g, ps.upd, t)))
            if (step + 1 < nsteps || stage + 1 < s)
                if (!grid_barrier(bs, nb, limit_ns)) return;
        }
    }
}
#undef PERSIST_ITEMS

// items of one problem for a work-list kind (0 = not run)
long long items_of(const grmhd_ctx* cx, int kind)
{
    const Dims& g = ctx_dims(cx);
    if (kind == WL_IMP) return (long long)g.n[0] * g.n[1] * g.n[2];
    if (kind >= WL_FLUX && kind < WL_FLUX + 3) {
        const int d = kind - WL_FLUX;
        if (!g.act[d]) return 0;
        long long other = 1;
        for (int e = 0; e < 3; e++)
            if (e != d) other *= g.n[e];
        return (long long)((g.n[d] + kMarch) / kMarch) * other;
    }
    if (kind >= WL_EMF && kind < WL_EMF + 3) {
        const int c = kind - WL_EMF, a = (c + 1) % 3, bd = (c + 2) % 3;
        if (!(g.act[a] || g.act[bd]) || ctx_fused_emf_dir(cx, c) >= 0) return 0;
        if (g.act[a] && g.act[bd]) return (long long)((g.n[bd] + kMarch) / kMarch) * g.n[c] * (g.n[a] + 1);
        long long w = 1;
        for (int d = 0; d < 3; d++) w *= (d == c) ? g.n[d] : (g.act[d] ? g.n[d] + 1 : 1);
        return w;
    }
    long long w = 1;
    for (int d = 0; d < 3; d++) w *= g.act[d] ? g.n[d] + 1 : 1;
    return w;
}

}  // namespace

struct grmhd_batch_s {
    int n, s;
    bool mixed;
    std::vector<grmhd_ctx*> ctx;
    std::vector<double> dt;             // per problem, last uploaded
    std::vector<ProbStage> desc;        // host copy, n * s
    ProbStage* d_desc;                  // device table
    Chunk* d_chunks;                    // device chunk lists
    size_t chunk_cap;                   // capacity (chunks) of d_chunks
    // per work-list kind and metric flag: chunk offset / count, and launch shape
    int off[WL_KINDS][2], cnt[WL_KINDS][2];
    Cfg cfg[WL_KINDS];
    int nsm;
    std::vector<int> fixed_probs;       // problems with FIXED boundaries
    BarrierState* d_bar;                // persistent launch: grid barrier (device)
    double wait_limit_s;                // persistent launch: limit of each barrier wait
    int persist_blocks;                 // persistent launch: co-resident blocks (0: not yet known)
};

namespace {

grmhd_status build_lists(grmhd_batch* b, cudaStream_t st)
{
    std::vector<Chunk> all;
    for (int kind = 0; kind < WL_KINDS; kind++)
        for (int m = 0; m < 2; m++) {
            b->off[kind][m] = (int)all.size();
            for (int p = 0; p < b->n; p++) {
                const grmhd_ctx* c = b->ctx[p];
                if ((ctx_metric(c) ? 1 : 0) != m) continue;
                const long long w = items_of(c, kind);
                for (long long a = 0; a < w; a += b->cfg[kind].items) {
                    Chunk k;
                    k.prob = p;
                    k.pad = 0;
                    k.begin = a;
                    k.end = std::min(w, a + (long long)b->cfg[kind].items);
                    all.push_back(k);
                }
            }
            b->cnt[kind][m] = (int)all.size() - b->off[kind][m];
        }
    if (all.size() > b->chunk_cap) return batch_fail(GRMHD_ERR_SCRATCH, "batch work lists exceed the scratch");
    cudaError_t e = cudaMemcpyAsync(b->d_chunks, all.data(), all.size() * sizeof(Chunk), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return batch_fail(GRMHD_ERR_CUDA, "batch work-list upload failed");
    return GRMHD_OK;
}

void fill_desc(grmhd_batch* b, int p, double dt)
{
    grmhd_ctx* c = b->ctx[p];
    for (int i = 0; i < b->s; i++) {
        ProbStage& ps = b->desc[(size_t)p * b->s + i];
        memset(&ps, 0, sizeof ps);
        ps.g = ctx_dims(c);
        for (int d = 0; d < 3; d++) set_march(ps.g, d, kMarch);   // every batched march is kMarch long
        ctx_stage_args(c, i, dt, &ps.imp, &ps.upd);
        for (int v = 0; v < 8; v++) ps.p64.p[v] = ps.imp.prim.p[v];
        for (int v = 0; v < 11; v++) ps.p32.p[v] = ctx_p32(c, v);
        ps.bfs = ps.imp.bf;
        ps.psi = ps.imp.psi;
        ps.alp = ps.imp.alp;
        for (int d = 0; d < 3; d++) {
            for (int v = 0; v < 8; v++) ps.F64[d].p[v] = ctx_flux64(c, d, v);
            ps.Eh64[d] = ctx_emf64(c, d);
        }
        for (int k = 0; k < 3; k++) {
            const int d = ctx_fused_emf_dir(c, k);
            if (d < 0) continue;
            ps.fe64[d][k] = ctx_emf64(c, k);
        }
        for (int d = 0; d < 3; d++)
            for (int v = 0; v < 8; v++)
                ps.upd.F[d][v] = !ps.g.act[d] ? nullptr : ps.F64[d].p[v];
        ps.upd.f32 = ctx_mixed(c) ? 1 : 0;
        for (int k = 0; k < 3; k++) ps.upd.Eh[k] = ps.Eh64[k];
        for (int v = 0; v < 8; v++) ps.upd.prim[v] = ps.imp.prim.p[v];
        for (int v = 0; v < 11; v++) ps.upd.p32[v] = ps.p32.p[v];
        for (int k = 0; k < 3; k++) ps.upd.bf[k] = ps.bfs.p[k];
        ps.upd.psi = ps.psi;
        ps.upd.alp = ps.alp;
        ps.fixed = ctx_any_fixed(c) ? 1 : 0;
    }
}

int grid_of(const grmhd_batch* b, int kind, int m)
{
    const int nch = b->cnt[kind][m];
    const int cap = b->nsm * (2048 / b->cfg[kind].threads);
    return std::max(1, std::min(nch, cap));
}

// launches of one stage for the kinds selected in `mask` (bit per work-list kind)
cudaError_t launch_stage(grmhd_batch* b, int stage, cudaStream_t st, unsigned mask = 0xffu)
{
    const ProbStage* P = b->d_desc;
    const int s = b->s;
    for (int m = 0; m < 2; m++) {
        const int kind = WL_IMP;
        if (!(mask >> kind & 1u) || !b->cnt[kind][m]) continue;
        const Chunk* ch = b->d_chunks + b->off[kind][m];
        const int nch = b->cnt[kind][m], th = b->cfg[kind].threads, gr = grid_of(b, kind, m);
        if (b->mixed) {
            if (m) kb_implicit<true, true><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
            else kb_implicit<false, true><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
        } else {
            if (m) kb_implicit<true, false><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
            else kb_implicit<false, false><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
        }
    }
    for (int d = 0; d < 3; d++)
        for (int m = 0; m < 2; m++) {
            const int kind = WL_FLUX + d;
            if (!(mask >> kind & 1u) || !b->cnt[kind][m]) continue;
            const Chunk* ch = b->d_chunks + b->off[kind][m];
            const int nch = b->cnt[kind][m], th = b->cfg[kind].threads, gr = grid_of(b, kind, m);
#define KB_FLUX(DD, MM)                                                                 \
    if (b->mixed) kb_flux<DD, MM, float><<<gr, th, 0, st>>>(P, s, stage, ch, nch); \
    else kb_flux<DD, MM, double><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
            if (d == 0) { if (m) { KB_FLUX(0, true) } else { KB_FLUX(0, false) } }
            else if (d == 1) { if (m) { KB_FLUX(1, true) } else { KB_FLUX(1, false) } }
            else { if (m) { KB_FLUX(2, true) } else { KB_FLUX(2, false) } }
#undef KB_FLUX
        }
    for (int c = 0; c < 3; c++)
        for (int m = 0; m < 2; m++) {
            const int kind = WL_EMF + c;
            if (!(mask >> kind & 1u) || !b->cnt[kind][m]) continue;
            const Chunk* ch = b->d_chunks + b->off[kind][m];
            const int nch = b->cnt[kind][m], th = b->cfg[kind].threads, gr = grid_of(b, kind, m);
#define KB_EMF(CC, MM)                                                                 \
    if (b->mixed) kb_emf<CC, MM, float><<<gr, th, 0, st>>>(P, s, stage, ch, nch); \
    else kb_emf<CC, MM, double><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
            if (c == 0) { if (m) { KB_EMF(0, true) } else { KB_EMF(0, false) } }
            else if (c == 1) { if (m) { KB_EMF(1, true) } else { KB_EMF(1, false) } }
            else { if (m) { KB_EMF(2, true) } else { KB_EMF(2, false) } }
#undef KB_EMF
        }
    for (int m = 0; m < 2; m++) {
        const int kind = WL_UPD;
        if (!(mask >> kind & 1u) || !b->cnt[kind][m]) continue;
        const Chunk* ch = b->d_chunks + b->off[kind][m];
        const int nch = b->cnt[kind][m], th = b->cfg[kind].threads, gr = grid_of(b, kind, m);
        if (b->mixed) {
            if (m) kb_update<true, true><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
            else kb_update<false, true><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
        } else {
            if (m) kb_update<true, false><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
            else kb_update<false, false><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
        }
    }
    return cudaGetLastError();
}

size_t chunk_capacity(grmhd_ctx* const* ctxs, int n)
{
    size_t cap = 0;
    for (int kind = 0; kind < WL_KINDS; kind++)
        for (int p = 0; p < n; p++) {
            const long long w = items_of(ctxs[p], kind);
            cap += (size_t)((w + kMinItems - 1) / kMinItems);
        }
    return cap;
}

}  // namespace

extern "C" {

grmhd_status grmhd_batch_scratch_bytes(grmhd_ctx* const* ctxs, int n, size_t* bytes)
{
    if (!ctxs || n < 1 || !bytes) return batch_fail(GRMHD_ERR_ARG, "grmhd_batch_scratch_bytes: bad arguments");
    int s = 0;
    for (int p = 0; p < n; p++) {
        if (!ctxs[p] || !ctx_bound(ctxs[p])) return batch_fail(GRMHD_ERR_STATE, "every context must be bound");
        if (ctx_glm(ctxs[p]))
            return batch_fail(GRMHD_ERR_ARG, "batched execution supports constrained transport (GRMHD_DIVB_CT) only");
        if (ctx_ideal(ctxs[p]))
            return batch_fail(GRMHD_ERR_ARG, "batched execution takes the resistive edge EMF only");
        if (ctx_ppm(ctxs[p]))
            return batch_fail(GRMHD_ERR_ARG, "batched execution takes the MC reconstruction only");
        s = ctx_stages(ctxs[p]);
    }
    *bytes = rup(sizeof(ProbStage) * (size_t)n * s) + rup(sizeof(Chunk) * chunk_capacity(ctxs, n)) +
             rup(sizeof(BarrierState));
    return GRMHD_OK;
}

grmhd_status grmhd_batch_create(grmhd_ctx* const* ctxs, int n, void* scratch, size_t scratch_bytes,
                                grmhd_batch** out)
{
    if (!ctxs || n < 1 || !scratch || !out) return batch_fail(GRMHD_ERR_ARG, "grmhd_batch_create: bad arguments");
    size_t need = 0;
    grmhd_status s = grmhd_batch_scratch_bytes(ctxs, n, &need);
    if (s != GRMHD_OK) return s;
    if (scratch_bytes < need) return batch_fail(GRMHD_ERR_SCRATCH, "batch scratch smaller than grmhd_batch_scratch_bytes");
    if ((uintptr_t)scratch % kAlign) return batch_fail(GRMHD_ERR_SCRATCH, "batch scratch must be 256-byte aligned");
    for (int p = 1; p < n; p++) {
        if (!ctx_same_scheme(ctxs[0], ctxs[p]))
            return batch_fail(GRMHD_ERR_ARG, "batched problems must share the tableau and the precision");
    }
    grmhd_batch* b = new (std::nothrow) grmhd_batch_s();
    if (!b) return batch_fail(GRMHD_ERR_ARG, "out of host memory");
    b->n = n;
    b->s = ctx_stages(ctxs[0]);
    b->mixed = ctx_mixed(ctxs[0]);
    b->ctx.assign(ctxs, ctxs + n);
    b->dt.assign(n, 0.0);
    b->desc.resize((size_t)n * b->s);
    b->d_desc = (ProbStage*)scratch;
    b->d_chunks = (Chunk*)((char*)scratch + rup(sizeof(ProbStage) * (size_t)n * b->s));
    b->chunk_cap = chunk_capacity(ctxs, n);
    b->d_bar = (BarrierState*)((char*)b->d_chunks + rup(sizeof(Chunk) * b->chunk_cap));
    b->wait_limit_s = 1.0;
    b->persist_blocks = 0;
    b->nsm = ctx_nsm(ctxs[0]);
    for (int k = 0; k < WL_KINDS; k++) b->cfg[k] = kCands[1];
    for (int p = 0; p < n; p++) {
        fill_desc(b, p, 0.0);
        if (ctx_any_fixed(ctxs[p])) b->fixed_probs.push_back(p);
    }
    s = build_lists(b, 0);
    if (s != GRMHD_OK) {
        delete b;
        return s;
    }
    *out = b;
    return GRMHD_OK;
}

grmhd_status grmhd_batch_set_dt(grmhd_batch* b, const double* dt, grmhd_stream_t stream)
{
    if (!b || !dt) return batch_fail(GRMHD_ERR_ARG, "grmhd_batch_set_dt: bad arguments");
    bool dirty = false;
    for (int p = 0; p < b->n; p++) {
        if (!(dt[p] > 0.0)) return batch_fail(GRMHD_ERR_ARG, "every dt must be positive");
        if (dt[p] != b->dt[p]) {
            b->dt[p] = dt[p];
            fill_desc(b, p, dt[p]);
            dirty = true;
        }
    }
    if (dirty) {
        cudaError_t e = cudaMemcpyAsync(b->d_desc, b->desc.data(), b->desc.size() * sizeof(ProbStage),
                                        cudaMemcpyHostToDevice, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) return batch_fail(GRMHD_ERR_CUDA, "batch descriptor upload failed");
    }
    return GRMHD_OK;
}

grmhd_status grmhd_batch_step(grmhd_batch* b, grmhd_stream_t stream)
{
    NvtxRange nv("grmhd_batch_step");
    if (!b) return batch_fail(GRMHD_ERR_ARG, "batch is NULL");
    for (int p = 0; p < b->n; p++)
        if (!(b->dt[p] > 0.0)) return batch_fail(GRMHD_ERR_STATE, "call grmhd_batch_set_dt before stepping");
    cudaStream_t st = (cudaStream_t)stream;
    for (int p : b->fixed_probs) {
        cudaError_t e = ctx_copy_fixed_faces(b->ctx[p], st);
        if (e != cudaSuccess) return batch_fail(GRMHD_ERR_CUDA, "fixed-boundary face copy failed");
    }
    for (int i = 0; i < b->s; i++) {
        cudaError_t e = launch_stage(b, i, st);
        if (e != cudaSuccess) return batch_fail(GRMHD_ERR_CUDA, "batched stage launch failed");
    }
    return GRMHD_OK;
}

grmhd_status grmhd_batch_autotune(grmhd_batch* b, int reps, grmhd_stream_t stream)
{
    if (!b) return batch_fail(GRMHD_ERR_ARG, "batch is NULL");
    for (int p = 0; p < b->n; p++)
        if (!(b->dt[p] > 0.0)) return batch_fail(GRMHD_ERR_STATE, "call grmhd_batch_set_dt before tuning");
    if (reps < 1) reps = 3;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return batch_fail(GRMHD_ERR_CUDA, "cudaEventCreate failed");
    // stage 0 reads the bound state and writes only scratch; the one piece of
    // scratch that carries over between steps -- the stage primitives, which are the
    // next Newton solve's starting point -- and the failure count are saved to the
    // host and restored afterwards, so tuning changes no later result.  The implicit
    // kernel runs first once so that every later kernel reads this stage's
    // primitives.
    std::vector<std::vector<double>> saved(b->n);
    for (int p = 0; p < b->n; p++)
        if (ctx_save_guess(b->ctx[p], saved[p], st) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return batch_fail(GRMHD_ERR_CUDA, "saving the Newton starting point failed");
        }
    grmhd_status res = GRMHD_OK;
    for (int kind = 0; kind < WL_KINDS && res == GRMHD_OK; kind++) {
        if (!b->cnt[kind][0] && !b->cnt[kind][1]) continue;
        float best = 1e30f;
        int bi = 1;
        for (int ci = 0; ci < kNCand; ci++) {
            b->cfg[kind] = kCands[ci];
            if ((res = build_lists(b, st)) != GRMHD_OK) break;
            if (launch_stage(b, 0, st, 1u << WL_IMP) != cudaSuccess) { res = batch_fail(GRMHD_ERR_CUDA, "tune"); break; }
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps; r++) launch_stage(b, 0, st, 1u << kind);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) { res = batch_fail(GRMHD_ERR_CUDA, "tune sync"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bi = ci; }
        }
        b->cfg[kind] = kCands[bi];
    }
    if (res == GRMHD_OK) res = build_lists(b, st);
    for (int p = 0; p < b->n; p++)
        if (ctx_restore_guess(b->ctx[p], saved[p], st) != cudaSuccess && res == GRMHD_OK)
            res = batch_fail(GRMHD_ERR_CUDA, "restoring the Newton starting point failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return res;
}

grmhd_status grmhd_batch_set_wait_limit(grmhd_batch* b, double seconds)
{
    if (!b || !(seconds >= 0.0) || !(seconds <= 60.0))
        return batch_fail(GRMHD_ERR_ARG, "grmhd_batch_set_wait_limit: a limit in [0, 60] seconds");
    b->wait_limit_s = seconds;
    return GRMHD_OK;
}

grmhd_status grmhd_batch_persistent_status(grmhd_batch* b, grmhd_stream_t stream)
{
    if (!b) return batch_fail(GRMHD_ERR_ARG, "batch is NULL");
    BarrierState h;
    cudaError_t e = cudaMemcpyAsync(&h, b->d_bar, sizeof h, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return batch_fail(GRMHD_ERR_CUDA, "reading the persistent launch's status failed");
    if (h.err) return batch_fail(GRMHD_ERR_TIMEOUT, "a grid barrier wait of the persistent launch ran out of time");
    return GRMHD_OK;
}

grmhd_status grmhd_batch_step_persistent(grmhd_batch* b, int nsteps, int synchronize, grmhd_stream_t stream)
{
    NvtxRange nv("grmhd_batch_step_persistent");
    if (!b || nsteps < 1) return batch_fail(GRMHD_ERR_ARG, "grmhd_batch_step_persistent: bad arguments");
    for (int p = 0; p < b->n; p++)
        if (!(b->dt[p] > 0.0)) return batch_fail(GRMHD_ERR_STATE, "call grmhd_batch_set_dt before stepping");
    cudaStream_t st = (cudaStream_t)stream;
    const bool mixed = b->mixed;
    const void* fn = mixed ? (const void*)kb_persistent<float> : (const void*)kb_persistent<double>;
    if (b->persist_blocks < 1) {
        int dev = 0, coop = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (e == cudaSuccess && coop)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 128, 0);
        if (e != cudaSuccess || !coop || per_sm < 1)
            return batch_fail(GRMHD_ERR_CUDA, "the device cannot run the persistent (cooperative) launch");
        b->persist_blocks = per_sm * b->nsm;
    }
    // the barrier starts at zero; a memset node, so the call can be graph-captured
    cudaError_t e = cudaMemsetAsync(b->d_bar, 0, sizeof(BarrierState), st);
    if (e != cudaSuccess) return batch_fail(GRMHD_ERR_CUDA, "barrier reset failed");
    PersistLists L;
    L.ch = b->d_chunks;
    int total = 0;
    for (int k = 0; k < WL_KINDS; k++)
        for (int m = 0; m < 2; m++) {
            L.off[k][m] = b->off[k][m];
            L.cnt[k][m] = b->cnt[k][m];
            total += b->cnt[k][m];
        }
    const ProbStage* P = b->d_desc;
    int n = b->n, s = b->s, any_fixed = b->fixed_probs.empty() ? 0 : 1;
    BarrierState* bar = b->d_bar;
    unsigned long long limit = (unsigned long long)(b->wait_limit_s * 1e9);
    // no more blocks than co-resident ones (the barrier needs them all), nor than chunks
    const int blocks = std::max(1, std::min(b->persist_blocks, total));
    void* args[] = {(void*)&P, (void*)&n, (void*)&s, (void*)&L, (void*)&bar, (void*)&nsteps, (void*)&limit,
                    (void*)&any_fixed};
    e = cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(128), args, 0, st);
    if (e != cudaSuccess) return batch_fail(GRMHD_ERR_CUDA, "persistent launch failed");
    return synchronize ? grmhd_batch_persistent_status(b, stream) : GRMHD_OK;
}

grmhd_status grmhd_batch_config(const grmhd_batch* b, int* threads, int* items)
{
    if (!b) return batch_fail(GRMHD_ERR_ARG, "batch is NULL");
    for (int k = 0; k < WL_KINDS; k++) {
        if (threads) threads[k] = b->cfg[k].threads;
        if (items) items[k] = b->cfg[k].items;
    }
    return GRMHD_OK;
}

grmhd_status grmhd_batch_destroy(grmhd_batch* b)
{
    delete b;
    return GRMHD_OK;
}

}  // extern "C"

namespace grmhd {
GRMHD_OOB_READER(oob_batch)
}  // namespace grmhd
