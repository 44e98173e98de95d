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
    FluxOut<double> F64[3];   // fluxes and edge EMFs: FP64 for both precisions
    double* Eh64[3];
    double* fe64[3][3];   // [D][C]: edge EMFs written by the D-flux kernel (flat 1-D / 2-D)
    UpdateArgs upd;
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

template <bool M>
__global__ void __launch_bounds__(256) kb_implicit(const ProbStage* __restrict__ P, int s, int stage,
                                                  const Chunk* __restrict__ ch, int nch)
{
    for (int i = blockIdx.x; i < nch; i += gridDim.x) {
        const Chunk k = ch[i];
        const ProbStage& ps = P[k.prob * s + stage];
        for (long long t = k.begin + threadIdx.x; t < k.end; t += blockDim.x) implicit_item<M>(ps.g, ps.imp, t);
    }
}

template <typename T> __device__ __forceinline__ const PrimIn<T>& prim_of(const ProbStage& ps);
template <> __device__ __forceinline__ const PrimIn<double>& prim_of<double>(const ProbStage& ps) { return ps.p64; }
template <> __device__ __forceinline__ const PrimIn<float>& prim_of<float>(const ProbStage& ps) { return ps.p32; }
// item t: kMarch consecutive D-faces (flux_march_item)
template <int D, bool M, typename T>
__global__ void __launch_bounds__(256) kb_flux(const ProbStage* __restrict__ P, int s, int stage,
                                              const Chunk* __restrict__ ch, int nch)
{
    for (int i = blockIdx.x; i < nch; i += gridDim.x) {
        const Chunk k = ch[i];
        const ProbStage& ps = P[k.prob * s + stage];
        for (long long t = k.begin + threadIdx.x; t < k.end; t += blockDim.x)
            flux_march_item<D, M, T>(ps.g, prim_of<T>(ps), ps.bfs, ps.psi, ps.alp, ps.F64[D], nullptr, ps.fe64[D], t);
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

template <bool M>
__global__ void __launch_bounds__(256) kb_update(const ProbStage* __restrict__ P, int s, int stage,
                                                const Chunk* __restrict__ ch, int nch)
{
    for (int i = blockIdx.x; i < nch; i += gridDim.x) {
        const Chunk k = ch[i];
        const ProbStage& ps = P[k.prob * s + stage];
        for (long long t = k.begin + threadIdx.x; t < k.end; t += blockDim.x) update_item<M>(ps.g, ps.upd, t);
    }
}

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
        for (int k = 0; k < 3; k++) ps.upd.Eh[k] = ps.Eh64[k];
        for (int v = 0; v < 8; v++) ps.upd.prim[v] = ps.imp.prim.p[v];
        for (int k = 0; k < 3; k++) ps.upd.bf[k] = ps.bfs.p[k];
        ps.upd.psi = ps.psi;
        ps.upd.alp = ps.alp;
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
        if (m) kb_implicit<true><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
        else kb_implicit<false><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
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
        if (m) kb_update<true><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
        else kb_update<false><<<gr, th, 0, st>>>(P, s, stage, ch, nch);
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
    *bytes = rup(sizeof(ProbStage) * (size_t)n * s) + rup(sizeof(Chunk) * chunk_capacity(ctxs, n));
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
