// Batched instances behind the C ABI: n independent simulations stepped with
// one launch per step kernel over all of them (block offsets per instance in
// a device table), captured once per step parity in a CUDA graph, with the
// stream-collide tile shape picked by timing the candidates on the batch.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_handle.cuh"

using namespace lbm;

namespace {

constexpr int kMaxBatch = 4096;
constexpr size_t kAlign = 256;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Stream-collide tile shapes (threads x rows of one block, 128 threads),
// and with BF16 / FP16 storage a fourth candidate: the staged kernel
// (persistent blocks, 128 x 1 row tiles copied into shared memory ahead).
const dim3 kTiles[] = {dim3(128, 1), dim3(64, 2), dim3(32, 4)};
constexpr int kNumTiles = 3;
constexpr int kStagedTile = kNumTiles;
int candidates(int storage) { return storage == LBM_STORE_FP32 ? kNumTiles : kNumTiles + 1; }
// The block shape a candidate's block offsets and records are built for.
dim3 tile_shape(int t) { return kTiles[t == kStagedTile ? 0 : t]; }

// Stream-collide bucket table: at most 4 (n + 1) buckets.
int bucket_cap(int n) { return 4 * (n + 1); }

// Device tables: InstArgs [n], block offsets [phases][n + 1], stream-collide
// records [n] and buckets [4 (n + 1)], the staged kernel's work counter.
size_t table_bytes(int n)
{
    return round_up((size_t)n * sizeof(InstArgs), kAlign) +
           round_up((size_t)kBatchPhases * (n + 1) * sizeof(int), kAlign) +
           round_up((size_t)n * sizeof(ScInst), kAlign) + round_up((size_t)bucket_cap(n) * sizeof(int), kAlign) +
           kAlign;
}

} // namespace

struct lbm_batch {
    std::vector<lbm_handle *> hs;
    std::vector<int> poff; // per-instance parity offsets
    int n = 0, storage = 0, parity = 0, zone_max = 0;
    cudaStream_t stream = nullptr, cap = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    InstArgs *d_inst = nullptr;
    int *d_start = nullptr; // [kBatchPhases][n + 1]
    ScInst *d_sc = nullptr; // [n] stream-collide records
    int *d_bucket = nullptr; // [4 (n + 1)] stream-collide buckets
    unsigned *d_counter = nullptr; // [2] the staged kernel's work counter and done count
    int sc_shift = 0;
    int total[kBatchPhases] = {};
    int tile = 0, sc_resident = 1, links_ahead = 1;
    size_t links_smem = 0;
    cudaGraphExec_t gexec[4][2] = {}; // 2^l steps (l = 0..3) from each parity
    long long launches = 0;
    int sticky = LBM_OK;
};

namespace {

int fail_cuda(lbm_batch *b, cudaError_t e)
{
    if (e == cudaSuccess) return LBM_OK;
    if (b) b->sticky = LBM_ECUDA;
    return LBM_ECUDA;
}

#define BCK(b, call)                                      \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return fail_cuda(b, e_);   \
    } while (0)

// Block offsets of every phase for the current tile shape, uploaded to the
// device table (synchronously on the batch's stream).
int upload_starts(lbm_batch *b)
{
    std::vector<int> st((size_t)kBatchPhases * (b->n + 1), 0);
    for (int ph = 0; ph < kBatchPhases; ++ph) b->total[ph] = 0;
    for (int i = 0; i < b->n; ++i) {
        int blocks[kBatchPhases];
        batch_blocks(b->hs[i]->D, tile_shape(b->tile), blocks);
        for (int ph = 0; ph < kBatchPhases; ++ph) {
            st[(size_t)ph * (b->n + 1) + i] = b->total[ph];
            b->total[ph] += blocks[ph];
        }
    }
    for (int ph = 0; ph < kBatchPhases; ++ph) st[(size_t)ph * (b->n + 1) + b->n] = b->total[ph];
    // stream-collide: per-instance records (first block, tiles per row and
    // the exact reciprocal of the latter) and buckets of 2^shift blocks,
    // each holding the instance its first block belongs to
    const int V = b->storage == LBM_STORE_FP32 ? 1 : 2;
    const int tx = (int)tile_shape(b->tile).x;
    std::vector<ScInst> sc(b->n);
    for (int i = 0; i < b->n; ++i) {
        ScInst &e = sc[i];
        e.start = st[(size_t)kBStream * (b->n + 1) + i];
        e.gx = (b->hs[i]->D.pitch / V + tx - 1) / tx;
        int l = 0;
        while ((1ll << l) < e.gx) ++l;
        e.s = 31 + l;
        e.m = (1ull << e.s) / (unsigned long long)e.gx + 1ull;
        e.pad = 0;
    }
    const int tot = b->total[kBStream];
    int shift = 0;
    while ((tot >> shift) + 1 > bucket_cap(b->n)) ++shift;
    std::vector<int> bk((size_t)(tot >> shift) + 1);
    for (int k = 0, i = 0; k < (int)bk.size(); ++k) {
        const long long g = (long long)k << shift;
        while (i + 1 < b->n && sc[i + 1].start <= g) ++i;
        bk[k] = i;
    }
    b->sc_shift = shift;
    BCK(b, cudaMemcpyAsync(b->d_start, st.data(), st.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_sc, sc.data(), sc.size() * sizeof(ScInst), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_bucket, bk.data(), bk.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->sc_resident = stream_collide_batch_resident(b->storage, tile_shape(b->tile));
    return LBM_OK;
}

const int *starts(const lbm_batch *b, int ph) { return b->d_start + (size_t)ph * (b->n + 1); }

// Stream-collide of every instance with the current candidate.
cudaError_t launch_sc(const lbm_batch *b, int par, cudaStream_t st)
{
    if (b->tile == kStagedTile)
        return launch_stream_collide_staged_batch(b->d_inst, b->d_sc, b->d_bucket, b->sc_shift, b->n,
                                                  b->total[kBStream], b->storage, par, b->d_counter, st);
    return launch_stream_collide_batch(b->d_inst, b->d_sc, b->d_bucket, b->sc_shift, b->n, b->total[kBStream],
                                       b->storage, par, kTiles[b->tile], b->sc_resident, st);
}

// One step of every instance, in the order of lbm_step: links -> particles
// (and raster) -> flags -> stream-collide beside the general path.
int enqueue_batch_step(lbm_batch *b, int par, cudaStream_t st)
{
    const InstArgs *I = b->d_inst;
    const int n = b->n;
    BCK(b, launch_links_batch(I, starts(b, kBLinks), n, b->total[kBLinks], b->storage, par, b->links_ahead,
                              b->links_smem, st));
    BCK(b, launch_particles_batch(I, starts(b, kBParticles), n, b->total[kBParticles], par, st));
    BCK(b, launch_flags_batch(I, starts(b, kBFlags), n, b->total[kBFlags], par, st));
    BCK(b, cudaEventRecord(b->fork, st));
    BCK(b, cudaStreamWaitEvent(b->side, b->fork, 0));
    BCK(b, launch_boundary_batch(I, starts(b, kBBoundary), n, b->total[kBBoundary], b->storage, par, b->side));
    BCK(b, cudaEventRecord(b->join, b->side));
    BCK(b, launch_sc(b, par, st));
    BCK(b, cudaStreamWaitEvent(st, b->join, 0));
    return LBM_OK;
}

void drop_graphs(lbm_batch *b)
{
    for (int l = 0; l < 4; ++l)
        for (int p = 0; p < 2; ++p)
            if (b->gexec[l][p]) {
                cudaGraphExecDestroy(b->gexec[l][p]);
                b->gexec[l][p] = nullptr;
            }
}

// Graph of `steps` consecutive batch steps from parity par (as lbm_step's:
// an edge inside a graph costs less than a launch of the next graph).
int capture_batch(lbm_batch *b, int par, int steps, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    for (int k = 0; k < steps && !rc; ++k) rc = enqueue_batch_step(b, par ^ (k & 1), b->cap);
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    BCK(b, e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    BCK(b, e);
    return LBM_OK;
}

int check_handles(lbm_handle *const *hs, int32_t n)
{
    if (!hs || n < 1 || n > kMaxBatch) return LBM_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || hs[i]->sticky) return hs[i] ? hs[i]->sticky : LBM_EINVAL;
        if (hs[i]->D.storage != hs[0]->D.storage || hs[i]->D.direct) return LBM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return LBM_EINVAL;
    }
    return LBM_OK;
}

} // namespace

extern "C" {

int lbm_batch_footprint(lbm_handle *const *hs, int32_t n, size_t *bytes)
{
    if (!bytes) return LBM_EINVAL;
    int rc = check_handles(hs, n);
    if (rc) return rc;
    *bytes = table_bytes(n);
    return LBM_OK;
}

int lbm_batch_create(lbm_batch **out, lbm_handle *const *hs, int32_t n, void *d_workspace, size_t ws_bytes,
                     void *stream)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    int rc = check_handles(hs, n);
    if (rc) return rc;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) % kAlign)) return LBM_EINVAL;
    if (ws_bytes < table_bytes(n)) return LBM_ENOSPC;
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_EINVAL;
    b->hs.assign(hs, hs + n);
    b->poff.assign(n, 0);
    b->n = n;
    b->storage = hs[0]->D.storage;
    b->tile = b->storage == LBM_STORE_FP32 ? 0 : kStagedTile; // until lbm_batch_autotune picks
    b->parity = 0; // instance i runs at parity b->parity ^ poff[i]
    b->stream = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_workspace);
    b->d_inst = reinterpret_cast<InstArgs *>(ws);
    size_t at = round_up((size_t)n * sizeof(InstArgs), kAlign);
    b->d_start = reinterpret_cast<int *>(ws + at);
    at += round_up((size_t)kBatchPhases * (n + 1) * sizeof(int), kAlign);
    b->d_sc = reinterpret_cast<ScInst *>(ws + at);
    at += round_up((size_t)n * sizeof(ScInst), kAlign);
    b->d_bucket = reinterpret_cast<int *>(ws + at);
    at += round_up((size_t)bucket_cap(n) * sizeof(int), kAlign);
    b->d_counter = reinterpret_cast<unsigned *>(ws + at);
    auto fail = [&](int code) {
        lbm_batch_destroy(b);
        return code;
    };
    std::vector<InstArgs> inst(n);
    for (int i = 0; i < n; ++i) {
        lbm_handle *h = hs[i];
        // every handle's own work must be complete before the batch runs
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(LBM_ECUDA);
        inst[i].D = h->D;
        inst[i].A[0] = h->A[0];
        inst[i].A[1] = h->A[1];
        inst[i].own[0] = h->own[0];
        inst[i].own[1] = h->own[1];
        inst[i].poff = h->parity;
        inst[i].pad = 0;
        b->poff[i] = h->parity;
        b->zone_max = std::max(b->zone_max, h->D.zone_max);
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess)
        return fail(LBM_ECUDA);
    if (cudaMemcpyAsync(b->d_inst, inst.data(), n * sizeof(InstArgs), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(unsigned), b->stream) != cudaSuccess)
        return fail(LBM_ECUDA);
    if (prepare_links_batch(std::max(b->zone_max, 4), b->storage, &b->links_smem, &b->links_ahead) !=
        cudaSuccess)
        return fail(LBM_ECUDA);
    if ((rc = upload_starts(b))) return fail(rc);
    *out = b;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch *b, int32_t reps, int32_t *choice, double *best_ms)
{
    if (!b || reps < 1) return LBM_EINVAL;
    if (b->sticky) return b->sticky;
    // stream-collide alone reads A[parity] and writes only A[parity ^ 1],
    // which the next step overwrites: timing it changes no state
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_tile = b->tile;
    int rc = LBM_OK;
    for (int t = 0; t < candidates(b->storage) && !rc; ++t) {
        b->tile = t;
        if ((rc = upload_starts(b))) break;
        for (int w = 0; w < 2 && !rc; ++w)
            if (launch_sc(b, b->parity, b->stream) != cudaSuccess) rc = fail_cuda(b, cudaErrorLaunchFailure);
        if (rc || cudaEventRecord(e0, b->stream) != cudaSuccess) break;
        for (int r = 0; r < reps && !rc; ++r)
            if (launch_sc(b, b->parity, b->stream) != cudaSuccess) rc = fail_cuda(b, cudaErrorLaunchFailure);
        float ms = 0.f;
        if (rc || cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = rc ? rc : fail_cuda(b, cudaErrorUnknown);
            break;
        }
        if (ms < best) {
            best = ms;
            best_tile = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->tile = best_tile;
    drop_graphs(b);
    if ((rc = upload_starts(b))) return rc;
    if (choice) *choice = best_tile;
    if (best_ms) *best_ms = (double)best / reps;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int32_t nsteps)
{
    if (!b || nsteps < 0) return LBM_EINVAL;
    if (b->sticky) return b->sticky;
    for (int i = 0; i < b->n; ++i)
        if (b->hs[i]->parity != (b->parity ^ b->poff[i])) return LBM_EINVAL; // a handle was stepped on its own
    int per_step = 0;
    for (int ph = 0; ph < kBatchPhases; ++ph) per_step += ph != kBRaster && b->total[ph] > 0;
    for (int32_t k = 0; k < nsteps;) {
        // the largest graph (8, 4, 2 or 1 steps) that fits what is left
        int l = 3;
        while ((1 << l) > nsteps - k) --l;
        const int m = 1 << l;
        int rc;
        cudaGraphExec_t &g = b->gexec[l][b->parity];
        if (!g && (rc = capture_batch(b, b->parity, m, &g))) return rc;
        BCK(b, cudaGraphLaunch(g, b->stream));
        b->parity ^= m & 1;
        for (int i = 0; i < b->n; ++i) b->hs[i]->parity ^= m & 1;
        b->launches += (long long)m * per_step;
        k += m;
    }
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch *b, int32_t *which)
{
    if (!b) return LBM_EINVAL;
    if (which) *which = -1;
    BCK(b, cudaStreamSynchronize(b->stream));
    if (b->sticky) return b->sticky;
    // every handle reads its own device error word now (each failing one
    // holds its error, sticky), and the first failure is reported
    int first = LBM_OK;
    for (int i = 0; i < b->n; ++i) {
        const int rc = lbm_sync(b->hs[i]);
        if (rc && first == LBM_OK) {
            first = rc;
            if (which) *which = i;
        }
    }
    return first;
}

int64_t lbm_batch_launch_count(lbm_batch *b) { return b ? b->launches : 0; }

int lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return LBM_EINVAL;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->side) {
        cudaStreamSynchronize(b->side);
        cudaStreamDestroy(b->side);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    delete b;
    return LBM_OK;
}

} // extern "C"
