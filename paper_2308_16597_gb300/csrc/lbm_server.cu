// Request loop behind the C ABI: simulations of different sizes admitted by
// device-memory footprint into a caller-owned pool, advanced together in one
// batch (continuous batching: the batch is rebuilt whenever requests join or
// leave), and retired to host memory when their step budget is spent.
#include <algorithm>
#include <deque>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "lbm_handle.cuh"

namespace {

constexpr size_t kPoolAlign = 256;
// per instance: its arguments, block offsets, stream-collide record and
// four buckets (the 64 KB beyond covers the tables' alignment)
static_assert(sizeof(lbm::InstArgs) + lbm::kBatchPhases * sizeof(int) + sizeof(lbm::ScInst) + 4 * sizeof(int) <=
                  1024,
              "the table region reserves 1 KB per instance");

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit sub-allocator over [0, size) of the pool, with coalescing of
// neighbouring free ranges.  Offsets and sizes are multiples of 256 bytes.
class Pool {
  public:
    explicit Pool(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round_up(std::max<size_t>(bytes, 1), kPoolAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, next = it->first + bytes;
            free_.erase(it);
            if (rest) free_[next] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(std::max<size_t>(bytes, 1), kPoolAlign);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const
    {
        size_t m = 0;
        for (const auto &f : free_) m = std::max(m, f.second);
        return m;
    }

  private:
    std::map<size_t, size_t> free_; // offset -> size
};

enum ReqState { kQueued = 0, kActive = 1, kDone = 2, kFailed = 3 };

struct Request {
    int64_t id = 0;
    lbm_domain d{};
    lbm_params prm{};
    std::vector<lbm_particle> parts;
    int64_t steps = 0, done = 0;
    size_t bytes = 0, off = 0;
    lbm_handle *h = nullptr;
    int state = kQueued, err = LBM_OK;
    std::vector<float> fields; // 4 x ny x nx after retirement
    std::vector<lbm_particle> out;
};

} // namespace

struct lbm_server {
    char *pool_base = nullptr;
    size_t pool_bytes = 0;
    Pool *pool = nullptr;
    int max_active = 1;
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int64_t next_id = 1;
    std::unordered_map<int64_t, Request *> reqs;
    std::deque<Request *> queue;
    std::vector<Request *> active;
    lbm_batch *batch = nullptr;
    size_t table_off = 0, table_bytes = 0;
};

namespace {

void drop_batch(lbm_server *s)
{
    if (s->batch) {
        lbm_batch_destroy(s->batch);
        s->batch = nullptr;
    }
}

// Fields and particles to host memory, then the request's device memory back
// to the pool.
void retire(lbm_server *s, Request *r, int err)
{
    if (!err) {
        const size_t nn = (size_t)r->d.nx * r->d.ny;
        r->fields.resize(4 * nn);
        r->out.resize(r->parts.size());
        err = lbm_get_fields(r->h, r->fields.data(), r->fields.data() + nn, r->fields.data() + 2 * nn,
                             r->fields.data() + 3 * nn, 0);
        if (!err) err = lbm_get_particles(r->h, r->out.data(), (int32_t)r->out.size());
    }
    lbm_destroy(r->h);
    r->h = nullptr;
    s->pool->release(r->off, r->bytes);
    r->state = err ? kFailed : kDone;
    r->err = err;
    if (err) {
        r->fields.clear();
        r->out.clear();
    }
}

} // namespace

extern "C" {

int lbm_server_create(lbm_server **out, void *d_pool, size_t pool_bytes, int32_t max_active, void *stream)
{
    if (!out || !d_pool || (reinterpret_cast<uintptr_t>(d_pool) % kPoolAlign) || pool_bytes < kPoolAlign ||
        max_active < 1 || max_active > 4096)
        return LBM_EINVAL;
    lbm_server *s = new (std::nothrow) lbm_server();
    if (!s) return LBM_EINVAL;
    s->pool_base = static_cast<char *>(d_pool);
    s->pool_bytes = pool_bytes / kPoolAlign * kPoolAlign;
    s->pool = new (std::nothrow) Pool(s->pool_bytes);
    // the batch tables (about 0.5 KB per instance) take a fixed region at the
    // start of the pool, so that a batch can always be built
    s->table_bytes = round_up((size_t)max_active * 1024 + 65536, kPoolAlign);
    if (s->pool && (s->table_bytes >= s->pool_bytes || !s->pool->alloc(s->table_bytes, &s->table_off))) {
        lbm_server_destroy(s);
        return LBM_ENOSPC;
    }
    s->max_active = max_active;
    s->stream = static_cast<cudaStream_t>(stream);
    if (!s->pool || cudaEventCreate(&s->e0) != cudaSuccess || cudaEventCreate(&s->e1) != cudaSuccess) {
        lbm_server_destroy(s);
        return LBM_ECUDA;
    }
    *out = s;
    return LBM_OK;
}

int lbm_server_submit(lbm_server *s, const lbm_domain *d, const lbm_particle *p, int32_t n, const lbm_params *prm,
                      int64_t steps, int64_t *id)
{
    if (!s || !d || !prm || !id || steps < 1 || n < 0 || (n > 0 && !p)) return LBM_EINVAL;
    if (prm->flags & LBM_FLAG_DIRECT_LINKS) return LBM_EINVAL; // batches use the index array
    size_t bytes = 0;
    int rc = lbm_query_footprint(d, p, n, prm, &bytes);
    if (rc) return rc;
    // a request larger than the whole pool could never be admitted
    if (round_up(bytes, kPoolAlign) > s->pool_bytes - s->table_bytes) return LBM_ENOSPC;
    Request *r = new (std::nothrow) Request();
    if (!r) return LBM_EINVAL;
    r->id = s->next_id++;
    r->d = *d;
    r->prm = *prm;
    r->parts.assign(p, p + n);
    r->steps = steps;
    r->bytes = bytes;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *id = r->id;
    return LBM_OK;
}

int lbm_server_tick(lbm_server *s, int32_t max_steps, lbm_server_stats *st)
{
    if (!s || max_steps < 1) return LBM_EINVAL;
    lbm_server_stats S{};
    bool changed = false;
    // admission: head of the queue first, while memory and slots allow
    while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
        Request *r = s->queue.front();
        size_t off = 0;
        if (!s->pool->alloc(r->bytes, &off)) break;
        r->off = off;
        s->queue.pop_front();
        const int rc = lbm_init(&r->h, &r->d, r->parts.data(), (int32_t)r->parts.size(), &r->prm,
                                s->pool_base + off, r->bytes, s->stream);
        if (rc) {
            s->pool->release(off, r->bytes);
            r->h = nullptr;
            r->state = kFailed;
            r->err = rc;
            continue;
        }
        r->state = kActive;
        s->active.push_back(r);
        changed = true;
        ++S.admitted;
    }
    if (!s->active.empty()) {
        if (changed || !s->batch) {
            drop_batch(s);
            std::vector<lbm_handle *> hs;
            for (Request *r : s->active) hs.push_back(r->h);
            int rc = lbm_batch_create(&s->batch, hs.data(), (int32_t)hs.size(), s->pool_base + s->table_off,
                                      s->table_bytes, s->stream);
            if (rc) return rc;
        }
        int64_t steps = max_steps;
        for (Request *r : s->active) steps = std::min<int64_t>(steps, r->steps - r->done);
        if (cudaEventRecord(s->e0, s->stream) != cudaSuccess) return LBM_ECUDA;
        int rc = lbm_batch_step(s->batch, (int32_t)steps);
        if (rc) return rc;
        if (cudaEventRecord(s->e1, s->stream) != cudaSuccess) return LBM_ECUDA;
        int32_t which = -1;
        rc = lbm_batch_sync(s->batch, &which);
        // an error of the batch itself (not of one instance): no step can be
        // counted as done
        if (rc && which < 0) return rc;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->e0, s->e1);
        S.steps = (int32_t)steps;
        S.ms = ms;
        for (Request *r : s->active) {
            r->done += steps;
            S.updates += (int64_t)r->d.nx * r->d.ny * steps;
        }
        // retire finished (and failed) requests; the batch, which refers to
        // their handles, is rebuilt on the next tick
        std::vector<Request *> keep;
        for (int i = 0; i < (int)s->active.size(); ++i) {
            Request *r = s->active[i];
            const int err = (rc && i == which) ? rc : r->h->sticky;
            if (err || r->done >= r->steps) {
                drop_batch(s);
                retire(s, r, err);
                ++S.retired;
            } else {
                keep.push_back(r);
            }
        }
        s->active.swap(keep);
    }
    S.active = (int32_t)s->active.size();
    S.queued = (int32_t)s->queue.size();
    if (st) *st = S;
    return LBM_OK;
}

int lbm_server_status(lbm_server *s, int64_t id, int32_t *err)
{
    if (!s) return LBM_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return -1;
    if (err) *err = it->second->err;
    return it->second->state;
}

int lbm_server_result(lbm_server *s, int64_t id, float *drho, float *ux, float *uy, float *T, lbm_particle *p,
                      int32_t n)
{
    if (!s) return LBM_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return LBM_EINVAL;
    Request *r = it->second;
    if (r->state == kFailed) return r->err;
    if (r->state != kDone || n != (int32_t)r->out.size() || !drho || !ux || !uy || !T || (n > 0 && !p))
        return LBM_EINVAL;
    const size_t nn = (size_t)r->d.nx * r->d.ny;
    float *dst[4] = {drho, ux, uy, T};
    for (int f = 0; f < 4; ++f) std::copy(r->fields.begin() + f * nn, r->fields.begin() + (f + 1) * nn, dst[f]);
    std::copy(r->out.begin(), r->out.end(), p);
    s->reqs.erase(it);
    delete r;
    return LBM_OK;
}

int lbm_server_destroy(lbm_server *s)
{
    if (!s) return LBM_EINVAL;
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_batch(s);
    for (auto &kv : s->reqs) {
        if (kv.second->h) lbm_destroy(kv.second->h);
        delete kv.second;
    }
    if (s->e0) cudaEventDestroy(s->e0);
    if (s->e1) cudaEventDestroy(s->e1);
    delete s->pool;
    delete s;
    return LBM_OK;
}

} // extern "C"
