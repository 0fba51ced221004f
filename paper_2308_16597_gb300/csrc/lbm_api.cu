// Host side of the C ABI declared in include/lbm.h: workspace layout,
// argument validation, initialisation, the per-step launch sequence (direct
// or replayed from a captured CUDA graph), read-back and checkpoint hooks.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "lbm_handle.cuh"

using namespace lbm;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kDistTailPad = 256; // bytes after each distribution buffer
constexpr size_t kStageBytes = size_t(4) << 20;
constexpr int kGraphLevels = 4; // replayed graphs hold 1, 2, 4 or 8 steps
constexpr int kOrderSteps = 256; // steps between recomputations of the link order

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }


bool finite(double v) { return std::isfinite(v); }

int validate(const lbm_domain *d, const lbm_particle *p, int32_t n, const lbm_params *prm)
{
    if (!d || !prm || n < 0 || (n > 0 && !p)) return LBM_EINVAL;
    if (d->nx < 4 || d->ny < 4 || d->reserved != 0) return LBM_EINVAL;
    if ((long long)d->nx * d->ny > (1ll << 31) - 1) return LBM_EINVAL;
    if (!(prm->nu > 0) || !(prm->alpha > 0) || !finite(prm->nu) || !finite(prm->alpha)) return LBM_EINVAL;
    if (prm->storage != LBM_STORE_FP32 && prm->storage != LBM_STORE_BF16 && prm->storage != LBM_STORE_FP16)
        return LBM_EINVAL;
    const double rates[] = {prm->s_e, prm->s_eps, prm->s_q, prm->q_e, prm->q_nu};
    for (double r : rates)
        if (!finite(r) || r >= 2.0) return LBM_EINVAL;
    const double vals[] = {prm->g, prm->beta, prm->T0, prm->rho_f, prm->T_init, prm->eps_w,
                           prm->s_rep, prm->body_fx, prm->body_fy};
    for (double v : vals)
        if (!finite(v)) return LBM_EINVAL;
    if (n > 0 && !(prm->eps_w > 0)) return LBM_EINVAL;
    for (int i = 0; i < 4; ++i)
        if (!finite(d->T_wall[i])) return LBM_EINVAL;
    const bool px = d->bc & LBM_BC_PERIODIC_X, py = d->bc & LBM_BC_PERIODIC_Y;
    double rmax = 0.0;
    for (int a = 0; a < n; ++a) {
        const lbm_particle &P = p[a];
        const double v[] = {P.x, P.y, P.ux, P.uy, P.theta, P.omega, P.r, P.rho, P.T, P.b};
        for (double x : v)
            if (!finite(x)) return LBM_EINVAL;
        if (P.r < 1.0 || P.rho <= 0.0 || P.b < 0.0) return LBM_EINVAL;
        // an ellipse: 1 <= b < r, and theta within the exact range of the
        // angle reduction by pi/2
        if (is_ellipse(P.r, P.b) && (P.b < 1.0 || P.b > P.r || std::fabs(P.theta) > 1.6e6)) return LBM_EINVAL;
        // the link kernel holds a particle's zone in shared memory
        if (!link_zone_supported(zone_size(P.r), prm->storage)) return LBM_EINVAL;
        // a disk stays inside the cavity; next to a periodic seam it keeps two
        // nodes of clearance so that no link or stencil wraps around
        const double mx = px ? 2.0 : -0.5, my = py ? 2.0 : -0.5;
        if (P.x - P.r < mx || P.x + P.r > d->nx - 1 - (px ? 2.0 : -0.5)) return LBM_EINVAL;
        if (P.y - P.r < my || P.y + P.r > d->ny - 1 - (py ? 2.0 : -0.5)) return LBM_EINVAL;
        rmax = std::max(rmax, P.r);
    }
    // overlapping disks (cell hash with cell size 2 rmax)
    if (n > 1) {
        const double cs = 2.0 * rmax;
        std::unordered_map<long long, std::vector<int>> cells;
        auto key = [](long long cx, long long cy) { return (cx << 32) ^ (cy & 0xffffffffll); };
        for (int a = 0; a < n; ++a) {
            long long cx = (long long)std::floor(p[a].x / cs), cy = (long long)std::floor(p[a].y / cs);
            for (long long gx = cx - 1; gx <= cx + 1; ++gx)
                for (long long gy = cy - 1; gy <= cy + 1; ++gy) {
                    auto it = cells.find(key(gx, gy));
                    if (it == cells.end()) continue;
                    for (int b : it->second) {
                        double dx = p[a].x - p[b].x, dy = p[a].y - p[b].y;
                        if (std::sqrt(dx * dx + dy * dy) < p[a].r + p[b].r) return LBM_EINVAL;
                    }
                }
            cells[key(cx, cy)].push_back(a);
        }
    }
    return LBM_OK;
}

void layout(const lbm_domain *d, const lbm_particle *p, int32_t n, int storage, double s_rep, Layout &L)
{
    L.pitch = (int)round_up((size_t)d->nx, 32);
    L.ps = (long long)round_up((size_t)L.pitch * d->ny, 64);
    L.nslots = 0;
    for (int a = 0; a < n; ++a) L.nslots += (size_t)slot_capacity(p[a].r);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = round_up(off + std::max<size_t>(bytes, 1), kAlign);
        return o;
    };
    const size_t nn = (size_t)d->nx * d->ny;
    // each distribution buffer has a tail pad: the stream-collide fast path
    // reads up to 33 elements past the last row of the last plane
    for (int b = 0; b < 2; ++b) L.A[b] = take((size_t)kPop * L.ps * storage_bytes(storage) + kDistTailPad);
    for (int b = 0; b < 2; ++b) L.own[b] = take(nn * sizeof(int));
    L.flags = take((size_t)L.pitch * d->ny);
    L.slot_node = take(L.nslots * sizeof(int));
    L.slot_q = take(L.nslots * sizeof(float));
    L.slot_base = take((size_t)(n + 1) * sizeof(int));
    L.cur = take((size_t)kPartFields * n * sizeof(double));
    L.nxt = take((size_t)kPartFields * n * sizeof(double));
    L.prev = take((size_t)2 * n * sizeof(double));
    L.force = take((size_t)3 * n * sizeof(double));
    L.pos4 = take((size_t)n * sizeof(float4));
    L.prc = take((size_t)n * sizeof(float2));
    L.lsum = take((size_t)n * sizeof(LinkSums));
    for (int b = 0; b < 3; ++b) L.geo[b] = take((size_t)n * sizeof(GeomRec));
    L.pconst = take((size_t)n * sizeof(double4));
    L.lorder = take((size_t)n * sizeof(int));
    L.status = take(sizeof(Status));
    L.pack = take((size_t)n * sizeof(lbm_particle));
    L.stage_rows = (int)std::max<size_t>(1, std::min<size_t>(d->ny, kStageBytes / (16 * (size_t)d->nx)));
    L.stage = take((size_t)4 * L.stage_rows * d->nx * sizeof(float));
    // newborn nodes of one step: a disk moving less than one node per step
    // uncovers fewer than 2N nodes; room for 4N per particle
    int zmax = 0;
    for (int a = 0; a < n; ++a) zmax = std::max(zmax, zone_size(p[a].r));
    L.newborn_cap = std::max(1024, 4 * n * zmax);
    L.newborn = take((size_t)L.newborn_cap * sizeof(int));
    // each zone row's run of inside nodes, at the current and the next positions
    for (int b = 0; b < 2; ++b) L.runs[b] = take((size_t)n * std::max(zmax, 1) * sizeof(int2));
    L.near = take(((size_t)d->ny * near_tiles_per_row(storage, L.pitch) + 31) / 32 * sizeof(unsigned));
    L.dsum = take((size_t)n * sizeof(DirectSums));
    // cell grid of the pair screening: side 2 r_max + s + 2 (every pair in
    // reach lies in neighbouring cells), grown to hold at most 4 Mi cells
    double rmax = 1.0;
    for (int a = 0; a < n; ++a) rmax = std::max(rmax, p[a].r);
    double side = 2.0 * rmax + std::max(s_rep, 0.0) + 2.0;
    side = std::max(side, std::sqrt((double)d->nx * d->ny / (double)(1 << 22)));
    L.cell_side = side;
    L.cell_gx = n > 0 ? std::max(1, (int)std::ceil(d->nx / side)) : 1;
    L.cell_gy = n > 0 ? std::max(1, (int)std::ceil(d->ny / side)) : 1;
    const size_t ncell = (size_t)L.cell_gx * L.cell_gy;
    for (int b = 0; b < 2; ++b) L.cells[b] = take((ncell + 1 + ncell * kCellCap) * sizeof(int));
    L.total = off;
}

PartSoA soa_at(char *base, size_t off, int n)
{
    double *b = reinterpret_cast<double *>(base + off);
    return PartSoA{b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n, b + 6 * n, b + 7 * n, b + 8 * n, b + 9 * n};
}

const char *kKernelNames[kNumKernelKinds] = {"link_gather_bb_force", "particle_update",
                                             "owner_raster",
                                             "node_flags",           "stream_collide",
                                             "boundary_refill",
                                             "init_collide",         "fields",
                                             "near_mask",            "stream_collide_near"};

} // namespace


namespace {

int cuda_fail(lbm_handle *h, cudaError_t e)
{
    if (e == cudaSuccess) return LBM_OK;
    if (h) h->sticky = LBM_ECUDA;
    return LBM_ECUDA;
}

#define CK(h, call)                                      \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(h, e_); \
    } while (0)

int fold_events(lbm_handle *h)
{
    for (size_t i = 0; i < h->ev_used; ++i) {
        float ms = 0.f;
        CK(h, cudaEventSynchronize(h->ev[i].b));
        CK(h, cudaEventElapsedTime(&ms, h->ev[i].a, h->ev[i].b));
        h->acc_ms[h->ev[i].kind] += ms;
        h->acc_n[h->ev[i].kind] += 1;
    }
    h->ev_used = 0;
    return LBM_OK;
}

template <typename F>
int timed(lbm_handle *h, int kind, cudaStream_t st, F &&launch)
{
    const bool t = h->timing && st == h->stream;
    if (t) {
        if (h->ev_used >= 32768) {
            int rc = fold_events(h);
            if (rc) return rc;
        }
        if (h->ev_used == h->ev.size()) {
            lbm_handle::Ev e{};
            CK(h, cudaEventCreate(&e.a));
            CK(h, cudaEventCreate(&e.b));
            h->ev.push_back(e);
        }
        h->ev[h->ev_used].kind = kind;
        CK(h, cudaEventRecord(h->ev[h->ev_used].a, st));
    }
    CK(h, launch());
    if (t) {
        CK(h, cudaEventRecord(h->ev[h->ev_used].b, st));
        ++h->ev_used;
    }
    ++h->launches;
    return LBM_OK;
}

// One time step, in the order
//   gather + bounce-back + force (particle state at n, owner map at n; also
//   clears the other owner map over the zones at n - 1)
//   -> particle update (n -> n+1) with the raster of the new positions
//   -> flags at n+1
//   -> fused stream + collide of A_n into A_{n+1}, beside the general path
//      (frame and newborn nodes, refill).
int enqueue_step(lbm_handle *h, int par, cudaStream_t st)
{
    const Dev &D = h->D;
    void *Ain = h->A[par], *Aout = h->A[par ^ 1];
    int *oc = h->own[par], *on = h->own[par ^ 1];
    int rc;
    const bool serial = h->timing && st == h->stream; // per-kernel timing: one kernel at a time
    const bool overlap = h->np > 0 && (h->prm.flags & LBM_FLAG_OVERLAP);
    if (overlap) {
        // the lattice away from every particle needs nothing of this step's
        // particle work: stream-collide those tiles beside it
        if (serial) {
            if ((rc = timed(h, kKNearMask, st, [&] { return launch_near_mask(D, st); }))) return rc;
            if ((rc = timed(h, kKStreamCollide, st, [&] { return launch_stream_collide(D, Ain, Aout, kSCFar, st); })))
                return rc;
        } else {
            CK(h, cudaEventRecord(h->fork0, st));
            CK(h, cudaStreamWaitEvent(h->far, h->fork0, 0));
            if ((rc = timed(h, kKNearMask, h->far, [&] { return launch_near_mask(D, h->far); }))) return rc;
            if ((rc = timed(h, kKStreamCollide, h->far,
                            [&] { return launch_stream_collide(D, Ain, Aout, kSCFar, h->far); })))
                return rc;
            CK(h, cudaEventRecord(h->join0, h->far));
        }
    }
    if (h->np > 0) {
        if ((rc = timed(h, kKLinks, st, [&] {
                 return D.direct ? launch_links_direct(D, Ain, oc, on, par, st)
                                 : launch_links(D, Ain, oc, on, par, st);
             })))
            return rc;
    }
    // particle update and raster of the new positions (one kernel)
    if ((rc = timed(h, kKParticles, st, [&] { return launch_particles(D, par, on, st); }))) return rc;
    if (h->np > 0) {
        if ((rc = timed(h, kKFlags, st, [&] { return launch_flags(D, oc, on, 1, par, st); }))) return rc;
    }
    if (overlap && !serial) CK(h, cudaStreamWaitEvent(st, h->join0, 0));
    const int kind = overlap ? kKStreamCollideNear : kKStreamCollide;
    const int mode = overlap ? kSCNear : kSCAll;
    if (serial) {
        if ((rc = timed(h, kind, st, [&] { return launch_stream_collide(D, Ain, Aout, mode, st); }))) return rc;
        return timed(h, kKBoundary, st, [&] { return launch_boundary(D, Ain, Aout, oc, par, st); });
    }
    // k_boundary and k_stream_collide write disjoint nodes of Aout and read
    // only inputs complete at this point: run them side by side
    CK(h, cudaEventRecord(h->fork, st));
    CK(h, cudaStreamWaitEvent(h->side, h->fork, 0));
    if ((rc = timed(h, kKBoundary, h->side, [&] { return launch_boundary(D, Ain, Aout, oc, par, h->side); })))
        return rc;
    CK(h, cudaEventRecord(h->join, h->side));
    if ((rc = timed(h, kind, st, [&] { return launch_stream_collide(D, Ain, Aout, mode, st); }))) return rc;
    CK(h, cudaStreamWaitEvent(st, h->join, 0));
    return LBM_OK;
}

int kernels_per_step(const lbm_handle *h)
{
    if (h->np == 0) return 3;
    return ((h->prm.flags & LBM_FLAG_OVERLAP) ? 7 : 5) + ((h->prm.flags & LBM_FLAG_DIRECT_LINKS) ? 1 : 0);
}

// Graph of `steps` consecutive steps from parity par (an even count ends on
// par again).  Consecutive graph launches on a stream cost about 4 us more
// per step than kernel edges inside one graph (at 4000^2 / 4800 disks:
// 0.3785 ms per step with one step per graph, 0.3751 with four, 0.3746 with
// eight, 0.3745 with sixteen).
int capture(lbm_handle *h, int par, int steps, cudaGraphExec_t *out)
{
    if (!h->cap) CK(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    const long long before = h->launches;
    int rc = LBM_OK;
    for (int k = 0; k < steps && !rc; ++k) rc = enqueue_step(h, par ^ (k & 1), h->cap);
    h->launches = before;
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    CK(h, e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(h, e);
    return LBM_OK;
}

int device_error(lbm_handle *h)
{
    unsigned err = 0;
    CK(h, cudaMemcpy(&err, &h->D.status->err, sizeof err, cudaMemcpyDeviceToHost));
    if (err & kErrNumeric) return LBM_ENUMERIC;
    if (err & kErrDomain) return LBM_EDOMAIN;
    if (err & kErrOverflow) return LBM_EOVERFLOW;
    if (err & kErrTimeout) return LBM_ETIMEOUT;
    if (err & kErrBounds) return LBM_EBOUNDS;
    return LBM_OK;
}

int sync_status(lbm_handle *h)
{
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->sticky) return h->sticky;
    int rc = device_error(h);
    if (rc) h->sticky = rc;
    return rc;
}

void fill_dev(lbm_handle *h)
{
    Dev &D = h->D;
    const lbm_params &P = h->prm;
    const Layout &L = h->L;
    char *ws = h->ws;
    D.nx = h->d.nx;
    D.ny = h->d.ny;
    D.pitch = L.pitch;
    D.np = h->np;
    D.ps = L.ps;
    D.storage = P.storage;
    D.per_x = (h->d.bc & LBM_BC_PERIODIC_X) ? 1 : 0;
    D.per_y = (h->d.bc & LBM_BC_PERIODIC_Y) ? 1 : 0;
    const double s_nu = 1.0 / (3.0 * P.nu + 0.5);
    D.s_nu = (float)s_nu;
    D.s_e = (float)(P.s_e > 0 ? P.s_e : 1.0);
    D.s_eps = (float)(P.s_eps > 0 ? P.s_eps : 1.0);
    D.s_q = (float)(P.s_q > 0 ? P.s_q : 8.0 * (2.0 - s_nu) / (8.0 - s_nu));
    D.q_k = (float)(1.0 / (P.alpha / 0.2 + 0.5));
    D.q_e = (float)(P.q_e > 0 ? P.q_e : 1.0);
    D.q_nu = (float)(P.q_nu > 0 ? P.q_nu : 1.0);
    {
        // a_i = (m_i - s_i (m_i - m_eq,i) + (1 - s_i / 2) F_i) / |M_i|^2 with
        // |M_i|^2 = 36 (e, eps), 12 (q), 4 (p); D2Q5 norms 1/2, 1/20, 1/4
        const double se = D.s_e, sp = D.s_eps, sq = D.s_q, sn = D.s_nu, qk = D.q_k, qe = D.q_e, qn = D.q_nu;
        D.kA1 = (float)((1.0 - se) / 36.0); D.kB1 = (float)(se / 36.0); D.kC1 = (float)((1.0 - 0.5 * se) / 6.0);
        D.kA2 = (float)((1.0 - sp) / 36.0); D.kB2 = (float)(sp / 36.0); D.kC2 = (float)((1.0 - 0.5 * sp) / 6.0);
        D.kA4 = (float)((1.0 - sq) / 12.0); D.kB4 = (float)(sq / 12.0); D.kC4 = (float)((1.0 - 0.5 * sq) / 12.0);
        D.kA7 = (float)((1.0 - sn) / 4.0); D.kB7 = (float)(sn / 4.0); D.kC7 = (float)((1.0 - 0.5 * sn) / 2.0);
        D.kC8 = (float)((1.0 - 0.5 * sn) / 4.0);
        D.kG1 = (float)(0.5 * (1.0 - qk)); D.kG2 = (float)(0.5 * qk);
        D.kG3 = (float)(0.05 * (1.0 - qe)); D.kG4 = (float)(0.1 * qe); D.kG5 = (float)(0.25 * (1.0 - qn));
    }
    D.gbeta = (float)(P.g * P.beta);
    D.T0 = (float)P.T0;
    D.bfx = (float)P.body_fx;
    D.bfy = (float)P.body_fy;
    {
        // times a power of two: exact, so the collision on scaled values
        // rounds exactly as the one on the values themselves
        const float sc = kHalfScale;
        for (int i = 0; i < 12; ++i) D.ksc[i] = 0.f;
        D.ksc[kScC1] = sc * D.kC1; D.ksc[kScC2] = sc * D.kC2; D.ksc[kScB4] = sc * D.kB4;
        D.ksc[kScB7] = sc * D.kB7; D.ksc[kScC7] = sc * D.kC7; D.ksc[kScC8] = sc * D.kC8;
        D.ksc[kScG2] = sc * D.kG2; D.ksc[kScThree] = sc * 3.f; D.ksc[kScBfx] = sc * D.bfx;
    }
    for (int i = 0; i < 4; ++i) D.Twall[i] = (float)h->d.T_wall[i];
    D.g = P.g;
    D.rho_f = P.rho_f;
    D.eps_w = P.eps_w;
    D.s_rep = P.s_rep;
    D.fixed = (P.flags & LBM_FLAG_FIXED_PARTICLES) ? 1 : 0;
    D.flags = reinterpret_cast<uint8_t *>(ws + L.flags);
    D.newborn = reinterpret_cast<int *>(ws + L.newborn);
    D.newborn_cap = L.newborn_cap;
    for (int b = 0; b < 2; ++b) D.runs[b] = reinterpret_cast<int2 *>(ws + L.runs[b]);
    D.near = reinterpret_cast<unsigned *>(ws + L.near);
    D.dsum = reinterpret_cast<DirectSums *>(ws + L.dsum);
    D.direct = (P.flags & LBM_FLAG_DIRECT_LINKS) ? 1 : 0;
    // the staged stream-collide pays with 16-bit storage only (BF16 at
    // 4000^2: 166.9 against 180.4 us; FP32: 292 or more against 272 us)
    D.sc_staged = (P.storage != LBM_STORE_FP32 && !(P.flags & LBM_FLAG_SC_UNSTAGED)) ? 1 : 0;
    D.sc_extra_tx = (P.flags & LBM_FLAG_TEST_WAIT_TIMEOUT) ? 1 : 0;
    D.all_pairs = (P.flags & LBM_FLAG_ALL_PAIRS) ? 1 : 0;
    D.near_tpr = near_tiles_per_row(P.storage, L.pitch);
    D.slot_node = reinterpret_cast<int *>(ws + L.slot_node);
    D.slot_q = reinterpret_cast<float *>(ws + L.slot_q);
    D.slot_base = reinterpret_cast<int *>(ws + L.slot_base);
    D.cur = soa_at(ws, L.cur, h->np);
    D.nxt = soa_at(ws, L.nxt, h->np);
    D.px = reinterpret_cast<double *>(ws + L.prev);
    D.py = D.px + h->np;
    D.force = reinterpret_cast<double *>(ws + L.force);
    D.pos4 = reinterpret_cast<float4 *>(ws + L.pos4);
    D.nslots = (long long)L.nslots;
    D.a_elems = (long long)kPop * L.ps + (long long)(kDistTailPad / storage_bytes(D.storage));
    D.prc = reinterpret_cast<float2 *>(ws + L.prc);
    D.lsum = reinterpret_cast<LinkSums *>(ws + L.lsum);
    D.geo_prev = reinterpret_cast<GeomRec *>(ws + L.geo[0]);
    D.geo_cur = reinterpret_cast<GeomRec *>(ws + L.geo[1]);
    D.geo_nxt = reinterpret_cast<GeomRec *>(ws + L.geo[2]);
    D.pconst = reinterpret_cast<double4 *>(ws + L.pconst);
    D.lorder = reinterpret_cast<int *>(ws + L.lorder);
    D.status = reinterpret_cast<Status *>(ws + L.status);
    D.cell_gx = L.cell_gx;
    D.cell_gy = L.cell_gy;
    D.cell_inv = (float)(1.0 / L.cell_side);
    for (int b = 0; b < 2; ++b) D.cells[b] = reinterpret_cast<int *>(ws + L.cells[b]);
    for (int b = 0; b < 2; ++b) {
        h->A[b] = ws + L.A[b];
        h->own[b] = reinterpret_cast<int *>(ws + L.own[b]);
    }
}

// Upload a particle array into the current state (and the copies the step
// keeps), then build the owner map and flags of those positions.
int upload_particles(lbm_handle *h, const lbm_particle *p)
{
    const int n = h->np;
    if (n == 0) return LBM_OK;
    std::vector<double> soa((size_t)kPartFields * n);
    for (int a = 0; a < n; ++a) {
        const double v[kPartFields] = {p[a].x, p[a].y, p[a].ux, p[a].uy, p[a].theta, p[a].omega,
                                       p[a].r, p[a].rho, p[a].T, p[a].b};
        for (int f = 0; f < kPartFields; ++f) soa[(size_t)f * n + a] = v[f];
    }
    const size_t bytes = soa.size() * sizeof(double);
    CK(h, cudaMemcpyAsync(h->D.cur.x, soa.data(), bytes, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->D.nxt.x, h->D.cur.x, bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->D.px, h->D.cur.x, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int rebuild_maps(lbm_handle *h)
{
    const size_t nn = (size_t)h->d.nx * h->d.ny;
    CK(h, cudaMemsetAsync(h->own[0], 0xff, nn * sizeof(int), h->stream));
    CK(h, cudaMemsetAsync(h->own[1], 0xff, nn * sizeof(int), h->stream));
    CK(h, cudaMemsetAsync(h->D.flags, 0, (size_t)h->L.pitch * h->d.ny, h->stream));
    int *oc = h->own[h->parity];
    CK(h, launch_geom_init(h->D, h->stream));
    CK(h, launch_cells_init(h->D, h->stream));
    CK(h, launch_link_order(h->D, h->stream));
    h->since_order = 0;
    CK(h, launch_raster(h->D, oc, h->D.geo_cur, h->D.cur, h->D.runs[h->parity], h->stream));
    CK(h, launch_flags(h->D, oc, oc, 0, h->parity, h->stream));
    // no newborn node yet
    CK(h, cudaMemsetAsync(&h->D.status->nb, 0, sizeof(unsigned), h->stream));
    // the owner map one step back, which the first clear expects in the other buffer
    PartSoA prev = h->D.cur;
    prev.x = h->D.px;
    prev.y = h->D.py;
    CK(h, launch_raster(h->D, h->own[h->parity ^ 1], h->D.geo_prev, prev, nullptr, h->stream));
    return LBM_OK;
}

} // namespace

extern "C" {

const char *lbm_strerror(int code)
{
    switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOSPC: return "workspace too small";
    case LBM_ENUMERIC: return "non-finite or non-physical density/temperature";
    case LBM_EDOMAIN: return "a particle crossed a cavity wall";
    case LBM_EOVERFLOW: return "a fixed index array line holds more than one link";
    case LBM_ETIMEOUT: return "a bounded device wait gave up";
    case LBM_ECUDA: return "CUDA runtime error";
    case LBM_EBOUNDS: return "an index outside its buffer (bounds-checked build)";
    default: return "unknown error";
    }
}

int lbm_query_footprint(const lbm_domain *d, const lbm_particle *p, int32_t n, const lbm_params *prm,
                        size_t *bytes)
{
    if (!bytes) return LBM_EINVAL;
    int rc = validate(d, p, n, prm);
    if (rc) return rc;
    Layout L;
    layout(d, p, n, prm->storage, prm->s_rep, L);
    *bytes = L.total;
    return LBM_OK;
}

int lbm_init(lbm_handle **out, const lbm_domain *d, const lbm_particle *p, int32_t n,
             const lbm_params *prm, void *d_workspace, size_t ws_bytes, void *stream)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    int rc = validate(d, p, n, prm);
    if (rc) return rc;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) % kAlign)) return LBM_EINVAL;
    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_EINVAL;
    h->d = *d;
    h->prm = *prm;
    h->np = n;
    layout(d, p, n, prm->storage, prm->s_rep, h->L);
    if (ws_bytes < h->L.total) {
        delete h;
        return LBM_ENOSPC;
    }
    h->ws = static_cast<char *>(d_workspace);
    h->stream = static_cast<cudaStream_t>(stream);
    fill_dev(h);
    h->D.zone_max = 0;
    for (int a = 0; a < n; ++a) h->D.zone_max = std::max(h->D.zone_max, zone_size(p[a].r));
    auto fail = [&](int code) {
        lbm_destroy(h);
        return code;
    };
    if (cudaMemsetAsync(h->D.status, 0, sizeof(Status), h->stream) != cudaSuccess) return fail(LBM_ECUDA);
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->far, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->fork0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join0, cudaEventDisableTiming) != cudaSuccess)
        return fail(LBM_ECUDA);
    if (prepare_links(h->D) != cudaSuccess) return fail(LBM_ECUDA);
    if (n > 0) {
        std::vector<int> base(n + 1, 0);
        for (int a = 0; a < n; ++a) base[a + 1] = base[a] + slot_capacity(p[a].r);
        if (cudaMemcpyAsync(h->D.slot_base, base.data(), base.size() * sizeof(int),
                            cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
            return fail(LBM_ECUDA);
        if (cudaMemsetAsync(h->D.slot_node, 0xff, h->L.nslots * sizeof(int), h->stream) != cudaSuccess)
            return fail(LBM_ECUDA);
        if (cudaMemsetAsync(h->D.slot_q, 0, h->L.nslots * sizeof(float), h->stream) != cudaSuccess)
            return fail(LBM_ECUDA);
        if (cudaMemsetAsync(h->D.force, 0, 3 * (size_t)n * sizeof(double), h->stream) != cudaSuccess)
            return fail(LBM_ECUDA);
        if ((rc = upload_particles(h, p))) return fail(rc);
    }
    if ((rc = rebuild_maps(h))) return fail(rc);
    // both buffers zeroed whole (the gaps between planes, where the plane
    // stride exceeds ny x pitch, and the tail pad included), so that state
    // images hold no leftover bytes of the workspace
    const size_t abytes = (size_t)kPop * h->L.ps * storage_bytes(h->D.storage) + kDistTailPad;
    for (int b = 0; b < 2; ++b)
        if (cudaMemsetAsync(h->A[b], 0, abytes, h->stream) != cudaSuccess) return fail(LBM_ECUDA);
    if (launch_init_collide(h->D, h->A[1], h->A[0], (float)prm->T_init, 0, h->stream) != cudaSuccess)
        return fail(LBM_ECUDA);
    if ((rc = sync_status(h))) return fail(rc);
    *out = h;
    return LBM_OK;
}

int lbm_step(lbm_handle *h, int32_t nsteps)
{
    if (!h || nsteps < 0) return LBM_EINVAL;
    if (h->sticky) return h->sticky;
    const bool graph = !(h->prm.flags & LBM_FLAG_NO_GRAPH) && !h->timing;
    int rc;
    for (int32_t k = 0; k < nsteps;) {
        // the link order follows the particles every kOrderSteps steps
        if (h->since_order >= kOrderSteps) {
            CK(h, launch_link_order(h->D, h->stream));
            ++h->launches;
            h->since_order = 0;
        }
        if (graph) {
            // the largest graph (8, 4, 2 or 1 steps) that fits what is left
            int l = kGraphLevels - 1;
            while ((1 << l) > nsteps - k) --l;
            const int n = 1 << l;
            cudaGraphExec_t &g = h->gexec[l][h->parity];
            if (!g && (rc = capture(h, h->parity, n, &g))) return rc;
            CK(h, cudaGraphLaunch(g, h->stream));
            h->launches += (long long)n * kernels_per_step(h);
            h->parity ^= n & 1;
            h->since_order += n;
            k += n;
        } else {
            if ((rc = enqueue_step(h, h->parity, h->stream))) return rc;
            h->parity ^= 1;
            ++h->since_order;
            ++k;
        }
    }
    return LBM_OK;
}

int lbm_sync(lbm_handle *h)
{
    if (!h) return LBM_EINVAL;
    return sync_status(h);
}

int lbm_get_fields(lbm_handle *h, float *rho, float *ux, float *uy, float *T, int32_t on_device)
{
    if (!h || !rho || !ux || !uy || !T) return LBM_EINVAL;
    const void *A = h->A[h->parity];
    const int nx = h->d.nx, ny = h->d.ny;
    if (on_device) {
        CK(h, launch_fields(h->D, A, 0, ny, rho, ux, uy, T, h->stream));
        return h->sticky;
    }
    int rc = sync_status(h);
    if (rc) return rc;
    float *st = reinterpret_cast<float *>(h->ws + h->L.stage);
    const int R = h->L.stage_rows;
    float *outs[4] = {rho, ux, uy, T};
    for (int r0 = 0; r0 < ny; r0 += R) {
        const int rows = std::min(R, ny - r0);
        const size_t cnt = (size_t)rows * nx;
        CK(h, launch_fields(h->D, A, r0, rows, st, st + cnt, st + 2 * cnt, st + 3 * cnt, h->stream));
        for (int f = 0; f < 4; ++f)
            CK(h, cudaMemcpyAsync(outs[f] + (size_t)r0 * nx, st + f * cnt, cnt * sizeof(float),
                                  cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

int lbm_get_particles(lbm_handle *h, lbm_particle *out, int32_t n)
{
    if (!h || n != h->np || (n > 0 && !out)) return LBM_EINVAL;
    if (n > 0) {
        lbm_particle *pk = reinterpret_cast<lbm_particle *>(h->ws + h->L.pack);
        CK(h, launch_pack_particles(h->D, pk, h->stream));
        CK(h, cudaMemcpyAsync(out, pk, (size_t)n * sizeof(lbm_particle), cudaMemcpyDeviceToHost,
                              h->stream));
    }
    return sync_status(h);
}

int lbm_get_particles_async(lbm_handle *h, lbm_particle *out, int32_t n)
{
    if (!h || n != h->np || (n > 0 && !out)) return LBM_EINVAL;
    if (h->sticky) return h->sticky;
    if (n > 0) {
        lbm_particle *pk = reinterpret_cast<lbm_particle *>(h->ws + h->L.pack);
        CK(h, launch_pack_particles(h->D, pk, h->stream));
        CK(h, cudaMemcpyAsync(out, pk, (size_t)n * sizeof(lbm_particle), cudaMemcpyDeviceToHost,
                              h->stream));
    }
    return LBM_OK;
}

int lbm_get_forces(lbm_handle *h, double *out, int32_t n)
{
    if (!h || n != h->np || (n > 0 && !out)) return LBM_EINVAL;
    if (n > 0)
        CK(h, cudaMemcpyAsync(out, h->D.force, 3 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    return sync_status(h);
}

int lbm_destroy(lbm_handle *h)
{
    if (!h) return LBM_EINVAL;
    if (h->stream || h->cap) cudaStreamSynchronize(h->stream);
    for (int l = 0; l < kGraphLevels; ++l)
        for (int b = 0; b < 2; ++b)
            if (h->gexec[l][b]) cudaGraphExecDestroy(h->gexec[l][b]);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->far) {
        cudaStreamSynchronize(h->far);
        cudaStreamDestroy(h->far);
    }
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->fork0) cudaEventDestroy(h->fork0);
    if (h->join0) cudaEventDestroy(h->join0);
    for (auto &e : h->ev) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    delete h;
    return LBM_OK;
}

int lbm_get_owner(lbm_handle *h, int32_t *out)
{
    if (!h || !out) return LBM_EINVAL;
    CK(h, cudaMemcpyAsync(out, h->own[h->parity], (size_t)h->d.nx * h->d.ny * sizeof(int),
                          cudaMemcpyDeviceToHost, h->stream));
    return sync_status(h);
}

int lbm_get_slots(lbm_handle *h, int32_t *node, float *q, int64_t cap, int64_t *count)
{
    if (!h || !count || cap < 0) return LBM_EINVAL;
    *count = (int64_t)h->L.nslots;
    const size_t m = std::min<size_t>((size_t)cap, h->L.nslots);
    if (m > 0) {
        if (!node || !q) return LBM_EINVAL;
        CK(h, cudaMemcpyAsync(node, h->D.slot_node, m * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaMemcpyAsync(q, h->D.slot_q, m * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    }
    return sync_status(h);
}

// State image: distributions (current buffer), owner map, flags, particle
// state and previous positions.
static size_t state_parts(const lbm_handle *h, size_t sz[5])
{
    sz[0] = (size_t)kPop * h->L.ps * storage_bytes(h->D.storage);
    sz[1] = (size_t)h->d.nx * h->d.ny * sizeof(int);
    sz[2] = (size_t)h->L.pitch * h->d.ny;
    sz[3] = (size_t)kPartFields * h->np * sizeof(double);
    sz[4] = (size_t)2 * h->np * sizeof(double);
    return sz[0] + sz[1] + sz[2] + sz[3] + sz[4];
}

int lbm_state_bytes(lbm_handle *h, size_t *bytes)
{
    if (!h || !bytes) return LBM_EINVAL;
    size_t sz[5];
    *bytes = state_parts(h, sz);
    return LBM_OK;
}

int lbm_get_state(lbm_handle *h, void *buf, size_t bytes)
{
    size_t sz[5];
    if (!h || !buf || bytes < state_parts(h, sz)) return LBM_EINVAL;
    int rc = sync_status(h);
    if (rc) return rc;
    const void *src[5] = {h->A[h->parity], h->own[h->parity], h->D.flags, h->D.cur.x, h->D.px};
    char *o = static_cast<char *>(buf);
    for (int i = 0; i < 5; ++i) {
        if (sz[i]) CK(h, cudaMemcpyAsync(o, src[i], sz[i], cudaMemcpyDeviceToHost, h->stream));
        o += sz[i];
    }
    return sync_status(h);
}

int lbm_set_state(lbm_handle *h, const void *buf, size_t bytes)
{
    size_t sz[5];
    if (!h || !buf || bytes < state_parts(h, sz)) return LBM_EINVAL;
    CK(h, cudaStreamSynchronize(h->stream));
    void *dst[5] = {h->A[h->parity], h->own[h->parity], h->D.flags, h->D.cur.x, h->D.px};
    const char *in = static_cast<const char *>(buf);
    for (int i = 0; i < 5; ++i) {
        if (sz[i]) CK(h, cudaMemcpyAsync(dst[i], in, sz[i], cudaMemcpyHostToDevice, h->stream));
        in += sz[i];
    }
    if (h->np > 0) {
        CK(h, cudaMemcpyAsync(h->D.nxt.x, h->D.cur.x, sz[3], cudaMemcpyDeviceToDevice, h->stream));
        // owner map one step back, expected by the next clear
        const size_t nn = (size_t)h->d.nx * h->d.ny;
        CK(h, cudaMemsetAsync(h->own[h->parity ^ 1], 0xff, nn * sizeof(int), h->stream));
        PartSoA prev = h->D.cur;
        prev.x = h->D.px;
        prev.y = h->D.py;
        CK(h, launch_geom_init(h->D, h->stream));
        CK(h, launch_cells_init(h->D, h->stream));
        CK(h, launch_link_order(h->D, h->stream));
        h->since_order = 0;
        CK(h, launch_raster(h->D, h->own[h->parity ^ 1], h->D.geo_prev, prev, nullptr, h->stream));
        // the row runs of the restored positions (their raster rewrites the
        // restored owner map with the values it holds), and the newborn
        // list of the restored flags, which the next step returns to fluid
        CK(h, launch_raster(h->D, h->own[h->parity], h->D.geo_cur, h->D.cur, h->D.runs[h->parity], h->stream));
        CK(h, cudaMemsetAsync(&h->D.status->nb, 0, sizeof(unsigned), h->stream));
        CK(h, launch_collect_newborn(h->D, h->stream));
    }
    return sync_status(h);
}

int lbm_set_distributions(lbm_handle *h, const double *f, const double *g)
{
    if (!h || !f || !g) return LBM_EINVAL;
    int rc = sync_status(h);
    if (rc) return rc;
    const int nx = h->d.nx, ny = h->d.ny, pitch = h->L.pitch;
    const long long ps = h->L.ps;
    const size_t nn = (size_t)nx * ny;
    // pre-collision image in the storage type, collided on the device
    const int es = storage_bytes(h->D.storage);
    std::vector<unsigned char> img((size_t)kPop * ps * es, 0);
    for (int p = 0; p < kPop; ++p)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t s = (size_t)j * nx + i;
                const double v = p < kQ9 ? f[(size_t)p * nn + s] - w9d(p) : g[(size_t)(p - kQ9) * nn + s];
                // a non-finite value stays so: at a fluid node the collision
                // reports it (LBM_ENUMERIC), at a solid node it is dropped
                const float x = (float)v;
                const size_t at = (size_t)p * ps + (size_t)j * pitch + i;
                if (h->D.storage == LBM_STORE_BF16) reinterpret_cast<__nv_bfloat16 *>(img.data())[at] = Elem<__nv_bfloat16>::st(x);
                else if (h->D.storage == LBM_STORE_FP16) reinterpret_cast<__half *>(img.data())[at] = Elem<__half>::st(x);
                else reinterpret_cast<float *>(img.data())[at] = x;
            }
    void *scratch = h->A[h->parity ^ 1];
    CK(h, cudaMemcpyAsync(scratch, img.data(), img.size(), cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_init_collide(h->D, scratch, h->A[h->parity], 0.f, 1, h->stream));
    return sync_status(h);
}

int lbm_get_counters(lbm_handle *h, int64_t *out8)
{
    if (!h || !out8) return LBM_EINVAL;
    int rc = sync_status(h);
    if (rc) return rc;
    unsigned long long c[kNumCounters];
    CK(h, cudaMemcpy(c, h->D.status->cnt[h->parity ^ 1], sizeof c, cudaMemcpyDeviceToHost));
    for (int i = 0; i < kNumCounters; ++i) out8[i] = (int64_t)c[i];
    return LBM_OK;
}

int lbm_kernel_timing(lbm_handle *h, int32_t enable)
{
    if (!h) return LBM_EINVAL;
    h->timing = enable != 0;
    return LBM_OK;
}

int lbm_kernel_times(lbm_handle *h, double *ms, int64_t *launches, int32_t nk)
{
    if (!h || !ms || !launches || nk < 0) return LBM_EINVAL;
    CK(h, cudaStreamSynchronize(h->stream));
    int rc = fold_events(h);
    if (rc) return rc;
    for (int k = 0; k < nk && k < kNumKernelKinds; ++k) {
        ms[k] = h->acc_ms[k];
        launches[k] = h->acc_n[k];
        h->acc_ms[k] = 0.0;
        h->acc_n[k] = 0;
    }
    return LBM_OK;
}

int32_t lbm_kernel_count(void) { return kNumKernelKinds; }

const char *lbm_kernel_name(int32_t k)
{
    return (k >= 0 && k < kNumKernelKinds) ? kKernelNames[k] : "";
}

int64_t lbm_launch_count(lbm_handle *h) { return h ? h->launches : -1; }

int lbm_binary_version(int32_t *version)
{
    if (!version) return LBM_EINVAL;
    int v = 0;
    if (stream_collide_binary_version(&v) != cudaSuccess) return LBM_ECUDA;
    *version = v;
    return LBM_OK;
}

} // extern "C"
