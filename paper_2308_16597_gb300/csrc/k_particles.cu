// Particle-side kernels of one time step:
//   k_links      indirect-addressing gather of fluid-particle links into the
//                fixed index array (Sec. 3), curved bounce-back of f and g on
//                each link (Sec. 2.3) and the momentum-exchange force and
//                torque (Sec. 2.4, Eq. force / Eq. torque) reduced per
//                particle in FP64;
//   k_particles  Newton-Euler update with gravity, buoyancy and spring
//                repulsion (Sec. 2.2, Sec. 2.4);
//   k_clear, k_raster, k_flags
//                owner map and node flags at the new positions.
#include "lbm_internal.cuh"

namespace lbm {

namespace {

constexpr int kLinkThreads = 288;
constexpr int kBoxThreads = 128;
constexpr int kPartThreads = 1024;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ bool inside(const Dev &D, int i, int j)
{
    return i >= 0 && i < D.nx && j >= 0 && j < D.ny;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

} // namespace

// One CTA per particle; thread s handles slot s (and s + 128, ...) of the
// particle's 12N - 12 fixed slots.  The slot of (direction k, line) is fixed
// by the zone geometry, so the gather needs no atomics and the per-particle
// reduction is a deterministic tree.
//
// The CTA first copies its zone (plus the two-node margin the bounce-back
// stencil reaches) into shared memory: the owner map and the 12 planes the
// rules read (f1..f8 and g1..g4), in whole 16-byte chunks with cp.async, so
// the scattered reads of the links become one coalesced burst per particle.
// It also issues bulk L2 prefetches of the zone rows of the particle `ahead`
// places later, so that particle's copies hit L2.  Bounce-back values are
// written into the solid node x_f + e_k in direction kbar of A in HBM, where
// the next pull stream picks them up: each (solid node, kbar) belongs to one
// link, and every read is of a fluid node, so the writes never race the reads.
constexpr int kTilePlanes = 12;

// Double-float warp sum (lane 0 receives the result).
__device__ __forceinline__ void warp_df_sum(float &h, float &l)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, h, o);
        const float l2 = __shfl_down_sync(0xffffffffu, l, o);
        df_add(h, l, h2, l2);
    }
}

__host__ __device__ inline int pow2_at_least(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
// Link-kernel shared memory for zones of side N: the 12-plane tile
// [wy][wx] (wy = N + 4 rows, wx a power of two >= N + 7 columns, 16-byte
// aligned start), the owner window [N + 4][ws] (ws a power of two >= N + 4),
// and per-slot counters, link nodes and the compacted list of valid slots.
__host__ __device__ inline int link_tile_wy(int N) { return N + 4; }
__host__ __device__ inline int link_tile_wx(int N) { return pow2_at_least(N + 7); }
__host__ __device__ inline int link_win_ws(int N) { return pow2_at_least(N + 4); }
size_t link_smem_bytes(int N)
{
    const int wy = link_tile_wy(N), wx = link_tile_wx(N), ws = link_win_ws(N), cap = 12 * N - 12;
    return (size_t)kTilePlanes * wy * wx * sizeof(float) + (size_t)(N + 4) * ws * sizeof(int) +
           (size_t)3 * cap * sizeof(int);
}

// Global plane of tile plane t: f1..f8 then g1..g4.
__device__ __forceinline__ int tile_global_plane(int t) { return t < 8 ? t + 1 : t + 2; }

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void prefetch_zone(const Dev &D, const float *A, const GeomRec &G)
{
    const int N = G.N, wy = link_tile_wy(N), wx = link_tile_wx(N);
    const int XA = (G.X0 - 2) & ~3, YA = G.Y0 - 2;
    const int lo = max(XA, 0), hi = min(XA + wx, D.pitch);
    if (hi <= lo) return;
    for (int idx = threadIdx.x; idx < kTilePlanes * wy; idx += kLinkThreads) {
        const int t = idx / wy, row = YA + idx % wy;
        if (row < 0 || row >= D.ny) continue;
        const float *sp = A + (long long)tile_global_plane(t) * D.ps + (long long)row * D.pitch + lo;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sp), "r"((unsigned)(hi - lo) * 4u)
                     : "memory");
    }
}

// Fixed slot (Sec. 3) of the link from zone node (a, b) along e_k, or -1 for
// a corner line that cannot carry a link.
__device__ __forceinline__ int slot_of(int k, int a, int b, int N)
{
    const int M = 2 * N - 3;
    switch (k) {
    case 1: return b;
    case 2: return N + a;
    case 3: return 2 * N + b;
    case 4: return 3 * N + a;
    default: {
        const int line = (k == 5 || k == 7) ? a - b + N - 2 : a + b - 1;
        if (line < 0 || line >= M) return -1;
        return 4 * N + (k - 5) * M + line;
    }
    }
}

// One CTA per particle.  Phases:
//  1. copy the zone (plus the two-node margin of the bounce-back stencil)
//     into shared memory: the 12 planes the rules read (f1..f8, g1..g4) with
//     16-byte cp.async, and the owner map; also issue bulk L2 prefetches of
//     the zone rows of the particle `ahead` places later in launch order;
//  2. every zone node that is fluid tests its eight neighbours; a neighbour
//     owned by this particle makes a link, recorded in the link's fixed slot
//     of the index array (direction k, line through the zone; Sec. 3);
//  3. the valid slots are compacted in slot order (a block-wide prefix), so
//     thread i takes the i-th link: the work is balanced and the reduction
//     order is fixed, hence the forces are bit-reproducible;
//  4. each link: wall fraction q, curved bounce-back of f and g (Sec. 2.3)
//     written into the solid node x_f + e_k (direction kbar) of A in HBM,
//     where the next pull stream picks it up (one link per (solid node, kbar),
//     and every read is of a fluid node), and the momentum-exchange bracket
//     of Eq. force / Eq. torque, reduced per particle.
__global__ void __launch_bounds__(kLinkThreads)
    k_links(const Dev D, float *A, const int *__restrict__ own, int parity, int ahead)
{
    extern __shared__ __align__(16) float ltile[];
    __shared__ int s_warp[kLinkThreads / 32 + 1];
    __shared__ unsigned s_over;
    const int p = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const GeomRec G = D.geo_cur[p];
    const DiskDF dk = geom_df(G);
    const float Ux = G.ux, Uy = G.uy, Om = G.om, wT = G.wT;
    const int N = G.N, cap = 12 * N - 12;
    const int X0 = G.X0, Y0 = G.Y0;
    const int base = D.slot_base[p];
    if (tid == 0) {
        D.pos4[p] = make_float4(dk.xh, dk.yh, dk.xl, dk.yl);
        D.prc[p] = make_float2(G.r, G.C);
        s_over = 0u;
    }
    if (p + ahead < D.np) prefetch_zone(D, A, D.geo_cur[p + ahead]);

    const int Nm = D.zone_max;
    const int wy = link_tile_wy(Nm), wx = link_tile_wx(Nm), ws = link_win_ws(Nm);
    const int XA = (X0 - 2) & ~3, YA = Y0 - 2;
    int *win = reinterpret_cast<int *>(ltile + kTilePlanes * wy * wx); // [N + 4][ws]
    int *cnt = win + (Nm + 4) * ws;                                    // [cap] links per slot
    int *info = cnt + 12 * Nm - 12;                                    // [cap] (b << 16) | a
    int *list = info + 12 * Nm - 12;                                   // [cap] valid slots in order

    // ---- 1. tile and owner window
    {
        const int cpr = wx >> 2, lcpr = __ffs(cpr) - 1, per_plane = wy * cpr;
        for (int t = 0; t < kTilePlanes; ++t) {
            const float *src = A + (long long)tile_global_plane(t) * D.ps;
            for (int e = tid; e < per_plane; e += kLinkThreads) {
                const int row = e >> lcpr, c = e & (cpr - 1);
                const int gy = YA + row, gx = XA + 4 * c;
                if (gy < 0 || gy >= D.ny || gx < 0 || gx + 4 > D.pitch) continue;
                cp_async16(ltile + (t * wy + row) * wx + 4 * c, src + (long long)gy * D.pitch + gx);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        const int lws = __ffs(ws) - 1;
        for (int e = tid; e < (N + 4) * ws; e += kLinkThreads) {
            const int row = e >> lws, col = e & (ws - 1);
            if (col >= N + 4) continue;
            const int i = X0 - 2 + col, j = Y0 - 2 + row;
            win[e] = inside(D, i, j) ? own[(long long)j * D.nx + i] : -2;
        }
        for (int e = tid; e < cap; e += kLinkThreads) cnt[e] = 0;
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
    }
    auto owner_at = [&](int i, int j) -> int { return win[(j - Y0 + 2) * ws + (i - X0 + 2)]; };
    auto tv = [&](int t, int i, int j) -> float { return ltile[(t * wy + (j - YA)) * wx + (i - XA)]; };

    // ---- 2. link detection, one zone node per thread
    {
        const int lws = __ffs(ws) - 1;
        for (int e = tid; e < N * ws; e += kLinkThreads) {
            const int bb = e >> lws, aa = e & (ws - 1);
            if (aa >= N) continue;
            const int w0 = (bb + 2) * ws + (aa + 2);
            if (win[w0] != -1) continue;
#pragma unroll
            for (int k = 1; k < kQ9; ++k) {
                if (win[w0 + ey(k) * ws + ex(k)] != p) continue;
                const int sl = slot_of(k, aa, bb, N);
                if (sl < 0) {
                    s_over = 1u;
                    continue;
                }
                if (atomicAdd(&cnt[sl], 1) == 0) info[sl] = (bb << 16) | aa;
                else s_over = 1u;
            }
        }
        __syncthreads();
    }

    // ---- 3. compaction of the valid slots in slot order
    int nvalid = 0;
    for (int s0 = 0; s0 < cap; s0 += kLinkThreads) {
        const int sl = s0 + tid;
        const bool v = sl < cap && cnt[sl] > 0;
        const unsigned m = __ballot_sync(0xffffffffu, v);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int w = 0; w < kLinkThreads / 32; ++w) {
                const int c = s_warp[w];
                s_warp[w] = acc;
                acc += c;
            }
            s_warp[kLinkThreads / 32] = acc;
        }
        __syncthreads();
        if (v) list[nvalid + s_warp[warp] + __popc(m & ((1u << lane) - 1u))] = sl;
        else if (sl < cap) {
            D.slot_node[base + sl] = -1;
            D.slot_q[base + sl] = 0.f;
        }
        nvalid += s_warp[kLinkThreads / 32];
        __syncthreads();
    }

    // ---- 4. bounce-back and momentum exchange, thread i on the i-th link
    float sbx = 0.f, sby = 0.f, stq = 0.f; // link brackets of Eq. force / Eq. torque
    int ax_x = 0, ax_y = 0, ax_t = 0, dg_x = 0, dg_y = 0, dg_t = 0; // exact constant parts
    unsigned c_lin = 0, c_simple = 0, c_th = 0;
    for (int li = tid; li < nvalid; li += kLinkThreads) {
        const int sl = list[li];
        int k, line;
        slot_dir_line(sl, N, k, line);
        const int kx = ex(k), ky = ey(k);
        const int fi = X0 + (info[sl] & 0xffff), fj = Y0 + (info[sl] >> 16);
        float dxf, dyf;
        const float q = link_q_df(fi, fj, k, dk, dxf, dyf);
        D.slot_node[base + sl] = fj * D.nx + fi;
        D.slot_q[base + sl] = q;

        // curved bounce-back in deviation form: every rule is an affine
        // combination of populations of equal weight, so it holds for
        // f~ = f - w unchanged
        const int kb = opp(k);
        const int i1 = fi - kx, j1 = fj - ky, i2 = fi - 2 * kx, j2 = fj - 2 * ky;
        const bool have1 = owner_at(i1, j1) == -1;
        const bool have2 = owner_at(i2, j2) == -1;
        const int ii1 = have1 ? i1 : fi, jj1 = have1 ? j1 : fj;
        const int ii2 = have2 ? i2 : fi, jj2 = have2 ? j2 : fj;
        const float fk0 = tv(k - 1, fi, fj), fk1 = tv(k - 1, ii1, jj1), fk2 = tv(k - 1, ii2, jj2);
        const float fb0 = tv(kb - 1, fi, fj), fb1 = tv(kb - 1, ii1, jj1);
        const float rx = dxf + q * kx, ry = dyf + q * ky;
        const float uwx = Ux - Om * ry, uwy = Uy + Om * rx;
        const float wall = 6.f * w9(k) * -(kx * uwx + ky * uwy); // 2 w rho0 e_kbar.u_w / c_s^2
        int lvl;
        const float fnew = bouzidi32(q, fk0, fk1, fk2, fb0, fb1, have1, have2, wall, lvl);
        c_lin += lvl == 1;
        c_simple += lvl == 2;
        const long long ns = (long long)(fj + ky) * D.pitch + (fi + kx);
        A[kb * D.ps + ns] = fnew;
        if (k <= 4) {
            const float gnew = thermal32(q, tv(8 + k - 1, fi, fj), tv(8 + k - 1, ii1, jj1),
                                         tv(8 + kb - 1, fi, fj), have1, wT);
            c_th += !have1;
            A[(kQ9 + kb) * D.ps + ns] = gnew;
        }
        // momentum exchange: with f = w + f~ the bracket of Eq. force is
        // 2 w_k e_k + [f~_k^+ (e_k - u_w) - f~_kbar (e_kbar - u_w)]; the
        // constant part and its torque 2 w_k ((i - x_c) e_k,y - (j - y_c) e_k,x)
        // (q drops out) are kept as exact integer sums, assembled in FP64 by
        // the particle update
        const float bx = fk0 * (kx - uwx) - fnew * (-kx - uwx);
        const float by = fk0 * (ky - uwy) - fnew * (-ky - uwy);
        sbx += bx;
        sby += by;
        stq += rx * by - ry * bx;
        const int tz = fi * ky - fj * kx;
        if (k <= 4) { ax_x += kx; ax_y += ky; ax_t += tz; }
        else { dg_x += kx; dg_y += ky; dg_t += tz; }
    }

    __shared__ float red[6][kLinkThreads / 32];
    __shared__ int icnt[9][kLinkThreads / 32];
    float fxl = 0.f, fyl = 0.f, tzl = 0.f;
    warp_df_sum(sbx, fxl);
    warp_df_sum(sby, fyl);
    warp_df_sum(stq, tzl);
    const unsigned F = 0xffffffffu;
    const int iv[9] = {(int)__reduce_add_sync(F, c_lin), (int)__reduce_add_sync(F, c_simple),
                       (int)__reduce_add_sync(F, c_th), (int)__reduce_add_sync(F, (unsigned)ax_x),
                       (int)__reduce_add_sync(F, (unsigned)ax_y), (int)__reduce_add_sync(F, (unsigned)ax_t),
                       (int)__reduce_add_sync(F, (unsigned)dg_x), (int)__reduce_add_sync(F, (unsigned)dg_y),
                       (int)__reduce_add_sync(F, (unsigned)dg_t)};
    if (lane == 0) {
        red[0][warp] = sbx; red[1][warp] = fxl;
        red[2][warp] = sby; red[3][warp] = fyl;
        red[4][warp] = stq; red[5][warp] = tzl;
        for (int c = 0; c < 9; ++c) icnt[c][warp] = iv[c];
    }
    __syncthreads();
    if (tid == 0) {
        LinkSums S;
        S.fx_h = red[0][0]; S.fx_l = red[1][0];
        S.fy_h = red[2][0]; S.fy_l = red[3][0];
        S.tz_h = red[4][0]; S.tz_l = red[5][0];
        int a9[9];
        for (int c = 0; c < 9; ++c) a9[c] = icnt[c][0];
        for (int w = 1; w < kLinkThreads / 32; ++w) {
            df_add(S.fx_h, S.fx_l, red[0][w], red[1][w]);
            df_add(S.fy_h, S.fy_l, red[2][w], red[3][w]);
            df_add(S.tz_h, S.tz_l, red[4][w], red[5][w]);
            for (int c = 0; c < 9; ++c) a9[c] += icnt[c][w];
        }
        S.ax_x = a9[3]; S.ax_y = a9[4]; S.ax_t = a9[5];
        S.dg_x = a9[6]; S.dg_y = a9[7]; S.dg_t = a9[8];
        S.pad[0] = S.pad[1] = S.pad[2] = S.pad[3] = 0;
        D.lsum[p] = S;
        unsigned long long *C = D.status->cnt[parity];
        if (a9[0]) atomicAdd(&C[kCntBzLinear], (unsigned long long)a9[0]);
        if (a9[1]) atomicAdd(&C[kCntBzSimple], (unsigned long long)a9[1]);
        if (a9[2]) atomicAdd(&C[kCntThermHalf], (unsigned long long)a9[2]);
        if (nvalid) atomicAdd(&C[kCntLinks], (unsigned long long)nvalid);
        if (s_over) atomicOr(&D.status->err, kErrOverflow);
    }
}

// Spring repulsion magnitude of Sec. 2.4 for a gap (distance to the wall
// plane, or centre distance minus both radii): zero beyond the threshold s,
// else (C/eps) ((gap - s)/s)^2 along the gap vector.
__device__ __forceinline__ double repulsion(double gap, double s, double eps, double C)
{
    if (gap > s) return 0.0;
    const double t = (gap - s) / s;
    return C / eps * t * t;
}

// Total force = hydrodynamic (assembled from the link sums) + buoyant weight
// -(rho_p - rho_f) pi r^2 g y-hat + repulsion (walls, and every other disk
// with C_ab the mean of the two force scales C = pi r^2 (rho_p - rho_f) g).
// Each block takes 32 particles: warp w screens particle w against all disks
// in shared-memory tiles (FP32 centres with a one-lattice-unit margin) and
// evaluates the pairs in reach from double-float centre differences; lane l
// of warp 0 then sums, integrates and stores particle l in FP64, so 32
// particles share every FP64 instruction.  Integration: U' = U + F/M,
// X' = X + (U + U')/2, Omega' = Omega + T/I, theta' = theta + (Omega + Omega')/2
// with M = rho_p pi r^2 and I = M r^2 / 2.
constexpr int kPartTile = 512;

// Pair repulsion on disk a from disk b (FP32 from double-float centres).
__device__ __noinline__ void pair_force(float4 pa, float2 ca, float4 pb, float2 cb, float s_rep,
                                        float inv_eps, float &fh_x, float &fl_x, float &fh_y,
                                        float &fl_y)
{
    float hx, ex_, hy, ey_;
    two_sum(pa.x, -pb.x, hx, ex_);
    two_sum(pa.y, -pb.y, hy, ey_);
    const float dx = hx + (ex_ + (pa.z - pb.z));
    const float dy = hy + (ey_ + (pa.w - pb.w));
    const float dist = sqrtf(dx * dx + dy * dy);
    const float gap = dist - ca.x - cb.x;
    if (gap > s_rep) return;
    const float t = (gap - s_rep) / s_rep;
    const float mag = 0.5f * (ca.y + cb.y) * inv_eps * t * t;
    df_add(fh_x, fl_x, mag * dx / dist, 0.f);
    df_add(fh_y, fl_y, mag * dy / dist, 0.f);
}

__global__ void __launch_bounds__(kPartThreads) k_particles(const Dev D, int parity)
{
    __shared__ float4 sp[kPartTile];
    __shared__ float2 sc[kPartTile];
    __shared__ float sred[4][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a = blockIdx.x * 32 + warp;
    if (blockIdx.x == 0 && threadIdx.x < kNumCounters) D.status->cnt[parity ^ 1][threadIdx.x] = 0ull;
    const bool me = a < D.np;
    float4 pa = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 ca = make_float2(1.f, 0.f);
    if (me) {
        pa = D.pos4[a];
        ca = D.prc[a];
    }
    const float s_rep = (float)D.s_rep, inv_eps = (float)(1.0 / D.eps_w);
    const float reach = s_rep + 1.f;
    float fhx = 0.f, flx = 0.f, fhy = 0.f, fly = 0.f;
    for (int t0 = 0; t0 < D.np; t0 += kPartTile) {
        const int nb = min(kPartTile, D.np - t0);
        __syncthreads();
        for (int k = threadIdx.x; k < nb; k += kPartThreads) {
            sp[k] = D.pos4[t0 + k];
            sc[k] = D.prc[t0 + k];
        }
        __syncthreads();
        if (!me) continue;
        for (int u = lane; u < nb; u += 32) {
            const float4 o = sp[u];
            const float dxf = pa.x - o.x, dyf = pa.y - o.y, lim = ca.x + sc[u].x + reach;
            if (dxf * dxf + dyf * dyf > lim * lim || t0 + u == a) continue;
            pair_force(pa, ca, o, sc[u], s_rep, inv_eps, fhx, flx, fhy, fly);
        }
    }
    warp_df_sum(fhx, flx);
    warp_df_sum(fhy, fly);
    if (lane == 0) {
        sred[0][warp] = fhx; sred[1][warp] = flx;
        sred[2][warp] = fhy; sred[3][warp] = fly;
    }
    __syncthreads();
    if (warp != 0) return;
    const int b = blockIdx.x * 32 + lane;
    if (b >= D.np) return;
    double x = D.cur.x[b], y = D.cur.y[b], ux = D.cur.ux[b], uy = D.cur.uy[b];
    double th = D.cur.th[b], om = D.cur.om[b];
    const double r = D.cur.r[b], rho = D.cur.rho[b];
    double Fx, Fy, Tz;
    assemble_force(D.lsum[b], x, y, Fx, Fy, Tz);
    D.force[3 * b + 0] = Fx;
    D.force[3 * b + 1] = Fy;
    D.force[3 * b + 2] = Tz;
    const double Cb = kPi * r * r * (rho - D.rho_f) * D.g;
    Fy -= (rho - D.rho_f) * kPi * r * r * D.g;
    if (!D.per_x) {
        Fx += repulsion((x + 0.5) - r, D.s_rep, D.eps_w, Cb);
        Fx -= repulsion(((double)D.nx - 0.5 - x) - r, D.s_rep, D.eps_w, Cb);
    }
    if (!D.per_y) {
        Fy += repulsion((y + 0.5) - r, D.s_rep, D.eps_w, Cb);
        Fy -= repulsion(((double)D.ny - 0.5 - y) - r, D.s_rep, D.eps_w, Cb);
    }
    Fx += (double)sred[0][lane] + (double)sred[1][lane];
    Fy += (double)sred[2][lane] + (double)sred[3][lane];
    if (!D.fixed) {
        const double M = rho * kPi * r * r, I = 0.5 * M * r * r;
        const double ux1 = ux + Fx / M, uy1 = uy + Fy / M, om1 = om + Tz / I;
        x += 0.5 * (ux + ux1);
        y += 0.5 * (uy + uy1);
        th += 0.5 * (om + om1);
        ux = ux1;
        uy = uy1;
        om = om1;
    }
    if (x - r < -0.5 || x + r > (double)D.nx - 0.5 || y - r < -0.5 || y + r > (double)D.ny - 0.5)
        atomicOr(&D.status->err, kErrDomain);
    const double T = D.cur.T[b];
    D.nxt.x[b] = x; D.nxt.y[b] = y; D.nxt.ux[b] = ux; D.nxt.uy[b] = uy; D.nxt.th[b] = th;
    D.nxt.om[b] = om; D.nxt.r[b] = r; D.nxt.rho[b] = rho; D.nxt.T[b] = T;
    D.geo_nxt[b] = make_geom(x, y, r, ux, uy, om, T, rho, D.rho_f, D.g);
}

// Zone of a disk at (x, y) with radius r: N x N nodes from
// (floor(x - r) - 1, floor(y - r) - 1); it holds every node of the disk and
// every fluid node linked to it.
struct Box {
    int X0, Y0, N;
};
__device__ __forceinline__ Box box_of(const GeomRec &G) { return Box{G.X0, G.Y0, G.N}; }

// Reset the zone of each disk's position one step back in the owner map
// that is about to receive the new positions, and in the flag map.
__global__ void __launch_bounds__(kBoxThreads) k_clear(const Dev D, int *own_nxt)
{
    const int p = blockIdx.x;
    const Box B = box_of(D.geo_prev[p]);
    for (int idx = threadIdx.x; idx < B.N * B.N; idx += kBoxThreads) {
        const int i = B.X0 + idx % B.N, j = B.Y0 + idx / B.N;
        if (!inside(D, i, j)) continue;
        own_nxt[(long long)j * D.nx + i] = -1;
        D.flags[(long long)j * D.pitch + i] = kFluid;
    }
}

// Owner map: node (i,j) belongs to disk p iff (i - x)^2 + (j - y)^2 <= r^2
// (exact FP64); where disks overlap the highest index wins (atomicMax, so
// the result does not depend on the launch order).  One warp per disk, one
// lane per zone row: the predicate holds on one contiguous run of each row
// (it is monotone in |i - x|), so the run is found from an FP32 estimate of
// its ends and settled with the exact predicate at the ends only.
__global__ void __launch_bounds__(kBoxThreads)
    k_raster(const Dev D, int *own, const GeomRec *__restrict__ geo, const PartSoA pos)
{
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (kBoxThreads / 32) + (threadIdx.x >> 5);
    if (p >= D.np) return;
    const GeomRec G = geo[p];
    const double x = pos.x[p], y = pos.y[p], r = pos.r[p]; // for the FP64 fallback only
    const Box B = box_of(G);
    const DiskDF dk = geom_df(G);
    const int ic = G.ic; // the node of each row nearest the centre
    for (int b = lane; b < B.N; b += 32) {
        const int j = B.Y0 + b;
        if (j < 0 || j >= D.ny) continue;
        if (!in_disk_df(ic, j, dk, x, y, r)) continue; // then no node of the row is inside
        float dyh, dyl;
        df_offset(j, dk.yh, dk.yl, dyh, dyl);
        const float h = sqrtf(fmaxf(dk.r2h - dyh * dyh, 0.f));
        const int xmin = B.X0, xmax = B.X0 + B.N - 1;
        int lo = min(ic, (int)ceilf(dk.xh - h)), hi = max(ic, (int)floorf(dk.xh + h));
        lo = max(lo, xmin);
        hi = min(hi, xmax);
        while (lo > xmin && in_disk_df(lo - 1, j, dk, x, y, r)) --lo;
        while (!in_disk_df(lo, j, dk, x, y, r)) ++lo;
        while (hi < xmax && in_disk_df(hi + 1, j, dk, x, y, r)) ++hi;
        while (!in_disk_df(hi, j, dk, x, y, r)) --hi;
        lo = max(lo, 0);
        hi = min(hi, D.nx - 1);
        int *row = own + (long long)j * D.nx;
        for (int i = lo; i <= hi; ++i) atomicMax(row + i, p);
    }
}

// Flags over the zones of the old and the new position: solid at the new
// time, newborn (solid before, fluid now) or fluid.  Then each block moves
// its particle's new state into the current slot and keeps the old position
// for the next clear.
__global__ void __launch_bounds__(kBoxThreads)
    k_flags(const Dev D, const int *__restrict__ own_cur, const int *__restrict__ own_nxt, int rotate)
{
    const int p = blockIdx.x;
    const Box B0 = box_of(D.geo_cur[p]);
    const Box B1 = box_of(D.geo_nxt[p]);
    for (int pass = 0; pass < 2; ++pass) {
        const Box B = pass ? B1 : B0;
        for (int idx = threadIdx.x; idx < B.N * B.N; idx += kBoxThreads) {
            const int i = B.X0 + idx % B.N, j = B.Y0 + idx / B.N;
            if (!inside(D, i, j)) continue;
            const long long n = (long long)j * D.nx + i;
            const uint8_t f = own_nxt[n] >= 0 ? kSolid : own_cur[n] >= 0 ? kNewborn : kFluid;
            D.flags[(long long)j * D.pitch + i] = f;
        }
    }
    if (!rotate) return;
    __syncthreads();
    switch (threadIdx.x) {
    case 0: D.px[p] = D.cur.x[p]; D.cur.x[p] = D.nxt.x[p]; break;
    case 1: D.py[p] = D.cur.y[p]; D.cur.y[p] = D.nxt.y[p]; break;
    case 2: D.cur.ux[p] = D.nxt.ux[p]; break;
    case 3: D.cur.uy[p] = D.nxt.uy[p]; break;
    case 4: D.cur.th[p] = D.nxt.th[p]; break;
    case 5: D.cur.om[p] = D.nxt.om[p]; break;
    case 6: D.geo_prev[p] = D.geo_cur[p]; break;
    default: break;
    }
    __syncthreads();
    if (threadIdx.x == 0) D.geo_cur[p] = D.geo_nxt[p];
}

// Geometry records of the current state and of the previous positions.
__global__ void k_geom_init(const Dev D)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= D.np) return;
    const GeomRec G = make_geom(D.cur.x[a], D.cur.y[a], D.cur.r[a], D.cur.ux[a], D.cur.uy[a],
                                D.cur.om[a], D.cur.T[a], D.cur.rho[a], D.rho_f, D.g);
    D.geo_cur[a] = G;
    D.geo_nxt[a] = G;
    D.geo_prev[a] = make_geom(D.px[a], D.py[a], D.cur.r[a], 0.0, 0.0, 0.0, D.cur.T[a], D.cur.rho[a],
                              D.rho_f, D.g);
}

__global__ void k_pack_particles(const Dev D, lbm_particle *out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= D.np) return;
    lbm_particle P;
    P.x = D.cur.x[a]; P.y = D.cur.y[a]; P.ux = D.cur.ux[a]; P.uy = D.cur.uy[a];
    P.theta = D.cur.th[a]; P.omega = D.cur.om[a]; P.r = D.cur.r[a]; P.rho = D.cur.rho[a];
    P.T = D.cur.T[a];
    out[a] = P;
}

cudaError_t prepare_links(Dev &D)
{
    D.link_ahead = 1;
    if (D.np == 0) return cudaSuccess;
    const size_t smem = link_smem_bytes(D.zone_max);
    cudaError_t e = cudaFuncSetAttribute(k_links, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0, dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_links, kLinkThreads, smem)) != cudaSuccess)
        return e;
    D.link_ahead = max(1, sms * per_sm);
    return cudaSuccess;
}

cudaError_t launch_links(const Dev &D, float *A, const int *own_cur, int parity, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_links<<<D.np, kLinkThreads, link_smem_bytes(D.zone_max), s>>>(D, A, own_cur, parity, D.link_ahead);
    return cudaGetLastError();
}

cudaError_t launch_particles(const Dev &D, int parity, cudaStream_t s)
{
    const int blocks = D.np > 0 ? (D.np + 31) / 32 : 1;
    k_particles<<<blocks, kPartThreads, 0, s>>>(D, parity);
    return cudaGetLastError();
}

cudaError_t launch_clear(const Dev &D, int *own_nxt, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_clear<<<D.np, kBoxThreads, 0, s>>>(D, own_nxt);
    return cudaGetLastError();
}

cudaError_t launch_raster(const Dev &D, int *own, const GeomRec *geo, const PartSoA &pos, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    const int per = kBoxThreads / 32;
    k_raster<<<(D.np + per - 1) / per, kBoxThreads, 0, s>>>(D, own, geo, pos);
    return cudaGetLastError();
}

cudaError_t launch_geom_init(const Dev &D, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_geom_init<<<(D.np + 127) / 128, 128, 0, s>>>(D);
    return cudaGetLastError();
}

cudaError_t launch_flags(const Dev &D, const int *own_cur, const int *own_nxt, int rotate,
                         cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_flags<<<D.np, kBoxThreads, 0, s>>>(D, own_cur, own_nxt, rotate);
    return cudaGetLastError();
}

cudaError_t launch_pack_particles(const Dev &D, lbm_particle *out, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_pack_particles<<<(D.np + 127) / 128, 128, 0, s>>>(D, out);
    return cudaGetLastError();
}

} // namespace lbm
