// Particle-side kernels of one time step:
//   k_links      indirect-addressing gather of fluid-particle links into the
//                fixed index array (Sec. 3), curved bounce-back of f and g on
//                each link (Sec. 2.3) and the momentum-exchange force and
//                torque (Sec. 2.4, Eq. force / Eq. torque) summed per
//                particle in exact fixed point; entry of each particle in
//                the pair-screening grid;
//   k_particles  pair screening through the cell grid, Newton-Euler update
//                with gravity, buoyancy and spring repulsion (Sec. 2.2,
//                Sec. 2.4) in FP64, and the raster of the new positions into
//                the next owner map (cleared over the old zones by k_links);
//   k_flags      node flags at the new positions and the newborn list;
// plus the initialisation kernels (k_raster, k_geom_init), the
// direct-addressing comparison (k_direct_prep, k_links_direct), the near-tile
// bitmap of the opt-in split stream-collide (k_near_mask) and the batched
// forms of the step kernels.
#include <climits>
#include <mutex>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

constexpr int kLinkThreads = 128;
constexpr int kBoxThreads = 128;
constexpr int kPartThreads = 256;
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

// The link kernel's window for zones of side N: the zone plus the two-node
// margin of the bounce-back stencil, wy = N + 4 rows of wx = N + 4 columns
// from (X0 - 2, Y0 - 2); wx is at most 64 (the fluid and owner masks of a row
// are 64-bit words).
__host__ __device__ inline int link_tile_wy(int N) { return N + 4; }
__host__ __device__ inline int link_tile_wx(int N) { return N + 4; }
__host__ __device__ inline int link_occ_words(int N) { return (12 * N - 12 + 31) / 32; }

// Shared memory: the fluid and owner row masks [wy] (u64 each), slot
// occupancy words and their prefix [words], and per slot the link node and
// the compacted slot list.
size_t link_smem_bytes(int N, int storage)
{
    (void)storage;
    const size_t cap = (size_t)12 * N - 12;
    return (size_t)2 * link_tile_wy(N) * sizeof(unsigned long long) +
           (size_t)2 * link_occ_words(N) * sizeof(unsigned) + cap * 2 * sizeof(int);
}

bool link_zone_supported(int N, int storage)
{
    return link_tile_wx(N) <= 64 && link_smem_bytes(N, storage) <= (size_t)200 * 1024;
}

// Fixed slot (Sec. 3) of the link from zone node (a, b) along e_k, or -1 for
// a corner line that cannot carry a link.  Axis directions: e1/e3 by row b,
// e2/e4 by column a (N lines each); diagonals: e5/e7 by a - b + N - 2, e6/e8
// by a + b - 1 (2N - 3 lines each).  Branch-free, so that the lanes of a warp
// with different directions do not diverge.
__device__ __forceinline__ int slot_of(int k, int a, int b, int N)
{
    const int M = 2 * N - 3;
    const bool axis = k <= 4, odd = k & 1;
    const int line = odd ? (axis ? b : a - b + N - 2) : (axis ? a : a + b - 1);
    const int slot = axis ? (k - 1) * N + line : 4 * N + (k - 5) * M + line;
    return (axis || (line >= 0 && line < M)) ? slot : -1;
}

// Counts (and overflow flag) of the screening grid of the next step, which
// the next step's link kernel fills: block p of the np blocks of a
// per-particle kernel clears its share.  The grid was last read by the
// previous step's update.
__device__ __forceinline__ void clear_cells_slice(const Dev &D, int parity, int p, int tid, int nthreads)
{
    int *grid = D.cells[parity ^ 1];
    const int nc = D.cell_gx * D.cell_gy + 1, per = (nc + D.np - 1) / D.np;
    const int c1 = min(nc, (p + 1) * per);
    for (int c = p * per + tid; c < c1; c += nthreads)
        if (in_bounds(D, c, (long long)nc * (1 + kCellCap))) grid[c] = 0;
}

// Entry of particle b at (xh, yh) in a screening grid (cleared beforehand);
// a full cell flags the grid, whose next screening then scans all pairs.
__device__ __forceinline__ void cell_insert(const Dev &D, int *grid, int b, float xh, float yh)
{
    const int ncell = D.cell_gx * D.cell_gy, c = cell_of(D, xh, yh);
    const long long size = (long long)(ncell + 1) + (long long)ncell * kCellCap;
    if (!in_bounds(D, c, ncell)) return;
    const int k = atomicAdd(grid + c, 1);
    if (k < kCellCap) {
        if (in_bounds(D, ncell + 1 + (long long)c * kCellCap + k, size)) grid[ncell + 1 + c * kCellCap + k] = b;
    } else grid[ncell] = 1;
}

// The last step's newborn nodes (fluid now, listed by the flags kernel of
// that step) go back to plain fluid: the flags kernel of this step rewrites
// only the nodes whose class changes at the particles' edges.  Entries of
// block p of np blocks of nthreads threads.
__device__ __forceinline__ void revert_newborn(const Dev &D, int p, int tid, int nthreads)
{
    const int nb = min((int)D.status->nb, D.newborn_cap);
    for (int e = p * nthreads + tid; e < nb; e += D.np * nthreads) {
        const int v = D.newborn[e], n = v < 0 ? ~v : v;
        const int y = n / D.nx, x = n - y * D.nx;
        if (in_bounds(D, (long long)y * D.pitch + x, (long long)D.ny * D.pitch)) D.flags[(long long)y * D.pitch + x] = kFluid;
    }
}

// One CTA per particle.  Phases:
//  0. clear this CTA's share of the screening grid the next step's link
//     kernel fills, and the particle's zone one step back in the owner map
//     that the raster fills next; return the last step's newborn nodes to
//     fluid;
//  1. the warps read the owner map over the particle's window (zone plus
//     the two-node margin of the bounce-back stencil) and record per row a
//     fluid mask and an owned-by-this-particle mask (one ballot per 32
//     nodes); thread 0 publishes the particle's screening record (and the
//     FP64 frame of an ellipse); a warp prefetches into L2 the owner rows of
//     the particle
//     `ahead` places later in launch order (one residency wave ahead).
//     (Prefetching the populations of that particle's window as well, by
//     tensor or row prefetches, or of this particle's links as they are
//     found, measured slower: the kernel is bound by its latency chains and
//     issue, not by DRAM, and the extra traffic and instructions cost more
//     than the hits gained);
//  2. thread (k, b) intersects the fluid mask of zone row b with the owner
//     mask of row b + e_k,y shifted by e_k,x: each set bit is a link, which
//     claims its fixed slot of the index array (direction k, line through
//     the zone; Sec. 3) in an occupancy bitmap;
//  3. the occupied slots are compacted in slot order (popcount prefix), so
//     thread i takes the i-th link and the work is balanced;
//  4. each link: wall fraction q, curved bounce-back of f and g (Sec. 2.3)
//     from the populations read at x_f, x_f - e_k and x_f - 2 e_k,
//     written into the solid node x_f + e_k (direction kbar) of A in HBM,
//     where the next pull stream picks it up (one link per (solid node, kbar),
//     and every read is of a fluid node, so the writes never race the reads),
//     and the momentum-exchange bracket of Eq. force / Eq. torque, summed
//     in exact fixed point per thread, per warp and over the warps (so the
//     forces are bit-reproducible);
//  5. the particle enters the screening grid of this step's update.
template <typename T>
__device__ __forceinline__ void links_body(const Dev &D, T *A, const int *__restrict__ own,
                                           int *__restrict__ own_nxt, int parity, const int p, const int pa)
{
    using E = Elem<T>;
    extern __shared__ __align__(16) unsigned char lsm[];
    __shared__ int s_nvalid;
    __shared__ unsigned s_over;
    __shared__ EllFrame s_ell;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const GeomRec G = D.geo_cur[p];
    const int N = G.N, cap = 12 * N - 12;
    const int X0 = G.X0, Y0 = G.Y0;
    const int base = D.slot_base[p];

    const int Nm = D.zone_max;
    const int wy = link_tile_wy(Nm), wx = link_tile_wx(Nm);
    const int XA = X0 - 2, YA = Y0 - 2, off = 2;
    unsigned long long *Fm = reinterpret_cast<unsigned long long *>(lsm); // [wy]
    unsigned long long *Om = Fm + wy;                                       // [wy]
    const int nw = link_occ_words(Nm), capm = 12 * Nm - 12;
    unsigned *occ = reinterpret_cast<unsigned *>(Om + wy); // [nw]
    unsigned *pre = occ + nw;                               // [nw]
    int *info = reinterpret_cast<int *>(pre + nw);          // [cap] k | a << 4 | b << 12 of the slot's link
    int *list = info + capm;                                // [cap] valid slots in order

    // ---- 0. the screening grid the particle update fills next: this CTA's
    // slice of its counts; the owner map the raster fills next (positions
    // n + 1) still holds positions n - 1: clear this particle's zone of that
    // time
    clear_cells_slice(D, parity, p, tid, kLinkThreads);
    revert_newborn(D, p, tid, kLinkThreads);
    {
        const GeomRec Gp = D.geo_prev[p];
        for (int r = warp; r < Gp.N; r += kLinkThreads / 32) {
            const int j = Gp.Y0 + r;
            if (j < 0 || j >= D.ny) continue;
            for (int c = lane; c < Gp.N; c += 32) {
                const int i = Gp.X0 + c;
                if (i >= 0 && i < D.nx) own_nxt[(long long)j * D.nx + i] = -1;
            }
        }
    }

    // ---- 1. owner masks (all warps) and the look-ahead prefetch
    if (tid == 0) {
        s_over = 0u;
        const DiskDF d0 = geom_df(G);
        D.pos4[p] = make_float4(d0.xh, d0.yh, d0.xl, d0.yl);
        D.prc[p] = make_float2(G.r, G.C);
        if (G.r < 0.f) s_ell = ell_frame(D.cur.x[p], D.cur.y[p], D.cur.th[p], D.cur.r[p], D.cur.b[p]);
    }
    {
        // owner rows in chunks of four per warp, all four loads issued before
        // the first ballot, so a chunk costs one memory latency
        constexpr int kW = kLinkThreads / 32;
        for (int r0 = 0; r0 < wy; r0 += 4 * kW) {
            int vlo[4], vhi[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int r = r0 + warp + t * kW, j = YA + r, i = XA + lane;
                vlo[t] = (r < wy && inside(D, i, j)) ? own[(long long)j * D.nx + i] : -2;
                vhi[t] = (wx > 32 && r < wy && inside(D, i + 32, j)) ? own[(long long)j * D.nx + i + 32] : -2;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (r0 + t * kW >= wy) break; // no warp has a row left
                const int r = r0 + warp + t * kW;
                const unsigned lo_f = __ballot_sync(0xffffffffu, vlo[t] == -1);
                const unsigned lo_o = __ballot_sync(0xffffffffu, vlo[t] == p);
                unsigned hi_f = 0u, hi_o = 0u;
                if (wx > 32) {
                    hi_f = __ballot_sync(0xffffffffu, vhi[t] == -1);
                    hi_o = __ballot_sync(0xffffffffu, vhi[t] == p);
                }
                if (lane == 0 && r < wy) {
                    Fm[r] = ((unsigned long long)hi_f << 32) | lo_f;
                    Om[r] = ((unsigned long long)hi_o << 32) | lo_o;
                }
            }
        }
    }
    // L2 prefetch of the owner rows of particle pa, the one a residency wave
    // later in launch order (none: pa < 0)
    if (warp == 1 && pa >= 0) {
        const GeomRec Ga = D.geo_cur[pa];
        const int xa = Ga.X0 - 2, ya = Ga.Y0 - 2;
        for (int r = lane; r < 2 * wy; r += 32) {
            const int j = ya + (r >> 1), i = min(max(xa + (r & 1) * (wx - 1), 0), D.nx - 1);
            if (j >= 0 && j < D.ny)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(own + (long long)j * D.nx + i) : "memory");
        }
    }
    for (int w = tid; w < nw; w += kLinkThreads) occ[w] = 0u;
    __syncthreads();

    // ---- 2. link detection: item (k, b), one mask intersection per row;
    // items run direction-major.  A warp's links are spread evenly over its
    // lanes (a prefix sum of the items' bit counts; lane j takes the j-th
    // link of the warp), since a few rows (the flat top and bottom of a disk
    // for e2 / e4) hold many links and most hold one
    {
        const unsigned F = 0xffffffffu;
        const unsigned long long Z = ((1ull << N) - 1ull) << off;
        for (int e0 = warp * 32; e0 < 8 * N; e0 += kLinkThreads) {
            const int e = e0 + lane;
            unsigned long long m = 0ull;
            int k = 1, b = 0;
            if (e < 8 * N) {
                k = 1 + e / N;
                b = e - (k - 1) * N;
                const int kx = ex(k), ky = ey(k);
                const unsigned long long o = Om[b + 2 + ky];
                m = Fm[b + 2] & (kx > 0 ? o >> 1 : kx < 0 ? o << 1 : o) & Z;
            }
            const int cnt = __popcll(m);
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(F, inc, o);
                if (lane >= o) inc += t;
            }
            const int total = __shfl_sync(F, inc, 31), excl = inc - cnt;
            for (int j0 = 0; j0 < total; j0 += 32) {
                const int j = j0 + lane;
                // the item holding link j: the last lane whose first link is
                // at or before j
                int l = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int ec = __shfl_sync(F, excl, l + step);
                    if (ec <= j) l += step;
                }
                unsigned long long ml = __shfl_sync(F, m, l);
                const int kl = __shfl_sync(F, k, l), bl = __shfl_sync(F, b, l), el = __shfl_sync(F, excl, l);
                if (j >= total) continue;
                for (int t = j - el; t > 0; --t) ml &= ml - 1ull; // drop the lower links of the item
                const int a = (__ffsll((long long)ml) - 1) - off;
                const int sl = slot_of(kl, a, bl, N);
                if (sl < 0) {
                    s_over = 1u;
                    continue;
                }
                const unsigned bit = 1u << (sl & 31);
                if (atomicOr(&occ[sl >> 5], bit) & bit) s_over = 1u;
                else info[sl] = kl | (a << 4) | (bl << 12);
            }
        }
    }
    __syncthreads();

    // ---- 3. compaction of the occupied slots in slot order
    const int nwp = (cap + 31) >> 5;
    if (warp == 0) {
        const unsigned c = lane < nwp ? (unsigned)__popc(occ[lane]) : 0u;
        unsigned inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane < nwp) pre[lane] = inc - c;
        if (lane == 31) s_nvalid = (int)inc;
    }
    __syncthreads();
    const int nvalid = s_nvalid;
    for (int sl = tid; sl < cap; sl += kLinkThreads) {
        const unsigned w = occ[sl >> 5], bit = 1u << (sl & 31);
        if (w & bit) list[pre[sl >> 5] + __popc(w & (bit - 1u))] = sl;
        else if (in_bounds(D, (long long)base + sl, D.nslots)) {
            D.slot_node[base + sl] = -1;
            D.slot_q[base + sl] = 0.f;
        }
    }
    __syncthreads();

    // ---- 4. bounce-back and momentum exchange, thread i on the i-th link
    const DiskDF dk = geom_df(G);
    const bool ell = G.r < 0.f; // an ellipse: q in FP64
    const float Ux = G.ux, Uy = G.uy, Om_ = G.om, wT = G.wT;
    // populations of fluid nodes: no CTA writes them during this kernel
    const T *Ar = A;
    auto tv = [&](int plane, int i, int j) -> float {
        const long long e = (long long)plane * D.ps + (long long)j * D.pitch + i;
        return in_bounds(D, e, D.a_elems) ? E::ld(__ldg(Ar + e)) : 0.f;
    };
    auto fluid = [&](int i, int j) -> bool { return (Fm[j - YA] >> (i - XA)) & 1ull; };
    // one round per kLinkThreads links: every warp sums its round at once
    // (exact integer sums), lane 0 adds it to the warp's total; no
    // accumulator stays live across rounds
    __shared__ LinkSums s_ws[kLinkThreads / 32];
    __shared__ int s_wc[kLinkThreads / 32][3];
    const int rounds = (nvalid + kLinkThreads - 1) / kLinkThreads;
    for (int it = 0; it < rounds; ++it) {
        const int li = it * kLinkThreads + tid;
        LinkAcc acc;
        if (li < nvalid) {
            const int sl = list[li];
            const int inf = info[sl], k = inf & 15;
            const int kx = ex(k), ky = ey(k);
            const int fi = X0 + ((inf >> 4) & 255), fj = Y0 + (inf >> 12);
            float dxf, dyf;
            const float q = ell ? link_q_ellipse(fi, fj, k, s_ell, dxf, dyf) : link_q_df(fi, fj, k, dk, dxf, dyf);
            if (in_bounds(D, (long long)base + sl, D.nslots)) {
                D.slot_node[base + sl] = fj * D.nx + fi;
                D.slot_q[base + sl] = q;
            }

            // curved bounce-back in deviation form: every rule is an affine
            // combination of populations of equal weight, so it holds for
            // f~ = f - w unchanged
            const int kb = opp(k);
            const int i1 = fi - kx, j1 = fj - ky, i2 = fi - 2 * kx, j2 = fj - 2 * ky;
            const bool have1 = fluid(i1, j1);
            const bool have2 = fluid(i2, j2);
            const int ii1 = have1 ? i1 : fi, jj1 = have1 ? j1 : fj;
            const int ii2 = have2 ? i2 : fi, jj2 = have2 ? j2 : fj;
            const float fk0 = tv(k, fi, fj), fk1 = tv(k, ii1, jj1), fk2 = tv(k, ii2, jj2);
            const float fb0 = tv(kb, fi, fj), fb1 = tv(kb, ii1, jj1);
            const float rx = dxf + q * kx, ry = dyf + q * ky;
            const float uwx = Ux - Om_ * ry, uwy = Uy + Om_ * rx;
            const float wall = 6.f * w9(k) * -(kx * uwx + ky * uwy); // 2 w rho0 e_kbar.u_w / c_s^2
            int lvl;
            const float fnew = bouzidi32(q, fk0, fk1, fk2, fb0, fb1, have1, have2, wall, lvl);
            const long long ns = (long long)(fj + ky) * D.pitch + (fi + kx);
            if (in_bounds(D, kb * D.ps + ns, D.a_elems)) A[kb * D.ps + ns] = E::st(fnew);
            if (k <= 4) {
                const float gnew = thermal32(q, tv(kQ9 + k, fi, fj), tv(kQ9 + k, ii1, jj1),
                                             tv(kQ9 + kb, fi, fj), have1, wT);
                if (in_bounds(D, (kQ9 + kb) * D.ps + ns, D.a_elems)) A[(kQ9 + kb) * D.ps + ns] = E::st(gnew);
            }
            // momentum exchange: with f = w + f~ the bracket of Eq. force is
            // 2 w_k e_k + [f~_k^+ (e_k - u_w) - f~_kbar (e_kbar - u_w)]; the
            // constant part and its torque 2 w_k ((i - x_c) e_k,y - (j - y_c) e_k,x)
            // (q drops out) are kept as exact integer sums, assembled in FP64 by
            // the particle update
            const float bx = fk0 * (kx - uwx) - fnew * (-kx - uwx);
            const float by = fk0 * (ky - uwy) - fnew * (-ky - uwy);
            acc.add(bx, by, rx * by - ry * bx, k, lvl, k <= 4 && !have1, fi * ky - fj * kx);
        }
        LinkSums Sw;
        int c3w[3];
        acc.finish(Sw, c3w);
        if (lane == 0) {
            if (it == 0) {
                s_ws[warp] = Sw;
                s_wc[warp][0] = c3w[0]; s_wc[warp][1] = c3w[1]; s_wc[warp][2] = c3w[2];
            } else {
                add_sums(s_ws[warp], Sw);
                s_wc[warp][0] += c3w[0]; s_wc[warp][1] += c3w[1]; s_wc[warp][2] += c3w[2];
            }
        }
    }
    if (rounds == 0 && lane == 0) { // no link
        LinkSums Sz;
        Sz.fx = Sz.fy = Sz.tz = 0;
        Sz.ax_x = Sz.ax_y = Sz.ax_t = Sz.dg_x = Sz.dg_y = Sz.dg_t = 0;
        s_ws[warp] = Sz;
        s_wc[warp][0] = s_wc[warp][1] = s_wc[warp][2] = 0;
    }
    // ---- 5. the particle's sums over the warps (exact integer sums, so the
    // grouping does not matter)
    __syncthreads();
    if (tid == 0) {
        LinkSums S = s_ws[0];
        int c3[3] = {s_wc[0][0], s_wc[0][1], s_wc[0][2]};
#pragma unroll
        for (int w = 1; w < kLinkThreads / 32; ++w) {
            add_sums(S, s_ws[w]);
            c3[0] += s_wc[w][0]; c3[1] += s_wc[w][1]; c3[2] += s_wc[w][2];
        }
        {
            D.lsum[p] = S;
            unsigned long long *C = D.status->cnt[parity];
            if (c3[0]) atomicAdd(&C[kCntBzLinear], (unsigned long long)c3[0]);
            if (c3[1]) atomicAdd(&C[kCntBzSimple], (unsigned long long)c3[1]);
            if (c3[2]) atomicAdd(&C[kCntThermHalf], (unsigned long long)c3[2]);
            if (nvalid) atomicAdd(&C[kCntLinks], (unsigned long long)nvalid);
            if (s_over) atomicOr(&D.status->err, kErrOverflow);
        }
    }
    // the particle's position into the screening grid this step's update
    // reads (its counts cleared by the previous step's link kernel): the
    // atomic's round trip ends the CTA instead of lengthening the update
    if (tid == 32) cell_insert(D, D.cells[parity], p, G.xh, G.yh);
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
// Each block takes 8 particles: warp w screens particle w against the
// particles listed in the 3 x 3 cells of the screening grid around its cell
// (filled with the step's starting positions by the link kernel; every
// pair in reach is among them), or, when a cell of that grid overflowed,
// against all particles in shared-memory tiles of 1600, and evaluates the
// pairs in reach from double-float centre differences, summed in 64-bit
// fixed point so that the result is the same whichever way the pairs were
// found and in whatever order; lane l of warp 0 then sums, integrates and
// stores particle l in FP64 (its constants 1/M, 1/I, W and C, and its
// geometry record, staged by the last warp while the others screen), and
// warp w rasters particle w.  Small
// blocks let four of them share an SM, so that the latency of one block's
// loads and FP64 tail overlaps the others' work.  Integration:
// U' = U + F/M, X' = X + (U + U')/2, Omega' = Omega + T/I,
// theta' = theta + (Omega + Omega')/2 with M = rho_p pi r^2 and I = M r^2 / 2
// (M = rho_p pi r b and I = M (r^2 + b^2) / 4 for an ellipse).
constexpr int kPartTile = 1600;
constexpr int kPartPerBlock = kPartThreads / 32;

// Support distance of particle p along the unit vector (nx, ny): its radius
// for a disk.
__device__ __forceinline__ double support_of(const Dev &D, int p, double nx, double ny)
{
    const double r = D.cur.r[p], b = D.cur.b[p];
    if (!is_ellipse(r, b)) return r;
    return ell_support(ell_frame(0.0, 0.0, D.cur.th[p], r, b), nx, ny);
}

// Pair repulsion on particle a from particle b when either is an ellipse, in
// FP64: the gap along the line of centres is the centre distance minus both
// support distances along it.
__device__ __noinline__ void pair_force_ellipse(const Dev &D, int a, int b, long long &sx, long long &sy)
{
    const double dx = D.cur.x[a] - D.cur.x[b], dy = D.cur.y[a] - D.cur.y[b];
    const double dist = sqrt(dx * dx + dy * dy);
    const double gap = dist - support_of(D, a, -dx / dist, -dy / dist) - support_of(D, b, dx / dist, dy / dist);
    if (gap > D.s_rep) return;
    auto scale = [&](int p) {
        const double r = D.cur.r[p], pb = D.cur.b[p];
        return kPi * r * (is_ellipse(r, pb) ? pb : r) * (D.cur.rho[p] - D.rho_f) * D.g;
    };
    const double mag = repulsion(gap, D.s_rep, D.eps_w, 0.5 * (scale(a) + scale(b)));
    sx += fix_of(mag * dx / dist);
    sy += fix_of(mag * dy / dist);
}

// Pair repulsion on disk a from disk b (FP32 from double-float centres).
__device__ __noinline__ void pair_force(float4 pa, float2 ca, float4 pb, float2 cb, float s_rep,
                                        float inv_eps, long long &sx, long long &sy)
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
    sx += fix_of(mag * dx / dist);
    sy += fix_of(mag * dy / dist);
}

// Screening of particle a (position pa, (r, C) ca) against candidate b:
// circumscribed circles within reach (r < 0 marks an ellipse), then the
// pair force.
__device__ __forceinline__ void screen_pair(const Dev &D, int a, float4 pa, float2 ca, int b, float4 pb, float2 cb,
                                            float s_rep, float inv_eps, long long &sx, long long &sy)
{
    const float dxf = pa.x - pb.x, dyf = pa.y - pb.y, lim = fabsf(ca.x) + fabsf(cb.x) + s_rep + 1.f;
    if (dxf * dxf + dyf * dyf > lim * lim || b == a) return;
    if (ca.x < 0.f || cb.x < 0.f) pair_force_ellipse(D, a, b, sx, sy);
    else pair_force(pa, ca, pb, cb, s_rep, inv_eps, sx, sy);
}

// Zone of a disk at (x, y) with radius r: N x N nodes from
// (floor(x - r) - 1, floor(y - r) - 1); it holds every node of the disk and
// every fluid node linked to it.
struct Box {
    int X0, Y0, N;
};
__device__ __forceinline__ Box box_of(const GeomRec &G) { return Box{G.X0, G.Y0, G.N}; }

// Writes of a warp's raster: lane l holds the run [lo, hi] of zone row
// b0 + l (empty when lo > hi); the warp then stores row after row, lanes on
// consecutive nodes, so each row's atomicMax requests coalesce.
__device__ __forceinline__ void write_runs(const Dev &D, int *own, const Box &B, int b0, int lo, int hi, int p)
{
    const int lane = threadIdx.x & 31, nr = min(32, B.N - b0);
    for (int r = 0; r < nr; ++r) {
        const int l = __shfl_sync(0xffffffffu, lo, r), h = __shfl_sync(0xffffffffu, hi, r);
        const long long j0 = (long long)(B.Y0 + b0 + r) * D.nx;
        for (int i = l + lane; i <= h; i += 32)
            if (in_bounds(D, j0 + i, (long long)D.nx * D.ny)) atomicMax(own + j0 + i, p);
    }
}

// Run of row j of one ellipse.  Along a row the ellipse form is a convex
// quadratic in i, so the inside nodes form one run; when the run is not
// empty the node nearest the vertex of the parabola lies in it (checked with
// its two neighbours, against rounding of the vertex).  The run's ends are
// estimated from the quadratic's roots (FP32) and settled with the predicate
// at the ends only: FP32 outside the rounding band, the exact FP64 form
// inside it.
__device__ __noinline__ void ellipse_run(const Dev &D, const Box B, const GeomRec G, double x, double y, double th,
                                         double r, double pb, int j, int &lo_out, int &hi_out)
{
    lo_out = 1;
    hi_out = 0;
    if (j < 0 || j >= D.ny) return;
    const int xmin = B.X0, xmax = B.X0 + B.N - 1;
    const EllDF F = ell_df(G.xh, G.xl, G.yh, G.yl, G.w0, G.w1, r, pb);
    auto inside = [&](int i) -> bool {
        const int side = ell_side_df(i, j, F);
        if (side) return side < 0;
        return in_ellipse(i, j, ell_frame(x, y, th, r, pb));
    };
    const float c = F.c, s = F.s;
    const float A2 = c * c * F.b2 + s * s * F.a2; // dx^2 coefficient
    const float Bc = c * s * (F.b2 - F.a2);       // half the dx dy coefficient
    const float Cc = s * s * F.b2 + c * c * F.a2; // dy^2 coefficient
    float dyh, dyl;
    df_offset(j, G.yh, G.yl, dyh, dyl);
    const float dy = dyh + dyl;
    const float B1 = Bc * dy, C0 = Cc * dy * dy - F.ab;
    const float mid = (G.xh - B1 / A2) + G.xl;
    const int im = (int)floorf(mid + 0.5f);
    const int in = inside(im) ? im : inside(im - 1) ? im - 1 : inside(im + 1) ? im + 1 : INT_MIN;
    if (in == INT_MIN) return; // then no node of the row is inside
    const float h = sqrtf(fmaxf(B1 * B1 - A2 * C0, 0.f)) / A2;
    int lo = max(min(in, (int)ceilf(mid - h)), xmin), hi = min(max(in, (int)floorf(mid + h)), xmax);
    while (lo > xmin && inside(lo - 1)) --lo;
    while (!inside(lo)) ++lo;
    while (hi < xmax && inside(hi + 1)) ++hi;
    while (!inside(hi)) --hi;
    lo_out = max(lo, 0);
    hi_out = min(hi, D.nx - 1);
}

// Run of row j of one disk: the node nearest the centre decides whether the
// row meets the disk; the ends come from an FP32 estimate settled with the
// exact predicate.
__device__ __forceinline__ void disk_run(const Dev &D, const Box &B, const GeomRec &G, double x, double y, double r,
                                         int j, int &lo_out, int &hi_out)
{
    lo_out = 1;
    hi_out = 0;
    if (j < 0 || j >= D.ny) return;
    const DiskDF dk = geom_df(G);
    const int ic = G.ic; // the node of each row nearest the centre
    if (!in_disk_df(ic, j, dk, x, y, r)) return; // then no node of the row is inside
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
    lo_out = max(lo, 0);
    hi_out = min(hi, D.nx - 1);
}

// Raster of one particle by one warp: lane per zone row for the runs, then
// coalesced writes.  runs (may be null): the particle's row runs (lo, hi),
// empty when lo > hi, kept for the next step's flags.
__device__ __forceinline__ void raster_one(const Dev &D, int *own, const GeomRec &G, double x, double y, double r,
                                           double th, double pb, int p, int2 *runs)
{
    const int lane = threadIdx.x & 31;
    const Box B = box_of(G);
    for (int b0 = 0; b0 < B.N; b0 += 32) {
        const int j = B.Y0 + b0 + lane;
        int lo = 1, hi = 0;
        if (b0 + lane < B.N) {
            if (G.r < 0.f) ellipse_run(D, B, G, x, y, th, r, pb, j, lo, hi);
            else disk_run(D, B, G, x, y, r, j, lo, hi);
            if (runs && in_bounds(D, (long long)p * D.zone_max + b0 + lane, (long long)D.np * D.zone_max))
                runs[b0 + lane] = make_int2(lo, hi);
        }
        write_runs(D, own, B, b0, lo, hi, p);
    }
}

// Support distances of an ellipse along the wall normals x-hat and y-hat
// (kept out of line: the disk path does not carry its registers).
__device__ __noinline__ void wall_supports(double th, double r, double b, double &hx, double &hy)
{
    const EllFrame E = ell_frame(0.0, 0.0, th, r, b);
    hx = ell_support(E, 1.0, 0.0);
    hy = ell_support(E, 0.0, 1.0);
}

// New state of a particle as the raster needs it.
struct RasterIn {
    GeomRec G;
    double x, y, r, th, b;
};

// Constants of the update of a particle (they depend only on its shape and
// density): 1/M, 1/I, the buoyant weight W = (rho_p - rho_f) A g and the
// repulsion force scale C = A (rho_p - rho_f) g, with the area A = pi r^2
// (pi r b for an ellipse), M = rho_p A and I = M r^2 / 2 (M (r^2 + b^2) / 4
// for an ellipse).  The update multiplies by 1/M and 1/I, which differs
// from dividing by M and I by at most one rounding of the increment.
__device__ __forceinline__ double4 part_consts(double r, double b, double rho, double rho_f, double g)
{
    const bool ell = is_ellipse(r, b);
    const double rb = ell ? b : r;
    const double M = rho * kPi * r * rb, I = ell ? 0.25 * M * (r * r + b * b) : 0.5 * M * r * r;
    return make_double4(1.0 / M, 1.0 / I, (rho - rho_f) * kPi * r * rb * g, kPi * r * rb * (rho - rho_f) * g);
}

// FP64 tail of the particle update for particle b: total force, Newton-Euler
// step, domain checks, new state and geometry record.  (psx, psy: the pair
// repulsion in fixed point; out: the new state for the raster; st, ls, Gc, pk: the
// particle's state fields x, y, ux, uy, theta, omega, r, rho, T, b, its link
// sums, its current geometry record and its constants, staged in shared
// memory during the screening.)
__device__ __forceinline__ void particle_tail(const Dev &D, int b, int parity, long long psx, long long psy, RasterIn &out,
                                              const double *st, const LinkSums &ls, const GeomRec &Gc,
                                              const double4 &pk)
{
    double x = st[0], y = st[1], ux = st[2], uy = st[3];
    double th = st[4], om = st[5];
    const double r = st[6], rho = st[7], pb = st[9];
    // an ellipse: wall gaps to its support distances along the wall normals
    const bool ell = is_ellipse(r, pb);
    double Fx, Fy, Tz;
    if (D.direct) {
        const DirectSums &ds = D.dsum[b];
        LinkSums S;
        S.fx = fix_force(ds.f[0]);
        S.fy = fix_force(ds.f[1]);
        S.tz = fix_torque(ds.f[2]);
        S.ax_x = ds.c[0]; S.ax_y = ds.c[1]; S.ax_t = ds.c[2];
        S.dg_x = ds.c[3]; S.dg_y = ds.c[4]; S.dg_t = ds.c[5];
        assemble_force(S, x, y, Fx, Fy, Tz);
    } else {
        assemble_force(ls, x, y, Fx, Fy, Tz);
    }
    D.force[3 * b + 0] = Fx;
    D.force[3 * b + 1] = Fy;
    D.force[3 * b + 2] = Tz;
    const double Cb = pk.w;
    Fy -= pk.z;
    double hx = r, hy = r;
    if (ell) wall_supports(th, r, pb, hx, hy);
    // A wall gap takes the FP64 repulsion only where the FP32 centre of the
    // current geometry record puts it within the threshold plus a margin
    // (mar) far above that centre's rounding error (half an FP32 spacing,
    // 2.4e-4 at 4096): elsewhere the repulsion is zero either way, and GB300
    // runs FP64 at a small fraction of its FP32 rate.
    const float mar = 1e-3f + 2.4e-7f * (float)(D.nx + D.ny), near = (float)D.s_rep + mar;
    const float hxf = (float)hx, hyf = (float)hy, nxf = (float)D.nx, nyf = (float)D.ny;
    if (!D.per_x) {
        if ((Gc.xh + 0.5f) - hxf <= near) Fx += repulsion((x + 0.5) - hx, D.s_rep, D.eps_w, Cb);
        if ((nxf - 0.5f - Gc.xh) - hxf <= near) Fx -= repulsion(((double)D.nx - 0.5 - x) - hx, D.s_rep, D.eps_w, Cb);
    }
    if (!D.per_y) {
        if ((Gc.yh + 0.5f) - hyf <= near) Fy += repulsion((y + 0.5) - hy, D.s_rep, D.eps_w, Cb);
        if ((nyf - 0.5f - Gc.yh) - hyf <= near) Fy -= repulsion(((double)D.ny - 0.5 - y) - hy, D.s_rep, D.eps_w, Cb);
    }
    if (psx) Fx += fix_value(psx);
    if (psy) Fy += fix_value(psy);
    if (!D.fixed) {
        const double ux1 = ux + Fx * pk.x, uy1 = uy + Fy * pk.x, om1 = om + Tz * pk.y;
        x += 0.5 * (ux + ux1);
        y += 0.5 * (uy + uy1);
        th += 0.5 * (om + om1);
        ux = ux1;
        uy = uy1;
        om = om1;
    }
    // a disk that would leave the cavity, move a node or more in one step
    // (beyond the reach of the near-tile bitmap), or whose state is no longer
    // finite raises the (sticky) domain error and stays where it was, so that
    // its zone stays inside the arrays every later kernel indexes
    // (decided in FP32 with the margin mar where that is certain, else in
    // FP64; a non-finite state fails both)
    const double xo = st[0], yo = st[1];
    const float xf = (float)x, yf = (float)y, rf = (float)r;
    const bool surely_in = xf - rf >= mar - 0.5f && xf + rf <= nxf - 0.5f - mar && yf - rf >= mar - 0.5f &&
                           yf + rf <= nyf - 0.5f - mar && fabsf(xf - Gc.xh) < 1.f - mar &&
                           fabsf(yf - Gc.yh) < 1.f - mar;
    if (!surely_in && !(x - r >= -0.5 && x + r <= (double)D.nx - 0.5 && y - r >= -0.5 && y + r <= (double)D.ny - 0.5 &&
                        fabs(x - xo) < 1.0 && fabs(y - yo) < 1.0)) {
        atomicOr(&D.status->err, kErrDomain);
        x = xo;
        y = yo;
    }
    const double T = st[8];
    D.nxt.x[b] = x; D.nxt.y[b] = y; D.nxt.ux[b] = ux; D.nxt.uy[b] = uy; D.nxt.th[b] = th;
    D.nxt.om[b] = om; D.nxt.r[b] = r; D.nxt.rho[b] = rho; D.nxt.T[b] = T; D.nxt.b[b] = pb;
    const GeomRec Gn = move_geom(Gc, x, y, r, pb, th, ux, uy, om);
    D.geo_nxt[b] = Gn;
    out.G = Gn;
    out.x = x; out.y = y; out.r = r; out.th = th; out.b = pb;
}

__device__ __forceinline__ void particles_body(const Dev &D, int parity, int *own_nxt, const int blk)
{
    __shared__ float4 sp[kPartTile];
    __shared__ float2 sc[kPartTile];
    __shared__ long long sred[2][kPartPerBlock];
    __shared__ RasterIn sras[kPartPerBlock]; // the tail's results, handed to the raster warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a = blk * kPartPerBlock + warp;
    if (blk == 0 && threadIdx.x < kNumCounters) D.status->cnt[parity ^ 1][threadIdx.x] = 0ull;
    if (blk == 0 && threadIdx.x == 0) D.status->nb = 0u;
    const bool me = a < D.np;
    // the last warp stages the tail's inputs (the block's particle states and
    // link sums) while every warp screens, so that the FP64 tail starts
    // without a global round trip
    __shared__ double s_cur[kPartPerBlock][kPartFields];
    __shared__ LinkSums s_ls[kPartPerBlock];
    __shared__ GeomRec s_geo[kPartPerBlock];
    __shared__ double4 s_pk[kPartPerBlock];
    if (warp == kPartPerBlock - 1) {
        for (int t = lane; t < kPartPerBlock * kPartFields; t += 32) {
            const int q = t / kPartFields, f = t - q * kPartFields, bq = blk * kPartPerBlock + q;
            if (bq < D.np) s_cur[q][f] = D.cur.x[(long long)f * D.np + bq];
        }
        static_assert(sizeof(GeomRec) == 64, "a geometry record is 16 words");
        for (int t = lane; t < kPartPerBlock * 16; t += 32) {
            const int q = t >> 4, w = t & 15, bq = blk * kPartPerBlock + q;
            if (bq < D.np) reinterpret_cast<int *>(&s_geo[q])[w] = reinterpret_cast<const int *>(&D.geo_cur[bq])[w];
        }
        if (lane < kPartPerBlock && blk * kPartPerBlock + lane < D.np) s_pk[lane] = D.pconst[blk * kPartPerBlock + lane];
        if (!D.direct)
            for (int t = lane; t < kPartPerBlock * 8; t += 32) {
                const int q = t >> 3, w = t & 7, bq = blk * kPartPerBlock + q;
                if (bq < D.np) reinterpret_cast<long long *>(&s_ls[q])[w] = reinterpret_cast<const long long *>(&D.lsum[bq])[w];
            }
    }
    float4 pa = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 ca = make_float2(1.f, 0.f);
    if (me) {
        pa = D.pos4[a];
        ca = D.prc[a];
    }
    const float s_rep = (float)D.s_rep, inv_eps = (float)(1.0 / D.eps_w);
    long long sx = 0, sy = 0; // pair repulsion, fixed point
    const int *grid = D.cells[parity];
    const int gx = D.cell_gx, gy = D.cell_gy, ncell = gx * gy;
    if (!grid[ncell] && !D.all_pairs) {
        // candidates from the 3 x 3 cells around a's cell: lane l < 9 holds
        // cell l's count; candidate t goes to lane t mod 32
        int cnt = 0, cell = 0;
        if (me && lane < 9) {
            const int c0 = cell_of(D, pa.x, pa.y);
            const int cx = c0 % gx + lane % 3 - 1, cy = c0 / gx + lane / 3 - 1;
            if (cx >= 0 && cx < gx && cy >= 0 && cy < gy) {
                cell = cy * gx + cx;
                cnt = min(__ldg(grid + cell), kCellCap);
            }
        }
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const int total = __shfl_sync(0xffffffffu, inc, 8), excl = inc - cnt;
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int b = -1;
#pragma unroll
            for (int l = 0; l < 9; ++l) {
                const int e = __shfl_sync(0xffffffffu, excl, l), n = __shfl_sync(0xffffffffu, cnt, l);
                const int c = __shfl_sync(0xffffffffu, cell, l);
                if (t >= e && t < e + n) b = __ldg(grid + ncell + 1 + c * kCellCap + (t - e));
            }
            if (b >= 0) screen_pair(D, a, pa, ca, b, D.pos4[b], D.prc[b], s_rep, inv_eps, sx, sy);
        }
    } else {
        // a cell overflowed: every pair, in shared-memory tiles
        for (int t0 = 0; t0 < D.np; t0 += kPartTile) {
            const int nb = min(kPartTile, D.np - t0);
            __syncthreads();
#pragma unroll 8
            for (int k = threadIdx.x; k < nb; k += kPartThreads) {
                sp[k] = D.pos4[t0 + k];
                sc[k] = D.prc[t0 + k];
            }
            __syncthreads();
            if (!me) continue;
            for (int u = lane; u < nb; u += 32) screen_pair(D, a, pa, ca, t0 + u, sp[u], sc[u], s_rep, inv_eps, sx, sy);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
        sred[0][warp] = sx;
        sred[1][warp] = sy;
    }
    __syncthreads();
    const int b = blk * kPartPerBlock + lane;
    if (warp == 0 && lane < kPartPerBlock && b < D.np)
        particle_tail(D, b, parity, sred[0][lane], sred[1][lane], sras[lane], s_cur[lane], s_ls[lane],
                      s_geo[lane], s_pk[lane]);
    // then the owner map at the new positions: warp w rasters the block's
    // particle w (its own new state only, so no other block is waited for)
    __syncthreads();
    if (a < D.np) {
        const RasterIn &R = sras[warp];
        raster_one(D, own_nxt, R.G, R.x, R.y, R.r, R.th, R.b, a, D.runs[parity ^ 1] + (long long)a * D.zone_max);
    }
}



// Owner map: node (i,j) belongs to disk p iff (i - x)^2 + (j - y)^2 <= r^2
// (exact FP64; for an ellipse u^2 b^2 + v^2 a^2 <= a^2 b^2 in its frame);
// where particles overlap the highest index wins (atomicMax, so
// the result does not depend on the launch order).  One warp per particle,
// one lane per zone row: the predicate holds on one contiguous run of each
// row (it is monotone in |i - x|), so the run is found from an FP32 estimate
// of its ends and settled with the exact predicate at the ends only; the
// runs are then written row by row with coalesced atomicMax requests.

__device__ __forceinline__ void raster_body(const Dev &D, int *own, const GeomRec *__restrict__ geo,
                                            const PartSoA &pos, int2 *runs, const int blk)
{
    const int p = blk * (kBoxThreads / 32) + (threadIdx.x >> 5);
    if (p >= D.np) return;
    raster_one(D, own, geo[p], pos.x[p], pos.y[p], pos.r[p], pos.th[p], pos.b[p], p,
               runs ? runs + (long long)p * D.zone_max : nullptr);
}

// Class of a node from the two owner maps: solid at the new time, newborn
// (solid before, fluid now) or fluid.
__device__ __forceinline__ uint8_t node_class(int oc, int on) { return on >= 0 ? kSolid : oc >= 0 ? kNewborn : kFluid; }

// A newborn node into this step's list (j * nx + i off the cavity frame,
// ~(j * nx + i) on it, where the general path takes it anyway).
__device__ __forceinline__ void list_newborn(const Dev &D, int i, int j)
{
    const unsigned at = atomicAdd(&D.status->nb, 1u);
    const int n = j * D.nx + i;
    const bool frame = i == 0 || i == D.nx - 1 || j == 0 || j == D.ny - 1;
    if (at < (unsigned)D.newborn_cap) D.newborn[at] = frame ? ~n : n;
    else atomicOr(&D.status->err, kErrOverflow);
}

// Nodes of run [lo, hi] of row j outside run [xlo, xhi] (one or two
// intervals; all of it when [xlo, xhi] is empty), in order.
template <typename F>
__device__ __forceinline__ void run_minus(int lo, int hi, int xlo, int xhi, F &&f)
{
    if (xlo > xhi) {
        for (int i = lo; i <= hi; ++i) f(i);
        return;
    }
    for (int i = lo; i <= min(hi, xlo - 1); ++i) f(i);
    for (int i = max(lo, xhi + 1); i <= hi; ++i) f(i);
}

// Node flags of a step.  Before it, every node holds its class for the
// previous step (the link kernel has returned that step's newborn nodes to
// fluid); a node's class can only change where it enters or leaves a
// particle, so the team of particle p visits, row by row, the nodes of its
// disk at the new position outside its disk at the current one (solid now:
// every disk holding a node writes the same class) and the nodes of its
// current disk outside the new one (solid if another particle now holds
// them, else newborn, listed once, by the particle that owned the node),
// from the row runs the rasters kept.  A team of TEAM warps per particle
// (one warp when the particles alone fill the GPU, else 2 or 4), lane l on
// rows l, l + 32 TEAM, ...  Team warp 0 also moves the particle's new state
// into the current slot and keeps the old position for the next clear.
// Initialisation (rotate == 0): every node of the zone rectangle from the
// owner map (own_cur == own_nxt), nothing listed.
template <int TEAM>
__device__ __forceinline__ void flags_body(const Dev &D, const int *__restrict__ own_cur,
                                           const int *__restrict__ own_nxt, int rotate, int parity, const int p)
{
    const int lane = threadIdx.x & 31, tw = (threadIdx.x >> 5) % TEAM;
    // a team past the last particle still reaches the block barrier below
    const bool act = p < D.np; // uniform across the team
    Box Bb{0, 0, 0}, Bc{0, 0, 0};
    if (act) {
        Bb = box_of(D.geo_cur[p]);
        Bc = box_of(D.geo_nxt[p]);
    }
    if (rotate) {
        // the new state moves into the current slot (and the current position
        // into the previous one) while the other threads work on the flags;
        // every thread of the team has read the boxes before
        if (TEAM == 1) __syncwarp();
        else __syncthreads();
        if (act && tw == 0) switch (lane) {
        case 0: D.px[p] = D.cur.x[p]; D.cur.x[p] = D.nxt.x[p]; break;
        case 1: D.py[p] = D.cur.y[p]; D.cur.y[p] = D.nxt.y[p]; break;
        case 2: D.cur.ux[p] = D.nxt.ux[p]; break;
        case 3: D.cur.uy[p] = D.nxt.uy[p]; break;
        case 4: D.cur.th[p] = D.nxt.th[p]; break;
        case 5: D.cur.om[p] = D.nxt.om[p]; break;
        case 6: D.geo_prev[p] = D.geo_cur[p]; D.geo_cur[p] = D.geo_nxt[p]; break;
        default: break;
        }
    }
    if (!act) return;
    const long long nflags = (long long)D.ny * D.pitch;
    if (!rotate) {
        // every node of the zone (one position: own_cur == own_nxt)
        for (int r = tw; r < Bb.N; r += TEAM) {
            const int j = Bb.Y0 + r;
            if (j < 0 || j >= D.ny) continue;
            for (int c = lane; c < Bb.N; c += 32) {
                const int i = Bb.X0 + c;
                if (i < 0 || i >= D.nx) continue;
                const int n = j * D.nx + i;
                const long long o = (long long)j * D.pitch + i;
                if (in_bounds(D, o, nflags)) D.flags[o] = node_class(own_cur[n], own_nxt[n]);
            }
        }
        return;
    }
    const int2 *Ro = D.runs[parity] + (long long)p * D.zone_max;     // current position
    const int2 *Rn = D.runs[parity ^ 1] + (long long)p * D.zone_max; // new position
    const int ylo = min(Bb.Y0, Bc.Y0), yhi = max(Bb.Y0 + Bb.N, Bc.Y0 + Bc.N);
    for (int j = ylo + tw * 32 + lane; j < yhi; j += TEAM * 32) {
        if (j < 0 || j >= D.ny) continue;
        int2 o = make_int2(1, 0), w = make_int2(1, 0);
        if (j - Bb.Y0 >= 0 && j - Bb.Y0 < Bb.N) o = Ro[j - Bb.Y0];
        if (j - Bc.Y0 >= 0 && j - Bc.Y0 < Bc.N) w = Rn[j - Bc.Y0];
        const long long row = (long long)j * D.pitch;
        // entering the particle: solid at the new time
        run_minus(w.x, w.y, o.x, o.y, [&](int i) {
            if (in_bounds(D, row + i, nflags)) D.flags[row + i] = kSolid;
        });
        // leaving it: newborn unless another particle holds the node now
        run_minus(o.x, o.y, w.x, w.y, [&](int i) {
            const int n = j * D.nx + i;
            const int oc = own_cur[n];
            const uint8_t f = node_class(oc, own_nxt[n]);
            if (in_bounds(D, row + i, nflags)) D.flags[row + i] = f;
            if (f == kNewborn && oc == p) list_newborn(D, i, j);
        });
    }
}

// Near-tile bitmap: every warp tile (one row, 32 V nodes) that meets a
// particle's zone at the current position widened by kNearMargin nodes.  One
// thread per particle and zone row; the bitmap is cleared beforehand.
__global__ void __launch_bounds__(128) k_near_mask(const Dev D, int span)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int Nm = D.zone_max + 2 * kNearMargin;
    const int p = g / Nm, r = g - p * Nm;
    if (p >= D.np) return;
    const GeomRec G = D.geo_cur[p];
    const int j = G.Y0 - kNearMargin + r;
    if (r >= G.N + 2 * kNearMargin || j < 0 || j >= D.ny) return;
    const int x0 = max(G.X0 - kNearMargin, 0), x1 = min(G.X0 + G.N - 1 + kNearMargin, D.pitch - 1);
    for (int t = x0 / span; t <= x1 / span; ++t) {
        const int b = j * D.near_tpr + t;
        atomicOr(D.near + (b >> 5), 1u << (b & 31));
    }
}

// ---- direct addressing (comparison with the index array)
// Per particle: clear its zone one step back in the next owner map, return
// the last step's newborn nodes to fluid, publish its centre for the pair
// screening, zero its sums.
__global__ void __launch_bounds__(kBoxThreads) k_direct_prep(const Dev D, int *__restrict__ own_nxt, int parity)
{
    const int p = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    clear_cells_slice(D, parity, p, threadIdx.x, kBoxThreads);
    revert_newborn(D, p, threadIdx.x, kBoxThreads);
    const GeomRec Gp = D.geo_prev[p];
    for (int r = warp; r < Gp.N; r += kBoxThreads / 32) {
        const int j = Gp.Y0 + r;
        if (j < 0 || j >= D.ny) continue;
        for (int c = lane; c < Gp.N; c += 32) {
            const int i = Gp.X0 + c;
            if (i >= 0 && i < D.nx) own_nxt[(long long)j * D.nx + i] = -1;
        }
    }
    if (threadIdx.x == 0) {
        const GeomRec G = D.geo_cur[p];
        const DiskDF d0 = geom_df(G);
        D.pos4[p] = make_float4(d0.xh, d0.yh, d0.xl, d0.yl);
        D.prc[p] = make_float2(G.r, G.C);
        cell_insert(D, D.cells[parity], p, G.xh, G.yh);
    }
    if (threadIdx.x < 3) D.dsum[p].f[threadIdx.x] = 0.0;
    if (threadIdx.x < 6) D.dsum[p].c[threadIdx.x] = 0;
}

// One thread per lattice node (the straightforward mapping the paper starts
// from, Sec. 3): a fluid node tests its eight neighbours in the owner map
// and, for each one owned by a particle, applies the same wall fraction,
// bounce-back and momentum-exchange bracket as the index-array kernel, adding
// the bracket to the particle's sums with FP64 atomics.  Only nodes next to
// a disk do work, so most threads of a block idle.
template <typename T>
__global__ void __launch_bounds__(128)
    k_links_direct(const Dev D, T *A, const int *__restrict__ own, int parity)
{
    using E = Elem<T>;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    unsigned cnt[4] = {0u, 0u, 0u, 0u}; // links, linear, simple, thermal half-way
    if (i < D.nx && own[(long long)j * D.nx + i] == -1) {
        auto fluid = [&](int a, int b) {
            return a >= 0 && a < D.nx && b >= 0 && b < D.ny && own[(long long)b * D.nx + a] == -1;
        };
        auto tv = [&](int t, int a, int b) -> float {
            return E::ld(A[(long long)t * D.ps + (long long)b * D.pitch + a]);
        };
#pragma unroll 1
        for (int k = 1; k < kQ9; ++k) {
            const int kx = ex(k), ky = ey(k), si = i + kx, sj = j + ky;
            if (si < 0 || si >= D.nx || sj < 0 || sj >= D.ny) continue;
            const int p = own[(long long)sj * D.nx + si];
            if (p < 0) continue;
            const GeomRec G = D.geo_cur[p];
            float dxf, dyf;
            const float q = G.r < 0.f ? link_q_ellipse(i, j, k,
                                                       ell_frame(D.cur.x[p], D.cur.y[p], D.cur.th[p], D.cur.r[p],
                                                                 D.cur.b[p]),
                                                       dxf, dyf)
                                      : link_q_df(i, j, k, geom_df(G), dxf, dyf);
            const int kb = opp(k);
            const int i1 = i - kx, j1 = j - ky, i2 = i - 2 * kx, j2 = j - 2 * ky;
            const bool have1 = fluid(i1, j1), have2 = fluid(i2, j2);
            const int ii1 = have1 ? i1 : i, jj1 = have1 ? j1 : j;
            const int ii2 = have2 ? i2 : i, jj2 = have2 ? j2 : j;
            const float fk0 = tv(k, i, j), fk1 = tv(k, ii1, jj1), fk2 = tv(k, ii2, jj2);
            const float fb0 = tv(kb, i, j), fb1 = tv(kb, ii1, jj1);
            const float rx = dxf + q * kx, ry = dyf + q * ky;
            const float uwx = G.ux - G.om * ry, uwy = G.uy + G.om * rx;
            const float wall = 6.f * w9(k) * -(kx * uwx + ky * uwy);
            int lvl;
            const float fnew = bouzidi32(q, fk0, fk1, fk2, fb0, fb1, have1, have2, wall, lvl);
            const long long ns = (long long)sj * D.pitch + si;
            if (in_bounds(D, kb * D.ps + ns, D.a_elems)) A[kb * D.ps + ns] = E::st(fnew);
            if (k <= 4) {
                const float gnew = thermal32(q, tv(kQ9 + k, i, j), tv(kQ9 + k, ii1, jj1), tv(kQ9 + kb, i, j), have1,
                                             G.wT);
                if (in_bounds(D, (kQ9 + kb) * D.ps + ns, D.a_elems)) A[(kQ9 + kb) * D.ps + ns] = E::st(gnew);
                cnt[3] += !have1;
            }
            const float bx = fk0 * (kx - uwx) - fnew * (-kx - uwx);
            const float by = fk0 * (ky - uwy) - fnew * (-ky - uwy);
            DirectSums &ds = D.dsum[p];
            atomicAdd(&ds.f[0], (double)bx);
            atomicAdd(&ds.f[1], (double)by);
            atomicAdd(&ds.f[2], (double)(rx * by - ry * bx));
            const int tz = i * ky - j * kx, o = k <= 4 ? 0 : 3;
            if (kx) atomicAdd(&ds.c[o], kx);
            if (ky) atomicAdd(&ds.c[o + 1], ky);
            if (tz) atomicAdd(&ds.c[o + 2], tz);
            cnt[0] += 1u;
            cnt[1] += lvl == 1;
            cnt[2] += lvl == 2;
        }
    }
    // counters: one atomic per warp
    const unsigned F = 0xffffffffu;
    unsigned long long *C = D.status->cnt[parity];
    const unsigned c0 = __reduce_add_sync(F, cnt[0]), c1 = __reduce_add_sync(F, cnt[1]);
    const unsigned c2 = __reduce_add_sync(F, cnt[2]), c3 = __reduce_add_sync(F, cnt[3]);
    if ((threadIdx.x & 31) == 0) {
        if (c0) atomicAdd(&C[kCntLinks], (unsigned long long)c0);
        if (c1) atomicAdd(&C[kCntBzLinear], (unsigned long long)c1);
        if (c2) atomicAdd(&C[kCntBzSimple], (unsigned long long)c2);
        if (c3) atomicAdd(&C[kCntThermHalf], (unsigned long long)c3);
    }
}

// ---- single-instance kernels
// 16 CTAs per SM (the 2,048-thread limit; 32 registers): the kernel is
// latency-bound, and 16 particles in flight per SM instead of the 9 that 56
// registers allow beat the few spilled registers (80 against 91 us per step
// on the 4000^2 / 4800-disk benchmark).
constexpr int kLinkCtasPerSm = 16;
template <typename T>
__global__ void __launch_bounds__(kLinkThreads, kLinkCtasPerSm)
    k_links(const Dev D, T *A, const int *__restrict__ own,
            int *__restrict__ own_nxt, int parity, int ahead)
{
    // CTAs in the link order (descending y, the rows stream-collide wrote
    // last first)
    const int b = (int)blockIdx.x;
    links_body<T>(D, A, own, own_nxt, parity, __ldg(D.lorder + b), b + ahead < D.np ? __ldg(D.lorder + b + ahead) : -1);
}
__global__ void __launch_bounds__(kPartThreads, 4) k_particles(const Dev D, int parity, int *own_nxt)
{
    particles_body(D, parity, own_nxt, (int)blockIdx.x);
}
__global__ void __launch_bounds__(kBoxThreads)
    k_raster(const Dev D, int *own, const GeomRec *__restrict__ geo, const PartSoA pos, int2 *runs)
{
    raster_body(D, own, geo, pos, runs, (int)blockIdx.x);
}
template <int TEAM>
__global__ void __launch_bounds__(kBoxThreads, 9)
    k_flags(const Dev D, const int *__restrict__ own_cur, const int *__restrict__ own_nxt, int rotate, int parity)
{
    flags_body<TEAM>(D, own_cur, own_nxt, rotate, parity,
                     (int)blockIdx.x * (kBoxThreads / 32 / TEAM) + (int)(threadIdx.x >> 5) / TEAM);
}

// ---- batched kernels: one grid over all instances (InstArgs table, block
// offsets `start`).  The link kernel's look-ahead owner-row prefetch stays
// within the instance.
template <typename T>
__global__ void __launch_bounds__(kLinkThreads, kLinkCtasPerSm)
    k_links_batch(const InstArgs *__restrict__ I, const int *__restrict__ start, int n, int parity, int ahead)
{
    __shared__ Dev sD;
    const int i = batch_find(start, n, (int)blockIdx.x);
    const InstArgs &a = I[i];
    copy_dev(sD, a.D);
    const int par = parity ^ a.poff;
    const int b = (int)blockIdx.x - __ldg(start + i);
    links_body<T>(sD, static_cast<T *>(a.A[par]), a.own[par], a.own[par ^ 1], par, b, b + ahead < sD.np ? b + ahead : -1);
}
__global__ void __launch_bounds__(kPartThreads, 4)
    k_particles_batch(const InstArgs *__restrict__ I, const int *__restrict__ start, int n, int parity)
{
    __shared__ Dev sD;
    const int i = batch_find(start, n, (int)blockIdx.x);
    copy_dev(sD, I[i].D);
    const int par = parity ^ I[i].poff;
    particles_body(sD, par, I[i].own[par ^ 1], (int)blockIdx.x - __ldg(start + i));
}
__global__ void __launch_bounds__(kBoxThreads)
    k_raster_batch(const InstArgs *__restrict__ I, const int *__restrict__ start, int n, int parity)
{
    __shared__ Dev sD;
    const int i = batch_find(start, n, (int)blockIdx.x);
    const InstArgs &a = I[i];
    copy_dev(sD, a.D);
    raster_body(sD, a.own[parity ^ a.poff ^ 1], sD.geo_nxt, sD.nxt, sD.runs[parity ^ a.poff ^ 1],
                (int)blockIdx.x - __ldg(start + i));
}
__global__ void __launch_bounds__(kBoxThreads)
    k_flags_batch(const InstArgs *__restrict__ I, const int *__restrict__ start, int n, int parity)
{
    __shared__ Dev sD;
    const int i = batch_find(start, n, (int)blockIdx.x);
    const InstArgs &a = I[i];
    copy_dev(sD, a.D);
    const int par = parity ^ a.poff;
    flags_body<1>(sD, a.own[par], a.own[par ^ 1], 1, par,
                  ((int)blockIdx.x - __ldg(start + i)) * (kBoxThreads / 32) + (int)(threadIdx.x >> 5));
}

// Geometry records of the current state and of the previous positions.
__global__ void k_geom_init(const Dev D)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= D.np) return;
    const GeomRec G = make_geom(D.cur.x[a], D.cur.y[a], D.cur.r[a], D.cur.b[a], D.cur.th[a], D.cur.ux[a],
                                D.cur.uy[a], D.cur.om[a], D.cur.T[a], D.cur.rho[a], D.rho_f, D.g);
    D.geo_cur[a] = G;
    D.geo_nxt[a] = G;
    D.pconst[a] = part_consts(D.cur.r[a], D.cur.b[a], D.cur.rho[a], D.rho_f, D.g);
    // (the orientation one step back is not kept: the current one, which
    // only shapes the raster of that owner map inside the same zone)
    D.geo_prev[a] = make_geom(D.px[a], D.py[a], D.cur.r[a], D.cur.b[a], D.cur.th[a], 0.0, 0.0, 0.0, D.cur.T[a],
                              D.cur.rho[a], D.rho_f, D.g);
}

// Link order: the particles by descending y in kOrderBands bands of rows,
// counting-sorted by one block (inside a band, in the order of the block's
// shared-memory atomics).  Stream-collide writes the rows in ascending y,
// so the rows it wrote last are still in L2 when the next link kernel
// gathers from them, and the CTAs of the particles there run first (at
// 4000^2 / 4800 disks: link kernel 78.6 against 84.0 us, step 0.3697
// against 0.3750 ms).  Only the order of the CTAs changes, not what any of
// them computes.
constexpr int kOrderBands = 1024;
__global__ void __launch_bounds__(kOrderBands) k_link_order(const Dev D)
{
    __shared__ int cnt[kOrderBands], at[kOrderBands];
    const int t = threadIdx.x;
    auto band = [&](int p) {
        const double y = D.cur.y[p];
        const int b = (int)((double)kOrderBands * (((double)D.ny - 1.0) - y) / (double)D.ny);
        return min(max(b, 0), kOrderBands - 1);
    };
    cnt[t] = 0;
    __syncthreads();
    for (int p = t; p < D.np; p += kOrderBands) atomicAdd(&cnt[band(p)], 1);
    __syncthreads();
    at[t] = cnt[t];
    __syncthreads();
    for (int o = 1; o < kOrderBands; o <<= 1) { // inclusive prefix sum
        const int v = t >= o ? at[t - o] : 0;
        __syncthreads();
        at[t] += v;
        __syncthreads();
    }
    at[t] -= cnt[t]; // first position of band t
    __syncthreads();
    for (int p = t; p < D.np; p += kOrderBands) {
        const int pos = atomicAdd(&at[band(p)], 1);
        if (in_bounds(D, pos, D.np)) D.lorder[pos] = p;
    }
}

__global__ void k_pack_particles(const Dev D, lbm_particle *out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= D.np) return;
    lbm_particle P;
    P.x = D.cur.x[a]; P.y = D.cur.y[a]; P.ux = D.cur.ux[a]; P.uy = D.cur.uy[a];
    P.theta = D.cur.th[a]; P.omega = D.cur.om[a]; P.r = D.cur.r[a]; P.rho = D.cur.rho[a];
    P.T = D.cur.T[a]; P.b = D.cur.b[a];
    out[a] = P;
}

namespace {

template <typename T>
void *link_kernel()
{
    return reinterpret_cast<void *>(&k_links<T>);
}

void *link_kernel_for(int storage)
{
    switch (storage) {
    case LBM_STORE_BF16: return link_kernel<__nv_bfloat16>();
    case LBM_STORE_FP16: return link_kernel<__half>();
    default: return link_kernel<float>();
    }
}

} // namespace

cudaError_t prepare_links(Dev &D)
{
    D.link_ahead = 1;
    D.flag_team = 1;
    if (D.np == 0) return cudaSuccess;
    const size_t smem = link_smem_bytes(D.zone_max, D.storage);
    const void *fn = link_kernel_for(D.storage);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0, dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLinkThreads, smem)) != cudaSuccess)
        return e;
    D.link_ahead = max(1, sms * per_sm); // particles (CTAs) resident at once
    // flags: one warp per particle when there are enough particles to fill
    // the GPU (about 36 warps per SM), else teams of 2 or 4 warps
    const int warps = sms * 36;
    D.flag_team = D.np * 2 > warps ? 1 : D.np * 4 > warps ? 2 : 4;
    return cudaSuccess;
}

cudaError_t launch_links(const Dev &D, void *A, const int *own_cur, int *own_nxt, int parity,
                         cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    const size_t smem = link_smem_bytes(D.zone_max, D.storage);
    const int grid = D.np;
    switch (D.storage) {
    case LBM_STORE_FP32:
        k_links<float><<<grid, kLinkThreads, smem, s>>>(D, static_cast<float *>(A), own_cur, own_nxt, parity,
                                                        D.link_ahead);
        break;
    case LBM_STORE_BF16:
        k_links<__nv_bfloat16><<<grid, kLinkThreads, smem, s>>>(D, static_cast<__nv_bfloat16 *>(A), own_cur,
                                                                own_nxt, parity, D.link_ahead);
        break;
    case LBM_STORE_FP16:
        k_links<__half><<<grid, kLinkThreads, smem, s>>>(D, static_cast<__half *>(A), own_cur, own_nxt, parity,
                                                         D.link_ahead);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---- batched launches (one grid over all instances)
cudaError_t prepare_links_batch(int zone_max, int storage, size_t *smem, int *ahead)
{
    *smem = link_smem_bytes(zone_max, storage);
    const void *fn = storage == LBM_STORE_BF16   ? reinterpret_cast<const void *>(&k_links_batch<__nv_bfloat16>)
                     : storage == LBM_STORE_FP16 ? reinterpret_cast<const void *>(&k_links_batch<__half>)
                                                 : reinterpret_cast<const void *>(&k_links_batch<float>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0, dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLinkThreads, *smem)) != cudaSuccess)
        return e;
    *ahead = max(1, sms * per_sm);
    return cudaSuccess;
}

cudaError_t launch_links_batch(const InstArgs *I, const int *start, int n, int total, int storage, int parity,
                               int ahead, size_t smem, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    switch (storage) {
    case LBM_STORE_FP32: k_links_batch<float><<<total, kLinkThreads, smem, s>>>(I, start, n, parity, ahead); break;
    case LBM_STORE_BF16:
        k_links_batch<__nv_bfloat16><<<total, kLinkThreads, smem, s>>>(I, start, n, parity, ahead);
        break;
    case LBM_STORE_FP16: k_links_batch<__half><<<total, kLinkThreads, smem, s>>>(I, start, n, parity, ahead); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_particles_batch(const InstArgs *I, const int *start, int n, int total, int parity,
                                   cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    k_particles_batch<<<total, kPartThreads, 0, s>>>(I, start, n, parity);
    return cudaGetLastError();
}

cudaError_t launch_raster_batch(const InstArgs *I, const int *start, int n, int total, int parity, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    k_raster_batch<<<total, kBoxThreads, 0, s>>>(I, start, n, parity);
    return cudaGetLastError();
}

cudaError_t launch_flags_batch(const InstArgs *I, const int *start, int n, int total, int parity, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    k_flags_batch<<<total, kBoxThreads, 0, s>>>(I, start, n, parity);
    return cudaGetLastError();
}

// Blocks of each batched step kernel for one instance.
void batch_blocks(const Dev &D, dim3 sc_block, int out[kBatchPhases])
{
    const int V = D.storage == LBM_STORE_FP32 ? 1 : 2;
    out[kBLinks] = D.np;
    out[kBParticles] = D.np > 0 ? (D.np + kPartPerBlock - 1) / kPartPerBlock : 1;
    out[kBRaster] = (D.np + kBoxThreads / 32 - 1) / (kBoxThreads / 32);
    out[kBFlags] = (D.np + kBoxThreads / 32 - 1) / (kBoxThreads / 32);
    out[kBStream] = ((D.pitch / V + (int)sc_block.x - 1) / (int)sc_block.x) *
                    ((D.ny + (int)sc_block.y - 1) / (int)sc_block.y);
    out[kBBoundary] = kBoundaryBlocksPerInstance;
}

cudaError_t launch_near_mask(const Dev &D, cudaStream_t s)
{
    const size_t words = ((size_t)D.ny * D.near_tpr + 31) / 32;
    cudaError_t e = cudaMemsetAsync(D.near, 0, words * sizeof(unsigned), s);
    if (e != cudaSuccess || D.np == 0) return e;
    const int span = 32 * (D.storage == LBM_STORE_FP32 ? 1 : 2);
    const long long threads = (long long)D.np * (D.zone_max + 2 * kNearMargin);
    k_near_mask<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(D, span);
    return cudaGetLastError();
}

cudaError_t launch_links_direct(const Dev &D, void *A, const int *own_cur, int *own_nxt, int parity,
                                cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_direct_prep<<<D.np, kBoxThreads, 0, s>>>(D, own_nxt, parity);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((D.nx + 127) / 128, D.ny);
    switch (D.storage) {
    case LBM_STORE_FP32: k_links_direct<float><<<grid, 128, 0, s>>>(D, static_cast<float *>(A), own_cur, parity); break;
    case LBM_STORE_BF16:
        k_links_direct<__nv_bfloat16><<<grid, 128, 0, s>>>(D, static_cast<__nv_bfloat16 *>(A), own_cur, parity);
        break;
    case LBM_STORE_FP16: k_links_direct<__half><<<grid, 128, 0, s>>>(D, static_cast<__half *>(A), own_cur, parity); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_particles(const Dev &D, int parity, int *own_nxt, cudaStream_t s)
{
    const int blocks = D.np > 0 ? (D.np + kPartPerBlock - 1) / kPartPerBlock : 1;
    k_particles<<<blocks, kPartThreads, 0, s>>>(D, parity, own_nxt);
    return cudaGetLastError();
}

cudaError_t launch_raster(const Dev &D, int *own, const GeomRec *geo, const PartSoA &pos, int2 *runs, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    const int per = kBoxThreads / 32;
    k_raster<<<(D.np + per - 1) / per, kBoxThreads, 0, s>>>(D, own, geo, pos, runs);
    return cudaGetLastError();
}

cudaError_t launch_geom_init(const Dev &D, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_geom_init<<<(D.np + 127) / 128, 128, 0, s>>>(D);
    return cudaGetLastError();
}

cudaError_t launch_link_order(const Dev &D, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_link_order<<<1, kOrderBands, 0, s>>>(D);
    return cudaGetLastError();
}

cudaError_t launch_cells_init(const Dev &D, cudaStream_t s)
{
    const size_t counts = ((size_t)D.cell_gx * D.cell_gy + 1) * sizeof(int);
    for (int b = 0; b < 2; ++b) {
        const cudaError_t e = cudaMemsetAsync(D.cells[b], 0, counts, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_flags(const Dev &D, const int *own_cur, const int *own_nxt, int rotate, int parity,
                         cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    const int per = kBoxThreads / 32 / max(D.flag_team, 1); // particles per block
    const int grid = (D.np + per - 1) / per;
    switch (D.flag_team) {
    case 4: k_flags<4><<<grid, kBoxThreads, 0, s>>>(D, own_cur, own_nxt, rotate, parity); break;
    case 2: k_flags<2><<<grid, kBoxThreads, 0, s>>>(D, own_cur, own_nxt, rotate, parity); break;
    default: k_flags<1><<<grid, kBoxThreads, 0, s>>>(D, own_cur, own_nxt, rotate, parity); break;
    }
    return cudaGetLastError();
}

// Newborn nodes of a restored state: every node whose flag says newborn
// goes into the list (emptied first by the caller), which the next step's
// link kernel returns to fluid.
__global__ void k_collect_newborn(const Dev D)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= D.nx) return;
    if (D.flags[(long long)j * D.pitch + i] == kNewborn) list_newborn(D, i, j);
}

cudaError_t launch_collect_newborn(const Dev &D, cudaStream_t s)
{
    k_collect_newborn<<<dim3((D.nx + 127) / 128, D.ny), 128, 0, s>>>(D);
    return cudaGetLastError();
}

cudaError_t launch_pack_particles(const Dev &D, lbm_particle *out, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_pack_particles<<<(D.np + 127) / 128, 128, 0, s>>>(D, out);
    return cudaGetLastError();
}

} // namespace lbm
