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

constexpr int kLinkThreads = 128;
constexpr int kBoxThreads = 128;
constexpr int kPartThreads = 128;
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
// reduction is a deterministic tree.  Bounce-back values are written into the
// solid node x_f + e_k in direction kbar of the post-collision array A, where
// the next pull stream picks them up: each (solid node, kbar) belongs to one
// link, and every read is of a fluid node, so the writes never race the reads.
__global__ void __launch_bounds__(kLinkThreads)
    k_links(const Dev D, float *A, const int *__restrict__ own, int parity)
{
    const int p = blockIdx.x;
    const double xc = D.cur.x[p], yc = D.cur.y[p], r = D.cur.r[p];
    const float Ux = (float)D.cur.ux[p], Uy = (float)D.cur.uy[p], Om = (float)D.cur.om[p];
    const float wT = 0.2f * (float)D.cur.T[p]; // 2 w_k T_w for D2Q5
    const int N = zone_size(r), cap = 12 * N - 12;
    const int X0 = (int)floor(xc - r) - 1, Y0 = (int)floor(yc - r) - 1;
    const int base = D.slot_base[p];
    double Fx = 0.0, Fy = 0.0, Tz = 0.0;
    unsigned c_lin = 0, c_simple = 0, c_th = 0, c_links = 0, c_over = 0;

    for (int s = threadIdx.x; s < cap; s += kLinkThreads) {
        int k, line;
        slot_dir_line(s, N, k, line);
        const int kx = ex(k), ky = ey(k);
        int found = 0, fi = 0, fj = 0;
        for (int t = 0; t < N; ++t) {
            int a, b;
            if (!zone_point(k, N, line, t, a, b)) continue;
            const int i = X0 + a, j = Y0 + b;
            if (!inside(D, i, j) || own[(long long)j * D.nx + i] != -1) continue;
            const int si = i + kx, sj = j + ky;
            if (!inside(D, si, sj) || own[(long long)sj * D.nx + si] != p) continue;
            if (++found == 1) {
                fi = i;
                fj = j;
            }
        }
        c_over += found > 1;
        int node = -1;
        float q = 0.f;
        if (found) {
            node = fj * D.nx + fi;
            q = (float)link_q(fi, fj, k, xc, yc, r);
        }
        D.slot_node[base + s] = node;
        D.slot_q[base + s] = q;
        if (!found) continue;
        ++c_links;

        // ---- curved bounce-back (Sec. 2.3) in deviation form: every rule is
        // an affine combination of populations of equal weight, so it holds
        // for f~ = f - w unchanged.
        const int kb = opp(k);
        const int i1 = fi - kx, j1 = fj - ky, i2 = fi - 2 * kx, j2 = fj - 2 * ky;
        const bool have1 = inside(D, i1, j1) && own[(long long)j1 * D.nx + i1] == -1;
        const bool have2 = inside(D, i2, j2) && own[(long long)j2 * D.nx + i2] == -1;
        const long long n0 = (long long)fj * D.pitch + fi;
        const long long n1 = have1 ? (long long)j1 * D.pitch + i1 : n0;
        const long long n2 = have2 ? (long long)j2 * D.pitch + i2 : n0;
        const float fk0 = A[k * D.ps + n0], fk1 = A[k * D.ps + n1], fk2 = A[k * D.ps + n2];
        const float fb0 = A[kb * D.ps + n0], fb1 = A[kb * D.ps + n1];
        const double dxi = __dsub_rn((double)fi, xc), dyj = __dsub_rn((double)fj, yc);
        const float rx = (float)dxi + q * kx, ry = (float)dyj + q * ky;
        const float uwx = Ux - Om * ry, uwy = Uy + Om * rx;
        const float wall = 6.f * w9(k) * -(kx * uwx + ky * uwy); // 2 w rho0 e_kbar.u_w / c_s^2
        float fnew;
        if (q <= 0.5f) {
            if (have1 && have2) {
                fnew = q * (2.f * q + 1.f) * fk0 + (1.f - 4.f * q * q) * fk1 -
                       q * (1.f - 2.f * q) * fk2 + wall;
            } else if (have1) {
                fnew = 2.f * q * fk0 + (1.f - 2.f * q) * fk1 + wall;
                ++c_lin;
            } else {
                fnew = fk0 + wall;
                ++c_simple;
            }
        } else if (have1) {
            const float cq = 1.f / (q * (2.f * q + 1.f));
            fnew = cq * fk0 + (2.f * q - 1.f) / q * fb0 - (2.f * q - 1.f) / (2.f * q + 1.f) * fb1 +
                   cq * wall;
        } else {
            const float h = 0.5f / q;
            fnew = h * fk0 + (2.f * q - 1.f) * h * fb0 + h * wall;
            ++c_lin;
        }
        const long long ns = (long long)(fj + ky) * D.pitch + (fi + kx);
        A[kb * D.ps + ns] = fnew;
        if (k <= 4) {
            const float gk0 = A[(kQ9 + k) * D.ps + n0];
            float gnew;
            if (have1) {
                const float c23 = (2.f * q - 1.f) / (2.f * q + 1.f), c4 = 2.f / (2.f * q + 1.f);
                gnew = -gk0 + c23 * (A[(kQ9 + k) * D.ps + n1] + A[(kQ9 + kb) * D.ps + n0]) + c4 * wT;
            } else {
                gnew = -gk0 + wT;
                ++c_th;
            }
            A[(kQ9 + kb) * D.ps + ns] = gnew;
        }

        // ---- momentum exchange.  With f = w + f~ the bracket of Eq. force is
        // 2 w_k e_k + [f~_k^+ (e_k - u_w) - f~_kbar (e_kbar - u_w)]; the constant
        // part is added in FP64, and its torque 2 w_k (x_f - x_c) x e_k does not
        // depend on q.
        const float bx = fk0 * (kx - uwx) - fnew * (-kx - uwx);
        const float by = fk0 * (ky - uwy) - fnew * (-ky - uwy);
        const double cF = 2.0 * w9d(k);
        Fx += cF * kx + (double)bx;
        Fy += cF * ky + (double)by;
        Tz += cF * (dxi * ky - dyj * kx) + (double)(rx * by - ry * bx);
    }

    __shared__ double red[3][kLinkThreads / 32];
    __shared__ unsigned cnt[5][kLinkThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Fx = warp_sum(Fx);
    Fy = warp_sum(Fy);
    Tz = warp_sum(Tz);
    c_lin = warp_sum(c_lin);
    c_simple = warp_sum(c_simple);
    c_th = warp_sum(c_th);
    c_links = warp_sum(c_links);
    c_over = warp_sum(c_over);
    if (lane == 0) {
        red[0][warp] = Fx;
        red[1][warp] = Fy;
        red[2][warp] = Tz;
        cnt[0][warp] = c_lin;
        cnt[1][warp] = c_simple;
        cnt[2][warp] = c_th;
        cnt[3][warp] = c_links;
        cnt[4][warp] = c_over;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sx = 0.0, sy = 0.0, st = 0.0;
        unsigned a[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < kLinkThreads / 32; ++w) {
            sx += red[0][w];
            sy += red[1][w];
            st += red[2][w];
            for (int c = 0; c < 5; ++c) a[c] += cnt[c][w];
        }
        D.force[3 * p + 0] = sx;
        D.force[3 * p + 1] = sy;
        D.force[3 * p + 2] = st;
        unsigned long long *C = D.status->cnt[parity];
        if (a[0]) atomicAdd(&C[kCntBzLinear], (unsigned long long)a[0]);
        if (a[1]) atomicAdd(&C[kCntBzSimple], (unsigned long long)a[1]);
        if (a[2]) atomicAdd(&C[kCntThermHalf], (unsigned long long)a[2]);
        if (a[3]) atomicAdd(&C[kCntLinks], (unsigned long long)a[3]);
        if (a[4]) atomicOr(&D.status->err, kErrOverflow);
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

// One thread per particle.  Total force = hydrodynamic + buoyant weight
// -(rho_p - rho_f) pi r^2 g y-hat + repulsion (walls, then every other disk,
// with C_ab the mean of the two force scales C = pi r^2 (rho_p - rho_f) g).
// Other disks are screened in FP32 tiles with a one-lattice-unit margin and
// evaluated in FP64.  Integration: U' = U + F/M, X' = X + (U + U')/2,
// Omega' = Omega + T/I, theta' = theta + (Omega + Omega')/2 with
// M = rho_p pi r^2 and I = M r^2 / 2.
__global__ void __launch_bounds__(kPartThreads) k_particles(const Dev D, int parity)
{
    __shared__ float sx[kPartThreads], sy[kPartThreads], sr[kPartThreads];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x < kNumCounters) D.status->cnt[parity ^ 1][threadIdx.x] = 0ull;
    const bool me = a < D.np;
    double x = 0, y = 0, ux = 0, uy = 0, th = 0, om = 0, r = 1, rho = 1, T = 0;
    if (me) {
        x = D.cur.x[a]; y = D.cur.y[a]; ux = D.cur.ux[a]; uy = D.cur.uy[a];
        th = D.cur.th[a]; om = D.cur.om[a]; r = D.cur.r[a]; rho = D.cur.rho[a]; T = D.cur.T[a];
    }
    const double Ca = kPi * r * r * (rho - D.rho_f) * D.g;
    double Fx = 0.0, Fy = 0.0, Tz = 0.0;
    if (me) {
        Fx = D.force[3 * a + 0];
        Fy = D.force[3 * a + 1] - (rho - D.rho_f) * kPi * r * r * D.g;
        Tz = D.force[3 * a + 2];
        if (!D.per_x) {
            Fx += repulsion((x + 0.5) - r, D.s_rep, D.eps_w, Ca);
            Fx -= repulsion(((double)D.nx - 0.5 - x) - r, D.s_rep, D.eps_w, Ca);
        }
        if (!D.per_y) {
            Fy += repulsion((y + 0.5) - r, D.s_rep, D.eps_w, Ca);
            Fy -= repulsion(((double)D.ny - 0.5 - y) - r, D.s_rep, D.eps_w, Ca);
        }
    }
    const float xf = (float)x, yf = (float)y, rf = (float)r, reach = (float)D.s_rep + 1.f;
    for (int t0 = 0; t0 < D.np; t0 += kPartThreads) {
        const int b = t0 + threadIdx.x;
        __syncthreads();
        if (b < D.np) {
            sx[threadIdx.x] = (float)D.cur.x[b];
            sy[threadIdx.x] = (float)D.cur.y[b];
            sr[threadIdx.x] = (float)D.cur.r[b];
        }
        __syncthreads();
        const int nb = min(kPartThreads, D.np - t0);
        if (!me) continue;
        for (int u = 0; u < nb; ++u) {
            const float dxf = xf - sx[u], dyf = yf - sy[u], lim = rf + sr[u] + reach;
            if (dxf * dxf + dyf * dyf > lim * lim || t0 + u == a) continue;
            const int bb = t0 + u;
            const double dx = x - D.cur.x[bb], dy = y - D.cur.y[bb];
            const double dist = sqrt(dx * dx + dy * dy);
            const double rb = D.cur.r[bb];
            const double gap = dist - r - rb;
            if (gap > D.s_rep) continue;
            const double Cb = kPi * rb * rb * (D.cur.rho[bb] - D.rho_f) * D.g;
            const double mag = repulsion(gap, D.s_rep, D.eps_w, 0.5 * (Ca + Cb));
            Fx += mag * dx / dist;
            Fy += mag * dy / dist;
        }
    }
    if (!me) return;
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
    D.nxt.x[a] = x; D.nxt.y[a] = y; D.nxt.ux[a] = ux; D.nxt.uy[a] = uy; D.nxt.th[a] = th;
    D.nxt.om[a] = om; D.nxt.r[a] = r; D.nxt.rho[a] = rho; D.nxt.T[a] = T;
}

// Zone of a disk at (x, y) with radius r: N x N nodes from
// (floor(x - r) - 1, floor(y - r) - 1); it holds every node of the disk and
// every fluid node linked to it.
struct Box {
    int X0, Y0, N;
};
__device__ __forceinline__ Box box_of(double x, double y, double r)
{
    return Box{(int)floor(x - r) - 1, (int)floor(y - r) - 1, zone_size(r)};
}

// Reset the zone of each disk's position one step back in the owner map
// that is about to receive the new positions, and in the flag map.
__global__ void __launch_bounds__(kBoxThreads) k_clear(const Dev D, int *own_nxt)
{
    const int p = blockIdx.x;
    const Box B = box_of(D.px[p], D.py[p], D.cur.r[p]);
    for (int idx = threadIdx.x; idx < B.N * B.N; idx += kBoxThreads) {
        const int i = B.X0 + idx % B.N, j = B.Y0 + idx / B.N;
        if (!inside(D, i, j)) continue;
        own_nxt[(long long)j * D.nx + i] = -1;
        D.flags[(long long)j * D.pitch + i] = kFluid;
    }
}

// Owner map: node (i,j) belongs to disk p iff (i - x)^2 + (j - y)^2 <= r^2
// (exact FP64); where disks overlap the highest index wins (atomicMax, so
// the result does not depend on the launch order).
__global__ void __launch_bounds__(kBoxThreads) k_raster(const Dev D, int *own, const PartSoA pos)
{
    const int p = blockIdx.x;
    const double x = pos.x[p], y = pos.y[p], r = pos.r[p];
    const Box B = box_of(x, y, r);
    for (int idx = threadIdx.x; idx < B.N * B.N; idx += kBoxThreads) {
        const int i = B.X0 + idx % B.N, j = B.Y0 + idx / B.N;
        if (!inside(D, i, j) || !in_disk(i, j, x, y, r)) continue;
        atomicMax(&own[(long long)j * D.nx + i], p);
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
    const double r = D.cur.r[p];
    const Box B0 = box_of(D.cur.x[p], D.cur.y[p], r);
    const Box B1 = box_of(D.nxt.x[p], D.nxt.y[p], r);
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
    default: break;
    }
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

cudaError_t launch_links(const Dev &D, float *A, const int *own_cur, int parity, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_links<<<D.np, kLinkThreads, 0, s>>>(D, A, own_cur, parity);
    return cudaGetLastError();
}

cudaError_t launch_particles(const Dev &D, int parity, cudaStream_t s)
{
    const int blocks = D.np > 0 ? (D.np + kPartThreads - 1) / kPartThreads : 1;
    k_particles<<<blocks, kPartThreads, 0, s>>>(D, parity);
    return cudaGetLastError();
}

cudaError_t launch_clear(const Dev &D, int *own_nxt, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_clear<<<D.np, kBoxThreads, 0, s>>>(D, own_nxt);
    return cudaGetLastError();
}

cudaError_t launch_raster(const Dev &D, int *own, const PartSoA &pos, cudaStream_t s)
{
    if (D.np == 0) return cudaSuccess;
    k_raster<<<D.np, kBoxThreads, 0, s>>>(D, own, pos);
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
