// Fused pull-stream + MRT collision of the flow (D2Q9) and temperature (D2Q5)
// distributions with Boussinesq buoyancy (Sec. 2.1, Eq. f and Eq. g), and the
// refilling of newborn nodes (Sec. 2.5) on the general path.
//
// Layout: 14 planes (9 flow deviations f~ = f - w, 5 temperature populations
// g) of [ny][pitch] elements (FP32, BF16 or scaled FP16; arithmetic in FP32),
// ping-ponged between two buffers.  A plane row is read once and written once
// per step: 112 (FP32) or 56 (16-bit) algorithmic bytes per node.
//
// One thread per node.  A pull from x - 1 or x + 1 takes the value from the
// neighbouring lane by a warp shuffle (one scalar load at the warp edge), so
// the x-shifted planes cost no extra HBM traffic.  The nodes of the cavity
// frame (walls, periodic seams) and newborn nodes take a general (scalar)
// path in a second, small kernel (k_boundary) that runs concurrently with
// the streaming kernel and keeps that code and its registers out of it.
// With 16-bit storage a thread holds two nodes, collided together on paired
// FP32 instructions.
#include "lbm_internal.cuh"

namespace lbm {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Post-collision value pulled into node (x, y) for population p, general
// form: the source x - e is read directly, wrapped across a periodic seam, or
// replaced across a wall by half-way bounce-back (f) or anti-bounce-back with
// the wall temperature (g).  In deviation form the half-way rule keeps its
// shape because w_i = w_ibar.
template <typename T>
__device__ float pull_general(const Dev &D, const T *__restrict__ A, int x, int y, int p)
{
    using E = Elem<T>;
    const int d = pdir(p);
    int xs = x - ex(d), ys = y - ey(d);
    bool wall = false;
    if (xs < 0 || xs >= D.nx) {
        if (D.per_x) xs = xs < 0 ? xs + D.nx : xs - D.nx;
        else wall = true;
    }
    if (ys < 0 || ys >= D.ny) {
        if (D.per_y) ys = ys < 0 ? ys + D.ny : ys - D.ny;
        else wall = true;
    }
    if (!wall) {
        const long long e = (long long)p * D.ps + (long long)ys * D.pitch + xs;
        return in_bounds(D, e, D.a_elems) ? E::ld(A[e]) : 0.f;
    }
    const long long self = (long long)y * D.pitch + x;
    const long long e = (long long)(p < kQ9 ? opp(d) : kQ9 + opp(d)) * D.ps + self;
    const float v = in_bounds(D, e, D.a_elems) ? E::ld(A[e]) : 0.f;
    if (p < kQ9) return v;
    const int side = d == 1 ? 0 : d == 3 ? 1 : d == 2 ? 2 : 3;
    return -v + 2.f * w5(d) * D.Twall[side];
}

// Values pulled into a node on the general path; for a newborn node the
// refilling of Sec. 2.5 instead: e_c maximises n . e_c (FP64, ties to the
// lowest index, n the outward normal at the new position), f is extrapolated from the nodes
// x + m e_c (m = 1, 2, 3) that are fluid at both times (quadratic, linear,
// copy, or f_eq(1, u_w)), its momentum is set to rho u_w, and
// g = g_eq(T_w, u_w).
// Returns 0 for a general pull, else 1 + the refill class (1 quadratic,
// 2 linear, 3 copy, 4 equilibrium).
// The pull of plane p at the side node (x, y), x = 0 or nx - 1, of a row
// between the first and the last, for a plane whose source lies across the
// side wall or the periodic seam (pull_general restricted to that case).
template <typename T>
__device__ __forceinline__ float side_pull(const Dev &D, const T *__restrict__ A, int x, int y, int p)
{
    using E = Elem<T>;
    const int d = pdir(p);
    if (D.per_x) {
        const int xs = x == 0 ? D.nx - 1 : 0;
        const long long e = (long long)p * D.ps + (long long)(y - ey(d)) * D.pitch + xs;
        return in_bounds(D, e, D.a_elems) ? E::ld(A[e]) : 0.f;
    }
    const long long e = (long long)(p < kQ9 ? opp(d) : kQ9 + opp(d)) * D.ps + (long long)y * D.pitch + x;
    const float v = in_bounds(D, e, D.a_elems) ? E::ld(A[e]) : 0.f;
    if (p < kQ9) return v;
    return -v + 2.f * w5(d) * D.Twall[d == 1 ? 0 : 1];
}

template <typename T>
__device__ __forceinline__ int slow_node(const Dev &D, const T *__restrict__ A,
                                      const int *__restrict__ own_cur, int x, int y, uint8_t fl,
                                      float *out)
{
    if (fl != kNewborn) {
#pragma unroll
        for (int p = 0; p < kPop; ++p) out[p] = pull_general(D, A, x, y, p);
        return 0;
    }
    const int pid = own_cur[(long long)y * D.nx + x];
    const double xc = D.cur.x[pid], yc = D.cur.y[pid];
    const double dx = __dsub_rn((double)x, xc), dy = __dsub_rn((double)y, yc);
    // outward normal: (dx, dy) for a disk, the gradient of the ellipse form
    // for an ellipse
    double nx = dx, ny = dy;
    const double pr = D.cur.r[pid], pb = D.cur.b[pid];
    if (is_ellipse(pr, pb)) ell_normal(ell_frame(xc, yc, D.cur.th[pid], pr, pb), dx, dy, nx, ny);
    int c = 1;
    double best = __dadd_rn(__dmul_rn((double)ex(1), nx), __dmul_rn((double)ey(1), ny));
    for (int k = 2; k < kQ9; ++k) {
        double v = __dadd_rn(__dmul_rn((double)ex(k), nx), __dmul_rn((double)ey(k), ny));
        if (v > best) {
            best = v;
            c = k;
        }
    }
    const float uwx = (float)(D.cur.ux[pid] - D.cur.om[pid] * dy);
    const float uwy = (float)(D.cur.uy[pid] + D.cur.om[pid] * dx);
    int nvalid = 0;
    for (int m = 1; m <= 3; ++m) {
        int a = x + m * ex(c), b = y + m * ey(c);
        if (a < 0 || a >= D.nx || b < 0 || b >= D.ny) break;
        if (D.flags[(long long)b * D.pitch + a] != kFluid) break;
        nvalid = m;
    }
    float fh[kQ9];
    if (nvalid == 0) {
        const float uu = uwx * uwx + uwy * uwy;
        for (int i = 0; i < kQ9; ++i) {
            float eu = ex(i) * uwx + ey(i) * uwy;
            fh[i] = w9(i) * (3.f * eu + 4.5f * eu * eu - 1.5f * uu);
        }
    } else {
        float c1 = nvalid == 3 ? 3.f : nvalid == 2 ? 2.f : 1.f;
        float c2 = nvalid == 3 ? -3.f : nvalid == 2 ? -1.f : 0.f;
        float c3 = nvalid == 3 ? 1.f : 0.f;
        const int x1 = x + ex(c), y1 = y + ey(c);
#pragma unroll
        for (int i = 0; i < kQ9; ++i) {
            float v = c1 * pull_general(D, A, x1, y1, i);
            if (nvalid >= 2) v += c2 * pull_general(D, A, x1 + ex(c), y1 + ey(c), i);
            if (nvalid >= 3) v += c3 * pull_general(D, A, x1 + 2 * ex(c), y1 + 2 * ey(c), i);
            fh[i] = v;
        }
    }
    // velocity constraint: j = rho u_w, every other moment kept; the x- and
    // y-momentum rows of the moment basis have squared norm 6
    float rho = 1.f, jx = 0.f, jy = 0.f;
    for (int i = 0; i < kQ9; ++i) {
        rho += fh[i];
        jx += ex(i) * fh[i];
        jy += ey(i) * fh[i];
    }
    const float djx = (rho * uwx - jx) * (1.f / 6.f), djy = (rho * uwy - jy) * (1.f / 6.f);
    for (int i = 0; i < kQ9; ++i) out[i] = fh[i] + ex(i) * djx + ey(i) * djy;
    const float Tw = (float)D.cur.T[pid];
    for (int i = 0; i < kQ5; ++i) out[kQ9 + i] = w5(i) * Tw * (1.f + 5.f * (ex(i) * uwx + ey(i) * uwy));
    return 4 - nvalid;
}

// Arithmetic of the collision on one node (float) or on two nodes at once
// (float2, Blackwell's paired FP32 instructions).  Every operation is a
// round-to-nearest add, multiply or fused multiply-add, so both forms give
// the same bits per node, and no kernel that inlines them fuses differently.
template <typename F>
struct FOps;
template <>
struct FOps<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ float bc(float v) { return v; }
    static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.f, a); }
};
template <>
struct FOps<float2> {
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    // a - b = RN(b (-1) + a): exact product, one rounding
    static __device__ __forceinline__ float2 sub(float2 a, float2 b)
    {
        return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
    }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
    static __device__ __forceinline__ float2 rcp(float2 a)
    {
        return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y));
    }
};
__device__ __forceinline__ bool phys_ok(float rho, float T)
{
    return (rho > 0.25f) && (rho < 4.f) && (fabsf(T) < 1e30f);
}

// MRT collision in deviation form (Eq. f with Guo forcing in moment space,
// Eq. g), in place on c[14] (one node per lane of F).  ok: whether each
// node's density and temperature are finite and physical.  kS: c holds the
// populations times 2^12 (FP16 storage's scale) and receives the results
// times 2^12; every product of a scaled term takes the scale through a
// scaled constant or one exact multiplication, so the results are those of
// the unscaled collision times 2^12, bit for bit.
template <typename F, bool kS = false>
__device__ __forceinline__ void collide_t(const Dev &D, F *c, bool &ok0, bool &ok1)
{
    using O = FOps<F>;
    auto K = [&](float plain, int scaled) { return kS ? D.ksc[scaled] : plain; };
    const F f0 = c[0], f1 = c[1], f2 = c[2], f3 = c[3], f4 = c[4];
    const F f5 = c[5], f6 = c[6], f7 = c[7], f8 = c[8];
    // pair sums and differences shared by the moments
    const F u13 = O::add(f1, f3), d13 = O::sub(f1, f3), u24 = O::add(f2, f4), d24 = O::sub(f2, f4);
    const F s56 = O::add(f5, f6), d56 = O::sub(f5, f6), s78 = O::add(f7, f8), d87 = O::sub(f8, f7);
    const F sa = O::add(u13, u24), sd = O::add(s56, s78);
    const F drho = O::add(O::add(f0, sa), sd);
    const F rho = kS ? O::fma(drho, O::bc(1.f / kHalfScale), O::bc(1.f)) : O::add(O::bc(1.f), drho);
    const F e = O::add(d56, d87), g = O::sub(s56, s78);
    const F jx = O::add(d13, e), jy = O::add(d24, g);
    const F T = O::add(O::add(O::add(c[9], c[10]), O::add(c[11], c[12])), c[13]);
    const F Tu = kS ? O::mul(T, O::bc(1.f / kHalfScale)) : T; // the temperature itself
    const F Fx = O::bc(D.bfx);
    const F Fy = O::fma(O::mul(rho, O::bc(D.gbeta)), O::sub(Tu, O::bc(D.T0)), O::bc(D.bfy));
    const F FxS = kS ? O::bc(D.ksc[kScBfx]) : Fx, FyS = kS ? O::mul(Fy, O::bc(kHalfScale)) : Fy;
    const F inv = O::rcp(rho), invS = kS ? O::mul(inv, O::bc(1.f / kHalfScale)) : inv;
    const F ux = O::mul(O::fma(O::bc(0.5f), FxS, jx), invS), uy = O::mul(O::fma(O::bc(0.5f), FyS, jy), invS);
    const F m1 = O::fma(O::bc(2.f), sd, O::fma(O::bc(-4.f), f0, O::sub(O::bc(0.f), sa))); // -4 f0 - sa + 2 sd
    const F m2 = O::fma(O::bc(4.f), f0, O::fma(O::bc(-2.f), sa, sd));                     // 4 f0 - 2 sa + sd
    const F m4 = O::fma(O::bc(-2.f), d13, e); // 2 (f3 - f1) + (f5 - f6) + (f8 - f7)
    const F m6 = O::fma(O::bc(-2.f), d24, g); // 2 (f4 - f2) + (f5 + f6) - (f7 + f8)
    const F m7 = O::sub(u13, u24);
    const F m8 = O::sub(O::add(f5, f7), O::add(f6, f8));
    const F uu = O::fma(ux, ux, O::mul(uy, uy));
    const F uF = O::fma(ux, Fx, O::mul(uy, Fy));
    const F ru = O::mul(O::mul(O::bc(K(3.f, kScThree)), rho), uu);
    // a_i = post-collision moment i / |M_i|^2, the rates and norms folded
    // into the coefficients k*: m_i - s_i (m_i - m_eq,i) + (1 - s_i / 2) F_i
    const F a0 = O::mul(drho, O::bc(1.f / 9.f));
    const F a1 = O::fma(O::bc(D.kA1), m1,
                        O::fma(O::bc(D.kB1), O::fma(O::bc(-2.f), drho, ru), O::mul(O::bc(K(D.kC1, kScC1)), uF)));
    const F a2 =
        O::fma(O::bc(D.kA2), m2, O::fma(O::bc(D.kB2), O::sub(drho, ru), O::mul(O::bc(-K(D.kC2, kScC2)), uF)));
    const F a3 = O::mul(O::add(jx, FxS), O::bc(1.f / 6.f)), a5 = O::mul(O::add(jy, FyS), O::bc(1.f / 6.f));
    const F rux = O::mul(rho, ux), ruy = O::mul(rho, uy);
    const F a4 = O::fma(O::bc(D.kA4), m4, O::fma(O::bc(-K(D.kB4, kScB4)), rux, O::mul(O::bc(-D.kC4), FxS)));
    const F a6 = O::fma(O::bc(D.kA4), m6, O::fma(O::bc(-K(D.kB4, kScB4)), ruy, O::mul(O::bc(-D.kC4), FyS)));
    const F pxx = O::fma(ux, ux, O::mul(O::sub(O::bc(0.f), uy), uy)); // ux^2 - uy^2
    const F fxx = O::fma(ux, Fx, O::mul(O::sub(O::bc(0.f), uy), Fy)); // ux Fx - uy Fy
    const F fxy = O::fma(ux, Fy, O::mul(uy, Fx));                     // ux Fy + uy Fx
    const F a7 = O::fma(O::bc(D.kA7), m7,
                        O::fma(O::bc(K(D.kB7, kScB7)), O::mul(rho, pxx), O::mul(O::bc(K(D.kC7, kScC7)), fxx)));
    const F a8 = O::fma(O::bc(D.kA7), m8,
                        O::fma(O::bc(K(D.kB7, kScB7)), O::mul(rux, uy), O::mul(O::bc(K(D.kC8, kScC8)), fxy)));
    // f = M^T a
    const F base = O::fma(O::bc(-2.f), a2, O::sub(a0, a1)), dbase = O::fma(O::bc(2.f), a1, O::add(a0, a2));
    const F h34 = O::fma(O::bc(-2.f), a4, a3), h56 = O::fma(O::bc(-2.f), a6, a5);
    const F s34 = O::add(a3, a4), s56a = O::add(a5, a6);
    c[0] = O::fma(O::bc(4.f), a2, O::fma(O::bc(-4.f), a1, a0));
    c[1] = O::add(O::add(base, h34), a7);
    c[2] = O::sub(O::add(base, h56), a7);
    c[3] = O::add(O::sub(base, h34), a7);
    c[4] = O::sub(O::sub(base, h56), a7);
    c[5] = O::add(O::add(O::add(dbase, s34), s56a), a8);
    c[6] = O::sub(O::add(O::sub(dbase, s34), s56a), a8);
    c[7] = O::add(O::sub(O::sub(dbase, s34), s56a), a8);
    c[8] = O::sub(O::sub(O::add(dbase, s34), s56a), a8);
    // D2Q5: n = (T, g1-g3, g2-g4, -4g0 + g1+g2+g3+g4, g1-g2+g3-g4),
    // n_eq = (T, T ux, T uy, -2T, 0); g = N^T diag(1/5, 1/2, 1/2, 1/20, 1/4) n
    const F g0 = c[9], g1 = c[10], g2 = c[11], g3 = c[12], g4 = c[13];
    const F n1 = O::sub(g1, g3), n2 = O::sub(g2, g4);
    const F n3 = O::fma(O::bc(-4.f), g0, O::add(O::add(g1, g2), O::add(g3, g4)));
    const F n4 = O::sub(O::add(g1, g3), O::add(g2, g4));
    const F b0 = O::mul(T, O::bc(0.2f));
    const F b1 = O::fma(O::bc(D.kG1), n1, O::mul(O::bc(K(D.kG2, kScG2)), O::mul(Tu, ux)));
    const F b2 = O::fma(O::bc(D.kG1), n2, O::mul(O::bc(K(D.kG2, kScG2)), O::mul(Tu, uy)));
    const F b3 = O::fma(O::bc(D.kG3), n3, O::mul(O::bc(-D.kG4), T));
    const F b4 = O::mul(O::bc(D.kG5), n4);
    const F b03 = O::add(b0, b3);
    c[9] = O::fma(O::bc(-4.f), b3, b0);
    c[10] = O::add(O::add(b03, b1), b4);
    c[11] = O::sub(O::add(b03, b2), b4);
    c[12] = O::add(O::sub(b03, b1), b4);
    c[13] = O::sub(O::sub(b03, b2), b4);
    if constexpr (sizeof(F) == sizeof(float)) {
        ok0 = phys_ok(reinterpret_cast<const float &>(rho), reinterpret_cast<const float &>(Tu));
        ok1 = ok0;
    } else {
        const float2 r2 = reinterpret_cast<const float2 &>(rho), t2 = reinterpret_cast<const float2 &>(Tu);
        ok0 = phys_ok(r2.x, t2.x);
        ok1 = phys_ok(r2.y, t2.y);
    }
}
// One node: false for a non-finite or non-physical density/temperature.
__device__ __forceinline__ bool collide(const Dev &D, float *c)
{
    bool ok, unused;
    collide_t<float>(D, c, ok, unused);
    return ok;
}

// Per-thread counts of newborn nodes and of refill fallbacks (linear, copy,
// equilibrium), added to the step's counters once per thread.
__device__ __noinline__ void flush_counters(const Dev &D, int parity, const unsigned *n4)
{
    unsigned long long *C = D.status->cnt[parity];
    if (n4[0]) atomicAdd(&C[kCntNewborn], (unsigned long long)n4[0]);
    if (n4[1]) atomicAdd(&C[kCntRfLinear], (unsigned long long)n4[1]);
    if (n4[2]) atomicAdd(&C[kCntRfCopy], (unsigned long long)n4[2]);
    if (n4[3]) atomicAdd(&C[kCntRfEq], (unsigned long long)n4[3]);
}

} // namespace

// ---------------------------------------------------------------------------
// Stream-collide kernel.  One thread per node; a block covers 128 consecutive
// nodes of a row and blocks are launched in row order, so the blocks resident
// at any moment read and write a compact band of rows of every plane.  Each
// plane is read with one 4-byte load per thread at the pulled position: the
// x - e_x shift is taken from the neighbouring lane by a warp shuffle (one
// extra scalar load at the warp edge), so every plane row crosses HBM once.
//
// Look-ahead prefetch: lanes 0..13 of every block issue one bulk L2 prefetch
// each (cp.async.bulk.prefetch.L2) of the 14 source row segments of the block
// `ahead` positions later in launch order, where `ahead` is the number of
// blocks resident on the GPU.  By the time that block runs its loads hit L2,
// so the memory latency of one wave overlaps the collisions of the previous
// wave without holding registers.  (On the 4000^2 benchmark case, when it
// was introduced: 0.73 of the copy bandwidth against 0.56 without it, about
// 53 us per launch.)
// ---------------------------------------------------------------------------
constexpr int kSCThreads = 128;

// V consecutive stored elements moved as one aligned vector.
template <typename T, int V>
struct Vec;
template <>
struct Vec<float, 1> {
    using W = float;
    __device__ static void unpack(W w, float *v) { v[0] = w; }
    __device__ static W pack(const float *v) { return v[0]; }
};
template <>
struct Vec<float, 2> {
    using W = float2;
    __device__ static void unpack(W w, float *v) { v[0] = w.x; v[1] = w.y; }
    __device__ static W pack(const float *v) { return make_float2(v[0], v[1]); }
};
template <>
struct Vec<__nv_bfloat16, 2> {
    using W = __nv_bfloat162;
    __device__ static void unpack(W w, float *v)
    {
        const float2 f = __bfloat1622float2(w);
        v[0] = f.x;
        v[1] = f.y;
    }
    __device__ static W pack(const float *v) { return __floats2bfloat162_rn(v[0], v[1]); }
};
template <>
struct Vec<__half, 2> {
    using W = __half2;
    __device__ static void unpack(W w, float *v)
    {
        const float2 f = __half22float2(w);
        v[0] = f.x * (1.f / kHalfScale);
        v[1] = f.y * (1.f / kHalfScale);
    }
    __device__ static W pack(const float *v) { return __floats2half2_rn(v[0] * kHalfScale, v[1] * kHalfScale); }
};

// Loads and stores of the fused stream-collide kernels: FP16 values stay in
// their stored scale (times 2^12) and the collision runs on the scaled
// values (collide_t<F, true>, the same bits); every other storage as Elem
// and Vec.
template <typename T>
struct Io {
    static constexpr bool kScaled = false;
    __device__ static float ld(T v) { return Elem<T>::ld(v); }
    __device__ static T st(float v) { return Elem<T>::st(v); }
};
template <>
struct Io<__half> {
    static constexpr bool kScaled = true;
    __device__ static float ld(__half v) { return __half2float(v); }
    __device__ static __half st(float v) { return __float2half_rn(v); }
};
template <typename T, int V>
struct VecIo : Vec<T, V> {
};
template <>
struct VecIo<__half, 2> {
    using W = __half2;
    __device__ static void unpack(W w, float *v)
    {
        const float2 f = __half22float2(w);
        v[0] = f.x;
        v[1] = f.y;
    }
    __device__ static W pack(const float *v) { return __floats2half2_rn(v[0], v[1]); }
};

// Whether warp tile t of row y is within reach of a particle this step.
__device__ __forceinline__ bool tile_near(const Dev &D, int y, int t)
{
    const int b = y * D.near_tpr + t;
    return (__ldg(D.near + (b >> 5)) >> (b & 31)) & 1u;
}

// Stream-collide kernel, V consecutive nodes per thread (one vector load and
// one vector store per plane); FP32 runs V = 1, the 16-bit storages V = 2 so
// that every load still moves four bytes.  mode selects all warp tiles, or
// only those away from / within reach of this step's particles.
// Look-ahead target of a grid launch: the block `ahead` places later in
// launch order, ahead = ahead_y grid rows + ahead_x blocks (ahead_x < gx).
__device__ __forceinline__ void ahead_block(const Blk &blk, int ahead_y, int ahead_x, int &bx, int &by)
{
    bx = blk.x + ahead_x;
    by = blk.y + ahead_y;
    if (bx >= blk.gx) {
        bx -= blk.gx;
        ++by;
    }
}

// Look-ahead prefetch of a block: lanes 0..13 of its first row of threads
// issue one bulk L2 prefetch each of the 14 source row segments of block
// (bx, by) of a grid over D (in a pass, only of rows holding that pass's
// tiles).
template <typename T, int V, int mode>
__device__ __forceinline__ void prefetch_block(const Dev &D, const T *__restrict__ Ain, int bx, int by)
{
    constexpr int kAl = 16 / (int)sizeof(T); // elements per 16 bytes
    const int span = (int)blockDim.x * V;   // nodes of a row per block
    if (threadIdx.x < kPop && threadIdx.y == 0) {
        // L2 prefetch of the source rows of the block at (pf_x, pf_y), the
        // one that runs about a residency wave later
        const int yb = by * (int)blockDim.y;
        const int xs = bx * span;
        const int lo = max(xs - kAl, 0), hi = min(xs + span + kAl, D.pitch);
        const int p = threadIdx.x;
        for (int yy = yb; yy < min(yb + (int)blockDim.y, D.ny) && hi > lo; ++yy) {
            if constexpr (mode != kSCAll) { // only rows of this pass's tiles
                bool want = false;
                for (int t = xs / (32 * V); t * 32 * V < min(xs + span, D.pitch); ++t)
                    want |= tile_near(D, yy, t) == (mode == kSCNear);
                if (!want) continue;
            }
            int ys = yy - ey(pdir(p));
            if (ys < 0 || ys >= D.ny) {
                if (!D.per_y) continue;
                ys = ys < 0 ? ys + D.ny : ys - D.ny;
            }
            const T *sp = Ain + (long long)p * D.ps + (long long)ys * D.pitch + lo;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sp),
                         "r"((unsigned)((hi - lo) * (int)sizeof(T)))
                         : "memory");
        }
    }
}

template <typename T, int V, bool kSharedFlags>
__device__ __forceinline__ void sc_tail(const Dev &D, const T *__restrict__ Ain, T *__restrict__ Aout,
                                        float (&c)[V][kPop], int x0, int y, const uint8_t *sflags);

// pf_x < 0: no look-ahead prefetch here (the caller issues its own).
template <typename T, int V, int mode = kSCAll>
__device__ __forceinline__ void sc_body(const Dev &D, const T *__restrict__ Ain, T *__restrict__ Aout, int pf_x,
                                        int pf_y, const Blk blk)
{
    using E = Elem<T>;
    using VW = typename Vec<T, V>::W;
    const int lane = threadIdx.x & 31;
    if (pf_x >= 0) prefetch_block<T, V, mode>(D, Ain, pf_x, pf_y);
    const int x0 = (blk.x * (int)blockDim.x + (int)threadIdx.x) * V;
    const int y = blk.y * (int)blockDim.y + (int)threadIdx.y;
    if (y >= D.ny) return; // uniform across the warp: blockDim.x is a multiple of 32
    // a warp wholly past the pitch (where the grid's last block of a row
    // overhangs it) has no node: it returns before its first load
    if (x0 - lane * V >= D.pitch) return;
    if constexpr (mode != kSCAll)
        if (tile_near(D, y, (x0 - (lane * V)) / (32 * V)) != (mode == kSCNear))
            return; // the other pass's tile (uniform across the warp)
    const bool act = x0 < D.pitch; // the pitch is a multiple of 32, so all V nodes are in the row
    float c[V][kPop];
    // A warp off the first and last row (the common case) pulls without any
    // wall, seam or range test.  In the first and last warp of a row, the
    // reads past the row's ends (x = -1, x >= nx, lanes past the pitch: at
    // most 32 V + 1 elements, since a warp starts below the pitch) land in
    // the previous plane (every plane with e_x = 1 has index p >= 1), the
    // next row or the buffer's tail pad, so they stay inside the buffer; the
    // values they bring feed only the planes of the side nodes x = 0 and
    // x = nx - 1 that pull across a wall or seam, which the general pull
    // replaces below, and the padding past nx, which is zeroed.
    const bool interior = y >= 1 && y + 1 < D.ny;
    if (interior) {
        const T *b0 = Ain + (long long)y * D.pitch + x0;
#pragma unroll
        for (int p = 0; p < kPop; ++p) {
            const int d = pdir(p);
            const int dx = ex(d), dy = ey(d);
            const T *src = b0 + (long long)p * D.ps - (long long)dy * D.pitch;
            const long long e = (long long)(src - Ain); // element index, for the bounds checks
            float v[V];
            if (in_bounds(D, e, D.a_elems - V + 1)) VecIo<T, V>::unpack(__ldg(reinterpret_cast<const VW *>(src)), v);
            else {
#pragma unroll
                for (int k = 0; k < V; ++k) v[k] = 0.f;
            }
            if (dx == 0) {
#pragma unroll
                for (int k = 0; k < V; ++k) c[k][p] = v[k];
            } else if (dx == 1) { // pull from x - 1
                float l = __shfl_up_sync(kFull, v[V - 1], 1);
                if (lane == 0) l = in_bounds(D, e - 1, D.a_elems) ? Io<T>::ld(__ldg(src - 1)) : 0.f;
                c[0][p] = l;
#pragma unroll
                for (int k = 1; k < V; ++k) c[k][p] = v[k - 1];
            } else { // pull from x + 1
                float r = __shfl_down_sync(kFull, v[0], 1);
                if (lane == 31) r = in_bounds(D, e + V, D.a_elems) ? Io<T>::ld(__ldg(src + V)) : 0.f;
#pragma unroll
                for (int k = 0; k + 1 < V; ++k) c[k][p] = v[k + 1];
                c[V - 1][p] = r;
            }
        }
    } else {
#pragma unroll
        for (int p = 0; p < kPop; ++p) {
            const int d = pdir(p);
            const int dx = ex(d), dy = ey(d);
            int ys = y - dy;
            bool rowok = ys >= 0 && ys < D.ny;
            if (!rowok && D.per_y) {
                ys = ys < 0 ? ys + D.ny : ys - D.ny;
                rowok = true;
            }
            const T *src = Ain + (long long)p * D.ps + (long long)(rowok ? ys : 0) * D.pitch;
            float v[V];
            if (act && rowok) VecIo<T, V>::unpack(__ldg(reinterpret_cast<const VW *>(src + x0)), v);
            else {
#pragma unroll
                for (int k = 0; k < V; ++k) v[k] = 0.f;
            }
            if (dx == 0) {
#pragma unroll
                for (int k = 0; k < V; ++k) c[k][p] = v[k];
            } else if (dx == 1) { // pull from x - 1
                float l = __shfl_up_sync(kFull, v[V - 1], 1);
                if (lane == 0) l = (act && rowok && x0 >= 1) ? Io<T>::ld(__ldg(src + x0 - 1)) : 0.f;
                c[0][p] = l;
#pragma unroll
                for (int k = 1; k < V; ++k) c[k][p] = v[k - 1];
            } else { // pull from x + 1
                float r = __shfl_down_sync(kFull, v[0], 1);
                if (lane == 31) r = (act && rowok && x0 + V < D.pitch) ? Io<T>::ld(__ldg(src + x0 + V)) : 0.f;
#pragma unroll
                for (int k = 0; k + 1 < V; ++k) c[k][p] = v[k + 1];
                c[V - 1][p] = r;
            }
        }
    }
    if (!act) return;
    sc_tail<T, V, false>(D, Ain, Aout, c, x0, y, nullptr);
}

// The part of a stream-collide update after the interior pulls, for the V
// nodes x0 .. x0 + V - 1 of row y whose pulled values c holds: the side
// nodes' wall or seam planes, the collision, the stores and the numeric
// check.  The nodes' flags are read from sflags (shared memory) or, without
// kSharedFlags, from the flag map where they are used (an address computed
// earlier and held cost the one-block-per-tile kernels registers).
template <typename T, int V, bool kSharedFlags>
__device__ __forceinline__ void sc_tail(const Dev &D, const T *__restrict__ Ain, T *__restrict__ Aout,
                                        float (&c)[V][kPop], int x0, int y, const uint8_t *sflags)
{
    using VW = typename Vec<T, V>::W;
    constexpr float kIo = Io<T>::kScaled ? kHalfScale : 1.f; // the side pulls' values in the kernel's scale
    const bool interior = y >= 1 && y + 1 < D.ny;
    // The nodes x = 0 and x = nx - 1 of the rows between the first and the
    // last: the planes that pull across a side wall or the periodic seam
    // take the wall rule or the far side's value (side_pull: the general
    // pull that k_boundary applies to the first and last rows, restricted
    // to that case, inlined: as a call it cost the 16-bit kernel 4 us of
    // its 180 through register allocation); every other plane
    // is the fast path's.  This warp thus writes whole sectors at the row's
    // ends, and the side columns need no scattered pass of their own.
    if (interior) {
        if (x0 == 0) {
#pragma unroll
            for (int p = 0; p < kPop; ++p)
                if (ex(pdir(p)) == 1) c[0][p] = side_pull(D, Ain, 0, y, p) * kIo;
        }
        const int kl = D.nx - 1 - x0;
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (k == kl) {
#pragma unroll
                for (int p = 0; p < kPop; ++p)
                    if (ex(pdir(p)) == -1) c[k][p] = side_pull(D, Ain, D.nx - 1, y, p) * kIo;
            }
    }
    bool ok = true, gen[V], anygen = false;
    if constexpr (V == 2) {
        // both nodes collided at once on paired FP32 instructions; solid
        // nodes (and the padding past nx) are zeroed after
        bool fluid[2];
        // both nodes' flags in one 2-byte load (x0 is even)
        const uint8_t *flp = kSharedFlags ? sflags : D.flags + (long long)y * D.pitch + x0;
        const unsigned short fl2 = *reinterpret_cast<const unsigned short *>(flp);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int x = x0 + k;
            const unsigned fl = (fl2 >> (8 * k)) & 0xffu;
            fluid[k] = x < D.nx && fl != kSolid;
            // newborn nodes and the first and last rows belong to k_boundary,
            // which writes them
            gen[k] = fluid[k] && (fl == kNewborn || y == 0 || y == D.ny - 1);
            anygen |= gen[k];
        }
        float2 cc[kPop];
#pragma unroll
        for (int p = 0; p < kPop; ++p) cc[p] = make_float2(c[0][p], c[1][p]);
        bool ok0, ok1;
        collide_t<float2, Io<T>::kScaled>(D, cc, ok0, ok1);
#pragma unroll
        for (int p = 0; p < kPop; ++p) {
            c[0][p] = cc[p].x;
            c[1][p] = cc[p].y;
        }
        if (!(fluid[0] && fluid[1])) { // solid nodes and the padding past nx hold zeros
#pragma unroll
            for (int p = 0; p < kPop; ++p) {
                if (!fluid[0]) c[0][p] = 0.f;
                if (!fluid[1]) c[1][p] = 0.f;
            }
        }
        ok = (!fluid[0] || gen[0] || ok0) && (!fluid[1] || gen[1] || ok1);
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int x = x0 + k;
            const uint8_t fl = kSharedFlags ? sflags[k] : D.flags[(long long)y * D.pitch + x];
            gen[k] = false;
            if (x < D.nx && fl != kSolid) {
                // newborn nodes and the first and last rows belong to
                // k_boundary, which writes them
                gen[k] = fl == kNewborn || y == 0 || y == D.ny - 1;
                if (!gen[k]) ok &= collide(D, c[k]);
            } else {
#pragma unroll
                for (int p = 0; p < kPop; ++p) c[k][p] = 0.f;
            }
            anygen |= gen[k];
        }
    }
    const long long d0 = (long long)y * D.pitch + x0;
    T *dst = Aout + d0;
    if (!anygen) {
#pragma unroll
        for (int p = 0; p < kPop; ++p) {
            float v[V];
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = c[k][p];
            if (in_bounds(D, d0 + (long long)p * D.ps, D.a_elems - V + 1))
                *reinterpret_cast<VW *>(dst + (long long)p * D.ps) = VecIo<T, V>::pack(v);
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (!gen[k]) {
#pragma unroll
                for (int p = 0; p < kPop; ++p)
                    if (in_bounds(D, d0 + (long long)p * D.ps + k, D.a_elems))
                        dst[(long long)p * D.ps + k] = Io<T>::st(c[k][p]);
            }
    }
    if (!ok) atomicOr(&D.status->err, kErrNumeric);
}

// General path, beside the stream-collide kernel (it reads only the previous
// state and writes only nodes that kernel leaves alone): the fluid nodes of
// the first and last rows (walls, periodic seams) and the newborn nodes
// listed by k_flags, each pulled (or refilled, Sec. 2.5) by slow_node and
// collided.  (The side columns' fluid nodes between those rows are the
// stream-collide kernel's.)
// A fixed grid strides over the 2 nx nodes of the two rows and then the
// list, whose length the device holds; a listed node on the frame (~n) is
// taken from the list unless it lies in those rows.
template <typename T>
__device__ __forceinline__ void boundary_body(const Dev &D, const T *__restrict__ Ain, T *__restrict__ Aout,
                                              const int *__restrict__ own_cur, int parity, const Blk blk)
{
    using E = Elem<T>;
    const int nx = D.nx, ny = D.ny;
    const int nframe = 2 * nx;
    const int nlist = min((int)D.status->nb, D.newborn_cap);
    unsigned n4[4] = {0u, 0u, 0u, 0u};
    bool ok = true;
    for (int idx = blk.x * (int)blockDim.x + (int)threadIdx.x; idx < nframe + nlist; idx += blk.gx * (int)blockDim.x) {
        int x, y;
        if (idx < nx) { x = idx; y = 0; }
        else if (idx < nframe) { x = idx - nx; y = ny - 1; }
        else {
            const int v = D.newborn[idx - nframe], n = v < 0 ? ~v : v;
            y = n / nx;
            x = n - y * nx;
            if (v < 0 && (y == 0 || y == ny - 1)) continue; // visited above
        }
        const long long o = (long long)y * D.pitch + x;
        const uint8_t fl = D.flags[o];
        if (fl == kSolid) continue;
        float c[kPop];
        const int r = slow_node(D, Ain, own_cur, x, y, fl, c);
        if (r) {
            n4[0] += 1u;
            n4[1] += r == 2;
            n4[2] += r == 3;
            n4[3] += r == 4;
        }
        ok &= collide(D, c);
#pragma unroll
        for (int p = 0; p < kPop; ++p)
            if (in_bounds(D, (long long)p * D.ps + o, D.a_elems)) Aout[(long long)p * D.ps + o] = E::st(c[p]);
    }
    flush_counters(D, parity, n4);
    if (!ok) atomicOr(&D.status->err, kErrNumeric);
}

// Blocks per SM that measured best on the 4000^2 benchmark: FP32 10 (48
// registers; 268 us against 272 with 8 and 279 with 12), 16-bit storage 9
// (at most 56 registers, a few spilled: BF16 180.8 us against 184.6 with 8
// and 181.8 with 10; the kernel waits on L2 latency as much as on issue, so
// the ninth block's warps outweigh the spills).
template <typename T, int V, int mode>
__global__ void __launch_bounds__(kSCThreads, V == 1 ? 10 : 9)
    k_stream_collide(const Dev D, const T *__restrict__ Ain, T *__restrict__ Aout, int ahead_y, int ahead_x)
{
    const Blk blk = this_blk();
    int bx, by;
    ahead_block(blk, ahead_y, ahead_x, bx, by);
    sc_body<T, V, mode>(D, Ain, Aout, bx, by, blk);
}


// ---------------------------------------------------------------------------
// Staged stream-collide (the whole-lattice pass with BF16 / FP16 storage).
// The same update as k_stream_collide, bit for bit, organised around shared
// memory: a persistent grid of 128-thread blocks takes row tiles of 128 V
// nodes in row order from a device counter (kStChunk consecutive tiles per
// claim, handed out one iteration ahead by thread 0), and each block keeps
// kStStages tiles in flight.  For a tile, 15 bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on the stage's mbarrier) bring
// the 14 planes' source row segments, each with 16 bytes more on the side
// its plane pulls from, and the tile's flags (over a batch a sixteenth brings
// the tile's instance record); lanes 0-3 of the four warps issue one each
// (st_lane, st_issue).  The block collides one tile from shared memory while
// the copies of the next ones are in flight: the memory latency overlaps the
// arithmetic without holding registers, and every pulled value is a
// shared-memory load at a fixed offset from one base (no shuffles, no edge
// loads, no per-plane address arithmetic).  Rows stay in launch order, so
// the tiles in flight form a compact band of rows, as in k_stream_collide.
//
// Shared memory per stage: 14 plane segments of 128 V + 2 H elements
// (H = 16 bytes of elements; node x_s + i at element H + i), then the
// tile's 128 V flag bytes.  The reads past a row's ends (x = -H .. -1 for a
// plane pulling from x - 1, which has index p >= 1, so the previous plane or
// row lies there; x = pitch .. pitch + H - 1 for one pulling from x + 1, the
// next row, plane or the buffer's tail pad) feed only the side nodes' wall or
// seam planes, which sc_tail replaces, and the zeroed padding.  The first and
// last rows read clamped source rows: every fluid node there belongs to
// k_boundary, and the others are stored as zeros.
//
// Every wait on an mbarrier is bounded (one second of the global timer);
// one that runs out records kErrTimeout (LBM_ETIMEOUT), and the block waits,
// again bounded, for its copies still in flight before it leaves.
// ---------------------------------------------------------------------------
#ifndef LBM_ST_STAGES
#define LBM_ST_STAGES 3
#endif
constexpr int kStStages = LBM_ST_STAGES;
#ifndef LBM_ST_MINB
#define LBM_ST_MINB 8
#endif
constexpr unsigned long long kStWaitNs = 1000000000ull;

template <typename T, int V, bool kInst = false>
struct StGeo {
    static constexpr int W = kSCThreads * V;                     // nodes of a tile
    static constexpr int H = 16 / (int)sizeof(T);                // halo elements on a pulled side
    static constexpr int SEG_B = (W + 2 * H) * (int)sizeof(T);   // bytes of a plane segment
    static constexpr int FLAGS_OFF = kPop * SEG_B;               // the tile's flags
    // with kInst (a batch): the tile's instance record (state, buffers)
    static constexpr int INST_OFF = (FLAGS_OFF + W + 15) / 16 * 16;
    static constexpr int INST_B = kInst ? (int)sizeof(InstArgs) : 0;
    static constexpr int STAGE_B = (INST_OFF + INST_B + 127) / 128 * 128;
    static constexpr int SMEM_B = kStStages * STAGE_B + 128;     // + barriers and tile slots
};
static_assert(sizeof(InstArgs) % 16 == 0, "an instance record is copied whole by a bulk copy");
// Planes whose source lies one node to the side (e_x != 0): they copy H
// elements more.
__host__ __device__ constexpr int shifted_planes()
{
    int n = 0;
    for (int p = 0; p < kPop; ++p) n += ex(pdir(p)) != 0;
    return n;
}

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned bar, unsigned tx)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity)
{
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity to complete, for at most kStWaitNs.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > kStWaitNs) return false;
    return true;
}
__device__ __forceinline__ void bulk_to_smem(unsigned dst, const void *src, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Shared memory after the stages: a `full` barrier per stage (complete when
// the tile's copies have landed), the tile of each stage (instance, row y,
// first column xs; y < 0: no tile), and two slots that pass the next claimed
// tile from thread 0 to the block.
template <typename T, int V, bool kInst = false>
struct StTail {
    unsigned long long *full;
    int4 *stile, *snext;
    int *chunk; // thread 0's claim state: the index of the last tile handed out, tiles left in its chunk
    __device__ explicit StTail(unsigned char *sm)
    {
        full = reinterpret_cast<unsigned long long *>(sm + kStStages * StGeo<T, V, kInst>::STAGE_B);
        stile = reinterpret_cast<int4 *>(sm + kStStages * StGeo<T, V, kInst>::STAGE_B + 32);
        snext = stile + kStStages;
        chunk = reinterpret_cast<int *>(snext + 2);
    }
};
static_assert(kStStages * 8 <= 32 && 32 + (kStStages + 2) * 16 + 8 <= 128, "staged stream-collide: tail layout");

// The copy a thread issues for every tile, fixed for the launch: copy c
// (planes 0..13, then the flags, then in a batch the tile's instance record)
// belongs to lane c % 4 of warp c / 4, so no warp carries the copies alone.  Three registers: the copy (-1 none, kPop
// the flags), its shared-memory destination in stage 0, and for a plane its
// row shift e_y + 1 (bits 0-1) and whether it pulls from x - 1 (bit 2) or
// x + 1 (bit 3), i.e. takes H elements more on that side.
struct StLane {
    int c;
    unsigned dst;
    int meta;
};
template <typename T, int V, bool kInst = false>
__device__ __forceinline__ StLane st_lane(unsigned char *sm)
{
    using G = StGeo<T, V, kInst>;
    const int lane = threadIdx.x & 31, c = (threadIdx.x >> 5) * 4 + lane;
    if (kInst && lane < 4 && c == kPop + 1) return StLane{c, smem_addr(sm + G::INST_OFF), 0}; // the record
    if (lane >= 4 || c > kPop) return StLane{-1, 0u, 0};
    if (c == kPop) return StLane{c, smem_addr(sm + G::FLAGS_OFF), 0};
    const int d = pdir(c), dx = ex(d);
    return StLane{c, smem_addr(sm + c * G::SEG_B) + (unsigned)((dx == 1 ? 0 : G::H) * (int)sizeof(T)),
                  (ey(d) + 1) | (dx == 1 ? 4 : 0) | (dx == -1 ? 8 : 0)};
}

// The block loads the tile of row y, columns xs .. xs + W - 1 (of the
// instance whose state D and Ain hold), into stage s, each thread issuing its
// copy; thread 0 first records the tile and
// announces the bytes (a copy that lands before the announcement only makes
// the byte count negative for a while; the phase cannot complete before
// thread 0's arrival).  y < 0: nothing to load, the stage's phase completes
// at once and tells the block to stop.  Every thread passes the same tile.
template <typename T, int V, bool kInst = false>
__device__ __forceinline__ void st_issue(const Dev &D, const T *__restrict__ Ain, unsigned char *sm, int s, int4 tile,
                                         const StLane &L, const InstArgs *rec = nullptr)
{
    using G = StGeo<T, V, kInst>;
    const StTail<T, V, kInst> t(sm);
    const unsigned b = smem_addr(t.full + s);
    const int y = tile.y, xs = tile.z;
    const int n = min(G::W, D.pitch - xs); // nodes of the tile
    if (threadIdx.x == 0) {
        t.stile[s] = tile;
        if (y < 0) mbar_arrive(b);
        else
            mbar_arrive_tx(b, (unsigned)(n * (kPop * (int)sizeof(T) + 1) + shifted_planes() * 16 + G::INST_B +
                                         D.sc_extra_tx));
    }
    if (y < 0 || L.c < 0) return;
    const unsigned dst = L.dst + (unsigned)(s * G::STAGE_B);
    if (kInst && L.c == kPop + 1) { // the tile's instance record
        bulk_to_smem(dst, rec, (unsigned)G::INST_B, b);
        return;
    }
    if (L.c == kPop) { // the tile's flags
        bulk_to_smem(dst, D.flags + (long long)y * D.pitch + xs, (unsigned)n, b);
        return;
    }
    int ys = y - ((L.meta & 3) - 1);
    if ((unsigned)ys >= (unsigned)D.ny) {
        if (D.per_y) ys = ys < 0 ? ys + D.ny : ys - D.ny;
        else ys = min(max(ys, 0), D.ny - 1); // the first or last row: values unused
    }
    const int halo = (L.meta & 12) ? G::H : 0;
    long long e = (long long)L.c * D.ps + (long long)ys * D.pitch + xs - ((L.meta & 4) ? G::H : 0);
    if (!(in_bounds(D, e, D.a_elems) && in_bounds(D, e + n + halo - 1, D.a_elems))) e = 0; // checked builds
    bulk_to_smem(dst, Ain + e, (unsigned)((n + halo) * (int)sizeof(T)), b);
}

// Tiles claimed per step of the work counter: consecutive tiles, the first
// looked up, the others found from it (next column, next row, or, at the
// end of an instance, looked up), so the counter's round trip and the
// lookup's dependent loads come once per kStChunk tiles.
constexpr int kStChunk = 4;

// The staged loop over the tiles a policy P hands out: P::decode(it) maps a
// tile index to a tile (int4: instance, row, first column; row -1 past the
// end), P::next(t, it) gives tile it from tile it - 1, P::dev / ain / aout
// give an instance's state and buffers, P::ctr the work counter (in chunks
// of kStChunk tiles) and the done count after it, P::err the error word a
// timeout is recorded in.
template <typename T, int V, typename P>
__device__ __forceinline__ void staged_body(const P &pol)
{
    constexpr bool kInst = P::kInst;
    using G = StGeo<T, V, kInst>;
    using E = Elem<T>;
    using VW = typename Vec<T, V>::W;
    extern __shared__ __align__(128) unsigned char sm[];
    const StTail<T, V, kInst> t(sm);
    const int tid = threadIdx.x;
    const StLane L = st_lane<T, V, kInst>(sm);
    unsigned *ctr = pol.ctr();
    // thread 0: the tile after `last`, the last one it handed out
    auto claim = [&](int4 last) {
        int it = t.chunk[0], left = t.chunk[1];
        if (left == 0) {
            it = (int)atomicAdd(ctr, 1u) * kStChunk;
            left = kStChunk;
            last = pol.decode(it);
        } else {
            last = pol.next(last, ++it);
        }
        t.chunk[0] = it;
        t.chunk[1] = left - 1;
        return last;
    };

    // thread 0 claims the first kStStages tiles (after the first one past
    // the end, none): kStStages - 1 to load now, one for the first refill
    if (tid == 0) {
        for (int s = 0; s < kStStages; ++s) mbar_init(smem_addr(t.full + s), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        t.chunk[1] = 0;
        int4 tile = make_int4(0, 0, 0, 0);
        for (int s = 0; s < kStStages; ++s) {
            tile = tile.y < 0 ? tile : claim(tile);
            if (s + 1 < kStStages) t.stile[s] = tile;
            else t.snext[0] = tile;
        }
    }
    __syncthreads();
    for (int s = 0; s + 1 < kStStages; ++s) {
        const int4 tile = t.stile[s];
        __syncthreads(); // every thread has read the slot st_issue rewrites
        st_issue<T, V, kInst>(pol.dev(tile.x), pol.ain(tile.x), sm, s, tile, L, pol.rec(tile.x));
    }
    bool timeout = false;
    int k = 0;
    for (;; ++k) {
        const int s = k % kStStages;
        // refill the stage the block finished with in the last iteration
        // with the tile claimed then; thread 0 claims the one after it
        const int4 nt = t.snext[k & 1];
        st_issue<T, V, kInst>(pol.dev(nt.x), pol.ain(nt.x), sm, (k + kStStages - 1) % kStStages, nt, L,
                              pol.rec(nt.x));
        int4 claimed = make_int4(0, -1, 0, 0);
        if (tid == 0 && nt.y >= 0) claimed = claim(nt);
        const bool got = mbar_wait(smem_addr(t.full + s), (unsigned)(k / kStStages) & 1u);
        const int4 tile = got ? t.stile[s] : make_int4(0, -1, 0, 0);
        const int y = tile.y;
        if (y >= 0) {
            const unsigned char *sb = sm + s * G::STAGE_B;
            // a batch's instance record came with the tile
            const InstArgs *rec = reinterpret_cast<const InstArgs *>(sb + G::INST_OFF);
            const Dev &D = kInst ? rec->D : pol.dev(tile.x);
            const int x0 = tile.z + tid * V;
            if (x0 < D.pitch) { // threads past the pitch have no node
                float c[V][kPop];
#pragma unroll
                for (int p = 0; p < kPop; ++p) {
                    const int dx = ex(pdir(p));
                    const T *seg = reinterpret_cast<const T *>(sb + p * G::SEG_B) + G::H + tid * V;
                    if constexpr (V == 1) {
                        c[0][p] = E::ld(seg[-dx]);
                    } else {
                        float a[2];
                        VecIo<T, V>::unpack(*reinterpret_cast<const VW *>(seg), a);
                        if (dx == 0) {
                            c[0][p] = a[0];
                            c[1][p] = a[1];
                        } else if (dx == 1) { // pull from x - 1
                            float l[2];
                            VecIo<T, V>::unpack(*reinterpret_cast<const VW *>(seg - 2), l);
                            c[0][p] = l[1];
                            c[1][p] = a[0];
                        } else { // pull from x + 1
                            float r[2];
                            VecIo<T, V>::unpack(*reinterpret_cast<const VW *>(seg + 2), r);
                            c[0][p] = a[1];
                            c[1][p] = r[0];
                        }
                    }
                }
                const T *ain;
                T *aout;
                if constexpr (kInst) {
                    const int par = pol.parity ^ rec->poff;
                    ain = static_cast<const T *>(rec->A[par]);
                    aout = static_cast<T *>(rec->A[par ^ 1]);
                } else {
                    ain = pol.ain(tile.x);
                    aout = pol.aout(tile.x);
                }
                sc_tail<T, V, true>(D, ain, aout, c, x0, y, sb + G::FLAGS_OFF + tid * V);
            }
        }
        if (tid == 0) t.snext[(k + 1) & 1] = claimed;
        // every thread is done with stage s and has read snext[k & 1]; stop
        // together at the end of the work or after a wait ran out
        if (__syncthreads_or(y < 0)) {
            timeout = __syncthreads_or(!got);
            break;
        }
    }
    if (timeout) {
        if (tid == 0) atomicOr(pol.err(), kErrTimeout);
        // copies may still be in flight into the stages of iterations k ..
        // k + kStStages - 1: wait for them (bounded) before leaving
        for (int j = k; j < k + kStStages; ++j)
            if (!mbar_wait(smem_addr(t.full + j % kStStages), (unsigned)(j / kStStages) & 1u)) break;
        __syncthreads();
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(ctr + 1, 1u) == gridDim.x - 1) { // the last block: reset for the next launch
            ctr[0] = 0u;
            ctr[1] = 0u;
            __threadfence();
        }
    }
}

// One instance: tiles in row order, ntx per row.
template <typename T, int V>
struct StSingle {
    static constexpr bool kInst = false;
    const Dev &D;
    const T *Ain;
    T *Aout;
    int ntx, nitems;
    __device__ int4 decode(int it) const
    {
        if (it >= nitems) return make_int4(0, -1, 0, 0);
        const int y = it / ntx;
        return make_int4(0, y, (it - y * ntx) * StGeo<T, V>::W, 0);
    }
    __device__ int4 next(int4 t, int it) const
    {
        if (t.y < 0 || it >= nitems) return make_int4(0, -1, 0, 0);
        t.z += StGeo<T, V>::W;
        if (t.z >= D.pitch) {
            t.z = 0;
            ++t.y;
        }
        return t;
    }
    __device__ const Dev &dev(int) const { return D; }
    __device__ const InstArgs *rec(int) const { return nullptr; }
    __device__ const T *ain(int) const { return Ain; }
    __device__ T *aout(int) const { return Aout; }
    __device__ unsigned *ctr() const { return &D.status->sc_next; }
    __device__ unsigned *err() const { return &D.status->err; }
};
static_assert(offsetof(Status, sc_done) == offsetof(Status, sc_next) + sizeof(unsigned), "work counter pair");

// A batch: the tiles of all instances, instance by instance, found through
// the batch's stream-collide records and buckets of the 128 x 1 tile shape
// (one 128 V-node row tile per block); a timeout is recorded in instance 0's
// error word (the batch's sync reads every instance's).
template <typename T, int V>
struct StBatch {
    static constexpr bool kInst = true;
    const InstArgs *__restrict__ I;
    const ScInst *__restrict__ sc;
    const int *__restrict__ bucket;
    int shift, n, total, parity;
    unsigned *counter;
    __device__ int4 decode(int it) const
    {
        if (it >= total) return make_int4(0, -1, 0, 0);
        const int i = sc_find(sc, bucket, shift, n, it);
        int bx, by;
        sc_tile(sc + i, it, bx, by);
        return make_int4(i, by, bx * StGeo<T, V, true>::W, 0);
    }
    __device__ int4 next(int4 t, int it) const
    {
        if (t.y < 0 || it >= total) return make_int4(0, -1, 0, 0);
        const Dev &D = I[t.x].D;
        t.z += StGeo<T, V, true>::W;
        if (t.z >= D.pitch) {
            t.z = 0;
            if (++t.y >= D.ny) return decode(it); // the next instance
        }
        return t;
    }
    __device__ const Dev &dev(int i) const { return I[i].D; }
    __device__ const InstArgs *rec(int i) const { return I + i; }
    __device__ const T *ain(int i) const { return static_cast<const T *>(I[i].A[parity ^ I[i].poff]); }
    __device__ T *aout(int i) const { return static_cast<T *>(I[i].A[parity ^ I[i].poff ^ 1]); }
    __device__ unsigned *ctr() const { return counter; }
    __device__ unsigned *err() const { return &I[0].D.status->err; }
};

template <typename T, int V>
__global__ void __launch_bounds__(kSCThreads, LBM_ST_MINB)
    k_stream_collide_staged(const Dev D, const T *__restrict__ Ain, T *__restrict__ Aout, int ntx, int nitems)
{
    staged_body<T, V>(StSingle<T, V>{D, Ain, Aout, ntx, nitems});
}

template <typename T, int V>
__global__ void __launch_bounds__(kSCThreads, LBM_ST_MINB)
    k_stream_collide_staged_batch(const InstArgs *__restrict__ I, const ScInst *__restrict__ sc,
                                  const int *__restrict__ bucket, int shift, int n, int total, int parity,
                                  unsigned *counter)
{
    staged_body<T, V>(StBatch<T, V>{I, sc, bucket, shift, n, total, parity, counter});
}

template <typename T>
__global__ void __launch_bounds__(128)
    k_boundary(const Dev D, const T *__restrict__ Ain, T *__restrict__ Aout, const int *__restrict__ own_cur,
               int parity)
{
    boundary_body<T>(D, Ain, Aout, own_cur, parity, this_blk());
}

// Batched forms: one grid over all instances.  Stream-collide blocks are
// laid out per instance as gx x gy tiles of the instance's lattice (gx from
// its pitch); a block finds its instance and tile from two small tables (a
// bucket table and the per-instance records, no search and no division),
// and prefetches the block `resident` places later in the launch over all
// instances (often one of a later instance: prefetching only within the
// block's own instance left most blocks of small instances without a
// prefetch).
template <typename T, int V>
__global__ void __launch_bounds__(kSCThreads, V == 1 ? 10 : 9) // as k_stream_collide (BF16 ensemble: 0.516 against 0.522 ms per step with 8)
    k_stream_collide_batch(const InstArgs *__restrict__ I, const ScInst *__restrict__ sc,
                           const int *__restrict__ bucket, int shift, int n, int total, int parity, int resident)
{
    // the look-ahead target is the block `resident` places later in the
    // launch over all instances, which is often in a later instance
    const int tg = (int)blockIdx.x + resident;
    if (threadIdx.x < kPop && threadIdx.y == 0 && tg < total) {
        const int j = sc_find(sc, bucket, shift, n, tg);
        const InstArgs &t = I[j];
        int bx, by;
        sc_tile(sc + j, tg, bx, by);
        prefetch_block<T, V, kSCAll>(t.D, static_cast<const T *>(t.A[parity ^ t.poff]), bx, by);
    }
    const int i = sc_find(sc, bucket, shift, n, (int)blockIdx.x);
    const InstArgs &a = I[i];
    int bx, by;
    sc_tile(sc + i, (int)blockIdx.x, bx, by);
    const Blk blk{bx, by, 0, 0}; // the grid extents are not used by the body
    const int par = parity ^ a.poff;
    sc_body<T, V>(a.D, static_cast<const T *>(a.A[par]), static_cast<T *>(a.A[par ^ 1]), -1, 0, blk);
}

template <typename T>
__global__ void __launch_bounds__(128)
    k_boundary_batch(const InstArgs *__restrict__ I, const int *__restrict__ start, int n, int parity)
{
    __shared__ Dev sD;
    const int i = batch_find(start, n, (int)blockIdx.x);
    const InstArgs &a = I[i];
    copy_dev(sD, a.D);
    const int s0 = __ldg(start + i);
    const Blk blk{(int)blockIdx.x - s0, 0, __ldg(start + i + 1) - s0, 1};
    const int par = parity ^ a.poff;
    boundary_body<T>(sD, static_cast<const T *>(a.A[par]), static_cast<T *>(a.A[par ^ 1]), a.own[par], par,
                     blk);
}

// Collision without streaming, for the initial state and for distributions
// supplied by the caller (mode 1 reads pre-collision values from Ain).
template <typename T>
__global__ void k_init_collide(const Dev D, const T *__restrict__ Ain, T *__restrict__ Aout, float T_init,
                               int mode)
{
    using E = Elem<T>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= D.pitch || y >= D.ny) return;
    const long long n = (long long)y * D.pitch + x;
    float c[kPop];
    const bool live = x < D.nx && D.flags[n] != kSolid;
    for (int p = 0; p < kPop; ++p) {
        if (mode == 1) c[p] = E::ld(Ain[(long long)p * D.ps + n]);
        else c[p] = p < kQ9 ? 0.f : w5(p - kQ9) * T_init;
    }
    if (live) {
        if (!collide(D, c)) atomicOr(&D.status->err, kErrNumeric);
    } else {
        for (int p = 0; p < kPop; ++p) c[p] = 0.f;
    }
    for (int p = 0; p < kPop; ++p) Aout[(long long)p * D.ps + n] = E::st(c[p]);
}

// rho - 1, u, T from the post-collision state: the collision keeps rho and
// T and adds F to the momentum, so u = (sum e f+ - F/2)/rho equals the
// pre-collision (sum e f + F/2)/rho of Sec. 2.1.
template <typename S>
__global__ void k_fields(const Dev D, const S *__restrict__ A, int row0, float *rho_o, float *ux_o,
                         float *uy_o, float *T_o)
{
    using E = Elem<S>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = row0 + blockIdx.y;
    if (x >= D.nx || y >= D.ny) return;
    const long long n = (long long)y * D.pitch + x;
    const long long o = (long long)blockIdx.y * D.nx + x;
    if (D.flags[n] == kSolid) {
        const float nan = __int_as_float(0x7fc00000);
        rho_o[o] = nan; ux_o[o] = nan; uy_o[o] = nan; T_o[o] = nan;
        return;
    }
    float f[kQ9], T = 0.f, drho = 0.f, jx = 0.f, jy = 0.f;
    for (int i = 0; i < kQ9; ++i) {
        f[i] = E::ld(A[(long long)i * D.ps + n]);
        drho += f[i];
        jx += ex(i) * f[i];
        jy += ey(i) * f[i];
    }
    for (int i = 0; i < kQ5; ++i) T += E::ld(A[(long long)(kQ9 + i) * D.ps + n]);
    const float rho = 1.f + drho;
    const float Fx = D.bfx, Fy = rho * D.gbeta * (T - D.T0) + D.bfy;
    rho_o[o] = drho;
    ux_o[o] = (jx - 0.5f * Fx) / rho;
    uy_o[o] = (jy - 0.5f * Fy) / rho;
    T_o[o] = T;
}

namespace {

template <typename T, int V, int mode>
cudaError_t stream_collide_m(const Dev &D, const void *Ain, void *Aout, cudaStream_t s)
{
    static int resident = 0;
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide<T, V, mode>, kSCThreads, 0);
        resident = max(1, sms * per_sm);
    }
    const int tx = D.pitch / V; // threads per row (the pitch is a multiple of 32)
    int bx = ((tx + 31) / 32) * 32;
    if (bx > kSCThreads) bx = kSCThreads;
    const int by = kSCThreads / bx;
    dim3 block(bx, by);
    dim3 grid((tx + bx - 1) / bx, (D.ny + by - 1) / by);
    k_stream_collide<T, V, mode><<<grid, block, 0, s>>>(D, static_cast<const T *>(Ain), static_cast<T *>(Aout),
                                                        resident / (int)grid.x, resident % (int)grid.x);
    return cudaGetLastError();
}

// Blocks of a staged kernel the GPU holds at once (carveout set to the
// largest shared-memory share first).
template <typename K>
int staged_resident(K kernel, int smem)
{
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess) return 0;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kSCThreads, smem) != cudaSuccess) return 0;
    return max(1, sms * per_sm);
}

// The staged kernel's grid: as many blocks as the GPU holds at once (they
// claim tiles from the work counter, so blocks that start late, behind the
// boundary kernel's, take fewer).
template <typename T, int V>
cudaError_t stream_collide_staged(const Dev &D, const void *Ain, void *Aout, cudaStream_t s)
{
    using G = StGeo<T, V>;
    static int resident = 0;
    if (!resident && !(resident = staged_resident(k_stream_collide_staged<T, V>, G::SMEM_B)))
        return cudaErrorInvalidValue;
    const int ntx = (D.pitch + G::W - 1) / G::W;
    const int nitems = ntx * D.ny;
    k_stream_collide_staged<T, V><<<min(resident, nitems), kSCThreads, G::SMEM_B, s>>>(
        D, static_cast<const T *>(Ain), static_cast<T *>(Aout), ntx, nitems);
    return cudaGetLastError();
}

template <typename T, int V>
cudaError_t stream_collide_staged_batch(const InstArgs *I, const ScInst *sc, const int *bucket, int shift, int n,
                                        int total, int parity, unsigned *counter, cudaStream_t s)
{
    using G = StGeo<T, V, true>;
    static int resident = 0;
    if (!resident && !(resident = staged_resident(k_stream_collide_staged_batch<T, V>, G::SMEM_B)))
        return cudaErrorInvalidValue;
    k_stream_collide_staged_batch<T, V><<<min(resident, total), kSCThreads, G::SMEM_B, s>>>(I, sc, bucket, shift, n,
                                                                                          total, parity, counter);
    return cudaGetLastError();
}

template <typename T, int V>
cudaError_t stream_collide_t(const Dev &D, const void *Ain, void *Aout, int mode, cudaStream_t s)
{
    switch (mode) {
    case kSCFar: return stream_collide_m<T, V, kSCFar>(D, Ain, Aout, s);
    case kSCNear: return stream_collide_m<T, V, kSCNear>(D, Ain, Aout, s);
    default:
        return D.sc_staged ? stream_collide_staged<T, V>(D, Ain, Aout, s)
                           : stream_collide_m<T, V, kSCAll>(D, Ain, Aout, s);
    }
}

template <typename T>
cudaError_t boundary_t(const Dev &D, const void *Ain, void *Aout, const int *own_cur, int parity, cudaStream_t s)
{
    static int blocks = 0;
    if (!blocks) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks = max(1, 2 * sms);
    }
    k_boundary<T><<<blocks, 128, 0, s>>>(D, static_cast<const T *>(Ain), static_cast<T *>(Aout), own_cur, parity);
    return cudaGetLastError();
}

template <typename T>
cudaError_t init_collide_t(const Dev &D, const void *Ain, void *Aout, float T_init, int mode, cudaStream_t s)
{
    dim3 block(128);
    dim3 grid((D.pitch + 127) / 128, D.ny);
    k_init_collide<T><<<grid, block, 0, s>>>(D, static_cast<const T *>(Ain), static_cast<T *>(Aout), T_init,
                                             mode);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fields_t(const Dev &D, const void *A, int row0, int rows, float *rho, float *ux, float *uy,
                     float *Tf, cudaStream_t s)
{
    dim3 block(128);
    dim3 grid((D.nx + 127) / 128, rows);
    k_fields<T><<<grid, block, 0, s>>>(D, static_cast<const T *>(A), row0, rho, ux, uy, Tf);
    return cudaGetLastError();
}

} // namespace

int near_tiles_per_row(int storage, int pitch)
{
    const int span = 32 * (storage == LBM_STORE_FP32 ? 1 : 2);
    return (pitch + span - 1) / span;
}

cudaError_t launch_stream_collide(const Dev &D, const void *Ain, void *Aout, int mode, cudaStream_t s)
{
    switch (D.storage) {
    case LBM_STORE_FP32: return stream_collide_t<float, 1>(D, Ain, Aout, mode, s);
    case LBM_STORE_BF16: return stream_collide_t<__nv_bfloat16, 2>(D, Ain, Aout, mode, s);
    case LBM_STORE_FP16: return stream_collide_t<__half, 2>(D, Ain, Aout, mode, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t stream_collide_binary_version(int *version)
{
    cudaFuncAttributes a{};
    const cudaError_t e = cudaFuncGetAttributes(&a, k_stream_collide<float, 1, kSCAll>);
    if (e == cudaSuccess) *version = a.binaryVersion;
    return e;
}

cudaError_t launch_boundary(const Dev &D, const void *Ain, void *Aout, const int *own_cur, int parity,
                            cudaStream_t s)
{
    switch (D.storage) {
    case LBM_STORE_FP32: return boundary_t<float>(D, Ain, Aout, own_cur, parity, s);
    case LBM_STORE_BF16: return boundary_t<__nv_bfloat16>(D, Ain, Aout, own_cur, parity, s);
    case LBM_STORE_FP16: return boundary_t<__half>(D, Ain, Aout, own_cur, parity, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stream_collide_batch(const InstArgs *I, const ScInst *sc, const int *bucket, int shift, int n,
                                        int total, int storage, int parity, dim3 block, int resident,
                                        cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    switch (storage) {
    case LBM_STORE_FP32:
        k_stream_collide_batch<float, 1><<<total, block, 0, s>>>(I, sc, bucket, shift, n, total, parity, resident);
        break;
    case LBM_STORE_BF16:
        k_stream_collide_batch<__nv_bfloat16, 2>
            <<<total, block, 0, s>>>(I, sc, bucket, shift, n, total, parity, resident);
        break;
    case LBM_STORE_FP16:
        k_stream_collide_batch<__half, 2><<<total, block, 0, s>>>(I, sc, bucket, shift, n, total, parity, resident);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_boundary_batch(const InstArgs *I, const int *start, int n, int total, int storage, int parity,
                                  cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    switch (storage) {
    case LBM_STORE_FP32: k_boundary_batch<float><<<total, 128, 0, s>>>(I, start, n, parity); break;
    case LBM_STORE_BF16: k_boundary_batch<__nv_bfloat16><<<total, 128, 0, s>>>(I, start, n, parity); break;
    case LBM_STORE_FP16: k_boundary_batch<__half><<<total, 128, 0, s>>>(I, start, n, parity); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_stream_collide_staged_batch(const InstArgs *I, const ScInst *sc, const int *bucket, int shift,
                                               int n, int total, int storage, int parity, unsigned *counter,
                                               cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    switch (storage) {
    case LBM_STORE_BF16:
        return stream_collide_staged_batch<__nv_bfloat16, 2>(I, sc, bucket, shift, n, total, parity, counter, s);
    case LBM_STORE_FP16: return stream_collide_staged_batch<__half, 2>(I, sc, bucket, shift, n, total, parity, counter, s);
    default: return cudaErrorInvalidValue;
    }
}

int stream_collide_batch_resident(int storage, dim3 block)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nt = (int)(block.x * block.y);
    switch (storage) {
    case LBM_STORE_BF16:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_batch<__nv_bfloat16, 2>, nt, 0);
        break;
    case LBM_STORE_FP16:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_batch<__half, 2>, nt, 0);
        break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_batch<float, 1>, nt, 0);
    }
    return max(1, sms * per_sm);
}

cudaError_t launch_init_collide(const Dev &D, const void *Ain, void *Aout, float T_init, int mode,
                                cudaStream_t s)
{
    switch (D.storage) {
    case LBM_STORE_FP32: return init_collide_t<float>(D, Ain, Aout, T_init, mode, s);
    case LBM_STORE_BF16: return init_collide_t<__nv_bfloat16>(D, Ain, Aout, T_init, mode, s);
    case LBM_STORE_FP16: return init_collide_t<__half>(D, Ain, Aout, T_init, mode, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fields(const Dev &D, const void *A, int row0, int rows, float *rho, float *ux, float *uy,
                          float *T, cudaStream_t s)
{
    switch (D.storage) {
    case LBM_STORE_FP32: return fields_t<float>(D, A, row0, rows, rho, ux, uy, T, s);
    case LBM_STORE_BF16: return fields_t<__nv_bfloat16>(D, A, row0, rows, rho, ux, uy, T, s);
    case LBM_STORE_FP16: return fields_t<__half>(D, A, row0, rows, rho, ux, uy, T, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace lbm
