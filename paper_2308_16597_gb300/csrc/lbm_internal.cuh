// Internal declarations of the sm_103a lattice Boltzmann library: lattice
// constants, the device view of the caller's workspace, exact geometry
// helpers and the kernel launchers.  Not part of the public ABI (lbm.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Lattices (Sec. 2.1).  D2Q9 e0..e8 as in lbm.h; D2Q5 uses e0..e4.  The 14
// stored populations are the 9 flow deviations f~_i = f_i - w_i followed by
// the 5 raw temperature populations g_i.
// ---------------------------------------------------------------------------
constexpr int kQ9 = 9;
constexpr int kQ5 = 5;
constexpr int kPop = 14;

__host__ __device__ constexpr int ex(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i)
{
    return i == 0 ? 0 : i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5;
}
// D2Q9 weights (4/9, 1/9, 1/36).
__host__ __device__ constexpr float w9(int i) { return i == 0 ? 4.f / 9.f : i <= 4 ? 1.f / 9.f : 1.f / 36.f; }
__host__ __device__ constexpr double w9d(int i) { return i == 0 ? 4.0 / 9.0 : i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0; }
// D2Q5 weights for an energy-moment equilibrium a T with a = -2:
// w0 = (1 - a)/5 = 3/5, w1..4 = (4 + a)/20 = 1/10; c_sT^2 = (4 + a)/10 = 1/5.
__host__ __device__ constexpr float w5(int i) { return i == 0 ? 0.6f : 0.1f; }
// Population index p in [0, 14) -> lattice direction.
__host__ __device__ constexpr int pdir(int p) { return p < kQ9 ? p : p - kQ9; }

// ---------------------------------------------------------------------------
// Storage of the 14 planes (lbm_params.storage).  Every kernel computes in
// FP32: a load widens, a store rounds to nearest even.  FP16 holds the values
// scaled by 2^12, so that deviations down to 1.5e-8 stay in its normal range
// (stored magnitudes up to 16; larger ones overflow to infinity and raise
// LBM_ENUMERIC); the power-of-two scale is exact both ways.  BF16 has FP32's
// exponent range and needs no scale.
// ---------------------------------------------------------------------------
template <typename T>
struct Elem;
template <>
struct Elem<float> {
    __host__ __device__ static float ld(float v) { return v; }
    __host__ __device__ static float st(float v) { return v; }
};
template <>
struct Elem<__nv_bfloat16> {
    __host__ __device__ static float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    __host__ __device__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};
constexpr float kHalfScale = 4096.f;
template <>
struct Elem<__half> {
    __host__ __device__ static float ld(__half v) { return __half2float(v) * (1.f / kHalfScale); }
    __host__ __device__ static __half st(float v) { return __float2half_rn(v * kHalfScale); }
};
// Indices of Dev::ksc.
enum { kScC1 = 0, kScC2, kScB4, kScB7, kScC7, kScC8, kScG2, kScThree, kScBfx, kNumSc };
// Bytes per stored population.
__host__ __device__ constexpr int storage_bytes(int storage) { return storage == LBM_STORE_FP32 ? 4 : 2; }

// Per-node state bytes of the flag map.
constexpr uint8_t kFluid = 0;   // fluid at the previous and the current time
constexpr uint8_t kSolid = 1;   // inside a particle at the current time
constexpr uint8_t kNewborn = 2; // uncovered by a particle during the last step

// Device error bits (sticky, mapped to LBM_E* on the host).
constexpr unsigned kErrNumeric = 1u;
constexpr unsigned kErrDomain = 2u;
constexpr unsigned kErrOverflow = 4u;
constexpr unsigned kErrTimeout = 8u;
constexpr unsigned kErrBounds = 16u; // builds with -DLBM_CHECK only

// Counter slots (see lbm_get_counters).
enum { kCntBzLinear = 0, kCntBzSimple, kCntThermHalf, kCntRfLinear, kCntRfCopy, kCntRfEq,
       kCntNewborn, kCntLinks, kNumCounters };

struct Status {
    unsigned int err;
    unsigned int pad;
    unsigned long long cnt[2][kNumCounters]; // double-buffered by step parity
    unsigned int nb;     // newborn nodes listed this step (reset by the particle update)
    unsigned int nb_pad;
    // the staged stream-collide's work counter (next row tile to claim) and
    // the count of its blocks done; the last block done resets both to 0
    unsigned int sc_next;
    unsigned int sc_done;
};

// Structure-of-arrays particle state on the device (FP64).
struct PartSoA {
    double *x, *y, *ux, *uy, *th, *om, *r, *rho, *T, *b;
};
constexpr int kPartFields = 10; // doubles per particle in a PartSoA

// Everything a kernel needs, passed by value.
struct Dev {
    int nx, ny, pitch, np;
    long long ps; // plane stride in elements
    int storage;  // LBM_STORE_*: element type of the planes
    int per_x, per_y;
    // physics (FP32 for the lattice, FP64 for particles)
    float s_e, s_eps, s_q, s_nu, q_k, q_e, q_nu;
    // the relaxation rates folded with the moment norms (see collide())
    float kA1, kB1, kC1, kA2, kB2, kC2, kA4, kB4, kC4, kA7, kB7, kC7, kC8, kG1, kG2, kG3, kG4, kG5;
    float gbeta, T0, bfx, bfy;
    // FP16 storage: constants of the collision times the storage scale 2^12,
    // for the fused stream-collide kernels, which collide the scaled values
    // (kScC1 ... below; the last three words pad the record)
    float ksc[12];
    float Twall[4];
    double g, rho_f, eps_w, s_rep;
    int fixed;
    int zone_max;      // largest zone side N over the particles (sizes the link kernel's tile)
    int link_ahead;    // link-kernel CTAs resident on the GPU (distance of its L2 prefetch)
    int flag_team;     // warps per particle in the flags kernel (1, 2 or 4)
    // device buffers
    uint8_t *flags;    // [ny][pitch]
    int *newborn;      // [newborn_cap]: this step's newborn nodes, j * nx + i off the cavity frame, ~(j * nx + i) on it
    int newborn_cap;
    int2 *runs[2];     // [np][zone_max] by step parity: each zone row's run (lo, hi) of nodes inside the particle
    unsigned *near;    // bit per warp tile (row, 32 V nodes) within reach of a particle this step
    int near_tpr;      // warp tiles per row of that bitmap
    long long nslots;  // slots of the fixed index array
    long long a_elems; // elements of each distribution buffer, its tail pad included
    int *slot_node;    // [nslots]
    float *slot_q;     // [nslots]
    int *slot_base;    // [np + 1]
    PartSoA cur, nxt;  // state at n (and n+1 after the raster rotation) / new state
    double *px, *py;   // positions one step back (boxes to clear)
    double *force;     // [3 np]: hydrodynamic Fx, Fy, Tz of the last step
    float4 *pos4;      // [np]: centre as double-float (xh, yh, xl, yl) at the start of the step
    float2 *prc;       // [np]: (GeomRec r, C) in FP32 for the pair screening (r < 0: an ellipse)
    struct LinkSums *lsum; // [np]: link-kernel sums, assembled into force by the particle update
    struct DirectSums *dsum; // [np]: the same sums accumulated by atomics (direct addressing)
    int direct;            // links found by the node-parallel scan instead of the index array
    int sc_staged;         // whole-lattice stream-collide through the staged kernel (else one block per tile)
    int sc_extra_tx;       // bytes the staged kernel announces beyond its copies (tests of its bounded waits)
    struct GeomRec *geo_prev, *geo_cur, *geo_nxt; // [np] each: FP32/int geometry of the three positions
    double4 *pconst;   // [np]: constants of the update (1/M, 1/I, weight W, repulsion scale C)
    int *lorder;       // [np]: the link kernel's CTA order (particles by descending y)
    // pair screening: a grid of square cells of side 1 / cell_inv >= 2 r_max
    // + s + 2, so that every pair in reach sits in the same or neighbouring
    // cells; per parity [cell_gx * cell_gy + 1] counts (the last one flags an
    // overflowing cell), then kCellCap particle ids per cell
    int cell_gx, cell_gy;
    float cell_inv;
    int *cells[2];
    int all_pairs; // screen all pairs instead (LBM_FLAG_ALL_PAIRS)
    Status *status;
};
constexpr int kCellCap = 16;

// Bounds-checked builds (-DLBM_CHECK): in_bounds(D, i, n) is false for an
// index i outside [0, n) and records kErrBounds (LBM_EBOUNDS at the next
// synchronising call); the caller then skips the access.  The checks stand
// in for a memory checker: they cover the scattered writes of the particle
// kernels and every read of the stream-collide fast path.  Without
// LBM_CHECK the function is constant true and compiles away.
__device__ __forceinline__ bool in_bounds(const Dev &D, long long i, long long n)
{
#ifdef LBM_CHECK
    if (i < 0 || i >= n) {
        atomicOr(&D.status->err, kErrBounds);
        return false;
    }
#else
    (void)D; (void)i; (void)n;
#endif
    return true;
}
__device__ __forceinline__ int cell_of(const Dev &D, float xh, float yh)
{
    const int cx = min(max((int)(xh * D.cell_inv), 0), D.cell_gx - 1);
    const int cy = min(max((int)(yh * D.cell_inv), 0), D.cell_gy - 1);
    return cy * D.cell_gx + cx;
}
// Pair forces are summed in 64-bit fixed point (units of 2^-40): integer
// addition is exact and associative, so the sum does not depend on the order
// in which a particle's neighbours are found.
__device__ __forceinline__ long long fix_of(float v) { return __float2ll_rn(v * 0x1p40f); }
__device__ __forceinline__ long long fix_of(double v) { return __double2ll_rn(v * 0x1p40); }
__device__ __forceinline__ double fix_value(long long v) { return (double)v * 0x1p-40; }

// ---------------------------------------------------------------------------
// Exact FP64 geometry shared by raster, gather and refill.  Every operation is
// a correctly rounded IEEE operation with no FMA contraction, so the results
// agree bit for bit with any other implementation of the same expressions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_disk(int i, int j, double xc, double yc, double r)
{
    double dx = __dsub_rn((double)i, xc);
    double dy = __dsub_rn((double)j, yc);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= __dmul_rn(r, r);
}

// Wall fraction q (Sec. 2.3) of the link (i,j) -> (i,j) + e_k on the circle
// (xc, yc, r): t = (|d|^2 - r^2) / (-(d.e) + sqrt((d.e)^2 - |e|^2 (|d|^2 - r^2))).
__device__ __forceinline__ double link_q(int i, int j, int k, double xc, double yc, double r)
{
    double dx = __dsub_rn((double)i, xc);
    double dy = __dsub_rn((double)j, yc);
    double de = __dadd_rn(__dmul_rn((double)ex(k), dx), __dmul_rn((double)ey(k), dy));
    double a = (double)(ex(k) * ex(k) + ey(k) * ey(k));
    double c = __dsub_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(r, r));
    double disc = __dsub_rn(__dmul_rn(de, de), __dmul_rn(a, c));
    if (disc < 0.0) disc = 0.0;
    double t = __ddiv_rn(c, __dadd_rn(-de, __dsqrt_rn(disc)));
    return t > 1.0 ? 1.0 : t;
}

// ---------------------------------------------------------------------------
// Elliptical particles (Sec. 2.6, Appendix A): semi-axes a = r along the body
// axis at angle theta and b; 0 < b != r.  Every operation below is a
// correctly rounded FP64 operation with no FMA contraction, so the owner map
// and the wall fractions are reproducible bit for bit by any implementation
// of the same expressions.  The ellipse lies inside the circle of radius r,
// so the zone of a disk of radius r holds it and its links.
// ---------------------------------------------------------------------------
__host__ __device__ inline bool is_ellipse(double r, double b) { return b > 0.0 && b != r; }

// cos and sin of theta: Cody-Waite reduction by pi/2 (pi/2 split into a
// 33-bit head, so k times the head is exact for |k| < 2^20, and a tail), then
// the Taylor series of sin (to t^17) and cos (to t^16) on [-pi/4, pi/4] in
// Horner form, truncation below 1e-17; the quadrant k mod 4 picks the signs.
__device__ __forceinline__ void cos_sin_rn(double theta, double &c, double &s)
{
    const double two_over_pi = 0.63661977236758134308;
    const double pio2_hi = 1.5707963267341256e+00;
    const double pio2_lo = 6.0771005065061922e-11;
    const double k = floor(__dadd_rn(__dmul_rn(theta, two_over_pi), 0.5));
    const double t = __dsub_rn(__dsub_rn(theta, __dmul_rn(k, pio2_hi)), __dmul_rn(k, pio2_lo));
    const double t2 = __dmul_rn(t, t);
    // odd series: 1/17!, -1/15!, ..., -1/3!; even series: 1/16!, ..., -1/2!
    // (each 1/n! correctly rounded to FP64, written out)
    const double sc[8] = {2.8114572543455206e-15, -7.647163731819816e-13, 1.6059043836821613e-10,
                          -2.505210838544172e-08, 2.7557319223985893e-06, -0.0001984126984126984,
                          0.008333333333333333,   -0.16666666666666666};
    const double cc[8] = {4.779477332387385e-14,  -1.1470745597729725e-11, 2.08767569878681e-09,
                          -2.755731922398589e-07, 2.48015873015873e-05,    -0.001388888888888889,
                          0.041666666666666664,   -0.5};
    double ps = sc[0], pc = cc[0];
#pragma unroll
    for (int n = 1; n < 8; ++n) {
        ps = __dadd_rn(__dmul_rn(ps, t2), sc[n]);
        pc = __dadd_rn(__dmul_rn(pc, t2), cc[n]);
    }
    const double sn = __dadd_rn(t, __dmul_rn(t, __dmul_rn(t2, ps)));
    const double cn = __dadd_rn(1.0, __dmul_rn(t2, pc));
    const long long q = (long long)k & 3;
    c = q == 0 ? cn : q == 1 ? -sn : q == 2 ? -cn : sn;
    s = q == 0 ? sn : q == 1 ? cn : q == 2 ? -sn : -cn;
}

// An ellipse in the form its predicates use: centre, cos/sin of theta, a^2, b^2.
struct EllFrame {
    double x, y, c, s, a2, b2;
};
__device__ __forceinline__ EllFrame ell_frame(double x, double y, double th, double r, double b)
{
    EllFrame E;
    E.x = x;
    E.y = y;
    cos_sin_rn(th, E.c, E.s);
    E.a2 = __dmul_rn(r, r);
    E.b2 = __dmul_rn(b, b);
    return E;
}
// (dx, dy) in the body frame: u along the major axis, v along the minor one.
__device__ __forceinline__ void ell_uv(const EllFrame &E, double dx, double dy, double &u, double &v)
{
    u = __dadd_rn(__dmul_rn(dx, E.c), __dmul_rn(dy, E.s));
    v = __dsub_rn(__dmul_rn(dy, E.c), __dmul_rn(dx, E.s));
}
// u^2 b^2 + v^2 a^2 (the ellipse is where it is <= a^2 b^2)
__device__ __forceinline__ double ell_form(const EllFrame &E, double u, double v)
{
    return __dadd_rn(__dmul_rn(__dmul_rn(u, u), E.b2), __dmul_rn(__dmul_rn(v, v), E.a2));
}
__device__ __forceinline__ bool in_ellipse(int i, int j, const EllFrame &E)
{
    double u, v;
    ell_uv(E, __dsub_rn((double)i, E.x), __dsub_rn((double)j, E.y), u, v);
    return ell_form(E, u, v) <= __dmul_rn(E.a2, E.b2);
}
// Wall fraction q of the link (i, j) -> (i, j) + e_k on the ellipse: the
// smaller root t of F(d + t e) = 0, F(w) = u(w)^2 b^2 + v(w)^2 a^2 - a^2 b^2,
// i.e. P2 t^2 + 2 P1 t + P0 = 0, as t = P0 / (-P1 + sqrt(P1^2 - P2 P0))
// (P0 > 0 outside, P1 < 0 towards the ellipse: no cancellation).  Also
// returns d = (i, j) - centre rounded to FP32.
__device__ __forceinline__ float link_q_ellipse(int i, int j, int k, const EllFrame &E, float &dxf, float &dyf)
{
    const double dx = __dsub_rn((double)i, E.x), dy = __dsub_rn((double)j, E.y);
    double du, dv, eu, ev;
    ell_uv(E, dx, dy, du, dv);
    ell_uv(E, (double)ex(k), (double)ey(k), eu, ev);
    const double P2 = ell_form(E, eu, ev);
    const double P1 = __dadd_rn(__dmul_rn(__dmul_rn(du, eu), E.b2), __dmul_rn(__dmul_rn(dv, ev), E.a2));
    const double P0 = __dsub_rn(ell_form(E, du, dv), __dmul_rn(E.a2, E.b2));
    double disc = __dsub_rn(__dmul_rn(P1, P1), __dmul_rn(P2, P0));
    if (disc < 0.0) disc = 0.0;
    double t = __ddiv_rn(P0, __dadd_rn(-P1, __dsqrt_rn(disc)));
    dxf = (float)dx;
    dyf = (float)dy;
    return (float)(t > 1.0 ? 1.0 : t);
}
// Outward normal at an offset (dx, dy) from the centre, unnormalised: the
// gradient of u^2 / a^2 + v^2 / b^2 (up to a factor 2) in lattice axes.
__device__ __forceinline__ void ell_normal(const EllFrame &E, double dx, double dy, double &nx, double &ny)
{
    double u, v;
    ell_uv(E, dx, dy, u, v);
    const double gu = __ddiv_rn(u, E.a2), gv = __ddiv_rn(v, E.b2);
    nx = __dsub_rn(__dmul_rn(gu, E.c), __dmul_rn(gv, E.s));
    ny = __dadd_rn(__dmul_rn(gu, E.s), __dmul_rn(gv, E.c));
}
// Support distance along the unit vector n: sqrt(a^2 (n.u)^2 + b^2 (n.v)^2).
__device__ __forceinline__ double ell_support(const EllFrame &E, double nx, double ny)
{
    double u, v;
    ell_uv(E, nx, ny, u, v);
    return __dsqrt_rn(__dadd_rn(__dmul_rn(__dmul_rn(E.a2, u), u), __dmul_rn(__dmul_rn(E.b2, v), v)));
}

// Effective zone of Sec. 3: N = ceil(2r) + 3 nodes per side starting at
// floor(c - r) - 1 (equal to the paper's INT(c + r) - INT(c - r) + 3 for
// integer radii); 12N - 12 fixed slots.
__host__ __device__ inline int zone_size(double r) { return (int)ceil(2.0 * r) + 3; }
__host__ __device__ inline int slot_capacity(double r) { return 12 * zone_size(r) - 12; }

// ---------------------------------------------------------------------------
// Double-float arithmetic in FP32 (an unevaluated sum hi + lo).  GB300 runs
// FP64 at 2 lanes per SM per cycle, so every warp-wide FP64 instruction holds
// the SM's FP64 pipe for ~16 cycles; geometry and reductions therefore use
// error-free transformations in FP32: Knuth's TwoSum and the FMA-based
// TwoProduct (Dekker / Ogita-Rump-Oishi).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = a * b;
    e = fmaf(a, b, -p);
}
// (h, l) += (h2, l2)
__device__ __forceinline__ void df_add(float &h, float &l, float h2, float l2)
{
    float s, e;
    two_sum(h, h2, s, e);
    h = s;
    l = l + l2 + e;
}

// A disk with its centre split as x = xh + xl, y = yh + yl and r^2 = r2h + r2l
// (built once per disk in FP64).
struct DiskDF {
    float xh, xl, yh, yl, r2h, r2l;
};
__device__ __forceinline__ DiskDF disk_df(double x, double y, double r)
{
    DiskDF d;
    d.xh = (float)x;
    d.xl = (float)(x - (double)d.xh);
    d.yh = (float)y;
    d.yl = (float)(y - (double)d.yh);
    const double r2 = r * r;
    d.r2h = (float)r2;
    d.r2l = (float)(r2 - (double)d.r2h);
    return d;
}
// i - xc as (h, l), accurate to ~1e-12 absolute.
__device__ __forceinline__ void df_offset(int i, float xh, float xl, float &h, float &l)
{
    float e;
    two_sum((float)i, -xh, h, e);
    l = e - xl;
}
// |d|^2 - r^2 for d = (i, j) - centre as an unevaluated sum t + low, with
// |error| < 1e-9 for |d| < 64 and centre coordinates below 4096 (the error
// grows with the coordinates' FP32 spacing).  Also returns d as double-float
// components.
__device__ __forceinline__ void disk_gap2_df(int i, int j, const DiskDF &D, float &t, float &low, float &dxh,
                                             float &dxl, float &dyh, float &dyl)
{
    df_offset(i, D.xh, D.xl, dxh, dxl);
    df_offset(j, D.yh, D.yl, dyh, dyl);
    float p1, e1, p2, e2, s, es, et;
    two_prod(dxh, dxh, p1, e1);
    two_prod(dyh, dyh, p2, e2);
    two_sum(p1, p2, s, es);
    two_sum(s, -D.r2h, t, et);
    low = ((e1 + e2) + (es + et)) - D.r2l + 2.f * (dxh * dxl + dyh * dyl) + (dxl * dxl + dyl * dyl);
}
// The same, rounded to FP32.
__device__ __forceinline__ float disk_gap2(int i, int j, const DiskDF &D, float &dxh, float &dxl,
                                           float &dyh, float &dyl)
{
    float t, low;
    disk_gap2_df(i, j, D, t, low, dxh, dxl, dyh, dyl);
    return t + low;
}
// Exact disk predicate (the FP64 one above) decided in FP32 except inside a
// band of +-1e-6 around the circle, where FP64 rounding could matter.
__device__ __forceinline__ bool in_disk_df(int i, int j, const DiskDF &D, double xc, double yc,
                                           double r)
{
    float a, b, c, d;
    const float g = disk_gap2(i, j, D, a, b, c, d);
    if (g < -1e-6f) return true;
    if (g > 1e-6f) return false;
    return in_disk(i, j, xc, yc, r);
}

// Wall fraction q of the link from (i, j) along e_k to the circle: the
// cancellation-free closed form q = c / (-de + sqrt(de^2 - |e|^2 c)) with
// c = |d|^2 - r^2 and de = d.e (de < 0 on a link).  c, de and the
// discriminant are carried in double-float, so that near-tangent links,
// whose small discriminant magnifies its absolute error by 1 / (2 sqrt(disc)),
// see errors of about 1e-9 there instead of FP32 roundings of de^2 and c;
// the square root, the sum and the division are FP32.  With u = 2^-24 (the
// largest relative error of one FP32 rounding) and den = -de + sqrt(disc):
//   |q - q_exact| <= 4.5 u q + (e_c + q e_de + q e_disc / (2 sqrt(disc))) / den,
// e_c <= 2e-9, e_de <= 5e-11, e_disc <= 1e-8 for |d| < 32 and centre
// coordinates below 4096 (the three scale with the coordinates' FP32 spacing
// beyond).  Also returns d (FP32) for the wall velocity and torque.
__device__ __forceinline__ float link_q_df(int i, int j, int k, const DiskDF &D, float &dxf,
                                           float &dyf)
{
    float dxh, dxl, dyh, dyl, ch, cl;
    disk_gap2_df(i, j, D, ch, cl, dxh, dxl, dyh, dyl);
    float sh, se, deh, del;
    two_sum((float)ex(k) * dxh, (float)ey(k) * dyh, sh, se);
    two_sum(sh, se + ((float)ex(k) * dxl + (float)ey(k) * dyl), deh, del);
    // disc = de^2 - a c in double-float (a = |e_k|^2 is 1 or 2: a ch is exact)
    const float a = (float)(ex(k) * ex(k) + ey(k) * ey(k));
    float p, pe, s2, e2;
    two_prod(deh, deh, p, pe);
    two_sum(p, -a * ch, s2, e2);
    const float disc = fmaxf(s2 + (e2 + ((pe + 2.f * deh * del) - a * cl)), 0.f);
    dxf = dxh + dxl;
    dyf = dyh + dyl;
    return fminf((ch + cl) / (sqrtf(disc) - (deh + del)), 1.f);
}

// The ellipse predicate decided in FP32 (offsets from the double-float
// centre, FP32 cos/sin, a^2, b^2), except inside a band around the boundary
// wide enough to hold every FP32 rounding: with R = r + 3 bounding |d| on the
// zone, the FP32 value of F = u^2 b^2 + v^2 a^2 - a^2 b^2 is within
// 3.3e-6 R^2 a^2 of the exact one, and the band is 1e-5 R^2 a^2.  Outside the
// band the FP32 sign is the exact sign.
struct EllDF {
    float xh, xl, yh, yl, c, s, a2, b2, ab, band;
};
__device__ __forceinline__ EllDF ell_df(float xh, float xl, float yh, float yl, float c, float s, double r,
                                        double b)
{
    EllDF E;
    E.xh = xh; E.xl = xl; E.yh = yh; E.yl = yl; E.c = c; E.s = s;
    E.a2 = (float)(r * r);
    E.b2 = (float)(b * b);
    E.ab = (float)(r * r * b * b);
    const float R = (float)r + 3.f;
    E.band = 1e-5f * R * R * E.a2;
    return E;
}
// -1: inside, +1: outside, 0: inside the band (decide in FP64).
__device__ __forceinline__ int ell_side_df(int i, int j, const EllDF &E)
{
    float dxh, dxl, dyh, dyl;
    df_offset(i, E.xh, E.xl, dxh, dxl);
    df_offset(j, E.yh, E.yl, dyh, dyl);
    const float dx = dxh + dxl, dy = dyh + dyl;
    const float u = dx * E.c + dy * E.s, v = dy * E.c - dx * E.s;
    const float F = (u * u) * E.b2 + (v * v) * E.a2 - E.ab;
    return F < -E.band ? -1 : F > E.band ? 1 : 0;
}

// Geometry of one disk position in the forms the per-warp kernels use, built
// once per particle and step in FP64 (one lane per particle) so that no warp
// repeats FP64 work: the double-float centre and r^2, the zone (origin, side),
// the row centre index floor(x + 1/2), FP32 velocities and 2 w_k T_w, and the
// radius (negated for an ellipse, whose semi-major axis it is) and repulsion
// force scale C = A (rho_p - rho_f) g with the area A = pi r^2 (pi r b for an
// ellipse).  w0, w1: r^2 as double-float for a disk; cos theta and sin theta
// in FP32 for an ellipse.
struct GeomRec {
    float xh, xl, yh, yl, w0, w1, r, C;
    int X0, Y0, N, ic;
    float ux, uy, om, wT;
};
__device__ __forceinline__ GeomRec make_geom(double x, double y, double r, double b, double th, double ux,
                                             double uy, double om, double T, double rho, double rho_f, double g)
{
    GeomRec G;
    const DiskDF d = disk_df(x, y, r);
    G.xh = d.xh; G.xl = d.xl; G.yh = d.yh; G.yl = d.yl; G.w0 = d.r2h; G.w1 = d.r2l;
    const bool ell = is_ellipse(r, b);
    if (ell) {
        double c, s;
        cos_sin_rn(th, c, s);
        G.w0 = (float)c;
        G.w1 = (float)s;
    }
    G.r = ell ? -(float)r : (float)r;
    G.C = (float)(3.14159265358979323846 * r * (ell ? b : r) * (rho - rho_f) * g);
    G.N = zone_size(r);
    G.X0 = (int)floor(x - r) - 1;
    G.Y0 = (int)floor(y - r) - 1;
    G.ic = (int)floor(x + 0.5);
    G.ux = (float)ux; G.uy = (float)uy; G.om = (float)om; G.wT = (float)(0.2 * T);
    return G;
}
// make_geom at another position and motion of the same particle: the fields
// that depend only on its shape, density and temperature (r, C, the zone
// side, r^2 of a disk, 2 w_k T_w) are those of its record G at any other
// position, so the result has the same bits as make_geom.
__device__ __forceinline__ GeomRec move_geom(GeomRec G, double x, double y, double r, double b, double th, double ux,
                                             double uy, double om)
{
    G.xh = (float)x;
    G.xl = (float)(x - (double)G.xh);
    G.yh = (float)y;
    G.yl = (float)(y - (double)G.yh);
    if (is_ellipse(r, b)) {
        double c, s;
        cos_sin_rn(th, c, s);
        G.w0 = (float)c;
        G.w1 = (float)s;
    }
    G.X0 = (int)floor(x - r) - 1;
    G.Y0 = (int)floor(y - r) - 1;
    G.ic = (int)floor(x + 0.5);
    G.ux = (float)ux; G.uy = (float)uy; G.om = (float)om;
    return G;
}
__device__ __forceinline__ DiskDF geom_df(const GeomRec &G)
{
    DiskDF d;
    d.xh = G.xh; d.xl = G.xl; d.yh = G.yh; d.yl = G.yl; d.r2h = G.w0; d.r2l = G.w1;
    return d;
}

// Per-particle sums of the link kernel: the variable part of Eq. force /
// Eq. torque in 64-bit fixed point (units of 2^-50 for the force, 2^-46 for
// the torque: integer addition is exact and associative, so the sums do not
// depend on how the links are grouped or ordered), and the exact integer
// sums of the constant part 2 w_k e_k (axis links: 2w = 2/9, diagonal: 1/18)
// and its torque moment 2 w_k (i e_k,y - j e_k,x).
struct LinkSums {
    long long fx, fy, tz;
    int ax_x, ax_y, ax_t, dg_x, dg_y, dg_t;
    int pad[4];
};
__device__ __forceinline__ long long fix_force(float v) { return __float2ll_rn(v * 0x1p50f); }
__device__ __forceinline__ long long fix_torque(float v) { return __float2ll_rn(v * 0x1p46f); }
__device__ __forceinline__ long long fix_force(double v) { return __double2ll_rn(v * 0x1p50); }
__device__ __forceinline__ long long fix_torque(double v) { return __double2ll_rn(v * 0x1p46); }
// Direct addressing: the variable parts in FP64 and the constant parts as
// integers, accumulated link by link with atomics (order not fixed).
struct DirectSums {
    double f[3];  // Fx, Fy, Tz brackets
    int c[6];     // ax_x, ax_y, ax_t, dg_x, dg_y, dg_t
};
// Per-link momentum-exchange sums.  Each thread adds its links (add), then
// finish() sums a warp's threads; the sums are exact, so every kernel that
// sums links gets the same bits however it distributes them.  bx, by, tq:
// the variable part of Eq. force / Eq. torque of a link; k its direction;
// lvl its Bouzidi fallback level; half whether its thermal rule fell back to
// half-way; tz the torque moment i e_k,y - j e_k,x of its constant part.
struct LinkAcc {
    long long fx = 0, fy = 0, tq = 0;
    int axx = 0, axy = 0, axt = 0, dgx = 0, dgy = 0, dgt = 0, cl = 0, cs = 0, ct = 0;

    __device__ __forceinline__ void add(float bx, float by, float t, int k, int lvl, bool half, int tz)
    {
        fx += fix_force(bx);
        fy += fix_force(by);
        tq += fix_torque(t);
        cl += lvl == 1;
        cs += lvl == 2;
        ct += half;
        if (k <= 4) { axx += ex(k); axy += ey(k); axt += tz; }
        else { dgx += ex(k); dgy += ey(k); dgt += tz; }
    }
    // Whole warp; the sums land in S and cnt3 (fallback counts: linear,
    // simple, thermal half-way) on every lane.
    __device__ __forceinline__ void finish(LinkSums &S, int *cnt3)
    {
        const unsigned F = 0xffffffffu;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(F, fx, o);
            fy += __shfl_xor_sync(F, fy, o);
            tq += __shfl_xor_sync(F, tq, o);
        }
        S.fx = fx; S.fy = fy; S.tz = tq;
        S.ax_x = (int)__reduce_add_sync(F, (unsigned)axx);
        S.ax_y = (int)__reduce_add_sync(F, (unsigned)axy);
        S.ax_t = (int)__reduce_add_sync(F, (unsigned)axt);
        S.dg_x = (int)__reduce_add_sync(F, (unsigned)dgx);
        S.dg_y = (int)__reduce_add_sync(F, (unsigned)dgy);
        S.dg_t = (int)__reduce_add_sync(F, (unsigned)dgt);
        S.pad[0] = S.pad[1] = S.pad[2] = S.pad[3] = 0;
        cnt3[0] = (int)__reduce_add_sync(F, (unsigned)cl);
        cnt3[1] = (int)__reduce_add_sync(F, (unsigned)cs);
        cnt3[2] = (int)__reduce_add_sync(F, (unsigned)ct);
    }
};
// S += T (the sums of another group of links).
__device__ __forceinline__ void add_sums(LinkSums &S, const LinkSums &T)
{
    S.fx += T.fx; S.fy += T.fy; S.tz += T.tz;
    S.ax_x += T.ax_x; S.ax_y += T.ax_y; S.ax_t += T.ax_t;
    S.dg_x += T.dg_x; S.dg_y += T.dg_y; S.dg_t += T.dg_t;
}

// Reduction of per-link results stored in shared memory, by one warp, in
// link order.  code: k | fallback level << 4 | thermal half-way << 6.
__device__ __forceinline__ void reduce_links(const float *bx, const float *by, const float *tq,
                                             const int *code, const int *tz, int n, LinkSums &S,
                                             int *cnt3)
{
    LinkAcc acc;
    for (int i = (int)(threadIdx.x & 31); i < n; i += 32) {
        const int c = code[i];
        acc.add(bx[i], by[i], tq[i], c & 15, (c >> 4) & 3, (c >> 6) & 1, tz[i]);
    }
    acc.finish(S, cnt3);
}

// Hydrodynamic force (Fx, Fy) and torque of a particle centred at (xc, yc).
__device__ __forceinline__ void assemble_force(const LinkSums &S, double xc, double yc, double &Fx,
                                               double &Fy, double &Tz)
{
    const double cax = 2.0 / 9.0, cdg = 1.0 / 18.0;
    const double Fcx = cax * (double)S.ax_x + cdg * (double)S.dg_x;
    const double Fcy = cax * (double)S.ax_y + cdg * (double)S.dg_y;
    const double Tc = cax * (double)S.ax_t + cdg * (double)S.dg_t - xc * Fcy + yc * Fcx;
    Fx = Fcx + (double)S.fx * 0x1p-50;
    Fy = Fcy + (double)S.fy * 0x1p-50;
    Tz = Tc + (double)S.tz * 0x1p-46;
}

// Bouzidi quadratic bounce-back (Sec. 2.3) in deviation form, with the
// linear and simple fallbacks when a stencil node is not fluid.  fk0, fk1,
// fk2 = f~_k^+ at x_f, x_f - e_k, x_f - 2e_k; fb0, fb1 = f~_kbar^+ at x_f,
// x_f - e_k; wall = 2 w_k rho0 e_kbar.u_w / c_s^2.  *lvl: 0 quadratic,
// 1 linear, 2 simple.
__device__ __forceinline__ float bouzidi32(float q, float fk0, float fk1, float fk2, float fb0,
                                           float fb1, bool have1, bool have2, float wall, int &lvl)
{
    if (q <= 0.5f) {
        if (have1 && have2) {
            lvl = 0;
            return q * (2.f * q + 1.f) * fk0 + (1.f - 4.f * q * q) * fk1 - q * (1.f - 2.f * q) * fk2 +
                   wall;
        }
        if (have1) {
            lvl = 1;
            return 2.f * q * fk0 + (1.f - 2.f * q) * fk1 + wall;
        }
        lvl = 2;
        return fk0 + wall;
    }
    // q > 1/2: coefficients from the two reciprocals 1/q and 1/(2q + 1)
    const float rq = __frcp_rn(q);
    if (have1) {
        lvl = 0;
        const float r1 = __frcp_rn(2.f * q + 1.f);
        const float cc = rq * r1, t = 2.f * q - 1.f;
        return cc * fk0 + t * rq * fb0 - t * r1 * fb1 + cc * wall;
    }
    lvl = 1;
    const float h = 0.5f * rq;
    return h * fk0 + (2.f * q - 1.f) * h * fb0 + h * wall;
}

// Li et al. curved Dirichlet rule for g (Sec. 2.3), c_d1 = -1,
// c_d2 = c_d3 = (2q-1)/(2q+1), c_d4 = 2/(2q+1); half-way anti-bounce-back
// without x_f - e_k.  wT = 2 w_k T_w.
__device__ __forceinline__ float thermal32(float q, float gk0, float gk1, float gb0, bool have1,
                                           float wT)
{
    if (have1) {
        const float r1 = __frcp_rn(2.f * q + 1.f);
        return -gk0 + (2.f * q - 1.f) * r1 * (gk1 + gb0) + 2.f * r1 * wT;
    }
    return -gk0 + wT;
}

// Zone point (a, b) of the t-th node on line `line` of direction k; false
// when it falls outside the N x N zone.  e1/e3: rows (line = b); e2/e4:
// columns (line = a); e5/e7: constant a - b (line = a - b + N - 2); e6/e8:
// constant a + b (line = a + b - 1).
__host__ __device__ inline bool zone_point(int k, int N, int line, int t, int &a, int &b)
{
    if (k == 1 || k == 3) {
        a = t;
        b = line;
    } else if (k == 2 || k == 4) {
        a = line;
        b = t;
    } else if (k == 5 || k == 7) {
        a = t;
        b = t - (line - (N - 2));
    } else {
        a = t;
        b = (line + 1) - t;
    }
    return b >= 0 && b < N;
}

// Walk of line `line` of direction k in zone coordinates (a = column,
// b = row): the valid points are (a0 + t da, b0 + t db), t = 0 .. cnt - 1 (the
// same points as zone_point, in the same order, without per-point tests).
__host__ __device__ inline void line_walk(int k, int N, int line, int &a0, int &b0, int &da, int &db,
                                          int &cnt)
{
    if (k == 1 || k == 3) {
        a0 = 0; b0 = line; da = 1; db = 0; cnt = N;
    } else if (k == 2 || k == 4) {
        a0 = line; b0 = 0; da = 0; db = 1; cnt = N;
    } else if (k == 5 || k == 7) {
        const int m = line - (N - 2); // b = a - m
        const int t0 = m > 0 ? m : 0, t1 = (N - 1 + m) < (N - 1) ? (N - 1 + m) : (N - 1);
        a0 = t0; b0 = t0 - m; da = 1; db = 1; cnt = t1 - t0 + 1;
    } else {
        const int sm = line + 1; // b = sm - a
        const int t0 = (sm - N + 1) > 0 ? (sm - N + 1) : 0, t1 = sm < (N - 1) ? sm : (N - 1);
        a0 = t0; b0 = sm - t0; da = 1; db = -1; cnt = t1 - t0 + 1;
    }
}

// Slot s of a zone of size N -> direction k and line.
__host__ __device__ inline void slot_dir_line(int s, int N, int &k, int &line)
{
    if (s < 4 * N) {
        k = 1 + s / N;
        line = s % N;
    } else {
        int t = s - 4 * N, m = 2 * N - 3;
        k = 5 + t / m;
        line = t % m;
    }
}

// ---------------------------------------------------------------------------
// Batched instances.  Every step kernel is a device body that takes the
// position of its block within one instance's launch (Blk): the
// single-instance kernels fill it from the built-in indices, the batched
// kernels from the block's slice of one grid over all instances, whose
// per-instance block offsets are `start` (start[i] <= block < start[i + 1]).
// ---------------------------------------------------------------------------
struct Blk {
    int x, y, gx, gy;
};
__device__ __forceinline__ Blk this_blk()
{
    return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y};
}
// Instance whose slice holds batched block g (binary search over n + 1
// offsets; instances with no blocks in this launch are skipped).
__device__ __forceinline__ int batch_find(const int *__restrict__ start, int n, int g)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}
// Block-wide copy of an instance's Dev into shared memory (all threads of
// the block call it; it ends with a barrier).
__device__ __forceinline__ void copy_dev(Dev &dst, const Dev &src)
{
    static_assert(sizeof(Dev) % 4 == 0, "Dev is copied as 32-bit words");
    const int t = (int)(threadIdx.y * blockDim.x + threadIdx.x), nt = (int)(blockDim.x * blockDim.y);
    for (int w = t; w < (int)(sizeof(Dev) / 4); w += nt)
        reinterpret_cast<int *>(&dst)[w] = __ldg(reinterpret_cast<const int *>(&src) + w);
    __syncthreads();
}
// Per-instance arguments of the batched kernels (device table).
struct InstArgs {
    Dev D;
    void *A[2];   // distribution buffers by step parity
    int *own[2];  // owner maps by step parity
    int poff;     // the instance's step parity = the batch's parity ^ poff
    int pad;
};

// Stream-collide blocks of one instance in a batched launch: its first
// block, its tiles per row gx, and a multiplier m and shift s with
// local / gx = (local * m) >> s exactly for every 0 <= local < 2^31
// (division by an invariant integer, Granlund and Montgomery 1994:
// s = 31 + ceil(log2 gx), m = floor(2^s / gx) + 1).
struct ScInst {
    unsigned long long m;
    int start, gx, s, pad;
};
// Instance holding stream-collide block g: the instance the bucket of g
// starts in (buckets of 2^shift blocks), then forward over the instances
// that start inside the bucket.
__device__ __forceinline__ int sc_find(const ScInst *__restrict__ sc, const int *__restrict__ bucket, int shift,
                                       int n, int g)
{
    int i = __ldg(bucket + (g >> shift));
    while (i + 1 < n && __ldg(&sc[i + 1].start) <= g) ++i;
    return i;
}
// Tile (bx, by) of stream-collide block g within its instance's gx-wide
// grid of tiles.
__device__ __forceinline__ void sc_tile(const ScInst *__restrict__ e, int g, int &bx, int &by)
{
    const unsigned local = (unsigned)(g - __ldg(&e->start));
    by = (int)(((unsigned long long)local * __ldg(&e->m)) >> __ldg(&e->s));
    bx = (int)local - by * __ldg(&e->gx);
}

// ---------------------------------------------------------------------------
// Kernel launchers (defined in k_fluid.cu and k_particles.cu).
// ---------------------------------------------------------------------------
enum KernelKind { kKLinks = 0, kKParticles, kKRaster, kKFlags, kKStreamCollide,
                  kKBoundary, kKInit, kKFields, kKNearMask, kKStreamCollideNear, kNumKernelKinds };

// Stream-collide passes: every warp tile, or only the tiles away from (far)
// or within reach of (near) this step's particles.
enum SCMode { kSCAll = 0, kSCFar = 1, kSCNear = 2 };
// Nodes added around each particle's zone in the near-tile bitmap: covers the
// zones one step back and one step ahead of a disk that moves less than one
// node per step.
constexpr int kNearMargin = 2;

// Planes are passed untyped: their element type is D.storage.
cudaError_t launch_stream_collide(const Dev &D, const void *Ain, void *Aout, int mode, cudaStream_t s);
// Binary (SASS) architecture of the loaded stream-collide kernel, as
// cudaFuncGetAttributes reports it (major * 10 + minor).
cudaError_t stream_collide_binary_version(int *version);
// Near-tile bitmap of this step (clears it first).
cudaError_t launch_near_mask(const Dev &D, cudaStream_t s);
// Direct addressing (the paper's comparison for its index array): a per-
// particle preparation (owner-map clear, centres, zeroed sums) and one thread
// per lattice node testing its eight neighbours.
cudaError_t launch_links_direct(const Dev &D, void *A, const int *own_cur, int *own_nxt, int parity,
                                cudaStream_t s);
// Warp tiles per row of the near-tile bitmap for a storage and pitch.
int near_tiles_per_row(int storage, int pitch);
// Nodes the stream-collide kernel leaves to the general path: the first and
// last rows (y = 0, ny - 1) and the listed newborn nodes.
cudaError_t launch_boundary(const Dev &D, const void *Ain, void *Aout, const int *own_cur, int parity,
                            cudaStream_t s);
// mode 0: fluid at rest (unit density, T_init) then collide; mode 1: collide
// the pre-collision values read from Ain at each node.
cudaError_t launch_init_collide(const Dev &D, const void *Ain, void *Aout, float T_init, int mode,
                                cudaStream_t s);
cudaError_t launch_fields(const Dev &D, const void *A, int row0, int rows, float *rho, float *ux,
                          float *uy, float *T, cudaStream_t s);
cudaError_t launch_links(const Dev &D, void *A, const int *own_cur, int *own_nxt, int parity,
                         cudaStream_t s);
// Shared memory of the link kernel for zones of side N; prepare_links sets the
// kernel's shared-memory limit and D.link_ahead (call outside stream capture).
size_t link_smem_bytes(int N, int storage);
// Whether the link kernel holds a zone of side N (tile rows of at most 64
// columns, shared memory within 200 KB).
bool link_zone_supported(int N, int storage);
cudaError_t prepare_links(Dev &D);
// Particle update, then the raster of the new positions into own_nxt.
cudaError_t launch_particles(const Dev &D, int parity, int *own_nxt, cudaStream_t s);
// runs (may be null): where each particle's zone-row runs go, for the flags
// of the next step.
cudaError_t launch_raster(const Dev &D, int *own, const struct GeomRec *geo, const PartSoA &pos, int2 *runs,
                          cudaStream_t s);
// rotate == 0: the flags of one position from scratch; rotate == 1: a step's
// flags from the row runs of parity (current) and parity ^ 1 (new).
cudaError_t launch_flags(const Dev &D, const int *own_cur, const int *own_nxt, int rotate, int parity,
                         cudaStream_t s);
// The newborn list of a restored state, from its flags (the list is empty).
cudaError_t launch_collect_newborn(const Dev &D, cudaStream_t s);
cudaError_t launch_pack_particles(const Dev &D, lbm_particle *out, cudaStream_t s);
// Geometry records of the current state (into cur, nxt and prev) and of the
// previous positions (into prev), for init and restore.
cudaError_t launch_geom_init(const Dev &D, cudaStream_t s);
// Screening grids: both cleared (the first step's link kernel enters the
// current positions).
cudaError_t launch_cells_init(const Dev &D, cudaStream_t s);
// The link kernel's CTA order from the current positions (descending y).
cudaError_t launch_link_order(const Dev &D, cudaStream_t s);

// Batched step kernels over an InstArgs table (one grid over all instances;
// `start` holds the n + 1 block offsets of the launch, `total` its blocks).
enum BatchPhase { kBLinks = 0, kBParticles, kBRaster, kBFlags, kBStream, kBBoundary, kBatchPhases };
constexpr int kBoundaryBlocksPerInstance = 8;
void batch_blocks(const Dev &D, dim3 sc_block, int out[kBatchPhases]);
cudaError_t prepare_links_batch(int zone_max, int storage, size_t *smem, int *ahead);
cudaError_t launch_links_batch(const InstArgs *I, const int *start, int n, int total, int storage, int parity,
                               int ahead, size_t smem, cudaStream_t s);
cudaError_t launch_particles_batch(const InstArgs *I, const int *start, int n, int total, int parity,
                                   cudaStream_t s);
cudaError_t launch_raster_batch(const InstArgs *I, const int *start, int n, int total, int parity, cudaStream_t s);
cudaError_t launch_flags_batch(const InstArgs *I, const int *start, int n, int total, int parity, cudaStream_t s);
cudaError_t launch_stream_collide_batch(const InstArgs *I, const ScInst *sc, const int *bucket, int shift, int n,
                                        int total, int storage, int parity, dim3 block, int resident,
                                        cudaStream_t s);
cudaError_t launch_boundary_batch(const InstArgs *I, const int *start, int n, int total, int storage, int parity,
                                  cudaStream_t s);
int stream_collide_batch_resident(int storage, dim3 block);
// The staged stream-collide over a batch (BF16 / FP16 storage): sc and
// bucket built for the 128 x 1 tile shape; counter: two zeroed words of
// device memory the launch leaves zeroed.
cudaError_t launch_stream_collide_staged_batch(const InstArgs *I, const ScInst *sc, const int *bucket, int shift,
                                               int n, int total, int storage, int parity, unsigned *counter,
                                               cudaStream_t s);

} // namespace lbm
