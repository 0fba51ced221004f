// Allocation-free variant of the link kernel: gather the fixed index array
// of fluid-particle links, apply the curved bounce-back on every link and
// reduce the momentum-exchange force and torque per particle, with the index
// array held in a file-scope device array instead of a caller workspace.
//
// Who needs it: code that may not allocate device memory at the point where
// it computes particle forces, e.g. a host application whose device memory
// is owned by another allocator or pool it cannot extend, or a caller inside
// a section where cudaMalloc is not allowed.  Such a caller still owns and
// passes the distributions, the owner map, the particles and the force
// output; the only scratch (the index array) lives here.
//
// The array holds 2,097,152 slots (node + wall fraction, 8 bytes each) and
// the slot offsets of up to 32,768 particles: 16 MiB + 128 KiB held on every
// GPU that loads the library, for the life of the process.  All calls share
// it and it keeps the contents of the last call, so calls whose GPU work
// overlaps (on two streams, or from two threads) race on it.  Every call
// looks up the array's device address on the current device
// (cudaGetSymbolAddress); the first call on a device also loads the
// library's device code there, so make that first call before any stream
// capture.
#include <climits>
#include <cmath>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr long long kStaticSlots = 1ll << 21;   // 2,097,152 slots
constexpr int kStaticParticles = 1 << 15;       // 32,768 particles
constexpr int kThreads = 256;

// [slot nodes: int32 x kStaticSlots][wall fractions: float x kStaticSlots]
// [slot offsets: int32 x (kStaticParticles + 1)][reject flag: uint32]
constexpr size_t kScratchBytes =
    (size_t)kStaticSlots * 8 + ((size_t)kStaticParticles + 1) * 4 + 256;

static __device__ __align__(256) unsigned char g_link_scratch[kScratchBytes];

struct Scratch {
    int *node;
    float *q;
    int *base;
    unsigned *reject; // set when a radius exceeds r_max for this call
};

__host__ __device__ inline Scratch carve(unsigned char *p)
{
    Scratch s;
    s.node = reinterpret_cast<int *>(p);
    s.q = reinterpret_cast<float *>(p + (size_t)kStaticSlots * 4);
    s.base = reinterpret_cast<int *>(p + (size_t)kStaticSlots * 8);
    s.reject = reinterpret_cast<unsigned *>(p + (size_t)kStaticSlots * 8 +
                                            ((size_t)kStaticParticles + 1) * 4);
    return s;
}

struct View {
    float *A;
    long long ps;
    int pitch, nx, ny, n;
    double r_max;
    const int *own;
    const lbm_particle *P;
    double *F;
};

// Slot offsets: running sum of 12N - 12 over the particles (one thread).
// The reject flag is rewritten on every call: set when some radius exceeds
// the r_max the host checked the capacity against, or when a particle breaks
// the shape rule of lbm_init (semi-minor axis b negative, or, for an
// ellipse, b below 1 or above the semi-major axis r, or |theta| above 1.6e6),
// since the zone and the slot capacity are sized from r.
__global__ void k_static_bases(View v, unsigned char *scratch)
{
    Scratch s = carve(scratch);
    if (threadIdx.x == 0) {
        int acc = 0;
        unsigned bad = 0u;
        for (int a = 0; a < v.n; ++a) {
            s.base[a] = acc;
            const double r = v.P[a].r, b = v.P[a].b;
            const bool shape_ok = b >= 0.0 && (!is_ellipse(r, b) || (b >= 1.0 && b <= r &&
                                                                     fabs(v.P[a].theta) <= 1.6e6));
            if (!(r >= 1.0 && r <= v.r_max) || !shape_ok) bad = 1u;
            else acc += slot_capacity(r);
        }
        s.base[v.n] = acc;
        *s.reject = bad;
    }
}

__device__ __forceinline__ bool in_box(const View &v, int i, int j)
{
    return i >= 0 && i < v.nx && j >= 0 && j < v.ny;
}

// Phase 1: one CTA per particle fills its 12N - 12 slots (Sec. 3 mapping).
// A line holding two links is marked -2 (the particle's force becomes NaN).
__global__ void __launch_bounds__(kThreads) k_static_gather(View v, unsigned char *scratch)
{
    Scratch s = carve(scratch);
    if (*s.reject) return;
    const int p = blockIdx.x;
    const double xc = v.P[p].x, yc = v.P[p].y, r = v.P[p].r;
    const DiskDF dk = disk_df(xc, yc, r);
    const bool ell = is_ellipse(r, v.P[p].b);
    EllFrame E{};
    if (ell) E = ell_frame(xc, yc, v.P[p].theta, r, v.P[p].b);
    const int N = zone_size(r), cap = 12 * N - 12;
    const int X0 = (int)floor(xc - r) - 1, Y0 = (int)floor(yc - r) - 1;
    const int base = s.base[p];
    for (int t0 = threadIdx.x; t0 < cap; t0 += kThreads) {
        int k, line;
        slot_dir_line(t0, N, k, line);
        int found = 0, fi = 0, fj = 0;
        for (int t = 0; t < N; ++t) {
            int a, b;
            if (!zone_point(k, N, line, t, a, b)) continue;
            const int i = X0 + a, j = Y0 + b;
            if (!in_box(v, i, j) || v.own[(long long)j * v.nx + i] != -1) continue;
            const int si = i + ex(k), sj = j + ey(k);
            if (!in_box(v, si, sj) || v.own[(long long)sj * v.nx + si] != p) continue;
            if (++found == 1) {
                fi = i;
                fj = j;
            }
        }
        float dxf, dyf;
        s.node[base + t0] = found > 1 ? -2 : found ? fj * v.nx + fi : -1;
        s.q[base + t0] = !found ? 0.f : ell ? link_q_ellipse(fi, fj, k, E, dxf, dyf) : link_q_df(fi, fj, k, dk, dxf, dyf);
    }
}

// Phase 2: bounce-back and momentum exchange on the gathered slots, with the
// same device helpers, per-link arithmetic, exact fixed-point sums (here by
// one warp over the valid slots in slot order) and FP64 assembly as the
// workspace kernels, so the forces agree bit for bit.
// Shared memory: the compacted slot list and the per-link results,
// 24 bytes per slot of the largest zone.
__global__ void __launch_bounds__(kThreads) k_static_bbforce(View v, unsigned char *scratch, int capm)
{
    Scratch s = carve(scratch);
    const int p = blockIdx.x;
    if (*s.reject) {
        if (threadIdx.x < 3) v.F[3 * p + threadIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    __shared__ int s_warp[kThreads / 32 + 1];
    extern __shared__ int list[]; // [capm] valid slots in slot order, then the per-link results
    float *lbx = reinterpret_cast<float *>(list + capm);
    float *lby = lbx + capm;
    float *ltq = lby + capm;
    int *lcode = reinterpret_cast<int *>(ltq + capm);
    int *ltz = lcode + capm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double xc = v.P[p].x, yc = v.P[p].y, r = v.P[p].r;
    const DiskDF dk = disk_df(xc, yc, r);
    const bool ell = is_ellipse(r, v.P[p].b);
    const float Ux = (float)v.P[p].ux, Uy = (float)v.P[p].uy, Om = (float)v.P[p].omega;
    const float wT = (float)(0.2 * v.P[p].T);
    const int N = zone_size(r), cap = 12 * N - 12;
    const int base = s.base[p];
    int broken = 0, nvalid = 0;
    float *A = v.A;
    const long long ps = v.ps;
    for (int s0 = 0; s0 < cap; s0 += kThreads) {
        const int sl = s0 + tid;
        const int node = sl < cap ? s.node[base + sl] : -1;
        broken |= node == -2;
        const bool valid = node >= 0;
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                const int c = s_warp[w];
                s_warp[w] = acc;
                acc += c;
            }
            s_warp[kThreads / 32] = acc;
        }
        __syncthreads();
        if (valid) list[nvalid + s_warp[warp] + __popc(m & ((1u << lane) - 1u))] = sl;
        nvalid += s_warp[kThreads / 32];
        __syncthreads();
    }
    for (int li = tid; li < nvalid; li += kThreads) {
        const int sl2 = list[li];
        const int nd = s.node[base + sl2];
        int k, line;
        slot_dir_line(sl2, N, k, line);
        const float q = s.q[base + sl2];
        const int fi = nd % v.nx, fj = nd / v.nx;
        const int kx = ex(k), ky = ey(k), kb = opp(k);
        const int i1 = fi - kx, j1 = fj - ky, i2 = fi - 2 * kx, j2 = fj - 2 * ky;
        const bool have1 = in_box(v, i1, j1) && v.own[(long long)j1 * v.nx + i1] == -1;
        const bool have2 = in_box(v, i2, j2) && v.own[(long long)j2 * v.nx + i2] == -1;
        const long long n0 = (long long)fj * v.pitch + fi;
        const long long n1 = have1 ? (long long)j1 * v.pitch + i1 : n0;
        const long long n2 = have2 ? (long long)j2 * v.pitch + i2 : n0;
        const float fk0 = A[k * ps + n0], fk1 = A[k * ps + n1], fk2 = A[k * ps + n2];
        const float fb0 = A[kb * ps + n0], fb1 = A[kb * ps + n1];
        float dxh, dxl, dyh, dyl;
        df_offset(fi, dk.xh, dk.xl, dxh, dxl);
        df_offset(fj, dk.yh, dk.yl, dyh, dyl);
        // an ellipse: the offset rounded from FP64, as the step's link kernel has it
        const float dxf = ell ? (float)((double)fi - xc) : dxh + dxl;
        const float dyf = ell ? (float)((double)fj - yc) : dyh + dyl;
        const float rx = dxf + q * kx, ry = dyf + q * ky;
        const float uwx = Ux - Om * ry, uwy = Uy + Om * rx;
        const float wall = 6.f * w9(k) * -(kx * uwx + ky * uwy);
        int lvl;
        const float fnew = bouzidi32(q, fk0, fk1, fk2, fb0, fb1, have1, have2, wall, lvl);
        const long long ns = (long long)(fj + ky) * v.pitch + (fi + kx);
        A[kb * ps + ns] = fnew;
        if (k <= 4)
            A[(kQ9 + kb) * ps + ns] = thermal32(q, A[(kQ9 + k) * ps + n0], A[(kQ9 + k) * ps + n1],
                                                A[(kQ9 + kb) * ps + n0], have1, wT);
        const float bx = fk0 * (kx - uwx) - fnew * (-kx - uwx);
        const float by = fk0 * (ky - uwy) - fnew * (-ky - uwy);
        lbx[li] = bx;
        lby[li] = by;
        ltq[li] = rx * by - ry * bx;
        lcode[li] = k | (lvl << 4) | ((k <= 4 && !have1) ? 64 : 0);
        ltz[li] = fi * ky - fj * kx;
    }
    broken = __syncthreads_or(broken);
    if (warp == 0) {
        LinkSums S;
        int c3[3];
        reduce_links(lbx, lby, ltq, lcode, ltz, nvalid, S, c3);
        if (lane == 0) {
            double Fx, Fy, Tz;
            assemble_force(S, xc, yc, Fx, Fy, Tz);
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            v.F[3 * p + 0] = broken ? nan : Fx;
            v.F[3 * p + 1] = broken ? nan : Fy;
            v.F[3 * p + 2] = broken ? nan : Tz;
        }
    }
}

// Device address of the static array on the current device.  Looked up on
// every call rather than cached: the query is cheap once the device code is
// loaded, and a cached address would go stale when the context is reset
// (cudaDeviceReset), which places the array anew.  In host code the array's
// name is only a host-side stand-in, never a device address.
int scratch_address(unsigned char **out)
{
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_link_scratch) != cudaSuccess || !ptr) return LBM_ECUDA;
    *out = static_cast<unsigned char *>(ptr);
    return LBM_OK;
}

} // namespace
} // namespace lbm

extern "C" int lbm_link_forces_noalloc(float *d_dist, int64_t plane_stride, int32_t pitch,
                                       const int32_t *d_owner, int32_t nx, int32_t ny,
                                       const lbm_particle *d_particles, int32_t n, double r_max,
                                       double *d_forces, void *stream)
{
    using namespace lbm;
    if (n < 0 || nx < 1 || ny < 1 || pitch < nx || plane_stride < (int64_t)pitch * ny) return LBM_EINVAL;
    // the index array stores j * nx + i as int32
    if ((long long)nx * ny > INT_MAX) return LBM_EINVAL;
    if (n == 0) return LBM_OK;
    if (!d_dist || !d_owner || !d_particles || !d_forces || !(r_max >= 1.0) || r_max > 1e6)
        return LBM_EINVAL;
    if (n > kStaticParticles || (long long)n * slot_capacity(r_max) > kStaticSlots) return LBM_ENOSPC;
    // the force kernel holds the slot list and per-link results of the
    // largest zone in shared memory
    const int capm = slot_capacity(r_max);
    const size_t smem = (size_t)capm * 6 * sizeof(int);
    if (smem > (size_t)200 * 1024) return LBM_ENOSPC;
    unsigned char *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    View v{d_dist, (long long)plane_stride, pitch, nx, ny, n, r_max, d_owner, d_particles, d_forces};
    k_static_bases<<<1, 32, 0, s>>>(v, scratch);
    k_static_gather<<<n, kThreads, 0, s>>>(v, scratch);
    if (smem > (size_t)48 * 1024 &&
        cudaFuncSetAttribute(k_static_bbforce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return LBM_ECUDA;
    k_static_bbforce<<<n, kThreads, smem, s>>>(v, scratch, capm);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}
