// Device helpers shared by the 2D and 3D step kernels: vector types of one
// velocity group, compensated sums, the limiter, block reductions and the
// TMA / mbarrier primitives (inline PTX).
#pragma once
#include "dvm_internal.h"

namespace dvm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kLog2e = 1.4426950408889634074;

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

template <typename T>
__device__ __forceinline__ void vld(const typename Vec<T>::type *p, T (&r)[Vec<T>::W])
{
    typename Vec<T>::type a = __ldg(p);
    if constexpr (Vec<T>::W == 4) { r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w; }
    else { r[0] = a.x; r[1] = a.y; }
}

template <typename T>
__device__ __forceinline__ void vst(typename Vec<T>::type *p, const T (&r)[Vec<T>::W])
{
    if constexpr (Vec<T>::W == 4) *p = make_float4(r[0], r[1], r[2], r[3]);
    else *p = make_double2(r[0], r[1]);
}

__device__ __forceinline__ float dexp2(float x) { return exp2f(x); }
__device__ __forceinline__ double dexp2(double x) { return exp2(x); }
__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }

// Two FP32 values in one 64-bit register pair, for the packed FP32
// instructions of sm_100 and later (add/sub/mul/fma.rn.f32x2: each lane is
// the correctly rounded scalar operation).
struct F2 { unsigned long long v; };
__device__ __forceinline__ F2 f2(float a, float b)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ F2 f2(float a) { return f2(a, a); }
__device__ __forceinline__ void f2_get(F2 x, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ F2 add2(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b)
{
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b)
{
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// minmod: 0 unless both arguments have the same strict sign, else the one of
// smaller magnitude.
template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    const T m = fmin(fabs(a), fabs(b));
    return a * b > T(0) ? copysign(m, a) : T(0);
}

// Compensated (Kahan) accumulator in FP32, plain sum in FP64.
template <typename T> struct Acc {
    T s = 0, c = 0;
    __device__ __forceinline__ void add(T x)
    {
        if constexpr (sizeof(T) == 4) {
            T y = x - c;
            T t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += x;
        }
    }
    // merge another (s, c) pair: (s1 - c1) + (s2 - c2) via TwoSum
    __device__ __forceinline__ void merge(T s2, T c2)
    {
        if constexpr (sizeof(T) == 4) {
            T t = s + s2;
            T bp = t - s;
            T e = (s - (t - bp)) + (s2 - bp);
            c = (c + c2) - e;
            s = t;
        } else {
            s += s2;
        }
    }
    __device__ __forceinline__ void warp_reduce()
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T s2 = __shfl_xor_sync(0xffffffffu, s, o);
            T c2 = __shfl_xor_sync(0xffffffffu, c, o);
            merge(s2, c2);
        }
    }
    __device__ __forceinline__ T value() const { return s - c; }
};

// Velocity chunks of the state-moment kernels (set-up and output): a block
// holds 32 consecutive cells of a row and kMomChunks warps, one chunk of the
// velocity groups each.
constexpr int kMomChunks = 8;

// Merges the compensated sums of the kMomChunks warps of a block into warp 0,
// chunk by chunk in order (the same result on every run).
template <typename T, int NM>
__device__ __forceinline__ void merge_chunks(Acc<T> (&s)[NM])
{
    __shared__ T sh[NM][2][kMomChunks][32];
    const int w = threadIdx.y, l = threadIdx.x;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        sh[m][0][w][l] = s[m].s;
        sh[m][1][w][l] = s[m].c;
    }
    __syncthreads();
    if (w == 0)
        for (int k = 1; k < kMomChunks; ++k)
#pragma unroll
            for (int m = 0; m < NM; ++m) s[m].merge(sh[m][0][k][l], sh[m][1][k][l]);
}

// A scalar in the state precision without FP64 arithmetic in FP32 kernels.
template <typename T>
__device__ __forceinline__ T pick(float f, double d)
{
    if constexpr (sizeof(T) == 4) return f;
    else return d;
}

// minmod(a, b) = median(a, b, 0): 0 unless a and b have the same strict sign,
// else the one of smaller magnitude (three min/max operations, exact).
template <typename T>
__device__ __forceinline__ T minmod3(T a, T b)
{
    return fmax(fmin(a, b), fmin(fmax(a, b), T(0)));
}

// min(|a|, |b|) with the sign bit sign(a) XOR sign(b): non-negative exactly
// when a and b have the same sign (one instruction on sm_86 and later).
__device__ __forceinline__ float min_xorsign_abs(float a, float b)
{
    float r;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// x with its sign flipped where s is negative (one bit operation).
__device__ __forceinline__ float xorsign(float x, float s)
{
    return __int_as_float(__float_as_int(x) ^ (__float_as_int(s) & (int)0x80000000));
}

// FP32: the magnitude max(min_xorsign_abs(a, b), 0) with the sign of a,
// which is the sign of the result where it is not zero (three operations;
// the same number, up to the sign of a zero).
__device__ __forceinline__ float minmod3(float a, float b)
{
    return xorsign(fmaxf(min_xorsign_abs(a, b), 0.f), a);
}

// The same for FP64 with integer operations on the bit patterns: the
// magnitudes of IEEE-754 doubles order as their bits without the sign, and
// the result is one of the arguments or zero, so it is exact (a zero result
// may differ in the sign of zero).  The integer pipe is far wider than the
// FP64 pipe, which on this part carries two lanes per clock per SM.
__device__ __forceinline__ double minmod3(double a, double b)
{
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const unsigned long long ma = (unsigned long long)ia & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long mb = (unsigned long long)ib & 0x7FFFFFFFFFFFFFFFull;
    const long long r = ma <= mb ? ia : ib;
    return (ia ^ ib) < 0 ? 0.0 : __longlong_as_double(r);
}

// The two limiter values of one axis that share the difference a: the
// downwind face minmod(b, a) and the upwind face minmod(a, c) (exact: each
// is one of its arguments or zero).
__device__ __forceinline__ void minmod_pair(float b, float a, float c, float &mo, float &mi)
{
    // magnitudes (see minmod_mag_pair); both values carry the sign of a
    mo = xorsign(fmaxf(min_xorsign_abs(b, a), 0.f), a);
    mi = xorsign(fmaxf(min_xorsign_abs(a, c), 0.f), a);
}
__device__ __forceinline__ void minmod_pair(double b, double a, double c, double &mo, double &mi)
{
    mo = minmod3(b, a);
    mi = minmod3(a, c);
}

// Magnitudes of the two limiter values of minmod_pair: |minmod(b, a)| =
// max(min_xorsign_abs(b, a), 0) and |minmod(a, c)| likewise.  Both limiter
// values, where not zero, have the sign of a.
__device__ __forceinline__ void minmod_mag_pair(float b, float a, float c, float &mo, float &mi)
{
    mo = fmaxf(min_xorsign_abs(b, a), 0.f);
    mi = fmaxf(min_xorsign_abs(a, c), 0.f);
}

// 2^x by the hardware approximation (relative error a few ulp; results below
// the smallest normal number flush to 0).
__device__ __forceinline__ float ex2_fast(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename T>
__device__ __forceinline__ void sld(const typename Vec<T>::type *p, T (&r)[Vec<T>::W])
{
    typename Vec<T>::type a = *p;
    if constexpr (Vec<T>::W == 4) { r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w; }
    else { r[0] = a.x; r[1] = a.y; }
}

// ---- TMA and mbarrier primitives (inline PTX, sm_90+)
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: false if the phase did not complete
// within kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (long it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Compensated block sum (all threads return the total); red holds 2 values
// per warp.
template <typename T>
__device__ __forceinline__ T block_acc(Acc<T> a, T *red)
{
    a.warp_reduce();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) { red[2 * warp] = a.s; red[2 * warp + 1] = a.c; }
    __syncthreads();
    Acc<T> t;
    for (int w = 0; w < nw; ++w) t.merge(red[2 * w], red[2 * w + 1]);
    return t.value();
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red)
{
    // deterministic block reduction (fixed tree)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = 0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

// Slab index of cell (i, j), -2 <= i < nx + 2, -2 <= j < ny + 2: the slab is
// the grid padded by two cells on every side, and the padding holds the
// boundary-condition values (Maxwellian ghosts, periodic images or
// zero-gradient copies), so a neighbour within two cells is a plain index.
__device__ __forceinline__ long nbr(const Grid2D &g, int i, int j)
{
    return (long)(j + 2) * (g.nx + 4) + (i + 2);
}

// Cell coordinates of interior cell k = j*nx + i (2D grids have fewer than
// 2^31 cells, so 32-bit arithmetic suffices).
__device__ __forceinline__ void cell_ij(const Grid2D &g, long k, int &i, int &j)
{
    const int kk = (int)k;
    j = kk / g.nx;
    i = kk - j * g.nx;
}

// Slab index of interior cell k.
__device__ __forceinline__ long pcell(const Grid2D &g, long k)
{
    int i, j;
    cell_ij(g, k, i, j);
    return nbr(g, i, j);
}

// Offset of (comp, p) within the device layout; add slab index * W.
template <typename T>
__device__ __forceinline__ long ebase(const Grid2D &g, int comp, int p)
{
    constexpr int W = Vec<T>::W;
    return ((long)(p / W) * 2 + comp) * g.slab * W + (p % W);
}

// Element (interior cell k, comp, p) of the device layout.
template <typename T>
__device__ __forceinline__ long didx(const Grid2D &g, long k, int comp, int p)
{
    return ebase<T>(g, comp, p) + pcell(g, k) * Vec<T>::W;
}

// Padding cells that mirror interior cell (i, j) on periodic and
// zero-gradient sides (at most two along each axis); -1 where unused.
template <typename I>
__device__ __forceinline__ void mirrors(const Grid2D &g, int i, int j, I (&m)[4])
{
    m[0] = m[1] = m[2] = m[3] = -1;
    if (g.bc[0] == DVM_BC_PERIODIC) {
        if (i < 2) m[0] = (I)nbr(g, i + g.nx, j);
        else if (i >= g.nx - 2) m[0] = (I)nbr(g, i - g.nx, j);
    } else {
        if (i == 0 && g.bc[0] == DVM_BC_ZEROGRAD) { m[0] = (I)nbr(g, -1, j); m[1] = (I)nbr(g, -2, j); }
        if (i == g.nx - 1 && g.bc[1] == DVM_BC_ZEROGRAD) { m[0] = (I)nbr(g, g.nx, j); m[1] = (I)nbr(g, g.nx + 1, j); }
    }
    if (g.bc[2] == DVM_BC_PERIODIC) {
        if (j < 2) m[2] = (I)nbr(g, i, j + g.ny);
        else if (j >= g.ny - 2) m[2] = (I)nbr(g, i, j - g.ny);
    } else {
        if (j == 0 && g.bc[2] == DVM_BC_ZEROGRAD) { m[2] = (I)nbr(g, i, -1); m[3] = (I)nbr(g, i, -2); }
        if (j == g.ny - 1 && g.bc[3] == DVM_BC_ZEROGRAD) { m[2] = (I)nbr(g, i, g.ny); m[3] = (I)nbr(g, i, g.ny + 1); }
    }
}

// Per-velocity coefficients: vx, vy, nu_x = |vx| dt/dx, nu_y = |vy| dt/dy.
// Padded velocities carry a huge speed (their Maxwellian is 0) and zero
// Courant numbers.
template <typename T> struct alignas(4 * sizeof(T)) VCoef { T vx, vy, nux, nuy; };

template <typename T>
__device__ __forceinline__ VCoef<T> ld_coef(const VCoef<T> *p)
{
    VCoef<T> c;
    if constexpr (sizeof(T) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        c.vx = a.x; c.vy = a.y; c.nux = a.z; c.nuy = a.w;
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        c.vx = a.x; c.vy = a.y; c.nux = b.x; c.nuy = b.y;
    }
    return c;
}

// Sector of a wall point for piecewise wall temperatures: the first s with
// cross(d_s, r) >= 0 and cross(d_{s+1}, r) < 0.
__device__ __forceinline__ double wall_temperature(const BodyParams &b, double rx, double ry)
{
    if (b.nseg <= 0) return b.Tw;
    for (int s = 0; s < b.nseg; ++s) {
        int t = (s + 1) % b.nseg;
        double p = b.seg_dir[2 * s] * ry - b.seg_dir[2 * s + 1] * rx;
        double q = b.seg_dir[2 * t] * ry - b.seg_dir[2 * t + 1] * rx;
        if (p >= 0 && q < 0) return b.Tw_seg[s];
    }
    return b.Tw_seg[0];
}

// One member (virtual cell) of a control volume, as the update needs it.
struct __align__(16) CvMember {
    long pc;                  // slab index
    long mir[4];              // padding mirrors (-1: none)
    int i, j;
    double L[4];              // Cartesian edge lengths at t^n: x-, x+, y-, y+
    double lw, nwx, nwy;      // wall edge at t^n (lw = 0: no wall)
    double sb;                // virtual-cell area at t^n
    int wslot;                // wall slot, -1 if none
    int mask;                 // limiter mask of the faces
    int live, keep;           // non-solid at t^n / at t^{n+1}
};

// A control volume: members in cell order, the master's slab index and the
// area ratios of Eq. ExSchemeDD, all fixed between geometry updates.
struct __align__(16) CvInfo {
    int nm;
    int ok;                   // S^{n+1,*} > 0
    long pcm;
    double a;                 // S^n / S^{n+1,*}
    double bco;               // dt / S^{n+1,*}
    double Sn;
    CvMember mem[kMaxMembers];
};

}  // namespace
}  // namespace dvm
