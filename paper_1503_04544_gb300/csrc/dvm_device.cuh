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

}  // namespace
}  // namespace dvm
