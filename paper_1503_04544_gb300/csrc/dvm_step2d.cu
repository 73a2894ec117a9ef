// 2D time step of the cut-cell discrete-velocity method (arXiv:1503.04544,
// Sec. 3.3.5): fusion (Eq. FusionDD), wall density and stress (Eqs.
// BoundaryDDv, StressTensorDD), force/torque and rotation (Eqs. eq-force,
// eq-torque, motionDD_posit, motionDD_vit), fluxes and explicit update of the
// reduced pair (f, g) (Eqs. FluxDD, ExSchemeDD, BGKDD) and distribution
// (Eq. UpdateDD).  Device layout: see dvm_internal.h.
//
// Kernels of one step (fixed obstacle): k_wall (FP64 wall density, wall
// fluxes, force/torque, rigid-body update in its last block), k_bulk (every
// gas cell that is a control volume on its own), k_special (cut and merged
// control volumes).  A moving obstacle adds the geometry of t^{n+1}, the
// control volumes of t^n and k_fusion before them.
//
// k_bulk: one thread per cell, 32 consecutive cells in x per warp and kRows
// rows per block; the velocity grid is split over blockIdx.z.  Each thread
// walks its velocity groups, reads its cell and the upwind/downwind
// neighbours of the group (the upwind side is uniform across the warp), and
// writes the new state and the partial moments of its split.  The moments of
// the state at t^n are the sums of the partials written by the previous step.
#include <cudaTypedefs.h>

#include <cstdio>
#include <string>

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

// Element (cell, comp, p) of the device layout.
template <typename T>
__device__ __forceinline__ long didx(const Grid2D &g, long cell, int comp, int p)
{
    constexpr int W = Vec<T>::W;
    return ((long)(p / W) * 2 + comp) * g.slab * W + cell * W + (p % W);
}

// Slab index of cell (i, j) or of the ghost cell that replaces it beyond a
// side: periodic wrap, Maxwellian ghost, zero-gradient copy of the boundary.
__device__ __forceinline__ long nbr(const Grid2D &g, int i, int j)
{
    const long nc = (long)g.nx * g.ny;
    if (i < 0) {
        if (g.bc[0] == DVM_BC_PERIODIC) i = ((i % g.nx) + g.nx) % g.nx;
        else if (g.bc[0] == DVM_BC_MAXWELLIAN) return nc + g.gofs[0] + j;
        else i = 0;
    } else if (i >= g.nx) {
        if (g.bc[1] == DVM_BC_PERIODIC) i = i % g.nx;
        else if (g.bc[1] == DVM_BC_MAXWELLIAN) return nc + g.gofs[1] + j;
        else i = g.nx - 1;
    }
    if (j < 0) {
        if (g.bc[2] == DVM_BC_PERIODIC) j = ((j % g.ny) + g.ny) % g.ny;
        else if (g.bc[2] == DVM_BC_MAXWELLIAN) return nc + g.gofs[2] + i;
        else j = 0;
    } else if (j >= g.ny) {
        if (g.bc[3] == DVM_BC_PERIODIC) j = j % g.ny;
        else if (g.bc[3] == DVM_BC_MAXWELLIAN) return nc + g.gofs[3] + i;
        else j = g.ny - 1;
    }
    return (long)j * g.nx + i;
}

// Primitive variables (Eq. MacroscopicDDv; T from E = rho|u|^2/2 + 3/2 rho T)
// from the reduced sums s0 = sum f, s1 = sum vx f, s2 = sum vy f,
// s3 = sum (|v|^2/2 f + g).
template <typename T>
__device__ __forceinline__ bool primitives(double dv, T s0, T s1, T s2, T s3, T &rho, T &ux, T &uy, T &tmp)
{
    rho = s0 * T(dv);
    ux = s1 / s0;
    uy = s2 / s0;
    tmp = (T(2) * (s3 / s0) - (ux * ux + uy * uy)) / T(3);
    return rho > T(0) && tmp > T(0);
}

// Sum of the S partial moments of a cell ([S][4][nc] layout).
template <typename T>
__device__ __forceinline__ void gather_partials(const T *part, int S, long nc, long cell, T (&s)[4])
{
    Acc<T> a[4];
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) a[m].merge(part[((long)q * 4 + m) * nc + cell], T(0));
#pragma unroll
    for (int m = 0; m < 4; ++m) s[m] = a[m].value();
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

template <typename T> struct BulkArgs {
    Grid2D g;
    int S;
    const T *fin;
    T *fout;
    const T *pin;             // partial moments of f^n   [S][4][nc]
    T *pout;                  // partial moments of f^n+1 [S][4][nc]
    const uint8_t *flags;
    const VCoef<T> *vt;       // [nvp]
    const int8_t *gsign;      // [ngrp][2]
    int *err;
};

// ------------------------------------------------------------ bulk kernel
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

constexpr int kStageBytes = 2 * kTileY * kTileX * 16;     // both components of one group

// Update of one component of one velocity group for the thread's cell from
// the shared-memory tile (Eq. ExSchemeDD on a full gas cell, fluxes of Eq.
// FluxDD in difference form with the limited reconstruction), moment sums.
// c0 is the tile index of the cell; ox/oy the tile strides of one cell
// step along x/y towards the upwind side (per element in the mixed case).
template <typename T, bool MUSCL, int COMP, bool UNIFORM>
__device__ __forceinline__ void bulk_tile(const typename Vec<T>::type *t, int c0, int ux1, int uy1,
                                          const T (&vx)[Vec<T>::W], const T (&vy)[Vec<T>::W],
                                          const T (&nux)[Vec<T>::W], const T (&nuy)[Vec<T>::W],
                                          const T (&feq)[Vec<T>::W], T wxm, T wxp, T wym, T wyp, T r,
                                          T (&out)[Vec<T>::W], T &q0, T &q1, T &q2, T &q3)
{
    constexpr int W = Vec<T>::W;
    T f[W];
    sld<T>(t + c0, f);
    if (UNIFORM) {
        // ux1/uy1: tile offset of the upwind neighbour (+-1 or +-kTileX)
        T u1[W], w1[W], d1[W], u2[W], e1[W], w2[W];
        sld<T>(t + c0 - ux1, u1);
        sld<T>(t + c0 - uy1, w1);
        if (MUSCL) {
            sld<T>(t + c0 + ux1, d1);
            sld<T>(t + c0 - 2 * ux1, u2);
            sld<T>(t + c0 + uy1, e1);
            sld<T>(t + c0 - 2 * uy1, w2);
        }
        const bool px = ux1 > 0, py = uy1 > 0;
        const T cxo = px ? wxp : wxm, cxi = px ? wxm : wxp;
        const T cyo = py ? wyp : wym, cyi = py ? wym : wyp;
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const T ax = f[e] - u1[e], ay = f[e] - w1[e];
            T dfx = ax, dfy = ay;
            if (MUSCL) {
                dfx += (T(1) - nux[e]) * (cxo * minmod3(d1[e] - f[e], ax) - cxi * minmod3(ax, u1[e] - u2[e]));
                dfy += (T(1) - nuy[e]) * (cyo * minmod3(e1[e] - f[e], ay) - cyi * minmod3(ay, w1[e] - w2[e]));
            }
            out[e] = f[e] - nux[e] * dfx - nuy[e] * dfy + r * (feq[e] - f[e]);
        }
    } else {
        T xm[W], xp[W], ym[W], yp[W], xm2[W], xp2[W], ym2[W], yp2[W];
        sld<T>(t + c0 - 1, xm); sld<T>(t + c0 + 1, xp);
        sld<T>(t + c0 - kTileX, ym); sld<T>(t + c0 + kTileX, yp);
        if (MUSCL) {
            sld<T>(t + c0 - 2, xm2); sld<T>(t + c0 + 2, xp2);
            sld<T>(t + c0 - 2 * kTileX, ym2); sld<T>(t + c0 + 2 * kTileX, yp2);
        }
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const bool px = vx[e] >= T(0), py = vy[e] >= T(0);
            const T u1 = px ? xm[e] : xp[e], w1 = py ? ym[e] : yp[e];
            const T ax = f[e] - u1, ay = f[e] - w1;
            T dfx = ax, dfy = ay;
            if (MUSCL) {
                const T d1 = px ? xp[e] : xm[e], u2 = px ? xm2[e] : xp2[e];
                const T e1 = py ? yp[e] : ym[e], w2 = py ? ym2[e] : yp2[e];
                const T cxo = px ? wxp : wxm, cxi = px ? wxm : wxp;
                const T cyo = py ? wyp : wym, cyi = py ? wym : wyp;
                dfx += (T(1) - nux[e]) * (cxo * minmod3(d1 - f[e], ax) - cxi * minmod3(ax, u1 - u2));
                dfy += (T(1) - nuy[e]) * (cyo * minmod3(e1 - f[e], ay) - cyi * minmod3(ay, w1 - w2));
            }
            out[e] = f[e] - nux[e] * dfx - nuy[e] * dfy + r * (feq[e] - f[e]);
        }
    }
#pragma unroll
    for (int e = 0; e < W; ++e) {
        if (COMP == 0) {
            q0 += out[e];
            q1 += vx[e] * out[e];
            q2 += vy[e] * out[e];
            q3 += T(0.5) * (vx[e] * vx[e] + vy[e] * vy[e]) * out[e];
        } else {
            q3 += out[e];
        }
    }
}

// Bulk update.  Block = 32 x kRows cells; the velocity groups of split
// blockIdx.z stream through a kStages-deep ring of shared-memory tiles
// (the block's cells plus a two-cell halo, both components of one group),
// each filled by one TMA tensor load completing on an mbarrier.  Halo cells
// beyond the domain are replaced by their boundary-condition values after
// the load.  Every thread of the block takes part in the waits and barriers;
// only threads of plain cells compute.
template <typename T, bool MUSCL>
__global__ void __launch_bounds__(32 * kRows, 2) k_bulk(BulkArgs<T> a, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    V *ring = reinterpret_cast<V *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    const Grid2D &g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * kRows;
    const int i = i0 + tx, j = j0 + ty;
    const bool inside = i < g.nx && j < g.ny;
    const long nc = (long)g.nx * g.ny;
    const long cell = inside ? (long)j * g.nx + i : 0;
    const int split = blockIdx.z;
    const int gps = (g.ngrp + a.S - 1) / a.S;
    const int g0 = split * gps, g1 = min(g0 + gps, g.ngrp);
    const int ngr = max(g1 - g0, 0);
    const uint8_t fl = inside ? a.flags[cell] : 0;
    const bool plain = (fl & kPlain) != 0, zero = (fl & kZero) != 0;
    const V *fin = reinterpret_cast<const V *>(a.fin);
    V *fout = reinterpret_cast<V *>(a.fout);

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        mbar_fence_init();
        for (int st = 0; st < kStages - 1 && st < ngr; ++st) {
            mbar_expect_tx(&bars[st], kStageBytes);
            tma_load_3d(ring + (long)st * (kStageBytes / 16), &tmap, &bars[st], (i0 - 2) * W, j0 - 2, (g0 + st) * 2);
        }
    }

    // equilibrium of the cell at t^n
    T A = 0, c2 = 0, r = 0, gfac = 0, ux = 0, uy = 0;
    if (plain) {
        T s[4];
        gather_partials(a.pin, a.S, nc, cell, s);
        T rho, tmp;
        if (!primitives<T>(g.dv, s[0], s[1], s[2], s[3], rho, ux, uy, tmp)) atomicExch(&a.err[kErrNonphys], 1);
        A = rho / (T(2.0 * kPi) * tmp);
        c2 = T(kLog2e) / (T(2) * tmp);
        r = T(g.dt / g.tau0) * rho;
        gfac = tmp / T(2);
    }
    const int mask = fl >> kMaskShift;
    // limiter weights of the faces x-, x+, y-, y+ (1/2 where the limited
    // reconstruction is allowed, 0 where the flux falls back to first order)
    const T wxm = (mask & 1) ? T(0.5) : T(0), wxp = (mask & 2) ? T(0.5) : T(0);
    const T wym = (mask & 4) ? T(0.5) : T(0), wyp = (mask & 8) ? T(0.5) : T(0);
    const int c0 = (ty + 2) * kTileX + tx + 2;
    const bool edge = i0 - 2 < 0 || i0 + 34 > g.nx || j0 - 2 < 0 || j0 + kRows + 2 > g.ny;
    __syncthreads();

    Acc<T> m0, m1, m2, m3;
    T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
    int fold = 0;
    for (int it = 0; it < ngr; ++it) {
        const int q = g0 + it, st = it % kStages;
        const uint32_t parity = (uint32_t)((it / kStages) & 1);
        if (tid == 0 && it + kStages - 1 < ngr) {
            const int s2 = (it + kStages - 1) % kStages;
            mbar_expect_tx(&bars[s2], kStageBytes);
            tma_load_3d(ring + (long)s2 * (kStageBytes / 16), &tmap, &bars[s2], (i0 - 2) * W, j0 - 2,
                        (g0 + it + kStages - 1) * 2);
        }
        const bool ok = mbar_wait(&bars[st], parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(&a.err[kErrTimeout], 1);
                // let the copies already issued land before the block exits
                for (int k2 = it; k2 < it + kStages && k2 < ngr; ++k2)
                    mbar_wait(&bars[k2 % kStages], (uint32_t)((k2 / kStages) & 1));
            }
            __syncthreads();
            return;
        }
        V *tile = ring + (long)st * (kStageBytes / 16);
        if (edge) {
            // halo cells beyond the domain: boundary-condition values
            for (int e = tid; e < 2 * kTileY * kTileX; e += 32 * kRows) {
                const int comp = e / (kTileY * kTileX), rem = e % (kTileY * kTileX);
                const int rr = rem / kTileX, cc = rem % kTileX;
                const int gi = i0 - 2 + cc, gj = j0 - 2 + rr;
                const bool inx = gi >= 0 && gi < g.nx, iny = gj >= 0 && gj < g.ny;
                const bool cross = (cc >= 2 && cc < 34) || (rr >= 2 && rr < kRows + 2);
                if ((inx && iny) || !cross) continue;
                if (!inx && !iny) continue;
                tile[e] = fin[((long)q * 2 + comp) * g.slab + nbr(g, gi, gj)];
            }
            __syncthreads();
        }
        if (plain) {
            const int sx = a.gsign[2 * q], sy = a.gsign[2 * q + 1];
            T vx[W], vy[W], nux[W], nuy[W], feq[W], out[W];
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const VCoef<T> vc = ld_coef(a.vt + q * W + e);
                vx[e] = vc.vx; vy[e] = vc.vy; nux[e] = vc.nux; nuy[e] = vc.nuy;
                const T dx = vc.vx - ux, dy = vc.vy - uy;
                feq[e] = A * dexp2(-(dx * dx + dy * dy) * c2);
            }
            V *o0 = fout + (long)q * 2 * g.slab + cell;
            if (sx != 0 && sy != 0) {
                const int ux1 = sx > 0 ? 1 : -1, uy1 = sy > 0 ? kTileX : -kTileX;
                bulk_tile<T, MUSCL, 0, true>(tile, c0, ux1, uy1, vx, vy, nux, nuy, feq, wxm, wxp, wym, wyp, r,
                                             out, q0, q1, q2, q3);
                vst<T>(o0, out);
#pragma unroll
                for (int e = 0; e < W; ++e) feq[e] *= gfac;
                bulk_tile<T, MUSCL, 1, true>(tile + kTileY * kTileX, c0, ux1, uy1, vx, vy, nux, nuy, feq, wxm,
                                             wxp, wym, wyp, r, out, q0, q1, q2, q3);
                vst<T>(o0 + g.slab, out);
            } else {
                bulk_tile<T, MUSCL, 0, false>(tile, c0, 1, kTileX, vx, vy, nux, nuy, feq, wxm, wxp, wym, wyp, r,
                                              out, q0, q1, q2, q3);
                vst<T>(o0, out);
#pragma unroll
                for (int e = 0; e < W; ++e) feq[e] *= gfac;
                bulk_tile<T, MUSCL, 1, false>(tile + kTileY * kTileX, c0, 1, kTileX, vx, vy, nux, nuy, feq, wxm,
                                              wxp, wym, wyp, r, out, q0, q1, q2, q3);
                vst<T>(o0 + g.slab, out);
            }
            // fold the plain sums of 8 groups into the compensated sums
            if (++fold == 8) {
                m0.add(q0); m1.add(q1); m2.add(q2); m3.add(q3);
                q0 = q1 = q2 = q3 = 0;
                fold = 0;
            }
        } else if (zero) {
            T z[W];
#pragma unroll
            for (int e = 0; e < W; ++e) z[e] = 0;
            vst<T>(fout + (long)q * 2 * g.slab + cell, z);
            vst<T>(fout + ((long)q * 2 + 1) * g.slab + cell, z);
        }
        __syncthreads();      // the stage is refilled at the next iteration
    }
    if (plain) {
        m0.add(q0); m1.add(q1); m2.add(q2); m3.add(q3);
        a.pout[((long)split * 4 + 0) * nc + cell] = m0.value();
        a.pout[((long)split * 4 + 1) * nc + cell] = m1.value();
        a.pout[((long)split * 4 + 2) * nc + cell] = m2.value();
        a.pout[((long)split * 4 + 3) * nc + cell] = m3.value();
    } else if (zero) {
#pragma unroll
        for (int m = 0; m < 4; ++m) a.pout[((long)split * 4 + m) * nc + cell] = 0;
    }
}

// ------------------------------------------------------------ control volumes
struct CvArgs {
    Grid2D g;
    Geo2D Gn, Gp;
    const int32_t *master;
    const uint8_t *flags;
    const int32_t *spec_list;
    const int32_t *wall_list;
    const int32_t *wslot;
    const int32_t *counts;
    int cap;
    int S;
    int *err;
};

// Ordered list of the members of control volume m (cells whose master is m),
// scanned in row-major order over the window reachable by the master search.
__device__ int gather_members(const CvArgs &c, long m, int32_t *mem)
{
    __shared__ int wcnt[16];
    const Grid2D &g = c.g;
    const int R = kMaxWalk, Wd = 2 * kMaxWalk + 1, npos = Wd * Wd;
    const int mi = (int)(m % g.nx), mj = (int)(m / g.nx);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int total = 0;
    for (int base = 0; base < npos; base += 32 * nw) {
        int pos = base + warp * 32 + lane;
        bool hit = false;
        if (pos < npos) {
            int ii = mi - R + pos % Wd, jj = mj - R + pos / Wd;
            if (ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny)
                hit = c.master[(long)jj * g.nx + ii] == (int32_t)m;
        }
        unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = total;
        for (int w = 0; w < warp; ++w) off += wcnt[w];
        int rank = off + __popc(bal & ((1u << lane) - 1u));
        if (hit) {
            if (rank < kMaxMembers) {
                int ii = mi - R + pos % Wd, jj = mj - R + pos / Wd;
                mem[rank] = jj * g.nx + ii;
            } else {
                atomicExch(&c.err[kErrCapacity], 1);
            }
        }
        int add = 0;
        for (int w = 0; w < nw; ++w) add += wcnt[w];
        total += add;
        __syncthreads();
    }
    return total < kMaxMembers ? total : kMaxMembers;
}

template <typename T>
__device__ __forceinline__ T face_flux(T L, T v, T nu, T fAA, T fA, T fB, T fBB, bool muscl)
{
    if (!muscl) return L * (fmin(v, T(0)) * fB + fmax(v, T(0)) * fA);
    T fr;
    if (v > T(0)) fr = fA + T(0.5) * (T(1) - nu) * minmod(fB - fA, fA - fAA);
    else if (v < T(0)) fr = fB - T(0.5) * (T(1) - nu) * minmod(fBB - fB, fB - fA);
    else return T(0);
    return L * (v * fr);
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

// Write the moment sums of a control volume to a member: split 0 holds the
// sums, the other splits 0 (solid members get zeros).
template <typename T>
__device__ __forceinline__ void write_member_partials(T *part, int S, long nc, long k, bool keep,
                                                      T s0, T s1, T s2, T s3)
{
    for (int q = 0; q < S; ++q) {
        const bool z = q > 0 || !keep;
        part[((long)q * 4 + 0) * nc + k] = z ? T(0) : s0;
        part[((long)q * 4 + 1) * nc + k] = z ? T(0) : s1;
        part[((long)q * 4 + 2) * nc + k] = z ? T(0) : s2;
        part[((long)q * 4 + 3) * nc + k] = z ? T(0) : s3;
    }
}

// Fusion (Eq. FusionDD): f_CV = sum sbar f / S over a merged control volume,
// written back to every member, with the moment sums of the result.
template <typename T>
__global__ void __launch_bounds__(256) k_fusion(CvArgs c, T *f, T *part)
{
    __shared__ int32_t mem[kMaxMembers];
    __shared__ double sb[kMaxMembers];
    __shared__ double red[8 * 4];
    const Grid2D &g = c.g;
    const long nc = (long)g.nx * g.ny;
    const int n = min(c.counts[0], c.cap);
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const long m = c.spec_list[idx];
        const int nm = gather_members(c, m, mem);
        if (nm <= 1) continue;
        double S = 0;
        for (int q = 0; q < nm; ++q) S += c.Gn.sbar[mem[q]];
        for (int q = threadIdx.x; q < nm; q += blockDim.x) sb[q] = c.Gn.sbar[mem[q]];
        __syncthreads();
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int comp = 0; comp < 2; ++comp)
            for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
                double s = 0;
                for (int q = 0; q < nm; ++q) s += sb[q] * (double)f[didx<T>(g, mem[q], comp, p)];
                const T fcv = (T)(s / S);
                for (int q = 0; q < nm; ++q) f[didx<T>(g, mem[q], comp, p)] = fcv;
                const double vx = g.vxmin + (p % g.nvx) * g.dvx, vy = g.vymin + (p / g.nvx) * g.dvy;
                if (comp == 0) { a0 += fcv; a1 += vx * fcv; a2 += vy * fcv; a3 += 0.5 * (vx * vx + vy * vy) * fcv; }
                else a3 += fcv;
            }
        a0 = block_sum(a0, red); a1 = block_sum(a1, red + 8);
        a2 = block_sum(a2, red + 16); a3 = block_sum(a3, red + 24);
        if (threadIdx.x < nm)
            write_member_partials<T>(part, c.S, nc, mem[threadIdx.x], c.Gn.type[mem[threadIdx.x]] != DVM_SOLID,
                                     (T)a0, (T)a1, (T)a2, (T)a3);
        __syncthreads();
    }
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

// Wall density (Eq. BoundaryDDv), stress (Eq. StressTensorDD), the wall-edge
// flux of every velocity (Eq. FluxDD) and the cell's force and torque
// (Eqs. eq-force, eq-torque), in FP64.  The wall velocity is
// u_w = u_c + (r - c)^perp omega (Eq. uwDD) at t^n.  The last block to finish
// sums the force and torque over the wall list in list order, advances the
// angular velocity (Eq. motionDD_vit) and records the history.
template <typename T>
__global__ void __launch_bounds__(256) k_wall(CvArgs c, BodyParams b, BodyDev *body, const T *f,
                                              T *wflux, double *wphi, double *wcontrib, int *ticket,
                                              double *hist, int moving)
{
    __shared__ double red[8 * 8];
    __shared__ double ex[kMaxAxisNv], ey[kMaxAxisNv];
    __shared__ double sphi;
    __shared__ bool last;
    const Grid2D &g = c.g;
    const int n = min(c.counts[1], c.cap);
    const double omega = body->omega;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const long k = c.wall_list[idx];
        const double rx = c.Gn.rwx[k] - b.cx, ry = c.Gn.rwy[k] - b.cy;
        const double uwx = b.vbx - ry * omega, uwy = b.vby + rx * omega;
        const double Tw = wall_temperature(b, rx, ry);
        const double nwx = c.Gn.nwx[k], nwy = c.Gn.nwy[k], lw = c.Gn.lw[k];
        // separable Maxwellian M[1, u_w, T_w] = ex[p1] ey[p2] / (2 pi T_w)
        for (int q = threadIdx.x; q < g.nvx + g.nvy; q += blockDim.x) {
            if (q < g.nvx) { double d = g.vxmin + q * g.dvx - uwx; ex[q] = exp(-(d * d) / (2.0 * Tw)); }
            else { int qq = q - g.nvx; double d = g.vymin + qq * g.dvy - uwy; ey[qq] = exp(-(d * d) / (2.0 * Tw)); }
        }
        __syncthreads();
        const double cm = 1.0 / (2.0 * kPi * Tw);
        double num = 0, den = 0, ixx = 0, ixy = 0, iyy = 0, oxx = 0, oxy = 0, oyy = 0;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const int p1 = p % g.nvx, p2 = p / g.nvx;
            const double ax = g.vxmin + p1 * g.dvx - uwx, ay = g.vymin + p2 * g.dvy - uwy;
            const double cp = ax * nwx + ay * nwy;
            if (cp > 0) {
                const double fv = (double)f[didx<T>(g, k, 0, p)];
                num += cp * fv;
                oxx += ax * ax * fv; oxy += ax * ay * fv; oyy += ay * ay * fv;
            } else if (cp < 0) {
                const double m1 = cm * ex[p1] * ey[p2];
                den += cp * m1;
                ixx += ax * ax * m1; ixy += ax * ay * m1; iyy += ay * ay * m1;
            }
        }
        num = block_sum(num, red); den = block_sum(den, red + 8);
        ixx = block_sum(ixx, red + 16); ixy = block_sum(ixy, red + 24); iyy = block_sum(iyy, red + 32);
        oxx = block_sum(oxx, red + 40); oxy = block_sum(oxy, red + 48); oyy = block_sum(oyy, red + 56);
        if (threadIdx.x == 0) {
            const double phi = -(num * g.dv) / (den * g.dv);
            const double sxx = (phi * ixx + oxx) * g.dv, sxy = (phi * ixy + oxy) * g.dv;
            const double syy = (phi * iyy + oyy) * g.dv;
            const double fx = (sxx * nwx + sxy * nwy) * lw, fy = (sxy * nwx + syy * nwy) * lw;
            wphi[idx] = phi;
            wcontrib[3 * idx] = fx;
            wcontrib[3 * idx + 1] = fy;
            wcontrib[3 * idx + 2] = rx * fy - ry * fx;
            sphi = phi;
        }
        __syncthreads();
        const double phi = sphi;
        for (int comp = 0; comp < 2; ++comp)
            for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
                const int p1 = p % g.nvx, p2 = p / g.nvx;
                const double ax = g.vxmin + p1 * g.dvx - uwx, ay = g.vymin + p2 * g.dvy - uwy;
                const double cp = ax * nwx + ay * nwy;
                const double m1 = cm * ex[p1] * ey[p2];
                const double fw = comp == 0 ? phi * m1 : phi * (Tw / 2.0 * m1);
                const double fv = (double)f[didx<T>(g, k, comp, p)];
                wflux[((long)idx * 2 + comp) * g.nv + p] = (T)(lw * (fmin(cp, 0.0) * fw + fmax(cp, 0.0) * fv));
            }
        __syncthreads();
    }
    // the last block sums the contributions in list order
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double fx = 0, fy = 0, tq = 0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        fx += wcontrib[3 * t]; fy += wcontrib[3 * t + 1]; tq += wcontrib[3 * t + 2];
    }
    fx = block_sum(fx, red); fy = block_sum(fy, red + 8); tq = block_sum(tq, red + 16);
    if (threadIdx.x == 0) {
        body->F[0] = fx; body->F[1] = fy; body->F[2] = 0; body->torque = tq;
        const double om1 = moving ? body->omega + g.dt * tq / b.inertia : body->omega;
        body->theta = body->theta1;
        body->omega = om1;
        body->trig[0] = body->trig[2];
        body->trig[1] = body->trig[3];
        double *h = hist + 6 * (body->step % kHistCap);
        h[0] = fx; h[1] = fy; h[2] = 0; h[3] = tq; h[4] = body->theta; h[5] = om1;
        body->step += 1;
        *ticket = 0;
    }
}

// Value of virtual cell (i, j), component comp, velocity p, with the
// domain boundary conditions.
template <typename T>
__device__ __forceinline__ T fval(const Grid2D &g, const T *f, int i, int j, int comp, int p)
{
    return f[didx<T>(g, nbr(g, i, j), comp, p)];
}

// Explicit update of one control volume (Eq. ExSchemeDD): fluxes across the
// Cartesian edges of every member (Eq. FluxDD) plus its wall-edge flux,
// area ratio S^n / S^{n+1,*}, relaxation, then distribution to the members
// (Eq. UpdateDD; members solid at t^{n+1} hold 0) and the moment sums.
template <typename T>
__global__ void __launch_bounds__(256) k_special(CvArgs c, const T *fin, T *fout, const T *pin,
                                                 T *pout, const T *wflux)
{
    __shared__ int32_t mem[kMaxMembers];
    __shared__ T L[kMaxMembers][4];           // lx-, lx+, ly-, ly+
    __shared__ int32_t ws[kMaxMembers];       // wall slot
    __shared__ int8_t mk[kMaxMembers];        // limiter mask
    __shared__ int8_t live[kMaxMembers];      // non-solid at t^n
    __shared__ int8_t keep[kMaxMembers];      // non-solid at t^{n+1}
    __shared__ double red[8 * 4];
    const Grid2D &g = c.g;
    const long nc = (long)g.nx * g.ny;
    const int n = min(c.counts[0], c.cap);
    const int W1 = g.nx + 1;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const long m = c.spec_list[idx];
        const int nm = gather_members(c, m, mem);
        for (int q = threadIdx.x; q < nm; q += blockDim.x) {
            const long k = mem[q];
            const int i = (int)(k % g.nx), j = (int)(k / g.nx);
            L[q][0] = (T)c.Gn.lx[(long)j * W1 + i];
            L[q][1] = (T)c.Gn.lx[(long)j * W1 + i + 1];
            L[q][2] = (T)c.Gn.ly[(long)j * g.nx + i];
            L[q][3] = (T)c.Gn.ly[(long)(j + 1) * g.nx + i];
            ws[q] = c.wslot[k];
            mk[q] = (int8_t)(c.flags[k] >> kMaskShift);
            live[q] = c.Gn.type[k] != DVM_SOLID;
            keep[q] = c.Gp.type[k] != DVM_SOLID;
        }
        __syncthreads();
        double Sn = 0, Sp = 0;
        for (int q = 0; q < nm; ++q) { Sn += c.Gn.sbar[mem[q]]; Sp += c.Gp.sbar[mem[q]]; }
        if (!(Sp > 0)) {
            if (threadIdx.x == 0) atomicExch(&c.err[kErrGeometry], 1);
            __syncthreads();
            continue;
        }
        T s[4];
        gather_partials(pin, c.S, nc, m, s);
        T rho, ux, uy, tmp;
        if (!primitives<T>(g.dv, s[0], s[1], s[2], s[3], rho, ux, uy, tmp) && threadIdx.x == 0)
            atomicExch(&c.err[kErrNonphys], 1);
        const T a = T(Sn / Sp), bco = T(g.dt / Sp), r = T(g.dt / g.tau0) * rho;
        const T A = rho / (T(2.0 * kPi) * tmp);
        Acc<T> s0, s1, s2, s3;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const int p1 = p % g.nvx, p2 = p / g.nvx;
            const T vx = T(g.vxmin + p1 * g.dvx), vy = T(g.vymin + p2 * g.dvy);
            const T nux = fabs(vx) * T(g.dt / g.dx), nuy = fabs(vy) * T(g.dt / g.dy);
            const T dxu = vx - ux, dyu = vy - uy;
            const T feq0 = A * dexp(-(dxu * dxu + dyu * dyu) / (T(2) * tmp));
            for (int comp = 0; comp < 2; ++comp) {
                T R = 0;
                for (int q = 0; q < nm; ++q) {
                    if (!live[q]) continue;
                    const long k = mem[q];
                    const int i = (int)(k % g.nx), j = (int)(k / g.nx);
                    const T fc = fin[didx<T>(g, k, comp, p)];
                    const T fxm1 = fval(g, fin, i - 1, j, comp, p), fxp1 = fval(g, fin, i + 1, j, comp, p);
                    const T fym1 = fval(g, fin, i, j - 1, comp, p), fyp1 = fval(g, fin, i, j + 1, comp, p);
                    T fxm2 = 0, fxp2 = 0, fym2 = 0, fyp2 = 0;
                    if (mk[q]) {
                        fxm2 = fval(g, fin, i - 2, j, comp, p); fxp2 = fval(g, fin, i + 2, j, comp, p);
                        fym2 = fval(g, fin, i, j - 2, comp, p); fyp2 = fval(g, fin, i, j + 2, comp, p);
                    }
                    const T Fxp = face_flux<T>(L[q][1], vx, nux, fxm1, fc, fxp1, fxp2, mk[q] & 2);
                    const T Fxm = face_flux<T>(L[q][0], vx, nux, fxm2, fxm1, fc, fxp1, mk[q] & 1);
                    const T Fyp = face_flux<T>(L[q][3], vy, nuy, fym1, fc, fyp1, fyp2, mk[q] & 8);
                    const T Fym = face_flux<T>(L[q][2], vy, nuy, fym2, fym1, fc, fyp1, mk[q] & 4);
                    const T Fw = ws[q] >= 0 ? wflux[((long)ws[q] * 2 + comp) * g.nv + p] : T(0);
                    R += (Fxp - Fxm) + (Fyp - Fym) + Fw;
                }
                const T fcv = fin[didx<T>(g, m, comp, p)];
                const T feq = comp == 0 ? feq0 : tmp / T(2) * feq0;
                const T fn = a * fcv - bco * R + a * r * (feq - fcv);
                for (int q = 0; q < nm; ++q) fout[didx<T>(g, mem[q], comp, p)] = keep[q] ? fn : T(0);
                if (comp == 0) {
                    s0.add(fn); s1.add(vx * fn); s2.add(vy * fn);
                    s3.add(T(0.5) * (vx * vx + vy * vy) * fn);
                } else {
                    s3.add(fn);
                }
            }
        }
        const double t0 = block_sum((double)s0.value(), red), t1 = block_sum((double)s1.value(), red + 8);
        const double t2 = block_sum((double)s2.value(), red + 16), t3 = block_sum((double)s3.value(), red + 24);
        if (threadIdx.x < nm) write_member_partials<T>(pout, c.S, nc, mem[threadIdx.x], keep[threadIdx.x],
                                                       (T)t0, (T)t1, (T)t2, (T)t3);
        __syncthreads();
    }
}

// Body position at t^{n+1} (Eq. motionDD_posit) and its trigonometry.
__global__ void k_advance(BodyDev *b, double dt, int moving)
{
    if (threadIdx.x != 0) return;
    b->theta1 = moving ? b->theta + dt * b->omega : b->theta;
    b->trig[2] = cos(b->theta1);
    b->trig[3] = sin(b->theta1);
}

// Moment sums of the current state for every cell (warp per cell), written
// as split 0 of the partials (other splits 0).  Solid cells give zeros.
template <typename T>
__global__ void __launch_bounds__(256) k_partials(Grid2D g, int S, const T *f, T *part,
                                                  const int8_t *type, int *err)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long nc = (long)g.nx * g.ny;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= nc) return;
    Acc<T> s0, s1, s2, s3;
    for (int p = lane; p < g.nv; p += 32) {
        const T vx = T(g.vxmin + (p % g.nvx) * g.dvx), vy = T(g.vymin + (p / g.nvx) * g.dvy);
        const T fv = f[didx<T>(g, cell, 0, p)];
        s0.add(fv); s1.add(vx * fv); s2.add(vy * fv);
        s3.add(T(0.5) * (vx * vx + vy * vy) * fv);
        s3.add(f[didx<T>(g, cell, 1, p)]);
    }
    s0.warp_reduce(); s1.warp_reduce(); s2.warp_reduce(); s3.warp_reduce();
    if (lane == 0) {
        const bool keep = type[cell] != DVM_SOLID;
        if (keep) {
            T rho, ux, uy, tmp;
            if (!primitives<T>(g.dv, s0.value(), s1.value(), s2.value(), s3.value(), rho, ux, uy, tmp))
                atomicExch(&err[kErrNonphys], 1);
        }
        write_member_partials<T>(part, S, nc, cell, keep, s0.value(), s1.value(), s2.value(), s3.value());
    }
}

// FP64 moments for output: rho, ux, uy, uz(=0), T per cell.
template <typename T>
__global__ void __launch_bounds__(256) k_moments_out(Grid2D g, const T *f, double *out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= (long)g.nx * g.ny) return;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int p = lane; p < g.nv; p += 32) {
        const double vx = g.vxmin + (p % g.nvx) * g.dvx, vy = g.vymin + (p / g.nvx) * g.dvy;
        const double fv = (double)f[didx<T>(g, cell, 0, p)];
        s0 += fv; s1 += vx * fv; s2 += vy * fv;
        s3 += 0.5 * (vx * vx + vy * vy) * fv + (double)f[didx<T>(g, cell, 1, p)];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o); s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o); s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    if (lane == 0) {
        double *o5 = out + cell * 5;
        const double rho = s0 * g.dv;
        if (!(rho > 0)) { for (int q = 0; q < 5; ++q) o5[q] = 0; return; }
        const double ux = s1 * g.dv / rho, uy = s2 * g.dv / rho;
        o5[0] = rho; o5[1] = ux; o5[2] = uy; o5[3] = 0;
        o5[4] = (2.0 * (s3 * g.dv) / rho - (ux * ux + uy * uy)) / 3.0;
    }
}

// Maxwellian state from per-cell primitives (rho, ux, uy, uz, T); solid
// cells get 0 (Eq. BGKDD for g).
template <typename T>
__global__ void k_init(Grid2D g, const double *prim, const int8_t *type, T *f)
{
    const long nc = (long)g.nx * g.ny;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * g.nv) return;
    const long k = t / g.nv;
    const int p = (int)(t % g.nv);
    const double *q = prim + 5 * k;
    double m = 0;
    if (type[k] != DVM_SOLID && q[0] > 0) {
        const double ax = g.vxmin + (p % g.nvx) * g.dvx - q[1];
        const double ay = g.vymin + (p / g.nvx) * g.dvy - q[2];
        m = q[0] / (2.0 * kPi * q[4]) * exp(-(ax * ax + ay * ay) / (2.0 * q[4]));
    }
    f[didx<T>(g, k, 0, p)] = (T)m;
    f[didx<T>(g, k, 1, p)] = (T)(q[4] / 2.0 * m);
}

// Ghost cells of a Maxwellian side from (rho, ux, uy, uz, T) per side cell,
// written into both state buffers.
template <typename T>
__global__ void k_ghost(Grid2D g, const double *prim, int side, int nside, T *f0, T *f1)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nside * g.nv) return;
    const long q = t / g.nv;
    const int p = (int)(t % g.nv);
    const double *s = prim + 5 * q;
    const double ax = g.vxmin + (p % g.nvx) * g.dvx - s[1];
    const double ay = g.vymin + (p / g.nvx) * g.dvy - s[2];
    const double m = s[0] / (2.0 * kPi * s[4]) * exp(-(ax * ax + ay * ay) / (2.0 * s[4]));
    const long cell = (long)g.nx * g.ny + g.gofs[side] + q;
    f0[didx<T>(g, cell, 0, p)] = (T)m;
    f0[didx<T>(g, cell, 1, p)] = (T)(s[4] / 2.0 * m);
    f1[didx<T>(g, cell, 0, p)] = (T)m;
    f1[didx<T>(g, cell, 1, p)] = (T)(s[4] / 2.0 * m);
}

// Conversion between the public layout [cell][comp][p] and the device layout.
template <typename T>
__global__ void k_pack(Grid2D g, const T *src, T *dst, int to_dev)
{
    const long nc = (long)g.nx * g.ny;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * 2 * g.nv) return;
    const long k = t / (2L * g.nv);
    const int comp = (int)((t / g.nv) % 2), p = (int)(t % g.nv);
    const long d = didx<T>(g, k, comp, p);
    if (to_dev) dst[d] = src[t];
    else dst[t] = src[d];
}

// Zero the state of every solid cell (they belong to no control volume).
template <typename T>
__global__ void k_zero_solid(Grid2D g, const int8_t *type, T *f)
{
    const long nc = (long)g.nx * g.ny;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * 2 * g.nvp) return;
    const long k = t % nc;
    if (type[k] != DVM_SOLID) return;
    const long rest = t / nc;
    const int comp = (int)(rest % 2), p = (int)(rest / 2);
    f[didx<T>(g, k, comp, p)] = T(0);
}

// Per-cell mass sbar * sum_p f dv (FP64), then a fixed-order sum.
template <typename T>
__global__ void __launch_bounds__(256) k_mass_cells(Grid2D g, const T *f, const double *sbar, double *cm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= (long)g.nx * g.ny) return;
    double s = 0;
    for (int p = lane; p < g.nv; p += 32) s += (double)f[didx<T>(g, cell, 0, p)];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) cm[cell] = sbar[cell] * (s * g.dv);
}

__global__ void __launch_bounds__(1024) k_sum(const double *x, long n, double *out)
{
    __shared__ double red[32];
    double s = 0;
    for (long t = threadIdx.x; t < n; t += blockDim.x) s += x[t];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

// Per-velocity coefficients and per-group sign of the velocity components.
template <typename T>
__global__ void k_tables(Grid2D g, VCoef<T> *vt, int8_t *gsign)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int W = Vec<T>::W;
    if (p < g.nvp) {
        VCoef<T> c;
        if (p < g.nv) {
            const T vx = T(g.vxmin + (p % g.nvx) * g.dvx), vy = T(g.vymin + (p / g.nvx) * g.dvy);
            c.vx = vx; c.vy = vy;
            c.nux = fabs(vx) * T(g.dt / g.dx);
            c.nuy = fabs(vy) * T(g.dt / g.dy);
        } else {
            c.vx = T(1e4); c.vy = T(1e4); c.nux = 0; c.nuy = 0;
        }
        vt[p] = c;
    }
    if (p < g.ngrp) {
        bool xp = true, xn = true, yp = true, yn = true;
        for (int e = 0; e < W; ++e) {
            const int q = p * W + e;
            if (q >= g.nv) continue;
            const T vx = T(g.vxmin + (q % g.nvx) * g.dvx), vy = T(g.vymin + (q / g.nvx) * g.dvy);
            xp = xp && vx >= T(0); xn = xn && vx <= T(0);
            yp = yp && vy >= T(0); yn = yn && vy <= T(0);
        }
        gsign[2 * p] = xp ? 1 : (xn ? -1 : 0);
        gsign[2 * p + 1] = yp ? 1 : (yn ? -1 : 0);
    }
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

template <typename T, bool MUSCL>
cudaError_t launch_bulk(dvm_ctx *c, const BulkArgs<T> &a)
{
    const size_t smem = (size_t)kStages * kStageBytes + kStages * sizeof(uint64_t);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_bulk<T, MUSCL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(nblk(c->nx, 32), nblk(c->ny, kRows), c->S), block(32, kRows);
    k_bulk<T, MUSCL><<<grid, block, smem, c->stream>>>(a, c->tmap[c->cur]);
    return cudaGetLastError();
}

template <typename T>
cudaError_t step2d_t(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    BodyParams bp = body_params(c);
    const bool body = c->body.shape != DVM_SHAPE_NONE;
    const bool moving = c->moving;
    T *fin = (T *)c->f[c->cur], *fout = (T *)c->f[1 - c->cur];
    T *pin = (T *)c->part[c->cur], *pout = (T *)c->part[1 - c->cur];
    cudaError_t e = cudaSuccess;
    if (moving) {
        k_advance<<<1, 32, 0, c->stream>>>(c->d_body, c->dt, 1);
        if ((e = geometry2d_level(c, 1 - c->gcur, body_trig(c, 2))) != cudaSuccess) return e;
        if ((e = masters_flags2d(c, true)) != cudaSuccess) return e;
        c->launches += 8;
    }
    CvArgs cv;
    cv.g = g;
    cv.Gn = c->geo[c->gcur];
    cv.Gp = moving ? c->geo[1 - c->gcur] : c->geo[c->gcur];
    cv.master = c->master; cv.flags = c->flags;
    cv.spec_list = c->spec_list; cv.wall_list = c->wall_list; cv.wslot = c->wslot;
    cv.counts = c->counts; cv.cap = c->list_cap; cv.S = c->S;
    cv.err = c->d_err;
    const int cvgrid = 2 * 152;
    if (body) {
        if (moving || c->need_fusion) {
            k_fusion<T><<<cvgrid, 256, 0, c->stream>>>(cv, fin, pin);
            c->launches += 1;
        }
        k_wall<T><<<cvgrid, 256, 0, c->stream>>>(cv, bp, c->d_body, fin, (T *)c->wflux, c->wphi,
                                                  c->wcontrib, c->ticket, c->d_hist, moving ? 1 : 0);
        c->launches += 1;
    }
    BulkArgs<T> a;
    a.g = g; a.S = c->S; a.fin = fin; a.fout = fout; a.pin = pin; a.pout = pout;
    a.flags = c->flags; a.vt = (const VCoef<T> *)c->vtab; a.gsign = c->gsign; a.err = c->d_err;
    if ((e = timing_mark(c, 0)) != cudaSuccess) return e;
    e = c->scheme == DVM_MUSCL ? launch_bulk<T, true>(c, a) : launch_bulk<T, false>(c, a);
    if (e != cudaSuccess) return e;
    if ((e = timing_mark(c, 1)) != cudaSuccess) return e;
    c->launches += 1;
    if (body) {
        k_special<T><<<cvgrid, 256, 0, c->stream>>>(cv, fin, fout, pin, pout, (const T *)c->wflux);
        c->launches += 1;
    }
    c->cur = 1 - c->cur;
    if (moving) c->gcur = 1 - c->gcur;
    c->need_fusion = false;
    c->steps_done++;
    return cudaGetLastError();
}

}  // namespace

// TMA descriptors of the two state buffers: a 3D view (x: cells of a row
// times the W velocities of a group, y: rows, z: group and component) of
// the interior cells of each slab; the box is the bulk kernel's tile.
int make_tensor_maps2d(dvm_ctx *c)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return DVM_ERR_CUDA;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const int W = c->W;
    const cuuint64_t dims[3] = {(cuuint64_t)c->nx * W, (cuuint64_t)c->ny, (cuuint64_t)2 * c->ngrp};
    const cuuint64_t strides[2] = {(cuuint64_t)c->nx * W * c->elem, (cuuint64_t)c->slab * W * c->elem};
    const cuuint32_t box[3] = {(cuuint32_t)kTileX * W, (cuuint32_t)kTileY, 2};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = c->prec == DVM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    for (int b = 0; b < 2; ++b) {
        CUresult r = encode(&c->tmap[b], dt, 3, c->f[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
            return DVM_ERR_CUDA;
        }
    }
    return DVM_OK;
}

size_t vcoef_bytes(int prec) { return prec == DVM_FP32 ? sizeof(VCoef<float>) : sizeof(VCoef<double>); }

cudaError_t step2d(dvm_ctx *c)
{
    return c->prec == DVM_FP32 ? step2d_t<float>(c) : step2d_t<double>(c);
}

cudaError_t tables2d(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    const int n = c->nvp > c->ngrp ? c->nvp : c->ngrp;
    if (c->prec == DVM_FP32)
        k_tables<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, (VCoef<float> *)c->vtab, c->gsign);
    else
        k_tables<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, (VCoef<double> *)c->vtab, c->gsign);
    return cudaGetLastError();
}

cudaError_t partials_from_state2d(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    const long nc = (long)c->nx * c->ny;
    if (c->prec == DVM_FP32)
        k_partials<float><<<nblk(nc, 8), 256, 0, c->stream>>>(g, c->S, (const float *)c->f[c->cur],
                                                              (float *)c->part[c->cur], c->geo[c->gcur].type, c->d_err);
    else
        k_partials<double><<<nblk(nc, 8), 256, 0, c->stream>>>(g, c->S, (const double *)c->f[c->cur],
                                                               (double *)c->part[c->cur], c->geo[c->gcur].type, c->d_err);
    return cudaGetLastError();
}

cudaError_t moments_out2d(dvm_ctx *c, double *d_out)
{
    Grid2D g = grid2d(c);
    const long nc = (long)c->nx * c->ny;
    if (c->prec == DVM_FP32)
        k_moments_out<float><<<nblk(nc, 8), 256, 0, c->stream>>>(g, (const float *)c->f[c->cur], d_out);
    else
        k_moments_out<double><<<nblk(nc, 8), 256, 0, c->stream>>>(g, (const double *)c->f[c->cur], d_out);
    return cudaGetLastError();
}

cudaError_t init_maxwellian2d(dvm_ctx *c, const double *d_prim)
{
    Grid2D g = grid2d(c);
    const long n = (long)c->nx * c->ny * c->nv;
    if (c->prec == DVM_FP32)
        k_init<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, d_prim, c->geo[c->gcur].type, (float *)c->f[c->cur]);
    else
        k_init<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, d_prim, c->geo[c->gcur].type, (double *)c->f[c->cur]);
    return cudaGetLastError();
}

cudaError_t ghost2d(dvm_ctx *c, int side, const double *d_prim, int nside)
{
    Grid2D g = grid2d(c);
    const long n = (long)nside * c->nv;
    if (c->prec == DVM_FP32)
        k_ghost<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, d_prim, side, nside, (float *)c->f[0], (float *)c->f[1]);
    else
        k_ghost<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, d_prim, side, nside, (double *)c->f[0], (double *)c->f[1]);
    return cudaGetLastError();
}

cudaError_t pack2d(dvm_ctx *c, const void *pub, void *dev)
{
    Grid2D g = grid2d(c);
    const long n = (long)c->nx * c->ny * 2 * c->nv;
    if (c->prec == DVM_FP32)
        k_pack<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, (const float *)pub, (float *)dev, 1);
    else
        k_pack<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, (const double *)pub, (double *)dev, 1);
    return cudaGetLastError();
}

cudaError_t zero_solid2d(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    const long n = (long)c->nx * c->ny * 2 * c->nvp;
    for (int b = 0; b < 2; ++b) {
        if (c->prec == DVM_FP32)
            k_zero_solid<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, c->geo[c->gcur].type, (float *)c->f[b]);
        else
            k_zero_solid<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, c->geo[c->gcur].type, (double *)c->f[b]);
    }
    return cudaGetLastError();
}

cudaError_t unpack2d(dvm_ctx *c, const void *dev, void *pub)
{
    Grid2D g = grid2d(c);
    const long n = (long)c->nx * c->ny * 2 * c->nv;
    if (c->prec == DVM_FP32)
        k_pack<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, (const float *)dev, (float *)pub, 0);
    else
        k_pack<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, (const double *)dev, (double *)pub, 0);
    return cudaGetLastError();
}

cudaError_t mass2d(dvm_ctx *c, double *d_scratch, double *d_out)
{
    Grid2D g = grid2d(c);
    const long nc = (long)c->nx * c->ny;
    // mass of the state at t^n with the areas of t^n (members of a control
    // volume hold its value, so this is Eq. def-masse)
    if (c->prec == DVM_FP32)
        k_mass_cells<float><<<nblk(nc, 8), 256, 0, c->stream>>>(g, (const float *)c->f[c->cur], c->geo[c->gcur].sbar, d_scratch);
    else
        k_mass_cells<double><<<nblk(nc, 8), 256, 0, c->stream>>>(g, (const double *)c->f[c->cur], c->geo[c->gcur].sbar, d_scratch);
    k_sum<<<1, 1024, 0, c->stream>>>(d_scratch, nc, d_out);
    return cudaGetLastError();
}

}  // namespace dvm
