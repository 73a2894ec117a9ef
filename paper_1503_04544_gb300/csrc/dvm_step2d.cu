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
#include <type_traits>

#include "dvm_device.cuh"

namespace dvm {
namespace {


// Primitive variables (Eq. MacroscopicDDv; T from E = rho|u|^2/2 + 3/2 rho T)
// from the reduced sums s0 = sum f, s1 = sum vx f, s2 = sum vy f,
// s3 = sum (|v|^2/2 f + g).

template <typename T>
__device__ __forceinline__ bool primitives(T dv, T s0, T s1, T s2, T s3, T &rho, T &ux, T &uy, T &tmp)
{
    rho = s0 * dv;
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


template <typename T> struct BulkArgs {
    Grid2D g;
    int S;
    int Sin;                  // partial-sum slots of pin (S, or 1 for summed moments of a velocity split)
    const T *fin;
    T *fout;
    const T *pin;             // partial moments of f^n   [S][4][nc]
    T *pout;                  // partial moments of f^n+1 [S][4][nc]
    const uint8_t *flags;
    const VCoef<T> *vt;       // [nvp]
    const ulonglong2 *pt;     // [ngrp][7] packed-pair coefficients (FP32 path)
    const int8_t *gsign;      // [ngrp][2]
    const T *eqp;             // [4][nc] conservative equilibrium parameters, or null (direct moments)
    const T *qh;              // [2][nc] heat flux of the control volume at t^n (Shakhov model), used when hin is null
    const T *hin;             // Shakhov: raw heat-flux moments of f^n [S][5][nc] and their reference velocity [2][nc]
    T *hout;                  // Shakhov: the same for f^n+1
    T pr1;                    // 1 - Pr (Shakhov model)
    uint32_t *bits;           // [ngrp][bslab] limiter branches of the downwind faces (recording only)
    int bpitch;               // row pitch of the branch words
    long bslab;               // branch words per group
    int *err;
};

// ------------------------------------------------------------ bulk kernel
constexpr int kStageBytes = 2 * kTileY * kTileX * 16;     // both components of one group


// Branch the limited reconstruction of a downwind face took (recorded for the
// discrete adjoint): 1 when minmod returned its first argument a (the
// downwind difference), 2 when it returned the second b (the upwind
// difference; also on a tie), 0 when it returned 0 or the face is first order.
template <typename T>
__device__ __forceinline__ uint32_t branch_bits(T m, T a, T b, T w)
{
    return (w == T(0) || m == T(0)) ? 0u : (m == b ? 2u : (m == a ? 1u : 0u));
}

// Update of one component of one velocity group for the thread's cell from
// the shared-memory tile (Eq. ExSchemeDD on a full gas cell, fluxes of Eq.
// FluxDD in difference form with the limited reconstruction), moment sums.
// c0 is the tile index of the cell; ux1/uy1 the tile offsets of one cell step
// towards the upwind side along x/y (sign-uniform groups), else per element.
// With REC the branches of the two downwind faces are or-ed into bw at bit
// ((COMP * 2 + axis) * W + e) * 2.
template <typename T, bool MUSCL, int COMP, bool UNIFORM, bool REC>
__device__ __forceinline__ void bulk_tile(const typename Vec<T>::type *t, int c0, int ux1, int uy1,
                                          const T (&vx)[Vec<T>::W], const T (&vy)[Vec<T>::W],
                                          const T (&nux)[Vec<T>::W], const T (&nuy)[Vec<T>::W],
                                          const T (&feq)[Vec<T>::W], T wxm, T wxp, T wym, T wyp, T r,
                                          T (&out)[Vec<T>::W], T &q0, T &q1, T &q2, T &q3, uint32_t &bw)
{
    constexpr int W = Vec<T>::W;
    T f[W];
    sld<T>(t + c0, f);
    if (UNIFORM) {
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
                const T bx = d1[e] - f[e], by = e1[e] - f[e], cx = u1[e] - u2[e], cy = w1[e] - w2[e];
                const T mxo = minmod3(bx, ax), myo = minmod3(by, ay), mxi = minmod3(ax, cx), myi = minmod3(ay, cy);
                dfx += (T(1) - nux[e]) * (cxo * mxo - cxi * mxi);
                dfy += (T(1) - nuy[e]) * (cyo * myo - cyi * myi);
                if (REC) {
                    bw |= branch_bits(mxo, bx, ax, cxo) << (((COMP * 2 + 0) * W + e) * 2);
                    bw |= branch_bits(myo, by, ay, cyo) << (((COMP * 2 + 1) * W + e) * 2);
                }
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
                const T bx = d1 - f[e], by = e1 - f[e], cx = u1 - u2, cy = w1 - w2;
                const T mxo = minmod3(bx, ax), myo = minmod3(by, ay), mxi = minmod3(ax, cx), myi = minmod3(ay, cy);
                dfx += (T(1) - nux[e]) * (cxo * mxo - cxi * mxi);
                dfy += (T(1) - nuy[e]) * (cyo * myo - cyi * myi);
                if (REC) {
                    bw |= branch_bits(mxo, bx, ax, cxo) << (((COMP * 2 + 0) * W + e) * 2);
                    bw |= branch_bits(myo, by, ay, cyo) << (((COMP * 2 + 1) * W + e) * 2);
                }
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

// Packed FP32 form of bulk_tile for a sign-uniform group with the limited
// reconstruction: the differences, the flux combination, the update and the
// moment sums on pairs of velocities with the f32x2 instructions (the minmod
// min/max stay scalar).  Same formulas as bulk_tile; the moment sums go to
// per-lane accumulators Q (q0, q1, q2, q3 of bulk_tile).  P: per-element
// coefficient pairs -nux, -nuy, 1 - nux, 1 - nuy, vx, vy, |v|^2/2.
struct PairCoef { F2 nnx[2], nny[2], onx[2], ony[2], vx[2], vy[2], ke[2]; };

// Branch code of a minmod value of magnitude m (b: its second argument): 0
// for zero, 2 for b (also on a tie), else 1.
__device__ __forceinline__ uint32_t bcode(float m, float b) { return m == 0.f ? 0u : (m == fabsf(b) ? 2u : 1u); }

template <int COMP, bool REC>
__device__ __forceinline__ void bulk_tile_x2(const float4 *t, int c0, int ux1, int uy1, const PairCoef &P,
                                             const F2 (&feq)[2], float wxm, float wxp, float wym, float wyp, F2 r,
                                             float (&out)[4], F2 (&Q)[4], uint32_t &bw)
{
    float f[4], u1[4], w1[4], d1[4], u2[4], e1[4], w2[4];
    sld<float>(t + c0, f);
    sld<float>(t + c0 - ux1, u1);
    sld<float>(t + c0 - uy1, w1);
    sld<float>(t + c0 + ux1, d1);
    sld<float>(t + c0 - 2 * ux1, u2);
    sld<float>(t + c0 + uy1, e1);
    sld<float>(t + c0 - 2 * uy1, w2);
    const bool px = ux1 > 0, py = uy1 > 0;
    const float cxo = px ? wxp : wxm, cxi = px ? wxm : wxp;
    const float cyo = py ? wyp : wym, cyi = py ? wym : wyp;
    const F2 CXO = f2(cxo), NCXI = f2(-cxi), CYO = f2(cyo), NCYI = f2(-cyi);
    uint32_t lo = 0;                  // branch codes before the face-weight masks
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int a0 = 2 * h, a1 = 2 * h + 1;
        const F2 F = f2(f[a0], f[a1]), U1 = f2(u1[a0], u1[a1]), W1 = f2(w1[a0], w1[a1]);
        const F2 AX = sub2(F, U1), AY = sub2(F, W1);
        const F2 BX = sub2(f2(d1[a0], d1[a1]), F), BY = sub2(f2(e1[a0], e1[a1]), F);
        const F2 CX = sub2(U1, f2(u2[a0], u2[a1])), CY = sub2(W1, f2(w2[a0], w2[a1]));
        // the limited terms cxo mo - cxi mi from the magnitudes of the two
        // limiter values, which (where not zero) share the sign of a: the same
        // numbers as from the signed values, in fewer scalar min/max
        float ax[2], ay[2], bx[2], by[2], cx[2], cy[2], mxo[2], mxi[2], myo[2], myi[2];
        f2_get(AX, ax[0], ax[1]); f2_get(AY, ay[0], ay[1]);
        f2_get(BX, bx[0], bx[1]); f2_get(BY, by[0], by[1]);
        f2_get(CX, cx[0], cx[1]); f2_get(CY, cy[0], cy[1]);
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            minmod_mag_pair(bx[l], ax[l], cx[l], mxo[l], mxi[l]);
            minmod_mag_pair(by[l], ay[l], cy[l], myo[l], myi[l]);
            if (REC) {
                const int e = 2 * h + l;
                lo |= bcode(mxo[l], ax[l]) << (((COMP * 2 + 0) * 4 + e) * 2);
                lo |= bcode(myo[l], ay[l]) << (((COMP * 2 + 1) * 4 + e) * 2);
            }
        }
        float tx[2], ty[2];
        f2_get(fma2(NCXI, f2(mxi[0], mxi[1]), mul2(CXO, f2(mxo[0], mxo[1]))), tx[0], tx[1]);
        f2_get(fma2(NCYI, f2(myi[0], myi[1]), mul2(CYO, f2(myo[0], myo[1]))), ty[0], ty[1]);
        const F2 TX = f2(xorsign(tx[0], ax[0]), xorsign(tx[1], ax[1]));
        const F2 TY = f2(xorsign(ty[0], ay[0]), xorsign(ty[1], ay[1]));
        const F2 DFX = fma2(P.onx[h], TX, AX), DFY = fma2(P.ony[h], TY, AY);
        F2 O = fma2(P.nnx[h], DFX, F);
        O = fma2(P.nny[h], DFY, O);
        O = fma2(r, sub2(feq[h], F), O);
        f2_get(O, out[a0], out[a1]);
        if (COMP == 0) {
            Q[0] = add2(Q[0], O);
            Q[1] = fma2(P.vx[h], O, Q[1]);
            Q[2] = fma2(P.vy[h], O, Q[2]);
            Q[3] = fma2(P.ke[h], O, Q[3]);
        } else {
            Q[3] = add2(Q[3], O);
        }
    }
    if (REC) {
        // first-order faces record no branch: x fields 0x00FF00FF, y fields 0xFF00FF00
        const uint32_t mo = (cxo != 0.f ? 0x00FF00FFu : 0u) | (cyo != 0.f ? 0xFF00FF00u : 0u);
        bw |= lo & mo;
    }
}

// Adds the two lanes of each packed moment sum to q0..q3 and clears them.
template <typename T>
__device__ __forceinline__ void fold_pairs(F2 (&Q)[4], T &q0, T &q1, T &q2, T &q3)
{
    float a, b;
    f2_get(Q[0], a, b); q0 += a + b;
    f2_get(Q[1], a, b); q1 += a + b;
    f2_get(Q[2], a, b); q2 += a + b;
    f2_get(Q[3], a, b); q3 += a + b;
#pragma unroll
    for (int m = 0; m < 4; ++m) Q[m] = f2(0.f);
}

// Compensated sums of the FP32 Shakhov variant of the bulk kernel, kept in
// shared memory (rows [m][sum, compensation], one column per thread) to
// leave the registers to the update: the four moments and the five raw
// heat-flux moments.
constexpr int kSaccRows = 9;
constexpr size_t kSaccBytes = (size_t)kSaccRows * 2 * 32 * kRows * sizeof(float);

__device__ __forceinline__ void sacc_add(float *sa, int m, int tid, float x)
{
    constexpr int N = 32 * kRows;
    Acc<float> a;
    a.s = sa[(2 * m) * N + tid];
    a.c = sa[(2 * m + 1) * N + tid];
    a.add(x);
    sa[(2 * m) * N + tid] = a.s;
    sa[(2 * m + 1) * N + tid] = a.c;
}

__device__ __forceinline__ float sacc_value(const float *sa, int m, int tid)
{
    constexpr int N = 32 * kRows;
    Acc<float> a;
    a.s = sa[(2 * m) * N + tid];
    a.c = sa[(2 * m + 1) * N + tid];
    return a.value();
}

// Adds both lanes of the per-lane sums Q (n of them) to the shared
// compensated sums from row m0 on and clears them.
template <int n>
__device__ __forceinline__ void fold_lanes(F2 (&Q)[n], int m0, float *sa, int tid)
{
#pragma unroll
    for (int m = 0; m < n; ++m) {
        float a, b;
        f2_get(Q[m], a, b);
        sacc_add(sa, m0 + m, tid, a + b);
        Q[m] = f2(0.f);
    }
}

// Compile-time choice between two variables.
template <bool A, typename T>
__device__ __forceinline__ T &sel(T &a, T &b)
{
    if constexpr (A) return a; else return b;
}

// Raw heat-flux moments (Shakhov model) of one component of a pair of
// velocities about the origin, from the velocity table only: component 0
// (f) adds vx ke f, vy ke f, vx^2 f, vx vy f, vy^2 f to H[0..4] (ke =
// |v|^2/2), component 1 (g) adds vx g, vy g to H[0], H[1].  With the
// moments of the cell, its heat flux about its own velocity u is
//   q = H_(x,y) - u.P_(.,x|y) - u E + rho u |u|^2
// (P the second moments, E = sum (ke f + g)); the same identity holds about
// any reference velocity u_r with u - u_r in place of u.
template <int COMP>
__device__ __forceinline__ void hmom_x2(F2 O, F2 VX, F2 VY, F2 KE, F2 (&H)[5])
{
    if (COMP == 0) {
        const F2 TX = mul2(VX, O), TY = mul2(VY, O);
        H[2] = fma2(VX, TX, H[2]);
        H[3] = fma2(VY, TX, H[3]);
        H[4] = fma2(VY, TY, H[4]);
        H[0] = fma2(KE, TX, H[0]);
        H[1] = fma2(KE, TY, H[1]);
    } else {
        H[0] = fma2(VX, O, H[0]);
        H[1] = fma2(VY, O, H[1]);
    }
}

// The same over one FP32 velocity group (values o at velocities vx, vy).
template <int COMP>
__device__ __forceinline__ void hmom_group(const float (&o)[4], const float (&vx)[4], const float (&vy)[4],
                                           F2 (&H)[5])
{
#pragma unroll
    for (int e = 0; e < 4; e += 2) {
        const F2 VX = f2(vx[e], vx[e + 1]), VY = f2(vy[e], vy[e + 1]);
        const F2 KE = mul2(f2(0.5f), fma2(VX, VX, mul2(VY, VY)));
        hmom_x2<COMP>(f2(o[e], o[e + 1]), VX, VY, KE, H);
    }
}

// Store of one (group, component) vector of a cell and of its padding
// mirrors (cells within two cells of a periodic or zero-gradient side).
template <typename T>
__device__ __forceinline__ void store_cell(typename Vec<T>::type *slab, int pc, const int (&mir)[4], bool anymir,
                                           const T (&v)[Vec<T>::W])
{
    vst<T>(slab + pc, v);
    if (anymir) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (mir[k] >= 0) vst<T>(slab + mir[k], v);
    }
}

// Bulk update.  Block = 32 x kRows cells; the velocity groups of split
// blockIdx.z stream through a kStages-deep ring of shared-memory tiles
// (the block's cells plus a two-cell halo, both components of one group),
// each filled by one TMA tensor load that completes on the stage's "full"
// mbarrier; each warp releases a stage on its "empty" mbarrier once it has
// read it, and thread 0 refills a stage only after all warps released it.
// Every wait is bounded: on timeout the kernel records kErrTimeout and goes
// on without blocking.  Threads of non-plain cells only take part in the
// barriers.
// With REC (recomputation for the discrete adjoint) each plain cell also
// writes the limiter branches of its downwind faces, one word per group at
// its padded index (row pitch bpitch).
// With SHAK (the Shakhov model, Eq. ShakhovDD, explicit scheme) the cell
// relaxes towards f_S = M [1 + k c.q (|c|^2/T - 4)], g_S = T/2 M [1 + k c.q
// (|c|^2/T - 2)], k = (1 - Pr) / (5 rho T^2), with the heat flux q of the
// cell at t^n: from the raw moments of f^n that the previous step left in
// hin (shifted to the cell's velocity, see hmom_x2), or from k_heatflux when
// hin is null.  The FP32 variant leaves the raw moments of f^{n+1} about the
// origin in hout for the next step.
template <typename T, bool MUSCL, bool REC, bool SHAK>
__global__ void __launch_bounds__(32 * kRows, 2) k_bulk(BulkArgs<T> a, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int W = Vec<T>::W;
    // raw heat-flux moments of the new state (FP32 only: an FP64 step is
    // bound by the FP64 pipe, where one more read of f^n by k_heatflux costs
    // less than these sums)
    constexpr bool HRAW = SHAK && sizeof(T) == 4;
    using V = typename Vec<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    V *ring = reinterpret_cast<V *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    const Grid2D &g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * kRows;
    const int i = i0 + tx, j = j0 + ty;
    const bool inside = i < g.nx && j < g.ny;
    const long nc = (long)g.nx * g.ny;
    const long cell = inside ? (long)j * g.nx + i : 0;
    const int pc = (int)nbr(g, i, j);
    const int split = blockIdx.z;
    const int gps = (g.ngrp + a.S - 1) / a.S;
    const int g0 = split * gps, g1 = min(g0 + gps, g.ngrp);
    const int ngr = max(g1 - g0, 0);
    const uint8_t fl = inside ? a.flags[cell] : 0;
    const bool plain = (fl & kPlain) != 0, zero = (fl & kZero) != 0;
    V *fout = reinterpret_cast<V *>(a.fout);

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], kRows);
        }
        mbar_fence_init();
        for (int st = 0; st < kStages - 1 && st < ngr; ++st) {
            mbar_expect_tx(&full[st], kStageBytes);
            tma_load_3d(ring + (long)st * (kStageBytes / 16), &tmap, &full[st], i0 * W, j0, (g0 + st) * 2);
        }
    }

    // equilibrium of the cell at t^n
    T A = 0, c2 = 0, r = 0, gfac = 0, ux = 0, uy = 0, el0 = 0, e1x = 0, e1y = 0;
    T kqx = 0, kqy = 0, iT = 0, l2a4 = 0, nkuq = 0;  // Shakhov: k q_x, k q_y, 1/T, 2 log2(A)/log2(e) - 4, -k u.q
    if (plain) {
        T s[4];
        gather_partials(a.pin, a.Sin, nc, cell, s);
        T rho, tmp;
        if (!primitives<T>(pick<T>(g.dv_f, g.dv), s[0], s[1], s[2], s[3], rho, ux, uy, tmp))
            atomicExch(&a.err[kErrNonphys], 1);
        r = pick<T>(g.dt_tau0_f, g.dt_tau0) * rho;
        if (a.eqp) {
            // conservative equilibrium (Sec. 3.1): tau from the direct
            // density, the Maxwellian from the Newton parameters
            rho = a.eqp[cell]; ux = a.eqp[nc + cell]; uy = a.eqp[2 * nc + cell]; tmp = a.eqp[3 * nc + cell];
        }
        A = rho / (T(2.0 * kPi) * tmp);
        c2 = T(kLog2e) / (T(2) * tmp);
        gfac = tmp / T(2);
        if constexpr (SHAK) {
            T qx = 0, qy = 0;
            if (HRAW && a.hin) {
                // heat flux at t^n from the raw moments of f^n that the
                // previous step wrote, about their reference velocity u_r
                // (the origin, or the control volume's velocity at t^{n-1}
                // for cells that k_special wrote): w = u - u_r and
                // E' = sum (|v - u_r|^2/2 f + g)
                Acc<T> h[5];
                for (int sp = 0; sp < a.S; ++sp)
#pragma unroll
                    for (int m = 0; m < 5; ++m) h[m].merge(a.hin[((long)sp * 5 + m) * nc + cell], T(0));
                const long ur = (long)a.S * 5 * nc + cell;
                const T urx = a.hin[ur], ury = a.hin[ur + nc];
                const T wx = ux - urx, wy = uy - ury;
                const T e1 = s[3] - urx * s[1] - ury * s[2] + T(0.5) * (urx * urx + ury * ury) * s[0];
                const T rw2 = s[0] * (wx * wx + wy * wy);
                const T dv = pick<T>(g.dv_f, g.dv);
                qx = dv * (h[0].value() - wx * h[2].value() - wy * h[3].value() - wx * e1 + wx * rw2);
                qy = dv * (h[1].value() - wx * h[3].value() - wy * h[4].value() - wy * e1 + wy * rw2);
            } else {
                qx = a.qh[cell];
                qy = a.qh[nc + cell];
            }
            const T k = a.pr1 / (T(5) * rho * tmp * tmp);
            kqx = k * qx;
            kqy = k * qy;
            iT = T(1) / tmp;
            l2a4 = T(2.0 / kLog2e) * log2(A) - T(4);
            nkuq = -(kqx * ux + kqy * uy);
        }
        // log2 M(v) = el0 + e1x vx + e1y vy - c2 |v|^2 (packed path)
        el0 = log2(A) - c2 * (ux * ux + uy * uy);
        e1x = T(2) * c2 * ux;
        e1y = T(2) * c2 * uy;
    }
    const int mask = fl >> kMaskShift;
    // limiter weights of the faces x-, x+, y-, y+ (1/2 where the limited
    // reconstruction is allowed, 0 where the flux falls back to first order)
    const T wxm = (mask & 1) ? T(0.5) : T(0), wxp = (mask & 2) ? T(0.5) : T(0);
    const T wym = (mask & 4) ? T(0.5) : T(0), wyp = (mask & 8) ? T(0.5) : T(0);
    const int c0 = (ty + 2) * kTileX + tx + 2;
    int mir[4];               // padded indices fit in 32 bits (checked at context creation)
    mirrors(g, i, j, mir);
    const bool anymir = __any_sync(0xffffffffu, inside && (mir[0] >= 0 || mir[2] >= 0));
    __syncthreads();

    // FP64: the Maxwellian along a row of the uniform v_x grid by the
    // recurrence M(v + dv) = M(v) R(v), R(v + dv) = R(v) Qm with
    // Qm = 2^(-2 c2 dv^2), restarted from a direct evaluation every 8
    // velocities and at every row start (relative error below 30 ulp)
    T Mrun = 0, Rrun = 0, Qm = 0;
    const bool mrec = sizeof(T) == 8 && g.nvx % W == 0;
    if (sizeof(T) == 8 && plain) Qm = dexp2(T(-2) * c2 * T(g.dvx) * T(g.dvx));
    // the exponent's per-cell terms as pairs (packed path)
    F2 EL0, E1X, E1Y, NC2;
    if constexpr (sizeof(T) == 4 && MUSCL) {
        EL0 = f2(el0); E1X = f2(e1x); E1Y = f2(e1y); NC2 = f2(-2.f * c2);
    }
    Acc<T> m0, m1, m2, m3;
    T q0 = 0, q1 = 0, q2 = 0, q3 = 0;
    F2 Qp[4];                 // per-lane sums of the packed FP32 path
#pragma unroll
    for (int m = 0; m < 4; ++m) Qp[m] = f2(0.f);
    // FP32 Shakhov: raw heat-flux moments of f^{n+1} about the origin, per
    // lane over 16 groups, then (with the four moments) into the shared
    // compensated sums
    F2 Hp[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) Hp[m] = f2(0.f);
    float *sacc = reinterpret_cast<float *>(smem + kStages * kStageBytes + 2 * kStages * sizeof(uint64_t));
    if constexpr (HRAW) {
#pragma unroll
        for (int m = 0; m < 2 * kSaccRows; ++m) sacc[m * 32 * kRows + tid] = 0;
    }
    int fold = 0;
    for (int it = 0; it < ngr; ++it) {
        const int q = g0 + it, st = it % kStages;
        if (tid == 0 && it + kStages - 1 < ngr) {
            const int k = it + kStages - 1, s2 = k % kStages;
            if (k >= kStages && !mbar_wait(&empty[s2], (uint32_t)((k / kStages - 1) & 1)))
                atomicExch(&a.err[kErrTimeout], 1);
            mbar_expect_tx(&full[s2], kStageBytes);
            tma_load_3d(ring + (long)s2 * (kStageBytes / 16), &tmap, &full[s2], i0 * W, j0, (g0 + k) * 2);
        }
        if (!mbar_wait(&full[st], (uint32_t)((it / kStages) & 1))) atomicExch(&a.err[kErrTimeout], 1);
        const V *tile = ring + (long)st * (kStageBytes / 16);
        V *o0 = fout + (long)q * 2 * g.slab;
        if (plain) {
            const int sx = a.gsign[2 * q], sy = a.gsign[2 * q + 1];
            T vx[W], vy[W], nux[W], nuy[W], feq[W], out[W];
            uint32_t bw = 0;
            // the FP32 Shakhov variant keeps every moment sum in the per-lane
            // pairs: the scalar path's sums of this group go there at its end
            T t0 = 0, t1 = 0, t2 = 0, t3 = 0;
            T &p0 = sel<HRAW>(t0, q0), &p1 = sel<HRAW>(t1, q1), &p2 = sel<HRAW>(t2, q2), &p3 = sel<HRAW>(t3, q3);
            if constexpr (sizeof(T) == 4 && MUSCL) {
                if (sx != 0 && sy != 0) {
                    // packed FP32 path of the sign-uniform groups, coefficients
                    // from the group's rows of the packed table
                    const int ux1 = sx > 0 ? 1 : -1, uy1 = sy > 0 ? kTileX : -kTileX;
                    PairCoef P;
                    {
                        const ulonglong2 *pt = a.pt + (long)q * 7;
                        F2 *rows[7] = {P.nnx, P.nny, P.onx, P.ony, P.vx, P.vy, P.ke};
#pragma unroll
                        for (int k = 0; k < 7; ++k) {
                            const ulonglong2 v = __ldg(pt + k);
                            rows[k][0].v = v.x;
                            rows[k][1].v = v.y;
                        }
                    }
                    F2 fq[2], fg[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        {
                            // log2 M = el0 - 2 c2 |v|^2/2 + e1x vx + e1y vy
                            F2 X = fma2(NC2, P.ke[h], EL0);
                            X = fma2(E1X, P.vx[h], X);
                            X = fma2(E1Y, P.vy[h], X);
                            float x0, x1;
                            f2_get(X, x0, x1);
                            fq[h] = f2(ex2_fast(x0), ex2_fast(x1));
                            if constexpr (SHAK) {
                                // |c|^2/T - 4 = 2 (log2 A - log2 M) / log2 e - 4,
                                // k c.q = kqx vx + kqy vy - (kqx ux + kqy uy);
                                // f_S = M + M k c.q (|c|^2/T - 4) and
                                // g_S = T/2 (f_S + 2 M k c.q)
                                const F2 D4 = fma2(f2(float(-2.0 / kLog2e)), X, f2(l2a4));
                                const F2 KCQ = fma2(P.vx[h], f2(kqx), fma2(P.vy[h], f2(kqy), f2(nkuq)));
                                const F2 MK = mul2(fq[h], KCQ);
                                fq[h] = fma2(MK, D4, fq[h]);
                                fg[h] = mul2(f2(gfac), fma2(MK, f2(2.f), fq[h]));
                            }
                        }
                    }
                    const F2 r2 = f2(r);
                    bulk_tile_x2<0, REC>(tile, c0, ux1, uy1, P, fq, wxm, wxp, wym, wyp, r2, out, Qp, bw);
                    store_cell<T>(o0, pc, mir, anymir, out);
                    if constexpr (SHAK) {
                        hmom_x2<0>(f2(out[0], out[1]), P.vx[0], P.vy[0], P.ke[0], Hp);
                        hmom_x2<0>(f2(out[2], out[3]), P.vx[1], P.vy[1], P.ke[1], Hp);
                    }
                    if constexpr (SHAK) {
                        fq[0] = fg[0]; fq[1] = fg[1];
                    } else {
                        const F2 gf = f2(gfac);
                        fq[0] = mul2(fq[0], gf); fq[1] = mul2(fq[1], gf);
                    }
                    bulk_tile_x2<1, REC>(tile + kTileY * kTileX, c0, ux1, uy1, P, fq, wxm, wxp, wym, wyp, r2, out,
                                         Qp, bw);
                    store_cell<T>(o0 + g.slab, pc, mir, anymir, out);
                    if constexpr (SHAK) {
                        hmom_x2<1>(f2(out[0], out[1]), P.vx[0], P.vy[0], P.ke[0], Hp);
                        hmom_x2<1>(f2(out[2], out[3]), P.vx[1], P.vy[1], P.ke[1], Hp);
                    }
                    goto stored;
                }
            }
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const VCoef<T> vc = ld_coef(a.vt + q * W + e);
                vx[e] = vc.vx; vy[e] = vc.vy; nux[e] = vc.nux; nuy[e] = vc.nuy;
            }
            if (sizeof(T) == 8 && mrec) {
                const int p0 = q * W;
                if (it % (8 / W) == 0 || p0 % g.nvx == 0) {
                    const T dx = vx[0] - ux, dy = vy[0] - uy;
                    Mrun = A * dexp2(-(dx * dx + dy * dy) * c2);
                    Rrun = dexp2(-c2 * (T(2) * dx * T(g.dvx) + T(g.dvx) * T(g.dvx)));
                }
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    feq[e] = Mrun;
                    Mrun *= Rrun;
                    Rrun *= Qm;
                }
            } else {
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    const T dx = vx[e] - ux, dy = vy[e] - uy;
                    feq[e] = A * dexp2(-(dx * dx + dy * dy) * c2);
                }
            }
            // Shakhov: the equilibria of f and g (the BGK g equilibrium T/2 M
            // is formed in place after the f update)
            T feqg[W];
            if constexpr (SHAK) {
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    const T dx = vx[e] - ux, dy = vy[e] - uy;
                    const T kcq = kqx * dx + kqy * dy, d2 = (dx * dx + dy * dy) * iT;
                    feqg[e] = gfac * feq[e] * fma(kcq, d2 - T(2), T(1));
                    feq[e] *= fma(kcq, d2 - T(4), T(1));
                }
            }
            if (sx != 0 && sy != 0) {
                const int ux1 = sx > 0 ? 1 : -1, uy1 = sy > 0 ? kTileX : -kTileX;
                bulk_tile<T, MUSCL, 0, true, REC>(tile, c0, ux1, uy1, vx, vy, nux, nuy, feq, wxm, wxp, wym, wyp, r,
                                                  out, p0, p1, p2, p3, bw);
                store_cell<T>(o0, pc, mir, anymir, out);
                if constexpr (HRAW) hmom_group<0>(out, vx, vy, Hp);
                if constexpr (!SHAK) {
#pragma unroll
                    for (int e = 0; e < W; ++e) feqg[e] = feq[e] * gfac;
                }
                bulk_tile<T, MUSCL, 1, true, REC>(tile + kTileY * kTileX, c0, ux1, uy1, vx, vy, nux, nuy, feqg, wxm,
                                                  wxp, wym, wyp, r, out, p0, p1, p2, p3, bw);
                store_cell<T>(o0 + g.slab, pc, mir, anymir, out);
                if constexpr (HRAW) hmom_group<1>(out, vx, vy, Hp);
            } else {
                bulk_tile<T, MUSCL, 0, false, REC>(tile, c0, 1, kTileX, vx, vy, nux, nuy, feq, wxm, wxp, wym, wyp, r,
                                                   out, p0, p1, p2, p3, bw);
                store_cell<T>(o0, pc, mir, anymir, out);
                if constexpr (HRAW) hmom_group<0>(out, vx, vy, Hp);
                if constexpr (!SHAK) {
#pragma unroll
                    for (int e = 0; e < W; ++e) feqg[e] = feq[e] * gfac;
                }
                bulk_tile<T, MUSCL, 1, false, REC>(tile + kTileY * kTileX, c0, 1, kTileX, vx, vy, nux, nuy, feqg,
                                                   wxm, wxp, wym, wyp, r, out, p0, p1, p2, p3, bw);
                store_cell<T>(o0 + g.slab, pc, mir, anymir, out);
                if constexpr (HRAW) hmom_group<1>(out, vx, vy, Hp);
            }
            if constexpr (HRAW) {
                Qp[0] = add2(Qp[0], f2(t0, 0.f)); Qp[1] = add2(Qp[1], f2(t1, 0.f));
                Qp[2] = add2(Qp[2], f2(t2, 0.f)); Qp[3] = add2(Qp[3], f2(t3, 0.f));
            }
        stored:
            if (REC) a.bits[(long)q * a.bslab + (long)(j + 2) * a.bpitch + i + 2] = bw;
            // fold the plain sums of 8 groups (16 in the FP32 Shakhov variant)
            // into the compensated sums
            if (++fold == (HRAW ? 16 : 8)) {
                if constexpr (HRAW) {
                    fold_lanes<4>(Qp, 0, sacc, tid);
                    fold_lanes<5>(Hp, 4, sacc, tid);
                } else {
                    if constexpr (sizeof(T) == 4 && MUSCL) fold_pairs(Qp, q0, q1, q2, q3);
                    m0.add(q0); m1.add(q1); m2.add(q2); m3.add(q3);
                    q0 = q1 = q2 = q3 = 0;
                }
                fold = 0;
            }
        } else if (zero) {
            T z[W];
#pragma unroll
            for (int e = 0; e < W; ++e) z[e] = 0;
            store_cell<T>(o0, pc, mir, anymir, z);
            store_cell<T>(o0 + g.slab, pc, mir, anymir, z);
        }
        __syncwarp();
        if (tx == 0) mbar_arrive(&empty[st]);
    }
    if (tid == 0) {
        // every issued copy has landed before the block exits (normally
        // already observed by the waits above)
        for (int k = max(ngr - kStages, 0); k < ngr; ++k) mbar_wait(&full[k % kStages], (uint32_t)((k / kStages) & 1));
    }
    if (plain) {
        if constexpr (HRAW) {
            fold_lanes<4>(Qp, 0, sacc, tid);
            fold_lanes<5>(Hp, 4, sacc, tid);
#pragma unroll
            for (int m = 0; m < 4; ++m) a.pout[((long)split * 4 + m) * nc + cell] = sacc_value(sacc, m, tid);
#pragma unroll
            for (int m = 0; m < 5; ++m) a.hout[((long)split * 5 + m) * nc + cell] = sacc_value(sacc, 4 + m, tid);
            // the reference velocity of these sums: the origin
            if (split == 0) {
                a.hout[(long)a.S * 5 * nc + cell] = 0;
                a.hout[((long)a.S * 5 + 1) * nc + cell] = 0;
            }
        } else {
            if constexpr (sizeof(T) == 4 && MUSCL) fold_pairs(Qp, q0, q1, q2, q3);
            m0.add(q0); m1.add(q1); m2.add(q2); m3.add(q3);
            a.pout[((long)split * 4 + 0) * nc + cell] = m0.value();
            a.pout[((long)split * 4 + 1) * nc + cell] = m1.value();
            a.pout[((long)split * 4 + 2) * nc + cell] = m2.value();
            a.pout[((long)split * 4 + 3) * nc + cell] = m3.value();
        }
    } else if (zero) {
#pragma unroll
        for (int m = 0; m < 4; ++m) a.pout[((long)split * 4 + m) * nc + cell] = 0;
        if constexpr (HRAW) {
#pragma unroll
            for (int m = 0; m < 5; ++m) a.hout[((long)split * 5 + m) * nc + cell] = 0;
            if (split == 0) {
                a.hout[(long)a.S * 5 * nc + cell] = 0;
                a.hout[((long)a.S * 5 + 1) * nc + cell] = 0;
            }
        }
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
    int Sin;                  // partial-sum slots of the moments read (S, or 1 for summed moments)
    int gps;                  // velocity groups per split
    const void *cvinfo;       // control-volume records
    const void *vt;           // per-velocity coefficients (state precision)
    const void *eqp;          // [4][nc] conservative equilibrium parameters, or null
    int shak;                 // the Shakhov model under the explicit scheme
    void *hout;               // Shakhov: raw heat-flux moments of f^n+1 [S][5][nc] and reference velocity [2][nc]
    double pr1;               // 1 - Pr (Shakhov model)
    int *err;
};

// Velocity range [v0, v1) of split s.
__device__ __forceinline__ void split_range(const CvArgs &c, int s, int W, int &v0, int &v1)
{
    v0 = s * c.gps * W;
    v1 = min(c.g.nv, v0 + c.gps * W);
}

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

// Control-volume records of every control volume in the list (once per
// geometry): members from the master search, their slab indices, padding
// mirrors, edge lengths, wall edges and the area ratios.
__global__ void __launch_bounds__(256) k_members(CvArgs c, CvInfo *info)
{
    __shared__ int32_t mem[kMaxMembers];
    const Grid2D &g = c.g;
    const int n = min(c.counts[0], c.cap);
    const int W1 = g.nx + 1;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const long m = c.spec_list[idx];
        const int nm = gather_members(c, m, mem);
        CvInfo &I = info[idx];
        if (threadIdx.x < nm) {
            const long k = mem[threadIdx.x];
            CvMember &M = I.mem[threadIdx.x];
            int i, j;
            cell_ij(g, k, i, j);
            M.i = i; M.j = j;
            M.pc = nbr(g, i, j);
            mirrors(g, i, j, M.mir);
            M.L[0] = c.Gn.lx[(long)j * W1 + i];
            M.L[1] = c.Gn.lx[(long)j * W1 + i + 1];
            M.L[2] = c.Gn.ly[(long)j * g.nx + i];
            M.L[3] = c.Gn.ly[(long)(j + 1) * g.nx + i];
            M.wslot = c.wslot[k];
            const bool wall = M.wslot >= 0;
            M.lw = wall ? c.Gn.lw[k] : 0.0;
            M.nwx = c.Gn.nwx[k];
            M.nwy = c.Gn.nwy[k];
            M.sb = c.Gn.sbar[k];
            M.mask = c.flags[k] >> kMaskShift;
            M.live = c.Gn.type[k] != DVM_SOLID;
            M.keep = c.Gp.type[k] != DVM_SOLID;
            if (k == m) I.pcm = M.pc;
        }
        if (threadIdx.x == 0) {
            double Sn = 0, Sp = 0;
            for (int q = 0; q < nm; ++q) { Sn += c.Gn.sbar[mem[q]]; Sp += c.Gp.sbar[mem[q]]; }
            I.nm = nm;
            I.ok = Sp > 0;
            I.Sn = Sn;
            I.a = Sp > 0 ? Sn / Sp : 0.0;
            I.bco = Sp > 0 ? g.dt / Sp : 0.0;
            if (!(Sp > 0)) atomicExch(&c.err[kErrGeometry], 1);
        }
        __syncthreads();
    }
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

// Write the moment sums of one velocity split to a member (zeros if the
// member is solid).
template <typename T>
__device__ __forceinline__ void write_split_partials(T *part, int s, long nc, long k, bool keep,
                                                     T s0, T s1, T s2, T s3)
{
    part[((long)s * 4 + 0) * nc + k] = keep ? s0 : T(0);
    part[((long)s * 4 + 1) * nc + k] = keep ? s1 : T(0);
    part[((long)s * 4 + 2) * nc + k] = keep ? s2 : T(0);
    part[((long)s * 4 + 3) * nc + k] = keep ? s3 : T(0);
}

// Fusion (Eq. FusionDD): f_CV = sum sbar f / S over a merged control volume,
// written back to every member, with the moment sums of the result.  One
// work item is one control volume and one velocity split.
template <typename T>
__global__ void __launch_bounds__(256) k_fusion(CvArgs c, T *f, T *part)
{
    __shared__ T red[8 * 2];
    const Grid2D &g = c.g;
    const CvInfo *info = reinterpret_cast<const CvInfo *>(c.cvinfo);
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(c.vt);
    const long nc = (long)g.nx * g.ny;
    const int n = min(c.counts[0], c.cap) * c.S;
    for (int item = blockIdx.x; item < n; item += gridDim.x) {
        const CvInfo &I = info[item / c.S];
        const int sp = item % c.S;
        const int nm = I.nm;
        if (nm <= 1) continue;
        int v0, v1;
        split_range(c, sp, Vec<T>::W, v0, v1);
        const double S = I.Sn;
        Acc<T> a0, a1, a2, a3;
        for (int comp = 0; comp < 2; ++comp)
            for (int p = v0 + threadIdx.x; p < v1; p += blockDim.x) {
                const long base = ebase<T>(g, comp, p);
                double acc = 0;
                for (int q = 0; q < nm; ++q) acc += I.mem[q].sb * (double)f[base + I.mem[q].pc * Vec<T>::W];
                const T fcv = (T)(acc / S);
                for (int q = 0; q < nm; ++q) {
                    f[base + I.mem[q].pc * Vec<T>::W] = fcv;
                    for (int t = 0; t < 4; ++t)
                        if (I.mem[q].mir[t] >= 0) f[base + I.mem[q].mir[t] * Vec<T>::W] = fcv;
                }
                const VCoef<T> vc = ld_coef(vt + p);
                if (comp == 0) {
                    a0.add(fcv); a1.add(vc.vx * fcv); a2.add(vc.vy * fcv);
                    a3.add(T(0.5) * (vc.vx * vc.vx + vc.vy * vc.vy) * fcv);
                } else {
                    a3.add(fcv);
                }
            }
        const T t0 = block_acc(a0, red), t1 = block_acc(a1, red), t2 = block_acc(a2, red), t3 = block_acc(a3, red);
        if (threadIdx.x < nm) {
            const CvMember &M = I.mem[threadIdx.x];
            const long k = (long)M.j * g.nx + M.i;
            write_split_partials<T>(part, sp, nc, k, M.live != 0, t0, t1, t2, t3);
        }
        __syncthreads();
    }
}


// Wall density (Eq. BoundaryDDv), stress (Eq. StressTensorDD), force and
// torque (Eqs. eq-force, eq-torque), in FP64.  The wall velocity is
// u_w = u_c + (r - c)^perp omega (Eq. uwDD) at t^n.  A work item is one wall
// cell and one velocity split: it writes the split's sums over outgoing
// velocities (of f) and incoming ones (of M[1, u_w, T_w]).  The last block to
// finish combines the splits of every wall cell in list order: wall density
// phi, stress, force and torque, their sum over the body, the angular
// velocity at t^{n+1} (Eq. motionDD_vit) and the history record.  It leaves
// (phi, u_w, T_w) of each wall cell for the control-volume kernel.
struct WallGeom {
    double rx, ry, uwx, uwy, Tw, nwx, nwy, lw;
};

__device__ __forceinline__ WallGeom wall_geom(const CvArgs &c, const BodyParams &b, long k, double omega)
{
    WallGeom w;
    w.rx = c.Gn.rwx[k] - b.cx;
    w.ry = c.Gn.rwy[k] - b.cy;
    w.uwx = b.vbx - w.ry * omega;
    w.uwy = b.vby + w.rx * omega;
    w.Tw = wall_temperature(b, w.rx, w.ry);
    w.nwx = c.Gn.nwx[k];
    w.nwy = c.Gn.nwy[k];
    w.lw = c.Gn.lw[k];
    return w;
}

// mode 0: the whole wall step.  A velocity split (Sec. 5.2) runs it in two
// halves around the caller's sum over the ranks: mode 1 writes each wall
// cell's eight sums over this context's velocities to xw[8 * slot] and stops;
// mode 2 reads the summed eight values from xw and does the rest.
// The velocities of the wall sums and their sign against the wall normal are
// FP64 in both precisions (the split into incoming and outgoing velocities
// is decided as in FP64); the products and the compensated sums are in the
// state precision (for an FP32 state, FP32 products and compensated sums,
// about 1e-7 relative); the wall density, the stress, the force, the torque
// and the rotation are FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_wall(CvArgs c, BodyParams b, BodyDev *body, const T *f,
                                              double *wdat, double *wcontrib, int *ticket,
                                              double *hist, int moving, int mode, double *xw)
{
    __shared__ double red[8 * 8];
    __shared__ double ex[kMaxAxisNv], ey[kMaxAxisNv];
    __shared__ double wsc[6];   // uwx, uwy, nwx, nwy, 1/(2 pi Tw), 2 Tw
    using WA = typename std::conditional<sizeof(T) == 4, float, double>::type;   // wall-sum type
    __shared__ WA wred[8 * 2];
    __shared__ bool last;
    const Grid2D &g = c.g;
    const int nw = min(c.counts[1], c.cap);
    const double omega = body->omega;
    const int tid = threadIdx.x;
    for (int idx = blockIdx.x; idx < nw; idx += gridDim.x) {
        const long k = c.wall_list[idx];
        double r0, r1, r2, r3, r4, r5, r6, r7;
        if (mode == 2) {
            const double *x = xw + 8L * idx;
            r0 = x[0]; r1 = x[1]; r2 = x[2]; r3 = x[3]; r4 = x[4]; r5 = x[5]; r6 = x[6]; r7 = x[7];
        } else {
        if (tid == 0) {
            const WallGeom w = wall_geom(c, b, k, omega);
            wsc[0] = w.uwx; wsc[1] = w.uwy; wsc[2] = w.nwx; wsc[3] = w.nwy;
            wsc[4] = 1.0 / (2.0 * kPi * w.Tw); wsc[5] = 2.0 * w.Tw;
        }
        __syncthreads();
        const double uwx = wsc[0], uwy = wsc[1], nwx = wsc[2], nwy = wsc[3], cm = wsc[4], twoTw = wsc[5];
        // separable Maxwellian M[1, u_w, T_w] = ex[p1] ey[p2] / (2 pi T_w)
        for (int q = tid; q < g.nvx + g.nvy; q += blockDim.x) {
            if (q < g.nvx) { const double d = g.vxmin + q * g.dvx - uwx; ex[q] = exp(-(d * d) / twoTw); }
            else { const int qq = q - g.nvx; const double d = g.vymin + qq * g.dvy - uwy; ey[qq] = exp(-(d * d) / twoTw); }
        }
        __syncthreads();
        const long pck = pcell(g, k) * Vec<T>::W;
        Acc<WA> a0, a1, a2, a3, a4, a5, a6, a7;
        int p1 = tid % g.nvx, p2 = tid / g.nvx;
        const int dp1 = blockDim.x % g.nvx, dp2 = blockDim.x / g.nvx;
        for (int p = tid; p < g.nv; p += blockDim.x) {
            const double ax = g.vxmin + p1 * g.dvx - uwx, ay = g.vymin + p2 * g.dvy - uwy;
            const double cp = ax * nwx + ay * nwy;
            const WA cw = (WA)cp, axw = (WA)ax, ayw = (WA)ay;
            if (cp > 0.0) {
                const WA fv = (WA)f[ebase<T>(g, 0, p) + pck];
                a0.add(cw * fv);
                a5.add(axw * axw * fv); a6.add(axw * ayw * fv); a7.add(ayw * ayw * fv);
            } else if (cp < 0.0) {
                const WA m1 = (WA)(cm * ex[p1] * ey[p2]);
                a1.add(cw * m1);
                a2.add(axw * axw * m1); a3.add(axw * ayw * m1); a4.add(ayw * ayw * m1);
            }
            p1 += dp1; p2 += dp2;
            if (p1 >= g.nvx) { p1 -= g.nvx; p2 += 1; }
        }
        r0 = block_acc(a0, wred); r1 = block_acc(a1, wred); r2 = block_acc(a2, wred);
        r3 = block_acc(a3, wred); r4 = block_acc(a4, wred); r5 = block_acc(a5, wred);
        r6 = block_acc(a6, wred); r7 = block_acc(a7, wred);
        if (mode == 1) {
            if (tid == 0) {
                double *x = xw + 8L * idx;
                x[0] = r0; x[1] = r1; x[2] = r2; x[3] = r3; x[4] = r4; x[5] = r5; x[6] = r6; x[7] = r7;
            }
            __syncthreads();
            continue;
        }
        }
        if (tid == 0) {
            const WallGeom w = wall_geom(c, b, k, omega);
            const double phi = -(r0 * g.dv) / (r1 * g.dv);
            const double sxx = (phi * r2 + r5) * g.dv, sxy = (phi * r3 + r6) * g.dv;
            const double syy = (phi * r4 + r7) * g.dv;
            const double fkx = (sxx * w.nwx + sxy * w.nwy) * w.lw, fky = (sxy * w.nwx + syy * w.nwy) * w.lw;
            wcontrib[3 * idx] = fkx;
            wcontrib[3 * idx + 1] = fky;
            wcontrib[3 * idx + 2] = w.rx * fky - w.ry * fkx;
            double *d = wdat + 4L * idx;
            d[0] = phi; d[1] = w.uwx; d[2] = w.uwy; d[3] = w.Tw;
        }
        __syncthreads();
    }
    if (mode == 1) return;
    // the last block sums the contributions in list order
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double fx = 0, fy = 0, tq = 0;
    for (int t = tid; t < nw; t += blockDim.x) {
        fx += wcontrib[3 * t]; fy += wcontrib[3 * t + 1]; tq += wcontrib[3 * t + 2];
    }
    fx = block_sum(fx, red); fy = block_sum(fy, red + 8); tq = block_sum(tq, red + 16);
    if (tid == 0) {
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
    constexpr int W = Vec<T>::W;
    return f[((long)(p / W) * 2 + comp) * g.slab * W + nbr(g, i, j) * W + (p % W)];
}

// Explicit update of one control volume (Eq. ExSchemeDD): fluxes across the
// Cartesian edges of every member (Eq. FluxDD) and across its wall edge with
// the diffuse-reflection state f_w = phi M[1, u_w, T_w], g_w = T_w/2 f_w on
// incoming velocities (Eq. BoundaryDDv; phi from the FP64 wall kernel), area
// ratio S^n / S^{n+1,*}, relaxation, then distribution to the members (Eq.
// UpdateDD; members solid at t^{n+1} hold 0) and the moment sums of the
// velocity split.  One work item is one control volume and one split.
// Copy of one control-volume record into shared memory (16-byte words).
__device__ __forceinline__ void load_info(const CvInfo *src, CvInfo *dst)
{
    static_assert(sizeof(CvInfo) % 16 == 0, "CvInfo is copied in 16-byte words");
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int q = threadIdx.x; q < (int)(sizeof(CvInfo) / 16); q += blockDim.x) d4[q] = __ldg(s4 + q);
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_special(CvArgs c, const T *fin, T *fout, const T *pin,
                                                 T *pout, const double *wdat)
{
    __shared__ T red[8 * 2];
    __shared__ __align__(16) CvInfo I;
    const Grid2D &g = c.g;
    const CvInfo *info = reinterpret_cast<const CvInfo *>(c.cvinfo);
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(c.vt);
    const long nc = (long)g.nx * g.ny;
    const int n = min(c.counts[0], c.cap) * c.S;
    constexpr int W = Vec<T>::W;
    for (int item = blockIdx.x; item < n; item += gridDim.x) {
        const int idx = item / c.S, sp = item % c.S;
        load_info(info + idx, &I);
        if (!I.ok) { __syncthreads(); continue; }
        const int nm = I.nm;
        int v0, v1;
        split_range(c, sp, W, v0, v1);
        const long m = c.spec_list[idx];
        T s[4];
        gather_partials(pin, c.Sin, nc, m, s);
        T rho, ux, uy, tmp;
        if (!primitives<T>(pick<T>(g.dv_f, g.dv), s[0], s[1], s[2], s[3], rho, ux, uy, tmp) && threadIdx.x == 0 && sp == 0)
            atomicExch(&c.err[kErrNonphys], 1);
        const T a = (T)I.a, bco = (T)I.bco, r = pick<T>(g.dt_tau0_f, g.dt_tau0) * rho;
        if (c.eqp) {
            const T *e = static_cast<const T *>(c.eqp);
            rho = e[m]; ux = e[nc + m]; uy = e[2 * nc + m]; tmp = e[3 * nc + m];
        }
        const T A = rho / (T(2.0 * kPi) * tmp);
        const T i2T = T(1) / (T(2) * tmp);
        // Shakhov (Eq. ShakhovDD): k q with the heat flux of the control
        // volume at t^n, summed here over every velocity of its (fused) state
        T kqx = 0, kqy = 0;
        if (c.shak) {
            Acc<T> h0, h1;
            for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
                const VCoef<T> vc = ld_coef(vt + p);
                const T dx = vc.vx - ux, dy = vc.vy - uy;
                const T fa = fin[ebase<T>(g, 0, p) + I.pcm * W], fb = fin[ebase<T>(g, 1, p) + I.pcm * W];
                const T w = T(0.5) * (dx * dx + dy * dy) * fa + fb;
                h0.add(dx * w);
                h1.add(dy * w);
            }
            const T dv = pick<T>(g.dv_f, g.dv);
            const T qx = block_acc(h0, red) * dv, qy = block_acc(h1, red) * dv;
            const T k = T(c.pr1) / (T(5) * rho * tmp * tmp);
            kqx = k * qx;
            kqy = k * qy;
        }
        Acc<T> s0, s1, s2, s3;
        Acc<T> hs[5];     // Shakhov: raw heat-flux moments of the new state about (ux, uy)
        for (int p = v0 + threadIdx.x; p < v1; p += blockDim.x) {
            const VCoef<T> vc = ld_coef(vt + p);
            const T vx = vc.vx, vy = vc.vy, nux = vc.nux, nuy = vc.nuy;
            const T dxu = vx - ux, dyu = vy - uy;
            const T feq0 = A * dexp(-(dxu * dxu + dyu * dyu) * i2T);
            T sf = T(1), sg = T(1);
            if (c.shak) {
                const T kcq = kqx * dxu + kqy * dyu, d2 = (dxu * dxu + dyu * dyu) * T(2) * i2T;
                sf = fma(kcq, d2 - T(4), T(1));
                sg = fma(kcq, d2 - T(2), T(1));
            }
            const long base0 = ebase<T>(g, 0, p), base1 = ebase<T>(g, 1, p);
            T R0 = 0, R1 = 0;
            for (int q = 0; q < nm; ++q) {
                const CvMember &M = I.mem[q];
                if (!M.live) continue;
                const int i = M.i, j = M.j;
                const bool mus = M.mask != 0;
                T Fw0 = 0, Fw1 = 0;
                const T f0 = fin[base0 + M.pc * W], f1 = fin[base1 + M.pc * W];
                if (M.wslot >= 0) {
                    // diffuse reflection: incoming state f_w and the flux
                    // lw [min(c, 0) f_w + max(c, 0) f] across the wall edge
                    const double *d = wdat + 4L * M.wslot;
                    const T phi = (T)d[0], uwx = (T)d[1], uwy = (T)d[2], Tw = (T)d[3];
                    const T ax = vx - uwx, ay = vy - uwy;
                    const T cw = ax * (T)M.nwx + ay * (T)M.nwy;
                    const T m1 = dexp(-(ax * ax + ay * ay) / (T(2) * Tw)) / (T(2.0 * kPi) * Tw);
                    const T lw = (T)M.lw;
                    Fw0 = lw * (fmin(cw, T(0)) * (phi * m1) + fmax(cw, T(0)) * f0);
                    Fw1 = lw * (fmin(cw, T(0)) * (phi * (Tw / T(2) * m1)) + fmax(cw, T(0)) * f1);
                }
#pragma unroll
                for (int comp = 0; comp < 2; ++comp) {
                    const long base = comp == 0 ? base0 : base1;
                    const T fc = comp == 0 ? f0 : f1;
                    const T fxm1 = fin[base + nbr(g, i - 1, j) * W], fxp1 = fin[base + nbr(g, i + 1, j) * W];
                    const T fym1 = fin[base + nbr(g, i, j - 1) * W], fyp1 = fin[base + nbr(g, i, j + 1) * W];
                    T fxm2 = 0, fxp2 = 0, fym2 = 0, fyp2 = 0;
                    if (mus) {
                        fxm2 = fin[base + nbr(g, i - 2, j) * W]; fxp2 = fin[base + nbr(g, i + 2, j) * W];
                        fym2 = fin[base + nbr(g, i, j - 2) * W]; fyp2 = fin[base + nbr(g, i, j + 2) * W];
                    }
                    const T Fxp = face_flux<T>((T)M.L[1], vx, nux, fxm1, fc, fxp1, fxp2, M.mask & 2);
                    const T Fxm = face_flux<T>((T)M.L[0], vx, nux, fxm2, fxm1, fc, fxp1, M.mask & 1);
                    const T Fyp = face_flux<T>((T)M.L[3], vy, nuy, fym1, fc, fyp1, fyp2, M.mask & 8);
                    const T Fym = face_flux<T>((T)M.L[2], vy, nuy, fym2, fym1, fc, fyp1, M.mask & 4);
                    const T Rq = (Fxp - Fxm) + (Fyp - Fym) + (comp == 0 ? Fw0 : Fw1);
                    if (comp == 0) R0 += Rq; else R1 += Rq;
                }
            }
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
                const long base = comp == 0 ? base0 : base1;
                const T fcv = fin[base + I.pcm * W];
                const T feq = comp == 0 ? feq0 * sf : tmp / T(2) * feq0 * sg;
                const T fn = a * fcv - bco * (comp == 0 ? R0 : R1) + a * r * (feq - fcv);
                for (int q = 0; q < nm; ++q) {
                    const CvMember &M = I.mem[q];
                    const T v = M.keep ? fn : T(0);
                    fout[base + M.pc * W] = v;
                    for (int t = 0; t < 4; ++t)
                        if (M.mir[t] >= 0) fout[base + M.mir[t] * W] = v;
                }
                if (comp == 0) {
                    s0.add(fn); s1.add(vx * fn); s2.add(vy * fn);
                    s3.add(T(0.5) * (vx * vx + vy * vy) * fn);
                } else {
                    s3.add(fn);
                }
                if (c.hout) {
                    if (comp == 0) {
                        const T tx = dxu * fn, ty = dyu * fn, k2 = T(0.5) * (dxu * dxu + dyu * dyu);
                        hs[0].add(k2 * tx); hs[1].add(k2 * ty);
                        hs[2].add(dxu * tx); hs[3].add(dyu * tx); hs[4].add(dyu * ty);
                    } else {
                        hs[0].add(dxu * fn); hs[1].add(dyu * fn);
                    }
                }
            }
        }
        const T t0 = block_acc(s0, red), t1 = block_acc(s1, red);
        const T t2 = block_acc(s2, red), t3 = block_acc(s3, red);
        if (threadIdx.x < nm) {
            const CvMember &M = I.mem[threadIdx.x];
            write_split_partials<T>(pout, sp, nc, (long)M.j * g.nx + M.i, M.keep != 0, t0, t1, t2, t3);
        }
        if (c.hout) {
            T hv[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) hv[q] = block_acc(hs[q], red);
            if (threadIdx.x < nm) {
                const CvMember &M = I.mem[threadIdx.x];
                const long k = (long)M.j * g.nx + M.i;
                const bool keep = M.keep != 0;
                T *ho = static_cast<T *>(c.hout);
#pragma unroll
                for (int q = 0; q < 5; ++q) ho[((long)sp * 5 + q) * nc + k] = keep ? hv[q] : T(0);
                if (sp == 0) {
                    ho[(long)c.S * 5 * nc + k] = keep ? ux : T(0);
                    ho[((long)c.S * 5 + 1) * nc + k] = keep ? uy : T(0);
                }
            }
        }
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

// Moment sums of cells (i, j) of one row over a chunk of the velocity
// groups: f, v_x f, v_y f and |v|^2/2 f + g (Eq. MacroscopicDDv), per group
// plain over its lanes and compensated across groups.  The lanes of a warp
// are 32 consecutive cells, so each group's vector of the 32 cells is one
// coalesced read; warp threadIdx.y takes the threadIdx.y-th of kMomChunks
// chunks.

template <typename T>
__device__ __forceinline__ void state_sums2d(const Grid2D &g, const T *f, const VCoef<T> *vt, int i, int j,
                                             Acc<T> (&s)[4])
{
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    if (i >= g.nx) return;
    const int gps = (g.ngrp + kMomChunks - 1) / kMomChunks;
    const int q0 = threadIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    const long pc = nbr(g, i, j);
    const V *fv = reinterpret_cast<const V *>(f);
    for (int q = q0; q < q1; ++q) {
        T a[W], b[W];
        vld<T>(fv + (long)q * 2 * g.slab + pc, a);
        vld<T>(fv + ((long)q * 2 + 1) * g.slab + pc, b);
        T t0 = 0, t1 = 0, t2 = 0, t3 = 0;
#pragma unroll
        for (int e = 0; e < W; ++e) {
            if (q * W + e >= g.nv) continue;
            const VCoef<T> c = ld_coef(vt + q * W + e);
            t0 += a[e];
            t1 += c.vx * a[e];
            t2 += c.vy * a[e];
            t3 += T(0.5) * (c.vx * c.vx + c.vy * c.vy) * a[e] + b[e];
        }
        s[0].add(t0); s[1].add(t1); s[2].add(t2); s[3].add(t3);
    }
}

// Partial moment sums of a state (set-up, not the time step): the whole sum
// goes to split 0, zeros to the others and to solid cells.
template <typename T>
__global__ void __launch_bounds__(32 * kMomChunks) k_partials(Grid2D g, int S, const T *f, const VCoef<T> *vt,
                                                              T *part, const int8_t *type, int *err)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y;
    Acc<T> s[4];
    state_sums2d<T>(g, f, vt, i, j, s);
    merge_chunks<T, 4>(s);
    if (threadIdx.y != 0 || i >= g.nx) return;
    const long nc = (long)g.nx * g.ny, cell = (long)j * g.nx + i;
    const bool keep = type[cell] != DVM_SOLID;
    if (keep) {
        T rho, ux, uy, tmp;
        if (!primitives<T>(pick<T>(g.dv_f, g.dv), s[0].value(), s[1].value(), s[2].value(), s[3].value(), rho, ux,
                           uy, tmp))
            atomicExch(&err[kErrNonphys], 1);
    }
    write_member_partials<T>(part, S, nc, cell, keep, s[0].value(), s[1].value(), s[2].value(), s[3].value());
}

// Moments for output: rho, ux, uy, uz (= 0), T per cell, formed in FP64 from
// the sums (compensated in the state precision).
template <typename T>
__global__ void __launch_bounds__(32 * kMomChunks) k_moments_out(Grid2D g, const T *f, const VCoef<T> *vt,
                                                                 double *out)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y;
    Acc<T> s[4];
    state_sums2d<T>(g, f, vt, i, j, s);
    merge_chunks<T, 4>(s);
    if (threadIdx.y != 0 || i >= g.nx) return;
    double *o5 = out + ((long)j * g.nx + i) * 5;
    const double s0 = (double)s[0].s - (double)s[0].c, s1 = (double)s[1].s - (double)s[1].c;
    const double s2 = (double)s[2].s - (double)s[2].c, s3 = (double)s[3].s - (double)s[3].c;
    const double rho = s0 * g.dv;
    if (!(rho > 0)) {
        for (int q = 0; q < 5; ++q) o5[q] = 0;
        return;
    }
    const double ux = s1 * g.dv / rho, uy = s2 * g.dv / rho;
    o5[0] = rho; o5[1] = ux; o5[2] = uy; o5[3] = 0;
    o5[4] = (2.0 * (s3 * g.dv) / rho - (ux * ux + uy * uy)) / 3.0;
}

// Implicit relaxation of the first-order semi-implicit scheme (Eq.
// ImpSchemeDD), after a transport pass that ran without relaxation: the
// moments at t^{n+1} are those of the transported values (the collision term
// sums to zero over the velocities), read from the partial sums the transport
// kernels wrote.  Every gas cell relaxes towards their Maxwellian,
// f = (f* + nu M) / (1 + nu) and g = (g* + nu T/2 M) / (1 + nu) with
// nu = dt / tau^{n+1} = (dt / tau0) rho, in place and in its padding mirrors,
// and the partial sums become those of the relaxed state (split 0; zeros in
// the others).  Cells solid at t^{n+1} (type) keep their zero state.
// Block = 32 consecutive cells of a row x kMomChunks warps, one chunk of the
// velocity groups each.
// 2^x for the relaxation kernel: the hardware approximation in FP32.
__device__ __forceinline__ float exp2_relax(float x) { return ex2_fast(x); }
__device__ __forceinline__ double exp2_relax(double x) { return exp2(x); }

// With SHAK (the Shakhov model, Eq. ShakhovDD) the equilibrium carries the
// heat flux at t^{n+1}, q = q_T / (1 + nu Pr), q_T that of the transported
// values (the heat-flux moment of the scheme with the model's (1 - Pr) q):
// a first pass over the cell's velocities sums q_T, the second relaxes
// towards f_S = M [1 + k c.q (|c|^2/T - 4)], g_S = T/2 M [1 + k c.q (|c|^2/T - 2)],
// k = (1 - Pr) / (5 rho T^2).
// The moments of the transported values come from mom (Smom partial-sum
// slots: this context's S, or 1 for the sums of a velocity split over the
// ranks); the moment sums of the relaxed values go to part (S slots).
// CONS: the equilibrium from the conservative parameters eqp (Sec. 3.1), a
// variant of its own so that the plain one keeps its registers (the pass is
// bound by memory latency, and 64 registers give four blocks per SM).
template <typename T, bool SHAK, bool CONS>
__global__ void __launch_bounds__(32 * kMomChunks) k_imex(Grid2D g, int S, T dt_tau0, T *f, const VCoef<T> *vt,
                                                          const T *mom, int Smom, T *part, const int8_t *type,
                                                          const T *eqp, T Pr, int *err)
{
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    __shared__ T qsh[2][32];
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y;
    const long nc = (long)g.nx * g.ny, cell = (long)j * g.nx + i;
    bool gas = i < g.nx && type[cell] != DVM_SOLID;
    T s[4] = {T(0), T(0), T(0), T(0)};
    if (gas) gather_partials(mom, Smom, nc, cell, s);
    T rho = 0, ux = 0, uy = 0, tmp = 0;
    if (gas && !primitives<T>(pick<T>(g.dv_f, g.dv), s[0], s[1], s[2], s[3], rho, ux, uy, tmp)) {
        if (threadIdx.y == 0) atomicExch(&err[kErrNonphys], 1);
        gas = false;
    }
    Acc<T> a4[4];
    const int gps = (g.ngrp + kMomChunks - 1) / kMomChunks;
    const int q0 = threadIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    const long pc = nbr(g, i, j);
    V *fv = reinterpret_cast<V *>(f);
    T qx = 0, qy = 0;
    if constexpr (SHAK) {
        // heat flux of the transported values about their velocity
        Acc<T> hq[2];
        if (gas) {
            for (int q = q0; q < q1; ++q) {
                T a[W], b[W];
                vld<T>(fv + (long)q * 2 * g.slab + pc, a);
                vld<T>(fv + ((long)q * 2 + 1) * g.slab + pc, b);
                T t0 = 0, t1 = 0;
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    if (q * W + e >= g.nv) continue;
                    const VCoef<T> c = ld_coef(vt + q * W + e);
                    const T dx = c.vx - ux, dy = c.vy - uy;
                    const T w = T(0.5) * (dx * dx + dy * dy) * a[e] + b[e];
                    t0 += dx * w;
                    t1 += dy * w;
                }
                hq[0].add(t0);
                hq[1].add(t1);
            }
        }
        merge_chunks<T, 2>(hq);
        if (threadIdx.y == 0) {
            const T rel = T(1) / (T(1) + dt_tau0 * rho * Pr);
            qsh[0][threadIdx.x] = hq[0].value() * pick<T>(g.dv_f, g.dv) * rel;
            qsh[1][threadIdx.x] = hq[1].value() * pick<T>(g.dv_f, g.dv) * rel;
        }
        __syncthreads();
        qx = qsh[0][threadIdx.x];
        qy = qsh[1][threadIdx.x];
    }
    if (gas) {
        const T nu = dt_tau0 * rho, inv = T(1) / (T(1) + nu);
        if constexpr (CONS) {
            // conservative equilibrium of the transported state (Sec. 3.1)
            rho = eqp[cell]; ux = eqp[nc + cell]; uy = eqp[2 * nc + cell]; tmp = eqp[3 * nc + cell];
        }
        const T A = rho / (T(2.0 * kPi) * tmp), c2 = T(kLog2e) / (T(2) * tmp), half = tmp / T(2);
        const T kk = SHAK ? (T(1) - Pr) / (T(5) * rho * tmp * tmp) : T(0), iT = T(1) / tmp;
        long mir[4];
        mirrors(g, i, j, mir);
#pragma unroll 2
        for (int q = q0; q < q1; ++q) {
            V *pa = fv + (long)q * 2 * g.slab, *pb = pa + g.slab;
            T a[W], b[W];
            vld<T>(pa + pc, a);
            vld<T>(pb + pc, b);
            T t0 = 0, t1 = 0, t2 = 0, t3 = 0;
#pragma unroll
            for (int e = 0; e < W; ++e) {
                if (q * W + e >= g.nv) continue;
                const VCoef<T> c = ld_coef(vt + q * W + e);
                const T dx = c.vx - ux, dy = c.vy - uy;
                const T M = A * exp2_relax(-(dx * dx + dy * dy) * c2);
                T sf = T(1), sg = T(1);
                if constexpr (SHAK) {
                    const T h = kk * (dx * qx + dy * qy), d2 = (dx * dx + dy * dy) * iT;
                    sf += h * (d2 - T(4));
                    sg += h * (d2 - T(2));
                }
                a[e] = (a[e] + nu * M * sf) * inv;
                b[e] = (b[e] + nu * half * M * sg) * inv;
                t0 += a[e];
                t1 += c.vx * a[e];
                t2 += c.vy * a[e];
                t3 += T(0.5) * (c.vx * c.vx + c.vy * c.vy) * a[e] + b[e];
            }
            vst<T>(pa + pc, a);
            vst<T>(pb + pc, b);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (mir[k] >= 0) {
                    vst<T>(pa + mir[k], a);
                    vst<T>(pb + mir[k], b);
                }
            a4[0].add(t0); a4[1].add(t1); a4[2].add(t2); a4[3].add(t3);
        }
    }
    merge_chunks<T, 4>(a4);
    if (threadIdx.y != 0 || i >= g.nx) return;
    write_member_partials<T>(part, S, nc, cell, gas, a4[0].value(), a4[1].value(), a4[2].value(), a4[3].value());
}

// Maxwellian state from per-cell primitives (rho, ux, uy, uz, T); solid
// cells get 0 (Eq. BGKDD for g).
template <typename T>
__global__ void k_init(Grid2D g, const double *prim, const int8_t *type, T *f)
{
    const long k = blockIdx.x;            // one block per cell, threads over velocities
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    if (p >= g.nv) return;
    const long pc = pcell(g, k) * Vec<T>::W;
    const double *q = prim + 5 * k;
    double m = 0;
    if (type[k] != DVM_SOLID && q[0] > 0) {
        const double ax = g.vxmin + (p % g.nvx) * g.dvx - q[1];
        const double ay = g.vymin + (p / g.nvx) * g.dvy - q[2];
        m = q[0] / (2.0 * kPi * q[4]) * exp(-(ax * ax + ay * ay) / (2.0 * q[4]));
    }
    f[ebase<T>(g, 0, p) + pc] = (T)m;
    f[ebase<T>(g, 1, p) + pc] = (T)(q[4] / 2.0 * m);
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
    constexpr int W = Vec<T>::W;
    const long base0 = ((long)(p / W) * 2) * g.slab * W + (p % W);
    const long base1 = base0 + g.slab * W;
    for (int layer = 1; layer <= 2; ++layer) {
        long pcg;
        if (side == 0) pcg = nbr(g, -layer, (int)q);
        else if (side == 1) pcg = nbr(g, g.nx - 1 + layer, (int)q);
        else if (side == 2) pcg = nbr(g, (int)q, -layer);
        else pcg = nbr(g, (int)q, g.ny - 1 + layer);
        f0[base0 + pcg * W] = (T)m;
        f0[base1 + pcg * W] = (T)(s[4] / 2.0 * m);
        f1[base0 + pcg * W] = (T)m;
        f1[base1 + pcg * W] = (T)(s[4] / 2.0 * m);
    }
}

// Padding of periodic and zero-gradient sides from the interior of a state
// buffer (both layers, every group and component).
template <typename T>
__global__ void k_halo(Grid2D g, T *f)
{
    constexpr int W = Vec<T>::W;
    const long per = 2L * (g.nx + g.ny);      // padding cells of one layer (cross arms)
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * per * 2 * g.nvp) return;
    const long hc = t % (2 * per);            // padding cell: layer, side, position
    const long rest = t / (2 * per);
    const int comp = (int)(rest % 2), p = (int)(rest / 2);
    const int layer = (int)(hc / per) + 1;
    long pos = hc % per;
    int side, q;
    if (pos < g.ny) { side = 0; q = (int)pos; }
    else if (pos < 2L * g.ny) { side = 1; q = (int)(pos - g.ny); }
    else if (pos < 2L * g.ny + g.nx) { side = 2; q = (int)(pos - 2L * g.ny); }
    else { side = 3; q = (int)(pos - 2L * g.ny - g.nx); }
    const int kind = g.bc[side];
    if (kind == DVM_BC_MAXWELLIAN) return;
    int di, dj, si, sj;
    if (side == 0) { di = -layer; dj = q; si = kind == DVM_BC_PERIODIC ? g.nx - layer : 0; sj = q; }
    else if (side == 1) { di = g.nx - 1 + layer; dj = q; si = kind == DVM_BC_PERIODIC ? layer - 1 : g.nx - 1; sj = q; }
    else if (side == 2) { di = q; dj = -layer; si = q; sj = kind == DVM_BC_PERIODIC ? g.ny - layer : 0; }
    else { di = q; dj = g.ny - 1 + layer; si = q; sj = kind == DVM_BC_PERIODIC ? layer - 1 : g.ny - 1; }
    const long base = ((long)(p / W) * 2 + comp) * g.slab * W + (p % W);
    f[base + nbr(g, di, dj) * W] = f[base + nbr(g, si, sj) * W];
}

// Conversion between the public layout [cell][comp][p] and the device layout.
template <typename T>
__global__ void k_pack(Grid2D g, const T *src, T *dst, int to_dev)
{
    const long k = blockIdx.x;            // one block per cell, threads over (comp, p)
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= 2 * g.nv) return;
    const int comp = e >= g.nv, p = e - comp * g.nv;
    const long t = k * 2L * g.nv + e;
    const long d = ebase<T>(g, comp, p) + pcell(g, k) * Vec<T>::W;
    if (to_dev) dst[d] = src[t];
    else dst[t] = src[d];
}

// Zero the state of every solid cell (they belong to no control volume): one
// thread per cell and chunk of the velocity groups (blockIdx.y); only the
// threads of solid cells store, whole group vectors of both components.
template <typename T>
__global__ void k_zero_solid(Grid2D g, const int8_t *type, T *f)
{
    using V = typename Vec<T>::type;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long)g.nx * g.ny || type[k] != DVM_SOLID) return;
    const int gps = (g.ngrp + gridDim.y - 1) / gridDim.y;
    const int q0 = blockIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    const long pc = pcell(g, k);
    V *fv = reinterpret_cast<V *>(f);
    const T z[Vec<T>::W] = {};
    for (int q = q0; q < q1; ++q) {
        vst<T>(fv + (long)q * 2 * g.slab + pc, z);
        vst<T>(fv + ((long)q * 2 + 1) * g.slab + pc, z);
    }
}

// Per-cell mass sbar * sum_p f dv (FP64), then a fixed-order sum.
template <typename T>
__global__ void __launch_bounds__(256) k_mass_cells(Grid2D g, const T *f, const double *sbar, double *cm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= (long)g.nx * g.ny) return;
    double s = 0;
    const long pc = pcell(g, cell) * Vec<T>::W;
    for (int p = lane; p < g.nv; p += 32) s += (double)f[ebase<T>(g, 0, p) + pc];
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

// Per-velocity coefficients, per-group sign of the velocity components and
// the FP32 coefficients of each group in the order of the packed path: seven
// float4 rows -nux, -nuy, 1 - nux, 1 - nuy, vx, vy, |v|^2/2 over the group's
// four lanes (lanes 0, 1 and 2, 3 form the two pairs).
template <typename T>
__global__ void k_tables(Grid2D g, VCoef<T> *vt, int8_t *gsign, float4 *ptab)
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
        float row[7][4];
        for (int e = 0; e < 4; ++e) {
            const int q = p * 4 + e;
            float vx = 1e4f, vy = 1e4f, nux = 0.f, nuy = 0.f;    // padding lanes: feq = 0, no transport
            if (q < g.nv) {
                vx = float(g.vxmin + (q % g.nvx) * g.dvx);
                vy = float(g.vymin + (q / g.nvx) * g.dvy);
                nux = fabsf(vx) * float(g.dt / g.dx);
                nuy = fabsf(vy) * float(g.dt / g.dy);
            }
            row[0][e] = -nux; row[1][e] = -nuy;
            row[2][e] = 1.f - nux; row[3][e] = 1.f - nuy;
            row[4][e] = vx; row[5][e] = vy;
            row[6][e] = 0.5f * (vx * vx + vy * vy);
        }
        if (W == 4)
            for (int r = 0; r < 7; ++r) ptab[p * 7 + r] = make_float4(row[r][0], row[r][1], row[r][2], row[r][3]);
    }
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

template <typename T, bool MUSCL, bool REC, bool SHAK>
cudaError_t launch_bulk(dvm_ctx *c, const BulkArgs<T> &a)
{
    const size_t smem = (size_t)kStages * kStageBytes + 2 * kStages * sizeof(uint64_t) +
                        (SHAK && sizeof(T) == 4 ? kSaccBytes : 0);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_bulk<T, MUSCL, REC, SHAK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // the device's greatest launch priority: the side-stream kernels beside
    // it (wall and control volumes) take an SM's registers only when none of
    // the bulk kernel's own blocks waits for them
    static const int prio = [] {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return greatest;
    }();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk(c->nx, 32), nblk(c->ny, kRows), c->S);
    cfg.blockDim = dim3(32, kRows);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_bulk<T, MUSCL, REC, SHAK>, a, c->tmap[c->cur]);
}

// Moment sums of each cell over this context's velocities, folded over the
// S velocity splits in fixed order: x[m][cell] = sum_s part[s][m][cell]
// (the data a velocity split exchanges, Sec. 5.2), in FP64.
template <typename T>
__global__ void k_fold_partials(const T *part, int S, long nc, double *x)
{
    const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= nc) return;
    T s[4];
    gather_partials(part, S, nc, cell, s);
#pragma unroll
    for (int m = 0; m < 4; ++m) x[(long)m * nc + cell] = (double)s[m];
}

// The summed moment sums back in the state precision, one slot.
template <typename T>
__global__ void k_unfold_partials(const double *x, long n, T *part)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) part[t] = (T)x[t];
}

// The bookkeeping that ends a step: the new state is the current one.
cudaError_t end_step2d(dvm_ctx *c, bool hkeep)
{
    c->cur = 1 - c->cur;
    if (c->moving) c->gcur = 1 - c->gcur;
    c->need_fusion = false;
    c->hvalid = hkeep;
    c->steps_done++;
    return cudaGetLastError();
}

// The relaxation of the semi-implicit scheme (Eq. ImpSchemeDD) on the
// transported values f[1 - cur], with their moments from mom (Smom slots).
template <typename T>
cudaError_t imex_relax2d(dvm_ctx *c, const T *mom, int Smom)
{
    const Grid2D g = grid2d(c);
    T *fout = (T *)c->f[1 - c->cur], *pout = (T *)c->part[1 - c->cur];
    const bool cons = c->eq_mode == DVM_EQ_CONSERVATIVE;
    const dim3 grid(nblk(c->nx, 32), c->ny), block(32, kMomChunks);
    const int8_t *type1 = c->geo[c->moving ? 1 - c->gcur : c->gcur].type;    // cell types at t^{n+1}
    cudaError_t e;
    // conservative equilibrium parameters of the transported state
    if (cons && (e = eqpar(c, mom, Smom)) != cudaSuccess) return e;
    const T r0 = T(c->dt / c->tau0);
    const VCoef<T> *vt = (const VCoef<T> *)c->vtab;
    if (c->model == DVM_SHAKHOV)
        k_imex<T, true, false><<<grid, block, 0, c->stream>>>(g, c->S, r0, fout, vt, mom, Smom, pout, type1, nullptr,
                                                              T(c->Pr), c->d_err);
    else if (cons)
        k_imex<T, false, true><<<grid, block, 0, c->stream>>>(g, c->S, r0, fout, vt, mom, Smom, pout, type1,
                                                              (const T *)c->eqp, T(1), c->d_err);
    else
        k_imex<T, false, false><<<grid, block, 0, c->stream>>>(g, c->S, r0, fout, vt, mom, Smom, pout, type1,
                                                               nullptr, T(1), c->d_err);
    c->launches += 1;
    return cudaGetLastError();
}

// Phase 3 of a semi-implicit step of a velocity split: the relaxation from
// the moment sums of the transported values summed over the ranks (xbuf).
template <typename T>
cudaError_t split_relax2d_t(dvm_ctx *c, const double *xbuf)
{
    const long nc = (long)c->nc;
    T *mom = (T *)c->split_in;
    k_unfold_partials<T><<<nblk(4 * nc, 256), 256, 0, c->stream>>>(xbuf, 4 * nc, mom);
    c->launches += 1;
    cudaError_t e = imex_relax2d<T>(c, mom, 1);
    if (e != cudaSuccess) return e;
    return end_step2d(c, false);
}

// One step in phases.  phase 0: the whole step.  A velocity split (Sec. 5.2:
// each rank holds every cell for a slab of the velocity grid) runs it as
// phase 1, which ends with this context's contributions in xbuf (FP64: the
// moment sums of F^n of every cell, [4][nc], then the eight wall sums of every
// wall cell, [wall slot][8]), and phase 2, which takes xbuf summed over the
// ranks and finishes the step.  Under the semi-implicit scheme phase 2 ends
// with this context's moment sums of the transported values in xbuf ([4][nc])
// and phase 3 takes them summed over the ranks and relaxes.
template <typename T>
cudaError_t step2d_t(dvm_ctx *c, int phase, double *xbuf)
{
    Grid2D g = grid2d(c);
    // the semi-implicit scheme (Eq. ImpSchemeDD) transports without
    // relaxation here; k_imex relaxes at the end of the step
    const bool imex = c->time_scheme == DVM_IMEX;
    if (imex) {
        g.dt_tau0 = 0.0;
        g.dt_tau0_f = 0.f;
    }
    BodyParams bp = body_params(c);
    const bool body = c->body.shape != DVM_SHAPE_NONE;
    const bool moving = c->moving;
    const long nc = (long)c->nc;
    T *fin = (T *)c->f[c->cur], *fout = (T *)c->f[1 - c->cur];
    T *pin = (T *)c->part[c->cur], *pout = (T *)c->part[1 - c->cur];
    cudaError_t e = cudaSuccess;
    if (moving && phase != 2) {
        k_advance<<<1, 32, 0, c->stream>>>(c->d_body, c->dt, 1);
        if ((e = geometry2d_level(c, 1 - c->gcur, body_trig(c, 2))) != cudaSuccess) return e;
        if ((e = masters_flags2d(c, true)) != cudaSuccess) return e;
        c->launches += 9;
    }
    CvArgs cv{};
    cv.g = g;
    cv.Gn = c->geo[c->gcur];
    cv.Gp = moving ? c->geo[1 - c->gcur] : c->geo[c->gcur];
    cv.master = c->master; cv.flags = c->flags;
    cv.spec_list = c->spec_list; cv.wall_list = c->wall_list; cv.wslot = c->wslot;
    cv.counts = c->counts; cv.cap = c->list_cap; cv.S = c->S;
    cv.Sin = phase == 2 ? 1 : c->S;
    cv.gps = (c->ngrp + c->S - 1) / c->S;
    cv.cvinfo = c->cvinfo; cv.vt = c->vtab;
    const bool cons = c->eq_mode == DVM_EQ_CONSERVATIVE;
    cv.eqp = cons && !imex ? c->eqp : nullptr;
    // the Shakhov model under the explicit scheme relaxes towards its
    // equilibrium inside the step, with the heat flux of F^n from the raw
    // moments the previous step left (k_heatflux when there are none)
    const bool shak = c->model == DVM_SHAKHOV && !imex;
    const bool hkeep = shak && c->prec == DVM_FP32;      // raw heat-flux moments kept (FP32)
    const bool hraw = hkeep && c->hvalid;
    cv.shak = shak ? 1 : 0;
    cv.hout = hkeep ? c->hpart[1 - c->cur] : nullptr;
    cv.pr1 = 1.0 - c->Pr;
    cv.err = c->d_err;
    const int cvgrid = 4 * 152;
    double *xw = xbuf ? xbuf + 4 * nc : nullptr;
    if (phase != 2) {
        if (body && (moving || c->need_fusion)) {
            k_fusion<T><<<cvgrid, 256, 0, c->stream>>>(cv, fin, pin);
            c->launches += 1;
        }
        if (phase == 1) {
            // this rank's moment sums of f_CV^n and wall sums, to be summed
            // over the ranks by the caller
            k_fold_partials<T><<<nblk(nc, 256), 256, 0, c->stream>>>(pin, c->S, nc, xbuf);
            c->launches += 1;
            if (body) {
                k_wall<T><<<cvgrid, 256, 0, c->stream>>>(cv, bp, c->d_body, fin, c->wphi, c->wcontrib, c->ticket,
                                                          c->d_hist, moving ? 1 : 0, 1, xw);
                c->launches += 1;
            }
            return cudaGetLastError();
        }
    } else {
        // the summed moments of f_CV^n, one slot in the state precision
        pin = (T *)c->split_in;
        k_unfold_partials<T><<<nblk(4 * nc, 256), 256, 0, c->stream>>>(xbuf, 4 * nc, pin);
        c->launches += 1;
    }
    const int Sin = phase == 2 ? 1 : c->S;
    // conservative equilibrium parameters of f_CV^n (after fusion)
    if (cons && !imex && (e = eqpar(c, pin, Sin)) != cudaSuccess) return e;
    // heat flux of every control volume at t^n (after fusion) when no raw
    // moments of F^n are at hand
    if (shak && !hraw && (e = heatflux2d(c, fin, pin)) != cudaSuccess) return e;
    if (body) {
        // the wall kernel (wall density, stress, force, rotation) and then the
        // control-volume kernel run on the side stream beside the bulk kernel:
        // both read F^n and write only the cut and merged control volumes,
        // the bulk kernel only the plain cells
        if ((e = cudaEventRecord(c->ev_wfork, c->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(c->wstream, c->ev_wfork, 0)) != cudaSuccess) return e;
        k_wall<T><<<cvgrid, 256, 0, c->wstream>>>(cv, bp, c->d_body, fin, c->wphi, c->wcontrib, c->ticket,
                                                   c->d_hist, moving ? 1 : 0, phase == 2 ? 2 : 0, xw);
        c->launches += 1;
    }
    BulkArgs<T> a{};
    a.g = g; a.S = c->S; a.Sin = Sin; a.fin = fin; a.fout = fout; a.pin = pin; a.pout = pout;
    a.flags = c->flags; a.vt = (const VCoef<T> *)c->vtab; a.gsign = c->gsign; a.err = c->d_err;
    a.pt = (const ulonglong2 *)c->ptab;
    a.eqp = cons && !imex ? (const T *)c->eqp : nullptr;
    a.qh = shak && !hraw ? (const T *)c->qheat : nullptr;
    a.hin = hraw ? (const T *)c->hpart[c->cur] : nullptr;
    a.hout = hkeep ? (T *)c->hpart[1 - c->cur] : nullptr;
    a.pr1 = T(1.0 - c->Pr);
    a.bits = c->rec_bits;
    a.bpitch = bits_pitch(c);
    a.bslab = bits_slab(c);
    if ((e = timing_mark(c, 0)) != cudaSuccess) return e;
    if (shak) e = c->scheme != DVM_MUSCL ? launch_bulk<T, false, false, true>(c, a) : launch_bulk<T, true, false, true>(c, a);
    else if (c->scheme != DVM_MUSCL) e = launch_bulk<T, false, false, false>(c, a);
    else e = c->rec_bits ? launch_bulk<T, true, true, false>(c, a) : launch_bulk<T, true, false, false>(c, a);
    if (e != cudaSuccess) return e;
    if ((e = timing_mark(c, 1)) != cudaSuccess) return e;
    c->launches += 1;
    if (body) {
        k_special<T><<<cvgrid, 256, 0, c->wstream>>>(cv, fin, fout, pin, pout, c->wphi);
        if ((e = cudaEventRecord(c->ev_wjoin, c->wstream)) != cudaSuccess) return e;
        // the step ends when both streams are done
        if ((e = cudaStreamWaitEvent(c->stream, c->ev_wjoin, 0)) != cudaSuccess) return e;
        c->launches += 1;
    }
    if (imex) {
        if (phase == 2) {
            // velocity split: this rank's moment sums of the transported
            // values; the ranks sum them before dvm_split_relax (phase 3)
            k_fold_partials<T><<<nblk(nc, 256), 256, 0, c->stream>>>(pout, c->S, nc, xbuf);
            c->launches += 1;
            return cudaGetLastError();
        }
        if ((e = imex_relax2d<T>(c, pout, c->S)) != cudaSuccess) return e;
    }
    return end_step2d(c, hkeep);
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return nullptr;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return encode;
}

// TMA descriptor of a buffer of limiter-branch words ([ngrp][ny + 4][pitch]
// uint32): one box is the block's tile (36 x 12 words) of one group.
int encode_bits_map2d(dvm_ctx *c, void *buf, CUtensorMap *map)
{
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) { set_error("cuTensorMapEncodeTiled is not available from the driver"); return DVM_ERR_CUDA; }
    const cuuint64_t dims[3] = {(cuuint64_t)bits_pitch(c), (cuuint64_t)(c->ny + 4), (cuuint64_t)c->ngrp};
    const cuuint64_t strides[2] = {(cuuint64_t)bits_pitch(c) * 4, (cuuint64_t)bits_slab(c) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kTileX, (cuuint32_t)kTileY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, buf, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return DVM_ERR_CUDA;
    }
    return DVM_OK;
}

// TMA descriptor of a state buffer in the device layout (any buffer with the
// layout of f[0], f[1]).
int encode_tensor_map2d(dvm_ctx *c, void *buf, CUtensorMap *map)
{
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) { set_error("cuTensorMapEncodeTiled is not available from the driver"); return DVM_ERR_CUDA; }
    const int W = c->W;
    const cuuint64_t dims[3] = {(cuuint64_t)(c->nx + 4) * W, (cuuint64_t)(c->ny + 4), (cuuint64_t)2 * c->ngrp};
    const cuuint64_t strides[2] = {(cuuint64_t)(c->nx + 4) * W * c->elem, (cuuint64_t)c->slab * W * c->elem};
    const cuuint32_t box[3] = {(cuuint32_t)kTileX * W, (cuuint32_t)kTileY, 2};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = c->prec == DVM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    CUresult r = encode(map, dt, 3, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return DVM_ERR_CUDA;
    }
    return DVM_OK;
}

// TMA descriptors of the two state buffers: a 3D view (x: padded cells of a
// row times the W velocities of a group, y: padded rows, z: group and
// component) of each slab; the box is the bulk kernel's tile with its halo.
int make_tensor_maps2d(dvm_ctx *c)
{
    for (int b = 0; b < 2; ++b) {
        const int rc = encode_tensor_map2d(c, c->f[b], &c->tmap[b]);
        if (rc != DVM_OK) return rc;
    }
    return DVM_OK;
}

size_t vcoef_bytes(int prec) { return prec == DVM_FP32 ? sizeof(VCoef<float>) : sizeof(VCoef<double>); }

size_t cvinfo_bytes() { return sizeof(CvInfo); }

cudaError_t members2d(dvm_ctx *c, bool moving)
{
    CvArgs cv{};
    cv.g = grid2d(c);
    cv.Gn = c->geo[c->gcur];
    cv.Gp = moving ? c->geo[1 - c->gcur] : c->geo[c->gcur];
    cv.master = c->master; cv.flags = c->flags; cv.wslot = c->wslot;
    cv.spec_list = c->spec_list; cv.counts = c->counts; cv.cap = c->list_cap;
    cv.err = c->d_err;
    k_members<<<4 * 152, 256, 0, c->stream>>>(cv, (CvInfo *)c->cvinfo);
    return cudaGetLastError();
}

// Fusion (Eq. FusionDD) of the state buffer f in place, moment sums into
// part (a scratch of S x 4 x nc elements).
cudaError_t fusion2d(dvm_ctx *c, void *f, void *part)
{
    CvArgs cv{};
    cv.g = grid2d(c);
    cv.Gn = c->geo[c->gcur];
    cv.Gp = c->geo[c->gcur];
    cv.master = c->master; cv.flags = c->flags;
    cv.spec_list = c->spec_list; cv.wall_list = c->wall_list; cv.wslot = c->wslot;
    cv.counts = c->counts; cv.cap = c->list_cap; cv.S = c->S;
    cv.gps = (c->ngrp + c->S - 1) / c->S;
    cv.cvinfo = c->cvinfo; cv.vt = c->vtab;
    cv.err = c->d_err;
    if (c->prec == DVM_FP32) k_fusion<float><<<4 * 152, 256, 0, c->stream>>>(cv, (float *)f, (float *)part);
    else k_fusion<double><<<4 * 152, 256, 0, c->stream>>>(cv, (double *)f, (double *)part);
    return cudaGetLastError();
}

cudaError_t step2d(dvm_ctx *c)
{
    return c->prec == DVM_FP32 ? step2d_t<float>(c, 0, nullptr) : step2d_t<double>(c, 0, nullptr);
}

// Velocity split: phase 1 (this rank's sums into xbuf), phase 2 (finish the
// step from xbuf summed over the ranks; semi-implicit scheme: the transport,
// and this rank's moment sums of the transported values into xbuf) or phase
// 3 (semi-implicit scheme: the relaxation from xbuf summed over the ranks).
cudaError_t split_step2d(dvm_ctx *c, int phase, void *xbuf)
{
    double *x = static_cast<double *>(xbuf);
    if (phase == 3) return c->prec == DVM_FP32 ? split_relax2d_t<float>(c, x) : split_relax2d_t<double>(c, x);
    return c->prec == DVM_FP32 ? step2d_t<float>(c, phase, x) : step2d_t<double>(c, phase, x);
}

cudaError_t tables2d(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    const int n = c->nvp > c->ngrp ? c->nvp : c->ngrp;
    if (c->prec == DVM_FP32)
        k_tables<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, (VCoef<float> *)c->vtab, c->gsign,
                                                              (float4 *)c->ptab);
    else
        k_tables<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, (VCoef<double> *)c->vtab, c->gsign,
                                                               (float4 *)c->ptab);
    return cudaGetLastError();
}

cudaError_t partials_from_state2d(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    const dim3 grid(nblk(c->nx, 32), c->ny), block(32, kMomChunks);
    if (c->prec == DVM_FP32)
        k_partials<float><<<grid, block, 0, c->stream>>>(g, c->S, (const float *)c->f[c->cur],
                                                         (const VCoef<float> *)c->vtab, (float *)c->part[c->cur],
                                                         c->geo[c->gcur].type, c->d_err);
    else
        k_partials<double><<<grid, block, 0, c->stream>>>(g, c->S, (const double *)c->f[c->cur],
                                                          (const VCoef<double> *)c->vtab, (double *)c->part[c->cur],
                                                          c->geo[c->gcur].type, c->d_err);
    return cudaGetLastError();
}

cudaError_t moments_out2d(dvm_ctx *c, double *d_out)
{
    Grid2D g = grid2d(c);
    const dim3 grid(nblk(c->nx, 32), c->ny), block(32, kMomChunks);
    if (c->prec == DVM_FP32)
        k_moments_out<float><<<grid, block, 0, c->stream>>>(g, (const float *)c->f[c->cur],
                                                            (const VCoef<float> *)c->vtab, d_out);
    else
        k_moments_out<double><<<grid, block, 0, c->stream>>>(g, (const double *)c->f[c->cur],
                                                             (const VCoef<double> *)c->vtab, d_out);
    return cudaGetLastError();
}

cudaError_t init_maxwellian2d(dvm_ctx *c, const double *d_prim)
{
    Grid2D g = grid2d(c);
    dim3 grid((unsigned)(c->nx * c->ny), nblk(c->nv, 256));
    if (c->prec == DVM_FP32)
        k_init<float><<<grid, 256, 0, c->stream>>>(g, d_prim, c->geo[c->gcur].type, (float *)c->f[c->cur]);
    else
        k_init<double><<<grid, 256, 0, c->stream>>>(g, d_prim, c->geo[c->gcur].type, (double *)c->f[c->cur]);
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
    dim3 grid((unsigned)(c->nx * c->ny), nblk(2 * c->nv, 256));
    if (c->prec == DVM_FP32)
        k_pack<float><<<grid, 256, 0, c->stream>>>(g, (const float *)pub, (float *)dev, 1);
    else
        k_pack<double><<<grid, 256, 0, c->stream>>>(g, (const double *)pub, (double *)dev, 1);
    return cudaGetLastError();
}

cudaError_t zero_solid2d(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    const dim3 grid(nblk((long)c->nx * c->ny, 256), 8);
    for (int b = 0; b < 2; ++b) {
        if (c->prec == DVM_FP32)
            k_zero_solid<float><<<grid, 256, 0, c->stream>>>(g, c->geo[c->gcur].type, (float *)c->f[b]);
        else
            k_zero_solid<double><<<grid, 256, 0, c->stream>>>(g, c->geo[c->gcur].type, (double *)c->f[b]);
    }
    return cudaGetLastError();
}

cudaError_t halo2d(dvm_ctx *c, int buf)
{
    Grid2D g = grid2d(c);
    const long n = 2 * 2L * (c->nx + c->ny) * 2 * c->nvp;
    if (c->prec == DVM_FP32) k_halo<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, (float *)c->f[buf]);
    else k_halo<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, (double *)c->f[buf]);
    return cudaGetLastError();
}

cudaError_t unpack2d(dvm_ctx *c, const void *dev, void *pub)
{
    Grid2D g = grid2d(c);
    dim3 grid((unsigned)(c->nx * c->ny), nblk(2 * c->nv, 256));
    if (c->prec == DVM_FP32)
        k_pack<float><<<grid, 256, 0, c->stream>>>(g, (const float *)dev, (float *)pub, 0);
    else
        k_pack<double><<<grid, 256, 0, c->stream>>>(g, (const double *)dev, (double *)pub, 0);
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
