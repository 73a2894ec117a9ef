// 3D time step of the cut-cell discrete-velocity method (arXiv:1503.04544,
// Sec. 5, Eq. eq-schema3D) for the full distribution F and a fixed obstacle:
// wall density and stress of the diffuse wall (3D forms of Eqs. BoundaryDDv
// and StressTensorDD), force and torque about the z axis, fluxes across the
// six Cartesian faces of every virtual cell (each direction with its own
// velocity component) and across its wall face, explicit update of each
// control volume with BGK relaxation toward the 3D Maxwellian, distribution
// to the members (Eq. UpdateDD).
//
// Device layout: element (cell, p) at (q * slab + P(i, j, k)) * W + e for the
// velocity group q and lane e of the padded velocity index (Grid3D), with
// P(i, j, k) = ((k + 2)(ny + 4) + j + 2)(nx + 4) + i + 2: every group is a
// slab of the grid padded by two cells on each side that holds the boundary
// condition, so a neighbour within two cells along an axis is a plain index.
//
// Kernels of one step: k_wall3 (FP64 wall density, force and torque; the
// last block sums them in list order), k_bulk3 (every gas cell that is a
// control volume on its own), k_special3 (cut and merged control volumes).
// k_bulk3 assigns one thread to a column of cells along z; a warp covers 32
// consecutive cells along x, so the velocity of a group (hence the upwind
// side along y and z) is uniform across the warp.  The velocity groups are
// split over blockIdx.z; each block streams the planes of its column through
// shared memory with TMA, writes the new state and accumulates the moments of
// the new state for the next step.
#include <cudaTypedefs.h>

#include <cstdio>
#include <string>

#include "dvm_device.cuh"

namespace dvm {
namespace {

constexpr int kCoef3 = 6;            // per-cell coefficients of the bulk kernel
constexpr int kCoef3S = 11;          // the same with the Shakhov model's five

template <typename T> struct alignas(2 * sizeof(T)) VX3 { T vx, nux; };
template <typename T> struct alignas(4 * sizeof(T)) VYZ3 { T vy, vz, nuy, nuz; };

// Slab index of cell (i, j, k), each within two cells of the grid.
__device__ __forceinline__ int nbr3(const Grid3D &g, int i, int j, int k)
{
    return ((k + 2) * (g.ny + 4) + (j + 2)) * (g.nx + 4) + (i + 2);
}

__device__ __forceinline__ void cell_ijk(const Grid3D &g, int q, int &i, int &j, int &k)
{
    const int r = q / g.nx;
    i = q - r * g.nx;
    k = r / g.ny;
    j = r - k * g.ny;
}

__device__ __forceinline__ int pcell3(const Grid3D &g, int q)
{
    int i, j, k;
    cell_ijk(g, q, i, j, k);
    return nbr3(g, i, j, k);
}

// Element offset of padded velocity p at slab index pc.
__device__ __forceinline__ long pidx3(const Grid3D &g, int p, int pc)
{
    const int grp = p / g.W;
    return ((long)grp * g.slab + pc) * g.W + (p - grp * g.W);
}

// Padded index of public velocity p = (p3 nvy + p2) nvx + p1.
__device__ __forceinline__ int padded3(const Grid3D &g, int p)
{
    const int r = p / g.nvx;
    return r * g.nvxp + (p - r * g.nvx);
}

// Padding cells that mirror interior cell (i, j, k) on periodic and
// zero-gradient sides (two per axis at most); -1 where unused.
__device__ __forceinline__ void mirrors3(const Grid3D &g, int i, int j, int k, int (&m)[6])
{
#pragma unroll
    for (int t = 0; t < 6; ++t) m[t] = -1;
    if (g.bc[0] == DVM_BC_PERIODIC) {
        if (i < 2) m[0] = nbr3(g, i + g.nx, j, k);
        else if (i >= g.nx - 2) m[0] = nbr3(g, i - g.nx, j, k);
    } else {
        if (i == 0 && g.bc[0] == DVM_BC_ZEROGRAD) { m[0] = nbr3(g, -1, j, k); m[1] = nbr3(g, -2, j, k); }
        if (i == g.nx - 1 && g.bc[1] == DVM_BC_ZEROGRAD) { m[0] = nbr3(g, g.nx, j, k); m[1] = nbr3(g, g.nx + 1, j, k); }
    }
    if (g.bc[2] == DVM_BC_PERIODIC) {
        if (j < 2) m[2] = nbr3(g, i, j + g.ny, k);
        else if (j >= g.ny - 2) m[2] = nbr3(g, i, j - g.ny, k);
    } else {
        if (j == 0 && g.bc[2] == DVM_BC_ZEROGRAD) { m[2] = nbr3(g, i, -1, k); m[3] = nbr3(g, i, -2, k); }
        if (j == g.ny - 1 && g.bc[3] == DVM_BC_ZEROGRAD) { m[2] = nbr3(g, i, g.ny, k); m[3] = nbr3(g, i, g.ny + 1, k); }
    }
    if (g.bc[4] == DVM_BC_PERIODIC) {
        if (k < 2) m[4] = nbr3(g, i, j, k + g.nz);
        else if (k >= g.nz - 2) m[4] = nbr3(g, i, j, k - g.nz);
    } else {
        if (k == 0 && g.bc[4] == DVM_BC_ZEROGRAD) { m[4] = nbr3(g, i, j, -1); m[5] = nbr3(g, i, j, -2); }
        if (k == g.nz - 1 && g.bc[5] == DVM_BC_ZEROGRAD) { m[4] = nbr3(g, i, j, g.nz); m[5] = nbr3(g, i, j, g.nz + 1); }
    }
}

__device__ __forceinline__ bool near_side3(const Grid3D &g, int i, int j, int k)
{
    return i < 2 || i >= g.nx - 2 || j < 2 || j >= g.ny - 2 || k < 2 || k >= g.nz - 2;
}

// Primitive variables from the sums s0 = sum F, s1..3 = sum v F,
// s4 = sum |v|^2/2 F (Eq. MacroscopicTD; T from E = rho|u|^2/2 + 3/2 rho T).
template <typename T>
__device__ __forceinline__ bool primitives3(T dv, const T (&s)[5], T &rho, T &ux, T &uy, T &uz, T &tmp)
{
    rho = s[0] * dv;
    ux = s[1] / s[0];
    uy = s[2] / s[0];
    uz = s[3] / s[0];
    tmp = (T(2) * (s[4] / s[0]) - (ux * ux + uy * uy + uz * uz)) / T(3);
    return rho > T(0) && tmp > T(0);
}

// Sum of the S partial moments of a cell ([S][5][nc] layout).
template <typename T>
__device__ __forceinline__ void gather_partials3(const T *part, int S, long nc, long cell, T (&s)[5])
{
    Acc<T> a[5];
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 5; ++m) a[m].merge(part[((long)q * 5 + m) * nc + cell], T(0));
#pragma unroll
    for (int m = 0; m < 5; ++m) s[m] = a[m].value();
}

// 1 / (2 pi T)^{3/2}
template <typename T>
__device__ __forceinline__ T norm3(T tmp)
{
    const T a = T(2.0 * kPi) * tmp;
    return T(1) / (a * sqrt(a));
}

// ------------------------------------------------------------ bulk kernel
template <typename T> struct Bulk3Args {
    Grid3D g;
    int S, nzc;
    int Sin;                  // partial-sum slots of pin (S, or 1 for summed moments of a velocity split)
    const T *fin;
    T *fout;
    const T *pin;             // partial moments of F^n   [S][5][nc]
    T *pout;                  // partial moments of F^n+1 [S][5][nc]
    const uint16_t *flags;
    const VX3<T> *vxt;        // [nvxp]
    const VYZ3<T> *vyz;       // [nvy * nvz]
    const T *eqp;             // [5][nc] conservative equilibrium parameters, or null (direct moments)
    const T *qh;              // [3][nc] heat flux of the control volume at t^n (Shakhov model)
    T pr1;                    // 1 - Pr (Shakhov model)
    int *err;
};

constexpr int kZc3 = 4;                           // z-planes per block column
constexpr int kRing3 = 8;                         // shared-memory planes in flight
constexpr int kPlaneX = 32 + 4;                   // tile width plus a two-cell halo

// Tile rows of the bulk kernel (one consumer warp each): 11 in FP32, so that
// with the producer warp the block's 12 warps put 3 on each SM sub-partition
// and a thread may hold up to 168 registers (it uses about 160, without
// spills; 12 rows would cap it at 128); 8 in FP64 (shared memory of the
// per-cell state).
template <typename T> __host__ __device__ constexpr int rows3() { return sizeof(T) == 4 ? 11 : 8; }
template <typename T> __host__ __device__ constexpr int plane_cells3() { return kPlaneX * (rows3<T>() + 4); }
// Ring slot stride in 16-byte cells: every slot is the destination of a
// tensor copy and starts on a 128-byte boundary.
template <typename T> __host__ __device__ constexpr int plane_stride3() { return (plane_cells3<T>() * 16 + 127) / 128 * 8; }

// Velocity tables staged in shared memory by the bulk kernel: all of v_x and
// up to kVyzStage (v_y, v_z) pairs (more are read from global memory).
constexpr int kVyzStage = 512;

template <typename T, bool SHAK>
size_t bulk3_smem()
{
    const int ncoef = SHAK ? kCoef3S : kCoef3;
    return (size_t)kRing3 * plane_stride3<T>() * 16 + (size_t)kZc3 * (ncoef + 10) * 32 * rows3<T>() * sizeof(T) +
           2 * kRing3 * sizeof(uint64_t) + (size_t)kMaxAxisNv * sizeof(VX3<T>) + (size_t)kVyzStage * sizeof(VYZ3<T>);
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z, int w)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// Flux difference along one axis in units of the Courant number on a full gas
// cell (Eq. eq-schema3D), with the neighbours taken on the upwind side:
// a = F - F_up plus the limited reconstructions of the outgoing and incoming
// faces; ko, ki are (1 - nu)/2 where the face stencil is all gas, else 0.
template <typename T, bool MUSCL>
__device__ __forceinline__ T dflux(T f, T u1, T u2, T d1, T ko, T ki)
{
    const T a = f - u1;
    if (!MUSCL) return a;
    T mo, mi;
    minmod_pair(d1 - f, a, u1 - u2, mo, mi);
    return fma(-ki, mi, fma(ko, mo, a));
}

// 2^x in the state precision: the hardware approximation in FP32.
__device__ __forceinline__ float exp2_state(float x) { return ex2_fast(x); }
__device__ __forceinline__ double exp2_state(double x) { return exp2(x); }

// Bulk update of every gas cell that is a control volume on its own.
//
// Block = a tile of 32 x R cells in (x, y) and a column of kZc3 cells in z
// (blockIdx.z = split * nzc + column), R consumer warps (one per tile row)
// and one producer warp.  For each velocity group of its split the producer
// streams the kZc3 + 4 planes of the column (tile plus a two-cell halo, one
// TMA load each) into a ring of kRing3 shared-memory stages, refilling a stage
// once every consumer warp has released it.  The consumers march up the
// column: x/y neighbours come from the plane's stage; along z the cell values,
// their differences and the face value at z + 1/2 (the z - 1/2 face of the
// next cell) roll through registers.  Every wait is bounded and records
// kErrTimeout instead of blocking.  The neighbours of a group are taken on its
// upwind side (uniform within a group along y and z, and along x except for
// the group that contains v_x = 0).  Moments of the new state are summed per
// cell in registers over 8 groups, then folded into compensated sums in
// shared memory.
// With SHAK (the Shakhov model, FP32) the cells relax towards F_S = M [1 +
// k c.q (|c|^2/T - 5)], k = (1 - Pr) / (5 rho T^2), with the heat flux q of
// the cell at t^n from k_heatflux3: |c|^2/T from the Maxwellian's base-2
// exponent and k c.q linear in v, four operations per velocity.
template <typename T, bool MUSCL, bool SHAK>
__global__ void __launch_bounds__(32 * (rows3<T>() + 1), 1)
    k_bulk3(Bulk3Args<T> a, const __grid_constant__ CUtensorMap tmap)
{
    static_assert(!SHAK || sizeof(T) == 4, "the Shakhov variant of the bulk kernel is FP32");
    constexpr int W = Vec<T>::W, ZC = kZc3, R = rows3<T>(), NT = 32 * R, NP = ZC + 4;
    constexpr int NCO = SHAK ? kCoef3S : kCoef3;
    constexpr int PC = plane_stride3<T>(), PB = plane_cells3<T>() * 16;
    static_assert((PC * 16) % 128 == 0, "tensor-copy destinations start on 128-byte boundaries");
    using V = typename Vec<T>::type;
    extern __shared__ __align__(128) unsigned char sm3[];
    V *ring = reinterpret_cast<V *>(sm3);
    T *coef = reinterpret_cast<T *>(sm3 + kRing3 * PC * 16);        // [ZC][NCO][NT]
    T *ksum = coef + ZC * NCO * NT;                                  // [ZC][5][2][NT]
    uint64_t *full = reinterpret_cast<uint64_t *>(ksum + ZC * 10 * NT);
    uint64_t *empty = full + kRing3;
    VX3<T> *svx = reinterpret_cast<VX3<T> *>(empty + kRing3);          // [kMaxAxisNv]
    VYZ3<T> *svyz = reinterpret_cast<VYZ3<T> *>(svx + kMaxAxisNv);       // [kVyzStage]
    const Grid3D &g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const bool producer = ty == R;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * R;
    const int i = i0 + tx, j = j0 + ty;
    const int zc = blockIdx.z % a.nzc, split = blockIdx.z / a.nzc;
    const int z0 = zc * ZC;
    const long nc = (long)g.nx * g.ny * g.nz;
    const int gps = (g.ngrp + a.S - 1) / a.S;
    const int g0 = split * gps, g1 = min(g0 + gps, g.ngrp);
    const int ngr = max(g1 - g0, 0);
    const int total = ngr * NP;
    const bool inij = !producer && i < g.nx && j < g.ny;
    const int sz = (g.nx + 4) * (g.ny + 4);

    if (tid == 0) {
        for (int st = 0; st < kRing3; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], R);
        }
        mbar_fence_init();
    }
    // the velocity tables of the groups, staged once per block
    const int nyz = g.nvy * g.nvz;
    const bool stage_yz = nyz <= kVyzStage;
    for (int q = tid; q < g.nvxp; q += blockDim.x * blockDim.y) svx[q] = a.vxt[q];
    if (stage_yz)
        for (int q = tid; q < nyz; q += blockDim.x * blockDim.y) svyz[q] = a.vyz[q];
    const VX3<T> *vxtab = svx;
    const VYZ3<T> *vyztab = stage_yz ? svyz : a.vyz;
    // per-cell data of the column: flags, and for plain cells the
    // equilibrium in the form log2 M(v) = c0 + vx (c1 - c2 vx) - c2 dyz(v)
    uint32_t plainm = 0, zerom = 0, mirm = 0, masks = 0;   // masks: byte t = limiter mask of cell t
    static_assert(ZC <= 4, "one mask byte per column cell");
    if (!producer) {
#pragma unroll
        for (int t = 0; t < ZC; ++t) {
            const int k = z0 + t;
            const bool in = inij && k < g.nz;
            const long cell = ((long)k * g.ny + j) * g.nx + i;
            const uint16_t fl = in ? a.flags[cell] : 0;
            T *cz = coef + t * NCO * NT + tid;
            if (fl & kPlain) {
                plainm |= 1u << t;
                T s[5];
                gather_partials3(a.pin, a.Sin, nc, cell, s);
                T rho, ux, uy, uz, tmp;
                if (!primitives3<T>(pick<T>(g.dv_f, g.dv), s, rho, ux, uy, uz, tmp)) atomicExch(&a.err[kErrNonphys], 1);
                cz[5 * NT] = pick<T>(g.dt_tau0_f, g.dt_tau0) * rho;
                if (a.eqp) {
                    // conservative equilibrium (Sec. 3.1): tau from the direct
                    // density, the Maxwellian from the Newton parameters
                    rho = a.eqp[cell]; ux = a.eqp[nc + cell]; uy = a.eqp[2 * nc + cell];
                    uz = a.eqp[3 * nc + cell]; tmp = a.eqp[4 * nc + cell];
                }
                const T c2 = T(kLog2e) / (T(2) * tmp);
                cz[0] = log2(rho * norm3(tmp)) - c2 * ux * ux;
                cz[NT] = T(2) * c2 * ux;
                cz[2 * NT] = c2;
                cz[3 * NT] = uy;
                cz[4 * NT] = uz;
                if constexpr (SHAK) {
                    // k q, -k u.q and 2 log2(A) / log2(e) - 5
                    const T kk = a.pr1 / (T(5) * rho * tmp * tmp);
                    const T kqx = kk * a.qh[cell], kqy = kk * a.qh[nc + cell], kqz = kk * a.qh[2 * nc + cell];
                    cz[6 * NT] = kqx;
                    cz[7 * NT] = kqy;
                    cz[8 * NT] = kqz;
                    cz[9 * NT] = -(kqx * ux + kqy * uy + kqz * uz);
                    cz[10 * NT] = T(2.0 / kLog2e) * log2(rho * norm3(tmp)) - T(5);
                }
            }
            if (fl & kZero) zerom |= 1u << t;
            masks |= (uint32_t)((fl >> kMaskShift3) & 0x3F) << (8 * t);
            if (in && near_side3(g, i, j, k)) mirm |= 1u << t;
#pragma unroll
            for (int m = 0; m < 10; ++m) ksum[(t * 10 + m) * NT + tid] = T(0);
        }
    }
    __syncthreads();

    if (producer) {
        if (tx == 0) {
            for (int s = 0; s < total; ++s) {
                const int slot = s % kRing3;
                if (s >= kRing3 && !mbar_wait(&empty[slot], (uint32_t)(((s / kRing3) - 1) & 1)))
                    atomicExch(&a.err[kErrTimeout], 1);
                mbar_expect_tx(&full[slot], PB);
                const int gi = s / NP, o = s - gi * NP;
                // plane z0 - 2 + o of the column, padded index z0 + o
                tma_load_4d(ring + slot * PC, &tmap, &full[slot], i0 * W, j0, z0 + o, g0 + gi);
            }
            // every issued copy has landed before the block exits
            for (int s = max(total - kRing3, 0); s < total; ++s)
                mbar_wait(&full[s % kRing3], (uint32_t)((s / kRing3) & 1));
        }
        return;
    }

    const int c0 = (ty + 2) * kPlaneX + tx + 2;
    const int pc0 = inij ? nbr3(g, i, j, z0) : 0;
    auto wait_full = [&](int s) -> const V * {
        const int slot = s % kRing3;
        if (!mbar_wait(&full[slot], (uint32_t)((s / kRing3) & 1))) atomicExch(&a.err[kErrTimeout], 1);
        return ring + slot * PC;
    };
    auto release = [&](int s) {
        __syncwarp();
        if (tx == 0) mbar_arrive(&empty[s % kRing3]);
    };

    T q[ZC][5];
#pragma unroll
    for (int t = 0; t < ZC; ++t)
#pragma unroll
        for (int m = 0; m < 5; ++m) q[t][m] = T(0);
    int fold = 0;
    V *const fout = reinterpret_cast<V *>(a.fout);
    for (int gi = 0; gi < ngr; ++gi) {
        const int grp = g0 + gi;
        const int yz = grp / g.nxg, xg = grp - yz * g.nxg;
        const VYZ3<T> cyz = vyztab[yz];
        T vx[W], nux[W], kx[W];
        bool xpos = true, xneg = true;
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const VX3<T> cx = vxtab[xg * W + e];
            vx[e] = cx.vx;
            nux[e] = cx.nux;
            kx[e] = T(0.5) * (T(1) - cx.nux);
            xpos = xpos && cx.vx >= T(0);
            xneg = xneg && cx.vx <= T(0);
        }
        const bool xuni = xpos || xneg;
        const int ox = xpos ? 1 : -1;
        const bool py = cyz.vy >= T(0), pz = cyz.vz >= T(0);
        const int oy = py ? kPlaneX : -kPlaneX;
        const T ky = T(0.5) * (T(1) - cyz.nuy), kz = T(0.5) * (T(1) - cyz.nuz);
        const T nzs = pz ? cyz.nuz : -cyz.nuz;
        const T vyz2 = cyz.vy * cyz.vy + cyz.vz * cyz.vz;
        V *dst = fout + (long)grp * g.slab;
        const int base = gi * NP;
        // rolling window along z: f at z - 1, z, z + 1 and the differences
        // d(z - 1/2) = f(z) - f(z - 1), d(z + 1/2)
        T fm1[W], f0[W], fp1[W], dm[W], dp[W], phim[W];
        {
            T fm2[W];
            sld<T>(wait_full(base) + c0, fm2);
            sld<T>(wait_full(base + 1) + c0, fm1);
            sld<T>(wait_full(base + 2) + c0, f0);
            sld<T>(wait_full(base + 3) + c0, fp1);
            release(base);
            release(base + 1);
            // face value at z0 - 1/2
            const T kw = (masks & 16u) ? kz : T(0);
#pragma unroll
            for (int e = 0; e < W; ++e) {
                dm[e] = f0[e] - fm1[e];
                dp[e] = fp1[e] - f0[e];
            }
            if (!MUSCL) {
#pragma unroll
                for (int e = 0; e < W; ++e) phim[e] = pz ? fm1[e] : f0[e];
            } else if (pz) {
#pragma unroll
                for (int e = 0; e < W; ++e) phim[e] = fma(kw, minmod3(dm[e], fm1[e] - fm2[e]), fm1[e]);
            } else {
#pragma unroll
                for (int e = 0; e < W; ++e) phim[e] = fma(-kw, minmod3(dp[e], dm[e]), f0[e]);
            }
        }
#pragma unroll
        for (int t = 0; t < ZC; ++t) {
            // the plane of z was waited for as the z + 2 centre two steps ago
            const V *pl = ring + ((base + t + 2) % kRing3) * PC;
            T fp2[W];
            sld<T>(wait_full(base + t + 4) + c0, fp2);
            const uint32_t mk = (masks >> (8 * t)) & 0x3Fu;
            // face value at z + 1/2, the z - 1/2 face of the next cell
            T phip[W], dpp[W];
#pragma unroll
            for (int e = 0; e < W; ++e) dpp[e] = fp2[e] - fp1[e];
            if (!MUSCL) {
#pragma unroll
                for (int e = 0; e < W; ++e) phip[e] = pz ? f0[e] : fp1[e];
            } else {
                const T kw = (mk & 32u) ? kz : T(0);
                if (pz) {
#pragma unroll
                    for (int e = 0; e < W; ++e) phip[e] = fma(kw, minmod3(dp[e], dm[e]), f0[e]);
                } else {
#pragma unroll
                    for (int e = 0; e < W; ++e) phip[e] = fma(-kw, minmod3(dpp[e], dp[e]), fp1[e]);
                }
            }
            const bool pl_t = (plainm >> t) & 1u;
            if (pl_t || ((zerom >> t) & 1u)) {
                T out[W];
                if (pl_t) {
                    const T *cz = coef + t * NCO * NT + tid;
                    const T c0c = cz[0], c1 = cz[NT], c2 = cz[2 * NT], uy = cz[3 * NT], uz = cz[4 * NT], r = cz[5 * NT];
                    const T dyv = cyz.vy - uy, dzv = cyz.vz - uz;
                    const T cg = c0c - c2 * (dyv * dyv + dzv * dzv);
                    // Shakhov: k c.q = kqx vx + (kqy vy + kqz vz - k u.q)
                    T kqx = 0, kyz = 0, l5 = 0;
                    if constexpr (SHAK) {
                        kqx = cz[6 * NT];
                        kyz = fma(cz[7 * NT], cyz.vy, fma(cz[8 * NT], cyz.vz, cz[9 * NT]));
                        l5 = cz[10 * NT];
                    }
                    const T omr = T(1) - r;
                    const T kyo = (mk & (py ? 8u : 4u)) ? ky : T(0), kyi = (mk & (py ? 4u : 8u)) ? ky : T(0);
                    T yu1[W], yu2[W], yd1[W];
                    sld<T>(pl + c0 - oy, yu1);
                    if (MUSCL) {
                        sld<T>(pl + c0 - 2 * oy, yu2);
                        sld<T>(pl + c0 + oy, yd1);
                    }
                    T dfx[W];
                    if (xuni) {
                        const T xo = (mk & (xpos ? 2u : 1u)) ? T(1) : T(0), xi = (mk & (xpos ? 1u : 2u)) ? T(1) : T(0);
                        T xu1[W], xu2[W], xd1[W];
                        sld<T>(pl + c0 - ox, xu1);
                        if (MUSCL) {
                            sld<T>(pl + c0 - 2 * ox, xu2);
                            sld<T>(pl + c0 + ox, xd1);
                        }
#pragma unroll
                        for (int e = 0; e < W; ++e)
                            dfx[e] = dflux<T, MUSCL>(f0[e], xu1[e], MUSCL ? xu2[e] : T(0), MUSCL ? xd1[e] : T(0),
                                                     xo * kx[e], xi * kx[e]);
                    } else {
                        T xm1[W], xp1[W], xm2[W], xp2[W];
                        sld<T>(pl + c0 - 1, xm1);
                        sld<T>(pl + c0 + 1, xp1);
                        if (MUSCL) {
                            sld<T>(pl + c0 - 2, xm2);
                            sld<T>(pl + c0 + 2, xp2);
                        }
                        const T kxm = (mk & 1u) ? T(1) : T(0), kxp = (mk & 2u) ? T(1) : T(0);
#pragma unroll
                        for (int e = 0; e < W; ++e) {
                            const bool px = vx[e] >= T(0);
                            dfx[e] = dflux<T, MUSCL>(f0[e], px ? xm1[e] : xp1[e], MUSCL ? (px ? xm2[e] : xp2[e]) : T(0),
                                                     px ? xp1[e] : xm1[e], kx[e] * (px ? kxp : kxm),
                                                     kx[e] * (px ? kxm : kxp));
                        }
                    }
                    T s = 0, sx = 0, sxx = 0;
#pragma unroll
                    for (int e = 0; e < W; ++e) {
                        const T dfy = dflux<T, MUSCL>(f0[e], yu1[e], MUSCL ? yu2[e] : T(0), MUSCL ? yd1[e] : T(0), kyo, kyi);
                        const T xe = fma(fma(-c2, vx[e], c1), vx[e], cg);
                        T feq = exp2_state(xe);
                        if constexpr (SHAK) {
                            // |c|^2/T - 5 = 2 (log2 A - log2 M) / log2 e - 5
                            const T mk5 = feq * fma(kqx, vx[e], kyz);
                            feq = fma(mk5, fma(T(-2.0 / kLog2e), xe, l5), feq);
                        }
                        T o = fma(r, feq, omr * f0[e]);
                        o = fma(-nux[e], dfx[e], o);
                        o = fma(-cyz.nuy, dfy, o);
                        o = fma(-nzs, phip[e] - phim[e], o);     // nzs carries the sign of v_z
                        out[e] = o;
                        s += o;
                        sx = fma(vx[e], o, sx);
                        sxx = fma(vx[e] * vx[e], o, sxx);
                    }
                    q[t][0] += s;
                    q[t][1] += sx;
                    q[t][2] = fma(cyz.vy, s, q[t][2]);
                    q[t][3] = fma(cyz.vz, s, q[t][3]);
                    q[t][4] += T(0.5) * fma(vyz2, s, sxx);
                } else {
#pragma unroll
                    for (int e = 0; e < W; ++e) out[e] = T(0);
                }
                const int pc = pc0 + t * sz;
                vst<T>(dst + pc, out);
                if ((mirm >> t) & 1u) {
                    int mir[6];
                    mirrors3(g, i, j, z0 + t, mir);
#pragma unroll
                    for (int u = 0; u < 6; ++u)
                        if (mir[u] >= 0) vst<T>(dst + mir[u], out);
                }
            }
#pragma unroll
            for (int e = 0; e < W; ++e) {
                phim[e] = phip[e];
                dm[e] = dp[e];
                dp[e] = dpp[e];
                fm1[e] = f0[e];
                f0[e] = fp1[e];
                fp1[e] = fp2[e];
            }
            release(base + t + 2);
        }
        release(base + ZC + 2);
        release(base + ZC + 3);
        // fold the plain sums of 8 groups into the compensated sums
        if (++fold == 8 || gi + 1 == ngr) {
            fold = 0;
#pragma unroll
            for (int t = 0; t < ZC; ++t)
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    T *ks = ksum + (t * 10 + 2 * m) * NT + tid;
                    Acc<T> acc;
                    acc.s = ks[0];
                    acc.c = ks[NT];
                    acc.add(q[t][m]);
                    ks[0] = acc.s;
                    ks[NT] = acc.c;
                    q[t][m] = T(0);
                }
        }
    }
#pragma unroll
    for (int t = 0; t < ZC; ++t) {
        if (!(((plainm | zerom) >> t) & 1u)) continue;
        const long cell = ((long)(z0 + t) * g.ny + j) * g.nx + i;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const T *ks = ksum + (t * 10 + 2 * m) * NT + tid;
            a.pout[((long)split * 5 + m) * nc + cell] = ks[0] - ks[NT];
        }
    }
}

// ------------------------------------------------------------ control volumes
struct Cv3Args {
    Grid3D g;
    Geo3D G;
    const int32_t *master;
    const uint16_t *flags;
    const int32_t *spec_list;
    const int32_t *wall_list;
    const int32_t *wslot;
    const int32_t *counts;
    int cap;
    int S;
    int Sin;                  // partial-sum slots of the moments read (S, or 1 for summed moments)
    int gps;
    const void *cvinfo;
    const void *vxt;
    const void *vyz;
    const void *eqp;          // [5][nc] conservative equilibrium parameters, or null
    const void *qh;           // [3][nc] heat flux of the control volume at t^n (Shakhov model, FP32), or null
    double pr1;               // 1 - Pr (Shakhov model)
    int *err;
};

// One member (virtual cell) of a control volume.
struct __align__(16) CvMember3 {
    int pc;                   // slab index
    int mir[6];               // padding mirrors (-1: none)
    int cell;                 // cell index
    int wslot;                // wall slot, -1 if none
    int mask;                 // limiter mask of the six faces
    int live;                 // non-solid (fixed obstacle: always)
    int pad;
    double A[6];              // face areas x-, x+, y-, y+, z-, z+
    double sw, nwx, nwy, nwz; // wall face (sw = 0: none)
    double vol;
};

struct __align__(16) CvInfo3 {
    int nm, ok, pcm, pad;
    double bco;               // dt / S (fixed obstacle: S^n = S^{n+1,*})
    double S;
    CvMember3 mem[kMaxMembers3];
};

// Ordered members of control volume m (cells whose master is m) within the
// window reachable by the master search.
__device__ int gather_members3(const Cv3Args &c, int m, int32_t *mem)
{
    __shared__ int wcnt[8];
    const Grid3D &g = c.g;
    const int R = kMaxWalk, Wd = 2 * kMaxWalk + 1, npos = Wd * Wd * Wd;
    int mi, mj, mk;
    cell_ijk(g, m, mi, mj, mk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int total = 0;
    for (int base = 0; base < npos; base += 32 * nw) {
        const int pos = base + warp * 32 + lane;
        bool hit = false;
        int ii = 0, jj = 0, kk = 0;
        if (pos < npos) {
            ii = mi - R + pos % Wd;
            jj = mj - R + (pos / Wd) % Wd;
            kk = mk - R + pos / (Wd * Wd);
            if (ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny && kk >= 0 && kk < g.nz)
                hit = c.master[((long)kk * g.ny + jj) * g.nx + ii] == m;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = total;
        for (int w = 0; w < warp; ++w) off += wcnt[w];
        const int rank = off + __popc(bal & ((1u << lane) - 1u));
        if (hit) {
            if (rank < kMaxMembers3) mem[rank] = (kk * g.ny + jj) * g.nx + ii;
            else atomicExch(&c.err[kErrCapacity], 1);
        }
        int add = 0;
        for (int w = 0; w < nw; ++w) add += wcnt[w];
        total += add;
        __syncthreads();
    }
    return total < kMaxMembers3 ? total : kMaxMembers3;
}

// Members are listed in z-major order of the window; the fixed order keeps
// the sums deterministic.  Sorting is not needed: the order only has to be
// the same on every call.
__global__ void __launch_bounds__(256) k_members3(Cv3Args c, CvInfo3 *info)
{
    __shared__ int32_t mem[kMaxMembers3];
    const Grid3D &g = c.g;
    const int n = min(c.counts[0], c.cap);
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const int m = c.spec_list[idx];
        const int nm = gather_members3(c, m, mem);
        CvInfo3 &I = info[idx];
        if (threadIdx.x < nm) {
            const int q = mem[threadIdx.x];
            CvMember3 &M = I.mem[threadIdx.x];
            int i, j, k;
            cell_ijk(g, q, i, j, k);
            M.cell = q;
            M.pc = nbr3(g, i, j, k);
            mirrors3(g, i, j, k, M.mir);
            const long xf = ((long)k * g.ny + j) * (g.nx + 1) + i;
            const long yf = ((long)k * (g.ny + 1) + j) * g.nx + i;
            const long zf = ((long)k * g.ny + j) * g.nx + i;
            M.A[0] = c.G.ax[xf]; M.A[1] = c.G.ax[xf + 1];
            M.A[2] = c.G.ay[yf]; M.A[3] = c.G.ay[yf + g.nx];
            M.A[4] = c.G.az[zf]; M.A[5] = c.G.az[zf + (long)g.nx * g.ny];
            M.wslot = c.wslot[q];
            const bool wall = M.wslot >= 0;
            M.sw = wall ? c.G.sw[q] : 0.0;
            M.nwx = c.G.nwx[q]; M.nwy = c.G.nwy[q]; M.nwz = c.G.nwz[q];
            M.vol = c.G.vol[q];
            M.mask = (c.flags[q] >> kMaskShift3) & 0x3F;
            M.live = c.G.type[q] != DVM_SOLID;
            M.pad = 0;
            if (q == m) I.pcm = M.pc;
        }
        if (threadIdx.x == 0) {
            double S = 0;
            for (int t = 0; t < nm; ++t) S += c.G.vol[mem[t]];
            I.nm = nm;
            I.ok = S > 0;
            I.S = S;
            I.bco = S > 0 ? g.dt / S : 0.0;
            I.pad = 0;
            if (!(S > 0)) atomicExch(&c.err[kErrGeometry], 1);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void load_info3(const CvInfo3 *src, CvInfo3 *dst)
{
    static_assert(sizeof(CvInfo3) % 16 == 0, "CvInfo3 is copied in 16-byte words");
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int q = threadIdx.x; q < (int)(sizeof(CvInfo3) / 16); q += blockDim.x) d4[q] = __ldg(s4 + q);
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T face_flux3(T L, T v, T nu, T fAA, T fA, T fB, T fBB, bool muscl)
{
    if (!muscl) return L * (fmin(v, T(0)) * fB + fmax(v, T(0)) * fA);
    T fr;
    if (v > T(0)) fr = fA + T(0.5) * (T(1) - nu) * minmod(fB - fA, fA - fAA);
    else if (v < T(0)) fr = fB - T(0.5) * (T(1) - nu) * minmod(fBB - fB, fB - fA);
    else return T(0);
    return L * (v * fr);
}

template <typename T>
__device__ __forceinline__ void write_split_partials3(T *part, int s, long nc, long k, const T (&t)[5])
{
#pragma unroll
    for (int m = 0; m < 5; ++m) part[((long)s * 5 + m) * nc + k] = t[m];
}

// Velocity of padded index p from the tables.
template <typename T>
__device__ __forceinline__ void vel3(const Grid3D &g, const VX3<T> *vxt, const VYZ3<T> *vyz, int p, T &vx, T &vy,
                                     T &vz, T &nux, T &nuy, T &nuz)
{
    const int grp = p / g.W, e = p - grp * g.W;
    const int yz = grp / g.nxg;
    const VX3<T> cx = vxt[(grp - yz * g.nxg) * g.W + e];
    const VYZ3<T> c = vyz[yz];
    vx = cx.vx; nux = cx.nux;
    vy = c.vy; vz = c.vz; nuy = c.nuy; nuz = c.nuz;
}

// Fusion (3D form of Eq. FusionDD): F_CV = sum vol F / S over a merged
// control volume, written back to every member, with the moment sums.  One
// work item is one control volume and one velocity split.
template <typename T>
__global__ void __launch_bounds__(256) k_fusion3(Cv3Args c, T *f, T *part)
{
    __shared__ T red[8 * 2];
    const Grid3D &g = c.g;
    const CvInfo3 *info = reinterpret_cast<const CvInfo3 *>(c.cvinfo);
    const VX3<T> *vxt = reinterpret_cast<const VX3<T> *>(c.vxt);
    const VYZ3<T> *vyz = reinterpret_cast<const VYZ3<T> *>(c.vyz);
    const long nc = (long)g.nx * g.ny * g.nz;
    const int n = min(c.counts[0], c.cap) * c.S;
    for (int item = blockIdx.x; item < n; item += gridDim.x) {
        const CvInfo3 &I = info[item / c.S];
        const int sp = item % c.S;
        const int nm = I.nm;
        if (nm <= 1) continue;
        const int v0 = sp * c.gps * g.W, v1 = min(g.nvp, v0 + c.gps * g.W);
        const double S = I.S;
        Acc<T> a[5];
        for (int p = v0 + threadIdx.x; p < v1; p += blockDim.x) {
            double acc = 0;
            for (int t = 0; t < nm; ++t) acc += I.mem[t].vol * (double)f[pidx3(g, p, I.mem[t].pc)];
            const T fcv = (T)(acc / S);
            for (int t = 0; t < nm; ++t) {
                f[pidx3(g, p, I.mem[t].pc)] = fcv;
                for (int u = 0; u < 6; ++u)
                    if (I.mem[t].mir[u] >= 0) f[pidx3(g, p, I.mem[t].mir[u])] = fcv;
            }
            T vx, vy, vz, nux, nuy, nuz;
            vel3(g, vxt, vyz, p, vx, vy, vz, nux, nuy, nuz);
            a[0].add(fcv); a[1].add(vx * fcv); a[2].add(vy * fcv); a[3].add(vz * fcv);
            a[4].add(T(0.5) * (vx * vx + vy * vy + vz * vz) * fcv);
        }
        T t[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) t[m] = block_acc(a[m], red);
        if (threadIdx.x < nm) write_split_partials3<T>(part, sp, nc, I.mem[threadIdx.x].cell, t);
        __syncthreads();
    }
}

// Wall density phi (zero net mass flux across the wall face), stress
// Sigma = sum (v - u_w)(v - u_w)^T F_w dv and the force Sigma n_w S_w on the
// body (3D forms of Eqs. BoundaryDDv, StressTensorDD, eq-force), torque about
// the z axis through the centre (Eq. eq-torque), u_w = u_c + omega e_z x
// (r - c) (Eq. uwDD).  One block per wall cell: products and compensated sums
// in the state precision over all velocities, phi and the stress in FP64 by
// thread 0.  The last block sums the cells in list order into the body
// record and the history.  (phi, u_w, T_w) of each wall cell are left for
// the control-volume kernel.
template <typename T>
// mode 0: the whole wall step; a velocity split runs mode 1 (this rank's 14
// sums of every wall cell into xw[14 * slot], FP64) and, after the caller's
// sum over the ranks, mode 2 (the rest from the summed values).
__global__ void __launch_bounds__(256) k_wall3(Cv3Args c, BodyParams b, BodyDev *body, const T *f, double *wdat,
                                               double *wcontrib, int *ticket, double *hist, int mode, double *xw)
{
    __shared__ double red[8 * 8];
    __shared__ T ex[kMaxAxisNv], ey[kMaxAxisNv], ez[kMaxAxisNv];
    __shared__ T wsc[8];
    __shared__ T wred[8 * 2];
    __shared__ bool last;
    const Grid3D &g = c.g;
    const VX3<T> *vxt = reinterpret_cast<const VX3<T> *>(c.vxt);
    const VYZ3<T> *vyz = reinterpret_cast<const VYZ3<T> *>(c.vyz);
    const int nw = min(c.counts[1], c.cap);
    const double omega = body->omega;
    const int tid = threadIdx.x;
    for (int idx = blockIdx.x; idx < nw; idx += gridDim.x) {
        const int q = c.wall_list[idx];
        const double rx = c.G.rwx[q] - b.cx, ry = c.G.rwy[q] - b.cy;
        const double uwx = b.vbx - ry * omega, uwy = b.vby + rx * omega, uwz = 0.0;
        double rr[14];
        if (mode == 2) {
#pragma unroll
            for (int t = 0; t < 14; ++t) rr[t] = xw[14L * idx + t];
        } else {
        if (tid == 0) {
            wsc[0] = (T)uwx; wsc[1] = (T)uwy; wsc[2] = (T)uwz;
            wsc[3] = (T)c.G.nwx[q]; wsc[4] = (T)c.G.nwy[q]; wsc[5] = (T)c.G.nwz[q];
            wsc[6] = (T)(2.0 * b.Tw);
            const double a2 = 2.0 * kPi * b.Tw;
            wsc[7] = (T)(1.0 / (a2 * sqrt(a2)));
        }
        __syncthreads();
        const T ux = wsc[0], uy = wsc[1], uz = wsc[2], nx = wsc[3], ny = wsc[4], nz = wsc[5], twoTw = wsc[6];
        const T cm = wsc[7];
        // separable Maxwellian M[1, u_w, T_w] = cm ex[p1] ey[p2] ez[p3]
        for (int t = tid; t < g.nvx + g.nvy + g.nvz; t += blockDim.x) {
            if (t < g.nvx) { const T d = vxt[t].vx - ux; ex[t] = dexp(-(d * d) / twoTw); }
            else if (t < g.nvx + g.nvy) {
                const int p2 = t - g.nvx;
                const T d = vyz[p2].vy - uy;
                ey[p2] = dexp(-(d * d) / twoTw);
            } else {
                const int p3 = t - g.nvx - g.nvy;
                const T d = vyz[p3 * g.nvy].vz - uz;
                ez[p3] = dexp(-(d * d) / twoTw);
            }
        }
        __syncthreads();
        const int pc = pcell3(g, q);
        // a[0] = sum_{c>0} c F, a[1] = sum_{c<0} c M, a[2..7] = sum_{c<0} (v-u_w)(v-u_w) M,
        // a[8..13] = sum_{c>0} (v-u_w)(v-u_w) F   (xx, xy, xz, yy, yz, zz)
        Acc<T> a[14];
        for (int p = tid; p < g.nv; p += blockDim.x) {
            const int p1 = p % g.nvx, r = p / g.nvx;
            const int p3 = r / g.nvy, p2 = r - p3 * g.nvy;
            const T vx = vxt[p1].vx, vy = vyz[r].vy, vz = vyz[r].vz;
            const T ax = vx - ux, ay = vy - uy, az = vz - uz;
            const T cp = ax * nx + ay * ny + az * nz;
            if (cp > T(0)) {
                const T fv = f[pidx3(g, r * g.nvxp + p1, pc)];
                a[0].add(cp * fv);
                a[8].add(ax * ax * fv); a[9].add(ax * ay * fv); a[10].add(ax * az * fv);
                a[11].add(ay * ay * fv); a[12].add(ay * az * fv); a[13].add(az * az * fv);
            } else if (cp < T(0)) {
                const T m1 = cm * ex[p1] * ey[p2] * ez[p3];
                a[1].add(cp * m1);
                a[2].add(ax * ax * m1); a[3].add(ax * ay * m1); a[4].add(ax * az * m1);
                a[5].add(ay * ay * m1); a[6].add(ay * az * m1); a[7].add(az * az * m1);
            }
        }
#pragma unroll
        for (int t = 0; t < 14; ++t) rr[t] = (double)block_acc(a[t], wred);
        if (mode == 1) {
            if (tid == 0)
#pragma unroll
                for (int t = 0; t < 14; ++t) xw[14L * idx + t] = rr[t];
            __syncthreads();
            continue;
        }
        }
        if (tid == 0) {
            const double dv = g.dv;
            const double phi = -(rr[0] * dv) / (rr[1] * dv);
            double S6[6];
            for (int t = 0; t < 6; ++t) S6[t] = (phi * rr[2 + t] + rr[8 + t]) * dv;
            const double nxd = c.G.nwx[q], nyd = c.G.nwy[q], nzd = c.G.nwz[q], sw = c.G.sw[q];
            const double fx = (S6[0] * nxd + S6[1] * nyd + S6[2] * nzd) * sw;
            const double fy = (S6[1] * nxd + S6[3] * nyd + S6[4] * nzd) * sw;
            const double fz = (S6[2] * nxd + S6[4] * nyd + S6[5] * nzd) * sw;
            double *wc = wcontrib + 4L * idx;
            wc[0] = fx; wc[1] = fy; wc[2] = fz; wc[3] = rx * fy - ry * fx;
            double *d = wdat + 6L * idx;
            d[0] = phi; d[1] = uwx; d[2] = uwy; d[3] = uwz; d[4] = b.Tw; d[5] = 0;
        }
        __syncthreads();
    }
    if (mode == 1) return;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double fx = 0, fy = 0, fz = 0, tq = 0;
    for (int t = tid; t < nw; t += blockDim.x) {
        fx += wcontrib[4 * t]; fy += wcontrib[4 * t + 1]; fz += wcontrib[4 * t + 2]; tq += wcontrib[4 * t + 3];
    }
    fx = block_sum(fx, red); fy = block_sum(fy, red + 8); fz = block_sum(fz, red + 16); tq = block_sum(tq, red + 24);
    if (tid == 0) {
        body->F[0] = fx; body->F[1] = fy; body->F[2] = fz; body->torque = tq;
        double *h = hist + 6 * (body->step % kHistCap);
        h[0] = fx; h[1] = fy; h[2] = fz; h[3] = tq; h[4] = body->theta; h[5] = body->omega;
        body->step += 1;
        *ticket = 0;
    }
}

// Explicit update of one control volume (Eq. eq-schema3D): fluxes across the
// six faces of every member and across its wall face with the diffuse state
// F_w = phi M[1, u_w, T_w] on incoming velocities, relaxation, distribution
// to the members and the moment sums of the velocity split.  One work item is
// one control volume and one split.
template <typename T>
__global__ void __launch_bounds__(256) k_special3(Cv3Args c, const T *fin, T *fout, const T *pin, T *pout,
                                                  const double *wdat)
{
    __shared__ T red[8 * 2];
    __shared__ __align__(16) CvInfo3 I;
    const Grid3D &g = c.g;
    const CvInfo3 *info = reinterpret_cast<const CvInfo3 *>(c.cvinfo);
    const VX3<T> *vxt = reinterpret_cast<const VX3<T> *>(c.vxt);
    const VYZ3<T> *vyz = reinterpret_cast<const VYZ3<T> *>(c.vyz);
    const long nc = (long)g.nx * g.ny * g.nz;
    const int n = min(c.counts[0], c.cap) * c.S;
    const int sy = g.nx + 4, sz = (g.nx + 4) * (g.ny + 4);
    for (int item = blockIdx.x; item < n; item += gridDim.x) {
        const int idx = item / c.S, sp = item % c.S;
        load_info3(info + idx, &I);
        if (!I.ok) { __syncthreads(); continue; }
        const int nm = I.nm;
        const int v0 = sp * c.gps * g.W, v1 = min(g.nvp, v0 + c.gps * g.W);
        const int m = c.spec_list[idx];
        T s[5];
        gather_partials3(pin, c.Sin, nc, m, s);
        T rho, ux, uy, uz, tmp;
        if (!primitives3<T>(pick<T>(g.dv_f, g.dv), s, rho, ux, uy, uz, tmp) && threadIdx.x == 0 && sp == 0)
            atomicExch(&c.err[kErrNonphys], 1);
        const T bco = (T)I.bco, r = pick<T>(g.dt_tau0_f, g.dt_tau0) * rho;
        if (c.eqp) {
            const T *e = static_cast<const T *>(c.eqp);
            rho = e[m]; ux = e[nc + m]; uy = e[2 * nc + m]; uz = e[3 * nc + m]; tmp = e[4 * nc + m];
        }
        const T A = rho * norm3(tmp);
        const T i2T = T(1) / (T(2) * tmp);
        // Shakhov (Sec. 2.1): k q with the heat flux of the control volume
        T kqx = 0, kqy = 0, kqz = 0;
        if (c.qh) {
            const T *qh = static_cast<const T *>(c.qh);
            const T kk = T(c.pr1) / (T(5) * rho * tmp * tmp);
            kqx = kk * qh[m];
            kqy = kk * qh[nc + m];
            kqz = kk * qh[2 * nc + m];
        }
        Acc<T> acc[5];
        for (int p = v0 + threadIdx.x; p < v1; p += blockDim.x) {
            T vx, vy, vz, nux, nuy, nuz;
            vel3(g, vxt, vyz, p, vx, vy, vz, nux, nuy, nuz);
            const int grp = p / g.W, e = p - grp * g.W;
            const T *fg = fin + (long)grp * g.slab * g.W + e;     // element of slab index s: fg[s * W]
            const int Wd = g.W;
            T R = 0;
            for (int t = 0; t < nm; ++t) {
                const CvMember3 &M = I.mem[t];
                if (!M.live) continue;
                const int pc = M.pc;
                const T fc = fg[(long)pc * Wd];
                T Fw = 0;
                if (M.wslot >= 0) {
                    const double *d = wdat + 6L * M.wslot;
                    const T phi = (T)d[0], uwx = (T)d[1], uwy = (T)d[2], uwz = (T)d[3], Tw = (T)d[4];
                    const T ax = vx - uwx, ay = vy - uwy, az = vz - uwz;
                    const T cw = ax * (T)M.nwx + ay * (T)M.nwy + az * (T)M.nwz;
                    const T m1 = dexp(-(ax * ax + ay * ay + az * az) / (T(2) * Tw)) * norm3(Tw);
                    Fw = (T)M.sw * (fmin(cw, T(0)) * (phi * m1) + fmax(cw, T(0)) * fc);
                }
                const bool mxm = M.mask & 1, mxp = M.mask & 2, mym = M.mask & 4, myp = M.mask & 8;
                const bool mzm = M.mask & 16, mzp = M.mask & 32;
                const T xm1 = fg[(long)(pc - 1) * Wd], xp1 = fg[(long)(pc + 1) * Wd];
                const T ym1 = fg[(long)(pc - sy) * Wd], yp1 = fg[(long)(pc + sy) * Wd];
                const T zm1 = fg[(long)(pc - sz) * Wd], zp1 = fg[(long)(pc + sz) * Wd];
                T xm2 = 0, xp2 = 0, ym2 = 0, yp2 = 0, zm2 = 0, zp2 = 0;
                if (M.mask) {
                    xm2 = fg[(long)(pc - 2) * Wd]; xp2 = fg[(long)(pc + 2) * Wd];
                    ym2 = fg[(long)(pc - 2 * sy) * Wd]; yp2 = fg[(long)(pc + 2 * sy) * Wd];
                    zm2 = fg[(long)(pc - 2 * sz) * Wd]; zp2 = fg[(long)(pc + 2 * sz) * Wd];
                }
                const T Fxp = face_flux3<T>((T)M.A[1], vx, nux, xm1, fc, xp1, xp2, mxp);
                const T Fxm = face_flux3<T>((T)M.A[0], vx, nux, xm2, xm1, fc, xp1, mxm);
                const T Fyp = face_flux3<T>((T)M.A[3], vy, nuy, ym1, fc, yp1, yp2, myp);
                const T Fym = face_flux3<T>((T)M.A[2], vy, nuy, ym2, ym1, fc, yp1, mym);
                const T Fzp = face_flux3<T>((T)M.A[5], vz, nuz, zm1, fc, zp1, zp2, mzp);
                const T Fzm = face_flux3<T>((T)M.A[4], vz, nuz, zm2, zm1, fc, zp1, mzm);
                R += (Fxp - Fxm) + (Fyp - Fym) + (Fzp - Fzm) + Fw;
            }
            const T fcv = fg[(long)I.pcm * Wd];
            const T dxu = vx - ux, dyu = vy - uy, dzu = vz - uz;
            const T c2u = dxu * dxu + dyu * dyu + dzu * dzu;
            T feq = A * dexp(-c2u * i2T);
            if (c.qh) feq *= fma(kqx * dxu + kqy * dyu + kqz * dzu, c2u * T(2) * i2T - T(5), T(1));
            const T fn = fcv - bco * R + r * (feq - fcv);
            T *og = fout + (long)grp * g.slab * g.W + e;
            for (int t = 0; t < nm; ++t) {
                const CvMember3 &M = I.mem[t];
                og[(long)M.pc * Wd] = fn;
                for (int u = 0; u < 6; ++u)
                    if (M.mir[u] >= 0) og[(long)M.mir[u] * Wd] = fn;
            }
            acc[0].add(fn); acc[1].add(vx * fn); acc[2].add(vy * fn); acc[3].add(vz * fn);
            acc[4].add(T(0.5) * (vx * vx + vy * vy + vz * vz) * fn);
        }
        T t5[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) t5[q] = block_acc(acc[q], red);
        if (threadIdx.x < nm) write_split_partials3<T>(pout, sp, nc, I.mem[threadIdx.x].cell, t5);
        __syncthreads();
    }
}

// ------------------------------------------------------------ state services
// Moment sums of cells (i, j, k) of one x-row over a chunk of the velocity
// groups: F, v_x F, v_y F, v_z F and |v|^2/2 F (Eq. MacroscopicTD), per
// group plain over its lanes and compensated across groups.  The lanes of a
// warp are 32 consecutive cells, so each group's vector of the 32 cells is
// one coalesced read; warp threadIdx.y takes the threadIdx.y-th of
// kMomChunks chunks.
template <typename T>
__device__ __forceinline__ void state_sums3d(const Grid3D &g, const T *f, const VX3<T> *vxt, const VYZ3<T> *vyz,
                                             int i, int j, int k, Acc<T> (&s)[5])
{
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    if (i >= g.nx) return;
    const int gps = (g.ngrp + kMomChunks - 1) / kMomChunks;
    const int q0 = threadIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    if (q0 >= q1) return;
    const long pc = nbr3(g, i, j, k);
    const V *fv = reinterpret_cast<const V *>(f);
    int r = q0 / g.nxg, xg = q0 - r * g.nxg;
    for (int q = q0; q < q1; ++q) {
        T a[W];
        vld<T>(fv + (long)q * g.slab + pc, a);
        T t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const int p1 = xg * W + e;
            if (p1 >= g.nvx) continue;
            const T vx = vxt[p1].vx;
            t0 += a[e];
            t1 += vx * a[e];
            t2 += vx * vx * a[e];
        }
        const VYZ3<T> cy = vyz[r];
        s[0].add(t0);
        s[1].add(t1);
        s[2].add(cy.vy * t0);
        s[3].add(cy.vz * t0);
        s[4].add(T(0.5) * fma(cy.vy * cy.vy + cy.vz * cy.vz, t0, t2));
        if (++xg == g.nxg) {
            xg = 0;
            ++r;
        }
    }
}

// Partial moment sums of a state (set-up, not the time step): the whole sum
// goes to split 0, zeros to the others and to solid cells.
template <typename T>
__global__ void __launch_bounds__(32 * kMomChunks) k_partials3(Grid3D g, int S, const T *f, const VX3<T> *vxt,
                                                               const VYZ3<T> *vyz, T *part, const int8_t *type,
                                                               int *err)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    Acc<T> s[5];
    state_sums3d<T>(g, f, vxt, vyz, i, j, k, s);
    merge_chunks<T, 5>(s);
    if (threadIdx.y != 0 || i >= g.nx) return;
    const long nc = (long)g.nx * g.ny * g.nz, cell = ((long)k * g.ny + j) * g.nx + i;
    const bool keep = type[cell] != DVM_SOLID;
    T v[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) v[m] = keep ? s[m].value() : T(0);
    if (keep) {
        T rho, ux, uy, uz, tmp;
        if (!primitives3<T>(pick<T>(g.dv_f, g.dv), v, rho, ux, uy, uz, tmp)) atomicExch(&err[kErrNonphys], 1);
    }
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 5; ++m) part[((long)q * 5 + m) * nc + cell] = q == 0 ? v[m] : T(0);
}

// Moments for output: rho, ux, uy, uz, T per cell, formed in FP64 from the
// sums (compensated in the state precision).
template <typename T>
__global__ void __launch_bounds__(32 * kMomChunks) k_moments_out3(Grid3D g, const T *f, const VX3<T> *vxt,
                                                                  const VYZ3<T> *vyz, double *out)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    Acc<T> s[5];
    state_sums3d<T>(g, f, vxt, vyz, i, j, k, s);
    merge_chunks<T, 5>(s);
    if (threadIdx.y != 0 || i >= g.nx) return;
    double *o5 = out + (((long)k * g.ny + j) * g.nx + i) * 5;
    double d[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) d[m] = (double)s[m].s - (double)s[m].c;
    const double rho = d[0] * g.dv;
    if (!(rho > 0)) {
        for (int q = 0; q < 5; ++q) o5[q] = 0;
        return;
    }
    const double ux = d[1] * g.dv / rho, uy = d[2] * g.dv / rho, uz = d[3] * g.dv / rho;
    o5[0] = rho; o5[1] = ux; o5[2] = uy; o5[3] = uz;
    o5[4] = (2.0 * (d[4] * g.dv) / rho - (ux * ux + uy * uy + uz * uz)) / 3.0;
}

// Implicit relaxation of the semi-implicit scheme (Eq. ImpSchemeDD) in 3D,
// after a transport pass without relaxation: every gas cell relaxes towards
// the Maxwellian of the moments of its transported values (mom, Smom slots:
// this context's partial sums, or those summed over the ranks of a velocity
// split), F = (F* + nu M) / (1 + nu) with nu = (dt / tau0) rho, in place and
// in its padding mirrors; the partial sums part become those of this
// context's relaxed values.
// Block = 32 consecutive cells of an x-row x kMomChunks warps, one chunk of
// the velocity groups each.
template <typename T, bool SHAK>
__global__ void __launch_bounds__(32 * kMomChunks) k_imex3(Grid3D g, int S, T dt_tau0, T *f, const VX3<T> *vxt,
                                                           const VYZ3<T> *vyz, const T *mom, int Smom, T *part,
                                                           const int8_t *type, const T *eqp, T Pr, int *err)
{
    // SHAK: the Shakhov model (Sec. 2.1) with the heat flux at t^{n+1},
    // q = q_T / (1 + nu Pr), q_T = sum c |c|^2/2 F dv of the transported
    // values; F_S = M [1 + (1 - Pr) c.q (|c|^2/T - 5) / (5 rho T^2)]
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    __shared__ T qsh[3][32];
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const long nc = (long)g.nx * g.ny * g.nz, cell = ((long)k * g.ny + j) * g.nx + i;
    bool gas = i < g.nx && type[cell] != DVM_SOLID;
    T s[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (gas) gather_partials3(mom, Smom, nc, cell, s);
    T rho = 0, ux = 0, uy = 0, uz = 0, tmp = 0;
    if (gas && !primitives3<T>(pick<T>(g.dv_f, g.dv), s, rho, ux, uy, uz, tmp)) {
        if (threadIdx.y == 0) atomicExch(&err[kErrNonphys], 1);
        gas = false;
    }
    Acc<T> a5[5];
    const int gps = (g.ngrp + kMomChunks - 1) / kMomChunks;
    const int q0 = threadIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    const long pc = nbr3(g, i, j, k);
    V *fv = reinterpret_cast<V *>(f);
    T qx = 0, qy = 0, qz = 0;
    if constexpr (SHAK) {
        Acc<T> hq[3];
        if (gas) {
            int r = q0 / g.nxg, xg = q0 - r * g.nxg;
            for (int q = q0; q < q1; ++q) {
                T a[W];
                vld<T>(fv + (long)q * g.slab + pc, a);
                const VYZ3<T> cy = vyz[r];
                const T dy = cy.vy - uy, dz = cy.vz - uz, dyz = dy * dy + dz * dz;
                T t0 = 0, t1 = 0;
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    const int p1 = xg * W + e;
                    if (p1 >= g.nvx) continue;
                    const T dx = vxt[p1].vx - ux, w = T(0.5) * (dx * dx + dyz) * a[e];
                    t0 += dx * w;
                    t1 += w;
                }
                hq[0].add(t0);
                hq[1].add(dy * t1);
                hq[2].add(dz * t1);
                if (++xg == g.nxg) {
                    xg = 0;
                    ++r;
                }
            }
        }
        merge_chunks<T, 3>(hq);
        if (threadIdx.y == 0) {
            const T rel = pick<T>(g.dv_f, g.dv) / (T(1) + dt_tau0 * rho * Pr);
#pragma unroll
            for (int d = 0; d < 3; ++d) qsh[d][threadIdx.x] = hq[d].value() * rel;
        }
        __syncthreads();
        qx = qsh[0][threadIdx.x];
        qy = qsh[1][threadIdx.x];
        qz = qsh[2][threadIdx.x];
    }
    if (gas && q0 < q1) {
        const T nu = dt_tau0 * rho, inv = T(1) / (T(1) + nu);
        if (eqp) {
            // conservative equilibrium of the transported state (Sec. 3.1)
            rho = eqp[cell]; ux = eqp[nc + cell]; uy = eqp[2 * nc + cell]; uz = eqp[3 * nc + cell];
            tmp = eqp[4 * nc + cell];
        }
        const T A = rho * norm3(tmp), c2 = T(kLog2e) / (T(2) * tmp);
        const T kk = SHAK ? (T(1) - Pr) / (T(5) * rho * tmp * tmp) : T(0), iT = T(1) / tmp;
        int mir[6];
        mirrors3(g, i, j, k, mir);
        int r = q0 / g.nxg, xg = q0 - r * g.nxg;
#pragma unroll 2
        for (int q = q0; q < q1; ++q) {
            V *pa = fv + (long)q * g.slab;
            T a[W];
            vld<T>(pa + pc, a);
            const VYZ3<T> cy = vyz[r];
            const T dyz = (cy.vy - uy) * (cy.vy - uy) + (cy.vz - uz) * (cy.vz - uz);
            const T hyz = kk * ((cy.vy - uy) * qy + (cy.vz - uz) * qz);
            T t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const int p1 = xg * W + e;
                if (p1 >= g.nvx) continue;
                const T vx = vxt[p1].vx, dx = vx - ux;
                T M = A * exp2_state(-(dx * dx + dyz) * c2);
                if constexpr (SHAK) M *= T(1) + (kk * dx * qx + hyz) * ((dx * dx + dyz) * iT - T(5));
                a[e] = (a[e] + nu * M) * inv;
                t0 += a[e];
                t1 += vx * a[e];
                t2 += vx * vx * a[e];
            }
            vst<T>(pa + pc, a);
#pragma unroll
            for (int m = 0; m < 6; ++m)
                if (mir[m] >= 0) vst<T>(pa + mir[m], a);
            a5[0].add(t0);
            a5[1].add(t1);
            a5[2].add(cy.vy * t0);
            a5[3].add(cy.vz * t0);
            a5[4].add(T(0.5) * fma(cy.vy * cy.vy + cy.vz * cy.vz, t0, t2));
            if (++xg == g.nxg) {
                xg = 0;
                ++r;
            }
        }
    }
    merge_chunks<T, 5>(a5);
    if (threadIdx.y != 0 || i >= g.nx) return;
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 5; ++m) part[((long)q * 5 + m) * nc + cell] = (q == 0 && gas) ? a5[m].value() : T(0);
}

__device__ __forceinline__ double maxw3(const double *q, double vx, double vy, double vz)
{
    const double ax = vx - q[1], ay = vy - q[2], az = vz - q[3];
    const double a2 = 2.0 * kPi * q[4];
    return q[0] / (a2 * sqrt(a2)) * exp(-(ax * ax + ay * ay + az * az) / (2.0 * q[4]));
}

// Maxwellian state from per-cell primitives (rho, ux, uy, uz, T); solid cells
// get 0.  One block row per cell, threads over the public velocities.
template <typename T>
__global__ void k_init3(Grid3D g, const double *prim, const int8_t *type, T *f)
{
    const int q = blockIdx.x;
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    if (p >= g.nv) return;
    const int p1 = p % g.nvx, r = p / g.nvx;
    const int p3 = r / g.nvy, p2 = r - p3 * g.nvy;
    const double *s = prim + 5L * q;
    double m = 0;
    if (type[q] != DVM_SOLID && s[0] > 0)
        m = maxw3(s, g.vxmin + p1 * g.dvx, g.vymin + p2 * g.dvy, g.vzmin + p3 * g.dvz);
    f[pidx3(g, r * g.nvxp + p1, pcell3(g, q))] = (T)m;
}

// Ghost cells of a Maxwellian side (both layers, both state buffers).
template <typename T>
__global__ void k_ghost3(Grid3D g, const double *prim, int side, int nside, T *f0, T *f1)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nside * g.nv) return;
    const int q = (int)(t / g.nv), p = (int)(t % g.nv);
    const int p1 = p % g.nvx, r = p / g.nvx;
    const int p3 = r / g.nvy, p2 = r - p3 * g.nvy;
    const double m = maxw3(prim + 5L * q, g.vxmin + p1 * g.dvx, g.vymin + p2 * g.dvy, g.vzmin + p3 * g.dvz);
    // side cell q: row-major over the two remaining axes
    int a, b;
    if (side < 2) { a = q % g.ny; b = q / g.ny; }          // (j, k)
    else if (side < 4) { a = q % g.nx; b = q / g.nx; }     // (i, k)
    else { a = q % g.nx; b = q / g.nx; }                   // (i, j)
    const int pp = r * g.nvxp + p1;
    for (int layer = 1; layer <= 2; ++layer) {
        int pc;
        if (side == 0) pc = nbr3(g, -layer, a, b);
        else if (side == 1) pc = nbr3(g, g.nx - 1 + layer, a, b);
        else if (side == 2) pc = nbr3(g, a, -layer, b);
        else if (side == 3) pc = nbr3(g, a, g.ny - 1 + layer, b);
        else if (side == 4) pc = nbr3(g, a, b, -layer);
        else pc = nbr3(g, a, b, g.nz - 1 + layer);
        f0[pidx3(g, pp, pc)] = (T)m;
        f1[pidx3(g, pp, pc)] = (T)m;
    }
}

// Padding of periodic and zero-gradient sides from the interior (both
// layers, every padded velocity).
template <typename T>
__global__ void k_halo3(Grid3D g, T *f)
{
    const long fx = (long)g.ny * g.nz, fy = (long)g.nx * g.nz, fz = (long)g.nx * g.ny;
    const long per = 2 * (fx + fy + fz);      // padding cells of one layer
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * per * g.nvp) return;
    const long hc = t % (2 * per);
    const int p = (int)(t / (2 * per));
    const int layer = (int)(hc / per) + 1;
    long pos = hc % per;
    int side;
    if (pos < 2 * fx) { side = pos < fx ? 0 : 1; pos = pos % fx; }
    else if (pos < 2 * fx + 2 * fy) { pos -= 2 * fx; side = pos < fy ? 2 : 3; pos = pos % fy; }
    else { pos -= 2 * fx + 2 * fy; side = pos < fz ? 4 : 5; pos = pos % fz; }
    const int kind = g.bc[side];
    if (kind == DVM_BC_MAXWELLIAN) return;
    const bool per_ = kind == DVM_BC_PERIODIC;
    int di, dj, dk, si, sj, sk;
    if (side < 2) {
        const int j = (int)(pos % g.ny), k = (int)(pos / g.ny);
        dj = sj = j; dk = sk = k;
        if (side == 0) { di = -layer; si = per_ ? g.nx - layer : 0; }
        else { di = g.nx - 1 + layer; si = per_ ? layer - 1 : g.nx - 1; }
    } else if (side < 4) {
        const int i = (int)(pos % g.nx), k = (int)(pos / g.nx);
        di = si = i; dk = sk = k;
        if (side == 2) { dj = -layer; sj = per_ ? g.ny - layer : 0; }
        else { dj = g.ny - 1 + layer; sj = per_ ? layer - 1 : g.ny - 1; }
    } else {
        const int i = (int)(pos % g.nx), j = (int)(pos / g.nx);
        di = si = i; dj = sj = j;
        if (side == 4) { dk = -layer; sk = per_ ? g.nz - layer : 0; }
        else { dk = g.nz - 1 + layer; sk = per_ ? layer - 1 : g.nz - 1; }
    }
    f[pidx3(g, p, nbr3(g, di, dj, dk))] = f[pidx3(g, p, nbr3(g, si, sj, sk))];
}

// Conversion between the public layout [cell][p] and the device layout.
template <typename T>
__global__ void k_pack3(Grid3D g, const T *src, T *dst, int to_dev)
{
    const int q = blockIdx.x;
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    if (p >= g.nv) return;
    const long t = (long)q * g.nv + p;
    const long d = pidx3(g, padded3(g, p), pcell3(g, q));
    if (to_dev) dst[d] = src[t];
    else dst[t] = src[d];
}

// Zero the state of every solid cell: one thread per cell and chunk of the
// velocity groups (blockIdx.y); only the threads of solid cells store.
template <typename T>
__global__ void k_zero_solid3(Grid3D g, const int8_t *type, T *f)
{
    using V = typename Vec<T>::type;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long)g.nx * g.ny * g.nz || type[k] != DVM_SOLID) return;
    const int gps = (g.ngrp + gridDim.y - 1) / gridDim.y;
    const int q0 = blockIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    const long pc = pcell3(g, (int)k);
    V *fv = reinterpret_cast<V *>(f);
    const T z[Vec<T>::W] = {};
    for (int q = q0; q < q1; ++q) vst<T>(fv + (long)q * g.slab + pc, z);
}

template <typename T>
__global__ void __launch_bounds__(256) k_mass_cells3(Grid3D g, const T *f, const double *vol, double *cm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= (long)g.nx * g.ny * g.nz) return;
    double s = 0;
    const int pc = pcell3(g, (int)cell);
    for (int p = lane; p < g.nvp; p += 32) s += (double)f[pidx3(g, p, pc)];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) cm[cell] = vol[cell] * (s * g.dv);
}

__global__ void __launch_bounds__(1024) k_sum3(const double *x, long n, double *out)
{
    __shared__ double red[32];
    double s = 0;
    for (long t = threadIdx.x; t < n; t += blockDim.x) s += x[t];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

template <typename T>
__global__ void k_tables3(Grid3D g, VX3<T> *vxt, VYZ3<T> *vyz)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < g.nvxp) {
        VX3<T> c;
        if (t < g.nvx) {
            c.vx = T(g.vxmin + t * g.dvx);
            c.nux = fabs(c.vx) * T(g.dt / g.dx);
        } else {
            c.vx = T(1e4);      // padding: zero state, vanishing equilibrium
            c.nux = 0;
        }
        vxt[t] = c;
    }
    if (t < g.nvy * g.nvz) {
        const int p2 = t % g.nvy, p3 = t / g.nvy;
        VYZ3<T> c;
        c.vy = T(g.vymin + p2 * g.dvy);
        c.vz = T(g.vzmin + p3 * g.dvz);
        c.nuy = fabs(c.vy) * T(g.dt / g.dy);
        c.nuz = fabs(c.vz) * T(g.dt / g.dz);
        vyz[t] = c;
    }
}

inline unsigned nb3(long n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T>
const VX3<T> *vx_table(const dvm_ctx *c) { return reinterpret_cast<const VX3<T> *>(c->vtab); }

template <typename T>
const VYZ3<T> *vyz_table(const dvm_ctx *c)
{
    return reinterpret_cast<const VYZ3<T> *>(reinterpret_cast<const char *>(c->vtab) + (size_t)c->nvxp * sizeof(VX3<T>));
}

template <typename T, bool MUSCL, bool SHAK>
cudaError_t launch_bulk3(dvm_ctx *c, const Bulk3Args<T> &a)
{
    const size_t smem = bulk3_smem<T, SHAK>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_bulk3<T, MUSCL, SHAK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(nb3(c->nx, 32), nb3(c->ny, rows3<T>()), (unsigned)(a.nzc * a.S)), block(32, rows3<T>() + 1);
    k_bulk3<T, MUSCL, SHAK><<<grid, block, smem, c->stream>>>(a, c->tmap[c->cur]);
    return cudaGetLastError();
}

// The bulk kernel for the scheme, and its Shakhov variant in FP32.
template <typename T>
cudaError_t launch_bulk3_any(dvm_ctx *c, const Bulk3Args<T> &a, bool shak)
{
    if constexpr (sizeof(T) == 4) {
        if (shak) return c->scheme == DVM_MUSCL ? launch_bulk3<T, true, true>(c, a) : launch_bulk3<T, false, true>(c, a);
    }
    return c->scheme == DVM_MUSCL ? launch_bulk3<T, true, false>(c, a) : launch_bulk3<T, false, false>(c, a);
}

Cv3Args cv3_args(dvm_ctx *c)
{
    Cv3Args cv{};
    cv.g = grid3d(c);
    cv.G = c->geo3;
    cv.master = c->master; cv.flags = c->flags3;
    cv.spec_list = c->spec_list; cv.wall_list = c->wall_list; cv.wslot = c->wslot;
    cv.counts = c->counts; cv.cap = c->list_cap; cv.S = c->S; cv.Sin = c->S;
    cv.gps = (c->ngrp + c->S - 1) / c->S;
    cv.cvinfo = c->cvinfo;
    cv.vxt = c->vtab;
    cv.vyz = reinterpret_cast<const char *>(c->vtab) + (size_t)c->nvxp * 2 * c->elem;
    cv.err = c->d_err;
    return cv;
}

// Moment sums of each cell over this context's velocities, folded over the
// S velocity splits in fixed order, in FP64 (the data a velocity split
// exchanges, Sec. 5.2).
template <typename T>
__global__ void k_fold_partials3(const T *part, int S, long nc, double *x)
{
    const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= nc) return;
    T s[5];
    gather_partials3(part, S, nc, cell, s);
#pragma unroll
    for (int m = 0; m < 5; ++m) x[(long)m * nc + cell] = (double)s[m];
}

template <typename T>
__global__ void k_unfold_partials3(const double *x, long n, T *part)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) part[t] = (T)x[t];
}

// The bookkeeping that ends a step: the new state is the current one.
cudaError_t end_step3d(dvm_ctx *c)
{
    c->cur = 1 - c->cur;
    c->need_fusion = false;
    c->steps_done++;
    return cudaGetLastError();
}

// The relaxation of the semi-implicit scheme (Eq. ImpSchemeDD) on the
// transported values f[1 - cur], with their moments from mom (Smom slots).
template <typename T>
cudaError_t imex_relax3d(dvm_ctx *c, const T *mom, int Smom)
{
    const Grid3D g = grid3d(c);
    T *fout = (T *)c->f[1 - c->cur], *pout = (T *)c->part[1 - c->cur];
    const bool cons = c->eq_mode == DVM_EQ_CONSERVATIVE;
    const dim3 grid(nb3(c->nx, 32), c->ny, c->nz), block(32, kMomChunks);
    cudaError_t e;
    // conservative equilibrium parameters of the transported state
    if (cons && (e = eqpar(c, mom, Smom)) != cudaSuccess) return e;
    if (c->model == DVM_SHAKHOV)
        k_imex3<T, true><<<grid, block, 0, c->stream>>>(g, c->S, T(c->dt / c->tau0), fout, vx_table<T>(c),
                                                        vyz_table<T>(c), mom, Smom, pout, c->geo3.type, nullptr,
                                                        T(c->Pr), c->d_err);
    else
        k_imex3<T, false><<<grid, block, 0, c->stream>>>(g, c->S, T(c->dt / c->tau0), fout, vx_table<T>(c),
                                                         vyz_table<T>(c), mom, Smom, pout, c->geo3.type,
                                                         cons ? (const T *)c->eqp : nullptr, T(1), c->d_err);
    c->launches += 1;
    return cudaGetLastError();
}

// One step in phases, as in 2D: 0 the whole step; a velocity split runs
// phase 1 (this rank's moment sums [5][nc] and wall sums [wall slot][14]
// into the FP64 buffer xbuf) and phase 2 (the rest, from xbuf summed over
// the ranks).  Under the semi-implicit scheme phase 2 ends with this rank's
// moment sums of the transported values in xbuf ([5][nc]) and phase 3 takes
// them summed over the ranks and relaxes.
template <typename T>
cudaError_t step3d_t(dvm_ctx *c, int phase, double *xbuf)
{
    Grid3D g = grid3d(c);
    // the semi-implicit scheme (Eq. ImpSchemeDD) transports without
    // relaxation here; k_imex3 relaxes at the end of the step
    const bool imex = c->time_scheme == DVM_IMEX;
    if (imex) {
        g.dt_tau0 = 0.0;
        g.dt_tau0_f = 0.f;
    }
    const BodyParams bp = body_params(c);
    const bool body = c->body.shape != DVM_SHAPE_NONE;
    const long nc = (long)c->nc;
    T *fin = (T *)c->f[c->cur], *fout = (T *)c->f[1 - c->cur];
    T *pin = (T *)c->part[c->cur], *pout = (T *)c->part[1 - c->cur];
    cudaError_t e;
    Cv3Args cv = cv3_args(c);
    cv.g = g;                 // without the relaxation rate for the semi-implicit scheme
    const bool cons = c->eq_mode == DVM_EQ_CONSERVATIVE;
    cv.eqp = cons && !imex ? c->eqp : nullptr;
    const int cvgrid = 4 * 152;
    double *xw = xbuf ? xbuf + 5 * nc : nullptr;
    if (phase != 2) {
        if (body && c->need_fusion) {
            k_fusion3<T><<<cvgrid, 256, 0, c->stream>>>(cv, fin, pin);
            c->launches += 1;
        }
        if (phase == 1) {
            k_fold_partials3<T><<<nb3(nc, 256), 256, 0, c->stream>>>(pin, c->S, nc, xbuf);
            c->launches += 1;
            if (body) {
                k_wall3<T><<<cvgrid, 256, 0, c->stream>>>(cv, bp, c->d_body, fin, c->wphi, c->wcontrib, c->ticket,
                                                           c->d_hist, 1, xw);
                c->launches += 1;
            }
            return cudaGetLastError();
        }
    } else {
        // the summed moments of F_CV^n, one slot in the state precision
        pin = (T *)c->split_in;
        k_unfold_partials3<T><<<nb3(5 * nc, 256), 256, 0, c->stream>>>(xbuf, 5 * nc, pin);
        c->launches += 1;
    }
    const int Sin = phase == 2 ? 1 : c->S;
    cv.Sin = Sin;
    // conservative equilibrium parameters of F_CV^n (after fusion)
    if (cons && !imex && (e = eqpar(c, pin, Sin)) != cudaSuccess) return e;
    // the Shakhov model under the explicit scheme in FP32: the heat flux of
    // every control volume at t^n (after fusion), and the step kernels relax
    // towards its equilibrium (FP64: the post-pass k_shakhov3)
    const bool shak = c->model == DVM_SHAKHOV && !imex && c->prec == DVM_FP32;
    if (shak && (e = heatflux3d(c, fin, pin)) != cudaSuccess) return e;
    cv.qh = shak ? c->qheat : nullptr;
    cv.pr1 = 1.0 - c->Pr;
    if (body) {
        // the wall kernel and then the control-volume kernel run on the side
        // stream beside the bulk kernel: both read F^n and write only the cut
        // and merged control volumes, the bulk kernel only the plain cells
        if ((e = cudaEventRecord(c->ev_wfork, c->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(c->wstream, c->ev_wfork, 0)) != cudaSuccess) return e;
        k_wall3<T><<<cvgrid, 256, 0, c->wstream>>>(cv, bp, c->d_body, fin, c->wphi, c->wcontrib, c->ticket,
                                                    c->d_hist, phase == 2 ? 2 : 0, xw);
        c->launches += 1;
    }
    Bulk3Args<T> a{};
    a.g = g; a.S = c->S; a.Sin = Sin; a.nzc = (c->nz + kZc3 - 1) / kZc3;
    a.eqp = cons && !imex ? (const T *)c->eqp : nullptr;
    a.qh = shak ? (const T *)c->qheat : nullptr;
    a.pr1 = T(1.0 - c->Pr);
    a.fin = fin; a.fout = fout; a.pin = pin; a.pout = pout;
    a.flags = c->flags3; a.vxt = vx_table<T>(c); a.vyz = vyz_table<T>(c); a.err = c->d_err;
    if ((e = timing_mark(c, 0)) != cudaSuccess) return e;
    e = launch_bulk3_any<T>(c, a, shak);
    if (e != cudaSuccess) return e;
    if ((e = timing_mark(c, 1)) != cudaSuccess) return e;
    c->launches += 1;
    if (body) {
        k_special3<T><<<cvgrid, 256, 0, c->wstream>>>(cv, fin, fout, pin, pout, c->wphi);
        if ((e = cudaEventRecord(c->ev_wjoin, c->wstream)) != cudaSuccess) return e;
        // the step ends when both streams are done
        if ((e = cudaStreamWaitEvent(c->stream, c->ev_wjoin, 0)) != cudaSuccess) return e;
        c->launches += 1;
    }
    if (imex) {
        if (phase == 2) {
            // a velocity split relaxes in phase 3, from the moment sums of
            // the transported values summed over the ranks
            k_fold_partials3<T><<<nb3(nc, 256), 256, 0, c->stream>>>(pout, c->S, nc, xbuf);
            c->launches += 1;
            return cudaGetLastError();
        }
        if ((e = imex_relax3d<T>(c, pout, c->S)) != cudaSuccess) return e;
    }
    return end_step3d(c);
}

// Phase 3 of a semi-implicit step of a velocity split: the relaxation from
// the moment sums of the transported values summed over the ranks (xbuf).
template <typename T>
cudaError_t split_relax3d_t(dvm_ctx *c, const double *xbuf)
{
    const long nc = (long)c->nc;
    T *mom = (T *)c->split_in;
    k_unfold_partials3<T><<<nb3(5 * nc, 256), 256, 0, c->stream>>>(xbuf, 5 * nc, mom);
    c->launches += 1;
    cudaError_t e = imex_relax3d<T>(c, mom, 1);
    if (e != cudaSuccess) return e;
    return end_step3d(c);
}

}  // namespace

// TMA descriptors of the two state buffers: a 4D view (x: padded cells of a
// row times the W velocities of a group, y: padded rows, z: padded planes,
// w: velocity group) with the bulk kernel's plane box (tile plus halo).
int make_tensor_maps3d(dvm_ctx *c)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult qr;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
        if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return DVM_ERR_CUDA;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const int W = c->W;
    const cuuint64_t dims[4] = {(cuuint64_t)(c->nx + 4) * W, (cuuint64_t)(c->ny + 4), (cuuint64_t)(c->nz + 4),
                                (cuuint64_t)c->ngrp};
    const cuuint64_t row = (cuuint64_t)(c->nx + 4) * W * c->elem;
    const cuuint64_t strides[3] = {row, row * (c->ny + 4), (cuuint64_t)c->slab * W * c->elem};
    const cuuint32_t box[4] = {(cuuint32_t)kPlaneX * W,
                               (cuuint32_t)(c->prec == DVM_FP32 ? rows3<float>() : rows3<double>()) + 4, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = c->prec == DVM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    for (int b = 0; b < 2; ++b) {
        CUresult r = encode(&c->tmap[b], dt, 4, c->f[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled (3D) failed (" + std::to_string((int)r) + ")");
            return DVM_ERR_CUDA;
        }
    }
    return DVM_OK;
}

size_t vtab3_bytes(const dvm_ctx *c) { return (size_t)c->nvxp * 2 * c->elem + (size_t)c->nvy * c->nvz * 4 * c->elem; }

size_t cvinfo3_bytes() { return sizeof(CvInfo3); }

cudaError_t members3d(dvm_ctx *c)
{
    k_members3<<<4 * 152, 256, 0, c->stream>>>(cv3_args(c), (CvInfo3 *)c->cvinfo);
    return cudaGetLastError();
}

cudaError_t step3d(dvm_ctx *c)
{
    return c->prec == DVM_FP32 ? step3d_t<float>(c, 0, nullptr) : step3d_t<double>(c, 0, nullptr);
}

// Velocity split: phase 1 (this rank's sums into xbuf) or phase 2 (finish
// the step from xbuf summed over the ranks).
cudaError_t split_step3d(dvm_ctx *c, int phase, void *xbuf)
{
    double *x = static_cast<double *>(xbuf);
    if (phase == 3) return c->prec == DVM_FP32 ? split_relax3d_t<float>(c, x) : split_relax3d_t<double>(c, x);
    return c->prec == DVM_FP32 ? step3d_t<float>(c, phase, x) : step3d_t<double>(c, phase, x);
}

cudaError_t tables3d(dvm_ctx *c)
{
    const Grid3D g = grid3d(c);
    const int n = c->nvxp > c->nvy * c->nvz ? c->nvxp : c->nvy * c->nvz;
    if (c->prec == DVM_FP32)
        k_tables3<float><<<nb3(n, 256), 256, 0, c->stream>>>(g, (VX3<float> *)c->vtab, (VYZ3<float> *)vyz_table<float>(c));
    else
        k_tables3<double><<<nb3(n, 256), 256, 0, c->stream>>>(g, (VX3<double> *)c->vtab,
                                                                (VYZ3<double> *)vyz_table<double>(c));
    return cudaGetLastError();
}

cudaError_t partials_from_state3d(dvm_ctx *c)
{
    const Grid3D g = grid3d(c);
    const dim3 grid(nb3(c->nx, 32), c->ny, c->nz), block(32, kMomChunks);
    if (c->prec == DVM_FP32)
        k_partials3<float><<<grid, block, 0, c->stream>>>(g, c->S, (const float *)c->f[c->cur], vx_table<float>(c),
                                                          vyz_table<float>(c), (float *)c->part[c->cur], c->geo3.type,
                                                          c->d_err);
    else
        k_partials3<double><<<grid, block, 0, c->stream>>>(g, c->S, (const double *)c->f[c->cur],
                                                           vx_table<double>(c), vyz_table<double>(c),
                                                           (double *)c->part[c->cur], c->geo3.type, c->d_err);
    return cudaGetLastError();
}

cudaError_t moments_out3d(dvm_ctx *c, double *d_out)
{
    const Grid3D g = grid3d(c);
    const dim3 grid(nb3(c->nx, 32), c->ny, c->nz), block(32, kMomChunks);
    if (c->prec == DVM_FP32)
        k_moments_out3<float><<<grid, block, 0, c->stream>>>(g, (const float *)c->f[c->cur], vx_table<float>(c),
                                                             vyz_table<float>(c), d_out);
    else
        k_moments_out3<double><<<grid, block, 0, c->stream>>>(g, (const double *)c->f[c->cur], vx_table<double>(c),
                                                              vyz_table<double>(c), d_out);
    return cudaGetLastError();
}

cudaError_t init_maxwellian3d(dvm_ctx *c, const double *d_prim)
{
    const Grid3D g = grid3d(c);
    dim3 grid((unsigned)c->nc, nb3(c->nv, 256));
    if (c->prec == DVM_FP32)
        k_init3<float><<<grid, 256, 0, c->stream>>>(g, d_prim, c->geo3.type, (float *)c->f[c->cur]);
    else
        k_init3<double><<<grid, 256, 0, c->stream>>>(g, d_prim, c->geo3.type, (double *)c->f[c->cur]);
    return cudaGetLastError();
}

cudaError_t ghost3d(dvm_ctx *c, int side, const double *d_prim, int nside)
{
    const Grid3D g = grid3d(c);
    const long n = (long)nside * c->nv;
    if (c->prec == DVM_FP32)
        k_ghost3<float><<<nb3(n, 256), 256, 0, c->stream>>>(g, d_prim, side, nside, (float *)c->f[0], (float *)c->f[1]);
    else
        k_ghost3<double><<<nb3(n, 256), 256, 0, c->stream>>>(g, d_prim, side, nside, (double *)c->f[0], (double *)c->f[1]);
    return cudaGetLastError();
}

cudaError_t pack3d(dvm_ctx *c, const void *pub, void *dev)
{
    const Grid3D g = grid3d(c);
    dim3 grid((unsigned)c->nc, nb3(c->nv, 256));
    if (c->prec == DVM_FP32) k_pack3<float><<<grid, 256, 0, c->stream>>>(g, (const float *)pub, (float *)dev, 1);
    else k_pack3<double><<<grid, 256, 0, c->stream>>>(g, (const double *)pub, (double *)dev, 1);
    return cudaGetLastError();
}

cudaError_t unpack3d(dvm_ctx *c, const void *dev, void *pub)
{
    const Grid3D g = grid3d(c);
    dim3 grid((unsigned)c->nc, nb3(c->nv, 256));
    if (c->prec == DVM_FP32) k_pack3<float><<<grid, 256, 0, c->stream>>>(g, (const float *)dev, (float *)pub, 0);
    else k_pack3<double><<<grid, 256, 0, c->stream>>>(g, (const double *)dev, (double *)pub, 0);
    return cudaGetLastError();
}

cudaError_t zero_solid3d(dvm_ctx *c)
{
    const Grid3D g = grid3d(c);
    const dim3 grid(nb3(c->nc, 256), 8);
    for (int b = 0; b < 2; ++b) {
        if (c->prec == DVM_FP32) k_zero_solid3<float><<<grid, 256, 0, c->stream>>>(g, c->geo3.type, (float *)c->f[b]);
        else k_zero_solid3<double><<<grid, 256, 0, c->stream>>>(g, c->geo3.type, (double *)c->f[b]);
    }
    return cudaGetLastError();
}

cudaError_t halo3d(dvm_ctx *c, int buf)
{
    const Grid3D g = grid3d(c);
    const long per = 2L * ((long)c->ny * c->nz + (long)c->nx * c->nz + (long)c->nx * c->ny);
    const long n = 2 * per * c->nvp;
    if (c->prec == DVM_FP32) k_halo3<float><<<nb3(n, 256), 256, 0, c->stream>>>(g, (float *)c->f[buf]);
    else k_halo3<double><<<nb3(n, 256), 256, 0, c->stream>>>(g, (double *)c->f[buf]);
    return cudaGetLastError();
}

cudaError_t mass3d(dvm_ctx *c, double *d_scratch, double *d_out)
{
    const Grid3D g = grid3d(c);
    if (c->prec == DVM_FP32)
        k_mass_cells3<float><<<nb3(c->nc, 8), 256, 0, c->stream>>>(g, (const float *)c->f[c->cur], c->geo3.vol, d_scratch);
    else
        k_mass_cells3<double><<<nb3(c->nc, 8), 256, 0, c->stream>>>(g, (const double *)c->f[c->cur], c->geo3.vol, d_scratch);
    k_sum3<<<1, 1024, 0, c->stream>>>(d_scratch, c->nc, d_out);
    return cudaGetLastError();
}

}  // namespace dvm
