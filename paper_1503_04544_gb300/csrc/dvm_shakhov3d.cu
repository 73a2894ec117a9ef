// Shakhov collision model for the full 3D distribution F (arXiv:1503.04544,
// Sec. 2.1) under the explicit scheme (Eq. eq-schema3D): relaxation towards
//   F_S = M [1 + (1 - Pr) c.q (|c|^2/T - 5) / (5 P T)],
// c = v - u, P = rho T (R = 1), with the heat flux q = sum c |c|^2/2 F dv of
// the control volume at t^n.
//
// FP32: k_heatflux3 writes q of every cell's control volume before the step,
// and the step kernels (k_bulk3, k_special3) relax towards F_S themselves.
// FP64: the step kernels relax towards M, and k_shakhov3 adds the difference
//   (dt/tau) k c.q (|c|^2/T - 5) M,   k = (1 - Pr) / (5 rho T^2),
// to every gas cell after the step (the obstacle is fixed, so the area ratio
// of the scheme's relaxation term is 1); it then rewrites the moment sums of
// the new state.  (The FP64 bulk kernel's shared memory has no room for the
// Shakhov coefficients of its column cells.)
#include "dvm_device.cuh"

namespace dvm {
namespace {

template <typename T> struct alignas(2 * sizeof(T)) VxEntry { T vx, nux; };
template <typename T> struct alignas(4 * sizeof(T)) VyzEntry { T vy, vz, nuy, nuz; };

// Slab index of cell (i, j, k), each within two cells of the grid.
__device__ __forceinline__ long slab3(const Grid3D &g, int i, int j, int k)
{
    return ((long)(k + 2) * (g.ny + 4) + (j + 2)) * (g.nx + 4) + (i + 2);
}

// Padding cells that mirror interior cell (i, j, k) on periodic and
// zero-gradient sides (two per axis at most); -1 where unused.
__device__ __forceinline__ void side_mirrors3(const Grid3D &g, int i, int j, int k, long (&m)[6])
{
#pragma unroll
    for (int t = 0; t < 6; ++t) m[t] = -1;
    if (g.bc[0] == DVM_BC_PERIODIC) {
        if (i < 2) m[0] = slab3(g, i + g.nx, j, k);
        else if (i >= g.nx - 2) m[0] = slab3(g, i - g.nx, j, k);
    } else {
        if (i == 0 && g.bc[0] == DVM_BC_ZEROGRAD) { m[0] = slab3(g, -1, j, k); m[1] = slab3(g, -2, j, k); }
        if (i == g.nx - 1 && g.bc[1] == DVM_BC_ZEROGRAD) { m[0] = slab3(g, g.nx, j, k); m[1] = slab3(g, g.nx + 1, j, k); }
    }
    if (g.bc[2] == DVM_BC_PERIODIC) {
        if (j < 2) m[2] = slab3(g, i, j + g.ny, k);
        else if (j >= g.ny - 2) m[2] = slab3(g, i, j - g.ny, k);
    } else {
        if (j == 0 && g.bc[2] == DVM_BC_ZEROGRAD) { m[2] = slab3(g, i, -1, k); m[3] = slab3(g, i, -2, k); }
        if (j == g.ny - 1 && g.bc[3] == DVM_BC_ZEROGRAD) { m[2] = slab3(g, i, g.ny, k); m[3] = slab3(g, i, g.ny + 1, k); }
    }
    if (g.bc[4] == DVM_BC_PERIODIC) {
        if (k < 2) m[4] = slab3(g, i, j, k + g.nz);
        else if (k >= g.nz - 2) m[4] = slab3(g, i, j, k - g.nz);
    } else {
        if (k == 0 && g.bc[4] == DVM_BC_ZEROGRAD) { m[4] = slab3(g, i, j, -1); m[5] = slab3(g, i, j, -2); }
        if (k == g.nz - 1 && g.bc[5] == DVM_BC_ZEROGRAD) { m[4] = slab3(g, i, j, g.nz); m[5] = slab3(g, i, j, g.nz + 1); }
    }
}

__device__ __forceinline__ float exp2_s3(float x) { return ex2_fast(x); }
__device__ __forceinline__ double exp2_s3(double x) { return exp2(x); }

// Heat flux of the control volume of cell (i, j, k) at t^n, for a block of 32
// consecutive cells of an x-row x kMomChunks warps, each warp one chunk of
// the velocity groups: the primitives from the partial sums of its master,
// q from the master's F^n (after fusion), compensated sums merged over the
// chunks in fixed order into qsh (every warp of the block reads them after
// the barrier).  gas is false for solid cells and cells in no control volume.
template <typename T>
__device__ __forceinline__ void cv_heat_flux3(const Grid3D &g, int S, const T *fin, const T *pin,
                                              const VxEntry<T> *vxt, const VyzEntry<T> *vyz, const int32_t *master,
                                              const int8_t *type, int *err, int i, int j, int k, T (&qsh)[3][32],
                                              bool &gas, T &rho, T &ux, T &uy, T &uz, T &tmp)
{
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    const long nc = (long)g.nx * g.ny * g.nz, cell = ((long)k * g.ny + j) * g.nx + i;
    const T dv = pick<T>(g.dv_f, g.dv);
    gas = i < g.nx && type[cell] != DVM_SOLID;
    const long m = gas ? (long)master[cell] : -1;
    gas = gas && m >= 0;
    rho = ux = uy = uz = tmp = 0;
    if (gas) {
        Acc<T> a[5];
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int f = 0; f < 5; ++f) a[f].merge(pin[((long)q * 5 + f) * nc + m], T(0));
        const T s0 = a[0].value();
        rho = s0 * dv;
        ux = a[1].value() / s0;
        uy = a[2].value() / s0;
        uz = a[3].value() / s0;
        tmp = (T(2) * (a[4].value() / s0) - (ux * ux + uy * uy + uz * uz)) / T(3);
        if (!(rho > T(0) && tmp > T(0))) {
            if (threadIdx.y == 0) atomicExch(&err[kErrNonphys], 1);
            gas = false;
        }
    }
    const int gps = (g.ngrp + kMomChunks - 1) / kMomChunks;
    const int q0 = threadIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    Acc<T> hq[3];
    if (gas && q0 < q1) {
        const int mk = (int)(m / ((long)g.nx * g.ny)), mr = (int)(m - (long)mk * g.nx * g.ny);
        const long pm = slab3(g, mr % g.nx, mr / g.nx, mk);
        const V *fv = reinterpret_cast<const V *>(fin);
        int r = q0 / g.nxg, xg = q0 - r * g.nxg;
        for (int q = q0; q < q1; ++q) {
            T a[W];
            vld<T>(fv + (long)q * g.slab + pm, a);
            const VyzEntry<T> cy = vyz[r];
            const T cyv = cy.vy - uy, czv = cy.vz - uz, dyz = cyv * cyv + czv * czv;
            T t0 = 0, t1 = 0;
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const int p1 = xg * W + e;
                if (p1 >= g.nvx) continue;
                const T dx = vxt[p1].vx - ux;
                const T w = T(0.5) * (dx * dx + dyz) * a[e];
                t0 += dx * w;
                t1 += w;
            }
            hq[0].add(t0);
            hq[1].add(cyv * t1);
            hq[2].add(czv * t1);
            if (++xg == g.nxg) {
                xg = 0;
                ++r;
            }
        }
    }
    merge_chunks<T, 3>(hq);
    if (threadIdx.y == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) qsh[d][threadIdx.x] = hq[d].value() * dv;
    }
    __syncthreads();
}

// The heat flux of every cell's control volume at t^n into q[3][nc] (0 for
// solid cells and cells in no control volume).
template <typename T>
__global__ void __launch_bounds__(32 * kMomChunks)
    k_heatflux3(Grid3D g, int S, const T *fin, const T *pin, const VxEntry<T> *vxt, const VyzEntry<T> *vyz,
                const int32_t *master, const int8_t *type, T *q, int *err)
{
    __shared__ T qsh[3][32];
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    bool gas;
    T rho, ux, uy, uz, tmp;
    cv_heat_flux3(g, S, fin, pin, vxt, vyz, master, type, err, i, j, k, qsh, gas, rho, ux, uy, uz, tmp);
    if (threadIdx.y != 0 || i >= g.nx) return;
    const long nc = (long)g.nx * g.ny * g.nz, cell = ((long)k * g.ny + j) * g.nx + i;
#pragma unroll
    for (int d = 0; d < 3; ++d) q[d * nc + cell] = gas ? qsh[d][threadIdx.x] : T(0);
}

// FP64: pass 1 (cv_heat_flux3), then pass 2 adds the Shakhov term to F^{n+1}
// of the cell and its padding mirrors and sums the five moments of the
// result.  Solid cells keep their zero state and sums.
template <typename T>
__global__ void __launch_bounds__(32 * kMomChunks)
    k_shakhov3(Grid3D g, int S, T dt_tau0, T pr1, const T *fin, const T *pin, T *fout, T *pout,
               const VxEntry<T> *vxt, const VyzEntry<T> *vyz, const int32_t *master, const int8_t *type, int *err)
{
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    __shared__ T qsh[3][32];
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const long nc = (long)g.nx * g.ny * g.nz, cell = ((long)k * g.ny + j) * g.nx + i;
    bool gas;
    T rho, ux, uy, uz, tmp;
    cv_heat_flux3(g, S, fin, pin, vxt, vyz, master, type, err, i, j, k, qsh, gas, rho, ux, uy, uz, tmp);
    const int gps = (g.ngrp + kMomChunks - 1) / kMomChunks;
    const int q0 = threadIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    const T qx = qsh[0][threadIdx.x], qy = qsh[1][threadIdx.x], qz = qsh[2][threadIdx.x];
    // pass 2: the Shakhov term on F^{n+1}
    Acc<T> a5[5];
    if (gas && q0 < q1) {
        const T tw = T(2.0 * kPi) * tmp;
        const T A = rho / (tw * sqrt(tw)), c2 = T(kLog2e) / (T(2) * tmp);
        const T kk = dt_tau0 * rho * pr1 / (T(5) * rho * tmp * tmp);     // (dt/tau) k
        const T iT = T(1) / tmp;
        const long pc = slab3(g, i, j, k);
        long mir[6];
        side_mirrors3(g, i, j, k, mir);
        V *fo = reinterpret_cast<V *>(fout);
        int r = q0 / g.nxg, xg = q0 - r * g.nxg;
        for (int q = q0; q < q1; ++q) {
            V *pa = fo + (long)q * g.slab;
            T a[W];
            vld<T>(pa + pc, a);
            const VyzEntry<T> cy = vyz[r];
            const T cyv = cy.vy - uy, czv = cy.vz - uz, dyz = cyv * cyv + czv * czv;
            const T qyz = cyv * qy + czv * qz;
            T t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const int p1 = xg * W + e;
                if (p1 >= g.nvx) continue;
                const T vx = vxt[p1].vx, dx = vx - ux, d2 = dx * dx + dyz;
                const T h = kk * (dx * qx + qyz) * (A * exp2_s3(-d2 * c2));
                a[e] += h * (d2 * iT - T(5));
                t0 += a[e];
                t1 += vx * a[e];
                t2 += vx * vx * a[e];
            }
            vst<T>(pa + pc, a);
#pragma unroll
            for (int t = 0; t < 6; ++t)
                if (mir[t] >= 0) vst<T>(pa + mir[t], a);
            a5[0].add(t0);
            a5[1].add(t1);
            a5[2].add(cy.vy * t0);
            a5[3].add(cy.vz * t0);
            a5[4].add(T(0.5) * ((cy.vy * cy.vy + cy.vz * cy.vz) * t0 + t2));
            if (++xg == g.nxg) {
                xg = 0;
                ++r;
            }
        }
    }
    merge_chunks<T, 5>(a5);
    if (threadIdx.y != 0 || i >= g.nx) return;
    // split 0 holds the sums, the other splits zeros (solid cells: zeros)
    for (int q = 0; q < S; ++q) {
        const bool z = q > 0 || !gas;
#pragma unroll
        for (int f = 0; f < 5; ++f) pout[((long)q * 5 + f) * nc + cell] = z ? T(0) : a5[f].value();
    }
}

template <typename T>
cudaError_t shakhov3d_t(dvm_ctx *c)
{
    // the step has swapped the buffers: F^n is the other one now
    const T *fin = (const T *)c->f[1 - c->cur], *pin = (const T *)c->part[1 - c->cur];
    T *fout = (T *)c->f[c->cur], *pout = (T *)c->part[c->cur];
    const Grid3D g = grid3d(c);
    const VxEntry<T> *vxt = reinterpret_cast<const VxEntry<T> *>(c->vtab);
    const VyzEntry<T> *vyz = reinterpret_cast<const VyzEntry<T> *>(reinterpret_cast<const char *>(c->vtab) +
                                                                   (size_t)c->nvxp * sizeof(VxEntry<T>));
    const dim3 grid((unsigned)((c->nx + 31) / 32), (unsigned)c->ny, (unsigned)c->nz), block(32, kMomChunks);
    cudaError_t e = timing_mark_kernel(c, 2, 0);
    if (e != cudaSuccess) return e;
    k_shakhov3<T><<<grid, block, 0, c->stream>>>(g, c->S, T(c->dt / c->tau0), T(1.0 - c->Pr), fin, pin, fout, pout,
                                                  vxt, vyz, c->master, c->geo3.type, c->d_err);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return timing_mark_kernel(c, 2, 1);
}

template <typename T>
cudaError_t heatflux3d_t(dvm_ctx *c, const void *f, const void *part)
{
    const Grid3D g = grid3d(c);
    const VxEntry<T> *vxt = reinterpret_cast<const VxEntry<T> *>(c->vtab);
    const VyzEntry<T> *vyz = reinterpret_cast<const VyzEntry<T> *>(reinterpret_cast<const char *>(c->vtab) +
                                                                   (size_t)c->nvxp * sizeof(VxEntry<T>));
    const dim3 grid((unsigned)((c->nx + 31) / 32), (unsigned)c->ny, (unsigned)c->nz), block(32, kMomChunks);
    cudaError_t e = timing_mark_kernel(c, 2, 0);
    if (e != cudaSuccess) return e;
    k_heatflux3<T><<<grid, block, 0, c->stream>>>(g, c->S, (const T *)f, (const T *)part, vxt, vyz, c->master,
                                                   c->geo3.type, (T *)c->qheat, c->d_err);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return timing_mark_kernel(c, 2, 1);
}

}  // namespace

cudaError_t heatflux3d(dvm_ctx *c, const void *f, const void *part)
{
    return c->prec == DVM_FP32 ? heatflux3d_t<float>(c, f, part) : heatflux3d_t<double>(c, f, part);
}

cudaError_t shakhov3d(dvm_ctx *c)
{
    return c->prec == DVM_FP32 ? shakhov3d_t<float>(c) : shakhov3d_t<double>(c);
}

}  // namespace dvm
