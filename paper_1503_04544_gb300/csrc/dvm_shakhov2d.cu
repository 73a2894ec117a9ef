// Heat flux of the control volumes at t^n for the Shakhov collision model of
// the reduced 2D (f, g) equations (arXiv:1503.04544, Sec. 2.2, Eq.
// ShakhovDD) under the explicit scheme (Eq. ExSchemeDD).  The model relaxes
// towards
//   f_S = M [1 + (1 - Pr) c.q (|c|^2/T - 4) / (5 P T)],
//   g_S = T/2 M [1 + (1 - Pr) c.q (|c|^2/T - 2) / (5 P T)],
// c = v - u, P = rho T (R = 1), where q = sum c (|c|^2/2 f + g) dv is the heat
// flux of the control volume at t^n (Eq. MacroscopicDDv).  The step kernels
// (k_bulk, k_special) form f_S and g_S in place of the Maxwellian; the heat
// flux, a sum over every velocity, comes from k_heatflux before them.
#include "dvm_device.cuh"

namespace dvm {
namespace {

// Sum of the S partial moment sums of a cell ([S][4][nc] layout).
template <typename T>
__device__ __forceinline__ void cell_sums(const T *part, int S, long nc, long cell, T (&s)[4])
{
    Acc<T> a[4];
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) a[m].merge(part[((long)q * 4 + m) * nc + cell], T(0));
#pragma unroll
    for (int m = 0; m < 4; ++m) s[m] = a[m].value();
}

// Block = 32 consecutive cells of a row x kMomChunks warps, each warp one
// chunk of the velocity groups: the heat flux of the cell's control volume
// from F^n (its master's values after fusion) about the control volume's
// velocity, compensated sums merged over the chunks in fixed order, into
// q[2][nc].  Cells in no control volume get 0.
template <typename T>
__global__ void __launch_bounds__(32 * kMomChunks)
    k_heatflux(Grid2D g, int S, const T *fin, const T *pin, const VCoef<T> *vt, const int32_t *master, T *q, int *err)
{
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y;
    const long nc = (long)g.nx * g.ny, cell = (long)j * g.nx + i;
    const T dv = pick<T>(g.dv_f, g.dv);
    const long m = i < g.nx ? (long)master[cell] : -1;
    bool gas = m >= 0;
    T ux = 0, uy = 0;
    if (gas) {
        T s[4];
        cell_sums(pin, S, nc, m, s);
        if (s[0] > T(0)) {
            ux = s[1] / s[0];
            uy = s[2] / s[0];
        } else {
            if (threadIdx.y == 0) atomicExch(&err[kErrNonphys], 1);
            gas = false;
        }
    }
    const int gps = (g.ngrp + kMomChunks - 1) / kMomChunks;
    const int q0 = threadIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    Acc<T> hq[2];
    if (gas) {
        const long pm = pcell(g, m);
        const V *fv = reinterpret_cast<const V *>(fin);
        for (int q = q0; q < q1; ++q) {
            T a[W], b[W];
            vld<T>(fv + (long)q * 2 * g.slab + pm, a);
            vld<T>(fv + ((long)q * 2 + 1) * g.slab + pm, b);
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
    if (threadIdx.y != 0 || i >= g.nx) return;
    q[cell] = gas ? hq[0].value() * dv : T(0);
    q[nc + cell] = gas ? hq[1].value() * dv : T(0);
}

template <typename T>
cudaError_t heatflux2d_t(dvm_ctx *c, const void *f, const void *part)
{
    const Grid2D g = grid2d(c);
    const dim3 grid((unsigned)((c->nx + 31) / 32), (unsigned)c->ny), block(32, kMomChunks);
    cudaError_t e = timing_mark_kernel(c, 2, 0);
    if (e != cudaSuccess) return e;
    k_heatflux<T><<<grid, block, 0, c->stream>>>(g, c->S, (const T *)f, (const T *)part, (const VCoef<T> *)c->vtab,
                                                  c->master, (T *)c->qheat, c->d_err);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return timing_mark_kernel(c, 2, 1);
}

}  // namespace

cudaError_t heatflux2d(dvm_ctx *c, const void *f, const void *part)
{
    return c->prec == DVM_FP32 ? heatflux2d_t<float>(c, f, part) : heatflux2d_t<double>(c, f, part);
}

}  // namespace dvm
