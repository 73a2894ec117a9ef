// Shakhov collision model for the reduced 2D (f, g) equations
// (arXiv:1503.04544, Sec. 2.2, Eq. ShakhovDD) under the explicit scheme
// (Eq. ExSchemeDD).  The model relaxes towards
//   f_S = M [1 + (1 - Pr) c.q (|c|^2/T - 4) / (5 P T)],
//   g_S = T/2 M [1 + (1 - Pr) c.q (|c|^2/T - 2) / (5 P T)],
// c = v - u, P = rho T (R = 1), where q = sum c (|c|^2/2 f + g) dv is the heat
// flux of the control volume at t^n (Eq. MacroscopicDDv).  The step kernels
// relax towards M; the scheme's relaxation term differs from theirs by
//   a (dt/tau) (f_S - M) = a (dt/tau) k c.q (|c|^2/T - 4) M,   k = (1 - Pr) / (5 rho T^2),
// and the g counterpart, with a = S^n / S^{n+1,*} the area ratio of the
// control volume (1 for a fixed obstacle and for every plain cell), which
// k_shakhov adds to every gas cell after the step, with the moments and heat
// flux of the cell's control volume at t^n.  It then rewrites the moment sums
// of the new state.
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

// rho, u and T from the sums of Eq. MacroscopicDDv (E = rho|u|^2/2 + 3/2 rho T).
template <typename T>
__device__ __forceinline__ bool cell_primitives(T dv, const T (&s)[4], T &rho, T &ux, T &uy, T &tmp)
{
    rho = s[0] * dv;
    ux = s[1] / s[0];
    uy = s[2] / s[0];
    tmp = (T(2) * (s[3] / s[0]) - (ux * ux + uy * uy)) / T(3);
    return rho > T(0) && tmp > T(0);
}

__device__ __forceinline__ float exp2_s(float x) { return ex2_fast(x); }
__device__ __forceinline__ double exp2_s(double x) { return exp2(x); }

// Block = 32 consecutive cells of a row x kMomChunks warps, each warp one
// chunk of the velocity groups.  Pass 1 sums the heat flux of the cell's
// control volume from F^n (its master's values after fusion), pass 2 adds the
// Shakhov term to F^{n+1} of the cell and its padding mirrors and sums the
// moments of the result.  Solid cells keep their zero state and zero sums.
template <typename T>
__global__ void __launch_bounds__(32 * kMomChunks)
    k_shakhov(Grid2D g, int S, T dt_tau0, T pr1, const T *fin, const T *pin, T *fout, T *pout,
              const VCoef<T> *vt, const int32_t *master, const int8_t *type, const uint8_t *flags,
              const double *ratio, int *err)
{
    constexpr int W = Vec<T>::W;
    using V = typename Vec<T>::type;
    __shared__ T qsh[2][32];
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y;
    const long nc = (long)g.nx * g.ny, cell = (long)j * g.nx + i;
    const T dv = pick<T>(g.dv_f, g.dv);
    bool gas = i < g.nx && type[cell] != DVM_SOLID;
    const long m = gas ? (long)master[cell] : -1;
    gas = gas && m >= 0;
    T rho = 0, ux = 0, uy = 0, tmp = 0;
    if (gas) {
        T s[4];
        cell_sums(pin, S, nc, m, s);
        if (!cell_primitives(dv, s, rho, ux, uy, tmp)) {
            if (threadIdx.y == 0) atomicExch(&err[kErrNonphys], 1);
            gas = false;
        }
    }
    const int gps = (g.ngrp + kMomChunks - 1) / kMomChunks;
    const int q0 = threadIdx.y * gps, q1 = min(q0 + gps, g.ngrp);
    // pass 1: heat flux of the control volume at t^n
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
    if (threadIdx.y == 0) {
        qsh[0][threadIdx.x] = hq[0].value() * dv;
        qsh[1][threadIdx.x] = hq[1].value() * dv;
    }
    __syncthreads();
    const T qx = qsh[0][threadIdx.x], qy = qsh[1][threadIdx.x];
    // pass 2: the Shakhov term on F^{n+1}
    Acc<T> a4[4];
    if (gas) {
        const T A = rho / (T(2.0 * kPi) * tmp), c2 = T(kLog2e) / (T(2) * tmp);
        // a (dt/tau) k, a the area ratio of a moving obstacle's control volume
        const T ar = ratio && (flags[cell] & kSpecial) ? (T)ratio[cell] : T(1);
        const T kk = ar * dt_tau0 * rho * pr1 / (T(5) * rho * tmp * tmp);
        const T iT = T(1) / tmp, half = tmp / T(2);
        const long pc = nbr(g, i, j);
        long mir[4];
        mirrors(g, i, j, mir);
        V *fo = reinterpret_cast<V *>(fout);
        for (int q = q0; q < q1; ++q) {
            V *pa = fo + (long)q * 2 * g.slab, *pb = pa + g.slab;
            T a[W], b[W];
            vld<T>(pa + pc, a);
            vld<T>(pb + pc, b);
            T t0 = 0, t1 = 0, t2 = 0, t3 = 0;
#pragma unroll
            for (int e = 0; e < W; ++e) {
                if (q * W + e >= g.nv) continue;
                const VCoef<T> c = ld_coef(vt + q * W + e);
                const T dx = c.vx - ux, dy = c.vy - uy, d2 = dx * dx + dy * dy;
                const T h = kk * (dx * qx + dy * qy) * (A * exp2_s(-d2 * c2));
                a[e] += h * (d2 * iT - T(4));
                b[e] += half * h * (d2 * iT - T(2));
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
    // split 0 holds the sums, the other splits zeros (solid cells: zeros)
    for (int q = 0; q < S; ++q) {
        const bool z = q > 0 || !gas;
#pragma unroll
        for (int k = 0; k < 4; ++k) pout[((long)q * 4 + k) * nc + cell] = z ? T(0) : a4[k].value();
    }
}

template <typename T>
cudaError_t shakhov2d_t(dvm_ctx *c)
{
    // the step has swapped the buffers: F^n is the other one now
    const T *fin = (const T *)c->f[1 - c->cur], *pin = (const T *)c->part[1 - c->cur];
    T *fout = (T *)c->f[c->cur], *pout = (T *)c->part[c->cur];
    const Grid2D g = grid2d(c);
    const dim3 grid((unsigned)((c->nx + 31) / 32), (unsigned)c->ny), block(32, kMomChunks);
    cudaError_t e = timing_mark_kernel(c, 2, 0);
    if (e != cudaSuccess) return e;
    k_shakhov<T><<<grid, block, 0, c->stream>>>(g, c->S, T(c->dt / c->tau0), T(1.0 - c->Pr), fin, pin, fout, pout,
                                                 (const VCoef<T> *)c->vtab, c->master, c->geo[c->gcur].type,
                                                 c->flags, c->moving ? c->cv_ratio : nullptr, c->d_err);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return timing_mark_kernel(c, 2, 1);
}

}  // namespace

cudaError_t shakhov2d(dvm_ctx *c)
{
    return c->prec == DVM_FP32 ? shakhov2d_t<float>(c) : shakhov2d_t<double>(c);
}

}  // namespace dvm
