// 2D time step of the cut-cell discrete-velocity method (arXiv:1503.04544,
// Sec. 3.3.5): fusion (Eq. FusionDD), wall density and stress (Eqs.
// BoundaryDDv, StressTensorDD), force/torque and rotation (Eqs. eq-force,
// eq-torque, motionDD_posit, motionDD_vit), fluxes and explicit update of the
// reduced pair (f, g) (Eqs. FluxDD, ExSchemeDD, BGKDD) and distribution
// (Eq. UpdateDD).
//
// State layout: [cell][comp][p], comp 0 = f, 1 = g, p = p2*nvx + p1.
//
// k_bulk updates every gas cell that forms a control volume on its own (all
// but a thin layer around the obstacle): one warp per cell, each lane a
// vector of VEC consecutive velocities of one velocity row, looping over the
// velocity grid; fluxes, relaxation and the moments of the new state are
// fused so that each step reads and writes the state once.  Cut and merged
// cells go through k_special, one block per control volume.
#include <cstdio>

#include "dvm_internal.h"

namespace dvm {
namespace {

constexpr double kPi = 3.14159265358979323846;

template <typename T> struct VecT;
template <> struct VecT<float> { using v4 = float4; using v2 = float2; };
template <> struct VecT<double> { using v4 = double4; using v2 = double2; };

template <typename T, int V>
__device__ __forceinline__ void vload(const T *p, T (&r)[V])
{
    if constexpr (V == 4 && sizeof(T) == 4) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    } else if constexpr (V == 2 && sizeof(T) == 4) {
        float2 a = __ldg(reinterpret_cast<const float2 *>(p));
        r[0] = a.x; r[1] = a.y;
    } else if constexpr (V == 2 && sizeof(T) == 8) {
        double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        r[0] = a.x; r[1] = a.y;
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) r[e] = __ldg(p + e);
    }
}

template <typename T, int V>
__device__ __forceinline__ void vstore(T *p, const T (&r)[V])
{
    if constexpr (V == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
    } else if constexpr (V == 2 && sizeof(T) == 4) {
        *reinterpret_cast<float2 *>(p) = make_float2(r[0], r[1]);
    } else if constexpr (V == 2 && sizeof(T) == 8) {
        *reinterpret_cast<double2 *>(p) = make_double2(r[0], r[1]);
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) p[e] = r[e];
    }
}

__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }

// minmod: 0 unless both arguments have the same strict sign, else the one of
// smaller magnitude.
template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    if (a > T(0) && b > T(0)) return a < b ? a : b;
    if (a < T(0) && b < T(0)) return a > b ? a : b;
    return T(0);
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

template <typename T> struct StepArgs {
    Grid2D g;
    const T *fin;
    T *fout;
    T *mom;                   // [nc][8]: rho ux uy uz T
    const uint8_t *flags;
    const T *ghost[4];
    int *err;
};

// Base pointer of the state of cell (i, j) or of its ghost beyond a side.
template <typename T>
__device__ __forceinline__ const T *cell_ptr(const StepArgs<T> &a, int i, int j)
{
    const Grid2D &g = a.g;
    const long cs = 2L * g.nv;
    if (i < 0) {
        if (g.bc[0] == DVM_BC_PERIODIC) i = ((i % g.nx) + g.nx) % g.nx;
        else if (g.bc[0] == DVM_BC_MAXWELLIAN) return a.ghost[0] + j * cs;
        else i = 0;
    } else if (i >= g.nx) {
        if (g.bc[1] == DVM_BC_PERIODIC) i = i % g.nx;
        else if (g.bc[1] == DVM_BC_MAXWELLIAN) return a.ghost[1] + j * cs;
        else i = g.nx - 1;
    }
    if (j < 0) {
        if (g.bc[2] == DVM_BC_PERIODIC) j = ((j % g.ny) + g.ny) % g.ny;
        else if (g.bc[2] == DVM_BC_MAXWELLIAN) return a.ghost[2] + i * cs;
        else j = 0;
    } else if (j >= g.ny) {
        if (g.bc[3] == DVM_BC_PERIODIC) j = j % g.ny;
        else if (g.bc[3] == DVM_BC_MAXWELLIAN) return a.ghost[3] + i * cs;
        else j = g.ny - 1;
    }
    return a.fin + ((long)j * g.nx + i) * cs;
}

// Moments (Eq. MacroscopicDDv) of a cell from the reduced sums
// s0 = sum f, s1 = sum vx f, s2 = sum vy f, s3 = sum (|v|^2/2 f + g).
template <typename T>
__device__ __forceinline__ void store_moments(T *m, double dv, T s0, T s1, T s2, T s3, int *err)
{
    T rho = s0 * T(dv);
    T ux = s1 / s0, uy = s2 / s0;
    T temp = (T(2) * (s3 / s0) - (ux * ux + uy * uy)) / T(3);
    if (!(rho > T(0)) || !(temp > T(0))) atomicExch(&err[kErrNonphys], 1);
    m[0] = rho; m[1] = ux; m[2] = uy; m[3] = 0; m[4] = temp;
}

// ------------------------------------------------------------ bulk kernel
template <typename T, int VEC, bool MUSCL>
__global__ void __launch_bounds__(256) k_bulk(StepArgs<T> a)
{
    extern __shared__ unsigned char smem_raw[];
    const Grid2D &g = a.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *ex = reinterpret_cast<T *>(smem_raw) + warp * (g.nvx + g.nvy);
    T *ey = ex + g.nvx;
    const long nc = (long)g.nx * g.ny;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= nc) return;
    const uint8_t fl = a.flags[cell];
    const long cs = 2L * g.nv;
    if (!(fl & kPlain)) {
        if (fl & kZero) {
            T z[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) z[e] = 0;
            for (int p = lane * VEC; p < 2 * g.nv; p += 32 * VEC) vstore<T, VEC>(a.fout + cell * cs + p, z);
            if (lane < 8) a.mom[cell * 8 + lane] = 0;
        }
        return;
    }
    const int i = (int)(cell % g.nx), j = (int)(cell / g.nx);
    // equilibrium of the cell at t^n (separable Maxwellian tables)
    const T rho = a.mom[cell * 8 + 0], ux = a.mom[cell * 8 + 1], uy = a.mom[cell * 8 + 2];
    const T tmp = a.mom[cell * 8 + 4];
    const T inv2T = T(1) / (T(2) * tmp);
    for (int q = lane; q < g.nvx; q += 32) {
        T d = T(g.vxmin + q * g.dvx) - ux;
        ex[q] = dexp(-(d * d) * inv2T);
    }
    for (int q = lane; q < g.nvy; q += 32) {
        T d = T(g.vymin + q * g.dvy) - uy;
        ey[q] = dexp(-(d * d) * inv2T);
    }
    __syncwarp();
    const T A = rho / (T(2.0 * kPi) * tmp);
    const T gfac = tmp / T(2);
    const T r = T(g.dt / g.tau0) * rho;
    const T dtdx = T(g.dt / g.dx), dtdy = T(g.dt / g.dy);

    const T *self = a.fin + cell * cs;
    const T *xm1 = cell_ptr(a, i - 1, j), *xp1 = cell_ptr(a, i + 1, j);
    const T *ym1 = cell_ptr(a, i, j - 1), *yp1 = cell_ptr(a, i, j + 1);
    const T *xm2 = MUSCL ? cell_ptr(a, i - 2, j) : nullptr, *xp2 = MUSCL ? cell_ptr(a, i + 2, j) : nullptr;
    const T *ym2 = MUSCL ? cell_ptr(a, i, j - 2) : nullptr, *yp2 = MUSCL ? cell_ptr(a, i, j + 2) : nullptr;
    const int mask = fl >> kMaskShift;
    T *out = a.fout + cell * cs;

    Acc<T> s0, s1, s2, s3;
    for (int base = lane * VEC; base < g.nv; base += 32 * VEC) {
        const int p1 = base % g.nvx, p2 = base / g.nvx;
        const T vy = T(g.vymin + p2 * g.dvy);
        const T vx0 = T(g.vxmin + p1 * g.dvx), vx1 = T(g.vxmin + (p1 + VEC - 1) * g.dvx);
        const bool sx = vx0 + vx1 >= T(0), sy = vy >= T(0);
        // upstream (u1, u2) and downstream (d1) neighbours along each axis
        const T *xu1 = sx ? xm1 : xp1, *xd1 = sx ? xp1 : xm1, *xu2 = sx ? xm2 : xp2;
        const T *yu1 = sy ? ym1 : yp1, *yd1 = sy ? yp1 : ym1, *yu2 = sy ? ym2 : yp2;
        // limiter allowed on the outflow / inflow face of each axis
        const bool mxo = sx ? (mask & 2) : (mask & 1), mxi = sx ? (mask & 1) : (mask & 2);
        const bool myo = sy ? (mask & 8) : (mask & 4), myi = sy ? (mask & 4) : (mask & 8);
        const T nuy = fabs(vy) * dtdy;
        const T cy = T(0.5) * (T(1) - nuy);
        const T eyv = ey[p2];
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
            const long o = (long)comp * g.nv + base;
            T f[VEC], u1[VEC], d1[VEC], w1[VEC], e1[VEC], u2[VEC], w2[VEC], res[VEC];
            vload<T, VEC>(self + o, f);
            vload<T, VEC>(xu1 + o, u1);
            vload<T, VEC>(yu1 + o, w1);
            if (MUSCL) {
                vload<T, VEC>(xd1 + o, d1);
                vload<T, VEC>(xu2 + o, u2);
                vload<T, VEC>(yd1 + o, e1);
                vload<T, VEC>(yu2 + o, w2);
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const T vx = T(g.vxmin + (p1 + e) * g.dvx);
                const T nux = fabs(vx) * dtdx;
                T fox = f[e], fix = u1[e], foy = f[e], fiy = w1[e];
                if (MUSCL) {
                    const T cx = T(0.5) * (T(1) - nux);
                    if (mxo) fox += cx * minmod(d1[e] - f[e], f[e] - u1[e]);
                    if (mxi) fix += cx * minmod(f[e] - u1[e], u1[e] - u2[e]);
                    if (myo) foy += cy * minmod(e1[e] - f[e], f[e] - w1[e]);
                    if (myi) fiy += cy * minmod(f[e] - w1[e], w1[e] - w2[e]);
                }
                T feq = A * ex[p1 + e] * eyv;
                if (comp == 1) feq *= gfac;
                const T fn = f[e] - nux * (fox - fix) - nuy * (foy - fiy) + r * (feq - f[e]);
                res[e] = fn;
                if (comp == 0) {
                    s0.add(fn);
                    s1.add(vx * fn);
                    s2.add(vy * fn);
                    s3.add(T(0.5) * (vx * vx + vy * vy) * fn);
                } else {
                    s3.add(fn);
                }
            }
            vstore<T, VEC>(out + o, res);
        }
    }
    s0.warp_reduce(); s1.warp_reduce(); s2.warp_reduce(); s3.warp_reduce();
    if (lane == 0)
        store_moments<T>(a.mom + cell * 8, g.dv, s0.value(), s1.value(), s2.value(), s3.value(), a.err);
}

// ------------------------------------------------------------ control volumes
struct CvArgs {
    Grid2D g;
    Geo2D Gn, Gp;
    const int32_t *master;
    const uint8_t *flags;
    const int32_t *spec_list;
    const int32_t *wall_list;
    const int32_t *counts;
    int cap;                  // capacity of spec_list and wall_list
    const double *wphi, *wux, *wuy, *wT;
    int *err;
};

// Ordered list of the members of control volume m (cells whose master is m),
// scanned in row-major order over the window reachable by the master search.
// Returns the count (capped at kMaxMembers with the capacity flag set).
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

// Fusion (Eq. FusionDD): f_CV = sum sbar f / S over a merged control volume,
// written back to every member, with the moments of the result.
template <typename T>
__global__ void __launch_bounds__(256) k_fusion(CvArgs c, T *f, T *mom)
{
    __shared__ int32_t mem[kMaxMembers];
    __shared__ double sb[kMaxMembers];
    __shared__ double red[8 * 4];
    const Grid2D &g = c.g;
    const int n = min(c.counts[0], c.cap);
    const long cs = 2L * g.nv;
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
                for (int q = 0; q < nm; ++q) s += sb[q] * (double)f[mem[q] * cs + comp * g.nv + p];
                const T fcv = (T)(s / S);
                for (int q = 0; q < nm; ++q) f[mem[q] * cs + comp * g.nv + p] = fcv;
                const double vx = g.vxmin + (p % g.nvx) * g.dvx, vy = g.vymin + (p / g.nvx) * g.dvy;
                if (comp == 0) { a0 += fcv; a1 += vx * fcv; a2 += vy * fcv; a3 += 0.5 * (vx * vx + vy * vy) * fcv; }
                else a3 += fcv;
            }
        a0 = block_sum(a0, red); a1 = block_sum(a1, red + 8);
        a2 = block_sum(a2, red + 16); a3 = block_sum(a3, red + 24);
        if (threadIdx.x < nm) {
            T *mm = mom + (long)mem[threadIdx.x] * 8;
            store_moments<T>(mm, g.dv, (T)a0, (T)a1, (T)a2, (T)a3, c.err);
        }
        __syncthreads();
    }
}

// Wall density (Eq. BoundaryDDv), stress (Eq. StressTensorDD) and the
// cell's force and torque contribution (Eqs. eq-force, eq-torque), FP64.
// The wall velocity is u_w = u_c + (r - c)^perp omega (Eq. uwDD) at t^n; with
// nseg > 0 the wall temperature is that of the angular sector of r - c.
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

template <typename T>
__global__ void __launch_bounds__(256) k_wall(CvArgs c, BodyParams b, const BodyDev *body,
                                              const T *f, double *wphi, double *wux, double *wuy,
                                              double *wT, double *wcontrib)
{
    __shared__ double red[8 * 8];
    const Grid2D &g = c.g;
    const int n = min(c.counts[1], c.cap);
    const long cs = 2L * g.nv;
    const double omega = body->omega;
    const int ni = g.i1 - g.i0;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const long k = c.wall_list[idx];
        const double rx = c.Gn.rwx[k] - b.cx, ry = c.Gn.rwy[k] - b.cy;
        const double uwx = b.vbx - ry * omega, uwy = b.vby + rx * omega;
        const double Tw = wall_temperature(b, rx, ry);
        const double nwx = c.Gn.nwx[k], nwy = c.Gn.nwy[k], lw = c.Gn.lw[k];
        const double cm = 1.0 / (2.0 * kPi * Tw);
        double num = 0, den = 0, ixx = 0, ixy = 0, iyy = 0, oxx = 0, oxy = 0, oyy = 0;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const double ax = g.vxmin + (p % g.nvx) * g.dvx - uwx;
            const double ay = g.vymin + (p / g.nvx) * g.dvy - uwy;
            const double cp = ax * nwx + ay * nwy;
            if (cp > 0) {
                const double fv = (double)f[k * cs + p];
                num += cp * fv;
                oxx += ax * ax * fv; oxy += ax * ay * fv; oyy += ay * ay * fv;
            } else if (cp < 0) {
                const double m1 = cm * exp(-(ax * ax + ay * ay) / (2.0 * Tw));
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
            wphi[k] = phi; wux[k] = uwx; wuy[k] = uwy; wT[k] = Tw;
            const int i = (int)(k % g.nx), j = (int)(k / g.nx);
            const long t = (long)(j - g.j0) * ni + (i - g.i0);
            wcontrib[3 * t] = fx;
            wcontrib[3 * t + 1] = fy;
            wcontrib[3 * t + 2] = rx * fy - ry * fx;
        }
        __syncthreads();
    }
}

// Value of virtual cell (i, j), component comp, velocity p, with the
// domain boundary conditions.
template <typename T>
__device__ __forceinline__ T fval(const Grid2D &g, const T *f, const T *const *ghost, int i, int j,
                                  int comp, int p)
{
    const long cs = 2L * g.nv;
    if (i < 0) {
        if (g.bc[0] == DVM_BC_PERIODIC) i = ((i % g.nx) + g.nx) % g.nx;
        else if (g.bc[0] == DVM_BC_MAXWELLIAN) return ghost[0][j * cs + comp * g.nv + p];
        else i = 0;
    } else if (i >= g.nx) {
        if (g.bc[1] == DVM_BC_PERIODIC) i = i % g.nx;
        else if (g.bc[1] == DVM_BC_MAXWELLIAN) return ghost[1][j * cs + comp * g.nv + p];
        else i = g.nx - 1;
    }
    if (j < 0) {
        if (g.bc[2] == DVM_BC_PERIODIC) j = ((j % g.ny) + g.ny) % g.ny;
        else if (g.bc[2] == DVM_BC_MAXWELLIAN) return ghost[2][i * cs + comp * g.nv + p];
        else j = 0;
    } else if (j >= g.ny) {
        if (g.bc[3] == DVM_BC_PERIODIC) j = j % g.ny;
        else if (g.bc[3] == DVM_BC_MAXWELLIAN) return ghost[3][i * cs + comp * g.nv + p];
        else j = g.ny - 1;
    }
    return f[((long)j * g.nx + i) * cs + comp * g.nv + p];
}

// Explicit update of one control volume (Eq. ExSchemeDD): fluxes across the
// Cartesian and wall edges of every member (Eq. FluxDD), area ratio
// S^n / S^{n+1,*}, relaxation, then distribution to the members (Eq.
// UpdateDD; members solid at t^{n+1} hold 0) and the moments of the result.
template <typename T>
__global__ void __launch_bounds__(256) k_special(CvArgs c, const T *fin, T *fout, T *mom,
                                                 const T *g0, const T *g1, const T *g2, const T *g3)
{
    __shared__ int32_t mem[kMaxMembers];
    __shared__ double L[kMaxMembers][5];      // lx-, lx+, ly-, ly+, lw
    __shared__ double W[kMaxMembers][6];      // nwx, nwy, phi, uwx, uwy, Tw
    __shared__ int8_t mk[kMaxMembers];        // limiter mask
    __shared__ int8_t live[kMaxMembers];      // non-solid at t^n
    __shared__ int8_t keep[kMaxMembers];      // non-solid at t^{n+1}
    __shared__ double red[8 * 4];
    const Grid2D &g = c.g;
    const T *ghost[4] = {g0, g1, g2, g3};
    const int n = min(c.counts[0], c.cap);
    const long cs = 2L * g.nv;
    const int W1 = g.nx + 1;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const long m = c.spec_list[idx];
        const int nm = gather_members(c, m, mem);
        for (int q = threadIdx.x; q < nm; q += blockDim.x) {
            const long k = mem[q];
            const int i = (int)(k % g.nx), j = (int)(k / g.nx);
            L[q][0] = c.Gn.lx[(long)j * W1 + i];
            L[q][1] = c.Gn.lx[(long)j * W1 + i + 1];
            L[q][2] = c.Gn.ly[(long)j * g.nx + i];
            L[q][3] = c.Gn.ly[(long)(j + 1) * g.nx + i];
            const bool wall = c.Gn.type[k] == DVM_CUT && c.Gn.lw[k] > 0;
            L[q][4] = wall ? c.Gn.lw[k] : 0.0;
            W[q][0] = c.Gn.nwx[k]; W[q][1] = c.Gn.nwy[k];
            W[q][2] = wall ? c.wphi[k] : 0.0;
            W[q][3] = wall ? c.wux[k] : 0.0; W[q][4] = wall ? c.wuy[k] : 0.0;
            W[q][5] = wall ? c.wT[k] : 1.0;
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
        const T rho = mom[m * 8], ux = mom[m * 8 + 1], uy = mom[m * 8 + 2], tmp = mom[m * 8 + 4];
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
                    const T fc = fin[k * cs + comp * g.nv + p];
                    const T fxm1 = fval(g, fin, ghost, i - 1, j, comp, p), fxp1 = fval(g, fin, ghost, i + 1, j, comp, p);
                    const T fym1 = fval(g, fin, ghost, i, j - 1, comp, p), fyp1 = fval(g, fin, ghost, i, j + 1, comp, p);
                    T fxm2 = 0, fxp2 = 0, fym2 = 0, fyp2 = 0;
                    if (mk[q]) {
                        fxm2 = fval(g, fin, ghost, i - 2, j, comp, p); fxp2 = fval(g, fin, ghost, i + 2, j, comp, p);
                        fym2 = fval(g, fin, ghost, i, j - 2, comp, p); fyp2 = fval(g, fin, ghost, i, j + 2, comp, p);
                    }
                    const T Fxp = face_flux<T>(T(L[q][1]), vx, nux, fxm1, fc, fxp1, fxp2, mk[q] & 2);
                    const T Fxm = face_flux<T>(T(L[q][0]), vx, nux, fxm2, fxm1, fc, fxp1, mk[q] & 1);
                    const T Fyp = face_flux<T>(T(L[q][3]), vy, nuy, fym1, fc, fyp1, fyp2, mk[q] & 8);
                    const T Fym = face_flux<T>(T(L[q][2]), vy, nuy, fym2, fym1, fc, fyp1, mk[q] & 4);
                    T Fw = 0;
                    if (L[q][4] > 0) {
                        const double ax = (g.vxmin + p1 * g.dvx) - W[q][3];
                        const double ay = (g.vymin + p2 * g.dvy) - W[q][4];
                        const double cp = ax * W[q][0] + ay * W[q][1];
                        const double Tw = W[q][5];
                        const double m1 = exp(-(ax * ax + ay * ay) / (2.0 * Tw)) / (2.0 * kPi * Tw);
                        const double fw = comp == 0 ? W[q][2] * m1 : W[q][2] * (Tw / 2.0 * m1);
                        Fw = (T)(L[q][4] * (fmin(cp, 0.0) * fw + fmax(cp, 0.0) * (double)fc));
                    }
                    R += (Fxp - Fxm) + (Fyp - Fym) + Fw;
                }
                const T fcv = fin[m * cs + comp * g.nv + p];
                const T feq = comp == 0 ? feq0 : tmp / T(2) * feq0;
                const T fn = a * fcv - bco * R + a * r * (feq - fcv);
                for (int q = 0; q < nm; ++q)
                    fout[(long)mem[q] * cs + comp * g.nv + p] = keep[q] ? fn : T(0);
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
        if (threadIdx.x < nm) {
            T *mm = mom + (long)mem[threadIdx.x] * 8;
            if (keep[threadIdx.x]) store_moments<T>(mm, g.dv, (T)t0, (T)t1, (T)t2, (T)t3, c.err);
            else for (int q = 0; q < 8; ++q) mm[q] = 0;
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

// Force and torque of the step (fixed-order sum over the body box), angular
// velocity at t^{n+1} (Eq. motionDD_vit) and the history record.
__global__ void __launch_bounds__(256) k_reduce_ode(const double *wcontrib, int nbox, BodyDev *b,
                                                   BodyParams bp, double dt, int moving,
                                                   double *hist, long long step)
{
    __shared__ double red[8 * 3];
    double fx = 0, fy = 0, tq = 0;
    for (int t = threadIdx.x; t < nbox; t += blockDim.x) {
        fx += wcontrib[3 * t]; fy += wcontrib[3 * t + 1]; tq += wcontrib[3 * t + 2];
    }
    fx = block_sum(fx, red); fy = block_sum(fy, red + 8); tq = block_sum(tq, red + 16);
    if (threadIdx.x == 0) {
        b->F[0] = fx; b->F[1] = fy; b->F[2] = 0; b->torque = tq;
        const double om1 = moving ? b->omega + dt * tq / bp.inertia : b->omega;
        b->theta = b->theta1;
        b->omega = om1;
        b->trig[0] = b->trig[2];
        b->trig[1] = b->trig[3];
        double *h = hist + 6 * (step % kHistCap);
        h[0] = fx; h[1] = fy; h[2] = 0; h[3] = tq; h[4] = b->theta; h[5] = om1;
    }
}

// Moments of the current state for every cell (warp per cell), used when a
// state is installed.  Solid cells (zero state) give zeros.
template <typename T>
__global__ void __launch_bounds__(256) k_moments(Grid2D g, const T *f, T *mom, const int8_t *type,
                                                 int *err)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= (long)g.nx * g.ny) return;
    const T *fk = f + cell * 2L * g.nv;
    Acc<T> s0, s1, s2, s3;
    for (int p = lane; p < g.nv; p += 32) {
        const T vx = T(g.vxmin + (p % g.nvx) * g.dvx), vy = T(g.vymin + (p / g.nvx) * g.dvy);
        const T fv = fk[p];
        s0.add(fv); s1.add(vx * fv); s2.add(vy * fv);
        s3.add(T(0.5) * (vx * vx + vy * vy) * fv);
        s3.add(fk[g.nv + p]);
    }
    s0.warp_reduce(); s1.warp_reduce(); s2.warp_reduce(); s3.warp_reduce();
    if (lane == 0) {
        if (type[cell] == DVM_SOLID) {
            for (int q = 0; q < 8; ++q) mom[cell * 8 + q] = 0;
        } else {
            store_moments<T>(mom + cell * 8, g.dv, s0.value(), s1.value(), s2.value(), s3.value(), err);
        }
    }
}

// FP64 moments for output: rho, ux, uy, uz(=0), T per cell.
template <typename T>
__global__ void __launch_bounds__(256) k_moments_out(Grid2D g, const T *f, double *out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= (long)g.nx * g.ny) return;
    const T *fk = f + cell * 2L * g.nv;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int p = lane; p < g.nv; p += 32) {
        const double vx = g.vxmin + (p % g.nvx) * g.dvx, vy = g.vymin + (p / g.nvx) * g.dvy;
        const double fv = (double)fk[p];
        s0 += fv; s1 += vx * fv; s2 += vy * fv;
        s3 += 0.5 * (vx * vx + vy * vy) * fv + (double)fk[g.nv + p];
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
    f[k * 2L * g.nv + p] = (T)m;
    f[k * 2L * g.nv + g.nv + p] = (T)(q[4] / 2.0 * m);
}

// Ghost states of a Maxwellian side from (rho, ux, uy, uz, T) per side cell.
template <typename T>
__global__ void k_ghost(Grid2D g, const double *prim, int ncell_side, T *gh)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)ncell_side * g.nv) return;
    const long q = t / g.nv;
    const int p = (int)(t % g.nv);
    const double *s = prim + 5 * q;
    const double ax = g.vxmin + (p % g.nvx) * g.dvx - s[1];
    const double ay = g.vymin + (p / g.nvx) * g.dvy - s[2];
    const double m = s[0] / (2.0 * kPi * s[4]) * exp(-(ax * ax + ay * ay) / (2.0 * s[4]));
    gh[q * 2L * g.nv + p] = (T)m;
    gh[q * 2L * g.nv + g.nv + p] = (T)(s[4] / 2.0 * m);
}

// Per-cell mass sbar * sum_p f dv (FP64), then a fixed-order sum.
template <typename T>
__global__ void __launch_bounds__(256) k_mass_cells(Grid2D g, const T *f, const double *sbar, double *cm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long cell = (long)blockIdx.x * 8 + warp;
    if (cell >= (long)g.nx * g.ny) return;
    double s = 0;
    for (int p = lane; p < g.nv; p += 32) s += (double)f[cell * 2L * g.nv + p];
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

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

template <typename T, int VEC, bool MUSCL>
cudaError_t launch_bulk(dvm_ctx *c, const StepArgs<T> &a)
{
    const long nc = (long)c->nx * c->ny;
    const size_t sm = 8 * (size_t)(c->nvx + c->nvy) * sizeof(T);
    k_bulk<T, VEC, MUSCL><<<nblk(nc, 8), 256, sm, c->stream>>>(a);
    return cudaGetLastError();
}

// Widest vector such that every aligned group of VEC velocities along x lies
// in one row and has one sign of v_x (zero allowed).
int pick_vec(const dvm_ctx *c, int vmax)
{
    for (int v = vmax; v > 1; v >>= 1) {
        if (c->nvx % v) continue;
        bool ok = true;
        for (int g0 = 0; g0 < c->nvx && ok; g0 += v) {
            double a = c->vxmin + g0 * c->dvx, b = c->vxmin + (g0 + v - 1) * c->dvx;
            if (a < 0 && b > 0) ok = false;
        }
        if (ok) return v;
    }
    return 1;
}

template <typename T>
cudaError_t step2d_t(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    BodyParams bp = body_params(c);
    const bool body = c->body.shape != DVM_SHAPE_NONE;
    const bool moving = c->moving;
    const int nbox = (g.i1 - g.i0) * (g.j1 - g.j0);
    T *fin = (T *)c->f[c->cur], *fout = (T *)c->f[1 - c->cur];
    T *mom = (T *)c->mom;
    cudaError_t e = cudaSuccess;
    if (body) {
        k_advance<<<1, 32, 0, c->stream>>>(c->d_body, c->dt, moving ? 1 : 0);
        c->launches += 1;
        if (moving) {
            c->launches += 6;
            if ((e = geometry2d_level(c, 1 - c->gcur, body_trig(c, 2))) != cudaSuccess) return e;
            if ((e = masters_flags2d(c, true)) != cudaSuccess) return e;
        }
    }
    CvArgs cv;
    cv.g = g;
    cv.Gn = c->geo[c->gcur];
    cv.Gp = moving ? c->geo[1 - c->gcur] : c->geo[c->gcur];
    cv.master = c->master; cv.flags = c->flags;
    cv.spec_list = c->spec_list; cv.wall_list = c->wall_list; cv.counts = c->counts;
    cv.wphi = c->wphi; cv.wux = c->wux; cv.wuy = c->wuy; cv.wT = c->wT;
    cv.err = c->d_err;
    cv.cap = c->list_cap;
    const int cvgrid = 4 * 152;
    if (body) {
        if (moving || c->need_fusion) {
            k_fusion<T><<<cvgrid, 256, 0, c->stream>>>(cv, fin, mom);
            c->launches += 1;
        }
        c->launches += 1;
        k_wall<T><<<cvgrid, 256, 0, c->stream>>>(cv, bp, c->d_body, fin, c->wphi, c->wux, c->wuy,
                                                  c->wT, c->wcontrib);
    }
    StepArgs<T> a;
    a.g = g; a.fin = fin; a.fout = fout; a.mom = mom; a.flags = c->flags; a.err = c->d_err;
    for (int s = 0; s < 4; ++s) a.ghost[s] = (const T *)c->ghost[s];
    const bool muscl = c->scheme == DVM_MUSCL;
    const int vec = pick_vec(c, sizeof(T) == 4 ? 4 : 2);
    if ((e = timing_mark(c, 0)) != cudaSuccess) return e;
    if (sizeof(T) == 4 && vec == 4) e = muscl ? launch_bulk<T, 4, true>(c, a) : launch_bulk<T, 4, false>(c, a);
    else if (vec >= 2) e = muscl ? launch_bulk<T, 2, true>(c, a) : launch_bulk<T, 2, false>(c, a);
    else e = muscl ? launch_bulk<T, 1, true>(c, a) : launch_bulk<T, 1, false>(c, a);
    if (e != cudaSuccess) return e;
    if ((e = timing_mark(c, 1)) != cudaSuccess) return e;
    c->launches += 1;
    if (body) {
        k_special<T><<<cvgrid, 256, 0, c->stream>>>(cv, fin, fout, mom, a.ghost[0], a.ghost[1],
                                                     a.ghost[2], a.ghost[3]);
        k_reduce_ode<<<1, 256, 0, c->stream>>>(c->wcontrib, nbox, c->d_body, bp, c->dt,
                                               moving ? 1 : 0, c->d_hist, c->steps_done);
        c->launches += 2;
    }
    c->cur = 1 - c->cur;
    if (moving) c->gcur = 1 - c->gcur;
    c->need_fusion = false;
    c->steps_done++;
    return cudaGetLastError();
}

}  // namespace

cudaError_t step2d(dvm_ctx *c)
{
    return c->prec == DVM_FP32 ? step2d_t<float>(c) : step2d_t<double>(c);
}

cudaError_t moments2d(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    const long nc = (long)c->nx * c->ny;
    if (c->prec == DVM_FP32)
        k_moments<float><<<nblk(nc, 8), 256, 0, c->stream>>>(g, (const float *)c->f[c->cur],
                                                             (float *)c->mom, c->geo[c->gcur].type, c->d_err);
    else
        k_moments<double><<<nblk(nc, 8), 256, 0, c->stream>>>(g, (const double *)c->f[c->cur],
                                                              (double *)c->mom, c->geo[c->gcur].type, c->d_err);
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
        k_ghost<float><<<nblk(n, 256), 256, 0, c->stream>>>(g, d_prim, nside, (float *)c->ghost[side]);
    else
        k_ghost<double><<<nblk(n, 256), 256, 0, c->stream>>>(g, d_prim, nside, (double *)c->ghost[side]);
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
