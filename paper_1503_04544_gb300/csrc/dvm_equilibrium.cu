// Conservative discrete equilibrium (arXiv:1503.04544, Sec. 3.1, the
// paragraph after Eq. MacroscopicDDv): the (rho, u, T) put into the
// equilibrium of a control volume are not its direct moments but the ones
// whose discrete equilibrium on the velocity grid has the same discrete
// moments (mass, momentum, energy) as the state, so that the collision term
// conserves them exactly on the grid.  The paper finds them by a Newton
// algorithm; the root does not depend on the variant.
//
// k_eqpar: one thread per cell, plain Newton steps from the direct moments.
// The Maxwellian is separable on the Cartesian velocity grid,
// M(v) = K prod_a e_a(v_a) with e_a = exp(-(v_a - u_a)^2 / (2T)) and
// K = rho / (2 pi T)^(D/2), so every discrete moment and every entry of the
// Jacobian is K times a product of 1D sums over one axis:
//   R_a^j = sum_k v_k^j e_a(v_k) h_a,  j = 0..4,
// with dR^j/du = (R^{j+1} - u R^j) / T and
// dR^j/dT = (R^{j+2} - 2 u R^{j+1} + u^2 R^j) / (2 T^2).  An iteration costs
// sum_a n_a exponentials instead of prod_a n_a.  Equations (D = 2 reduced,
// g_eq = T/2 M; D = 3 full F):
//   K R_x^0 R_y^0 (R_z^0)             = rho_f           (mass)
//   K R_a^1 prod_{b != a} R_b^0       = (rho u_a)_f     (momentum)
//   K/2 sum_a R_a^2 prod_{b != a} R_b^0 (+ T/2 mass)    = E_f (energy)
// The cell's moment sums are the partial sums the step kernels write.  The
// FP32 path solves in FP32 with the hardware exp2, the FP64 path in FP64.
#include <cuda_runtime.h>

#include "dvm_device.cuh"

namespace dvm {
namespace {

constexpr int kNewtonMax = 10;
constexpr int kEqThreads = 64;

template <typename T> __device__ __forceinline__ T eq_exp2(T x);
template <> __device__ __forceinline__ float eq_exp2<float>(float x) { return ex2_fast(x); }
template <> __device__ __forceinline__ double eq_exp2<double>(double x) { return exp2(x); }

struct EqArgs {
    long nc;
    int S;                    // partial-sum slots
    const void *part;         // [S][D + 2][nc] moment sums (2D: f, vx f, vy f, |v|^2/2 f + g)
    void *eqp;                // [D + 2][nc] rho, u_1..u_D, T of the equilibrium
    int n[3];                 // velocity points per axis
    double v0[3], h[3];       // v_k = v0 + k h
    double dv;                // velocity cell measure
    int *err;
};

// Solves A x = b for n = N by Gaussian elimination with partial pivoting
// (the largest remaining |A[i][k]| is brought to row k by conditional swaps,
// so every index is a compile-time constant and A stays in registers); false
// for a zero pivot.
template <typename T, int N>
__device__ __forceinline__ bool solve_n(T (&A)[N][N], T (&b)[N], T (&x)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const bool sw = fabs(A[i][k]) > fabs(A[k][k]);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T u = A[k][j], v = A[i][j];
                A[k][j] = sw ? v : u;
                A[i][j] = sw ? u : v;
            }
            const T u = b[k], v = b[i];
            b[k] = sw ? v : u;
            b[i] = sw ? u : v;
        }
        if (!(fabs(A[k][k]) > T(0))) return false;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const T l = A[i][k] / A[k][k];
#pragma unroll
            for (int j = k; j < N; ++j) A[i][j] -= l * A[k][j];
            b[i] -= l * b[k];
        }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        T s = b[i];
#pragma unroll
        for (int j = i + 1; j < N; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return true;
}

// One row of moments and Jacobian: w K prod_a R_a^{e_a}, e = (e_0, .., e_{D-1}).
template <typename T, int D>
__device__ __forceinline__ void add_term(const T (&R)[D][5], const T (&dRu)[D][3], const T (&dRT)[D][3],
                                         const int (&e)[D], T w, T K, T dKdT, T rho, T &m, T (&Jrow)[D + 2])
{
    T P = T(1);
#pragma unroll
    for (int a = 0; a < D; ++a) P *= R[a][e[a]];
    m += w * K * P;
    Jrow[0] += w * K * P / rho;
    T dT = dKdT * P;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        T rest = T(1);
#pragma unroll
        for (int b = 0; b < D; ++b)
            if (b != a) rest *= R[b][e[b]];
        Jrow[1 + a] += w * K * dRu[a][e[a]] * rest;
        dT += K * dRT[a][e[a]] * rest;
    }
    Jrow[D + 1] += w * dT;
}

// Sums over one velocity axis, R^j = sum_k v_k^j exp2(-(v_k - u)^2 c) h,
// j = 0..4 (returned by value, so that no array is indexed at run time).
template <typename T> struct Sum5 { T r0, r1, r2, r3, r4; };

template <typename T>
__device__ __forceinline__ Sum5<T> axis_sums(const T *v, int n, T u, T c, T h)
{
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
    for (int k = 0; k < n; ++k) {
        const T vk = v[k], x = vk - u;
        T p = eq_exp2<T>(-(x * x) * c) * h;
        s0 += p; p *= vk; s1 += p; p *= vk; s2 += p; p *= vk; s3 += p; p *= vk; s4 += p;
    }
    return Sum5<T>{s0, s1, s2, s3, s4};
}

// One thread per cell.
template <typename T, int D>
__global__ void __launch_bounds__(kEqThreads) k_eqpar(EqArgs a)
{
    constexpr int N = D + 2;
    __shared__ T vax[3][kMaxAxisNv];
    for (int k = threadIdx.x; k < kMaxAxisNv; k += blockDim.x) {
        vax[0][k] = k < a.n[0] ? T(a.v0[0] + k * a.h[0]) : T(0);
        vax[1][k] = k < a.n[1] ? T(a.v0[1] + k * a.h[1]) : T(0);
        vax[2][k] = D == 3 && k < a.n[2] ? T(a.v0[2] + k * a.h[2]) : T(0);
    }
    __syncthreads();
    const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.nc) return;
    const T *part = static_cast<const T *>(a.part);
    T *eqp = static_cast<T *>(a.eqp);
    Acc<T> acc[N];
    for (int q = 0; q < a.S; ++q)
#pragma unroll
        for (int m = 0; m < N; ++m) acc[m].merge(part[((long)q * N + m) * a.nc + cell], T(0));
    const T dv = T(a.dv);
    T tgt[N];
#pragma unroll
    for (int m = 0; m < N; ++m) tgt[m] = acc[m].value() * dv;
    T th[N];
#pragma unroll
    for (int m = 0; m < N; ++m) th[m] = T(0);
    if (tgt[0] > T(0)) {
        // direct moments: the start of the iteration
        th[0] = tgt[0];
        T u2 = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            th[1 + d] = tgt[1 + d] / tgt[0];
            u2 += th[1 + d] * th[1 + d];
        }
        th[N - 1] = (T(2) * tgt[N - 1] / tgt[0] - u2) / T(3);
        // stop once a step is below tol (relative to rho, sqrt(T), T); a
        // last step below loose (the rounding floor of the FP32 sums on hot
        // or cold cells) is accepted, a larger one or a non-positive
        // density or temperature is an error
        const T tol = sizeof(T) == 4 ? T(1e-6) : T(1e-13);
        const T loose = sizeof(T) == 4 ? T(1e-4) : T(1e-10);
        bool ok = th[N - 1] > T(0), done = false;
        T last = T(1);
        T dir[N];
#pragma unroll
        for (int m = 0; m < N; ++m) dir[m] = th[m];
        const T hx = T(a.h[0]), hy = T(a.h[1]), hz = T(a.h[2]);
        for (int it = 0; it < kNewtonMax && ok && !done; ++it) {
            const T rho = th[0], Tt = th[N - 1];
            const T c = T(kLog2e) / (T(2) * Tt);
            T R[D][5], dRu[D][3], dRT[D][3];
            {
                const Sum5<T> sx = axis_sums<T>(vax[0], a.n[0], th[1], c, hx);
                const Sum5<T> sy = axis_sums<T>(vax[1], a.n[1], th[2], c, hy);
                R[0][0] = sx.r0; R[0][1] = sx.r1; R[0][2] = sx.r2; R[0][3] = sx.r3; R[0][4] = sx.r4;
                R[1][0] = sy.r0; R[1][1] = sy.r1; R[1][2] = sy.r2; R[1][3] = sy.r3; R[1][4] = sy.r4;
                if constexpr (D == 3) {
                    const Sum5<T> sz = axis_sums<T>(vax[2], a.n[2], th[3], c, hz);
                    R[D - 1][0] = sz.r0; R[D - 1][1] = sz.r1; R[D - 1][2] = sz.r2; R[D - 1][3] = sz.r3;
                    R[D - 1][4] = sz.r4;
                }
            }
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const T u = th[1 + d];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    dRu[d][j] = (R[d][j + 1] - u * R[d][j]) / Tt;
                    dRT[d][j] = (R[d][j + 2] - T(2) * u * R[d][j + 1] + u * u * R[d][j]) / (T(2) * Tt * Tt);
                }
            }
            T K = rho / (T(2.0 * kPi) * Tt);
            if (D == 3) K /= sqrt(T(2.0 * kPi) * Tt);
            const T dKdT = -K * T(D) / (T(2) * Tt);
            T m[N], J[N][N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                m[i] = T(0);
#pragma unroll
                for (int j = 0; j < N; ++j) J[i][j] = T(0);
            }
            {
                int e[D];
#pragma unroll
                for (int d = 0; d < D; ++d) e[d] = 0;
                add_term<T, D>(R, dRu, dRT, e, T(1), K, dKdT, rho, m[0], J[0]);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    e[d] = 1;
                    add_term<T, D>(R, dRu, dRT, e, T(1), K, dKdT, rho, m[1 + d], J[1 + d]);
                    e[d] = 2;
                    add_term<T, D>(R, dRu, dRT, e, T(0.5), K, dKdT, rho, m[N - 1], J[N - 1]);
                    e[d] = 0;
                }
            }
            if (D == 2) {
                // the g component: T/2 M adds T/2 times the mass row to the
                // energy, and M/2 to its T derivative
#pragma unroll
                for (int j = 0; j < N; ++j) J[N - 1][j] += Tt / T(2) * J[0][j];
                J[N - 1][N - 1] += m[0] / T(2);
                m[N - 1] += Tt / T(2) * m[0];
            }
            T res[N], step[N];
#pragma unroll
            for (int i = 0; i < N; ++i) res[i] = tgt[i] - m[i];
            if (!solve_n<T, N>(J, res, step)) { ok = false; break; }
            T big = fabs(step[0]) / rho;
            const T st = sqrt(Tt);
#pragma unroll
            for (int d = 0; d < D; ++d) big = fmax(big, fabs(step[1 + d]) / st);
            big = fmax(big, fabs(step[N - 1]) / Tt);
#pragma unroll
            for (int i = 0; i < N; ++i) th[i] += step[i];
            ok = th[0] > T(0) && th[N - 1] > T(0) && big == big;
            done = big < tol;
            last = big;
        }
        if (!ok || !(done || last < loose)) {
            atomicExch(&a.err[kErrNonphys], 1);
#pragma unroll
            for (int i = 0; i < N; ++i) th[i] = dir[i];
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) eqp[(long)i * a.nc + cell] = th[i];
}

}  // namespace

// Equilibrium parameters of every cell from the moment sums `part` (S slots
// of the layout of the context's partial sums) into c->eqp.
cudaError_t eqpar(dvm_ctx *c, const void *part, int S)
{
    EqArgs a;
    a.nc = c->nc;
    a.S = S;
    a.part = part;
    a.eqp = c->eqp;
    // the whole velocity grid (that of the velocity split when one is set:
    // the moment sums are then over every rank's velocities)
    for (int d = 0; d < 3; ++d) { a.n[d] = c->gnv[d]; a.v0[d] = c->gv0[d]; a.h[d] = c->gdv[d]; }
    a.dv = c->gdv[0] * c->gdv[1] * (c->dim == 3 ? c->gdv[2] : 1.0);
    a.err = c->d_err;
    const unsigned blocks = (unsigned)((c->nc + kEqThreads - 1) / kEqThreads);
    if (c->dim == 2) {
        if (c->prec == DVM_FP32) k_eqpar<float, 2><<<blocks, kEqThreads, 0, c->stream>>>(a);
        else k_eqpar<double, 2><<<blocks, kEqThreads, 0, c->stream>>>(a);
    } else {
        if (c->prec == DVM_FP32) k_eqpar<float, 3><<<blocks, kEqThreads, 0, c->stream>>>(a);
        else k_eqpar<double, 3><<<blocks, kEqThreads, 0, c->stream>>>(a);
    }
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace dvm
