// Discrete adjoint of the 2D fixed-body step (arXiv:1503.04544, Sec. 3.3.5)
// for the drag J = F_x of the state after N steps (Eqs. StressTensorDD,
// eq-force), with respect to the state, the per-sector wall temperatures and
// the Maxwellian inflow states; the paper has no adjoint, the method's step
// is differentiated as it stands.
//
// One step is F^n -> fusion (Eq. FusionDD) -> moments, wall density, fluxes,
// explicit update with relaxation (Eqs. BGKDD, BoundaryDDv, FluxDD,
// ExSchemeDD) -> distribution (Eq. UpdateDD).  Its transposed Jacobian is
// applied to lambda^{n+1} in the reverse order:
//   k_adj_mu       transpose of the distribution: mu = sum of lambda over the
//                  members of each cut/merged control volume;
//   k_adj_relax    per control volume and velocity split: the relaxation
//                  through the moments (sums over the velocities of
//                  mu dM/d(rho, u, T)), finished by k_adj_relax_fin;
//   k_adj_gather_* per (cell, velocity): relaxation terms and the face-flux
//                  transposes of every face whose stencil reads the cell;
//                  the limiter derivative is the one of the branch the
//                  forward step took (recorded by the recomputation for
//                  the cells deep in the gas, re-derived from F^n elsewhere);
//   k_adj_wall_*   per wall cell: the diffuse flux and the wall density
//                  coupling (Eq. BoundaryDDv), and dJ/dT_w;
//   k_adj_pads*    the boundary pads: the step reads them but does not
//                  update them, so their sensitivities are gathered like a
//                  cell's and folded back onto the cells they copy
//                  (periodic, zero-gradient) or chained to (rho, u, T) of
//                  the Maxwellian ghost state;
//   k_adj_fuseT    transpose of the fusion of merged control volumes; it
//                  also forms mu of the result for the next transposed
//                  step, which then skips k_adj_mu.
// The driver dvm_drag_adjoint checkpoints the forward run every K steps,
// recomputes each segment onto a device tape and sweeps it backwards.
#include <cstring>
#include <string>
#include <vector>

#include "dvm_device.cuh"

namespace dvm {
namespace {

struct AdjArgs {
    Grid2D g;
    Geo2D G;
    BodyParams b;
    const int32_t *master;
    const uint8_t *flags;
    const int32_t *spec_list;
    const int32_t *wall_list;
    const int32_t *counts;
    int cap;
    const void *cvinfo;
    const void *vt;
    const int32_t *cvx;       // special control-volume index of a cell's master, -1 if plain
    const void *bown;         // dt / S of the cell's control volume (state precision), 0 if none
    int muscl;
    double omega;
    int *err;                 // device error flags (kErrTimeout)
};

// minmod with the derivative of the branch taken (ties: the second argument).
template <typename T>
__device__ __forceinline__ void minmod_d(T a, T b, T &da, T &db)
{
    da = db = T(0);
    if (a > T(0) && b > T(0)) { if (a < b) da = T(1); else db = T(1); }
    else if (a < T(0) && b < T(0)) { if (a > b) da = T(1); else db = T(1); }
}

// Derivatives of the face flux L v phi(fAA, fA, fB, fBB) (Eq. FluxDD with the
// limited reconstruction) with respect to its four stencil values.
template <typename T>
__device__ __forceinline__ void face_flux_d(T L, T v, T nu, T fAA, T fA, T fB, T fBB, bool muscl, T (&d)[4])
{
    d[0] = d[1] = d[2] = d[3] = T(0);
    if (!muscl) { d[1] = L * fmax(v, T(0)); d[2] = L * fmin(v, T(0)); return; }
    const T k = T(0.5) * (T(1) - nu);
    T da, db;
    if (v > T(0)) {
        minmod_d(fB - fA, fA - fAA, da, db);
        d[1] = L * v * (T(1) + k * (db - da));
        d[2] = L * v * (k * da);
        d[0] = L * v * (-k * db);
    } else if (v < T(0)) {
        minmod_d(fBB - fB, fB - fA, da, db);
        d[2] = L * v * (T(1) - k * (db - da));
        d[3] = L * v * (-k * da);
        d[1] = L * v * (k * db);
    }
}

// Adjoint of the control volume that owns cell k (mu), for component comp and
// padded velocity p; b of that control volume.
template <typename T>
__device__ __forceinline__ T mu_of(const AdjArgs &a, const T *lam, const T *mucv, int k, int comp, int p)
{
    const int cx = a.cvx[k];
    if (cx >= 0) return mucv[((long)cx * 2 + comp) * a.g.nvp + p];
    return lam[ebase<T>(a.g, comp, p) + pcell(a.g, k) * Vec<T>::W];
}

// mu of cell k for the W velocities of the group starting at p.
template <typename T>
__device__ __forceinline__ void mu_of_v(const AdjArgs &a, const T *lam, const T *mucv, int k, int comp, int p,
                                        T (&r)[Vec<T>::W])
{
    using V = typename Vec<T>::type;
    const int cx = a.cvx[k];
    if (cx >= 0) vld<T>(reinterpret_cast<const V *>(mucv + ((long)cx * 2 + comp) * a.g.nvp + p), r);
    else vld<T>(reinterpret_cast<const V *>(lam + ebase<T>(a.g, comp, p)) + pcell(a.g, k), r);
}

// ------------------------------------------------------------ set-up
__global__ void k_adj_rev(const int32_t *spec_list, const int32_t *counts, int cap, int32_t *rev)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < min(counts[0], cap)) rev[spec_list[idx]] = idx;
}

template <typename T>
__global__ void k_adj_setup(Grid2D g, const int32_t *master, const uint8_t *flags, const int32_t *rev,
                            const CvInfo *info, int32_t *cvx, T *bown)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long)g.nx * g.ny) return;
    const int m = master[k];
    if (m < 0) { cvx[k] = -1; bown[k] = T(0); return; }
    if (flags[m] & kSpecial) {
        const int idx = rev[m];
        cvx[k] = idx;
        bown[k] = (T)info[idx].bco;
    } else {
        cvx[k] = -1;
        bown[k] = (T)(g.dt / (g.dx * g.dy));
    }
}

// ------------------------------------------------------------ step kernels
// mu of every cut or merged control volume: the sum of lambda over its
// members (one block per (control volume, chunk of velocities)).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_mu(AdjArgs a, const T *lam, T *mucv)
{
    __shared__ long pcs[kMaxMembers];
    const CvInfo &I = reinterpret_cast<const CvInfo *>(a.cvinfo)[blockIdx.x];
    constexpr int W = Vec<T>::W;
    const int nm = I.nm;
    if (threadIdx.x < nm) pcs[threadIdx.x] = I.mem[threadIdx.x].pc * W;
    __syncthreads();
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= 2 * a.g.nvp) return;
    const int comp = e / a.g.nvp, p = e - comp * a.g.nvp;
    const long base = ebase<T>(a.g, comp, p);
    T s = 0;
    for (int t = 0; t < nm; ++t) s += lam[base + pcs[t]];
    mucv[((long)blockIdx.x * 2 + comp) * a.g.nvp + p] = s;
}

// Relaxation through the moments, per control volume and velocity split
// (one thread per master cell, 32 consecutive cells along x per warp, vector
// loads of each velocity group; split blockIdx.z takes every gridDim.z-th
// block of groups): with G = F - b R + r (Feq - F), r = dt rho / tau0, the
// partial sums over the split of mu r dFeq/d(rho, ux, uy, T) and of
// mu (Feq - F) dt/tau0, rpart[z][5][nc].
template <typename T>
__device__ __forceinline__ void cell_moments(const Grid2D &g, const T *part, int S, long m, T &rho, T &ux, T &uy,
                                             T &E, T &tmp)
{
    const long nc = (long)g.nx * g.ny;
    Acc<T> s0, s1, s2, s3;
    for (int q = 0; q < S; ++q) {
        s0.merge(part[((long)q * 4 + 0) * nc + m], T(0));
        s1.merge(part[((long)q * 4 + 1) * nc + m], T(0));
        s2.merge(part[((long)q * 4 + 2) * nc + m], T(0));
        s3.merge(part[((long)q * 4 + 3) * nc + m], T(0));
    }
    const T dv = pick<T>(g.dv_f, g.dv);
    rho = s0.value() * dv;
    ux = s1.value() / s0.value();
    uy = s2.value() / s0.value();
    E = s3.value() * dv;
    tmp = (T(2) * E / rho - (ux * ux + uy * uy)) / T(3);
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_relax(AdjArgs a, const T *f, const T *part, int S, const T *lam,
                                                   const T *mucv, T *rpart)
{
    const Grid2D &g = a.g;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int m = j * g.nx + i;
    if (a.master[m] != m) return;
    constexpr int W = Vec<T>::W;
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(a.vt);
    const long pc = nbr(g, i, j) * W;
    const long nc = (long)g.nx * g.ny;
    T rho, ux, uy, E, tmp;
    cell_moments<T>(g, part, S, m, rho, ux, uy, E, tmp);
    const T dtt = pick<T>(g.dt_tau0_f, g.dt_tau0);
    const T r = dtt * rho;
    const T A = rho / (T(2.0 * kPi) * tmp), i2T = T(1) / (T(2) * tmp), c2 = T(kLog2e) * i2T;
    const T h = tmp / T(2);
    const int cx = a.cvx[m];
    const int gps = (g.ngrp + gridDim.z - 1) / gridDim.z;
    const int q0 = blockIdx.z * gps, q1 = min(q0 + gps, g.ngrp);
    // with u = mu_f + T/2 mu_g: dM/drho = M / rho, dM/du = M (v - u) / T,
    // dM/dT = M (|v - u|^2 / (2T) - 1) / T, d(T/2 M) = T/2 dM + M/2 dT; the
    // factors 1/rho and 1/T are applied once after the sums
    Acc<T> a0, a1, a2, a3, ar;
    for (int q = q0; q < q1; ++q) {
        const int p = q * W;
        T fv[W], gv[W], mf[W], mg[W];
        vld<T>(reinterpret_cast<const typename Vec<T>::type *>(f + ebase<T>(g, 0, p) + pc), fv);
        vld<T>(reinterpret_cast<const typename Vec<T>::type *>(f + ebase<T>(g, 1, p) + pc), gv);
        if (cx >= 0) {
#pragma unroll
            for (int e = 0; e < W; ++e) {
                mf[e] = mucv[((long)cx * 2) * g.nvp + p + e];
                mg[e] = mucv[((long)cx * 2 + 1) * g.nvp + p + e];
            }
        } else {
            vld<T>(reinterpret_cast<const typename Vec<T>::type *>(lam + ebase<T>(g, 0, p) + pc), mf);
            vld<T>(reinterpret_cast<const typename Vec<T>::type *>(lam + ebase<T>(g, 1, p) + pc), mg);
        }
        T t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, tr = 0;
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const VCoef<T> vc = ld_coef(vt + p + e);
            const T ax = vc.vx - ux, ay = vc.vy - uy, a2 = ax * ax + ay * ay;
            const T M = A * dexp2(-a2 * c2);
            const T mu = M * (mf[e] + h * mg[e]);
            t0 += mu;
            t1 += mu * ax;
            t2 += mu * ay;
            t3 += mu * (a2 * i2T - T(1));
            t4 += mg[e] * M;
            tr += mf[e] * (M - fv[e]) + mg[e] * (h * M - gv[e]);
        }
        a0.add(t0); a1.add(t1); a2.add(t2); a3.add(t3 + t4 * T(0.5) * tmp); ar.add(tr);
    }
    const T rr = r / rho, rt = r / tmp;
    T *o = rpart + (long)blockIdx.z * 5 * nc + m;
    o[0] = rr * a0.value(); o[nc] = rt * a1.value(); o[2 * nc] = rt * a2.value(); o[3 * nc] = rt * a3.value();
    o[4 * nc] = dtt * ar.value();
}

// Sum of the splits and the chain to the conserved moments:
// aux[m] = (r, S0, S1, S2, S3), S = d/d(rho, rho ux, rho uy, E).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_relax_fin(AdjArgs a, const T *part, int S, const T *rpart, int Z,
                                                       T *aux)
{
    const Grid2D &g = a.g;
    const long m = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nc = (long)g.nx * g.ny;
    if (m >= nc || a.master[m] != m) return;
    T rho, ux, uy, E, tmp;
    cell_moments<T>(g, part, S, m, rho, ux, uy, E, tmp);
    Acc<T> q0, q1, q2, q3, qr;
    for (int z = 0; z < Z; ++z) {
        const T *o = rpart + (long)z * 5 * nc + m;
        q0.merge(o[0], T(0)); q1.merge(o[nc], T(0)); q2.merge(o[2 * nc], T(0)); q3.merge(o[3 * nc], T(0));
        qr.merge(o[4 * nc], T(0));
    }
    const T r = pick<T>(g.dt_tau0_f, g.dt_tau0) * rho;
    const T sp0 = q0.value() + qr.value(), sp1 = q1.value(), sp2 = q2.value(), sp3 = q3.value();
    const T S0 = sp0 - sp1 * ux / rho - sp2 * uy / rho +
                 sp3 * (T(-2) * E / (rho * rho) + T(2) * (ux * ux + uy * uy) / rho) / T(3);
    const T S1 = sp1 / rho - sp3 * T(2) * ux / (T(3) * rho);
    const T S2 = sp2 / rho - sp3 * T(2) * uy / (T(3) * rho);
    const T S3 = sp3 * T(2) / (T(3) * rho);
    T *o = aux + 5 * m;
    o[0] = r; o[1] = S0; o[2] = S1; o[3] = S2; o[4] = S3;
}

// Sum over the faces along one axis whose stencil reads padded position
// (ti, tj) -- a cell, or a boundary pad along the axis -- of the weight W_f
// (adjoint of the two control volumes the face separates) times the flux
// derivative at that stencil slot, for the W velocities of the group at p.
// The faces are those between positions ii and ii + 1 along the axis for
// ii = c - 2 .. c + 1.  The step reads the pads but does not update them: a
// pad on either side of a face adds no weight, and a face between two pads
// none at all.
template <typename T>
__device__ void gather_axis(const AdjArgs &a, const T *f, const T *lam, const T *mucv, int axis, int ti, int tj,
                            int comp, int p, const T (&v)[Vec<T>::W], const T (&nu)[Vec<T>::W],
                            T (&acc)[Vec<T>::W])
{
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    const Grid2D &g = a.g;
    const int n = axis == 0 ? g.nx : g.ny;
    const int c = axis == 0 ? ti : tj;
    const V *F = reinterpret_cast<const V *>(f + ebase<T>(g, comp, p));
    const T *bown = reinterpret_cast<const T *>(a.bown);
    for (int ii = c - 2; ii <= c + 1; ++ii) {
        const bool aint = ii >= 0 && ii < n, bint = ii + 1 >= 0 && ii + 1 < n;
        if (!aint && !bint) continue;
        // the face between A (position ii) and B (position ii + 1) along the axis
        const int ia = axis == 0 ? ii : ti, ja = axis == 0 ? tj : ii;
        const int ib = axis == 0 ? ii + 1 : ti, jb = axis == 0 ? tj : ii + 1;
        const int A = aint ? ja * g.nx + ia : -1;
        const int B = bint ? jb * g.nx + ib : -1;
        // length and limiter flag as the forward step uses them
        T L;
        bool lim;
        if (A >= 0) {
            L = axis == 0 ? (T)a.G.lx[(long)ja * (g.nx + 1) + ia + 1] : (T)a.G.ly[(long)(ja + 1) * g.nx + ia];
            lim = a.muscl && ((a.flags[A] >> kMaskShift) & (axis == 0 ? 2 : 8));
        } else {
            L = axis == 0 ? (T)a.G.lx[(long)jb * (g.nx + 1) + ib] : (T)a.G.ly[(long)jb * g.nx + ib];
            lim = a.muscl && ((a.flags[B] >> kMaskShift) & (axis == 0 ? 1 : 4));
        }
        if (L == T(0)) continue;
        const T bA = A >= 0 ? bown[A] : T(0), bB = B >= 0 ? bown[B] : T(0);
        if (bA == T(0) && bB == T(0)) continue;
        T Wf[W], mA[W], mB[W];
        if (bA != T(0)) mu_of_v<T>(a, lam, mucv, A, comp, p, mA);
        if (bB != T(0)) mu_of_v<T>(a, lam, mucv, B, comp, p, mB);
#pragma unroll
        for (int e = 0; e < W; ++e) Wf[e] = (bA != T(0) ? -bA * mA[e] : T(0)) + (bB != T(0) ? bB * mB[e] : T(0));
        // stencil AA, A, B, BB (positions ii - 1 .. ii + 2, within the padding)
        T fv[4][W];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int pos = ii - 1 + t;
            vld<T>(F + nbr(g, axis == 0 ? pos : ti, axis == 0 ? tj : pos), fv[t]);
        }
        const int slot = c - ii + 1;
#pragma unroll
        for (int e = 0; e < W; ++e) {
            T d[4];
            face_flux_d<T>(L, v[e], nu[e], fv[0][e], fv[1][e], fv[2][e], fv[3][e], lim, d);
            acc[e] += Wf[e] * d[slot];
        }
    }
}

// What the generic gather needs of one face whose stencil reads a listed
// cell, fixed for a fixed body: the adjoint sources of its two sides (>= 0:
// padded cell of lambda; < 0: -(index + 1) of a merged control volume's mu),
// their weights b (0 for a pad), the face length, the padded cells of its
// four stencil values, the stencil slot of the listed cell, and whether the
// limiter is used (bit 0) and the record is live (bit 1).
template <typename T> struct __align__(16) FaceRec {
    int srcA, srcB;
    int fpos[4];
    T L, bA, bB;
    int bits;                 // 1: limiter, 2: live; slot in bits 4..5
};

// Face records of the listed cells: record (idx, axis, t) is the face
// between positions c - 2 + t and c - 1 + t along the axis (the loop of
// gather_axis); one thread per record.
template <typename T>
__global__ void k_adj_listrec(AdjArgs a, const int32_t *list, int nlist, FaceRec<T> *rec)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nlist * 8) return;
    const Grid2D &g = a.g;
    const int idx = (int)(t >> 3), axis = (int)((t >> 2) & 1), slotf = (int)(t & 3);
    const int k = list[idx];
    int ti, tj;
    cell_ij(g, k, ti, tj);
    const int n = axis == 0 ? g.nx : g.ny;
    const int c = axis == 0 ? ti : tj;
    const int ii = c - 2 + slotf;
    FaceRec<T> R{};
    const bool aint = ii >= 0 && ii < n, bint = ii + 1 >= 0 && ii + 1 < n;
    if (aint || bint) {
        const int ia = axis == 0 ? ii : ti, ja = axis == 0 ? tj : ii;
        const int ib = axis == 0 ? ii + 1 : ti, jb = axis == 0 ? tj : ii + 1;
        const int A = aint ? ja * g.nx + ia : -1;
        const int B = bint ? jb * g.nx + ib : -1;
        T L;
        bool lim;
        if (A >= 0) {
            L = axis == 0 ? (T)a.G.lx[(long)ja * (g.nx + 1) + ia + 1] : (T)a.G.ly[(long)(ja + 1) * g.nx + ia];
            lim = a.muscl && ((a.flags[A] >> kMaskShift) & (axis == 0 ? 2 : 8));
        } else {
            L = axis == 0 ? (T)a.G.lx[(long)jb * (g.nx + 1) + ib] : (T)a.G.ly[(long)jb * g.nx + ib];
            lim = a.muscl && ((a.flags[B] >> kMaskShift) & (axis == 0 ? 1 : 4));
        }
        const T *bown = reinterpret_cast<const T *>(a.bown);
        const T bA = A >= 0 ? bown[A] : T(0), bB = B >= 0 ? bown[B] : T(0);
        if (L != T(0) && (bA != T(0) || bB != T(0))) {
            const auto src = [&](int cell) { return a.cvx[cell] >= 0 ? -(a.cvx[cell] + 1) : (int)pcell(g, cell); };
            R.srcA = bA != T(0) ? src(A) : 0;
            R.srcB = bB != T(0) ? src(B) : 0;
            for (int q = 0; q < 4; ++q) {
                const int pos = ii - 1 + q;
                R.fpos[q] = (int)nbr(g, axis == 0 ? pos : ti, axis == 0 ? tj : pos);
            }
            R.L = L; R.bA = bA; R.bB = bB;
            R.bits = (lim ? 1 : 0) | 2 | ((c - ii + 1) << 4);
        }
    }
    rec[t] = R;
}

// lambda or mu of an adjoint source for the W velocities at p.
template <typename T>
__device__ __forceinline__ void src_load(const Grid2D &g, const T *lam, const T *mucv, int src, int comp, int p,
                                         T (&r)[Vec<T>::W])
{
    using V = typename Vec<T>::type;
    if (src < 0) vld<T>(reinterpret_cast<const V *>(mucv + ((long)(-src - 1) * 2 + comp) * g.nvp + p), r);
    else vld<T>(reinterpret_cast<const V *>(lam + ebase<T>(g, comp, p)) + src, r);
}

// Generic gather over the listed cells from their face records: relaxation
// terms for control-volume masters and the face-flux transposes along both
// axes.  A block takes 64 (listed cell, velocity group) items, consecutive on
// consecutive listed cells; its four quarters take the (component, axis)
// pairs, four face records each, and the sums meet in shared memory.
constexpr int kRecItems = 64;
template <typename T>
__global__ void __launch_bounds__(4 * kRecItems) k_adj_gather_rec(AdjArgs a, const T *f, const T *lam,
                                                                  const T *mucv, const T *aux, const int32_t *list,
                                                                  int nlist, const FaceRec<T> *rec, T *lam_out)
{
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    __shared__ T part[4][kRecItems][W];
    const Grid2D &g = a.g;
    const int sub = threadIdx.x / kRecItems, it = threadIdx.x % kRecItems;
    const int comp = sub >> 1, ax = sub & 1;
    const long t = (long)blockIdx.x * kRecItems + it;
    const bool live = t < (long)nlist * g.ngrp;
    const int q = live ? (int)(t / nlist) : 0, idx = live ? (int)(t % nlist) : 0;
    const int p = q * W;
    T acc[W];
#pragma unroll
    for (int e = 0; e < W; ++e) acc[e] = T(0);
    if (live) {
        T v[W], nu[W];
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const VCoef<T> vc = ld_coef(reinterpret_cast<const VCoef<T> *>(a.vt) + p + e);
            v[e] = ax ? vc.vy : vc.vx;
            nu[e] = ax ? vc.nuy : vc.nux;
        }
        const V *F = reinterpret_cast<const V *>(f + ebase<T>(g, comp, p));
        const FaceRec<T> *R0 = rec + (long)idx * 8 + ax * 4;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const FaceRec<T> R = R0[r];
            if (!(R.bits & 2)) continue;
            T mA[W], mB[W], fv[4][W];
            if (R.bA != T(0)) src_load<T>(g, lam, mucv, R.srcA, comp, p, mA);
            if (R.bB != T(0)) src_load<T>(g, lam, mucv, R.srcB, comp, p, mB);
#pragma unroll
            for (int u = 0; u < 4; ++u) vld<T>(F + R.fpos[u], fv[u]);
            const int slot = (R.bits >> 4) & 3;
            const bool lim = R.bits & 1;
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const T Wf = (R.bA != T(0) ? -R.bA * mA[e] : T(0)) + (R.bB != T(0) ? R.bB * mB[e] : T(0));
                T d[4];
                face_flux_d<T>(R.L, v[e], nu[e], fv[0][e], fv[1][e], fv[2][e], fv[3][e], lim, d);
                acc[e] += Wf * d[slot];
            }
        }
    }
#pragma unroll
    for (int e = 0; e < W; ++e) part[sub][it][e] = acc[e];
    __syncthreads();
    if (sub >= 2 || !live) return;
    // quarter 0 and 1: component 0 and 1 of the item, relaxation terms
    const int k = list[idx];
    T out[W], vx[W], vy[W];
#pragma unroll
    for (int e = 0; e < W; ++e) {
        const VCoef<T> vc = ld_coef(reinterpret_cast<const VCoef<T> *>(a.vt) + p + e);
        vx[e] = vc.vx; vy[e] = vc.vy;
        out[e] = T(0);
    }
    if (a.master[k] == k) {
        const T dv = pick<T>(g.dv_f, g.dv);
        const T *o = aux + 5 * (long)k;
        T m[W];
        mu_of_v<T>(a, lam, mucv, k, sub, p, m);
#pragma unroll
        for (int e = 0; e < W; ++e)
            out[e] = m[e] * (T(1) - o[0]) +
                     (sub == 0 ? dv * (o[1] + o[2] * vx[e] + o[3] * vy[e] + o[4] * T(0.5) * (vx[e] * vx[e] + vy[e] * vy[e]))
                               : dv * o[4]);
    }
#pragma unroll
    for (int e = 0; e < W; ++e) {
        out[e] += part[sub * 2][it][e] + part[sub * 2 + 1][it][e];
        if (p + e >= g.nv) out[e] = T(0);
    }
    vst<T>(reinterpret_cast<V *>(lam_out + ebase<T>(g, sub, p)) + pcell(g, k), out);
}

// Transpose of the face fluxes along one axis for a cell deep in the gas, in
// the upwind direction u of the velocity: the face downwind of position m
// carries |v| L phi_m from m to m + u, phi_m = F_m + k mm(F_{m+u} - F_m,
// F_m - F_{m-u}) with k = (1 - nu)/2, and its adjoint weight is b |v| L
// (lambda_{m+u} - lambda_m) = nu (lambda_{m+u} - lambda_m) between plain
// cells (b = dt/(dx dy)).  The cell receives the weights of the faces
// downwind of k - u, k, k + u times the derivative of their phi with respect
// to F_k; sm, sk, sp are the recorded branches of those three faces (1: the
// first minmod argument, 2: the second, 0: none or first order).
// lm, l0, lp, lq: lambda at k - u, k, k + u, k + 2u (0 at pads).
template <typename T, bool MUSCL>
__device__ __forceinline__ T adj_axis(T kap, T lm, T l0, T lp, T lq, uint32_t sm, uint32_t sk, uint32_t sp)
{
    const T wk = lp - l0;
    if (!MUSCL) return wk;
    T corr = T(0);
    if (sk & 1u) corr -= wk;
    else if (sk & 2u) corr += wk;
    if (sm & 1u) corr += l0 - lm;
    if (sp & 2u) corr -= lq - lp;
    return wk + kap * corr;
}

// Shared-memory stages of the fast gather: lambda of both components of one
// velocity group over the block's cells and a two-cell halo, and the branch
// words of the same tile (row of 36 words), 128-byte aligned.
constexpr int kAdjStages = 4;
constexpr int kAdjLamBytes = 2 * kTileY * kTileX * 16;
constexpr int kAdjBitsBytes = ((kTileY * kTileX * 4 + 127) / 128) * 128;
constexpr int kAdjStageBytes = kAdjLamBytes + kAdjBitsBytes;
static_assert(kAdjLamBytes % 128 == 0 && kAdjStageBytes % 128 == 0,
              "tensor-copy destinations start on 128-byte boundaries");

// Fast gather for the cells flagged in fast[] (one thread per cell, 32 x
// kRows cells per block, the velocity groups split over blockIdx.z),
// relaxation terms included.  Reads lambda^{n+1} and, for MUSCL, the limiter
// branches recorded for F^n, not F^n itself.  Each group's tile of lambda
// (both components) and of the branch words arrives by TMA in a
// kAdjStages-deep shared-memory ring on "full" mbarriers; each warp releases
// a stage on its "empty" mbarrier, and thread 0 refills a stage only after
// all warps released it.  Every wait is bounded (on timeout the kernel sets
// kErrTimeout and goes on).  Other cells are left to k_adj_gather_rec.
template <typename T, bool MUSCL>
__global__ void __launch_bounds__(32 * kRows, 2) k_adj_gather_fast(AdjArgs a, const __grid_constant__ CUtensorMap lmap,
                                                                   const __grid_constant__ CUtensorMap bmap,
                                                                   const int8_t *gsign, const T *aux,
                                                                   const uint8_t *fast, T *lam_out)
{
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr uint32_t kBytes = MUSCL ? kAdjLamBytes + kTileY * kTileX * 4 : kAdjLamBytes;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kAdjStages * kAdjStageBytes);
    uint64_t *empty = full + kAdjStages;
    const Grid2D &g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * kRows;
    const int i = i0 + tx, j = j0 + ty;
    const bool inside = i < g.nx && j < g.ny;
    const long k = inside ? (long)j * g.nx + i : 0;
    const bool isfast = inside && fast[k];
    const int gps = (g.ngrp + gridDim.z - 1) / gridDim.z;
    const int g0 = blockIdx.z * gps, g1 = min(g0 + gps, g.ngrp);
    const int ngr = max(g1 - g0, 0);
    const auto issue = [&](int st, int q) {
        unsigned char *dst = smem + (long)st * kAdjStageBytes;
        mbar_expect_tx(&full[st], kBytes);
        tma_load_3d(dst, &lmap, &full[st], i0 * W, j0, q * 2);
        if (MUSCL) tma_load_3d(dst + kAdjLamBytes, &bmap, &full[st], i0, j0, q);
    };
    if (tid == 0) {
        for (int st = 0; st < kAdjStages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], kRows);
        }
        mbar_fence_init();
        for (int st = 0; st < kAdjStages - 1 && st < ngr; ++st) issue(st, g0 + st);
    }
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(a.vt);
    T omr = 0, S0 = 0, S1 = 0, S2 = 0, S3 = 0;
    if (isfast) {
        const T *o = aux + 5 * k;
        omr = T(1) - o[0]; S0 = o[1]; S1 = o[2]; S2 = o[3]; S3 = o[4];
    }
    const T dv = pick<T>(g.dv_f, g.dv);
    const long pc = nbr(g, i, j);
    const int c0 = (ty + 2) * kTileX + tx + 2;
    __syncthreads();

    for (int it = 0; it < ngr; ++it) {
        const int q = g0 + it, st = it % kAdjStages;
        if (tid == 0 && it + kAdjStages - 1 < ngr) {
            const int kk = it + kAdjStages - 1, s2 = kk % kAdjStages;
            if (kk >= kAdjStages && !mbar_wait(&empty[s2], (uint32_t)((kk / kAdjStages - 1) & 1)))
                atomicExch(&a.err[kErrTimeout], 1);
            issue(s2, g0 + kk);
        }
        if (!mbar_wait(&full[st], (uint32_t)((it / kAdjStages) & 1))) atomicExch(&a.err[kErrTimeout], 1);
        if (isfast) {
            const unsigned char *base = smem + (long)st * kAdjStageBytes;
            const uint32_t *bt = reinterpret_cast<const uint32_t *>(base + kAdjLamBytes);
            const int p = q * W;
            T vx[W], vy[W], nux[W], nuy[W], rel0[W];
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const VCoef<T> vc = ld_coef(vt + p + e);
                vx[e] = vc.vx; vy[e] = vc.vy; nux[e] = vc.nux; nuy[e] = vc.nuy;
                rel0[e] = dv * (S0 + S1 * vx[e] + S2 * vy[e] + S3 * T(0.5) * (vx[e] * vx[e] + vy[e] * vy[e]));
            }
            const int sgx = gsign[2 * q], sgy = gsign[2 * q + 1];
            uint32_t bo = 0, bxm = 0, bxp = 0, bym = 0, byp = 0;
            if (MUSCL) {
                bo = bt[c0]; bxm = bt[c0 - 1]; bxp = bt[c0 + 1]; bym = bt[c0 - kTileX]; byp = bt[c0 + kTileX];
            }
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
                const V *t = reinterpret_cast<const V *>(base) + comp * kTileY * kTileX;
                T l0[W], out[W];
                sld<T>(t + c0, l0);
                if (sgx != 0 && sgy != 0) {
                    // upwind direction uniform over the group
                    const int ux = sgx > 0 ? 1 : -1, uy = sgy > 0 ? kTileX : -kTileX;
                    T xm[W], xp[W], xq[W], ym[W], yp[W], yq[W];
                    sld<T>(t + c0 + ux, xp);
                    sld<T>(t + c0 + uy, yp);
                    if (MUSCL) {
                        sld<T>(t + c0 - ux, xm); sld<T>(t + c0 + 2 * ux, xq);
                        sld<T>(t + c0 - uy, ym); sld<T>(t + c0 + 2 * uy, yq);
                    }
                    const uint32_t smx = sgx > 0 ? bxm : bxp, spx = sgx > 0 ? bxp : bxm;
                    const uint32_t smy = sgy > 0 ? bym : byp, spy = sgy > 0 ? byp : bym;
#pragma unroll
                    for (int e = 0; e < W; ++e) {
                        const int shx = ((comp * 2 + 0) * W + e) * 2, shy = ((comp * 2 + 1) * W + e) * 2;
                        T nu = l0[e] * omr + (comp == 0 ? rel0[e] : dv * S3);
                        nu += nux[e] * adj_axis<T, MUSCL>(T(0.5) * (T(1) - nux[e]), MUSCL ? xm[e] : T(0), l0[e],
                                                          xp[e], MUSCL ? xq[e] : T(0), smx >> shx, bo >> shx,
                                                          spx >> shx);
                        nu += nuy[e] * adj_axis<T, MUSCL>(T(0.5) * (T(1) - nuy[e]), MUSCL ? ym[e] : T(0), l0[e],
                                                          yp[e], MUSCL ? yq[e] : T(0), smy >> shy, bo >> shy,
                                                          spy >> shy);
                        out[e] = p + e < g.nv ? nu : T(0);
                    }
                } else {
                    // per-element direction
                    T x2m[W], x1m[W], x1p[W], x2p[W], y2m[W], y1m[W], y1p[W], y2p[W];
                    sld<T>(t + c0 - 2, x2m); sld<T>(t + c0 - 1, x1m); sld<T>(t + c0 + 1, x1p); sld<T>(t + c0 + 2, x2p);
                    sld<T>(t + c0 - 2 * kTileX, y2m); sld<T>(t + c0 - kTileX, y1m);
                    sld<T>(t + c0 + kTileX, y1p); sld<T>(t + c0 + 2 * kTileX, y2p);
#pragma unroll
                    for (int e = 0; e < W; ++e) {
                        const int shx = ((comp * 2 + 0) * W + e) * 2, shy = ((comp * 2 + 1) * W + e) * 2;
                        const bool px = vx[e] >= T(0), py = vy[e] >= T(0);
                        T nu = l0[e] * omr + (comp == 0 ? rel0[e] : dv * S3);
                        nu += nux[e] * adj_axis<T, MUSCL>(T(0.5) * (T(1) - nux[e]), px ? x1m[e] : x1p[e], l0[e],
                                                          px ? x1p[e] : x1m[e], px ? x2p[e] : x2m[e],
                                                          (px ? bxm : bxp) >> shx, bo >> shx, (px ? bxp : bxm) >> shx);
                        nu += nuy[e] * adj_axis<T, MUSCL>(T(0.5) * (T(1) - nuy[e]), py ? y1m[e] : y1p[e], l0[e],
                                                          py ? y1p[e] : y1m[e], py ? y2p[e] : y2m[e],
                                                          (py ? bym : byp) >> shy, bo >> shy, (py ? byp : bym) >> shy);
                        out[e] = p + e < g.nv ? nu : T(0);
                    }
                }
                vst<T>(reinterpret_cast<V *>(lam_out + ebase<T>(g, comp, p)) + pc, out);
            }
        }
        __syncwarp();
        if (tx == 0) mbar_arrive(&empty[st]);
    }
    if (tid == 0) {
        // every issued copy has landed before the block exits
        for (int kk = max(ngr - kAdjStages, 0); kk < ngr; ++kk)
            mbar_wait(&full[kk % kAdjStages], (uint32_t)((kk / kAdjStages) & 1));
    }
}

// Pads beyond a side, from its boundary cell (lambda of the pads is 0, the
// branch word of the inner pad P1 is the one its boundary face recorded):
// for a velocity entering through the side the inner pad receives nu
// (lambda_0 (1 - k s1(P1) + k s2(P1)) - k s2(0) (lambda_1 - lambda_0)) and the
// outer pad -nu k s2(P1) lambda_0; for one leaving, the inner pad receives
// -nu k s1(0) lambda_0.  lambda_1 is the next cell inwards; the return value
// is the sum over both pads (both copy the boundary cell, or both hold the
// same ghost value).
template <typename T, bool MUSCL>
__device__ __forceinline__ T pad_pair(bool inward, T nu, T l0, T l1, uint32_t bp1, uint32_t bo)
{
    const T kap = T(0.5) * (T(1) - nu);
    if (inward) {
        T r = l0;
        if (MUSCL) {
            if (bp1 & 1u) r -= kap * l0;
            else if (bp1 & 2u) r += kap * l0;
            if (bo & 2u) r -= kap * (l1 - l0);
            if (bp1 & 2u) r -= kap * l0;
        }
        return nu * r;
    }
    return (MUSCL && (bo & 1u)) ? -nu * kap * l0 : T(0);
}

// Branch words of the boundary faces: for every plain cell on a side and
// velocity group, the limiter branch of its face on that side for the
// velocities entering through it, minmod(F_0 - F_P1, F_P1 - F_P2) with P1, P2
// the pads beyond the face (the upwind face of the cell, "downwind" of P1),
// written at the padded index of P1 in the branch words of F^n.  Same
// operands and direction rule as the forward step (the group's sign when its
// velocities share it, else each element's); 0 where the face is first
// order.  One thread per (side, side cell, velocity group).
template <typename T>
__device__ __forceinline__ uint32_t branch_code(T m, T b) { return m == T(0) ? 0u : (m == b ? 2u : 1u); }

template <typename T>
__global__ void __launch_bounds__(256) k_adj_padwords(Grid2D g, const T *f, const uint8_t *flags, const int8_t *gsign,
                                                      const VCoef<T> *vt, uint32_t *bits, long bslab, int bpitch)
{
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    const int nmax = g.nx > g.ny ? g.nx : g.ny;
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long per = (long)nmax * g.ngrp;
    if (t >= 4 * per) return;
    const int side = (int)(t / per);
    t %= per;
    const int q = (int)(t % nmax), grp = (int)(t / nmax), p = grp * W;
    const int axis = side >> 1;
    const int n = axis == 0 ? g.nx : g.ny, nside = axis == 0 ? g.ny : g.nx;
    if (q >= nside) return;
    const int ib = (side & 1) ? n - 1 : 0;
    const int ci = axis == 0 ? ib : q, cj = axis == 0 ? q : ib;
    const uint8_t fl = flags[(long)cj * g.nx + ci];
    if (!(fl & kPlain)) return;
    const int di = axis == 0 ? ((side & 1) ? 1 : -1) : 0, dj = axis == 1 ? ((side & 1) ? 1 : -1) : 0;
    // the incoming face on this side: x- / x+ / y- / y+ limiter mask bit
    const bool wi = (fl >> kMaskShift) & (1 << side);
    const int sg = gsign[2 * grp + axis];
    uint32_t word = 0;
    if (wi) {
        for (int comp = 0; comp < 2; ++comp) {
            const V *F = reinterpret_cast<const V *>(f + ebase<T>(g, comp, p));
            T f0[W], f1[W], f2v[W];
            vld<T>(F + nbr(g, ci, cj), f0);
            vld<T>(F + nbr(g, ci + di, cj + dj), f1);
            vld<T>(F + nbr(g, ci + 2 * di, cj + 2 * dj), f2v);
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const VCoef<T> vc = ld_coef(vt + p + e);
                const T v = axis == 0 ? vc.vx : vc.vy;
                const bool pos = sg != 0 ? sg > 0 : v >= T(0);
                const bool entering = (side & 1) ? !pos : pos;
                if (!entering) continue;
                const T a = f0[e] - f1[e], c = f1[e] - f2v[e];
                word |= branch_code(minmod3(a, c), c) << (((comp * 2 + axis) * W + e) * 2);
            }
        }
    }
    bits[(long)grp * bslab + (long)(cj + dj + 2) * bpitch + ci + di + 2] = word;
}

// Pads of a zero-gradient or Maxwellian side whose boundary cell is a fast
// cell (one thread per (side, side cell, velocity group), after the fast
// gather; the two sides of one axis together, as they touch distinct cells):
// folded onto the boundary cell (zero-gradient) or summed over the steps
// into pacc (Maxwellian; a reduction without return, one adder per address
// and step, so the sum is deterministic).
// The term of one pad: side, side cell q, velocity group grp.
template <typename T, bool MUSCL>
__device__ __forceinline__ void pad_fast_one(const AdjArgs &a, const T *lam, const uint32_t *bits, long bslab,
                                             int bpitch, int side, int q, int grp, double *pacc, int nmax,
                                             T *lam_out)
{
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    const Grid2D &g = a.g;
    pacc += (long)side * nmax * 2 * g.nv;
    const int p = grp * W;
    const int axis = side >> 1;
    const int n = axis == 0 ? g.nx : g.ny;
    const int ib = (side & 1) ? n - 1 : 0;                  // boundary cell along the axis
    const int ci = axis == 0 ? ib : q, cj = axis == 0 ? q : ib;
    const int di = axis == 0 ? ((side & 1) ? 1 : -1) : 0, dj = axis == 1 ? ((side & 1) ? 1 : -1) : 0;
    uint32_t bo = 0, bp1 = 0;
    if (MUSCL) {
        const uint32_t *bq = bits + (long)grp * bslab;
        bo = bq[(long)(cj + 2) * bpitch + ci + 2];
        bp1 = bq[(long)(cj + dj + 2) * bpitch + ci + di + 2];
    }
    T vv[W], nu[W];
#pragma unroll
    for (int e = 0; e < W; ++e) {
        const VCoef<T> vc = ld_coef(reinterpret_cast<const VCoef<T> *>(a.vt) + p + e);
        vv[e] = axis == 0 ? vc.vx : vc.vy;
        nu[e] = axis == 0 ? vc.nux : vc.nuy;
    }
    for (int comp = 0; comp < 2; ++comp) {
        const V *L = reinterpret_cast<const V *>(lam + ebase<T>(g, comp, p));
        T l0[W], l1[W], ps[W];
        vld<T>(L + nbr(g, ci, cj), l0);
        vld<T>(L + nbr(g, ci - di, cj - dj), l1);
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const int sh = ((comp * 2 + axis) * W + e) * 2;
            const bool inward = (side & 1) ? vv[e] < T(0) : vv[e] > T(0);
            ps[e] = p + e < g.nv ? pad_pair<T, MUSCL>(inward, nu[e], l0[e], l1[e], bp1 >> sh, bo >> sh) : T(0);
        }
        if (g.bc[side] == DVM_BC_MAXWELLIAN) {
            double *o = pacc + ((long)q * 2 + comp) * g.nv + p;
#pragma unroll
            for (int e = 0; e < W; ++e)
                if (p + e < g.nv) atomicAdd(o + e, (double)ps[e]);
        } else {
            V *o = reinterpret_cast<V *>(lam_out + ebase<T>(g, comp, p)) + nbr(g, ci, cj);
            T cur[W];
            vld<T>(o, cur);
#pragma unroll
            for (int e = 0; e < W; ++e) cur[e] += ps[e];
            vst<T>(o, cur);
        }
    }
}

// Pads of a zero-gradient or Maxwellian side whose boundary cell is a fast
// cell (one thread per (side, side cell, velocity group), after the fast
// gather; the two sides of one axis together, as they touch distinct cells):
// folded onto the boundary cell (zero-gradient) or summed over the steps
// into pacc (Maxwellian; a reduction without return, one adder per address
// and step, so the sum is deterministic).
template <typename T, bool MUSCL>
__global__ void __launch_bounds__(256) k_adj_pads_fast(AdjArgs a, const T *lam, const uint32_t *bits, long bslab,
                                                       int bpitch, int side0, int sides, int nside, int padmask,
                                                       const uint8_t *fast, double *pacc, int nmax, T *lam_out)
{
    const Grid2D &g = a.g;
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long per = (long)nside * g.ngrp;
    if (t >= per * sides) return;
    const int side = side0 + (int)(t / per);
    t %= per;
    if (!((padmask >> side) & 1)) return;
    const int q = (int)(t % nside), grp = (int)(t / nside);
    const int axis = side >> 1;
    const int ib = (side & 1) ? (axis == 0 ? g.nx : g.ny) - 1 : 0;
    if (!fast[axis == 0 ? (long)q * g.nx + ib : (long)ib * g.nx + q]) return;
    pad_fast_one<T, MUSCL>(a, lam, bits, bslab, bpitch, side, q, grp, pacc, nmax, lam_out);
}

// The same for the four sides in one launch (nx, ny > 1).  A corner cell's
// x-side and y-side terms both land on it when both sides fold onto the
// boundary cell: the x side's thread then adds the y side's term after its
// own (the order of one launch per axis), so no two threads update one cell.
template <typename T, bool MUSCL>
__global__ void __launch_bounds__(256) k_adj_pads_fast4(AdjArgs a, const T *lam, const uint32_t *bits, long bslab,
                                                        int bpitch, int padmask, const uint8_t *fast, double *pacc,
                                                        int nmax, T *lam_out)
{
    const Grid2D &g = a.g;
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long perx = (long)g.ny * g.ngrp, pery = (long)g.nx * g.ngrp;
    if (t >= 2 * (perx + pery)) return;
    int side;
    if (t < 2 * perx) {
        side = (int)(t / perx);
        t %= perx;
    } else {
        t -= 2 * perx;
        side = 2 + (int)(t / pery);
        t %= pery;
    }
    if (!((padmask >> side) & 1)) return;
    const int nside = side < 2 ? g.ny : g.nx;
    const int q = (int)(t % nside), grp = (int)(t / nside);
    const auto folds = [&](int s) { return ((padmask >> s) & 1) && g.bc[s] != DVM_BC_MAXWELLIAN; };
    const int axis = side >> 1;
    const int ib = (side & 1) ? (axis == 0 ? g.nx : g.ny) - 1 : 0;
    if (!fast[axis == 0 ? (long)q * g.nx + ib : (long)ib * g.nx + q]) return;
    // a corner of a folding y side: left to the x side's thread when that folds too
    if (axis == 1 && folds(side) && (q == 0 || q == g.nx - 1) && folds(q == 0 ? 0 : 1)) return;
    pad_fast_one<T, MUSCL>(a, lam, bits, bslab, bpitch, side, q, grp, pacc, nmax, lam_out);
    if (axis == 0 && folds(side) && (q == 0 || q == g.ny - 1) && folds(q == 0 ? 2 : 3))
        pad_fast_one<T, MUSCL>(a, lam, bits, bslab, bpitch, q == 0 ? 2 : 3, side == 0 ? 0 : g.nx - 1, grp, pacc,
                               nmax, lam_out);
}

// Cells eligible for the fast gather: plain gas cells whose neighbours within
// two cells along each axis are plain gas cells or boundary pads (a pad adds
// no adjoint weight; the branch of a face between a pad and a plain cell is
// recorded by that cell).
__global__ void k_adj_fastmask(Grid2D g, const uint8_t *flags, uint8_t *fast)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long)g.nx * g.ny) return;
    int i, j;
    cell_ij(g, k, i, j);
    bool ok = (flags[k] & kPlain) != 0;
    for (int d = -2; d <= 2 && ok; ++d) {
        const int ii = i + d, jj = j + d;
        ok = (ii < 0 || ii >= g.nx || (flags[(long)j * g.nx + ii] & kPlain)) &&
             (jj < 0 || jj >= g.ny || (flags[(long)jj * g.nx + i] & kPlain));
    }
    fast[k] = ok ? 1 : 0;
}

// Side cells whose pads the generic pad kernel has to gather (all of them on
// periodic sides, those whose boundary cell is not a fast cell elsewhere).
__global__ void k_adj_padcount(Grid2D g, const uint8_t *fast, int padsides, int *cnt)
{
    const int side = blockIdx.y;
    const int nside = side < 2 ? g.ny : g.nx;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nside) return;
    bool need = true;
    if ((padsides >> side) & 1) {
        const int tb = (side & 1) ? (side < 2 ? g.nx : g.ny) - 1 : 0;
        need = !fast[side < 2 ? (long)q * g.nx + tb : (long)tb * g.nx + q];
    }
    if (need) atomicAdd(&cnt[side], 1);
}

// Compact list of the cells in a control volume that are not eligible for
// the fast gather (one block); cells in no control volume keep lambda = 0.
__global__ void __launch_bounds__(1024) k_adj_slowlist(long nc, const uint8_t *fast, const int32_t *master,
                                                      int32_t *list, int *count)
{
    __shared__ int wsum[32];
    __shared__ int tot;
    int n = 0;
    for (long base = 0; base < nc; base += blockDim.x) {
        const long k = base + threadIdx.x;
        const bool slow = k < nc && !fast[k] && master[k] >= 0;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const unsigned bal = __ballot_sync(0xffffffffu, slow);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { const int v = wsum[w]; wsum[w] = acc; acc += v; }
            tot = acc;
        }
        __syncthreads();
        if (slow) list[n + wsum[warp] + __popc(bal & ((1u << lane) - 1u))] = (int32_t)k;
        n += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = n;
}

struct WallAdj {
    double uwx, uwy, Tw, rx, ry, nwx, nwy, lw;
    int sector;
};

// Sector index of a wall point (the rule of wall_temperature).
__device__ __forceinline__ int wall_sector_idx(const BodyParams &b, double rx, double ry)
{
    for (int s = 0; s < b.nseg; ++s) {
        const int t = (s + 1) % b.nseg;
        const double p = b.seg_dir[2 * s] * ry - b.seg_dir[2 * s + 1] * rx;
        const double q = b.seg_dir[2 * t] * ry - b.seg_dir[2 * t + 1] * rx;
        if (p >= 0 && q < 0) return s;
    }
    return 0;
}

__device__ __forceinline__ WallAdj wall_adj(const AdjArgs &a, long k)
{
    WallAdj w;
    w.rx = a.G.rwx[k] - a.b.cx;
    w.ry = a.G.rwy[k] - a.b.cy;
    w.uwx = a.b.vbx - w.ry * a.omega;
    w.uwy = a.b.vby + w.rx * a.omega;
    w.Tw = wall_temperature(a.b, w.rx, w.ry);
    w.sector = a.b.nseg > 0 ? wall_sector_idx(a.b, w.rx, w.ry) : 0;
    w.nwx = a.G.nwx[k]; w.nwy = a.G.nwy[k]; w.lw = a.G.lw[k];
    return w;
}

// Per (wall cell, velocity): c = (v - u_w) . n_w, and M1, dM1/dT_w for c < 0;
// in FP64 (the objective) and in the state precision (the transposed steps).
struct __align__(16) WallVel {
    double cp, m1, dm1;
};
template <typename T> struct WallVelT {
    T cp, m1, dm1;
};

// Per wall cell, once per adjoint run (the body is fixed): the wall data,
// and per velocity c = (v - u_w) . n_w and, for the velocities leaving the
// gas (c < 0), the wall Maxwellian M1 = M[1, u_w, T_w] and dM1/dT_w; with
// D = sum_{c<0} c M1 dv and dD/dT_w.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_wall_pre(AdjArgs a, int nw, WallAdj *wadj, WallVel *wm, WallVelT<T> *wt,
                                                      double2 *wd, int32_t *wsec)
{
    __shared__ double red[8 * 2];
    const Grid2D &g = a.g;
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(a.vt);
    const double dv = g.dv;
    for (int idx = blockIdx.x; idx < nw; idx += gridDim.x) {
        const WallAdj w = wall_adj(a, a.wall_list[idx]);
        const double cmw = 1.0 / (2.0 * kPi * w.Tw);
        double den = 0, dD = 0;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const VCoef<T> vc = ld_coef(vt + p);
            const double ax = (double)vc.vx - w.uwx, ay = (double)vc.vy - w.uwy;
            const double cp = ax * w.nwx + ay * w.nwy;
            double m1 = 0, dm1 = 0;
            if (cp < 0) {
                const double a2 = ax * ax + ay * ay;
                m1 = cmw * exp(-a2 / (2.0 * w.Tw));
                dm1 = m1 * (a2 / (2.0 * w.Tw * w.Tw) - 1.0 / w.Tw);
                den += cp * m1 * dv;
                dD += cp * dm1 * dv;
            }
            wm[(long)idx * g.nv + p] = WallVel{cp, m1, dm1};
            wt[(long)idx * g.nv + p] = WallVelT<T>{(T)cp, (T)m1, (T)dm1};
        }
        den = block_sum(den, red);
        dD = block_sum(dD, red + 8);
        if (threadIdx.x == 0) {
            wadj[idx] = w;
            wd[idx] = make_double2(den, dD);
            wsec[idx] = w.sector;
        }
        __syncthreads();
    }
}

// Wall cells of a transposed step: the diffuse flux lw (min(c,0) phi M1 +
// max(c,0) F) of the update, through phi = -sum_{c>0} c f dv / D, D =
// sum_{c<0} c M1 dv, with dJ/dT_w per wall slot.  One block per wall cell;
// the per-velocity terms in the state precision with compensated sums (FP64
// arithmetic is scarce on this GPU), phi and the T_w chain in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_wall_step(AdjArgs a, int nw, const WallAdj *wadj,
                                                       const WallVelT<T> *wt, const double2 *wd, const T *f,
                                                       const T *lam, const T *mucv, T *lam_out, double *gtw)
{
    __shared__ T red[8 * 2];
    const Grid2D &g = a.g;
    const T *bown = reinterpret_cast<const T *>(a.bown);
    constexpr int W = Vec<T>::W;
    for (int idx = blockIdx.x; idx < nw; idx += gridDim.x) {
        const int k = a.wall_list[idx];
        const WallAdj w = wadj[idx];
        const long pk = pcell(g, k) * W;
        const T hT = (T)(0.5 * w.Tw), blw = -bown[k] * (T)w.lw;
        const WallVelT<T> *tab = wt + (long)idx * g.nv;
        Acc<T> num, sphi, sTw;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const WallVelT<T> m = tab[p];
            if (m.cp > T(0)) {
                num.add(m.cp * f[ebase<T>(g, 0, p) + pk]);
            } else if (m.cp < T(0)) {
                const T w0 = blw * mu_of<T>(a, lam, mucv, k, 0, p);
                const T w1 = blw * mu_of<T>(a, lam, mucv, k, 1, p);
                sphi.add(m.cp * m.m1 * (w0 + w1 * hT));
                sTw.add(m.cp * (w0 * m.dm1 + w1 * (T(0.5) * m.m1 + hT * m.dm1)));   // times phi below
            }
        }
        const double numd = (double)block_acc(num, red) * g.dv;
        const double sphid = (double)block_acc(sphi, red);
        const double sTwd = (double)block_acc(sTw, red);
        const double2 D = wd[idx];
        const double phi = -numd / D.x;
        const T sd = (T)(-sphid * g.dv / D.x);
        // per-velocity terms of the wall cell
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const T cp = tab[p].cp;
            if (!(cp > T(0))) continue;
            const long e0 = ebase<T>(g, 0, p) + pk, e1 = ebase<T>(g, 1, p) + pk;
            lam_out[e0] += cp * (sd + blw * mu_of<T>(a, lam, mucv, k, 0, p));
            lam_out[e1] += cp * blw * mu_of<T>(a, lam, mucv, k, 1, p);
        }
        if (threadIdx.x == 0) gtw[idx] += phi * sTwd + sphid * (-phi / D.x) * D.y;
        __syncthreads();
    }
}

// The objective J = F_x of the wall stress (Eqs. StressTensorDD, eq-force) on
// the wall cells: dJ/dF into lambda (outgoing velocities directly, incoming
// ones through phi = -sum_{c>0} c f dv / D), J per wall slot and its direct
// T_w derivative.  One block per wall cell, FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_wall_obj(AdjArgs a, int nw, const WallAdj *wadj, const WallVel *wm,
                                                      const double2 *wd, const T *f, T *lam_out, double *gtw,
                                                      double *jwall)
{
    __shared__ double red[8 * 5];
    const Grid2D &g = a.g;
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(a.vt);
    constexpr int W = Vec<T>::W;
    const double dv = g.dv;
    for (int idx = blockIdx.x; idx < nw; idx += gridDim.x) {
        const int k = a.wall_list[idx];
        const WallAdj w = wadj[idx];
        const long pk = pcell(g, k) * W;
        const WallVel *tab = wm + (long)idx * g.nv;
        // sums over the velocities (the dv of num, sxx, sxy applied after the sums)
        double num = 0, sphi = 0, sTw = 0, sxx = 0, sxy = 0;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const WallVel m = tab[p];
            const VCoef<T> vc = ld_coef(vt + p);
            const double ax = (double)vc.vx - w.uwx, ay = (double)vc.vy - w.uwy;
            if (m.cp > 0) {
                const double fv = (double)f[ebase<T>(g, 0, p) + pk];
                num += m.cp * fv;
                sxx += ax * ax * fv; sxy += ax * ay * fv;
            } else if (m.cp < 0) {
                const double wgt = (ax * ax * w.nwx + ax * ay * w.nwy) * w.lw * dv;
                sphi += wgt * m.m1;
                sTw += wgt * m.dm1;          // times phi below
            }
        }
        num = block_sum(num, red) * dv; sphi = block_sum(sphi, red + 8); sTw = block_sum(sTw, red + 16);
        sxx = block_sum(sxx, red + 24) * dv; sxy = block_sum(sxy, red + 32) * dv;
        const double2 D = wd[idx];
        const double phi = -num / D.x, sd = -sphi * dv / D.x;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const double cp = tab[p].cp;
            if (!(cp > 0)) continue;
            const VCoef<T> vc = ld_coef(vt + p);
            const double ax = (double)vc.vx - w.uwx, ay = (double)vc.vy - w.uwy;
            const long e0 = ebase<T>(g, 0, p) + pk;
            lam_out[e0] = (T)((double)lam_out[e0] + sd * cp + (ax * ax * w.nwx + ax * ay * w.nwy) * w.lw * dv);
        }
        if (threadIdx.x == 0) {
            gtw[idx] += phi * sTw + sphi * (-phi / D.x) * D.y;
            // the incoming part of the stress: phi times the M1 sums
            jwall[idx] = (sxx * w.nwx + sxy * w.nwy) * w.lw + phi * sphi;
        }
        __syncthreads();
    }
}

// Transpose of the fusion: lam_k = (sbar_k / S) sum_{j in CV} nu_j for merged
// control volumes (one block per (control volume, chunk of velocities)).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_fuseT(AdjArgs a, T *lam_out, T *mucv)
{
    __shared__ long pcs[kMaxMembers];
    __shared__ T ratio[kMaxMembers];
    const CvInfo &I = reinterpret_cast<const CvInfo *>(a.cvinfo)[blockIdx.x];
    constexpr int W = Vec<T>::W;
    const int nm = I.nm;
    if (nm <= 1 && !mucv) return;
    if (threadIdx.x < nm) {
        pcs[threadIdx.x] = I.mem[threadIdx.x].pc * W;
        ratio[threadIdx.x] = (T)(I.mem[threadIdx.x].sb / I.Sn);
    }
    __syncthreads();
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= 2 * a.g.nvp) return;
    const int comp = e / a.g.nvp, p = e - comp * a.g.nvp;
    const long base = ebase<T>(a.g, comp, p);
    T s = 0;
    for (int t = 0; t < nm; ++t) s += lam_out[base + pcs[t]];
    if (nm > 1)
        for (int t = 0; t < nm; ++t) lam_out[base + pcs[t]] = ratio[t] * s;
    if (mucv) {
        // the member sums of the next transposed step, summed as k_adj_mu
        // sums them (the members' values in member order)
        T m = 0;
        for (int t = 0; t < nm; ++t) m += nm > 1 ? ratio[t] * s : lam_out[base + pcs[t]];
        mucv[((long)blockIdx.x * 2 + comp) * a.g.nvp + p] = m;
    }
}

// The two pad layers of one side: their sensitivities (the flux transposes
// along the side's axis that read them) go to the cells they copy -- the
// boundary cell for a zero-gradient side, the periodic images -- or, for a
// Maxwellian side, are summed over the steps per (side cell, component,
// velocity) into pacc (the ghost state is the same at every step; the chain
// to (rho, u, T) is k_adj_ghost_chain).  One thread per (side cell,
// velocity group); the sides are launched one after the other (a corner
// cell receives from two sides).  Side cells whose boundary cell is a fast
// cell of a zero-gradient or Maxwellian side are left to k_adj_pads_fast.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_pads(AdjArgs a, const T *f, const T *lam, const T *mucv, int side,
                                                  int nside, const uint8_t *fast, int padsides, double *pacc,
                                                  T *lam_out)
{
    constexpr int W = Vec<T>::W;
    const Grid2D &g = a.g;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nside * g.ngrp) return;
    const int q = (int)(t % nside), p = (int)(t / nside) * W;
    const int axis = side < 2 ? 0 : 1;
    const int kind = g.bc[side];
    const int n = axis == 0 ? g.nx : g.ny;
    // the boundary cell of a zero-gradient or Maxwellian side took them if it
    // is a fast cell
    if ((padsides >> side) & 1) {
        const int tb = (side & 1) ? n - 1 : 0;
        if (fast[axis == 0 ? (long)q * g.nx + tb : (long)tb * g.nx + q]) return;
    }
    // positions of the inner (1) and outer (2) pad along the axis, and the
    // cells they copy
    const int c1 = (side & 1) ? n : -1, c2 = (side & 1) ? n + 1 : -2;
    const int i1 = axis == 0 ? c1 : q, j1 = axis == 0 ? q : c1;
    const int i2 = axis == 0 ? c2 : q, j2 = axis == 0 ? q : c2;
    T v[W], nu[W];
#pragma unroll
    for (int e = 0; e < W; ++e) {
        const VCoef<T> vc = ld_coef(reinterpret_cast<const VCoef<T> *>(a.vt) + p + e);
        v[e] = axis == 0 ? vc.vx : vc.vy;
        nu[e] = axis == 0 ? vc.nux : vc.nuy;
    }
    int t1, t2;
    if (kind == DVM_BC_PERIODIC) {
        t1 = (side & 1) ? 0 : n - 1;
        t2 = n > 1 ? ((side & 1) ? 1 : n - 2) : t1;
    } else {
        t1 = t2 = (side & 1) ? n - 1 : 0;
    }
    const long k1 = axis == 0 ? (long)q * g.nx + t1 : (long)t1 * g.nx + q;
    const long k2 = axis == 0 ? (long)q * g.nx + t2 : (long)t2 * g.nx + q;
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {
        const int comp = u >> 1, layer = u & 1;
        T e[W];
#pragma unroll
        for (int x = 0; x < W; ++x) e[x] = T(0);
        gather_axis<T>(a, f, lam, mucv, axis, layer ? i2 : i1, layer ? j2 : j1, comp, p, v, nu, e);
#pragma unroll
        for (int x = 0; x < W; ++x) {
            if (p + x >= g.nv) continue;
            if (kind == DVM_BC_MAXWELLIAN) pacc[((long)q * 2 + comp) * g.nv + p + x] += (double)e[x];
            else lam_out[ebase<T>(g, comp, p + x) + pcell(g, layer ? k2 : k1) * W] += e[x];
        }
    }
}

// Chain of the summed ghost sensitivities of a Maxwellian side to (rho, ux,
// uy, T) of each side cell (ghost f = M[rho, u, T], g = T/2 M in both
// layers); one block per side cell.
__global__ void __launch_bounds__(256) k_adj_ghost_chain(Grid2D g, int nside, const double *prim, const double *pacc,
                                                         double *gbc)
{
    __shared__ double red[8 * 4];
    for (int q = blockIdx.x; q < nside; q += gridDim.x) {
        const double *st = prim + 5L * q;
        double o0 = 0, o1 = 0, o2 = 0, o3 = 0;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const double s0 = pacc[((long)q * 2) * g.nv + p], s1 = pacc[((long)q * 2 + 1) * g.nv + p];
            const double vx = g.vxmin + (p % g.nvx) * g.dvx, vy = g.vymin + (p / g.nvx) * g.dvy;
            const double ax = vx - st[1], ay = vy - st[2], a2 = ax * ax + ay * ay;
            const double M = st[0] / (2.0 * kPi * st[4]) * exp(-a2 / (2.0 * st[4]));
            const double d0 = M / st[0], d1 = M * ax / st[4], d2 = M * ay / st[4];
            const double d3 = M * (a2 / (2.0 * st[4] * st[4]) - 1.0 / st[4]);
            const double h = st[4] / 2.0;
            o0 += s0 * d0 + s1 * h * d0;
            o1 += s0 * d1 + s1 * h * d1;
            o2 += s0 * d2 + s1 * h * d2;
            o3 += s0 * d3 + s1 * (M / 2.0 + h * d3);
        }
        o0 = block_sum(o0, red); o1 = block_sum(o1, red + 8); o2 = block_sum(o2, red + 16); o3 = block_sum(o3, red + 24);
        if (threadIdx.x == 0) {
            double *o = gbc + 5L * q;
            o[0] = o0; o[1] = o1; o[2] = o2; o[3] = 0; o[4] = o3;
        }
        __syncthreads();
    }
}

// dJ/d(rho, ux, uy, uz, T) of a Maxwellian initial state from lambda^0 (one
// thread per cell, 32 consecutive cells along x per warp).  With u = lambda_f
// + T/2 lambda_g: dJ/drho = sum u M / rho, dJ/du = sum u M (v - u) / T, dJ/dT =
// sum u M (|v - u|^2 / (2T) - 1) / T + sum lambda_g M / 2; the Maxwellian and
// the compensated sums in the state precision, the final factors in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_init(Grid2D g, const T *lam, const double *prim, const int8_t *type,
                                                  double *gout)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const long k = (long)j * g.nx + i;
    const double *st = prim + 5 * k;
    double o0 = 0, o1 = 0, o2 = 0, o3 = 0;
    if (type[k] != DVM_SOLID && st[0] > 0) {
        constexpr int W = Vec<T>::W;
        const long pk = nbr(g, i, j) * W;
        const T ux = (T)st[1], uy = (T)st[2], tmp = (T)st[4];
        const T A = (T)(st[0] / (2.0 * kPi * st[4])), i2T = (T)(0.5 / st[4]), c2 = (T)(kLog2e * 0.5 / st[4]);
        const T h = tmp / T(2);
        Acc<T> a0, a1, a2, a3, a4;
        for (int p0 = 0; p0 < g.nvp; p0 += W) {
            T l0[W], l1[W];
            vld<T>(reinterpret_cast<const typename Vec<T>::type *>(lam + ebase<T>(g, 0, p0) + pk), l0);
            vld<T>(reinterpret_cast<const typename Vec<T>::type *>(lam + ebase<T>(g, 1, p0) + pk), l1);
            T t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0;
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const int p = p0 + e;
                if (p >= g.nv) break;
                const T ax = (T)(g.vxmin + (p % g.nvx) * g.dvx) - ux, ay = (T)(g.vymin + (p / g.nvx) * g.dvy) - uy;
                const T q2 = ax * ax + ay * ay;
                const T M = A * dexp2(-q2 * c2);
                const T mu = M * (l0[e] + h * l1[e]);
                t0 += mu; t1 += mu * ax; t2 += mu * ay; t3 += mu * (q2 * i2T - T(1)); t4 += l1[e] * M;
            }
            a0.add(t0); a1.add(t1); a2.add(t2); a3.add(t3); a4.add(t4);
        }
        o0 = (double)a0.value() / st[0];
        o1 = (double)a1.value() / st[4];
        o2 = (double)a2.value() / st[4];
        o3 = (double)a3.value() / st[4] + 0.5 * (double)a4.value();
    }
    double *o = gout + 5 * k;
    o[0] = o0; o[1] = o1; o[2] = o2; o[3] = 0; o[4] = o3;
}

inline unsigned nba(long n, int b) { return (unsigned)((n + b - 1) / b); }

// Adjoint workspace of a context (allocated on first use).
struct AdjWork {
    size_t bytes_state = 0;
    void *lam[2] = {nullptr, nullptr};
    void *mucv = nullptr, *aux = nullptr, *bown = nullptr;
    int32_t *cvx = nullptr, *rev = nullptr;
    double *gtw = nullptr, *jwall = nullptr, *gbc = nullptr, *ginit = nullptr;
    int32_t *wsec = nullptr;
    uint8_t *fast = nullptr;                         // cells of the fast gather
    int32_t *slow = nullptr, *nslow_d = nullptr;     // the other cells
    int nslow = 0;
    int padneed[4] = {0, 0, 0, 0};                   // side cells left to the generic pad kernel
    int ncv = 0;                                     // cut and merged control volumes
    cudaStream_t side = nullptr;                     // second stream of a transposed step
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_pw0 = nullptr, ev_pw = nullptr;
    bool mu_ready = false;                           // mucv holds the member sums of the next lambda^{n+1}
    cudaStream_t rstream = nullptr;                  // recomputation, one segment ahead of the reverse sweep
    cudaEvent_t ev_rec[2] = {nullptr, nullptr};      // recomputation into tape set s done
    cudaEvent_t ev_used[2] = {nullptr, nullptr};     // transposed steps reading tape set s done
    void *frec = nullptr;                            // FaceRec per (listed cell, axis, face)
    void *rpart = nullptr;                           // [Z][5][nc] split sums of the relaxation transpose
    int Z = 1, Zf = 1;                               // velocity splits of the relaxation and the fast gather
    std::vector<uint32_t *> tbits, sbits;            // limiter branches per tape slot / per segment end
    std::vector<CUtensorMap> tbmap, sbmap;           // their TMA descriptors
    CUtensorMap lmap[2];                             // TMA descriptors of lam[0], lam[1]
    int nw = 0, nw_cap = 0;                          // wall cells and the capacity of the wall tables
    WallAdj *wadj = nullptr;                         // per wall cell: wall data
    WallVel *wm = nullptr;                           // per wall cell and velocity: c, M1, dM1/dT_w
    void *wt = nullptr;                              // the same in the state precision
    double2 *wd = nullptr;                           // per wall cell: (D, dD/dT_w)
    double *pacc = nullptr;                          // [side][cell][comp][nv] Maxwellian pad sensitivities
    void *fin = nullptr, *finpart = nullptr;         // F^N and its partial moments
    void *scratch_part = nullptr;                    // partial moments written by a tape fusion
    std::vector<void *> ckpt, ckpt_part, tape, ptape;
    std::vector<CUtensorMap> tmaps;                  // TMA descriptors of the tape buffers
    std::vector<CUtensorMap> cmaps;                  // TMA descriptors of the checkpoints
    // kept segments (written by the forward run, never recomputed): slots
    // 1..K-1 of each, their partial moments and descriptors, and the branch
    // words of steps 0..K-2
    std::vector<void *> ktape, kptape;
    std::vector<CUtensorMap> kmaps;
    std::vector<uint32_t *> kbits;
    std::vector<CUtensorMap> kbmaps;
    int cap = 0;
};

void release(AdjWork &w)
{
    for (int b = 0; b < 2; ++b) cudaFree(w.lam[b]);
    cudaFree(w.mucv); cudaFree(w.aux); cudaFree(w.bown); cudaFree(w.cvx); cudaFree(w.rev);
    cudaFree(w.gtw); cudaFree(w.jwall); cudaFree(w.gbc); cudaFree(w.ginit); cudaFree(w.wsec);
    cudaFree(w.fin); cudaFree(w.finpart); cudaFree(w.scratch_part);
    cudaFree(w.fast); cudaFree(w.slow); cudaFree(w.nslow_d); cudaFree(w.rpart);
    cudaFree(w.wadj); cudaFree(w.wm); cudaFree(w.wt); cudaFree(w.wd); cudaFree(w.pacc); cudaFree(w.frec);
    if (w.ev_fork) cudaEventDestroy(w.ev_fork);
    if (w.ev_join) cudaEventDestroy(w.ev_join);
    if (w.ev_pw0) cudaEventDestroy(w.ev_pw0);
    if (w.ev_pw) cudaEventDestroy(w.ev_pw);
    if (w.side) cudaStreamDestroy(w.side);
    for (int q = 0; q < 2; ++q) {
        if (w.ev_rec[q]) cudaEventDestroy(w.ev_rec[q]);
        if (w.ev_used[q]) cudaEventDestroy(w.ev_used[q]);
    }
    if (w.rstream) cudaStreamDestroy(w.rstream);
    for (uint32_t *p : w.tbits) cudaFree(p);
    for (uint32_t *p : w.sbits) cudaFree(p);
    for (void *p : w.ckpt) cudaFree(p);
    for (void *p : w.ckpt_part) cudaFree(p);
    for (void *p : w.tape) cudaFree(p);
    for (void *p : w.ptape) cudaFree(p);
    for (void *p : w.ktape) cudaFree(p);
    for (void *p : w.kptape) cudaFree(p);
    for (uint32_t *p : w.kbits) cudaFree(p);
    w = AdjWork();
}

// Copy of the padding frame (two cells on every side: boundary ghosts and
// mirrors) of every (group, component) slab of src into dst; a buffer that
// the step writes takes the pads it does not write from the state.
template <typename T>
__global__ void k_adj_copy_pads(Grid2D g, const T *src, T *dst)
{
    using V = typename Vec<T>::type;
    const int nxp = g.nx + 4;
    const int nframe = 4 * nxp + 4 * g.ny;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nframe * 2 * g.ngrp) return;
    const int q = (int)(t / nframe), f = (int)(t - (long)q * nframe);
    int i, j;
    if (f < 4 * nxp) {
        const int r = f / nxp;
        i = f - r * nxp;
        j = r < 2 ? r : g.ny + r;          // padded rows 0, 1, ny + 2, ny + 3
    } else {
        const int u = f - 4 * nxp, cidx = u / g.ny;
        j = 2 + (u - cidx * g.ny);
        i = cidx < 2 ? cidx : g.nx + cidx; // padded columns 0, 1, nx + 2, nx + 3
    }
    const long o = (long)q * g.slab + (long)j * nxp + i;
    reinterpret_cast<V *>(dst)[o] = reinterpret_cast<const V *>(src)[o];
}

AdjArgs adj_args(dvm_ctx *c, const AdjWork &w)
{
    AdjArgs a;
    a.g = grid2d(c);
    a.G = c->geo[c->gcur];
    a.b = body_params(c);
    a.master = c->master; a.flags = c->flags;
    a.spec_list = c->spec_list; a.wall_list = c->wall_list; a.counts = c->counts;
    a.cap = c->list_cap; a.cvinfo = c->cvinfo; a.vt = c->vtab;
    a.cvx = w.cvx; a.bown = w.bown;
    a.muscl = c->scheme == DVM_MUSCL;
    a.omega = c->body.omega;
    a.err = c->d_err;
    return a;
}

// One reverse step: lam_in = lambda^{n+1}, f = F^n (device layout), bits =
// the limiter branches the step took (MUSCL) -> lam_out.
// Sides whose pads k_adj_pads_fast takes from fast boundary cells:
// zero-gradient sides and Maxwellian sides with a parameter state.
inline int pad_sides(const dvm_ctx *c)
{
    int m = 0;
    for (int s = 0; s < 4; ++s)
        if (c->bc[s] == DVM_BC_ZEROGRAD || (c->bc[s] == DVM_BC_MAXWELLIAN && c->d_bcstate[s])) m |= 1 << s;
    return m;
}

template <typename T, bool MUSCL>
cudaError_t launch_gather_fast(dvm_ctx *c, const AdjArgs &a, const AdjWork &w, const CUtensorMap &lmap,
                               const CUtensorMap *bmap, T *lam_out)
{
    const size_t smem = (size_t)kAdjStages * kAdjStageBytes + 2 * kAdjStages * sizeof(uint64_t);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_gather_fast<T, MUSCL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid(nba(c->nx, 32), nba(c->ny, kRows), w.Zf), block(32, kRows);
    k_adj_gather_fast<T, MUSCL><<<grid, block, smem, c->stream>>>(a, lmap, bmap ? *bmap : lmap, c->gsign,
                                                                   (const T *)w.aux, w.fast, lam_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_step(dvm_ctx *c, AdjWork &w, const T *f, const T *part, const uint32_t *bits,
                         const CUtensorMap *bmap, int lin, T *lam_out)
{
    const T *lam_in = (const T *)w.lam[lin];
    const AdjArgs a = adj_args(c, w);
    T *mucv = (T *)w.mucv, *aux = (T *)w.aux;
    cudaError_t e;
    if (bits) {
        // the pad words feed only the fast gather and the pads: on the side
        // stream, beside the relaxation transpose
        if ((e = cudaEventRecord(w.ev_pw0, c->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(w.side, w.ev_pw0, 0)) != cudaSuccess) return e;
        const int nmax = c->nx > c->ny ? c->nx : c->ny;
        k_adj_padwords<T><<<nba(4L * nmax * c->ngrp, 256), 256, 0, w.side>>>(
            a.g, f, c->flags, c->gsign, (const VCoef<T> *)c->vtab, const_cast<uint32_t *>(bits), bits_slab(c),
            bits_pitch(c));
        if ((e = cudaEventRecord(w.ev_pw, w.side)) != cudaSuccess) return e;
    }
    const dim3 cvg((unsigned)(w.ncv > 0 ? w.ncv : 1), nba(2L * c->nvp, 256));
    // the member sums of lambda^{n+1}, unless the previous transposed step's
    // fusion transpose wrote them
    if (w.ncv > 0 && !w.mu_ready) k_adj_mu<T><<<cvg, 256, 0, c->stream>>>(a, lam_in, mucv);
    w.mu_ready = false;
    const dim3 cgrid(nba(c->nx, 32), nba(c->ny, 8)), cblock(32, 8);
    k_adj_relax<T><<<dim3(cgrid.x, cgrid.y, w.Z), cblock, 0, c->stream>>>(a, f, part, c->S, lam_in, mucv,
                                                                          (T *)w.rpart);
    k_adj_relax_fin<T><<<nba(c->nc, 256), 256, 0, c->stream>>>(a, part, c->S, (const T *)w.rpart, w.Z, aux);
    // the listed cells (record gather, then the wall terms of the wall cells
    // among them) on the side stream, concurrently with the fast cells and
    // their pads: the two write disjoint cells
    e = cudaEventRecord(w.ev_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(w.side, w.ev_fork, 0);
    if (e != cudaSuccess) return e;
    if (w.nslow > 0)
        k_adj_gather_rec<T><<<nba((long)w.nslow * c->ngrp, kRecItems), 4 * kRecItems, 0, w.side>>>(
            a, f, lam_in, mucv, aux, w.slow, w.nslow, (const FaceRec<T> *)w.frec, lam_out);
    if (w.nw > 0)
        k_adj_wall_step<T><<<w.nw, 256, 0, w.side>>>(a, w.nw, w.wadj, (const WallVelT<T> *)w.wt, w.wd, f, lam_in,
                                                      mucv, lam_out, w.gtw);
    if ((e = cudaEventRecord(w.ev_join, w.side)) != cudaSuccess) return e;
    if (bits && (e = cudaStreamWaitEvent(c->stream, w.ev_pw, 0)) != cudaSuccess) return e;
    e = c->scheme == DVM_MUSCL ? launch_gather_fast<T, true>(c, a, w, w.lmap[lin], bmap, lam_out)
                               : launch_gather_fast<T, false>(c, a, w, w.lmap[lin], nullptr, lam_out);
    if (e != cudaSuccess) return e;
    int launched = 7;
    const int nside[4] = {c->ny, c->ny, c->nx, c->nx};
    const int nmax = c->nx > c->ny ? c->nx : c->ny;
    const int ps = pad_sides(c);
    if (c->nx > 1 && c->ny > 1 && ps) {
        // the four sides in one launch
        const unsigned nb = nba(2L * (c->nx + c->ny) * c->ngrp, 256);
        if (c->scheme == DVM_MUSCL)
            k_adj_pads_fast4<T, true><<<nb, 256, 0, c->stream>>>(a, lam_in, bits, bits_slab(c), bits_pitch(c), ps,
                                                                 w.fast, w.pacc, nmax, lam_out);
        else
            k_adj_pads_fast4<T, false><<<nb, 256, 0, c->stream>>>(a, lam_in, nullptr, 0, 0, ps, w.fast, w.pacc, nmax,
                                                                  lam_out);
        ++launched;
    }
    for (int ax = 0; ax < 2 && !(c->nx > 1 && c->ny > 1); ++ax) {
        // both sides of the axis in one launch when they touch distinct cells
        const int n = ax == 0 ? c->nx : c->ny;
        for (int s = 2 * ax; s < 2 * ax + 2; s += n > 1 ? 2 : 1) {
            const int sides = n > 1 ? 2 : 1;
            if (!((ps >> s) & (sides == 2 ? 3 : 1))) continue;
            const unsigned nb = nba((long)nside[s] * c->ngrp * sides, 256);
            if (c->scheme == DVM_MUSCL)
                k_adj_pads_fast<T, true><<<nb, 256, 0, c->stream>>>(a, lam_in, bits, bits_slab(c), bits_pitch(c), s,
                                                                    sides, nside[s], ps, w.fast, w.pacc, nmax,
                                                                    lam_out);
            else
                k_adj_pads_fast<T, false><<<nb, 256, 0, c->stream>>>(a, lam_in, nullptr, 0, 0, s, sides, nside[s], ps,
                                                                     w.fast, w.pacc, nmax, lam_out);
            ++launched;
        }
    }
    if ((e = cudaStreamWaitEvent(c->stream, w.ev_join, 0)) != cudaSuccess) return e;
    for (int s = 0; s < 4; ++s) {
        if (c->bc[s] == DVM_BC_MAXWELLIAN && !c->d_bcstate[s]) continue;
        if (w.padneed[s] == 0) continue;
        k_adj_pads<T><<<nba((long)nside[s] * c->ngrp, 256), 256, 0, c->stream>>>(
            a, f, lam_in, mucv, s, nside[s], w.fast, ps, w.pacc + (long)s * nmax * 2 * c->nv, lam_out);
        ++launched;
    }
    if (w.ncv > 0) {
        k_adj_fuseT<T><<<cvg, 256, 0, c->stream>>>(a, lam_out, mucv);
        w.mu_ready = true;
    }
    c->launches += launched;
    return cudaGetLastError();
}

// Adds a state in the public layout [cell][comp][p] (a linear objective's
// dJ/dF^N) to lambda in the padded device layout (interior cells only; the
// pads stay 0).
template <typename T>
__global__ void k_adj_seed(Grid2D g, const T *pub, T *lam)
{
    const long k = blockIdx.x;            // one block per cell, threads over (comp, p)
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= 2 * g.nv) return;
    const int comp = e >= g.nv, p = e - comp * g.nv;
    const long d = ebase<T>(g, comp, p) + pcell(g, k) * Vec<T>::W;
    lam[d] += pub[k * 2L * g.nv + e];
}

// The adjoint sweep for J = [with_drag] F_x(F^N) + <seed, F^N>: the drag
// objective seeds lambda^N through the wall stress and the fusion transpose,
// a linear functional adds its dJ/dF^N = seed (public layout, host or
// device); lambda^0 = dJ/dF^0 can be returned in the public layout.
template <typename T>
int drag_adjoint_t(dvm_ctx *c, int nsteps, int K, double *J, double *gTw, double *const *gbc, double *gprim0,
                   double *ms_forward, double *ms_reverse, int with_drag, const void *seed, int seed_dev,
                   void *lam0, int lam0_dev)
{
    if (!c->adj) c->adj = new AdjWork();
    AdjWork &w = *static_cast<AdjWork *>(c->adj);
    const size_t bytes = c->dev_elems * c->elem;
    const size_t partb = (size_t)c->S * 4 * c->nc * c->elem;
    const int nmax = c->nx > c->ny ? c->nx : c->ny;
    const int nseg = (nsteps + K - 1) / K;
    const auto seglen = [&](int sgi) {
        const int n0 = sgi * K, n1 = (n0 + K < nsteps) ? n0 + K : nsteps;
        return n1 - n0;
    };
    cudaError_t e = cudaSuccess;
#define AC(call) do { e = (call); if (e != cudaSuccess) return cuda_fail(e, #call); } while (0)
    if (w.bytes_state != bytes || w.cap != c->list_cap) {
        release(w);
        for (int b = 0; b < 2; ++b) {
            AC(cudaMalloc(&w.lam[b], bytes));
            const int rc = encode_tensor_map2d(c, w.lam[b], &w.lmap[b]);
            if (rc != DVM_OK) return rc;
        }
        AC(cudaMalloc(&w.aux, (size_t)c->nc * 5 * c->elem));
        AC(cudaMalloc(&w.bown, (size_t)c->nc * c->elem));
        AC(cudaMalloc(&w.cvx, sizeof(int32_t) * c->nc));
        AC(cudaMalloc(&w.rev, sizeof(int32_t) * c->nc));
        AC(cudaMalloc(&w.gbc, sizeof(double) * 5 * 4 * nmax));
        AC(cudaMalloc(&w.ginit, sizeof(double) * 5 * c->nc));
        AC(cudaMalloc(&w.mucv, (size_t)c->list_cap * 2 * c->nvp * c->elem));
        AC(cudaMalloc(&w.gtw, sizeof(double) * c->list_cap));
        AC(cudaMalloc(&w.jwall, sizeof(double) * c->list_cap));
        AC(cudaMalloc(&w.wsec, sizeof(int32_t) * c->list_cap));
        AC(cudaMalloc(&w.fin, bytes));
        AC(cudaMalloc(&w.finpart, partb));
        AC(cudaMalloc(&w.scratch_part, partb));
        AC(cudaMalloc(&w.fast, c->nc));
        AC(cudaMalloc(&w.slow, sizeof(int32_t) * c->nc));
        AC(cudaMalloc(&w.frec, sizeof(FaceRec<T>) * 8 * c->nc));
        AC(cudaMalloc(&w.nslow_d, 5 * sizeof(int)));
        AC(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
        AC(cudaStreamCreateWithFlags(&w.rstream, cudaStreamNonBlocking));
        for (int q = 0; q < 2; ++q) {
            AC(cudaEventCreateWithFlags(&w.ev_rec[q], cudaEventDisableTiming));
            AC(cudaEventCreateWithFlags(&w.ev_used[q], cudaEventDisableTiming));
        }
        AC(cudaEventCreateWithFlags(&w.ev_fork, cudaEventDisableTiming));
        AC(cudaEventCreateWithFlags(&w.ev_join, cudaEventDisableTiming));
        AC(cudaEventCreateWithFlags(&w.ev_pw0, cudaEventDisableTiming));
        AC(cudaEventCreateWithFlags(&w.ev_pw, cudaEventDisableTiming));
        w.Z = c->ngrp < 8 ? c->ngrp : 8;
        w.Zf = c->ngrp < 4 ? c->ngrp : 4;
        AC(cudaMalloc(&w.pacc, sizeof(double) * 4 * nmax * 2 * c->nv));
        AC(cudaMalloc(&w.rpart, (size_t)w.Z * 5 * c->nc * c->elem));
        w.bytes_state = bytes;
        w.cap = c->list_cap;
    }
    while ((int)w.ckpt.size() < nseg) {
        void *p = nullptr, *q = nullptr;
        AC(cudaMalloc(&p, bytes));
        AC(cudaMalloc(&q, partb));
        w.ckpt.push_back(p);
        w.ckpt_part.push_back(q);
        CUtensorMap m;
        const int rc = encode_tensor_map2d(c, p, &m);
        if (rc != DVM_OK) return rc;
        w.cmaps.push_back(m);
    }
    const bool rec = c->scheme == DVM_MUSCL;
    const size_t bitsb = (size_t)c->ngrp * bits_slab(c) * sizeof(uint32_t);
    // kept segments: the last nkeep of the run, whose tapes the forward run
    // writes within the budget of dvm_set_adjoint_tape (and the device's free
    // memory less a margin); a failed allocation keeps fewer
    int nkeep = 0;
    if (K > 1 && c->adj_tape > 0) {
        const size_t kseg = (size_t)(K - 1) * (bytes + partb + (rec ? bitsb : 0));
        size_t fr = 0, tot = 0;
        AC(cudaMemGetInfo(&fr, &tot));
        const size_t have = (size_t)w.ktape.size() / (K - 1) * kseg;      // already held
        const size_t margin = (size_t)4 << 30;
        const size_t avail = fr + have > margin ? fr + have - margin : 0;
        const size_t budget = c->adj_tape < avail ? c->adj_tape : avail;
        nkeep = (int)(budget / kseg < (size_t)nseg ? budget / kseg : (size_t)nseg);
    }
    {
        const size_t nslots = (size_t)nkeep * (K - 1);
        while (w.ktape.size() > nslots) {          // fewer than before: free the rest
            cudaFree(w.ktape.back()); cudaFree(w.kptape.back());
            w.ktape.pop_back(); w.kptape.pop_back(); w.kmaps.pop_back();
            if (!w.kbits.empty()) { cudaFree(w.kbits.back()); w.kbits.pop_back(); w.kbmaps.pop_back(); }
        }
        while (w.ktape.size() < nslots) {
            void *p = nullptr, *q = nullptr;
            uint32_t *b = nullptr;
            if (cudaMalloc(&p, bytes) != cudaSuccess || cudaMalloc(&q, partb) != cudaSuccess ||
                (rec && cudaMalloc(&b, bitsb) != cudaSuccess)) {
                cudaGetLastError();
                cudaFree(p); cudaFree(q); cudaFree(b);
                break;
            }
            CUtensorMap m;
            int rc = encode_tensor_map2d(c, p, &m);
            if (rc != DVM_OK) { cudaFree(p); cudaFree(q); cudaFree(b); return rc; }
            w.ktape.push_back(p);
            w.kptape.push_back(q);
            w.kmaps.push_back(m);
            if (rec) {
                AC(cudaMemsetAsync(b, 0, bitsb, c->stream));
                CUtensorMap bm;
                rc = encode_bits_map2d(c, b, &bm);
                if (rc != DVM_OK) { cudaFree(b); return rc; }
                w.kbits.push_back(b);
                w.kbmaps.push_back(bm);
            }
        }
        nkeep = K > 1 ? (int)(w.ktape.size() / (K - 1)) : 0;
    }
    const int first_kept = nseg - nkeep;
    // segment sgi's tape is kept (its interior slots come from the forward run)
    const auto kept = [&](int sgi) { return sgi >= first_kept && seglen(sgi) > 1; };
    const auto kidx = [&](int sgi, int t) { return (size_t)(sgi - first_kept) * (K - 1) + (t - 1); };
    // a kept segment after a kept segment: the previous one's last step
    // writes its checkpoint (no copy of the live state)
    const auto direct = [&](int sgi) { return sgi >= 1 && kept(sgi - 1) && kept(sgi); };
    bool recompute_any = false;
    for (int sgi = 0; sgi < first_kept; ++sgi) recompute_any = recompute_any || seglen(sgi) > 1;
    // two tape sets: the recomputation of one segment fills one while the
    // reverse sweep reads the other
    while (recompute_any && (int)w.tape.size() < 2 * K) {
        void *p = nullptr, *q = nullptr;
        AC(cudaMalloc(&p, bytes));
        AC(cudaMalloc(&q, partb));
        w.tape.push_back(p);
        w.ptape.push_back(q);
        CUtensorMap m;
        const int rc = encode_tensor_map2d(c, p, &m);
        if (rc != DVM_OK) return rc;
        w.tmaps.push_back(m);
    }
    // limiter branches of the tape states (MUSCL): one buffer per tape slot but
    // the last, whose branches the checkpointed forward run records once per
    // segment; pad words that no cell writes stay 0
    for (int pass = 0; pass < 2 && rec; ++pass) {
        std::vector<uint32_t *> &v = pass ? w.sbits : w.tbits;
        std::vector<CUtensorMap> &mv = pass ? w.sbmap : w.tbmap;
        const int want = pass ? nseg : (recompute_any ? 2 * (K - 1) : 0);
        while ((int)v.size() < want) {
            uint32_t *p = nullptr;
            AC(cudaMalloc(&p, bitsb));
            AC(cudaMemsetAsync(p, 0, bitsb, c->stream));
            v.push_back(p);
            CUtensorMap m;
            const int rc = encode_bits_map2d(c, p, &m);
            if (rc != DVM_OK) return rc;
            mv.push_back(m);
        }
    }
    // the tape buffers take the boundary padding (Maxwellian ghosts) of the state
    if (recompute_any)
        for (int t = 0; t < K; ++t)
            AC(cudaMemcpyAsync(w.tape[t], c->f[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
    {
        const Grid2D g = grid2d(c);
        const long nf = (long)(4 * (c->nx + 4) + 4 * c->ny) * 2 * c->ngrp;
        for (size_t u = 0; u < w.ktape.size(); ++u)
            k_adj_copy_pads<T><<<nba(nf, 256), 256, 0, c->stream>>>(g, (const T *)c->f[c->cur], (T *)w.ktape[u]);
        for (int sgi = 1; sgi < nseg; ++sgi)
            if (direct(sgi))
                k_adj_copy_pads<T><<<nba(nf, 256), 256, 0, c->stream>>>(g, (const T *)c->f[c->cur], (T *)w.ckpt[sgi]);
        AC(cudaGetLastError());
    }
    AC(cudaMemsetAsync(w.gbc, 0, sizeof(double) * 5 * 4 * nmax, c->stream));
    AC(cudaMemsetAsync(w.gtw, 0, sizeof(double) * c->list_cap, c->stream));
    {
        const Grid2D g = grid2d(c);
        k_adj_rev<<<nba(c->list_cap, 256), 256, 0, c->stream>>>(c->spec_list, c->counts, c->list_cap, w.rev);
        k_adj_setup<T><<<nba(c->nc, 256), 256, 0, c->stream>>>(g, c->master, c->flags, w.rev, (const CvInfo *)c->cvinfo,
                                                                w.cvx, (T *)w.bown);
        k_adj_fastmask<<<nba(c->nc, 256), 256, 0, c->stream>>>(g, c->flags, w.fast);
        k_adj_slowlist<<<1, 1024, 0, c->stream>>>(c->nc, w.fast, c->master, w.slow, w.nslow_d);
        AC(cudaMemcpyAsync(&w.nslow, w.nslow_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        int32_t cnt0[2];
        AC(cudaMemcpyAsync(cnt0, c->counts, sizeof(cnt0), cudaMemcpyDeviceToHost, c->stream));
        AC(cudaMemsetAsync(w.nslow_d + 1, 0, 4 * sizeof(int), c->stream));
        k_adj_padcount<<<dim3(nba(nmax, 256), 4), 256, 0, c->stream>>>(g, w.fast, pad_sides(c), w.nslow_d + 1);
        AC(cudaMemcpyAsync(w.padneed, w.nslow_d + 1, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        AC(cudaStreamSynchronize(c->stream));
        w.nw = cnt0[1] < c->list_cap ? cnt0[1] : c->list_cap;
        w.ncv = cnt0[0] < c->list_cap ? cnt0[0] : c->list_cap;
        if (w.nw > w.nw_cap) {
            cudaFree(w.wadj); cudaFree(w.wm); cudaFree(w.wt); cudaFree(w.wd);
            w.wadj = nullptr; w.wm = nullptr; w.wt = nullptr; w.wd = nullptr; w.nw_cap = 0;
            AC(cudaMalloc(&w.wadj, sizeof(WallAdj) * w.nw));
            AC(cudaMalloc(&w.wm, sizeof(WallVel) * w.nw * c->nv));
            AC(cudaMalloc(&w.wt, sizeof(WallVelT<double>) * w.nw * c->nv));
            AC(cudaMalloc(&w.wd, sizeof(double2) * w.nw));
            w.nw_cap = w.nw;
        }
        if (w.nslow > 0)
            k_adj_listrec<T><<<nba((long)w.nslow * 8, 256), 256, 0, c->stream>>>(adj_args(c, w), w.slow, w.nslow,
                                                                              (FaceRec<T> *)w.frec);
        if (w.nw > 0)
            k_adj_wall_pre<T><<<w.nw, 256, 0, c->stream>>>(adj_args(c, w), w.nw, w.wadj, w.wm, (WallVelT<T> *)w.wt,
                                                            w.wd, w.wsec);
        AC(cudaMemsetAsync(w.pacc, 0, sizeof(double) * 4 * nmax * 2 * c->nv, c->stream));
    }
    cudaEvent_t ev[3];
    for (int q = 0; q < 3; ++q) AC(cudaEventCreate(&ev[q]));
    const bool fuse0 = c->need_fusion;
    const long long steps0 = c->steps_done;
    void *f_orig[2] = {c->f[0], c->f[1]}, *p_orig[2] = {c->part[0], c->part[1]};
    const CUtensorMap tm_orig[2] = {c->tmap[0], c->tmap[1]};
    AC(cudaEventRecord(ev[0], c->stream));
    // forward with checkpoints every K steps; a kept segment's steps write its
    // tape (step t of the segment reads slot t, slot 0 being the live state or
    // the checkpoint, and writes slot t + 1; its last step writes the next
    // segment's checkpoint when that segment is kept, else the other live
    // buffer) and record their limiter branches
    for (int n = 0; n < nsteps; ++n) {
        const int sgi = n / K, t = n % K, len = seglen(sgi);
        if (t == 0 && !direct(sgi)) {
            AC(cudaMemcpyAsync(w.ckpt[sgi], c->f[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
            AC(cudaMemcpyAsync(w.ckpt_part[sgi], c->part[c->cur], partb, cudaMemcpyDeviceToDevice, c->stream));
        }
        const bool last = t == len - 1;
        // the last step of each segment records its limiter branches
        if (rec && last) c->rec_bits = w.sbits[sgi];
        if (!kept(sgi)) {
            const cudaError_t es = step2d(c);
            c->rec_bits = nullptr;
            AC(es);
            continue;
        }
        const int L = c->cur;
        if (t > 0) {
            c->f[L] = w.ktape[kidx(sgi, t)];
            c->part[L] = w.kptape[kidx(sgi, t)];
            c->tmap[L] = w.kmaps[kidx(sgi, t)];
        } else if (direct(sgi)) {
            c->f[L] = w.ckpt[sgi];
            c->part[L] = w.ckpt_part[sgi];
            c->tmap[L] = w.cmaps[sgi];
        }
        if (!last) {
            c->f[1 - L] = w.ktape[kidx(sgi, t + 1)];
            c->part[1 - L] = w.kptape[kidx(sgi, t + 1)];
            c->tmap[1 - L] = w.kmaps[kidx(sgi, t + 1)];
            if (rec) c->rec_bits = w.kbits[kidx(sgi, t + 1)];
        } else if (sgi + 1 < nseg && direct(sgi + 1)) {
            c->f[1 - L] = w.ckpt[sgi + 1];
            c->part[1 - L] = w.ckpt_part[sgi + 1];
            c->tmap[1 - L] = w.cmaps[sgi + 1];
        }
        const cudaError_t es = step2d(c);
        c->rec_bits = nullptr;
        c->f[0] = f_orig[0]; c->f[1] = f_orig[1];
        c->part[0] = p_orig[0]; c->part[1] = p_orig[1];
        c->tmap[0] = tm_orig[0]; c->tmap[1] = tm_orig[1];
        if (!last) c->cur = L;      // the state is in the tape, the live buffers keep their parity
        AC(es);
    }
    AC(cudaEventRecord(ev[1], c->stream));
    AC(cudaMemcpyAsync(w.fin, c->f[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
    AC(cudaMemcpyAsync(w.finpart, c->part[c->cur], partb, cudaMemcpyDeviceToDevice, c->stream));
    dvm::BodyDev body_end;
    AC(cudaMemcpyAsync(&body_end, c->d_body, sizeof(body_end), cudaMemcpyDeviceToHost, c->stream));
    const AdjArgs a = adj_args(c, w);
    // objective on F^N: lambda^N = fusion^T dJ/dF
    int lin = 0;                                      // lambda^{n+1} is lam[lin]
    T *lamA = (T *)w.lam[0];
    // cells in no control volume and the pads keep lambda = 0 in both buffers
    AC(cudaMemsetAsync(w.lam[0], 0, bytes, c->stream));
    AC(cudaMemsetAsync(w.lam[1], 0, bytes, c->stream));
    AC(cudaMemsetAsync(w.jwall, 0, sizeof(double) * c->list_cap, c->stream));
    if (with_drag) {
        if (w.nw > 0)
            k_adj_wall_obj<T><<<w.nw, 256, 0, c->stream>>>(a, w.nw, w.wadj, w.wm, w.wd, (const T *)c->f[c->cur], lamA,
                                                            w.gtw, w.jwall);
        if (w.ncv > 0)
            k_adj_fuseT<T><<<dim3((unsigned)w.ncv, nba(2L * c->nvp, 256)), 256, 0, c->stream>>>(a, lamA,
                                                                                              (T *)nullptr);
    }
    // the public-layout staging buffer of the seed and of lambda^0
    if ((seed || lam0) && !c->d_pub) AC(cudaMalloc(&c->d_pub, c->state_elems * c->elem));
    if (seed) {
        // a linear functional of F^N as the step leaves it (members of a
        // merged control volume hold its value; no fusion transpose)
        AC(cudaMemcpyAsync(c->d_pub, seed, c->state_elems * c->elem,
                           seed_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
        k_adj_seed<T><<<dim3((unsigned)c->nc, nba(2L * c->nv, 256)), 256, 0, c->stream>>>(grid2d(c),
                                                                                         (const T *)c->d_pub, lamA);
    }
    // reverse sweep, segment by segment: recompute the segment onto the tape
    // (each step writes the next tape buffer) unless the forward run kept it,
    // then apply the transposed steps backwards
    const int cur_orig = c->cur;
    w.mu_ready = false;              // lambda^N took the objective and the seed after any fusion transpose
    cudaStream_t main_stream = c->stream;
    // tape slot 0 of segment sgi is its checkpoint; slot t > 0 is slot t of
    // the kept tape or of tape set sgi % 2; step t writes slot t + 1 (state
    // and partial moments)
    const auto fslot = [&](int sgi, int t) {
        return t == 0 ? w.ckpt[sgi] : (kept(sgi) ? w.ktape[kidx(sgi, t)] : w.tape[(sgi & 1) * K + t]);
    };
    const auto pslot = [&](int sgi, int t) {
        return t == 0 ? w.ckpt_part[sgi] : (kept(sgi) ? w.kptape[kidx(sgi, t)] : w.ptape[(sgi & 1) * K + t]);
    };
    const auto mslot = [&](int sgi, int t) { return t == 0 ? w.cmaps[sgi] : w.tmaps[(sgi & 1) * K + t]; };
    const auto bslot = [&](int sgi, int t) { return (sgi & 1) * (K - 1) + t; };
    bool used[2] = {false, false};
    // recomputation of segment sgi on the recomputation stream
    const auto recompute = [&](int sgi) -> cudaError_t {
        const int set = sgi & 1, len = seglen(sgi);
        cudaError_t er = cudaSuccess;
        if (used[set] && (er = cudaStreamWaitEvent(w.rstream, w.ev_used[set], 0)) != cudaSuccess) return er;
        c->stream = w.rstream;
        // the step linearises around the fused state (members of merged control
        // volumes are equal after every step, not necessarily in the initial state)
        if (sgi == 0 && fuse0) er = fusion2d(c, fslot(0, 0), pslot(0, 0));
        c->need_fusion = false;
        for (int t = 0; er == cudaSuccess && t + 1 < len; ++t) {
            c->f[c->cur] = fslot(sgi, t);
            c->f[1 - c->cur] = fslot(sgi, t + 1);
            c->part[c->cur] = pslot(sgi, t);
            c->part[1 - c->cur] = pslot(sgi, t + 1);
            c->tmap[c->cur] = mslot(sgi, t);
            c->tmap[1 - c->cur] = mslot(sgi, t + 1);
            if (rec) c->rec_bits = w.tbits[bslot(sgi, t)];
            er = step2d(c);
            c->rec_bits = nullptr;
            c->cur = 1 - c->cur;            // keep the same slot parity: step2d advanced it
        }
        c->f[0] = f_orig[0]; c->f[1] = f_orig[1];
        c->part[0] = p_orig[0]; c->part[1] = p_orig[1];
        c->tmap[0] = tm_orig[0]; c->tmap[1] = tm_orig[1];
        c->cur = cur_orig;
        c->stream = main_stream;
        if (er == cudaSuccess) er = cudaEventRecord(w.ev_rec[set], w.rstream);
        return er;
    };
    // the checkpoints are written by the forward run on the main stream
    AC(cudaStreamWaitEvent(w.rstream, ev[1], 0));
    // a kept first segment linearises around the fused initial state as well
    if (fuse0 && kept(0)) AC(fusion2d(c, fslot(0, 0), pslot(0, 0)));
    if (!kept(nseg - 1)) AC(recompute(nseg - 1));
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int set = sgi & 1, len = seglen(sgi);
        const bool kp = kept(sgi);
        if (sgi > 0 && !kept(sgi - 1)) AC(recompute(sgi - 1));   // the next segment, while this one is swept
        if (!kp) AC(cudaStreamWaitEvent(c->stream, w.ev_rec[set], 0));
        for (int t = len - 1; t >= 0; --t) {
            // the branches of step t: recorded by the forward run for the last
            // step and for every step of a kept segment (step t wrote slot t + 1)
            const CUtensorMap *bm = !rec ? nullptr
                                         : (t == len - 1 ? &w.sbmap[sgi]
                                                         : (kp ? &w.kbmaps[kidx(sgi, t + 1)] : &w.tbmap[bslot(sgi, t)]));
            const uint32_t *bits = !rec ? nullptr
                                        : (t == len - 1 ? w.sbits[sgi]
                                                        : (kp ? w.kbits[kidx(sgi, t + 1)] : w.tbits[bslot(sgi, t)]));
            AC(adjoint_step<T>(c, w, (const T *)fslot(sgi, t), (const T *)pslot(sgi, t), bits, bm, lin,
                               (T *)w.lam[1 - lin]));
            lin = 1 - lin;
        }
        if (!kp) {
            AC(cudaEventRecord(w.ev_used[set], c->stream));
            used[set] = true;
        }
    }
    AC(cudaEventRecord(ev[2], c->stream));
    // J and dJ/dT_w per sector: ordered sums over the wall list on the host
    int32_t cnt[2];
    std::vector<double> jw((size_t)c->list_cap), gt((size_t)c->list_cap);
    std::vector<int32_t> ws((size_t)c->list_cap);
    AC(cudaMemcpyAsync(cnt, c->counts, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    AC(cudaMemcpyAsync(jw.data(), w.jwall, sizeof(double) * c->list_cap, cudaMemcpyDeviceToHost, c->stream));
    AC(cudaMemcpyAsync(gt.data(), w.gtw, sizeof(double) * c->list_cap, cudaMemcpyDeviceToHost, c->stream));
    AC(cudaMemcpyAsync(ws.data(), w.wsec, sizeof(int32_t) * c->list_cap, cudaMemcpyDeviceToHost, c->stream));
    const int nside[4] = {c->ny, c->ny, c->nx, c->nx};
    for (int s = 0; s < 4; ++s)
        if (c->bc[s] == DVM_BC_MAXWELLIAN && c->d_bcstate[s])
            k_adj_ghost_chain<<<nside[s], 256, 0, c->stream>>>(grid2d(c), nside[s], c->d_bcstate[s],
                                                               w.pacc + (long)s * nmax * 2 * c->nv,
                                                               w.gbc + 5L * s * nmax);
    for (int s = 0; s < 4; ++s) {
        if (!gbc || !gbc[s]) continue;
        if (c->bc[s] != DVM_BC_MAXWELLIAN) { std::memset(gbc[s], 0, sizeof(double) * 5 * nside[s]); continue; }
        AC(cudaMemcpyAsync(gbc[s], w.gbc + 5L * s * nmax, sizeof(double) * 5 * nside[s], cudaMemcpyDeviceToHost, c->stream));
    }
    if (lam0) {
        // dJ/dF^0 in the public layout
        AC(unpack2d(c, w.lam[lin], c->d_pub));
        AC(cudaMemcpyAsync(lam0, c->d_pub, c->state_elems * c->elem,
                           lam0_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    }
    if (gprim0) {
        if (!c->have_prim0) { set_error("dvm_drag_adjoint: gprim0 needs a state set by dvm_init_maxwellian"); return DVM_ERR_STATE; }
        k_adj_init<T><<<dim3(nba(c->nx, 32), nba(c->ny, 8)), dim3(32, 8), 0, c->stream>>>(
            grid2d(c), (const T *)w.lam[lin], c->d_prim0, c->geo[c->gcur].type, w.ginit);
        AC(cudaMemcpyAsync(gprim0, w.ginit, sizeof(double) * 5 * c->nc, cudaMemcpyDeviceToHost, c->stream));
    }
    // leave the context at F^N, as after nsteps forward steps
    AC(cudaMemcpyAsync(c->f[c->cur], w.fin, bytes, cudaMemcpyDeviceToDevice, c->stream));
    AC(cudaMemcpyAsync(c->part[c->cur], w.finpart, partb, cudaMemcpyDeviceToDevice, c->stream));
    AC(cudaMemcpyAsync(c->d_body, &body_end, sizeof(body_end), cudaMemcpyHostToDevice, c->stream));
    AC(cudaStreamSynchronize(c->stream));
    c->need_fusion = false;
    c->steps_done = steps0 + nsteps;
    const int nw = cnt[1] < c->list_cap ? cnt[1] : c->list_cap;
    double s = 0;
    for (int q = 0; q < nw; ++q) s += jw[q];
    *J = s;
    const int ns = c->body.nseg > 0 ? c->body.nseg : 1;
    for (int q = 0; q < ns; ++q) gTw[q] = 0;
    for (int q = 0; q < nw; ++q) gTw[ws[q] < ns ? ws[q] : 0] += gt[q];
    float f1 = 0, f2 = 0;
    AC(cudaEventElapsedTime(&f1, ev[0], ev[1]));
    AC(cudaEventElapsedTime(&f2, ev[1], ev[2]));
    if (ms_forward) *ms_forward = f1;
    if (ms_reverse) *ms_reverse = f2;
    for (int q = 0; q < 3; ++q) cudaEventDestroy(ev[q]);
#undef AC
    return DVM_OK;
}

}  // namespace

int drag_adjoint2d(dvm_ctx *c, int nsteps, int K, double *J, double *gTw, double *const *gbc, double *gprim0,
                   double *ms_forward, double *ms_reverse, int with_drag, const void *seed, int seed_dev, void *lam0,
                   int lam0_dev)
{
    return c->prec == DVM_FP32 ? drag_adjoint_t<float>(c, nsteps, K, J, gTw, gbc, gprim0, ms_forward, ms_reverse,
                                                       with_drag, seed, seed_dev, lam0, lam0_dev)
                               : drag_adjoint_t<double>(c, nsteps, K, J, gTw, gbc, gprim0, ms_forward, ms_reverse,
                                                        with_drag, seed, seed_dev, lam0, lam0_dev);
}

// The kept tape buffers beyond what max_bytes allows go now (the adjoint
// call re-allocates what its budget needs).
void trim_adjoint_tape2d(dvm_ctx *c, size_t max_bytes)
{
    if (!c->adj) return;
    AdjWork &w = *static_cast<AdjWork *>(c->adj);
    if (w.ktape.empty()) return;
    const size_t per = w.bytes_state + (size_t)c->S * 4 * c->nc * c->elem +
                       (w.kbits.empty() ? 0 : (size_t)c->ngrp * bits_slab(c) * sizeof(uint32_t));
    while (!w.ktape.empty() && w.ktape.size() * per > max_bytes) {
        cudaFree(w.ktape.back()); cudaFree(w.kptape.back());
        w.ktape.pop_back(); w.kptape.pop_back(); w.kmaps.pop_back();
        if (!w.kbits.empty()) { cudaFree(w.kbits.back()); w.kbits.pop_back(); w.kbmaps.pop_back(); }
    }
}

void free_adjoint2d(dvm_ctx *c)
{
    if (!c->adj) return;
    AdjWork *w = static_cast<AdjWork *>(c->adj);
    release(*w);
    delete w;
    c->adj = nullptr;
}

}  // namespace dvm
