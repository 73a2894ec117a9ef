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
//   k_adj_mu      transpose of the distribution: mu = sum of lambda over the
//                 members of each cut/merged control volume;
//   k_adj_relax   per control volume: the relaxation through the moments
//                 (sums over the velocities of mu dM/d(rho, u, T));
//   k_adj_gather  per (cell, velocity): relaxation terms and the face-flux
//                 transposes of every face whose stencil reads the cell (the
//                 limiter derivative is the one of the branch the forward
//                 step takes), boundary pads folded back onto the cells they
//                 copy;
//   k_adj_wall    per wall cell: the diffuse flux and the wall density
//                 coupling (Eq. BoundaryDDv), and dJ/dT_w;
//   k_adj_fuseT   transpose of the fusion of merged control volumes;
//   k_adj_ghost   sensitivities of the Maxwellian ghost cells, chained to
//                 (rho, u, T) of each inflow cell.
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
};

struct Loc { int cell, side, q; };

// Source of the padded value at cell (i, j) within two cells of the grid: an
// interior cell, or a Maxwellian ghost (side, index along the side).
__device__ __forceinline__ Loc locate(const Grid2D &g, int i, int j)
{
    Loc L{-1, -1, -1};
    if (i < 0) {
        if (g.bc[0] == DVM_BC_PERIODIC) i += g.nx;
        else if (g.bc[0] == DVM_BC_MAXWELLIAN) { L.side = 0; L.q = j; return L; }
        else i = 0;
    } else if (i >= g.nx) {
        if (g.bc[1] == DVM_BC_PERIODIC) i -= g.nx;
        else if (g.bc[1] == DVM_BC_MAXWELLIAN) { L.side = 1; L.q = j; return L; }
        else i = g.nx - 1;
    }
    if (j < 0) {
        if (g.bc[2] == DVM_BC_PERIODIC) j += g.ny;
        else if (g.bc[2] == DVM_BC_MAXWELLIAN) { L.side = 2; L.q = i; return L; }
        else j = 0;
    } else if (j >= g.ny) {
        if (g.bc[3] == DVM_BC_PERIODIC) j -= g.ny;
        else if (g.bc[3] == DVM_BC_MAXWELLIAN) { L.side = 3; L.q = i; return L; }
        else j = g.ny - 1;
    }
    L.cell = j * g.nx + i;
    return L;
}

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
// mu of every cut or merged control volume: the sum of lambda over its members.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_mu(AdjArgs a, const T *lam, T *mucv)
{
    const CvInfo *info = reinterpret_cast<const CvInfo *>(a.cvinfo);
    const int n = min(a.counts[0], a.cap);
    constexpr int W = Vec<T>::W;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const CvInfo &I = info[idx];
        for (int e = threadIdx.x; e < 2 * a.g.nvp; e += blockDim.x) {
            const int comp = e / a.g.nvp, p = e - comp * a.g.nvp;
            const long base = ebase<T>(a.g, comp, p);
            T s = 0;
            for (int t = 0; t < I.nm; ++t) s += lam[base + I.mem[t].pc * W];
            mucv[((long)idx * 2 + comp) * a.g.nvp + p] = s;
        }
    }
}

// Relaxation through the moments, per control volume (one thread per master
// cell, 32 consecutive cells along x per warp, vector loads of each velocity
// group): with G = F - b R + r (Feq - F), r = dt rho / tau0, the moment
// sensitivities S = d/d(rho, rho u, E) of sum_p mu r Feq + mu (Feq - F)
// dt/tau0 drho.  aux[m] = (r, S0, S1, S2, S3).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_relax(AdjArgs a, const T *f, const T *part, int S, const T *lam,
                                                   const T *mucv, T *aux)
{
    const Grid2D &g = a.g;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int m = j * g.nx + i;
    if (a.master[m] != m) return;
    constexpr int W = Vec<T>::W;
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(a.vt);
    const long pc = nbr(g, i, j) * W;
    // moments of F^n: the partial sums the forward step read ([S][4][nc])
    const long nc = (long)g.nx * g.ny;
    Acc<T> s0, s1, s2, s3;
    for (int q = 0; q < S; ++q) {
        s0.merge(part[((long)q * 4 + 0) * nc + m], T(0));
        s1.merge(part[((long)q * 4 + 1) * nc + m], T(0));
        s2.merge(part[((long)q * 4 + 2) * nc + m], T(0));
        s3.merge(part[((long)q * 4 + 3) * nc + m], T(0));
    }
    const T dv = pick<T>(g.dv_f, g.dv);
    const T rho = s0.value() * dv, ux = s1.value() / s0.value(), uy = s2.value() / s0.value();
    const T E = s3.value() * dv;
    const T tmp = (T(2) * E / rho - (ux * ux + uy * uy)) / T(3);
    const T dtt = pick<T>(g.dt_tau0_f, g.dt_tau0);
    const T r = dtt * rho;
    const T A = rho / (T(2.0 * kPi) * tmp), i2T = T(1) / (T(2) * tmp);
    const int cx = a.cvx[m];
    Acc<T> q0, q1, q2, q3, qr;
    for (int p = 0; p < g.nvp; p += W) {
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
        T t0 = 0, t1 = 0, t2 = 0, t3 = 0, tr = 0;
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const VCoef<T> vc = ld_coef(vt + p + e);
            const T ax = vc.vx - ux, ay = vc.vy - uy, a2 = ax * ax + ay * ay;
            const T M = A * dexp(-a2 * i2T);
            // dM/d(rho, ux, uy, T) and d(T/2 M)/d(...)
            const T d0 = M / rho, d1 = M * ax / tmp, d2 = M * ay / tmp, d3 = M * (a2 * i2T / tmp - T(1) / tmp);
            const T h = tmp / T(2);
            t0 += mf[e] * d0 + mg[e] * h * d0;
            t1 += mf[e] * d1 + mg[e] * h * d1;
            t2 += mf[e] * d2 + mg[e] * h * d2;
            t3 += mf[e] * d3 + mg[e] * (M / T(2) + h * d3);
            tr += mf[e] * (M - fv[e]) + mg[e] * (h * M - gv[e]);
        }
        q0.add(r * t0); q1.add(r * t1); q2.add(r * t2); q3.add(r * t3); qr.add(tr * dtt);
    }
    const T sp0 = q0.value() + qr.value(), sp1 = q1.value(), sp2 = q2.value(), sp3 = q3.value();
    const T S0 = sp0 - sp1 * ux / rho - sp2 * uy / rho +
                 sp3 * (T(-2) * E / (rho * rho) + T(2) * (ux * ux + uy * uy) / rho) / T(3);
    const T S1 = sp1 / rho - sp3 * T(2) * ux / (T(3) * rho);
    const T S2 = sp2 / rho - sp3 * T(2) * uy / (T(3) * rho);
    const T S3 = sp3 * T(2) / (T(3) * rho);
    T *o = aux + 5 * (long)m;
    o[0] = r; o[1] = S0; o[2] = S1; o[3] = S2; o[4] = S3;
}

// Sum over the faces along one axis whose stencil reads position (ci, cj) of
// the weight W_f (adjoint of the two control volumes the face separates)
// times the flux derivative at that stencil slot.  The faces are those
// between columns ii and ii + 1 for ii = c - 2 .. c + 1 along the axis; a
// slot counts when its value comes from the target (cell or ghost).
template <typename T, bool ALIASFREE>
__device__ T gather_axis(const AdjArgs &a, const T *f, const T *lam, const T *mucv, int axis, int ti, int tj,
                         Loc target, int comp, int p, T v, T nu)
{
    const Grid2D &g = a.g;
    constexpr int W = Vec<T>::W;
    const int n = axis == 0 ? g.nx : g.ny;
    const bool per = g.bc[axis == 0 ? 0 : 2] == DVM_BC_PERIODIC;
    const int c = axis == 0 ? ti : tj;
    const long eb = ebase<T>(g, comp, p);
    const T *bown = reinterpret_cast<const T *>(a.bown);
    T acc = 0;
    for (int ii = c - 2; ii <= c + 1; ++ii) {
        int fi = ii;
        if (per) { if (fi < 0) fi += n; else if (fi >= n) fi -= n; }
        else if (fi < -1 || fi > n - 1) continue;       // not a face of any cell
        // the face between A (column fi) and B (column fi + 1) along the axis
        int ia = axis == 0 ? fi : ti, ja = axis == 0 ? tj : fi;
        int ib = axis == 0 ? fi + 1 : ti, jb = axis == 0 ? tj : fi + 1;
        if (ib >= g.nx) ib -= g.nx;                     // periodic wrap of B
        if (jb >= g.ny) jb -= g.ny;
        const bool aint = per || fi >= 0, bint = per || fi + 1 <= n - 1;
        const int A = aint ? ja * g.nx + ia : -1;
        const int B = bint ? jb * g.nx + ib : -1;
        // length and limiter flag as the forward step uses them
        T L;
        bool lim = false;
        if (A >= 0) {
            L = axis == 0 ? (T)a.G.lx[(long)ja * (g.nx + 1) + ia + 1] : (T)a.G.ly[(long)(ja + 1) * g.nx + ia];
            lim = a.muscl && ((a.flags[A] >> kMaskShift) & (axis == 0 ? 2 : 8));
        } else {
            L = axis == 0 ? (T)a.G.lx[(long)jb * (g.nx + 1) + ib] : (T)a.G.ly[(long)jb * g.nx + ib];
            lim = a.muscl && ((a.flags[B] >> kMaskShift) & (axis == 0 ? 1 : 4));
        }
        if (L == T(0)) continue;
        const T Wf = (A >= 0 ? -bown[A] * mu_of<T>(a, lam, mucv, A, comp, p) : T(0)) +
                     (B >= 0 ? bown[B] * mu_of<T>(a, lam, mucv, B, comp, p) : T(0));
        if (Wf == T(0)) continue;
        // stencil AA, A, B, BB in padded coordinates around the face
        T fv[4];
        int si[4], sj[4];
        for (int t = 0; t < 4; ++t) {
            si[t] = axis == 0 ? fi - 1 + t : ti;
            sj[t] = axis == 0 ? tj : fi - 1 + t;
            fv[t] = f[eb + nbr(g, si[t], sj[t]) * W];
        }
        T d[4];
        face_flux_d<T>(L, v, nu, fv[0], fv[1], fv[2], fv[3], lim, d);
        if (ALIASFREE) {
            // away from the sides only the slot at the cell's own position reads it
            acc += Wf * d[c - ii + 1];
        } else {
            for (int t = 0; t < 4; ++t) {
                if (d[t] == T(0)) continue;
                const Loc l = locate(g, si[t], sj[t]);
                if (l.cell == target.cell && l.side == target.side && l.q == target.q) acc += Wf * d[t];
            }
        }
    }
    return acc;
}

// nu of one (cell, velocity): relaxation terms for control-volume masters and
// the face-flux transposes (generic: any cell, any boundary).
template <typename T>
__device__ __forceinline__ void gather_generic(const AdjArgs &a, const T *f, const T *lam, const T *mucv, const T *aux,
                                               T *lam_out, int k, int p)
{
    const Grid2D &g = a.g;
    constexpr int W = Vec<T>::W;
    const long pk = pcell(g, k) * W;
    if (a.master[k] < 0 || p >= g.nv) {
        lam_out[ebase<T>(g, 0, p) + pk] = T(0);
        lam_out[ebase<T>(g, 1, p) + pk] = T(0);
        return;
    }
    const VCoef<T> vc = ld_coef(reinterpret_cast<const VCoef<T> *>(a.vt) + p);
    int ki, kj;
    cell_ij(g, k, ki, kj);
    const Loc me{k, -1, -1};
    const bool ismaster = a.master[k] == k;
    const T dv = pick<T>(g.dv_f, g.dv);
    for (int comp = 0; comp < 2; ++comp) {
        T nu = 0;
        if (ismaster) {
            const T *o = aux + 5 * (long)k;
            nu += mu_of<T>(a, lam, mucv, k, comp, p) * (T(1) - o[0]);
            nu += comp == 0 ? dv * (o[1] + o[2] * vc.vx + o[3] * vc.vy + o[4] * T(0.5) * (vc.vx * vc.vx + vc.vy * vc.vy))
                            : dv * o[4];
        }
        if (ki >= 2 && ki < g.nx - 2 && kj >= 2 && kj < g.ny - 2) {
            nu += gather_axis<T, true>(a, f, lam, mucv, 0, ki, kj, me, comp, p, vc.vx, vc.nux);
            nu += gather_axis<T, true>(a, f, lam, mucv, 1, ki, kj, me, comp, p, vc.vy, vc.nuy);
        } else {
            nu += gather_axis<T, false>(a, f, lam, mucv, 0, ki, kj, me, comp, p, vc.vx, vc.nux);
            nu += gather_axis<T, false>(a, f, lam, mucv, 1, ki, kj, me, comp, p, vc.vy, vc.nuy);
        }
        lam_out[ebase<T>(g, comp, p) + pk] = nu;
    }
}

// Generic gather over the listed cells (those near walls, merged control
// volumes or non-periodic sides), one thread per (listed cell, velocity).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_gather_list(AdjArgs a, const T *f, const T *lam, const T *mucv,
                                                         const T *aux, const int32_t *list, int nlist, T *lam_out)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nlist * a.g.nvp) return;
    gather_generic<T>(a, f, lam, mucv, aux, lam_out, list[t / a.g.nvp], (int)(t % a.g.nvp));
}

// Transpose of the face fluxes along one axis for a cell deep in the gas
// (all cells within three along the axis are plain gas cells and no
// non-periodic side is within reach): with W_f = b (mu_B - mu_A) L and the
// limited face value phi = F_up + k mm(...) the cell receives, for v > 0,
//   W(k+1/2) (1 + k (db - da))_{k+1/2} + W(k-1/2) k da_{k-1/2} - W(k+3/2) k db_{k+3/2}
// and the mirror image for v < 0 (da, db: the branch the forward minmod takes).
// f2m..f2p: F at offsets -2..+2, l2m..l2p: mu at offsets -2..+2; bl = b L v.
template <typename T, bool MUSCL>
__device__ __forceinline__ T adj_axis(T bl, T nu, T f2m, T f1m, T f0, T f1p, T f2p, T l2m, T l1m, T l0, T l1p, T l2p)
{
    if (bl == T(0)) return T(0);
    if (!MUSCL) return bl > T(0) ? bl * (l1p - l0) : bl * (l0 - l1m);
    const T k = T(0.5) * (T(1) - nu);
    T da, db, r;
    if (bl > T(0)) {
        minmod_d(f1p - f0, f0 - f1m, da, db);            // face k+1/2
        r = (l1p - l0) * (T(1) + k * (db - da));
        minmod_d(f0 - f1m, f1m - f2m, da, db);           // face k-1/2
        r += (l0 - l1m) * (k * da);
        minmod_d(f2p - f1p, f1p - f0, da, db);           // face k+3/2
        r -= (l2p - l1p) * (k * db);
    } else {
        minmod_d(f1p - f0, f0 - f1m, da, db);            // face k-1/2 (k is its B)
        r = (l0 - l1m) * (T(1) - k * (db - da));
        minmod_d(f2p - f1p, f1p - f0, da, db);           // face k+1/2 (k is its A)
        r += (l1p - l0) * (k * db);
        minmod_d(f0 - f1m, f1m - f2m, da, db);           // face k-3/2 (k is its BB)
        r -= (l1m - l2m) * (k * da);
    }
    return bl * r;
}

// Fast gather for the cells flagged in fast[] (one thread per cell, 32
// consecutive cells along x per warp, vector loads of each velocity group),
// relaxation terms included; other cells are left to k_adj_gather_list.
template <typename T, bool MUSCL>
__global__ void __launch_bounds__(256) k_adj_gather_fast(AdjArgs a, const T *f, const T *lam, const T *aux,
                                                         const uint8_t *fast, T *lam_out)
{
    const Grid2D &g = a.g;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int k = j * g.nx + i;
    if (!fast[k]) return;
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(a.vt);
    const long pc = nbr(g, i, j);
    const long sy = g.nx + 4;
    const T *o = aux + 5 * (long)k;
    const T r = o[0], S0 = o[1], S1 = o[2], S2 = o[3], S3 = o[4];
    const T dv = pick<T>(g.dv_f, g.dv);
    const T *bown = reinterpret_cast<const T *>(a.bown);
    const T b = bown[k];
    const T Lx = (T)g.dy, Ly = (T)g.dx;
    for (int p = 0; p < g.nvp; p += W) {
        T vx[W], vy[W], nux[W], nuy[W];
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const VCoef<T> vc = ld_coef(vt + p + e);
            vx[e] = vc.vx; vy[e] = vc.vy; nux[e] = vc.nux; nuy[e] = vc.nuy;
        }
        for (int comp = 0; comp < 2; ++comp) {
            const V *F = reinterpret_cast<const V *>(f + ebase<T>(g, comp, p));
            const V *Lm = reinterpret_cast<const V *>(lam + ebase<T>(g, comp, p));
            T c0[W], fx[4][W], fy[4][W], l0[W], lx[4][W], ly[4][W];
            vld<T>(F + pc, c0);
            vld<T>(Lm + pc, l0);
            const long offx[4] = {-2, -1, 1, 2};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                vld<T>(F + pc + offx[t], fx[t]);
                vld<T>(F + pc + offx[t] * sy, fy[t]);
                vld<T>(Lm + pc + offx[t], lx[t]);
                vld<T>(Lm + pc + offx[t] * sy, ly[t]);
            }
            T out[W];
#pragma unroll
            for (int e = 0; e < W; ++e) {
                T nu = l0[e] * (T(1) - r);
                nu += comp == 0 ? dv * (S0 + S1 * vx[e] + S2 * vy[e] + S3 * T(0.5) * (vx[e] * vx[e] + vy[e] * vy[e]))
                                : dv * S3;
                if (p + e < g.nv) {
                    nu += adj_axis<T, MUSCL>(b * Lx * vx[e], nux[e], fx[0][e], fx[1][e], c0[e], fx[2][e], fx[3][e],
                                             lx[0][e], lx[1][e], l0[e], lx[2][e], lx[3][e]);
                    nu += adj_axis<T, MUSCL>(b * Ly * vy[e], nuy[e], fy[0][e], fy[1][e], c0[e], fy[2][e], fy[3][e],
                                             ly[0][e], ly[1][e], l0[e], ly[2][e], ly[3][e]);
                } else {
                    nu = T(0);
                }
                out[e] = nu;
            }
            vst<T>(reinterpret_cast<V *>(lam_out + ebase<T>(g, comp, p)) + pc, out);
        }
    }
}

// Cells eligible for the fast gather: plain gas cells whose neighbours within
// three cells along each axis are plain gas cells, at least two cells from
// every side (no boundary pad then aliases the cell, and the faces it reads
// separate interior cells; the adjoint buffers carry no boundary padding).
__global__ void k_adj_fastmask(Grid2D g, const uint8_t *flags, uint8_t *fast)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long)g.nx * g.ny) return;
    int i, j;
    cell_ij(g, k, i, j);
    bool ok = (flags[k] & kPlain) != 0 && i >= 2 && i < g.nx - 2 && j >= 2 && j < g.ny - 2;
    for (int d = -3; d <= 3 && ok; ++d) {
        const int ii = i + d, jj = j + d;
        // neighbours beyond a side are boundary values: the face masks of the
        // forward step count them as gas
        ok = (ii < 0 || ii >= g.nx || (flags[(long)j * g.nx + ii] & kPlain)) &&
             (jj < 0 || jj >= g.ny || (flags[(long)jj * g.nx + i] & kPlain));
    }
    fast[k] = ok ? 1 : 0;
}

// Compact list of the cells not eligible for the fast gather (one block).
__global__ void __launch_bounds__(1024) k_adj_slowlist(long nc, const uint8_t *fast, int32_t *list, int *count)
{
    __shared__ int wsum[32];
    __shared__ int tot;
    int n = 0;
    for (long base = 0; base < nc; base += blockDim.x) {
        const long k = base + threadIdx.x;
        const bool slow = k < nc && !fast[k];
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

// Wall cells: the diffuse flux lw (min(c,0) phi Mw + max(c,0) F) of the update
// (objective = 0) or the force functional (objective = 1), through phi =
// -sum_{c>0} c f dv / D, D = sum_{c<0} c M1 dv, with dJ/dT_w per wall slot.
// One block per wall cell, FP64 reductions.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_wall(AdjArgs a, const T *f, const T *lam, const T *mucv, T *lam_out,
                                                  double *gtw, double *jwall, int32_t *wsec, int objective)
{
    __shared__ double red[8 * 8];
    const Grid2D &g = a.g;
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(a.vt);
    const T *bown = reinterpret_cast<const T *>(a.bown);
    const int nw = min(a.counts[1], a.cap);
    constexpr int W = Vec<T>::W;
    const double dv = g.dv;
    for (int idx = blockIdx.x; idx < nw; idx += gridDim.x) {
        const int k = a.wall_list[idx];
        const WallAdj w = wall_adj(a, k);
        const long pk = pcell(g, k) * W;
        const double cmw = 1.0 / (2.0 * kPi * w.Tw);
        const double bk = objective ? 0.0 : (double)bown[k];
        double num = 0, den = 0, sphi = 0, sTw = 0, dD = 0, sxx = 0, sxy = 0;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const VCoef<T> vc = ld_coef(vt + p);
            const double ax = (double)vc.vx - w.uwx, ay = (double)vc.vy - w.uwy;
            const double cp = ax * w.nwx + ay * w.nwy;
            if (cp > 0) {
                const double fv = (double)f[ebase<T>(g, 0, p) + pk];
                num += cp * fv * dv;
                sxx += ax * ax * fv * dv; sxy += ax * ay * fv * dv;
            } else if (cp < 0) {
                const double a2 = ax * ax + ay * ay;
                const double m1 = cmw * exp(-a2 / (2.0 * w.Tw));
                const double dm1 = m1 * (a2 / (2.0 * w.Tw * w.Tw) - 1.0 / w.Tw);
                den += cp * m1 * dv;
                dD += cp * dm1 * dv;
                if (objective) {
                    const double wgt = (ax * ax * w.nwx + ax * ay * w.nwy) * w.lw * dv;
                    sphi += wgt * m1;
                    sTw += wgt * dm1;          // times phi below
                } else {
                    const double w0 = -bk * (double)mu_of<T>(a, lam, mucv, k, 0, p);
                    const double w1 = -bk * (double)mu_of<T>(a, lam, mucv, k, 1, p);
                    sphi += w.lw * cp * (w0 * m1 + w1 * w.Tw / 2.0 * m1);
                    sTw += w.lw * cp * (w0 * dm1 + w1 * (m1 / 2.0 + w.Tw / 2.0 * dm1));   // times phi below
                }
            }
        }
        num = block_sum(num, red); den = block_sum(den, red + 8); sphi = block_sum(sphi, red + 16);
        sTw = block_sum(sTw, red + 24); dD = block_sum(dD, red + 32);
        sxx = block_sum(sxx, red + 40); sxy = block_sum(sxy, red + 48);
        const double phi = -num / den;
        // per-velocity terms of the wall cell
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const VCoef<T> vc = ld_coef(vt + p);
            const double ax = (double)vc.vx - w.uwx, ay = (double)vc.vy - w.uwy;
            const double cp = ax * w.nwx + ay * w.nwy;
            if (!(cp > 0)) continue;
            const long e0 = ebase<T>(g, 0, p) + pk, e1 = ebase<T>(g, 1, p) + pk;
            double add0 = sphi * (-cp * dv / den), add1 = 0;
            if (objective) {
                add0 += (ax * ax * w.nwx + ax * ay * w.nwy) * w.lw * dv;
            } else {
                add0 += -bk * (double)mu_of<T>(a, lam, mucv, k, 0, p) * w.lw * cp;
                add1 += -bk * (double)mu_of<T>(a, lam, mucv, k, 1, p) * w.lw * cp;
            }
            lam_out[e0] = (T)((double)lam_out[e0] + add0);
            if (add1 != 0) lam_out[e1] = (T)((double)lam_out[e1] + add1);
        }
        if (threadIdx.x == 0) {
            gtw[idx] += phi * sTw + sphi * (-phi / den) * dD;
            wsec[idx] = w.sector;
            if (objective) {
                // the incoming part of the stress: phi times the M1 sums
                const double sin_xx_xy = sphi;          // sum (ax^2 nwx + ax ay nwy) lw dv M1
                jwall[idx] = (sxx * w.nwx + sxy * w.nwy) * w.lw + phi * sin_xx_xy;
            }
        }
        __syncthreads();
    }
}

// Transpose of the fusion: lam_k = (sbar_k / S) sum_{j in CV} nu_j for merged
// control volumes.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_fuseT(AdjArgs a, T *lam_out)
{
    const CvInfo *info = reinterpret_cast<const CvInfo *>(a.cvinfo);
    const int n = min(a.counts[0], a.cap);
    constexpr int W = Vec<T>::W;
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        const CvInfo &I = info[idx];
        if (I.nm <= 1) continue;
        for (int e = threadIdx.x; e < 2 * a.g.nvp; e += blockDim.x) {
            const int comp = e / a.g.nvp, p = e - comp * a.g.nvp;
            const long base = ebase<T>(a.g, comp, p);
            T s = 0;
            for (int t = 0; t < I.nm; ++t) s += lam_out[base + I.mem[t].pc * W];
            for (int t = 0; t < I.nm; ++t) lam_out[base + I.mem[t].pc * W] = (T)(I.mem[t].sb / I.Sn) * s;
        }
    }
}

// Maxwellian ghost cells: sensitivity of the ghost value of side s, index q,
// then chained to (rho, ux, uy, T) of that side cell; one block per side cell.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_ghost(AdjArgs a, const T *f, const T *lam, const T *mucv, int side,
                                                   int nside, const double *prim, double *gbc)
{
    __shared__ double red[8 * 4];
    const Grid2D &g = a.g;
    const VCoef<T> *vt = reinterpret_cast<const VCoef<T> *>(a.vt);
    const int axis = side < 2 ? 0 : 1;
    for (int q = blockIdx.x; q < nside; q += gridDim.x) {
        // a cell adjacent to the ghost along the side's axis anchors the gather
        int ti, tj;
        if (side == 0) { ti = 0; tj = q; }
        else if (side == 1) { ti = g.nx - 1; tj = q; }
        else if (side == 2) { ti = q; tj = 0; }
        else { ti = q; tj = g.ny - 1; }
        const Loc target{-1, side, q};
        const double *st = prim + 5L * q;
        double o0 = 0, o1 = 0, o2 = 0, o3 = 0;
        for (int p = threadIdx.x; p < g.nv; p += blockDim.x) {
            const VCoef<T> vc = ld_coef(vt + p);
            const T v = axis == 0 ? vc.vx : vc.vy, nu = axis == 0 ? vc.nux : vc.nuy;
            const double s0 = (double)gather_axis<T, false>(a, f, lam, mucv, axis, ti, tj, target, 0, p, v, nu);
            const double s1 = (double)gather_axis<T, false>(a, f, lam, mucv, axis, ti, tj, target, 1, p, v, nu);
            const double ax = (double)vc.vx - st[1], ay = (double)vc.vy - st[2], a2 = ax * ax + ay * ay;
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
            o[0] += o0; o[1] += o1; o[2] += o2; o[4] += o3;
        }
        __syncthreads();
    }
}

// dJ/d(rho, ux, uy, uz, T) of a Maxwellian initial state from lambda^0 (one
// thread per cell, 32 consecutive cells along x per warp, FP64 sums).
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
        for (int p0 = 0; p0 < g.nvp; p0 += W) {
            T l0[W], l1[W];
            vld<T>(reinterpret_cast<const typename Vec<T>::type *>(lam + ebase<T>(g, 0, p0) + pk), l0);
            vld<T>(reinterpret_cast<const typename Vec<T>::type *>(lam + ebase<T>(g, 1, p0) + pk), l1);
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const int p = p0 + e;
                if (p >= g.nv) break;
                const double vx = g.vxmin + (p % g.nvx) * g.dvx, vy = g.vymin + (p / g.nvx) * g.dvy;
                const double ax = vx - st[1], ay = vy - st[2], a2 = ax * ax + ay * ay;
                const double M = st[0] / (2.0 * kPi * st[4]) * exp(-a2 / (2.0 * st[4]));
                const double d0 = M / st[0], d1 = M * ax / st[4], d2 = M * ay / st[4];
                const double d3 = M * (a2 / (2.0 * st[4] * st[4]) - 1.0 / st[4]);
                const double h = st[4] / 2.0;
                o0 += (double)l0[e] * d0 + (double)l1[e] * h * d0;
                o1 += (double)l0[e] * d1 + (double)l1[e] * h * d1;
                o2 += (double)l0[e] * d2 + (double)l1[e] * h * d2;
                o3 += (double)l0[e] * d3 + (double)l1[e] * (M / 2.0 + h * d3);
            }
        }
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
    void *fin = nullptr, *finpart = nullptr;         // F^N and its partial moments
    void *scratch_part = nullptr;                    // partial moments written by a tape fusion
    std::vector<void *> ckpt, ckpt_part, tape, ptape;
    std::vector<CUtensorMap> tmaps;                  // TMA descriptors of the tape buffers
    int cap = 0;
};

void release(AdjWork &w)
{
    for (int b = 0; b < 2; ++b) cudaFree(w.lam[b]);
    cudaFree(w.mucv); cudaFree(w.aux); cudaFree(w.bown); cudaFree(w.cvx); cudaFree(w.rev);
    cudaFree(w.gtw); cudaFree(w.jwall); cudaFree(w.gbc); cudaFree(w.ginit); cudaFree(w.wsec);
    cudaFree(w.fin); cudaFree(w.finpart); cudaFree(w.scratch_part);
    cudaFree(w.fast); cudaFree(w.slow); cudaFree(w.nslow_d);
    for (void *p : w.ckpt) cudaFree(p);
    for (void *p : w.ckpt_part) cudaFree(p);
    for (void *p : w.tape) cudaFree(p);
    for (void *p : w.ptape) cudaFree(p);
    w = AdjWork();
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
    return a;
}

// One reverse step: lam_in = lambda^{n+1}, f = F^n (device layout) -> lam_out.
template <typename T>
cudaError_t adjoint_step(dvm_ctx *c, AdjWork &w, const T *f, const T *part, const T *lam_in, T *lam_out)
{
    const AdjArgs a = adj_args(c, w);
    const int cvgrid = 4 * 152;
    T *mucv = (T *)w.mucv, *aux = (T *)w.aux;
    k_adj_mu<T><<<cvgrid, 256, 0, c->stream>>>(a, lam_in, mucv);
    const dim3 cgrid(nba(c->nx, 32), nba(c->ny, 8)), cblock(32, 8);
    k_adj_relax<T><<<cgrid, cblock, 0, c->stream>>>(a, f, part, c->S, lam_in, mucv, aux);
    if (c->scheme == DVM_MUSCL)
        k_adj_gather_fast<T, true><<<cgrid, cblock, 0, c->stream>>>(a, f, lam_in, aux, w.fast, lam_out);
    else
        k_adj_gather_fast<T, false><<<cgrid, cblock, 0, c->stream>>>(a, f, lam_in, aux, w.fast, lam_out);
    if (w.nslow > 0)
        k_adj_gather_list<T><<<nba((long)w.nslow * c->nvp, 256), 256, 0, c->stream>>>(a, f, lam_in, mucv, aux, w.slow,
                                                                                      w.nslow, lam_out);
    k_adj_wall<T><<<cvgrid, 256, 0, c->stream>>>(a, f, lam_in, mucv, lam_out, w.gtw, w.jwall, w.wsec, 0);
    k_adj_fuseT<T><<<cvgrid, 256, 0, c->stream>>>(a, lam_out);
    const int nside[4] = {c->ny, c->ny, c->nx, c->nx};
    const int nmax = c->nx > c->ny ? c->nx : c->ny;
    for (int s = 0; s < 4; ++s)
        if (c->bc[s] == DVM_BC_MAXWELLIAN && c->d_bcstate[s])
            k_adj_ghost<T><<<nside[s], 256, 0, c->stream>>>(a, f, lam_in, mucv, s, nside[s], c->d_bcstate[s],
                                                            w.gbc + 5L * s * nmax);
    c->launches += 6;
    return cudaGetLastError();
}

template <typename T>
int drag_adjoint_t(dvm_ctx *c, int nsteps, int K, double *J, double *gTw, double *const *gbc, double *gprim0,
                   double *ms_forward, double *ms_reverse)
{
    if (!c->adj) c->adj = new AdjWork();
    AdjWork &w = *static_cast<AdjWork *>(c->adj);
    const size_t bytes = c->dev_elems * c->elem;
    const size_t partb = (size_t)c->S * 4 * c->nc * c->elem;
    const int nmax = c->nx > c->ny ? c->nx : c->ny;
    const int nseg = (nsteps + K - 1) / K;
    cudaError_t e = cudaSuccess;
#define AC(call) do { e = (call); if (e != cudaSuccess) return cuda_fail(e, #call); } while (0)
    if (w.bytes_state != bytes || w.cap != c->list_cap) {
        release(w);
        for (int b = 0; b < 2; ++b) AC(cudaMalloc(&w.lam[b], bytes));
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
        AC(cudaMalloc(&w.nslow_d, sizeof(int)));
        w.bytes_state = bytes;
        w.cap = c->list_cap;
    }
    while ((int)w.ckpt.size() < nseg) {
        void *p = nullptr, *q = nullptr;
        AC(cudaMalloc(&p, bytes));
        AC(cudaMalloc(&q, partb));
        w.ckpt.push_back(p);
        w.ckpt_part.push_back(q);
    }
    while ((int)w.tape.size() < K) {
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
    // the tape buffers take the boundary padding (Maxwellian ghosts) of the state
    for (int t = 0; t < K; ++t)
        AC(cudaMemcpyAsync(w.tape[t], c->f[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
    AC(cudaMemsetAsync(w.gbc, 0, sizeof(double) * 5 * 4 * nmax, c->stream));
    AC(cudaMemsetAsync(w.gtw, 0, sizeof(double) * c->list_cap, c->stream));
    {
        const Grid2D g = grid2d(c);
        k_adj_rev<<<nba(c->list_cap, 256), 256, 0, c->stream>>>(c->spec_list, c->counts, c->list_cap, w.rev);
        k_adj_setup<T><<<nba(c->nc, 256), 256, 0, c->stream>>>(g, c->master, c->flags, w.rev, (const CvInfo *)c->cvinfo,
                                                                w.cvx, (T *)w.bown);
        k_adj_fastmask<<<nba(c->nc, 256), 256, 0, c->stream>>>(g, c->flags, w.fast);
        k_adj_slowlist<<<1, 1024, 0, c->stream>>>(c->nc, w.fast, w.slow, w.nslow_d);
        AC(cudaMemcpyAsync(&w.nslow, w.nslow_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        AC(cudaStreamSynchronize(c->stream));
    }
    cudaEvent_t ev[3];
    for (int q = 0; q < 3; ++q) AC(cudaEventCreate(&ev[q]));
    const bool fuse0 = c->need_fusion;
    const long long steps0 = c->steps_done;
    AC(cudaEventRecord(ev[0], c->stream));
    // forward with checkpoints every K steps
    for (int n = 0; n < nsteps; ++n) {
        if (n % K == 0) {
            AC(cudaMemcpyAsync(w.ckpt[n / K], c->f[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
            AC(cudaMemcpyAsync(w.ckpt_part[n / K], c->part[c->cur], partb, cudaMemcpyDeviceToDevice, c->stream));
        }
        AC(step2d(c));
    }
    AC(cudaEventRecord(ev[1], c->stream));
    AC(cudaMemcpyAsync(w.fin, c->f[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
    AC(cudaMemcpyAsync(w.finpart, c->part[c->cur], partb, cudaMemcpyDeviceToDevice, c->stream));
    dvm::BodyDev body_end;
    AC(cudaMemcpyAsync(&body_end, c->d_body, sizeof(body_end), cudaMemcpyDeviceToHost, c->stream));
    const AdjArgs a = adj_args(c, w);
    const int cvgrid = 4 * 152;
    // objective on F^N: lambda^N = fusion^T dJ/dF
    T *lamA = (T *)w.lam[0], *lamB = (T *)w.lam[1];
    AC(cudaMemsetAsync(lamA, 0, bytes, c->stream));
    k_adj_wall<T><<<cvgrid, 256, 0, c->stream>>>(a, (const T *)c->f[c->cur], lamA, (const T *)w.mucv, lamA, w.gtw,
                                                 w.jwall, w.wsec, 1);
    k_adj_fuseT<T><<<cvgrid, 256, 0, c->stream>>>(a, lamA);
    // reverse sweep, segment by segment: recompute the segment onto the tape
    // (each step writes the next tape buffer), then apply the transposed steps
    // backwards
    void *f_orig[2] = {c->f[0], c->f[1]};
    const CUtensorMap tm_orig[2] = {c->tmap[0], c->tmap[1]};
    const int cur_orig = c->cur;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int n0 = sgi * K, n1 = (n0 + K < nsteps) ? n0 + K : nsteps, len = n1 - n0;
        AC(cudaMemcpyAsync(w.tape[0], w.ckpt[sgi], bytes, cudaMemcpyDeviceToDevice, c->stream));
        AC(cudaMemcpyAsync(c->part[c->cur], w.ckpt_part[sgi], partb, cudaMemcpyDeviceToDevice, c->stream));
        // the step linearises around the fused state (members of merged control
        // volumes are equal after every step, not necessarily in the initial state)
        if (sgi == 0 && fuse0) AC(fusion2d(c, w.tape[0], c->part[c->cur]));
        c->need_fusion = false;
        for (int t = 0; t < len; ++t) {
            if (t + 1 < len) {
                c->f[c->cur] = w.tape[t];
                c->f[1 - c->cur] = w.tape[t + 1];
                c->tmap[c->cur] = w.tmaps[t];
                c->tmap[1 - c->cur] = w.tmaps[t + 1];
                AC(step2d(c));
                AC(cudaMemcpyAsync(w.ptape[t], c->part[1 - c->cur], partb, cudaMemcpyDeviceToDevice, c->stream));
            } else {
                AC(cudaMemcpyAsync(w.ptape[t], c->part[c->cur], partb, cudaMemcpyDeviceToDevice, c->stream));
            }
        }
        c->f[0] = f_orig[0]; c->f[1] = f_orig[1];
        c->tmap[0] = tm_orig[0]; c->tmap[1] = tm_orig[1];
        c->cur = cur_orig;
        for (int t = len - 1; t >= 0; --t) {
            AC(adjoint_step<T>(c, w, (const T *)w.tape[t], (const T *)w.ptape[t], lamA, lamB));
            T *tt = lamA; lamA = lamB; lamB = tt;
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
    for (int s = 0; s < 4; ++s) {
        if (!gbc || !gbc[s]) continue;
        if (c->bc[s] != DVM_BC_MAXWELLIAN) { std::memset(gbc[s], 0, sizeof(double) * 5 * nside[s]); continue; }
        AC(cudaMemcpyAsync(gbc[s], w.gbc + 5L * s * nmax, sizeof(double) * 5 * nside[s], cudaMemcpyDeviceToHost, c->stream));
    }
    if (gprim0) {
        if (!c->have_prim0) { set_error("dvm_drag_adjoint: gprim0 needs a state set by dvm_init_maxwellian"); return DVM_ERR_STATE; }
        k_adj_init<T><<<dim3(nba(c->nx, 32), nba(c->ny, 8)), dim3(32, 8), 0, c->stream>>>(grid2d(c), lamA, c->d_prim0,
                                                                                      c->geo[c->gcur].type, w.ginit);
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
                   double *ms_forward, double *ms_reverse)
{
    return c->prec == DVM_FP32 ? drag_adjoint_t<float>(c, nsteps, K, J, gTw, gbc, gprim0, ms_forward, ms_reverse)
                               : drag_adjoint_t<double>(c, nsteps, K, J, gTw, gbc, gprim0, ms_forward, ms_reverse);
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
