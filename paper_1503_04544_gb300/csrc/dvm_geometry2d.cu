// 2D cut-cell geometry on the device (Appendix A of arXiv:1503.04544):
// nodal level set, cell types, Cartesian edge lengths, wall edge, area,
// master search and per-cell flags for the step kernels.
//
// This translation unit is compiled with --fmad=false: every quantity is a
// composition of correctly rounded +, -, *, /, sqrt, min and max, so the
// result is reproducible bit for bit by any IEEE-754 implementation that
// evaluates the same expressions in the same order.
#include "dvm_internal.h"

namespace dvm {
namespace {

__device__ __forceinline__ double levelset(const BodyParams &b, double ct, double st,
                                           double x, double y)
{
    double ddx = x - b.cx, ddy = y - b.cy;
    if (b.shape == DVM_SHAPE_CIRCLE) return sqrt(ddx * ddx + ddy * ddy) - b.ra;
    if (b.shape == DVM_SHAPE_ELLIPSE) {
        // first-order distance g / |grad g| of the rotated ellipse
        double xr = ct * ddx + st * ddy;
        double yr = -st * ddx + ct * ddy;
        double a2 = b.ra * b.ra, b2 = b.rb * b.rb;
        double g = xr * xr / a2 + yr * yr / b2 - 1.0;
        double gx = 2.0 * xr / a2, gy = 2.0 * yr / b2;
        double nrm = sqrt(gx * gx + gy * gy);
        if (nrm > 0) return g / nrm;
        return -(b.ra < b.rb ? b.ra : b.rb);
    }
    // containers: the gas inside
    if (b.shape == DVM_SHAPE_DISK_CONTAINER) return b.ra - sqrt(ddx * ddx + ddy * ddy);
    if (b.shape == DVM_SHAPE_BOX_CONTAINER) {
        const double x0 = b.cx - b.ra, x1 = b.cx + b.ra, y0 = b.cy - b.rb, y1 = b.cy + b.rb;
        return fmin(fmin(x - x0, x1 - x), fmin(y - y0, y1 - y));
    }
    return 1.0;
}

// Appendix A.1: nodes exactly on the wall are moved by 1e-10 dx.
__device__ __forceinline__ double clamp_phi(double p, double dx)
{
    double eps = 1e-10 * dx;
    if (p >= 0) return p > eps ? p : eps;
    return -p > eps ? p : -eps;
}

// Gas part of a Cartesian edge between nodal values p0 and p1 (length h).
__device__ __forceinline__ double edge_len(double p0, double p1, double h)
{
    if (p0 > 0 && p1 > 0) return h;
    if (p0 < 0 && p1 < 0) return 0.0;
    double o = h * (p0 / (p0 - p1));
    return p0 > 0 ? o : h - o;
}

__global__ void k_nodes(Grid2D g, BodyParams b, Geo2D G, const double *trig)
{
    int na = g.i1 - g.i0 + 1, nb = g.j1 - g.j0 + 1;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na * nb) return;
    int a = g.i0 + t % na, bb = g.j0 + t / na;
    double x = g.xmin + a * g.dx, y = g.ymin + bb * g.dy;
    G.phi[(long)bb * (g.nx + 1) + a] = clamp_phi(levelset(b, trig[0], trig[1], x, y), g.dx);
}

__global__ void k_edges(Grid2D g, Geo2D G)
{
    // vertical edges a in [i0, i1], rows j in [j0, j1); horizontal edges
    // b in [j0, j1], columns i in [i0, i1)
    int nvert = (g.i1 - g.i0 + 1) * (g.j1 - g.j0);
    int nhor = (g.i1 - g.i0) * (g.j1 - g.j0 + 1);
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int W = g.nx + 1;
    if (t < nvert) {
        int na = g.i1 - g.i0 + 1;
        int a = g.i0 + t % na, j = g.j0 + t / na;
        G.lx[(long)j * W + a] = edge_len(G.phi[(long)j * W + a], G.phi[(long)(j + 1) * W + a], g.dy);
    } else if (t < nvert + nhor) {
        t -= nvert;
        int ni = g.i1 - g.i0;
        int i = g.i0 + t % ni, bb = g.j0 + t / ni;
        G.ly[(long)bb * g.nx + i] = edge_len(G.phi[(long)bb * W + i], G.phi[(long)bb * W + i + 1], g.dx);
    }
}

__global__ void k_cells(Grid2D g, Geo2D G, int *err)
{
    int ni = g.i1 - g.i0, nj = g.j1 - g.j0;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ni * nj) return;
    int i = g.i0 + t % ni, j = g.j0 + t / ni;
    long k = (long)j * g.nx + i;
    const int W = g.nx + 1;
    double pmm = G.phi[(long)j * W + i], ppm = G.phi[(long)j * W + i + 1];
    double ppp = G.phi[(long)(j + 1) * W + i + 1], pmp = G.phi[(long)(j + 1) * W + i];
    double m = fmin(fmin(pmm, ppm), fmin(ppp, pmp));
    double M = fmax(fmax(pmm, ppm), fmax(ppp, pmp));
    G.cgas[k] = (0.25 * (((pmm + ppm) + ppp) + pmp)) > 0;   // Eq. (ii)
    double lw = 0, nwx = 0, nwy = 0, rwx = 0, rwy = 0, sbar;
    int8_t type;
    if (m > 0) {
        type = DVM_GAS;
        sbar = g.dx * g.dy;
    } else if (M < 0) {
        type = DVM_SOLID;
        sbar = 0;
    } else {
        type = DVM_CUT;
        double px[4], py[4];
        int n = 0;
        // crossings on the edges x-, x+, y-, y+ in the cell frame
        if ((pmm > 0) != (pmp > 0)) { px[n] = 0;    py[n] = g.dy * (pmm / (pmm - pmp)); ++n; }
        if ((ppm > 0) != (ppp > 0)) { px[n] = g.dx; py[n] = g.dy * (ppm / (ppm - ppp)); ++n; }
        if ((pmm > 0) != (ppm > 0)) { px[n] = g.dx * (pmm / (pmm - ppm)); py[n] = 0;    ++n; }
        if ((pmp > 0) != (ppp > 0)) { px[n] = g.dx * (pmp / (pmp - ppp)); py[n] = g.dy; ++n; }
        if (n != 2) {
            atomicExch(&err[kErrGeometry], 1);   // saddle cell: two wall pieces
            sbar = 0;
        } else {
            double lxm = G.lx[(long)j * W + i], lxp = G.lx[(long)j * W + i + 1];
            double lym = G.ly[(long)j * g.nx + i], lyp = G.ly[(long)(j + 1) * g.nx + i];
            double ex = px[1] - px[0], ey = py[1] - py[0];
            lw = sqrt(ex * ex + ey * ey);
            double rx = 0.5 * (px[0] + px[1]), ry = 0.5 * (py[0] + py[1]);
            // Green-formula normal, oriented into the solid
            nwx = (lxm - lxp) / lw;
            nwy = (lym - lyp) / lw;
            rwx = (g.xmin + i * g.dx) + rx;
            rwy = (g.ymin + j * g.dy) + ry;
            sbar = 0.5 * (lxp * g.dx + lyp * g.dy + lw * (rx * nwx + ry * nwy));
        }
    }
    G.type[k] = type;
    G.lw[k] = lw; G.nwx[k] = nwx; G.nwy[k] = nwy; G.rwx[k] = rwx; G.rwy[k] = rwy;
    G.sbar[k] = sbar;
}

__global__ void k_clear_hs(Grid2D g, uint8_t *hs)
{
    int ni = g.i1 - g.i0, nj = g.j1 - g.j0;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ni * nj) return;
    hs[(long)(g.j0 + t / ni) * g.nx + g.i0 + t % ni] = 0;
}

// Master search of Appendix A.3 (ties: x+, x-, y+, y-).  A cell solid at t^n
// but not at t^{n+1} walks with its t^{n+1} edges; the stopping test is
// Eq. (ii) at t^n.
__global__ void k_masters(Grid2D g, Geo2D Gn, Geo2D Gp, int32_t *master, uint8_t *hs, int *err)
{
    int ni = g.i1 - g.i0, nj = g.j1 - g.j0;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ni * nj) return;
    int i = g.i0 + t % ni, j = g.j0 + t / ni;
    long k = (long)j * g.nx + i;
    if (Gn.type[k] == DVM_SOLID && Gp.type[k] == DVM_SOLID) { master[k] = -1; return; }
    const int W = g.nx + 1;
    int ci = i, cj = j;
    bool ok = false;
    for (int it = 0; it <= kMaxWalk; ++it) {
        long q = (long)cj * g.nx + ci;
        if (Gn.cgas[q]) { ok = true; break; }
        const Geo2D &G = Gn.type[q] != DVM_SOLID ? Gn : Gp;
        double lxm = G.lx[(long)cj * W + ci], lxp = G.lx[(long)cj * W + ci + 1];
        double lym = G.ly[(long)cj * g.nx + ci], lyp = G.ly[(long)(cj + 1) * g.nx + ci];
        double M = fmax(fmax(lxp, lxm), fmax(lyp, lym));
        if (!(M > 0)) break;
        if (lxp == M) ci++;
        else if (lxm == M) ci--;
        else if (lyp == M) cj++;
        else cj--;
        if (ci < g.i0 || ci >= g.i1 || cj < g.j0 || cj >= g.j1) break;
    }
    if (!ok) { atomicExch(&err[kErrGeometry], 1); master[k] = -1; return; }
    long m = (long)cj * g.nx + ci;
    master[k] = (int32_t)m;
    if (m != k) hs[m] = 1;
}

// Gas test for the limiter stencil; ghost cells beyond non-periodic sides
// count as gas.
__device__ __forceinline__ bool gas_at(const Grid2D &g, const int8_t *type, int i, int j)
{
    if (i < 0) { if (g.bc[0] != DVM_BC_PERIODIC) return true; i += g.nx; }
    else if (i >= g.nx) { if (g.bc[1] != DVM_BC_PERIODIC) return true; i -= g.nx; }
    if (j < 0) { if (g.bc[2] != DVM_BC_PERIODIC) return true; j += g.ny; }
    else if (j >= g.ny) { if (g.bc[3] != DVM_BC_PERIODIC) return true; j -= g.ny; }
    return type[(long)j * g.nx + i] == DVM_GAS;
}

__global__ void k_flags(Grid2D g, Geo2D Gn, Geo2D Gp, const int32_t *master, const uint8_t *hs,
                        uint8_t *flags, bool moving, bool muscl)
{
    int ni = g.i1 - g.i0, nj = g.j1 - g.j0;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ni * nj) return;
    int i = g.i0 + t % ni, j = g.j0 + t / ni;
    long k = (long)j * g.nx + i;
    uint8_t f = 0;
    int32_t m = master[k];
    if (m < 0) {
        f = moving ? kZero : 0;
    } else if (Gn.type[k] == DVM_GAS && Gp.type[k] == DVM_GAS && m == k && !hs[k]) {
        f = kPlain;
    } else {
        f = kSpecial;
    }
    if (muscl) {
        const int8_t *ty = Gn.type;
        bool gm2 = gas_at(g, ty, i - 2, j), gm1 = gas_at(g, ty, i - 1, j), g0 = gas_at(g, ty, i, j);
        bool gp1 = gas_at(g, ty, i + 1, j), gp2 = gas_at(g, ty, i + 2, j);
        bool hm2 = gas_at(g, ty, i, j - 2), hm1 = gas_at(g, ty, i, j - 1);
        bool hp1 = gas_at(g, ty, i, j + 1), hp2 = gas_at(g, ty, i, j + 2);
        uint8_t mask = 0;
        if (gm2 && gm1 && g0 && gp1) mask |= 1;   // face x-
        if (gm1 && g0 && gp1 && gp2) mask |= 2;   // face x+
        if (hm2 && hm1 && g0 && hp1) mask |= 4;   // face y-
        if (hm1 && g0 && hp1 && hp2) mask |= 8;   // face y+
        f |= mask << kMaskShift;
    }
    flags[k] = f;
}

// Exclusive block-wide prefix count of a predicate (1024 threads).
__device__ int block_excl_scan(bool pred, int *wsum, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned b = __ballot_sync(0xffffffffu, pred);
    int pre = __popc(b & ((1u << lane) - 1u));
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        wsum[lane] = inc - v;
        if (lane == 31) *total = inc;
    }
    __syncthreads();
    int r = wsum[warp] + pre;
    __syncthreads();
    return r;
}

// Control-volume masters and wall cells of the box, listed in cell order
// (deterministic, so that the force and torque sums have a fixed order).
__global__ void __launch_bounds__(1024) k_lists(Grid2D g, Geo2D Gn, const int32_t *master,
                                                const uint8_t *flags, int32_t *spec_list,
                                                int32_t *wall_list, int32_t *wslot,
                                                int32_t *counts, int cap, int *err)
{
    __shared__ int wsum[32];
    __shared__ int tot;
    const int ni = g.i1 - g.i0, nbox = ni * (g.j1 - g.j0);
    int nspec = 0, nwall = 0;
    for (int base = 0; base < nbox; base += blockDim.x) {
        const int t = base + threadIdx.x;
        bool sp = false, wl = false;
        long k = 0;
        if (t < nbox) {
            k = (long)(g.j0 + t / ni) * g.nx + g.i0 + t % ni;
            sp = (flags[k] & kSpecial) && master[k] == (int32_t)k;
            wl = Gn.type[k] == DVM_CUT && Gn.lw[k] > 0;
        }
        int ps = block_excl_scan(sp, wsum, &tot) + nspec;
        __syncthreads();
        nspec += tot;
        __syncthreads();
        int pw = block_excl_scan(wl, wsum, &tot) + nwall;
        __syncthreads();
        nwall += tot;
        if (t < nbox) {
            if (sp) { if (ps < cap) spec_list[ps] = (int32_t)k; else atomicExch(&err[kErrCapacity], 1); }
            wslot[k] = wl && pw < cap ? pw : -1;
            if (wl) { if (pw < cap) wall_list[pw] = (int32_t)k; else atomicExch(&err[kErrCapacity], 1); }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        counts[0] = nspec < cap ? nspec : cap;
        counts[1] = nwall < cap ? nwall : cap;
    }
}

__global__ void k_static_fill(Grid2D g, Geo2D G, int32_t *master, uint8_t *flags, uint8_t *hs,
                              int32_t *wslot, bool muscl)
{
    long nc = (long)g.nx * g.ny;
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nc) {
        G.type[t] = DVM_GAS; G.cgas[t] = 1;
        G.lw[t] = 0; G.nwx[t] = 0; G.nwy[t] = 0; G.rwx[t] = 0; G.rwy[t] = 0;
        G.sbar[t] = g.dx * g.dy;
        master[t] = (int32_t)t;
        hs[t] = 0;
        wslot[t] = -1;
        flags[t] = kPlain | (muscl ? (uint8_t)(0xF << kMaskShift) : 0);
    }
    long nvert = (long)(g.nx + 1) * g.ny;
    if (t < nvert) G.lx[t] = g.dy;
    long nhor = (long)g.nx * (g.ny + 1);
    if (t < nhor) G.ly[t] = g.dx;
    long nnode = (long)(g.nx + 1) * (g.ny + 1);
    if (t < nnode) G.phi[t] = 1.0;
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

cudaError_t init_static_geometry2d(dvm_ctx *c)
{
    Grid2D g = grid2d(c);
    long n = (long)(c->nx + 1) * (c->ny + 1);
    for (int l = 0; l < 2; ++l)
        k_static_fill<<<nblk(n, 256), 256, 0, c->stream>>>(g, c->geo[l], c->master, c->flags,
                                                           c->hs, c->wslot, c->scheme == DVM_MUSCL);
    return cudaGetLastError();
}

cudaError_t geometry2d_level(dvm_ctx *c, int level, const double *d_trig)
{
    Grid2D g = grid2d(c);
    if (g.i1 <= g.i0 || g.j1 <= g.j0) return cudaSuccess;
    BodyParams b = body_params(c);
    const Geo2D &G = c->geo[level];
    int nn = (g.i1 - g.i0 + 1) * (g.j1 - g.j0 + 1);
    k_nodes<<<nblk(nn, 256), 256, 0, c->stream>>>(g, b, G, d_trig);
    int ne = (g.i1 - g.i0 + 1) * (g.j1 - g.j0) + (g.i1 - g.i0) * (g.j1 - g.j0 + 1);
    k_edges<<<nblk(ne, 256), 256, 0, c->stream>>>(g, G);
    int ncell = (g.i1 - g.i0) * (g.j1 - g.j0);
    k_cells<<<nblk(ncell, 256), 256, 0, c->stream>>>(g, G, c->d_err);
    return cudaGetLastError();
}

cudaError_t masters_flags2d(dvm_ctx *c, bool moving)
{
    Grid2D g = grid2d(c);
    if (g.i1 <= g.i0 || g.j1 <= g.j0) return cudaSuccess;
    int ncell = (g.i1 - g.i0) * (g.j1 - g.j0);
    const Geo2D &Gn = c->geo[c->gcur];
    const Geo2D &Gp = moving ? c->geo[1 - c->gcur] : c->geo[c->gcur];
    k_clear_hs<<<nblk(ncell, 256), 256, 0, c->stream>>>(g, c->hs);
    k_masters<<<nblk(ncell, 256), 256, 0, c->stream>>>(g, Gn, Gp, c->master, c->hs, c->d_err);
    k_flags<<<nblk(ncell, 256), 256, 0, c->stream>>>(g, Gn, Gp, c->master, c->hs, c->flags, moving,
                                                     c->scheme == DVM_MUSCL);
    k_lists<<<1, 1024, 0, c->stream>>>(g, Gn, c->master, c->flags, c->spec_list, c->wall_list,
                                       c->wslot, c->counts, c->list_cap, c->d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return members2d(c, moving);
    return cudaGetLastError();
}

}  // namespace dvm
