// 3D cut-cell geometry on the device (arXiv:1503.04544, Sec. 5; the paper
// leaves the 3D geometry to the reader).  Reading: every Cartesian face gets
// the gas area of the 2D virtual-cell construction of Appendix A applied to
// its four nodes; the wall face closes the polyhedron,
// S_w n_w = (A_x- - A_x+, A_y- - A_y+, A_z- - A_z+); the wall centre is the
// mean of the crossings of the level set with the twelve cell edges; the
// volume follows from the divergence theorem in the cell frame.  The master
// search of Appendix A.3 walks across the largest of the six faces (ties:
// x+, x-, y+, y-, z+, z-).
//
// Compiled with --fmad=false: every quantity is a composition of correctly
// rounded +, -, *, /, sqrt, min and max evaluated in a fixed order, so any
// IEEE-754 implementation of the same expressions reproduces it bit for bit.
#include "dvm_internal.h"

namespace dvm {
namespace {

__device__ __forceinline__ double levelset3(const BodyParams &b, double x, double y, double z)
{
    const double ddx = x - b.cx, ddy = y - b.cy, ddz = z - b.cz;
    if (b.shape == DVM_SHAPE_SPHERE) return sqrt(ddx * ddx + ddy * ddy + ddz * ddz) - b.ra;
    return 1.0;
}

// Appendix A.1: nodes exactly on the wall are moved by 1e-10 dx.
__device__ __forceinline__ double clamp_phi3(double p, double dx)
{
    const double eps = 1e-10 * dx;
    if (p >= 0) return p > eps ? p : eps;
    return -p > eps ? p : -eps;
}

// Gas part of an edge of length h between nodal values p0 and p1.
__device__ __forceinline__ double edge_len3(double p0, double p1, double h)
{
    if (p0 > 0 && p1 > 0) return h;
    if (p0 < 0 && p1 < 0) return 0.0;
    const double o = h * (p0 / (p0 - p1));
    return p0 > 0 ? o : h - o;
}

// Gas area of a face with nodal values p00 (u=0, w=0), p10 (u=h1, w=0),
// p11 (u=h1, w=h2), p01 (u=0, w=h2): the Green formula of Appendix A in the
// face's own frame.  A face crossed twice (saddle) raises kErrGeometry.
__device__ double face_area(double p00, double p10, double p11, double p01, double h1, double h2, int *err)
{
    const double m = fmin(fmin(p00, p10), fmin(p11, p01));
    const double M = fmax(fmax(p00, p10), fmax(p11, p01));
    if (m > 0) return h1 * h2;
    if (M < 0) return 0.0;
    const double lum = edge_len3(p00, p01, h2), lup = edge_len3(p10, p11, h2);
    const double lwp = edge_len3(p01, p11, h1);
    const double lwm = edge_len3(p00, p10, h1);
    double pu[2], pw[2];
    int n = 0;
    // crossings in a fixed order: u = 0, u = h1, w = 0, w = h2
    if ((p00 > 0) != (p01 > 0)) { if (n < 2) { pu[n] = 0;  pw[n] = h2 * (p00 / (p00 - p01)); } ++n; }
    if ((p10 > 0) != (p11 > 0)) { if (n < 2) { pu[n] = h1; pw[n] = h2 * (p10 / (p10 - p11)); } ++n; }
    if ((p00 > 0) != (p10 > 0)) { if (n < 2) { pu[n] = h1 * (p00 / (p00 - p10)); pw[n] = 0;  } ++n; }
    if ((p01 > 0) != (p11 > 0)) { if (n < 2) { pu[n] = h1 * (p01 / (p01 - p11)); pw[n] = h2; } ++n; }
    if (n != 2) { atomicExch(&err[kErrGeometry], 1); return 0.0; }
    const double eu = pu[1] - pu[0], ew = pw[1] - pw[0];
    const double lw = sqrt(eu * eu + ew * ew);
    const double ru = 0.5 * (pu[0] + pu[1]), rw = 0.5 * (pw[0] + pw[1]);
    const double nu = (lum - lup) / lw, nw = (lwm - lwp) / lw;
    return 0.5 * (lup * h1 + lwp * h2 + lw * (ru * nu + rw * nw));
}

__device__ __forceinline__ long node3(const Grid3D &g, int a, int b, int c)
{
    return ((long)c * (g.ny + 1) + b) * (g.nx + 1) + a;
}

__global__ void k_nodes3(Grid3D g, BodyParams b, Geo3D G)
{
    const long nn = (long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nn) return;
    const int a = (int)(t % (g.nx + 1));
    const long r = t / (g.nx + 1);
    const int bb = (int)(r % (g.ny + 1)), c = (int)(r / (g.ny + 1));
    G.phi[t] = clamp_phi3(levelset3(b, g.xmin + a * g.dx, g.ymin + bb * g.dy, g.zmin + c * g.dz), g.dx);
}

// Face areas: x-faces a of (j, k), y-faces b of (i, k), z-faces c of (i, j).
__global__ void k_faces3(Grid3D g, Geo3D G, int *err)
{
    const long nxf = (long)(g.nx + 1) * g.ny * g.nz;
    const long nyf = (long)g.nx * (g.ny + 1) * g.nz;
    const long nzf = (long)g.nx * g.ny * (g.nz + 1);
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nxf) {
        const int a = (int)(t % (g.nx + 1));
        const long r = t / (g.nx + 1);
        const int j = (int)(r % g.ny), k = (int)(r / g.ny);
        G.ax[t] = face_area(G.phi[node3(g, a, j, k)], G.phi[node3(g, a, j + 1, k)], G.phi[node3(g, a, j + 1, k + 1)],
                            G.phi[node3(g, a, j, k + 1)], g.dy, g.dz, err);
        return;
    }
    t -= nxf;
    if (t < nyf) {
        const int i = (int)(t % g.nx);
        const long r = t / g.nx;
        const int bb = (int)(r % (g.ny + 1)), k = (int)(r / (g.ny + 1));
        G.ay[t] = face_area(G.phi[node3(g, i, bb, k)], G.phi[node3(g, i + 1, bb, k)], G.phi[node3(g, i + 1, bb, k + 1)],
                            G.phi[node3(g, i, bb, k + 1)], g.dx, g.dz, err);
        return;
    }
    t -= nyf;
    if (t < nzf) {
        const int i = (int)(t % g.nx);
        const long r = t / g.nx;
        const int j = (int)(r % g.ny), c = (int)(r / g.ny);
        G.az[t] = face_area(G.phi[node3(g, i, j, c)], G.phi[node3(g, i + 1, j, c)], G.phi[node3(g, i + 1, j + 1, c)],
                            G.phi[node3(g, i, j + 1, c)], g.dx, g.dy, err);
    }
}

__global__ void k_cells3(Grid3D g, Geo3D G)
{
    const long nc = (long)g.nx * g.ny * g.nz;
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    const int i = (int)(q % g.nx);
    const long r = q / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    // nodes: (i,j,k) (i+1,j,k) (i+1,j+1,k) (i,j+1,k), then the same at k+1
    double p[8];
    p[0] = G.phi[node3(g, i, j, k)];         p[1] = G.phi[node3(g, i + 1, j, k)];
    p[2] = G.phi[node3(g, i + 1, j + 1, k)]; p[3] = G.phi[node3(g, i, j + 1, k)];
    p[4] = G.phi[node3(g, i, j, k + 1)];     p[5] = G.phi[node3(g, i + 1, j, k + 1)];
    p[6] = G.phi[node3(g, i + 1, j + 1, k + 1)]; p[7] = G.phi[node3(g, i, j + 1, k + 1)];
    double m = p[0], M = p[0], s = p[0];
    for (int t = 1; t < 8; ++t) { m = fmin(m, p[t]); M = fmax(M, p[t]); s = s + p[t]; }
    G.cgas[q] = 0.125 * s > 0;        // Eq. (ii) with the eight nodes
    double sw = 0, nwx = 0, nwy = 0, nwz = 0, rwx = 0, rwy = 0, rwz = 0, vol;
    int8_t type;
    if (m > 0) {
        type = DVM_GAS;
        vol = g.dx * g.dy * g.dz;
    } else if (M < 0) {
        type = DVM_SOLID;
        vol = 0;
    } else {
        type = DVM_CUT;
        const long xf = ((long)k * g.ny + j) * (g.nx + 1) + i;
        const long yf = ((long)k * (g.ny + 1) + j) * g.nx + i;
        const long zf = ((long)k * g.ny + j) * g.nx + i;
        const double axm = G.ax[xf], axp = G.ax[xf + 1];
        const double aym = G.ay[yf], ayp = G.ay[yf + g.nx];
        const double azm = G.az[zf], azp = G.az[zf + (long)g.nx * g.ny];
        const double wx = axm - axp, wy = aym - ayp, wz = azm - azp;
        sw = sqrt(wx * wx + wy * wy + wz * wz);
        // the twelve edges: four along x, four along y, four along z
        const int E0[12] = {0, 3, 4, 7, 0, 1, 4, 5, 0, 1, 3, 2};
        const int E1[12] = {1, 2, 5, 6, 3, 2, 7, 6, 4, 5, 7, 6};
        double rx = 0, ry = 0, rz = 0;
        int nc2 = 0;
        for (int e = 0; e < 12; ++e) {
            const double p0 = p[E0[e]], p1 = p[E1[e]];
            if ((p0 > 0) == (p1 > 0)) continue;
            const double tt = p0 / (p0 - p1);
            const int a0 = E0[e], a1 = E1[e];
            // unit-cube coordinates of the corners: x = bit pattern of the
            // node order above
            const double o0x = (a0 == 1 || a0 == 2 || a0 == 5 || a0 == 6) ? 1.0 : 0.0;
            const double o0y = (a0 == 2 || a0 == 3 || a0 == 6 || a0 == 7) ? 1.0 : 0.0;
            const double o0z = a0 >= 4 ? 1.0 : 0.0;
            const double o1x = (a1 == 1 || a1 == 2 || a1 == 5 || a1 == 6) ? 1.0 : 0.0;
            const double o1y = (a1 == 2 || a1 == 3 || a1 == 6 || a1 == 7) ? 1.0 : 0.0;
            const double o1z = a1 >= 4 ? 1.0 : 0.0;
            rx += g.dx * (o0x + tt * (o1x - o0x));
            ry += g.dy * (o0y + tt * (o1y - o0y));
            rz += g.dz * (o0z + tt * (o1z - o0z));
            ++nc2;
        }
        rx /= nc2; ry /= nc2; rz /= nc2;
        nwx = sw > 0 ? wx / sw : 0;
        nwy = sw > 0 ? wy / sw : 0;
        nwz = sw > 0 ? wz / sw : 0;
        rwx = (g.xmin + i * g.dx) + rx;
        rwy = (g.ymin + j * g.dy) + ry;
        rwz = (g.zmin + k * g.dz) + rz;
        vol = (axp * g.dx + ayp * g.dy + azp * g.dz + sw * (rx * nwx + ry * nwy + rz * nwz)) / 3.0;
    }
    G.type[q] = type;
    G.sw[q] = sw; G.nwx[q] = nwx; G.nwy[q] = nwy; G.nwz[q] = nwz;
    G.rwx[q] = rwx; G.rwy[q] = rwy; G.rwz[q] = rwz;
    G.vol[q] = vol;
}

// Master search (Appendix A.3 with six faces) of a fixed obstacle.
__global__ void k_masters3(Grid3D g, Geo3D G, int32_t *master, uint8_t *hs, int *err)
{
    const long nc = (long)g.nx * g.ny * g.nz;
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    if (G.type[q] == DVM_SOLID) { master[q] = -1; return; }
    int ci = (int)(q % g.nx);
    const long r = q / g.nx;
    int cj = (int)(r % g.ny), ck = (int)(r / g.ny);
    bool ok = false;
    for (int it = 0; it <= kMaxWalk; ++it) {
        const long c = ((long)ck * g.ny + cj) * g.nx + ci;
        if (G.cgas[c]) { ok = true; break; }
        const long xf = ((long)ck * g.ny + cj) * (g.nx + 1) + ci;
        const long yf = ((long)ck * (g.ny + 1) + cj) * g.nx + ci;
        const long zf = ((long)ck * g.ny + cj) * g.nx + ci;
        const double axm = G.ax[xf], axp = G.ax[xf + 1];
        const double aym = G.ay[yf], ayp = G.ay[yf + g.nx];
        const double azm = G.az[zf], azp = G.az[zf + (long)g.nx * g.ny];
        const double M = fmax(fmax(fmax(axp, axm), fmax(ayp, aym)), fmax(azp, azm));
        if (!(M > 0)) break;
        if (axp == M) ci++;
        else if (axm == M) ci--;
        else if (ayp == M) cj++;
        else if (aym == M) cj--;
        else if (azp == M) ck++;
        else ck--;
        if (ci < 0 || ci >= g.nx || cj < 0 || cj >= g.ny || ck < 0 || ck >= g.nz) break;
    }
    if (!ok) { atomicExch(&err[kErrGeometry], 1); master[q] = -1; return; }
    const long m = ((long)ck * g.ny + cj) * g.nx + ci;
    master[q] = (int32_t)m;
    if (m != q) hs[m] = 1;
}

__device__ __forceinline__ int wrap3(int a, int n, int bc, bool &ghost)
{
    if (a >= 0 && a < n) return a;
    if (bc != DVM_BC_PERIODIC) { ghost = true; return 0; }
    return a < 0 ? a + n : a - n;
}

// Gas test of the limiter stencil: ghost cells beyond non-periodic sides
// count as gas.
__device__ __forceinline__ bool gas3(const Grid3D &g, const int8_t *type, int i, int j, int k)
{
    bool ghost = false;
    i = i < 0 ? wrap3(i, g.nx, g.bc[0], ghost) : (i >= g.nx ? wrap3(i, g.nx, g.bc[1], ghost) : i);
    j = j < 0 ? wrap3(j, g.ny, g.bc[2], ghost) : (j >= g.ny ? wrap3(j, g.ny, g.bc[3], ghost) : j);
    k = k < 0 ? wrap3(k, g.nz, g.bc[4], ghost) : (k >= g.nz ? wrap3(k, g.nz, g.bc[5], ghost) : k);
    if (ghost) return true;
    return type[((long)k * g.ny + j) * g.nx + i] == DVM_GAS;
}

__global__ void k_flags3(Grid3D g, Geo3D G, const int32_t *master, const uint8_t *hs, uint16_t *flags, bool muscl)
{
    const long nc = (long)g.nx * g.ny * g.nz;
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    const int i = (int)(q % g.nx);
    const long r = q / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    uint16_t f = 0;
    const int32_t m = master[q];
    if (m < 0) f = 0;
    else if (G.type[q] == DVM_GAS && m == q && !hs[q]) f = kPlain;
    else f = kSpecial;
    if (muscl) {
        const int8_t *ty = G.type;
        const bool c0 = gas3(g, ty, i, j, k);
        uint16_t mask = 0;
        if (gas3(g, ty, i - 2, j, k) && gas3(g, ty, i - 1, j, k) && c0 && gas3(g, ty, i + 1, j, k)) mask |= 1;
        if (gas3(g, ty, i - 1, j, k) && c0 && gas3(g, ty, i + 1, j, k) && gas3(g, ty, i + 2, j, k)) mask |= 2;
        if (gas3(g, ty, i, j - 2, k) && gas3(g, ty, i, j - 1, k) && c0 && gas3(g, ty, i, j + 1, k)) mask |= 4;
        if (gas3(g, ty, i, j - 1, k) && c0 && gas3(g, ty, i, j + 1, k) && gas3(g, ty, i, j + 2, k)) mask |= 8;
        if (gas3(g, ty, i, j, k - 2) && gas3(g, ty, i, j, k - 1) && c0 && gas3(g, ty, i, j, k + 1)) mask |= 16;
        if (gas3(g, ty, i, j, k - 1) && c0 && gas3(g, ty, i, j, k + 1) && gas3(g, ty, i, j, k + 2)) mask |= 32;
        f |= (uint16_t)(mask << kMaskShift3);
    }
    flags[q] = f;
}

// Exclusive block-wide prefix count of a predicate (1024 threads).
__device__ int block_excl_scan3(bool pred, int *wsum, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(0xffffffffu, pred);
    const int pre = __popc(b & ((1u << lane) - 1u));
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    if (warp == 0) {
        const int v = wsum[lane];
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        wsum[lane] = inc - v;
        if (lane == 31) *total = inc;
    }
    __syncthreads();
    const int res = wsum[warp] + pre;
    __syncthreads();
    return res;
}

// Control-volume masters and wall cells in cell order (deterministic sums).
__global__ void __launch_bounds__(1024) k_lists3(Grid3D g, Geo3D G, const int32_t *master, const uint16_t *flags,
                                                 int32_t *spec_list, int32_t *wall_list, int32_t *wslot,
                                                 int32_t *counts, int cap, int *err)
{
    __shared__ int wsum[32];
    __shared__ int tot;
    const long nc = (long)g.nx * g.ny * g.nz;
    int nspec = 0, nwall = 0;
    for (long base = 0; base < nc; base += blockDim.x) {
        const long q = base + threadIdx.x;
        bool sp = false, wl = false;
        if (q < nc) {
            sp = (flags[q] & kSpecial) && master[q] == (int32_t)q;
            wl = G.type[q] == DVM_CUT && G.sw[q] > 0;
        }
        const int ps = block_excl_scan3(sp, wsum, &tot) + nspec;
        __syncthreads();
        nspec += tot;
        __syncthreads();
        const int pw = block_excl_scan3(wl, wsum, &tot) + nwall;
        __syncthreads();
        nwall += tot;
        if (q < nc) {
            if (sp) { if (ps < cap) spec_list[ps] = (int32_t)q; else atomicExch(&err[kErrCapacity], 1); }
            wslot[q] = wl && pw < cap ? pw : -1;
            if (wl) { if (pw < cap) wall_list[pw] = (int32_t)q; else atomicExch(&err[kErrCapacity], 1); }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        counts[0] = nspec < cap ? nspec : cap;
        counts[1] = nwall < cap ? nwall : cap;
    }
}

__global__ void k_static3(Grid3D g, Geo3D G, int32_t *master, uint16_t *flags, uint8_t *hs, int32_t *wslot,
                          bool muscl)
{
    const long nc = (long)g.nx * g.ny * g.nz;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nc) {
        G.type[t] = DVM_GAS; G.cgas[t] = 1;
        G.sw[t] = 0; G.nwx[t] = 0; G.nwy[t] = 0; G.nwz[t] = 0;
        G.rwx[t] = 0; G.rwy[t] = 0; G.rwz[t] = 0;
        G.vol[t] = g.dx * g.dy * g.dz;
        master[t] = (int32_t)t;
        hs[t] = 0;
        wslot[t] = -1;
        flags[t] = kPlain | (muscl ? (uint16_t)(0x3F << kMaskShift3) : 0);
    }
    if (t < (long)(g.nx + 1) * g.ny * g.nz) G.ax[t] = g.dy * g.dz;
    if (t < (long)g.nx * (g.ny + 1) * g.nz) G.ay[t] = g.dx * g.dz;
    if (t < (long)g.nx * g.ny * (g.nz + 1)) G.az[t] = g.dx * g.dy;
    if (t < (long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1)) G.phi[t] = 1.0;
}

__global__ void k_clear_hs3(long n, uint8_t *hs)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) hs[t] = 0;
}

inline unsigned nblk3(long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t init_static_geometry3d(dvm_ctx *c)
{
    const Grid3D g = grid3d(c);
    const long n = (long)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    k_static3<<<nblk3(n, 256), 256, 0, c->stream>>>(g, c->geo3, c->master, c->flags3, c->hs, c->wslot,
                                                    c->scheme == DVM_MUSCL);
    return cudaGetLastError();
}

cudaError_t geometry3d(dvm_ctx *c)
{
    const Grid3D g = grid3d(c);
    const BodyParams b = body_params(c);
    const long nn = (long)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    k_nodes3<<<nblk3(nn, 256), 256, 0, c->stream>>>(g, b, c->geo3);
    const long nf = (long)(c->nx + 1) * c->ny * c->nz + (long)c->nx * (c->ny + 1) * c->nz +
                    (long)c->nx * c->ny * (c->nz + 1);
    k_faces3<<<nblk3(nf, 256), 256, 0, c->stream>>>(g, c->geo3, c->d_err);
    k_cells3<<<nblk3(c->nc, 256), 256, 0, c->stream>>>(g, c->geo3);
    return cudaGetLastError();
}

cudaError_t masters_flags3d(dvm_ctx *c)
{
    const Grid3D g = grid3d(c);
    k_clear_hs3<<<nblk3(c->nc, 256), 256, 0, c->stream>>>(c->nc, c->hs);
    k_masters3<<<nblk3(c->nc, 256), 256, 0, c->stream>>>(g, c->geo3, c->master, c->hs, c->d_err);
    k_flags3<<<nblk3(c->nc, 256), 256, 0, c->stream>>>(g, c->geo3, c->master, c->hs, c->flags3,
                                                        c->scheme == DVM_MUSCL);
    k_lists3<<<1, 1024, 0, c->stream>>>(g, c->geo3, c->master, c->flags3, c->spec_list, c->wall_list, c->wslot,
                                        c->counts, c->list_cap, c->d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return members3d(c);
}

}  // namespace dvm
