/*
 * Plain FP64 CPU oracle for the cut-cell discrete-velocity method of
 * Dechriste & Mieussens (arXiv:1503.04544).  TEST INFRASTRUCTURE ONLY: see
 * dvm_oracle.h.  Readings of passages that are silent, ambiguous or garbled
 * are marked "reading:" where they are applied.
 *
 * 2D path: reduced (f, g) BGK model (Sec. 2.2, Eq. BGKDD), explicit
 * first-order scheme on control volumes (Eq. ExSchemeDD) with upwind fluxes
 * (Eq. FluxDD), discrete diffuse reflection (Eq. BoundaryDDv), the 7-step
 * iteration of Sec. 3.3.5 and the Appendix A geometry.
 */
#include "dvm_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXWALK 8
static const double ORC_PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- physics */

/* Relaxation time scale, Sec. 5 (3D radiometer): tau = sqrt(pi)/2 *
 * (rho0/rho) * Kn L / sqrt(2 R T0).  With R = T0 = rho0 = 1 this returns
 * tau0 such that tau = tau0 / rho. */
double orc_tau0(const orc_cfg *c)
{
    return sqrt(ORC_PI) / 2.0 * c->Kn * c->Lref / sqrt(2.0);
}

static double axis_vmax(int n, double vmin, double vmax)
{
    double dv = (vmax - vmin) / n;
    double a = fabs(vmin), b = fabs(vmin + (n - 1) * dv);
    return a > b ? a : b;
}

/* Time step.  reading: the CFL condition of Sec. 3.4.1 is garbled; the step
 * is dt = CFL / sum_d (max_p |v_{p,d}| / dx_d). */
double orc_dt(const orc_cfg *c)
{
    if (c->dt > 0) return c->dt;
    double s = axis_vmax(c->nvx, c->vxmin, c->vxmax) / ((c->xmax - c->xmin) / c->nx)
             + axis_vmax(c->nvy, c->vymin, c->vymax) / ((c->ymax - c->ymin) / c->ny);
    if (c->dim == 3)
        s += axis_vmax(c->nvz, c->vzmin, c->vzmax) / ((c->zmax - c->zmin) / c->nz);
    return c->cfl / s;
}

/* Reduced 2D Maxwellian of Sec. 2.2 with R = 1. */
static double maxw2d(double rho, double ux, double uy, double T, double vx, double vy)
{
    double ax = vx - ux, ay = vy - uy;
    return rho / (2.0 * ORC_PI * T) * exp(-(ax * ax + ay * ay) / (2.0 * T));
}

/* 3D Maxwellian of Eq. MaxwellianTD with R = 1. */
static double maxw3d(double rho, double ux, double uy, double uz, double T,
                     double vx, double vy, double vz)
{
    double ax = vx - ux, ay = vy - uy, az = vz - uz;
    return rho / pow(2.0 * ORC_PI * T, 1.5) * exp(-(ax * ax + ay * ay + az * az) / (2.0 * T));
}

/* ---------------------------------------------------------------- geometry */

/* Level set of Appendix A: signed distance, negative inside the solid.
 * reading: the ellipse uses the first-order distance g/|grad g|. */
static double levelset2d(const orc_cfg *c, double ct, double st, double x, double y)
{
    double ddx = x - c->cx, ddy = y - c->cy;
    if (c->shape == ORC_SHAPE_CIRCLE) {
        return sqrt(ddx * ddx + ddy * ddy) - c->ra;
    } else if (c->shape == ORC_SHAPE_ELLIPSE) {
        double xr = ct * ddx + st * ddy;
        double yr = -st * ddx + ct * ddy;
        double a2 = c->ra * c->ra, b2 = c->rb * c->rb;
        double g = xr * xr / a2 + yr * yr / b2 - 1.0;
        double gx = 2.0 * xr / a2, gy = 2.0 * yr / b2;
        double nrm = sqrt(gx * gx + gy * gy);
        if (nrm > 0) return g / nrm;
        return -(c->ra < c->rb ? c->ra : c->rb);
    }
    return 1.0;
}

/* Clamp of Appendix A.1: phi := sign(phi) max(|phi|, 1e-10 dx), sign(0)=+. */
static double clamp_phi(double p, double dx)
{
    double eps = 1e-10 * dx;
    if (p >= 0) return p > eps ? p : eps;
    return -p > eps ? p : -eps;
}

/* Gas length of one Cartesian edge from its two nodal values (Appendix A.2).
 * reading: the printed formula counts a fully gaseous edge twice; the gas
 * part is taken once, measured in the edge's own frame from node 0. */
static double edge_gas_length(double p0, double p1, double h)
{
    if (p0 > 0 && p1 > 0) return h;
    if (p0 < 0 && p1 < 0) return 0.0;
    double o = h * (p0 / (p0 - p1));   /* crossing offset from node 0 */
    return p0 > 0 ? o : h - o;
}

int orc_geometry2d(const orc_cfg *c, double ct, double st, orc_geo2d *g)
{
    const int nx = c->nx, ny = c->ny;
    const double dx = (c->xmax - c->xmin) / nx, dy = (c->ymax - c->ymin) / ny;
    for (int b = 0; b <= ny; ++b)
        for (int a = 0; a <= nx; ++a) {
            double x = c->xmin + a * dx, y = c->ymin + b * dy;
            g->phi[b * (nx + 1) + a] = clamp_phi(levelset2d(c, ct, st, x, y), dx);
        }
#define PHI(a, b) g->phi[(b) * (nx + 1) + (a)]
    for (int j = 0; j < ny; ++j)
        for (int a = 0; a <= nx; ++a)
            g->lx[j * (nx + 1) + a] = edge_gas_length(PHI(a, j), PHI(a, j + 1), dy);
    for (int b = 0; b <= ny; ++b)
        for (int i = 0; i < nx; ++i)
            g->ly[b * nx + i] = edge_gas_length(PHI(i, b), PHI(i + 1, b), dx);
    int err = ORC_OK;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            double pmm = PHI(i, j), ppm = PHI(i + 1, j), ppp = PHI(i + 1, j + 1), pmp = PHI(i, j + 1);
            double m = fmin(fmin(pmm, ppm), fmin(ppp, pmp));
            double M = fmax(fmax(pmm, ppm), fmax(ppp, pmp));
            /* Eq. (ii): centre in gas from the mean of the 4 nodal values */
            g->cgas[k] = (0.25 * (((pmm + ppm) + ppp) + pmp)) > 0;
            g->lw[k] = 0; g->nwx[k] = 0; g->nwy[k] = 0;
            g->rwx[k] = 0; g->rwy[k] = 0;
            if (m > 0) {            /* gas cell: parameter table of Sec. 3.2.2 */
                g->type[k] = ORC_GAS;
                g->sbar[k] = dx * dy;
                continue;
            }
            if (M < 0) {
                g->type[k] = ORC_SOLID;
                g->sbar[k] = 0;
                continue;
            }
            g->type[k] = ORC_CUT;
            /* crossing points in the cell frame, edge order x-, x+, y-, y+ */
            double px[4], py[4];
            int nc = 0;
            if ((pmm > 0) != (pmp > 0)) { px[nc] = 0;  py[nc] = dy * (pmm / (pmm - pmp)); ++nc; }
            if ((ppm > 0) != (ppp > 0)) { px[nc] = dx; py[nc] = dy * (ppm / (ppm - ppp)); ++nc; }
            if ((pmm > 0) != (ppm > 0)) { px[nc] = dx * (pmm / (pmm - ppm)); py[nc] = 0;  ++nc; }
            if ((pmp > 0) != (ppp > 0)) { px[nc] = dx * (pmp / (pmp - ppp)); py[nc] = dy; ++nc; }
            if (nc != 2) { err = ORC_ERR_GEOMETRY; g->sbar[k] = 0; continue; }  /* saddle */
            double lxm = g->lx[j * (nx + 1) + i], lxp = g->lx[j * (nx + 1) + i + 1];
            double lym = g->ly[j * nx + i], lyp = g->ly[(j + 1) * nx + i];
            double ex = px[1] - px[0], ey = py[1] - py[0];
            double lw = sqrt(ex * ex + ey * ey);
            double rx = 0.5 * (px[0] + px[1]), ry = 0.5 * (py[0] + py[1]);
            /* reading: the Green-formula normal of Appendix A.2 is printed
             * with the opposite sign; n_w must point into the solid. */
            double nx_ = (lxm - lxp) / lw, ny_ = (lym - lyp) / lw;
            g->lw[k] = lw; g->nwx[k] = nx_; g->nwy[k] = ny_;
            g->rwx[k] = (c->xmin + i * dx) + rx;
            g->rwy[k] = (c->ymin + j * dy) + ry;
            /* Green formula of Appendix A.4 in the cell frame: the x- and y-
             * edges lie on the frame axes and contribute nothing. */
            g->sbar[k] = 0.5 * (lxp * dx + lyp * dy + lw * (rx * nx_ + ry * ny_));
        }
#undef PHI
    return err;
}

/* Master search, Eq. (fusion) of Appendix A.3.
 * reading: ties of the sequential tests resolve with the priority x+, x-,
 * y+, y-; a cell that is solid at t^n but not at t^{n+1} (appearing) walks
 * with its t^{n+1} edges; the stopping test is Eq. (ii) at t^n. */
int orc_masters2d(const orc_cfg *c, const orc_geo2d *gn, const orc_geo2d *gp,
                  int32_t *master)
{
    const int nx = c->nx, ny = c->ny;
    int err = ORC_OK;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            master[k] = -1;
            if (gn->type[k] == ORC_SOLID && gp->type[k] == ORC_SOLID) continue;
            int ci = i, cj = j, it = 0, ok = 0;
            while (it <= ORC_MAXWALK) {
                int q = cj * nx + ci;
                if (gn->cgas[q]) { ok = 1; break; }
                const orc_geo2d *g = gn->type[q] != ORC_SOLID ? gn : gp;
                double lxm = g->lx[cj * (nx + 1) + ci], lxp = g->lx[cj * (nx + 1) + ci + 1];
                double lym = g->ly[cj * nx + ci], lyp = g->ly[(cj + 1) * nx + ci];
                double M = fmax(fmax(lxp, lxm), fmax(lyp, lym));
                if (!(M > 0)) break;
                if (lxp == M) ci++;
                else if (lxm == M) ci--;
                else if (lyp == M) cj++;
                else cj--;
                if (ci < 0 || ci >= nx || cj < 0 || cj >= ny) break;
                ++it;
            }
            if (!ok) { err = ORC_ERR_GEOMETRY; continue; }
            master[k] = cj * nx + ci;
        }
    return err;
}

/* ------------------------------------------------------- initial condition */

int orc_init_maxwellian(const orc_cfg *c, const double *rho, const double *ux,
                        const double *uy, const double *uz, const double *T,
                        double *F)
{
    const int nv1 = c->nvx, nv2 = c->nvy, nv3 = c->dim == 3 ? c->nvz : 1;
    const int nv = nv1 * nv2 * nv3;
    const long ncell = (long)c->nx * c->ny * (c->dim == 3 ? c->nz : 1);
    const int ncomp = c->dim == 3 ? 1 : 2;
    const double dvx = (c->vxmax - c->vxmin) / nv1, dvy = (c->vymax - c->vymin) / nv2;
    const double dvz = c->dim == 3 ? (c->vzmax - c->vzmin) / nv3 : 0;
    for (long k = 0; k < ncell; ++k) {
        double *fk = F + k * ncomp * nv;
        for (int p3 = 0; p3 < nv3; ++p3)
            for (int p2 = 0; p2 < nv2; ++p2)
                for (int p1 = 0; p1 < nv1; ++p1) {
                    int p = (p3 * nv2 + p2) * nv1 + p1;
                    double vx = c->vxmin + p1 * dvx, vy = c->vymin + p2 * dvy;
                    if (rho[k] <= 0) {
                        for (int q = 0; q < ncomp; ++q) fk[q * nv + p] = 0;
                        continue;
                    }
                    if (c->dim == 3) {
                        double vz = c->vzmin + p3 * dvz;
                        fk[p] = maxw3d(rho[k], ux[k], uy[k], uz[k], T[k], vx, vy, vz);
                    } else {
                        double m = maxw2d(rho[k], ux[k], uy[k], T[k], vx, vy);
                        fk[p] = m;
                        fk[nv + p] = T[k] / 2.0 * m;       /* Eq. BGKDD: g = RT/2 M */
                    }
                }
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- moments */

/* Discrete moments, Eq. MacroscopicDDv (2D) and Eq. MacroscopicTD summed
 * over the grid (3D); T from E = rho|u|^2/2 + 3/2 rho R T (Sec. 2.1). */
static int cell_moments(const orc_cfg *c, const double *fk, double *rho,
                        double *u, double *T)
{
    const int nv1 = c->nvx, nv2 = c->nvy, nv3 = c->dim == 3 ? c->nvz : 1;
    const int nv = nv1 * nv2 * nv3;
    const double dvx = (c->vxmax - c->vxmin) / nv1, dvy = (c->vymax - c->vymin) / nv2;
    const double dvz = c->dim == 3 ? (c->vzmax - c->vzmin) / nv3 : 1.0;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, sE = 0;
    for (int p3 = 0; p3 < nv3; ++p3)
        for (int p2 = 0; p2 < nv2; ++p2)
            for (int p1 = 0; p1 < nv1; ++p1) {
                int p = (p3 * nv2 + p2) * nv1 + p1;
                double vx = c->vxmin + p1 * dvx, vy = c->vymin + p2 * dvy;
                double vz = c->dim == 3 ? c->vzmin + p3 * dvz : 0.0;
                double f = fk[p];
                s0 += f; s1 += vx * f; s2 += vy * f; s3 += vz * f;
                if (c->dim == 3) sE += 0.5 * (vx * vx + vy * vy + vz * vz) * f;
                else sE += 0.5 * (vx * vx + vy * vy) * f + fk[nv + p];
            }
    double dv = dvx * dvy * (c->dim == 3 ? dvz : 1.0);
    *rho = s0 * dv;
    if (!(*rho > 0)) { u[0] = u[1] = u[2] = 0; *T = 0; return ORC_ERR_NONPHYSICAL; }
    u[0] = s1 * dv / *rho;
    u[1] = s2 * dv / *rho;
    u[2] = s3 * dv / *rho;
    double E = sE * dv;
    *T = (2.0 * E / *rho - (u[0] * u[0] + u[1] * u[1] + u[2] * u[2])) / 3.0;
    return *T > 0 ? ORC_OK : ORC_ERR_NONPHYSICAL;
}

int orc_moments(const orc_cfg *c, const double *F, double *rho, double *ux,
                double *uy, double *uz, double *T)
{
    const int nv = c->nvx * c->nvy * (c->dim == 3 ? c->nvz : 1);
    const long ncell = (long)c->nx * c->ny * (c->dim == 3 ? c->nz : 1);
    const int ncomp = c->dim == 3 ? 1 : 2;
    for (long k = 0; k < ncell; ++k) {
        double u[3];
        cell_moments(c, F + k * ncomp * nv, &rho[k], u, &T[k]);
        ux[k] = u[0]; uy[k] = u[1];
        if (uz) uz[k] = u[2];
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- 2D step */

typedef struct {
    const orc_cfg *c;
    int nx, ny, nv, nv1, nv2;
    double dx, dy, dvx, dvy, dt;
    double *ghost[4];         /* Maxwellian ghost states per boundary cell */
    const double *F;          /* virtual-cell values after fusion          */
    const orc_geo2d *g;       /* geometry at t^n                            */
} orc_ctx2d;

/* Value of a virtual cell, extended by the domain boundary conditions.
 * reading: periodic wrap; Maxwellian sides hold the prescribed state in
 * every ghost layer; zero-gradient copies the boundary cell. */
static double fval2d(const orc_ctx2d *x, int i, int j, int comp, int p)
{
    const orc_cfg *c = x->c;
    if (i < 0) {
        if (c->bc[0] == ORC_BC_PERIODIC) i += x->nx;
        else if (c->bc[0] == ORC_BC_MAXWELLIAN) return x->ghost[0][((long)j * 2 + comp) * x->nv + p];
        else i = 0;
    } else if (i >= x->nx) {
        if (c->bc[1] == ORC_BC_PERIODIC) i -= x->nx;
        else if (c->bc[1] == ORC_BC_MAXWELLIAN) return x->ghost[1][((long)j * 2 + comp) * x->nv + p];
        else i = x->nx - 1;
    }
    if (j < 0) {
        if (c->bc[2] == ORC_BC_PERIODIC) j += x->ny;
        else if (c->bc[2] == ORC_BC_MAXWELLIAN) return x->ghost[2][((long)i * 2 + comp) * x->nv + p];
        else j = 0;
    } else if (j >= x->ny) {
        if (c->bc[3] == ORC_BC_PERIODIC) j -= x->ny;
        else if (c->bc[3] == ORC_BC_MAXWELLIAN) return x->ghost[3][((long)i * 2 + comp) * x->nv + p];
        else j = x->ny - 1;
    }
    return x->F[(((long)j * x->nx + i) * 2 + comp) * x->nv + p];
}

/* Gas test used by the limiter fallback; ghost cells count as gas. */
static int isgas2d(const orc_ctx2d *x, int i, int j)
{
    const orc_cfg *c = x->c;
    if (i < 0) { if (c->bc[0] != ORC_BC_PERIODIC) return 1; i += x->nx; }
    else if (i >= x->nx) { if (c->bc[1] != ORC_BC_PERIODIC) return 1; i -= x->nx; }
    if (j < 0) { if (c->bc[2] != ORC_BC_PERIODIC) return 1; j += x->ny; }
    else if (j >= x->ny) { if (c->bc[3] != ORC_BC_PERIODIC) return 1; j -= x->ny; }
    return x->g->type[j * x->nx + i] == ORC_GAS;
}

/* minmod(a, b): 0 unless a and b have the same strict sign, else the one of
 * smaller magnitude. */
static double minmod(double a, double b)
{
    if (a > 0 && b > 0) return a < b ? a : b;
    if (a < 0 && b < 0) return a > b ? a : b;
    return 0.0;
}

/* Numerical flux across one Cartesian edge of length L with the cell A on
 * its minus side and B on its plus side (Eq. FluxDD).
 * reading (MUSCL): the paper leaves the second-order scheme to future work;
 * the limited flux is the one-step van Leer form
 *   v>0: f_A + (1-nu)/2 minmod(f_B - f_A, f_A - f_AA)
 *   v<0: f_B - (1-nu)/2 minmod(f_BB - f_B, f_B - f_A),  nu = |v| dt/dx,
 * used only when AA, A, B, BB are all gas cells. */
static double face_flux(double L, double v, double nu, double fAA, double fA,
                        double fB, double fBB, int muscl)
{
    if (!muscl) return L * (fmin(v, 0.0) * fB + fmax(v, 0.0) * fA);
    double fr;
    if (v > 0) fr = fA + 0.5 * (1.0 - nu) * minmod(fB - fA, fA - fAA);
    else if (v < 0) fr = fB - 0.5 * (1.0 - nu) * minmod(fBB - fB, fB - fA);
    else return 0.0;
    return L * (v * fr);
}

/* Sector of a wall point for piecewise wall temperatures: the first s with
 * cross(d_s, r) >= 0 and cross(d_{s+1}, r) < 0. */
static int wall_sector(const orc_cfg *c, double rx, double ry)
{
    for (int s = 0; s < c->nseg; ++s) {
        int t = (s + 1) % c->nseg;
        double a = c->seg_dir[2 * s] * ry - c->seg_dir[2 * s + 1] * rx;
        double b = c->seg_dir[2 * t] * ry - c->seg_dir[2 * t + 1] * rx;
        if (a >= 0 && b < 0) return s;
    }
    return 0;
}

static void make_ghosts2d(orc_ctx2d *x)
{
    const orc_cfg *c = x->c;
    for (int s = 0; s < 4; ++s) {
        x->ghost[s] = NULL;
        if (c->bc[s] != ORC_BC_MAXWELLIAN) continue;
        int n = s < 2 ? x->ny : x->nx;
        x->ghost[s] = malloc(sizeof(double) * (size_t)n * 2 * x->nv);
        for (int q = 0; q < n; ++q) {
            const double *st = c->bc_state[s] + 5 * q;   /* rho ux uy uz T */
            for (int p2 = 0; p2 < x->nv2; ++p2)
                for (int p1 = 0; p1 < x->nv1; ++p1) {
                    int p = p2 * x->nv1 + p1;
                    double vx = c->vxmin + p1 * x->dvx, vy = c->vymin + p2 * x->dvy;
                    double m = maxw2d(st[0], st[1], st[2], st[4], vx, vy);
                    x->ghost[s][((long)q * 2 + 0) * x->nv + p] = m;
                    x->ghost[s][((long)q * 2 + 1) * x->nv + p] = st[4] / 2.0 * m;
                }
        }
    }
}

static void alloc_geo2d(orc_geo2d *g, int nx, int ny)
{
    long nc = (long)nx * ny;
    g->phi = malloc(sizeof(double) * (nx + 1) * (ny + 1));
    g->type = malloc(nc); g->cgas = malloc(nc);
    g->lx = malloc(sizeof(double) * (nx + 1) * ny);
    g->ly = malloc(sizeof(double) * nx * (ny + 1));
    g->lw = malloc(sizeof(double) * nc);
    g->nwx = malloc(sizeof(double) * nc); g->nwy = malloc(sizeof(double) * nc);
    g->rwx = malloc(sizeof(double) * nc); g->rwy = malloc(sizeof(double) * nc);
    g->sbar = malloc(sizeof(double) * nc);
}

static void free_geo2d(orc_geo2d *g)
{
    free(g->phi); free(g->type); free(g->cgas); free(g->lx); free(g->ly);
    free(g->lw); free(g->nwx); free(g->nwy); free(g->rwx); free(g->rwy); free(g->sbar);
}

double orc_mass2d(const orc_cfg *c, const double *F)
{
    const int nx = c->nx, ny = c->ny, nv = c->nvx * c->nvy;
    const double dv = (c->vxmax - c->vxmin) / c->nvx * ((c->vymax - c->vymin) / c->nvy);
    orc_geo2d g;
    alloc_geo2d(&g, nx, ny);
    orc_geometry2d(c, cos(c->theta), sin(c->theta), &g);
    /* Eq. def-masse with every member of a control volume holding the
     * control-volume value: M = sum_cells sbar sum_p f dv. */
    double M = 0;
    for (long k = 0; k < (long)nx * ny; ++k) {
        double s = 0;
        for (int p = 0; p < nv; ++p) s += F[k * 2 * nv + p];
        M += g.sbar[k] * (s * dv);
    }
    free_geo2d(&g);
    return M;
}

int orc_run2d(const orc_cfg *c, double *F, int nsteps, orc_hist *h,
              double *theta_out, double *omega_out)
{
    if (c->dim != 2 || c->nx < 2 || c->ny < 1 || c->nvx < 1 || c->nvy < 1) return ORC_ERR_ARG;
    orc_ctx2d X;
    X.c = c; X.nx = c->nx; X.ny = c->ny; X.nv1 = c->nvx; X.nv2 = c->nvy;
    X.nv = X.nv1 * X.nv2;
    X.dx = (c->xmax - c->xmin) / c->nx; X.dy = (c->ymax - c->ymin) / c->ny;
    X.dvx = (c->vxmax - c->vxmin) / c->nvx; X.dvy = (c->vymax - c->vymin) / c->nvy;
    X.dt = orc_dt(c);
    const int nx = X.nx, ny = X.ny, nv = X.nv;
    const long nc = (long)nx * ny;
    const double dt = X.dt, dx = X.dx, dy = X.dy, dv = X.dvx * X.dvy;
    const double tau0 = orc_tau0(c);
    const int moving = c->movable && c->shape != ORC_SHAPE_NONE;
    make_ghosts2d(&X);

    orc_geo2d ga, gb, *gn = &ga, *gp = &gb;
    alloc_geo2d(&ga, nx, ny); alloc_geo2d(&gb, nx, ny);
    double theta = c->theta, omega = c->omega;
    int err = orc_geometry2d(c, cos(theta), sin(theta), gn);
    int32_t *master = malloc(sizeof(int32_t) * nc);
    int32_t *mstart = malloc(sizeof(int32_t) * (nc + 1));
    int32_t *mlist = malloc(sizeof(int32_t) * nc);
    int32_t *cnt = malloc(sizeof(int32_t) * nc);
    double *Sn = malloc(sizeof(double) * nc), *Sp = malloc(sizeof(double) * nc);
    double *mrho = malloc(sizeof(double) * nc), *mux = malloc(sizeof(double) * nc);
    double *muy = malloc(sizeof(double) * nc), *mT = malloc(sizeof(double) * nc);
    double *wphi = malloc(sizeof(double) * nc), *wux = malloc(sizeof(double) * nc);
    double *wuy = malloc(sizeof(double) * nc), *wT = malloc(sizeof(double) * nc);
    double *Fnew = malloc(sizeof(double) * nc * 2 * nv);
    double *vx = malloc(sizeof(double) * X.nv1), *vy = malloc(sizeof(double) * X.nv2);
    for (int p1 = 0; p1 < X.nv1; ++p1) vx[p1] = c->vxmin + p1 * X.dvx;
    for (int p2 = 0; p2 < X.nv2; ++p2) vy[p2] = c->vymin + p2 * X.dvy;

    for (int step = 0; step < nsteps && err == ORC_OK; ++step) {
        /* Step 1: body position at t^{n+1} (Eq. motionDD_posit). */
        double theta1 = moving ? theta + dt * omega : theta;
        /* Step 3 geometry is needed by the master search of appearing cells. */
        if (moving) err = orc_geometry2d(c, cos(theta1), sin(theta1), gp);
        else gp = gn;
        if (err) break;
        /* Step 2: control volumes sigma^n and fusion (Eq. FusionDD). */
        err = orc_masters2d(c, gn, gp, master);
        if (err) break;
        for (long k = 0; k < nc; ++k) { cnt[k] = 0; Sn[k] = 0; Sp[k] = 0; }
        for (long k = 0; k < nc; ++k)
            if (master[k] >= 0) {
                cnt[master[k]]++;
                Sn[master[k]] += gn->sbar[k];
                Sp[master[k]] += gp->sbar[k];
            }
        mstart[0] = 0;
        for (long k = 0; k < nc; ++k) mstart[k + 1] = mstart[k] + cnt[k];
        for (long k = 0; k < nc; ++k) cnt[k] = 0;
        for (long k = 0; k < nc; ++k)
            if (master[k] >= 0) { int m = master[k]; mlist[mstart[m] + cnt[m]++] = (int32_t)k; }
        #pragma omp parallel for schedule(dynamic, 64)
        for (long m = 0; m < nc; ++m) {
            int nm = mstart[m + 1] - mstart[m];
            if (nm <= 1) continue;
            for (int comp = 0; comp < 2; ++comp)
                for (int p = 0; p < nv; ++p) {
                    double s = 0;
                    for (int q = mstart[m]; q < mstart[m + 1]; ++q) {
                        long kk = mlist[q];
                        s += gn->sbar[kk] * F[(kk * 2 + comp) * nv + p];
                    }
                    double fcv = s / Sn[m];
                    for (int q = mstart[m]; q < mstart[m + 1]; ++q)
                        F[((long)mlist[q] * 2 + comp) * nv + p] = fcv;   /* reading: c14 */
                }
        }
        X.F = F; X.g = gn;
        /* moments of f_CV^n and the BGK equilibrium inputs (Eq. BGKDD) */
        int nonphys = 0;
        #pragma omp parallel for reduction(|:nonphys)
        for (long m = 0; m < nc; ++m) {
            if (mstart[m + 1] - mstart[m] == 0) continue;
            double u[3], r, T;
            if (cell_moments(c, F + m * 2 * nv, &r, u, &T)) nonphys = 1;
            mrho[m] = r; mux[m] = u[0]; muy[m] = u[1]; mT[m] = T;
        }
        if (nonphys) { err = ORC_ERR_NONPHYSICAL; break; }
        /* Step 4: wall density phi (Eq. BoundaryDDv) at every wall edge;
         * Step 5: stress (Eq. StressTensorDD), force and torque
         * (Eqs. eq-force, eq-torque). */
        double Fx = 0, Fy = 0, Tq = 0;
        for (long k = 0; k < nc; ++k) {
            if (gn->type[k] != ORC_CUT || !(gn->lw[k] > 0)) continue;
            double rx = gn->rwx[k] - c->cx, ry = gn->rwy[k] - c->cy;
            double uwx = c->vbx - ry * omega, uwy = c->vby + rx * omega;   /* Eq. uwDD */
            double Tw = c->nseg > 0 ? c->Tw_seg[wall_sector(c, rx, ry)] : c->Tw;
            double nwx = gn->nwx[k], nwy = gn->nwy[k];
            const double *fk = F + k * 2 * nv;
            double num = 0, den = 0;
            for (int p2 = 0; p2 < X.nv2; ++p2)
                for (int p1 = 0; p1 < X.nv1; ++p1) {
                    int p = p2 * X.nv1 + p1;
                    double cp = (vx[p1] - uwx) * nwx + (vy[p2] - uwy) * nwy;
                    if (cp > 0) num += cp * fk[p] * dv;
                    else if (cp < 0) den += cp * maxw2d(1.0, uwx, uwy, Tw, vx[p1], vy[p2]) * dv;
                }
            double phi = -num / den;
            double sxx = 0, sxy = 0, syy = 0;
            for (int p2 = 0; p2 < X.nv2; ++p2)
                for (int p1 = 0; p1 < X.nv1; ++p1) {
                    int p = p2 * X.nv1 + p1;
                    double ax = vx[p1] - uwx, ay = vy[p2] - uwy;
                    double cp = ax * nwx + ay * nwy;
                    double fv;
                    if (cp < 0) fv = phi * maxw2d(1.0, uwx, uwy, Tw, vx[p1], vy[p2]);
                    else if (cp > 0) fv = fk[p];
                    else continue;
                    sxx += ax * ax * fv * dv; sxy += ax * ay * fv * dv; syy += ay * ay * fv * dv;
                }
            double fkx = (sxx * nwx + sxy * nwy) * gn->lw[k];
            double fky = (sxy * nwx + syy * nwy) * gn->lw[k];
            Fx += fkx; Fy += fky;
            Tq += rx * fky - ry * fkx;
            wphi[k] = phi; wux[k] = uwx; wuy[k] = uwy; wT[k] = Tw;
        }
        double omega1 = moving ? omega + dt * Tq / c->inertia : omega;   /* Eq. motionDD_vit */
        /* Step 6: explicit scheme (Eq. ExSchemeDD) on every control volume. */
        int badcv = 0;
        #pragma omp parallel reduction(|:badcv)
        {
            double *R = malloc(sizeof(double) * 2 * nv);
            #pragma omp for schedule(dynamic, 16)
            for (long m = 0; m < nc; ++m) {
                if (mstart[m + 1] - mstart[m] == 0) continue;
                if (!(Sp[m] > 0)) { badcv = 1; continue; }
                for (int q = 0; q < 2 * nv; ++q) R[q] = 0;
                for (int q = mstart[m]; q < mstart[m + 1]; ++q) {
                    long k = mlist[q];
                    if (gn->type[k] == ORC_SOLID) continue;   /* appearing cell: no edges at t^n */
                    int i = (int)(k % nx), j = (int)(k / nx);
                    int mus = c->scheme == ORC_MUSCL;
                    int mxp = mus && isgas2d(&X, i - 1, j) && isgas2d(&X, i, j) &&
                              isgas2d(&X, i + 1, j) && isgas2d(&X, i + 2, j);
                    int mxm = mus && isgas2d(&X, i - 2, j) && isgas2d(&X, i - 1, j) &&
                              isgas2d(&X, i, j) && isgas2d(&X, i + 1, j);
                    int myp = mus && isgas2d(&X, i, j - 1) && isgas2d(&X, i, j) &&
                              isgas2d(&X, i, j + 1) && isgas2d(&X, i, j + 2);
                    int mym = mus && isgas2d(&X, i, j - 2) && isgas2d(&X, i, j - 1) &&
                              isgas2d(&X, i, j) && isgas2d(&X, i, j + 1);
                    double lxp = gn->lx[j * (nx + 1) + i + 1], lxm = gn->lx[j * (nx + 1) + i];
                    double lyp = gn->ly[(j + 1) * nx + i], lym = gn->ly[j * nx + i];
                    int wall = gn->type[k] == ORC_CUT && gn->lw[k] > 0;
                    for (int comp = 0; comp < 2; ++comp)
                        for (int p2 = 0; p2 < X.nv2; ++p2)
                            for (int p1 = 0; p1 < X.nv1; ++p1) {
                                int p = p2 * X.nv1 + p1;
                                double v1 = vx[p1], v2 = vy[p2];
                                double nu1 = fabs(v1) * dt / dx, nu2 = fabs(v2) * dt / dy;
                                double fxp = face_flux(lxp, v1, nu1,
                                    fval2d(&X, i - 1, j, comp, p), fval2d(&X, i, j, comp, p),
                                    fval2d(&X, i + 1, j, comp, p), fval2d(&X, i + 2, j, comp, p), mxp);
                                double fxm = face_flux(lxm, v1, nu1,
                                    fval2d(&X, i - 2, j, comp, p), fval2d(&X, i - 1, j, comp, p),
                                    fval2d(&X, i, j, comp, p), fval2d(&X, i + 1, j, comp, p), mxm);
                                double fyp = face_flux(lyp, v2, nu2,
                                    fval2d(&X, i, j - 1, comp, p), fval2d(&X, i, j, comp, p),
                                    fval2d(&X, i, j + 1, comp, p), fval2d(&X, i, j + 2, comp, p), myp);
                                double fym = face_flux(lym, v2, nu2,
                                    fval2d(&X, i, j - 2, comp, p), fval2d(&X, i, j - 1, comp, p),
                                    fval2d(&X, i, j, comp, p), fval2d(&X, i, j + 1, comp, p), mym);
                                double fw = 0;
                                if (wall) {
                                    double ax = v1 - wux[k], ay = v2 - wuy[k];
                                    double cp = ax * gn->nwx[k] + ay * gn->nwy[k];
                                    double mw = maxw2d(1.0, wux[k], wuy[k], wT[k], v1, v2);
                                    double fwall = comp == 0 ? wphi[k] * mw
                                                             : wphi[k] * (wT[k] / 2.0 * mw);  /* reading: c13 */
                                    fw = gn->lw[k] * (fmin(cp, 0.0) * fwall +
                                                      fmax(cp, 0.0) * F[(k * 2 + comp) * nv + p]);
                                }
                                R[comp * nv + p] += (fxp - fxm) + (fyp - fym) + fw;
                            }
                }
                double tau = tau0 / mrho[m];
                double a = Sn[m] / Sp[m], b = dt / Sp[m], r = dt / tau;
                for (int comp = 0; comp < 2; ++comp)
                    for (int p2 = 0; p2 < X.nv2; ++p2)
                        for (int p1 = 0; p1 < X.nv1; ++p1) {
                            int p = p2 * X.nv1 + p1;
                            double fcv = F[(m * 2 + comp) * nv + p];
                            double feq = maxw2d(mrho[m], mux[m], muy[m], mT[m], vx[p1], vy[p2]);
                            if (comp == 1) feq = mT[m] / 2.0 * feq;
                            Fnew[(m * 2 + comp) * nv + p] = a * fcv - b * R[comp * nv + p] + a * r * (feq - fcv);
                        }
            }
            free(R);
        }
        if (badcv) { err = ORC_ERR_GEOMETRY; break; }
        /* Step 7: distribution (Eq. UpdateDD).  reading: cells that are
         * solid at t^{n+1} hold zero. */
        #pragma omp parallel for
        for (long k = 0; k < nc; ++k) {
            int m = master[k];
            double *dst = F + k * 2 * nv;
            if (m < 0 || gp->type[k] == ORC_SOLID) { memset(dst, 0, sizeof(double) * 2 * nv); continue; }
            memcpy(dst, Fnew + (long)m * 2 * nv, sizeof(double) * 2 * nv);
        }
        if (h) {
            if (h->Fx) h->Fx[step] = Fx;
            if (h->Fy) h->Fy[step] = Fy;
            if (h->torque) h->torque[step] = Tq;
            if (h->theta) h->theta[step] = theta1;
            if (h->omega) h->omega[step] = omega1;
            if (h->mass) {
                double M = 0;
                for (long k = 0; k < nc; ++k) {
                    double s = 0;
                    for (int p = 0; p < nv; ++p) s += F[k * 2 * nv + p];
                    M += gp->sbar[k] * (s * dv);
                }
                h->mass[step] = M;
            }
        }
        theta = theta1; omega = omega1;
        if (moving) { orc_geo2d *t = gn; gn = gp; gp = t; }
    }
    if (theta_out) *theta_out = theta;
    if (omega_out) *omega_out = omega;
    free_geo2d(&ga); free_geo2d(&gb);
    free(master); free(mstart); free(mlist); free(cnt); free(Sn); free(Sp);
    free(mrho); free(mux); free(muy); free(mT);
    free(wphi); free(wux); free(wuy); free(wT); free(Fnew); free(vx); free(vy);
    for (int s = 0; s < 4; ++s) free(X.ghost[s]);
    return err;
}
