/*
 * Plain FP64 CPU oracle for the cut-cell discrete-velocity method of
 * Dechriste & Mieussens (arXiv:1503.04544).  TEST INFRASTRUCTURE ONLY: see
 * dvm_oracle.h.  Readings of passages that are silent, ambiguous or garbled
 * are marked "reading:" where they are applied.
 *
 * 2D path: reduced (f, g) BGK model (Sec. 2.2, Eq. BGKDD), explicit
 * first-order scheme on control volumes (Eq. ExSchemeDD) with upwind fluxes
 * (Eq. FluxDD), discrete diffuse reflection (Eq. BoundaryDDv), the 7-step
 * iteration of Sec. 3.3.5 and the Appendix A geometry.  With
 * time_scheme = ORC_IMEX the update is the first-order semi-implicit scheme
 * (Eq. ImpSchemeDD) instead, in 2D and 3D.  With model = ORC_SHAKHOV the
 * explicit scheme relaxes towards the Shakhov equilibrium (Eq. ShakhovDD in
 * 2D, the form of Sec. 2.1 in 3D) with the heat flux of the control volume.
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
 * reading: the ellipse uses the first-order distance g/|grad g|; a box
 * container the least of the four signed distances to its sides. */
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
    } else if (c->shape == ORC_SHAPE_DISK_CONTAINER) {
        /* the gas inside the disk */
        return c->ra - sqrt(ddx * ddx + ddy * ddy);
    } else if (c->shape == ORC_SHAPE_BOX_CONTAINER) {
        /* the gas inside the box: the least distance to its four sides */
        double x0 = c->cx - c->ra, x1 = c->cx + c->ra, y0 = c->cy - c->rb, y1 = c->cy + c->rb;
        return fmin(fmin(x - x0, x1 - x), fmin(y - y0, y1 - y));
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

/* ------------------------------------------- conservative discrete equilibrium */

/* Solve A x = b (n <= 5) by Gaussian elimination with partial pivoting;
 * A and b are overwritten.  Returns 0 on success, 1 for a singular matrix. */
static int solve_small(int n, double A[5][5], double *b, double *x)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i][k]) > fabs(A[piv][k])) piv = i;
        if (!(fabs(A[piv][k]) > 0)) return 1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) { double t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t; }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double l = A[i][k] / A[k][k];
            for (int j = k; j < n; ++j) A[i][j] -= l * A[k][j];
            b[i] -= l * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return 0;
}

/* Conservative equilibrium parameters (Sec. 3.1, the paragraph after Eq.
 * MacroscopicDDv): the (rho, u, T) put into the equilibrium are not the direct
 * moments of the state but the ones whose discrete equilibrium has the same
 * discrete moments as the state, so that the collision term conserves mass,
 * momentum and energy exactly on the velocity grid.  With theta = (rho, u, T)
 * and the equilibrium E_p(theta) = M[rho, u, T](v_p) (2D: and T/2 M for g),
 * the equations are, for phi = 1, v_d and the energy weight,
 *   sum_p phi(v_p) E_p(theta) dv = sum_p phi(v_p) f_p dv,
 * 2D energy: sum (|v|^2/2 + T/2) M dv = sum (|v|^2/2 f + g) dv;
 * 3D energy: sum |v|^2/2 M dv = sum |v|^2/2 F dv.
 * The root does not depend on the variant of Newton's method that finds it;
 * this one takes plain Newton steps from the direct moments, with the exact
 * Jacobian summed over the whole grid:
 *   dM/drho = M / rho, dM/du_d = M (v_d - u_d) / T,
 *   dM/dT = M (|v - u|^2 / (2 T^2) - dim / (2 T)),
 * and in 2D the energy row also gets d(T/2 M)/dT = T/2 dM/dT + M/2.  Stops
 * when the largest step, relative to rho, sqrt(T) (velocities) and T, is
 * below 1e-13 (one more step then follows from the quadratic convergence
 * already taken), at most 50 steps. */
static int conservative_params(const orc_cfg *c, const double *fk, double *rho, double *u, double *T,
                               int *iters)
{
    const int D = c->dim, n = D + 2;
    const int nv1 = c->nvx, nv2 = c->nvy, nv3 = D == 3 ? c->nvz : 1;
    const int nv = nv1 * nv2 * nv3;
    const double dvx = (c->vxmax - c->vxmin) / nv1, dvy = (c->vymax - c->vymin) / nv2;
    const double dvz = D == 3 ? (c->vzmax - c->vzmin) / nv3 : 1.0;
    const double dv = dvx * dvy * dvz;
    /* moments of the state */
    double tgt[5] = {0, 0, 0, 0, 0};
    for (int p3 = 0; p3 < nv3; ++p3)
        for (int p2 = 0; p2 < nv2; ++p2)
            for (int p1 = 0; p1 < nv1; ++p1) {
                int p = (p3 * nv2 + p2) * nv1 + p1;
                double v[3] = {c->vxmin + p1 * dvx, c->vymin + p2 * dvy, D == 3 ? c->vzmin + p3 * dvz : 0.0};
                double f = fk[p];
                tgt[0] += f * dv;
                for (int d = 0; d < D; ++d) tgt[1 + d] += v[d] * f * dv;
                double e = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * f;
                if (D == 2) e += fk[nv + p];
                tgt[n - 1] += e * dv;
            }
    int rc = cell_moments(c, fk, rho, u, T);
    if (rc) return rc;
    double th[5];
    th[0] = *rho;
    for (int d = 0; d < D; ++d) th[1 + d] = u[d];
    th[n - 1] = *T;
    int it = 0, done = 0;
    for (it = 0; it < 50 && !done; ++it) {
        double m[5] = {0, 0, 0, 0, 0}, J[5][5];
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) J[i][j] = 0;
        const double r = th[0], Tt = th[n - 1];
        if (!(r > 0) || !(Tt > 0)) return ORC_ERR_NONPHYSICAL;
        double uu[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) uu[d] = th[1 + d];
        for (int p3 = 0; p3 < nv3; ++p3)
            for (int p2 = 0; p2 < nv2; ++p2)
                for (int p1 = 0; p1 < nv1; ++p1) {
                    double v[3] = {c->vxmin + p1 * dvx, c->vymin + p2 * dvy, D == 3 ? c->vzmin + p3 * dvz : 0.0};
                    double M = D == 3 ? maxw3d(r, uu[0], uu[1], uu[2], Tt, v[0], v[1], v[2])
                                      : maxw2d(r, uu[0], uu[1], Tt, v[0], v[1]);
                    double c2 = 0;
                    for (int d = 0; d < D; ++d) c2 += (v[d] - uu[d]) * (v[d] - uu[d]);
                    double dM[5];
                    dM[0] = M / r;
                    for (int d = 0; d < D; ++d) dM[1 + d] = M * (v[d] - uu[d]) / Tt;
                    dM[n - 1] = M * (c2 / (2.0 * Tt * Tt) - D / (2.0 * Tt));
                    double half_v2 = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                    double phi[5];
                    phi[0] = 1.0;
                    for (int d = 0; d < D; ++d) phi[1 + d] = v[d];
                    phi[n - 1] = D == 2 ? half_v2 + Tt / 2.0 : half_v2;
                    for (int i = 0; i < n; ++i) {
                        m[i] += phi[i] * M * dv;
                        for (int j = 0; j < n; ++j) J[i][j] += phi[i] * dM[j] * dv;
                    }
                    if (D == 2) J[n - 1][n - 1] += 0.5 * M * dv;   /* d(T/2)/dT times M, from g */
                }
        double res[5], step[5];
        for (int i = 0; i < n; ++i) res[i] = tgt[i] - m[i];
        if (solve_small(n, J, res, step)) return ORC_ERR_NONPHYSICAL;
        double big = fabs(step[0]) / th[0];
        for (int d = 0; d < D; ++d) big = fmax(big, fabs(step[1 + d]) / sqrt(Tt));
        big = fmax(big, fabs(step[n - 1]) / Tt);
        for (int i = 0; i < n; ++i) th[i] += step[i];
        if (big < 1e-13) done = 1;
    }
    if (iters) *iters = it;
    if (!done) return ORC_ERR_NONPHYSICAL;
    *rho = th[0];
    for (int d = 0; d < 3; ++d) u[d] = d < D ? th[1 + d] : 0.0;
    *T = th[n - 1];
    return (*rho > 0 && *T > 0) ? ORC_OK : ORC_ERR_NONPHYSICAL;
}

/* Equilibrium parameters of one cell: the direct moments (Eq.
 * MacroscopicDDv), or the conservative ones of Sec. 3.1. */
static int equilibrium_params(const orc_cfg *c, const double *fk, double *rho, double *u, double *T)
{
    if (c->conservative) return conservative_params(c, fk, rho, u, T, NULL);
    return cell_moments(c, fk, rho, u, T);
}

int orc_equilibrium_params(const orc_cfg *c, const double *fk, double *out, int *iters)
{
    double rho, u[3] = {0, 0, 0}, T;
    int rc;
    if (iters) *iters = 0;
    if (c->conservative) rc = conservative_params(c, fk, &rho, u, &T, iters);
    else rc = cell_moments(c, fk, &rho, u, &T);
    out[0] = rho; out[1] = u[0]; out[2] = u[1]; out[3] = u[2]; out[4] = T;
    return rc;
}

/* ---------------------------------------------------------- collision model */

/* Heat flux of one cell's state about its velocity u (R = 1): reduced 2D
 * q = sum (v - u)(|v - u|^2/2 f + g) dv (Eq. MacroscopicDDv), 3D
 * q = sum (v - u)|v - u|^2/2 F dv (the heat flux of Sec. 2.1). */
static void cell_heat_flux(const orc_cfg *c, const double *fk, const double *u, double *q)
{
    const int nv1 = c->nvx, nv2 = c->nvy, nv3 = c->dim == 3 ? c->nvz : 1;
    const int nv = nv1 * nv2 * nv3;
    const double dvx = (c->vxmax - c->vxmin) / nv1, dvy = (c->vymax - c->vymin) / nv2;
    const double dvz = c->dim == 3 ? (c->vzmax - c->vzmin) / nv3 : 1.0;
    double s[3] = {0, 0, 0};
    for (int p3 = 0; p3 < nv3; ++p3)
        for (int p2 = 0; p2 < nv2; ++p2)
            for (int p1 = 0; p1 < nv1; ++p1) {
                int p = (p3 * nv2 + p2) * nv1 + p1;
                double ax = c->vxmin + p1 * dvx - u[0], ay = c->vymin + p2 * dvy - u[1];
                double az = c->dim == 3 ? c->vzmin + p3 * dvz - u[2] : 0.0;
                double w = 0.5 * (ax * ax + ay * ay + az * az) * fk[p];
                if (c->dim == 2) w += fk[nv + p];
                s[0] += ax * w; s[1] += ay * w; s[2] += az * w;
            }
    double dv = dvx * dvy * (c->dim == 3 ? dvz : 1.0);
    q[0] = s[0] * dv; q[1] = s[1] * dv; q[2] = s[2] * dv;
}

/* Equilibrium of the collision model at velocity v (R = 1, P = rho T).
 * BGK: the Maxwellian, and in 2D g = T/2 M (Eq. BGKDD).  Shakhov: the
 * Maxwellian times 1 + (1 - Pr)(v - u).q (|v - u|^2/T - 5)/(5 P T) in 3D
 * (Sec. 2.1); in 2D f and g of Eq. ShakhovDD, with -4 and -2 in place of -5. */
static void equilibrium_at(const orc_cfg *c, double rho, const double *u, double T, const double *q,
                           double vx, double vy, double vz, double *fe, double *ge)
{
    if (c->dim == 3) {
        double M = maxw3d(rho, u[0], u[1], u[2], T, vx, vy, vz);
        if (c->model == ORC_SHAKHOV) {
            double ax = vx - u[0], ay = vy - u[1], az = vz - u[2];
            double cq = ax * q[0] + ay * q[1] + az * q[2];
            M *= 1.0 + (1.0 - c->Pr) * cq * ((ax * ax + ay * ay + az * az) / T - 5.0) / (5.0 * rho * T * T);
        }
        *fe = M;
        return;
    }
    double M = maxw2d(rho, u[0], u[1], T, vx, vy);
    double sf = 1.0, sg = 1.0;
    if (c->model == ORC_SHAKHOV) {
        double ax = vx - u[0], ay = vy - u[1];
        double cq = ax * q[0] + ay * q[1];
        double c2 = (ax * ax + ay * ay) / T;
        double k = (1.0 - c->Pr) * cq / (5.0 * rho * T * T);
        sf = 1.0 + k * (c2 - 4.0);
        sg = 1.0 + k * (c2 - 2.0);
    }
    *fe = M * sf;
    if (ge) *ge = T / 2.0 * M * sg;
}

static int model_ok(const orc_cfg *c)
{
    if (c->conservative && c->model != ORC_BGK) return 0;   /* conservative equilibrium: BGK */
    if (c->model == ORC_BGK) return 1;
    return c->model == ORC_SHAKHOV && c->Pr >= 0;
}

int orc_heat_flux(const orc_cfg *c, const double *fk, double *q)
{
    double rho, u[3], T;
    int rc = cell_moments(c, fk, &rho, u, &T);
    cell_heat_flux(c, fk, u, q);
    return rc;
}

int orc_equilibrium(const orc_cfg *c, double rho, const double *u, double T,
                    const double *q, double *fk)
{
    if (!model_ok(c) || !(rho > 0) || !(T > 0)) return ORC_ERR_ARG;
    const int nv1 = c->nvx, nv2 = c->nvy, nv3 = c->dim == 3 ? c->nvz : 1;
    const int nv = nv1 * nv2 * nv3;
    const double dvx = (c->vxmax - c->vxmin) / nv1, dvy = (c->vymax - c->vymin) / nv2;
    const double dvz = c->dim == 3 ? (c->vzmax - c->vzmin) / nv3 : 1.0;
    for (int p3 = 0; p3 < nv3; ++p3)
        for (int p2 = 0; p2 < nv2; ++p2)
            for (int p1 = 0; p1 < nv1; ++p1) {
                int p = (p3 * nv2 + p2) * nv1 + p1;
                double vz = c->dim == 3 ? c->vzmin + p3 * dvz : 0.0;
                equilibrium_at(c, rho, u, T, q, c->vxmin + p1 * dvx, c->vymin + p2 * dvy, vz, &fk[p],
                               c->dim == 2 ? &fk[nv + p] : NULL);
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

/* Periodic image of index a on an axis of n cells (any a, also when the
 * stencil reaches further than n cells). */
/* Implicit relaxation of the first-order semi-implicit scheme (Eq.
 * ImpSchemeDD) on the transported values fk of one control volume (the first
 * two terms of the scheme).  Summing the scheme over the velocities makes the
 * collision term vanish, so rho, u and T at t^{n+1} are the moments of the
 * transported values; with them f^{n+1} = (f_T + nu M) / (1 + nu), where
 * nu = dt / tau^{n+1} = dt rho^{n+1} / tau0 and M is the Maxwellian of
 * Eq. BGKDD (2D: g_T relaxes towards T/2 M).  reading: with the direct
 * moments the discrete moments of M are taken equal to rho, u, T, as in the
 * explicit scheme; with the conservative parameters of Sec. 3.1 they are
 * equal by construction, so the relaxed state keeps the discrete moments of
 * the transported one. */
static int imex_relax(const orc_cfg *c, double dt, double tau0, double *fk)
{
    double rho, u[3], T, rd, ud[3], Td;
    if (cell_moments(c, fk, &rd, ud, &Td)) return ORC_ERR_NONPHYSICAL;
    /* tau from the direct density; the Maxwellian from the equilibrium
     * parameters (direct or conservative, Sec. 3.1) */
    if (equilibrium_params(c, fk, &rho, u, &T)) return ORC_ERR_NONPHYSICAL;
    const double nu = dt * rd / tau0;
    /* Shakhov (Eq. ShakhovDD): the equilibrium holds the heat flux at
     * t^{n+1}.  reading: taking the heat-flux moment of the scheme with the
     * model's property that its equilibrium carries (1 - Pr) q gives
     * q^{n+1} = q_T / (1 + nu Pr), q_T the heat flux of the transported
     * values about their own velocity (Eq. MacroscopicDDv). */
    double q[3] = {0, 0, 0};
    if (c->model == ORC_SHAKHOV) {
        double qt[3];
        cell_heat_flux(c, fk, ud, qt);
        for (int d = 0; d < 3; ++d) q[d] = qt[d] / (1.0 + nu * c->Pr);
    }
    const int nv1 = c->nvx, nv2 = c->nvy, nv3 = c->dim == 3 ? c->nvz : 1;
    const int nv = nv1 * nv2 * nv3;
    const double dvx = (c->vxmax - c->vxmin) / nv1, dvy = (c->vymax - c->vymin) / nv2;
    const double dvz = c->dim == 3 ? (c->vzmax - c->vzmin) / nv3 : 1.0;
    for (int p3 = 0; p3 < nv3; ++p3)
        for (int p2 = 0; p2 < nv2; ++p2)
            for (int p1 = 0; p1 < nv1; ++p1) {
                int p = (p3 * nv2 + p2) * nv1 + p1;
                double vx = c->vxmin + p1 * dvx, vy = c->vymin + p2 * dvy;
                double vz = c->dim == 3 ? c->vzmin + p3 * dvz : 0.0;
                double fe, ge;
                equilibrium_at(c, rho, u, T, q, vx, vy, vz, &fe, c->dim == 3 ? NULL : &ge);
                fk[p] = (fk[p] + nu * fe) / (1.0 + nu);
                if (c->dim == 2) fk[nv + p] = (fk[nv + p] + nu * ge) / (1.0 + nu);
            }
    return ORC_OK;
}

static int wrap(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

/* Value of a virtual cell, extended by the domain boundary conditions.
 * reading: periodic wrap; Maxwellian sides hold the prescribed state in
 * every ghost layer; zero-gradient copies the boundary cell. */
static double fval2d(const orc_ctx2d *x, int i, int j, int comp, int p)
{
    const orc_cfg *c = x->c;
    if (i < 0) {
        if (c->bc[0] == ORC_BC_PERIODIC) i = wrap(i, x->nx);
        else if (c->bc[0] == ORC_BC_MAXWELLIAN) return x->ghost[0][((long)j * 2 + comp) * x->nv + p];
        else i = 0;
    } else if (i >= x->nx) {
        if (c->bc[1] == ORC_BC_PERIODIC) i = wrap(i, x->nx);
        else if (c->bc[1] == ORC_BC_MAXWELLIAN) return x->ghost[1][((long)j * 2 + comp) * x->nv + p];
        else i = x->nx - 1;
    }
    if (j < 0) {
        if (c->bc[2] == ORC_BC_PERIODIC) j = wrap(j, x->ny);
        else if (c->bc[2] == ORC_BC_MAXWELLIAN) return x->ghost[2][((long)i * 2 + comp) * x->nv + p];
        else j = 0;
    } else if (j >= x->ny) {
        if (c->bc[3] == ORC_BC_PERIODIC) j = wrap(j, x->ny);
        else if (c->bc[3] == ORC_BC_MAXWELLIAN) return x->ghost[3][((long)i * 2 + comp) * x->nv + p];
        else j = x->ny - 1;
    }
    return x->F[(((long)j * x->nx + i) * 2 + comp) * x->nv + p];
}

/* Gas test used by the limiter fallback; ghost cells count as gas. */
static int isgas2d(const orc_ctx2d *x, int i, int j)
{
    const orc_cfg *c = x->c;
    if (i < 0) { if (c->bc[0] != ORC_BC_PERIODIC) return 1; i = wrap(i, x->nx); }
    else if (i >= x->nx) { if (c->bc[1] != ORC_BC_PERIODIC) return 1; i = wrap(i, x->nx); }
    if (j < 0) { if (c->bc[2] != ORC_BC_PERIODIC) return 1; j = wrap(j, x->ny); }
    else if (j >= x->ny) { if (c->bc[3] != ORC_BC_PERIODIC) return 1; j = wrap(j, x->ny); }
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
    if (!model_ok(c)) return ORC_ERR_ARG;
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
    double *tau_rho = malloc(sizeof(double) * nc);
    double *mq = calloc((size_t)nc * 3, sizeof(double));
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
        /* moments of f_CV^n and the BGK equilibrium inputs (Eq. BGKDD): the
         * direct density sets tau; the equilibrium takes the direct moments
         * or the conservative parameters of Sec. 3.1 */
        int nonphys = 0;
        #pragma omp parallel for reduction(|:nonphys)
        for (long m = 0; m < nc; ++m) {
            if (mstart[m + 1] - mstart[m] == 0) continue;
            double u[3], r, T;
            if (cell_moments(c, F + m * 2 * nv, &r, u, &T)) nonphys = 1;
            tau_rho[m] = r;
            if (c->model == ORC_SHAKHOV) cell_heat_flux(c, F + m * 2 * nv, u, mq + 3 * m);
            if (c->conservative && c->time_scheme == ORC_EXPLICIT &&
                conservative_params(c, F + m * 2 * nv, &r, u, &T, NULL)) nonphys = 1;
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
        /* Step 6: explicit scheme (Eq. ExSchemeDD), or the first-order
         * semi-implicit one (Eq. ImpSchemeDD), on every control volume. */
        int badcv = 0, badrelax = 0;
        #pragma omp parallel reduction(|:badcv, badrelax)
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
                double tau = tau0 / tau_rho[m];
                double a = Sn[m] / Sp[m], b = dt / Sp[m], r = dt / tau;
                if (c->time_scheme == ORC_IMEX) {
                    for (int comp = 0; comp < 2; ++comp)
                        for (int p = 0; p < nv; ++p)
                            Fnew[(m * 2 + comp) * nv + p] = a * F[(m * 2 + comp) * nv + p] - b * R[comp * nv + p];
                    if (imex_relax(c, dt, tau0, Fnew + m * 2 * nv)) badrelax = 1;
                    continue;
                }
                const double um[3] = {mux[m], muy[m], 0.0};
                for (int p2 = 0; p2 < X.nv2; ++p2)
                    for (int p1 = 0; p1 < X.nv1; ++p1) {
                        int p = p2 * X.nv1 + p1;
                        double eq[2];
                        equilibrium_at(c, mrho[m], um, mT[m], mq + 3 * m, vx[p1], vy[p2], 0.0, &eq[0], &eq[1]);
                        for (int comp = 0; comp < 2; ++comp) {
                            double fcv = F[(m * 2 + comp) * nv + p];
                            Fnew[(m * 2 + comp) * nv + p] = a * fcv - b * R[comp * nv + p] + a * r * (eq[comp] - fcv);
                        }
                    }
            }
            free(R);
        }
        if (badcv) { err = ORC_ERR_GEOMETRY; break; }
        if (badrelax) { err = ORC_ERR_NONPHYSICAL; break; }
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
    free(mrho); free(mux); free(muy); free(mT); free(mq); free(tau_rho);
    free(wphi); free(wux); free(wuy); free(wT); free(Fnew); free(vx); free(vy);
    for (int s = 0; s < 4; ++s) free(X.ghost[s]);
    return err;
}

/* ================================================================ 3D
 * Full-distribution BGK in 3D (Sec. 5): the same steps with seven-face
 * virtual cells.  reading: the geometry that the paper leaves to the reader
 * is built face by face from the 2D construction of Appendix A; the wall face
 * closes the polyhedron, S_w n_w = -sum_faces A_f n_f; the volume follows
 * from the divergence theorem in the cell frame, where the faces at the
 * frame's origin contribute nothing and the wall plane passes through the
 * centroid of the edge crossings.  Only fixed obstacles are handled in 3D. */

static double levelset3d(const orc_cfg *c, double x, double y, double z)
{
    double ddx = x - c->cx, ddy = y - c->cy, ddz = z - c->cz;
    if (c->shape == ORC_SHAPE_SPHERE) return sqrt(ddx * ddx + ddy * ddy + ddz * ddz) - c->ra;
    if (c->shape == ORC_SHAPE_CIRCLE) {          /* infinite circular cylinder */
        if (c->axis == 0) return sqrt(ddy * ddy + ddz * ddz) - c->ra;
        if (c->axis == 1) return sqrt(ddx * ddx + ddz * ddz) - c->ra;
        return sqrt(ddx * ddx + ddy * ddy) - c->ra;
    }
    return 1.0;
}

/* Gas area of a square face with nodal values p00 (u=0,w=0), p10 (u=h1,w=0),
 * p11 (u=h1,w=h2), p01 (u=0,w=h2): the 2D virtual-cell area (Appendix A)
 * evaluated in the plane of the face. */
static double face_area(double p00, double p10, double p11, double p01, double h1, double h2, int *err)
{
    double m = fmin(fmin(p00, p10), fmin(p11, p01));
    double M = fmax(fmax(p00, p10), fmax(p11, p01));
    if (m > 0) return h1 * h2;
    if (M < 0) return 0.0;
    double lum = edge_gas_length(p00, p01, h2), lup = edge_gas_length(p10, p11, h2);
    double lwm = edge_gas_length(p00, p10, h1), lwp = edge_gas_length(p01, p11, h1);
    double pu[4], pw[4];
    int n = 0;
    if ((p00 > 0) != (p01 > 0)) { pu[n] = 0;  pw[n] = h2 * (p00 / (p00 - p01)); ++n; }
    if ((p10 > 0) != (p11 > 0)) { pu[n] = h1; pw[n] = h2 * (p10 / (p10 - p11)); ++n; }
    if ((p00 > 0) != (p10 > 0)) { pu[n] = h1 * (p00 / (p00 - p10)); pw[n] = 0;  ++n; }
    if ((p01 > 0) != (p11 > 0)) { pu[n] = h1 * (p01 / (p01 - p11)); pw[n] = h2; ++n; }
    if (n != 2) { *err = ORC_ERR_GEOMETRY; return 0.0; }
    double eu = pu[1] - pu[0], ew = pw[1] - pw[0];
    double lw = sqrt(eu * eu + ew * ew);
    double ru = 0.5 * (pu[0] + pu[1]), rw = 0.5 * (pw[0] + pw[1]);
    double nu = (lum - lup) / lw, nw = (lwm - lwp) / lw;
    return 0.5 * (lup * h1 + lwp * h2 + lw * (ru * nu + rw * nw));
}

int orc_geometry3d(const orc_cfg *c, orc_geo3d *g)
{
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    const double dx = (c->xmax - c->xmin) / nx, dy = (c->ymax - c->ymin) / ny, dz = (c->zmax - c->zmin) / nz;
    int err = ORC_OK;
#define N3(a, b, cc) g->phi[((long)(cc) * (ny + 1) + (b)) * (nx + 1) + (a)]
    for (int cc = 0; cc <= nz; ++cc)
        for (int b = 0; b <= ny; ++b)
            for (int a = 0; a <= nx; ++a)
                N3(a, b, cc) = clamp_phi(levelset3d(c, c->xmin + a * dx, c->ymin + b * dy, c->zmin + cc * dz), dx);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int a = 0; a <= nx; ++a)
                g->ax[((long)k * ny + j) * (nx + 1) + a] =
                    face_area(N3(a, j, k), N3(a, j + 1, k), N3(a, j + 1, k + 1), N3(a, j, k + 1), dy, dz, &err);
    for (int k = 0; k < nz; ++k)
        for (int b = 0; b <= ny; ++b)
            for (int i = 0; i < nx; ++i)
                g->ay[((long)k * (ny + 1) + b) * nx + i] =
                    face_area(N3(i, b, k), N3(i + 1, b, k), N3(i + 1, b, k + 1), N3(i, b, k + 1), dx, dz, &err);
    for (int cc = 0; cc <= nz; ++cc)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                g->az[((long)cc * ny + j) * nx + i] =
                    face_area(N3(i, j, cc), N3(i + 1, j, cc), N3(i + 1, j + 1, cc), N3(i, j + 1, cc), dx, dy, &err);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long q = ((long)k * ny + j) * nx + i;
                double p[8] = {N3(i, j, k), N3(i + 1, j, k), N3(i + 1, j + 1, k), N3(i, j + 1, k),
                               N3(i, j, k + 1), N3(i + 1, j, k + 1), N3(i + 1, j + 1, k + 1), N3(i, j + 1, k + 1)};
                double m = p[0], M = p[0], s = p[0];
                for (int t = 1; t < 8; ++t) { m = fmin(m, p[t]); M = fmax(M, p[t]); s = s + p[t]; }
                g->cgas[q] = 0.125 * s > 0;     /* Eq. (ii) with the 8 nodes */
                g->sw[q] = 0; g->nwx[q] = g->nwy[q] = g->nwz[q] = 0;
                g->rwx[q] = g->rwy[q] = g->rwz[q] = 0;
                if (m > 0) { g->type[q] = ORC_GAS; g->vol[q] = dx * dy * dz; continue; }
                if (M < 0) { g->type[q] = ORC_SOLID; g->vol[q] = 0; continue; }
                g->type[q] = ORC_CUT;
                double axm = g->ax[((long)k * ny + j) * (nx + 1) + i], axp = g->ax[((long)k * ny + j) * (nx + 1) + i + 1];
                double aym = g->ay[((long)k * (ny + 1) + j) * nx + i], ayp = g->ay[((long)k * (ny + 1) + j + 1) * nx + i];
                double azm = g->az[((long)k * ny + j) * nx + i], azp = g->az[((long)(k + 1) * ny + j) * nx + i];
                double wx = axm - axp, wy = aym - ayp, wz = azm - azp;
                double sw = sqrt(wx * wx + wy * wy + wz * wz);
                /* crossings of the 12 edges in the cell frame */
                static const int E[12][2] = {{0, 1}, {3, 2}, {4, 5}, {7, 6},     /* along x */
                                             {0, 3}, {1, 2}, {4, 7}, {5, 6},     /* along y */
                                             {0, 4}, {1, 5}, {3, 7}, {2, 6}};    /* along z */
                static const double O[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                               {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
                double rx = 0, ry = 0, rz = 0;
                int nc = 0;
                for (int e = 0; e < 12; ++e) {
                    double p0 = p[E[e][0]], p1 = p[E[e][1]];
                    if ((p0 > 0) == (p1 > 0)) continue;
                    double t = p0 / (p0 - p1);
                    const double *o0 = O[E[e][0]], *o1 = O[E[e][1]];
                    rx += dx * (o0[0] + t * (o1[0] - o0[0]));
                    ry += dy * (o0[1] + t * (o1[1] - o0[1]));
                    rz += dz * (o0[2] + t * (o1[2] - o0[2]));
                    ++nc;
                }
                rx /= nc; ry /= nc; rz /= nc;
                double nwx = sw > 0 ? wx / sw : 0, nwy = sw > 0 ? wy / sw : 0, nwz = sw > 0 ? wz / sw : 0;
                g->sw[q] = sw; g->nwx[q] = nwx; g->nwy[q] = nwy; g->nwz[q] = nwz;
                g->rwx[q] = (c->xmin + i * dx) + rx;
                g->rwy[q] = (c->ymin + j * dy) + ry;
                g->rwz[q] = (c->zmin + k * dz) + rz;
                g->vol[q] = (axp * dx + ayp * dy + azp * dz + sw * (rx * nwx + ry * nwy + rz * nwz)) / 3.0;
            }
#undef N3
    return err;
}

/* Master search with the six faces (ties: x+, x-, y+, y-, z+, z-). */
int orc_masters3d(const orc_cfg *c, const orc_geo3d *g, int32_t *master)
{
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    int err = ORC_OK;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long q = ((long)k * ny + j) * nx + i;
                master[q] = -1;
                if (g->type[q] == ORC_SOLID) continue;
                int ci = i, cj = j, ck = k, it = 0, ok = 0;
                while (it <= ORC_MAXWALK) {
                    long r = ((long)ck * ny + cj) * nx + ci;
                    if (g->cgas[r]) { ok = 1; break; }
                    double axm = g->ax[((long)ck * ny + cj) * (nx + 1) + ci], axp = g->ax[((long)ck * ny + cj) * (nx + 1) + ci + 1];
                    double aym = g->ay[((long)ck * (ny + 1) + cj) * nx + ci], ayp = g->ay[((long)ck * (ny + 1) + cj + 1) * nx + ci];
                    double azm = g->az[((long)ck * ny + cj) * nx + ci], azp = g->az[((long)(ck + 1) * ny + cj) * nx + ci];
                    double M = fmax(fmax(fmax(axp, axm), fmax(ayp, aym)), fmax(azp, azm));
                    if (!(M > 0)) break;
                    if (axp == M) ci++;
                    else if (axm == M) ci--;
                    else if (ayp == M) cj++;
                    else if (aym == M) cj--;
                    else if (azp == M) ck++;
                    else ck--;
                    if (ci < 0 || ci >= nx || cj < 0 || cj >= ny || ck < 0 || ck >= nz) break;
                    ++it;
                }
                if (!ok) { err = ORC_ERR_GEOMETRY; continue; }
                master[q] = (int32_t)(((long)ck * ny + cj) * nx + ci);
            }
    return err;
}

typedef struct {
    const orc_cfg *c;
    int nx, ny, nz, nv, nv1, nv2, nv3;
    double dx, dy, dz, dvx, dvy, dvz, dt;
    double *ghost[6];
    const double *F;
    const orc_geo3d *g;
} orc_ctx3d;

/* Value of cell (i, j, k) with the domain boundary conditions (same readings
 * as in 2D, per axis). */
static double fval3d(const orc_ctx3d *x, int i, int j, int k, int p)
{
    const orc_cfg *c = x->c;
    if (i < 0) {
        if (c->bc[0] == ORC_BC_PERIODIC) i = wrap(i, x->nx);
        else if (c->bc[0] == ORC_BC_MAXWELLIAN) return x->ghost[0][((long)k * x->ny + j) * x->nv + p];
        else i = 0;
    } else if (i >= x->nx) {
        if (c->bc[1] == ORC_BC_PERIODIC) i = wrap(i, x->nx);
        else if (c->bc[1] == ORC_BC_MAXWELLIAN) return x->ghost[1][((long)k * x->ny + j) * x->nv + p];
        else i = x->nx - 1;
    }
    if (j < 0) {
        if (c->bc[2] == ORC_BC_PERIODIC) j = wrap(j, x->ny);
        else if (c->bc[2] == ORC_BC_MAXWELLIAN) return x->ghost[2][((long)k * x->nx + i) * x->nv + p];
        else j = 0;
    } else if (j >= x->ny) {
        if (c->bc[3] == ORC_BC_PERIODIC) j = wrap(j, x->ny);
        else if (c->bc[3] == ORC_BC_MAXWELLIAN) return x->ghost[3][((long)k * x->nx + i) * x->nv + p];
        else j = x->ny - 1;
    }
    if (k < 0) {
        if (c->bc[4] == ORC_BC_PERIODIC) k = wrap(k, x->nz);
        else if (c->bc[4] == ORC_BC_MAXWELLIAN) return x->ghost[4][((long)j * x->nx + i) * x->nv + p];
        else k = 0;
    } else if (k >= x->nz) {
        if (c->bc[5] == ORC_BC_PERIODIC) k = wrap(k, x->nz);
        else if (c->bc[5] == ORC_BC_MAXWELLIAN) return x->ghost[5][((long)j * x->nx + i) * x->nv + p];
        else k = x->nz - 1;
    }
    return x->F[(((long)k * x->ny + j) * x->nx + i) * x->nv + p];
}

static int isgas3d(const orc_ctx3d *x, int i, int j, int k)
{
    const orc_cfg *c = x->c;
    if (i < 0) { if (c->bc[0] != ORC_BC_PERIODIC) return 1; i = wrap(i, x->nx); }
    else if (i >= x->nx) { if (c->bc[1] != ORC_BC_PERIODIC) return 1; i = wrap(i, x->nx); }
    if (j < 0) { if (c->bc[2] != ORC_BC_PERIODIC) return 1; j = wrap(j, x->ny); }
    else if (j >= x->ny) { if (c->bc[3] != ORC_BC_PERIODIC) return 1; j = wrap(j, x->ny); }
    if (k < 0) { if (c->bc[4] != ORC_BC_PERIODIC) return 1; k = wrap(k, x->nz); }
    else if (k >= x->nz) { if (c->bc[5] != ORC_BC_PERIODIC) return 1; k = wrap(k, x->nz); }
    return x->g->type[((long)k * x->ny + j) * x->nx + i] == ORC_GAS;
}

static void alloc_geo3d(orc_geo3d *g, int nx, int ny, int nz)
{
    long nc = (long)nx * ny * nz;
    g->phi = malloc(sizeof(double) * (nx + 1) * (ny + 1) * (long)(nz + 1));
    g->type = malloc(nc); g->cgas = malloc(nc);
    g->ax = malloc(sizeof(double) * (nx + 1) * (long)ny * nz);
    g->ay = malloc(sizeof(double) * nx * (long)(ny + 1) * nz);
    g->az = malloc(sizeof(double) * nx * (long)ny * (nz + 1));
    g->sw = malloc(sizeof(double) * nc);
    g->nwx = malloc(sizeof(double) * nc); g->nwy = malloc(sizeof(double) * nc); g->nwz = malloc(sizeof(double) * nc);
    g->rwx = malloc(sizeof(double) * nc); g->rwy = malloc(sizeof(double) * nc); g->rwz = malloc(sizeof(double) * nc);
    g->vol = malloc(sizeof(double) * nc);
}

static void free_geo3d(orc_geo3d *g)
{
    free(g->phi); free(g->type); free(g->cgas); free(g->ax); free(g->ay); free(g->az); free(g->sw);
    free(g->nwx); free(g->nwy); free(g->nwz); free(g->rwx); free(g->rwy); free(g->rwz); free(g->vol);
}

double orc_mass3d(const orc_cfg *c, const double *F)
{
    const int nv = c->nvx * c->nvy * c->nvz;
    const double dv = (c->vxmax - c->vxmin) / c->nvx * ((c->vymax - c->vymin) / c->nvy) *
                      ((c->vzmax - c->vzmin) / c->nvz);
    orc_geo3d g;
    alloc_geo3d(&g, c->nx, c->ny, c->nz);
    orc_geometry3d(c, &g);
    double M = 0;
    const long nc = (long)c->nx * c->ny * c->nz;
    for (long q = 0; q < nc; ++q) {
        double s = 0;
        for (int p = 0; p < nv; ++p) s += F[q * nv + p];
        M += g.vol[q] * (s * dv);
    }
    free_geo3d(&g);
    return M;
}

int orc_run3d(const orc_cfg *c, double *F, int nsteps, orc_hist *h)
{
    if (c->dim != 3 || c->movable || !model_ok(c)) return ORC_ERR_ARG;
    orc_ctx3d X;
    X.c = c; X.nx = c->nx; X.ny = c->ny; X.nz = c->nz;
    X.nv1 = c->nvx; X.nv2 = c->nvy; X.nv3 = c->nvz; X.nv = X.nv1 * X.nv2 * X.nv3;
    X.dx = (c->xmax - c->xmin) / c->nx; X.dy = (c->ymax - c->ymin) / c->ny; X.dz = (c->zmax - c->zmin) / c->nz;
    X.dvx = (c->vxmax - c->vxmin) / c->nvx; X.dvy = (c->vymax - c->vymin) / c->nvy;
    X.dvz = (c->vzmax - c->vzmin) / c->nvz;
    X.dt = orc_dt(c);
    const int nx = X.nx, ny = X.ny, nz = X.nz, nv = X.nv;
    const long nc = (long)nx * ny * nz;
    const double dt = X.dt, dv = X.dvx * X.dvy * X.dvz, tau0 = orc_tau0(c);
    /* ghosts of Maxwellian sides */
    for (int s = 0; s < 6; ++s) {
        X.ghost[s] = NULL;
        if (c->bc[s] != ORC_BC_MAXWELLIAN) continue;
        long n = s < 2 ? (long)ny * nz : (s < 4 ? (long)nx * nz : (long)nx * ny);
        X.ghost[s] = malloc(sizeof(double) * n * nv);
        for (long q = 0; q < n; ++q) {
            const double *st = c->bc_state[s] + 5 * q;
            for (int p3 = 0; p3 < X.nv3; ++p3)
                for (int p2 = 0; p2 < X.nv2; ++p2)
                    for (int p1 = 0; p1 < X.nv1; ++p1) {
                        int p = (p3 * X.nv2 + p2) * X.nv1 + p1;
                        X.ghost[s][q * nv + p] = maxw3d(st[0], st[1], st[2], st[3], st[4], c->vxmin + p1 * X.dvx,
                                                        c->vymin + p2 * X.dvy, c->vzmin + p3 * X.dvz);
                    }
        }
    }
    orc_geo3d geo;
    alloc_geo3d(&geo, nx, ny, nz);
    int err = orc_geometry3d(c, &geo);
    int32_t *master = malloc(sizeof(int32_t) * nc);
    if (!err) err = orc_masters3d(c, &geo, master);
    int32_t *mstart = malloc(sizeof(int32_t) * (nc + 1)), *mlist = malloc(sizeof(int32_t) * nc), *cnt = malloc(sizeof(int32_t) * nc);
    double *S = malloc(sizeof(double) * nc);
    double *mr = malloc(sizeof(double) * nc), *mu = malloc(sizeof(double) * 3 * nc), *mT = malloc(sizeof(double) * nc);
    double *tau_rho = malloc(sizeof(double) * nc);
    double *mq = calloc((size_t)nc * 3, sizeof(double));
    double *wphi = malloc(sizeof(double) * nc), *wu = malloc(sizeof(double) * 3 * nc), *wT = malloc(sizeof(double) * nc);
    double *Fnew = malloc(sizeof(double) * nc * nv);
    double *vx = malloc(sizeof(double) * X.nv1), *vy = malloc(sizeof(double) * X.nv2), *vz = malloc(sizeof(double) * X.nv3);
    for (int q = 0; q < X.nv1; ++q) vx[q] = c->vxmin + q * X.dvx;
    for (int q = 0; q < X.nv2; ++q) vy[q] = c->vymin + q * X.dvy;
    for (int q = 0; q < X.nv3; ++q) vz[q] = c->vzmin + q * X.dvz;
    if (!err) {
        for (long q = 0; q < nc; ++q) { cnt[q] = 0; S[q] = 0; }
        for (long q = 0; q < nc; ++q) if (master[q] >= 0) { cnt[master[q]]++; S[master[q]] += geo.vol[q]; }
        mstart[0] = 0;
        for (long q = 0; q < nc; ++q) mstart[q + 1] = mstart[q] + cnt[q];
        for (long q = 0; q < nc; ++q) cnt[q] = 0;
        for (long q = 0; q < nc; ++q) if (master[q] >= 0) { int m = master[q]; mlist[mstart[m] + cnt[m]++] = (int32_t)q; }
    }
    X.g = &geo;
    for (int step = 0; step < nsteps && err == ORC_OK; ++step) {
        /* fusion (3D form of Eq. FusionDD) */
        #pragma omp parallel for schedule(dynamic, 64)
        for (long m = 0; m < nc; ++m) {
            if (mstart[m + 1] - mstart[m] <= 1) continue;
            for (int p = 0; p < nv; ++p) {
                double s = 0;
                for (int q = mstart[m]; q < mstart[m + 1]; ++q) s += geo.vol[mlist[q]] * F[(long)mlist[q] * nv + p];
                double fcv = s / S[m];
                for (int q = mstart[m]; q < mstart[m + 1]; ++q) F[(long)mlist[q] * nv + p] = fcv;
            }
        }
        X.F = F;
        int nonphys = 0;
        #pragma omp parallel for reduction(|:nonphys)
        for (long m = 0; m < nc; ++m) {
            if (mstart[m + 1] - mstart[m] == 0) continue;
            double u[3], r, T;
            if (cell_moments(c, F + m * nv, &r, u, &T)) nonphys = 1;
            tau_rho[m] = r;
            if (c->model == ORC_SHAKHOV) cell_heat_flux(c, F + m * nv, u, mq + 3 * m);
            if (c->conservative && c->time_scheme == ORC_EXPLICIT &&
                conservative_params(c, F + m * nv, &r, u, &T, NULL)) nonphys = 1;
            mr[m] = r; mu[3 * m] = u[0]; mu[3 * m + 1] = u[1]; mu[3 * m + 2] = u[2]; mT[m] = T;
        }
        if (nonphys) { err = ORC_ERR_NONPHYSICAL; break; }
        /* wall density and stress (3D forms of Eqs. BoundaryTD, StressTensorDD) */
        double Fx = 0, Fy = 0, Fz = 0, Tq = 0;
        for (long q = 0; q < nc; ++q) {
            if (geo.type[q] != ORC_CUT || !(geo.sw[q] > 0)) continue;
            double rx = geo.rwx[q] - c->cx, ry = geo.rwy[q] - c->cy;
            double uw[3] = {c->vbx - ry * c->omega, c->vby + rx * c->omega, 0.0};
            double Tw = c->Tw, n[3] = {geo.nwx[q], geo.nwy[q], geo.nwz[q]};
            const double *fk = F + q * nv;
            double num = 0, den = 0;
            for (int p3 = 0; p3 < X.nv3; ++p3)
                for (int p2 = 0; p2 < X.nv2; ++p2)
                    for (int p1 = 0; p1 < X.nv1; ++p1) {
                        int p = (p3 * X.nv2 + p2) * X.nv1 + p1;
                        double a[3] = {vx[p1] - uw[0], vy[p2] - uw[1], vz[p3] - uw[2]};
                        double cp = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
                        if (cp > 0) num += cp * fk[p] * dv;
                        else if (cp < 0) den += cp * maxw3d(1.0, uw[0], uw[1], uw[2], Tw, vx[p1], vy[p2], vz[p3]) * dv;
                    }
            double phi = -num / den;
            double Sg[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            for (int p3 = 0; p3 < X.nv3; ++p3)
                for (int p2 = 0; p2 < X.nv2; ++p2)
                    for (int p1 = 0; p1 < X.nv1; ++p1) {
                        int p = (p3 * X.nv2 + p2) * X.nv1 + p1;
                        double a[3] = {vx[p1] - uw[0], vy[p2] - uw[1], vz[p3] - uw[2]};
                        double cp = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
                        double fv;
                        if (cp < 0) fv = phi * maxw3d(1.0, uw[0], uw[1], uw[2], Tw, vx[p1], vy[p2], vz[p3]);
                        else if (cp > 0) fv = fk[p];
                        else continue;
                        for (int r1 = 0; r1 < 3; ++r1)
                            for (int r2 = 0; r2 < 3; ++r2) Sg[r1][r2] += a[r1] * a[r2] * fv * dv;
                    }
            double fk3[3];
            for (int r1 = 0; r1 < 3; ++r1) fk3[r1] = (Sg[r1][0] * n[0] + Sg[r1][1] * n[1] + Sg[r1][2] * n[2]) * geo.sw[q];
            Fx += fk3[0]; Fy += fk3[1]; Fz += fk3[2];
            Tq += rx * fk3[1] - ry * fk3[0];
            wphi[q] = phi; wu[3 * q] = uw[0]; wu[3 * q + 1] = uw[1]; wu[3 * q + 2] = uw[2]; wT[q] = Tw;
        }
        /* explicit scheme (Eq. eq-schema3D), or the semi-implicit one */
        int badrelax3 = 0;
        #pragma omp parallel reduction(|:badrelax3)
        {
            double *R = malloc(sizeof(double) * nv);
            #pragma omp for schedule(dynamic, 16)
            for (long m = 0; m < nc; ++m) {
                if (mstart[m + 1] - mstart[m] == 0) continue;
                for (int p = 0; p < nv; ++p) R[p] = 0;
                for (int q = mstart[m]; q < mstart[m + 1]; ++q) {
                    long kq = mlist[q];
                    int i = (int)(kq % nx), j = (int)((kq / nx) % ny), k = (int)(kq / ((long)nx * ny));
                    int mus = c->scheme == ORC_MUSCL;
                    int mxp = mus && isgas3d(&X, i - 1, j, k) && isgas3d(&X, i, j, k) && isgas3d(&X, i + 1, j, k) && isgas3d(&X, i + 2, j, k);
                    int mxm = mus && isgas3d(&X, i - 2, j, k) && isgas3d(&X, i - 1, j, k) && isgas3d(&X, i, j, k) && isgas3d(&X, i + 1, j, k);
                    int myp = mus && isgas3d(&X, i, j - 1, k) && isgas3d(&X, i, j, k) && isgas3d(&X, i, j + 1, k) && isgas3d(&X, i, j + 2, k);
                    int mym = mus && isgas3d(&X, i, j - 2, k) && isgas3d(&X, i, j - 1, k) && isgas3d(&X, i, j, k) && isgas3d(&X, i, j + 1, k);
                    int mzp = mus && isgas3d(&X, i, j, k - 1) && isgas3d(&X, i, j, k) && isgas3d(&X, i, j, k + 1) && isgas3d(&X, i, j, k + 2);
                    int mzm = mus && isgas3d(&X, i, j, k - 2) && isgas3d(&X, i, j, k - 1) && isgas3d(&X, i, j, k) && isgas3d(&X, i, j, k + 1);
                    double axm = geo.ax[((long)k * ny + j) * (nx + 1) + i], axp = geo.ax[((long)k * ny + j) * (nx + 1) + i + 1];
                    double aym = geo.ay[((long)k * (ny + 1) + j) * nx + i], ayp = geo.ay[((long)k * (ny + 1) + j + 1) * nx + i];
                    double azm = geo.az[((long)k * ny + j) * nx + i], azp = geo.az[((long)(k + 1) * ny + j) * nx + i];
                    int wall = geo.type[kq] == ORC_CUT && geo.sw[kq] > 0;
                    for (int p3 = 0; p3 < X.nv3; ++p3)
                        for (int p2 = 0; p2 < X.nv2; ++p2)
                            for (int p1 = 0; p1 < X.nv1; ++p1) {
                                int p = (p3 * X.nv2 + p2) * X.nv1 + p1;
                                double v1 = vx[p1], v2 = vy[p2], v3 = vz[p3];
                                double n1 = fabs(v1) * dt / X.dx, n2 = fabs(v2) * dt / X.dy, n3 = fabs(v3) * dt / X.dz;
                                /* reading: each direction uses its own velocity component */
                                double fxp = face_flux(axp, v1, n1, fval3d(&X, i - 1, j, k, p), fval3d(&X, i, j, k, p),
                                                       fval3d(&X, i + 1, j, k, p), fval3d(&X, i + 2, j, k, p), mxp);
                                double fxm = face_flux(axm, v1, n1, fval3d(&X, i - 2, j, k, p), fval3d(&X, i - 1, j, k, p),
                                                       fval3d(&X, i, j, k, p), fval3d(&X, i + 1, j, k, p), mxm);
                                double fyp = face_flux(ayp, v2, n2, fval3d(&X, i, j - 1, k, p), fval3d(&X, i, j, k, p),
                                                       fval3d(&X, i, j + 1, k, p), fval3d(&X, i, j + 2, k, p), myp);
                                double fym = face_flux(aym, v2, n2, fval3d(&X, i, j - 2, k, p), fval3d(&X, i, j - 1, k, p),
                                                       fval3d(&X, i, j, k, p), fval3d(&X, i, j + 1, k, p), mym);
                                double fzp = face_flux(azp, v3, n3, fval3d(&X, i, j, k - 1, p), fval3d(&X, i, j, k, p),
                                                       fval3d(&X, i, j, k + 1, p), fval3d(&X, i, j, k + 2, p), mzp);
                                double fzm = face_flux(azm, v3, n3, fval3d(&X, i, j, k - 2, p), fval3d(&X, i, j, k - 1, p),
                                                       fval3d(&X, i, j, k, p), fval3d(&X, i, j, k + 1, p), mzm);
                                double fw = 0;
                                if (wall) {
                                    double a0 = v1 - wu[3 * kq], a1 = v2 - wu[3 * kq + 1], a2 = v3 - wu[3 * kq + 2];
                                    double cp = a0 * geo.nwx[kq] + a1 * geo.nwy[kq] + a2 * geo.nwz[kq];
                                    double fwall = wphi[kq] * maxw3d(1.0, wu[3 * kq], wu[3 * kq + 1], wu[3 * kq + 2], wT[kq], v1, v2, v3);
                                    fw = geo.sw[kq] * (fmin(cp, 0.0) * fwall + fmax(cp, 0.0) * F[kq * nv + p]);
                                }
                                R[p] += (fxp - fxm) + (fyp - fym) + (fzp - fzm) + fw;
                            }
                }
                double tau = tau0 / tau_rho[m];
                double a = 1.0, b = dt / S[m], r = dt / tau;   /* fixed body: V^n = V^{n+1,*} */
                if (c->time_scheme == ORC_IMEX) {
                    /* the semi-implicit scheme (Eq. ImpSchemeDD) in 3D */
                    for (int p = 0; p < nv; ++p) Fnew[m * nv + p] = a * F[m * nv + p] - b * R[p];
                    if (imex_relax(c, dt, tau0, Fnew + m * nv)) badrelax3 = 1;
                    continue;
                }
                for (int p3 = 0; p3 < X.nv3; ++p3)
                    for (int p2 = 0; p2 < X.nv2; ++p2)
                        for (int p1 = 0; p1 < X.nv1; ++p1) {
                            int p = (p3 * X.nv2 + p2) * X.nv1 + p1;
                            double fcv = F[m * nv + p];
                            double feq;
                            equilibrium_at(c, mr[m], mu + 3 * m, mT[m], mq + 3 * m, vx[p1], vy[p2], vz[p3], &feq, NULL);
                            Fnew[m * nv + p] = a * fcv - b * R[p] + a * r * (feq - fcv);
                        }
            }
            free(R);
        }
        if (badrelax3) { err = ORC_ERR_NONPHYSICAL; break; }
        #pragma omp parallel for
        for (long q = 0; q < nc; ++q) {
            int m = master[q];
            if (m < 0) { memset(F + q * nv, 0, sizeof(double) * nv); continue; }
            memcpy(F + q * nv, Fnew + (long)m * nv, sizeof(double) * nv);
        }
        if (h) {
            if (h->Fx) h->Fx[step] = Fx;
            if (h->Fy) h->Fy[step] = Fy;
            if (h->Fz) h->Fz[step] = Fz;
            if (h->torque) h->torque[step] = Tq;
            if (h->mass) {
                double M = 0;
                for (long q = 0; q < nc; ++q) {
                    double s = 0;
                    for (int p = 0; p < nv; ++p) s += F[q * nv + p];
                    M += geo.vol[q] * (s * dv);
                }
                h->mass[step] = M;
            }
        }
    }
    free_geo3d(&geo);
    free(master); free(mstart); free(mlist); free(cnt); free(S); free(mr); free(mu); free(mT); free(mq); free(tau_rho);
    free(wphi); free(wu); free(wT); free(Fnew); free(vx); free(vy); free(vz);
    for (int s = 0; s < 6; ++s) free(X.ghost[s]);
    return err;
}

/* ================================================================ 2D adjoint
 * Discrete adjoint (reverse-mode derivative) of the fixed-body 2D step, for
 * the drag J = F_x(F^N) of the state after N steps (Eqs. StressTensorDD,
 * eq-force on the fused state, as the step itself evaluates it).  The step is
 * the composition  F^n -> fusion (Eq. FusionDD) -> moments, wall density,
 * fluxes, explicit update with relaxation (Eqs. BGKDD, BoundaryDDv, FluxDD,
 * ExSchemeDD) -> distribution (Eq. UpdateDD); its transpose Jacobian is
 * applied in the reverse order.  The limiter is piecewise linear: its
 * derivative is the one of the branch the forward step takes (on a tie the
 * branch the forward minmod returns).  Written as plain loops over cells,
 * components and velocities, in the order of the forward code above. */

typedef struct { long cell; int side, q; } orc_loc;

/* Source of the value fval2d returns for cell (i, j): an interior cell, or a
 * ghost (Maxwellian side, index along the side). */
static orc_loc loc2d(const orc_ctx2d *x, int i, int j)
{
    const orc_cfg *c = x->c;
    orc_loc L = {-1, -1, -1};
    if (i < 0) {
        if (c->bc[0] == ORC_BC_PERIODIC) i = wrap(i, x->nx);
        else if (c->bc[0] == ORC_BC_MAXWELLIAN) { L.side = 0; L.q = j; return L; }
        else i = 0;
    } else if (i >= x->nx) {
        if (c->bc[1] == ORC_BC_PERIODIC) i = wrap(i, x->nx);
        else if (c->bc[1] == ORC_BC_MAXWELLIAN) { L.side = 1; L.q = j; return L; }
        else i = x->nx - 1;
    }
    if (j < 0) {
        if (c->bc[2] == ORC_BC_PERIODIC) j = wrap(j, x->ny);
        else if (c->bc[2] == ORC_BC_MAXWELLIAN) { L.side = 2; L.q = i; return L; }
        else j = 0;
    } else if (j >= x->ny) {
        if (c->bc[3] == ORC_BC_PERIODIC) j = wrap(j, x->ny);
        else if (c->bc[3] == ORC_BC_MAXWELLIAN) { L.side = 3; L.q = i; return L; }
        else j = x->ny - 1;
    }
    L.cell = (long)j * x->nx + i;
    return L;
}

/* minmod with the derivative of the branch taken: d/da, d/db in {0, 1}. */
static double minmod_d(double a, double b, double *da, double *db)
{
    *da = *db = 0.0;
    if (a > 0 && b > 0) { if (a < b) { *da = 1.0; return a; } *db = 1.0; return b; }
    if (a < 0 && b < 0) { if (a > b) { *da = 1.0; return a; } *db = 1.0; return b; }
    return 0.0;
}

/* Derivatives of face_flux with respect to fAA, fA, fB, fBB. */
static void face_flux_d(double L, double v, double nu, double fAA, double fA, double fB,
                        double fBB, int muscl, double d[4])
{
    d[0] = d[1] = d[2] = d[3] = 0.0;
    if (!muscl) { d[1] = L * fmax(v, 0.0); d[2] = L * fmin(v, 0.0); return; }
    const double k = 0.5 * (1.0 - nu);
    double da, db;
    if (v > 0) {            /* fA + k mm(fB - fA, fA - fAA) */
        minmod_d(fB - fA, fA - fAA, &da, &db);
        d[1] = L * v * (1.0 + k * (db - da));
        d[2] = L * v * (k * da);
        d[0] = L * v * (-k * db);
    } else if (v < 0) {     /* fB - k mm(fBB - fB, fB - fA) */
        minmod_d(fBB - fB, fB - fA, &da, &db);
        d[2] = L * v * (1.0 - k * (db - da));
        d[3] = L * v * (-k * da);
        d[1] = L * v * (k * db);
    }
}

/* Sensitivities of the 2D Maxwellian M[rho, u, T](v) and of T/2 M. */
static void maxw2d_d(double rho, double ux, double uy, double T, double vx, double vy,
                     double *m, double dm[4], double dg[4])
{
    const double ax = vx - ux, ay = vy - uy;
    *m = maxw2d(rho, ux, uy, T, vx, vy);
    dm[0] = *m / rho;
    dm[1] = *m * ax / T;
    dm[2] = *m * ay / T;
    dm[3] = *m * ((ax * ax + ay * ay) / (2.0 * T * T) - 1.0 / T);
    for (int q = 0; q < 3; ++q) dg[q] = T / 2.0 * dm[q];
    dg[3] = *m / 2.0 + T / 2.0 * dm[3];
}

typedef struct {
    long nc;
    int nv, ncv;
    int32_t *master, *mstart, *mlist;
    double *Sn;
} orc_cvs;

/* Fusion (Eq. FusionDD): Ft = F with every merged control volume replaced by
 * its area-weighted average. */
static void fuse2d(const orc_ctx2d *x, const orc_cvs *V, const double *F, double *Ft)
{
    const int nv = x->nv;
    memcpy(Ft, F, sizeof(double) * V->nc * 2 * nv);
    for (long m = 0; m < V->nc; ++m) {
        const int nm = V->mstart[m + 1] - V->mstart[m];
        if (nm <= 1) continue;
        for (int comp = 0; comp < 2; ++comp)
            for (int p = 0; p < nv; ++p) {
                double s = 0;
                for (int q = V->mstart[m]; q < V->mstart[m + 1]; ++q) {
                    long kk = V->mlist[q];
                    s += x->g->sbar[kk] * F[(kk * 2 + comp) * nv + p];
                }
                const double fcv = s / V->Sn[m];
                for (int q = V->mstart[m]; q < V->mstart[m + 1]; ++q)
                    Ft[((long)V->mlist[q] * 2 + comp) * nv + p] = fcv;
            }
    }
}

/* Transpose of the fusion: lam_k = (sbar_k / S) sum_{j in CV} nu_j. */
static void fuse2d_T(const orc_ctx2d *x, const orc_cvs *V, const double *nu, double *lam)
{
    const int nv = x->nv;
    memcpy(lam, nu, sizeof(double) * V->nc * 2 * nv);
    for (long m = 0; m < V->nc; ++m) {
        const int nm = V->mstart[m + 1] - V->mstart[m];
        if (nm <= 1) continue;
        for (int comp = 0; comp < 2; ++comp)
            for (int p = 0; p < nv; ++p) {
                double s = 0;
                for (int q = V->mstart[m]; q < V->mstart[m + 1]; ++q)
                    s += nu[((long)V->mlist[q] * 2 + comp) * nv + p];
                for (int q = V->mstart[m]; q < V->mstart[m + 1]; ++q) {
                    long kk = V->mlist[q];
                    lam[(kk * 2 + comp) * nv + p] = x->g->sbar[kk] / V->Sn[m] * s;
                }
            }
    }
}

/* Wall quantities of wall cell k for the state Ft: u_w, T_w, the incoming
 * normalisation D = sum_{c<0} c M1 dv and phi (Eq. BoundaryDDv). */
typedef struct { double uwx, uwy, Tw, D, phi, rx, ry; int sector; } orc_wall;

static orc_wall wall2d(const orc_ctx2d *x, long k, const double *Ft)
{
    const orc_cfg *c = x->c;
    const orc_geo2d *g = x->g;
    orc_wall w;
    w.rx = g->rwx[k] - c->cx; w.ry = g->rwy[k] - c->cy;
    w.uwx = c->vbx - w.ry * c->omega; w.uwy = c->vby + w.rx * c->omega;
    w.sector = c->nseg > 0 ? wall_sector(c, w.rx, w.ry) : 0;
    w.Tw = c->nseg > 0 ? c->Tw_seg[w.sector] : c->Tw;
    const double dv = x->dvx * x->dvy;
    double num = 0, den = 0;
    for (int p2 = 0; p2 < x->nv2; ++p2)
        for (int p1 = 0; p1 < x->nv1; ++p1) {
            const int p = p2 * x->nv1 + p1;
            const double vx = c->vxmin + p1 * x->dvx, vy = c->vymin + p2 * x->dvy;
            const double cp = (vx - w.uwx) * g->nwx[k] + (vy - w.uwy) * g->nwy[k];
            if (cp > 0) num += cp * Ft[k * 2 * x->nv + p] * dv;
            else if (cp < 0) den += cp * maxw2d(1.0, w.uwx, w.uwy, w.Tw, vx, vy) * dv;
        }
    w.D = den;
    w.phi = -num / den;
    return w;
}

/* dM1/dTw for M1 = M[1, u_w, T_w]. */
static double dM1_dTw(double m1, double ax, double ay, double Tw)
{
    return m1 * ((ax * ax + ay * ay) / (2.0 * Tw * Tw) - 1.0 / Tw);
}

int orc_adjoint2d(const orc_cfg *c, const double *F0, int nsteps, double *Jout, double *lam0,
                  double *gTw, double *gbc0, double *gbc1, double *gbc2, double *gbc3)
{
    return orc_adjoint2d_ex(c, F0, nsteps, 1, NULL, Jout, lam0, gTw, gbc0, gbc1, gbc2, gbc3);
}

/* The adjoint for J = [with_drag] F_x(F^N) + <seed, F^N>: the linear part's
 * gradient, the seed, joins lambda^N after the drag part's fusion transpose
 * (the drag is taken on the fused F^N, the functional on F^N itself). */
int orc_adjoint2d_ex(const orc_cfg *c, const double *F0, int nsteps, int with_drag, const double *seed,
                     double *Jout, double *lam0, double *gTw, double *gbc0, double *gbc1, double *gbc2,
                     double *gbc3)
{
    if (c->dim != 2 || c->movable || c->shape == ORC_SHAPE_NONE || nsteps < 0) return ORC_ERR_ARG;
    if (c->model != ORC_BGK || c->time_scheme != ORC_EXPLICIT || c->conservative) return ORC_ERR_ARG;
    orc_ctx2d X;
    X.c = c; X.nx = c->nx; X.ny = c->ny; X.nv1 = c->nvx; X.nv2 = c->nvy;
    X.nv = X.nv1 * X.nv2;
    X.dx = (c->xmax - c->xmin) / c->nx; X.dy = (c->ymax - c->ymin) / c->ny;
    X.dvx = (c->vxmax - c->vxmin) / c->nvx; X.dvy = (c->vymax - c->vymin) / c->nvy;
    X.dt = orc_dt(c);
    const int nx = X.nx, ny = X.ny, nv = X.nv;
    const long nc = (long)nx * ny, ns = nc * 2 * nv;
    const double dt = X.dt, dv = X.dvx * X.dvy, tau0 = orc_tau0(c);
    make_ghosts2d(&X);
    orc_geo2d geo;
    alloc_geo2d(&geo, nx, ny);
    int err = orc_geometry2d(c, cos(c->theta), sin(c->theta), &geo);
    X.g = &geo;
    orc_cvs V;
    V.nc = nc; V.nv = nv;
    V.master = malloc(sizeof(int32_t) * nc);
    V.mstart = malloc(sizeof(int32_t) * (nc + 1));
    V.mlist = malloc(sizeof(int32_t) * nc);
    V.Sn = calloc(nc, sizeof(double));
    int32_t *cnt = calloc(nc, sizeof(int32_t));
    if (!err) err = orc_masters2d(c, &geo, &geo, V.master);
    /* forward states F^0 .. F^N */
    double *Fs = malloc(sizeof(double) * ns * (size_t)(nsteps + 1));
    double *Ft = malloc(sizeof(double) * ns), *nu = calloc(ns, sizeof(double));
    double *lam = malloc(sizeof(double) * ns), *mu = malloc(sizeof(double) * ns);
    double *gg[4] = {NULL, NULL, NULL, NULL};        /* sensitivities to ghost values */
    double *gbc[4] = {gbc0, gbc1, gbc2, gbc3};
    const int nside[4] = {ny, ny, nx, nx};
    for (int s = 0; s < 4; ++s) {
        if (X.ghost[s]) gg[s] = calloc((size_t)nside[s] * 2 * nv, sizeof(double));
        if (gbc[s]) memset(gbc[s], 0, sizeof(double) * 5 * nside[s]);
    }
    const int ntw = c->nseg > 0 ? c->nseg : 1;
    memset(gTw, 0, sizeof(double) * ntw);
    if (err) goto done;
    for (long k = 0; k < nc; ++k) if (V.master[k] >= 0) { cnt[V.master[k]]++; V.Sn[V.master[k]] += geo.sbar[k]; }
    V.mstart[0] = 0;
    for (long k = 0; k < nc; ++k) V.mstart[k + 1] = V.mstart[k] + cnt[k];
    memset(cnt, 0, sizeof(int32_t) * nc);
    for (long k = 0; k < nc; ++k)
        if (V.master[k] >= 0) { int m = V.master[k]; V.mlist[V.mstart[m] + cnt[m]++] = (int32_t)k; }
    memcpy(Fs, F0, sizeof(double) * ns);
    for (int n = 0; n < nsteps && !err; ++n) {
        memcpy(Fs + (size_t)(n + 1) * ns, Fs + (size_t)n * ns, sizeof(double) * ns);
        err = orc_run2d(c, Fs + (size_t)(n + 1) * ns, 1, NULL, NULL, NULL);
    }
    if (err) goto done;

    /* objective: J = F_x of the fused final state; nu = dJ/dFt */
    {
        fuse2d(&X, &V, Fs + (size_t)nsteps * ns, Ft);
        memset(nu, 0, sizeof(double) * ns);
        double J = 0;
        for (long k = 0; k < nc && with_drag; ++k) {
            if (geo.type[k] != ORC_CUT || !(geo.lw[k] > 0)) continue;
            const orc_wall w = wall2d(&X, k, Ft);
            const double nwx = geo.nwx[k], nwy = geo.nwy[k], lw = geo.lw[k];
            double sxx = 0, sxy = 0, sphi = 0, sTw = 0, dD = 0;
            for (int p2 = 0; p2 < X.nv2; ++p2)
                for (int p1 = 0; p1 < X.nv1; ++p1) {
                    const int p = p2 * X.nv1 + p1;
                    const double vx = c->vxmin + p1 * X.dvx, vy = c->vymin + p2 * X.dvy;
                    const double ax = vx - w.uwx, ay = vy - w.uwy, cp = ax * nwx + ay * nwy;
                    const double wgt = (ax * ax * nwx + ax * ay * nwy) * lw * dv;   /* dFx / dF_w(p) */
                    if (cp > 0) {
                        const double f = Ft[k * 2 * nv + p];
                        sxx += ax * ax * f * dv; sxy += ax * ay * f * dv;
                        nu[k * 2 * nv + p] += wgt;
                    } else if (cp < 0) {
                        const double m1 = maxw2d(1.0, w.uwx, w.uwy, w.Tw, vx, vy);
                        const double dm1 = dM1_dTw(m1, ax, ay, w.Tw);
                        sxx += ax * ax * w.phi * m1 * dv; sxy += ax * ay * w.phi * m1 * dv;
                        sphi += wgt * m1;
                        sTw += wgt * w.phi * dm1;
                        dD += cp * dm1 * dv;
                    }
                }
            J += (sxx * nwx + sxy * nwy) * lw;
            /* phi = -num / D: dphi/df(p) = -c_p dv / D (c_p > 0); dphi/dTw = -phi / D dD/dTw */
            for (int p2 = 0; p2 < X.nv2; ++p2)
                for (int p1 = 0; p1 < X.nv1; ++p1) {
                    const int p = p2 * X.nv1 + p1;
                    const double vx = c->vxmin + p1 * X.dvx, vy = c->vymin + p2 * X.dvy;
                    const double cp = (vx - w.uwx) * nwx + (vy - w.uwy) * nwy;
                    if (cp > 0) nu[k * 2 * nv + p] += sphi * (-cp * dv / w.D);
                }
            gTw[w.sector] += sTw + sphi * (-w.phi / w.D) * dD;
        }
        *Jout = J;
        fuse2d_T(&X, &V, nu, lam);
        if (seed)
            for (long q = 0; q < ns; ++q) lam[q] += seed[q];
    }

    /* reverse sweep over the steps */
    for (int n = nsteps - 1; n >= 0; --n) {
        const double *Fn = Fs + (size_t)n * ns;
        fuse2d(&X, &V, Fn, Ft);
        X.F = Ft;
        /* transpose of the distribution: mu_m = sum of lam over the members */
        memset(mu, 0, sizeof(double) * ns);
        for (long k = 0; k < nc; ++k) {
            const int m = V.master[k];
            if (m < 0) continue;
            for (int q = 0; q < 2 * nv; ++q) mu[(long)m * 2 * nv + q] += lam[k * 2 * nv + q];
        }
        memset(nu, 0, sizeof(double) * ns);
        for (long m = 0; m < nc; ++m) {
            if (V.mstart[m + 1] - V.mstart[m] == 0) continue;
            const double *mm = mu + m * 2 * nv;
            const double *fc = Ft + m * 2 * nv;
            /* relaxation: G = fcv - b R + r (Feq - fcv), r = dt rho / tau0 */
            double u[3], rho, T;
            cell_moments(c, fc, &rho, u, &T);
            const double r = dt * rho / tau0, b = dt / V.Sn[m];
            double sp[4] = {0, 0, 0, 0};          /* d/d(rho, ux, uy, T) of sum mu r Feq */
            double srho_r = 0;                     /* via r(rho): sum mu (Feq - fcv) dt/tau0 */
            for (int p2 = 0; p2 < X.nv2; ++p2)
                for (int p1 = 0; p1 < X.nv1; ++p1) {
                    const int p = p2 * X.nv1 + p1;
                    const double vx = c->vxmin + p1 * X.dvx, vy = c->vymin + p2 * X.dvy;
                    double M, dm[4], dg[4];
                    maxw2d_d(rho, u[0], u[1], T, vx, vy, &M, dm, dg);
                    for (int q = 0; q < 4; ++q) sp[q] += r * (mm[p] * dm[q] + mm[nv + p] * dg[q]);
                    srho_r += (mm[p] * (M - fc[p]) + mm[nv + p] * (T / 2.0 * M - fc[nv + p])) * dt / tau0;
                    nu[m * 2 * nv + p] += mm[p] * (1.0 - r);
                    nu[m * 2 * nv + nv + p] += mm[nv + p] * (1.0 - r);
                }
            sp[0] += srho_r;
            /* chain (rho, ux, uy, T) -> conserved sums (m0, m1, m2, m3) = (rho, rho ux, rho uy, E) */
            const double E = rho * (0.5 * (u[0] * u[0] + u[1] * u[1]) + 1.5 * T);
            const double S0 = sp[0] - sp[1] * u[0] / rho - sp[2] * u[1] / rho +
                              sp[3] * (-2.0 * E / (rho * rho) + 2.0 * (u[0] * u[0] + u[1] * u[1]) / rho) / 3.0;
            const double S1 = sp[1] / rho - sp[3] * 2.0 * u[0] / (3.0 * rho);
            const double S2 = sp[2] / rho - sp[3] * 2.0 * u[1] / (3.0 * rho);
            const double S3 = sp[3] * 2.0 / (3.0 * rho);
            for (int p2 = 0; p2 < X.nv2; ++p2)
                for (int p1 = 0; p1 < X.nv1; ++p1) {
                    const int p = p2 * X.nv1 + p1;
                    const double vx = c->vxmin + p1 * X.dvx, vy = c->vymin + p2 * X.dvy;
                    nu[m * 2 * nv + p] += dv * (S0 + S1 * vx + S2 * vy + S3 * 0.5 * (vx * vx + vy * vy));
                    nu[m * 2 * nv + nv + p] += dv * S3;
                }
            /* transport of every member: G -= b R */
            for (int qq = V.mstart[m]; qq < V.mstart[m + 1]; ++qq) {
                const long k = V.mlist[qq];
                if (geo.type[k] == ORC_SOLID) continue;
                const int i = (int)(k % nx), j = (int)(k / nx);
                const int mus = c->scheme == ORC_MUSCL;
                const int mxp = mus && isgas2d(&X, i - 1, j) && isgas2d(&X, i, j) && isgas2d(&X, i + 1, j) && isgas2d(&X, i + 2, j);
                const int mxm = mus && isgas2d(&X, i - 2, j) && isgas2d(&X, i - 1, j) && isgas2d(&X, i, j) && isgas2d(&X, i + 1, j);
                const int myp = mus && isgas2d(&X, i, j - 1) && isgas2d(&X, i, j) && isgas2d(&X, i, j + 1) && isgas2d(&X, i, j + 2);
                const int mym = mus && isgas2d(&X, i, j - 2) && isgas2d(&X, i, j - 1) && isgas2d(&X, i, j) && isgas2d(&X, i, j + 1);
                const double lxp = geo.lx[j * (nx + 1) + i + 1], lxm = geo.lx[j * (nx + 1) + i];
                const double lyp = geo.ly[(j + 1) * nx + i], lym = geo.ly[j * nx + i];
                /* the four faces: sign in R, length, axis, stencil cells (AA, A, B, BB) */
                const struct { double sgn, L; int ax, muscl; int ci[4], cj[4]; } faces[4] = {
                    {+1.0, lxp, 0, mxp, {i - 1, i, i + 1, i + 2}, {j, j, j, j}},
                    {-1.0, lxm, 0, mxm, {i - 2, i - 1, i, i + 1}, {j, j, j, j}},
                    {+1.0, lyp, 1, myp, {i, i, i, i}, {j - 1, j, j + 1, j + 2}},
                    {-1.0, lym, 1, mym, {i, i, i, i}, {j - 2, j - 1, j, j + 1}}};
                for (int fa = 0; fa < 4; ++fa) {
                    orc_loc loc[4];
                    for (int t = 0; t < 4; ++t) loc[t] = loc2d(&X, faces[fa].ci[t], faces[fa].cj[t]);
                    for (int comp = 0; comp < 2; ++comp)
                        for (int p2 = 0; p2 < X.nv2; ++p2)
                            for (int p1 = 0; p1 < X.nv1; ++p1) {
                                const int p = p2 * X.nv1 + p1;
                                const double w = -b * mm[comp * nv + p] * faces[fa].sgn;
                                if (w == 0.0) continue;
                                const double vx = c->vxmin + p1 * X.dvx, vy = c->vymin + p2 * X.dvy;
                                const double v = faces[fa].ax == 0 ? vx : vy;
                                const double nuc = faces[fa].ax == 0 ? fabs(vx) * dt / X.dx : fabs(vy) * dt / X.dy;
                                double fv[4], d[4];
                                for (int t = 0; t < 4; ++t) fv[t] = fval2d(&X, faces[fa].ci[t], faces[fa].cj[t], comp, p);
                                face_flux_d(faces[fa].L, v, nuc, fv[0], fv[1], fv[2], fv[3], faces[fa].muscl, d);
                                for (int t = 0; t < 4; ++t) {
                                    if (d[t] == 0.0) continue;
                                    if (loc[t].cell >= 0) nu[(loc[t].cell * 2 + comp) * nv + p] += w * d[t];
                                    else gg[loc[t].side][((long)loc[t].q * 2 + comp) * nv + p] += w * d[t];
                                }
                            }
                }
                /* wall flux: lw (min(c,0) phi Mw + max(c,0) F) */
                if (geo.type[k] == ORC_CUT && geo.lw[k] > 0) {
                    const orc_wall ww = wall2d(&X, k, Ft);
                    const double nwx = geo.nwx[k], nwy = geo.nwy[k], lw = geo.lw[k];
                    double sphi = 0, sTw = 0, dD = 0;
                    for (int p2 = 0; p2 < X.nv2; ++p2)
                        for (int p1 = 0; p1 < X.nv1; ++p1) {
                            const int p = p2 * X.nv1 + p1;
                            const double vx = c->vxmin + p1 * X.dvx, vy = c->vymin + p2 * X.dvy;
                            const double ax = vx - ww.uwx, ay = vy - ww.uwy, cp = ax * nwx + ay * nwy;
                            const double w0 = -b * mm[p], w1 = -b * mm[nv + p];
                            if (cp > 0) {
                                nu[k * 2 * nv + p] += w0 * lw * cp;
                                nu[k * 2 * nv + nv + p] += w1 * lw * cp;
                            } else if (cp < 0) {
                                const double m1 = maxw2d(1.0, ww.uwx, ww.uwy, ww.Tw, vx, vy);
                                const double dm1 = dM1_dTw(m1, ax, ay, ww.Tw);
                                /* f_w = phi m1, g_w = phi Tw/2 m1 */
                                sphi += lw * cp * (w0 * m1 + w1 * ww.Tw / 2.0 * m1);
                                sTw += lw * cp * ww.phi * (w0 * dm1 + w1 * (m1 / 2.0 + ww.Tw / 2.0 * dm1));
                                dD += cp * dm1 * dv;
                            }
                        }
                    for (int p2 = 0; p2 < X.nv2; ++p2)
                        for (int p1 = 0; p1 < X.nv1; ++p1) {
                            const int p = p2 * X.nv1 + p1;
                            const double vx = c->vxmin + p1 * X.dvx, vy = c->vymin + p2 * X.dvy;
                            const double cp = (vx - ww.uwx) * nwx + (vy - ww.uwy) * nwy;
                            if (cp > 0) nu[k * 2 * nv + p] += sphi * (-cp * dv / ww.D);
                        }
                    gTw[ww.sector] += sTw + sphi * (-ww.phi / ww.D) * dD;
                }
            }
        }
        fuse2d_T(&X, &V, nu, lam);
    }
    memcpy(lam0, lam, sizeof(double) * ns);
    /* ghost sensitivities -> (rho, ux, uy, uz, T) of the Maxwellian sides */
    for (int s = 0; s < 4; ++s) {
        if (!gg[s] || !gbc[s]) continue;
        for (int q = 0; q < nside[s]; ++q) {
            const double *st = c->bc_state[s] + 5 * q;
            double *o = gbc[s] + 5 * q;
            for (int p2 = 0; p2 < X.nv2; ++p2)
                for (int p1 = 0; p1 < X.nv1; ++p1) {
                    const int p = p2 * X.nv1 + p1;
                    const double vx = c->vxmin + p1 * X.dvx, vy = c->vymin + p2 * X.dvy;
                    double M, dm[4], dg[4];
                    maxw2d_d(st[0], st[1], st[2], st[4], vx, vy, &M, dm, dg);
                    const double a0 = gg[s][((long)q * 2) * nv + p], a1 = gg[s][((long)q * 2 + 1) * nv + p];
                    o[0] += a0 * dm[0] + a1 * dg[0];
                    o[1] += a0 * dm[1] + a1 * dg[1];
                    o[2] += a0 * dm[2] + a1 * dg[2];
                    o[4] += a0 * dm[3] + a1 * dg[3];
                }
        }
    }
done:
    free_geo2d(&geo);
    free(V.master); free(V.mstart); free(V.mlist); free(V.Sn); free(cnt);
    free(Fs); free(Ft); free(nu); free(lam); free(mu);
    for (int s = 0; s < 4; ++s) { free(X.ghost[s]); free(gg[s]); }
    return err;
}

/* Transpose of the Maxwellian initial state (orc_init_maxwellian, 2D):
 * g[cell][5] = d<lam, F0>/d(rho, ux, uy, uz, T) of each cell. */
int orc_init_maxwellian_vjp(const orc_cfg *c, const double *rho, const double *ux, const double *uy,
                            const double *T, const double *lam, double *g)
{
    if (c->dim != 2) return ORC_ERR_ARG;
    const int nv1 = c->nvx, nv2 = c->nvy, nv = nv1 * nv2;
    const long ncell = (long)c->nx * c->ny;
    const double dvx = (c->vxmax - c->vxmin) / nv1, dvy = (c->vymax - c->vymin) / nv2;
    for (long k = 0; k < ncell; ++k) {
        double *o = g + 5 * k;
        for (int q = 0; q < 5; ++q) o[q] = 0;
        if (rho[k] <= 0) continue;
        for (int p2 = 0; p2 < nv2; ++p2)
            for (int p1 = 0; p1 < nv1; ++p1) {
                const int p = p2 * nv1 + p1;
                const double vx = c->vxmin + p1 * dvx, vy = c->vymin + p2 * dvy;
                double M, dm[4], dg[4];
                maxw2d_d(rho[k], ux[k], uy[k], T[k], vx, vy, &M, dm, dg);
                const double a0 = lam[(k * 2) * nv + p], a1 = lam[(k * 2 + 1) * nv + p];
                o[0] += a0 * dm[0] + a1 * dg[0];
                o[1] += a0 * dm[1] + a1 * dg[1];
                o[2] += a0 * dm[2] + a1 * dg[2];
                o[4] += a0 * dm[3] + a1 * dg[3];
            }
    }
    return ORC_OK;
}
