/*
 * Plain FP64 CPU oracle for the Cartesian cut-cell discrete-velocity method
 * (Dechriste & Mieussens, arXiv:1503.04544).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against the paper: only the tests, the smoke entry point and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the GPU path.
 *
 * Every routine is written as plain loops in the order the paper states the
 * method (Sec. 3.3.5 "Summary of the numerical scheme" for 2D, Sec. 5 for 3D,
 * Appendix A for the geometry).  Compiled with -ffp-contract=off so that the
 * geometry (a pure function of +,-,*,/,sqrt) is reproducible bit for bit.
 *
 * Layout of a distribution array: [cell][component][p], cell = j*nx + i
 * (3D: (k*ny + j)*nx + i), p = p2*nvx + p1 (3D: (p3*nvy + p2)*nvx + p1), the
 * velocity ordering of Sec. 3.1.  2D has two components (f, g) of the reduced
 * model (Sec. 2.2); 3D has one (F).
 */
#ifndef DVM_ORACLE_H
#define DVM_ORACLE_H
#include <stdint.h>

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_CFL = 2, ORC_ERR_GEOMETRY = 3,
       ORC_ERR_NONPHYSICAL = 4 };
enum { ORC_GAS = 0, ORC_CUT = 1, ORC_SOLID = 2 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_MAXWELLIAN = 1, ORC_BC_ZEROGRAD = 2 };
enum { ORC_SHAPE_NONE = 0, ORC_SHAPE_CIRCLE = 1, ORC_SHAPE_ELLIPSE = 2,
       ORC_SHAPE_SPHERE = 3, ORC_SHAPE_DISK_CONTAINER = 4, ORC_SHAPE_BOX_CONTAINER = 5 };
enum { ORC_UPWIND = 0, ORC_MUSCL = 1 };
enum { ORC_EXPLICIT = 0, ORC_IMEX = 1 };  /* Eq. ExSchemeDD | Eq. ImpSchemeDD */
enum { ORC_BGK = 0, ORC_SHAKHOV = 1 };    /* Eq. BGKDD | Eq. ShakhovDD (Sec. 2.1) */

/* Problem statement.  2D uses the x/y fields, 3D also the z ones. */
typedef struct {
    int dim;                       /* 2 or 3 */
    int nx, ny, nz;                /* cells per axis */
    double xmin, xmax, ymin, ymax, zmin, zmax;
    int nvx, nvy, nvz;             /* velocity points per axis */
    double vxmin, vxmax, vymin, vymax, vzmin, vzmax;
    double Kn, Lref, cfl, dt;      /* dt > 0 overrides the CFL rule */
    int scheme;                    /* ORC_UPWIND | ORC_MUSCL */
    int bc[6];                     /* x-, x+, y-, y+, z-, z+ */
    /* Maxwellian sides: (rho, ux, uy, uz, T) per boundary cell of that side,
     * ordered like the cells of the side (2D: j or i; 3D: row-major of the
     * two remaining axes). */
    const double *bc_state[6];
    /* obstacle */
    int shape;
    double cx, cy, cz, ra, rb;     /* circle/sphere radius ra; ellipse a=ra, b=rb */
    double theta, omega;           /* body angle and angular velocity */
    double vbx, vby;               /* translational velocity (kept fixed; the
                                      configurations only rotate) */
    double mass, inertia;
    int movable;                   /* 1: free rotation about (cx, cy) */
    double Tw;                     /* wall temperature */
    int nseg;                      /* >0: per-sector wall temperatures */
    const double *Tw_seg;          /* [nseg] */
    const double *seg_dir;         /* [2*nseg] sector boundary directions */
    int axis;                      /* 3D circle: axis of the infinite cylinder
                                      (0 x, 1 y, 2 z) */
    int time_scheme;               /* ORC_EXPLICIT (Eq. ExSchemeDD) or ORC_IMEX
                                      (first-order semi-implicit, Eq. ImpSchemeDD) */
    int model;                     /* ORC_BGK or ORC_SHAKHOV (explicit scheme only) */
    double Pr;                     /* Prandtl number of the Shakhov model */
    int conservative;              /* 0: the equilibrium takes the direct moments
                                      (Eq. MacroscopicDDv); 1: the (rho, u, T)
                                      whose discrete equilibrium has the discrete
                                      moments of the state (Sec. 3.1, Newton; BGK) */
} orc_cfg;

/* Geometry of one time level (2D): every array is caller-owned.          */
typedef struct {
    double *phi;      /* (nx+1)*(ny+1) nodal level set, node (a,b) at b*(nx+1)+a */
    int8_t *type;     /* nx*ny: ORC_GAS / ORC_CUT / ORC_SOLID                   */
    int8_t *cgas;     /* nx*ny: centre-in-gas test of Eq. (ii)                   */
    double *lx;       /* (nx+1)*ny vertical edges, edge a of row j at j*(nx+1)+a */
    double *ly;       /* nx*(ny+1) horizontal edges, edge b of column i at b*nx+i */
    double *lw;       /* nx*ny wall edge length                                  */
    double *nwx, *nwy;/* nx*ny wall normal (towards the solid)                   */
    double *rwx, *rwy;/* nx*ny wall edge centre (absolute)                       */
    double *sbar;     /* nx*ny virtual cell area                                 */
} orc_geo2d;

/* Diagnostics written by the runner, one entry per step (nullable).        */
typedef struct {
    double *Fx, *Fy, *Fz;   /* force on the body at t^n                     */
    double *torque;         /* torque about the z axis at t^n               */
    double *theta, *omega;  /* body state after the step                    */
    double *mass;           /* total mass after the step                    */
} orc_hist;

double orc_tau0(const orc_cfg *c);
double orc_dt(const orc_cfg *c);

int orc_geometry2d(const orc_cfg *c, double cos_t, double sin_t, orc_geo2d *g);
int orc_masters2d(const orc_cfg *c, const orc_geo2d *gn, const orc_geo2d *gnp1,
                  int32_t *master);
int orc_init_maxwellian(const orc_cfg *c, const double *rho, const double *ux,
                        const double *uy, const double *uz, const double *T,
                        double *F);
int orc_moments(const orc_cfg *c, const double *F, double *rho, double *ux,
                double *uy, double *uz, double *T);

/* Heat flux q[3] of one cell's state fk (layout [component][p]) about its own
 * velocity: reduced 2D q = sum (v - u)(|v - u|^2/2 f + g) dv (Eq.
 * MacroscopicDDv), 3D q = sum (v - u)|v - u|^2/2 F dv (Sec. 2.1). */
int orc_heat_flux(const orc_cfg *c, const double *fk, double *q);

/* Equilibrium of the configured collision model for (rho, u[3], T, q[3])
 * on the velocity grid, into one cell's state fk: BGK (Eq. BGKDD, the 3D
 * Maxwellian) or Shakhov (Eq. ShakhovDD in 2D, the 3D form of Sec. 2.1). */
int orc_equilibrium(const orc_cfg *c, double rho, const double *u, double T,
                    const double *q, double *fk);
/* Parameters (rho, u[3], T) of one cell's equilibrium for the configured
 * moments: the direct moments of fk (Eq. MacroscopicDDv), or with
 * c->conservative the root of the discrete conservation equations of
 * Sec. 3.1, found by Newton's method.  out[5] = rho, ux, uy, uz, T;
 * iters (nullable) receives the Newton iterations taken. */
int orc_equilibrium_params(const orc_cfg *c, const double *fk, double *out, int *iters);
int orc_run2d(const orc_cfg *c, double *F, int nsteps, orc_hist *h,
              double *theta_out, double *omega_out);
double orc_mass2d(const orc_cfg *c, const double *F);


/* ------------------------------------------------------------------ 3D */

/* Geometry of the 3D cut cells (reading of the extension of Appendix A that
 * the paper leaves to the reader, Sec. 5): faces carry the 2D virtual-cell
 * area of their four nodes; the wall face closes the polyhedron.  Arrays are
 * caller-owned. */
typedef struct {
    double *phi;      /* (nx+1)(ny+1)(nz+1) nodes, node (a,b,c) at (c*(ny+1)+b)*(nx+1)+a */
    int8_t *type;     /* nx*ny*nz                                                    */
    int8_t *cgas;     /* nx*ny*nz                                                    */
    double *ax;       /* (nx+1)*ny*nz x-faces, face a of (j,k) at (k*ny+j)*(nx+1)+a   */
    double *ay;       /* nx*(ny+1)*nz y-faces, face b of (i,k) at (k*(ny+1)+b)*nx+i   */
    double *az;       /* nx*ny*(nz+1) z-faces, face c of (i,j) at (c*ny+j)*nx+i       */
    double *sw;       /* wall face area                                              */
    double *nwx, *nwy, *nwz;   /* wall normal (towards the solid)                    */
    double *rwx, *rwy, *rwz;   /* wall centre (absolute)                             */
    double *vol;      /* virtual-cell volume                                         */
} orc_geo3d;

int orc_geometry3d(const orc_cfg *c, orc_geo3d *g);
int orc_masters3d(const orc_cfg *c, const orc_geo3d *g, int32_t *master);
int orc_run3d(const orc_cfg *c, double *F, int nsteps, orc_hist *h);
double orc_mass3d(const orc_cfg *c, const double *F);


/* ------------------------------------------------------------ 2D adjoint */

/* Drag J = F_x(F^N) after nsteps fixed-body steps from F0, and its discrete
 * adjoint: lam0 = dJ/dF0 (layout of F), gTw[nseg] (or gTw[0] for a uniform
 * wall) = dJ/dT_w, gbc_s[5 * side cells] = dJ/d(rho, ux, uy, uz, T) of the
 * Maxwellian side s (nullable; zeros for other sides). */
int orc_adjoint2d(const orc_cfg *c, const double *F0, int nsteps, double *J, double *lam0,
                  double *gTw, double *gbc0, double *gbc1, double *gbc2, double *gbc3);
/* The same for J = [with_drag] F_x(F^N) + <seed, F^N> (seed: dJ/dF^N of a
 * linear functional of the state after nsteps steps, layout of F; nullable). */
int orc_adjoint2d_ex(const orc_cfg *c, const double *F0, int nsteps, int with_drag, const double *seed,
                     double *J, double *lam0, double *gTw, double *gbc0, double *gbc1, double *gbc2,
                     double *gbc3);
int orc_init_maxwellian_vjp(const orc_cfg *c, const double *rho, const double *ux,
                            const double *uy, const double *T, const double *lam, double *g);

#endif
