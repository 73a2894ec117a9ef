// Internal declarations of libdvm shared by its CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cstddef>
#include <string>

#include "dvm.h"

namespace dvm {

constexpr int kMaxWalk = 8;          // bound of the master search (Appendix A.3)
constexpr int kBoxMargin = 12;       // cells between the body and the edge of its box
constexpr int kHistCap = 1 << 15;    // steps kept in the force/angle history
constexpr int kMaxMembers = 32;      // virtual cells per control volume
constexpr int kMaxAxisNv = 64;       // velocity points per axis

// cell flag bits
constexpr uint8_t kPlain = 1;        // gas cell alone in its control volume at t^n and t^{n+1}
constexpr uint8_t kZero = 2;         // solid at t^{n+1} and in no control volume: write 0
constexpr uint8_t kSpecial = 4;      // updated by the control-volume kernel
constexpr uint8_t kMaskShift = 4;    // bits 4..7: limiter allowed on faces x-, x+, y-, y+

// device error flag slots
enum { kErrNonphys = 0, kErrGeometry = 1, kErrCapacity = 2, kErrCount = 4 };

// One time level of the 2D geometry (Appendix A), FP64.
struct Geo2D {
    double *phi;      // (nx+1)*(ny+1)
    int8_t *type;     // nc
    int8_t *cgas;     // nc
    double *lx;       // (nx+1)*ny
    double *ly;       // nx*(ny+1)
    double *lw, *nwx, *nwy, *rwx, *rwy, *sbar;   // nc
};

// Rigid-body state on the device (FP64).
struct BodyDev {
    double theta, omega;      // at t^n
    double theta1;            // at t^{n+1}
    double trig[4];           // cos/sin of theta (t^n), cos/sin of theta1
    double F[3], torque;      // at t^n of the last step
};

// Parameters shared by the 2D kernels, passed by value.
struct Grid2D {
    int nx, ny, nvx, nvy, nv;
    double xmin, ymin, dx, dy;
    double vxmin, vymin, dvx, dvy, dv;
    double dt, tau0;
    int bc[4];
    int i0, i1, j0, j1;       // geometry box [i0, i1) x [j0, j1)
};

struct BodyParams {
    int shape, movable, nseg;
    double cx, cy, cz, ra, rb, vbx, vby, mass, inertia, Tw;
    const double *Tw_seg;     // device
    const double *seg_dir;    // device
};

}  // namespace dvm

struct dvm_ctx {
    int dim, nx, ny, nz;
    double xmin, xmax, ymin, ymax, zmin, zmax, dx, dy, dz;
    int nvx, nvy, nvz, nv;
    double vxmin, vxmax, vymin, vymax, vzmin, vzmax, dvx, dvy, dvz;
    double Kn, Lref, cfl, dt, tau0;
    int prec, scheme, ncomp, elem;
    long long nc;
    size_t state_elems;
    cudaStream_t stream;
    bool own_stream;
    int bc[6];
    void *ghost[6];               // device, [side cell][comp][p], state precision
    dvm_body body;
    double *d_Twseg, *d_segdir;
    void *f[2];
    int cur;
    void *mom;                    // [nc][8] state precision: rho ux uy uz T
    dvm::Geo2D geo[2];
    int gcur;
    int32_t *master;
    uint8_t *flags;
    uint8_t *hs;                  // has-slaves marks
    int32_t *spec_list, *wall_list, *counts;   // counts[0] = specials, [1] = walls
    int list_cap;
    double *wphi, *wux, *wuy, *wT;              // per cell, wall data of t^n
    double *wcontrib;             // per box cell: Fx, Fy, torque
    int i0, i1, j0, j1;
    dvm::BodyDev *d_body;
    double *d_hist;               // [kHistCap][6]
    long long steps_done;
    int *d_err;
    int *h_err;                   // pinned
    double *d_scratch;            // nc doubles (mass)
    double *d_out;                // nc*5 doubles (moments output)
    bool have_state, have_geo, need_fusion, moving;
    bool timing;
    void *ev_pool;                // std::vector<cudaEvent_t> of start/stop pairs
    int ev_used;
    long long launches;
};

namespace dvm {

void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);

dvm::Grid2D grid2d(const dvm_ctx *c);
dvm::BodyParams body_params(const dvm_ctx *c);

// geometry (dvm_geometry2d.cu)
cudaError_t geometry2d_level(dvm_ctx *c, int level, const double *d_cos_sin);
cudaError_t masters_flags2d(dvm_ctx *c, bool moving);
cudaError_t init_static_geometry2d(dvm_ctx *c);

// step kernels (dvm_step2d.cu)
cudaError_t moments2d(dvm_ctx *c);
cudaError_t init_maxwellian2d(dvm_ctx *c, const double *d_prim);
cudaError_t step2d(dvm_ctx *c);
cudaError_t mass2d(dvm_ctx *c, double *d_scratch, double *d_out);
cudaError_t moments_out2d(dvm_ctx *c, double *d_out);
cudaError_t ghost2d(dvm_ctx *c, int side, const double *d_prim, int nside);
cudaError_t timing_mark(dvm_ctx *c, int which);   // 0: before, 1: after the bulk kernel

inline double *body_trig(dvm_ctx *c, int which)
{
    return reinterpret_cast<double *>(reinterpret_cast<char *>(c->d_body) + offsetof(BodyDev, trig)) + which;
}

}  // namespace dvm
