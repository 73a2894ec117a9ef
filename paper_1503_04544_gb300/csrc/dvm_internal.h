// Internal declarations of libdvm shared by its CUDA translation units.
//
// Device layout of a distribution (2D, reduced pair f, g):
//   element (cell, comp, p) at ((p / W) * 2 + comp) * slab * W + P(cell) * W + p % W
// with W = 16 bytes / sizeof(T) velocities per group (4 in FP32, 2 in FP64)
// and the velocity count padded to a multiple of W with zero entries.  Each
// (group, component) slab is the cell grid padded by two cells on every side,
// P(i, j) = (j + 2) * (nx + 4) + i + 2; the padding holds the boundary
// condition (Maxwellian ghost states, or periodic images / zero-gradient
// copies that the kernels writing boundary cells keep up to date).  For one
// velocity group the states of consecutive cells are contiguous, so a warp of
// 32 consecutive cells in x reads 512 contiguous bytes, and the velocity
// (hence the upwind direction) is uniform across the warp.  The public layout
// of dvm.h ([cell][comp][p]) is converted on the way in and out.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <cstddef>
#include <string>

#include "dvm.h"

namespace dvm {

constexpr int kMaxWalk = 8;          // bound of the master search (Appendix A.3)
constexpr int kBoxMargin = 12;       // cells between the body and the edge of its box
constexpr int kHistCap = 1 << 15;    // steps kept in the force/angle history
constexpr int kMaxMembers = 16;      // virtual cells per control volume
constexpr int kMaxAxisNv = 64;       // velocity points per axis
constexpr int kRows = 8;             // cell rows per block of the bulk kernel
constexpr int kStages = 5;           // shared-memory stages of the bulk kernel's TMA ring
constexpr int kTileX = 32 + 4;       // tile width with a two-cell halo on each side
constexpr int kTileY = kRows + 4;    // tile height with a two-cell halo
// a stage of both components, 2 x kTileY x kTileX x 16 B, is a multiple of
// 128 B for any kRows: every stage of the bulk kernel's ring is a
// tensor-copy destination on a 128-byte boundary
static_assert((2 * kTileY * kTileX * 16) % 128 == 0, "tensor-copy destinations start on 128-byte boundaries");
constexpr long kWaitLimit = 1L << 20; // bound of every mbarrier wait (polls)

// cell flag bits
constexpr uint8_t kPlain = 1;        // gas cell alone in its control volume at t^n and t^{n+1}
constexpr uint8_t kZero = 2;         // solid at t^{n+1} and in no control volume: write 0
constexpr uint8_t kSpecial = 4;      // updated by the control-volume kernel
constexpr uint8_t kMaskShift = 4;    // bits 4..7: limiter allowed on faces x-, x+, y-, y+

// 3D cell flags (16 bits): kPlain, kZero, kSpecial as in 2D; bits 4..9 allow
// the limiter on the faces x-, x+, y-, y+, z-, z+
constexpr int kMaskShift3 = 4;
constexpr int kMaxMembers3 = 8;      // virtual cells per 3D control volume

// device error flag slots
enum { kErrNonphys = 0, kErrGeometry = 1, kErrCapacity = 2, kErrTimeout = 3, kErrCount = 4 };

// One time level of the 2D geometry (Appendix A), FP64.
struct Geo2D {
    double *phi;      // (nx+1)*(ny+1)
    int8_t *type;     // nc
    int8_t *cgas;     // nc
    double *lx;       // (nx+1)*ny
    double *ly;       // nx*(ny+1)
    double *lw, *nwx, *nwy, *rwx, *rwy, *sbar;   // nc
};

// Geometry of the 3D cut cells (faces from Appendix A applied to each face,
// the wall face closing the polyhedron), FP64.
struct Geo3D {
    double *phi;                       // (nx+1)(ny+1)(nz+1) nodes
    int8_t *type, *cgas;               // nc
    double *ax, *ay, *az;              // (nx+1)ny nz, nx(ny+1)nz, nx ny(nz+1) face areas
    double *sw, *nwx, *nwy, *nwz;      // nc wall face area and normal (into the solid)
    double *rwx, *rwy, *rwz;           // nc wall centre (absolute)
    double *vol;                       // nc virtual-cell volume
};

// Parameters shared by the 3D kernels.  Velocities are grouped by W along
// v_x with the v_x axis padded to nvxp = nxg * W points, so that v_y and v_z
// are uniform within a group; group q covers p1 = (q % nxg) * W + e,
// p2 = (q / nxg) % nvy, p3 = q / (nxg * nvy).
struct Grid3D {
    int nx, ny, nz, nvx, nvy, nvz, nv;
    int W, nvxp, nxg, nvp, ngrp;
    long slab;                // (nx + 4)(ny + 4)(nz + 4)
    double xmin, ymin, zmin, dx, dy, dz;
    double vxmin, vymin, vzmin, dvx, dvy, dvz, dv;
    double dt, tau0, dt_tau0;
    float dv_f, dt_tau0_f;
    int bc[6];
};

// Rigid-body state on the device (FP64).
struct BodyDev {
    double theta, omega;      // at t^n
    double theta1;            // at t^{n+1}
    double trig[4];           // cos/sin of theta (t^n), cos/sin of theta1
    double F[3], torque;      // at t^n of the last step
    long long step;           // steps completed
};

// Parameters shared by the 2D kernels, passed by value.
struct Grid2D {
    int nx, ny, nvx, nvy, nv;
    int W, nvp, ngrp;         // velocities per group, padded count, groups
    long slab;                // cells per slab: (nx + 4) * (ny + 4)
    double xmin, ymin, dx, dy;
    double vxmin, vymin, dvx, dvy, dv;
    double dt, tau0;
    double dt_tau0;           // dt / tau0
    float dv_f, dt_tau0_f;    // FP32 copies for the FP32 kernels
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
    CUtensorMap tmap[2];          // TMA descriptors of the two state buffers (2D or 3D view)
    int dim, nx, ny, nz;
    double xmin, xmax, ymin, ymax, zmin, zmax, dx, dy, dz;
    int nvx, nvy, nvz, nv;
    double vxmin, vxmax, vymin, vymax, vzmin, vzmax, dvx, dvy, dvz;
    double Kn, Lref, cfl, dt, tau0;
    int prec, scheme, ncomp, elem;
    long long nc;
    size_t state_elems;           // public layout: nc * ncomp * nv
    int W, nvp, ngrp;
    long slab;
    size_t dev_elems;             // device layout: ngrp * ncomp * slab * W
    int S;                        // velocity splits of the bulk kernel
    cudaStream_t stream;
    bool own_stream;
    cudaStream_t wstream;         // the wall kernel's stream (concurrent with the bulk kernel)
    cudaEvent_t ev_wfork, ev_wjoin;
    int bc[6];
    dvm_body body;
    double *d_Twseg, *d_segdir;
    void *f[2];
    int cur;
    void *part[2];                // [S][4][nc] partial moment sums, paired with f
    void *vtab;                   // [nvp][8] per-velocity coefficients (state precision)
    void *ptab;                   // [ngrp][7] float4: FP32 coefficients of a group in packed-pair order (2D)
    int8_t *gsign;                // [ngrp][2] sign of v_x, v_y in a group (0: mixed)
    dvm::Geo2D geo[2];
    dvm::Geo3D geo3;              // 3D geometry (fixed obstacle)
    uint16_t *flags3;             // 3D cell flags
    int nvxp, nxg;                // 3D velocity grouping (see Grid3D)
    int gcur;
    int32_t *master;
    uint8_t *flags;
    uint8_t *hs;                  // has-slaves marks
    int32_t *spec_list, *wall_list, *counts;   // counts[0] = specials, [1] = walls
    int32_t *wslot;               // wall slot of each cell, -1 if none
    void *cvinfo;                 // [control volume] CvInfo records (dvm_step2d.cu)
    int list_cap;
    void *wflux;                  // [wall slot][split][8] FP64 partial wall sums
    double *wphi;                 // [wall slot][4] wall density, u_w (2), T_w
    double *wcontrib;             // [wall slot][3] Fx, Fy, torque
    int *ticket;                  // block counter of the wall kernel
    int i0, i1, j0, j1;
    dvm::BodyDev *d_body;
    double *d_hist;               // [kHistCap][6]
    long long steps_done;
    int *d_err;
    int *h_err;                   // pinned
    double *d_scratch;            // nc doubles (mass)
    double *d_out;                // nc*5 doubles (moments output)
    void *d_pub;                  // staging buffer in the public layout
    double *d_bcstate[6];         // (rho, ux, uy, uz, T) per cell of each Maxwellian side
    double *d_prim0;              // primitives of the last dvm_init_maxwellian (nc * 5)
    bool have_prim0;
    void *adj;                    // adjoint workspace (dvm_adjoint2d.cu)
    size_t adj_tape;              // device bytes the adjoint may keep of the forward run's tape (dvm_set_adjoint_tape)
    uint32_t *rec_bits;           // if set, the 2D MUSCL bulk kernel records its limiter branches here
    bool have_state, have_geo, need_fusion, moving;
    int timing;                   // dvm_timing: 0 off, 1 the bulk kernel, 2 the Shakhov kernel
    void *ev_pool;                // std::vector<cudaEvent_t> of start/stop pairs
    int ev_used;
    bool graphs;                  // dvm_step replays two-step CUDA graphs (dvm_graphs)
    int time_scheme;              // DVM_EXPLICIT or DVM_IMEX (dvm_set_time_scheme)
    int model;                    // DVM_BGK or DVM_SHAKHOV (dvm_set_collision_model)
    double Pr;                    // Prandtl number of the Shakhov model
    int eq_mode;                  // DVM_EQ_DIRECT or DVM_EQ_CONSERVATIVE (dvm_set_equilibrium)
    int gnv[3];                   // the whole velocity grid: points, first velocity and step per axis
    double gv0[3], gdv[3];        //   (this context's own grid unless a velocity split is set)
    bool split;                   // dvm_set_velocity_split: steps through dvm_split_begin / _finish
    bool split_begun;             // dvm_split_begin done, dvm_split_finish pending
    bool split_relax;             // semi-implicit split step: transported, waiting for dvm_split_relax
    void *split_in;               // [4 or 5][nc] summed moment sums in the state precision (velocity split)
    void *qheat;                  // [D][nc] heat flux of each cell's control volume at t^n (Shakhov, state precision)
    void *hpart[2];               // 2D Shakhov, paired with part[]: raw heat-flux moments [S][5][nc] of the state
                                  // about a reference velocity [2][nc] per cell, written by the step that made it
    bool hvalid;                  // hpart[cur] belongs to f[cur] (else the step starts with k_heatflux)
    bool dt_given;                // dt came from dvm_physics, not from the CFL rule
    void *eqp;                    // [dim + 2][nc] conservative equilibrium parameters (state precision)
    void *snap_f, *snap_part;     // dvm_step: state and moment sums at the last checked step
    void *snap_scratch;           // dvm_step: moment sums of the state check
    void *snap_body;              // dvm_step: rigid-body record at the last checked step
    bool rollback_off;            // dvm_rollback(ctx, 0): dvm_step without snapshots
    void *gretired;               // std::vector<cudaGraphExec_t> launched, destroyed once the stream is idle
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
cudaError_t tables2d(dvm_ctx *c);
cudaError_t partials_from_state2d(dvm_ctx *c);
cudaError_t init_maxwellian2d(dvm_ctx *c, const double *d_prim);
cudaError_t step2d(dvm_ctx *c);
cudaError_t heatflux2d(dvm_ctx *c, const void *f, const void *part);
cudaError_t heatflux3d(dvm_ctx *c, const void *f, const void *part);   // [3][nc] heat flux into qheat (dvm_shakhov3d.cu)   // heat flux of F^n for the Shakhov step (dvm_shakhov2d.cu)
cudaError_t eqpar(dvm_ctx *c, const void *part, int S);         // conservative equilibrium parameters into c->eqp (dvm_equilibrium.cu)
cudaError_t split_step2d(dvm_ctx *c, int phase, void *xbuf);    // velocity split: 1 begin, 2 finish (dvm_step2d.cu)
cudaError_t split_step3d(dvm_ctx *c, int phase, void *xbuf);    // the same in 3D (dvm_step3d.cu)
cudaError_t fusion2d(dvm_ctx *c, void *f, void *part);          // Eq. FusionDD on a buffer
cudaError_t mass2d(dvm_ctx *c, double *d_scratch, double *d_out);
cudaError_t moments_out2d(dvm_ctx *c, double *d_out);
cudaError_t ghost2d(dvm_ctx *c, int side, const double *d_prim, int nside);
cudaError_t pack2d(dvm_ctx *c, const void *pub, void *dev);      // public -> device layout
cudaError_t unpack2d(dvm_ctx *c, const void *dev, void *pub);    // device -> public layout
cudaError_t zero_solid2d(dvm_ctx *c);                            // both state buffers
cudaError_t halo2d(dvm_ctx *c, int buf);                         // periodic / zero-gradient padding
cudaError_t members2d(dvm_ctx *c, bool moving);                  // control-volume records
cudaError_t timing_mark(dvm_ctx *c, int which);   // 0: before, 1: after the bulk kernel
cudaError_t timing_mark_kernel(dvm_ctx *c, int kernel, int which);   // the same for kernel 1 (bulk) or 2 (Shakhov)
int make_tensor_maps2d(dvm_ctx *c);                // TMA descriptors of f[0], f[1]
int encode_tensor_map2d(dvm_ctx *c, void *buf, CUtensorMap *map);
int encode_bits_map2d(dvm_ctx *c, void *buf, CUtensorMap *map);  // limiter-branch words (bits_pitch rows)
// adjoint (dvm_adjoint2d.cu)
int drag_adjoint2d(dvm_ctx *c, int nsteps, int K, double *J, double *gTw, double *const *gbc, double *gprim0,
                   double *ms_forward, double *ms_reverse, int with_drag, const void *seed, int seed_dev, void *lam0,
                   int lam0_dev);
void free_adjoint2d(dvm_ctx *c);
void trim_adjoint_tape2d(dvm_ctx *c, size_t max_bytes);   // frees kept tape buffers beyond max_bytes

// 3D (dvm_geometry3d.cu, dvm_step3d.cu)
dvm::Grid3D grid3d(const dvm_ctx *c);
cudaError_t init_static_geometry3d(dvm_ctx *c);
cudaError_t geometry3d(dvm_ctx *c);
cudaError_t masters_flags3d(dvm_ctx *c);
cudaError_t members3d(dvm_ctx *c);
cudaError_t tables3d(dvm_ctx *c);
cudaError_t partials_from_state3d(dvm_ctx *c);
cudaError_t init_maxwellian3d(dvm_ctx *c, const double *d_prim);
cudaError_t step3d(dvm_ctx *c);
cudaError_t mass3d(dvm_ctx *c, double *d_scratch, double *d_out);
cudaError_t moments_out3d(dvm_ctx *c, double *d_out);
cudaError_t ghost3d(dvm_ctx *c, int side, const double *d_prim, int nside);
cudaError_t pack3d(dvm_ctx *c, const void *pub, void *dev);
cudaError_t unpack3d(dvm_ctx *c, const void *dev, void *pub);
cudaError_t zero_solid3d(dvm_ctx *c);
cudaError_t halo3d(dvm_ctx *c, int buf);
size_t vtab3_bytes(const dvm_ctx *c);
int make_tensor_maps3d(dvm_ctx *c);                // TMA descriptors of f[0], f[1] (3D)
size_t cvinfo3_bytes();

// Limiter-branch words of the 2D MUSCL step (recorded for the adjoint): one
// uint32 per (velocity group, padded cell) with the row pitch rounded up to
// a multiple of 4 words (16-byte rows for TMA).
inline int bits_pitch(const dvm_ctx *c) { return (c->nx + 4 + 3) & ~3; }
inline long bits_slab(const dvm_ctx *c) { return (long)bits_pitch(c) * (c->ny + 4); }

inline double *body_trig(dvm_ctx *c, int which)
{
    return reinterpret_cast<double *>(reinterpret_cast<char *>(c->d_body) + offsetof(BodyDev, trig)) + which;
}

}  // namespace dvm
