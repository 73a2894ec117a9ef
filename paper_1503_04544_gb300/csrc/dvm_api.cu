// C-ABI of libdvm: context management, set-up, stepping and read-back.
// Every entry point returns a dvm_status and records a thread-local message.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dvm_internal.h"

namespace dvm {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *where)
{
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DVM_ERR_OOM : DVM_ERR_CUDA;
}

cudaError_t timing_mark(dvm_ctx *c, int which) { return timing_mark_kernel(c, 1, which); }

cudaError_t timing_mark_kernel(dvm_ctx *c, int kernel, int which)
{
    if (c->timing != kernel) return cudaSuccess;
    auto *pool = static_cast<std::vector<cudaEvent_t> *>(c->ev_pool);
    const size_t need = 2 * (size_t)(c->ev_used + 1);
    while (pool->size() < need) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        pool->push_back(e);
    }
    cudaError_t err = cudaEventRecord((*pool)[2 * c->ev_used + which], c->stream);
    if (which == 1) c->ev_used++;
    return err;
}

Grid2D grid2d(const dvm_ctx *c)
{
    Grid2D g;
    g.nx = c->nx; g.ny = c->ny; g.nvx = c->nvx; g.nvy = c->nvy; g.nv = c->nv;
    g.W = c->W; g.nvp = c->nvp; g.ngrp = c->ngrp; g.slab = c->slab;
    g.xmin = c->xmin; g.ymin = c->ymin; g.dx = c->dx; g.dy = c->dy;
    g.vxmin = c->vxmin; g.vymin = c->vymin; g.dvx = c->dvx; g.dvy = c->dvy;
    g.dv = c->dvx * c->dvy;
    g.dt = c->dt; g.tau0 = c->tau0;
    g.dt_tau0 = c->dt / c->tau0;
    g.dv_f = (float)g.dv;
    g.dt_tau0_f = (float)g.dt_tau0;
    for (int s = 0; s < 4; ++s) g.bc[s] = c->bc[s];
    g.i0 = c->i0; g.i1 = c->i1; g.j0 = c->j0; g.j1 = c->j1;
    return g;
}

Grid3D grid3d(const dvm_ctx *c)
{
    Grid3D g;
    g.nx = c->nx; g.ny = c->ny; g.nz = c->nz;
    g.nvx = c->nvx; g.nvy = c->nvy; g.nvz = c->nvz; g.nv = c->nv;
    g.W = c->W; g.nvxp = c->nvxp; g.nxg = c->nxg; g.nvp = c->nvp; g.ngrp = c->ngrp;
    g.slab = c->slab;
    g.xmin = c->xmin; g.ymin = c->ymin; g.zmin = c->zmin; g.dx = c->dx; g.dy = c->dy; g.dz = c->dz;
    g.vxmin = c->vxmin; g.vymin = c->vymin; g.vzmin = c->vzmin;
    g.dvx = c->dvx; g.dvy = c->dvy; g.dvz = c->dvz;
    g.dv = c->dvx * c->dvy * c->dvz;
    g.dt = c->dt; g.tau0 = c->tau0;
    g.dt_tau0 = c->dt / c->tau0;
    g.dv_f = (float)g.dv;
    g.dt_tau0_f = (float)g.dt_tau0;
    for (int s = 0; s < 6; ++s) g.bc[s] = c->bc[s];
    return g;
}

BodyParams body_params(const dvm_ctx *c)
{
    BodyParams b;
    b.shape = c->body.shape; b.movable = c->body.movable; b.nseg = c->body.nseg;
    b.cx = c->body.cx; b.cy = c->body.cy; b.cz = c->body.cz; b.ra = c->body.ra; b.rb = c->body.rb;
    b.vbx = c->body.vbx; b.vby = c->body.vby; b.mass = c->body.mass; b.inertia = c->body.inertia;
    b.Tw = c->body.Tw; b.Tw_seg = c->d_Twseg; b.seg_dir = c->d_segdir;
    return b;
}

size_t vcoef_bytes(int prec);
size_t cvinfo_bytes();

}  // namespace dvm

using namespace dvm;

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

static double axis_vmax(int n, double vmin, double vmax)
{
    double dv = (vmax - vmin) / n;
    double a = std::fabs(vmin), b = std::fabs(vmin + (n - 1) * dv);
    return a > b ? a : b;
}

static int side_cells(const dvm_ctx *c, int side)
{
    if (c->dim == 2) return side < 2 ? c->ny : c->nx;
    if (side < 2) return c->ny * c->nz;
    if (side < 4) return c->nx * c->nz;
    return c->nx * c->ny;
}

template <typename P> static cudaError_t dalloc(P **p, size_t bytes)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)p, bytes > 0 ? bytes : 16);
    return e;
}

static void free_geo(dvm::Geo2D &G)
{
    cudaFree(G.phi); cudaFree(G.type); cudaFree(G.cgas); cudaFree(G.lx); cudaFree(G.ly);
    cudaFree(G.lw); cudaFree(G.nwx); cudaFree(G.nwy); cudaFree(G.rwx); cudaFree(G.rwy);
    cudaFree(G.sbar);
    std::memset(&G, 0, sizeof(G));
}

static void free_geo3(dvm::Geo3D &G)
{
    cudaFree(G.phi); cudaFree(G.type); cudaFree(G.cgas); cudaFree(G.ax); cudaFree(G.ay); cudaFree(G.az);
    cudaFree(G.sw); cudaFree(G.nwx); cudaFree(G.nwy); cudaFree(G.nwz);
    cudaFree(G.rwx); cudaFree(G.rwy); cudaFree(G.rwz); cudaFree(G.vol);
    std::memset(&G, 0, sizeof(G));
}

// Executable graphs of finished dvm_step calls, destroyed once the stream has
// been synchronised (their launches have completed).
static void destroy_retired(dvm_ctx *c)
{
    auto *v = static_cast<std::vector<cudaGraphExec_t> *>(c->gretired);
    if (!v) return;
    for (cudaGraphExec_t x : *v) cudaGraphExecDestroy(x);
    v->clear();
}

static int check_flags(dvm_ctx *c)
{
    CK(cudaMemcpyAsync(c->h_err, c->d_err, kErrCount * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    destroy_retired(c);
    int rc = DVM_OK;
    if (c->h_err[kErrGeometry]) { set_error("geometry: saddle cell or master search left its bounds"); rc = DVM_ERR_GEOMETRY; }
    else if (c->h_err[kErrCapacity]) { set_error("geometry: control-volume list or member capacity exceeded"); rc = DVM_ERR_GEOMETRY; }
    else if (c->h_err[kErrNonphys]) { set_error("non-positive density or temperature"); rc = DVM_ERR_NONPHYSICAL; }
    else if (c->h_err[kErrTimeout]) { set_error("a bounded wait on a TMA transfer timed out"); rc = DVM_ERR_CUDA; }
    if (rc != DVM_OK) {
        // report once: the flags are cleared so that the context stays usable
        CK(cudaMemsetAsync(c->d_err, 0, kErrCount * sizeof(int), c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return rc;
}

// Dimension dispatch of the state services.
static cudaError_t st_ghost(dvm_ctx *c, int side, const double *d, int n)
{ return c->dim == 2 ? ghost2d(c, side, d, n) : ghost3d(c, side, d, n); }
static cudaError_t st_halo(dvm_ctx *c, int buf) { return c->dim == 2 ? halo2d(c, buf) : halo3d(c, buf); }
static cudaError_t st_zero_solid(dvm_ctx *c) { return c->dim == 2 ? zero_solid2d(c) : zero_solid3d(c); }
static cudaError_t st_partials(dvm_ctx *c) { return c->dim == 2 ? partials_from_state2d(c) : partials_from_state3d(c); }
static cudaError_t st_pack(dvm_ctx *c, const void *pub, void *dev) { return c->dim == 2 ? pack2d(c, pub, dev) : pack3d(c, pub, dev); }
static cudaError_t st_unpack(dvm_ctx *c, const void *dev, void *pub) { return c->dim == 2 ? unpack2d(c, dev, pub) : unpack3d(c, dev, pub); }
namespace dvm {
cudaError_t shakhov3d(dvm_ctx *c);   // the Shakhov term of the 3D step (dvm_shakhov3d.cu)
}

// One time step; with the Shakhov model its relaxation term follows the
// step (Eq. ShakhovDD in 2D, the form of Sec. 2.1 in 3D).
static cudaError_t st_step(dvm_ctx *c)
{
    cudaError_t e = c->dim == 2 ? step2d(c) : step3d(c);
    // the 2D step and the FP32 3D step relax towards the Shakhov equilibrium
    // themselves; the FP64 3D explicit step adds the Shakhov term after the
    // step; the semi-implicit schemes relax towards it in their relaxation
    // kernels
    if (e == cudaSuccess && c->model == DVM_SHAKHOV && c->time_scheme == DVM_EXPLICIT && c->dim == 3 &&
        c->prec == DVM_FP64)
        e = shakhov3d(c);
    return e;
}

// Why the Shakhov model cannot run on this context (nullptr: it can).
static const char *shakhov_unsupported(const dvm_ctx *c)
{
    if (c->split) return "Shakhov model: not with a velocity split (the heat flux needs its own exchange)";
    if (c->eq_mode != DVM_EQ_DIRECT) return "Shakhov model: the direct moments only (the conservative equilibrium is BGK)";
    return nullptr;
}

constexpr int kGraphMinSteps = 8;    // shorter runs are not worth a capture
constexpr size_t kGraphKeep = 64;    // launched graphs kept before a release

// `pairs` replays of a captured pair of steps.  A step writes the other state
// buffer (and, for a moving body, the other geometry level), so two steps
// leave the context's buffers as they found them and the pair replays as it
// is: one graph launch per two steps in place of their kernel launches and
// the gaps between them.  The capture advances the host bookkeeping of two
// steps that have not run (step and launch counts); it is put back and
// advanced per replay.  *done is the number of steps enqueued: 0 when the
// stream cannot be captured, the caller then steps launch by launch.
static cudaError_t graph_steps(dvm_ctx *c, int pairs, int *done)
{
    *done = 0;
    // a caller that never checks the flags would keep every launched graph:
    // past kGraphKeep of them, wait for the stream once and release them
    if (static_cast<std::vector<cudaGraphExec_t> *>(c->gretired)->size() >= kGraphKeep) {
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
        destroy_retired(c);
    }
    const long long steps0 = c->steps_done, launches0 = c->launches;
    const bool hvalid0 = c->hvalid;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    cudaError_t es = st_step(c);
    if (es == cudaSuccess) es = st_step(c);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
    const long long dl = c->launches - launches0;
    c->steps_done = steps0;
    c->launches = launches0;
    cudaGraphExec_t exec = nullptr;
    // the kernel nodes keep their own launch priorities (the bulk kernel's)
    const bool ok = es == cudaSuccess && ee == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        // not capturable here: nothing was enqueued, step launch by launch
        c->hvalid = hvalid0;
        cudaGetLastError();
        return cudaSuccess;
    }
    // destroyed once the stream has been synchronised
    static_cast<std::vector<cudaGraphExec_t> *>(c->gretired)->push_back(exec);
    for (int r = 0; r < pairs; ++r) {
        const cudaError_t e = cudaGraphLaunch(exec, c->stream);
        if (e != cudaSuccess) return e;
        c->steps_done += 2;
        c->launches += dl;
        *done += 2;
    }
    return cudaSuccess;
}
static cudaError_t st_moments(dvm_ctx *c, double *d) { return c->dim == 2 ? moments_out2d(c, d) : moments_out3d(c, d); }
static cudaError_t st_mass(dvm_ctx *c, double *s, double *d) { return c->dim == 2 ? mass2d(c, s, d) : mass3d(c, s, d); }
static cudaError_t st_init(dvm_ctx *c, const double *d) { return c->dim == 2 ? init_maxwellian2d(c, d) : init_maxwellian3d(c, d); }
static cudaError_t st_flags(dvm_ctx *c) { return c->dim == 2 ? masters_flags2d(c, false) : masters_flags3d(c); }

extern "C" {

const char *dvm_last_error(void) { return g_last_error.c_str(); }

int dvm_create(const dvm_grid *grid, const dvm_vgrid *vg, const dvm_physics *ph, int precision,
               int scheme, void *stream, dvm_ctx **out)
{
    if (!grid || !vg || !ph || !out) { set_error("null argument"); return DVM_ERR_ARG; }
    *out = nullptr;
    const int dim = grid->dim;
    if (dim != 2 && dim != 3) { set_error("dim must be 2 or 3"); return DVM_ERR_ARG; }
    if (grid->nx < 4 || grid->ny < 4 || (dim == 3 && grid->nz < 4) || vg->nvx < 1 || vg->nvy < 1 ||
        (dim == 3 && vg->nvz < 1)) {
        set_error("grid sizes: at least 4 cells per axis and one velocity"); return DVM_ERR_ARG;
    }
    if (vg->nvx > kMaxAxisNv || vg->nvy > kMaxAxisNv || (dim == 3 && vg->nvz > kMaxAxisNv)) {
        set_error("at most 64 velocities per axis"); return DVM_ERR_ARG;
    }
    if (precision != DVM_FP32 && precision != DVM_FP64) { set_error("precision must be 32 or 64"); return DVM_ERR_ARG; }
    if (scheme != DVM_UPWIND && scheme != DVM_MUSCL) { set_error("scheme"); return DVM_ERR_ARG; }
    if (!(grid->xmax > grid->xmin) || !(grid->ymax > grid->ymin) || !(vg->vxmax > vg->vxmin) ||
        !(vg->vymax > vg->vymin) || !(ph->Kn > 0) || !(ph->Lref > 0) ||
        (dim == 3 && (!(grid->zmax > grid->zmin) || !(vg->vzmax > vg->vzmin)))) {
        set_error("empty box, velocity window or non-positive Kn/Lref"); return DVM_ERR_ARG;
    }
    if (dim == 3 && (double)(grid->nx + 4) * (grid->ny + 4) * (grid->nz + 4) > 2.0e9) {
        set_error("3D grid too large for 32-bit slab indices"); return DVM_ERR_ARG;
    }
    if (dim == 2 && (double)(grid->nx + 4) * (grid->ny + 4) > 2.0e9) {
        set_error("2D grid too large for 32-bit slab indices"); return DVM_ERR_ARG;
    }
    dvm_ctx *c = new (std::nothrow) dvm_ctx();
    if (!c) { set_error("host allocation"); return DVM_ERR_OOM; }
    std::memset((void *)c, 0, sizeof(*c));
    c->dim = dim; c->nx = grid->nx; c->ny = grid->ny; c->nz = dim == 3 ? grid->nz : 1;
    c->xmin = grid->xmin; c->xmax = grid->xmax; c->ymin = grid->ymin; c->ymax = grid->ymax;
    c->zmin = grid->zmin; c->zmax = grid->zmax;
    c->dx = (c->xmax - c->xmin) / c->nx;
    c->dy = (c->ymax - c->ymin) / c->ny;
    c->dz = dim == 3 ? (c->zmax - c->zmin) / c->nz : 1.0;
    c->nvx = vg->nvx; c->nvy = vg->nvy; c->nvz = dim == 3 ? vg->nvz : 1;
    c->nv = c->nvx * c->nvy * c->nvz;
    c->vxmin = vg->vxmin; c->vxmax = vg->vxmax; c->vymin = vg->vymin; c->vymax = vg->vymax;
    c->vzmin = vg->vzmin; c->vzmax = vg->vzmax;
    c->dvx = (c->vxmax - c->vxmin) / c->nvx;
    c->dvy = (c->vymax - c->vymin) / c->nvy;
    c->dvz = dim == 3 ? (c->vzmax - c->vzmin) / c->nvz : 1.0;
    c->Kn = ph->Kn; c->Lref = ph->Lref; c->cfl = ph->cfl;
    // tau = sqrt(pi)/2 (rho0/rho) Kn L / sqrt(2 R T0), Sec. 5, R = T0 = rho0 = 1
    c->tau0 = std::sqrt(M_PI) / 2.0 * c->Kn * c->Lref / std::sqrt(2.0);
    c->dt_given = ph->dt > 0;
    if (ph->dt > 0) c->dt = ph->dt;
    else {
        double s = axis_vmax(c->nvx, c->vxmin, c->vxmax) / c->dx + axis_vmax(c->nvy, c->vymin, c->vymax) / c->dy;
        if (dim == 3) s += axis_vmax(c->nvz, c->vzmin, c->vzmax) / c->dz;
        c->dt = c->cfl / s;
    }
    if (!(c->dt > 0)) { delete c; set_error("time step"); return DVM_ERR_CFL; }
    c->prec = precision; c->scheme = scheme; c->ncomp = dim == 2 ? 2 : 1;
    c->elem = precision == DVM_FP32 ? 4 : 8;
    c->nc = (long long)c->nx * c->ny * c->nz;
    c->state_elems = (size_t)c->nc * c->ncomp * c->nv;
    c->W = 16 / c->elem;
    if (dim == 2) {
        c->nvp = (c->nv + c->W - 1) / c->W * c->W;
        c->ngrp = c->nvp / c->W;
        c->slab = (long)(c->nx + 4) * (c->ny + 4);
    } else {
        c->nvxp = (c->nvx + c->W - 1) / c->W * c->W;
        c->nxg = c->nvxp / c->W;
        c->nvp = c->nvxp * c->nvy * c->nvz;
        c->ngrp = c->nvp / c->W;
        c->slab = (long)(c->nx + 4) * (c->ny + 4) * (c->nz + 4);
    }
    c->dev_elems = (size_t)c->ngrp * c->ncomp * c->slab * c->W;
    if (dim == 2) {
        // velocity splits: the count that minimises the load of the busiest
        // SM, ceil(blocks / 152) blocks of (groups per split + 5) group
        // times each (5: the per-block prologue and pipeline fill, fitted
        // to measured bulk times); ties go to the smaller count
        const long blocks = (long)((c->nx + 31) / 32) * ((c->ny + kRows - 1) / kRows);
        int S = 1;
        long best = -1;
        for (int s = 1; s <= 16 && s <= c->ngrp; ++s) {
            const long per_sm = (blocks * s + 151) / 152;
            const long cost = per_sm * ((c->ngrp + s - 1) / s + 5);
            if (best < 0 || cost < best) { best = cost; S = s; }
        }
        c->S = S;
    } else {
        // one resident block per SM (tiles of 32 x 11 cells in FP32, 32 x 8 in
        // FP64, columns of 4 cells): the smallest split count giving at least
        // four waves on 152 SMs with a last wave at least 95% full, else the
        // best-filled count up to 24
        const long slots = 152;
        const int rows = precision == DVM_FP32 ? 11 : 8;
        const long blocks = (long)((c->nx + 31) / 32) * ((c->ny + rows - 1) / rows) * ((c->nz + 3) / 4);
        int best = 1;
        double best_eff = 0;
        for (int S = 1; S <= 24 && S <= c->ngrp; ++S) {
            const long nb = blocks * S, waves = (nb + slots - 1) / slots;
            const double eff = (double)nb / ((double)slots * waves);
            if (waves >= 4 && eff >= 0.95) { best = S; break; }
            if (eff > best_eff + 1e-9) { best_eff = eff; best = S; }
        }
        c->S = best;
    }
    const int nmom = dim == 2 ? 4 : 5;
    // the whole velocity grid is this context's own until a velocity split
    c->gnv[0] = c->nvx; c->gnv[1] = c->nvy; c->gnv[2] = dim == 3 ? c->nvz : 1;
    c->gv0[0] = c->vxmin; c->gv0[1] = c->vymin; c->gv0[2] = c->vzmin;
    c->gdv[0] = c->dvx; c->gdv[1] = c->dvy; c->gdv[2] = dim == 3 ? c->dvz : 1.0;
    {
        cudaError_t e = cudaStreamCreateWithFlags(&c->wstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_wfork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_wjoin, cudaEventDisableTiming);
        if (e != cudaSuccess) { delete c; return cuda_fail(e, "wall stream"); }
    }
    if (stream) { c->stream = (cudaStream_t)stream; c->own_stream = false; }
    else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaStreamCreate"); }
        c->own_stream = true;
    }
    for (int s = 0; s < 6; ++s) c->bc[s] = DVM_BC_PERIODIC;
    c->body.shape = DVM_SHAPE_NONE;
    c->i0 = c->i1 = c->j0 = c->j1 = 0;
    const size_t nc = (size_t)c->nc;
    cudaError_t e = cudaSuccess;
#define AL(p, b) if (e == cudaSuccess) e = dalloc(&(p), (b))
    AL(c->f[0], c->dev_elems * c->elem);
    AL(c->f[1], c->dev_elems * c->elem);
    AL(c->part[0], (size_t)c->S * nmom * nc * c->elem);
    AL(c->part[1], (size_t)c->S * nmom * nc * c->elem);
    AL(c->wslot, sizeof(int32_t) * nc);
    AL(c->ticket, sizeof(int));
    if (dim == 2) {
        AL(c->vtab, (size_t)c->nvp * vcoef_bytes(c->prec));
        AL(c->gsign, (size_t)2 * c->ngrp);
        AL(c->ptab, (size_t)c->ngrp * 7 * 16);
        for (int l = 0; l < 2; ++l) {
            dvm::Geo2D &G = c->geo[l];
            AL(G.phi, sizeof(double) * (c->nx + 1) * (c->ny + 1));
            AL(G.type, nc); AL(G.cgas, nc);
            AL(G.lx, sizeof(double) * (c->nx + 1) * c->ny);
            AL(G.ly, sizeof(double) * c->nx * (c->ny + 1));
            AL(G.lw, sizeof(double) * nc); AL(G.nwx, sizeof(double) * nc); AL(G.nwy, sizeof(double) * nc);
            AL(G.rwx, sizeof(double) * nc); AL(G.rwy, sizeof(double) * nc); AL(G.sbar, sizeof(double) * nc);
        }
        AL(c->flags, nc);
    } else {
        AL(c->vtab, vtab3_bytes(c));
        dvm::Geo3D &G = c->geo3;
        AL(G.phi, sizeof(double) * (c->nx + 1) * (c->ny + 1) * (size_t)(c->nz + 1));
        AL(G.type, nc); AL(G.cgas, nc);
        AL(G.ax, sizeof(double) * (c->nx + 1) * (size_t)c->ny * c->nz);
        AL(G.ay, sizeof(double) * c->nx * (size_t)(c->ny + 1) * c->nz);
        AL(G.az, sizeof(double) * c->nx * (size_t)c->ny * (c->nz + 1));
        AL(G.sw, sizeof(double) * nc); AL(G.nwx, sizeof(double) * nc); AL(G.nwy, sizeof(double) * nc);
        AL(G.nwz, sizeof(double) * nc); AL(G.rwx, sizeof(double) * nc); AL(G.rwy, sizeof(double) * nc);
        AL(G.rwz, sizeof(double) * nc); AL(G.vol, sizeof(double) * nc);
        AL(c->flags3, sizeof(uint16_t) * nc);
    }
    AL(c->master, sizeof(int32_t) * nc);
    AL(c->hs, nc);
    AL(c->counts, sizeof(int32_t) * 4);
    AL(c->d_body, sizeof(dvm::BodyDev));
    AL(c->d_hist, sizeof(double) * 6 * kHistCap);
    AL(c->d_err, sizeof(int) * kErrCount);
    AL(c->d_scratch, sizeof(double) * nc);
    AL(c->d_out, sizeof(double) * nc * 5);
#undef AL
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_err, sizeof(int) * kErrCount);
    if (e != cudaSuccess) { int rc = cuda_fail(e, "dvm_create allocation"); dvm_destroy(c); return rc; }
    cudaMemsetAsync(c->f[0], 0, c->dev_elems * c->elem, c->stream);
    cudaMemsetAsync(c->f[1], 0, c->dev_elems * c->elem, c->stream);
    cudaMemsetAsync(c->part[0], 0, (size_t)c->S * nmom * nc * c->elem, c->stream);
    cudaMemsetAsync(c->part[1], 0, (size_t)c->S * nmom * nc * c->elem, c->stream);
    cudaMemsetAsync(c->ticket, 0, sizeof(int), c->stream);
    cudaMemsetAsync(c->d_err, 0, sizeof(int) * kErrCount, c->stream);
    cudaMemsetAsync(c->d_body, 0, sizeof(dvm::BodyDev), c->stream);
    cudaMemsetAsync(c->d_hist, 0, sizeof(double) * 6 * kHistCap, c->stream);
    cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * 4, c->stream);
    if (dim == 2) {
        int rc = make_tensor_maps2d(c);
        if (rc != DVM_OK) { dvm_destroy(c); return rc; }
        e = init_static_geometry2d(c);
        if (e == cudaSuccess) e = tables2d(c);
    } else {
        int rc = make_tensor_maps3d(c);
        if (rc != DVM_OK) { dvm_destroy(c); return rc; }
        e = init_static_geometry3d(c);
        if (e == cudaSuccess) e = tables3d(c);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { int rc = cuda_fail(e, "dvm_create init"); dvm_destroy(c); return rc; }
    c->have_geo = true;
    c->ev_pool = new (std::nothrow) std::vector<cudaEvent_t>();
    c->gretired = new (std::nothrow) std::vector<cudaGraphExec_t>();
    c->graphs = true;
    if (!c->ev_pool || !c->gretired) { dvm_destroy(c); set_error("host allocation"); return DVM_ERR_OOM; }
    *out = c;
    return DVM_OK;
}

void dvm_destroy(dvm_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->f[0]); cudaFree(c->f[1]); cudaFree(c->part[0]); cudaFree(c->part[1]);
    cudaFree(c->vtab); cudaFree(c->ptab); cudaFree(c->gsign); cudaFree(c->wslot); cudaFree(c->ticket);
    cudaFree(c->wflux); cudaFree(c->d_pub);
    for (int l = 0; l < 2; ++l) free_geo(c->geo[l]);
    free_geo3(c->geo3);
    cudaFree(c->flags3);
    cudaFree(c->master); cudaFree(c->flags); cudaFree(c->hs);
    cudaFree(c->spec_list); cudaFree(c->wall_list); cudaFree(c->counts);
    cudaFree(c->wphi); cudaFree(c->wcontrib); cudaFree(c->cvinfo);
    cudaFree(c->d_body); cudaFree(c->d_hist); cudaFree(c->d_err);
    cudaFree(c->d_scratch); cudaFree(c->d_out); cudaFree(c->eqp); cudaFree(c->split_in); cudaFree(c->qheat);
    cudaFree(c->hpart[0]); cudaFree(c->hpart[1]);
    cudaFree(c->d_Twseg); cudaFree(c->d_segdir);
    for (int s = 0; s < 6; ++s) cudaFree(c->d_bcstate[s]);
    cudaFree(c->d_prim0);
    cudaFree(c->snap_f); cudaFree(c->snap_part); cudaFree(c->snap_scratch); cudaFree(c->snap_body);
    free_adjoint2d(c);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->gretired) {
        destroy_retired(c);
        delete static_cast<std::vector<cudaGraphExec_t> *>(c->gretired);
    }
    if (c->ev_pool) {
        auto *pool = static_cast<std::vector<cudaEvent_t> *>(c->ev_pool);
        for (cudaEvent_t e : *pool) cudaEventDestroy(e);
        delete pool;
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->ev_wfork) cudaEventDestroy(c->ev_wfork);
    if (c->ev_wjoin) cudaEventDestroy(c->ev_wjoin);
    if (c->wstream) cudaStreamDestroy(c->wstream);
    delete c;
}

int dvm_set_bc(dvm_ctx *c, int side, int kind, const double *state)
{
    if (!c || side < 0 || side >= 2 * c->dim) { set_error("side"); return DVM_ERR_ARG; }
    if (kind != DVM_BC_PERIODIC && kind != DVM_BC_MAXWELLIAN && kind != DVM_BC_ZEROGRAD) { set_error("kind"); return DVM_ERR_ARG; }
    if (kind == DVM_BC_MAXWELLIAN && !state) { set_error("Maxwellian side needs a state"); return DVM_ERR_ARG; }
    const int n = side_cells(c, side);
    if (kind == DVM_BC_MAXWELLIAN) {
        for (int q = 0; q < n; ++q)
            if (!(state[5 * q] > 0) || !(state[5 * q + 4] > 0)) { set_error("Maxwellian side: rho and T must be > 0"); return DVM_ERR_ARG; }
        // the side states stay on the device (the adjoint differentiates them)
        if (!c->d_bcstate[side]) CK(cudaMalloc(&c->d_bcstate[side], sizeof(double) * 5 * n));
        double *d = c->d_bcstate[side];
        cudaError_t e = cudaMemcpyAsync(d, state, sizeof(double) * 5 * n, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = st_ghost(c, side, d, n);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "dvm_set_bc");
    }
    c->bc[side] = kind;
    if (c->have_state) CK(st_halo(c, c->cur));
    // flags depend on the periodicity of the sides through the limiter masks
    if (c->body.shape != DVM_SHAPE_NONE) {
        cudaError_t e = st_flags(c);
        if (e != cudaSuccess) return cuda_fail(e, "dvm_set_bc flags");
        return check_flags(c);
    }
    return DVM_OK;
}

static int set_body3d(dvm_ctx *c, const dvm_body *b)
{
    if (b->shape != DVM_SHAPE_NONE && b->shape != DVM_SHAPE_SPHERE) {
        set_error("3D shapes: none, sphere"); return DVM_ERR_UNSUPPORTED;
    }
    if (b->shape != DVM_SHAPE_NONE && !(b->ra > 0)) { set_error("body size"); return DVM_ERR_ARG; }
    if (b->movable) { set_error("3D obstacles are fixed in this library version"); return DVM_ERR_UNSUPPORTED; }
    if (b->nseg > 0) { set_error("per-sector wall temperatures are 2D only"); return DVM_ERR_UNSUPPORTED; }
    c->body = *b;
    c->body.Tw_seg = nullptr; c->body.seg_dir = nullptr;
    c->moving = false;
    // list capacity: the cells of the box around the sphere (with margin)
    long nbox = 1;
    if (b->shape != DVM_SHAPE_NONE) {
        auto span = [](double cc, double R, double vmin, double h, int n) {
            int lo = (int)std::floor((cc - R - vmin) / h) - kBoxMargin;
            int hi = (int)std::ceil((cc + R - vmin) / h) + kBoxMargin;
            lo = lo < 0 ? 0 : (lo > n ? n : lo);
            hi = hi < 0 ? 0 : (hi > n ? n : hi);
            return (long)(hi - lo);
        };
        nbox = span(b->cx, b->ra, c->xmin, c->dx, c->nx) * span(b->cy, b->ra, c->ymin, c->dy, c->ny) *
               span(b->cz, b->ra, c->zmin, c->dz, c->nz);
        if (nbox < 1) nbox = 1;
    }
    cudaFree(c->spec_list); cudaFree(c->wall_list); cudaFree(c->wcontrib); cudaFree(c->wphi); cudaFree(c->cvinfo);
    c->spec_list = c->wall_list = nullptr; c->wcontrib = c->wphi = nullptr; c->cvinfo = nullptr;
    c->list_cap = (int)nbox;
    CK(cudaMalloc(&c->spec_list, sizeof(int32_t) * c->list_cap));
    CK(cudaMalloc(&c->wall_list, sizeof(int32_t) * c->list_cap));
    CK(cudaMalloc(&c->wcontrib, sizeof(double) * 4 * c->list_cap));
    CK(cudaMalloc(&c->wphi, sizeof(double) * 6 * c->list_cap));
    CK(cudaMalloc(&c->cvinfo, cvinfo3_bytes() * (size_t)c->list_cap));
    CK(cudaMemsetAsync(c->wcontrib, 0, sizeof(double) * 4 * c->list_cap, c->stream));
    CK(cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * 4, c->stream));
    dvm::BodyDev hb;
    std::memset(&hb, 0, sizeof(hb));
    hb.theta = b->theta; hb.omega = b->omega; hb.theta1 = b->theta;
    CK(cudaMemcpyAsync(c->d_body, &hb, sizeof(hb), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int) * kErrCount, c->stream));
    CK(init_static_geometry3d(c));
    if (b->shape != DVM_SHAPE_NONE) {
        CK(geometry3d(c));
        CK(masters_flags3d(c));
    }
    c->need_fusion = true;
    c->hvalid = false;
    c->steps_done = 0;
    return check_flags(c);
}

// A velocity-split step between its calls (dvm_split_begin ... finish, or
// finish ... relax): the state, the body and the scheme must not change.
static bool split_step_open(dvm_ctx *c, const char *fn)
{
    if (!c->split_begun && !c->split_relax) return false;
    set_error(std::string(fn) + ": a velocity-split step is in progress");
    return true;
}

int dvm_set_body(dvm_ctx *c, const dvm_body *b)
{
    if (!c || !b) { set_error("null argument"); return DVM_ERR_ARG; }
    if (split_step_open(c, "dvm_set_body")) return DVM_ERR_STATE;
    if (c->dim == 3) return set_body3d(c, b);
    const bool container = b->shape == DVM_SHAPE_DISK_CONTAINER || b->shape == DVM_SHAPE_BOX_CONTAINER;
    if (b->shape != DVM_SHAPE_NONE && b->shape != DVM_SHAPE_CIRCLE && b->shape != DVM_SHAPE_ELLIPSE && !container) {
        set_error("2D shapes: none, circle, ellipse, disk container, box container"); return DVM_ERR_UNSUPPORTED;
    }
    const bool two_sizes = b->shape == DVM_SHAPE_ELLIPSE || b->shape == DVM_SHAPE_BOX_CONTAINER;
    if (b->shape != DVM_SHAPE_NONE && (!(b->ra > 0) || (two_sizes && !(b->rb > 0)))) {
        set_error("body size"); return DVM_ERR_ARG;
    }
    if (container && b->movable) { set_error("a container is not movable"); return DVM_ERR_ARG; }
    if (b->movable && !(b->inertia > 0)) { set_error("movable body needs inertia > 0"); return DVM_ERR_ARG; }
    if (b->nseg > 0 && (!b->Tw_seg || !b->seg_dir)) { set_error("nseg > 0 needs Tw_seg and seg_dir"); return DVM_ERR_ARG; }
    c->body = *b;
    c->body.Tw_seg = nullptr; c->body.seg_dir = nullptr;
    cudaFree(c->d_Twseg); cudaFree(c->d_segdir);
    c->d_Twseg = c->d_segdir = nullptr;
    if (b->nseg > 0) {
        CK(cudaMalloc(&c->d_Twseg, sizeof(double) * b->nseg));
        CK(cudaMalloc(&c->d_segdir, sizeof(double) * 2 * b->nseg));
        CK(cudaMemcpy(c->d_Twseg, b->Tw_seg, sizeof(double) * b->nseg, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_segdir, b->seg_dir, sizeof(double) * 2 * b->nseg, cudaMemcpyHostToDevice));
    }
    c->moving = b->shape != DVM_SHAPE_NONE && b->movable;
    // box of cells that can be non-gas or have a non-gas cell within reach
    if (b->shape == DVM_SHAPE_NONE) {
        c->i0 = c->i1 = c->j0 = c->j1 = 0;
    } else if (container) {
        // the cells outside the container are solid: the whole grid
        c->i0 = 0; c->i1 = c->nx; c->j0 = 0; c->j1 = c->ny;
    } else {
        const double R = b->shape == DVM_SHAPE_ELLIPSE ? std::fmax(b->ra, b->rb) : b->ra;
        auto lo = [](double v, double h, int n) { int q = (int)std::floor(v / h) - kBoxMargin; return q < 0 ? 0 : (q > n ? n : q); };
        auto hi = [](double v, double h, int n) { int q = (int)std::ceil(v / h) + kBoxMargin; return q < 0 ? 0 : (q > n ? n : q); };
        c->i0 = lo(b->cx - R - c->xmin, c->dx, c->nx); c->i1 = hi(b->cx + R - c->xmin, c->dx, c->nx);
        c->j0 = lo(b->cy - R - c->ymin, c->dy, c->ny); c->j1 = hi(b->cy + R - c->ymin, c->dy, c->ny);
    }
    const int nbox = (c->i1 - c->i0) * (c->j1 - c->j0);
    cudaFree(c->spec_list); cudaFree(c->wall_list); cudaFree(c->wcontrib); cudaFree(c->wphi);
    cudaFree(c->wflux);
    c->spec_list = c->wall_list = nullptr; c->wcontrib = c->wphi = nullptr; c->wflux = nullptr;
    c->list_cap = nbox > 0 ? nbox : 1;
    CK(cudaMalloc(&c->spec_list, sizeof(int32_t) * c->list_cap));
    CK(cudaMalloc(&c->wall_list, sizeof(int32_t) * c->list_cap));
    CK(cudaMalloc(&c->wcontrib, sizeof(double) * 3 * c->list_cap));
    CK(cudaMalloc(&c->wphi, sizeof(double) * 4 * c->list_cap));
    cudaFree(c->cvinfo);
    CK(cudaMalloc(&c->cvinfo, cvinfo_bytes() * (size_t)c->list_cap));
    CK(cudaMalloc(&c->wflux, sizeof(double) * 8 * (size_t)c->list_cap * c->S));
    CK(cudaMemsetAsync(c->wcontrib, 0, sizeof(double) * 3 * c->list_cap, c->stream));
    CK(cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * 4, c->stream));
    dvm::BodyDev hb;
    std::memset(&hb, 0, sizeof(hb));
    hb.theta = b->theta; hb.omega = b->omega; hb.theta1 = b->theta;
    hb.trig[0] = std::cos(b->theta); hb.trig[1] = std::sin(b->theta);
    hb.trig[2] = hb.trig[0]; hb.trig[3] = hb.trig[1];
    CK(cudaMemcpyAsync(c->d_body, &hb, sizeof(hb), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int) * kErrCount, c->stream));
    c->gcur = 0;
    CK(init_static_geometry2d(c));
    if (b->shape != DVM_SHAPE_NONE) {
        CK(geometry2d_level(c, 0, body_trig(c, 0)));
        CK(geometry2d_level(c, 1, body_trig(c, 0)));
        CK(masters_flags2d(c, false));
    }
    c->need_fusion = true;
    c->hvalid = false;
    c->steps_done = 0;
    return check_flags(c);
}

int dvm_geometry2d_at(dvm_ctx *c, double cos_t, double sin_t)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (c->dim != 2) { set_error("dvm_geometry2d_at: 2D contexts only"); return DVM_ERR_ARG; }
    if (c->body.shape == DVM_SHAPE_NONE) return DVM_OK;
    double t[2] = {cos_t, sin_t};
    CK(cudaMemcpyAsync(body_trig(c, 0), t, sizeof(t), cudaMemcpyHostToDevice, c->stream));
    CK(geometry2d_level(c, c->gcur, body_trig(c, 0)));
    CK(masters_flags2d(c, false));
    c->need_fusion = true;
    c->hvalid = false;
    return check_flags(c);
}

int dvm_init_maxwellian(dvm_ctx *c, const double *rho, const double *ux, const double *uy,
                        const double *uz, const double *T)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (split_step_open(c, "dvm_init_maxwellian")) return DVM_ERR_STATE;
    const size_t nc = (size_t)c->nc;
    std::vector<double> prim(5 * nc);
    for (size_t k = 0; k < nc; ++k) {
        prim[5 * k] = rho ? rho[k] : 1.0;
        prim[5 * k + 1] = ux ? ux[k] : 0.0;
        prim[5 * k + 2] = uy ? uy[k] : 0.0;
        prim[5 * k + 3] = uz ? uz[k] : 0.0;
        prim[5 * k + 4] = T ? T[k] : 1.0;
        if (prim[5 * k] > 0 && !(prim[5 * k + 4] > 0)) { set_error("T must be > 0"); return DVM_ERR_ARG; }
    }
    if (!c->d_prim0) CK(cudaMalloc(&c->d_prim0, sizeof(double) * 5 * nc));
    double *d = c->d_prim0;    // kept: the adjoint chains dJ/dF^0 to these primitives
    CK(cudaMemcpyAsync(d, prim.data(), sizeof(double) * 5 * nc, cudaMemcpyHostToDevice, c->stream));
    c->have_prim0 = true;
    CK(st_init(c, d));
    CK(st_zero_solid(c));
    CK(st_halo(c, c->cur));
    CK(st_partials(c));
    c->have_state = true;
    c->need_fusion = true;
    c->hvalid = false;
    return check_flags(c);
}

static int ensure_pub(dvm_ctx *c)
{
    if (!c->d_pub) CK(cudaMalloc(&c->d_pub, c->state_elems * c->elem));
    return DVM_OK;
}

int dvm_set_state(dvm_ctx *c, const void *f, size_t bytes, int on_device)
{
    if (!c || !f) { set_error("null"); return DVM_ERR_ARG; }
    if (split_step_open(c, "dvm_set_state")) return DVM_ERR_STATE;
    if (bytes != c->state_elems * c->elem) { set_error("state size mismatch"); return DVM_ERR_ARG; }
    int rc = ensure_pub(c);
    if (rc != DVM_OK) return rc;
    CK(cudaMemcpyAsync(c->d_pub, f, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    CK(st_pack(c, c->d_pub, c->f[c->cur]));
    c->have_prim0 = false;
    CK(st_zero_solid(c));
    CK(st_halo(c, c->cur));
    CK(st_partials(c));
    c->have_state = true;
    c->need_fusion = true;
    c->hvalid = false;
    CK(cudaStreamSynchronize(c->stream));
    return DVM_OK;
}

int dvm_get_state(dvm_ctx *c, void *f, size_t bytes, int on_device)
{
    if (!c || !f) { set_error("null"); return DVM_ERR_ARG; }
    if (bytes != c->state_elems * c->elem) { set_error("state size mismatch"); return DVM_ERR_ARG; }
    int rc = ensure_pub(c);
    if (rc != DVM_OK) return rc;
    CK(st_unpack(c, c->f[c->cur], c->d_pub));
    CK(cudaMemcpyAsync(f, c->d_pub, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return DVM_OK;
}

// Checkpoint file: a fixed header, then the state in the public layout, the
// partial moment sums of the current buffer (device layout) and the device
// body record, so that a loaded context continues bit for bit as the saved
// one would have.  The header carries the sizes and schemes and a hash of
// everything else that defines the problem (problem_hash), so that a
// checkpoint of another obstacle, wall temperature, inflow or collision model
// is refused.
struct CheckpointHeader {
    char magic[8];            // "DVMCKPT1"
    int32_t version, dim, precision, scheme, time_scheme, S;
    int32_t nx, ny, nz, nvx, nvy, nvz, shape, movable, need_fusion, model;
    double dt, tau0;
    int64_t steps_done;
    uint64_t state_bytes, part_bytes, body_bytes;
    uint64_t problem;         // problem_hash
};
static const char kCkptMagic[8] = {'D', 'V', 'M', 'C', 'K', 'P', 'T', '1'};
static const int32_t kCkptVersion = 2;

// 64-bit FNV-1a over the bytes of a sequence of values.
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void bytes(const void *p, size_t n)
    {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t k = 0; k < n; ++k) { h ^= b[k]; h *= 1099511628211ull; }
    }
    void val(int32_t v) { bytes(&v, sizeof(v)); }
};

// Hash of the problem definition beyond the header's sizes: domain and
// velocity-grid extents, Kn, Lref, cfl, the collision model and Pr, the kind
// of every side and the states of the Maxwellian sides, and the obstacle
// (shape, centre, sizes, translation velocity, mass, inertia, movability,
// wall temperature and the per-sector temperatures and directions).  The
// body's angle and angular velocity are state, saved in the body record.
static int problem_hash(dvm_ctx *c, uint64_t *out)
{
    Fnv f;
    const double ext[] = {c->xmin, c->xmax, c->ymin, c->ymax, c->zmin, c->zmax, c->vxmin, c->vxmax,
                          c->vymin, c->vymax, c->vzmin, c->vzmax, c->Kn, c->Lref, c->cfl, c->Pr};
    f.bytes(ext, sizeof(ext));
    f.val((int32_t)c->model);
    f.val((int32_t)c->eq_mode);
    f.val((int32_t)c->split);
    for (int d = 0; d < 3; ++d) {
        f.val((int32_t)c->gnv[d]);
        f.bytes(&c->gv0[d], sizeof(double));
        f.bytes(&c->gdv[d], sizeof(double));
    }
    for (int side = 0; side < 2 * c->dim; ++side) {
        f.val((int32_t)c->bc[side]);
        if (c->bc[side] == DVM_BC_MAXWELLIAN && c->d_bcstate[side]) {
            std::vector<double> st((size_t)5 * side_cells(c, side));
            CK(cudaMemcpy(st.data(), c->d_bcstate[side], st.size() * sizeof(double), cudaMemcpyDeviceToHost));
            f.bytes(st.data(), st.size() * sizeof(double));
        }
    }
    const dvm_body &b = c->body;
    f.val((int32_t)b.shape);
    if (b.shape != DVM_SHAPE_NONE) {
        const double bd[] = {b.cx, b.cy, b.cz, b.ra, b.rb, b.vbx, b.vby, b.mass, b.inertia, b.Tw};
        f.bytes(bd, sizeof(bd));
        f.val((int32_t)b.movable);
        f.val((int32_t)b.nseg);
        if (b.nseg > 0 && c->d_Twseg && c->d_segdir) {
            std::vector<double> t((size_t)3 * b.nseg);
            CK(cudaMemcpy(t.data(), c->d_Twseg, sizeof(double) * b.nseg, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(t.data() + b.nseg, c->d_segdir, sizeof(double) * 2 * b.nseg, cudaMemcpyDeviceToHost));
            f.bytes(t.data(), t.size() * sizeof(double));
        }
    }
    *out = f.h;
    return DVM_OK;
}

static size_t part_bytes(const dvm_ctx *c)
{
    return (size_t)c->S * (c->dim == 2 ? 4 : 5) * (size_t)c->nc * c->elem;
}

int dvm_save(dvm_ctx *c, const char *path)
{
    if (!c || !path) { set_error("null argument"); return DVM_ERR_ARG; }
    if (!c->have_state) { set_error("dvm_save: no state"); return DVM_ERR_STATE; }
    CheckpointHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion; h.dim = c->dim; h.precision = c->prec; h.scheme = c->scheme; h.time_scheme = c->time_scheme;
    h.S = c->S; h.nx = c->nx; h.ny = c->ny; h.nz = c->nz; h.nvx = c->nvx; h.nvy = c->nvy; h.nvz = c->nvz;
    h.shape = c->body.shape; h.movable = c->body.movable; h.need_fusion = c->need_fusion ? 1 : 0;
    h.dt = c->dt; h.tau0 = c->tau0; h.steps_done = c->steps_done;
    h.state_bytes = c->state_elems * c->elem;
    h.part_bytes = part_bytes(c);
    h.body_bytes = sizeof(dvm::BodyDev);
    h.model = c->model;
    int rc = problem_hash(c, &h.problem);
    if (rc != DVM_OK) return rc;
    std::vector<char> state(h.state_bytes), part(h.part_bytes);
    dvm::BodyDev hb;
    rc = dvm_get_state(c, state.data(), state.size(), 0);
    if (rc != DVM_OK) return rc;
    CK(cudaMemcpyAsync(part.data(), c->part[c->cur], part.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&hb, c->d_body, sizeof(hb), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    FILE *fp = std::fopen(path, "wb");
    if (!fp) { set_error(std::string("dvm_save: cannot open ") + path); return DVM_ERR_ARG; }
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(state.data(), 1, state.size(), fp) == state.size() &&
              std::fwrite(part.data(), 1, part.size(), fp) == part.size() && std::fwrite(&hb, sizeof(hb), 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) { set_error(std::string("dvm_save: write failed: ") + path); return DVM_ERR_ARG; }
    return DVM_OK;
}

int dvm_load(dvm_ctx *c, const char *path)
{
    if (!c || !path) { set_error("null argument"); return DVM_ERR_ARG; }
    if (split_step_open(c, "dvm_load")) return DVM_ERR_STATE;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) { set_error(std::string("dvm_load: cannot open ") + path); return DVM_ERR_ARG; }
    uint64_t mine = 0;
    int hrc = problem_hash(c, &mine);
    if (hrc != DVM_OK) { std::fclose(fp); return hrc; }
    CheckpointHeader h;
    std::vector<char> state, part;
    dvm::BodyDev hb;
    bool ok = std::fread(&h, sizeof(h), 1, fp) == 1 && std::memcmp(h.magic, kCkptMagic, 8) == 0 &&
              h.version == kCkptVersion;
    // the checkpoint must come from a context of the same problem
    ok = ok && h.dim == c->dim && h.precision == c->prec && h.scheme == c->scheme && h.S == c->S &&
         h.nx == c->nx && h.ny == c->ny && h.nz == c->nz && h.nvx == c->nvx && h.nvy == c->nvy &&
         h.nvz == c->nvz && h.shape == c->body.shape && h.movable == c->body.movable && h.dt == c->dt &&
         h.tau0 == c->tau0 && h.state_bytes == c->state_elems * c->elem && h.part_bytes == part_bytes(c) &&
         h.body_bytes == sizeof(dvm::BodyDev) && (h.time_scheme == DVM_EXPLICIT || h.time_scheme == DVM_IMEX) &&
         h.model == c->model && h.problem == mine;
    if (ok) {
        state.resize(h.state_bytes);
        part.resize(h.part_bytes);
        ok = std::fread(state.data(), 1, state.size(), fp) == state.size() &&
             std::fread(part.data(), 1, part.size(), fp) == part.size() && std::fread(&hb, sizeof(hb), 1, fp) == 1;
    }
    std::fclose(fp);
    if (!ok) {
        set_error(std::string("dvm_load: not a checkpoint of this problem (grid, velocities, precision, schemes, "
                              "collision model, boundary states, body, wall temperatures, time step): ") + path);
        return DVM_ERR_ARG;
    }
    // the body first: a moving body's geometry is rebuilt at the saved angle
    // from the saved (cos, sin), which the saved run's current level used
    CK(cudaMemcpyAsync(c->d_body, &hb, sizeof(hb), cudaMemcpyHostToDevice, c->stream));
    if (c->dim == 2 && c->moving) {
        c->gcur = 0;
        CK(geometry2d_level(c, 0, body_trig(c, 2)));
        CK(geometry2d_level(c, 1, body_trig(c, 2)));
        CK(masters_flags2d(c, false));
    }
    int rc = dvm_set_state(c, state.data(), state.size(), 0);
    if (rc != DVM_OK) return rc;
    // the saved partial sums, not ones recomputed from the state
    CK(cudaMemcpyAsync(c->part[c->cur], part.data(), part.size(), cudaMemcpyHostToDevice, c->stream));
    c->need_fusion = h.need_fusion != 0;
    c->steps_done = h.steps_done;
    c->time_scheme = h.time_scheme;
    return check_flags(c);
}

int dvm_step_async(dvm_ctx *c, int nsteps)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    for (int d = 0; d < c->dim; ++d)
        if ((c->bc[2 * d] == DVM_BC_PERIODIC) != (c->bc[2 * d + 1] == DVM_BC_PERIODIC)) {
            set_error("opposite sides must both be periodic or both not");
            return DVM_ERR_ARG;
        }
    if (!c->have_state) { set_error("no state: call dvm_init_maxwellian or dvm_set_state"); return DVM_ERR_STATE; }
    if (nsteps < 0) { set_error("nsteps < 0"); return DVM_ERR_ARG; }
    if (c->split) {
        set_error("a velocity-split context steps through dvm_split_begin and dvm_split_finish");
        return DVM_ERR_STATE;
    }
    if (c->model == DVM_SHAKHOV)
        if (const char *why = shakhov_unsupported(c)) { set_error(why); return DVM_ERR_UNSUPPORTED; }
    int s = 0;
    // the first step after a state change (control-volume fusion), short runs
    // and runs with per-launch timing go launch by launch; the rest as
    // replays of a two-step graph (timing marks inside a graph, as event-record
    // nodes, cost about 1 % of the step)
    for (; s < nsteps && (s == 0 || c->need_fusion); ++s) {
        cudaError_t e = st_step(c);
        if (e != cudaSuccess) return cuda_fail(e, "dvm_step");
    }
    if (c->graphs && !c->timing && !c->rec_bits && nsteps - s >= kGraphMinSteps) {
        int done = 0;
        cudaError_t e = graph_steps(c, (nsteps - s) / 2, &done);
        if (e != cudaSuccess) return cuda_fail(e, "dvm_step (graph)");
        s += done;
    }
    for (; s < nsteps; ++s) {
        cudaError_t e = st_step(c);
        if (e != cudaSuccess) return cuda_fail(e, "dvm_step");
    }
    return DVM_OK;
}

int dvm_set_time_scheme(dvm_ctx *c, int scheme)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (scheme != DVM_EXPLICIT && scheme != DVM_IMEX) { set_error("time scheme must be DVM_EXPLICIT or DVM_IMEX"); return DVM_ERR_ARG; }
    if (split_step_open(c, "dvm_set_time_scheme")) return DVM_ERR_STATE;
    c->time_scheme = scheme;
    return DVM_OK;
}

int dvm_set_adjoint_tape(dvm_ctx *c, size_t max_bytes)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    c->adj_tape = max_bytes;
    if (c->dim == 2) trim_adjoint_tape2d(c, max_bytes);
    return DVM_OK;
}

int dvm_set_collision_model(dvm_ctx *c, int model, double Pr)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (model != DVM_BGK && model != DVM_SHAKHOV) { set_error("collision model must be DVM_BGK or DVM_SHAKHOV"); return DVM_ERR_ARG; }
    if (model == DVM_SHAKHOV) {
        if (!(Pr >= 0) || !std::isfinite(Pr)) { set_error("Prandtl number must be finite and >= 0"); return DVM_ERR_ARG; }
        if (const char *why = shakhov_unsupported(c)) { set_error(why); return DVM_ERR_UNSUPPORTED; }
    }
    if (model == DVM_SHAKHOV && !c->qheat) {
        // the heat flux of every cell [D][nc]; 2D also the raw heat-flux
        // moments of the state, paired with the partial sums
        const size_t hb = c->dim == 2 ? ((size_t)c->S * 5 + 2) * c->nc * c->elem : 0;
        if (cudaMalloc(&c->qheat, (size_t)c->dim * c->nc * c->elem) != cudaSuccess ||
            (hb && (cudaMalloc(&c->hpart[0], hb) != cudaSuccess || cudaMalloc(&c->hpart[1], hb) != cudaSuccess))) {
            cudaGetLastError();
            cudaFree(c->qheat); cudaFree(c->hpart[0]); cudaFree(c->hpart[1]);
            c->qheat = c->hpart[0] = c->hpart[1] = nullptr;
            set_error("dvm_set_collision_model: out of device memory");
            return DVM_ERR_OOM;
        }
    }
    c->hvalid = false;
    c->model = model;
    c->Pr = model == DVM_SHAKHOV ? Pr : 1.0;
    return DVM_OK;
}

int dvm_set_equilibrium(dvm_ctx *c, int mode)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (split_step_open(c, "dvm_set_equilibrium")) return DVM_ERR_STATE;
    if (mode != DVM_EQ_DIRECT && mode != DVM_EQ_CONSERVATIVE) {
        set_error("equilibrium mode must be DVM_EQ_DIRECT or DVM_EQ_CONSERVATIVE");
        return DVM_ERR_ARG;
    }
    if (mode == DVM_EQ_CONSERVATIVE && c->model != DVM_BGK) {
        set_error("the conservative equilibrium is implemented for the BGK model");
        return DVM_ERR_UNSUPPORTED;
    }
    if (mode == DVM_EQ_CONSERVATIVE && !c->eqp) {
        if (cudaMalloc(&c->eqp, (size_t)(c->dim + 2) * c->nc * c->elem) != cudaSuccess) {
            cudaGetLastError();
            c->eqp = nullptr;
            set_error("dvm_set_equilibrium: out of device memory");
            return DVM_ERR_OOM;
        }
    }
    c->eq_mode = mode;
    return DVM_OK;
}

int dvm_graphs(dvm_ctx *c, int enable)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    c->graphs = enable != 0;
    return DVM_OK;
}

int dvm_check(dvm_ctx *c)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    return check_flags(c);
}

// ---- dvm_step with a rollback to the last good step
// dvm_step runs chunks of up to kCheckChunk steps.  Before a chunk it copies
// the stepping state (state buffer, moment sums, rigid-body record, host
// counters) on the device; after it, it reads the flags and checks the
// moments of the chunk's last state.  If either fails, it goes back to the
// copy and steps one at a time with the same checks, and leaves the state at
// the input of the first step that failed.  The kernels are deterministic, so
// the replay meets the same states.
constexpr int kCheckChunk = 1024;

struct StepMark {
    int cur, gcur;
    long long steps;
    bool need_fusion;
};

static int ensure_snapshot(dvm_ctx *c)
{
    cudaError_t e = cudaSuccess;
    if (!c->snap_f) e = cudaMalloc(&c->snap_f, c->dev_elems * c->elem);
    if (e == cudaSuccess && !c->snap_part) e = cudaMalloc(&c->snap_part, part_bytes(c));
    if (e == cudaSuccess && !c->snap_scratch) e = cudaMalloc(&c->snap_scratch, part_bytes(c));
    if (e == cudaSuccess && !c->snap_body) e = cudaMalloc(&c->snap_body, sizeof(dvm::BodyDev));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("dvm_step: no device memory for the rollback copy of the state (dvm_rollback(ctx, 0) steps "
                  "without it)");
        return DVM_ERR_OOM;
    }
    return DVM_OK;
}

static cudaError_t take_snapshot(dvm_ctx *c, StepMark *m)
{
    m->cur = c->cur; m->gcur = c->gcur; m->steps = c->steps_done; m->need_fusion = c->need_fusion;
    cudaError_t e = cudaMemcpyAsync(c->snap_f, c->f[c->cur], c->dev_elems * c->elem, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->snap_part, c->part[c->cur], part_bytes(c), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->snap_body, c->d_body, sizeof(dvm::BodyDev), cudaMemcpyDeviceToDevice, c->stream);
    return e;
}

static cudaError_t restore_snapshot(dvm_ctx *c, const StepMark &m)
{
    c->cur = m.cur; c->gcur = m.gcur; c->steps_done = m.steps; c->need_fusion = m.need_fusion;
    c->hvalid = false;
    cudaError_t e = cudaMemcpyAsync(c->f[c->cur], c->snap_f, c->dev_elems * c->elem, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->part[c->cur], c->snap_part, part_bytes(c), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_body, c->snap_body, sizeof(dvm::BodyDev), cudaMemcpyDeviceToDevice, c->stream);
    // a moving body's current geometry level, from the cos/sin it was built with
    if (e == cudaSuccess && c->dim == 2 && c->moving) e = geometry2d_level(c, c->gcur, body_trig(c, 2));
    if (e == cudaSuccess && c->dim == 2 && c->moving) e = masters_flags2d(c, false);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, kErrCount * sizeof(int), c->stream);
    return e;
}

// Moments of the current state into the scratch sums: raises the
// non-physical flag for a gas cell with rho <= 0 or T <= 0.
static cudaError_t check_state(dvm_ctx *c)
{
    void *keep = c->part[c->cur];
    c->part[c->cur] = c->snap_scratch;
    const cudaError_t e = st_partials(c);
    c->part[c->cur] = keep;
    return e;
}

// Synchronises and tells whether a flag is raised (without clearing it).
static cudaError_t flags_raised(dvm_ctx *c, bool *raised)
{
    cudaError_t e = cudaMemcpyAsync(c->h_err, c->d_err, kErrCount * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    destroy_retired(c);
    *raised = false;
    for (int k = 0; k < kErrCount; ++k) *raised = *raised || c->h_err[k] != 0;
    return cudaSuccess;
}

int dvm_step(dvm_ctx *c, int nsteps)
{
    int rc = dvm_step_async(c, 0);             // the argument and state checks
    if (rc != DVM_OK) return rc;
    if (c->rollback_off) {
        rc = dvm_step_async(c, nsteps);
        if (rc != DVM_OK) return rc;
        return check_flags(c);
    }
    if (nsteps == 0) return check_flags(c);
    if ((rc = ensure_snapshot(c)) != DVM_OK) return rc;
    for (int done = 0; done < nsteps;) {
        const int n = nsteps - done < kCheckChunk ? nsteps - done : kCheckChunk;
        StepMark m;
        CK(take_snapshot(c, &m));
        if ((rc = dvm_step_async(c, n)) != DVM_OK) return rc;
        CK(check_state(c));
        bool bad = false;
        CK(flags_raised(c, &bad));
        if (bad) {
            CK(restore_snapshot(c, m));
            for (int k = 0; k < n; ++k) {
                CK(take_snapshot(c, &m));
                if ((rc = dvm_step_async(c, 1)) != DVM_OK) return rc;
                CK(check_state(c));
                CK(flags_raised(c, &bad));
                if (bad) {
                    rc = check_flags(c);       // message, flags cleared
                    CK(restore_snapshot(c, m));
                    CK(cudaStreamSynchronize(c->stream));
                    set_error(dvm_last_error() + std::string("; the state is left at step ") +
                              std::to_string(c->steps_done));
                    return rc;
                }
            }
        }
        done += n;
    }
    return check_flags(c);
}

int dvm_rollback(dvm_ctx *c, int enable)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    c->rollback_off = enable == 0;
    return DVM_OK;
}

// Scatter of the [cell][5] moment records into up to five device arrays.
__global__ void k_scatter5(const double *src, long nc, double *a0, double *a1, double *a2, double *a3, double *a4)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const double *r = src + 5 * k;
    if (a0) a0[k] = r[0];
    if (a1) a1[k] = r[1];
    if (a2) a2[k] = r[2];
    if (a3) a3[k] = r[3];
    if (a4) a4[k] = r[4];
}

int dvm_moments(dvm_ctx *c, double *rho, double *ux, double *uy, double *uz, double *T, int on_device)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (c->split) {
        set_error("dvm_moments: a velocity-split context holds a slab of the velocity grid; "
                  "the moments need the sums over every rank");
        return DVM_ERR_STATE;
    }
    const size_t nc = (size_t)c->nc;
    CK(st_moments(c, c->d_out));
    if (on_device) {
        k_scatter5<<<(unsigned)((nc + 255) / 256), 256, 0, c->stream>>>(c->d_out, (long)nc, rho, ux, uy, uz, T);
        CK(cudaGetLastError());
        c->launches += 1;
        CK(cudaStreamSynchronize(c->stream));
        return DVM_OK;
    }
    std::vector<double> h(5 * nc);
    CK(cudaMemcpyAsync(h.data(), c->d_out, sizeof(double) * 5 * nc, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < nc; ++k) {
        if (rho) rho[k] = h[5 * k];
        if (ux) ux[k] = h[5 * k + 1];
        if (uy) uy[k] = h[5 * k + 2];
        if (uz) uz[k] = h[5 * k + 3];
        if (T) T[k] = h[5 * k + 4];
    }
    return DVM_OK;
}

// ---- velocity split (Sec. 5.2)
int dvm_set_velocity_split(dvm_ctx *c, const dvm_vgrid *gv)
{
    if (!c || !gv) { set_error("null argument"); return DVM_ERR_ARG; }
    if (c->have_state || c->body.shape != DVM_SHAPE_NONE) {
        set_error("velocity split: set it right after dvm_create, before the body and the state");
        return DVM_ERR_STATE;
    }
    if (c->model != DVM_BGK) {
        set_error("velocity split: the BGK model only");
        return DVM_ERR_UNSUPPORTED;
    }
    const bool d3 = c->dim == 3;
    const int gn[3] = {gv->nvx, gv->nvy, d3 ? gv->nvz : 1};
    const double glo[3] = {gv->vxmin, gv->vymin, gv->vzmin}, ghi[3] = {gv->vxmax, gv->vymax, gv->vzmax};
    for (int d = 0; d < c->dim; ++d)
        if (gn[d] < 1 || gn[d] > kMaxAxisNv || !(ghi[d] > glo[d])) {
            set_error("velocity split: bad whole velocity grid (1 to 64 points per axis)");
            return DVM_ERR_ARG;
        }
    // the split axis is the last one (v_y in 2D, v_z in 3D); this context's
    // grid must be its rows [k0, k0 + n) with the other axes equal
    const int ax = c->dim - 1;
    const double gstep = (ghi[ax] - glo[ax]) / gn[ax];
    double *lo = d3 ? &c->vzmin : &c->vymin, *hi = d3 ? &c->vzmax : &c->vymax, *step = d3 ? &c->dvz : &c->dvy;
    const int nloc = d3 ? c->nvz : c->nvy;
    const double k0d = (*lo - glo[ax]) / gstep;
    const long k0 = std::lround(k0d);
    bool ok = std::fabs(gstep - *step) <= 1e-12 * gstep && std::fabs(k0d - (double)k0) <= 1e-9 && k0 >= 0 &&
              k0 + nloc <= gn[ax] && gv->nvx == c->nvx && gv->vxmin == c->vxmin && gv->vxmax == c->vxmax;
    if (d3) ok = ok && gv->nvy == c->nvy && gv->vymin == c->vymin && gv->vymax == c->vymax;
    if (!ok) {
        set_error("velocity split: the context's velocity grid is not a slab of rows of the last axis of the whole "
                  "grid (the other axes and the step equal, the first row an integer number of steps from the start)");
        return DVM_ERR_ARG;
    }
    for (int d = 0; d < 3; ++d) {
        c->gnv[d] = d < c->dim ? gn[d] : 1;
        c->gv0[d] = d < c->dim ? glo[d] : 0.0;
        c->gdv[d] = d < c->dim ? (ghi[d] - glo[d]) / gn[d] : 1.0;
    }
    // every rank takes the split axis' step of the whole grid and its first
    // row from the same expression, so that the quantities the ranks share
    // (the wall sums' dv, the force) are formed from bit-identical numbers
    *step = gstep;
    *lo = glo[ax] + (double)k0 * gstep;
    *hi = *lo + nloc * gstep;
    if (!c->dt_given) {
        // every rank takes the CFL time step of the whole velocity grid
        double sum = 0;
        for (int d = 0; d < c->dim; ++d)
            sum += axis_vmax(gn[d], glo[d], ghi[d]) / (d == 0 ? c->dx : d == 1 ? c->dy : c->dz);
        c->dt = c->cfl / sum;
    }
    CK(d3 ? tables3d(c) : tables2d(c));
    CK(cudaStreamSynchronize(c->stream));
    const int nmom = c->dim + 2;
    if (!c->split_in) {
        if (cudaMalloc(&c->split_in, (size_t)nmom * c->nc * c->elem) != cudaSuccess) {
            cudaGetLastError();
            c->split_in = nullptr;
            set_error("dvm_set_velocity_split: out of device memory");
            return DVM_ERR_OOM;
        }
    }
    c->split = true;
    return DVM_OK;
}

int dvm_split_size(dvm_ctx *c, size_t *count)
{
    if (!c || !count) { set_error("null argument"); return DVM_ERR_ARG; }
    if (!c->split) { set_error("dvm_split_size: no velocity split set"); return DVM_ERR_STATE; }
    const size_t nmom = c->dim + 2, nwall = c->dim == 2 ? 8 : 14;
    *count = nmom * c->nc + nwall * (c->body.shape != DVM_SHAPE_NONE ? c->list_cap : 0);
    return DVM_OK;
}

int dvm_split_begin(dvm_ctx *c, void *xbuf)
{
    if (!c || !xbuf) { set_error("null argument"); return DVM_ERR_ARG; }
    if (!c->split) { set_error("dvm_split_begin: no velocity split set"); return DVM_ERR_STATE; }
    if (!c->have_state) { set_error("no state: call dvm_init_maxwellian or dvm_set_state"); return DVM_ERR_STATE; }
    if (c->split_begun || c->split_relax) {
        set_error("dvm_split_begin: the previous step is not finished");
        return DVM_ERR_STATE;
    }
    for (int d = 0; d < c->dim; ++d)
        if ((c->bc[2 * d] == DVM_BC_PERIODIC) != (c->bc[2 * d + 1] == DVM_BC_PERIODIC)) {
            set_error("opposite sides must both be periodic or both not");
            return DVM_ERR_ARG;
        }
    cudaError_t e = c->dim == 2 ? split_step2d(c, 1, xbuf) : split_step3d(c, 1, xbuf);
    if (e != cudaSuccess) return cuda_fail(e, "dvm_split_begin");
    c->split_begun = true;
    return DVM_OK;
}

int dvm_split_finish(dvm_ctx *c, void *xbuf)
{
    if (!c || !xbuf) { set_error("null argument"); return DVM_ERR_ARG; }
    if (!c->split || !c->split_begun) { set_error("dvm_split_finish: no dvm_split_begin pending"); return DVM_ERR_STATE; }
    cudaError_t e = c->dim == 2 ? split_step2d(c, 2, xbuf) : split_step3d(c, 2, xbuf);
    c->split_begun = false;
    // the semi-implicit step waits for the second exchange
    c->split_relax = e == cudaSuccess && c->time_scheme == DVM_IMEX;
    if (e != cudaSuccess) return cuda_fail(e, "dvm_split_finish");
    return DVM_OK;
}

int dvm_split_relax(dvm_ctx *c, void *xbuf)
{
    if (!c || !xbuf) { set_error("null argument"); return DVM_ERR_ARG; }
    if (!c->split || !c->split_relax) {
        set_error("dvm_split_relax: no semi-implicit dvm_split_finish pending");
        return DVM_ERR_STATE;
    }
    cudaError_t e = c->dim == 2 ? split_step2d(c, 3, xbuf) : split_step3d(c, 3, xbuf);
    c->split_relax = false;
    if (e != cudaSuccess) return cuda_fail(e, "dvm_split_relax");
    return DVM_OK;
}

int dvm_wall_force(dvm_ctx *c, double *F, double *torque)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    dvm::BodyDev hb;
    CK(cudaMemcpyAsync(&hb, c->d_body, sizeof(hb), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (F) { F[0] = hb.F[0]; F[1] = hb.F[1]; F[2] = hb.F[2]; }
    if (torque) *torque = hb.torque;
    return DVM_OK;
}

int dvm_body_state(dvm_ctx *c, double *theta, double *omega)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    dvm::BodyDev hb;
    CK(cudaMemcpyAsync(&hb, c->d_body, sizeof(hb), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (theta) *theta = hb.theta;
    if (omega) *omega = hb.omega;
    return DVM_OK;
}

int dvm_history(dvm_ctx *c, double *Fx, double *Fy, double *Fz, double *torque, double *theta,
                double *omega, int n, int *count)
{
    if (!c || n < 0) { set_error("bad argument"); return DVM_ERR_ARG; }
    long long avail = c->steps_done < kHistCap ? c->steps_done : kHistCap;
    long long m = n < avail ? n : avail;
    std::vector<double> h(6 * (size_t)kHistCap);
    CK(cudaMemcpyAsync(h.data(), c->d_hist, sizeof(double) * 6 * kHistCap, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (long long q = 0; q < m; ++q) {
        long long step = c->steps_done - m + q;
        const double *r = &h[6 * (size_t)(step % kHistCap)];
        if (Fx) Fx[q] = r[0];
        if (Fy) Fy[q] = r[1];
        if (Fz) Fz[q] = r[2];
        if (torque) torque[q] = r[3];
        if (theta) theta[q] = r[4];
        if (omega) omega[q] = r[5];
    }
    if (count) *count = (int)m;
    return DVM_OK;
}

int dvm_mass(dvm_ctx *c, double *mass)
{
    if (!c || !mass) { set_error("null"); return DVM_ERR_ARG; }
    double *d = c->d_out;
    CK(st_mass(c, c->d_scratch, d));
    CK(cudaMemcpyAsync(mass, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return DVM_OK;
}

int dvm_info(dvm_ctx *c, double *dt, double *tau0, long long *ncell, int *nv, int *ncomp, int *elem)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (dt) *dt = c->dt;
    if (tau0) *tau0 = c->tau0;
    if (ncell) *ncell = c->nc;
    if (nv) *nv = c->nv;
    if (ncomp) *ncomp = c->ncomp;
    if (elem) *elem = c->elem;
    return DVM_OK;
}

int dvm_geometry2d(dvm_ctx *c, int8_t *type, int8_t *cgas, double *lx, double *ly, double *lw,
                   double *nwx, double *nwy, double *rwx, double *rwy, double *sbar, int32_t *master)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (c->dim != 2) { set_error("dvm_geometry2d: 2D contexts only"); return DVM_ERR_ARG; }
    const dvm::Geo2D &G = c->geo[c->gcur];
    const size_t nc = (size_t)c->nc;
    auto cp = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream) : cudaSuccess;
    };
    CK(cp(type, G.type, nc));
    CK(cp(cgas, G.cgas, nc));
    CK(cp(lx, G.lx, sizeof(double) * (c->nx + 1) * c->ny));
    CK(cp(ly, G.ly, sizeof(double) * c->nx * (c->ny + 1)));
    CK(cp(lw, G.lw, sizeof(double) * nc));
    CK(cp(nwx, G.nwx, sizeof(double) * nc));
    CK(cp(nwy, G.nwy, sizeof(double) * nc));
    CK(cp(rwx, G.rwx, sizeof(double) * nc));
    CK(cp(rwy, G.rwy, sizeof(double) * nc));
    CK(cp(sbar, G.sbar, sizeof(double) * nc));
    CK(cp(master, c->master, sizeof(int32_t) * nc));
    CK(cudaStreamSynchronize(c->stream));
    return DVM_OK;
}

int dvm_geometry3d(dvm_ctx *c, int8_t *type, int8_t *cgas, double *ax, double *ay, double *az, double *sw,
                   double *nwx, double *nwy, double *nwz, double *rwx, double *rwy, double *rwz, double *vol,
                   int32_t *master)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    if (c->dim != 3) { set_error("dvm_geometry3d: 3D contexts only"); return DVM_ERR_ARG; }
    const dvm::Geo3D &G = c->geo3;
    const size_t nc = (size_t)c->nc;
    auto cp = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream) : cudaSuccess;
    };
    CK(cp(type, G.type, nc));
    CK(cp(cgas, G.cgas, nc));
    CK(cp(ax, G.ax, sizeof(double) * (c->nx + 1) * (size_t)c->ny * c->nz));
    CK(cp(ay, G.ay, sizeof(double) * c->nx * (size_t)(c->ny + 1) * c->nz));
    CK(cp(az, G.az, sizeof(double) * c->nx * (size_t)c->ny * (c->nz + 1)));
    CK(cp(sw, G.sw, sizeof(double) * nc));
    CK(cp(nwx, G.nwx, sizeof(double) * nc));
    CK(cp(nwy, G.nwy, sizeof(double) * nc));
    CK(cp(nwz, G.nwz, sizeof(double) * nc));
    CK(cp(rwx, G.rwx, sizeof(double) * nc));
    CK(cp(rwy, G.rwy, sizeof(double) * nc));
    CK(cp(rwz, G.rwz, sizeof(double) * nc));
    CK(cp(vol, G.vol, sizeof(double) * nc));
    CK(cp(master, c->master, sizeof(int32_t) * nc));
    CK(cudaStreamSynchronize(c->stream));
    return DVM_OK;
}

// The checks every adjoint entry point makes.
static int adjoint_checks(dvm_ctx *c, int nsteps, int checkpoint_every)
{
    if (!c) { set_error("null argument"); return DVM_ERR_ARG; }
    if (c->dim != 2) { set_error("dvm_drag_adjoint: 2D contexts only"); return DVM_ERR_UNSUPPORTED; }
    if (c->time_scheme != DVM_EXPLICIT) {
        set_error("dvm_drag_adjoint: the explicit time scheme only");
        return DVM_ERR_UNSUPPORTED;
    }
    if (c->model != DVM_BGK) { set_error("dvm_drag_adjoint: the BGK model only"); return DVM_ERR_UNSUPPORTED; }
    if (c->eq_mode != DVM_EQ_DIRECT) {
        set_error("dvm_drag_adjoint: the direct moments only (not the conservative equilibrium)");
        return DVM_ERR_UNSUPPORTED;
    }
    if (c->split) { set_error("dvm_drag_adjoint: not with a velocity split"); return DVM_ERR_UNSUPPORTED; }
    if (c->body.shape == DVM_SHAPE_NONE || c->moving) {
        set_error("dvm_drag_adjoint: needs a fixed obstacle"); return DVM_ERR_UNSUPPORTED;
    }
    if (!c->have_state) { set_error("no state"); return DVM_ERR_STATE; }
    if (nsteps < 1 || checkpoint_every < 1) { set_error("nsteps and checkpoint_every must be >= 1"); return DVM_ERR_ARG; }
    for (int d = 0; d < 2; ++d)
        if ((c->bc[2 * d] == DVM_BC_PERIODIC) != (c->bc[2 * d + 1] == DVM_BC_PERIODIC)) {
            set_error("opposite sides must both be periodic or both not");
            return DVM_ERR_ARG;
        }
    return DVM_OK;
}

int dvm_drag_adjoint(dvm_ctx *c, int nsteps, int checkpoint_every, double *J, double *gTw, double *gbc0,
                     double *gbc1, double *gbc2, double *gbc3, double *gprim0, double *ms_forward,
                     double *ms_reverse)
{
    if (!c || !J || !gTw) { set_error("null argument"); return DVM_ERR_ARG; }
    int rc = adjoint_checks(c, nsteps, checkpoint_every);
    if (rc != DVM_OK) return rc;
    double *gbc[4] = {gbc0, gbc1, gbc2, gbc3};
    rc = drag_adjoint2d(c, nsteps, checkpoint_every, J, gTw, gbc, gprim0, ms_forward, ms_reverse, 1, nullptr, 0,
                        nullptr, 0);
    if (rc != DVM_OK) return rc;
    return check_flags(c);
}

int dvm_adjoint(dvm_ctx *c, int nsteps, int checkpoint_every, int with_drag, const void *seed, int seed_on_device,
                void *lambda0, int lambda0_on_device, double *J, double *gTw, double *gbc0, double *gbc1,
                double *gbc2, double *gbc3, double *gprim0)
{
    if (!c || !J || !gTw) { set_error("null argument"); return DVM_ERR_ARG; }
    if (!with_drag && !seed) { set_error("dvm_adjoint: no objective (with_drag = 0 and no seed)"); return DVM_ERR_ARG; }
    int rc = adjoint_checks(c, nsteps, checkpoint_every);
    if (rc != DVM_OK) return rc;
    double *gbc[4] = {gbc0, gbc1, gbc2, gbc3};
    rc = drag_adjoint2d(c, nsteps, checkpoint_every, J, gTw, gbc, gprim0, nullptr, nullptr, with_drag ? 1 : 0, seed,
                        seed_on_device, lambda0, lambda0_on_device);
    if (rc != DVM_OK) return rc;
    return check_flags(c);
}

int dvm_step_vjp(dvm_ctx *c, const void *lambda_np1, void *lambda_n, int on_device, double *gTw)
{
    if (!c || !lambda_np1 || !lambda_n || !gTw) { set_error("null argument"); return DVM_ERR_ARG; }
    double J = 0;
    return dvm_adjoint(c, 1, 1, 0, lambda_np1, on_device, lambda_n, on_device, &J, gTw, nullptr, nullptr, nullptr,
                       nullptr, nullptr);
}

int dvm_timing(dvm_ctx *c, int enable)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    c->timing = enable == 2 ? 2 : (enable != 0 ? 1 : 0);
    c->ev_used = 0;
    return DVM_OK;
}

int dvm_kernel_time(dvm_ctx *c, double *bulk_ms, long long *launches)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    CK(cudaStreamSynchronize(c->stream));
    auto *pool = static_cast<std::vector<cudaEvent_t> *>(c->ev_pool);
    double tot = 0;
    for (int q = 0; q < c->ev_used; ++q) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, (*pool)[2 * q], (*pool)[2 * q + 1]));
        tot += ms;
    }
    if (bulk_ms) *bulk_ms = tot;
    if (launches) *launches = c->ev_used;
    c->ev_used = 0;
    return DVM_OK;
}

int dvm_launches(dvm_ctx *c, long long *count)
{
    if (!c || !count) { set_error("null"); return DVM_ERR_ARG; }
    *count = c->launches;
    return DVM_OK;
}

int dvm_cell_counts(dvm_ctx *c, long long *nonsolid, long long *bulk, long long *cvs, long long *walls)
{
    if (!c) { set_error("null"); return DVM_ERR_ARG; }
    const size_t nc = (size_t)c->nc;
    std::vector<uint16_t> fl(nc);
    std::vector<int8_t> ty(nc);
    int32_t cnt[2] = {0, 0};
    if (c->dim == 2) {
        std::vector<uint8_t> f8(nc);
        CK(cudaMemcpyAsync(f8.data(), c->flags, nc, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (size_t k = 0; k < nc; ++k) fl[k] = f8[k];
    } else {
        CK(cudaMemcpyAsync(fl.data(), c->flags3, sizeof(uint16_t) * nc, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaMemcpyAsync(ty.data(), c->dim == 2 ? c->geo[c->gcur].type : c->geo3.type, nc, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(cnt, c->counts, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    long long ns = 0, nb = 0;
    for (size_t k = 0; k < nc; ++k) {
        ns += ty[k] != DVM_SOLID;
        nb += (fl[k] & kPlain) != 0;
    }
    const bool body = c->body.shape != DVM_SHAPE_NONE;
    if (nonsolid) *nonsolid = ns;
    if (bulk) *bulk = nb;
    if (cvs) *cvs = body ? cnt[0] : 0;
    if (walls) *walls = body ? cnt[1] : 0;
    return DVM_OK;
}

}  // extern "C"
