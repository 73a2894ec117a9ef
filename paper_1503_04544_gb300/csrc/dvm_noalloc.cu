// Total-mass diagnostic that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code inside a host framework whose
// allocator owns all device memory (a custom-call or plugin hook that must not
// allocate while it executes), or a loop with a fixed memory budget that may
// not grow its footprint once it runs.  dvm_mass_noalloc serves them: it computes the same
// quantity as dvm_mass from buffers the caller already holds, and keeps its
// only scratch, one partial mass per cell, in the file-scope device array
// below.  That array is part of the library image: every GPU on which the
// library is loaded holds it (8 MiB) until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dvm_internal.h"

namespace {

constexpr long long kNoAllocMaxCells = 1LL << 20;   // capacity of the static scratch
constexpr int kMaxDevices = 64;

// Per-cell partial masses of the last call.  Shared by every call on a device.
static __device__ __align__(256) double g_cell_mass[kNoAllocMaxCells];

// Device address of g_cell_mass, looked up once per device and CUDA context:
// a context created after a cudaDeviceReset holds its own copy of the array,
// so the address is looked up again when the current context's id changes
// (context ids are unique for the life of the process).
struct ScratchSlot {
    unsigned long long ctx_id;
    double *ptr;
};
std::mutex g_setup_mutex;
ScratchSlot g_scratch[kMaxDevices] = {};

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Id of the calling thread's current context; false if there is none yet or
// the driver does not provide the calls.
bool current_context_id(unsigned long long *id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PfnCtxGetCurrent>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PfnCtxGetId>(fn);
        looked_up = true;
    }
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Partial mass of one cell: sbar * sum_p f dv over the first component of a
// state in the public layout [cell][comp][p] (one warp per cell).
template <typename T>
__global__ void __launch_bounds__(256) k_cell_mass(const T *f, long long ncell, int ncomp, int nv,
                                                   const double *sbar, double dv, double *scratch)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long cell = (long long)blockIdx.x * 8 + warp;
    if (cell >= ncell) return;
    const T *fk = f + cell * ncomp * (long long)nv;
    double s = 0;
    for (int p = lane; p < nv; p += 32) s += (double)fk[p];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) scratch[cell] = sbar[cell] * (s * dv);
}

// Fixed-order sum of the per-cell masses into *out (one block).
__global__ void __launch_bounds__(1024) k_sum_mass(const double *scratch, long long n, double *out)
{
    __shared__ double red[32];
    double s = 0;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) s += scratch[t];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

// Address of the static scratch on the current device (set-up on the first
// call on a device, and again on the first call in a new context of it).
int scratch_on_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dvm::cuda_fail(e, "dvm_mass_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) { dvm::set_error("dvm_mass_noalloc: device index out of range"); return DVM_ERR_ARG; }
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchSlot &slot = g_scratch[dev];
    if (!slot.ptr || !have_id || slot.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cell_mass);
        if (e != cudaSuccess || !p) return dvm::cuda_fail(e, "dvm_mass_noalloc: cudaGetSymbolAddress");
        // the lookup makes the device's primary context current if none was
        unsigned long long now = 0;
        slot.ctx_id = current_context_id(&now) ? now : 0;
        slot.ptr = static_cast<double *>(p);
    }
    *out = slot.ptr;
    return DVM_OK;
}

}  // namespace

extern "C" int dvm_mass_noalloc(const void *f, int precision, long long ncell, int ncomp, int nv,
                                const double *sbar, double dv, double *mass, void *stream)
{
    if (!f || !sbar || !mass) { dvm::set_error("dvm_mass_noalloc: null pointer"); return DVM_ERR_ARG; }
    if (precision != DVM_FP32 && precision != DVM_FP64) { dvm::set_error("dvm_mass_noalloc: precision must be 32 or 64"); return DVM_ERR_ARG; }
    if (ncell < 1 || ncomp < 1 || nv < 1) { dvm::set_error("dvm_mass_noalloc: empty state"); return DVM_ERR_ARG; }
    if (ncell > kNoAllocMaxCells) {
        dvm::set_error("dvm_mass_noalloc: " + std::to_string(ncell) + " cells exceed the static scratch capacity of " +
                       std::to_string(kNoAllocMaxCells) + " cells; use dvm_mass");
        return DVM_ERR_ARG;
    }
    double *scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc != DVM_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((ncell + 7) / 8);
    // every entry of the scratch that k_sum_mass reads is written first by
    // k_cell_mass in the same call, so nothing needs clearing
    if (precision == DVM_FP32)
        k_cell_mass<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(f), ncell, ncomp, nv, sbar, dv, scratch);
    else
        k_cell_mass<double><<<blocks, 256, 0, st>>>(static_cast<const double *>(f), ncell, ncomp, nv, sbar, dv, scratch);
    k_sum_mass<<<1, 1024, 0, st>>>(scratch, ncell, mass);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dvm::cuda_fail(e, "dvm_mass_noalloc: launch");
    return DVM_OK;
}
