// sp_solve_noalloc: the solve of sp_solve with its workspace taken from a fixed
// device array compiled into this library, so that the call itself allocates no
// memory of any kind.
//
// Who needs it: code that must not allocate at the moment it solves.  cudaMalloc and
// cudaFree may synchronise the whole device, which stalls every other stream of a
// latency-bound time-stepping loop; a host framework may hand all device memory to
// its own pooling allocator and forbid raw allocations by the libraries it calls; and
// a memory budget fixed at start-up leaves no room for an allocation that can fail in
// the middle of a run.  Such callers build the plan (which does allocate: multiplier,
// twiddles) once, while they may, and then solve through this entry point.
//
// The scratch is one array per GPU that loads the library, held until the process
// exits.  Its device address is looked up once per device (cudaGetSymbolAddress,
// with that device current) on the first call made while it is the current device,
// and kept for the life of the process: make that first call before any stream
// capture, and do not call this entry point after cudaDeviceReset, which invalidates
// the kept address.  All calls share the array, so
// calls whose work overlaps on the GPU (other streams, other host threads, other
// plans) race on it and must be serialised by the caller.  No part of the scratch has
// to start at zero: every element a pass reads was written earlier in the same call.
#include <mutex>

#include "sp_internal.h"

// Capacity of the static workspace, in bytes (see SP_NOALLOC_MAX_BYTES in superpot.h).
static constexpr size_t kScratchBytes = (size_t)SP_NOALLOC_MAX_BYTES;

static __device__ __align__(256) unsigned char g_sp_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_addr[kMaxDevices];  // device address of g_sp_scratch per device ordinal

sp_status scratch_address(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return sp_fail(SP_ERR_INVALID, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        // `dev` is the current device here: the caller looked it up with cudaGetDevice.
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_sp_scratch);
        if (e != cudaSuccess || !ptr) return sp_cuda_check(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                                           "cudaGetSymbolAddress(static scratch)");
        g_addr[dev] = ptr;
    }
    *out = g_addr[dev];
    return SP_OK;
}

}  // namespace

extern "C" sp_status sp_solve_noalloc(const sp_plan p, const void* rho, void* u, sp_stream stream)
{
    sp_clear_error();
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (!rho || !u) return sp_fail(SP_ERR_INVALID, "rho and u must be non-NULL device pointers");
    if (!p->ready) return sp_fail(SP_ERR_NOT_READY, "sp_kernel_precompute has not been run on this plan");
    const size_t csize = (p->prec == SP_FP64 || p->prec == SP_DF32) ? 16 : 8;
    const size_t need = csize * (size_t)p->n[0] * (size_t)p->plane;
    if (need > kScratchBytes)
        return sp_fail(SP_ERR_UNSUPPORTED_SIZE,
                       "sp_solve_noalloc: this grid needs %zu bytes of workspace; the static scratch holds %zu",
                       need, kScratchBytes);
    int dev = 0;
    sp_status rc = sp_cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev != p->device)
        return sp_fail(SP_ERR_INVALID, "plan was created on device %d, current device is %d", p->device, dev);
    void* scratch = nullptr;
    if ((rc = scratch_address(dev, &scratch))) return rc;
    // A byte copy of the plan (plain values and pointers only) with the workspace
    // pointed at the static scratch; timing events are never recorded here.
    sp_plan_s view = *p;
    view.d_work = scratch;
    view.work_bytes = need;
    view.max_batch = 1;
    view.timing = false;
    if ((rc = sp_run_solve(&view, rho, u, 1, (cudaStream_t)stream))) return rc;
    // the plan's completion event (recording it allocates nothing): sp_plan_destroy
    // waits for it before freeing the multiplier and twiddles this solve reads
    return sp_record_done(p, (cudaStream_t)stream);
}
