// C ABI of the super-potential solver: plan creation and validation, precompute
// (Alg. 1), solves (Alg. 2), diagnostics.  See include/superpot.h for the contract.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "sp_internal.h"

static thread_local char g_err[1024] = "";

void sp_clear_error(void) { g_err[0] = 0; }

sp_status sp_fail(sp_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

sp_status sp_cuda_check(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return SP_OK;
    return sp_fail(e == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA, "%s: %s (%s)", what,
                   cudaGetErrorName(e), cudaGetErrorString(e));
}

sp_status sp_plan_alloc(sp_plan p, void** ptr, size_t bytes, const char* what)
{
    *ptr = nullptr;
    if (p->nalloc >= (int)(sizeof(p->alloc_ptr) / sizeof(p->alloc_ptr[0])))
        return sp_fail(SP_ERR_INVALID, "internal: too many plan allocations (%s)", what);
    void* q = nullptr;
    if (p->has_alloc) {
        q = p->alloc.alloc(bytes, p->device, p->alloc.ctx);
        if (!q) return sp_fail(SP_ERR_OOM, "allocator returned NULL for %s (%zu bytes)", what, bytes);
    } else {
        // stream-ordered on the plan's private stream, complete before the pointer is used
        cudaError_t e = cudaMallocAsync(&q, bytes, p->mem_st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->mem_st);
        if (e != cudaSuccess) {
            cudaGetLastError();  // allocation failures are not sticky: clear them
            return sp_fail(e == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA,
                           "cudaMallocAsync %s (%zu bytes): %s", what, bytes, cudaGetErrorName(e));
        }
    }
    p->alloc_ptr[p->nalloc] = q;
    p->alloc_bytes[p->nalloc] = bytes;
    ++p->nalloc;
    *ptr = q;
    return SP_OK;
}

// Release everything the plan owns, with the plan's device current.  Device memory of the
// library's own allocations is freed stream-ordered after the plan's last recorded work
// (no host wait); a caller's allocator gets its blocks back only after that work has
// completed (a host wait on the plan's event, not on the device).  Returns the status of
// that wait.
static cudaError_t free_plan(sp_plan p)
{
    if (!p) return cudaSuccess;
    cudaError_t err = cudaSuccess;
    if (p->has_alloc) {
        if (p->done_recorded) err = cudaEventSynchronize(p->done);
        for (int i = p->nalloc - 1; i >= 0; --i)
            p->alloc.release(p->alloc_ptr[i], p->alloc_bytes[i], p->device, p->alloc.ctx);
    } else if (p->mem_st) {
        if (p->done_recorded) err = cudaStreamWaitEvent(p->mem_st, p->done, 0);
        for (int i = p->nalloc - 1; i >= 0; --i) cudaFreeAsync(p->alloc_ptr[i], p->mem_st);
        cudaStreamDestroy(p->mem_st);  // released once its frees have run
    }
    if (p->ev) {
        for (cudaEvent_t e : *p->ev) cudaEventDestroy(e);
        delete p->ev;
    }
    if (p->done) cudaEventDestroy(p->done);
    if (p->staged) {
        for (int i = 0; i < 2; ++i)
            if (p->copy_st[i]) cudaStreamDestroy(p->copy_st[i]);
        for (int i = 0; i < 6; ++i)
            if (p->stage_ev[i]) cudaEventDestroy(p->stage_ev[i]);
    }
    free(p->h_gs_a);
    delete p;
    return err;
}

static const int kMaxLen = 2048;  // largest padded FFT length 2n per axis
static const int kGsCap = 4096;   // largest generated GS table

extern "C" sp_status sp_plan_create(sp_plan* out, const int n[3], const double box_lo[3],
                                    const double box_hi[3], int padding, const double* gs_w,
                                    const double* gs_a, int gs_terms, double eps,
                                    sp_precision prec, int max_batch)
{
    return sp_plan_create_ex(out, n, box_lo, box_hi, padding, gs_w, gs_a, gs_terms, eps, prec, max_batch, nullptr);
}

extern "C" sp_status sp_plan_create_ex(sp_plan* out, const int n[3], const double box_lo[3],
                                       const double box_hi[3], int padding, const double* gs_w,
                                       const double* gs_a, int gs_terms, double eps,
                                       sp_precision prec, int max_batch, const sp_allocator* allocator)
{
    g_err[0] = 0;
    if (!out) return sp_fail(SP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!n || !box_lo || !box_hi) return sp_fail(SP_ERR_INVALID, "n, box_lo and box_hi must be non-NULL");
    if (padding != 2) return sp_fail(SP_ERR_INVALID, "padding must be 2 (got %d)", padding);
    if (prec != SP_FP64 && prec != SP_FP32 && prec != SP_MIXED && prec != SP_DF32)
        return sp_fail(SP_ERR_INVALID, "unknown precision %d", (int)prec);
    if (max_batch < 1) return sp_fail(SP_ERR_INVALID, "max_batch must be >= 1 (got %d)", max_batch);
    if (allocator && (!allocator->alloc || !allocator->release))
        return sp_fail(SP_ERR_INVALID, "allocator: both alloc and release must be given");
    for (int ax = 0; ax < 3; ++ax) {
        if (n[ax] < 2 || 2 * n[ax] > kMaxLen)
            return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "n[%d] = %d: need n >= 2 and 2n <= %d", ax, n[ax], kMaxLen);
        if (!(isfinite(box_lo[ax]) && isfinite(box_hi[ax]) && box_hi[ax] > box_lo[ax]))
            return sp_fail(SP_ERR_INVALID, "box axis %d: need finite lo < hi", ax);
    }
    const bool user = gs_w || gs_a || gs_terms;
    if (user) {
        if (!gs_w || !gs_a || gs_terms < 1)
            return sp_fail(SP_ERR_INVALID, "GS table: give both arrays and gs_terms >= 1, or none");
        for (int s = 0; s < gs_terms; ++s)
            if (!(isfinite(gs_w[s]) && isfinite(gs_a[s]) && gs_a[s] > 0.0))
                return sp_fail(SP_ERR_INVALID, "GS table entry %d is not finite with a > 0", s);
    } else if (!(eps > 0.0 && eps < 1.0)) {
        return sp_fail(SP_ERR_INVALID, "eps must be in (0, 1) (got %g)", eps);
    }

    sp_plan p = new (std::nothrow) sp_plan_s();
    if (!p) return sp_fail(SP_ERR_OOM, "host allocation failed");
    cudaGetDevice(&p->device);
    if (allocator) {
        p->alloc = *allocator;
        p->has_alloc = true;
    }
    for (int ax = 0; ax < 3; ++ax) {
        p->n[ax] = n[ax];
        p->N[ax] = 2 * n[ax];
        p->lo[ax] = box_lo[ax];
        p->hi[ax] = box_hi[ax];
        p->h[ax] = (box_hi[ax] - box_lo[ax]) / (n[ax] - 1);
        p->L[ax] = n[ax] * p->h[ax];
        // a padded length with a prime factor above 7 has no radix plan: Bluestein's
        // algorithm, a circular convolution of length M = 2^k >= 2N - 1
        if (!sp_radix_plan(p->N[ax], &p->rp[ax])) {
            p->rp[ax].nst = 0;
            int M = 1;
            while (M < 2 * p->N[ax] - 1) M *= 2;
            p->blue_M[ax] = M;
            sp_radix_plan(M, &p->blue_rp[ax]);
        }
    }
    p->prec = prec;
    p->max_batch = max_batch;
    p->ldz = (n[2] + 1 + 7) & ~7;
    p->plane = 2LL * n[1] * p->ldz;
    p->eps = eps;
    p->delta = sqrt(p->L[0] * p->L[0] + p->L[1] * p->L[1] + p->L[2] * p->L[2]);
    p->h_tau = 0.1;
    p->eta = 1e-17;
    p->gs_user = user;
    // the generated table's length is fixed by eps and delta (eq. sin_1_x): known now
    const int terms = user ? gs_terms : sp_gs_terms(p);
    if (!user && (terms < 1 || terms > kGsCap)) {
        delete p;
        return sp_fail(SP_ERR_INVALID, "GS table of %d terms (eps %g): at most %d", terms, eps, kGsCap);
    }
    p->gs_cap = terms;
    p->gs_terms = terms;

    p->ev = new (std::nothrow) std::vector<cudaEvent_t>();
    p->h_gs_a = (double*)malloc(sizeof(double) * p->gs_cap);
    if (!p->h_gs_a || !p->ev) {
        free_plan(p);
        return sp_fail(SP_ERR_OOM, "host allocation failed");
    }
    if (user) memcpy(p->h_gs_a, gs_a, sizeof(double) * gs_terms);
    else sp_gs_exponents(p, p->h_gs_a);
    sp_status rc = SP_OK;
    if ((rc = sp_cuda_check(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming), "create plan event"))) {
        p->done = nullptr;
        free_plan(p);
        return rc;
    }
    if (!p->has_alloc &&
        (rc = sp_cuda_check(cudaStreamCreateWithFlags(&p->mem_st, cudaStreamNonBlocking), "create plan stream"))) {
        p->mem_st = nullptr;
        free_plan(p);
        return rc;
    }
#define SP_ALLOC(ptr, bytes)                                                           \
    do {                                                                               \
        if ((rc = sp_plan_alloc(p, (void**)&(ptr), (bytes), #ptr))) {                  \
            free_plan(p);                                                              \
            return rc;                                                                 \
        }                                                                              \
    } while (0)
    SP_ALLOC(p->d_status, 256);
    SP_ALLOC(p->d_gs_w, sizeof(double) * p->gs_cap);
    SP_ALLOC(p->d_gs_a, sizeof(double) * p->gs_cap);
    // 1D integral tables [s][k] per axis; axes with the same (n, L) share one
    for (int ax = 0; ax < 3; ++ax) {
        int same = -1;
        for (int q = 0; q < ax; ++q)
            if (p->n[q] == p->n[ax] && p->L[q] == p->L[ax]) { same = q; break; }
        if (same >= 0) {
            p->d_G[ax] = p->d_G[same];
            p->d_H[ax] = p->d_H[same];
            continue;
        }
        const size_t tb = sizeof(double) * (size_t)p->gs_cap * (n[ax] + 1);
        SP_ALLOC(p->d_G[ax], tb);
        SP_ALLOC(p->d_H[ax], tb);
    }
    const size_t mcount = (size_t)(n[0] + 1) * (n[1] + 1) * p->ldz;
    SP_ALLOC(p->d_M64, sizeof(double) * mcount);
    if (prec == SP_FP32 || prec == SP_MIXED) SP_ALLOC(p->d_M32, sizeof(float) * mcount);
    if (prec == SP_DF32) SP_ALLOC(p->d_Mdf, sizeof(df32) * mcount);
    for (int ax = 0; ax < 3; ++ax) {
        SP_ALLOC(p->d_tw64[ax], sizeof(cpx<double>) * p->N[ax]);
        SP_ALLOC(p->d_tw32[ax], sizeof(cpx<float>) * (p->N[ax] + SP_TW_STAGED_MAX));
        SP_ALLOC(p->d_twdf[ax], sizeof(cpx<df32>) * (p->N[ax] + SP_TW_STAGED_MAX));
    }
    for (int ax = 0; ax < 3; ++ax) {  // Bluestein tables: built on the host, copied once
        if (!p->blue_M[ax]) continue;
        SP_ALLOC(p->d_blue[ax], sp_bluestein_bytes(p, ax));
        std::vector<unsigned char> host(sp_bluestein_bytes(p, ax));
        sp_bluestein_fill(p, ax, host.data());
        // pageable source: the call returns once the bytes are staged, so host may go
        const cudaError_t ce = p->mem_st ? cudaMemcpyAsync(p->d_blue[ax], host.data(), host.size(),
                                                           cudaMemcpyHostToDevice, p->mem_st)
                                         : cudaMemcpy(p->d_blue[ax], host.data(), host.size(), cudaMemcpyHostToDevice);
        if ((rc = sp_cuda_check(ce, "Bluestein tables"))) {
            free_plan(p);
            return rc;
        }
    }
    const size_t csize = (prec == SP_FP64 || prec == SP_DF32) ? 16 : 8;
    p->work_bytes = csize * (size_t)max_batch * n[0] * (size_t)p->plane;
    SP_ALLOC(p->d_work, p->work_bytes);
#undef SP_ALLOC
    const cudaError_t ce = p->mem_st ? cudaMemsetAsync(p->d_status, 0, 256, p->mem_st) : cudaMemset(p->d_status, 0, 256);
    if ((rc = sp_cuda_check(ce == cudaSuccess && p->mem_st ? cudaStreamSynchronize(p->mem_st) : ce,
                            "clear status word"))) {
        free_plan(p);
        return rc;
    }
    if (user) {
        if ((rc = sp_cuda_check(cudaMemcpy(p->d_gs_w, gs_w, sizeof(double) * gs_terms, cudaMemcpyHostToDevice),
                                "copy GS weights")) ||
            (rc = sp_cuda_check(cudaMemcpy(p->d_gs_a, gs_a, sizeof(double) * gs_terms, cudaMemcpyHostToDevice),
                                "copy GS exponents"))) {
            free_plan(p);
            return rc;
        }
    }
    *out = p;
    return SP_OK;
}

sp_status sp_record_done(sp_plan p, cudaStream_t st)
{
    sp_status rc = sp_cuda_check(cudaEventRecord(p->done, st), "record plan event");
    if (rc == SP_OK) p->done_recorded = true;
    return rc;
}

extern "C" sp_status sp_kernel_precompute(sp_plan p, sp_stream stream)
{
    g_err[0] = 0;
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    sp_status rc = sp_check_device(p);
    if (rc) return rc;
    const size_t mcount = (size_t)(p->n[0] + 1) * (p->n[1] + 1) * p->ldz;
    if ((rc = sp_cuda_check(cudaMemsetAsync(p->d_M64, 0, sizeof(double) * mcount, st), "clear multiplier")))
        return rc;
    if ((rc = sp_setup_run(p, st))) return rc;
    if ((rc = sp_record_done(p, st))) return rc;
    p->ready = true;
    return SP_OK;
}

extern "C" sp_status sp_plan_set_kernel(sp_plan p, sp_kernel kind)
{
    g_err[0] = 0;
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (kind != SP_KERNEL_SUPERPOTENTIAL && kind != SP_KERNEL_GS_PLAIN)
        return sp_fail(SP_ERR_INVALID, "unknown kernel %d", (int)kind);
    p->kernel = (int)kind;
    p->ready = false;
    return SP_OK;
}

// The plan's memory lives on the device it was created on; launching its passes while
// another device is current would hand that device foreign pointers.
sp_status sp_check_device(const sp_plan p)
{
    int dev = -1;
    sp_status rc = sp_cuda_check(cudaGetDevice(&dev), "current device");
    if (rc) return rc;
    if (dev != p->device)
        return sp_fail(SP_ERR_INVALID, "plan was created on device %d, current device is %d", p->device, dev);
    return SP_OK;
}

static sp_status check_solve_args(sp_plan p, const void* rho, const void* u)
{
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (!rho || !u) return sp_fail(SP_ERR_INVALID, "rho and u must be non-NULL device pointers");
    if (!p->ready) return sp_fail(SP_ERR_NOT_READY, "sp_kernel_precompute has not been run on this plan");
    return sp_check_device(p);
}

extern "C" sp_status sp_solve(sp_plan p, const void* rho, void* u, sp_stream stream)
{
    g_err[0] = 0;
    sp_status rc = check_solve_args(p, rho, u);
    if (rc) return rc;
    if ((rc = sp_run_solve(p, rho, u, 1, (cudaStream_t)stream))) return rc;
    return sp_record_done(p, (cudaStream_t)stream);
}

extern "C" sp_status sp_solve_batched(sp_plan p, const void* rho, void* u, int batch, sp_stream stream)
{
    g_err[0] = 0;
    sp_status rc = check_solve_args(p, rho, u);
    if (rc) return rc;
    if (batch < 1 || batch > p->max_batch)
        return sp_fail(SP_ERR_INVALID, "batch %d outside [1, max_batch = %d]", batch, p->max_batch);
    if ((rc = sp_run_solve(p, rho, u, batch, (cudaStream_t)stream))) return rc;
    return sp_record_done(p, (cudaStream_t)stream);
}

extern "C" sp_status sp_forward_spectrum(sp_plan p, const void* rho, void* spec, sp_stream stream)
{
    g_err[0] = 0;
    sp_status rc = check_solve_args(p, rho, spec);
    if (rc) return rc;
    if ((rc = sp_run_forward(p, rho, spec, (cudaStream_t)stream))) return rc;
    return sp_record_done(p, (cudaStream_t)stream);
}

extern "C" sp_status sp_plan_destroy(sp_plan p)
{
    g_err[0] = 0;
    if (!p) return SP_OK;
    // wait for the plan's own last work and free on the plan's device, whichever device is
    // current
    int cur = -1;
    const bool switched = cudaGetDevice(&cur) == cudaSuccess && cur != p->device &&
                          cudaSetDevice(p->device) == cudaSuccess;
    cudaError_t e = free_plan(p);
    if (switched) cudaSetDevice(cur);
    return sp_cuda_check(e, "order the plan's release after its work");
}

extern "C" sp_status sp_plan_sync(sp_plan p)
{
    g_err[0] = 0;
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    sp_status rc = sp_check_device(p);
    if (rc) return rc;
    if (p->done_recorded && (rc = sp_cuda_check(cudaEventSynchronize(p->done), "wait for the plan's work")))
        return rc;
    if ((rc = sp_cuda_check(cudaGetLastError(), "pending device error"))) return rc;
    int status = 0;
    if ((rc = sp_cuda_check(cudaMemcpy(&status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost), "read status word")))
        return rc;
    if (status != 0) {
        if ((rc = sp_cuda_check(cudaMemset(p->d_status, 0, sizeof(int)), "clear status word"))) return rc;
        return sp_fail(SP_ERR_TIMEOUT, "a bounded device wait gave up (status %d): some work of the solve was not done",
                       status);
    }
    return SP_OK;
}

extern "C" size_t sp_plan_workspace_bytes(const sp_plan p) { return p ? p->work_bytes : 0; }

extern "C" int sp_plan_gs_terms(const sp_plan p) { return p ? p->gs_terms : 0; }

extern "C" sp_status sp_plan_copy_tables(sp_plan p, double* gs_w, double* gs_a, double* M, int axis,
                                         double* G, double* H)
{
    g_err[0] = 0;
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (!p->ready) return sp_fail(SP_ERR_NOT_READY, "sp_kernel_precompute has not been run on this plan");
    if ((G || H) && (axis < 0 || axis > 2)) return sp_fail(SP_ERR_INVALID, "axis must be 0, 1 or 2");
    sp_status rc;
    if ((rc = sp_check_device(p))) return rc;
    if (p->done_recorded && (rc = sp_cuda_check(cudaEventSynchronize(p->done), "wait for the plan's work")))
        return rc;
    const int S = p->gs_terms;
    if (gs_w && (rc = sp_cuda_check(cudaMemcpy(gs_w, p->d_gs_w, sizeof(double) * S, cudaMemcpyDeviceToHost),
                                    "copy GS weights")))
        return rc;
    if (gs_a && (rc = sp_cuda_check(cudaMemcpy(gs_a, p->d_gs_a, sizeof(double) * S, cudaMemcpyDeviceToHost),
                                    "copy GS exponents")))
        return rc;
    if (M) {
        const int n0p = p->n[0] + 1, n1p = p->n[1] + 1, n2p = p->n[2] + 1;
        std::vector<double> dev((size_t)n0p * n1p * p->ldz);
        if ((rc = sp_cuda_check(cudaMemcpy(dev.data(), p->d_M64, sizeof(double) * dev.size(),
                                           cudaMemcpyDeviceToHost), "copy multiplier")))
            return rc;
        for (int k0 = 0; k0 < n0p; ++k0)
            for (int k1 = 0; k1 < n1p; ++k1)
                for (int k2 = 0; k2 < n2p; ++k2)
                    M[((size_t)k0 * n1p + k1) * n2p + k2] = dev[((size_t)k1 * n0p + k0) * p->ldz + k2];
    }
    const size_t tb = sizeof(double) * (size_t)S * (p->n[axis < 0 ? 0 : axis] + 1);
    if (G && (rc = sp_cuda_check(cudaMemcpy(G, p->d_G[axis], tb, cudaMemcpyDeviceToHost), "copy G"))) return rc;
    if (H && (rc = sp_cuda_check(cudaMemcpy(H, p->d_H[axis], tb, cudaMemcpyDeviceToHost), "copy H"))) return rc;
    return SP_OK;
}

sp_status sp_mark(sp_plan p, cudaStream_t st)
{
    if (!p->timing) return SP_OK;
    std::vector<cudaEvent_t>& ev = *p->ev;
    if (p->ev_used == ev.size()) {  // the pool is exhausted: grow it (outside a reserved record)
        cudaEvent_t e;
        sp_status rc = sp_cuda_check(cudaEventCreate(&e), "create timing event");
        if (rc) return rc;
        ev.push_back(e);
    }
    return sp_cuda_check(cudaEventRecord(ev[p->ev_used++], st), "record timing event");
}

// Events for `solves` recorded solves (npass + 1 each; 8 passes assumed before the first
// solve tells the pass count).
static sp_status reserve_events(sp_plan p, int solves)
{
    const int per = (p->npass > 0 ? p->npass : 8) + 1;
    const size_t want = p->ev_used + (size_t)solves * per;
    std::vector<cudaEvent_t>& ev = *p->ev;
    while (ev.size() < want) {
        cudaEvent_t e;
        sp_status rc = sp_cuda_check(cudaEventCreate(&e), "create timing event");
        if (rc) return rc;
        ev.push_back(e);
    }
    return SP_OK;
}

extern "C" sp_status sp_plan_set_timing(sp_plan p, int enable)
{
    g_err[0] = 0;
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (enable < 0) return sp_fail(SP_ERR_INVALID, "enable must be >= 0 (got %d)", enable);
    p->timing = enable != 0;
    if (enable > 0) return reserve_events(p, enable);
    return SP_OK;
}

extern "C" int sp_plan_pass_times(sp_plan p, double* total_ms, int* launches, const char** names,
                                  int max_passes)
{
    g_err[0] = 0;
    if (!p) { sp_fail(SP_ERR_INVALID, "plan is NULL"); return -1; }
    const int np = p->npass;
    const int per = np + 1;
    for (int i = 0; i < max_passes && i < np; ++i) {
        if (total_ms) total_ms[i] = 0.0;
        if (launches) launches[i] = 0;
        if (names) names[i] = p->pass_name[i];
    }
    std::vector<cudaEvent_t>& ev = *p->ev;
    const size_t used = p->ev_used;
    if (np == 0 || used == 0) return np;
    if (used % per != 0) { sp_fail(SP_ERR_INVALID, "incomplete timing record"); return -1; }
    if (sp_cuda_check(cudaEventSynchronize(ev[used - 1]), "wait for timing events")) return -1;
    for (size_t s0 = 0; s0 < used; s0 += per) {
        for (int i = 0; i < np; ++i) {
            float ms = 0.f;
            if (sp_cuda_check(cudaEventElapsedTime(&ms, ev[s0 + i], ev[s0 + i + 1]), "elapsed time"))
                return -1;
            if (i < max_passes) {
                if (total_ms) total_ms[i] += ms;
                if (launches) launches[i] += 1;
            }
        }
    }
    p->ev_used = 0;  // the events stay in the pool for the next record
    return np;
}

extern "C" const char* sp_last_error(void) { return g_err; }

extern "C" const char* sp_version(void) { return "superpot 0.1 (sm_103a)"; }
