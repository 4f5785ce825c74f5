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

// Padded lengths the radix-2/3/4/5/7/8 passes can transform: products of 2, 3, 5 and 7.
static bool smooth2357(int m)
{
    if (m < 2) return false;
    for (int f : {2, 3, 5, 7})
        while (m % f == 0) m /= f;
    return m == 1;
}

static void free_plan(sp_plan p)
{
    if (!p) return;
    cudaFree(p->d_gs_w);
    cudaFree(p->d_gs_a);
    for (int ax = 0; ax < 3; ++ax) {
        bool owner = true;
        for (int q = 0; q < ax; ++q)
            if (p->d_G[q] == p->d_G[ax]) owner = false;
        if (owner) {
            cudaFree(p->d_G[ax]);
            cudaFree(p->d_H[ax]);
        }
        cudaFree(p->d_tw64[ax]);
        cudaFree(p->d_tw32[ax]);
        cudaFree(p->d_twdf[ax]);
    }
    cudaFree(p->d_M64);
    cudaFree(p->d_M32);
    cudaFree(p->d_Mdf);
    cudaFree(p->d_work);
    if (p->ev) {
        for (cudaEvent_t e : *p->ev) cudaEventDestroy(e);
        delete p->ev;
    }
    free(p->h_gs_a);
    delete p;
}

static const int kMaxLen = 2048;  // largest padded FFT length 2n per axis
static const int kGsCap = 4096;   // largest generated GS table

extern "C" sp_status sp_plan_create(sp_plan* out, const int n[3], const double box_lo[3],
                                    const double box_hi[3], int padding, const double* gs_w,
                                    const double* gs_a, int gs_terms, double eps,
                                    sp_precision prec, int max_batch)
{
    g_err[0] = 0;
    if (!out) return sp_fail(SP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!n || !box_lo || !box_hi) return sp_fail(SP_ERR_INVALID, "n, box_lo and box_hi must be non-NULL");
    if (padding != 2) return sp_fail(SP_ERR_INVALID, "padding must be 2 (got %d)", padding);
    if (prec != SP_FP64 && prec != SP_FP32 && prec != SP_MIXED && prec != SP_DF32)
        return sp_fail(SP_ERR_INVALID, "unknown precision %d", (int)prec);
    if (max_batch < 1) return sp_fail(SP_ERR_INVALID, "max_batch must be >= 1 (got %d)", max_batch);
    for (int ax = 0; ax < 3; ++ax) {
        if (n[ax] < 2 || !smooth2357(2 * n[ax]) || 2 * n[ax] > kMaxLen)
            return sp_fail(SP_ERR_UNSUPPORTED_SIZE,
                           "n[%d] = %d: need n >= 2 and 2n a product of 2s, 3s, 5s and 7s, 2n <= %d", ax,
                           n[ax], kMaxLen);
        if (prec == SP_DF32 && !sp_v2_supported(2 * n[ax]))
            return sp_fail(SP_ERR_UNSUPPORTED_SIZE,
                           "n[%d] = %d: double-float passes need 2n in {64, 128, 192, 256, 384, 512, 1024}", ax,
                           n[ax]);
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
    for (int ax = 0; ax < 3; ++ax) {
        p->n[ax] = n[ax];
        p->N[ax] = 2 * n[ax];
        p->lo[ax] = box_lo[ax];
        p->hi[ax] = box_hi[ax];
        p->h[ax] = (box_hi[ax] - box_lo[ax]) / (n[ax] - 1);
        p->L[ax] = n[ax] * p->h[ax];
        sp_radix_plan(p->N[ax], &p->rp[ax]);
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
    p->gs_cap = user ? gs_terms : kGsCap;
    p->gs_terms = user ? gs_terms : 0;

    p->ev = new (std::nothrow) std::vector<cudaEvent_t>();
    p->h_gs_a = (double*)malloc(sizeof(double) * p->gs_cap);
    if (!p->h_gs_a || !p->ev) {
        free_plan(p);
        return sp_fail(SP_ERR_OOM, "host allocation failed");
    }
    if (user) memcpy(p->h_gs_a, gs_a, sizeof(double) * gs_terms);
    sp_status rc = SP_OK;
#define SP_ALLOC(ptr, bytes)                                                           \
    do {                                                                               \
        if ((rc = sp_cuda_check(cudaMalloc((void**)&(ptr), (bytes)), "cudaMalloc " #ptr))) { \
            free_plan(p);                                                              \
            return rc;                                                                 \
        }                                                                              \
    } while (0)
    SP_ALLOC(p->d_gs_w, sizeof(double) * p->gs_cap);
    SP_ALLOC(p->d_gs_a, sizeof(double) * p->gs_cap);
    const size_t mcount = (size_t)(n[0] + 1) * (n[1] + 1) * p->ldz;
    SP_ALLOC(p->d_M64, sizeof(double) * mcount);
    if (prec == SP_FP32 || prec == SP_MIXED) SP_ALLOC(p->d_M32, sizeof(float) * mcount);
    if (prec == SP_DF32) SP_ALLOC(p->d_Mdf, sizeof(df32) * mcount);
    for (int ax = 0; ax < 3; ++ax) {
        SP_ALLOC(p->d_tw64[ax], sizeof(cpx<double>) * p->N[ax]);
        SP_ALLOC(p->d_tw32[ax], sizeof(cpx<float>) * (p->N[ax] + SP_TW_STAGED_MAX));
        SP_ALLOC(p->d_twdf[ax], sizeof(cpx<df32>) * (p->N[ax] + SP_TW_STAGED_MAX));
    }
    const size_t csize = (prec == SP_FP64 || prec == SP_DF32) ? 16 : 8;
    p->work_bytes = csize * (size_t)max_batch * n[0] * (size_t)p->plane;
    SP_ALLOC(p->d_work, p->work_bytes);
#undef SP_ALLOC
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
    return sp_run_solve(p, rho, u, 1, (cudaStream_t)stream);
}

extern "C" sp_status sp_solve_batched(sp_plan p, const void* rho, void* u, int batch, sp_stream stream)
{
    g_err[0] = 0;
    sp_status rc = check_solve_args(p, rho, u);
    if (rc) return rc;
    if (batch < 1 || batch > p->max_batch)
        return sp_fail(SP_ERR_INVALID, "batch %d outside [1, max_batch = %d]", batch, p->max_batch);
    return sp_run_solve(p, rho, u, batch, (cudaStream_t)stream);
}

extern "C" sp_status sp_forward_spectrum(sp_plan p, const void* rho, void* spec, sp_stream stream)
{
    g_err[0] = 0;
    sp_status rc = check_solve_args(p, rho, spec);
    if (rc) return rc;
    return sp_run_forward(p, rho, spec, (cudaStream_t)stream);
}

extern "C" sp_status sp_plan_destroy(sp_plan p)
{
    g_err[0] = 0;
    if (!p) return SP_OK;
    // wait for and free on the plan's own device, whichever device is current
    int cur = -1;
    const bool switched = cudaGetDevice(&cur) == cudaSuccess && cur != p->device &&
                          cudaSetDevice(p->device) == cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();
    free_plan(p);
    if (switched) cudaSetDevice(cur);
    return sp_cuda_check(e, "synchronise before destroy");
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
    if ((rc = sp_cuda_check(cudaDeviceSynchronize(), "synchronise before copy"))) return rc;
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
    cudaEvent_t e;
    sp_status rc = sp_cuda_check(cudaEventCreate(&e), "create timing event");
    if (rc) return rc;
    p->ev->push_back(e);
    return sp_cuda_check(cudaEventRecord(e, st), "record timing event");
}

extern "C" sp_status sp_plan_set_timing(sp_plan p, int enable)
{
    g_err[0] = 0;
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    p->timing = enable != 0;
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
    if (np == 0 || ev.empty()) return np;
    if (ev.size() % per != 0) { sp_fail(SP_ERR_INVALID, "incomplete timing record"); return -1; }
    if (sp_cuda_check(cudaEventSynchronize(ev.back()), "wait for timing events")) return -1;
    for (size_t s0 = 0; s0 < ev.size(); s0 += per) {
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
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    return np;
}

extern "C" const char* sp_last_error(void) { return g_err; }

extern "C" const char* sp_version(void) { return "superpot 0.1 (sm_103a)"; }
