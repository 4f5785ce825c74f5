// sp_solve_host: solves of host-resident densities end to end, with the host-to-device
// copy of the next input and the device-to-host copy of the previous result overlapping
// each solve (two copy streams, two staging buffers per direction).  Every solve is the
// one of sp_solve (Alg. 2); this file only orders copies and solves.
#include "sp_internal.h"

static sp_status make_staging(sp_plan p)
{
    if (p->staged) return SP_OK;
    const size_t io = (size_t)p->n[0] * p->n[1] * p->n[2] * (p->prec == SP_FP32 ? 4 : 8);
    sp_status rc;
    for (int i = 0; i < 4; ++i)
        if ((rc = sp_plan_alloc(p, &p->d_stage[i], io, "host-solve staging buffer"))) return rc;
    for (int i = 0; i < 2; ++i)
        if ((rc = sp_cuda_check(cudaStreamCreateWithFlags(&p->copy_st[i], cudaStreamNonBlocking), "copy stream")))
            return rc;
    for (int i = 0; i < 6; ++i)
        if ((rc = sp_cuda_check(cudaEventCreateWithFlags(&p->stage_ev[i], cudaEventDisableTiming), "copy event")))
            return rc;
    p->staged = true;
    return SP_OK;
}

extern "C" sp_status sp_solve_host(sp_plan p, const void* const* rho_h, void* const* u_h, int count,
                                   sp_stream stream)
{
    sp_clear_error();
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (count < 0) return sp_fail(SP_ERR_INVALID, "count must be >= 0 (got %d)", count);
    if (count > 0 && (!rho_h || !u_h)) return sp_fail(SP_ERR_INVALID, "rho_host and u_host must be non-NULL");
    for (int i = 0; i < count; ++i)
        if (!rho_h[i] || !u_h[i]) return sp_fail(SP_ERR_INVALID, "host array %d is NULL", i);
    if (!p->ready) return sp_fail(SP_ERR_NOT_READY, "sp_kernel_precompute has not been run on this plan");
    sp_status rc = sp_check_device(p);
    if (rc) return rc;
    if (count == 0) return SP_OK;
    if ((rc = make_staging(p))) return rc;
    cudaStream_t st = (cudaStream_t)stream, h2d = p->copy_st[0], d2h = p->copy_st[1];
    cudaEvent_t* loaded = p->stage_ev;
    cudaEvent_t* solved = p->stage_ev + 2;
    cudaEvent_t* fetched = p->stage_ev + 4;
    const size_t io = (size_t)p->n[0] * p->n[1] * p->n[2] * (p->prec == SP_FP32 ? 4 : 8);
    // staging buffers may still be in use by the previous call's work on `stream`
    if ((rc = sp_cuda_check(cudaEventRecord(solved[0], st), "order copies after earlier work"))) return rc;
    if ((rc = sp_cuda_check(cudaStreamWaitEvent(h2d, solved[0], 0), "order copies"))) return rc;
    if ((rc = sp_cuda_check(cudaStreamWaitEvent(d2h, solved[0], 0), "order copies"))) return rc;
#define SP_CK(call, what) \
    if ((rc = sp_cuda_check((call), what))) return rc
    for (int i = 0; i <= count; ++i) {
        if (i < count) {  // input i, once solve i-2 has released its buffer
            const int k = i & 1;
            if (i >= 2) SP_CK(cudaStreamWaitEvent(h2d, solved[k], 0), "wait for a free input buffer");
            SP_CK(cudaMemcpyAsync(p->d_stage[k], rho_h[i], io, cudaMemcpyHostToDevice, h2d), "copy density in");
            SP_CK(cudaEventRecord(loaded[k], h2d), "record input copy");
        }
        if (i >= 1) {  // solve i-1 once its input is in and result i-3 has left
            const int j = (i - 1) & 1;
            SP_CK(cudaStreamWaitEvent(st, loaded[j], 0), "wait for the input copy");
            if (i - 1 >= 2) SP_CK(cudaStreamWaitEvent(st, fetched[j], 0), "wait for a free output buffer");
            if ((rc = sp_run_solve(p, p->d_stage[j], p->d_stage[2 + j], 1, st))) return rc;
            SP_CK(cudaEventRecord(solved[j], st), "record solve");
            SP_CK(cudaStreamWaitEvent(d2h, solved[j], 0), "wait for the solve");
            SP_CK(cudaMemcpyAsync(u_h[i - 1], p->d_stage[2 + j], io, cudaMemcpyDeviceToHost, d2h), "copy potential out");
            SP_CK(cudaEventRecord(fetched[j], d2h), "record output copy");
        }
    }
    // the caller's stream completes only after the last result has reached the host
    SP_CK(cudaStreamWaitEvent(st, fetched[(count - 1) & 1], 0), "join the copy stream");
#undef SP_CK
    return sp_record_done(p, st);
}
