// v2 solve passes instantiated for FP32 arithmetic (FP32 and mixed-precision plans).
#include "sp_plane.cuh"

SP_V2_LINES(extern, float)
SP_V2_ALT(extern, float, 256)
SP_V2_ALT(extern, float, 512)
SP_V2_ALT(extern, float, 1024)

namespace v2 {
template <> const void* Tabs<float>::tw(sp_plan p, int ax) { return p->d_tw32[ax]; }
template <> const void* Tabs<float>::M(sp_plan p) { return p->d_M32; }
}  // namespace v2

sp_status sp_v2_solve_f32(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st, bool mixed)
{
    if (p->plane_fused && v2::plane_supported<float>(p))
        return mixed ? v2::solve_fused<float, double>(p, rho, u, batch, st, true)
                     : v2::solve_fused<float, float>(p, rho, u, batch, st, true);
    return mixed ? v2::solve<float, double>(p, rho, u, batch, st, true)
                 : v2::solve<float, float>(p, rho, u, batch, st, true);
}

bool sp_v2_plane_supported_f32(sp_plan p)
{
    for (int ax = 0; ax < 3; ++ax)
        if (!v2::len_ok(p->N[ax])) return false;
    return v2::plane_supported<float>(p);
}

// Mean milliseconds of `iters` whole solves of `batch` right-hand sides in the plan's
// current launch configuration (after one untimed solve), with the input and the output
// both inside the workspace: the values are meaningless, the work is that of a solve
// (no pass's amount of work depends on the data).  Host-synchronising; negative on error.
float sp_v2_time_solve_f32(sp_plan p, int batch, int iters, cudaStream_t st, bool mixed)
{
    const size_t io = (size_t)p->n[0] * p->n[1] * p->n[2] * (mixed ? 8 : 4) * batch;
    if (io > p->work_bytes || batch < 1 || batch > p->max_batch || iters < 1) return -1.f;
    sp_plan_s view = *p;
    view.timing = false;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.f;
    }
    sp_status rc = SP_OK;
    for (int it = -1; it < iters && rc == SP_OK; ++it) {  // it = -1: warm-up solve
        if (it == 0) cudaEventRecord(e0, st);
        rc = sp_v2_solve_f32(&view, p->d_work, p->d_work, batch, st, mixed);
    }
    cudaEventRecord(e1, st);
    float ms = -1.f;
    if (rc == SP_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        ms /= iters;
    else
        ms = -1.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

sp_status sp_v2_forward_f32(sp_plan p, const void* rho, void* spec, cudaStream_t st, bool mixed)
{
    return mixed ? v2::forward<float, double>(p, rho, spec, st) : v2::forward<float, float>(p, rho, spec, st);
}

float sp_v2_time_pass_f32(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st, bool mixed, int variant)
{
    return mixed ? v2::time_pass<float, double>(p, pass, tile, batch, iters, st, variant)
                 : v2::time_pass<float, float>(p, pass, tile, batch, iters, st, variant);
}

sp_status sp_v2_radices_f32(sp_plan p, int* out) { return v2::radices<float>(p, out); }

sp_status sp_v2_stage_twiddles_f32(sp_plan p, cudaStream_t st)
{
    return v2::stage_twiddles<float>(p, st);
}

sp_status sp_v2_persistent_f32(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st, bool mixed)
{
    return mixed ? v2::solve_persistent<float, double>(p, rho, u, batch, st)
                 : v2::solve_persistent<float, float>(p, rho, u, batch, st);
}

namespace {
struct HasAltF32 {
    template <int N> sp_status run() { return AltPlan<float, N>::exists ? SP_OK : SP_ERR_UNSUPPORTED_SIZE; }
};
}  // namespace

bool sp_v2_has_alt_f32(int N) { return v2::with_len(N, HasAltF32{}) == SP_OK; }
