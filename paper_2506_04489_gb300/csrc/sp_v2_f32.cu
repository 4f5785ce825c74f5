// v2 solve passes instantiated for FP32 arithmetic (FP32 and mixed-precision plans).
#include "sp_v2.cuh"

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
    return mixed ? v2::solve<float, double>(p, rho, u, batch, st, true)
                 : v2::solve<float, float>(p, rho, u, batch, st, true);
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
