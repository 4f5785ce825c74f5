// v2 solve passes instantiated for double-float arithmetic (FP64 input and output,
// passes on pairs of FP32 values, see sp_df32.cuh).
#include "sp_v2.cuh"

SP_V2_LINES(extern, df32)
SP_V2_ALT(extern, df32, 256)

namespace v2 {
template <> const void* Tabs<df32>::tw(sp_plan p, int ax) { return p->d_twdf[ax]; }
template <> const void* Tabs<df32>::M(sp_plan p) { return p->d_Mdf; }
}  // namespace v2

sp_status sp_v2_solve_df(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st)
{
    return v2::solve<df32, double>(p, rho, u, batch, st, true);
}

sp_status sp_v2_forward_df(sp_plan p, const void* rho, void* spec, cudaStream_t st)
{
    return v2::forward<df32, double>(p, rho, spec, st);
}

sp_status sp_v2_stage_twiddles_df(sp_plan p, cudaStream_t st)
{
    return v2::stage_twiddles<df32>(p, st);
}

float sp_v2_time_pass_df(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st, int variant)
{
    return v2::time_pass<df32, double>(p, pass, tile, batch, iters, st, variant);
}

sp_status sp_v2_radices_df(sp_plan p, int* out) { return v2::radices<df32>(p, out); }

sp_status sp_v2_persistent_df(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st)
{
    return v2::solve_persistent<df32, double>(p, rho, u, batch, st);
}

namespace {
struct HasAltDF {
    template <int N> sp_status run() { return AltPlan<df32, N>::exists ? SP_OK : SP_ERR_UNSUPPORTED_SIZE; }
};
}  // namespace

bool sp_v2_has_alt_df(int N) { return v2::with_len(N, HasAltDF{}) == SP_OK; }
