// v2 solve passes instantiated for native FP64 arithmetic.
#include "sp_v2.cuh"

SP_V2_LINES(extern, double)

namespace v2 {
template <> const void* Tabs<double>::tw(sp_plan p, int ax) { return p->d_tw64[ax]; }
template <> const void* Tabs<double>::M(sp_plan p) { return p->d_M64; }
}  // namespace v2

sp_status sp_v2_solve_f64(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st)
{
    return v2::solve<double, double>(p, rho, u, batch, st, true);
}

sp_status sp_v2_forward_f64(sp_plan p, const void* rho, void* spec, cudaStream_t st)
{
    return v2::forward<double, double>(p, rho, spec, st);
}

float sp_v2_time_pass_f64(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st, int variant)
{
    return v2::time_pass<double, double>(p, pass, tile, batch, iters, st, variant);
}

sp_status sp_v2_radices_f64(sp_plan p, int* out) { return v2::radices<double>(p, out); }

sp_status sp_v2_persistent_f64(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st)
{
    return v2::solve_persistent<double, double>(p, rho, u, batch, st);
}
