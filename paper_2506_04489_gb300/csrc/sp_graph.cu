// Batched execution helpers: the tile autotuner and CUDA-graph capture of a solve.
//
// The autotuner picks, per pass, the CTA tile of the register-resident passes (columns
// per CTA of the y and x line passes, pairs of real lines per CTA of the z passes) by
// timing every candidate on the plan's own workspace.  Tiles change which lines share a
// CTA, never the arithmetic of a line, so results are bitwise the same for every tile.
//
// A captured graph replays a (batched) solve on fixed buffers with one host-side launch:
// five kernel nodes, each over the whole batch, or (persistent plans) one cooperative
// kernel node running all five passes with grid barriers between them.
#include <new>

#include "sp_internal.h"

struct sp_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    sp_plan plan;  // its completion event is recorded after every replay
};

static float time_pass(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st, int variant)
{
    switch (p->prec) {
        case SP_FP64: return sp_v2_time_pass_f64(p, pass, tile, batch, iters, st, variant);
        case SP_FP32: return sp_v2_time_pass_f32(p, pass, tile, batch, iters, st, false, variant);
        case SP_MIXED: return sp_v2_time_pass_f32(p, pass, tile, batch, iters, st, true, variant);
        case SP_DF32: return sp_v2_time_pass_df(p, pass, tile, batch, iters, st, variant);
    }
    return -1.f;
}

extern "C" sp_status sp_plan_autotune(sp_plan p, int batch, sp_stream stream)
{
    sp_clear_error();
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (!p->ready) return sp_fail(SP_ERR_NOT_READY, "sp_kernel_precompute has not been run on this plan");
    if (batch < 1 || batch > p->max_batch)
        return sp_fail(SP_ERR_INVALID, "batch %d outside [1, max_batch = %d]", batch, p->max_batch);
    if (sp_status rc = sp_check_device(p)) return rc;
    for (int ax = 0; ax < 3; ++ax)
        if (!sp_v2_supported(p->N[ax])) return SP_OK;  // first-generation passes: nothing to tune
    cudaStream_t st = (cudaStream_t)stream;
    const int candidates[6] = {1, 2, 4, 8, 16, 32};
    int best_tile[3] = {0, 0, 0}, best_variant[3] = {0, 0, 0};
    for (int pass = 0; pass < 3; ++pass) {
        float best = -1.f;
        // the line passes (1: y, 2: x) also try the alternative radix plan of their length
        for (int variant = 0; variant < (pass == 0 ? 1 : 2); ++variant) {
            for (int c = 0; c < 6; ++c) {
                float ms = time_pass(p, pass, candidates[c], batch, 5, st, variant);
                sp_clear_error();  // tiles beyond a pass's limit, and absent plans, report an error: skip them
                if (ms > 0.f && (best < 0.f || ms < best)) {
                    best = ms;
                    best_tile[pass] = candidates[c];
                    best_variant[pass] = variant;
                }
            }
        }
        if (best < 0.f) return sp_fail(SP_ERR_CUDA, "autotune: no tile of pass %d ran", pass);
    }
    p->tile_z = best_tile[0];
    p->tile_line[1] = best_tile[1];
    p->tile_line[0] = best_tile[2];
    p->line_variant[1] = best_variant[1];
    p->line_variant[0] = best_variant[2];
    // FP32 and mixed: the fused three-pass schedule against the five passes, whole solves
    p->plane_fused = false;
    if ((p->prec == SP_FP32 || p->prec == SP_MIXED) && sp_v2_plane_supported_f32(p)) {
        const bool mixed = p->prec == SP_MIXED;
        const float five = sp_v2_time_solve_f32(p, batch, 5, st, mixed);
        p->plane_fused = true;
        const float fused = sp_v2_time_solve_f32(p, batch, 5, st, mixed);
        sp_clear_error();
        p->plane_fused = fused > 0.f && (five < 0.f || fused < five);
    }
    return sp_cuda_check(cudaStreamSynchronize(st), "autotune");
}

extern "C" sp_status sp_plan_launch_config(const sp_plan p, int* line_tiles, int* z_tile, int* line_plan, int* radices,
                                           int* schedule)
{
    sp_clear_error();
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (schedule) *schedule = p->persistent ? 2 : (p->plane_fused ? 1 : 0);
    if (line_tiles)
        for (int ax = 0; ax < 3; ++ax) line_tiles[ax] = p->tile_line[ax];
    if (z_tile) *z_tile = p->tile_z;
    if (line_plan)
        for (int ax = 0; ax < 3; ++ax) line_plan[ax] = p->line_variant[ax];
    if (radices) {
        for (int i = 0; i < 24; ++i) radices[i] = 0;
        bool v2 = true;
        for (int ax = 0; ax < 3; ++ax) v2 = v2 && sp_v2_supported(p->N[ax]);
        if (v2) {
            sp_status rc = SP_OK;
            switch (p->prec) {
                case SP_FP64: rc = sp_v2_radices_f64(p, radices); break;
                case SP_FP32:
                case SP_MIXED: rc = sp_v2_radices_f32(p, radices); break;
                case SP_DF32: rc = sp_v2_radices_df(p, radices); break;
            }
            if (rc) return rc;
        } else {  // first-generation passes: the runtime stage plans
            for (int ax = 0; ax < 3; ++ax)
                for (int s = 0; s < p->rp[ax].nst && s < 8; ++s) radices[8 * ax + s] = p->rp[ax].r[s];
        }
    }
    return SP_OK;
}

extern "C" sp_status sp_plan_set_launch_config(sp_plan p, const int* line_tiles, int z_tile, const int* line_plan,
                                               int schedule)
{
    sp_clear_error();
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (z_tile < 0) return sp_fail(SP_ERR_INVALID, "z_tile must be >= 0 (got %d)", z_tile);
    if (schedule < -1 || schedule > 1) return sp_fail(SP_ERR_INVALID, "schedule must be -1, 0 or 1 (got %d)", schedule);
    if (schedule == 1 && !((p->prec == SP_FP32 || p->prec == SP_MIXED) && sp_v2_plane_supported_f32(p)))
        return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "no fused plane passes for this grid and precision");
    if (line_tiles)
        for (int ax = 0; ax < 3; ++ax)
            if (line_tiles[ax] < 0) return sp_fail(SP_ERR_INVALID, "line_tiles[%d] must be >= 0", ax);
    if (line_plan) {
        if (line_plan[2] != 0) return sp_fail(SP_ERR_INVALID, "line_plan[2] must be 0 (the z passes have no line plan)");
        for (int ax = 0; ax < 2; ++ax) {
            if (line_plan[ax] != 0 && line_plan[ax] != 1)
                return sp_fail(SP_ERR_INVALID, "line_plan[%d] must be 0 or 1", ax);
            if (line_plan[ax] == 1) {
                const bool has = (p->prec == SP_FP32 || p->prec == SP_MIXED) ? sp_v2_has_alt_f32(p->N[ax])
                                 : p->prec == SP_DF32                         ? sp_v2_has_alt_df(p->N[ax])
                                                                              : false;
                if (!has)
                    return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "no alternative radix plan for axis %d (2n = %d) in this precision",
                                   ax, p->N[ax]);
            }
        }
    }
    if (line_tiles)
        for (int ax = 0; ax < 3; ++ax) p->tile_line[ax] = line_tiles[ax];
    p->tile_z = z_tile;
    if (line_plan)
        for (int ax = 0; ax < 2; ++ax) p->line_variant[ax] = line_plan[ax];
    if (schedule >= 0) p->plane_fused = schedule == 1;
    return SP_OK;
}

extern "C" sp_status sp_plan_tiles(const sp_plan p, int* line_tiles, int* z_tile)
{
    sp_clear_error();
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (line_tiles)
        for (int ax = 0; ax < 3; ++ax) line_tiles[ax] = p->tile_line[ax];
    if (z_tile) *z_tile = p->tile_z;
    return SP_OK;
}

extern "C" sp_status sp_graph_capture(sp_plan p, const void* rho, void* u, int batch, sp_stream stream,
                                      sp_graph* out)
{
    sp_clear_error();
    if (!out) return sp_fail(SP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (!rho || !u) return sp_fail(SP_ERR_INVALID, "rho and u must be non-NULL device pointers");
    if (!p->ready) return sp_fail(SP_ERR_NOT_READY, "sp_kernel_precompute has not been run on this plan");
    if (batch < 1 || batch > p->max_batch)
        return sp_fail(SP_ERR_INVALID, "batch %d outside [1, max_batch = %d]", batch, p->max_batch);
    if (!stream) return sp_fail(SP_ERR_INVALID, "graph capture needs a created stream, not the legacy default");
    if (sp_status rc0 = sp_check_device(p)) return rc0;
    cudaStream_t st = (cudaStream_t)stream;
    // one eager solve first: it sets every kernel attribute outside the capture
    sp_plan_s view = *p;
    view.timing = false;
    sp_status rc = sp_run_solve(&view, rho, u, batch, st);
    if (rc) return rc;
    if ((rc = sp_cuda_check(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture")))
        return rc;
    rc = sp_run_solve(&view, rho, u, batch, st);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if ((rc = sp_cuda_check(e, "end capture"))) return rc;
    cudaGraphExec_t exec = nullptr;
    if ((rc = sp_cuda_check(cudaGraphInstantiate(&exec, graph, 0), "instantiate graph"))) {
        cudaGraphDestroy(graph);
        return rc;
    }
    sp_graph g = new (std::nothrow) sp_graph_s;
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return sp_fail(SP_ERR_OOM, "host allocation failed");
    }
    g->graph = graph;
    g->exec = exec;
    g->plan = p;
    *out = g;
    return sp_record_done(p, st);
}

extern "C" sp_status sp_graph_launch(sp_graph g, sp_stream stream)
{
    sp_clear_error();
    if (!g) return sp_fail(SP_ERR_INVALID, "graph is NULL");
    sp_status rc = sp_cuda_check(cudaGraphLaunch(g->exec, (cudaStream_t)stream), "graph launch");
    if (rc) return rc;
    return sp_record_done(g->plan, (cudaStream_t)stream);
}

extern "C" sp_status sp_graph_destroy(sp_graph g)
{
    sp_clear_error();
    if (!g) return SP_OK;
    cudaError_t e = cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return sp_cuda_check(e, "destroy graph");
}

extern "C" sp_status sp_plan_set_persistent(sp_plan p, int enable)
{
    sp_clear_error();
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (enable && !(p->N[0] == p->N[1] && p->N[1] == p->N[2] && sp_v2_supported(p->N[0])))
        return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "the persistent solve needs a cubic grid with a compiled padded length");
    p->persistent = enable != 0;
    return SP_OK;
}

// Diagnostic of the bounded grid wait: `blocks` co-resident blocks of 32 threads each
// arrive once at a barrier that waits for `expected` arrivals.
__global__ void k_barrier_check(unsigned* count, int* status, unsigned expected, unsigned long long limit_ns)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        unsigned long long t0, t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        const unsigned long long max_polls = limit_ns / 16 + 1024;
        for (unsigned long long it = 0;; ++it) {
            if (*(volatile unsigned*)count >= expected) break;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (it >= max_polls || t - t0 > limit_ns) {
                atomicExch(status, 1);
                break;
            }
            __nanosleep(128);
        }
        __threadfence();
    }
    __syncthreads();
}

extern "C" sp_status sp_plan_barrier_check(sp_plan p, int blocks, int expected, double limit_ms, sp_stream stream)
{
    sp_clear_error();
    if (!p) return sp_fail(SP_ERR_INVALID, "plan is NULL");
    if (sp_status rc = sp_check_device(p)) return rc;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks < 1 || blocks > sms) return sp_fail(SP_ERR_INVALID, "blocks must be in [1, %d] (got %d)", sms, blocks);
    if (expected < 1) return sp_fail(SP_ERR_INVALID, "expected must be >= 1 (got %d)", expected);
    if (!(limit_ms > 0.0 && limit_ms <= 2000.0)) return sp_fail(SP_ERR_INVALID, "limit_ms must be in (0, 2000]");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned* bar = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(p->d_status) + 64);
    sp_status rc = sp_cuda_check(cudaMemsetAsync(bar, 0, sizeof(unsigned), st), "clear grid barrier");
    if (rc) return rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all blocks co-resident
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const unsigned long long limit_ns = (unsigned long long)(limit_ms * 1e6);
    if ((rc = sp_cuda_check(cudaLaunchKernelEx(&cfg, k_barrier_check, bar, p->d_status, (unsigned)expected, limit_ns),
                            "barrier check launch")))
        return rc;
    return sp_record_done(p, st);
}
