// Batched execution helpers: the tile autotuner and CUDA-graph capture of a solve.
//
// The autotuner picks, per pass, the CTA tile of the register-resident passes (columns
// per CTA of the y and x line passes, pairs of real lines per CTA of the z passes) by
// timing every candidate on the plan's own workspace.  Tiles change which lines share a
// CTA, never the arithmetic of a line, so results are bitwise the same for every tile.
//
// A captured graph replays a (batched) solve on fixed buffers with one host-side launch:
// five kernel nodes, each over the whole batch.
#include <new>

#include "sp_internal.h"

struct sp_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    sp_plan plan;  // its completion event is recorded after every replay
};

static float time_pass(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st)
{
    switch (p->prec) {
        case SP_FP64: return sp_v2_time_pass_f64(p, pass, tile, batch, iters, st);
        case SP_FP32: return sp_v2_time_pass_f32(p, pass, tile, batch, iters, st, false);
        case SP_MIXED: return sp_v2_time_pass_f32(p, pass, tile, batch, iters, st, true);
        case SP_DF32: return sp_v2_time_pass_df(p, pass, tile, batch, iters, st);
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
    int best_tile[3] = {0, 0, 0};
    for (int pass = 0; pass < 3; ++pass) {
        float best = -1.f;
        for (int c = 0; c < 6; ++c) {
            float ms = time_pass(p, pass, candidates[c], batch, 5, st);
            sp_clear_error();  // tiles beyond a pass's limit report an error: skip them
            if (ms > 0.f && (best < 0.f || ms < best)) {
                best = ms;
                best_tile[pass] = candidates[c];
            }
        }
        if (best < 0.f) return sp_fail(SP_ERR_CUDA, "autotune: no tile of pass %d ran", pass);
    }
    p->tile_z = best_tile[0];
    p->tile_line[1] = best_tile[1];
    p->tile_line[0] = best_tile[2];
    return sp_cuda_check(cudaStreamSynchronize(st), "autotune");
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
