// Multi-view form: a whole umgs_render captured once in a CUDA graph and
// replayed, and an autotuner for the tile size and compositor schedule.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"
#include "radix.cuh"

struct umgs_graph {
    umgs_ctx* ctx = nullptr;
    umgs_frame* frame = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;  // kernel launches captured into the graph
};

namespace umgs {

static umgs_status graph_fail(umgs_ctx* ctx, umgs_graph* gr, umgs_status st, const std::string& msg) {
    if (gr) {
        if (gr->exec) cudaGraphExecDestroy(gr->exec);
        if (gr->graph) cudaGraphDestroy(gr->graph);
        if (gr->cap) cudaStreamDestroy(gr->cap);
        delete gr;
    }
    return fail(ctx, st, msg);
}

}  // namespace umgs

using namespace umgs;

extern "C" {

umgs_status umgs_render_graph_create(umgs_ctx* ctx, umgs_frame* frame, const umgs_gaussians* g,
                                     const umgs_mesh* meshes, int32_t nmeshes, const umgs_camera* cams,
                                     int32_t ncams, const umgs_render_opts* opts, float* out_rgbt,
                                     float key_headroom, umgs_graph** out, void* stream) {
    if (!ctx || !frame || !out) return UMGS_ERR_INVALID_ARG;
    *out = nullptr;
    if (frame->ctx != ctx) return fail(ctx, UMGS_ERR_INVALID_ARG, "frame belongs to another context");
    if (!(key_headroom >= 1.f)) key_headroom = 1.25f;
    // 1) sizing render (ordinary, synchronising): validates the arguments,
    //    sizes every buffer and uploads the cameras
    umgs_render_opts so;
    umgs_default_render_opts(&so);
    if (opts) so = *opts;
    so.flags &= ~UMGS_RENDER_ASYNC;  // the sizing render reads the pair count back
    umgs_status st = umgs_render(ctx, g, meshes, nmeshes, cams, ncams, &so, out_rgbt, frame, stream);
    if (st != UMGS_OK) return st;
    cudaStream_t us = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(us) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaStreamSynchronize");
    // 2) capacity for the pairs, with headroom, and every buffer the capture touches
    const int64_t K = frame->num_keys;
    const int64_t Kcap = (int64_t)std::ceil((double)K * key_headroom) + 4096;
    const int64_t NR = (frame->ng + frame->nt) * frame->ncams;
    const int64_t M = frame->num_tiles;
    const int64_t nbmax = std::max({radix_blocks(Kcap), radix_blocks(NR), radix_blocks(M), (int64_t)1});
    if (reserve_binning(frame, Kcap, Kcap) != cudaSuccess) return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "pairs");
    if (frame->rs_hist.reserve(sizeof(uint32_t) * 256 * nbmax) != cudaSuccess)
        return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "histograms");
    for (DevBuf* b : {&frame->ord_k, &frame->ord_v, &frame->ord_k2, &frame->ord_v2})
        if (b->reserve(sizeof(uint32_t) * std::max<int64_t>(1, M)) != cudaSuccess)
            return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "tile order");
    if (so.split > 0) {
        if (reserve_split(frame, so.split, Kcap) != cudaSuccess)
            return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "work split buffers");
        if (frame->rs_hist.reserve(sizeof(uint32_t) * 256 *
                                   std::max(nbmax, radix_blocks(M + 2 * Kcap / so.split + 1))) != cudaSuccess)
            return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "histograms");
    }
    // 3) capture on a private stream
    umgs_graph* gr = new umgs_graph();
    gr->ctx = ctx;
    gr->frame = frame;
    if (cudaStreamCreateWithFlags(&gr->cap, cudaStreamNonBlocking) != cudaSuccess)
        return graph_fail(ctx, gr, UMGS_ERR_CUDA, "cudaStreamCreate");
    const bool prof = ctx->prof.on;
    ctx->prof.on = false;
    frame->nosync = true;
    frame->capture = true;
    frame->key_capacity = Kcap;
    umgs_render_opts o = so;
    if (o.tile_size == 0) o.tile_size = 16;
    const long long launches0 = g_kernel_launches.load();
    cudaError_t e = cudaStreamBeginCapture(gr->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = render_forward(ctx, g, meshes, nmeshes, cams, ncams, o, out_rgbt, frame, gr->cap);
        // captured launches do not run: they are counted per graph launch
        gr->kernels = g_kernel_launches.load() - launches0;
        count_launch(-gr->kernels);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(gr->cap, &graph);
        gr->graph = graph;
    }
    frame->nosync = false;
    frame->capture = false;
    ctx->prof.on = prof;
    if (e != cudaSuccess) return graph_fail(ctx, gr, UMGS_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorName(e));
    if (st != UMGS_OK) return graph_fail(ctx, gr, st, "render during capture: " + ctx->err);
    if ((e = cudaGraphInstantiate(&gr->exec, gr->graph, 0)) != cudaSuccess)
        return graph_fail(ctx, gr, UMGS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorName(e));
    frame->key_capacity = Kcap;
    *out = gr;
    ctx->err.clear();
    return UMGS_OK;
}

umgs_status umgs_graph_launch(umgs_graph* gr, void* stream) {
    if (!gr || !gr->exec) return UMGS_ERR_INVALID_ARG;
    const cudaError_t e = cudaGraphLaunch(gr->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(gr->ctx, e, "cudaGraphLaunch");
    count_launch(gr->kernels);
    return UMGS_OK;
}

umgs_status umgs_graph_check(umgs_graph* gr, void* stream) {
    if (!gr) return UMGS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const umgs_status st = frame_check(gr->frame, s);
    if (st == UMGS_ERR_CAPACITY) gr->ctx->err += ": re-create the graph";
    return st;
}

void umgs_graph_destroy(umgs_graph* gr) {
    if (!gr) return;
    if (gr->exec) cudaGraphExecDestroy(gr->exec);
    if (gr->graph) cudaGraphDestroy(gr->graph);
    if (gr->cap) cudaStreamDestroy(gr->cap);
    delete gr;
}

umgs_status umgs_autotune(umgs_ctx* ctx, const umgs_gaussians* g, const umgs_mesh* meshes, int32_t nmeshes,
                          const umgs_camera* cams, int32_t ncams, umgs_render_opts* inout, float* out_rgbt,
                          double* best_ms, void* stream) {
    if (!ctx || !inout) return UMGS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    umgs_frame* fr = nullptr;
    umgs_status st = umgs_frame_create(ctx, &fr);
    if (st != UMGS_OK) return st;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int tiles[3] = {8, 16, 32};
    const int scheds[4] = {0, 1, 2, 4};
    const int splits[4] = {0, 512, 1024, 2048};
    double best = 1e30;
    umgs_render_opts bo = *inout;
    // the soft-edge compositor has the grid launch only; no split with
    // soft edges or depth (the saved state is not kept while tuning)
    const int nsched = (inout->flags & UMGS_RENDER_SOFT_EDGE) ? 1 : 4;
    const int nsplit = (inout->flags & (UMGS_RENDER_SOFT_EDGE | UMGS_RENDER_DEPTH)) ? 1 : 4;
    for (int ti = 0; ti < 3 && st == UMGS_OK; ++ti)
        for (int si = 0; si < nsched && st == UMGS_OK; ++si)
        for (int pi = 0; pi < nsplit && st == UMGS_OK; ++pi) {
            umgs_render_opts o = *inout;
            o.tile_size = tiles[ti];
            o.sched = scheds[si];
            o.split = splits[pi];
            o.flags &= ~UMGS_RENDER_SAVE_BACKWARD;
            st = umgs_render(ctx, g, meshes, nmeshes, cams, ncams, &o, out_rgbt, fr, stream);  // warm-up
            if (st != UMGS_OK) break;
            cudaEventRecord(a, s);
            for (int r = 0; r < 3 && st == UMGS_OK; ++r)
                st = umgs_render(ctx, g, meshes, nmeshes, cams, ncams, &o, out_rgbt, fr, stream);
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (st == UMGS_OK && ms / 3.0 < best) { best = ms / 3.0; bo = o; }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    umgs_frame_destroy(fr);
    if (st != UMGS_OK) return st;
    bo.flags = inout->flags;
    *inout = bo;
    if (best_ms) *best_ms = best;
    return UMGS_OK;
}

}  // extern "C"
