// C ABI of libumgs: argument validation, contexts and frames.
#include <cstring>
#include <string>

#include "internal.h"

std::atomic<long long> g_kernel_launches{0};

namespace umgs {

umgs_status fail(umgs_ctx* ctx, umgs_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}

umgs_status cuda_fail(umgs_ctx* ctx, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(ctx, UMGS_ERR_CUDA, m);
}

// Alignment of the SH array that the colour kernel's vector loads need: a
// row of (degree + 1)^2 x 3 coefficients read as 16-byte words when its bytes
// are a multiple of 16, as 8-byte words when a multiple of 8.
static uintptr_t sh_alignment(int degree, int dtype) {
    const int row = (degree + 1) * (degree + 1) * 3 * (dtype == UMGS_BF16 ? 2 : 4);
    return row % 16 == 0 ? 16 : row % 8 == 0 ? 8 : 1;
}

}  // namespace umgs

using namespace umgs;

extern "C" {

umgs_status umgs_ctx_create(umgs_ctx** out, int device) {
    if (!out) return UMGS_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return UMGS_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return UMGS_ERR_CUDA;
    umgs_ctx* c = new umgs_ctx();
    c->device = device;
    if (cudaMallocHost(reinterpret_cast<void**>(&c->pinned), 64 * sizeof(int64_t)) != cudaSuccess) {
        delete c;
        return UMGS_ERR_OUT_OF_MEMORY;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (c->dstatus.reserve(16) != cudaSuccess || cudaMemset(c->dstatus.ptr, 0, 16) != cudaSuccess) {
        cudaFreeHost(c->pinned);
        delete c;
        return UMGS_ERR_OUT_OF_MEMORY;
    }
    c->default_frame = new umgs_frame();
    c->default_frame->ctx = c;
    c->default_frame->device = device;
    *out = c;
    return UMGS_OK;
}

void umgs_ctx_destroy(umgs_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->default_frame) {
        ctx->default_frame->release();
        delete ctx->default_frame;
    }
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    for (auto& r : ctx->prof.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->prof.pool) cudaEventDestroy(e);
    ctx->dstatus.release();
    ctx->vacc.release();
    ctx->vtab.release();
    ctx->bind_ws.release();
    ctx->bind_cams.release();
    ctx->bind_cnt.release();
    delete ctx;
    cudaGetLastError();  // leave no error of the teardown behind for the next call
}

const char* umgs_last_error(const umgs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

umgs_status umgs_ctx_sync(umgs_ctx* ctx, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(ctx->pinned, ctx->dstatus.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "umgs_ctx_sync");
    const int32_t st = (int32_t)(ctx->pinned[0] & 0xffffffff);
    if (st != 0) {
        cudaMemsetAsync(ctx->dstatus.ptr, 0, sizeof(int32_t), s);
        cudaStreamSynchronize(s);
        return fail(ctx, UMGS_ERR_INVALID_ARG, "a kernel saw an out-of-range face or vertex index (status " +
                                                   std::to_string(st) + ")");
    }
    return UMGS_OK;
}

long long umgs_kernel_launches(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

umgs_status umgs_profile_enable(umgs_ctx* ctx, int32_t on) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->prof.on = on != 0;
    return UMGS_OK;
}

umgs_status umgs_profile_read(umgs_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx || !ms || !launches) return UMGS_ERR_INVALID_ARG;
    for (int k = 0; k < UMGS_NUM_STAGES; ++k) { ms[k] = 0.0; launches[k] = 0; }
    umgs_status st = UMGS_OK;
    for (auto& r : ctx->prof.recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            st = fail(ctx, UMGS_ERR_CUDA, "cudaEventElapsedTime");
        if (r.stage >= 0 && r.stage < UMGS_NUM_STAGES) { ms[r.stage] += t; launches[r.stage] += 1; }
        ctx->prof.pool.push_back(r.a);
        ctx->prof.pool.push_back(r.b);
    }
    ctx->prof.recs.clear();
    return st;
}

void umgs_default_render_opts(umgs_render_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tile_size = 16;
    o->blend_mode = UMGS_BLEND_FULL;
    o->t_eps = 1e-4f;
}

umgs_status umgs_frame_create(umgs_ctx* ctx, umgs_frame** out) {
    if (!ctx || !out) return UMGS_ERR_INVALID_ARG;
    umgs_frame* f = new umgs_frame();
    f->ctx = ctx;
    f->device = ctx->device;
    *out = f;
    ctx->err.clear();
    return UMGS_OK;
}

void umgs_frame_destroy(umgs_frame* frame) {
    if (!frame) return;
    // (the device is the frame's own copy: its context may be gone already)
    cudaSetDevice(frame->device);
    cudaDeviceSynchronize();
    frame->release();
    delete frame;
    cudaGetLastError();  // leave no error of the teardown behind for the next call
}

umgs_status umgs_render(umgs_ctx* ctx, const umgs_gaussians* g, const umgs_mesh* meshes, int32_t nmeshes,
                        const umgs_camera* cams, int32_t ncams, const umgs_render_opts* opts_in, float* out_rgbt,
                        umgs_frame* frame, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    umgs_render_opts opts;
    umgs_default_render_opts(&opts);
    if (opts_in) opts = *opts_in;
    if (opts.tile_size == 0) opts.tile_size = 16;
    if (opts.tile_size != 8 && opts.tile_size != 16 && opts.tile_size != 32)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "tile_size must be 8, 16 or 32");
    if (opts.blend_mode < 0 || opts.blend_mode > 3) return fail(ctx, UMGS_ERR_INVALID_ARG, "unknown blend_mode");
    if ((opts.flags & UMGS_RENDER_T_PRODUCT) &&
        (opts.blend_mode != UMGS_BLEND_FULL || (opts.flags & UMGS_RENDER_SAVE_BACKWARD)))
        return fail(ctx, UMGS_ERR_INVALID_ARG, "UMGS_RENDER_T_PRODUCT needs FULL mode and no saved backward state");
    if ((opts.flags & UMGS_RENDER_DEPTH) &&
        (!frame || opts.blend_mode != UMGS_BLEND_FULL ||
         (opts.flags & (UMGS_RENDER_SAVE_BACKWARD | UMGS_RENDER_MIXED | UMGS_RENDER_T_PRODUCT))))
        return fail(ctx, UMGS_ERR_INVALID_ARG,
                    "UMGS_RENDER_DEPTH needs a frame, FULL mode and none of SAVE_BACKWARD, MIXED, T_PRODUCT");
    if ((opts.flags & UMGS_RENDER_SOFT_EDGE) &&
        (opts.blend_mode != UMGS_BLEND_FULL || !(opts.edge_sigma > 0.f) || !(opts.edge_sigma <= 16.f) ||
         opts.sched > 0 || (opts.flags & (UMGS_RENDER_MIXED | UMGS_RENDER_T_PRODUCT | UMGS_RENDER_DEPTH))))
        return fail(ctx, UMGS_ERR_INVALID_ARG,
                    "UMGS_RENDER_SOFT_EDGE needs FULL mode, 0 < edge_sigma <= 16, sched 0 and none of MIXED, "
                    "T_PRODUCT, DEPTH");
    if (opts.split != 0 &&
        (opts.split < 256 || opts.split > (1 << 20) ||
         (opts.flags & (UMGS_RENDER_SAVE_BACKWARD | UMGS_RENDER_DEPTH | UMGS_RENDER_SOFT_EDGE))))
        return fail(ctx, UMGS_ERR_INVALID_ARG,
                    "split must be 0 or 256..1048576, and not with SAVE_BACKWARD, DEPTH or SOFT_EDGE");
    if (!cams || ncams < 1) return fail(ctx, UMGS_ERR_INVALID_ARG, "need at least one camera");
    if (!out_rgbt) return fail(ctx, UMGS_ERR_INVALID_ARG, "out_rgbt is NULL");
    if (reinterpret_cast<uintptr_t>(out_rgbt) & 15)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "out_rgbt must be 16-byte aligned");
    if (nmeshes < 0 || (nmeshes > 0 && !meshes)) return fail(ctx, UMGS_ERR_INVALID_ARG, "bad mesh array");
    for (int c = 0; c < ncams; ++c) {
        if (cams[c].width != cams[0].width || cams[c].height != cams[0].height)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "all cameras must share width and height");
        if (cams[c].width < 1 || cams[c].height < 1 || cams[c].width > 32768 || cams[c].height > 32768)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "image size out of range (1..32768)");
        if (!(cams[c].fx > 0.f) || !(cams[c].fy > 0.f) || !(cams[c].near_z > 0.f))
            return fail(ctx, UMGS_ERR_INVALID_ARG, "fx, fy and near_z must be positive");
    }
    if (g && g->n > 0) {
        if (!g->means || !g->opacities || !g->sh) return fail(ctx, UMGS_ERR_INVALID_ARG, "Gaussian array is NULL");
        if (!g->cov3d && (!g->quats || !g->scales))
            return fail(ctx, UMGS_ERR_INVALID_ARG, "need quats+scales or cov3d");
        if (g->sh_degree < 0 || g->sh_degree > 3) return fail(ctx, UMGS_ERR_INVALID_ARG, "sh_degree must be 0..3");
        if (g->sh_dtype != UMGS_F32 && g->sh_dtype != UMGS_BF16)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "sh_dtype must be UMGS_F32 or UMGS_BF16");
        if (reinterpret_cast<uintptr_t>(g->sh) & (sh_alignment(g->sh_degree, g->sh_dtype) - 1))
            return fail(ctx, UMGS_ERR_INVALID_ARG,
                        "sh must be 16-byte aligned (8-byte for bfloat16 degree 1; see umgs_gaussians)");
    }
    if (g && g->n < 0) return fail(ctx, UMGS_ERR_INVALID_ARG, "negative Gaussian count");
    for (int m = 0; m < nmeshes; ++m) {
        const umgs_mesh& me = meshes[m];
        if (me.nf < 0 || me.nv < 0) return fail(ctx, UMGS_ERR_INVALID_ARG, "negative mesh size");
        const bool textured = me.uv || me.texture;
        if (textured && (!me.uv || !me.texture || me.tex_w < 1 || me.tex_h < 1))
            return fail(ctx, UMGS_ERR_INVALID_ARG, "a textured mesh needs uv, texture and tex_w, tex_h >= 1");
        if (me.nf > 0 && (!me.verts || !me.faces || (!me.vcolor && !textured) || me.nv < 1))
            return fail(ctx, UMGS_ERR_INVALID_ARG, "mesh array is NULL");
    }
    {   // unified 32-bit primitive ids; (camera, region) keys of 22 bits
        int64_t nprim = (g && g->n > 0) ? g->n : 0;
        for (int m = 0; m < nmeshes; ++m) nprim += meshes[m].nf;
        if (nprim > (int64_t)0xfffffffe)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "more than 4294967294 primitives (Gaussians + triangles)");
        const int64_t tx = (cams[0].width + opts.tile_size - 1) / opts.tile_size;
        const int64_t ty = (cams[0].height + opts.tile_size - 1) / opts.tile_size;
        const int64_t regions = (int64_t)ncams * ((tx + 7) / 8) * ((ty + 3) / 4);
        if (regions > ((int64_t)1 << 22))
            return fail(ctx, UMGS_ERR_INVALID_ARG,
                        "more than 2^22 regions of 8x4 tiles over the cameras (fewer cameras or larger tiles)");
    }
    umgs_frame* fr = frame ? frame : ctx->default_frame;
    if (fr->ctx != ctx) return fail(ctx, UMGS_ERR_INVALID_ARG, "frame belongs to another context");
    const bool async = (opts.flags & UMGS_RENDER_ASYNC) != 0;
    if (async && (!frame || frame->key_capacity < 1))
        return fail(ctx, UMGS_ERR_INVALID_ARG, "UMGS_RENDER_ASYNC needs a frame with a reserved pair capacity");
    umgs_gaussians empty;
    std::memset(&empty, 0, sizeof(empty));
    fr->nosync = async;
    const umgs_status st = render_forward(ctx, g ? g : &empty, meshes, nmeshes, cams, ncams, opts, out_rgbt, fr,
                                          static_cast<cudaStream_t>(stream));
    fr->nosync = false;
    return st;
}

umgs_status umgs_frame_reserve(umgs_frame* frame, int64_t key_capacity) {
    if (!frame || key_capacity < 1) return UMGS_ERR_INVALID_ARG;
    frame->key_capacity = key_capacity;
    return UMGS_OK;
}

umgs_status umgs_frame_check(umgs_frame* frame, void* stream) {
    if (!frame) return UMGS_ERR_INVALID_ARG;
    frame->ctx->err.clear();
    return frame_check(frame, static_cast<cudaStream_t>(stream));
}

umgs_status umgs_render_backward(umgs_ctx* ctx, umgs_frame* frame, const umgs_gaussians* g,
                                 const umgs_mesh* meshes, int32_t nmeshes, const float* dL_drgbt,
                                 const umgs_gaussian_grads* gg, const umgs_mesh_grads* mg, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    if (!frame || frame->ctx != ctx || !frame->valid) return fail(ctx, UMGS_ERR_INVALID_ARG, "no rendered frame");
    if (frame->blend_mode != UMGS_BLEND_FULL)
        return fail(ctx, UMGS_ERR_NOT_IMPLEMENTED, "backward is implemented for blend mode FULL");
    if (!frame->saved) return fail(ctx, UMGS_ERR_INVALID_ARG, "render without UMGS_RENDER_SAVE_BACKWARD");
    if (frame->mixed) return fail(ctx, UMGS_ERR_NOT_IMPLEMENTED, "backward of a mixed-precision render");
    if (!dL_drgbt) return fail(ctx, UMGS_ERR_INVALID_ARG, "dL_drgbt is NULL");
    if (reinterpret_cast<uintptr_t>(dL_drgbt) & 15)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "dL_drgbt must be 16-byte aligned");
    if (g && g->n > 0 && !g->cov3d && (reinterpret_cast<uintptr_t>(g->quats) & 15))
        return fail(ctx, UMGS_ERR_INVALID_ARG, "quats must be 16-byte aligned for the backward");
    if (gg && (reinterpret_cast<uintptr_t>(gg->quats) & 15))
        return fail(ctx, UMGS_ERR_INVALID_ARG, "the quats gradient must be 16-byte aligned");
    const int64_t ng = g ? g->n : 0;
    if (ng != frame->ng) return fail(ctx, UMGS_ERR_INVALID_ARG, "Gaussian count differs from the forward call");
    if (nmeshes != (int32_t)frame->mesh_offset.size() || (nmeshes > 0 && !meshes))
        return fail(ctx, UMGS_ERR_INVALID_ARG, "mesh count differs from the forward call");
    int64_t nt = 0;
    for (int m = 0; m < nmeshes; ++m) {
        nt += meshes[m].nf;
        if (meshes[m].uv || meshes[m].texture)
            return fail(ctx, UMGS_ERR_NOT_IMPLEMENTED, "backward of a textured mesh");
    }
    if (nt != frame->nt) return fail(ctx, UMGS_ERR_INVALID_ARG, "triangle count differs from the forward call");
    umgs_gaussians empty;
    std::memset(&empty, 0, sizeof(empty));
    return render_backward(ctx, frame, g ? g : &empty, meshes, nmeshes, dL_drgbt, gg, mg,
                           static_cast<cudaStream_t>(stream));
}

umgs_status umgs_deform(umgs_ctx* ctx, const umgs_gaussians* rest, const int32_t* face, const float* bary,
                        const float* proxy_v, const float* proxy_vd, const int32_t* proxy_f, int64_t nv,
                        int64_t nf, int32_t mode, float* out_means, float* out_cov3d, float* out_quats,
                        void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    if (!rest || rest->n < 0) return fail(ctx, UMGS_ERR_INVALID_ARG, "rest Gaussians missing");
    if ((mode & ~(UMGS_DEFORM_LITERAL | UMGS_DEFORM_ONE_RING)) != 0)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "bad mode");
    if (!proxy_v || !proxy_vd || !proxy_f || nv < 3 || nf < 1) return fail(ctx, UMGS_ERR_INVALID_ARG, "bad proxy mesh");
    if (rest->n > 0) {
        if (!rest->means || !face || !bary || !out_means || !out_cov3d)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL array");
        if (!rest->cov3d && (!rest->quats || !rest->scales))
            return fail(ctx, UMGS_ERR_INVALID_ARG, "need quats+scales or cov3d");
        if ((reinterpret_cast<uintptr_t>(face) | reinterpret_cast<uintptr_t>(bary)) & 15)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "face and bary must be 16-byte aligned");
    }
    return deform_forward(ctx, rest, face, bary, proxy_v, proxy_vd, proxy_f, nv, nf, mode, out_means, out_cov3d,
                          out_quats, static_cast<cudaStream_t>(stream));
}

umgs_status umgs_binding_compact(umgs_ctx* ctx, const int32_t* face, const float* bary, int64_t n,
                                 const int32_t* proxy_f, int64_t nv, int64_t nf, int32_t* out_count,
                                 int32_t* out_entries, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    if (n < 0 || nv < 3 || nf < 1 || !proxy_f) return fail(ctx, UMGS_ERR_INVALID_ARG, "bad sizes or proxy mesh");
    if (n > 0 && (!face || !bary || !out_count || !out_entries)) return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL array");
    if ((reinterpret_cast<uintptr_t>(bary) | reinterpret_cast<uintptr_t>(out_entries)) & 7)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "bary and out_entries must be 8-byte aligned");
    return binding_compact(ctx, face, bary, n, proxy_f, nv, nf, out_count, reinterpret_cast<int2*>(out_entries),
                           static_cast<cudaStream_t>(stream));
}

umgs_status umgs_deform_compact(umgs_ctx* ctx, const umgs_gaussians* rest, const int32_t* count,
                                const int32_t* entries, const float* proxy_v, const float* proxy_vd,
                                const int32_t* proxy_f, int64_t nv, int64_t nf, int32_t mode, float* out_means,
                                float* out_cov3d, float* out_quats, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    if (!rest || rest->n < 0) return fail(ctx, UMGS_ERR_INVALID_ARG, "rest Gaussians missing");
    if ((mode & ~(UMGS_DEFORM_LITERAL | UMGS_DEFORM_ONE_RING)) != 0)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "bad mode");
    if (!proxy_v || !proxy_vd || !proxy_f || nv < 3 || nf < 1) return fail(ctx, UMGS_ERR_INVALID_ARG, "bad proxy mesh");
    if (rest->n > 0) {
        if (!rest->means || !count || !entries || !out_means || !out_cov3d)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL array");
        if (!rest->cov3d && (!rest->quats || !rest->scales))
            return fail(ctx, UMGS_ERR_INVALID_ARG, "need quats+scales or cov3d");
        if (reinterpret_cast<uintptr_t>(entries) & 15)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "entries must be 16-byte aligned");
    }
    return deform_compact_forward(ctx, rest, count, reinterpret_cast<const int2*>(entries), proxy_v, proxy_vd,
                                  proxy_f, nv, nf, mode, out_means, out_cov3d, out_quats,
                                  static_cast<cudaStream_t>(stream));
}

umgs_status umgs_binding_csr(umgs_ctx* ctx, const int32_t* face, const float* bary, int64_t n,
                             const int32_t* proxy_f, int64_t nv, int64_t nf, int32_t* out_offsets,
                             int32_t* out_entries, int64_t cap, int64_t* out_total, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    if (n < 0 || nv < 3 || nf < 1 || !proxy_f || cap < 0 || !out_total || !out_offsets)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "bad sizes, proxy mesh or output");
    if (n > 0 && (!face || !bary)) return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL array");
    if (cap > 0 && !out_entries) return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL entries with cap > 0");
    if ((reinterpret_cast<uintptr_t>(bary) & 7) || (reinterpret_cast<uintptr_t>(out_entries) & 15))
        return fail(ctx, UMGS_ERR_INVALID_ARG, "bary must be 8-byte and out_entries 16-byte aligned");
    return binding_csr(ctx, face, bary, n, proxy_f, nv, nf, out_offsets, reinterpret_cast<int2*>(out_entries), cap,
                       out_total, static_cast<cudaStream_t>(stream));
}

umgs_status umgs_deform_csr(umgs_ctx* ctx, const umgs_gaussians* rest, const int32_t* offsets,
                            const int32_t* entries, const float* proxy_v, const float* proxy_vd,
                            const int32_t* proxy_f, int64_t nv, int64_t nf, int32_t mode, float* out_means,
                            float* out_cov3d, float* out_quats, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    if (!rest || rest->n < 0) return fail(ctx, UMGS_ERR_INVALID_ARG, "rest Gaussians missing");
    if ((mode & ~(UMGS_DEFORM_LITERAL | UMGS_DEFORM_ONE_RING)) != 0)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "bad mode");
    if (!proxy_v || !proxy_vd || !proxy_f || nv < 3 || nf < 1) return fail(ctx, UMGS_ERR_INVALID_ARG, "bad proxy mesh");
    if (rest->n > 0) {
        if (!rest->means || !offsets || !entries || !out_means || !out_cov3d)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL array");
        if (!rest->cov3d && (!rest->quats || !rest->scales))
            return fail(ctx, UMGS_ERR_INVALID_ARG, "need quats+scales or cov3d");
        if (reinterpret_cast<uintptr_t>(entries) & 15)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "entries must be 16-byte aligned");
    }
    return deform_compact_forward(ctx, rest, offsets, reinterpret_cast<const int2*>(entries), proxy_v, proxy_vd,
                                  proxy_f, nv, nf, mode, out_means, out_cov3d, out_quats,
                                  static_cast<cudaStream_t>(stream), true);
}

umgs_status umgs_bind(umgs_ctx* ctx, const umgs_gaussians* g, const float* proxy_v, const int32_t* proxy_f,
                      int64_t nv, int64_t nf, const umgs_camera* cams, int32_t ncams, int32_t mode, float k_sigma,
                      int32_t* out_face, float* out_bary, float* out_dist, uint8_t* out_flags,
                      int64_t* out_num_fallback, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    if (!g || g->n < 0) return fail(ctx, UMGS_ERR_INVALID_ARG, "Gaussians missing");
    if (mode != UMGS_BIND_BBX && mode != UMGS_BIND_CENTER && mode != UMGS_BIND_NEAREST)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "bad bind mode");
    if (!proxy_v || !proxy_f || nv < 3 || nf < 1) return fail(ctx, UMGS_ERR_INVALID_ARG, "bad proxy mesh");
    if (nf >= (1LL << 31)) return fail(ctx, UMGS_ERR_INVALID_ARG, "too many proxy faces");
    if (mode != UMGS_BIND_NEAREST && (!cams || ncams < 1))
        return fail(ctx, UMGS_ERR_INVALID_ARG, "ray-cast binding needs at least one camera");
    if (g->n > 0) {
        if (!g->means || !out_face || !out_bary || !out_dist || !out_flags)
            return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL array");
        if (mode == UMGS_BIND_BBX && (!g->quats || !g->scales))
            return fail(ctx, UMGS_ERR_INVALID_ARG, "BBX binding needs quats and scales");
        if (!(k_sigma > 0.f)) return fail(ctx, UMGS_ERR_INVALID_ARG, "k_sigma must be positive");
    }
    return bind_forward(ctx, g, proxy_v, proxy_f, nv, nf, cams, mode == UMGS_BIND_NEAREST ? 0 : ncams, mode, k_sigma,
                        out_face, out_bary, out_dist, out_flags, out_num_fallback, static_cast<cudaStream_t>(stream));
}

umgs_status umgs_deform_vertex_table(umgs_ctx* ctx, float* out_table, int64_t nv, void* stream) {
    if (!ctx || !out_table) return UMGS_ERR_INVALID_ARG;
    if (nv != ctx->vtab_rows || nv <= 0) return fail(ctx, UMGS_ERR_INVALID_ARG, "nv differs from the last umgs_deform");
    // the first 12 of the 16 floats of each internal row
    cudaError_t e = cudaMemcpy2DAsync(out_table, sizeof(float) * 12, ctx->vtab.ptr, sizeof(float) * 16,
                                      sizeof(float) * 12, (size_t)nv, cudaMemcpyDeviceToDevice,
                                      static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy2DAsync");
    return UMGS_OK;
}

umgs_status umgs_frame_counts(const umgs_frame* frame, int64_t* num_keys, int64_t* num_tiles) {
    if (!frame || !num_keys || !num_tiles) return UMGS_ERR_INVALID_ARG;
    if (!frame->valid) return UMGS_ERR_INVALID_ARG;
    *num_keys = frame->num_keys;
    *num_tiles = frame->num_tiles;
    return UMGS_OK;
}

umgs_status umgs_frame_evaluations(const umgs_frame* frame, int64_t* evals, void* stream) {
    if (!frame || !evals || !frame->valid) return UMGS_ERR_INVALID_ARG;
    if (cudaSetDevice(frame->ctx->device) != cudaSuccess) return fail(frame->ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    return frame_evaluations(frame, evals, static_cast<cudaStream_t>(stream));
}

umgs_status umgs_frame_stats_read(const umgs_frame* frame, umgs_frame_stats* out, void* stream) {
    if (!frame || !out || !frame->valid) return UMGS_ERR_INVALID_ARG;
    if (cudaSetDevice(frame->ctx->device) != cudaSuccess) return fail(frame->ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    return frame_stats(frame, out, static_cast<cudaStream_t>(stream));
}

umgs_status umgs_deform_fp64_faces(umgs_ctx* ctx, int64_t* count, void* stream) {
    if (!ctx || !count) return UMGS_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(ctx->pinned, ctx->dstatus.as<int32_t>() + 1, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the fp64 face count");
    int32_t v = 0;
    std::memcpy(&v, ctx->pinned, sizeof(v));
    *count = v;
    return UMGS_OK;
}

umgs_status umgs_frame_depth(const umgs_frame* frame, float* out_depth, void* stream) {
    if (!frame || !out_depth) return UMGS_ERR_INVALID_ARG;
    if (!frame->valid || !frame->has_depth)
        return fail(frame->ctx, UMGS_ERR_INVALID_ARG, "the last render into this frame kept no depth");
    if (cudaSetDevice(frame->ctx->device) != cudaSuccess) return fail(frame->ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    const cudaError_t e = cudaMemcpyAsync(out_depth, frame->depth.ptr,
                                          sizeof(float) * (int64_t)frame->ncams * frame->W * frame->H,
                                          cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(frame->ctx, e, "cudaMemcpyAsync(depth)");
    return UMGS_OK;
}

umgs_status umgs_frame_lists(const umgs_frame* frame, int64_t* tile_ptr, int32_t* ids, uint32_t* dbits,
                             void* stream) {
    if (!frame || !tile_ptr || !frame->valid) return UMGS_ERR_INVALID_ARG;
    if (frame->num_keys > 0 && (!ids || !dbits)) return UMGS_ERR_INVALID_ARG;
    return frame_lists(frame, tile_ptr, ids, dbits, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
