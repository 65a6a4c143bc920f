// Host-side internals of libumgs: context, frames, workspace, launchers.
#pragma once
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/umgs.h"
#include "common.cuh"

namespace umgs {

// A device buffer that only grows.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t n) {
        if (n <= bytes) return cudaSuccess;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        size_t want = n + n / 4 + 256;
        cudaError_t e = cudaMalloc(&ptr, want);
        if (e != cudaSuccess) { ptr = nullptr; return e; }
        bytes = want;
        return cudaSuccess;
    }
    void release() { if (ptr) cudaFree(ptr); ptr = nullptr; bytes = 0; }
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

}  // namespace umgs

// Everything one umgs_render call produces and umgs_render_backward consumes.
struct umgs_frame {
    umgs_ctx* ctx = nullptr;
    int device = 0;  // the context's device (umgs_frame_destroy may outlive the context)
    umgs::DevBuf cams, grec, trec, bin, tile_off;
    // binning: record depth keys/values (+ ping-pong), (region, id) pairs
    // (+ ping-pong), radix histograms and scan sums (the persistent
    // compositor's tile-order sort); per region its first pair, chunk count and first chunk; per
    // chunk and region tile the count and the count of earlier chunks; per
    // tile its list length and first entry; the tile lists
    umgs::DevBuf pk, pv, pk2, pv2, tk, tv, tk2, tv2, rs_hist, rs_hist2, rs_bsum;
    umgs::DevBuf lb_a, lb_b, lb_e, lb_s;  // look-back words: radix passes (alternating), emission, tile scan
    umgs::DevBuf rg_start, rg_nchunk, rg_coff, rg_ccnt, rg_cpre, tl_cnt, tl_off, tl_ids;
    uint32_t* ids = nullptr;    // tile lists: unified ids (tl_ids)
    umgs::DevBuf last, status;
    umgs::DevBuf tfin, ntri, stack;   // backward state (saved renders only)
    umgs::DevBuf depth;               // expected depth per pixel (UMGS_RENDER_DEPTH renders only)
    umgs::DevBuf textab;              // DevTex per textured mesh
    std::vector<umgs::DevCam> cams_host;  // the cameras last uploaded into `cams`
    void* cams_dev = nullptr;             // ... and the buffer they went to
    bool has_depth = false;
    umgs::DevBuf ggrad, tgrad, rerun_out;
    umgs::DevBuf fix_list;            // (camera, Gaussian) records whose conic is refined in fp64
    umgs::DevBuf ord_k, ord_v, ord_k2, ord_v2;  // tile (or work item) order of the persistent compositor
    umgs::DevBuf split_items, segbuf, seglast;  // per-tile work split: work items, segment composites
    int32_t stack_cap = 8;
    bool saved = false;
    bool mixed = false;               // Gaussian records in fp16 (GRec16)
    bool nosync = false;              // no host read-back inside umgs_render (async and graph capture)
    bool capture = false;             // inside a graph capture: buffers and cameras already in place
    int64_t key_capacity = 0;         // pair capacity when there is no read-back
    umgs_render_opts opts{};
    int64_t ng = 0, nt = 0;          // Gaussians, triangles (all meshes)
    int32_t ncams = 0, W = 0, H = 0;
    int32_t tile = 16, tiles_x = 0, tiles_y = 0;
    int64_t num_keys = 0, num_tiles = 0;
    int32_t blend_mode = 0;
    float t_eps = 1e-4f;
    float bg[3] = {0, 0, 0};
    bool valid = false;
    std::vector<int64_t> mesh_offset;  // unified id of each mesh's first face
    void release() {
        for (auto* b : {&cams, &grec, &trec, &bin, &tile_off, &pk, &pv, &pk2, &pv2, &tk, &tv, &tk2, &tv2,
                        &rs_hist, &rs_hist2, &rs_bsum, &rg_start, &rg_nchunk, &rg_coff, &rg_ccnt, &rg_cpre, &tl_cnt,
                        &tl_off, &tl_ids, &lb_a, &lb_b, &lb_e, &lb_s,
                        &last, &status, &tfin, &ntri, &stack, &depth, &textab, &ggrad, &tgrad, &rerun_out, &fix_list, &ord_k, &ord_v,
                        &ord_k2, &ord_v2, &split_items, &segbuf, &seglast})
            b->release();
        cams_host.clear();
        cams_dev = nullptr;
    }
};

// Kernels launched by this library in this process, all devices
// (umgs_kernel_launches).  Every launch site adds one; a launch of a captured
// graph adds the number of kernels captured into it.
extern std::atomic<long long> g_kernel_launches;
inline void count_launch(long long n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

namespace umgs {
// Launch `kernel` on `s` with programmatic stream serialisation: it may be
// scheduled before the preceding kernel of the stream finishes and must call
// pdl_enter() before touching anything that kernel writes.  Errors surface
// through cudaGetLastError like a <<< >>> launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    static_assert(sizeof...(KArgs) == sizeof...(Args), "kernel argument count");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
}  // namespace umgs

// Per-stage CUDA-event timing (umgs_profile_enable / umgs_profile_read).
struct StageProfiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;      // free events
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

struct umgs_ctx {
    int device = 0;
    StageProfiler prof;
    std::string err;
    umgs_frame* default_frame = nullptr;
    int64_t* pinned = nullptr;  // small pinned host scratch
    int num_sms = 0;
    umgs::DevBuf dstatus;       // device status word of asynchronous calls
    umgs::DevBuf vacc, vtab;    // deformation: per-vertex accumulators / transform table
    int64_t vtab_rows = 0;
    umgs::DevBuf bind_ws;       // binding workspace (grid header + cell entries)
    umgs::DevBuf bind_cams, bind_cnt;
    umgs::DevBuf order_ws;      // umgs_spatial_order workspace
};

namespace umgs {

umgs_status fail(umgs_ctx* ctx, umgs_status s, const std::string& msg);

// RAII bracket of one stage: records an event pair on `stream` when profiling is on.
struct StageTimer {
    umgs_ctx* ctx;
    int stage;
    cudaStream_t stream;
    cudaEvent_t a = nullptr;
    StageTimer(umgs_ctx* c, int s, cudaStream_t st) : ctx(c), stage(s), stream(st) {
        if (ctx->prof.on) { a = ctx->prof.get(); cudaEventRecord(a, stream); }
    }
    ~StageTimer() {
        if (a) {
            cudaEvent_t b = ctx->prof.get();
            cudaEventRecord(b, stream);
            ctx->prof.recs.push_back({stage, a, b});
        }
    }
};
umgs_status cuda_fail(umgs_ctx* ctx, cudaError_t e, const char* where);

umgs_status render_forward(umgs_ctx* ctx, const umgs_gaussians* g, const umgs_mesh* meshes, int32_t nmeshes,
                           const umgs_camera* cams, int32_t ncams, const umgs_render_opts& opts,
                           float* out_rgbt, umgs_frame* fr, cudaStream_t stream);

umgs_status deform_forward(umgs_ctx* ctx, const umgs_gaussians* g, const int32_t* face, const float* bary,
                           const float* V, const float* Vd, const int32_t* F, int64_t nv, int64_t nf, int32_t mode,
                           float* out_means, float* out_cov, float* out_quats, cudaStream_t stream);
umgs_status binding_compact(umgs_ctx* ctx, const int32_t* face, const float* bary, int64_t n, const int32_t* F,
                            int64_t nv, int64_t nf, int32_t* out_count, int2* out_entries, cudaStream_t stream);
umgs_status deform_compact_forward(umgs_ctx* ctx, const umgs_gaussians* g, const int32_t* count, const int2* entries,
                                   const float* V, const float* Vd, const int32_t* F, int64_t nv, int64_t nf,
                                   int32_t mode, float* out_means, float* out_cov, float* out_quats,
                                   cudaStream_t stream, bool csr = false);
umgs_status binding_csr(umgs_ctx* ctx, const int32_t* face, const float* bary, int64_t n, const int32_t* F,
                        int64_t nv, int64_t nf, int32_t* out_offsets, int2* out_entries, int64_t cap,
                        int64_t* out_total, cudaStream_t stream);

umgs_status bind_forward(umgs_ctx* ctx, const umgs_gaussians* g, const float* V, const int32_t* F, int64_t nv,
                         int64_t nf, const umgs_camera* cams, int32_t ncams, int32_t mode, float k_sigma,
                         int32_t* out_face, float* out_bary, float* out_dist, uint8_t* out_flags,
                         int64_t* out_num_fallback, cudaStream_t stream);

cudaError_t launch_composite(umgs_frame* fr, const umgs_render_opts& opts, float* out_rgbt, cudaStream_t stream);
// compositor of UMGS_RENDER_SOFT_EDGE renders (soft.cu)
cudaError_t launch_soft_composite(umgs_frame* fr, const umgs_render_opts& opts, float* out_rgbt, cudaStream_t stream);
cudaError_t reserve_binning(umgs_frame* fr, int64_t rcap, int64_t kcap);
// stable LSD radix sort of (k, v) on key bits [lo, lo + bits) (binning
// stage); the element count is read from n_dev (at most n_cap, which sizes
// the grids); key_mm: the optional key map of radix.cuh (RadixMap)
cudaError_t radix_sort_pairs(umgs_frame* fr, uint32_t* k, uint32_t* v, uint32_t* k2, uint32_t* v2,
                             const uint32_t* n_dev, int64_t n_cap, int bits, uint32_t** rk, uint32_t** rv,
                             cudaStream_t s, int lo = 0, const uint32_t* key_mm = nullptr);
// single-sweep passes of the binning stage's radix sorts (render.cu)
cudaError_t onesweep_sort(umgs_frame* fr, uint32_t* k, uint32_t* v, uint32_t* k2, uint32_t* v2,
                          const uint32_t* n_dev, int64_t n_cap, int lo, int npass, uint32_t* ghist,
                          uint32_t* counters, const uint32_t* mm, const uint32_t* n_culled, uint32_t* err,
                          cudaStream_t s);

umgs_status render_backward(umgs_ctx* ctx, umgs_frame* fr, const umgs_gaussians* g, const umgs_mesh* meshes,
                            int32_t nmeshes, const float* dL_drgbt, const umgs_gaussian_grads* gg,
                            const umgs_mesh_grads* mg, cudaStream_t stream);

umgs_status frame_check(umgs_frame* fr, cudaStream_t stream);
umgs_status frame_evaluations(const umgs_frame* fr, int64_t* evals, cudaStream_t stream);
umgs_status frame_stats(const umgs_frame* fr, umgs_frame_stats* out, cudaStream_t stream);
// first status word past the render's own (16 + the depth sort's key-map
// slots): two u64 evaluation counters (Gaussian, triangle)
constexpr int kStatusEvalWords = 16 + 2 * 32;
// then the work split's counters: work items, segment slots, persistent work counter
constexpr int kStatusSplitWords = kStatusEvalWords + 4;
// then the binning stage's single-sweep kernels: tile counters (depth-sort
// passes 0-3, region-sort passes, the pair emission, the tile scan), the
// depth sort's 4 x 256 and the region sort's 3 x 256 digit counts
constexpr int kStatusBinWords = kStatusSplitWords + 4;
constexpr int kBinCounters = 16;
constexpr int kBinRegionCounters = 4, kBinEmitCounter = 7, kBinScanCounter = 8;
constexpr int kBinCulledWord = 15;  // (in the counter words) culled records of the depth sort
constexpr int kStatusWords = kStatusBinWords + kBinCounters + 4 * 256 + 3 * 256;
// buffers of a render with the per-tile work split for kcap tile-list entries
cudaError_t reserve_split(umgs_frame* fr, int split, int64_t kcap);
umgs_status frame_lists(const umgs_frame* fr, int64_t* tile_ptr, int32_t* ids, uint32_t* dbits,
                        cudaStream_t stream);

}  // namespace umgs
