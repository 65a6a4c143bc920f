// Spatial order of a set of Gaussians (a layout tool with no paper
// counterpart): the permutation that sorts them by the Morton code of their
// means.  A model stored in that order keeps Gaussians that are close in
// space close in memory, so that the per-frame deformation (Eq. 12-13), which
// gathers the proxy-vertex rows of every Gaussian's binding, finds the rows of
// a block's Gaussians in the same few cache lines.
#include "internal.h"

namespace umgs {

// float <-> int with the order of the floats (for atomicMin / atomicMax)
__device__ __forceinline__ int ordered_int(float x) {
    const int i = __float_as_int(x);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void order_init_kernel(int* __restrict__ box) {
    if (threadIdx.x < 3) box[threadIdx.x] = 0x7fffffff;       // min x, y, z
    else if (threadIdx.x < 6) box[threadIdx.x] = (int)0x80000000;  // max x, y, z
}

// bounding box of the finite coordinates (grid-stride; one atomic per block
// and bound)
__global__ void order_box_kernel(const float* __restrict__ means, int64_t n, int* __restrict__ box) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const float x = means[3 * i + a];
            if (isfinite(x)) {
                lo[a] = fminf(lo[a], x);
                hi[a] = fmaxf(hi[a], x);
            }
        }
    __shared__ float s[6][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        for (int d = 16; d >= 1; d >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], d));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], d));
        }
        if (lane == 0) { s[a][w] = lo[a]; s[3 + a][w] = hi[a]; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        float v = s[a][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) v = a < 3 ? fminf(v, s[a][k]) : fmaxf(v, s[a][k]);
        if (isfinite(v)) {
            if (a < 3) atomicMin(&box[a], ordered_int(v));
            else atomicMax(&box[a], ordered_int(v));
        }
    }
}

// 10 bits per axis, interleaved (x in bit 0, y in bit 1, z in bit 2, ...)
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Morton code of each mean: per axis q = clamp((x - lo) * (1024 / (hi - lo)),
// 0, 1023) truncated (0 for a non-finite coordinate); keys = code, vals = index
__global__ void order_codes_kernel(const float* __restrict__ means, int64_t n, const int* __restrict__ box,
                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                   uint32_t* __restrict__ n_dev) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) *n_dev = (uint32_t)n;
    if (i >= n) return;
    uint32_t code = 0;
    for (int a = 0; a < 3; ++a) {
        const float lo = ordered_float(box[a]), hi = ordered_float(box[3 + a]);
        const float scale = 1024.f / fmaxf(hi - lo, 1e-30f);
        const float u = fminf(fmaxf((means[3 * i + a] - lo) * scale, 0.f), 1023.f);  // (NaN -> 0)
        code |= spread10((uint32_t)u) << a;
    }
    keys[i] = code;
    vals[i] = (uint32_t)i;
}

}  // namespace umgs

using namespace umgs;

extern "C" umgs_status umgs_spatial_order(umgs_ctx* ctx, const float* means, int64_t n, int32_t* out_perm,
                                          void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n < 0 || (n > 0 && (!means || !out_perm))) return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL array or negative size");
    if (n >= (int64_t)0x7fffffff) return fail(ctx, UMGS_ERR_INVALID_ARG, "more than 2^31 - 2 Gaussians");
    if (n == 0) return UMGS_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // workspace: box (8 ints), count, then keys / values and their ping-pong copies
    const size_t words = 16 + 4 * (size_t)n;
    cudaError_t e = ctx->order_ws.reserve(sizeof(uint32_t) * words);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "spatial order workspace");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "spatial order workspace");
    uint32_t* ws = ctx->order_ws.as<uint32_t>();
    int* box = reinterpret_cast<int*>(ws);
    uint32_t* n_dev = ws + 8;
    uint32_t *k = ws + 16, *v = k + n, *k2 = v + n, *v2 = k2 + n;
    order_init_kernel<<<1, 32, 0, s>>>(box), count_launch();
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms);
    order_box_kernel<<<grid, 256, 0, s>>>(means, n, box), count_launch();
    order_codes_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(means, n, box, k, v, n_dev), count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "spatial order kernels");
    uint32_t *rk = nullptr, *rv = nullptr;
    if ((e = radix_sort_pairs(ctx->default_frame, k, v, k2, v2, n_dev, n, 30, &rk, &rv, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "spatial order sort");
    if ((e = cudaMemcpyAsync(out_perm, rv, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "spatial order copy");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "spatial order");
    return UMGS_OK;
}
