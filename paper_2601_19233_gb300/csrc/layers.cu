// Separate-pass baseline (the scheme Sec. 4.1 and Fig. 5b compare the
// single pass against): two layers rendered apart, each with a zero
// background and its expected-depth output, are composited per pixel in the
// order of their depths and the background is added last.  Not a step of the
// method; it exists to measure what the single pass gets right.
#include "internal.h"

namespace umgs {

// per pixel: f = the nearer layer (a on equal depths), b = the other;
// C = C_f + T_f C_b + T_f T_b bg, T = T_f T_b
__global__ void composite_layers_kernel(const float4* __restrict__ a, const float* __restrict__ da,
                                        const float4* __restrict__ b, const float* __restrict__ db, int64_t n,
                                        float bg0, float bg1, float bg2, float4* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 la = a[i], lb = b[i];
    const bool a_front = !(db[i] < da[i]);
    const float4 f = a_front ? la : lb, k = a_front ? lb : la;
    const float T = f.w * k.w;
    out[i] = make_float4(f.x + f.w * k.x + T * bg0, f.y + f.w * k.y + T * bg1, f.z + f.w * k.z + T * bg2, T);
}

}  // namespace umgs

using namespace umgs;

extern "C" umgs_status umgs_composite_layers(umgs_ctx* ctx, const float* a_rgbt, const float* a_depth,
                                             const float* b_rgbt, const float* b_depth, int64_t npix,
                                             const float* bg, float* out_rgbt, void* stream) {
    if (!ctx) return UMGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (npix < 0 || (npix > 0 && (!a_rgbt || !a_depth || !b_rgbt || !b_depth || !out_rgbt)) || !bg)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "NULL array or negative size");
    if ((reinterpret_cast<uintptr_t>(a_rgbt) | reinterpret_cast<uintptr_t>(b_rgbt) |
         reinterpret_cast<uintptr_t>(out_rgbt)) & 15)
        return fail(ctx, UMGS_ERR_INVALID_ARG, "the rgbt arrays must be 16-byte aligned");
    if (npix == 0) return UMGS_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, UMGS_ERR_CUDA, "cudaSetDevice");
    composite_layers_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float4*>(a_rgbt), a_depth, reinterpret_cast<const float4*>(b_rgbt), b_depth, npix,
        bg[0], bg[1], bg[2], reinterpret_cast<float4*>(out_rgbt)),
        count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "composite_layers_kernel");
    return UMGS_OK;
}
