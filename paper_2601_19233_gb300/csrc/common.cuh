// Shared device definitions of libumgs (sm_103a).
//
// Canonical arithmetic: every float operation that decides WHICH fragments
// exist or in WHICH ORDER they are blended (pixel footprints of Gaussians,
// triangle snapping, depth keys, binding argmins) goes through the _rn
// intrinsics below, one IEEE binary32 operation each, never contracted into
// an FMA.  These decisions are therefore reproducible bit for bit by any
// IEEE-754 implementation that evaluates the same expression tree.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace umgs {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsq(float a) { return __fsqrt_rn(a); }
// ((a0*b0 + a1*b1) + a2*b2), each op rounded
__device__ __forceinline__ float dot3c(float a0, float a1, float a2, float b0, float b1, float b2) {
    return fa(fa(fm(a0, b0), fm(a1, b1)), fm(a2, b2));
}

// Camera as the kernels see it.
struct DevCam {
    float R[9];      // row-major rotation (world -> camera)
    float t[3];
    float fx, fy, cx, cy;
    int32_t W, H;
    float near_z;
    float campos[3]; // camera centre (colour direction only; not a decision)
    int32_t pad;
};

// Projected Gaussian record: 48 bytes, three 16-byte vectors.
//  q0 = (u, v, ca, cb), q1 = (cc, opacity, r, g), q2 = (b, rect_x, rect_y, -)
//  power2 = ca*dx^2 + cb*dx*dy + cc*dy^2 is the exponent in base 2:
//  alpha = min(0.99, opacity * exp2(power2)); rect_x = x_lo | x_hi << 16.
struct __align__(16) GRec {
    float4 q0, q1, q2;
};

// Mixed-precision Gaussian record: 32 bytes, two 16-byte vectors.  The
// screen position stays fp32 (fp16 loses sub-pixel precision above 2048 px);
// conic, opacity and colour are fp16; the rect is exact.
//  v0 = (u, v, half2(ca, cb), half2(cc, opacity)), v1 = (half2(r, g), half2(b, 0), rect_x, rect_y)
struct __align__(16) GRec16 {
    uint4 v0, v1;
};

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    return (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
}
__device__ __forceinline__ float half_lo(uint32_t p) { return __half2float(__ushort_as_half((unsigned short)(p & 0xffffu))); }
__device__ __forceinline__ float half_hi(uint32_t p) { return __half2float(__ushort_as_half((unsigned short)(p >> 16))); }

// Triangle record: 160 bytes, ten 16-byte vectors.
//  edge k (opposite vertex k of the orientation-corrected triangle):
//     E_k(sx, sy) = A_k*sx + B_k*sy + C_k in 1/256-px units, top-left bias
//     folded into C_k, sample covered <=> all E_k >= 0
//  u, v: unsnapped screen positions (ORIGINAL vertex order) for attributes
//  iz: 1/Z per vertex, col: vertex colours, alpha: per-vertex alpha;
//  const_alpha != 0 means alpha[0] is the face alpha (no interpolation).
struct __align__(16) TRec {
    int32_t A[3];
    int32_t B[3];
    int32_t const_alpha;
    int32_t pad0;
    long long C[3];
    long long pad1;
    float u[3], v[3];
    float iz[3];
    float col[9];
    float alpha[3];
    uint32_t rx, ry;  // pixel rect, lo | hi << 16 (as in BinInfo)
    float pad2;
};
static_assert(sizeof(GRec) == 48, "GRec size");
static_assert(sizeof(GRec16) == 32, "GRec16 size");
static_assert(sizeof(TRec) == 160, "TRec size");

// Per (camera, primitive) binning info: pixel rect packed as lo | hi << 16,
// depth bits; an empty rect (lo > hi) means culled.
struct __align__(16) BinInfo {
    uint32_t rx, ry, dbits, valid;
};

// 4 samples per pixel at the rotated-grid offsets (-2,-6), (6,-2), (-6,2),
// (2,6) / 16 px, i.e. these offsets in 1/256 px from the pixel centre.
__device__ __forceinline__ int sample_dx(int j) { return j == 0 ? -32 : j == 1 ? 96 : j == 2 ? -96 : 32; }
__device__ __forceinline__ int sample_dy(int j) { return j == 0 ? -96 : j == 1 ? -32 : j == 2 ? 32 : 96; }

// 2^x by the hardware approximation (ex2.approx.ftz: relative error ~2^-22,
// flushes results below 2^-126 to 0); used by the forward and the backward
// replay alike, so both take the same alpha decisions.
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Gaussian alpha at offset (dx, dy) from the projected mean, with a fixed
// operation sequence so the forward and the backward replay agree bit for bit:
// power2 = ca dx^2 + cb dx dy + cc dy^2 (base-2 exponent), alpha = o 2^power2.
__device__ __forceinline__ float gauss_power2(float ca, float cb, float cc, float dx, float dy) {
    return __fmaf_rn(cc, __fmul_rn(dy, dy), __fmaf_rn(cb, __fmul_rn(dx, dy), __fmul_rn(ca, __fmul_rn(dx, dx))));
}

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kLog2e = 1.4426950408889634f;

}  // namespace umgs
