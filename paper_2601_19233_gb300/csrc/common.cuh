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
//  q0 = (u, v, l0, l1), q1 = (l2, opacity, r, g), q2 = (b, rect_x, rect_y, Z)
//  (Z: camera depth of the mean, for the expected-depth output)
//  (l0, l1, l2): the conic's factor of gauss_power2, the exponent in base 2:
//  alpha = min(0.99, opacity * exp2(power2)); rect_x = x_lo | x_hi << 16.
struct __align__(16) GRec {
    float4 q0, q1, q2;
};

// Mixed-precision Gaussian record: 32 bytes, two 16-byte vectors.  The
// screen position stays fp32 (fp16 loses sub-pixel precision above 2048 px);
// conic, opacity and colour are fp16; the rect is exact.
//  v0 = (u, v, half2(l0, l1), half2(l2, opacity)), v1 = (half2(r, g), half2(b, 0), rect_x, rect_y)
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
//  const_alpha != 0 means alpha[0] is the face alpha (no interpolation);
//  tex > 0: a textured face, col[0..5] = the vertices' (u, v) and the colour
//  comes from texture tex - 1 of the render's texture table.
struct __align__(16) TRec {
    int32_t A[3];
    int32_t B[3];
    int32_t const_alpha;
    int32_t tex;
    long long C[3];
    long long orient;  // sign of the snapped integer area (+1 / -1): the setup's orientation
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

// Programmatic dependent launch (the kernels of a render are launched with
// programmatic stream serialisation): wait until the preceding kernel of the
// stream has finished and its writes are visible, then let the next kernel's
// blocks be scheduled while this one runs.  Without a programmatic
// predecessor the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Texture of a textured mesh: RGB float, row-major [h][w][3].
struct DevTex {
    const float* data;
    int32_t w, h;
    int64_t pad;
};

// Bilinear lookup with clamp-to-edge addressing: texel (i, j) sits at
// ((i + 0.5) / w, (j + 0.5) / h); the four texels around (u, v) are weighted
// by their distance.
__device__ __forceinline__ void sample_texture(const DevTex& tx, float u, float v, float (&c)[3]) {
    const float x = u * (float)tx.w - 0.5f, y = v * (float)tx.h - 0.5f;
    const float x0 = floorf(x), y0 = floorf(y);
    const float fx = x - x0, fy = y - y0;
    const int ix0 = (int)fminf(fmaxf(x0, 0.f), (float)(tx.w - 1)), ix1 = (int)fminf(fmaxf(x0 + 1.f, 0.f), (float)(tx.w - 1));
    const int iy0 = (int)fminf(fmaxf(y0, 0.f), (float)(tx.h - 1)), iy1 = (int)fminf(fmaxf(y0 + 1.f, 0.f), (float)(tx.h - 1));
    const float* r0 = tx.data + (int64_t)iy0 * tx.w * 3;
    const float* r1 = tx.data + (int64_t)iy1 * tx.w * 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float top = (1.f - fx) * r0[3 * ix0 + k] + fx * r0[3 * ix1 + k];
        const float bot = (1.f - fx) * r1[3 * ix0 + k] + fx * r1[3 * ix1 + k];
        c[k] = (1.f - fy) * top + fy * bot;
    }
}

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

// Gaussian exponent (base 2) at offset (dx, dy) from the projected mean.
// The record keeps the factor (l0, l1, l2) of the scaled conic: with
// Sigma2D = [[a, b], [b, c]], det = a c - b^2, the conic Q = Sigma2D^-1 and
// k = log2(e) / 2, k Q = L^T L for L = [[l0, l1], [0, l2]], l0 = sqrt(k c /
// det), l1 = -k b / (det l0), l2 = sqrt(k / c).  Then power2 = -k d^T Q d =
// -((l0 dx + l1 dy)^2 + (l2 dy)^2), a sum of two squares without the
// cancellation that A dx^2 + 2 B dx dy + C dy^2 suffers along an elongated
// footprint; alpha = o 2^power2.  A fixed operation sequence, so the forward
// and the backward replay agree bit for bit.
__device__ __forceinline__ float gauss_power2(float l0, float l1, float l2, float dx, float dy) {
    const float w1 = __fmaf_rn(l1, dy, __fmul_rn(l0, dx));
    const float w2 = __fmul_rn(l2, dy);
    return -__fmaf_rn(w1, w1, __fmul_rn(w2, w2));
}
// the base-2 conic of a factor: power2 = ca dx^2 + cb dx dy + cc dy^2
__device__ __forceinline__ void factor_conic(float l0, float l1, float l2, float& ca, float& cb, float& cc) {
    ca = -l0 * l0;
    cb = -2.f * l0 * l1;
    cc = -(l1 * l1 + l2 * l2);
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kHalfLog2e = 0.7213475204444817f;

// A projected covariance [[a, b], [b, c]] with det < kConicFp64 * a * c is
// near-singular: its conic is inverted in fp64 (the fp32 inverse would lose
// log2(a c / det) bits, about 7 at this bound, which keeps the fp32 alpha
// within 2e-5 of the exact one).
constexpr float kConicFp64 = 1.0f / 128.0f;

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;

// ---- warp <-> pixel layout of the compositors -------------------------------
// Warp w of a TS x TS tile (TS = 8, 16, 32) owns the 8 x 4 pixel block
// (w % (TS/8), w / (TS/8)); lane l is pixel (l % 8, l / 8) of that block.
// Near-square blocks let a record skip every warp whose block its footprint
// misses (the compositors build per-warp record lists from these masks).
template <int TS>
__device__ __forceinline__ void block_pixel(int t, int& lx, int& ly) {
    const int w = t >> 5, l = t & 31;
    lx = (w % (TS / 8)) * 8 + (l & 7);
    ly = (w / (TS / 8)) * 4 + (l >> 3);
}

// Blocks of 8 x BH pixels (bit wy * (TS/8) + wx for the block at (8 wx,
// BH wy); BH = 4: the warps of block_pixel) of the tile with origin
// (tx0, ty0) that meet the pixel box [x0,x1] x [y0,y1].
template <int TS, int BH = 4>
__device__ __forceinline__ uint32_t box_block_mask(int x0, int x1, int y0, int y1, int tx0, int ty0) {
    constexpr int LB = BH == 4 ? 2 : 3;
    x0 = max(x0, tx0); x1 = min(x1, tx0 + TS - 1);
    y0 = max(y0, ty0); y1 = min(y1, ty0 + TS - 1);
    if (x0 > x1 || y0 > y1) return 0u;
    const int wx0 = (x0 - tx0) >> 3, wx1 = (x1 - tx0) >> 3, wy0 = (y0 - ty0) >> LB, wy1 = (y1 - ty0) >> LB;
    const uint32_t cols = ((2u << wx1) - 1u) & ~((1u << wx0) - 1u);
    uint32_t m = 0u;
    for (int wy = wy0; wy <= wy1; ++wy) m |= cols << (wy * (TS / 8));
    return m;
}

// Blocks of 8 x BH pixels (as box_block_mask) of the tile with origin (tx0, ty0)
// whose pixels can hold a fragment of a Gaussian record with projected mean
// (u, v), conic factor (l0, l1, l2) (gauss_power2; base-2 conic ca dx^2 +
// cb dx dy + cc dy^2), opacity o and pixel rect [x0,x1] x [y0,y1].  A fragment needs
// the pixel in the rect and alpha >= 1/255, i.e. d = (dx, dy) inside the
// ellipse d^T Q d <= lim with Q = -[[ca, cb/2], [cb/2, cc]], lim =
// log2(255 o).  The ellipse lies inside the octagon bounded by its support
// in the directions x, y, x + y and x - y (h(n)^2 = lim n^T Q^-1 n); a block
// is kept when its pixel-centre rectangle meets that octagon.  The bounds
// are widened by 2% of lim plus 1% + 0.01 px, far beyond the rounding of this
// test and of the compositor's own alpha.  o < 1/255: no fragment; a conic
// that is not positive definite keeps every block of the rect.
template <int TS, int BH = 4>
__device__ __forceinline__ uint32_t gauss_block_mask(float u, float v, float l0, float l1, float l2, float o, int x0,
                                                     int x1, int y0, int y1, int tx0, int ty0) {
    constexpr int LB = BH == 4 ? 2 : 3;
    if (!(o >= kAlphaMin)) return 0u;
    float ca, cb, cc;
    factor_conic(l0, l1, l2, ca, cb, cc);
    const float qa = -ca, qb = -0.5f * cb, qc = -cc, det = qa * qc - qb * qb;
    if (!(qa > 0.f && qc > 0.f && det > 0.f)) return box_block_mask<TS, BH>(x0, x1, y0, y1, tx0, ty0);
    const float s = (__log2f(255.f * o) * 1.02f + 1e-4f) / det;  // lim Q^-1 = s [[qc, -qb], [-qb, qa]]
    const float hx = sqrtf(s * qc) * 1.01f + 0.01f, hy = sqrtf(s * qa) * 1.01f + 0.01f;
    const float hp = sqrtf(s * (qc + qa - 2.f * qb)) * 1.01f + 0.01f;  // direction x + y
    const float hm = sqrtf(s * (qc + qa + 2.f * qb)) * 1.01f + 0.01f;  // direction x - y
    x0 = max(max(x0, (int)floorf(u - hx - 0.5f)), tx0); x1 = min(min(x1, (int)ceilf(u + hx - 0.5f)), tx0 + TS - 1);
    y0 = max(max(y0, (int)floorf(v - hy - 0.5f)), ty0); y1 = min(min(y1, (int)ceilf(v + hy - 0.5f)), ty0 + TS - 1);
    if (x0 > x1 || y0 > y1) return 0u;
    const int wx0 = (x0 - tx0) >> 3, wx1 = (x1 - tx0) >> 3, wy0 = (y0 - ty0) >> LB, wy1 = (y1 - ty0) >> LB;
    uint32_t m = 0u;
    for (int wy = wy0; wy <= wy1; ++wy) {
        const float Y0 = (float)max(y0, ty0 + BH * wy) + 0.5f - v, Y1 = (float)min(y1, ty0 + BH * wy + BH - 1) + 0.5f - v;
        for (int wx = wx0; wx <= wx1; ++wx) {
            const float X0 = (float)max(x0, tx0 + 8 * wx) + 0.5f - u;
            const float X1 = (float)min(x1, tx0 + 8 * wx + 7) + 0.5f - u;
            if (X1 + Y1 >= -hp && X0 + Y0 <= hp && X1 - Y0 >= -hm && X0 - Y1 <= hm) m |= 1u << (wy * (TS / 8) + wx);
        }
    }
    return m;
}

}  // namespace umgs
