// Forward single-pass rasterization of Gaussians and triangles (Sec. 3.2).
//
// Pipeline per umgs_render call (all cameras in one set of launches):
//   1. project_gaussians / setup_triangles: one thread per primitive, looping
//      over cameras; canonical fp32 footprint (pixel rect) + depth key and a
//      compact record for the compositor; refine_conics_kernel recomputes the
//      few near-singular conics in fp64; shade_gaussians_kernel evaluates SH.
//   2. binning into per-tile lists in (depth bits, id) order:
//      a. every (camera, primitive) record sorted by its depth bits
//         (4 x 8-bit passes, stable, so equal depths stay in id order);
//      b. in that order every record emits one (region, id) pair per region
//         of 8 x 4 tiles its rect touches (offsets from an exclusive scan);
//      c. the pairs are sorted stably by region;
//      d. each region's pairs are expanded into the lists of its 32 tiles
//         (count pass, scans over chunks and tiles, ballot-ranked fill).
//   3. composite (composite.cu).
#include <cstdio>
#include <cstring>
#include <cmath>
#include <algorithm>

#include "internal.h"
#include "radix.cuh"

namespace umgs {

// ---------------------------------------------------------------------------
// spherical harmonics (3DGS colour model), degree <= 3, fp32: real SH with
// the Condon-Shortley phase, index l*l + (m + l), see shade_gaussians_kernel.

// ---------------------------------------------------------------------------
// canonical Gaussian covariance and projection

__device__ void cov3d_canonical(float qw, float qx, float qy, float qz, float sx, float sy, float sz, float S[6]) {
    float n = fsq(fa(fa(fa(fm(qw, qw), fm(qx, qx)), fm(qy, qy)), fm(qz, qz)));
    float w, x, y, z;
    if (n == 0.f) { w = 1.f; x = y = z = 0.f; }
    else { w = fdv(qw, n); x = fdv(qx, n); y = fdv(qy, n); z = fdv(qz, n); }
    float r[9];
    r[0] = fs(1.f, fm(2.f, fa(fm(y, y), fm(z, z))));
    r[1] = fm(2.f, fs(fm(x, y), fm(w, z)));
    r[2] = fm(2.f, fa(fm(x, z), fm(w, y)));
    r[3] = fm(2.f, fa(fm(x, y), fm(w, z)));
    r[4] = fs(1.f, fm(2.f, fa(fm(x, x), fm(z, z))));
    r[5] = fm(2.f, fs(fm(y, z), fm(w, x)));
    r[6] = fm(2.f, fs(fm(x, z), fm(w, y)));
    r[7] = fm(2.f, fa(fm(y, z), fm(w, x)));
    r[8] = fs(1.f, fm(2.f, fa(fm(x, x), fm(y, y))));
    float M[9];
    const float s[3] = {sx, sy, sz};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = fm(r[3 * i + j], s[j]);
    auto e = [&](int i, int j) { return dot3c(M[3 * i], M[3 * i + 1], M[3 * i + 2], M[3 * j], M[3 * j + 1], M[3 * j + 2]); };
    S[0] = e(0, 0); S[1] = e(0, 1); S[2] = e(0, 2); S[3] = e(1, 1); S[4] = e(1, 2); S[5] = e(2, 2);
}

// fp64 2D covariance for near-singular cases (same formula, double precision)
__device__ void cov2d_fp64(const DevCam& C, float mx, float my, float mz, const float* q, const float* s,
                           const float* c6, double& a, double& b, double& c) {
    const double R[9] = {C.R[0], C.R[1], C.R[2], C.R[3], C.R[4], C.R[5], C.R[6], C.R[7], C.R[8]};
    double X = R[0] * mx + R[1] * my + R[2] * mz + C.t[0];
    double Y = R[3] * mx + R[4] * my + R[5] * mz + C.t[1];
    double Z = R[6] * mx + R[7] * my + R[8] * mz + C.t[2];
    double S[3][3];
    if (c6) {
        S[0][0] = c6[0]; S[0][1] = S[1][0] = c6[1]; S[0][2] = S[2][0] = c6[2];
        S[1][1] = c6[3]; S[1][2] = S[2][1] = c6[4]; S[2][2] = c6[5];
    } else {
        double w = q[0], x = q[1], y = q[2], z = q[3];
        double n = sqrt(w * w + x * x + y * y + z * z);
        if (n == 0.0) { w = 1; x = y = z = 0; } else { w /= n; x /= n; y /= n; z /= n; }
        double r[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                          {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                          {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        double M[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = r[i][j] * (double)s[j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) S[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];
    }
    double limx = 1.3 * ((double)C.W / (2.0 * C.fx)), limy = 1.3 * ((double)C.H / (2.0 * C.fy));
    double xc = fmin(limx, fmax(-limx, X / Z)) * Z, yc = fmin(limy, fmax(-limy, Y / Z)) * Z;
    double J[2][3] = {{C.fx / Z, 0.0, -C.fx * xc / (Z * Z)}, {0.0, C.fy / Z, -C.fy * yc / (Z * Z)}};
    double T[2][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) T[i][k] = J[i][0] * R[k] + J[i][1] * R[3 + k] + J[i][2] * R[6 + k];
    double U[2][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) U[i][k] = T[i][0] * S[0][k] + T[i][1] * S[1][k] + T[i][2] * S[2][k];
    a = U[0][0] * T[0][0] + U[0][1] * T[0][1] + U[0][2] * T[0][2] + 0.3;
    b = U[0][0] * T[1][0] + U[0][1] * T[1][1] + U[0][2] * T[1][2];
    c = U[1][0] * T[1][0] + U[1][1] * T[1][1] + U[1][2] * T[1][2] + 0.3;
}

// Conic of a near-singular projected covariance, in fp64 (rare; kept out of
// line so the common path does not pay for its registers).
__device__ __noinline__ void conic_fp64(const DevCam& C, float mx, float my, float mz,
                                        const float* __restrict__ quats, const float* __restrict__ scales,
                                        const float* __restrict__ cov3d, int64_t i, float* out) {
    float q[4] = {0, 0, 0, 0}, s[3] = {0, 0, 0}, c6[6];
    if (cov3d) {
        for (int k = 0; k < 6; ++k) c6[k] = cov3d[6 * i + k];
    } else {
        for (int k = 0; k < 4; ++k) q[k] = quats[4 * i + k];
        for (int k = 0; k < 3; ++k) s[k] = scales[3 * i + k];
    }
    double A2, B2, C2;
    cov2d_fp64(C, mx, my, mz, q, s, cov3d ? c6 : nullptr, A2, B2, C2);
    const double d2 = A2 * C2 - B2 * B2;
    // the factor of gauss_power2: l0 = sqrt(k c / det), l1 = -k b / (det l0), l2 = sqrt(k / c)
    const double k = 0.5 * 1.4426950408889634;
    const double l0 = sqrt(k * C2 / d2);
    out[0] = (float)l0;
    out[1] = (float)(-k * B2 / (d2 * l0));
    out[2] = (float)sqrt(k / C2);
}

// fp64 conics of the (camera, Gaussian) records listed by project_gaussians;
// when the list overflowed every record is re-tested.
__global__ void refine_conics_kernel(const float* __restrict__ means, const float* __restrict__ quats,
                                     const float* __restrict__ scales, const float* __restrict__ cov3d, int64_t N,
                                     const DevCam* __restrict__ cams, int ncams, const BinInfo* __restrict__ bin,
                                     int64_t ntot, const unsigned* __restrict__ fix_count,
                                     const int64_t* __restrict__ fix_list, unsigned fix_cap, GRec* __restrict__ grec,
                                     GRec16* __restrict__ grec16) {
    pdl_enter();
    const unsigned cnt = *fix_count;
    const bool overflow = cnt > fix_cap;
    const int64_t total = overflow ? N * ncams : (int64_t)cnt;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ri = overflow ? k : fix_list[k];
        const int cam = (int)(ri / N);
        const int64_t i = ri - (int64_t)cam * N;
        if (!bin[(int64_t)cam * ntot + i].valid) continue;
        float cq[3];  // on overflow every visible record is refined (fp64 is never less accurate)
        conic_fp64(cams[cam], means[3 * i], means[3 * i + 1], means[3 * i + 2], quats, scales, cov3d, i, cq);
        if (grec16) {
            uint32_t* h = reinterpret_cast<uint32_t*>(grec16 + ri);
            const float o = half_hi(h[3]);
            h[2] = pack_half2(cq[0], cq[1]);
            h[3] = pack_half2(cq[2], o);
        } else {
            float* g = reinterpret_cast<float*>(grec + ri);
            g[2] = cq[0];
            g[3] = cq[1];
            g[4] = cq[2];
        }
    }
}

__global__ void __launch_bounds__(256, 2) project_gaussians_kernel(
    const float* __restrict__ means, const float* __restrict__ quats, const float* __restrict__ scales,
    const float* __restrict__ opac, const void* __restrict__ sh, int sh_dtype, int sh_deg,
    const float* __restrict__ cov3d, int64_t N, const DevCam* __restrict__ cams, int ncams,
    int ts, int tiles_x, int tiles_per_cam, GRec* __restrict__ grec, GRec16* __restrict__ grec16,
    BinInfo* __restrict__ bin, int64_t ntot_prims, unsigned* __restrict__ fix_count, int64_t* __restrict__ fix_list,
    unsigned fix_cap) {
    pdl_enter();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
    float S[6];
    if (cov3d) {
#pragma unroll
        for (int k = 0; k < 6; ++k) S[k] = cov3d[6 * i + k];
    } else {
        cov3d_canonical(quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3], scales[3 * i],
                        scales[3 * i + 1], scales[3 * i + 2], S);
    }
    const float o = opac[i];
    for (int cam = 0; cam < ncams; ++cam) {
        const DevCam& C = cams[cam];
        const int64_t ri = (int64_t)cam * N + i;           // record index
        const int64_t bidx = (int64_t)cam * ntot_prims + i;  // bin index
        const float* R = C.R;
        const float X = fa(dot3c(R[0], R[1], R[2], mx, my, mz), C.t[0]);
        const float Y = fa(dot3c(R[3], R[4], R[5], mx, my, mz), C.t[1]);
        const float Z = fa(dot3c(R[6], R[7], R[8], mx, my, mz), C.t[2]);
        bool valid = Z > C.near_z;
        const float u = fa(fdv(fm(C.fx, X), Z), C.cx);
        const float v = fa(fdv(fm(C.fy, Y), Z), C.cy);
        const float limx = fm(1.3f, fdv((float)C.W, fm(2.f, C.fx)));
        const float limy = fm(1.3f, fdv((float)C.H, fm(2.f, C.fy)));
        const float xc = fm(fminf(limx, fmaxf(-limx, fdv(X, Z))), Z);
        const float yc = fm(fminf(limy, fmaxf(-limy, fdv(Y, Z))), Z);
        const float z2 = fm(Z, Z);
        const float j00 = fdv(C.fx, Z), j11 = fdv(C.fy, Z);
        const float j02 = -fdv(fm(C.fx, xc), z2), j12 = -fdv(fm(C.fy, yc), z2);
        float T0[3], T1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T0[k] = fa(fm(j00, R[k]), fm(j02, R[6 + k]));
            T1[k] = fa(fm(j11, R[3 + k]), fm(j12, R[6 + k]));
        }
        // Sigma rows: [S0 S1 S2; S1 S3 S4; S2 S4 S5]
        const float Sm[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
        float U0[3], U1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            U0[k] = dot3c(T0[0], T0[1], T0[2], Sm[k], Sm[3 + k], Sm[6 + k]);
            U1[k] = dot3c(T1[0], T1[1], T1[2], Sm[k], Sm[3 + k], Sm[6 + k]);
        }
        float a = dot3c(U0[0], U0[1], U0[2], T0[0], T0[1], T0[2]);
        const float b = dot3c(U0[0], U0[1], U0[2], T1[0], T1[1], T1[2]);
        float c = dot3c(U1[0], U1[1], U1[2], T1[0], T1[1], T1[2]);
        a = fa(a, 0.3f);
        c = fa(c, 0.3f);
        const float det = fs(fm(a, c), fm(b, b));
        const float rx = fm(3.f, fsq(a)), ry = fm(3.f, fsq(c));
        valid = valid && det > 0.f && isfinite(u) && isfinite(v) && isfinite(rx) && isfinite(ry);
        const float xlo = fmaxf(ceilf(fs(fs(u, rx), 0.5f)), 0.f);
        const float xhi = fminf(floorf(fs(fa(u, rx), 0.5f)), (float)(C.W - 1));
        const float ylo = fmaxf(ceilf(fs(fs(v, ry), 0.5f)), 0.f);
        const float yhi = fminf(floorf(fs(fa(v, ry), 0.5f)), (float)(C.H - 1));
        valid = valid && xlo <= xhi && ylo <= yhi;
        BinInfo bi;
        bi.dbits = __float_as_uint(Z);
        bi.valid = valid ? 1u : 0u;
        if (!valid) {
            bi.rx = 1u;  // lo = 1 > hi = 0 : empty
            bi.ry = 1u;
            bin[bidx] = bi;
            continue;
        }
        const int ixlo = (int)xlo, ixhi = (int)xhi, iylo = (int)ylo, iyhi = (int)yhi;
        bi.rx = (uint32_t)ixlo | ((uint32_t)ixhi << 16);
        bi.ry = (uint32_t)iylo | ((uint32_t)iyhi << 16);
        bin[bidx] = bi;
        // conic factor of gauss_power2 (not a decision): fp32, or fp64 when
        // the 2x2 determinant is small relative to a*c (kConicFp64)
        float l0, l1, l2;
        {
            const float id = 1.f / det;
            l0 = sqrtf(kHalfLog2e * c * id);
            l1 = -kHalfLog2e * b * id / l0;
            l2 = sqrtf(kHalfLog2e / c);
        }
        if (det < kConicFp64 * a * c) {  // near-singular: refined in fp64 by refine_conics_kernel
            const unsigned slot = atomicAdd(fix_count, 1u);
            if (slot < fix_cap) fix_list[slot] = ri;
        }
        // colour is written by shade_gaussians_kernel
        if (grec16) {
            GRec16* hp = grec16 + ri;
            hp->v0 = make_uint4(__float_as_uint(u), __float_as_uint(v), pack_half2(l0, l1), pack_half2(l2, o));
            reinterpret_cast<uint2*>(&hp->v1)[1] = make_uint2(bi.rx, bi.ry);
        } else {
            float4* gp = reinterpret_cast<float4*>(grec + ri);
            gp[0] = make_float4(u, v, l0, l1);
            reinterpret_cast<float2*>(gp + 1)[0] = make_float2(l2, o);
            reinterpret_cast<float2*>(gp + 2)[0] = make_float2(0.f, __uint_as_float(bi.rx));
            reinterpret_cast<float2*>(gp + 2)[1] = make_float2(__uint_as_float(bi.ry), Z);  // Z: expected-depth output
        }
    }
}

// View-dependent colour of every visible (camera, Gaussian): one thread per
// Gaussian keeps its SH coefficients in registers across the cameras.  Rows
// whose bytes are a multiple of 16 (fp32 degree 1 and 3, bf16 degree 3) are
// first copied for the whole block with coalesced 16-byte loads into shared
// memory, at a pitch of an odd number of 16-byte words so that the threads'
// reads of their own rows meet no bank conflict.  The coefficients and the
// means are read before the wait on the preceding kernel.  That is safe:
// every kernel of the chain waits before it lets the next one start, so when
// this one starts, everything launched before its predecessor has finished
// (the render's status clearing and projection, and whatever the caller ran
// on the stream before the render, a deformation that wrote these means
// included), and the predecessor, the fp64 conic refinement, writes neither
// array.  The records and the visibility it and the projection write are
// read after the wait.
constexpr int kShadeThreads = 128;
template <int WR>
__device__ __forceinline__ void shade_stage_rows(const void* sh, int64_t base, int nb, uint4* __restrict__ rows) {
    if constexpr (WR > 0) {
        const uint4* src = reinterpret_cast<const uint4*>(static_cast<const unsigned char*>(sh) + base * (16 * WR));
        for (int q = threadIdx.x; q < nb * WR; q += kShadeThreads) {
            const int r = q / WR;
            rows[r * (WR | 1) + (q - r * WR)] = src[q];
        }
    }
}

template <int DEG>
__global__ void __launch_bounds__(kShadeThreads) shade_gaussians_kernel(const float* __restrict__ means, const void* __restrict__ sh,
                                                              int sh_dtype, int64_t N, const DevCam* __restrict__ cams,
                                                              int ncams, const BinInfo* __restrict__ bin, int64_t ntot,
                                                              GRec* __restrict__ grec, GRec16* __restrict__ grec16) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    // 16-byte words per staged row (0: the rows are read in place)
    constexpr int W32 = (12 * K) % 16 == 0 ? 12 * K / 16 : 0, W16 = (6 * K) % 16 == 0 ? 6 * K / 16 : 0;
    constexpr int WMAX = W32 > W16 ? W32 : W16;
    __shared__ uint4 s_rows[kShadeThreads * (WMAX | 1)];
    const bool bf = sh_dtype == UMGS_BF16;
    const int64_t base = (int64_t)blockIdx.x * kShadeThreads;
    const int64_t i = base + threadIdx.x;
    const int nb = (int)min((int64_t)kShadeThreads, N - base);
    if (bf) shade_stage_rows<W16>(sh, base, nb, s_rows);
    else shade_stage_rows<W32>(sh, base, nb, s_rows);
    float mx = 0.f, my = 0.f, mz = 0.f;
    if (i < N) { mx = means[3 * i]; my = means[3 * i + 1]; mz = means[3 * i + 2]; }
    pdl_enter();
    if ((bf ? W16 : W32) > 0) __syncthreads();
    if (i >= N) return;
    float c[3 * K];
    bool done_rows = false;
    if constexpr (W16 > 0) {
        if (bf) {
            const uint4* row = s_rows + threadIdx.x * (W16 | 1);
#pragma unroll
            for (int q = 0; q < W16; ++q) {
                const uint4 u = row[q];
                const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    c[8 * q + 2 * h] = __uint_as_float(w[h] << 16);
                    c[8 * q + 2 * h + 1] = __uint_as_float(w[h] & 0xffff0000u);
                }
            }
            done_rows = true;
        }
    }
    if constexpr (W32 > 0) {
        if (!bf) {
            const float4* row = reinterpret_cast<const float4*>(s_rows + threadIdx.x * (W32 | 1));
#pragma unroll
            for (int k = 0; k < W32; ++k) {
                const float4 t = row[k];
                c[4 * k] = t.x; c[4 * k + 1] = t.y; c[4 * k + 2] = t.z; c[4 * k + 3] = t.w;
            }
            done_rows = true;
        }
    }
    if (!done_rows && bf) {
        // 3K bf16 values per Gaussian: 8-byte loads where a row allows them
        constexpr int NB = 3 * K * 2;
        const unsigned char* p = static_cast<const unsigned char*>(sh) + i * NB;
        if (NB % 8 == 0) {
#pragma unroll
            for (int q = 0; q < NB / 8; ++q) {
                const uint2 u = reinterpret_cast<const uint2*>(p)[q];
                c[4 * q] = __uint_as_float(u.x << 16); c[4 * q + 1] = __uint_as_float(u.x & 0xffff0000u);
                c[4 * q + 2] = __uint_as_float(u.y << 16); c[4 * q + 3] = __uint_as_float(u.y & 0xffff0000u);
            }
        } else {
            const unsigned short* q = reinterpret_cast<const unsigned short*>(p);
#pragma unroll
            for (int k = 0; k < 3 * K; ++k) c[k] = __uint_as_float(((unsigned int)q[k]) << 16);
        }
    } else if (!done_rows) {
        const float* p = static_cast<const float*>(sh) + i * 3 * K;
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) c[k] = p[k];
    }
    for (int cam = 0; cam < ncams; ++cam) {
        if (!bin[(int64_t)cam * ntot + i].valid) continue;
        const DevCam& C = cams[cam];
        const float dx = mx - C.campos[0], dy = my - C.campos[1], dz = mz - C.campos[2];
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        const float x = dx * inv, y = dy * inv, z = dz * inv;
        float Y[K];
        Y[0] = 0.28209479177387814f;                                   // 1/(2 sqrt(pi))
        if (DEG > 0) {
            const float c1 = 0.4886025119029199f;                      // sqrt(3/(4 pi))
            Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
        }
        if (DEG > 1) {
            const float xx = x * x, yy = y * y, zz = z * z;
            Y[4] = 1.0925484305920792f * x * y;                        // sqrt(15/pi)/2
            Y[5] = -1.0925484305920792f * y * z;
            Y[6] = 0.31539156525252005f * (2.f * zz - xx - yy);       // sqrt(5/pi)/4
            Y[7] = -1.0925484305920792f * x * z;
            Y[8] = 0.5462742152960396f * (xx - yy);                    // sqrt(15/pi)/4
            if (DEG > 2) {
                Y[9] = -0.5900435899266435f * y * (3.f * xx - yy);    // sqrt(35/(2 pi))/4
                Y[10] = 2.890611442640554f * x * y * z;                // sqrt(105/pi)/2
                Y[11] = -0.4570457994644658f * y * (4.f * zz - xx - yy);  // sqrt(21/(2 pi))/4
                Y[12] = 0.3731763325901154f * z * (2.f * zz - 3.f * xx - 3.f * yy);  // sqrt(7/pi)/4
                Y[13] = -0.4570457994644658f * x * (4.f * zz - xx - yy);
                Y[14] = 1.445305721320277f * z * (xx - yy);            // sqrt(105/pi)/4
                Y[15] = -0.5900435899266435f * x * (xx - 3.f * yy);
            }
        }
        float rgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = fmaf(c[3 * k + ch], Y[k], acc);
            rgb[ch] = fmaxf(acc + 0.5f, 0.f);
        }
        if (grec16) {
            reinterpret_cast<uint2*>(&grec16[(int64_t)cam * N + i].v1)[0] =
                make_uint2(pack_half2(rgb[0], rgb[1]), pack_half2(rgb[2], 0.f));
        } else {
            float4* gp = reinterpret_cast<float4*>(grec + (int64_t)cam * N + i);
            reinterpret_cast<float2*>(gp + 1)[1] = make_float2(rgb[0], rgb[1]);
            reinterpret_cast<float*>(gp + 2)[0] = rgb[2];
        }
    }
}

// ---------------------------------------------------------------------------
// canonical triangle setup

__device__ __forceinline__ long long floor_div256(long long a) { return a >> 8; }
__device__ __forceinline__ long long ceil_div256(long long a) { return -((-a) >> 8); }

__global__ void __launch_bounds__(256) setup_triangles_kernel(
    const float* __restrict__ verts, const int32_t* __restrict__ faces, const float* __restrict__ vcolor,
    const float* __restrict__ valpha, const float* __restrict__ falpha, const float* __restrict__ uv, int tex,
    int64_t nv, int64_t nf,
    int64_t tri_base /* index of this mesh's first face among all triangles */, int64_t nt_total,
    int64_t id_base /* unified id of this mesh's first face */, const DevCam* __restrict__ cams, int ncams,
    int ts, int tiles_x, int tiles_per_cam, TRec* __restrict__ trec, BinInfo* __restrict__ bin,
    int64_t ntot_prims, int32_t* __restrict__ status,
    int dilate /* soft-edge coverage: rect widened by this many pixels */, float isig /* 1/edge_sigma or 0 */) {
    pdl_enter();
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int vid[3] = {faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]};
    bool idx_ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (vid[k] < 0 || vid[k] >= nv) idx_ok = false;
    if (!idx_ok) {
        atomicOr(status, 1);
        for (int cam = 0; cam < ncams; ++cam) {
            BinInfo bi; bi.rx = 1u; bi.ry = 1u; bi.dbits = 0u; bi.valid = 0u;
            bin[(int64_t)cam * ntot_prims + id_base + f] = bi;
        }
        return;
    }
    float P[3][3], col[9], al[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int d = 0; d < 3; ++d) P[k][d] = verts[3 * (int64_t)vid[k] + d];
    }
    if (uv) {  // textured: the vertices' (u, v) in col[0..5]
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            col[2 * k] = uv[2 * (int64_t)vid[k]];
            col[2 * k + 1] = uv[2 * (int64_t)vid[k] + 1];
            col[6 + k] = 0.f;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) col[3 * k + d] = vcolor[3 * (int64_t)vid[k] + d];
    }
    int const_alpha = 1;  // 0: interpolated vertex alpha, 1: face alpha, 2: no alpha (1)
    if (falpha) { al[0] = al[1] = al[2] = falpha[f]; }
    else if (valpha) { const_alpha = 0; al[0] = valpha[vid[0]]; al[1] = valpha[vid[1]]; al[2] = valpha[vid[2]]; }
    else { const_alpha = 2; al[0] = al[1] = al[2] = 1.f; }
    for (int cam = 0; cam < ncams; ++cam) {
        const DevCam& C = cams[cam];
        const float* R = C.R;
        float Zv[3], uv[3], vv[3];
        long long sx[3], sy[3];
        bool valid = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float X = fa(dot3c(R[0], R[1], R[2], P[k][0], P[k][1], P[k][2]), C.t[0]);
            const float Y = fa(dot3c(R[3], R[4], R[5], P[k][0], P[k][1], P[k][2]), C.t[1]);
            const float Z = fa(dot3c(R[6], R[7], R[8], P[k][0], P[k][1], P[k][2]), C.t[2]);
            const float u = fa(fdv(fm(C.fx, X), Z), C.cx);
            const float v = fa(fdv(fm(C.fy, Y), Z), C.cy);
            const bool ok = Z > C.near_z && isfinite(u) && isfinite(v) && fabsf(u) <= 16384.f && fabsf(v) <= 16384.f;
            valid = valid && ok;
            Zv[k] = Z; uv[k] = u; vv[k] = v;
            sx[k] = ok ? __float2ll_rn(fm(256.f, u)) : 0;
            sy[k] = ok ? __float2ll_rn(fm(256.f, v)) : 0;
        }
        const long long area = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sx[2] - sx[0]) * (sy[1] - sy[0]);
        valid = valid && area != 0;
        long long ox[3] = {sx[0], sx[1], sx[2]}, oy[3] = {sy[0], sy[1], sy[2]};
        if (area < 0) { ox[1] = sx[2]; ox[2] = sx[1]; oy[1] = sy[2]; oy[2] = sy[1]; }
        const long long xmin = min(sx[0], min(sx[1], sx[2])), xmax = max(sx[0], max(sx[1], sx[2]));
        const long long ymin = min(sy[0], min(sy[1], sy[2])), ymax = max(sy[0], max(sy[1], sy[2]));
        const long long xlo = max(ceil_div256(xmin - 224) - dilate, 0LL);
        const long long xhi = min(floor_div256(xmax - 32) + dilate, (long long)(C.W - 1));
        const long long ylo = max(ceil_div256(ymin - 224) - dilate, 0LL);
        const long long yhi = min(floor_div256(ymax - 32) + dilate, (long long)(C.H - 1));
        valid = valid && xlo <= xhi && ylo <= yhi;
        BinInfo bi;
        bi.dbits = __float_as_uint(fdv(fa(fa(Zv[0], Zv[1]), Zv[2]), 3.f));
        bi.valid = valid ? 1u : 0u;
        const int64_t bidx = (int64_t)cam * ntot_prims + id_base + f;
        if (!valid) { bi.rx = 1u; bi.ry = 1u; bin[bidx] = bi; continue; }
        bi.rx = (uint32_t)xlo | ((uint32_t)xhi << 16);
        bi.ry = (uint32_t)ylo | ((uint32_t)yhi << 16);
        bin[bidx] = bi;
        TRec t;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            const long long A = oy[a] - oy[b];
            const long long B = ox[b] - ox[a];
            const long long Cc = ox[a] * oy[b] - oy[a] * ox[b];
            const bool topleft = A > 0 || (A == 0 && B > 0);
            t.A[k] = (int32_t)A;
            t.B[k] = (int32_t)B;
            t.C[k] = Cc - (topleft ? 0 : 1);
            t.u[k] = uv[k];
            t.v[k] = vv[k];
            t.iz[k] = 1.f / Zv[k];
            t.alpha[k] = al[k];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) t.col[k] = col[k];
        t.const_alpha = const_alpha;
        t.tex = uv ? tex + 1 : 0;
        t.orient = area > 0 ? 1 : -1;
        t.rx = bi.rx;
        t.ry = bi.ry;
        t.pad2 = isig;  // soft-edge coverage: 1/edge_sigma (0: binary sample coverage)
        trec[(int64_t)cam * nt_total + tri_base + f] = t;
    }
}

// The frame's status words (n) and the tile scan's look-back words (nq),
// cleared at the start of every render.
__global__ void zero_words_kernel(uint32_t* __restrict__ p, int n, uint64_t* __restrict__ q, int64_t nq) {
    pdl_enter();
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0; i < n; i += stride) p[i] = 0u;
    for (int64_t i = i0; i < nq; i += stride) q[i] = 0ull;
}

// ---------------------------------------------------------------------------
// binning.  Every tile's list must hold the records whose pixel rect touches
// it, in (depth bits, id) order.  Instead of emitting one (tile, id) pair per
// covered tile and sorting all of them by tile, the records are
//   1. sorted once by depth bits (stable LSD radix sort of all (camera,
//      primitive) records; ties stay in id order),
//   2. emitted in that order as (region, id) pairs, a region being a block of
//      kRegionTX x kRegionTY tiles (4x fewer pairs than tiles at 1080p),
//   3. sorted stably by region (one 8-bit pass for up to 256 regions),
//   4. expanded region by region into the tile lists: each region's pairs
//      are cut into chunks of kRegionChunk; a counting pass gives every
//      (chunk, tile of the region) its count, an exclusive scan over the
//      chunks of a region and over all tiles gives each its first slot, and
//      a fill pass writes each id to its tiles in chunk order, ranking the
//      ids of a chunk per tile with warp ballots (so the order within a tile
//      is the region order, which is the depth order).

constexpr int kRegionTX = 8, kRegionTY = 4;  // tiles per region: one bit each of a 32-bit mask
// A (region, id) key carries the record's region-local tile rect in its low
// kRectBits bits (x0, x1: 3 bits each, y0, y1: 2 bits each) and the region
// index above them; the region sort skips the rect bits.
constexpr int kRectBits = 10;
constexpr int64_t kMaxRegions = (int64_t)1 << (32 - kRectBits);
constexpr int kRegionChunk = 2048;           // region pairs per count/fill block
constexpr int kRegionThreads = 256;

// Tiles and regions a record's tile rect meets (both 0 for a culled record).
struct RecordRects {
    int tx0, tx1, ty0, ty1;   // tile rect
    int gx0, gy0, gw, gh;     // region rect
};
__device__ __forceinline__ RecordRects record_rects(const BinInfo& b, int ts) {
    RecordRects r;
    r.tx0 = (int)(b.rx & 0xffff) / ts; r.tx1 = (int)(b.rx >> 16) / ts;
    r.ty0 = (int)(b.ry & 0xffff) / ts; r.ty1 = (int)(b.ry >> 16) / ts;
    r.gx0 = r.tx0 / kRegionTX;
    r.gy0 = r.ty0 / kRegionTY;
    r.gw = r.tx1 / kRegionTX - r.gx0 + 1;
    r.gh = r.ty1 / kRegionTY - r.gy0 + 1;
    return r;
}

// Per (camera, primitive) record, in record order (grid-stride, one block
// of 1024 threads per SM, so that a histogram bin takes one global atomic per
// SM):
// * the depth key (0xffffffff for culled records) and the record index,
//   the inputs of the depth sort;
// * for the depth sort's high digits (DepthDigits), ~min and max of the valid
//   keys: one atomic pair per block into slot blockIdx % kRadixMapSlots of
//   mm (mm[2s] = ~min, mm[2s+1] = max; all start at 0);
// * the depth sort's digit counts that need no minimum: the low and second
//   byte of every key (dhist[0..255], dhist[256..511]), the third byte of
//   the valid keys (dhist[512..767]) and the number of culled records;
// * the number of tiles and of regions the record's rect meets, summed
//   (64-bit, one atomic per block) into *ktotal (the length of all tile
//   lists together) and *rtotal (the number of (region, id) pairs);
// * and the look-back words of the emission and of the depth sort's first
//   pass cleared.
__global__ void __launch_bounds__(1024) prim_keys_kernel(const BinInfo* __restrict__ bin, int64_t n, int64_t ntot,
                                                         int ts, int regions_x, int regions_per_cam,
                                                         uint32_t* __restrict__ pk, uint32_t* __restrict__ pv,
                                                         uint32_t* __restrict__ n_dev, uint32_t* __restrict__ mm,
                                                         uint32_t* __restrict__ dhist, uint32_t* __restrict__ n_culled,
                                                         unsigned long long* __restrict__ ktotal,
                                                         unsigned long long* __restrict__ rtotal,
                                                         uint64_t* __restrict__ lbe, int64_t lbe_words,
                                                         uint32_t* __restrict__ lb0, int64_t lb0_words) {
    pdl_enter();
    constexpr int U = 4;  // records per thread and round, loaded together
    __shared__ uint32_t s_mm[2][32];
    __shared__ unsigned long long s_sum[2][32];
    __shared__ uint32_t s_cul[32];
    __shared__ uint32_t s_dh[3 * 256];
    const int t = threadIdx.x;
    for (int j = t; j < 3 * 256; j += blockDim.x) s_dh[j] = 0u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + t;
    if (i0 == 0) *n_dev = (uint32_t)n;
    for (int64_t j = i0; j < lbe_words; j += stride) lbe[j] = 0ull;
    for (int64_t j = i0; j < lb0_words; j += stride) lb0[j] = 0u;
    __syncthreads();
    uint32_t nmin = 0u, kmax = 0u, culled = 0u;  // ~min, max over this thread's valid keys
    unsigned long long tiles = 0, regions = 0;
    const int lane = t & 31;
    for (int64_t r0 = i0; r0 - lane < n; r0 += U * stride) {  // (warp-uniform trip count)
        BinInfo bb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = r0 + u * stride;
            if (i < n) bb[u] = bin[i];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = r0 + u * stride;
            const bool live = i < n;
            const bool valid = live && bb[u].valid;
            const uint32_t k = valid ? bb[u].dbits : 0xffffffffu;
            if (live) {
                pk[i] = k;
                pv[i] = (uint32_t)i;
            }
            // low and second byte: spread, plain atomics (culled records are
            // counted below); third byte: clustered, one atomic per distinct
            // value in the warp
            if (valid) {
                atomicAdd(&s_dh[k & 255u], 1u);
                atomicAdd(&s_dh[256 + ((k >> 8) & 255u)], 1u);
            }
            const uint32_t d2 = (k >> 16) & 255u;
            const unsigned peers = match_digit8(d2, valid);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_dh[512 + d2], (uint32_t)__popc(peers));
            culled += (live && !valid) ? 1u : 0u;
            if (!valid) continue;
            nmin = max(nmin, ~k);
            kmax = max(kmax, k);
            const RecordRects r = record_rects(bb[u], ts);
            tiles += (unsigned long long)((r.tx1 - r.tx0 + 1) * (r.ty1 - r.ty0 + 1));
            regions += (unsigned long long)(r.gw * r.gh);
        }
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        nmin = max(nmin, __shfl_xor_sync(0xffffffffu, nmin, d));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, d));
        culled += __shfl_xor_sync(0xffffffffu, culled, d);
        tiles += __shfl_xor_sync(0xffffffffu, tiles, d);
        regions += __shfl_xor_sync(0xffffffffu, regions, d);
    }
    if ((t & 31) == 0) {
        s_mm[0][t >> 5] = nmin; s_mm[1][t >> 5] = kmax;
        s_sum[0][t >> 5] = tiles; s_sum[1][t >> 5] = regions;
        s_cul[t >> 5] = culled;
    }
    __syncthreads();
    if (t == 0) {
        uint32_t a = 0u, c = 0u, cu = 0u;
        unsigned long long st = 0, sr = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = max(a, s_mm[0][w]); c = max(c, s_mm[1][w]);
            st += s_sum[0][w]; sr += s_sum[1][w]; cu += s_cul[w];
        }
        if (a | c) {
            uint32_t* slot = mm + 2 * (blockIdx.x % kRadixMapSlots);
            atomicMax(slot, a);
            atomicMax(slot + 1, c);
        }
        if (st) atomicAdd(ktotal, st);
        if (sr) atomicAdd(rtotal, sr);
        if (cu) {  // culled records: key 0xffffffff
            atomicAdd(n_culled, cu);
            s_dh[255] += cu;
            s_dh[256 + 255] += cu;
        }
    }
    __syncthreads();
    for (int j = t; j < 3 * 256; j += blockDim.x)
        if (s_dh[j]) atomicAdd(&dhist[j], s_dh[j]);
}

// (region, id) pairs of the depth-sorted records (the depth sort's result is
// in pv_b after an odd number of passes that ran, else in pv_a): record i
// owns the slots [off(i), off(i) + regions(i)), its regions in row-major
// order, with off the exclusive prefix of the region counts over the sorted
// records, found in the same kernel: a block (tile index from *counter)
// takes kEmitRecords consecutive records, warp w the w-th 256 of them in 8
// rounds of 32; per-warp scans and a scan over the warps give the block's
// offsets, and a warp look-back over the blocks before it (one word per
// block in lbe) the block's first slot.  Then each warp fills the
// (contiguous) slots of a round's 32 records together: lane l writes slots
// l, l + 32, ... of the round's range, finding the owning record by binary
// search over the round's exclusive prefix, so the writes are coalesced and
// a record with many regions does not hold up its warp.
// Capacity: when the tile lists would hold more than `kcap` entries (or more
// than 2^32 - 2), or the pairs more than `rcap`, nothing is emitted, the
// region-pair count *rn (the region sort's count) is set to 0 so that no tile
// list gets an entry, and the overflow is recorded: status bit 2 for a
// capacity, status[1] = 0xffffffff for the 32-bit limit.  Thread 0 of block 0
// also publishes the number of tile-list entries in status[1]; the blocks
// clear the look-back words of the region sort's first pass (lbr, tiles of
// `rtile` pairs) and count the digits of the region sort's `rpasses` 8-bit
// passes over the emitted pairs' region index (rhist[p * 256 + d]: pairs
// whose region r has (r >> 8p) & 255 == d; in depth order consecutive pairs
// rarely share a region, so plain shared-memory atomics).
constexpr int kEmitRounds = 8;
constexpr int kEmitRecords = 256 * kEmitRounds;
__global__ void __launch_bounds__(256) emit_region_pairs_kernel(
    const BinInfo* __restrict__ bin, const uint32_t* __restrict__ pv_a, const uint32_t* __restrict__ pv_b,
    const uint32_t* __restrict__ mm, int64_t n, int64_t ntot, int ts, int regions_x, int regions_per_cam,
    const unsigned long long* __restrict__ ktotal, const unsigned long long* __restrict__ rtotal, int64_t kcap,
    uint32_t* __restrict__ rk, uint32_t* __restrict__ rv, int64_t rcap, uint32_t* __restrict__ rn,
    int32_t* __restrict__ status, uint64_t* __restrict__ lbe, uint32_t* __restrict__ counter,
    PassLookback lbr, int64_t rtile, uint32_t* __restrict__ rhist, int rpasses) {
    pdl_enter();
    __shared__ uint32_t s_rh[3 * 256];
    __shared__ uint2 s_rect[kEmitRecords];  // per record of the block: tile rect (x0 | x1 << 16, y0 | y1 << 16)
    __shared__ uint32_t s_rec[kEmitRecords];  // ... and its record index
    __shared__ uint32_t s_wtot[8];
    __shared__ uint32_t s_id;
    __shared__ unsigned long long s_base[8];
    const unsigned long long K = *ktotal, RT = *rtotal;
    const bool over = K > (unsigned long long)kcap || K >= 0xffffffffull || RT > (unsigned long long)rcap;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (blockIdx.x == 0 && t == 0) {
        status[1] = (int32_t)(uint32_t)(K >= 0xffffffffull ? 0xffffffffull : K);
        if (over && K < 0xffffffffull) atomicOr(status, 4);
        *rn = over ? 0u : (uint32_t)RT;
    }
    if (over) return;
    {   // the region sort's first look-back words, for its live tiles
        const int64_t tiles = ((int64_t)RT + rtile - 1) / rtile;
        const int64_t words = tiles * 256, gwords = lookback_groups(tiles) * 256;
        const int64_t j0 = blockIdx.x * (int64_t)blockDim.x + t, stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t j = j0; j < words; j += stride) lbr.tiles[j] = 0u;
        for (int64_t j = j0; j < gwords; j += stride) lbr.groups[j] = 0ull;
    }
    for (int j = t; j < 3 * 256; j += blockDim.x) s_rh[j] = 0u;
    if (t == 0) s_id = atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t b = s_id;
    const uint32_t* __restrict__ pv = (depth_digits(mm).passes_run() & 1) ? pv_b : pv_a;
    const int64_t wbase = b * kEmitRecords + warp * 256;  // the warp's first record
    // 1. region counts, exclusive prefix within the warp's 256 records
    int cnt[kEmitRounds], excl[kEmitRounds];
    int run = 0;
#pragma unroll
    for (int j = 0; j < kEmitRounds; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        const int local = warp * 256 + j * 32 + lane;
        cnt[j] = 0;
        if (i < n) {
            const uint32_t rec = pv[i];
            const BinInfo bi = bin[rec];
            if (bi.valid) {
                const RecordRects r = record_rects(bi, ts);
                cnt[j] = r.gw * r.gh;
                s_rect[local] = make_uint2((uint32_t)r.tx0 | ((uint32_t)r.tx1 << 16),
                                           (uint32_t)r.ty0 | ((uint32_t)r.ty1 << 16));
                s_rec[local] = rec;
            }
        }
        int inc = cnt[j];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        excl[j] = run + inc - cnt[j];
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) s_wtot[warp] = (uint32_t)run;
    __syncthreads();
    // 2. the warps' offsets and the block's first slot (warp 0)
    if (warp == 0) {
        const uint32_t wt = lane < 8 ? s_wtot[lane] : 0u;
        uint32_t winc = wt;
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, winc, d);
            if (lane >= d) winc += y;
        }
        const uint32_t btot = __shfl_sync(0xffffffffu, winc, 7);
        if (lane == 0) lb_store(lbe + b, (b == 0 ? kLbInc : kLbAgg) | btot);
        const uint64_t bex = lookback_warp(lbe, b, reinterpret_cast<uint32_t*>(status));
        if (lane == 0 && b > 0) lb_store(lbe + b, kLbInc | (bex + btot));
        if (lane < 8) s_base[lane] = bex + (winc - wt);
    }
    __syncthreads();
    const int64_t warp_slot = (int64_t)s_base[warp];
    // 3. emission, round by round
#pragma unroll
    for (int j = 0; j < kEmitRounds; ++j) {
        if (wbase + j * 32 >= n) break;  // (warp-uniform)
        const int local = warp * 256 + j * 32 + lane;
        RecordRects rr{0, 0, 0, 0, 0, 0, 1, 0};
        uint32_t id = 0, rbase = 0;
        if (cnt[j] > 0) {  // (the rect and record staged in step 1, no second gather)
            const uint32_t rec = s_rec[local];
            const uint2 q = s_rect[local];
            const int cam = (int)(rec / ntot);
            id = (uint32_t)(rec - (int64_t)cam * ntot);
            rr.tx0 = (int)(q.x & 0xffffu); rr.tx1 = (int)(q.x >> 16);
            rr.ty0 = (int)(q.y & 0xffffu); rr.ty1 = (int)(q.y >> 16);
            rr.gx0 = rr.tx0 / kRegionTX;
            rr.gy0 = rr.ty0 / kRegionTY;
            rr.gw = rr.tx1 / kRegionTX - rr.gx0 + 1;
            rr.gh = rr.ty1 / kRegionTY - rr.gy0 + 1;
            rbase = (uint32_t)cam * (uint32_t)regions_per_cam;
        }
        const int e0 = __shfl_sync(0xffffffffu, excl[j], 0);
        const int ex = excl[j] - e0;  // exclusive prefix within the round
        const int total = __shfl_sync(0xffffffffu, ex + cnt[j], 31);
        const int64_t base = warp_slot + e0;
        for (int s0 = 0; s0 < total; s0 += 32) {
            const int s = s0 + lane;
            // owner: the last lane r with ex[r] <= s
            int r = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int c = r + step;
                const int e = __shfl_sync(0xffffffffu, ex, c & 31);
                if (c < 32 && e <= s) r = c;
            }
            const int re = __shfl_sync(0xffffffffu, ex, r);
            const int rx = __shfl_sync(0xffffffffu, rr.gx0, r);
            const int ry = __shfl_sync(0xffffffffu, rr.gy0, r);
            const int rw = __shfl_sync(0xffffffffu, rr.gw, r);
            const uint32_t rid = __shfl_sync(0xffffffffu, id, r);
            const uint32_t rrb = __shfl_sync(0xffffffffu, rbase, r);
            const int rtx0 = __shfl_sync(0xffffffffu, rr.tx0, r), rtx1 = __shfl_sync(0xffffffffu, rr.tx1, r);
            const int rty0 = __shfl_sync(0xffffffffu, rr.ty0, r), rty1 = __shfl_sync(0xffffffffu, rr.ty1, r);
            const int64_t o = base + s;
            if (s < total && o < rcap) {
                const int k = s - re;
                const int gy = ry + k / rw, gx = rx + k % rw;
                // the record's tiles inside region (gx, gy), region-local
                const int lx0 = max(rtx0 - gx * kRegionTX, 0), lx1 = min(rtx1 - gx * kRegionTX, kRegionTX - 1);
                const int ly0 = max(rty0 - gy * kRegionTY, 0), ly1 = min(rty1 - gy * kRegionTY, kRegionTY - 1);
                const uint32_t lrect = (uint32_t)(lx0 | (lx1 << 3) | (ly0 << 6) | (ly1 << 8));
                const uint32_t region = rrb + (uint32_t)(gy * regions_x + gx);
                rk[o] = (region << kRectBits) | lrect;
                rv[o] = rid;
                for (int q = 0; q < rpasses; ++q) atomicAdd(&s_rh[q * 256 + ((region >> (8 * q)) & 255u)], 1u);
            }
        }
    }
    __syncthreads();
    for (int j = t; j < rpasses * 256; j += blockDim.x)
        if (s_rh[j]) atomicAdd(&rhist[j], s_rh[j]);
}

// Region starts and chunk offsets of a render with at most 256 regions (one
// block), from the region counts of the region sort's histogram (the pairs
// of region r are rhist[r]; none when the lists overflowed, *rn == 0):
// rstart[r] = first pair of region r, rstart[R] = pair count; coff[r] =
// first count/fill chunk of region r, coff[R] = *nblk = chunk count.
__global__ void __launch_bounds__(256) region_scan_small_kernel(const uint32_t* __restrict__ rhist,
                                                                const uint32_t* __restrict__ rn, int64_t R,
                                                                uint32_t* __restrict__ rstart,
                                                                uint32_t* __restrict__ coff,
                                                                uint32_t* __restrict__ nblk) {
    pdl_enter();
    __shared__ uint32_t s_warp[32];
    const int t = threadIdx.x;
    const uint32_t c = (t < R && *rn != 0u) ? rhist[t] : 0u;
    uint32_t tot, ctot;
    const uint32_t st = block_exclusive_scan_256(c, s_warp, tot);
    const uint32_t ch = (c + kRegionChunk - 1) / kRegionChunk;
    const uint32_t co = block_exclusive_scan_256(ch, s_warp, ctot);
    if (t < R) {
        rstart[t] = st;
        coff[t] = co;
    }
    if (t == 0) {
        rstart[R] = tot;
        coff[R] = ctot;
        *nblk = ctot;
    }
}

// Region starts from the region-sorted keys: rstart[r] = first pair of region
// r (regions without pairs get the next region's start), rstart[R] = count.
// Grid-stride over the pairs: a pair whose region differs from its
// predecessor's writes the starts of the regions in between.
__global__ void region_starts_kernel(const uint32_t* __restrict__ rk, const uint32_t* __restrict__ rn, int64_t rcap,
                                     int64_t R, uint32_t* __restrict__ rstart) {
    pdl_enter();
    const int64_t n = min((int64_t)*rn, rcap);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n == 0) {
        for (int64_t r = i0; r <= R; r += stride) rstart[r] = 0u;
        return;
    }
    for (int64_t i = i0; i < n; i += stride) {
        const int64_t k = rk[i] >> kRectBits;
        const int64_t kp = i > 0 ? (int64_t)(rk[i - 1] >> kRectBits) : -1;
        for (int64_t r = kp + 1; r <= k; ++r) rstart[r] = (uint32_t)i;
        if (i == n - 1)
            for (int64_t r = k + 1; r <= R; ++r) rstart[r] = (uint32_t)n;
    }
}

// Inputs of the exclusive scans below, one uint32 per index.
struct ArrayIn {
    const uint32_t* a;
    __device__ uint32_t operator()(int64_t i) const { return a[i]; }
};
// number of count/fill chunks of region i
struct ChunksIn {
    const uint32_t* rstart;
    __device__ uint32_t operator()(int64_t i) const {
        return (rstart[i + 1] - rstart[i] + kRegionChunk - 1) / kRegionChunk;
    }
};
// list length of tile t (sum over its region's chunks); also writes, per
// chunk, the count of the region's earlier chunks for that tile (the
// chunk's first slot within the tile's list)
struct TileTotalIn {
    const uint32_t* coff;
    const uint32_t* nblk;
    const uint32_t* ccnt;
    uint32_t* cpre;
    int64_t R;
    int tiles_x, tiles_per_cam, regions_x, regions_per_cam;
    __device__ uint32_t operator()(int64_t t) const {
        const int cam = (int)(t / tiles_per_cam);
        const int lt = (int)(t - (int64_t)cam * tiles_per_cam);
        const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
        const int64_t r = (int64_t)cam * regions_per_cam + (ty / kRegionTY) * regions_x + tx / kRegionTX;
        const int l = (ty % kRegionTY) * kRegionTX + tx % kRegionTX;
        const uint32_t b0 = coff[r], b1 = r + 1 < R ? coff[r + 1] : *nblk;
        uint32_t run = 0;
        for (uint32_t b = b0; b < b1; ++b) {
            cpre[(int64_t)b * 32 + l] = run;
            run += ccnt[(int64_t)b * 32 + l];
        }
        return run;
    }
};

// Exclusive scan of n (<= kSmallScanMax) values in one block of 1024
// threads, 1024 per round: out[i] for i < n, out[n] = total = *total.
constexpr int64_t kSmallScanMax = 1 << 15;
template <class In, class Out>
__global__ void __launch_bounds__(1024) scan_small_kernel(In in, int64_t n, Out* __restrict__ out,
                                                          uint32_t* __restrict__ total) {
    pdl_enter();
    __shared__ uint32_t s_warp[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int64_t b = 0; b < n; b += 1024) {
        const int64_t i = b + threadIdx.x;
        const uint32_t x = i < n ? in(i) : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) s_warp[w] = inc;
        __syncthreads();
        if (w == 0) {
            uint32_t v = s_warp[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += y;
            }
            s_warp[lane] = v;
        }
        __syncthreads();
        if (i < n) out[i] = (Out)(carry + inc - x + (w > 0 ? s_warp[w - 1] : 0u));
        carry += s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[n] = (Out)carry;
        *total = carry;
    }
}

// Per-index values of an input functor (for the multi-block paths).
template <class In>
__global__ void gather_in_kernel(In in, int64_t n, uint32_t* __restrict__ out) {
    pdl_enter();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in(i);
}

// The region and chunk of count/fill block `blk` (< nblk): the last region
// whose first chunk is at or before it (regions without pairs own no chunk).
__device__ __forceinline__ int64_t region_of_chunk(const uint32_t* __restrict__ coff, int64_t R, uint32_t blk) {
    int64_t lo = 0, hi = R - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (coff[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Region-local tile mask of a (region, id) key: bit (ly * kRegionTX + lx)
// for every tile of the rect packed in its low kRectBits bits.
__device__ __forceinline__ uint32_t key_tile_mask(uint32_t key) {
    const int lx0 = key & 7, lx1 = (key >> 3) & 7, ly0 = (key >> 6) & 3, ly1 = (key >> 8) & 3;
    const uint32_t row = (0xffu >> (kRegionTX - 1 - lx1)) & (0xffu << lx0);
    const uint32_t rows = (0xffffffffu >> (8 * (kRegionTY - 1 - ly1))) & (0xffffffffu << (8 * ly0));
    return (row * 0x01010101u) & rows;
}
static_assert(kRegionTX == 8 && kRegionTY == 4, "key_tile_mask packs 8 tiles per byte, 4 rows");

struct RegionChunk {
    int64_t e0, e1;      // pair range of the chunk
    int tx0, ty0;        // first tile of the region
    int64_t tile0;       // global index of the region's first tile
};

__device__ __forceinline__ RegionChunk region_chunk(const uint32_t* __restrict__ coff, const uint32_t* __restrict__ rstart,
                                                    int64_t R, uint32_t blk, int regions_x, int regions_per_cam,
                                                    int tiles_x, int tiles_per_cam) {
    RegionChunk c;
    const int64_t r = region_of_chunk(coff, R, blk);
    const int64_t j = blk - coff[r];
    const int64_t s = rstart[r], e = rstart[r + 1];
    c.e0 = s + j * kRegionChunk;
    c.e1 = min(c.e0 + kRegionChunk, e);
    const int cam = (int)(r / regions_per_cam);
    const int lr = (int)(r - (int64_t)cam * regions_per_cam);
    const int gy = lr / regions_x, gx = lr - gy * regions_x;
    c.tx0 = gx * kRegionTX;
    c.ty0 = gy * kRegionTY;
    c.tile0 = (int64_t)cam * tiles_per_cam + (int64_t)c.ty0 * tiles_x + c.tx0;
    return c;
}

constexpr int kRegionItems = kRegionChunk / kRegionThreads;

// 32 x 32 bit-matrix transpose across a warp (recursive 2 x 2 block swaps):
// on entry lane r holds row r (bit c = element (r, c)); on exit lane c holds
// column c (bit r).  For tile masks this gives lane t the ballot of tile t.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
        const uint32_t m = j == 16 ? 0x0000ffffu : j == 8 ? 0x00ff00ffu : j == 4 ? 0x0f0f0f0fu : j == 2 ? 0x33333333u
                                                                                                     : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y << j) & ~m));
    }
    return x;
}

// Counting pass: per chunk and tile of its region, the number of the chunk's
// pairs whose record covers the tile (lane t of a warp counts tile t from the
// transposed masks).
__global__ void __launch_bounds__(kRegionThreads) region_count_kernel(
    const uint32_t* __restrict__ rk, const uint32_t* __restrict__ coff, const uint32_t* __restrict__ rstart,
    const uint32_t* __restrict__ nblk_dev, int64_t R, int regions_x, int regions_per_cam, int tiles_x,
    int tiles_per_cam, uint32_t* __restrict__ ccnt) {
    pdl_enter();
    __shared__ uint32_t s_cnt[kRegionThreads / 32][32];
    if (blockIdx.x >= *nblk_dev) return;
    const RegionChunk c = region_chunk(coff, rstart, R, blockIdx.x, regions_x, regions_per_cam, tiles_x,
                                       tiles_per_cam);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t m[kRegionItems];
#pragma unroll
    for (int q = 0; q < kRegionItems; ++q) {
        const int64_t e = c.e0 + q * kRegionThreads + threadIdx.x;
        m[q] = e < c.e1 ? key_tile_mask(rk[e]) : 0u;
    }
    uint32_t mine = 0;
#pragma unroll
    for (int q = 0; q < kRegionItems; ++q) mine += __popc(warp_transpose32(m[q]));
    s_cnt[warp][lane] = mine;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kRegionThreads / 32; ++w) s += s_cnt[w][threadIdx.x];
        ccnt[(int64_t)blockIdx.x * 32 + threadIdx.x] = s;
    }
}

// Fill pass: writes each pair's id into the lists of the tiles its record
// covers.  Rounds of 256 pairs in order; per tile, the warp's ballot (its
// transposed masks) ranks the pairs of a warp and a scan over the warps ranks
// the warps, so each tile receives the chunk's ids in pair order.  The ids
// are staged in shared memory, tile by
// tile (the chunk's tile counts are known from the counting pass), and then
// written out as contiguous runs; a chunk with more than kFillStage entries
// writes them directly.  Every warp keeps the per-tile running slots itself
// (lane t: tile t), so one barrier per round suffices, and ballots alternate
// between two buffers: a warp writes round q + 2's ballots only after the
// barrier of round q + 1, which every warp passes after its reads of round q.
constexpr int kFillStage = 10240;  // staged ids per chunk (40 KB)
__global__ void __launch_bounds__(kRegionThreads) region_fill_kernel(
    const uint32_t* __restrict__ rk, const uint32_t* __restrict__ rv, const uint32_t* __restrict__ coff,
    const uint32_t* __restrict__ rstart, const uint32_t* __restrict__ nblk_dev, int64_t R, int regions_x,
    int regions_per_cam, int tiles_x, int tiles_y, int tiles_per_cam, const int64_t* __restrict__ tile_off,
    const uint32_t* __restrict__ ccnt, const uint32_t* __restrict__ cpre, uint32_t* __restrict__ ids) {
    pdl_enter();
    constexpr int NW = kRegionThreads / 32;
    __shared__ uint32_t s_bal[2][NW][32];
    __shared__ uint32_t s_pre[2][NW][32];
    __shared__ uint32_t s_cst[33];    // staged start of each tile
    __shared__ uint32_t s_base[32];   // global first slot of each tile's run
    __shared__ uint32_t s_stage[kFillStage];
    if (blockIdx.x >= *nblk_dev) return;
    const RegionChunk c = region_chunk(coff, rstart, R, blockIdx.x, regions_x, regions_per_cam, tiles_x,
                                       tiles_per_cam);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        const int lx = lane % kRegionTX, ly = lane / kRegionTX;
        const bool exists = c.tx0 + lx < tiles_x && c.ty0 + ly < tiles_y;
        const uint32_t cnt = ccnt[(int64_t)blockIdx.x * 32 + lane];
        s_base[lane] = exists ? (uint32_t)tile_off[c.tile0 + (int64_t)ly * tiles_x + lx] +
                                    cpre[(int64_t)blockIdx.x * 32 + lane]
                              : 0u;
        uint32_t inc = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        s_cst[lane] = inc - cnt;
        if (lane == 31) s_cst[32] = inc;
    }
    __syncthreads();
    const bool staged = s_cst[32] <= (uint32_t)kFillStage;  // block-uniform
    // lane t of every warp: the next slot of tile t (staged or global),
    // advanced by every round's count of the whole block
    uint32_t run = staged ? s_cst[lane] : s_base[lane];
    uint32_t id[kRegionItems], m[kRegionItems];
#pragma unroll
    for (int q = 0; q < kRegionItems; ++q) {
        const int64_t e = c.e0 + q * kRegionThreads + threadIdx.x;
        const bool in = e < c.e1;
        m[q] = in ? key_tile_mask(rk[e]) : 0u;
        id[q] = in ? rv[e] : 0u;
    }
    uint32_t* const dst = staged ? s_stage : ids;
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int q = 0; q < kRegionItems; ++q) {
        if (c.e0 + q * kRegionThreads >= c.e1) break;  // block-uniform
        const int buf = q & 1;
        s_bal[buf][warp][lane] = warp_transpose32(m[q]);  // lane t: the warp's ballot of tile t
        __syncthreads();
        // lane t: this warp's first slot of tile t in this round (the counts of
        // the warps before it), and every warp advances its own running slots
        // by the round's total: no second barrier, no serial warp
        uint32_t pre = run;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t cw = __popc(s_bal[buf][w][lane]);
            pre += w < warp ? cw : 0u;
            run += cw;
        }
        s_pre[buf][warp][lane] = pre;  // (a row of this warp's own)
        __syncwarp();
        uint32_t mm = m[q];
        while (mm) {
            const int t = __ffs(mm) - 1;
            mm &= mm - 1u;
            dst[s_pre[buf][warp][t] + __popc(s_bal[buf][warp][t] & lt_mask)] = id[q];
        }
        __syncwarp();
    }
    if (!staged) return;
    __syncthreads();
    // staged slot k belongs to the last tile t with s_cst[t] <= k
    const uint32_t E = s_cst[32];
    for (uint32_t k = threadIdx.x; k < E; k += kRegionThreads) {
        int t = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1)
            if (t + step < 32 && s_cst[t + step] <= k) t += step;
        ids[s_base[t] + (k - s_cst[t])] = s_stage[k];
    }
}

// tile_off (int64, M + 1 entries) from a 32-bit tile scan and its total.
__global__ void tile_off_kernel(const uint32_t* __restrict__ toff, const uint32_t* __restrict__ total, int64_t M,
                                int64_t* __restrict__ off) {
    pdl_enter();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < M) off[t] = toff[t];
    else if (t == M) off[M] = *total;
}

// ---------------------------------------------------------------------------
// frame inspection: per tile (one thread each), its ids and their depth bits

__global__ void lists_kernel(const int64_t* __restrict__ off, const uint32_t* __restrict__ tids, int64_t M,
                             const BinInfo* __restrict__ bin, int64_t ntot, int tiles_per_cam,
                             int32_t* __restrict__ ids, uint32_t* __restrict__ dbits) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= M) return;
    const int64_t cam = t / tiles_per_cam;
    for (int64_t i = off[t]; i < off[t + 1]; ++i) {
        const uint32_t id = tids[i];
        ids[i] = (int32_t)id;
        dbits[i] = bin[cam * ntot + id].dbits;
    }
}


// exclusive scan of n uint32 counts into out; the grand total goes to *total (device)
cudaError_t scan_u32(umgs_frame* fr, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, cudaStream_t s) {
    const int64_t nb = (n + kRsTile - 1) / kRsTile;
    cudaError_t e = fr->rs_bsum.reserve(sizeof(uint32_t) * std::max<int64_t>(1, nb));
    if (e != cudaSuccess) return e;
    if (nb > (1 << 22)) return cudaErrorInvalidValue;
    uint32_t* overflow = reinterpret_cast<uint32_t*>(fr->status.as<int32_t>() + 9);
    launch_pdl(scan_reduce_kernel, (unsigned)nb, kRsThreads, 0, s, in, n, fr->rs_bsum.as<uint32_t>(), overflow);
    launch_pdl(scan_blocks_kernel, 1, 1024, 0, s, fr->rs_bsum.as<uint32_t>(), (int)nb, total, overflow);
    launch_pdl(scan_apply_kernel, (unsigned)nb, kRsThreads, 0, s, in, n, fr->rs_bsum.as<uint32_t>(), out);
    return cudaGetLastError();
}

// stable LSD radix sort of (k, v) on key bits [lo, lo + bits) (the bits above
// must be zero); the element count is read from device memory (n_dev, at most
// n_cap, which sizes the grids); ping-pongs with (k2, v2) and returns where
// the result ended
cudaError_t radix_sort_pairs(umgs_frame* fr, uint32_t* k, uint32_t* v, uint32_t* k2, uint32_t* v2,
                             const uint32_t* n_dev, int64_t n_cap, int bits, uint32_t** rk, uint32_t** rv,
                             cudaStream_t s, int lo, const uint32_t* key_mm) {
    const int64_t nb = radix_blocks(n_cap);
    const int items = radix_items(n_cap);
    const int64_t nh = 256 * nb;
    cudaError_t e = fr->rs_hist.reserve(sizeof(uint32_t) * nh);
    if (e != cudaSuccess) return e;
    e = fr->rs_hist2.reserve(sizeof(uint32_t) * 256);
    if (e != cudaSuccess) return e;
    uint32_t* hist = fr->rs_hist.as<uint32_t>();
    uint32_t* dtotal = fr->rs_hist2.as<uint32_t>();
    for (int shift = lo; shift < lo + bits; shift += 8) {
        if (items == 8) {
            launch_pdl(radix_upsweep_kernel<8>, (unsigned)nb, kRsThreads, 0, s, k, n_dev, n_cap, shift, (int)nb, hist,
                       key_mm);
        } else {
            launch_pdl(radix_upsweep_kernel<16>, (unsigned)nb, kRsThreads, 0, s, k, n_dev, n_cap, shift, (int)nb, hist,
                       key_mm);
        }
        launch_pdl(radix_hist_scan_kernel, 256, kRsThreads, 0, s, hist, (int)nb, n_dev, n_cap, kRsThreads * items, dtotal,
                   shift, key_mm);
        if (items == 8) {
            launch_pdl(radix_downsweep_kernel<8>, (unsigned)nb, kRsThreads, 0, s, k, v, n_dev, n_cap, shift, (int)nb, hist,
                       dtotal, k2, v2, key_mm);
        } else {
            launch_pdl(radix_downsweep_kernel<16>, (unsigned)nb, kRsThreads, 0, s, k, v, n_dev, n_cap, shift, (int)nb,
                       hist, dtotal, k2, v2, key_mm);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint32_t* t = k; k = k2; k2 = t;
        t = v; v = v2; v2 = t;
    }
    *rk = k;
    *rv = v;
    return cudaSuccess;
}

// Passes [0, npass) of the single-sweep stable LSD radix sort of (k, v) on
// the 8-bit digits at lo + 8p, or the depth sort's DepthDigits when mm is
// given (then npass = 4, ghist holds prim_keys_kernel's counts, n_culled the
// culled records, and pass 2 counts pass 3's digits into ghist[768..]);
// ghist: 256 digit counts per pass; counters: one zeroed tile counter per
// pass; the frame's lb_a / lb_b alternate as look-back words
// (lookback_layout for radix_blocks(n_cap) tiles; lb_a cleared beforehand for
// the first pass's live tiles).  The element count is
// read from n_dev (at most n_cap, which sizes the grids); the result is in
// (k2, v2) after an odd number of passes that ran, else in (k, v).
cudaError_t onesweep_sort(umgs_frame* fr, uint32_t* k, uint32_t* v, uint32_t* k2, uint32_t* v2,
                          const uint32_t* n_dev, int64_t n_cap, int lo, int npass, uint32_t* ghist,
                          uint32_t* counters, const uint32_t* mm, const uint32_t* n_culled, uint32_t* err,
                          cudaStream_t s) {
    const int64_t nb = radix_blocks(n_cap);
    const int items = radix_items(n_cap);
    const PassLookback lb[2] = {lookback_layout(fr->lb_a.ptr, nb), lookback_layout(fr->lb_b.ptr, nb)};
    const PassLookback none{nullptr, nullptr};
    for (int p = 0; p < npass; ++p) {
        const uint32_t* ki = (p & 1) ? k2 : k;
        const uint32_t* vi = (p & 1) ? v2 : v;
        uint32_t* ko = (p & 1) ? k : k2;
        uint32_t* vo = (p & 1) ? v : v2;
        const PassLookback nxt = p + 1 < npass ? lb[(p + 1) & 1] : none;
        const int shift = lo + 8 * p;
        const uint32_t* gh = ghist + 256 * p;
#define UMGS_PASS(IT, MP)                                                                                      \
    launch_pdl(onesweep_pass_kernel<IT, MP>, (unsigned)nb, kRsThreads, 0, s, ki, vi, n_dev, n_cap, shift, gh,  \
               lb[p & 1], nxt, counters + p, ko, vo, mm, n_culled, mm ? ghist + 3 * 256 : nullptr, err)
        if (mm) {
            if (items == 8) UMGS_PASS(8, true);
            else UMGS_PASS(16, true);
        } else {
            if (items == 8) UMGS_PASS(8, false);
            else UMGS_PASS(16, false);
        }
#undef UMGS_PASS
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// host orchestration

static inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// Buffers of the binning stage for `rcap` (region, id) pairs and `kcap`
// tile-list entries, for the frame's current image, tile size and cameras.
cudaError_t reserve_binning(umgs_frame* fr, int64_t rcap, int64_t kcap) {
    const int regions_x = (fr->tiles_x + kRegionTX - 1) / kRegionTX;
    const int64_t R = (int64_t)regions_x * ((fr->tiles_y + kRegionTY - 1) / kRegionTY) * fr->ncams;
    const int64_t M = fr->num_tiles;
    const int64_t nblk_max = (rcap + kRegionChunk - 1) / kRegionChunk + R;
    cudaError_t e;
    for (DevBuf* b : {&fr->tk, &fr->tv, &fr->tk2, &fr->tv2})
        if ((e = b->reserve(sizeof(uint32_t) * std::max<int64_t>(1, rcap))) != cudaSuccess) return e;
    if ((e = fr->tl_ids.reserve(sizeof(uint32_t) * std::max<int64_t>(1, kcap))) != cudaSuccess) return e;
    if ((e = fr->rg_start.reserve(sizeof(uint32_t) * (R + 1))) != cudaSuccess) return e;
    if ((e = fr->rg_nchunk.reserve(sizeof(uint32_t) * R)) != cudaSuccess) return e;
    if ((e = fr->rg_coff.reserve(sizeof(uint32_t) * (R + 1))) != cudaSuccess) return e;
    if ((e = fr->rg_ccnt.reserve(sizeof(uint32_t) * 32 * nblk_max)) != cudaSuccess) return e;
    if ((e = fr->rg_cpre.reserve(sizeof(uint32_t) * 32 * nblk_max)) != cudaSuccess) return e;
    if ((e = fr->tl_cnt.reserve(sizeof(uint32_t) * std::max<int64_t>(1, M))) != cudaSuccess) return e;
    if ((e = fr->tl_off.reserve(sizeof(uint32_t) * std::max<int64_t>(1, M))) != cudaSuccess) return e;
    // look-back words of the region sort's passes
    if ((e = fr->lb_a.reserve(lookback_bytes(radix_blocks(rcap)))) != cudaSuccess) return e;
    if ((e = fr->lb_b.reserve(lookback_bytes(radix_blocks(rcap)))) != cudaSuccess) return e;
    return cudaSuccess;
}

umgs_status render_forward(umgs_ctx* ctx, const umgs_gaussians* g, const umgs_mesh* meshes, int32_t nmeshes,
                           const umgs_camera* cams, int32_t ncams, const umgs_render_opts& opts, float* out_rgbt,
                           umgs_frame* fr, cudaStream_t stream) {
    const int ts = opts.tile_size;
    const bool soft = (opts.flags & UMGS_RENDER_SOFT_EDGE) != 0;
    const int W = cams[0].width, H = cams[0].height;
    const int tiles_x = (W + ts - 1) / ts, tiles_y = (H + ts - 1) / ts;
    const int tiles_per_cam = tiles_x * tiles_y;
    const int64_t M = (int64_t)tiles_per_cam * ncams;
    const int64_t Ng = g ? g->n : 0;
    int64_t Nt = 0;
    fr->mesh_offset.clear();
    for (int m = 0; m < nmeshes; ++m) { fr->mesh_offset.push_back(Ng + Nt); Nt += meshes[m].nf; }
    const int64_t Ntot = Ng + Nt;
    if (Ntot >= (int64_t)0xffffffffLL) return fail(ctx, UMGS_ERR_INVALID_ARG, "too many primitives (ids are 32-bit)");
    if (M >= (int64_t)1 << 31) return fail(ctx, UMGS_ERR_INVALID_ARG, "too many tiles");
    fr->valid = false;
    fr->ng = Ng; fr->nt = Nt; fr->ncams = ncams; fr->W = W; fr->H = H;
    fr->tile = ts; fr->tiles_x = tiles_x; fr->tiles_y = tiles_y; fr->num_tiles = M;
    fr->blend_mode = opts.blend_mode; fr->t_eps = opts.t_eps;
    fr->opts = opts;
    fr->bg[0] = opts.bg[0]; fr->bg[1] = opts.bg[1]; fr->bg[2] = opts.bg[2];

    cudaError_t e;
#define UMGS_TRY(x)                                                   \
    do {                                                              \
        e = (x);                                                      \
        if (e == cudaErrorMemoryAllocation) {                         \
            cudaGetLastError();                                       \
            return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, #x);             \
        }                                                             \
        if (e != cudaSuccess) return cuda_fail(ctx, e, #x);           \
    } while (0)

    UMGS_TRY(fr->cams.reserve(sizeof(DevCam) * ncams));
    const bool mixed = (opts.flags & UMGS_RENDER_MIXED) != 0;
    fr->mixed = mixed;
    UMGS_TRY(fr->grec.reserve((mixed ? sizeof(GRec16) : sizeof(GRec)) * std::max<int64_t>(1, Ng * ncams)));
    UMGS_TRY(fr->trec.reserve(sizeof(TRec) * std::max<int64_t>(1, Nt * ncams)));
    UMGS_TRY(fr->bin.reserve(sizeof(BinInfo) * std::max<int64_t>(1, Ntot * ncams)));
    UMGS_TRY(fr->tile_off.reserve(sizeof(int64_t) * (M + 1)));
    UMGS_TRY(fr->lb_s.reserve(sizeof(uint64_t) * ((M + 255) / 256)));
    // status words: [0] error bits, [1] number of tile-list entries (32-bit,
    // 0xffffffff when it does not fit), [2] largest saved-stack need, [3] fp64
    // conic list length, [4] tile count for the tile-order sort, [5] record
    // count for the depth sort, [6..7] (region, id) pairs counted (u64), [8] persistent
    // work counter, [9] scan overflow, [10..11] tile-list entries (u64),
    // [12] (region, id) pairs sorted (0 after an overflow), [13] count/fill
    // chunks, [14] tile-list entries from the tile scan, [15] unused,
    // [16 ..) the depth sort's key-map slots (~min, max); then the
    // evaluation and work-split counters and, from kStatusBinWords, the
    // tile counters and digit histograms of the single-sweep binning kernels
    static_assert(kStatusEvalWords == 16 + 2 * kRadixMapSlots, "status word layout");
    UMGS_TRY(fr->status.reserve(sizeof(int32_t) * kStatusWords));

    // cameras: host -> pinned staging -> device
    std::vector<DevCam> dc(ncams);
    for (int c = 0; c < ncams; ++c) {
        const umgs_camera& cm = cams[c];
        DevCam& d = dc[c];
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) d.R[3 * r + k] = cm.viewmat[4 * r + k];
            d.t[r] = cm.viewmat[4 * r + 3];
        }
        d.fx = cm.fx; d.fy = cm.fy; d.cx = cm.cx; d.cy = cm.cy;
        d.W = cm.width; d.H = cm.height; d.near_z = cm.near_z;
        for (int k = 0; k < 3; ++k) {
            double s = 0;
            for (int r = 0; r < 3; ++r) s -= (double)cm.viewmat[4 * r + k] * (double)cm.viewmat[4 * r + 3];
            d.campos[k] = (float)s;
        }
        d.pad = 0;
    }
    // (inside a graph capture the cameras were uploaded by the sizing render;
    // cameras equal to the frame's last upload into the same buffer are not
    // sent again)
    const bool same_cams = fr->cams_dev == fr->cams.ptr && fr->cams_host.size() == (size_t)ncams &&
                           std::memcmp(fr->cams_host.data(), dc.data(), sizeof(DevCam) * ncams) == 0;
    if (!fr->capture && !same_cams) {
        UMGS_TRY(cudaMemcpyAsync(fr->cams.ptr, dc.data(), sizeof(DevCam) * ncams, cudaMemcpyHostToDevice, stream));
        fr->cams_host = dc;
        fr->cams_dev = fr->cams.ptr;
    }
    // status words cleared by a kernel (not a memset node), so that the
    // programmatic launch chain runs on from the stream's previous kernel
    {
        const int64_t nq = (M + 255) / 256;  // the tile scan's look-back words
        const unsigned zg = (unsigned)std::min<int64_t>((std::max<int64_t>(nq, kStatusWords) + 1023) / 1024,
                                                        ctx->num_sms);
        launch_pdl(zero_words_kernel, zg, 256, 0, stream, reinterpret_cast<uint32_t*>(fr->status.ptr), kStatusWords,
                   fr->lb_s.as<uint64_t>(), nq);
    }

    const DevCam* dcams = fr->cams.as<DevCam>();
    const unsigned fix_cap = (unsigned)std::min<int64_t>(std::max<int64_t>(1, Ng * ncams), 1 << 22);
    UMGS_TRY(fr->fix_list.reserve(sizeof(int64_t) * fix_cap));
    if (Ng > 0) {
        StageTimer tm(ctx, UMGS_STAGE_PROJECT_GAUSSIANS, stream);
        launch_pdl(project_gaussians_kernel, grid_for(Ng, 256), 256, 0, stream, 
            g->means, g->quats, g->scales, g->opacities, g->sh, g->sh_dtype, g->sh_degree, g->cov3d, Ng, dcams,
            ncams, ts, tiles_x, tiles_per_cam, fr->grec.as<GRec>(), mixed ? fr->grec.as<GRec16>() : nullptr,
            fr->bin.as<BinInfo>(), Ntot, reinterpret_cast<unsigned*>(fr->status.as<int32_t>() + 3),
            fr->fix_list.as<int64_t>(), fix_cap);
        UMGS_TRY(cudaGetLastError());
        launch_pdl(refine_conics_kernel, 4 * ctx->num_sms, 128, 0, stream, 
            g->means, g->quats, g->scales, g->cov3d, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot,
            reinterpret_cast<unsigned*>(fr->status.as<int32_t>() + 3), fr->fix_list.as<int64_t>(), fix_cap,
            fr->grec.as<GRec>(), mixed ? fr->grec.as<GRec16>() : nullptr);
        UMGS_TRY(cudaGetLastError());
    }
    if (Ng > 0) {
        StageTimer tm(ctx, UMGS_STAGE_SHADE_GAUSSIANS, stream);
        const unsigned gb = grid_for(Ng, kShadeThreads);
        GRec16* g16 = mixed ? fr->grec.as<GRec16>() : nullptr;
        switch (g->sh_degree) {
            case 0: launch_pdl(shade_gaussians_kernel<0>, gb, kShadeThreads, 0, stream, g->means, g->sh, g->sh_dtype, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot, fr->grec.as<GRec>(), g16); break;
            case 1: launch_pdl(shade_gaussians_kernel<1>, gb, kShadeThreads, 0, stream, g->means, g->sh, g->sh_dtype, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot, fr->grec.as<GRec>(), g16); break;
            case 2: launch_pdl(shade_gaussians_kernel<2>, gb, kShadeThreads, 0, stream, g->means, g->sh, g->sh_dtype, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot, fr->grec.as<GRec>(), g16); break;
            default: launch_pdl(shade_gaussians_kernel<3>, gb, kShadeThreads, 0, stream, g->means, g->sh, g->sh_dtype, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot, fr->grec.as<GRec>(), g16); break;
        }
        UMGS_TRY(cudaGetLastError());
    }
    // texture table of the textured meshes (uploaded like the cameras)
    std::vector<DevTex> texs;
    std::vector<int> mesh_tex(std::max(1, (int)nmeshes), -1);
    for (int m = 0; m < nmeshes; ++m)
        if (meshes[m].uv && meshes[m].texture) {
            mesh_tex[m] = (int)texs.size();
            texs.push_back(DevTex{meshes[m].texture, meshes[m].tex_w, meshes[m].tex_h, 0});
        }
    UMGS_TRY(fr->textab.reserve(sizeof(DevTex) * std::max<size_t>(1, texs.size())));
    if (!texs.empty() && !fr->capture)
        UMGS_TRY(cudaMemcpyAsync(fr->textab.ptr, texs.data(), sizeof(DevTex) * texs.size(), cudaMemcpyHostToDevice,
                                 stream));
    int64_t tri_base = 0;
    for (int m = 0; m < nmeshes; ++m) {
        const umgs_mesh& me = meshes[m];
        if (me.nf > 0) {
            StageTimer tm(ctx, UMGS_STAGE_SETUP_TRIANGLES, stream);
            launch_pdl(setup_triangles_kernel, grid_for(me.nf, 256), 256, 0, stream, 
                me.verts, me.faces, me.vcolor, me.valpha, me.falpha, mesh_tex[m] >= 0 ? me.uv : nullptr,
                mesh_tex[m], me.nv, me.nf, tri_base, Nt, Ng + tri_base,
                dcams, ncams, ts, tiles_x, tiles_per_cam, fr->trec.as<TRec>(), fr->bin.as<BinInfo>(), Ntot,
                fr->status.as<int32_t>(), soft ? (int)ceilf(8.f * opts.edge_sigma) : 0,
                soft ? 1.f / opts.edge_sigma : 0.f);
            UMGS_TRY(cudaGetLastError());
        }
        tri_base += me.nf;
    }
    // ---- binning: depth sort of all records, (region, id) emission, stable
    // region sort, expansion into the tile lists (see prim_keys_kernel)
    const int64_t NR = Ntot * ncams;  // (camera, primitive) records
    const int regions_x = (tiles_x + kRegionTX - 1) / kRegionTX;
    const int regions_per_cam = regions_x * ((tiles_y + kRegionTY - 1) / kRegionTY);
    const int64_t R = (int64_t)regions_per_cam * ncams;
    if (R > kMaxRegions) return fail(ctx, UMGS_ERR_INVALID_ARG, "too many tile regions (cameras x regions > 2^22)");
    UMGS_TRY(fr->pk.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    UMGS_TRY(fr->pv.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    UMGS_TRY(fr->pk2.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    UMGS_TRY(fr->pv2.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    const int64_t nb_depth = radix_blocks(NR);
    UMGS_TRY(fr->lb_a.reserve(lookback_bytes(nb_depth)));
    UMGS_TRY(fr->lb_b.reserve(lookback_bytes(nb_depth)));
    const int64_t nb_emit = (NR + kEmitRecords - 1) / kEmitRecords;
    UMGS_TRY(fr->lb_e.reserve(sizeof(uint64_t) * std::max<int64_t>(1, nb_emit)));
    uint32_t* pk = fr->pk.as<uint32_t>();
    uint32_t* pv = fr->pv.as<uint32_t>();
    uint32_t* status_u = reinterpret_cast<uint32_t*>(fr->status.as<int32_t>());
    unsigned long long* ktotal = reinterpret_cast<unsigned long long*>(status_u + 10);
    unsigned long long* rtotal = reinterpret_cast<unsigned long long*>(status_u + 6);
    uint32_t* rn = status_u + 12;    // number of (region, id) pairs sorted
    uint32_t* nblk = status_u + 13;  // number of count/fill chunks
    uint32_t* ktot32 = status_u + 14;
    uint32_t* mm = status_u + 16;
    uint32_t* counters = status_u + kStatusBinWords;  // tile counters of the single-sweep kernels
    uint32_t* dhist = counters + kBinCounters;        // depth sort: 4 x 256 digit counts
    uint32_t* rhist = dhist + 4 * 256;                // region sort: 3 x 256 digit counts
    int rbits = 0;
    while (((int64_t)1 << rbits) < R) ++rbits;
    const int rpasses = (rbits + 7) / 8;  // region sort passes (none for a single region)
    if (NR > 0) {
        StageTimer tm(ctx, UMGS_STAGE_SCAN, stream);
        // (one block of 1024 threads per SM: a histogram bin takes one global atomic per SM)
        const unsigned pgrid = (unsigned)std::min<int64_t>(grid_for(NR, kHistThreads), ctx->num_sms);
        launch_pdl(prim_keys_kernel, pgrid, kHistThreads, 0, stream, fr->bin.as<BinInfo>(), NR, Ntot, ts, regions_x,
                   regions_per_cam, pk, pv, status_u + 5, mm, dhist, counters + kBinCulledWord, ktotal, rtotal,
                   fr->lb_e.as<uint64_t>(), nb_emit, fr->lb_a.as<uint32_t>(),
                   lookback_bytes(nb_depth) / (int64_t)sizeof(uint32_t));
        UMGS_TRY(cudaGetLastError());
        UMGS_TRY(onesweep_sort(fr, pk, pv, fr->pk2.as<uint32_t>(), fr->pv2.as<uint32_t>(), status_u + 5, NR, 0, 4,
                               dhist, counters, mm, counters + kBinCulledWord, status_u, stream));
    }
    int64_t Kcap, rcap;
    if (!fr->nosync) {
        // read back the status words: error bits, list entries, region pairs
        UMGS_TRY(cudaMemcpyAsync(ctx->pinned, fr->status.ptr, 16 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
        UMGS_TRY(cudaStreamSynchronize(stream));
        const uint32_t* w = reinterpret_cast<const uint32_t*>(ctx->pinned);
        const uint64_t K64 = (uint64_t)w[10] | ((uint64_t)w[11] << 32);
        const uint64_t R64 = (uint64_t)w[6] | ((uint64_t)w[7] << 32);
        if (w[0] & 1) return fail(ctx, UMGS_ERR_INVALID_ARG, "a face index is out of range");
        if (w[0] & kStatusLookbackTimeout) return fail(ctx, UMGS_ERR_TIMEOUT, "a binning look-back wait gave up");
        if (K64 >= 0xffffffffull) return fail(ctx, UMGS_ERR_CAPACITY, "more than 4294967294 (tile, primitive) pairs");
        fr->num_keys = (int64_t)K64;
        Kcap = (int64_t)K64;
        rcap = NR > 0 ? (int64_t)R64 : 0;  // (region pairs never outnumber list entries)
    } else {
        // no host read-back: the lists are held to the reserved capacity and
        // an overflow is flagged in the status word (bit 2); inside a capture
        // the buffers were sized beforehand
        Kcap = fr->key_capacity;
        rcap = Kcap;  // region pairs never outnumber list entries
        fr->num_keys = -1;
    }
    if (!fr->capture) UMGS_TRY(reserve_binning(fr, rcap, Kcap));
    fr->ids = fr->tl_ids.as<uint32_t>();
    const int items_r = radix_items(rcap);
    if (NR > 0) {
        StageTimer tm(ctx, UMGS_STAGE_SCATTER, stream);
        launch_pdl(emit_region_pairs_kernel, (unsigned)nb_emit, 256, 0, stream, fr->bin.as<BinInfo>(),
                   static_cast<const uint32_t*>(pv), static_cast<const uint32_t*>(fr->pv2.as<uint32_t>()),
                   static_cast<const uint32_t*>(mm), NR, Ntot, ts, regions_x, regions_per_cam, ktotal, rtotal, Kcap,
                   fr->tk.as<uint32_t>(), fr->tv.as<uint32_t>(), rcap, rn, fr->status.as<int32_t>(),
                   fr->lb_e.as<uint64_t>(), counters + kBinEmitCounter,
                   lookback_layout(fr->lb_a.ptr, radix_blocks(rcap)), (int64_t)kRsThreads * items_r, rhist,
                   std::max(1, rpasses));
        UMGS_TRY(cudaGetLastError());
    }
    {
        StageTimer tm(ctx, UMGS_STAGE_SORT, stream);
        uint32_t* rk = fr->tk.as<uint32_t>();
        uint32_t* rv = fr->tv.as<uint32_t>();
        if (NR > 0 && rcap > 0 && rpasses > 0) {
            UMGS_TRY(onesweep_sort(fr, fr->tk.as<uint32_t>(), fr->tv.as<uint32_t>(), fr->tk2.as<uint32_t>(),
                                   fr->tv2.as<uint32_t>(), rn, rcap, kRectBits, rpasses, rhist,
                                   counters + kBinRegionCounters, nullptr, nullptr, status_u, stream));
            if (rpasses & 1) {
                rk = fr->tk2.as<uint32_t>();
                rv = fr->tv2.as<uint32_t>();
            }
        }
        const int64_t nblk_max = (rcap + kRegionChunk - 1) / kRegionChunk + R;
        uint32_t* rstart = fr->rg_start.as<uint32_t>();
        uint32_t* coff = fr->rg_coff.as<uint32_t>();
        int64_t* toff64 = fr->tile_off.as<int64_t>();
        if (R <= 256) {
            // at most one region pass: its digit counts are the region counts
            launch_pdl(region_scan_small_kernel, 1, 256, 0, stream, static_cast<const uint32_t*>(rhist),
                       static_cast<const uint32_t*>(rn), R, rstart, coff, nblk);
        } else {
            const unsigned sgrid = (unsigned)std::min<int64_t>(grid_for(std::max(rcap, R + 1), 256), 8 * ctx->num_sms);
            launch_pdl(region_starts_kernel, sgrid, 256, 0, stream, rk, rn, rcap, R, rstart);
            UMGS_TRY(cudaGetLastError());
            if (R <= kSmallScanMax) {
                launch_pdl(scan_small_kernel<ChunksIn, uint32_t>, 1, 1024, 0, stream, ChunksIn{rstart}, R, coff, nblk);
            } else {
                launch_pdl(gather_in_kernel<ChunksIn>, grid_for(R, 256), 256, 0, stream, ChunksIn{rstart}, R,
                           fr->rg_nchunk.as<uint32_t>());
                UMGS_TRY(scan_u32(fr, fr->rg_nchunk.as<uint32_t>(), coff, R, nblk, stream));
            }
        }
        UMGS_TRY(cudaGetLastError());
        launch_pdl(region_count_kernel, (unsigned)nblk_max, kRegionThreads, 0, stream,
            rk, coff, rstart, nblk, R, regions_x, regions_per_cam, tiles_x, tiles_per_cam, fr->rg_ccnt.as<uint32_t>());
        UMGS_TRY(cudaGetLastError());
        const TileTotalIn tin{coff, nblk, fr->rg_ccnt.as<uint32_t>(), fr->rg_cpre.as<uint32_t>(), R, tiles_x,
                              tiles_per_cam, regions_x, regions_per_cam};
        // (one tile per thread: a tile's total walks its region's chunks)
        launch_pdl(scan_lookback_kernel<TileTotalIn, 1>, (unsigned)((M + 255) / 256), kRsThreads, 0, stream, tin, M,
                   toff64, ktot32, fr->lb_s.as<uint64_t>(), counters + kBinScanCounter, status_u);
        UMGS_TRY(cudaGetLastError());
        launch_pdl(region_fill_kernel, (unsigned)nblk_max, kRegionThreads, 0, stream,
            rk, rv, coff, rstart, nblk, R, regions_x, regions_per_cam, tiles_x, tiles_y, tiles_per_cam, toff64,
            fr->rg_ccnt.as<uint32_t>(), fr->rg_cpre.as<uint32_t>(), fr->tl_ids.as<uint32_t>());
        UMGS_TRY(cudaGetLastError());
    }
    UMGS_TRY(fr->last.reserve(sizeof(int32_t) * (int64_t)ncams * W * H));
    fr->has_depth = (opts.flags & UMGS_RENDER_DEPTH) != 0;
    if (fr->has_depth) UMGS_TRY(fr->depth.reserve(sizeof(float) * (int64_t)ncams * W * H));
    fr->saved = (opts.flags & UMGS_RENDER_SAVE_BACKWARD) != 0 && opts.blend_mode == UMGS_BLEND_FULL;
    if (fr->saved) {
        const int64_t npix = (int64_t)ncams * W * H;
        UMGS_TRY(fr->tfin.reserve(sizeof(float) * npix));
        UMGS_TRY(fr->ntri.reserve(sizeof(int32_t) * npix));
        UMGS_TRY(fr->stack.reserve(sizeof(float4) * npix * fr->stack_cap));
    }
    {
        StageTimer tm_comp(ctx, UMGS_STAGE_COMPOSITE, stream);
        if (soft) UMGS_TRY(launch_soft_composite(fr, opts, out_rgbt, stream));
        else UMGS_TRY(launch_composite(fr, opts, out_rgbt, stream));
    }
    fr->valid = true;
#undef UMGS_TRY
    return UMGS_OK;
}

umgs_status frame_check(umgs_frame* fr, cudaStream_t stream) {
    int32_t* w = reinterpret_cast<int32_t*>(fr->ctx->pinned);
    cudaError_t e = cudaMemcpyAsync(w, fr->status.ptr, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(fr->ctx, e, "reading the frame status");
    if (w[0] & 1) return fail(fr->ctx, UMGS_ERR_INVALID_ARG, "a face index is out of range");
    if (w[0] & kStatusLookbackTimeout) return fail(fr->ctx, UMGS_ERR_TIMEOUT, "a binning look-back wait gave up");
    if ((uint32_t)w[1] == 0xffffffffu)
        return fail(fr->ctx, UMGS_ERR_CAPACITY, "more than 4294967294 (tile, primitive) pairs");
    if (w[0] & 4)
        return fail(fr->ctx, UMGS_ERR_CAPACITY, "more (tile, primitive) pairs than the reserved capacity (" +
                                                     std::to_string(fr->key_capacity) + ")");
    return UMGS_OK;
}

umgs_status frame_lists(const umgs_frame* fr, int64_t* tile_ptr, int32_t* ids, uint32_t* dbits, cudaStream_t stream) {
    cudaError_t e = cudaMemcpyAsync(tile_ptr, fr->tile_off.ptr, sizeof(int64_t) * (fr->num_tiles + 1),
                                    cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(fr->ctx, e, "cudaMemcpyAsync(tile_ptr)");
    if (fr->num_keys > 0) {
        lists_kernel<<<grid_for(fr->num_tiles, 256), 256, 0, stream>>>(
            fr->tile_off.as<int64_t>(), fr->ids, fr->num_tiles, fr->bin.as<BinInfo>(), fr->ng + fr->nt,
            fr->tiles_x * fr->tiles_y, ids, dbits), count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(fr->ctx, e, "lists_kernel");
    }
    return UMGS_OK;
}

}  // namespace umgs
