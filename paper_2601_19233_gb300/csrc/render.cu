// Forward single-pass rasterization of Gaussians and triangles (Sec. 3.2).
//
// Pipeline per umgs_render call (all cameras in one set of launches):
//   1. project_gaussians / setup_triangles: one thread per primitive, looping
//      over cameras; canonical fp32 footprint (pixel rect) + depth key and a
//      compact record for the compositor; refine_conics_kernel recomputes the
//      few near-singular conics in fp64; shade_gaussians_kernel evaluates SH.
//   2. binning, a two-level stable radix sort (the onion sort):
//      a. every (camera, primitive) record sorted by its depth bits
//         (4 x 8-bit passes, stable, so equal depths stay in id order);
//      b. in that order every record emits one (tile, id) pair per tile its
//         rect touches (offsets from an exclusive scan of the tile counts);
//      c. the pairs are sorted stably by tile (8-bit passes over the tile
//         bits): each tile's list is then in (depth bits, id) order;
//      d. tile_ranges: per tile, the first index of its list (binary search).
//   3. composite: one CTA per tile, one thread per pixel; records of the
//      sorted list are staged through shared memory in batches; every pixel
//      blends its fragments front to back (Eq. 1-2 for Gaussians, Eq. 7-9
//      for entities of depth-adjacent triangles) and the CTA stops when
//      every pixel has T < t_eps (block-wide vote).
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
    out[0] = (float)(C2 / d2);
    out[1] = (float)(-B2 / d2);
    out[2] = (float)(A2 / d2);
}

// fp64 conics of the (camera, Gaussian) records listed by project_gaussians;
// when the list overflowed every record is re-tested.
__global__ void refine_conics_kernel(const float* __restrict__ means, const float* __restrict__ quats,
                                     const float* __restrict__ scales, const float* __restrict__ cov3d, int64_t N,
                                     const DevCam* __restrict__ cams, int ncams, const BinInfo* __restrict__ bin,
                                     int64_t ntot, const unsigned* __restrict__ fix_count,
                                     const int64_t* __restrict__ fix_list, unsigned fix_cap, GRec* __restrict__ grec,
                                     GRec16* __restrict__ grec16) {
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
            h[2] = pack_half2(-0.5f * kLog2e * cq[0], -kLog2e * cq[1]);
            h[3] = pack_half2(-0.5f * kLog2e * cq[2], o);
        } else {
            float* g = reinterpret_cast<float*>(grec + ri);
            g[2] = -0.5f * kLog2e * cq[0];
            g[3] = -kLog2e * cq[1];
            g[4] = -0.5f * kLog2e * cq[2];
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
        // conic (not a decision): fp32, or fp64 when the 2x2 determinant is
        // small relative to a*c (cancellation would cost > 10 bits)
        float ia, ib, ic;
        {
            const float id = 1.f / det;
            ia = c * id; ib = -b * id; ic = a * id;
        }
        if (det < 0.0009765625f * a * c) {  // near-singular: refined in fp64 by refine_conics_kernel
            const unsigned slot = atomicAdd(fix_count, 1u);
            if (slot < fix_cap) fix_list[slot] = ri;
        }
        // colour is written by shade_gaussians_kernel
        if (grec16) {
            GRec16* hp = grec16 + ri;
            hp->v0 = make_uint4(__float_as_uint(u), __float_as_uint(v),
                                pack_half2(-0.5f * kLog2e * ia, -kLog2e * ib), pack_half2(-0.5f * kLog2e * ic, o));
            reinterpret_cast<uint2*>(&hp->v1)[1] = make_uint2(bi.rx, bi.ry);
        } else {
            float4* gp = reinterpret_cast<float4*>(grec + ri);
            gp[0] = make_float4(u, v, -0.5f * kLog2e * ia, -kLog2e * ib);
            reinterpret_cast<float2*>(gp + 1)[0] = make_float2(-0.5f * kLog2e * ic, o);
            reinterpret_cast<float2*>(gp + 2)[0] = make_float2(0.f, __uint_as_float(bi.rx));
            reinterpret_cast<float*>(gp + 2)[2] = __uint_as_float(bi.ry);
        }
    }
}

// View-dependent colour of every visible (camera, Gaussian): one thread per
// Gaussian keeps its SH coefficients in registers across the cameras.
template <int DEG>
__global__ void __launch_bounds__(256) shade_gaussians_kernel(const float* __restrict__ means, const void* __restrict__ sh,
                                                              int sh_dtype, int64_t N, const DevCam* __restrict__ cams,
                                                              int ncams, const BinInfo* __restrict__ bin, int64_t ntot,
                                                              GRec* __restrict__ grec, GRec16* __restrict__ grec16) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float c[3 * K];
    if (sh_dtype == UMGS_BF16) {
        // 3K bf16 values per Gaussian: widest aligned vector loads (16 B for SH3)
        constexpr int NB = 3 * K * 2;
        const unsigned char* p = static_cast<const unsigned char*>(sh) + i * NB;
        if (NB % 16 == 0) {
#pragma unroll
            for (int q = 0; q < NB / 16; ++q) {
                const uint4 u = reinterpret_cast<const uint4*>(p)[q];
                const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    c[8 * q + 2 * h] = __uint_as_float(w[h] << 16);
                    c[8 * q + 2 * h + 1] = __uint_as_float(w[h] & 0xffff0000u);
                }
            }
        } else if (NB % 8 == 0) {
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
    } else if ((3 * K) % 4 == 0) {
        const float4* p = reinterpret_cast<const float4*>(static_cast<const float*>(sh) + i * 3 * K);
#pragma unroll
        for (int k = 0; k < 3 * K / 4; ++k) {
            const float4 t = p[k];
            c[4 * k] = t.x; c[4 * k + 1] = t.y; c[4 * k + 2] = t.z; c[4 * k + 3] = t.w;
        }
    } else {
        const float* p = static_cast<const float*>(sh) + i * 3 * K;
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) c[k] = p[k];
    }
    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
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
    const float* __restrict__ valpha, const float* __restrict__ falpha, int64_t nv, int64_t nf,
    int64_t tri_base /* index of this mesh's first face among all triangles */, int64_t nt_total,
    int64_t id_base /* unified id of this mesh's first face */, const DevCam* __restrict__ cams, int ncams,
    int ts, int tiles_x, int tiles_per_cam, TRec* __restrict__ trec, BinInfo* __restrict__ bin,
    int64_t ntot_prims, int32_t* __restrict__ status) {
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
        for (int d = 0; d < 3; ++d) {
            P[k][d] = verts[3 * (int64_t)vid[k] + d];
            col[3 * k + d] = vcolor[3 * (int64_t)vid[k] + d];
        }
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
        const long long xlo = max(ceil_div256(xmin - 224), 0LL), xhi = min(floor_div256(xmax - 32), (long long)(C.W - 1));
        const long long ylo = max(ceil_div256(ymin - 224), 0LL), yhi = min(floor_div256(ymax - 32), (long long)(C.H - 1));
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
        t.pad0 = 0; t.pad1 = 0;
#pragma unroll
        t.rx = bi.rx;
        t.ry = bi.ry;
        t.pad2 = 0.f;
        trec[(int64_t)cam * nt_total + tri_base + f] = t;
    }
}

// ---------------------------------------------------------------------------
// binning: a two-level stable radix sort (the "onion"): all (camera,
// primitive) records by depth bits, then the emitted (tile, primitive) pairs
// by tile.  Stability makes each tile's list come out in (depth bits, id)
// order without a per-tile sort.

__global__ void prim_keys_kernel(const BinInfo* __restrict__ bin, int64_t n, uint32_t* __restrict__ pk,
                                 uint32_t* __restrict__ pv, uint32_t* __restrict__ n_dev) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) *n_dev = (uint32_t)n;
    if (i >= n) return;
    const BinInfo b = bin[i];
    pk[i] = b.valid ? b.dbits : 0xffffffffu;
    pv[i] = (uint32_t)i;
}

__device__ __forceinline__ uint32_t tiles_of(const BinInfo& b, int ts) {
    if (!b.valid) return 0u;
    const int xlo = b.rx & 0xffff, xhi = b.rx >> 16, ylo = b.ry & 0xffff, yhi = b.ry >> 16;
    return (uint32_t)((xhi / ts - xlo / ts + 1) * (yhi / ts - ylo / ts + 1));
}

__global__ void tile_counts_kernel(const BinInfo* __restrict__ bin, const uint32_t* __restrict__ pv, int64_t n, int ts,
                                   uint32_t* __restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cnt[i] = tiles_of(bin[pv[i]], ts);
}

// (tile, id) pairs of the depth-sorted records: record i owns the slots
// [off[i], off[i] + tiles(i)), its tiles in row-major order.  Each warp takes
// 32 consecutive records and fills their (contiguous) slots together: lane l
// writes slots s = l, l + 32, ... of the warp's range, finding the owning
// record by binary search over the warp's exclusive prefix of tile counts,
// so the writes are coalesced and a record with many tiles does not hold up
// its warp.  Slots at or beyond `cap` are not written (the overflow is
// flagged in status bit 2); every slot below it is.
__global__ void __launch_bounds__(256) emit_pairs_kernel(const BinInfo* __restrict__ bin,
                                                         const uint32_t* __restrict__ pv,
                                                         const uint32_t* __restrict__ off, int64_t n, int64_t ntot,
                                                         int ts, int tiles_x, int tiles_per_cam,
                                                         uint32_t* __restrict__ tk, uint32_t* __restrict__ tv,
                                                         int64_t cap, int32_t* __restrict__ status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    if (i - lane >= n) return;  // whole warp past the end
    int xlo = 0, ylo = 0, w = 1, cnt = 0;
    uint32_t id = 0, tbase = 0;
    int64_t start = 0;
    if (i < n) {
        const uint32_t rec = pv[i];
        const BinInfo b = bin[rec];
        start = off[i];
        if (b.valid) {
            const int cam = (int)(rec / ntot);
            id = (uint32_t)(rec - (int64_t)cam * ntot);
            xlo = (int)(b.rx & 0xffff) / ts;
            const int xhi = (int)(b.rx >> 16) / ts;
            ylo = (int)(b.ry & 0xffff) / ts;
            const int yhi = (int)(b.ry >> 16) / ts;
            w = xhi - xlo + 1;
            cnt = w * (yhi - ylo + 1);
            tbase = (uint32_t)cam * (uint32_t)tiles_per_cam;
        }
    }
    // exclusive prefix of the counts within the warp
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int64_t base = __shfl_sync(0xffffffffu, start, 0);  // offsets are contiguous in record order
    if (lane == 0 && base + total > cap) atomicOr(status, 4);  // capacity overflow
    for (int s0 = 0; s0 < total; s0 += 32) {
        const int s = s0 + lane;
        // owner: the last lane r with excl[r] <= s
        int r = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int c = r + step;
            const int e = __shfl_sync(0xffffffffu, excl, c & 31);
            if (c < 32 && e <= s) r = c;
        }
        const int re = __shfl_sync(0xffffffffu, excl, r);
        const int rx = __shfl_sync(0xffffffffu, xlo, r);
        const int ry = __shfl_sync(0xffffffffu, ylo, r);
        const int rw = __shfl_sync(0xffffffffu, w, r);
        const uint32_t rid = __shfl_sync(0xffffffffu, id, r);
        const uint32_t rtb = __shfl_sync(0xffffffffu, tbase, r);
        const int64_t o = base + s;
        if (s < total && o < cap) {
            const int k = s - re;
            const int ty = ry + k / rw, tx = rx + k % rw;
            tk[o] = rtb + (uint32_t)(ty * tiles_x + tx);
            tv[o] = rid;
        }
    }
}

// tile_off[t] = first index of tile t in the sorted keys (lower bound).
// More pairs than the capacity (flagged by emit_pairs): the emission skipped
// records, so slots below the capacity may hold no pair; every tile is then
// left empty rather than reading them.
__global__ void tile_ranges_kernel(const uint32_t* __restrict__ tk, const uint32_t* __restrict__ K_dev, int64_t Kcap,
                                   int64_t M, int64_t* __restrict__ off) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t > M) return;
    const int64_t K = (int64_t)*K_dev > Kcap ? 0 : (int64_t)*K_dev;
    if (t == M) { off[M] = K; return; }
    int64_t lo = 0, hi = K;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (tk[mid] < (uint32_t)t) lo = mid + 1;
        else hi = mid;
    }
    off[t] = lo;
}

// ---------------------------------------------------------------------------
// compositor

constexpr int kBatch = 256;
// records staged per batch: 256, or 128 for 32x32 tiles (32 warps of lists)
template <int TS> struct BatchOf { static constexpr int value = TS == 32 ? 128 : 256; };

struct PixelState {
    float C[3];
    float T;
    float Tin;
    float t[4];
    float g_since;
    bool in_ent;
};

// SAVE: also keep what the backward pass needs: per pixel the final T and
// the number of covering triangle fragments, and per covering triangle
// fragment the four sub-sample transmittances before it (scaled by T_in/4)
// in a per-pixel stack of capacity `cap` (`need` records the largest count).
// MODE: UMGS_BLEND_* or kModeTProduct (FULL with the literal Eq. 6
// transmittance T <- T (1 - O_i alpha_i) inside an entity).
constexpr int kModeTProduct = 4;

template <int TS, bool SAVE, int MODE>
__device__ __forceinline__ void composite_tile(
    int tile, float4 (*__restrict__ s_rec)[10], uint32_t* __restrict__ s_id, uint32_t* __restrict__ s_wmask,
    uint8_t* __restrict__ s_list,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off,
    const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need) {
    constexpr int NT = TS * TS;
    constexpr int mode = MODE;
    const int cam = tile / tiles_per_cam;
    const int lt = tile - cam * tiles_per_cam;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    int lx, ly;
    block_pixel<TS>(threadIdx.x, lx, ly);
    const int px = tx * TS + lx, py = ty * TS + ly;
    const bool inside = px < W && py < H;
    const int64_t beg = off[tile], end = off[tile + 1];
    const GRec* G = grec + (int64_t)cam * Ng;
    const GRec16* G16 = grec16 ? grec16 + (int64_t)cam * Ng : nullptr;
    const TRec* TR = trec + (int64_t)cam * Nt;
    const float qx = px + 0.5f, qy = py + 0.5f;
    const long long scx = (long long)px * 256 + 128, scy = (long long)py * 256 + 128;

    PixelState st;
    st.C[0] = st.C[1] = st.C[2] = 0.f;
    st.T = 1.f; st.Tin = 1.f; st.g_since = 1.f;
    st.t[0] = st.t[1] = st.t[2] = st.t[3] = 1.f;
    st.in_ent = false;
    bool done = !inside;
    int last = 0;
    int sp = 0;
    const int64_t pix = ((int64_t)cam * H + py) * W + px;

    // warp w owns one 8 x 4 pixel block of the tile (block_pixel); every
    // record carries the mask of the blocks that can hold a fragment of it
    const int warp = threadIdx.x >> 5;
    const int tile_x0 = tx * TS, tile_y0 = ty * TS;
    const float pxf = (float)px, pyf = (float)py;
    constexpr int NB = BatchOf<TS>::value;
    for (int64_t b0 = beg; b0 < end; b0 += NB) {
        if (__syncthreads_count(done) == NT) break;
        const int n = (int)min((int64_t)NB, end - b0);
        const int lbase = (int)(b0 - beg) + 1;  // list position + 1 of the batch's first record
        for (int k = threadIdx.x; k < n; k += NT) {
            const uint32_t id = ids[b0 + k];
            s_id[k] = id;
            if (id >= Ng + Nt) {
                s_wmask[k] = 0u;  // not a record of this frame: no fragment
            } else if (id < Ng) {
                float4 a, b, c;
                if (G16) {  // fp16 record: widen to the fp32 layout
                    const uint4 h0 = G16[id].v0, h1 = G16[id].v1;
                    a = make_float4(__uint_as_float(h0.x), __uint_as_float(h0.y), half_lo(h0.z), half_hi(h0.z));
                    b = make_float4(half_lo(h0.w), half_hi(h0.w), half_lo(h1.x), half_hi(h1.x));
                    c = make_float4(half_lo(h1.y), __uint_as_float(h1.z), __uint_as_float(h1.w), 0.f);
                } else {
                    const float4* src = reinterpret_cast<const float4*>(G + id);
                    a = src[0]; b = src[1]; c = src[2];
                }
                const uint32_t rx = __float_as_uint(c.y), ry = __float_as_uint(c.z);
                s_rec[k][0] = a;
                s_rec[k][1] = make_float4(b.x, b.y, (float)(rx & 0xffff), (float)(rx >> 16));
                s_rec[k][2] = make_float4((float)(ry & 0xffff), (float)(ry >> 16), b.z, b.w);
                s_rec[k][3] = make_float4(c.x, 0.f, 0.f, 0.f);
                s_wmask[k] = gauss_block_mask<TS>(a.x, a.y, a.z, a.w, b.x, b.y, (int)(rx & 0xffff), (int)(rx >> 16),
                                                  (int)(ry & 0xffff), (int)(ry >> 16), tile_x0, tile_y0);
            } else {
                const float4* src = reinterpret_cast<const float4*>(TR + (id - Ng));
#pragma unroll
                for (int q = 0; q < 10; ++q) s_rec[k][q] = src[q];
                const TRec& tr = *reinterpret_cast<const TRec*>(&s_rec[k][0]);
                s_wmask[k] = box_block_mask<TS>((int)(tr.rx & 0xffff), (int)(tr.rx >> 16), (int)(tr.ry & 0xffff),
                                                (int)(tr.ry >> 16), tile_x0, tile_y0);
            }
        }
        __syncthreads();
        if (__any_sync(0xffffffffu, !done)) {
            // this warp's records of the batch, in order
            uint8_t* lst = s_list + warp * BatchOf<TS>::value;
            int cnt = 0;
            const int lane = threadIdx.x & 31;
            for (int c0 = 0; c0 < n; c0 += 32) {
                const bool mine = c0 + lane < n && ((s_wmask[c0 + lane] >> warp) & 1u);
                const unsigned bal = __ballot_sync(0xffffffffu, mine);
                if (mine) lst[cnt + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)(c0 + lane);
                cnt += __popc(bal);
            }
            __syncwarp();
            for (int li = 0; li < cnt; ++li) {
                const int k = lst[li];
                if (done) continue;
                const uint32_t id = s_id[k];
                if (id < Ng) {
                    const float4 q1 = s_rec[k][1], q2 = s_rec[k][2];
                    if (pxf < q1.z || pxf > q1.w || pyf < q2.x || pyf > q2.y) continue;
                    const float4 q0 = s_rec[k][0];
                    const float dx = __fsub_rn(qx, q0.x), dy = __fsub_rn(qy, q0.y);
                    const float p2 = gauss_power2(q0.z, q0.w, q1.x, dx, dy);
                    const float alpha = fminf(kAlphaMax, __fmul_rn(q1.y, fast_exp2(p2)));
                    if (alpha < kAlphaMin) continue;
                    const float w = alpha * st.T;
                    st.C[0] += w * q2.z; st.C[1] += w * q2.w; st.C[2] += w * s_rec[k][3].x;
                    st.T *= (1.f - alpha);
                    if (mode == UMGS_BLEND_ENTITY_ALL) st.g_since *= (1.f - alpha);
                    else st.in_ent = false;
                } else {
                    const TRec& t = *reinterpret_cast<const TRec*>(&s_rec[k][0]);
                    if (px < (int)(t.rx & 0xffff) || px > (int)(t.rx >> 16) || py < (int)(t.ry & 0xffff) ||
                        py > (int)(t.ry >> 16))
                        continue;
                    long long E[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) E[e] = (long long)t.A[e] * scx + (long long)t.B[e] * scy + t.C[e];
                    int mask = 0;
                    if (mode == UMGS_BLEND_DIRECT) {
                        mask = (E[0] >= 0 && E[1] >= 0 && E[2] >= 0) ? 0xf : 0;
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int sdx = sample_dx(j), sdy = sample_dy(j);
                            bool in = true;
#pragma unroll
                            for (int e = 0; e < 3; ++e) in = in && (E[e] + (long long)(t.A[e] * sdx + t.B[e] * sdy) >= 0);
                            mask |= in ? (1 << j) : 0;
                        }
                    }
                    if (mask == 0) continue;
                    // attributes at the pixel centre: perspective-correct
                    // barycentrics of the unsnapped triangle, clamped at 0
                    float lam[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const int a = (e + 1) % 3, b = (e + 2) % 3;
                        lam[e] = (t.u[a] - qx) * (t.v[b] - qy) - (t.u[b] - qx) * (t.v[a] - qy);
                    }
                    const float area = lam[0] + lam[1] + lam[2];
                    float wv[3];
                    if (area != 0.f) {
                        const float ia = 1.f / area;
#pragma unroll
                        for (int e = 0; e < 3; ++e) wv[e] = fmaxf(lam[e] * ia, 0.f) * t.iz[e];
                    } else {
#pragma unroll
                        for (int e = 0; e < 3; ++e) wv[e] = (1.f / 3.f) * t.iz[e];
                    }
                    const float ws = wv[0] + wv[1] + wv[2];
                    if (ws > 0.f) { const float is = 1.f / ws; wv[0] *= is; wv[1] *= is; wv[2] *= is; }
                    else { wv[0] = wv[1] = wv[2] = 1.f / 3.f; }
                    float col[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) col[c] = wv[0] * t.col[c] + wv[1] * t.col[3 + c] + wv[2] * t.col[6 + c];
                    float a = t.const_alpha ? t.alpha[0] : (wv[0] * t.alpha[0] + wv[1] * t.alpha[1] + wv[2] * t.alpha[2]);
                    a = fminf(fmaxf(a, 0.f), 1.f);
                    if (mode == UMGS_BLEND_DIRECT) {
                        const float w = a * st.T;
                        st.C[0] += w * col[0]; st.C[1] += w * col[1]; st.C[2] += w * col[2];
                        st.T *= (1.f - a);
                    } else if (mode == UMGS_BLEND_MSAA_ALL) {
                        const float O = 0.25f * (float)__popc(mask);
                        const float w = O * a * st.T;
                        st.C[0] += w * col[0]; st.C[1] += w * col[1]; st.C[2] += w * col[2];
                        st.T *= (1.f - O * a);
                    } else {
                        if (!st.in_ent) {
                            st.Tin = st.T;
                            st.t[0] = st.t[1] = st.t[2] = st.t[3] = 1.f;
                            st.g_since = 1.f;
                            st.in_ent = true;
                        }
                        if (SAVE && mode == UMGS_BLEND_FULL) {
                            if (sp < cap) {
                                const float q = 0.25f * st.Tin;
                                stack[(int64_t)sp * npix + pix] = make_float4(q * st.t[0], q * st.t[1], q * st.t[2], q * st.t[3]);
                            }
                            ++sp;
                        }
                        float O = 0.f;
#pragma unroll
                        for (int j = 0; j < 4; ++j) O += ((mask >> j) & 1) ? st.t[j] : 0.f;
                        O *= 0.25f;
                        const float w = st.Tin * O * a;
                        st.C[0] += w * col[0]; st.C[1] += w * col[1]; st.C[2] += w * col[2];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if ((mask >> j) & 1) st.t[j] *= (1.f - a);
                        const float tm = 0.25f * ((st.t[0] + st.t[1]) + (st.t[2] + st.t[3]));
                        if (mode == kModeTProduct) st.T *= (1.f - O * a);
                        else st.T = (mode == UMGS_BLEND_ENTITY_ALL) ? st.Tin * tm * st.g_since : st.Tin * tm;
                    }
                }
                last = lbase + k;
                if (st.T < t_eps) done = true;
            }
        }
    }
    if (inside) {
        out[pix] = make_float4(st.C[0] + st.T * bg0, st.C[1] + st.T * bg1, st.C[2] + st.T * bg2, st.T);
        // bit 31: the pixel stopped at T < t_eps after list position `last`
        if (out_last) out_last[pix] = last | (st.T < t_eps ? (int)0x80000000u : 0);
        if (SAVE) {
            out_tfin[pix] = st.T;
            out_ntri[pix] = sp;
            if (sp > cap) atomicMax(need, sp);
        }
    }
}


// one CTA per tile (grid launch)
template <int TS, bool SAVE, int MODE>
__global__ void __launch_bounds__(TS * TS) composite_kernel(
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need) {
    constexpr int NB = BatchOf<TS>::value;
    __shared__ float4 s_rec[NB][10];
    __shared__ uint32_t s_id[NB];
    __shared__ uint32_t s_wmask[NB];
    __shared__ uint8_t s_list[(TS * TS / 32) * NB];
    composite_tile<TS, SAVE, MODE>(blockIdx.x, s_rec, s_id, s_wmask, s_list, ids, off, grec, grec16, trec, Ng, Nt, tiles_x, tiles_per_cam, W, H, t_eps, bg0, bg1, bg2, out, out_last, out_tfin, out_ntri, stack, cap, npix, need);
}

// persistent launch: resident CTAs take tiles from an atomic queue in the
// order `order` (decreasing list length: the heaviest tiles start first)
template <int TS, bool SAVE, int MODE>
__global__ void __launch_bounds__(TS * TS) composite_persistent_kernel(
    const uint32_t* __restrict__ order, unsigned* __restrict__ work, int64_t M,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need) {
    constexpr int NB = BatchOf<TS>::value;
    __shared__ float4 s_rec[NB][10];
    __shared__ uint32_t s_id[NB];
    __shared__ uint32_t s_wmask[NB];
    __shared__ uint8_t s_list[(TS * TS / 32) * NB];
    __shared__ unsigned s_next;
    while (true) {
        if (threadIdx.x == 0) s_next = atomicAdd(work, 1u);
        __syncthreads();
        const unsigned k = s_next;
        __syncthreads();
        if ((int64_t)k >= M) break;
        composite_tile<TS, SAVE, MODE>((int)order[k], s_rec, s_id, s_wmask, s_list, ids, off, grec, grec16, trec, Ng, Nt, tiles_x, tiles_per_cam, W, H, t_eps, bg0, bg1, bg2, out, out_last, out_tfin, out_ntri, stack, cap, npix, need);
        __syncthreads();
    }
}

// tile order for the persistent launch: key = 0xffff - min(list length, 0xffff)
__global__ void tile_order_keys_kernel(const int64_t* __restrict__ off, int64_t M, uint32_t* __restrict__ k,
                                       uint32_t* __restrict__ v, uint32_t* __restrict__ m_dev) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t == 0) *m_dev = (uint32_t)M;
    if (t >= M) return;
    const int64_t c = off[t + 1] - off[t];
    k[t] = 0xffffu - (uint32_t)min(c, (int64_t)0xffff);
    v[t] = (uint32_t)t;
}

// ---------------------------------------------------------------------------
// frame inspection: split sorted keys into ids / depth bits

__global__ void lists_kernel(const uint32_t* __restrict__ tk, const uint32_t* __restrict__ tv, int64_t n, const BinInfo* __restrict__ bin, int64_t ntot, int tiles_per_cam,
                             int32_t* __restrict__ ids, uint32_t* __restrict__ dbits) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t id = tv[i];
    const int cam = (int)(tk[i] / (uint32_t)tiles_per_cam);
    ids[i] = (int32_t)id;
    dbits[i] = bin[(int64_t)cam * ntot + id].dbits;
}


cudaError_t radix_sort_pairs(umgs_frame* fr, uint32_t* k, uint32_t* v, uint32_t* k2, uint32_t* v2,
                             const uint32_t* n_dev, int64_t n_cap, int bits, uint32_t** rk, uint32_t** rv,
                             cudaStream_t s);

cudaError_t launch_composite(umgs_frame* fr, const umgs_render_opts& opts, float* out_rgbt, cudaStream_t stream) {
    const float te = opts.t_eps > 0.f ? opts.t_eps : -1.f;
    float4* out = reinterpret_cast<float4*>(out_rgbt);
    const int ts = fr->tile;
    const unsigned M = (unsigned)fr->num_tiles;
    const int tpc = fr->tiles_x * fr->tiles_y;
    const int64_t npix = (int64_t)fr->ncams * fr->W * fr->H;
    const bool save = fr->saved;
    if (save) cudaMemsetAsync(fr->status.as<int32_t>() + 2, 0, sizeof(int32_t), stream);
    const bool persist = opts.sched > 0;
    const uint32_t* order = nullptr;
    unsigned* work = nullptr;
    int nblk = 0;
    if (persist) {
        // tiles in decreasing order of list length (stable radix sort of 16-bit keys)
        cudaError_t e;
        if ((e = fr->ord_k.reserve(sizeof(uint32_t) * M)) != cudaSuccess) return e;
        if ((e = fr->ord_v.reserve(sizeof(uint32_t) * M)) != cudaSuccess) return e;
        if ((e = fr->ord_k2.reserve(sizeof(uint32_t) * M)) != cudaSuccess) return e;
        if ((e = fr->ord_v2.reserve(sizeof(uint32_t) * M)) != cudaSuccess) return e;
        uint32_t* mdev = reinterpret_cast<uint32_t*>(fr->status.as<int32_t>() + 4);
        work = reinterpret_cast<unsigned*>(fr->status.as<int32_t>() + 8);
        tile_order_keys_kernel<<<(M + 255) / 256, 256, 0, stream>>>(fr->tile_off.as<int64_t>(), M, fr->ord_k.as<uint32_t>(),
                                                                     fr->ord_v.as<uint32_t>(), mdev), count_launch();
        uint32_t* rk = nullptr;
        uint32_t* rv = nullptr;
        if ((e = radix_sort_pairs(fr, fr->ord_k.as<uint32_t>(), fr->ord_v.as<uint32_t>(), fr->ord_k2.as<uint32_t>(),
                                  fr->ord_v2.as<uint32_t>(), mdev, M, 16, &rk, &rv, stream)) != cudaSuccess)
            return e;
        order = rv;
        cudaMemsetAsync(work, 0, sizeof(unsigned), stream);
        nblk = opts.sched * fr->ctx->num_sms;
    }
#define UMGS_LAUNCH(TSV, SV, MV)                                                                                \
    if (persist) composite_persistent_kernel<TSV, SV, MV><<<nblk, TSV * TSV, 0, stream>>>(order, work, M,      \
        fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(), fr->mixed ? fr->grec.as<GRec16>() : nullptr,  \
        fr->trec.as<TRec>(), fr->ng,                                                                            \
        fr->nt, fr->tiles_x, tpc, fr->W, fr->H, te, opts.bg[0], opts.bg[1], opts.bg[2], out,                      \
        fr->last.as<int32_t>(), save ? fr->tfin.as<float>() : nullptr, save ? fr->ntri.as<int32_t>() : nullptr,   \
        save ? fr->stack.as<float4>() : nullptr, fr->stack_cap, npix, fr->status.as<int32_t>() + 2),            \
        count_launch();                                                                                         \
    else composite_kernel<TSV, SV, MV><<<M, TSV * TSV, 0, stream>>>(                                            \
        fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(), fr->mixed ? fr->grec.as<GRec16>() : nullptr,  \
        fr->trec.as<TRec>(), fr->ng,                                                                            \
        fr->nt, fr->tiles_x, tpc, fr->W, fr->H, te, opts.bg[0], opts.bg[1], opts.bg[2], out,                      \
        fr->last.as<int32_t>(), save ? fr->tfin.as<float>() : nullptr, save ? fr->ntri.as<int32_t>() : nullptr,   \
        save ? fr->stack.as<float4>() : nullptr, fr->stack_cap, npix, fr->status.as<int32_t>() + 2),            \
        count_launch()
    // the saved (backward) form exists for FULL only
#define UMGS_MODES(TSV)                                                                                         \
    if (save) { UMGS_LAUNCH(TSV, true, UMGS_BLEND_FULL); }                                                      \
    else if (mode == kModeTProduct) { UMGS_LAUNCH(TSV, false, kModeTProduct); }                                 \
    else if (mode == UMGS_BLEND_DIRECT) { UMGS_LAUNCH(TSV, false, UMGS_BLEND_DIRECT); }                         \
    else if (mode == UMGS_BLEND_MSAA_ALL) { UMGS_LAUNCH(TSV, false, UMGS_BLEND_MSAA_ALL); }                     \
    else if (mode == UMGS_BLEND_ENTITY_ALL) { UMGS_LAUNCH(TSV, false, UMGS_BLEND_ENTITY_ALL); }                 \
    else { UMGS_LAUNCH(TSV, false, UMGS_BLEND_FULL); }
    const int mode = (opts.blend_mode == UMGS_BLEND_FULL && (opts.flags & UMGS_RENDER_T_PRODUCT)) ? kModeTProduct
                                                                                                : opts.blend_mode;
    if (ts == 16) { UMGS_MODES(16) }
    else if (ts == 8) { UMGS_MODES(8) }
    else { UMGS_MODES(32) }
#undef UMGS_MODES
#undef UMGS_LAUNCH
    return cudaGetLastError();
}


// exclusive scan of n uint32 counts into out; the grand total goes to *total (device)
cudaError_t scan_u32(umgs_frame* fr, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, cudaStream_t s) {
    const int64_t nb = (n + kRsTile - 1) / kRsTile;
    cudaError_t e = fr->rs_bsum.reserve(sizeof(uint32_t) * std::max<int64_t>(1, nb));
    if (e != cudaSuccess) return e;
    if (nb > (1 << 22)) return cudaErrorInvalidValue;
    uint32_t* overflow = reinterpret_cast<uint32_t*>(fr->status.as<int32_t>() + 9);
    scan_reduce_kernel<<<(unsigned)nb, kRsThreads, 0, s>>>(in, n, fr->rs_bsum.as<uint32_t>(), overflow),
        count_launch();
    scan_blocks_kernel<<<1, 1024, 0, s>>>(fr->rs_bsum.as<uint32_t>(), (int)nb, total, overflow), count_launch();
    scan_apply_kernel<<<(unsigned)nb, kRsThreads, 0, s>>>(in, n, fr->rs_bsum.as<uint32_t>(), out), count_launch();
    return cudaGetLastError();
}

// stable LSD radix sort of (k, v) on the low `bits` bits; the element count
// is read from device memory (n_dev, at most n_cap, which sizes the grids);
// ping-pongs with (k2, v2) and returns where the result ended
cudaError_t radix_sort_pairs(umgs_frame* fr, uint32_t* k, uint32_t* v, uint32_t* k2, uint32_t* v2,
                             const uint32_t* n_dev, int64_t n_cap, int bits, uint32_t** rk, uint32_t** rv,
                             cudaStream_t s) {
    const int64_t n = n_cap;
    const int64_t nb = std::max<int64_t>(1, (n + kRsTile - 1) / kRsTile);
    const int64_t nh = 256 * nb;
    cudaError_t e = fr->rs_hist.reserve(sizeof(uint32_t) * nh);
    if (e != cudaSuccess) return e;
    e = fr->rs_hist2.reserve(sizeof(uint32_t) * 256);
    if (e != cudaSuccess) return e;
    uint32_t* hist = fr->rs_hist.as<uint32_t>();
    uint32_t* dtotal = fr->rs_hist2.as<uint32_t>();
    for (int shift = 0; shift < bits; shift += 8) {
        radix_upsweep_kernel<<<(unsigned)nb, kRsThreads, 0, s>>>(k, n_dev, n_cap, shift, (int)nb, hist), count_launch();
        radix_hist_scan_kernel<<<256, kRsThreads, 0, s>>>(hist, (int)nb, dtotal), count_launch();
        radix_downsweep_kernel<<<(unsigned)nb, kRsThreads, 0, s>>>(k, v, n_dev, n_cap, shift, (int)nb, hist, dtotal,
                                                                   k2, v2), count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint32_t* t = k; k = k2; k2 = t;
        t = v; v = v2; v2 = t;
    }
    *rk = k;
    *rv = v;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// host orchestration

static inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

umgs_status render_forward(umgs_ctx* ctx, const umgs_gaussians* g, const umgs_mesh* meshes, int32_t nmeshes,
                           const umgs_camera* cams, int32_t ncams, const umgs_render_opts& opts, float* out_rgbt,
                           umgs_frame* fr, cudaStream_t stream) {
    const int ts = opts.tile_size;
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
    // status words: [0] error bits, [1] number of (tile, id) pairs, [2] largest
    // saved-stack need, [3] fp64 conic list length, [4] tile count for the
    // tile-order sort, [5] record count for the depth sort, [6..7] evaluation
    // count (u64), [8] persistent work counter, [9] pair-count overflow
    UMGS_TRY(fr->status.reserve(sizeof(int32_t) * 16));

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
    // (inside a graph capture the cameras were uploaded by the sizing render)
    if (!fr->capture)
        UMGS_TRY(cudaMemcpyAsync(fr->cams.ptr, dc.data(), sizeof(DevCam) * ncams, cudaMemcpyHostToDevice, stream));
    UMGS_TRY(cudaMemsetAsync(fr->status.ptr, 0, sizeof(int32_t) * 16, stream));

    const DevCam* dcams = fr->cams.as<DevCam>();
    const unsigned fix_cap = (unsigned)std::min<int64_t>(std::max<int64_t>(1, Ng * ncams), 1 << 22);
    UMGS_TRY(fr->fix_list.reserve(sizeof(int64_t) * fix_cap));
    if (Ng > 0) {
        StageTimer tm(ctx, UMGS_STAGE_PROJECT_GAUSSIANS, stream);
        project_gaussians_kernel<<<grid_for(Ng, 256), 256, 0, stream>>>(
            g->means, g->quats, g->scales, g->opacities, g->sh, g->sh_dtype, g->sh_degree, g->cov3d, Ng, dcams,
            ncams, ts, tiles_x, tiles_per_cam, fr->grec.as<GRec>(), mixed ? fr->grec.as<GRec16>() : nullptr,
            fr->bin.as<BinInfo>(), Ntot, reinterpret_cast<unsigned*>(fr->status.as<int32_t>() + 3),
            fr->fix_list.as<int64_t>(), fix_cap), count_launch();
        UMGS_TRY(cudaGetLastError());
        refine_conics_kernel<<<4 * ctx->num_sms, 128, 0, stream>>>(
            g->means, g->quats, g->scales, g->cov3d, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot,
            reinterpret_cast<unsigned*>(fr->status.as<int32_t>() + 3), fr->fix_list.as<int64_t>(), fix_cap,
            fr->grec.as<GRec>(), mixed ? fr->grec.as<GRec16>() : nullptr), count_launch();
        UMGS_TRY(cudaGetLastError());
    }
    if (Ng > 0) {
        StageTimer tm(ctx, UMGS_STAGE_SHADE_GAUSSIANS, stream);
        const unsigned gb = grid_for(Ng, 256);
        GRec16* g16 = mixed ? fr->grec.as<GRec16>() : nullptr;
        switch (g->sh_degree) {
            case 0: shade_gaussians_kernel<0><<<gb, 256, 0, stream>>>(g->means, g->sh, g->sh_dtype, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot, fr->grec.as<GRec>(), g16), count_launch(); break;
            case 1: shade_gaussians_kernel<1><<<gb, 256, 0, stream>>>(g->means, g->sh, g->sh_dtype, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot, fr->grec.as<GRec>(), g16), count_launch(); break;
            case 2: shade_gaussians_kernel<2><<<gb, 256, 0, stream>>>(g->means, g->sh, g->sh_dtype, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot, fr->grec.as<GRec>(), g16), count_launch(); break;
            default: shade_gaussians_kernel<3><<<gb, 256, 0, stream>>>(g->means, g->sh, g->sh_dtype, Ng, dcams, ncams, fr->bin.as<BinInfo>(), Ntot, fr->grec.as<GRec>(), g16), count_launch(); break;
        }
        UMGS_TRY(cudaGetLastError());
    }
    int64_t tri_base = 0;
    for (int m = 0; m < nmeshes; ++m) {
        const umgs_mesh& me = meshes[m];
        if (me.nf > 0) {
            StageTimer tm(ctx, UMGS_STAGE_SETUP_TRIANGLES, stream);
            setup_triangles_kernel<<<grid_for(me.nf, 256), 256, 0, stream>>>(
                me.verts, me.faces, me.vcolor, me.valpha, me.falpha, me.nv, me.nf, tri_base, Nt, Ng + tri_base,
                dcams, ncams, ts, tiles_x, tiles_per_cam, fr->trec.as<TRec>(), fr->bin.as<BinInfo>(), Ntot,
                fr->status.as<int32_t>()), count_launch();
            UMGS_TRY(cudaGetLastError());
        }
        tri_base += me.nf;
    }
    // ---- binning: depth sort of all records, pair emission, stable tile sort
    const int64_t NR = Ntot * ncams;  // (camera, primitive) records
    UMGS_TRY(fr->pk.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    UMGS_TRY(fr->pv.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    UMGS_TRY(fr->pk2.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    UMGS_TRY(fr->pv2.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    UMGS_TRY(fr->pcnt.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    UMGS_TRY(fr->poff.reserve(sizeof(uint32_t) * std::max<int64_t>(1, NR)));
    uint32_t* pk = fr->pk.as<uint32_t>();
    uint32_t* pv = fr->pv.as<uint32_t>();
    uint32_t* status_u = reinterpret_cast<uint32_t*>(fr->status.as<int32_t>());
    if (NR > 0) {
        StageTimer tm(ctx, UMGS_STAGE_SCAN, stream);
        prim_keys_kernel<<<grid_for(NR, 256), 256, 0, stream>>>(fr->bin.as<BinInfo>(), NR, pk, pv, status_u + 5), count_launch();
        UMGS_TRY(cudaGetLastError());
        uint32_t* rk = nullptr;
        uint32_t* rv = nullptr;
        UMGS_TRY(radix_sort_pairs(fr, pk, pv, fr->pk2.as<uint32_t>(), fr->pv2.as<uint32_t>(), status_u + 5, NR, 32, &rk,
                                  &rv, stream));
        pk = rk;
        pv = rv;
        tile_counts_kernel<<<grid_for(NR, 256), 256, 0, stream>>>(fr->bin.as<BinInfo>(), pv, NR, ts,
                                                                  fr->pcnt.as<uint32_t>()), count_launch();
        UMGS_TRY(scan_u32(fr, fr->pcnt.as<uint32_t>(), fr->poff.as<uint32_t>(), NR, status_u + 1, stream));
    }
    int64_t Kcap;
    if (!fr->nosync) {
        // read back the number of pairs (and the status word)
        UMGS_TRY(cudaMemcpyAsync(ctx->pinned, fr->status.ptr, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
        UMGS_TRY(cudaStreamSynchronize(stream));
        const int32_t st = (int32_t)(ctx->pinned[0] & 0xffffffff);
        const int64_t K = NR > 0 ? (int64_t)(uint32_t)(ctx->pinned[0] >> 32) : 0;
        if (st & 1) return fail(ctx, UMGS_ERR_INVALID_ARG, "a face index is out of range");
        if (K == 0xffffffffll) return fail(ctx, UMGS_ERR_CAPACITY, "more than 4294967294 (tile, primitive) pairs");
        fr->num_keys = K;
        Kcap = K;
        UMGS_TRY(fr->tk.reserve(sizeof(uint32_t) * std::max<int64_t>(1, K)));
        UMGS_TRY(fr->tv.reserve(sizeof(uint32_t) * std::max<int64_t>(1, K)));
        UMGS_TRY(fr->tk2.reserve(sizeof(uint32_t) * std::max<int64_t>(1, K)));
        UMGS_TRY(fr->tv2.reserve(sizeof(uint32_t) * std::max<int64_t>(1, K)));
    } else {
        // no host read-back: the pairs are held to the reserved capacity and an
        // overflow is flagged in the status word (bit 2); inside a capture the
        // buffers were sized beforehand
        Kcap = fr->key_capacity;
        fr->num_keys = -1;
        if (!fr->capture) {
            UMGS_TRY(fr->tk.reserve(sizeof(uint32_t) * std::max<int64_t>(1, Kcap)));
            UMGS_TRY(fr->tv.reserve(sizeof(uint32_t) * std::max<int64_t>(1, Kcap)));
            UMGS_TRY(fr->tk2.reserve(sizeof(uint32_t) * std::max<int64_t>(1, Kcap)));
            UMGS_TRY(fr->tv2.reserve(sizeof(uint32_t) * std::max<int64_t>(1, Kcap)));
        }
    }
    fr->ids = fr->tv.as<uint32_t>();
    fr->tkeys = fr->tk.as<uint32_t>();
    if (NR > 0) {
        StageTimer tm(ctx, UMGS_STAGE_SCATTER, stream);
emit_pairs_kernel<<<grid_for(NR, 256), 256, 0, stream>>>(fr->bin.as<BinInfo>(), pv, fr->poff.as<uint32_t>(), NR,
                                                                 Ntot, ts, tiles_x, tiles_per_cam, fr->tk.as<uint32_t>(),
                                                                 fr->tv.as<uint32_t>(), Kcap, fr->status.as<int32_t>()),
            count_launch();
        UMGS_TRY(cudaGetLastError());
    }
    {
        StageTimer tm(ctx, UMGS_STAGE_SORT, stream);
        if (Kcap > 0) {
            int bits = 1;
            while (((int64_t)1 << bits) < M) ++bits;
            uint32_t* rk = nullptr;
            uint32_t* rv = nullptr;
            UMGS_TRY(radix_sort_pairs(fr, fr->tk.as<uint32_t>(), fr->tv.as<uint32_t>(), fr->tk2.as<uint32_t>(),
                                      fr->tv2.as<uint32_t>(), status_u + 1, Kcap, bits, &rk, &rv, stream));
            fr->tkeys = rk;
            fr->ids = rv;
        }
        tile_ranges_kernel<<<grid_for(M + 1, 256), 256, 0, stream>>>(fr->tkeys, status_u + 1, Kcap, M,
                                                                     fr->tile_off.as<int64_t>()), count_launch();
        UMGS_TRY(cudaGetLastError());
    }
    UMGS_TRY(fr->last.reserve(sizeof(int32_t) * (int64_t)ncams * W * H));
    fr->saved = (opts.flags & UMGS_RENDER_SAVE_BACKWARD) != 0 && opts.blend_mode == UMGS_BLEND_FULL;
    if (fr->saved) {
        const int64_t npix = (int64_t)ncams * W * H;
        UMGS_TRY(fr->tfin.reserve(sizeof(float) * npix));
        UMGS_TRY(fr->ntri.reserve(sizeof(int32_t) * npix));
        UMGS_TRY(fr->stack.reserve(sizeof(float4) * npix * fr->stack_cap));
    }
    {
        StageTimer tm_comp(ctx, UMGS_STAGE_COMPOSITE, stream);
        UMGS_TRY(launch_composite(fr, opts, out_rgbt, stream));
    }
    fr->valid = true;
#undef UMGS_TRY
    return UMGS_OK;
}

// N_alg of the last render (diagnostic, not part of the render): per pixel
// the entries of its tile list whose pixel rect holds the pixel, up to and
// including list position `last` when the pixel stopped at T < t_eps (bit 31
// of the compositor's `last`), else all of them.  One CTA per tile, one
// thread per pixel, summed into *count.
template <int TS>
__global__ void __launch_bounds__(TS * TS) eval_count_kernel(
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, const int32_t* __restrict__ last, unsigned long long* __restrict__ count) {
    const int tile = blockIdx.x;
    const int cam = tile / tiles_per_cam;
    const int lt = tile - cam * tiles_per_cam;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    int lx, ly;
    block_pixel<TS>(threadIdx.x, lx, ly);
    const int px = tx * TS + lx, py = ty * TS + ly;
    unsigned long long c = 0;
    if (px < W && py < H) {
        const int64_t beg = off[tile], end = off[tile + 1];
        const int32_t l = last[((int64_t)cam * H + py) * W + px];
        const int64_t lim = (l < 0) ? (int64_t)(l & 0x7fffffff) : end - beg;
        for (int64_t p = 0; p < lim; ++p) {
            const uint32_t id = ids[beg + p];
            uint32_t rx, ry;
            if (id >= Ng + Nt) continue;
            if (id < Ng) {
                if (grec16) {
                    const uint4 h1 = grec16[(int64_t)cam * Ng + id].v1;
                    rx = h1.z; ry = h1.w;
                } else {
                    const float4 c2 = reinterpret_cast<const float4*>(grec + (int64_t)cam * Ng + id)[2];
                    rx = __float_as_uint(c2.y); ry = __float_as_uint(c2.z);
                }
            } else {
                const TRec& t = trec[(int64_t)cam * Nt + (id - Ng)];
                rx = t.rx; ry = t.ry;
            }
            c += (px >= (int)(rx & 0xffff) && px <= (int)(rx >> 16) && py >= (int)(ry & 0xffff) &&
                  py <= (int)(ry >> 16)) ? 1ull : 0ull;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

umgs_status frame_evaluations(const umgs_frame* fr, int64_t* evals, cudaStream_t stream) {
    cudaError_t e;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(fr->status.as<int32_t>() + 6);
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), stream)) != cudaSuccess)
        return cuda_fail(fr->ctx, e, "cudaMemsetAsync");
    const int tpc = fr->tiles_x * fr->tiles_y;
    const unsigned M = (unsigned)fr->num_tiles;
    if (M > 0) {
#define UMGS_LAUNCH(TSV)                                                                                        \
        eval_count_kernel<TSV><<<M, TSV * TSV, 0, stream>>>(fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(), \
            fr->mixed ? fr->grec.as<GRec16>() : nullptr, fr->trec.as<TRec>(), fr->ng, fr->nt, fr->tiles_x, tpc,   \
            fr->W, fr->H, fr->last.as<int32_t>(), cnt), count_launch()
        if (fr->tile == 16) UMGS_LAUNCH(16);
        else if (fr->tile == 8) UMGS_LAUNCH(8);
        else UMGS_LAUNCH(32);
#undef UMGS_LAUNCH
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(fr->ctx, e, "eval_count_kernel");
    }
    unsigned long long v = 0;
    if ((e = cudaMemcpyAsync(fr->ctx->pinned, cnt, sizeof(v), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return cuda_fail(fr->ctx, e, "reading the evaluation count");
    std::memcpy(&v, fr->ctx->pinned, sizeof(v));
    *evals = (int64_t)v;
    return UMGS_OK;
}

umgs_status frame_check(umgs_frame* fr, cudaStream_t stream) {
    int32_t* w = reinterpret_cast<int32_t*>(fr->ctx->pinned);
    cudaError_t e = cudaMemcpyAsync(w, fr->status.ptr, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(fr->ctx, e, "reading the frame status");
    if (w[0] & 1) return fail(fr->ctx, UMGS_ERR_INVALID_ARG, "a face index is out of range");
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
        lists_kernel<<<grid_for(fr->num_keys, 256), 256, 0, stream>>>(
            fr->tkeys, fr->ids, fr->num_keys, fr->bin.as<BinInfo>(), fr->ng + fr->nt, fr->tiles_x * fr->tiles_y, ids,
            dbits), count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(fr->ctx, e, "lists_kernel");
    }
    return UMGS_OK;
}

}  // namespace umgs
