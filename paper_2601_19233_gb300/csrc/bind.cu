// Gaussian-centric binding of Gaussians to a proxy mesh (Sec. 3.3).
//
// From every camera a ray is cast towards each target (the Gaussian mean in
// CENTER mode, the 8 corners of its 3-sigma box in BBX mode); the ray is the
// half-line o + t (p - o), t > 0, and every hit counts.  The target is bound
// to the hit nearest to it (distance |t - 1| |p - o|; ties: lower camera,
// then lower face).  Targets no ray hits fall back to the closest point on
// the mesh; NEAREST mode uses the closest point for every target.
//
// The paper casts these rays with OptiX; here a uniform grid over the proxy
// replaces the BVH:
//   grid_stats   proxy AABB and mean edge length (one CTA)
//   grid_count / grid_fill   each face goes into every cell its AABB,
//                expanded by delta = 1e-3 cell, overlaps; cell entries carry
//                the face's three vertices (48 B) so a cell is one
//                contiguous run
//   bind_raycast one thread per target, looping over cameras; from the
//                target the ray is walked through the grid in both
//                directions (3D-DDA, boundary parameters recomputed from
//                cell indices at every step so no error accumulates) and a
//                walk stops once the cell entry distance exceeds the best
//                distance found so far
//   bind_nearest one thread per unbound target; Chebyshev rings of cells
//                around the target until no closer cell can exist
// Every ray/triangle test and every closest-point evaluation is the same
// sequence of IEEE float32 operations as the brute-force definition, so the
// chosen faces, barycentrics and distances are bit-exact; the grid only
// decides which faces get tested, and its margins keep that a superset of
// the faces that can win.
#include <cmath>
#include <vector>

#include "internal.h"

namespace umgs {

struct GridInfo {
    float org[3];
    float h;
    int dims[3];
    int ncells;
    float delta;  // registration margin
};

__global__ void grid_stats_kernel(const float* __restrict__ V, const int32_t* __restrict__ F, int64_t nv, int64_t nf,
                                  float* __restrict__ out /* min3 max3 edge_sum count */, int32_t* __restrict__ status) {
    __shared__ float smin[3][32], smax[3][32];
    __shared__ double ssum[32];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    double esum = 0.0;
    for (int64_t f = threadIdx.x; f < nf; f += blockDim.x) {
        const int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
        if (a < 0 || a >= nv || b < 0 || b >= nv || c < 0 || c >= nv) { atomicOr(status, 2); continue; }
        float P[3][3];
        for (int k = 0; k < 3; ++k) {
            const int v = k == 0 ? a : (k == 1 ? b : c);
            for (int d = 0; d < 3; ++d) {
                P[k][d] = V[3 * (int64_t)v + d];
                mn[d] = fminf(mn[d], P[k][d]);
                mx[d] = fmaxf(mx[d], P[k][d]);
            }
        }
        for (int k = 0; k < 3; ++k) {
            const int l = (k + 1) % 3;
            const float dx = P[k][0] - P[l][0], dy = P[k][1] - P[l][1], dz = P[k][2] - P[l][2];
            esum += sqrt((double)(dx * dx + dy * dy + dz * dz));
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        for (int d = 0; d < 3; ++d) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
        esum += __shfl_xor_sync(0xffffffffu, esum, o);
    }
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) { smin[d][w] = mn[d]; smax[d][w] = mx[d]; }
        ssum[w] = esum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x / 32;
        double s = 0;
        for (int d = 0; d < 3; ++d) {
            float a = INFINITY, b = -INFINITY;
            for (int k = 0; k < nw; ++k) { a = fminf(a, smin[d][k]); b = fmaxf(b, smax[d][k]); }
            out[d] = a;
            out[3 + d] = b;
        }
        for (int k = 0; k < nw; ++k) s += ssum[k];
        out[6] = (float)(s / (3.0 * (double)nf));
    }
}

__device__ __forceinline__ int cell_of(float x, float org, float h, int n) {
    int c = (int)floorf((x - org) / h);
    return min(max(c, 0), n - 1);
}

__global__ void grid_count_kernel(const float* __restrict__ V, const int32_t* __restrict__ F, int64_t nf, GridInfo gi,
                                  int32_t* __restrict__ cnt, float* __restrict__ fv_unused) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    float mn[3], mx[3];
    for (int d = 0; d < 3; ++d) { mn[d] = INFINITY; mx[d] = -INFINITY; }
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) {
            const float x = V[3 * (int64_t)F[3 * f + k] + d];
            mn[d] = fminf(mn[d], x); mx[d] = fmaxf(mx[d], x);
        }
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = cell_of(mn[d] - gi.delta, gi.org[d], gi.h, gi.dims[d]);
        hi[d] = cell_of(mx[d] + gi.delta, gi.org[d], gi.h, gi.dims[d]);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) atomicAdd(&cnt[(z * gi.dims[1] + y) * gi.dims[0] + x], 1);
}

__global__ void grid_fill_kernel(const float* __restrict__ V, const int32_t* __restrict__ F, int64_t nf, GridInfo gi,
                                 const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                                 float4* __restrict__ entries) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    float P[3][3], mn[3], mx[3];
    for (int d = 0; d < 3; ++d) { mn[d] = INFINITY; mx[d] = -INFINITY; }
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) {
            P[k][d] = V[3 * (int64_t)F[3 * f + k] + d];
            mn[d] = fminf(mn[d], P[k][d]); mx[d] = fmaxf(mx[d], P[k][d]);
        }
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = cell_of(mn[d] - gi.delta, gi.org[d], gi.h, gi.dims[d]);
        hi[d] = cell_of(mx[d] + gi.delta, gi.org[d], gi.h, gi.dims[d]);
    }
    const float4 e0 = make_float4(P[0][0], P[0][1], P[0][2], __int_as_float((int)f));
    const float4 e1 = make_float4(P[1][0], P[1][1], P[1][2], 0.f);
    const float4 e2 = make_float4(P[2][0], P[2][1], P[2][2], 0.f);
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                const int c = (z * gi.dims[1] + y) * gi.dims[0] + x;
                const int slot = start[c] + atomicAdd(&fill[c], 1);
                entries[3 * (int64_t)slot] = e0;
                entries[3 * (int64_t)slot + 1] = e1;
                entries[3 * (int64_t)slot + 2] = e2;
            }
}

__global__ void __launch_bounds__(1024) grid_scan_kernel(const int32_t* __restrict__ cnt, int n,
                                                         int32_t* __restrict__ start) {
    __shared__ int warp_sums[32];
    const int tid = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int b = min(tid * per, n), e = min(b + per, n);
    int local = 0;
    for (int k = b; k < e; ++k) local += cnt[k];
    int x = local;
    const int lane = tid & 31, warp = tid >> 5;
    for (int d = 1; d < 32; d <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
        for (int d = 1; d < 32; d <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    int run = x - local + (warp > 0 ? warp_sums[warp - 1] : 0);
    for (int k = b; k < e; ++k) { start[k] = run; run += cnt[k]; }
    if (tid == 1023) start[n] = warp_sums[31];
}

// ---- canonical target and primitive tests ---------------------------------

__device__ void bind_target(const float* __restrict__ means, const float* __restrict__ quats,
                            const float* __restrict__ scales, int64_t i, int corner, int mode, float k_sigma,
                            float p[3]) {
    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
    if (mode != UMGS_BIND_BBX) { p[0] = mx; p[1] = my; p[2] = mz; return; }
    const float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
    const float n = fsq(fa(fa(fa(fm(qw, qw), fm(qx, qx)), fm(qy, qy)), fm(qz, qz)));
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
    float off[3];
    for (int j = 0; j < 3; ++j) {
        const float ks = fm(k_sigma, scales[3 * i + j]);
        off[j] = ((corner >> j) & 1) ? ks : -ks;
    }
    p[0] = fa(mx, dot3c(r[0], r[1], r[2], off[0], off[1], off[2]));
    p[1] = fa(my, dot3c(r[3], r[4], r[5], off[0], off[1], off[2]));
    p[2] = fa(mz, dot3c(r[6], r[7], r[8], off[0], off[1], off[2]));
}

__device__ __forceinline__ void crossc(float a0, float a1, float a2, float b0, float b1, float b2, float& c0,
                                       float& c1, float& c2) {
    c0 = fs(fm(a1, b2), fm(a2, b1));
    c1 = fs(fm(a2, b0), fm(a0, b2));
    c2 = fs(fm(a0, b1), fm(a1, b0));
}

// Moller-Trumbore in canonical float32; returns true on a hit with u, v, t
__device__ __forceinline__ bool ray_tri(const float o[3], const float d[3], float4 A, float4 B, float4 C, float& u,
                                        float& v, float& t) {
    const float e1x = fs(B.x, A.x), e1y = fs(B.y, A.y), e1z = fs(B.z, A.z);
    const float e2x = fs(C.x, A.x), e2y = fs(C.y, A.y), e2z = fs(C.z, A.z);
    float px, py, pz;
    crossc(d[0], d[1], d[2], e2x, e2y, e2z, px, py, pz);
    const float det = dot3c(e1x, e1y, e1z, px, py, pz);
    const float tx = fs(o[0], A.x), ty = fs(o[1], A.y), tz = fs(o[2], A.z);
    const float un = dot3c(tx, ty, tz, px, py, pz);
    float qx, qy, qz;
    crossc(tx, ty, tz, e1x, e1y, e1z, qx, qy, qz);
    const float vn = dot3c(d[0], d[1], d[2], qx, qy, qz);
    const float tn = dot3c(e2x, e2y, e2z, qx, qy, qz);
    u = fdv(un, det);
    v = fdv(vn, det);
    t = fdv(tn, det);
    return det != 0.f && u >= 0.f && v >= 0.f && fa(u, v) <= 1.f && t > 0.f && isfinite(t);
}

// closest point on a triangle (region method), canonical float32
__device__ __forceinline__ void closest_tri(const float p[3], float4 A, float4 B, float4 C, float& b1, float& b2,
                                            float& d2) {
    const float abx = fs(B.x, A.x), aby = fs(B.y, A.y), abz = fs(B.z, A.z);
    const float acx = fs(C.x, A.x), acy = fs(C.y, A.y), acz = fs(C.z, A.z);
    const float apx = fs(p[0], A.x), apy = fs(p[1], A.y), apz = fs(p[2], A.z);
    const float d1 = dot3c(abx, aby, abz, apx, apy, apz), d2_ = dot3c(acx, acy, acz, apx, apy, apz);
    const float bpx = fs(p[0], B.x), bpy = fs(p[1], B.y), bpz = fs(p[2], B.z);
    const float d3 = dot3c(abx, aby, abz, bpx, bpy, bpz), d4 = dot3c(acx, acy, acz, bpx, bpy, bpz);
    const float cpx = fs(p[0], C.x), cpy = fs(p[1], C.y), cpz = fs(p[2], C.z);
    const float d5 = dot3c(abx, aby, abz, cpx, cpy, cpz), d6 = dot3c(acx, acy, acz, cpx, cpy, cpz);
    const float vc = fs(fm(d1, d4), fm(d3, d2_));
    const float vb = fs(fm(d5, d2_), fm(d1, d6));
    const float va = fs(fm(d3, d6), fm(d5, d4));
    const float n6 = fs(d4, d3), m6 = fs(d5, d6);
    if (d1 <= 0.f && d2_ <= 0.f) { b1 = 0.f; b2 = 0.f; }
    else if (d3 >= 0.f && d4 <= d3) { b1 = 1.f; b2 = 0.f; }
    else if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) { b1 = fdv(d1, fs(d1, d3)); b2 = 0.f; }
    else if (d6 >= 0.f && d5 <= d6) { b1 = 0.f; b2 = 1.f; }
    else if (vb <= 0.f && d2_ >= 0.f && d6 <= 0.f) { b1 = 0.f; b2 = fdv(d2_, fs(d2_, d6)); }
    else if (va <= 0.f && n6 >= 0.f && m6 >= 0.f) { const float r6 = fdv(n6, fa(n6, m6)); b1 = fs(1.f, r6); b2 = r6; }
    else { const float den = fa(fa(va, vb), vc); b1 = fdv(vb, den); b2 = fdv(vc, den); }
    const float qx = fa(A.x, fa(fm(abx, b1), fm(acx, b2)));
    const float qy = fa(A.y, fa(fm(aby, b1), fm(acy, b2)));
    const float qz = fa(A.z, fa(fm(abz, b1), fm(acz, b2)));
    const float dx = fs(p[0], qx), dy = fs(p[1], qy), dz = fs(p[2], qz);
    d2 = dot3c(dx, dy, dz, dx, dy, dz);
}

struct Best {
    float dist;
    int cam, face;
    float u, v;
    __device__ __forceinline__ bool better(float d, int c, int f) const {
        if (face < 0) return true;
        if (d != dist) return d < dist;
        if (c != cam) return c < cam;
        return f < face;
    }
};

// walk one direction of the ray from the target; tau = |t - 1|
__device__ void walk(const GridInfo& gi, const int32_t* __restrict__ start, const float4* __restrict__ ent,
                     const float o[3], const float d[3], const float p[3], float dn, float sgn, int cam, Best& best,
                     int& budget) {
    const float dir[3] = {sgn * d[0], sgn * d[1], sgn * d[2]};
    // parameter range inside the grid box: p + tau*dir, tau in [tlo, thi]
    float tlo = 0.f, thi = (sgn < 0.f) ? 1.f : INFINITY;  // backward walk stops at the camera (t = 0)
    for (int a = 0; a < 3; ++a) {
        const float lo = gi.org[a], hi = gi.org[a] + gi.h * gi.dims[a];
        if (dir[a] == 0.f) {
            if (p[a] < lo || p[a] > hi) return;
        } else {
            float t0 = (lo - p[a]) / dir[a], t1 = (hi - p[a]) / dir[a];
            if (t0 > t1) { const float t = t0; t0 = t1; t1 = t; }
            tlo = fmaxf(tlo, t0);
            thi = fminf(thi, t1);
        }
    }
    if (tlo > thi) return;
    float tau = tlo;
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = cell_of(p[a] + tau * dir[a], gi.org[a], gi.h, gi.dims[a]);
    const float slack = 1e-5f;
    while (true) {
        if (best.face >= 0 && tau * dn > best.dist * (1.f + slack) + gi.delta) return;
        if (--budget < 0) return;
        // faces of this cell
        const int cid = (c[2] * gi.dims[1] + c[1]) * gi.dims[0] + c[0];
        for (int k = start[cid]; k < start[cid + 1]; ++k) {
            const float4 A = ent[3 * (int64_t)k], B = ent[3 * (int64_t)k + 1], C = ent[3 * (int64_t)k + 2];
            float u, v, t;
            if (ray_tri(o, d, A, B, C, u, v, t)) {
                const float dist = fm(fabsf(fs(t, 1.f)), dn);
                const int f = __float_as_int(A.w);
                if (best.better(dist, cam, f)) { best.dist = dist; best.cam = cam; best.face = f; best.u = u; best.v = v; }
            }
        }
        // next cell: smallest boundary parameter, recomputed from the indices
        float tn = INFINITY;
        int ax = -1;
        for (int a = 0; a < 3; ++a) {
            if (dir[a] == 0.f) continue;
            const int nb = c[a] + (dir[a] > 0.f ? 1 : 0);
            const float tb = (gi.org[a] + gi.h * nb - p[a]) / dir[a];
            if (tb < tn) { tn = tb; ax = a; }
        }
        if (ax < 0 || tn > thi) return;
        tau = fmaxf(tau, tn);
        c[ax] += dir[ax] > 0.f ? 1 : -1;
        if (c[ax] < 0 || c[ax] >= gi.dims[ax]) return;
    }
}

__global__ void __launch_bounds__(128) bind_raycast_kernel(
    const float* __restrict__ means, const float* __restrict__ quats, const float* __restrict__ scales, int64_t n,
    int mode, float k_sigma, const DevCam* __restrict__ cams, int ncams, GridInfo gi, const int32_t* __restrict__ start,
    const float4* __restrict__ ent, int32_t* __restrict__ out_face, float* __restrict__ out_bary,
    float* __restrict__ out_dist, uint8_t* __restrict__ out_flags, int32_t* __restrict__ status) {
    const int per = (mode == UMGS_BIND_BBX) ? 8 : 1;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= n * per) return;
    const int64_t i = tid / per;
    const int corner = (int)(tid - i * per);
    float p[3];
    bind_target(means, quats, scales, i, corner, mode, k_sigma, p);
    Best best;
    best.face = -1; best.dist = 0.f; best.cam = 0; best.u = 0.f; best.v = 0.f;
    int budget = 1 << 22;  // cell visits; bounds the work of any single target
    for (int c = 0; c < ncams; ++c) {
        const float* R = cams[c].R;
        const float* t = cams[c].t;
        float o[3];
        for (int a = 0; a < 3; ++a) o[a] = -dot3c(R[a], R[3 + a], R[6 + a], t[0], t[1], t[2]);
        const float d[3] = {fs(p[0], o[0]), fs(p[1], o[1]), fs(p[2], o[2])};
        const float dn = fsq(dot3c(d[0], d[1], d[2], d[0], d[1], d[2]));
        if (!(dn > 0.f)) continue;
        walk(gi, start, ent, o, d, p, dn, 1.f, c, best, budget);
        walk(gi, start, ent, o, d, p, dn, -1.f, c, best, budget);
    }
    if (budget < 0) atomicOr(status, 4);
    const int reps = (mode == UMGS_BIND_BBX) ? 1 : 8;
    for (int r = 0; r < reps; ++r) {
        const int64_t slot = i * 8 + corner + r;
        if (best.face >= 0) {
            out_face[slot] = best.face;
            out_bary[2 * slot] = best.u;
            out_bary[2 * slot + 1] = best.v;
            out_dist[slot] = best.dist;
            out_flags[slot] = 1;
        } else {
            out_face[slot] = -1;
            out_flags[slot] = 0;
        }
    }
}

__global__ void __launch_bounds__(128) bind_nearest_kernel(
    const float* __restrict__ means, const float* __restrict__ quats, const float* __restrict__ scales, int64_t n,
    int mode, float k_sigma, GridInfo gi, const int32_t* __restrict__ start, const float4* __restrict__ ent,
    int32_t* __restrict__ out_face, float* __restrict__ out_bary, float* __restrict__ out_dist,
    uint8_t* __restrict__ out_flags, unsigned long long* __restrict__ nfallback) {
    const int per = (mode == UMGS_BIND_BBX) ? 8 : 1;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= n * per) return;
    const int64_t i = tid / per;
    const int corner = (int)(tid - i * per);
    const int64_t slot0 = i * 8 + corner;
    if (mode != UMGS_BIND_NEAREST && out_flags[slot0] == 1) return;
    float p[3];
    bind_target(means, quats, scales, i, corner, mode == UMGS_BIND_NEAREST ? UMGS_BIND_CENTER : mode, k_sigma, p);
    int c0[3];
    for (int a = 0; a < 3; ++a) c0[a] = cell_of(p[a], gi.org[a], gi.h, gi.dims[a]);
    const int rmax = max(gi.dims[0], max(gi.dims[1], gi.dims[2]));
    float bd2 = 0.f, bu = 0.f, bv = 0.f;
    int bf = -1;
    for (int r = 0; r <= rmax; ++r) {
        if (bf >= 0) {
            const float lb = (r - 1) * gi.h - gi.delta;
            if (lb > 0.f && lb * lb > bd2 * (1.f + 1e-5f)) break;
        }
        for (int z = c0[2] - r; z <= c0[2] + r; ++z) {
            if (z < 0 || z >= gi.dims[2]) continue;
            for (int y = c0[1] - r; y <= c0[1] + r; ++y) {
                if (y < 0 || y >= gi.dims[1]) continue;
                const bool edge_zy = (z == c0[2] - r || z == c0[2] + r || y == c0[1] - r || y == c0[1] + r);
                for (int x = c0[0] - r; x <= c0[0] + r; x += (edge_zy || r == 0) ? 1 : 2 * r) {
                    if (x < 0 || x >= gi.dims[0]) continue;
                    const int cid = (z * gi.dims[1] + y) * gi.dims[0] + x;
                    for (int k = start[cid]; k < start[cid + 1]; ++k) {
                        const float4 A = ent[3 * (int64_t)k], B = ent[3 * (int64_t)k + 1], C = ent[3 * (int64_t)k + 2];
                        float b1, b2, d2;
                        closest_tri(p, A, B, C, b1, b2, d2);
                        const int f = __float_as_int(A.w);
                        if (bf < 0 ? (d2 == d2) : (d2 < bd2 || (d2 == bd2 && f < bf))) {
                            bd2 = d2; bf = f; bu = b1; bv = b2;
                        }
                    }
                }
            }
        }
    }
    const int reps = (mode == UMGS_BIND_BBX) ? 1 : 8;
    for (int r = 0; r < reps; ++r) {
        const int64_t slot = slot0 + r;
        out_face[slot] = bf;
        out_bary[2 * slot] = bu;
        out_bary[2 * slot + 1] = bv;
        out_dist[slot] = fsq(bd2);
        out_flags[slot] = 2;
    }
    atomicAdd(nfallback, (unsigned long long)reps);
}

static inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

umgs_status bind_forward(umgs_ctx* ctx, const umgs_gaussians* g, const float* V, const int32_t* F, int64_t nv,
                         int64_t nf, const umgs_camera* cams, int32_t ncams, int32_t mode, float k_sigma,
                         int32_t* out_face, float* out_bary, float* out_dist, uint8_t* out_flags,
                         int64_t* out_num_fallback, cudaStream_t stream) {
    cudaError_t e;
#define UMGS_TRY(x)                                                                  \
    do {                                                                             \
        e = (x);                                                                     \
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, #x); } \
        if (e != cudaSuccess) return cuda_fail(ctx, e, #x);                         \
    } while (0)
    // workspace layout inside ctx->bind_ws is rebuilt per call
    DevBuf& ws = ctx->bind_ws;
    UMGS_TRY(ws.reserve(256));
    float* stats = ws.as<float>();
    UMGS_TRY(cudaMemsetAsync(ctx->dstatus.ptr, 0, sizeof(int32_t), stream));
    {
        StageTimer tm(ctx, UMGS_STAGE_BIND_GRID, stream);
        grid_stats_kernel<<<1, 1024, 0, stream>>>(V, F, nv, nf, stats, ctx->dstatus.as<int32_t>()), count_launch();
        UMGS_TRY(cudaGetLastError());
    }
    float hs[8];
    UMGS_TRY(cudaMemcpyAsync(hs, stats, sizeof(float) * 7, cudaMemcpyDeviceToHost, stream));
    int32_t st0 = 0;
    UMGS_TRY(cudaMemcpyAsync(&st0, ctx->dstatus.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    UMGS_TRY(cudaStreamSynchronize(stream));
    if (st0 & 2) return fail(ctx, UMGS_ERR_INVALID_ARG, "a proxy face index is out of range");
    GridInfo gi;
    float ext = 0.f;
    for (int d = 0; d < 3; ++d) ext = fmaxf(ext, hs[3 + d] - hs[d]);
    float h = 2.f * hs[6];
    if (!(h > 0.f)) h = fmaxf(ext, 1e-6f);
    long long cells;
    while (true) {
        cells = 1;
        for (int d = 0; d < 3; ++d) {
            const float pad = 1e-3f * h;
            gi.org[d] = hs[d] - pad;
            gi.dims[d] = std::max(1, std::min(1024, (int)ceilf((hs[3 + d] - hs[d] + 2 * pad) / h)));
            cells *= gi.dims[d];
        }
        if (cells <= (1LL << 24)) break;
        h *= 1.5f;
    }
    gi.h = h;
    gi.ncells = (int)cells;
    gi.delta = 1e-3f * h;
    // workspace: counts, fill, start, entries
    const size_t off_cnt = 256, off_fill = off_cnt + sizeof(int32_t) * (cells + 1);
    const size_t off_start = off_fill + sizeof(int32_t) * (cells + 1);
    const size_t off_ent0 = ((off_start + sizeof(int32_t) * (cells + 1) + 255) / 256) * 256;
    UMGS_TRY(ws.reserve(off_ent0));
    int32_t* cnt = reinterpret_cast<int32_t*>(ws.as<char>() + off_cnt);
    int32_t* fill = reinterpret_cast<int32_t*>(ws.as<char>() + off_fill);
    int32_t* start = reinterpret_cast<int32_t*>(ws.as<char>() + off_start);
    UMGS_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (cells + 1) * 2, stream));
    int32_t nent = 0;
    {
        StageTimer tm(ctx, UMGS_STAGE_BIND_GRID, stream);
        grid_count_kernel<<<grid_for(nf, 256), 256, 0, stream>>>(V, F, nf, gi, cnt, nullptr), count_launch();
        grid_scan_kernel<<<1, 1024, 0, stream>>>(cnt, (int)cells, start), count_launch();
        UMGS_TRY(cudaGetLastError());
    }
    UMGS_TRY(cudaMemcpyAsync(&nent, start + cells, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    UMGS_TRY(cudaStreamSynchronize(stream));
    const size_t need = off_ent0 + sizeof(float4) * 3 * (size_t)std::max(1, nent);
    if (need > ws.bytes) {
        // grow, keeping the counts/starts (copy the small header region)
        void* old = ws.ptr;
        size_t oldb = ws.bytes;
        void* nw = nullptr;
        UMGS_TRY(cudaMalloc(&nw, need + need / 4));
        UMGS_TRY(cudaMemcpyAsync(nw, old, std::min(oldb, off_ent0), cudaMemcpyDeviceToDevice, stream));
        UMGS_TRY(cudaStreamSynchronize(stream));
        cudaFree(old);
        ws.ptr = nw;
        ws.bytes = need + need / 4;
        cnt = reinterpret_cast<int32_t*>(ws.as<char>() + off_cnt);
        fill = reinterpret_cast<int32_t*>(ws.as<char>() + off_fill);
        start = reinterpret_cast<int32_t*>(ws.as<char>() + off_start);
    }
    float4* ent = reinterpret_cast<float4*>(ws.as<char>() + off_ent0);
    {
        StageTimer tm(ctx, UMGS_STAGE_BIND_GRID, stream);
        grid_fill_kernel<<<grid_for(nf, 256), 256, 0, stream>>>(V, F, nf, gi, start, fill, ent), count_launch();
        UMGS_TRY(cudaGetLastError());
    }
    // cameras
    std::vector<DevCam> dc(ncams);
    for (int c = 0; c < ncams; ++c) {
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) dc[c].R[3 * r + k] = cams[c].viewmat[4 * r + k];
            dc[c].t[r] = cams[c].viewmat[4 * r + 3];
        }
    }
    UMGS_TRY(ctx->bind_cams.reserve(sizeof(DevCam) * std::max(1, ncams)));
    if (ncams > 0)
        UMGS_TRY(cudaMemcpyAsync(ctx->bind_cams.ptr, dc.data(), sizeof(DevCam) * ncams, cudaMemcpyHostToDevice, stream));
    UMGS_TRY(ctx->bind_cnt.reserve(sizeof(unsigned long long)));
    UMGS_TRY(cudaMemsetAsync(ctx->bind_cnt.ptr, 0, sizeof(unsigned long long), stream));
    const int per = (mode == UMGS_BIND_BBX) ? 8 : 1;
    const int64_t ntg = g->n * per;
    if (ntg > 0) {
        if (mode != UMGS_BIND_NEAREST) {
            StageTimer tm(ctx, UMGS_STAGE_BIND_RAYCAST, stream);
            bind_raycast_kernel<<<grid_for(ntg, 128), 128, 0, stream>>>(
                g->means, g->quats, g->scales, g->n, mode, k_sigma, ctx->bind_cams.as<DevCam>(), ncams, gi, start, ent,
                out_face, out_bary, out_dist, out_flags, ctx->dstatus.as<int32_t>()), count_launch();
            UMGS_TRY(cudaGetLastError());
        }
        StageTimer tm(ctx, UMGS_STAGE_BIND_NEAREST, stream);
        bind_nearest_kernel<<<grid_for(ntg, 128), 128, 0, stream>>>(
            g->means, g->quats, g->scales, g->n, mode, k_sigma, gi, start, ent, out_face, out_bary, out_dist, out_flags,
            ctx->bind_cnt.as<unsigned long long>()), count_launch();
        UMGS_TRY(cudaGetLastError());
    }
    unsigned long long nfb = 0;
    int32_t st = 0;
    UMGS_TRY(cudaMemcpyAsync(&nfb, ctx->bind_cnt.ptr, sizeof(nfb), cudaMemcpyDeviceToHost, stream));
    UMGS_TRY(cudaMemcpyAsync(&st, ctx->dstatus.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    UMGS_TRY(cudaStreamSynchronize(stream));
    if (out_num_fallback) *out_num_fallback = (int64_t)nfb;
    if (st & 4) return fail(ctx, UMGS_ERR_CAPACITY, "a ray exceeded the cell-visit budget");
#undef UMGS_TRY
    return UMGS_OK;
}

}  // namespace umgs
