// Compositor of the forward pass (Sec. 3.2, Eq. 1-2 and 7-11) and the
// evaluation count of a rendered frame.
//
// One CTA per tile, two pixels per thread: records of the tile's sorted list
// are staged through shared memory in batches, every pixel blends its
// fragments front to back (Eq. 1-2 for Gaussians, Eq. 7-9 for entities of
// depth-adjacent triangles, background Eq. 10-11) and the CTA stops when
// every pixel has T < t_eps (block-wide vote).  A persistent variant takes
// tiles from an atomic queue in decreasing list length.
#include <cstdio>
#include <cstring>
#include <cmath>
#include <algorithm>

#include "internal.h"

namespace umgs {
// ---------------------------------------------------------------------------
// compositor

// ---- layout: two pixels per thread -----------------------------------------
// Warp w of a TS x TS tile owns the 8 x 8 pixel block (w % (TS/8), w / (TS/8));
// lane l holds the pixels (l % 8, l / 8) and (l % 8, l / 8 + 4) of it.  The
// two pixels share a column, so the record loads, the list walk, the rect
// test in x and the x part of a Gaussian's exponent are done once for both.
template <int TS> struct Layout {
    static constexpr int NW = TS * TS / 64;  // warps (8 x 8 blocks) per tile
    static constexpr int NT = 32 * NW;       // threads per tile
    static constexpr int NB = 256;           // records staged per batch
    static constexpr int RPT = (NB + NT - 1) / NT;  // records per thread in the staging
};
// resident CTAs per SM the 16 x 16 kernels are built for (80 registers, no
// spills; shared memory allows the same)
template <int TS> struct MinBlocks { static constexpr int value = TS == 16 ? 6 : 1; };
constexpr int kSlot = 11;      // 16-byte vectors of shared memory per staged triangle
constexpr int kTriSlots = 64;  // staged triangles per batch (a batch ends before the 65th)

// Per-pixel state of the blend.  The colour, the transmittance and the
// expected-depth sums of a thread's two pixels are held as (pixel 0, pixel 1)
// pairs in PairAcc, so that a Gaussian fragment updates both with one packed
// fp32 instruction each (fma.rn.f32x2: the same rounding as two scalar fmas).
struct PixelState {
    float Tin;
    float t[4];
    float g_since;
    bool in_ent;
    bool done;
    int last;
    int sp;
};
struct PairAcc {
    float2 C[3];
    float2 T;
    float2 D, Wd;  // expected-depth mode: sum w z, sum w
};

// Shared memory of the forward compositor: per batch the staged Gaussians
// as five 16-byte vectors, the pairs that the packed exponent of a thread's
// two pixels reads ((-u, -u, -v, -v), (l0, l0, l1, l1), (l2, l2, o, o)),
// then (r, g, b, Z) and the pixel rect (x0, x1 - x0, y0, y1 - y0) as
// integers; up to kTriSlots staged triangles (kSlot x 16
// bytes, stage_triangle), the ids and warp-block masks of the batch's
// records, one ballot of "is a triangle" per 32 records, each triangle
// record's slot, and per warp its list of entries (record | slot << 8 |
// 0x8000 for a triangle).
template <int TS>
struct CompositeSmem {
    static constexpr int NB = Layout<TS>::NB;
    float4 g[NB][5];
    float4 t[kTriSlots][kSlot];
    uint32_t id[NB];
    uint32_t wmask[NB];
    uint32_t tbal[NB / 32];
    uint8_t tslot[NB];
    uint16_t list[Layout<TS>::NW * NB];
};

// SAVE: also keep what the backward pass needs: per pixel the final T and
// the number of covering triangle fragments, and per covering triangle
// fragment the four sub-sample transmittances before it (scaled by T_in/4)
// in a per-pixel stack of capacity `cap` (`need` records the largest count).
// MODE: UMGS_BLEND_* or kModeTProduct (FULL with the literal Eq. 6
// transmittance T <- T (1 - O_i alpha_i) inside an entity).
constexpr int kModeTProduct = 4;
// kModeDepth: FULL blending that also accumulates each pixel's expected depth
// sum w z / sum w (w the blend weight; z the Gaussian mean's camera depth or
// the triangle's perspective-correct depth at the pixel centre) into
// out_depth (+inf where nothing blends).
constexpr int kModeDepth = 5;

// ---- triangle records staged for one tile ----------------------------------
// A triangle is staged for the tile it is composited in as kSlot 16-byte
// vectors (int4 / float4 views of the same slot):
//   w[0] = (E0_0, E0_1, E0_2, flags)  edge functions E_k (1/256 px units,
//          top-left bias included) at the centre of the tile's first pixel
//   w[1] = (A256_k, u_0), w[2] = (B256_k, v_0): change of E_k per pixel
//          step in x and in y (256 A_k, 256 B_k); vertex 0 on the screen
//   w[3] = (P_k, 0), w[4] = (Q_k, ia): sample j of a pixel is inside edge k
//          iff E_k + o_kj >= 0, o_k = (P_k, Q_k, -Q_k, -P_k) for the offsets
//          (-2,-6), (6,-2), (-6,2), (2,6) / 16 px, i.e. P = -32 A - 96 B and
//          Q = 96 A - 32 B; ia = 1 / (twice the signed screen area)
//   w[5..7] = (alpha_e | beta_e | gamma_e, c_e): lambda_e(q) = alpha_e +
//          beta_e qx + gamma_e qy is twice the signed area of (q, P_a, P_b),
//          (a, b) = (e+1, e+2), for q relative to vertex 0; c_e = iz_e ia
//          (perspective-correct barycentric weight per unit lambda)
//   w[8..10] = (colour or texture uv of vertex e, alpha_e)
// Integer coverage stays exact in int32 when every edge function over the
// tile's samples lies within +-2^30; an edge that every sample of the tile
// passes is replaced by the constant 1 (A = B = P = Q = 0), and a triangle
// with an edge no sample of the tile passes has no fragment there.  A record
// beyond that range (an edge of more than about 1,000 px crossing the tile)
// is flagged kTriWide and tested in int64 from its global record.
constexpr int kTriWide = 1, kTriConstAlpha = 2;

// a*b - c*d with one rounding of the result (Kahan's compensated form)
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// Stages triangle record t for the tile with origin (tx0, ty0) into slot w;
// returns the mask of the tile's 8 x 8 blocks that can hold a fragment of it.
template <int TS>
__device__ __forceinline__ uint32_t stage_triangle(const TRec& t, int tx0, int ty0, float4* __restrict__ w) {
    uint32_t m = box_block_mask<TS, 8>((int)(t.rx & 0xffff), (int)(t.rx >> 16), (int)(t.ry & 0xffff),
                                       (int)(t.ry >> 16), tx0, ty0);
    if (!m) return 0u;
    const long long cx0 = (long long)tx0 * 256 + 128, cy0 = (long long)ty0 * 256 + 128;
    constexpr long long kLim = 1LL << 30;
    int E0[3], A2[3], B2[3], P[3], Q[3], off[3];
    bool wide = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const long long A = t.A[k], B = t.B[k];
        const long long e = A * cx0 + B * cy0 + t.C[k];
        const long long a = A * 256, b = B * 256;
        const long long p = -32 * A - 96 * B, q = 96 * A - 32 * B;
        const long long o = max(llabs(p), llabs(q));
        const long long lo = e + min(0LL, a * (TS - 1)) + min(0LL, b * (TS - 1)) - o;
        const long long hi = e + max(0LL, a * (TS - 1)) + max(0LL, b * (TS - 1)) + o;
        if (hi < 0) return 0u;  // no sample of the tile is inside edge k
        if (lo >= 0) {          // every sample of the tile is inside edge k
            E0[k] = 1; A2[k] = B2[k] = P[k] = Q[k] = off[k] = 0;
            continue;
        }
        if (lo < -kLim || hi > kLim) wide = true;
        E0[k] = (int)e; A2[k] = (int)a; B2[k] = (int)b; P[k] = (int)p; Q[k] = (int)q; off[k] = (int)o;
    }
    if (!wide) {
        // drop the 8 x 8 blocks that an edge excludes entirely
        uint32_t mm = m;
        while (mm) {
            const int wb = __ffs(mm) - 1;
            mm &= mm - 1;
            const int bx = (wb % (TS / 8)) * 8, by = (wb / (TS / 8)) * 8;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int hi = E0[k] + A2[k] * bx + B2[k] * by + max(0, A2[k] * 7) + max(0, B2[k] * 7) + off[k];
                if (hi < 0) m &= ~(1u << wb);
            }
        }
        if (!m) return 0u;
    }
    int4* wi = reinterpret_cast<int4*>(w);
    const int flags = (wide ? kTriWide : 0) | (t.const_alpha ? kTriConstAlpha : 0) | (t.tex << 8);
    wi[0] = make_int4(E0[0], E0[1], E0[2], flags);
    wi[1] = make_int4(A2[0], A2[1], A2[2], __float_as_int(t.u[0]));
    wi[2] = make_int4(B2[0], B2[1], B2[2], __float_as_int(t.v[0]));
    // attribute planes relative to vertex 0 (the same for every tile, so
    // that images do not depend on the tile size)
    const float U[3] = {0.f, t.u[1] - t.u[0], t.u[2] - t.u[0]};
    const float V[3] = {0.f, t.v[1] - t.v[0], t.v[2] - t.v[0]};
    float al[3], be[3], ga[3], c[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int a = (e + 1) % 3, b = (e + 2) % 3;
        al[e] = diff_of_products(U[a], V[b], U[b], V[a]);
        be[e] = V[a] - V[b];
        ga[e] = U[b] - U[a];
    }
    const float area = al[0] + al[1] + al[2];
    float ia = 0.f;
    if (area != 0.f) {
        ia = 1.f / area;
#pragma unroll
        for (int e = 0; e < 3; ++e) c[e] = t.iz[e] * ia;
    } else {  // degenerate screen triangle: the three vertices weighted by 1/Z alike
#pragma unroll
        for (int e = 0; e < 3; ++e) { al[e] = 1.f; be[e] = ga[e] = 0.f; c[e] = t.iz[e] * (1.f / 3.f); }
    }
    wi[3] = make_int4(P[0], P[1], P[2], 0);
    wi[4] = make_int4(Q[0], Q[1], Q[2], __float_as_int(ia));
    w[5] = make_float4(al[0], al[1], al[2], c[0]);
    w[6] = make_float4(be[0], be[1], be[2], c[1]);
    w[7] = make_float4(ga[0], ga[1], ga[2], c[2]);
    w[8] = make_float4(t.col[0], t.col[1], t.col[2], t.alpha[0]);
    w[9] = make_float4(t.col[3], t.col[4], t.col[5], t.alpha[1]);
    w[10] = make_float4(t.col[6], t.col[7], t.col[8], t.alpha[2]);
    return m;
}

// Sample coverage (bit j: sample j) of the pixel (lx, ly) of the tile by a
// staged (not wide) triangle; DIRECT: 0xf iff the pixel centre is covered.
template <bool CENTRE>
__device__ __forceinline__ int staged_coverage(const float4* __restrict__ w, int lx, int ly) {
    const int4 e0 = reinterpret_cast<const int4*>(w)[0], a = reinterpret_cast<const int4*>(w)[1],
               b = reinterpret_cast<const int4*>(w)[2];
    const int E0 = e0.x + a.x * lx + b.x * ly, E1 = e0.y + a.y * lx + b.y * ly, E2 = e0.z + a.z * lx + b.z * ly;
    if (CENTRE) return (E0 >= 0 && E1 >= 0 && E2 >= 0) ? 0xf : 0;
    const int4 p = reinterpret_cast<const int4*>(w)[3], q = reinterpret_cast<const int4*>(w)[4];
    const bool s0 = (E0 + p.x >= 0) & (E1 + p.y >= 0) & (E2 + p.z >= 0);
    const bool s1 = (E0 + q.x >= 0) & (E1 + q.y >= 0) & (E2 + q.z >= 0);
    const bool s2 = (E0 >= q.x) & (E1 >= q.y) & (E2 >= q.z);
    const bool s3 = (E0 >= p.x) & (E1 >= p.y) & (E2 >= p.z);
    return (s0 ? 1 : 0) | (s1 ? 2 : 0) | (s2 ? 4 : 0) | (s3 ? 8 : 0);
}

// Sample coverage of pixel (px, py) by a global triangle record in int64.
__device__ __forceinline__ int record_coverage(const TRec& t, int px, int py, bool centre_only) {
    const long long scx = (long long)px * 256 + 128, scy = (long long)py * 256 + 128;
    long long E[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) E[e] = (long long)t.A[e] * scx + (long long)t.B[e] * scy + t.C[e];
    if (centre_only) return (E[0] >= 0 && E[1] >= 0 && E[2] >= 0) ? 0xf : 0;
    int mask = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int sdx = sample_dx(j), sdy = sample_dy(j);
        bool in = true;
#pragma unroll
        for (int e = 0; e < 3; ++e) in = in && (E[e] + (long long)(t.A[e] * sdx + t.B[e] * sdy) >= 0);
        mask |= in ? (1 << j) : 0;
    }
    return mask;
}

// One triangle record at one pixel: coverage, attributes, and the blend of
// the blend mode (Eq. 7-9 for FULL).  Returns true when it was a fragment.
template <bool SAVE, int MODE>
__device__ __forceinline__ bool blend_triangle(PixelState& st, float (&C)[3], float& T, float& D, float& Wd,
                                               const float4* __restrict__ w, const TRec* __restrict__ TR,
                                               uint32_t tid, int px, int py, int lx, int ly,
                                               float4* __restrict__ stack, int cap, int64_t npix, int64_t pix,
                                               const DevTex* __restrict__ textab) {
    constexpr int mode = MODE;
    const float qx = px + 0.5f, qy = py + 0.5f;
    const int flags = reinterpret_cast<const int4*>(w)[0].w;
    int mask;
    float wv[3], zt = 0.f;
    if (!(flags & kTriWide)) {
        mask = staged_coverage<MODE == UMGS_BLEND_DIRECT>(w, lx, ly);
        if (mask == 0) return false;
        // perspective-correct barycentrics at the pixel centre, clamped at 0
        const float4 fa = w[5], fb = w[6], fc = w[7];
        const float rqx = __fsub_rn(qx, __int_as_float(reinterpret_cast<const int4*>(w)[1].w));
        const float rqy = __fsub_rn(qy, __int_as_float(reinterpret_cast<const int4*>(w)[2].w));
        const float l0 = __fmaf_rn(fb.x, rqx, __fmaf_rn(fc.x, rqy, fa.x));
        const float l1 = __fmaf_rn(fb.y, rqx, __fmaf_rn(fc.y, rqy, fa.y));
        const float l2 = __fmaf_rn(fb.z, rqx, __fmaf_rn(fc.z, rqy, fa.z));
        wv[0] = fmaxf(l0 * fa.w, 0.f); wv[1] = fmaxf(l1 * fb.w, 0.f); wv[2] = fmaxf(l2 * fc.w, 0.f);
        if (mode == kModeDepth) {
            const float ia = __int_as_float(reinterpret_cast<const int4*>(w)[4].w);
            const float ls = ia != 0.f ? fmaxf(l0 * ia, 0.f) + fmaxf(l1 * ia, 0.f) + fmaxf(l2 * ia, 0.f) : 1.f;
            const float ws0 = wv[0] + wv[1] + wv[2];
            const TRec& t = TR[tid];
            zt = ws0 > 0.f ? ls / ws0 : 3.f / (t.iz[0] + t.iz[1] + t.iz[2]);
        }
    } else {  // wide record: int64 coverage and attributes from the global record
        const TRec& t = TR[tid];
        if (px < (int)(t.rx & 0xffff) || px > (int)(t.rx >> 16) || py < (int)(t.ry & 0xffff) ||
            py > (int)(t.ry >> 16))
            return false;
        mask = record_coverage(t, px, py, mode == UMGS_BLEND_DIRECT);
        if (mask == 0) return false;
        float lam[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int a = (e + 1) % 3, b = (e + 2) % 3;
            lam[e] = (t.u[a] - qx) * (t.v[b] - qy) - (t.u[b] - qx) * (t.v[a] - qy);
        }
        const float area = lam[0] + lam[1] + lam[2];
        if (area != 0.f) {
            const float ia = __fdividef(1.f, area);
#pragma unroll
            for (int e = 0; e < 3; ++e) wv[e] = fmaxf(lam[e] * ia, 0.f) * t.iz[e];
        } else {
#pragma unroll
            for (int e = 0; e < 3; ++e) wv[e] = (1.f / 3.f) * t.iz[e];
        }
        if (mode == kModeDepth) {
            const float ls = area != 0.f ? fmaxf(lam[0] / area, 0.f) + fmaxf(lam[1] / area, 0.f) +
                                               fmaxf(lam[2] / area, 0.f)
                                         : 1.f;
            const float ws0 = wv[0] + wv[1] + wv[2];
            zt = ws0 > 0.f ? ls / ws0 : 3.f / (t.iz[0] + t.iz[1] + t.iz[2]);
        }
    }
    const float ws = wv[0] + wv[1] + wv[2];
    if (ws > 0.f) { const float is = __fdividef(1.f, ws); wv[0] *= is; wv[1] *= is; wv[2] *= is; }
    else { wv[0] = wv[1] = wv[2] = 1.f / 3.f; }
    const float4 v0 = w[8], v1 = w[9], v2 = w[10];
    float col[3];
    if (flags >> 8) {  // textured face: (u, v) interpolated like a colour, then sampled
        const float tu = wv[0] * v0.x + wv[1] * v0.z + wv[2] * v1.y;
        const float tv = wv[0] * v0.y + wv[1] * v1.x + wv[2] * v1.z;
        sample_texture(textab[(flags >> 8) - 1], tu, tv, col);
    } else {
        col[0] = wv[0] * v0.x + wv[1] * v1.x + wv[2] * v2.x;
        col[1] = wv[0] * v0.y + wv[1] * v1.y + wv[2] * v2.y;
        col[2] = wv[0] * v0.z + wv[1] * v1.z + wv[2] * v2.z;
    }
    float a = (flags & kTriConstAlpha) ? v0.w : (wv[0] * v0.w + wv[1] * v1.w + wv[2] * v2.w);
    a = fminf(fmaxf(a, 0.f), 1.f);
    if (mode == UMGS_BLEND_DIRECT) {
        const float wt = a * T;
        C[0] += wt * col[0]; C[1] += wt * col[1]; C[2] += wt * col[2];
        T *= (1.f - a);
    } else if (mode == UMGS_BLEND_MSAA_ALL) {
        const float O = 0.25f * (float)__popc(mask);
        const float wt = O * a * T;
        C[0] += wt * col[0]; C[1] += wt * col[1]; C[2] += wt * col[2];
        T *= (1.f - O * a);
    } else {
        if (!st.in_ent) {
            st.Tin = T;
            st.t[0] = st.t[1] = st.t[2] = st.t[3] = 1.f;
            st.g_since = 1.f;
            st.in_ent = true;
        }
        if (SAVE && mode == UMGS_BLEND_FULL) {
            if (st.sp < cap) {
                const float q = 0.25f * st.Tin;
                stack[(int64_t)st.sp * npix + pix] = make_float4(q * st.t[0], q * st.t[1], q * st.t[2], q * st.t[3]);
            }
            ++st.sp;
        }
        float O = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) O += ((mask >> j) & 1) ? st.t[j] : 0.f;
        O *= 0.25f;
        const float wt = st.Tin * O * a;
        C[0] += wt * col[0]; C[1] += wt * col[1]; C[2] += wt * col[2];
        if (mode == kModeDepth) { D += wt * zt; Wd += wt; }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((mask >> j) & 1) st.t[j] *= (1.f - a);
        const float tm = 0.25f * ((st.t[0] + st.t[1]) + (st.t[2] + st.t[3]));
        if (mode == kModeTProduct) T *= (1.f - O * a);
        else T = (mode == UMGS_BLEND_ENTITY_ALL) ? st.Tin * tm * st.g_since : st.Tin * tm;
    }
    return true;
}

// Blend of a Gaussian fragment into both pixels of a thread (Eq. 1-2):
// alpha (a0, a1), where a pixel the fragment does not reach takes alpha 0,
// which leaves its colour, T and sums exactly as they were.
template <int MODE>
__device__ __forceinline__ void blend_gaussian2(PixelState (&st)[2], PairAcc& acc, bool t0, bool t1, float a0, float a1,
                                                float r, float g, float b, float z, int pos, float t_eps) {
    const float2 al = make_float2(t0 ? a0 : 0.f, t1 ? a1 : 0.f);
    const float2 w = __fmul2_rn(al, acc.T);
    acc.C[0] = __ffma2_rn(w, make_float2(r, r), acc.C[0]);
    acc.C[1] = __ffma2_rn(w, make_float2(g, g), acc.C[1]);
    acc.C[2] = __ffma2_rn(w, make_float2(b, b), acc.C[2]);
    if (MODE == kModeDepth) {
        acc.D = __ffma2_rn(w, make_float2(z, z), acc.D);
        acc.Wd = __fadd2_rn(acc.Wd, w);
    }
    acc.T = __ffma2_rn(make_float2(-al.x, -al.y), acc.T, acc.T);  // T (1 - alpha), one rounding
    if (MODE == UMGS_BLEND_ENTITY_ALL) {
        st[0].g_since *= (1.f - al.x);
        st[1].g_since *= (1.f - al.y);
    } else {
        st[0].in_ent = st[0].in_ent && !t0;
        st[1].in_ent = st[1].in_ent && !t1;
    }
    if (t0) st[0].last = pos;
    if (t1) st[1].last = pos;
    st[0].done = st[0].done || acc.T.x < t_eps;
    st[1].done = st[1].done || acc.T.y < t_eps;
}

template <int TS, bool SAVE, int MODE>
__device__ __forceinline__ void composite_tile(
    int tile, int64_t seg_beg, int64_t seg_end, float4* __restrict__ seg_out, int32_t* __restrict__ seg_last,
    CompositeSmem<TS>& sm,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off,
    const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need, float* __restrict__ out_depth, const DevTex* __restrict__ textab) {
    using L = Layout<TS>;
    constexpr int NT = L::NT, NB = L::NB, RPT = L::RPT;
    const int cam = tile / tiles_per_cam;
    const int lt = tile - cam * tiles_per_cam;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = (warp % (TS / 8)) * 8 + (lane & 7);
    const int ly0 = (warp / (TS / 8)) * 8 + (lane >> 3), ly1 = ly0 + 4;
    const int tile_x0 = tx * TS, tile_y0 = ty * TS;
    const int px = tile_x0 + lx, py0 = tile_y0 + ly0, py1 = tile_y0 + ly1;
    // the tile's list, or one segment [seg_beg, seg_end) of it (list
    // positions stay relative to the start of the tile's list)
    const int64_t beg = off[tile], end = seg_end >= 0 ? seg_end : off[tile + 1];
    const GRec* G = grec + (int64_t)cam * Ng;
    const GRec16* G16 = grec16 ? grec16 + (int64_t)cam * Ng : nullptr;
    const TRec* TR = trec + (int64_t)cam * Nt;
    const float qx = px + 0.5f, qy0 = py0 + 0.5f, qy1 = py1 + 0.5f;

    PixelState st[2];
    PairAcc acc;
    acc.C[0] = acc.C[1] = acc.C[2] = make_float2(0.f, 0.f);
    acc.T = make_float2(1.f, 1.f);
    acc.D = acc.Wd = make_float2(0.f, 0.f);
    const float2 qxx = make_float2(qx, qx), qyy = make_float2(qy0, qy1);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        st[p].Tin = 1.f; st[p].g_since = 1.f;
        st[p].t[0] = st[p].t[1] = st[p].t[2] = st[p].t[3] = 1.f;
        st[p].in_ent = false;
        st[p].last = 0;
        st[p].sp = 0;
    }
    st[0].done = !(px < W && py0 < H);
    st[1].done = !(px < W && py1 < H);
    const int64_t pix0 = ((int64_t)cam * H + py0) * W + px, pix1 = ((int64_t)cam * H + py1) * W + px;

    for (int64_t b0 = seg_beg >= 0 ? seg_beg : beg; b0 < end;) {
        int n = (int)min((int64_t)NB, end - b0);
        uint32_t rid[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int k = threadIdx.x + r * NT;
            rid[r] = k < n ? ids[b0 + k] : 0xffffffffu;
            const unsigned bal = __ballot_sync(0xffffffffu, rid[r] >= Ng && rid[r] < Ng + Nt);
            // (written before the barrier: read only between it and the
            // staging barrier, which every warp has passed by now)
            if (lane == 0 && k < NB) sm.tbal[k >> 5] = bal;
        }
        if (__syncthreads_count(st[0].done && st[1].done) == NT) break;
        // the batch ends before its (kTriSlots + 1)-th triangle (every thread
        // finds the same cut, and the number of triangles nT, from the ballots)
        int nT = 0;
        for (int wd = 0; wd < NB / 32 && wd * 32 < n; ++wd) {
            uint32_t m = sm.tbal[wd];
            const int c = __popc(m);
            if (nT + c > kTriSlots) {
                for (int j = nT; j < kTriSlots; ++j) m &= m - 1u;
                n = min(n, wd * 32 + __ffs(m) - 1);
                nT = kTriSlots;
                break;
            }
            nT += c;
        }
        const int lbase = (int)(b0 - beg) + 1;  // list position + 1 of the batch's first record
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int k = threadIdx.x + r * NT;
            if (k >= n) continue;
            const uint32_t id = rid[r];
            sm.id[k] = id;
            if (id >= Ng + Nt) {
                sm.wmask[k] = 0u;  // not a record of this frame: no fragment
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
                const int x0 = (int)(rx & 0xffff), x1 = (int)(rx >> 16), y0 = (int)(ry & 0xffff), y1 = (int)(ry >> 16);
                sm.g[k][0] = make_float4(-a.x, -a.x, -a.y, -a.y);
                sm.g[k][1] = make_float4(a.z, a.z, a.w, a.w);
                sm.g[k][2] = make_float4(b.x, b.x, b.y, b.y);
                sm.g[k][3] = make_float4(b.z, b.w, c.x, c.w);
                reinterpret_cast<int4*>(&sm.g[k][4])[0] = make_int4(x0, x1 - x0, y0, y1 - y0);
                sm.wmask[k] = gauss_block_mask<TS, 8>(a.x, a.y, a.z, a.w, b.x, b.y, x0, x1, y0, y1, tile_x0, tile_y0);
            }
        }
        // triangles, compacted over the threads: thread t stages the batch's
        // t-th triangle (slot t), so that the long triangle set-up does not
        // hold up the Gaussian records of 32 different warps
        for (int t = threadIdx.x; t < nT; t += NT) {
            int run = 0, wd = 0;
            uint32_t m = 0u;
            for (; wd < NB / 32; ++wd) {
                m = sm.tbal[wd];
                const int c = __popc(m);
                if (run + c > t) break;
                run += c;
            }
            if (wd >= NB / 32) break;  // (cannot happen: nT counts the ballots' bits)
            for (int j = run; j < t; ++j) m &= m - 1u;
            const int k = wd * 32 + __ffs(m) - 1;
            const uint32_t id = ids[b0 + k];
            sm.tslot[k] = (uint8_t)t;
            sm.wmask[k] = stage_triangle<TS>(TR[id - Ng], tile_x0, tile_y0, &sm.t[t][0]);
        }
        __syncthreads();
        b0 += n;
        if (__any_sync(0xffffffffu, !(st[0].done && st[1].done))) {
            // this warp's records of the batch, in order
            uint16_t* lst = sm.list + warp * NB;
            int cnt = 0;
            const uint32_t ng32 = (uint32_t)Ng;
            for (int c0 = 0; c0 < n; c0 += 32) {
                const int kk = c0 + lane;
                const bool mine = kk < n && ((sm.wmask[kk] >> warp) & 1u);
                const unsigned bal = __ballot_sync(0xffffffffu, mine);
                if (mine) {
                    const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                    const bool tri = sm.id[kk] >= ng32;
                    lst[pos] = (uint16_t)(tri ? (kk | (sm.tslot[kk] << 8) | 0x8000) : kk);
                }
                cnt += __popc(bal);
            }
            __syncwarp();
            for (int li = 0; li < cnt; ++li) {
                const int ent = lst[li];
                const int k = ent & 0xff;
                if (st[0].done && st[1].done) continue;
                if (!(ent & 0x8000)) {
                    const int4 r = reinterpret_cast<const int4*>(&sm.g[k][4])[0];  // (x0, w, y0, h)
                    const bool inx = (unsigned)(px - r.x) <= (unsigned)r.y;
                    const bool in0 = inx && (unsigned)(py0 - r.z) <= (unsigned)r.w && !st[0].done;
                    const bool in1 = inx && (unsigned)(py1 - r.z) <= (unsigned)r.w && !st[1].done;
                    if (!(in0 || in1)) continue;
                    // the exponent of both pixels in packed fp32 (the operation
                    // order and roundings of gauss_power2)
                    const float4 g0 = sm.g[k][0], g1 = sm.g[k][1], g2 = sm.g[k][2];
                    const float2 dx = __fadd2_rn(qxx, make_float2(g0.x, g0.y));
                    const float2 dy = __fadd2_rn(qyy, make_float2(g0.z, g0.w));
                    const float2 w1 = __ffma2_rn(make_float2(g1.z, g1.w), dy, __fmul2_rn(make_float2(g1.x, g1.y), dx));
                    const float2 w2 = __fmul2_rn(make_float2(g2.x, g2.y), dy);
                    const float2 pw = __ffma2_rn(w1, w1, __fmul2_rn(w2, w2));
                    const float2 e = __fmul2_rn(make_float2(g2.z, g2.w), make_float2(fast_exp2(-pw.x), fast_exp2(-pw.y)));
                    const float a0 = fminf(kAlphaMax, e.x), a1 = fminf(kAlphaMax, e.y);
                    const bool t0 = in0 && a0 >= kAlphaMin, t1 = in1 && a1 >= kAlphaMin;
                    if (!(t0 || t1)) continue;
                    const float4 g3 = sm.g[k][3];  // (r, g, b, Z)
                    blend_gaussian2<MODE>(st, acc, t0, t1, a0, a1, g3.x, g3.y, g3.z, g3.w, lbase + k, t_eps);
                } else {
                    const float4* w = &sm.t[(ent >> 8) & 0x7f][0];
                    const uint32_t tid = sm.id[k] - (uint32_t)Ng;
                    if (!st[0].done) {
                        float C[3] = {acc.C[0].x, acc.C[1].x, acc.C[2].x};
                        float T = acc.T.x, D = acc.D.x, Wd = acc.Wd.x;
                        if (blend_triangle<SAVE, MODE>(st[0], C, T, D, Wd, w, TR, tid, px, py0, lx, ly0, stack, cap,
                                                       npix, pix0, textab)) {
                            st[0].last = lbase + k;
                            if (T < t_eps) st[0].done = true;
                        }
                        acc.C[0].x = C[0]; acc.C[1].x = C[1]; acc.C[2].x = C[2];
                        acc.T.x = T; acc.D.x = D; acc.Wd.x = Wd;
                    }
                    if (!st[1].done) {
                        float C[3] = {acc.C[0].y, acc.C[1].y, acc.C[2].y};
                        float T = acc.T.y, D = acc.D.y, Wd = acc.Wd.y;
                        if (blend_triangle<SAVE, MODE>(st[1], C, T, D, Wd, w, TR, tid, px, py1, lx, ly1, stack, cap,
                                                       npix, pix1, textab)) {
                            st[1].last = lbase + k;
                            if (T < t_eps) st[1].done = true;
                        }
                        acc.C[0].y = C[0]; acc.C[1].y = C[1]; acc.C[2].y = C[2];
                        acc.T.y = T; acc.D.y = D; acc.Wd.y = Wd;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int py = p ? py1 : py0;
        if (!(px < W && py < H)) continue;
        const int64_t pix = p ? pix1 : pix0;
        const PixelState& s = st[p];
        const float C0 = p ? acc.C[0].y : acc.C[0].x, C1 = p ? acc.C[1].y : acc.C[1].x,
                    C2 = p ? acc.C[2].y : acc.C[2].x, T = p ? acc.T.y : acc.T.x;
        const float D = p ? acc.D.y : acc.D.x, Wd = p ? acc.Wd.y : acc.Wd.x;
        if (seg_out) {  // one segment of a split tile: its own composite, no background (split_merge_kernel)
            const int q = (p ? ly1 : ly0) * TS + lx;
            seg_out[q] = make_float4(C0, C1, C2, T);
            seg_last[q] = s.last;
            continue;
        }
        out[pix] = make_float4(C0 + T * bg0, C1 + T * bg1, C2 + T * bg2, T);
        // bit 31: the pixel stopped at T < t_eps after list position `last`
        if (out_last) out_last[pix] = s.last | (T < t_eps ? (int)0x80000000u : 0);
        if (SAVE) {
            out_tfin[pix] = T;
            out_ntri[pix] = s.sp;
            if (s.sp > cap) atomicMax(need, s.sp);
        }
        if (MODE == kModeDepth) out_depth[pix] = Wd > 0.f ? D / Wd : __int_as_float(0x7f800000);
    }
}


// one CTA per tile (grid launch)
template <int TS, bool SAVE, int MODE>
__global__ void __launch_bounds__(Layout<TS>::NT, MinBlocks<TS>::value) composite_kernel(
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need, float* __restrict__ out_depth, const DevTex* __restrict__ textab) {
    pdl_enter();
    __shared__ CompositeSmem<TS> sm;
    composite_tile<TS, SAVE, MODE>(blockIdx.x, -1, -1, nullptr, nullptr, sm, ids, off, grec, grec16, trec, Ng, Nt, tiles_x, tiles_per_cam, W, H, t_eps, bg0, bg1, bg2, out, out_last, out_tfin, out_ntri, stack, cap, npix, need, out_depth, textab);
}

// persistent launch: resident CTAs take tiles from an atomic queue in the
// order `order` (decreasing list length: the heaviest tiles start first)
template <int TS, bool SAVE, int MODE>
__global__ void __launch_bounds__(Layout<TS>::NT, MinBlocks<TS>::value) composite_persistent_kernel(
    const uint32_t* __restrict__ order, unsigned* __restrict__ work, int64_t M,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need, float* __restrict__ out_depth, const DevTex* __restrict__ textab) {
    pdl_enter();
    __shared__ CompositeSmem<TS> sm;
    __shared__ unsigned s_next;
    while (true) {
        if (threadIdx.x == 0) s_next = atomicAdd(work, 1u);
        __syncthreads();
        const unsigned k = s_next;
        __syncthreads();
        if ((int64_t)k >= M) break;
        composite_tile<TS, SAVE, MODE>((int)order[k], -1, -1, nullptr, nullptr, sm, ids, off, grec, grec16, trec, Ng, Nt, tiles_x, tiles_per_cam, W, H, t_eps, bg0, bg1, bg2, out, out_last, out_tfin, out_ntri, stack, cap, npix, need, out_depth, textab);
        __syncthreads();
    }
}

// ---- per-tile work split -----------------------------------------------------
// A tile whose list holds more than `split` records is composited as segments
// of `split` records on separate CTAs, each from T = 1, and the segments are
// merged per pixel front to back: C = sum_k (prod_{m<k} T_m) C_k, T = prod_k
// T_k (the composite of Eq. 1-2 regrouped; fp rounding differs from the whole
// tile).  Cuts are placed only in front of the list's first triangle record:
// an entity of depth-adjacent triangles (Eq. 7-9) would carry per-pixel
// state across a cut, and no entity can be open before a tile's first
// triangle.  A segment stops at its own T < t_eps, so it may blend a few
// fragments that the whole tile, already below t_eps, would drop: at most
// t_eps times the largest colour.
//
// Work item: int4 (tile, list begin, list end, meta), meta = slot | seg << 16 |
// nseg << 24; nseg = 1 is a whole tile (composited into the image).
constexpr int kMaxSegs = 64;

// one warp per tile: its segments, segment slots and work items
__global__ void split_plan_kernel(const int64_t* __restrict__ off, const uint32_t* __restrict__ ids, int64_t M,
                                  uint32_t ng, int split, int4* __restrict__ items, unsigned* __restrict__ nitems,
                                  unsigned* __restrict__ nslots, unsigned slots_cap) {
    pdl_enter();
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= M) return;  // (whole warps: M and the block size are warp-aligned per tile)
    const int64_t beg = off[t], end = off[t + 1], len = end - beg;
    int nseg = 1;
    if (len > split) {
        const int64_t lim = min(len, (int64_t)split * kMaxSegs);
        int64_t ftri = lim;  // position of the first triangle record (or the scan limit)
        for (int64_t c = 0; c < lim; c += 32) {
            const bool tri = c + lane < lim && ids[beg + c + lane] >= ng;
            const unsigned b = __ballot_sync(0xffffffffu, tri);
            if (b) { ftri = c + __ffs(b) - 1; break; }
        }
        // cuts at split, 2 split, ... that are <= ftri and < len
        nseg = 1 + (int)min(ftri / split, (len - 1) / split);
        nseg = min(nseg, kMaxSegs);
    }
    if (lane != 0) return;
    unsigned slot = 0;
    if (nseg > 1) {
        slot = atomicAdd(nslots, (unsigned)nseg);
        if (slot + nseg > slots_cap) nseg = 1;  // no room left: the tile is composited whole
    }
    const unsigned base = atomicAdd(nitems, (unsigned)nseg);  // < M + slots_cap: the items buffer's size
    for (int sg = 0; sg < nseg; ++sg) {
        const int64_t sb = beg + (int64_t)sg * split, se = sg == nseg - 1 ? end : sb + split;
        items[base + sg] = make_int4((int)t, (int)(uint32_t)sb, (int)(uint32_t)se,
                                     (int)(slot | ((unsigned)sg << 16) | ((unsigned)nseg << 24)));
    }
}

// order of the work items for the persistent launch (decreasing length)
__global__ void item_order_keys_kernel(const int4* __restrict__ items, const unsigned* __restrict__ nitems,
                                       int64_t cap, uint32_t* __restrict__ k, uint32_t* __restrict__ v) {
    pdl_enter();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= cap || i >= (int64_t)*nitems) return;
    const int4 it = items[i];
    const uint32_t len = (uint32_t)it.z - (uint32_t)it.y;
    k[i] = 0xffffu - min(len, 0xffffu);
    v[i] = (uint32_t)i;
}

// work item -> composite_tile arguments
template <int TS>
__device__ __forceinline__ void item_target(const int4 it, float4* segbuf, int32_t* seglast, int64_t& sb, int64_t& se,
                                            float4*& so, int32_t*& sl) {
    const unsigned meta = (unsigned)it.w;
    const unsigned nseg = meta >> 24;
    sb = (int64_t)(uint32_t)it.y;
    se = (int64_t)(uint32_t)it.z;
    if (nseg > 1) {
        const int64_t q = (int64_t)((meta & 0xffffu) + ((meta >> 16) & 0xffu)) * TS * TS;
        so = segbuf + q;
        sl = seglast + q;
    } else {
        so = nullptr;
        sl = nullptr;
    }
}

// one CTA per work item (grid sized for the item capacity)
template <int TS, int MODE>
__global__ void __launch_bounds__(Layout<TS>::NT, MinBlocks<TS>::value) composite_items_kernel(
    const int4* __restrict__ items, const unsigned* __restrict__ nitems, float4* __restrict__ segbuf,
    int32_t* __restrict__ seglast,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out,
    int32_t* __restrict__ out_last, const DevTex* __restrict__ textab) {
    pdl_enter();
    if (blockIdx.x >= *nitems) return;
    __shared__ CompositeSmem<TS> sm;
    const int4 it = items[blockIdx.x];
    int64_t sb, se;
    float4* so;
    int32_t* sl;
    item_target<TS>(it, segbuf, seglast, sb, se, so, sl);
    composite_tile<TS, false, MODE>(it.x, sb, se, so, sl, sm, ids, off, grec, grec16, trec, Ng, Nt, tiles_x,
                                    tiles_per_cam, W, H, t_eps, bg0, bg1, bg2, out, out_last, nullptr, nullptr,
                                    nullptr, 0, 0, nullptr, nullptr, textab);
}

// persistent launch over the work items in the order `order`
template <int TS, int MODE>
__global__ void __launch_bounds__(Layout<TS>::NT, MinBlocks<TS>::value) composite_items_persistent_kernel(
    const uint32_t* __restrict__ order, unsigned* __restrict__ work, const int4* __restrict__ items,
    const unsigned* __restrict__ nitems, float4* __restrict__ segbuf, int32_t* __restrict__ seglast,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out,
    int32_t* __restrict__ out_last, const DevTex* __restrict__ textab) {
    pdl_enter();
    __shared__ CompositeSmem<TS> sm;
    __shared__ unsigned s_next;
    const unsigned n = *nitems;
    while (true) {
        if (threadIdx.x == 0) s_next = atomicAdd(work, 1u);
        __syncthreads();
        const unsigned k = s_next;
        __syncthreads();
        if (k >= n) break;
        const int4 it = items[order[k]];
        int64_t sb, se;
        float4* so;
        int32_t* sl;
        item_target<TS>(it, segbuf, seglast, sb, se, so, sl);
        composite_tile<TS, false, MODE>(it.x, sb, se, so, sl, sm, ids, off, grec, grec16, trec, Ng, Nt, tiles_x,
                                        tiles_per_cam, W, H, t_eps, bg0, bg1, bg2, out, out_last, nullptr, nullptr,
                                        nullptr, 0, 0, nullptr, nullptr, textab);
        __syncthreads();
    }
}

// merge of the segments of every split tile (one CTA per work item; the
// tile's first segment does the work)
template <int TS>
__global__ void __launch_bounds__(256) split_merge_kernel(
    const int4* __restrict__ items, const unsigned* __restrict__ nitems, const float4* __restrict__ segbuf,
    const int32_t* __restrict__ seglast, int tiles_x, int tiles_per_cam, int W, int H, float t_eps, float bg0,
    float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last) {
    pdl_enter();
    if (blockIdx.x >= *nitems) return;
    const int4 it = items[blockIdx.x];
    const unsigned meta = (unsigned)it.w;
    const int nseg = (int)(meta >> 24), sg = (int)((meta >> 16) & 0xffu);
    if (nseg < 2 || sg != 0) return;
    const unsigned slot = meta & 0xffffu;
    const int tile = it.x;
    const int cam = tile / tiles_per_cam;
    const int lt = tile - cam * tiles_per_cam;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    for (int q = threadIdx.x; q < TS * TS; q += blockDim.x) {
        const int px = tx * TS + q % TS, py = ty * TS + q / TS;
        if (px >= W || py >= H) continue;
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
        int last = 0;
        for (int k = 0; k < nseg; ++k) {
            if (T < t_eps) break;  // the whole tile would have stopped before this segment
            const int64_t i = (int64_t)(slot + k) * TS * TS + q;
            const float4 r = segbuf[i];
            C0 += T * r.x; C1 += T * r.y; C2 += T * r.z;
            T *= r.w;
            const int l = seglast[i];
            if (l > 0) last = l;
        }
        const int64_t pix = ((int64_t)cam * H + py) * W + px;
        out[pix] = make_float4(C0 + T * bg0, C1 + T * bg1, C2 + T * bg2, T);
        if (out_last) out_last[pix] = last | (T < t_eps ? (int)0x80000000u : 0);
    }
}

// tile order for the persistent launch: key = 0xffff - min(list length, 0xffff)
__global__ void tile_order_keys_kernel(const int64_t* __restrict__ off, int64_t M, uint32_t* __restrict__ k,
                                       uint32_t* __restrict__ v, uint32_t* __restrict__ m_dev) {
    pdl_enter();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t == 0) *m_dev = (uint32_t)M;
    if (t >= M) return;
    const int64_t c = off[t + 1] - off[t];
    k[t] = 0xffffu - (uint32_t)min(c, (int64_t)0xffff);
    v[t] = (uint32_t)t;
}


// capacities of a split render with `kcap` tile-list entries: segment slots
// (two or more per split tile, each split tile holds more than `split`
// entries), at most 65,535 and 512 MB of segment buffers; work items
static void split_caps(const umgs_frame* fr, int split, int64_t kcap, int64_t* slots_cap, int64_t* items_cap) {
    const int64_t px = (int64_t)fr->tile * fr->tile;
    *slots_cap = std::max<int64_t>(1, std::min<int64_t>({65535, 2 * kcap / split + 1, (512LL << 20) / (px * 20)}));
    *items_cap = fr->num_tiles + *slots_cap;
}

cudaError_t reserve_split(umgs_frame* fr, int split, int64_t kcap) {
    int64_t slots_cap, items_cap;
    split_caps(fr, split, kcap, &slots_cap, &items_cap);
    const int64_t px = (int64_t)fr->tile * fr->tile;
    cudaError_t e;
    if ((e = fr->split_items.reserve(sizeof(int4) * items_cap)) != cudaSuccess) return e;
    if ((e = fr->segbuf.reserve(sizeof(float4) * slots_cap * px)) != cudaSuccess) return e;
    if ((e = fr->seglast.reserve(sizeof(int32_t) * slots_cap * px)) != cudaSuccess) return e;
    for (DevBuf* b : {&fr->ord_k, &fr->ord_v, &fr->ord_k2, &fr->ord_v2})
        if ((e = b->reserve(sizeof(uint32_t) * items_cap)) != cudaSuccess) return e;
    return cudaSuccess;
}

// a render with the per-tile work split (FULL / DIRECT / MSAA_ALL /
// ENTITY_ALL / T_PRODUCT; no saved state, no depth)
static cudaError_t launch_split_composite(umgs_frame* fr, const umgs_render_opts& opts, float4* out, float te,
                                          int mode, cudaStream_t stream) {
    const int split = opts.split;
    const int64_t kcap = fr->nosync ? fr->key_capacity : fr->num_keys;
    int64_t slots_cap, items_cap;
    split_caps(fr, split, kcap, &slots_cap, &items_cap);
    cudaError_t e;
    if (!fr->capture && (e = reserve_split(fr, split, kcap)) != cudaSuccess) return e;
    const int64_t M = fr->num_tiles;
    const int tpc = fr->tiles_x * fr->tiles_y;
    unsigned* nitems = reinterpret_cast<unsigned*>(fr->status.as<int32_t>() + kStatusSplitWords);
    unsigned* nslots = nitems + 1;
    unsigned* work = nitems + 2;
    int4* items = fr->split_items.as<int4>();
    launch_pdl(split_plan_kernel, (unsigned)((M * 32 + 255) / 256), 256, 0, stream, fr->tile_off.as<int64_t>(),
               fr->ids, M, (uint32_t)fr->ng, split, items, nitems, nslots, (unsigned)slots_cap);
    const bool persist = opts.sched > 0;
    const uint32_t* order = nullptr;
    if (persist) {
        launch_pdl(item_order_keys_kernel, (unsigned)((items_cap + 255) / 256), 256, 0, stream, items, nitems,
                   items_cap, fr->ord_k.as<uint32_t>(), fr->ord_v.as<uint32_t>());
        uint32_t* rk = nullptr;
        uint32_t* rv = nullptr;
        if ((e = radix_sort_pairs(fr, fr->ord_k.as<uint32_t>(), fr->ord_v.as<uint32_t>(), fr->ord_k2.as<uint32_t>(),
                                  fr->ord_v2.as<uint32_t>(), nitems, items_cap, 16, &rk, &rv, stream)) != cudaSuccess)
            return e;
        order = rv;
    }
    const int nblk = opts.sched * fr->ctx->num_sms;
    float4* sb = fr->segbuf.as<float4>();
    int32_t* sl = fr->seglast.as<int32_t>();
#define UMGS_SPLIT(TSV, MV)                                                                                     \
    if (persist) launch_pdl(composite_items_persistent_kernel<TSV, MV>, nblk, Layout<TSV>::NT, 0, stream, order, work, \
        items, nitems, sb, sl, fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(),                          \
        fr->mixed ? fr->grec.as<GRec16>() : nullptr, fr->trec.as<TRec>(), fr->ng, fr->nt, fr->tiles_x, tpc,      \
        fr->W, fr->H, te, opts.bg[0], opts.bg[1], opts.bg[2], out, fr->last.as<int32_t>(),                       \
        fr->textab.as<DevTex>());                                                                               \
    else launch_pdl(composite_items_kernel<TSV, MV>, (unsigned)items_cap, Layout<TSV>::NT, 0, stream, items, nitems,  \
        sb, sl, fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(),                                       \
        fr->mixed ? fr->grec.as<GRec16>() : nullptr, fr->trec.as<TRec>(), fr->ng, fr->nt, fr->tiles_x, tpc,      \
        fr->W, fr->H, te, opts.bg[0], opts.bg[1], opts.bg[2], out, fr->last.as<int32_t>(),                       \
        fr->textab.as<DevTex>());                                                                               \
    launch_pdl(split_merge_kernel<TSV>, (unsigned)items_cap, 256, 0, stream, items, nitems, sb, sl, fr->tiles_x,  \
               tpc, fr->W, fr->H, te, opts.bg[0], opts.bg[1], opts.bg[2], out, fr->last.as<int32_t>())
#define UMGS_SPLIT_MODES(TSV)                                                                                   \
    if (mode == kModeTProduct) { UMGS_SPLIT(TSV, kModeTProduct); }                                             \
    else if (mode == UMGS_BLEND_DIRECT) { UMGS_SPLIT(TSV, UMGS_BLEND_DIRECT); }                                \
    else if (mode == UMGS_BLEND_MSAA_ALL) { UMGS_SPLIT(TSV, UMGS_BLEND_MSAA_ALL); }                            \
    else if (mode == UMGS_BLEND_ENTITY_ALL) { UMGS_SPLIT(TSV, UMGS_BLEND_ENTITY_ALL); }                        \
    else { UMGS_SPLIT(TSV, UMGS_BLEND_FULL); }
    if (fr->tile == 16) { UMGS_SPLIT_MODES(16) }
    else if (fr->tile == 8) { UMGS_SPLIT_MODES(8) }
    else { UMGS_SPLIT_MODES(32) }
#undef UMGS_SPLIT_MODES
#undef UMGS_SPLIT
    return cudaGetLastError();
}

cudaError_t launch_composite(umgs_frame* fr, const umgs_render_opts& opts, float* out_rgbt, cudaStream_t stream) {
    const float te = opts.t_eps > 0.f ? opts.t_eps : -1.f;
    float4* out = reinterpret_cast<float4*>(out_rgbt);
    const int ts = fr->tile;
    const unsigned M = (unsigned)fr->num_tiles;
    const int tpc = fr->tiles_x * fr->tiles_y;
    const int64_t npix = (int64_t)fr->ncams * fr->W * fr->H;
    const bool save = fr->saved;
    if (opts.split > 0 && !save && !fr->has_depth) {
        const int mode = (opts.blend_mode == UMGS_BLEND_FULL && (opts.flags & UMGS_RENDER_T_PRODUCT)) ? kModeTProduct
                                                                                                   : opts.blend_mode;
        return launch_split_composite(fr, opts, out, te, mode, stream);
    }
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
        launch_pdl(tile_order_keys_kernel, (M + 255) / 256, 256, 0, stream, fr->tile_off.as<int64_t>(), M, fr->ord_k.as<uint32_t>(),
                                                                     fr->ord_v.as<uint32_t>(), mdev);
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
    if (persist) launch_pdl(composite_persistent_kernel<TSV, SV, MV>, nblk, Layout<TSV>::NT, 0, stream, order, work, M,      \
        fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(), fr->mixed ? fr->grec.as<GRec16>() : nullptr,  \
        fr->trec.as<TRec>(), fr->ng,                                                                            \
        fr->nt, fr->tiles_x, tpc, fr->W, fr->H, te, opts.bg[0], opts.bg[1], opts.bg[2], out,                      \
        fr->last.as<int32_t>(), save ? fr->tfin.as<float>() : nullptr, save ? fr->ntri.as<int32_t>() : nullptr,   \
        save ? fr->stack.as<float4>() : nullptr, fr->stack_cap, npix, fr->status.as<int32_t>() + 2,             \
        fr->has_depth ? fr->depth.as<float>() : nullptr, fr->textab.as<DevTex>());                                                                                         \
    else launch_pdl(composite_kernel<TSV, SV, MV>, M, Layout<TSV>::NT, 0, stream,                                             \
        fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(), fr->mixed ? fr->grec.as<GRec16>() : nullptr,  \
        fr->trec.as<TRec>(), fr->ng,                                                                            \
        fr->nt, fr->tiles_x, tpc, fr->W, fr->H, te, opts.bg[0], opts.bg[1], opts.bg[2], out,                      \
        fr->last.as<int32_t>(), save ? fr->tfin.as<float>() : nullptr, save ? fr->ntri.as<int32_t>() : nullptr,   \
        save ? fr->stack.as<float4>() : nullptr, fr->stack_cap, npix, fr->status.as<int32_t>() + 2,             \
        fr->has_depth ? fr->depth.as<float>() : nullptr, fr->textab.as<DevTex>())
    // the saved (backward) form exists for FULL only
#define UMGS_MODES(TSV)                                                                                         \
    if (save) { UMGS_LAUNCH(TSV, true, UMGS_BLEND_FULL); }                                                      \
    else if (mode == kModeDepth) { UMGS_LAUNCH(TSV, false, kModeDepth); }                                       \
    else if (mode == kModeTProduct) { UMGS_LAUNCH(TSV, false, kModeTProduct); }                                 \
    else if (mode == UMGS_BLEND_DIRECT) { UMGS_LAUNCH(TSV, false, UMGS_BLEND_DIRECT); }                         \
    else if (mode == UMGS_BLEND_MSAA_ALL) { UMGS_LAUNCH(TSV, false, UMGS_BLEND_MSAA_ALL); }                     \
    else if (mode == UMGS_BLEND_ENTITY_ALL) { UMGS_LAUNCH(TSV, false, UMGS_BLEND_ENTITY_ALL); }                 \
    else { UMGS_LAUNCH(TSV, false, UMGS_BLEND_FULL); }
    const int mode = fr->has_depth ? kModeDepth
                     : (opts.blend_mode == UMGS_BLEND_FULL && (opts.flags & UMGS_RENDER_T_PRODUCT)) ? kModeTProduct
                                                                                                  : opts.blend_mode;
    if (ts == 16) { UMGS_MODES(16) }
    else if (ts == 8) { UMGS_MODES(8) }
    else { UMGS_MODES(32) }
#undef UMGS_MODES
#undef UMGS_LAUNCH
    return cudaGetLastError();
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
    // count[0]: evaluations of Gaussian records, count[1]: of triangle records
    const int tile = blockIdx.x;
    const int cam = tile / tiles_per_cam;
    const int lt = tile - cam * tiles_per_cam;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    int lx, ly;
    block_pixel<TS>(threadIdx.x, lx, ly);
    const int px = tx * TS + lx, py = ty * TS + ly;
    unsigned long long c = 0, ct = 0;
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
            const unsigned long long in = (px >= (int)(rx & 0xffff) && px <= (int)(rx >> 16) &&
                                           py >= (int)(ry & 0xffff) && py <= (int)(ry >> 16)) ? 1ull : 0ull;
            if (id < Ng) c += in;
            else ct += in;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        ct += __shfl_xor_sync(0xffffffffu, ct, o);
    }
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
    if ((threadIdx.x & 31) == 0 && ct) atomicAdd(count + 1, ct);
}

// Evaluation counts of the last render: (Gaussian, triangle) (pixel, record) pairs.
static umgs_status count_evaluations(const umgs_frame* fr, int64_t* g_evals, int64_t* t_evals, cudaStream_t stream) {
    cudaError_t e;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(fr->status.as<int32_t>() + kStatusEvalWords);
    if ((e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), stream)) != cudaSuccess)
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
    unsigned long long v[2] = {0, 0};
    if ((e = cudaMemcpyAsync(fr->ctx->pinned, cnt, sizeof(v), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return cuda_fail(fr->ctx, e, "reading the evaluation count");
    std::memcpy(v, fr->ctx->pinned, sizeof(v));
    *g_evals = (int64_t)v[0];
    *t_evals = (int64_t)v[1];
    return UMGS_OK;
}

umgs_status frame_evaluations(const umgs_frame* fr, int64_t* evals, cudaStream_t stream) {
    int64_t g = 0, t = 0;
    const umgs_status st = count_evaluations(fr, &g, &t, stream);
    *evals = g + t;
    return st;
}

umgs_status frame_stats(const umgs_frame* fr, umgs_frame_stats* out, cudaStream_t stream) {
    umgs_status st = count_evaluations(fr, &out->gaussian_evals, &out->triangle_evals, stream);
    if (st != UMGS_OK) return st;
    // fp64 conic count (status word 3) and the list length, read after the
    // evaluation count's synchronisation
    uint32_t w[4];
    cudaError_t e = cudaMemcpyAsync(fr->ctx->pinned, fr->status.ptr, sizeof(w), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(fr->ctx, e, "reading the frame status");
    std::memcpy(w, fr->ctx->pinned, sizeof(w));
    out->fp64_conics = (int64_t)w[3];
    int64_t k = 0;
    if ((e = cudaMemcpyAsync(&k, fr->tile_off.as<int64_t>() + fr->num_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost,
                             stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return cuda_fail(fr->ctx, e, "reading the list length");
    out->list_entries = k;
    return UMGS_OK;
}

}  // namespace umgs
