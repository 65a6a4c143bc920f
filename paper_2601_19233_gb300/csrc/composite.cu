// Compositor of the forward pass (Sec. 3.2, Eq. 1-2 and 7-11) and the
// evaluation count of a rendered frame.
//
// One CTA per tile, one thread per pixel: records of the tile's sorted list
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

constexpr int kBatch = 256;
// records staged per batch: 256, or 128 for 32x32 tiles (32 warps of lists)
template <int TS> struct BatchOf { static constexpr int value = TS == 32 ? 128 : 256; };

struct PixelState {
    float C[3];
    float T;
    float D, Wd;  // expected-depth mode: sum w z, sum w
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
// kModeDepth: FULL blending that also accumulates each pixel's expected depth
// sum w z / sum w (w the blend weight; z the Gaussian mean's camera depth or
// the triangle's perspective-correct depth at the pixel centre) into
// out_depth (+inf where nothing blends).
constexpr int kModeDepth = 5;

template <int TS, bool SAVE, int MODE>
__device__ __forceinline__ void composite_tile(
    int tile, float4 (*__restrict__ s_rec)[10], uint32_t* __restrict__ s_id, uint32_t* __restrict__ s_wmask,
    uint8_t* __restrict__ s_list,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off,
    const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need, float* __restrict__ out_depth, const DevTex* __restrict__ textab) {
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
    const uint32_t ng32 = (uint32_t)Ng;  // unified ids are 32-bit: a 32-bit compare per fragment
    const GRec* G = grec + (int64_t)cam * Ng;
    const GRec16* G16 = grec16 ? grec16 + (int64_t)cam * Ng : nullptr;
    const TRec* TR = trec + (int64_t)cam * Nt;
    const float qx = px + 0.5f, qy = py + 0.5f;
    const long long scx = (long long)px * 256 + 128, scy = (long long)py * 256 + 128;

    PixelState st;
    st.C[0] = st.C[1] = st.C[2] = 0.f;
    st.T = 1.f; st.Tin = 1.f; st.g_since = 1.f;
    st.D = 0.f; st.Wd = 0.f;
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
                s_rec[k][3] = make_float4(c.x, c.w, 0.f, 0.f);  // (b, Z)
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
                if (id < ng32) {
                    const float4 q1 = s_rec[k][1], q2 = s_rec[k][2];
                    if (pxf < q1.z || pxf > q1.w || pyf < q2.x || pyf > q2.y) continue;
                    const float4 q0 = s_rec[k][0];
                    const float dx = __fsub_rn(qx, q0.x), dy = __fsub_rn(qy, q0.y);
                    const float p2 = gauss_power2(q0.z, q0.w, q1.x, dx, dy);
                    const float alpha = fminf(kAlphaMax, __fmul_rn(q1.y, fast_exp2(p2)));
                    if (alpha < kAlphaMin) continue;
                    const float w = alpha * st.T;
                    st.C[0] += w * q2.z; st.C[1] += w * q2.w; st.C[2] += w * s_rec[k][3].x;
                    if (mode == kModeDepth) { st.D += w * s_rec[k][3].y; st.Wd += w; }
                    st.T = __fmaf_rn(-alpha, st.T, st.T);  // T (1 - alpha), one rounding
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
                        const float ia = __fdividef(1.f, area);  // (fast division: screen areas stay far from 2^126)
#pragma unroll
                        for (int e = 0; e < 3; ++e) wv[e] = fmaxf(lam[e] * ia, 0.f) * t.iz[e];
                    } else {
#pragma unroll
                        for (int e = 0; e < 3; ++e) wv[e] = (1.f / 3.f) * t.iz[e];
                    }
                    const float ws = wv[0] + wv[1] + wv[2];
                    float zt = 0.f;  // perspective-correct depth at the pixel centre (depth mode)
                    if (mode == kModeDepth) {
                        const float ls = area != 0.f ? fmaxf(lam[0] / area, 0.f) + fmaxf(lam[1] / area, 0.f) +
                                                           fmaxf(lam[2] / area, 0.f)
                                                     : 1.f;
                        zt = ws > 0.f ? ls / ws : 3.f / (t.iz[0] + t.iz[1] + t.iz[2]);
                    }
                    if (ws > 0.f) { const float is = __fdividef(1.f, ws); wv[0] *= is; wv[1] *= is; wv[2] *= is; }
                    else { wv[0] = wv[1] = wv[2] = 1.f / 3.f; }
                    float col[3];
                    if (t.tex > 0) {  // textured face: (u, v) interpolated like a colour, then sampled
                        const float tu = wv[0] * t.col[0] + wv[1] * t.col[2] + wv[2] * t.col[4];
                        const float tv = wv[0] * t.col[1] + wv[1] * t.col[3] + wv[2] * t.col[5];
                        sample_texture(textab[t.tex - 1], tu, tv, col);
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            col[c] = wv[0] * t.col[c] + wv[1] * t.col[3 + c] + wv[2] * t.col[6 + c];
                    }
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
                        if (mode == kModeDepth) { st.D += w * zt; st.Wd += w; }
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
        if (mode == kModeDepth) out_depth[pix] = st.Wd > 0.f ? st.D / st.Wd : __int_as_float(0x7f800000);
    }
}


// one CTA per tile (grid launch)
template <int TS, bool SAVE, int MODE>
__global__ void __launch_bounds__(TS * TS) composite_kernel(
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const GRec16* __restrict__ grec16, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need, float* __restrict__ out_depth, const DevTex* __restrict__ textab) {
    pdl_enter();
    constexpr int NB = BatchOf<TS>::value;
    __shared__ float4 s_rec[NB][10];
    __shared__ uint32_t s_id[NB];
    __shared__ uint32_t s_wmask[NB];
    __shared__ uint8_t s_list[(TS * TS / 32) * NB];
    composite_tile<TS, SAVE, MODE>(blockIdx.x, s_rec, s_id, s_wmask, s_list, ids, off, grec, grec16, trec, Ng, Nt, tiles_x, tiles_per_cam, W, H, t_eps, bg0, bg1, bg2, out, out_last, out_tfin, out_ntri, stack, cap, npix, need, out_depth, textab);
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
    int64_t npix, int32_t* __restrict__ need, float* __restrict__ out_depth, const DevTex* __restrict__ textab) {
    pdl_enter();
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
        composite_tile<TS, SAVE, MODE>((int)order[k], s_rec, s_id, s_wmask, s_list, ids, off, grec, grec16, trec, Ng, Nt, tiles_x, tiles_per_cam, W, H, t_eps, bg0, bg1, bg2, out, out_last, out_tfin, out_ntri, stack, cap, npix, need, out_depth, textab);
        __syncthreads();
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
    if (persist) launch_pdl(composite_persistent_kernel<TSV, SV, MV>, nblk, TSV * TSV, 0, stream, order, work, M,      \
        fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(), fr->mixed ? fr->grec.as<GRec16>() : nullptr,  \
        fr->trec.as<TRec>(), fr->ng,                                                                            \
        fr->nt, fr->tiles_x, tpc, fr->W, fr->H, te, opts.bg[0], opts.bg[1], opts.bg[2], out,                      \
        fr->last.as<int32_t>(), save ? fr->tfin.as<float>() : nullptr, save ? fr->ntri.as<int32_t>() : nullptr,   \
        save ? fr->stack.as<float4>() : nullptr, fr->stack_cap, npix, fr->status.as<int32_t>() + 2,             \
        fr->has_depth ? fr->depth.as<float>() : nullptr, fr->textab.as<DevTex>());                                                                                         \
    else launch_pdl(composite_kernel<TSV, SV, MV>, M, TSV * TSV, 0, stream,                                             \
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
