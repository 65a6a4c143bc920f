// Compositor of UMGS_RENDER_SOFT_EDGE renders: blend mode FULL (Sec. 3.2,
// Eq. 1-2 for Gaussians, Eq. 7-9 for entities of depth-adjacent triangles,
// background Eq. 10-11) with the binary sample coverage o^j of a triangle
// replaced by the soft-edge coverage c^j of soft_edge.cuh.  A triangle is a
// fragment of every pixel of its (widened) pixel rect.
//
// One CTA per tile, one thread per pixel; warp w owns an 8 x 4 block of the
// tile (block_pixel).  Records of the tile's sorted list are staged through
// shared memory in batches of kSoftBatch together with the mask of the warp
// blocks that can hold a fragment of each (Gaussian: its alpha >= 1/255
// octagon; triangle: its widened rect), and every warp walks only its own
// records, in list order.  SAVE keeps the state
// composite_bwd_kernel<TS, true> replays: final T, the number of triangle
// fragments and, per triangle fragment, the four sample transmittances before
// it scaled by T_in/4.
#include "internal.h"
#include "soft_edge.cuh"

namespace umgs {

constexpr int kSoftBatch = 128;

template <int TS, bool SAVE>
__global__ void __launch_bounds__(TS * TS) composite_soft_kernel(
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off, const GRec* __restrict__ grec,
    const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x, int tiles_per_cam, int W, int H,
    float t_eps, float bg0, float bg1, float bg2, float4* __restrict__ out, int32_t* __restrict__ out_last,
    float* __restrict__ out_tfin, int32_t* __restrict__ out_ntri, float4* __restrict__ stack, int cap,
    int64_t npix, int32_t* __restrict__ need, const DevTex* __restrict__ textab) {
    pdl_enter();
    constexpr int NT = TS * TS;
    __shared__ float4 s_rec[kSoftBatch][10];
    __shared__ SoftEdges s_edges[kSoftBatch];  // per triangle record: its coverage constants
    __shared__ uint32_t s_id[kSoftBatch];
    __shared__ uint32_t s_wmask[kSoftBatch];
    __shared__ uint8_t s_list[(NT / 32) * kSoftBatch];
    const int tile = blockIdx.x;
    const int cam = tile / tiles_per_cam;
    const int lt = tile - cam * tiles_per_cam;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    int lx, ly;
    block_pixel<TS>(threadIdx.x, lx, ly);
    const int px = tx * TS + lx, py = ty * TS + ly;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile_x0 = tx * TS, tile_y0 = ty * TS;
    const bool inside = px < W && py < H;
    const int64_t beg = off[tile], end = off[tile + 1];
    const GRec* G = grec + (int64_t)cam * Ng;
    const TRec* TR = trec + (int64_t)cam * Nt;
    const float qx = px + 0.5f, qy = py + 0.5f;
    const int64_t pix = ((int64_t)cam * H + py) * W + px;

    float C[3] = {0.f, 0.f, 0.f};
    float T = 1.f, Tin = 1.f;
    float tj[4] = {1.f, 1.f, 1.f, 1.f};
    bool in_ent = false, done = !inside;
    int last = 0, sp = 0;
    for (int64_t b0 = beg; b0 < end; b0 += kSoftBatch) {
        if (__syncthreads_count(done) == NT) break;
        const int n = (int)min((int64_t)kSoftBatch, end - b0);
        for (int k = threadIdx.x; k < n; k += NT) {
            const uint32_t id = ids[b0 + k];
            s_id[k] = id;
            uint32_t wm = 0u;  // not a record of this frame: no fragment
            if (id < Ng) {
                const float4* src = reinterpret_cast<const float4*>(G + id);
                const float4 a = src[0], b = src[1], c = src[2];
                s_rec[k][0] = a; s_rec[k][1] = b; s_rec[k][2] = c;
                const uint32_t rx = __float_as_uint(c.y), ry = __float_as_uint(c.z);
                wm = gauss_block_mask<TS>(a.x, a.y, a.z, a.w, b.x, b.y, (int)(rx & 0xffff), (int)(rx >> 16),
                                          (int)(ry & 0xffff), (int)(ry >> 16), tile_x0, tile_y0);
            } else if (id < Ng + Nt) {
                const float4* src = reinterpret_cast<const float4*>(TR + (id - Ng));
#pragma unroll
                for (int q = 0; q < 10; ++q) s_rec[k][q] = src[q];
                const TRec& tr = *reinterpret_cast<const TRec*>(&s_rec[k][0]);
                wm = box_block_mask<TS>((int)(tr.rx & 0xffff), (int)(tr.rx >> 16), (int)(tr.ry & 0xffff),
                                        (int)(tr.ry >> 16), tile_x0, tile_y0);
                soft_edges(tr, s_edges[k]);
            }
            s_wmask[k] = wm;
        }
        __syncthreads();
        // this warp's records of the batch, in order
        uint8_t* lst = s_list + warp * kSoftBatch;
        int cnt = 0;
        for (int c0 = 0; c0 < n; c0 += 32) {
            const bool mine = c0 + lane < n && ((s_wmask[c0 + lane] >> warp) & 1u);
            const unsigned bal = __ballot_sync(0xffffffffu, mine);
            if (mine) lst[cnt + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)(c0 + lane);
            cnt += __popc(bal);
        }
        __syncwarp();
        for (int li = 0; li < cnt && !done; ++li) {
            const int k = lst[li];
            const uint32_t id = s_id[k];
            if (id < Ng) {
                // Gaussian (Eq. 1-2), as in the binary-coverage compositor
                const float4 q0 = s_rec[k][0], q1 = s_rec[k][1], q2 = s_rec[k][2];
                const uint32_t rx = __float_as_uint(q2.y), ry = __float_as_uint(q2.z);
                if (px < (int)(rx & 0xffff) || px > (int)(rx >> 16) || py < (int)(ry & 0xffff) || py > (int)(ry >> 16))
                    continue;
                const float dx = __fsub_rn(qx, q0.x), dy = __fsub_rn(qy, q0.y);
                const float alpha = fminf(kAlphaMax, __fmul_rn(q1.y, fast_exp2(gauss_power2(q0.z, q0.w, q1.x, dx, dy))));
                if (alpha < kAlphaMin) continue;
                const float w = alpha * T;
                C[0] += w * q1.z; C[1] += w * q1.w; C[2] += w * q2.x;
                T = __fmaf_rn(-alpha, T, T);
                in_ent = false;
            } else {
                const TRec& t = *reinterpret_cast<const TRec*>(&s_rec[k][0]);
                if (px < (int)(t.rx & 0xffff) || px > (int)(t.rx >> 16) || py < (int)(t.ry & 0xffff) ||
                    py > (int)(t.ry >> 16))
                    continue;
                float cov[4];
                soft_coverage_staged(t, s_edges[k], qx, qy, cov);
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
#pragma unroll
                for (int e = 0; e < 3; ++e) wv[e] = (area != 0.f ? fmaxf(lam[e] / area, 0.f) : (1.f / 3.f)) * t.iz[e];
                const float ws = wv[0] + wv[1] + wv[2];
#pragma unroll
                for (int e = 0; e < 3; ++e) wv[e] = ws > 0.f ? wv[e] / ws : (1.f / 3.f);
                float col[3];
                if (t.tex > 0) {
                    const float tu = wv[0] * t.col[0] + wv[1] * t.col[2] + wv[2] * t.col[4];
                    const float tv = wv[0] * t.col[1] + wv[1] * t.col[3] + wv[2] * t.col[5];
                    sample_texture(textab[t.tex - 1], tu, tv, col);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) col[c] = wv[0] * t.col[c] + wv[1] * t.col[3 + c] + wv[2] * t.col[6 + c];
                }
                float a = t.const_alpha ? t.alpha[0] : (wv[0] * t.alpha[0] + wv[1] * t.alpha[1] + wv[2] * t.alpha[2]);
                a = fminf(fmaxf(a, 0.f), 1.f);
                // entity (Eq. 7-9) with c^j for o^j
                if (!in_ent) {
                    Tin = T;
                    tj[0] = tj[1] = tj[2] = tj[3] = 1.f;
                    in_ent = true;
                }
                if (SAVE) {
                    if (sp < cap) {
                        const float q = 0.25f * Tin;
                        stack[(int64_t)sp * npix + pix] = make_float4(q * tj[0], q * tj[1], q * tj[2], q * tj[3]);
                    }
                    ++sp;
                }
                const float O = 0.25f * ((cov[0] * tj[0] + cov[1] * tj[1]) + (cov[2] * tj[2] + cov[3] * tj[3]));
                const float w = Tin * O * a;
                C[0] += w * col[0]; C[1] += w * col[1]; C[2] += w * col[2];
#pragma unroll
                for (int j = 0; j < 4; ++j) tj[j] *= 1.f - a * cov[j];
                T = Tin * (0.25f * ((tj[0] + tj[1]) + (tj[2] + tj[3])));
            }
            last = (int)(b0 - beg) + k + 1;
            if (T < t_eps) done = true;
        }
    }
    if (inside) {
        out[pix] = make_float4(C[0] + T * bg0, C[1] + T * bg1, C[2] + T * bg2, T);
        if (out_last) out_last[pix] = last | (T < t_eps ? (int)0x80000000u : 0);
        if (SAVE) {
            out_tfin[pix] = T;
            out_ntri[pix] = sp;
            if (sp > cap) atomicMax(need, sp);
        }
    }
}

cudaError_t launch_soft_composite(umgs_frame* fr, const umgs_render_opts& opts, float* out_rgbt,
                                  cudaStream_t stream) {
    const float te = opts.t_eps > 0.f ? opts.t_eps : -1.f;
    float4* out = reinterpret_cast<float4*>(out_rgbt);
    const unsigned M = (unsigned)fr->num_tiles;
    const int tpc = fr->tiles_x * fr->tiles_y;
    const int64_t npix = (int64_t)fr->ncams * fr->W * fr->H;
    const bool save = fr->saved;
    if (save) {
        cudaError_t e = cudaMemsetAsync(fr->status.as<int32_t>() + 2, 0, sizeof(int32_t), stream);
        if (e != cudaSuccess) return e;
    }
#define UMGS_LAUNCH(TSV, SV)                                                                                      \
    launch_pdl(composite_soft_kernel<TSV, SV>, M, TSV * TSV, 0, stream, fr->ids, fr->tile_off.as<int64_t>(),      \
               fr->grec.as<GRec>(), fr->trec.as<TRec>(), fr->ng, fr->nt, fr->tiles_x, tpc, fr->W, fr->H, te,      \
               opts.bg[0], opts.bg[1], opts.bg[2], out, fr->last.as<int32_t>(),                                   \
               save ? fr->tfin.as<float>() : nullptr, save ? fr->ntri.as<int32_t>() : nullptr,                    \
               save ? fr->stack.as<float4>() : nullptr, fr->stack_cap, npix, fr->status.as<int32_t>() + 2,        \
               fr->textab.as<DevTex>())
    if (fr->tile == 16) { if (save) UMGS_LAUNCH(16, true); else UMGS_LAUNCH(16, false); }
    else if (fr->tile == 8) { if (save) UMGS_LAUNCH(8, true); else UMGS_LAUNCH(8, false); }
    else { if (save) UMGS_LAUNCH(32, true); else UMGS_LAUNCH(32, false); }
#undef UMGS_LAUNCH
    return cudaGetLastError();
}

}  // namespace umgs
