// Backward pass of the single-pass composite (gradient of Sec. 3.2, Eq. 1-2, 7-9).
//
// composite_bwd  one CTA per tile, one thread per pixel.  The tile's sorted
//                list is replayed from the pixel's last blended fragment back
//                to the front, in batches staged through shared memory.
//                With U = dL/dT after the current fragment (U starts at
//                g.bg + dL/dT_final):
//                  Gaussian k:  T_k = T_{k+1} / (1 - alpha_k)   (alpha <= 0.99)
//                               dL/dalpha_k = T_k (g.c_k - U)
//                               U <- alpha_k g.c_k + (1 - alpha_k) U
//                  triangle k of an entity, per sub-sample stream j with
//                  s_j = T_in t_k^j / 4 read from the saved stack and
//                  a_j = o_k^j alpha_k:
//                               dL/da_j = s_j (g.c_k - U_j)
//                               U_j <- a_j g.c_k + (1 - a_j) U_j
//                  entering an entity from its back end sets U_j = U, leaving
//                  it through its front sets U = mean_j U_j; no division is
//                  needed for triangles, so opaque coverage is exact.
//                Per fragment the derivatives w.r.t. the projected record
//                (Gaussian: u, v, conic, opacity, RGB; triangle: unsnapped
//                screen positions, depths, vertex colours and alphas through
//                the perspective-correct interpolation) are reduced across
//                the warp (recursive halving, one component per lane) and
//                added to shared-memory accumulators of the batch, which are
//                flushed with one global atomic per record and component.
// project_gaussians_bwd / setup_triangles_bwd
//                chain rule from the records to the inputs (EWA projection,
//                covariance from quaternion and scale, SH colour), summed
//                over cameras.
#include <cmath>

#include "internal.h"
#include "soft_edge.cuh"

namespace umgs {

// Records per batch and the dynamic shared memory of a CTA: the records
// (160 B), their gradient accumulators (22 floats), ids, warp masks and the
// per-warp lists.  16x16 tiles stage 192 records (51 KB: four CTAs per SM).
template <int TS> struct BwdBatch { static constexpr int value = TS == 16 ? 192 : 128; };
template <int TS> constexpr int bwd_smem_bytes() {
    return BwdBatch<TS>::value * (160 + 88 + 4 + 4 + TS * TS / 32) + 4 * (TS * TS / 32) + 16;
}
// (soft-edge replays: then the records' coverage constants, SoftEdges, 16-byte aligned)
template <int TS> constexpr int bwd_soft_edges_offset() { return (bwd_smem_bytes<TS>() + 15) & ~15; }
template <int TS, bool SOFT> constexpr int bwd_smem_bytes_for() {
    return SOFT ? bwd_soft_edges_offset<TS>() + BwdBatch<TS>::value * (int)sizeof(SoftEdges) : bwd_smem_bytes<TS>();
}
constexpr float kLn2 = 0.6931471805599453f;

// Warp sum of V values per lane (V = 16 or 32) by recursive halving: at each
// step every lane keeps one half of its values, sends the other half to its
// partner and adds what it receives, so V - 1 shuffles (plus one for V = 16)
// replace the 5 V of one butterfly per value.  On return v[0] of lane L holds
// the warp sum of value L (V = 32) or of value L >> 1 (V = 16; both lanes of a
// pair hold it).
template <int V>
__device__ __forceinline__ void warp_sum_transpose(float (&v)[V], int lane) {
    static_assert(V == 16 || V == 32, "V");
#pragma unroll
    for (int half = V / 2, o = 16; half >= 1; half >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = up ? v[i] : v[i + half];
            const float keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    if (V == 16) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// 16x16 tiles: registers capped for four resident CTAs per SM (32 warps),
// which hides the per-batch barriers better than the three of an uncapped build
// SOFT: replay of a UMGS_RENDER_SOFT_EDGE render (soft-edge sample coverage
// c^j; a triangle is a fragment wherever its rect holds the pixel), with the
// gradient through c^j added to the vertex screen positions.
// (the soft replay holds more live values: two CTAs per SM, no register cap spills)
template <int TS, bool SOFT>
__global__ void __launch_bounds__(TS * TS, TS == 16 ? (SOFT ? 2 : 4) : 1) composite_bwd_kernel(
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off,
    const GRec* __restrict__ grec, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float bg0,
    float bg1, float bg2, const float4* __restrict__ dout, const int32_t* __restrict__ last,
    const float* __restrict__ tfin, const int32_t* __restrict__ ntri, const float4* __restrict__ stack, int64_t npix,
    float* __restrict__ ggrad, float* __restrict__ tgrad) {
    pdl_enter();
    constexpr int NT = TS * TS;
    constexpr int NW = NT / 32;
    constexpr int kBatchB = BwdBatch<TS>::value;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 (*s_rec)[10] = reinterpret_cast<float4 (*)[10]>(smem);
    float (*s_acc)[22] = reinterpret_cast<float (*)[22]>(smem + kBatchB * 160);  // per record gradient
    uint32_t* s_id = reinterpret_cast<uint32_t*>(smem + kBatchB * (160 + 88));
    uint32_t* s_wmask = s_id + kBatchB;
    int* s_wmax = reinterpret_cast<int*>(s_wmask + kBatchB);
    int& s_max = s_wmax[NW];
    uint8_t* s_list = reinterpret_cast<uint8_t*>(s_wmax + NW + 4);
    SoftEdges* s_edges = reinterpret_cast<SoftEdges*>(smem + bwd_soft_edges_offset<TS>());  // (SOFT only)
    const int tile = blockIdx.x;
    const int cam = tile / tiles_per_cam;
    const int lt = tile - cam * tiles_per_cam;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    int lx, ly;
    block_pixel<TS>(threadIdx.x, lx, ly);
    const int px = tx * TS + lx, py = ty * TS + ly;
    const bool inside = px < W && py < H;
    const int64_t beg = off[tile];
    const GRec* G = grec + (int64_t)cam * Ng;
    const TRec* TR = trec + (int64_t)cam * Nt;
    const float qx = px + 0.5f, qy = py + 0.5f;
    const long long scx = (long long)px * 256 + 128, scy = (long long)py * 256 + 128;
    const int64_t pix = ((int64_t)cam * H + py) * W + px;
    const int lane = threadIdx.x & 31;

    int nlast = 0, sp = 0;
    float T = 1.f, U = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
    if (inside) {
        nlast = last[pix] & 0x7fffffff;  // bit 31: stopped at T < t_eps
        sp = ntri[pix];
        T = tfin[pix];
        const float4 d = dout[pix];
        gr = d.x; gg = d.y; gb = d.z;
        U = gr * bg0 + gg * bg1 + gb * bg2 + d.w;
    }
    float Uj[4] = {0.f, 0.f, 0.f, 0.f};
    bool in_ent = false;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, nlast);
    {
        int wm = nlast;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wm = max(wm, __shfl_xor_sync(0xffffffffu, wm, o));
        if (lane == 0) s_wmax[warp] = wm;
    }
    __syncthreads();
    const int maxlast = s_max;
    const int wmaxlast = s_wmax[warp];
    const int tile_x0 = tx * TS, tile_y0 = ty * TS;

    for (int bend = maxlast; bend > 0; bend -= kBatchB) {
        const int b0 = max(0, bend - kBatchB);
        const int n = bend - b0;
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += NT) {
            const uint32_t id = ids[beg + b0 + k];
            s_id[k] = id;
            if (id >= Ng + Nt) {
                s_wmask[k] = 0u;  // not a record of this frame
            } else if (id < Ng) {
                const float4* src = reinterpret_cast<const float4*>(G + id);
                const float4 a = src[0], q1 = src[1], c = src[2];
                s_rec[k][0] = a; s_rec[k][1] = q1; s_rec[k][2] = c;
                const uint32_t rx = __float_as_uint(c.y), ry = __float_as_uint(c.z);
                s_wmask[k] = gauss_block_mask<TS>(a.x, a.y, a.z, a.w, q1.x, q1.y, (int)(rx & 0xffff), (int)(rx >> 16),
                                                  (int)(ry & 0xffff), (int)(ry >> 16), tile_x0, tile_y0);
            } else {
                const float4* src = reinterpret_cast<const float4*>(TR + (id - Ng));
#pragma unroll
                for (int q = 0; q < 10; ++q) s_rec[k][q] = src[q];
                const TRec& tr = *reinterpret_cast<const TRec*>(&s_rec[k][0]);
                s_wmask[k] = box_block_mask<TS>((int)(tr.rx & 0xffff), (int)(tr.rx >> 16), (int)(tr.ry & 0xffff),
                                                (int)(tr.ry >> 16), tile_x0, tile_y0);
                if (SOFT) soft_edges(tr, s_edges[k]);
            }
#pragma unroll
            for (int e = 0; e < 22; ++e) s_acc[k][e] = 0.f;
        }
        __syncthreads();
        // this warp's records of the batch (in order; replayed back to front)
        uint8_t* lst = s_list + warp * kBatchB;
        int cnt = 0;
        for (int c0 = 0; c0 < n; c0 += 32) {
            const bool mine = c0 + lane < n && b0 + c0 + lane < wmaxlast && ((s_wmask[c0 + lane] >> warp) & 1u);
            const unsigned bal = __ballot_sync(0xffffffffu, mine);
            if (mine) lst[cnt + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)(c0 + lane);
            cnt += __popc(bal);
        }
        __syncwarp();
        for (int li = cnt - 1; li >= 0; --li) {
            const int k = lst[li];
            const int pos = b0 + k;
            const bool active = inside && pos < nlast;
            const uint32_t id = s_id[k];
            if (id < Ng) {
                // ---- Gaussian fragment
                const float4 q0 = s_rec[k][0], q1 = s_rec[k][1], q2 = s_rec[k][2];
                const uint32_t rx = __float_as_uint(q2.y), ry = __float_as_uint(q2.z);
                const bool inrect = px >= (int)(rx & 0xffff) && px <= (int)(rx >> 16) && py >= (int)(ry & 0xffff) &&
                                    py <= (int)(ry >> 16);
                const float dx = __fsub_rn(qx, q0.x), dy = __fsub_rn(qy, q0.y);
                const float p2 = gauss_power2(q0.z, q0.w, q1.x, dx, dy);
                const float Gv = fast_exp2(p2);
                const float ag = __fmul_rn(q1.y, Gv);
                const float alpha = fminf(kAlphaMax, ag);
                const bool contrib = active && inrect && alpha >= kAlphaMin;
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = 0.f;
                if (contrib) {
                    if (in_ent) { U = 0.25f * ((Uj[0] + Uj[1]) + (Uj[2] + Uj[3])); in_ent = false; }
                    // (fast division: alpha <= 0.99 keeps the divisor in [0.01, 1])
                    const float Tk = __fdividef(T, 1.f - alpha);
                    const float gc = gr * q1.z + gg * q1.w + gb * q2.x;
                    const float dalpha = Tk * (gc - U);
                    const float w = Tk * alpha;
                    v[6] = w * gr; v[7] = w * gg; v[8] = w * gb;
                    U = alpha * gc + (1.f - alpha) * U;
                    T = Tk;
                    if (ag <= kAlphaMax) {
                        const float dpow = dalpha * alpha;
                        float ca, cb, cc;
                            factor_conic(q0.z, q0.w, q1.x, ca, cb, cc);
                            const float A = -2.f * kLn2 * ca, B = -kLn2 * cb, C = -2.f * kLn2 * cc;
                        v[0] = dpow * (A * dx + B * dy);
                        v[1] = dpow * (B * dx + C * dy);
                        v[2] = -0.5f * dpow * dx * dx;
                        v[3] = -dpow * dx * dy;
                        v[4] = -0.5f * dpow * dy * dy;
                        v[5] = dalpha * Gv;
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    warp_sum_transpose<16>(v, lane);
                    if ((lane & 1) == 0 && lane < 18 && v[0] != 0.f) atomicAdd(&s_acc[k][lane >> 1], v[0]);
                }
            } else {
                // ---- triangle fragment
                const TRec& t = *reinterpret_cast<const TRec*>(&s_rec[k][0]);
                int mask = 0;
                float cov[4] = {0.f, 0.f, 0.f, 0.f}, sg = 0.f, il[3], sgm[4][3];
                if (SOFT) {
                    if (active && px >= (int)(t.rx & 0xffff) && px <= (int)(t.rx >> 16) &&
                        py >= (int)(t.ry & 0xffff) && py <= (int)(t.ry >> 16)) {
                        mask = 0xf;  // a fragment of this pixel
                        soft_coverage_staged_bwd(t, s_edges[k], qx, qy, cov, sg, il, sgm);
                    }
                } else if (active) {
                    long long E[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) E[e] = (long long)t.A[e] * scx + (long long)t.B[e] * scy + t.C[e];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int sdx = sample_dx(j), sdy = sample_dy(j);
                        bool in = true;
#pragma unroll
                        for (int e = 0; e < 3; ++e) in = in && (E[e] + (long long)(t.A[e] * sdx + t.B[e] * sdy) >= 0);
                        mask |= in ? (1 << j) : 0;
                    }
                }
                const bool cover = mask != 0;
                float v[32];
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] = 0.f;
                if (cover) {
                    if (!in_ent) { Uj[0] = Uj[1] = Uj[2] = Uj[3] = U; in_ent = true; }
                    // replayed coverage equals the forward's, so sp > 0 here; the
                    // guard keeps a mismatch from reading outside the stack
                    float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (sp > 0) { --sp; s4 = stack[(int64_t)sp * npix + pix]; }
                    const float s[4] = {s4.x, s4.y, s4.z, s4.w};
                    // attributes, as in the forward
                    float e3[3];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const int a = (m + 1) % 3, b = (m + 2) % 3;
                        e3[m] = (t.u[a] - qx) * (t.v[b] - qy) - (t.u[b] - qx) * (t.v[a] - qy);
                    }
                    const float area = e3[0] + e3[1] + e3[2];
                    float lam[3], lh[3], wv[3];
                    const float ia = area != 0.f ? 1.f / area : 0.f;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        lam[m] = area != 0.f ? e3[m] * ia : (1.f / 3.f);
                        lh[m] = fmaxf(lam[m], 0.f);
                        wv[m] = lh[m] * t.iz[m];
                    }
                    const float ws = wv[0] + wv[1] + wv[2];
                    float w[3];
                    if (ws > 0.f) { const float is = 1.f / ws; w[0] = wv[0] * is; w[1] = wv[1] * is; w[2] = wv[2] * is; }
                    else { w[0] = w[1] = w[2] = 1.f / 3.f; }
                    float col[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) col[c] = w[0] * t.col[c] + w[1] * t.col[3 + c] + w[2] * t.col[6 + c];
                    const float araw = t.const_alpha ? t.alpha[0] : (w[0] * t.alpha[0] + w[1] * t.alpha[1] + w[2] * t.alpha[2]);
                    const float alpha = fminf(fmaxf(araw, 0.f), 1.f);
                    const float gc = gr * col[0] + gg * col[1] + gb * col[2];
                    float dalpha = 0.f, wsum = 0.f;
                    float dcov[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (SOFT) {  // o^j = c^j in [0, 1]
                            const float cj = cov[j];
                            dcov[j] = s[j] * alpha * (gc - Uj[j]);
                            dalpha += s[j] * cj * (gc - Uj[j]);
                            wsum += s[j] * cj * alpha;
                            Uj[j] = alpha * cj * gc + (1.f - alpha * cj) * Uj[j];
                        } else if ((mask >> j) & 1) {
                            dalpha += s[j] * (gc - Uj[j]);
                            wsum += s[j] * alpha;
                            Uj[j] = alpha * gc + (1.f - alpha) * Uj[j];
                        }
                    }
                    if (SOFT) soft_coverage_grad(t, qx, qy, cov, sg, il, sgm, dcov, &v[0], &v[3]);
                    T = (s[0] + s[1]) + (s[2] + s[3]);
                    const float dc[3] = {wsum * gr, wsum * gg, wsum * gb};
                    const float dar = (araw >= 0.f && araw <= 1.f) ? dalpha : 0.f;
                    // colour and alpha to vertices / weights
                    float dw[3];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        v[9 + 3 * m] = w[m] * dc[0];
                        v[10 + 3 * m] = w[m] * dc[1];
                        v[11 + 3 * m] = w[m] * dc[2];
                        dw[m] = t.col[3 * m] * dc[0] + t.col[3 * m + 1] * dc[1] + t.col[3 * m + 2] * dc[2];
                    }
                    if (t.const_alpha == 0) {
#pragma unroll
                        for (int m = 0; m < 3; ++m) { v[18 + m] = w[m] * dar; dw[m] += t.alpha[m] * dar; }
                    } else if (t.const_alpha == 1) {
                        v[18] = dar;
                    }
                    if (ws > 0.f) {
                        const float sdw = w[0] * dw[0] + w[1] * dw[1] + w[2] * dw[2];
                        const float is = 1.f / ws;
                        float dlam[3];
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            const float dwh = (dw[m] - sdw) * is;
                            const float diz = dwh * lh[m];
                            v[6 + m] = -diz * t.iz[m] * t.iz[m];
                            dlam[m] = (area != 0.f && lam[m] >= 0.f) ? dwh * t.iz[m] : 0.f;
                        }
                        if (area != 0.f) {
                            const float sl = dlam[0] * e3[0] + dlam[1] * e3[1] + dlam[2] * e3[2];
#pragma unroll
                            for (int m = 0; m < 3; ++m) {
                                const float de = dlam[m] * ia - sl * ia * ia;
                                const int a = (m + 1) % 3, b = (m + 2) % 3;
                                v[a] += de * (t.v[b] - qy);
                                v[3 + b] += de * (t.u[a] - qx);
                                v[b] -= de * (t.v[a] - qy);
                                v[3 + a] -= de * (t.u[b] - qx);
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, cover)) {
                    warp_sum_transpose<32>(v, lane);
                    if (lane < 21 && v[0] != 0.f) atomicAdd(&s_acc[k][lane], v[0]);
                }
            }
        }
        __syncthreads();
        // one global atomic per (record, component) of this tile's batch
        for (int k = threadIdx.x; k < n; k += NT) {
            const uint32_t id = s_id[k];
            if (id < Ng) {
                float* dst = ggrad + ((int64_t)cam * Ng + id) * 12;
#pragma unroll
                for (int e = 0; e < 9; ++e)
                    if (s_acc[k][e] != 0.f) atomicAdd(dst + e, s_acc[k][e]);
            } else {
                float* dst = tgrad + ((int64_t)cam * Nt + (id - Ng)) * 24;
#pragma unroll
                for (int e = 0; e < 21; ++e)
                    if (s_acc[k][e] != 0.f) atomicAdd(dst + e, s_acc[k][e]);
            }
        }
    }
}

// ---- two pixels per thread (binary coverage) ---------------------------------
// The replay of composite_bwd_kernel<TS, false> with the forward compositor's
// layout: warp w owns the 8 x 8 block (w % (TS/8), w / (TS/8)), lane l the
// pixels (l % 8, l / 8) and (l % 8, l / 8 + 4).  The arithmetic per pixel is
// unchanged; the two pixels' derivatives of a record are added in the lane
// before the warp reduction, so a record costs one reduction per 64 pixels.
template <int TS> struct Bwd2 {
    static constexpr int NT = TS * TS / 2;
    static constexpr int NW = NT / 32;
    static constexpr int NB = 128;  // records per batch
    static constexpr int SMEM = NB * (160 + 88 + 4 + 4) + NW * NB + 4 * NW + 16;
};

template <int TS>
__global__ void __launch_bounds__(Bwd2<TS>::NT, TS == 16 ? 5 : 1) composite_bwd2_kernel(
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ off,
    const GRec* __restrict__ grec, const TRec* __restrict__ trec, int64_t Ng, int64_t Nt, int tiles_x,
    int tiles_per_cam, int W, int H, float bg0,
    float bg1, float bg2, const float4* __restrict__ dout, const int32_t* __restrict__ last,
    const float* __restrict__ tfin, const int32_t* __restrict__ ntri, const float4* __restrict__ stack, int64_t npix,
    float* __restrict__ ggrad, float* __restrict__ tgrad) {
    pdl_enter();
    constexpr int NT = Bwd2<TS>::NT, NW = Bwd2<TS>::NW, kBatchB = Bwd2<TS>::NB;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 (*s_rec)[10] = reinterpret_cast<float4 (*)[10]>(smem);
    float (*s_acc)[22] = reinterpret_cast<float (*)[22]>(smem + kBatchB * 160);  // per record gradient
    uint32_t* s_id = reinterpret_cast<uint32_t*>(smem + kBatchB * (160 + 88));
    uint32_t* s_wmask = s_id + kBatchB;
    int* s_wmax = reinterpret_cast<int*>(s_wmask + kBatchB);
    int& s_max = s_wmax[NW];
    uint8_t* s_list = reinterpret_cast<uint8_t*>(s_wmax + NW + 4);
    const int tile = blockIdx.x;
    const int cam = tile / tiles_per_cam;
    const int lt = tile - cam * tiles_per_cam;
    const int ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = (warp % (TS / 8)) * 8 + (lane & 7);
    const int ly0 = (warp / (TS / 8)) * 8 + (lane >> 3);
    const int px = tx * TS + lx;
    const int64_t beg = off[tile];
    const GRec* G = grec + (int64_t)cam * Ng;
    const TRec* TR = trec + (int64_t)cam * Nt;
    const float qx = px + 0.5f;
    const long long scx = (long long)px * 256 + 128;

    int nlast[2], sp[2];
    float T[2], U[2], gr[2], gg[2], gb[2], Uj[2][4], qy[2];
    bool in_ent[2], inside[2];
    int64_t pix[2];
    long long scy[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int py = ty * TS + ly0 + 4 * p;
        qy[p] = py + 0.5f;
        scy[p] = (long long)py * 256 + 128;
        inside[p] = px < W && py < H;
        pix[p] = ((int64_t)cam * H + py) * W + px;
        nlast[p] = 0; sp[p] = 0;
        T[p] = 1.f; U[p] = 0.f; gr[p] = gg[p] = gb[p] = 0.f;
        if (inside[p]) {
            nlast[p] = last[pix[p]] & 0x7fffffff;  // bit 31: stopped at T < t_eps
            sp[p] = ntri[pix[p]];
            T[p] = tfin[pix[p]];
            const float4 d = dout[pix[p]];
            gr[p] = d.x; gg[p] = d.y; gb[p] = d.z;
            U[p] = d.x * bg0 + d.y * bg1 + d.z * bg2 + d.w;
        }
        Uj[p][0] = Uj[p][1] = Uj[p][2] = Uj[p][3] = 0.f;
        in_ent[p] = false;
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const int mylast = max(nlast[0], nlast[1]);
    atomicMax(&s_max, mylast);
    {
        int wm = mylast;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wm = max(wm, __shfl_xor_sync(0xffffffffu, wm, o));
        if (lane == 0) s_wmax[warp] = wm;
    }
    __syncthreads();
    const int maxlast = s_max;
    const int wmaxlast = s_wmax[warp];
    const int tile_x0 = tx * TS, tile_y0 = ty * TS;

    for (int bend = maxlast; bend > 0; bend -= kBatchB) {
        const int b0 = max(0, bend - kBatchB);
        const int n = bend - b0;
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += NT) {
            const uint32_t id = ids[beg + b0 + k];
            s_id[k] = id;
            if (id >= Ng + Nt) {
                s_wmask[k] = 0u;  // not a record of this frame
            } else if (id < Ng) {
                const float4* src = reinterpret_cast<const float4*>(G + id);
                const float4 a = src[0], q1 = src[1], c = src[2];
                s_rec[k][0] = a; s_rec[k][1] = q1; s_rec[k][2] = c;
                const uint32_t rx = __float_as_uint(c.y), ry = __float_as_uint(c.z);
                s_wmask[k] = gauss_block_mask<TS, 8>(a.x, a.y, a.z, a.w, q1.x, q1.y, (int)(rx & 0xffff),
                                                     (int)(rx >> 16), (int)(ry & 0xffff), (int)(ry >> 16), tile_x0,
                                                     tile_y0);
            } else {
                const float4* src = reinterpret_cast<const float4*>(TR + (id - Ng));
#pragma unroll
                for (int q = 0; q < 10; ++q) s_rec[k][q] = src[q];
                const TRec& tr = *reinterpret_cast<const TRec*>(&s_rec[k][0]);
                s_wmask[k] = box_block_mask<TS, 8>((int)(tr.rx & 0xffff), (int)(tr.rx >> 16), (int)(tr.ry & 0xffff),
                                                   (int)(tr.ry >> 16), tile_x0, tile_y0);
            }
#pragma unroll
            for (int e = 0; e < 22; ++e) s_acc[k][e] = 0.f;
        }
        __syncthreads();
        // this warp's records of the batch (in order; replayed back to front)
        uint8_t* lst = s_list + warp * kBatchB;
        int cnt = 0;
        for (int c0 = 0; c0 < n; c0 += 32) {
            const bool mine = c0 + lane < n && b0 + c0 + lane < wmaxlast && ((s_wmask[c0 + lane] >> warp) & 1u);
            const unsigned bal = __ballot_sync(0xffffffffu, mine);
            if (mine) lst[cnt + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)(c0 + lane);
            cnt += __popc(bal);
        }
        __syncwarp();
        for (int li = cnt - 1; li >= 0; --li) {
            const int k = lst[li];
            const int pos = b0 + k;
            const uint32_t id = s_id[k];
            if (id < Ng) {
                // ---- Gaussian fragment
                const float4 q0 = s_rec[k][0], q1 = s_rec[k][1], q2 = s_rec[k][2];
                const uint32_t rx = __float_as_uint(q2.y), ry = __float_as_uint(q2.z);
                const bool inx = px >= (int)(rx & 0xffff) && px <= (int)(rx >> 16);
                const float dx = __fsub_rn(qx, q0.x);
                // (the conic of the record, once for both pixels)
                float ca, cb, cc;
                factor_conic(q0.z, q0.w, q1.x, ca, cb, cc);
                const float A = -2.f * kLn2 * ca, B = -kLn2 * cb, C = -2.f * kLn2 * cc;
                const float Adx = A * dx, Bdx = B * dx;
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = 0.f;
                bool any = false;
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int py = ty * TS + ly0 + 4 * p;
                    const bool inrect = inx && py >= (int)(ry & 0xffff) && py <= (int)(ry >> 16);
                    const float dy = __fsub_rn(qy[p], q0.y);
                    const float p2 = gauss_power2(q0.z, q0.w, q1.x, dx, dy);
                    const float Gv = fast_exp2(p2);
                    const float ag = __fmul_rn(q1.y, Gv);
                    const float alpha = fminf(kAlphaMax, ag);
                    const bool contrib = inside[p] && pos < nlast[p] && inrect && alpha >= kAlphaMin;
                    if (contrib) {
                        any = true;
                        if (in_ent[p]) {
                            U[p] = 0.25f * ((Uj[p][0] + Uj[p][1]) + (Uj[p][2] + Uj[p][3]));
                            in_ent[p] = false;
                        }
                        // (fast division: alpha <= 0.99 keeps the divisor in [0.01, 1])
                        const float Tk = __fdividef(T[p], 1.f - alpha);
                        const float gc = gr[p] * q1.z + gg[p] * q1.w + gb[p] * q2.x;
                        const float dalpha = Tk * (gc - U[p]);
                        const float w = Tk * alpha;
                        v[6] += w * gr[p]; v[7] += w * gg[p]; v[8] += w * gb[p];
                        U[p] = alpha * gc + (1.f - alpha) * U[p];
                        T[p] = Tk;
                        if (ag <= kAlphaMax) {
                            const float dpow = dalpha * alpha;
                            v[0] += dpow * (Adx + B * dy);
                            v[1] += dpow * (Bdx + C * dy);
                            v[2] += -0.5f * dpow * dx * dx;
                            v[3] += -dpow * dx * dy;
                            v[4] += -0.5f * dpow * dy * dy;
                            v[5] += dalpha * Gv;
                        }
                    }
                }
                if (__any_sync(0xffffffffu, any)) {
                    warp_sum_transpose<16>(v, lane);
                    if ((lane & 1) == 0 && lane < 18 && v[0] != 0.f) atomicAdd(&s_acc[k][lane >> 1], v[0]);
                }
            } else {
                // ---- triangle fragment
                const TRec& t = *reinterpret_cast<const TRec*>(&s_rec[k][0]);
                float v[32];
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] = 0.f;
                bool any = false;
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    int mask = 0;
                    if (inside[p] && pos < nlast[p]) {
                        long long E[3];
#pragma unroll
                        for (int e = 0; e < 3; ++e)
                            E[e] = (long long)t.A[e] * scx + (long long)t.B[e] * scy[p] + t.C[e];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int sdx = sample_dx(j), sdy = sample_dy(j);
                            bool in = true;
#pragma unroll
                            for (int e = 0; e < 3; ++e)
                                in = in && (E[e] + (long long)(t.A[e] * sdx + t.B[e] * sdy) >= 0);
                            mask |= in ? (1 << j) : 0;
                        }
                    }
                    if (mask == 0) continue;
                    any = true;
                    const float qyp = qy[p];
                    if (!in_ent[p]) { Uj[p][0] = Uj[p][1] = Uj[p][2] = Uj[p][3] = U[p]; in_ent[p] = true; }
                    // replayed coverage equals the forward's, so sp > 0 here; the
                    // guard keeps a mismatch from reading outside the stack
                    float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (sp[p] > 0) { --sp[p]; s4 = stack[(int64_t)sp[p] * npix + pix[p]]; }
                    const float s[4] = {s4.x, s4.y, s4.z, s4.w};
                    // attributes, as in the forward
                    float e3[3];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const int a = (m + 1) % 3, b = (m + 2) % 3;
                        e3[m] = (t.u[a] - qx) * (t.v[b] - qyp) - (t.u[b] - qx) * (t.v[a] - qyp);
                    }
                    const float area = e3[0] + e3[1] + e3[2];
                    float lam[3], lh[3], wv[3];
                    const float ia = area != 0.f ? 1.f / area : 0.f;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        lam[m] = area != 0.f ? e3[m] * ia : (1.f / 3.f);
                        lh[m] = fmaxf(lam[m], 0.f);
                        wv[m] = lh[m] * t.iz[m];
                    }
                    const float ws = wv[0] + wv[1] + wv[2];
                    float w[3];
                    if (ws > 0.f) { const float is = 1.f / ws; w[0] = wv[0] * is; w[1] = wv[1] * is; w[2] = wv[2] * is; }
                    else { w[0] = w[1] = w[2] = 1.f / 3.f; }
                    float col[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) col[c] = w[0] * t.col[c] + w[1] * t.col[3 + c] + w[2] * t.col[6 + c];
                    const float araw = t.const_alpha ? t.alpha[0] : (w[0] * t.alpha[0] + w[1] * t.alpha[1] + w[2] * t.alpha[2]);
                    const float alpha = fminf(fmaxf(araw, 0.f), 1.f);
                    const float gc = gr[p] * col[0] + gg[p] * col[1] + gb[p] * col[2];
                    float dalpha = 0.f, wsum = 0.f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if ((mask >> j) & 1) {
                            dalpha += s[j] * (gc - Uj[p][j]);
                            wsum += s[j] * alpha;
                            Uj[p][j] = alpha * gc + (1.f - alpha) * Uj[p][j];
                        }
                    }
                    T[p] = (s[0] + s[1]) + (s[2] + s[3]);
                    const float dc[3] = {wsum * gr[p], wsum * gg[p], wsum * gb[p]};
                    const float dar = (araw >= 0.f && araw <= 1.f) ? dalpha : 0.f;
                    // colour and alpha to vertices / weights
                    float dw[3];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        v[9 + 3 * m] += w[m] * dc[0];
                        v[10 + 3 * m] += w[m] * dc[1];
                        v[11 + 3 * m] += w[m] * dc[2];
                        dw[m] = t.col[3 * m] * dc[0] + t.col[3 * m + 1] * dc[1] + t.col[3 * m + 2] * dc[2];
                    }
                    if (t.const_alpha == 0) {
#pragma unroll
                        for (int m = 0; m < 3; ++m) { v[18 + m] += w[m] * dar; dw[m] += t.alpha[m] * dar; }
                    } else if (t.const_alpha == 1) {
                        v[18] += dar;
                    }
                    if (ws > 0.f) {
                        const float sdw = w[0] * dw[0] + w[1] * dw[1] + w[2] * dw[2];
                        const float is = 1.f / ws;
                        float dlam[3];
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            const float dwh = (dw[m] - sdw) * is;
                            const float diz = dwh * lh[m];
                            v[6 + m] += -diz * t.iz[m] * t.iz[m];
                            dlam[m] = (area != 0.f && lam[m] >= 0.f) ? dwh * t.iz[m] : 0.f;
                        }
                        if (area != 0.f) {
                            const float sl = dlam[0] * e3[0] + dlam[1] * e3[1] + dlam[2] * e3[2];
#pragma unroll
                            for (int m = 0; m < 3; ++m) {
                                const float de = dlam[m] * ia - sl * ia * ia;
                                const int a = (m + 1) % 3, b = (m + 2) % 3;
                                v[a] += de * (t.v[b] - qyp);
                                v[3 + b] += de * (t.u[a] - qx);
                                v[b] -= de * (t.v[a] - qyp);
                                v[3 + a] -= de * (t.u[b] - qx);
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, any)) {
                    warp_sum_transpose<32>(v, lane);
                    if (lane < 21 && v[0] != 0.f) atomicAdd(&s_acc[k][lane], v[0]);
                }
            }
        }
        __syncthreads();
        // one global atomic per (record, component) of this tile's batch
        for (int k = threadIdx.x; k < n; k += NT) {
            const uint32_t id = s_id[k];
            if (id < Ng) {
                float* dst = ggrad + ((int64_t)cam * Ng + id) * 12;
#pragma unroll
                for (int e = 0; e < 9; ++e)
                    if (s_acc[k][e] != 0.f) atomicAdd(dst + e, s_acc[k][e]);
            } else if (id < Ng + Nt) {
                float* dst = tgrad + ((int64_t)cam * Nt + (id - Ng)) * 24;
#pragma unroll
                for (int e = 0; e < 21; ++e)
                    if (s_acc[k][e] != 0.f) atomicAdd(dst + e, s_acc[k][e]);
            }
        }
    }
}

// ---- records -> Gaussian parameters ---------------------------------------

// Real SH basis (Condon-Shortley phase, index l*l + (m + l)) of the unit
// direction (x, y, z) and its partial derivatives with respect to x, y, z.
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float (&Y)[(DEG + 1) * (DEG + 1)],
                                              float (&gx)[(DEG + 1) * (DEG + 1)], float (&gy)[(DEG + 1) * (DEG + 1)],
                                              float (&gz)[(DEG + 1) * (DEG + 1)]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
#pragma unroll
    for (int k = 0; k < K; ++k) { Y[k] = 0.f; gx[k] = gy[k] = gz[k] = 0.f; }
    Y[0] = 0.28209479177387814f;
    if constexpr (DEG > 0) {
        const float c1 = 0.4886025119029199f;
        Y[1] = -c1 * y; gy[1] = -c1;
        Y[2] = c1 * z;  gz[2] = c1;
        Y[3] = -c1 * x; gx[3] = -c1;
    }
    if constexpr (DEG > 1) {
        const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.5462742152960396f;
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = a * x * y;   gx[4] = a * y; gy[4] = a * x;
        Y[5] = -a * y * z;  gy[5] = -a * z; gz[5] = -a * y;
        Y[6] = b * (2.f * zz - xx - yy); gx[6] = -2.f * b * x; gy[6] = -2.f * b * y; gz[6] = 4.f * b * z;
        Y[7] = -a * x * z;  gx[7] = -a * z; gz[7] = -a * x;
        Y[8] = c * (xx - yy); gx[8] = 2.f * c * x; gy[8] = -2.f * c * y;
        if constexpr (DEG > 2) {
            const float d0 = -0.5900435899266435f, d1 = 2.890611442640554f, d2 = -0.4570457994644658f,
                        d3 = 0.3731763325901154f, d5 = 1.445305721320277f;
            Y[9] = d0 * y * (3.f * xx - yy);  gx[9] = 6.f * d0 * x * y; gy[9] = d0 * (3.f * xx - 3.f * yy);
            Y[10] = d1 * x * y * z;           gx[10] = d1 * y * z; gy[10] = d1 * x * z; gz[10] = d1 * x * y;
            Y[11] = d2 * y * (4.f * zz - xx - yy); gx[11] = -2.f * d2 * x * y; gy[11] = d2 * (4.f * zz - xx - 3.f * yy); gz[11] = 8.f * d2 * y * z;
            Y[12] = d3 * z * (2.f * zz - 3.f * xx - 3.f * yy); gx[12] = -6.f * d3 * x * z; gy[12] = -6.f * d3 * y * z; gz[12] = d3 * (6.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = d2 * x * (4.f * zz - xx - yy); gx[13] = d2 * (4.f * zz - 3.f * xx - yy); gy[13] = -2.f * d2 * x * y; gz[13] = 8.f * d2 * x * z;
            Y[14] = d5 * z * (xx - yy);       gx[14] = 2.f * d5 * x * z; gy[14] = -2.f * d5 * y * z; gz[14] = d5 * (xx - yy);
            Y[15] = d0 * x * (xx - 3.f * yy); gx[15] = d0 * (3.f * xx - 3.f * yy); gy[15] = -6.f * d0 * x * y;
        }
    }
}

// Gradient of one camera's colour (SH of the view direction dir = mean -
// camera centre, clamped at 0 after the +0.5 offset) with respect to the
// coefficients (added to dsh) and to the mean (added to dmu).  coef and dsh
// point at this Gaussian's 3K coefficients and gradients in shared memory.
template <int DEG>
__device__ __forceinline__ void sh_grad(const float* coef, float dx, float dy, float dz, const float drgb[3],
                                        float* dsh, float dmu[3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    // the direction is normalised as in the forward shading
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    const float x = dx * inv, y = dy * inv, z = dz * inv;
    float Y[K], gx[K], gy[K], gz[K];
    sh_basis_grad<DEG>(x, y, z, Y, gx, gy, gz);
    float gdx = 0.f, gdy = 0.f, gdz = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) acc = fmaf(coef[3 * k + c], Y[k], acc);
        const float g = (acc + 0.5f < 0.f) ? 0.f : drgb[c];  // clamped channel: no gradient
#pragma unroll
        for (int k = 0; k < K; ++k) {
            dsh[3 * k + c] += g * Y[k];
            const float gc = g * coef[3 * k + c];
            gdx += gc * gx[k]; gdy += gc * gy[k]; gdz += gc * gz[k];
        }
    }
    if (DEG > 0) {
        // project onto the tangent plane of the unit direction, divide by |dir|
        const float r = gdx * x + gdy * y + gdz * z;
        dmu[0] += (gdx - r * x) * inv; dmu[1] += (gdy - r * y) * inv; dmu[2] += (gdz - r * z) * inv;
    }
}

// One thread per Gaussian, 32 Gaussians per warp, kProjBwdWarps warps per
// CTA.  The warp's SH coefficients are staged through shared memory
// (coalesced in; rows padded to an odd length so the per-thread rows are
// conflict-free), the SH gradients are accumulated in a second such buffer
// and leave coalesced.  Every output element is written.
constexpr int kProjBwdWarps = 2;

template <int DEG>
__global__ void __launch_bounds__(kProjBwdWarps * 32) project_gaussians_bwd_kernel(
    const float* __restrict__ means, const float* __restrict__ quats, const float* __restrict__ scales,
    const void* __restrict__ sh, int sh_dtype, const float* __restrict__ cov3d, int64_t N,
    const DevCam* __restrict__ cams, int ncams, const BinInfo* __restrict__ bin, int64_t ntot,
    const float* __restrict__ ggrad, float* __restrict__ d_means, float* __restrict__ d_quats,
    float* __restrict__ d_scales, float* __restrict__ d_opac, float* __restrict__ d_sh, float* __restrict__ d_cov) {
    pdl_enter();
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int K3 = 3 * K;
    constexpr int KP = K3 | 1;
    __shared__ float s_sh[kProjBwdWarps][2][32 * KP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wbase = ((int64_t)blockIdx.x * kProjBwdWarps + warp) * 32;
    if (wbase >= N) return;  // whole warp (only warp-level synchronisation below)
    const int nw = N - wbase < 32 ? (int)(N - wbase) : 32;
    float* buf = s_sh[warp][0];
    float* gbuf = s_sh[warp][1];
    if (sh_dtype == UMGS_BF16) {
        const unsigned short* p = static_cast<const unsigned short*>(sh) + wbase * K3;
        for (int j = lane; j < nw * K3; j += 32) {
            const int g = j / K3;
            buf[g * KP + (j - g * K3)] = __uint_as_float(((unsigned int)p[j]) << 16);
        }
    } else {
        const float* p = static_cast<const float*>(sh) + wbase * K3;
        for (int j = lane; j < nw * K3; j += 32) {
            const int g = j / K3;
            buf[g * KP + (j - g * K3)] = p[j];
        }
    }
    const int64_t i = wbase + lane;
    const bool live = lane < nw;
    float* dsh = gbuf + lane * KP;
#pragma unroll
    for (int k = 0; k < K3; ++k) dsh[k] = 0.f;
    __syncwarp();
    if (live) {
        const float* coef = buf + lane * KP;
        const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
        // 3D covariance and its factors
        float S[9], Rq[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, s3[3] = {0, 0, 0}, qn[4] = {1, 0, 0, 0}, qlen = 1.f;
        if (cov3d) {
            const float* c = cov3d + 6 * i;
            S[0] = c[0]; S[1] = c[1]; S[2] = c[2]; S[3] = c[1]; S[4] = c[3]; S[5] = c[4]; S[6] = c[2]; S[7] = c[4]; S[8] = c[5];
        } else {
            const float4 q4 = reinterpret_cast<const float4*>(quats)[i];
            float w = q4.x, x = q4.y, y = q4.z, z = q4.w;
            qlen = sqrtf(w * w + x * x + y * y + z * z);
            if (qlen > 0.f) { w /= qlen; x /= qlen; y /= qlen; z /= qlen; } else { w = 1.f; x = y = z = 0.f; qlen = 1.f; }
            qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
            Rq[0] = 1.f - 2.f * (y * y + z * z); Rq[1] = 2.f * (x * y - w * z); Rq[2] = 2.f * (x * z + w * y);
            Rq[3] = 2.f * (x * y + w * z); Rq[4] = 1.f - 2.f * (x * x + z * z); Rq[5] = 2.f * (y * z - w * x);
            Rq[6] = 2.f * (x * z - w * y); Rq[7] = 2.f * (y * z + w * x); Rq[8] = 1.f - 2.f * (x * x + y * y);
            s3[0] = scales[3 * i]; s3[1] = scales[3 * i + 1]; s3[2] = scales[3 * i + 2];
            float M[9];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) M[3 * a + b] = Rq[3 * a + b] * s3[b];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) S[3 * a + b] = M[3 * a] * M[3 * b] + M[3 * a + 1] * M[3 * b + 1] + M[3 * a + 2] * M[3 * b + 2];
        }
        float dmu[3] = {0, 0, 0}, dS[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, dop = 0.f;
        for (int cam = 0; cam < ncams; ++cam) {
            if (!bin[(int64_t)cam * ntot + i].valid) continue;
            const float4* gv4 = reinterpret_cast<const float4*>(ggrad + ((int64_t)cam * N + i) * 12);
            const float4 g0 = gv4[0], g1 = gv4[1], g2 = gv4[2];
            const float du = g0.x, dv = g0.y, dA = g0.z, dB = g0.w, dC = g1.x, dO = g1.y;
            const float drgb[3] = {g1.z, g1.w, g2.x};
            if (du == 0.f && dv == 0.f && dA == 0.f && dB == 0.f && dC == 0.f && dO == 0.f && drgb[0] == 0.f &&
                drgb[1] == 0.f && drgb[2] == 0.f)
                continue;
            const DevCam& Cm = cams[cam];
            const float* R = Cm.R;
            const float X = R[0] * mx + R[1] * my + R[2] * mz + Cm.t[0];
            const float Yc = R[3] * mx + R[4] * my + R[5] * mz + Cm.t[1];
            const float Z = R[6] * mx + R[7] * my + R[8] * mz + Cm.t[2];
            const float iz = 1.f / Z, iz2 = iz * iz;
            const float limx = 1.3f * ((float)Cm.W / (2.f * Cm.fx)), limy = 1.3f * ((float)Cm.H / (2.f * Cm.fy));
            const float txz = X * iz, tyz = Yc * iz;
            const bool cx_in = txz >= -limx && txz <= limx, cy_in = tyz >= -limy && tyz <= limy;
            const float xc = fminf(limx, fmaxf(-limx, txz)) * Z, yc = fminf(limy, fmaxf(-limy, tyz)) * Z;
            const float J00 = Cm.fx * iz, J11 = Cm.fy * iz, J02 = -Cm.fx * xc * iz2, J12 = -Cm.fy * yc * iz2;
            float T0[3], T1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) { T0[k] = J00 * R[k] + J02 * R[6 + k]; T1[k] = J11 * R[3 + k] + J12 * R[6 + k]; }
            float U0[3], U1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                U0[k] = T0[0] * S[k] + T0[1] * S[3 + k] + T0[2] * S[6 + k];
                U1[k] = T1[0] * S[k] + T1[1] * S[3 + k] + T1[2] * S[6 + k];
            }
            const float a = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2] + 0.3f;
            const float b = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
            const float c = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2] + 0.3f;
            // conic Q = inv([[a b][b c]])
            float QA, QB, QC;
            const float det = a * c - b * b;
            if (det < kConicFp64 * a * c) {
                const double dd = (double)a * c - (double)b * b;
                QA = (float)(c / dd); QB = (float)(-b / dd); QC = (float)(a / dd);
            } else {
                const float id = 1.f / det;
                QA = c * id; QB = -b * id; QC = a * id;
            }
            // dL/dSigma2D = -Q G_Q Q with G_Q = [[dA, dB/2],[dB/2, dC]]
            const float g01 = 0.5f * dB;
            const float m00 = QA * dA + QB * g01, m01 = QA * g01 + QB * dC;
            const float m10 = QB * dA + QC * g01, m11 = QB * g01 + QC * dC;
            const float G00 = -(m00 * QA + m01 * QB), G01 = -(m00 * QB + m01 * QC), G11 = -(m10 * QB + m11 * QC);
            // Sigma2D = T S T^T: dS3 = T^T G T, dT = 2 G T S
            float GT0[3], GT1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) { GT0[k] = G00 * T0[k] + G01 * T1[k]; GT1[k] = G01 * T0[k] + G11 * T1[k]; }
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) dS[3 * p + q] += T0[p] * GT0[q] + T1[p] * GT1[q];
            float dT0[3], dT1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dT0[k] = 2.f * (GT0[0] * S[k] + GT0[1] * S[3 + k] + GT0[2] * S[6 + k]);
                dT1[k] = 2.f * (GT1[0] * S[k] + GT1[1] * S[3 + k] + GT1[2] * S[6 + k]);
            }
            // T = J R: dJ = dT R^T (only J00, J02, J11, J12 are variables)
            const float dJ00 = dT0[0] * R[0] + dT0[1] * R[1] + dT0[2] * R[2];
            const float dJ02 = dT0[0] * R[6] + dT0[1] * R[7] + dT0[2] * R[8];
            const float dJ11 = dT1[0] * R[3] + dT1[1] * R[4] + dT1[2] * R[5];
            const float dJ12 = dT1[0] * R[6] + dT1[1] * R[7] + dT1[2] * R[8];
            float dX = du * Cm.fx * iz, dY = dv * Cm.fy * iz;
            float dZ = -du * Cm.fx * X * iz2 - dv * Cm.fy * Yc * iz2;
            dZ += -dJ00 * Cm.fx * iz2 - dJ11 * Cm.fy * iz2;
            if (cx_in) { dX += -dJ02 * Cm.fx * iz2; dZ += dJ02 * 2.f * Cm.fx * X * iz2 * iz; }
            else { dZ += dJ02 * Cm.fx * copysignf(limx, txz) * iz2; }
            if (cy_in) { dY += -dJ12 * Cm.fy * iz2; dZ += dJ12 * 2.f * Cm.fy * Yc * iz2 * iz; }
            else { dZ += dJ12 * Cm.fy * copysignf(limy, tyz) * iz2; }
#pragma unroll
            for (int k = 0; k < 3; ++k) dmu[k] += R[k] * dX + R[3 + k] * dY + R[6 + k] * dZ;
            dop += dO;
            if (drgb[0] != 0.f || drgb[1] != 0.f || drgb[2] != 0.f)
                sh_grad<DEG>(coef, mx - Cm.campos[0], my - Cm.campos[1], mz - Cm.campos[2], drgb, dsh, dmu);
        }
        if (d_means) { d_means[3 * i] = dmu[0]; d_means[3 * i + 1] = dmu[1]; d_means[3 * i + 2] = dmu[2]; }
        if (d_opac) d_opac[i] = dop;
        // symmetrise dS (a function of the symmetric Sigma)
        const float G3[9] = {dS[0], 0.5f * (dS[1] + dS[3]), 0.5f * (dS[2] + dS[6]),
                             0.5f * (dS[1] + dS[3]), dS[4], 0.5f * (dS[5] + dS[7]),
                             0.5f * (dS[2] + dS[6]), 0.5f * (dS[5] + dS[7]), dS[8]};
        if (cov3d) {
            if (d_cov) {
                float* o = d_cov + 6 * i;
                o[0] = G3[0]; o[1] = 2.f * G3[1]; o[2] = 2.f * G3[2]; o[3] = G3[4]; o[4] = 2.f * G3[5]; o[5] = G3[8];
            }
        } else {
            // Sigma = M M^T, M = Rq diag(s): dM = 2 G3 M
            float M[9], dM[9];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) M[3 * a + b] = Rq[3 * a + b] * s3[b];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    dM[3 * a + b] = 2.f * (G3[3 * a] * M[b] + G3[3 * a + 1] * M[3 + b] + G3[3 * a + 2] * M[6 + b]);
            if (d_scales)
#pragma unroll
                for (int b = 0; b < 3; ++b) d_scales[3 * i + b] = dM[b] * Rq[b] + dM[3 + b] * Rq[3 + b] + dM[6 + b] * Rq[6 + b];
            if (d_quats) {
                float Gr[9];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) Gr[3 * a + b] = dM[3 * a + b] * s3[b];
                const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
                float dq[4];
                dq[0] = 2.f * (-z * Gr[1] + y * Gr[2] + z * Gr[3] - x * Gr[5] - y * Gr[6] + x * Gr[7]);
                dq[1] = 2.f * (y * Gr[1] + z * Gr[2] + y * Gr[3] - 2.f * x * Gr[4] - w * Gr[5] + z * Gr[6] + w * Gr[7] - 2.f * x * Gr[8]);
                dq[2] = 2.f * (-2.f * y * Gr[0] + x * Gr[1] + w * Gr[2] + x * Gr[3] + z * Gr[5] - w * Gr[6] + z * Gr[7] - 2.f * y * Gr[8]);
                dq[3] = 2.f * (-2.f * z * Gr[0] - w * Gr[1] + x * Gr[2] + w * Gr[3] - 2.f * z * Gr[4] + y * Gr[5] + x * Gr[6] + y * Gr[7]);
                const float dd = dq[0] * w + dq[1] * x + dq[2] * y + dq[3] * z;
                const float il = 1.f / qlen;
                reinterpret_cast<float4*>(d_quats)[i] =
                    make_float4((dq[0] - dd * w) * il, (dq[1] - dd * x) * il, (dq[2] - dd * y) * il, (dq[3] - dd * z) * il);
            }
        }
    }
    if (!d_sh) return;
    __syncwarp();
    float* o = d_sh + wbase * K3;
    for (int j = lane; j < nw * K3; j += 32) {
        const int g = j / K3;
        o[j] = gbuf[g * KP + (j - g * K3)];
    }
}

__global__ void __launch_bounds__(256) setup_triangles_bwd_kernel(
    const float* __restrict__ verts, const int32_t* __restrict__ faces, const float* __restrict__ valpha,
    const float* __restrict__ falpha, int64_t nf, int64_t tri_base, int64_t nt_total, int64_t id_base,
    const DevCam* __restrict__ cams, int ncams, const BinInfo* __restrict__ bin, int64_t ntot,
    const float* __restrict__ tgrad, float* __restrict__ d_verts, float* __restrict__ d_vcolor,
    float* __restrict__ d_valpha, float* __restrict__ d_falpha) {
    pdl_enter();
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int vid[3] = {faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]};
    float dfa = 0.f;
    for (int cam = 0; cam < ncams; ++cam) {
        if (!bin[(int64_t)cam * ntot + id_base + f].valid) continue;
        const float* gv = tgrad + ((int64_t)cam * nt_total + tri_base + f) * 24;
        const DevCam& Cm = cams[cam];
        const float* R = Cm.R;
        for (int k = 0; k < 3; ++k) {
            const float du = gv[k], dv = gv[3 + k], dZ0 = gv[6 + k];
            const float* P = verts + 3 * (int64_t)vid[k];
            if (d_verts && (du != 0.f || dv != 0.f || dZ0 != 0.f)) {
                const float X = R[0] * P[0] + R[1] * P[1] + R[2] * P[2] + Cm.t[0];
                const float Y = R[3] * P[0] + R[4] * P[1] + R[5] * P[2] + Cm.t[1];
                const float Z = R[6] * P[0] + R[7] * P[1] + R[8] * P[2] + Cm.t[2];
                const float iz = 1.f / Z;
                const float dX = du * Cm.fx * iz, dY = dv * Cm.fy * iz;
                const float dZ = dZ0 - du * Cm.fx * X * iz * iz - dv * Cm.fy * Y * iz * iz;
                for (int a = 0; a < 3; ++a)
                    atomicAdd(d_verts + 3 * (int64_t)vid[k] + a, R[a] * dX + R[3 + a] * dY + R[6 + a] * dZ);
            }
            if (d_vcolor)
                for (int c = 0; c < 3; ++c) {
                    const float g = gv[9 + 3 * k + c];
                    if (g != 0.f) atomicAdd(d_vcolor + 3 * (int64_t)vid[k] + c, g);
                }
            if (!falpha && valpha && d_valpha && gv[18 + k] != 0.f) atomicAdd(d_valpha + vid[k], gv[18 + k]);
        }
        if (falpha) dfa += gv[18];
    }
    if (falpha && d_falpha) d_falpha[f] = dfa;
}

static inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

umgs_status render_backward(umgs_ctx* ctx, umgs_frame* fr, const umgs_gaussians* g, const umgs_mesh* meshes,
                            int32_t nmeshes, const float* dL_drgbt, const umgs_gaussian_grads* gg,
                            const umgs_mesh_grads* mg, cudaStream_t stream) {
    cudaError_t e;
#define UMGS_TRY(x)                                                                  \
    do {                                                                             \
        e = (x);                                                                     \
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, #x); } \
        if (e != cudaSuccess) return cuda_fail(ctx, e, #x);                         \
    } while (0)
    const int64_t Ng = fr->ng, Nt = fr->nt, Ntot = Ng + Nt;
    const int64_t npix = (int64_t)fr->ncams * fr->W * fr->H;
    // saved stack large enough?  (the forward records the largest need)
    int32_t need = 0;
    UMGS_TRY(cudaMemcpyAsync(ctx->pinned, fr->status.as<int32_t>() + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    UMGS_TRY(cudaStreamSynchronize(stream));
    need = (int32_t)(ctx->pinned[0] & 0xffffffff);
    if (need > fr->stack_cap) {
        fr->stack_cap = need + need / 4 + 1;
        UMGS_TRY(fr->stack.reserve(sizeof(float4) * npix * fr->stack_cap));
        UMGS_TRY(fr->rerun_out.reserve(sizeof(float4) * npix));
        if (fr->opts.flags & UMGS_RENDER_SOFT_EDGE)
            UMGS_TRY(launch_soft_composite(fr, fr->opts, fr->rerun_out.as<float>(), stream));
        else
            UMGS_TRY(launch_composite(fr, fr->opts, fr->rerun_out.as<float>(), stream));
    }
    UMGS_TRY(fr->ggrad.reserve(sizeof(float) * 12 * std::max<int64_t>(1, Ng * fr->ncams)));
    UMGS_TRY(fr->tgrad.reserve(sizeof(float) * 24 * std::max<int64_t>(1, Nt * fr->ncams)));
    if (Ng > 0) UMGS_TRY(cudaMemsetAsync(fr->ggrad.ptr, 0, sizeof(float) * 12 * Ng * fr->ncams, stream));
    if (Nt > 0) UMGS_TRY(cudaMemsetAsync(fr->tgrad.ptr, 0, sizeof(float) * 24 * Nt * fr->ncams, stream));
    {
        StageTimer tm(ctx, UMGS_STAGE_BACKWARD_COMPOSITE, stream);
        const unsigned M = (unsigned)fr->num_tiles;
        const int tpc = fr->tiles_x * fr->tiles_y;
        const float4* dout = reinterpret_cast<const float4*>(dL_drgbt);
#define UMGS_LAUNCH(TSV, SOFTV)                                                                                  \
        /* per call: the attribute belongs to the current device */                                         \
        UMGS_TRY(cudaFuncSetAttribute(composite_bwd_kernel<TSV, SOFTV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (bwd_smem_bytes_for<TSV, SOFTV>())));                                      \
        launch_pdl(composite_bwd_kernel<TSV, SOFTV>, M, TSV * TSV, (bwd_smem_bytes_for<TSV, SOFTV>()), stream,           \
            fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(), fr->trec.as<TRec>(), Ng, Nt,               \
            fr->tiles_x, tpc, fr->W, fr->H, fr->bg[0], fr->bg[1], fr->bg[2], dout, fr->last.as<int32_t>(),         \
            fr->tfin.as<float>(), fr->ntri.as<int32_t>(), fr->stack.as<float4>(), npix, fr->ggrad.as<float>(),     \
            fr->tgrad.as<float>())
#define UMGS_LAUNCH2(TSV)                                                                                       \
        UMGS_TRY(cudaFuncSetAttribute(composite_bwd2_kernel<TSV>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                      Bwd2<TSV>::SMEM));                                                          \
        launch_pdl(composite_bwd2_kernel<TSV>, M, Bwd2<TSV>::NT, Bwd2<TSV>::SMEM, stream,                           \
            fr->ids, fr->tile_off.as<int64_t>(), fr->grec.as<GRec>(), fr->trec.as<TRec>(), Ng, Nt,               \
            fr->tiles_x, tpc, fr->W, fr->H, fr->bg[0], fr->bg[1], fr->bg[2], dout, fr->last.as<int32_t>(),         \
            fr->tfin.as<float>(), fr->ntri.as<int32_t>(), fr->stack.as<float4>(), npix, fr->ggrad.as<float>(),     \
            fr->tgrad.as<float>())
        const bool soft = (fr->opts.flags & UMGS_RENDER_SOFT_EDGE) != 0;
        if (fr->tile == 16) { if (soft) { UMGS_LAUNCH(16, true); } else { UMGS_LAUNCH2(16); } }
        else if (fr->tile == 8) { if (soft) { UMGS_LAUNCH(8, true); } else { UMGS_LAUNCH2(8); } }
        else { if (soft) { UMGS_LAUNCH(32, true); } else { UMGS_LAUNCH2(32); } }
#undef UMGS_LAUNCH2
#undef UMGS_LAUNCH
        UMGS_TRY(cudaGetLastError());
    }
    StageTimer tm(ctx, UMGS_STAGE_BACKWARD_PROJECT, stream);
    if (Ng > 0 && gg) {
        // every element of the requested outputs is written by the kernel
#define UMGS_LAUNCH(D)                                                                                          \
        launch_pdl(project_gaussians_bwd_kernel<D>, grid_for(Ng, kProjBwdWarps * 32), kProjBwdWarps * 32, 0, stream,                                 \
            g->means, g->quats, g->scales, g->sh, g->sh_dtype, g->cov3d, Ng, fr->cams.as<DevCam>(), fr->ncams,      \
            fr->bin.as<BinInfo>(), Ntot, fr->ggrad.as<float>(), gg->means, g->cov3d ? nullptr : gg->quats,         \
            g->cov3d ? nullptr : gg->scales, gg->opacities, gg->sh, g->cov3d ? gg->cov3d : nullptr)
        switch (g->sh_degree) {
            case 0: UMGS_LAUNCH(0); break;
            case 1: UMGS_LAUNCH(1); break;
            case 2: UMGS_LAUNCH(2); break;
            default: UMGS_LAUNCH(3); break;
        }
#undef UMGS_LAUNCH
        UMGS_TRY(cudaGetLastError());
    }
    int64_t tri_base = 0;
    for (int m = 0; m < nmeshes; ++m) {
        const umgs_mesh& me = meshes[m];
        if (mg) {
            const umgs_mesh_grads& o = mg[m];
            if (o.verts) UMGS_TRY(cudaMemsetAsync(o.verts, 0, sizeof(float) * 3 * me.nv, stream));
            if (o.vcolor) UMGS_TRY(cudaMemsetAsync(o.vcolor, 0, sizeof(float) * 3 * me.nv, stream));
            if (o.valpha) UMGS_TRY(cudaMemsetAsync(o.valpha, 0, sizeof(float) * me.nv, stream));
            if (o.falpha) UMGS_TRY(cudaMemsetAsync(o.falpha, 0, sizeof(float) * me.nf, stream));
            if (me.nf > 0) {
                launch_pdl(setup_triangles_bwd_kernel, grid_for(me.nf, 256), 256, 0, stream, 
                    me.verts, me.faces, me.valpha, me.falpha, me.nf, tri_base, Nt, Ng + tri_base, fr->cams.as<DevCam>(),
                    fr->ncams, fr->bin.as<BinInfo>(), Ntot, fr->tgrad.as<float>(), o.verts, o.vcolor, o.valpha,
                    o.falpha);
                UMGS_TRY(cudaGetLastError());
            }
        }
        tri_base += me.nf;
    }
#undef UMGS_TRY
    return UMGS_OK;
}

}  // namespace umgs
