// Soft-edge sample coverage of a triangle (UMGS_RENDER_SOFT_EDGE; an
// extension beyond the paper that makes the composite of Eq. 7-9
// differentiable in the vertex positions through coverage).
//
// For sample s_j of the pixel and edge e = (a, b) = (e+1, e+2) of the
// unsnapped projected triangle (record fields u, v):
//   lambda_e(s) = (u_a - s_x)(v_b - s_y) - (u_b - s_x)(v_a - s_y)
//     (twice the signed area of (s, P_a, P_b), the stable relative form),
//   d_e = sg lambda_e / |P_b - P_a|   (signed distance, positive inside;
//     sg = sign of the snapped integer area, TRec::orient),
//   c^j = prod_e sigmoid(d_e / sigma),  sigma = 1 / t.pad2.
// A triangle of zero area covers nothing.
#pragma once

#include "common.cuh"

namespace umgs {

// sg: the orientation the setup found from the snapped integer area (the
// one that orders the edge functions and culls zero-area triangles), not the
// fp32 area of the unsnapped vertices, whose sign can differ on a sliver
__device__ __forceinline__ float soft_orientation(const TRec& t) {
    return t.orient > 0 ? 1.f : (t.orient < 0 ? -1.f : 0.f);
}

// sigmoid(x) with the hardware exponential __expf (relative error ~2^-21 over
// the arguments that matter; exp(-x) overflows to inf for x < -88 and the
// result is then 0, the limit); forward and backward share it
__device__ __forceinline__ float soft_sigmoid(float x) { return 1.f / (1.f + __expf(-x)); }

// c^j of pixel centre (qx, qy) for the four samples; sg, inverse edge lengths
// and the per-(sample, edge) sigmoids are returned for the backward
__device__ __forceinline__ void soft_coverage(const TRec& t, float qx, float qy, float c[4], float& sg,
                                              float il[3], float sgm[4][3]) {
    sg = soft_orientation(t);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int a = (e + 1) % 3, b = (e + 2) % 3;
        const float ex = t.u[b] - t.u[a], ey = t.v[b] - t.v[a];
        const float L = sqrtf(ex * ex + ey * ey);
        il[e] = L > 0.f ? 1.f / L : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float sx = qx + (float)sample_dx(j) * (1.f / 256.f);
        const float sy = qy + (float)sample_dy(j) * (1.f / 256.f);
        float cj = sg != 0.f ? 1.f : 0.f;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int a = (e + 1) % 3, b = (e + 2) % 3;
            const float lam = (t.u[a] - sx) * (t.v[b] - sy) - (t.u[b] - sx) * (t.v[a] - sy);
            const float s = soft_sigmoid(sg * lam * il[e] * t.pad2);
            sgm[j][e] = s;
            cj *= s;
        }
        c[j] = cj;
    }
}

// Per-triangle constants of the forward's coverage, computed once per
// staged record: the scale of edge e's exponent k[e] = sg log2(e) / (L_e
// sigma) (k[3] = sg: 0 for a triangle of zero area, which covers nothing),
// and d[e][j], the change of lambda_e from the pixel centre to sample j
// (lambda_e is affine in the sample position: d = (v_a - v_b) dx_j +
// (u_b - u_a) dy_j).
struct SoftEdges {
    float k[4];
    float d[3][4];
    float il[4];  // 1 / L_e (0 for an edge of zero length; il[3] unused), for the backward
};
__device__ __forceinline__ void soft_edges(const TRec& t, SoftEdges& se) {
    const float sg = soft_orientation(t);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int a = (e + 1) % 3, b = (e + 2) % 3;
        const float ex = t.u[b] - t.u[a], ey = t.v[b] - t.v[a];
        const float L = sqrtf(ex * ex + ey * ey);
        se.k[e] = L > 0.f ? sg * 1.4426950408889634f * t.pad2 / L : 0.f;
        se.il[e] = L > 0.f ? 1.f / L : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            se.d[e][j] = (t.v[a] - t.v[b]) * ((float)sample_dx(j) * (1.f / 256.f)) +
                         (t.u[b] - t.u[a]) * ((float)sample_dy(j) * (1.f / 256.f));
    }
    se.k[3] = sg;
    se.il[3] = 0.f;
}
// c^j of pixel centre (qx, qy) from the staged constants: lambda_e at the
// centre (the relative form) plus the sample offsets, and per sample one
// reciprocal of the product of the three 1 + 2^(-k lambda) (the product of
// the three logistic terms; an overflow to inf gives 0, the limit)
__device__ __forceinline__ void soft_coverage_staged(const TRec& t, const SoftEdges& se, float qx, float qy,
                                                     float c[4]) {
    float lam[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int a = (e + 1) % 3, b = (e + 2) % 3;
        lam[e] = (t.u[a] - qx) * (t.v[b] - qy) - (t.u[b] - qx) * (t.v[a] - qy);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float den = 1.f;
#pragma unroll
        for (int e = 0; e < 3; ++e) den *= 1.f + fast_exp2(-se.k[e] * (lam[e] + se.d[e][j]));
        c[j] = se.k[3] != 0.f ? 1.f / den : 0.f;
    }
}

// The backward's form of soft_coverage from the staged constants: c^j and
// the per-(sample, edge) logistic terms the gradient needs, sg and 1/L_e
__device__ __forceinline__ void soft_coverage_staged_bwd(const TRec& t, const SoftEdges& se, float qx, float qy,
                                                         float c[4], float& sg, float il[3], float sgm[4][3]) {
    float lam[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int a = (e + 1) % 3, b = (e + 2) % 3;
        lam[e] = (t.u[a] - qx) * (t.v[b] - qy) - (t.u[b] - qx) * (t.v[a] - qy);
        il[e] = se.il[e];
    }
    sg = se.k[3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float cj = sg != 0.f ? 1.f : 0.f;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float sj = 1.f / (1.f + fast_exp2(-se.k[e] * (lam[e] + se.d[e][j])));
            sgm[j][e] = sj;
            cj *= sj;
        }
        c[j] = cj;
    }
}

// Adds d(sum_j dc[j] c^j) / d(u_k, v_k) to du[k], dv[k] (k = vertex):
// dc^j/dd_e = c^j (1 - sigmoid_e) / sigma and, with L = |P_b - P_a|,
// dd/dx = sg (dlambda/dx) / L - d (dL/dx) / L.
__device__ __forceinline__ void soft_coverage_grad(const TRec& t, float qx, float qy, const float c[4], float sg,
                                                   const float il[3], const float sgm[4][3], const float dc[4],
                                                   float du[3], float dv[3]) {
    if (sg == 0.f) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (dc[j] == 0.f || c[j] == 0.f) continue;
        const float sx = qx + (float)sample_dx(j) * (1.f / 256.f);
        const float sy = qy + (float)sample_dy(j) * (1.f / 256.f);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int a = (e + 1) % 3, b = (e + 2) % 3;
            const float gd = dc[j] * c[j] * (1.f - sgm[j][e]) * t.pad2;  // dL/dd_e
            const float lam = (t.u[a] - sx) * (t.v[b] - sy) - (t.u[b] - sx) * (t.v[a] - sy);
            const float d = sg * lam * il[e];
            const float ex = (t.u[b] - t.u[a]) * il[e], ey = (t.v[b] - t.v[a]) * il[e];  // unit edge
            const float k = sg * il[e], m = d * il[e];
            du[a] += gd * (k * (t.v[b] - sy) + m * ex);
            du[b] += gd * (-k * (t.v[a] - sy) - m * ex);
            dv[a] += gd * (-k * (t.u[b] - sx) + m * ey);
            dv[b] += gd * (k * (t.u[a] - sx) - m * ey);
        }
    }
}

}  // namespace umgs
