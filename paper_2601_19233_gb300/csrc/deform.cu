// Deformation transfer from the proxy mesh to the Gaussians (Sec. 3.3, Eq. 12-13).
//
//   face_gradients   one thread per proxy face: D_f = F'_f F_f^-1 with the
//                    frame F = [e1, e2, n / sqrt(|n|)] (fp64 inverse for
//                    sliver faces); area-weighted accumulation into the
//                    three vertices (atomics).
//   vertex_xforms    one thread per proxy vertex: D_v = sum / area, polar
//                    D_v = R_v S_v (Jacobi eigen-decomposition of D^T D),
//                    r_v = log R_v, Delta_v = V'_v - V_v -> a 64-byte row of
//                    the vertex table (Delta, r, S (6), rest position V_v;
//                    stays in L2: 10K vertices = 0.66 MB).
//   deform_gaussians eight threads per Gaussian (one per bound point): 3 vertex
//                    rows gathered from the table each, Eq. 12 interpolation,
//                    shuffle-reduced over the 8 points, Eq. 13 averaging,
//                    R' = exp(mean r), Sigma' = A Sigma A^T with A = R'S',
//                    mu' (FRAME or LITERAL), q' = quat(R') q.
//                    Streams 136 B in and 52 B out per Gaussian.
#include <cmath>
#include <mutex>

#include <cstring>
#include <string>

#include "internal.h"

namespace umgs {

constexpr int kStatusBadIndex = 2;
constexpr int64_t kVtabStride = 16;  // floats per vertex-table row

// ---- small 3x3 helpers (row-major) ---------------------------------------

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot3(const float a[3], const float b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// columns e1, e2, n/sqrt(|n|) of the face frame; returns |n|
__device__ float face_frame(const float a[3], const float b[3], const float c[3], float F[9]) {
    float e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    float e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    float n[3];
    cross3(e1, e2, n);
    const float nn = sqrtf(dot3(n, n));
    const float s = nn > 0.f ? rsqrtf(nn) : 0.f;
    for (int r = 0; r < 3; ++r) {
        F[3 * r + 0] = e1[r];
        F[3 * r + 1] = e2[r];
        F[3 * r + 2] = n[r] * s;
    }
    return nn;
}

__device__ bool inv3(const float M[9], float I[9]) {
    const float c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
    const float det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    if (!(fabsf(det) > 0.f)) return false;
    const float id = 1.f / det;
    I[0] = c00 * id; I[1] = (M[2] * M[7] - M[1] * M[8]) * id; I[2] = (M[1] * M[5] - M[2] * M[4]) * id;
    I[3] = c01 * id; I[4] = (M[0] * M[8] - M[2] * M[6]) * id; I[5] = (M[2] * M[3] - M[0] * M[5]) * id;
    I[6] = c02 * id; I[7] = (M[1] * M[6] - M[0] * M[7]) * id; I[8] = (M[0] * M[4] - M[1] * M[3]) * id;
    return true;
}

__device__ bool inv3_fp64(const float Mf[9], float I[9]) {
    double M[9];
    for (int k = 0; k < 9; ++k) M[k] = Mf[k];
    const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
    const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    if (!(fabs(det) > 0.0)) return false;
    const double id = 1.0 / det;
    I[0] = (float)(c00 * id); I[1] = (float)((M[2] * M[7] - M[1] * M[8]) * id); I[2] = (float)((M[1] * M[5] - M[2] * M[4]) * id);
    I[3] = (float)(c01 * id); I[4] = (float)((M[0] * M[8] - M[2] * M[6]) * id); I[5] = (float)((M[2] * M[3] - M[0] * M[5]) * id);
    I[6] = (float)(c02 * id); I[7] = (float)((M[1] * M[6] - M[0] * M[7]) * id); I[8] = (float)((M[0] * M[4] - M[1] * M[3]) * id);
    return true;
}

// Deformation gradient D = F' F^-1 of a sliver face entirely in fp64: the
// frames' cross products (|e1 x e2| is a small difference of large products
// for a sliver) and the inverse; the fp32 vertex positions are exact in fp64.
__device__ bool sliver_gradient_fp64(const float P[3][3], const float Q[3][3], float D[9]) {
    double Fr[9], Fd[9];
    for (int w = 0; w < 2; ++w) {
        const float (*X)[3] = w ? Q : P;
        double* F = w ? Fd : Fr;
        double e1[3], e2[3], n[3];
        for (int d = 0; d < 3; ++d) { e1[d] = (double)X[1][d] - X[0][d]; e2[d] = (double)X[2][d] - X[0][d]; }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0)) return false;
        const double sc = 1.0 / sqrt(nn);
        for (int r = 0; r < 3; ++r) { F[3 * r] = e1[r]; F[3 * r + 1] = e2[r]; F[3 * r + 2] = n[r] * sc; }
    }
    const double* M = Fr;
    const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
    const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    if (!(fabs(det) > 0.0)) return false;
    const double id = 1.0 / det;
    const double I[9] = {c00 * id, (M[2] * M[7] - M[1] * M[8]) * id, (M[1] * M[5] - M[2] * M[4]) * id,
                         c01 * id, (M[0] * M[8] - M[2] * M[6]) * id, (M[2] * M[3] - M[0] * M[5]) * id,
                         c02 * id, (M[1] * M[6] - M[0] * M[7]) * id, (M[0] * M[4] - M[1] * M[3]) * id};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            D[3 * i + j] = (float)(Fd[3 * i] * I[j] + Fd[3 * i + 1] * I[3 + j] + Fd[3 * i + 2] * I[6 + j]);
    return true;
}

__device__ __forceinline__ void matmul3(const float A[9], const float B[9], float C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// ---- K1a: per-face deformation gradients ----------------------------------

__global__ void __launch_bounds__(256) face_gradients_kernel(const float* __restrict__ V, const float* __restrict__ Vd,
                                                             const int32_t* __restrict__ F, int64_t nv, int64_t nf,
                                                             float* __restrict__ vacc, int32_t* __restrict__ status) {
    pdl_enter();
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) { atomicOr(status, kStatusBadIndex); return; }
    const int idx[3] = {i0, i1, i2};
    float P[3][3], Q[3][3];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) { P[k][d] = V[3 * (int64_t)idx[k] + d]; Q[k][d] = Vd[3 * (int64_t)idx[k] + d]; }
    float Fr[9], Fd[9], Fi[9], D[9];
    const float nn = face_frame(P[0], P[1], P[2], Fr);
    face_frame(Q[0], Q[1], Q[2], Fd);
    if (!(nn > 0.f)) return;  // degenerate rest face: zero weight
    // sliver: |n| = |e1||e2| sin(angle); its gradient (both frames and the
    // inverse) in fp64 when sin < 1e-3
    const float l1 = sqrtf(Fr[0] * Fr[0] + Fr[3] * Fr[3] + Fr[6] * Fr[6]);
    const float l2 = sqrtf(Fr[1] * Fr[1] + Fr[4] * Fr[4] + Fr[7] * Fr[7]);
    const bool sliver = nn < 1e-3f * l1 * l2;
    if (sliver) {
        atomicAdd(status + 1, 1);  // fp64 sliver faces of this deformation (umgs_deform_fp64_faces)
        if (!sliver_gradient_fp64(P, Q, D)) return;
    } else {
        if (!inv3(Fr, Fi)) return;
        matmul3(Fd, Fi, D);
    }
    const float area = 0.5f * nn;
    for (int k = 0; k < 3; ++k) {
        float* acc = vacc + 10 * (int64_t)idx[k];
        for (int e = 0; e < 9; ++e) atomicAdd(acc + e, area * D[e]);
        atomicAdd(acc + 9, area);
    }
}

// ---- K1b: per-vertex polar decomposition and log map ----------------------

// cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix A (destroyed);
// eigenvectors in the columns of V
__device__ void jacobi_eigen3(float A[9], float V[9]) {
    for (int k = 0; k < 9; ++k) V[k] = (k % 4 == 0) ? 1.f : 0.f;
    for (int sweep = 0; sweep < 10; ++sweep) {
        const float off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const float dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-14f * dia) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const float apq = A[3 * p + q];
            if (fabsf(apq) < 1e-30f) continue;
            const float theta = (A[3 * q + q] - A[3 * p + p]) / (2.f * apq);
            const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = rsqrtf(t * t + 1.f), s = t * c;
            // A <- J^T A J with J the (p,q) rotation
            for (int k = 0; k < 3; ++k) {  // columns p, q
                const float akp = A[3 * k + p], akq = A[3 * k + q];
                A[3 * k + p] = c * akp - s * akq;
                A[3 * k + q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {  // rows p, q
                const float apk = A[3 * p + k], aqk = A[3 * q + k];
                A[3 * p + k] = c * apk - s * aqk;
                A[3 * q + k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                const float vkp = V[3 * k + p], vkq = V[3 * k + q];
                V[3 * k + p] = c * vkp - s * vkq;
                V[3 * k + q] = s * vkp + c * vkq;
            }
        }
    }
}

// D = R S with R a proper rotation (det D < 0: smallest singular direction flipped)
__device__ void polar3(const float D[9], float R[9], float S6[6]) {
    float A[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[3 * i + j] = D[i] * D[j] + D[3 + i] * D[3 + j] + D[6 + i] * D[6 + j];
    float V[9];
    jacobi_eigen3(A, V);
    float lam[3] = {A[0], A[4], A[8]};
    // sort eigenpairs by decreasing eigenvalue
    int o[3] = {0, 1, 2};
    if (lam[o[0]] < lam[o[1]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
    if (lam[o[1]] < lam[o[2]]) { int t = o[1]; o[1] = o[2]; o[2] = t; }
    if (lam[o[0]] < lam[o[1]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
    float v[3][3];
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) v[k][r] = V[3 * r + o[k]];
    // right-handed V
    float c[3];
    cross3(v[0], v[1], c);
    if (dot3(c, v[2]) < 0.f) { v[2][0] = -v[2][0]; v[2][1] = -v[2][1]; v[2][2] = -v[2][2]; }
    // u1 = D v1 / |D v1|, u2 = D v2 orthogonalised, u3 = u1 x u2
    float u[3][3];
    for (int k = 0; k < 2; ++k)
        for (int r = 0; r < 3; ++r) u[k][r] = D[3 * r] * v[k][0] + D[3 * r + 1] * v[k][1] + D[3 * r + 2] * v[k][2];
    float n0 = sqrtf(dot3(u[0], u[0]));
    if (n0 > 0.f) for (int r = 0; r < 3; ++r) u[0][r] /= n0;
    else { u[0][0] = v[0][0]; u[0][1] = v[0][1]; u[0][2] = v[0][2]; }
    const float p = dot3(u[0], u[1]);
    for (int r = 0; r < 3; ++r) u[1][r] -= p * u[0][r];
    float n1 = sqrtf(dot3(u[1], u[1]));
    if (n1 > 1e-20f) for (int r = 0; r < 3; ++r) u[1][r] /= n1;
    else {  // rank <= 1: any unit vector orthogonal to u1
        float a[3] = {fabsf(u[0][0]) < 0.9f ? 1.f : 0.f, fabsf(u[0][0]) < 0.9f ? 0.f : 1.f, 0.f};
        cross3(u[0], a, u[1]);
        const float m = rsqrtf(dot3(u[1], u[1]));
        for (int r = 0; r < 3; ++r) u[1][r] *= m;
    }
    cross3(u[0], u[1], u[2]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[3 * i + j] = u[0][i] * v[0][j] + u[1][i] * v[1][j] + u[2][i] * v[2][j];
    // S = R^T D, symmetrised
    float S[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[3 * i + j] = R[i] * D[j] + R[3 + i] * D[3 + j] + R[6 + i] * D[6 + j];
    S6[0] = S[0]; S6[1] = 0.5f * (S[1] + S[3]); S6[2] = 0.5f * (S[2] + S[6]);
    S6[3] = S[4]; S6[4] = 0.5f * (S[5] + S[7]); S6[5] = S[8];
}

// axis-angle log of a rotation, angle in [0, pi]
__device__ void log_rot(const float R[9], float r[3]) {
    const float w[3] = {0.5f * (R[7] - R[5]), 0.5f * (R[2] - R[6]), 0.5f * (R[3] - R[1])};  // sin(t) * axis
    const float s = sqrtf(dot3(w, w));
    const float c = 0.5f * (R[0] + R[4] + R[8] - 1.f);
    const float th = atan2f(s, c);
    if (s > 1e-4f) {
        const float k = th / s;
        r[0] = k * w[0]; r[1] = k * w[1]; r[2] = k * w[2];
    } else if (c > 0.f) {  // near identity: th ~ s
        const float k = 1.f + s * s / 6.f;
        r[0] = k * w[0]; r[1] = k * w[1]; r[2] = k * w[2];
    } else {  // near pi: axis from (R + I)/2 = a a^T
        int j = 0;
        if (R[4] > R[3 * j + j]) j = 1;
        if (R[8] > R[3 * j + j]) j = 2;
        float a[3] = {0.5f * (R[j] + (j == 0)), 0.5f * (R[3 + j] + (j == 1)), 0.5f * (R[6 + j] + (j == 2))};
        const float m = rsqrtf(dot3(a, a));
        a[0] *= m; a[1] *= m; a[2] *= m;
        if (dot3(a, w) < 0.f) { a[0] = -a[0]; a[1] = -a[1]; a[2] = -a[2]; }
        r[0] = th * a[0]; r[1] = th * a[1]; r[2] = th * a[2];
    }
}

// the table row of vertex v from its transform D: polar D = R S, r = log R,
// Delta = V' - V and the rest position
__device__ __forceinline__ void write_vertex_row(const float (&D)[9], const float* __restrict__ V,
                                                 const float* __restrict__ Vd, int64_t v, float* __restrict__ vtab) {
    float R[9], S6[6], r[3];
    polar3(D, R, S6);
    log_rot(R, r);
    float4* o = reinterpret_cast<float4*>(vtab + kVtabStride * v);
    const float p0 = V[3 * v], p1 = V[3 * v + 1], p2 = V[3 * v + 2];
    o[0] = make_float4(Vd[3 * v] - p0, Vd[3 * v + 1] - p1, Vd[3 * v + 2] - p2, r[0]);
    o[1] = make_float4(r[1], r[2], S6[0], S6[1]);
    o[2] = make_float4(S6[2], S6[3], S6[4], S6[5]);
    o[3] = make_float4(p0, p1, p2, 0.f);
}

__global__ void __launch_bounds__(256) vertex_xforms_kernel(const float* __restrict__ V, const float* __restrict__ Vd,
                                                            const float* __restrict__ vacc, int64_t nv,
                                                            float* __restrict__ vtab) {
    pdl_enter();
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const float* a = vacc + 10 * v;
    float D[9];
    const float w = a[9];
    if (w > 0.f) { const float iw = 1.f / w; for (int k = 0; k < 9; ++k) D[k] = a[k] * iw; }
    else { for (int k = 0; k < 9; ++k) D[k] = (k % 4 == 0) ? 1.f : 0.f; }
    write_vertex_row(D, V, Vd, v, vtab);
}

// ---- one-ring reading of the per-vertex transform --------------------------
// D_v = (sum_j c_vj e'_vj e_vj^T + n'_v n_v^T)(sum_j c_vj e_vj e_vj^T + n_v n_v^T)^-1
// over the edges at v, c_vj = sum over the edge's faces of max(0, cot/2) of the
// opposite angle, N_v = sum of the faces' e1 x e2 at v, n_v = N_v / sqrt|N_v|
// (rest and deformed).  Per-vertex accumulators (21 floats): A (xx xy xz yy yz
// zz), B (row-major 3x3), N (3), N' (3).
constexpr int kOneRingAcc = 21;

__global__ void __launch_bounds__(256) one_ring_faces_kernel(const float* __restrict__ V, const float* __restrict__ Vd,
                                                             const int32_t* __restrict__ F, int64_t nv, int64_t nf,
                                                             float* __restrict__ vacc, int32_t* __restrict__ status) {
    pdl_enter();
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int idx[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
    for (int k = 0; k < 3; ++k)
        if (idx[k] < 0 || idx[k] >= nv) { atomicOr(status, kStatusBadIndex); return; }
    float P[3][3], Q[3][3];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) { P[k][d] = V[3 * (int64_t)idx[k] + d]; Q[k][d] = Vd[3 * (int64_t)idx[k] + d]; }
    for (int k = 0; k < 3; ++k) {  // edge (i, j) opposite corner k
        const int i = (k + 1) % 3, j = (k + 2) % 3;
        const float u1[3] = {P[i][0] - P[k][0], P[i][1] - P[k][1], P[i][2] - P[k][2]};
        const float u2[3] = {P[j][0] - P[k][0], P[j][1] - P[k][1], P[j][2] - P[k][2]};
        float cr[3];
        cross3(u1, u2, cr);
        const float len = sqrtf(dot3(cr, cr));
        const float w = len > 0.f ? fmaxf(0.5f * dot3(u1, u2) / len, 0.f) : 0.f;
        if (!(w > 0.f)) continue;
        const float e[3] = {P[j][0] - P[i][0], P[j][1] - P[i][1], P[j][2] - P[i][2]};
        const float ed[3] = {Q[j][0] - Q[i][0], Q[j][1] - Q[i][1], Q[j][2] - Q[i][2]};
        const float a6[6] = {w * e[0] * e[0], w * e[0] * e[1], w * e[0] * e[2],
                             w * e[1] * e[1], w * e[1] * e[2], w * e[2] * e[2]};
        for (const int vert : {idx[i], idx[j]}) {
            float* acc = vacc + kOneRingAcc * (int64_t)vert;
            for (int q = 0; q < 6; ++q) atomicAdd(acc + q, a6[q]);
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) atomicAdd(acc + 6 + 3 * r + c, w * ed[r] * e[c]);
        }
    }
    const float e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    const float e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    const float d1[3] = {Q[1][0] - Q[0][0], Q[1][1] - Q[0][1], Q[1][2] - Q[0][2]};
    const float d2[3] = {Q[2][0] - Q[0][0], Q[2][1] - Q[0][1], Q[2][2] - Q[0][2]};
    float n[3], nd[3];
    cross3(e1, e2, n);
    cross3(d1, d2, nd);
    for (int k = 0; k < 3; ++k) {
        float* acc = vacc + kOneRingAcc * (int64_t)idx[k];
        for (int d = 0; d < 3; ++d) { atomicAdd(acc + 15 + d, n[d]); atomicAdd(acc + 18 + d, nd[d]); }
    }
}

__global__ void __launch_bounds__(256) one_ring_vertices_kernel(const float* __restrict__ V,
                                                                const float* __restrict__ Vd,
                                                                const float* __restrict__ vacc, int64_t nv,
                                                                float* __restrict__ vtab) {
    pdl_enter();
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const float* a = vacc + kOneRingAcc * v;
    const float* N = a + 15;
    const float* Nd = a + 18;
    const float ln = sqrtf(dot3(N, N)), lnd = sqrtf(dot3(Nd, Nd));
    const float sn = ln > 0.f ? rsqrtf(ln) : 0.f, snd = lnd > 0.f ? rsqrtf(lnd) : 0.f;
    const float n[3] = {N[0] * sn, N[1] * sn, N[2] * sn}, nd[3] = {Nd[0] * snd, Nd[1] * snd, Nd[2] * snd};
    float A[9] = {a[0], a[1], a[2], a[1], a[3], a[4], a[2], a[4], a[5]};
    float B[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            A[3 * r + c] += n[r] * n[c];
            B[3 * r + c] = a[6 + 3 * r + c] + nd[r] * n[c];
        }
    float Ai[9], D[9];
    if (inv3_fp64(A, Ai)) matmul3(B, Ai, D);
    else for (int k = 0; k < 9; ++k) D[k] = (k % 4 == 0) ? 1.f : 0.f;  // isolated vertex: identity
    write_vertex_row(D, V, Vd, v, vtab);
}

// ---- K2: per-Gaussian update ------------------------------------------------

__device__ void exp_rot(const float r[3], float R[9], float q[4]) {
    const float th2 = dot3(r, r);
    const float th = sqrtf(th2);
    float A, B, hs, hc;  // R = I + A [r]x + B [r]x^2 ; q = (cos(th/2), sin(th/2)/th * r)
    if (th < 1e-3f) {
        A = 1.f - th2 / 6.f;
        B = 0.5f - th2 / 24.f;
        hs = 0.5f - th2 / 48.f;
        hc = 1.f - th2 / 8.f;
    } else {
        // one sincos of th/2: sin th = 2 s c, 1 - cos th = 2 s^2 (no cancellation)
        float s2, c2;
        sincosf(0.5f * th, &s2, &c2);
        const float ith = 1.f / th;
        hs = s2 * ith;
        A = 2.f * c2 * hs;
        B = 2.f * hs * hs;
        hc = c2;
    }
    const float x = r[0], y = r[1], z = r[2];
    R[0] = 1.f + B * (-(y * y + z * z)); R[1] = -A * z + B * x * y;         R[2] = A * y + B * x * z;
    R[3] = A * z + B * x * y;           R[4] = 1.f + B * (-(x * x + z * z)); R[5] = -A * x + B * y * z;
    R[6] = -A * y + B * x * z;          R[7] = A * x + B * y * z;          R[8] = 1.f + B * (-(x * x + y * y));
    q[0] = hc; q[1] = hs * x; q[2] = hs * y; q[3] = hs * z;
}

// Eq. 13 for one Gaussian from acc = scale^-1 x the means of its bound
// points' Eq. 12 interpolants (Delta, log R, S (6), rest position P) and
// bad (an index was out of range): writes the outputs selected by `which`
// (bit 0: mu', bit 1: Sigma', bit 2: q'; NaN and a status bit if bad).
__device__ __forceinline__ void deform_finish(const float (&acc)[15], float scale, int bad, bool live, int which,
                                              int64_t i, const float* __restrict__ means,
                                              const float* __restrict__ quats, const float* __restrict__ scales,
                                              const float* __restrict__ cov3d, int mode, float* __restrict__ out_means,
                                              float* __restrict__ out_cov, float* __restrict__ out_quats,
                                              int32_t* __restrict__ status) {
    if (!live || which == 0) return;
    if (bad) {
        if (which & 1) atomicOr(status, kStatusBadIndex);
        const float nanv = __int_as_float(0x7fc00000);
        if (which & 1) for (int d = 0; d < 3; ++d) out_means[3 * i + d] = nanv;
        if (which & 2) for (int d = 0; d < 6; ++d) out_cov[6 * i + d] = nanv;
        if ((which & 4) && out_quats) for (int d = 0; d < 4; ++d) out_quats[4 * i + d] = nanv;
        return;
    }
    const float e = scale;
    float rb[3] = {acc[3] * e, acc[4] * e, acc[5] * e};
    float Rp[9], qr[4];
    exp_rot(rb, Rp, qr);
    const float Sb[9] = {acc[6] * e, acc[7] * e, acc[8] * e, acc[7] * e, acc[9] * e, acc[10] * e,
                         acc[8] * e, acc[10] * e, acc[11] * e};
    float A[9];
    matmul3(Rp, Sb, A);
    if (which & 1) {
        const float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
        float mo[3];
        for (int d = 0; d < 3; ++d) mo[d] = mu[d] + acc[d] * e;
        if (mode == UMGS_DEFORM_FRAME) {
            const float rel[3] = {mu[0] - acc[12] * e, mu[1] - acc[13] * e, mu[2] - acc[14] * e};
            for (int d = 0; d < 3; ++d) mo[d] += A[3 * d] * rel[0] + A[3 * d + 1] * rel[1] + A[3 * d + 2] * rel[2] - rel[d];
        }
        for (int d = 0; d < 3; ++d) out_means[3 * i + d] = mo[d];
    }
    if ((which & 6) == 0) return;
    float qn[4] = {1.f, 0.f, 0.f, 0.f};
    float S[9];
    if (cov3d) {
        const float* c6 = cov3d + 6 * i;
        S[0] = c6[0]; S[1] = c6[1]; S[2] = c6[2]; S[3] = c6[1]; S[4] = c6[3]; S[5] = c6[4];
        S[6] = c6[2]; S[7] = c6[4]; S[8] = c6[5];
    } else {
        float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        const float nq2 = qw * qw + qx * qx + qy * qy + qz * qz;
        if (nq2 > 0.f) {
            const float inq = rsqrtf(nq2);
            qw *= inq; qx *= inq; qy *= inq; qz *= inq;
        } else {
            qw = 1.f; qx = qy = qz = 0.f;
        }
        qn[0] = qw; qn[1] = qx; qn[2] = qy; qn[3] = qz;
        if (which & 2) {
            const float r[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                                2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                                2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
            const float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
            float M[9];
            for (int a = 0; a < 3; ++a)
                for (int bb = 0; bb < 3; ++bb) M[3 * a + bb] = r[3 * a + bb] * s[bb];
            for (int a = 0; a < 3; ++a)
                for (int bb = 0; bb < 3; ++bb)
                    S[3 * a + bb] = M[3 * a] * M[3 * bb] + M[3 * a + 1] * M[3 * bb + 1] + M[3 * a + 2] * M[3 * bb + 2];
        }
    }
    if (which & 2) {
        float AS[9], Sig[9];
        matmul3(A, S, AS);
        for (int a = 0; a < 3; ++a)
            for (int bb = 0; bb < 3; ++bb)
                Sig[3 * a + bb] = AS[3 * a] * A[3 * bb] + AS[3 * a + 1] * A[3 * bb + 1] + AS[3 * a + 2] * A[3 * bb + 2];
        float* oc = out_cov + 6 * i;
        oc[0] = Sig[0]; oc[1] = Sig[1]; oc[2] = Sig[2]; oc[3] = Sig[4]; oc[4] = Sig[5]; oc[5] = Sig[8];
    }
    if ((which & 4) && out_quats) {
        // q' = qr * qn (Hamilton product), canonical sign w >= 0
        float o[4];
        o[0] = qr[0] * qn[0] - qr[1] * qn[1] - qr[2] * qn[2] - qr[3] * qn[3];
        o[1] = qr[0] * qn[1] + qr[1] * qn[0] + qr[2] * qn[3] - qr[3] * qn[2];
        o[2] = qr[0] * qn[2] - qr[1] * qn[3] + qr[2] * qn[0] + qr[3] * qn[1];
        o[3] = qr[0] * qn[3] + qr[1] * qn[2] - qr[2] * qn[1] + qr[3] * qn[0];
        const float sg = o[0] < 0.f ? -1.f : 1.f;
        for (int d = 0; d < 4; ++d) out_quats[4 * i + d] = sg * o[d];
    }
}

// One thread per (Gaussian, bound point): 8 consecutive lanes gather the
// Eq. 12 interpolants of one Gaussian's 8 points (independent loads, and a
// single broadcast when points share a face), reduce them with shuffles and
// then all 8 lanes evaluate Eq. 13; lanes 0-2 write mu', Sigma', q'.
__global__ void __launch_bounds__(256) deform_gaussians_kernel(
    const float* __restrict__ means, const float* __restrict__ quats, const float* __restrict__ scales,
    const float* __restrict__ cov3d, int64_t n, const int32_t* __restrict__ face, const float* __restrict__ bary,
    const float* __restrict__ V, const int32_t* __restrict__ F, int64_t nv, int64_t nf,
    const float* __restrict__ vtab, int mode, float* __restrict__ out_means, float* __restrict__ out_cov,
    float* __restrict__ out_quats, int32_t* __restrict__ status) {
    pdl_enter();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = tid >> 3;
    const int corner = (int)(tid & 7);
    const bool live = i < n;
    float acc[15];
#pragma unroll
    for (int e = 0; e < 15; ++e) acc[e] = 0.f;
    int bad = 0;
    if (live) {
        const int f = face[8 * i + corner];
        const float2 b = reinterpret_cast<const float2*>(bary)[8 * i + corner];
        if (f < 0 || f >= nf) {
            bad = 1;
        } else {
            const float w[3] = {1.f - b.x - b.y, b.x, b.y};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int v = F[3 * (int64_t)f + k];
                if (v < 0 || v >= nv) { bad = 1; continue; }
                const float4* row = reinterpret_cast<const float4*>(vtab + kVtabStride * (int64_t)v);
                const float4 t0 = row[0], t1 = row[1], t2 = row[2], t3 = row[3];
                const float px = t3.x, py = t3.y, pz = t3.z;
                const float wk = w[k];
                acc[0] += wk * t0.x; acc[1] += wk * t0.y; acc[2] += wk * t0.z;     // Delta
                acc[3] += wk * t0.w; acc[4] += wk * t1.x; acc[5] += wk * t1.y;     // log R
                acc[6] += wk * t1.z; acc[7] += wk * t1.w; acc[8] += wk * t2.x;     // S
                acc[9] += wk * t2.y; acc[10] += wk * t2.z; acc[11] += wk * t2.w;
                acc[12] += wk * px; acc[13] += wk * py; acc[14] += wk * pz;         // P
            }
        }
    }
    // sum over the 8 lanes of this Gaussian
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
        for (int e = 0; e < 15; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    deform_finish(acc, 0.125f, bad, live, corner < 3 ? 1 << corner : 0, i, means, quats, scales, cov3d, mode, out_means, out_cov,
                  out_quats, status);
}

// Compact binding (Sec. 3.3, Eq. 12-13 regrouped): every interpolant that
// Eq. 13 averages is linear in the vertex rows, so a Gaussian's means are
// sum_v w_v row(v) with w_v = (1/8) x the barycentric weights of vertex v
// summed over its 8 bound points.  One thread per Gaussian merges its 24
// (vertex, weight) terms into its distinct vertices (in order of first
// appearance); count -1 marks an out-of-range face or vertex index.
__global__ void __launch_bounds__(256) binding_compact_kernel(const int32_t* __restrict__ face,
                                                              const float* __restrict__ bary, int64_t n,
                                                              const int32_t* __restrict__ F, int64_t nv, int64_t nf,
                                                              int32_t* __restrict__ count,
                                                              int2* __restrict__ entries) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int2* out = entries + 24 * i;
    int c = 0;
    for (int p = 0; p < 8; ++p) {
        const int f = face[8 * i + p];
        const float2 b = reinterpret_cast<const float2*>(bary)[8 * i + p];
        if (f < 0 || f >= nf) { c = -1; break; }
        const float wk[3] = {1.f - b.x - b.y, b.x, b.y};
        bool bad = false;
        for (int k = 0; k < 3; ++k) {
            const int v = F[3 * (int64_t)f + k];
            if (v < 0 || v >= nv) { bad = true; break; }
            const float w = 0.125f * wk[k];
            int j = 0;
            while (j < c && out[j].x != v) ++j;
            if (j < c) out[j].y = __float_as_int(__int_as_float(out[j].y) + w);
            else { out[c] = make_int2(v, __float_as_int(w)); ++c; }
        }
        if (bad) { c = -1; break; }
    }
    count[i] = c;
}

// ---- compact binding as CSR ------------------------------------------------
// The distinct bound vertices and weights of Gaussian i occupy entries
// [offsets[i], offsets[i+1]) of one packed array, in order of first
// appearance, padded to an even count with a zero-weight copy of the first
// entry (the deformation reads two entries per 16-byte load).  A Gaussian
// with an out-of-range face or vertex index gets two (-1, 0) entries (the
// deformation then marks it bad).
__device__ int csr_distinct(const int32_t* __restrict__ face, const float* __restrict__ bary, int64_t i,
                            const int32_t* __restrict__ F, int64_t nv, int64_t nf, int2 out[24]) {
    int c = 0;
    for (int p = 0; p < 8; ++p) {
        const int f = face[8 * i + p];
        const float2 b = reinterpret_cast<const float2*>(bary)[8 * i + p];
        if (f < 0 || f >= nf) return -1;
        const float wk[3] = {1.f - b.x - b.y, b.x, b.y};
        for (int k = 0; k < 3; ++k) {
            const int v = F[3 * (int64_t)f + k];
            if (v < 0 || v >= nv) return -1;
            const float w = 0.125f * wk[k];
            int j = 0;
            while (j < c && out[j].x != v) ++j;
            if (j < c) out[j].y = __float_as_int(__int_as_float(out[j].y) + w);
            else { out[c] = make_int2(v, __float_as_int(w)); ++c; }
        }
    }
    return c;
}

__global__ void __launch_bounds__(256) binding_csr_count_kernel(const int32_t* __restrict__ face,
                                                               const float* __restrict__ bary, int64_t n,
                                                               const int32_t* __restrict__ F, int64_t nv, int64_t nf,
                                                               uint32_t* __restrict__ count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int2 tmp[24];
    const int c = csr_distinct(face, bary, i, F, nv, nf, tmp);
    count[i] = c < 0 ? 2u : (uint32_t)((c + 1) & ~1);
}

// exclusive scan of n counts into offsets[0..n] (offsets[n] = total), in one
// block of 1024 threads (a one-time step of the binding)
__global__ void __launch_bounds__(1024) binding_csr_scan_kernel(const uint32_t* __restrict__ count, int64_t n,
                                                               int32_t* __restrict__ offsets,
                                                               unsigned long long* __restrict__ total) {
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_base;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_base = 0;
    __syncthreads();
    for (int64_t b = 0; b < n; b += 1024) {
        const int64_t i = b + t;
        const unsigned long long v = i < n ? count[i] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const unsigned long long excl = s_base + (warp ? s_w[warp - 1] : 0ull) + x - v;
        if (i < n) offsets[i] = (int32_t)min(excl, 0x7fffffffull);
        __syncthreads();
        if (t == 1023) s_base += s_w[31];
        __syncthreads();
    }
    if (t == 0) {
        offsets[n] = (int32_t)min(s_base, 0x7fffffffull);
        *total = s_base;
    }
}

__global__ void __launch_bounds__(256) binding_csr_fill_kernel(const int32_t* __restrict__ face,
                                                              const float* __restrict__ bary, int64_t n,
                                                              const int32_t* __restrict__ F, int64_t nv, int64_t nf,
                                                              const int32_t* __restrict__ offsets,
                                                              int2* __restrict__ entries) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int2 tmp[24];
    const int c = csr_distinct(face, bary, i, F, nv, nf, tmp);
    int2* out = entries + offsets[i];
    if (c < 0) {
        out[0] = out[1] = make_int2(-1, 0);
        return;
    }
    for (int j = 0; j < c; ++j) out[j] = tmp[j];
    if (c & 1) out[c] = make_int2(tmp[0].x, 0);  // zero-weight padding
}

// Deformation over a compact binding.  A block of 256 threads takes 256
// Gaussians.  Gather phase, 4 rounds of 64 Gaussians: the four lanes of a
// Gaussian walk its entries together; for each entry lane p gathers float4 p
// of the vertex's 64-byte table row and accumulates those four of the 15
// interpolated components (one warp-wide row load touches 8 rows of 64
// contiguous bytes).  Entries are read two at a time (16-byte loads), four in
// flight per step.  The sums go to shared memory; then every thread finishes
// one Gaussian (Eq. 13 and all three outputs), so that math runs with every
// lane busy.
constexpr int kDefBlock = 256;
// CSR: `count` holds the offsets [n+1] of the packed entries (binding_csr_*)
template <bool CSR>
__global__ void __launch_bounds__(kDefBlock) deform_gaussians_compact_kernel(
    const float* __restrict__ means, const float* __restrict__ quats, const float* __restrict__ scales,
    const float* __restrict__ cov3d, int64_t n, const int32_t* __restrict__ count, const int2* __restrict__ entries,
    int64_t nv, const float* __restrict__ vtab, int mode, float* __restrict__ out_means,
    float* __restrict__ out_cov, float* __restrict__ out_quats, int32_t* __restrict__ status) {
    pdl_enter();
    __shared__ float s_acc[kDefBlock][17];  // odd row length: conflict-free row reads
    __shared__ int s_bad[kDefBlock];
    const int t = threadIdx.x;
    const int part = t & 3;
    const int64_t g0 = (int64_t)blockIdx.x * kDefBlock;
    const float4* tab = reinterpret_cast<const float4*>(vtab);
#pragma unroll
    for (int r = 0; r < kDefBlock / 64; ++r) {
        const int local = r * 64 + (t >> 2);
        const int64_t i = g0 + local;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        int bad = 0;
        int c = 0;
        int64_t start = 24 * i;
        if (i < n) {
            if (CSR) {
                start = count[i];
                c = count[i + 1] - count[i];
                if (c < 0 || c > 24 || (start & 1)) { bad = 1; c = 0; }
            } else {
                c = count[i];
                if (c < 0 || c > 24) { bad = 1; c = 0; }
            }
        }
        const int4* row = reinterpret_cast<const int4*>(entries + start);  // two entries per int4
        if (CSR) {
            // runs of even length: one 16-byte load takes two entries, no
            // tail; an index out of range reads row 0 with weight 0 and marks
            // the Gaussian bad
            const float4* tp = tab + part;
            const uint32_t unv = (uint32_t)min(nv, (int64_t)0xffffffff);
#pragma unroll 2
            for (int j = 0; j < c; j += 2) {
                const int4 e = row[j >> 1];
                const bool ok0 = (uint32_t)e.x < unv, ok1 = (uint32_t)e.z < unv;
                bad |= !(ok0 && ok1);
                const float4 t0 = tp[(uint64_t)(ok0 ? (uint32_t)e.x : 0u) << 2];
                const float4 t1 = tp[(uint64_t)(ok1 ? (uint32_t)e.z : 0u) << 2];
                const float w0 = ok0 ? __int_as_float(e.y) : 0.f, w1 = ok1 ? __int_as_float(e.w) : 0.f;
                a.x += w0 * t0.x; a.y += w0 * t0.y; a.z += w0 * t0.z; a.w += w0 * t0.w;
                a.x += w1 * t1.x; a.y += w1 * t1.y; a.z += w1 * t1.z; a.w += w1 * t1.w;
            }
            c = 0;  // (the padded form's loop below does nothing)
        }
        for (int j = 0; j < c; j += 4) {
            const int4 e01 = row[j >> 1];
            const int4 e23 = j + 2 < c ? row[(j >> 1) + 1] : make_int4(0, 0, 0, 0);
            const int vv[4] = {e01.x, e01.z, e23.x, e23.z};
            const int ww[4] = {e01.y, e01.w, e23.y, e23.w};
            float4 tq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool use = j + q < c;
                const int v = vv[q];
                if (use && (v < 0 || v >= nv)) bad = 1;
                tq[q] = (use && v >= 0 && v < nv) ? tab[4 * (int64_t)v + part] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float wk = j + q < c ? __int_as_float(ww[q]) : 0.f;
                a.x += wk * tq[q].x; a.y += wk * tq[q].y; a.z += wk * tq[q].z; a.w += wk * tq[q].w;
            }
        }
        // lane p of the Gaussian holds components 4p .. 4p+3 (the 16th is padding)
        s_acc[local][4 * part] = a.x;
        s_acc[local][4 * part + 1] = a.y;
        s_acc[local][4 * part + 2] = a.z;
        s_acc[local][4 * part + 3] = a.w;
        bad |= __shfl_xor_sync(0xffffffffu, bad, 1);
        bad |= __shfl_xor_sync(0xffffffffu, bad, 2);
        if (part == 0) s_bad[local] = bad;
    }
    __syncthreads();
    const int64_t i = g0 + t;
    if (i >= n) return;
    float acc[15];
#pragma unroll
    for (int e = 0; e < 15; ++e) acc[e] = s_acc[t][e];
    deform_finish(acc, 1.f, s_bad[t], true, 7, i, means, quats, scales, cov3d, mode, out_means, out_cov, out_quats,
                  status);
}

static inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// per-face gradients and the per-vertex table of the deformed proxy (A1)
// (also clears *word, the fp64 sliver-face count of the deformation)
__global__ void zero_floats_kernel(float* __restrict__ p, int64_t n, int32_t* __restrict__ word) {
    pdl_enter();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.f;
    if (i == 0 && word) *word = 0;
}

static umgs_status proxy_table(umgs_ctx* ctx, const float* V, const float* Vd, const int32_t* F, int64_t nv,
                               int64_t nf, bool one_ring, cudaStream_t stream) {
    cudaError_t e;
    const int64_t nacc = (one_ring ? kOneRingAcc : 10) * nv;
    if ((e = ctx->vacc.reserve(sizeof(float) * nacc)) != cudaSuccess) return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "vacc");
    if ((e = ctx->vtab.reserve(sizeof(float) * kVtabStride * nv)) != cudaSuccess)
        return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "vtab");
    ctx->vtab_rows = nv;
    // accumulators cleared by a kernel, so the programmatic launch chain runs on
    launch_pdl(zero_floats_kernel, grid_for(nacc, 256), 256, 0, stream, ctx->vacc.as<float>(), nacc,
               ctx->dstatus.as<int32_t>() + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "zero_floats_kernel");
    int32_t* status = ctx->dstatus.as<int32_t>();
    {
        StageTimer tm(ctx, UMGS_STAGE_DEFORM_FACES, stream);
        if (one_ring)
            launch_pdl(one_ring_faces_kernel, grid_for(nf, 256), 256, 0, stream, V, Vd, F, nv, nf, ctx->vacc.as<float>(),
                                                                         status);
        else
            launch_pdl(face_gradients_kernel, grid_for(nf, 256), 256, 0, stream, V, Vd, F, nv, nf, ctx->vacc.as<float>(),
                                                                         status);
    }
    {
        StageTimer tm(ctx, UMGS_STAGE_DEFORM_VERTICES, stream);
        if (one_ring)
            launch_pdl(one_ring_vertices_kernel, grid_for(nv, 256), 256, 0, stream, V, Vd, ctx->vacc.as<float>(), nv,
                                                                            ctx->vtab.as<float>());
        else
            launch_pdl(vertex_xforms_kernel, grid_for(nv, 256), 256, 0, stream, V, Vd, ctx->vacc.as<float>(), nv,
                                                                        ctx->vtab.as<float>());
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "proxy table kernels");
    return UMGS_OK;
}

umgs_status deform_forward(umgs_ctx* ctx, const umgs_gaussians* g, const int32_t* face, const float* bary,
                           const float* V, const float* Vd, const int32_t* F, int64_t nv, int64_t nf, int32_t mode,
                           float* out_means, float* out_cov, float* out_quats, cudaStream_t stream) {
    const umgs_status st = proxy_table(ctx, V, Vd, F, nv, nf, (mode & UMGS_DEFORM_ONE_RING) != 0, stream);
    mode &= 1;  // the mean update: FRAME or LITERAL
    if (st != UMGS_OK) return st;
    StageTimer tm(ctx, UMGS_STAGE_DEFORM_GAUSSIANS, stream);
    if (g->n > 0)
        launch_pdl(deform_gaussians_kernel, grid_for(8 * g->n, 256), 256, 0, stream, 
            g->means, g->quats, g->scales, g->cov3d, g->n, face, bary, V, F, nv, nf, ctx->vtab.as<float>(), mode,
            out_means, out_cov, out_quats, ctx->dstatus.as<int32_t>());
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "deform kernels");
    return UMGS_OK;
}

umgs_status binding_compact(umgs_ctx* ctx, const int32_t* face, const float* bary, int64_t n, const int32_t* F,
                            int64_t nv, int64_t nf, int32_t* out_count, int2* out_entries, cudaStream_t stream) {
    if (n > 0)
        binding_compact_kernel<<<grid_for(n, 256), 256, 0, stream>>>(face, bary, n, F, nv, nf, out_count,
                                                                     out_entries), count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "binding_compact_kernel");
    return UMGS_OK;
}

umgs_status binding_csr(umgs_ctx* ctx, const int32_t* face, const float* bary, int64_t n, const int32_t* F,
                        int64_t nv, int64_t nf, int32_t* out_offsets, int2* out_entries, int64_t cap,
                        int64_t* out_total, cudaStream_t stream) {
    cudaError_t e;
    if ((e = ctx->bind_cnt.reserve(sizeof(uint32_t) * std::max<int64_t>(1, n) + 16)) != cudaSuccess)
        return fail(ctx, UMGS_ERR_OUT_OF_MEMORY, "CSR counts");
    uint32_t* cnt = ctx->bind_cnt.as<uint32_t>();
    unsigned long long* tot = reinterpret_cast<unsigned long long*>(cnt + ((std::max<int64_t>(1, n) + 1) & ~1LL));
    if (n > 0)
        binding_csr_count_kernel<<<grid_for(n, 256), 256, 0, stream>>>(face, bary, n, F, nv, nf, cnt), count_launch();
    binding_csr_scan_kernel<<<1, 1024, 0, stream>>>(cnt, n, out_offsets, tot), count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "binding_csr kernels");
    unsigned long long total = 0;
    if ((e = cudaMemcpyAsync(ctx->pinned, tot, sizeof(total), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "reading the CSR size");
    std::memcpy(&total, ctx->pinned, sizeof(total));
    *out_total = (int64_t)total;
    if (total > 0x7fffffffull) return fail(ctx, UMGS_ERR_CAPACITY, "more than 2^31 - 1 binding entries");
    if ((int64_t)total > cap)
        return fail(ctx, UMGS_ERR_CAPACITY, "entries capacity " + std::to_string(cap) + " < " + std::to_string(total));
    if (n > 0)
        binding_csr_fill_kernel<<<grid_for(n, 256), 256, 0, stream>>>(face, bary, n, F, nv, nf, out_offsets,
                                                                      out_entries), count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "binding_csr_fill_kernel");
    return UMGS_OK;
}

umgs_status deform_compact_forward(umgs_ctx* ctx, const umgs_gaussians* g, const int32_t* count, const int2* entries,
                                   const float* V, const float* Vd, const int32_t* F, int64_t nv, int64_t nf,
                                   int32_t mode, float* out_means, float* out_cov, float* out_quats,
                                   cudaStream_t stream, bool csr) {
    const umgs_status st = proxy_table(ctx, V, Vd, F, nv, nf, (mode & UMGS_DEFORM_ONE_RING) != 0, stream);
    mode &= 1;  // the mean update: FRAME or LITERAL
    if (st != UMGS_OK) return st;
    StageTimer tm(ctx, UMGS_STAGE_DEFORM_GAUSSIANS, stream);
    if (g->n > 0) {
        if (csr)
            launch_pdl(deform_gaussians_compact_kernel<true>, grid_for(g->n, kDefBlock), kDefBlock, 0, stream,
                g->means, g->quats, g->scales, g->cov3d, g->n, count, entries, nv, ctx->vtab.as<float>(), mode,
                out_means, out_cov, out_quats, ctx->dstatus.as<int32_t>());
        else
            launch_pdl(deform_gaussians_compact_kernel<false>, grid_for(g->n, kDefBlock), kDefBlock, 0, stream,
                g->means, g->quats, g->scales, g->cov3d, g->n, count, entries, nv, ctx->vtab.as<float>(), mode,
                out_means, out_cov, out_quats, ctx->dstatus.as<int32_t>());
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "deform kernels");
    return UMGS_OK;
}

}  // namespace umgs

// ---------------------------------------------------------------------------
// Deformation without device allocation (no paper counterpart).
//
// Some callers cannot allocate device memory: a host application that
// reserves the whole device memory for its own allocator up front, a plugin
// inside a process whose device memory another runtime owns, or a real-time
// loop whose frame budget cannot absorb the synchronisation of cudaMalloc.
// umgs_deform_noalloc runs the same three deformation kernels as umgs_deform
// but keeps its scratch (per-vertex accumulators, vertex transform table and
// a status word) in the file-scope array below, so it needs no context and
// never calls cudaMalloc, cudaFree or any allocating library routine.
//
// The array holds UMGS_NOALLOC_MAX_PROXY_VERTICES vertices (26 floats each)
// plus 64 words; every GPU that loads the library keeps it (about 3.4 MB)
// until the process exits.  All calls share it: calls whose work overlaps
// on the GPU (other streams, other host threads) race on it.

namespace umgs {

constexpr int64_t kNoAllocMaxVerts = UMGS_NOALLOC_MAX_PROXY_VERTICES;
constexpr int64_t kNoAllocFloats = kNoAllocMaxVerts * (10 + kVtabStride) + 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

__global__ void noalloc_clear_kernel(float* __restrict__ p, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.f;
}

// Device address of g_noalloc_scratch on the current device, looked up once
// per device.  In host code the symbol is only a host-side stand-in, so the
// address must come from cudaGetSymbolAddress with that device current.  The
// cached address lives as long as the device's primary context: a
// cudaDeviceReset invalidates it (the header says so).
static cudaError_t noalloc_scratch_address(float** out) {
    constexpr int kMaxDev = 64;
    static float* addr[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = static_cast<float*>(p);
    }
    *out = addr[dev];
    return cudaSuccess;
}

}  // namespace umgs

extern "C" umgs_status umgs_deform_noalloc(const umgs_gaussians* rest, const int32_t* face, const float* bary,
                                           const float* proxy_v, const float* proxy_vd, const int32_t* proxy_f,
                                           int64_t nv, int64_t nf, int32_t mode, float* out_means,
                                           float* out_cov3d, float* out_quats, void* stream) {
    using namespace umgs;
    if (!rest || rest->n < 0) return UMGS_ERR_INVALID_ARG;
    if (mode != UMGS_DEFORM_FRAME && mode != UMGS_DEFORM_LITERAL) return UMGS_ERR_INVALID_ARG;
    if (!proxy_v || !proxy_vd || !proxy_f || nv < 3 || nf < 1) return UMGS_ERR_INVALID_ARG;
    if (nv > kNoAllocMaxVerts) return UMGS_ERR_CAPACITY;
    if (rest->n > 0) {
        if (!rest->means || !face || !bary || !out_means || !out_cov3d) return UMGS_ERR_INVALID_ARG;
        if (!rest->cov3d && (!rest->quats || !rest->scales)) return UMGS_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(face) | reinterpret_cast<uintptr_t>(bary)) & 15) return UMGS_ERR_INVALID_ARG;
    }
    float* base = nullptr;
    if (noalloc_scratch_address(&base) != cudaSuccess) return UMGS_ERR_CUDA;
    float* vacc = base;                                   // [nv,10]
    float* vtab = base + 10 * kNoAllocMaxVerts;           // [nv,16]
    int32_t* status = reinterpret_cast<int32_t*>(base + (10 + kVtabStride) * kNoAllocMaxVerts);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the accumulators and the status word keep the previous call's values
    noalloc_clear_kernel<<<grid_for(10 * nv, 256), 256, 0, s>>>(vacc, 10 * nv), count_launch();
    noalloc_clear_kernel<<<1, 64, 0, s>>>(reinterpret_cast<float*>(status), 64), count_launch();
    face_gradients_kernel<<<grid_for(nf, 256), 256, 0, s>>>(proxy_v, proxy_vd, proxy_f, nv, nf, vacc, status), count_launch();
    vertex_xforms_kernel<<<grid_for(nv, 256), 256, 0, s>>>(proxy_v, proxy_vd, vacc, nv, vtab), count_launch();
    if (rest->n > 0)
        deform_gaussians_kernel<<<grid_for(8 * rest->n, 256), 256, 0, s>>>(
            rest->means, rest->quats, rest->scales, rest->cov3d, rest->n, face, bary, proxy_v, proxy_f, nv, nf, vtab,
            mode, out_means, out_cov3d, out_quats, status), count_launch();
    return cudaGetLastError() == cudaSuccess ? UMGS_OK : UMGS_ERR_CUDA;
}
