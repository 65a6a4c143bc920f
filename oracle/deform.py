"""fp64 deformation transfer from a proxy mesh to Gaussians (test infrastructure only).

Sec. 3.3 "Deformation Transfer": every proxy vertex carries an offset
Delta = V' - V and a transform D = R S (polar decomposition); Eq. 12 carries
Delta, log R and S to the bound point P_i of each of the 8 BBX corners by
barycentric interpolation; Eq. 13 averages over the 8 corners and updates
the Gaussian: R' = exp(mean r_i), S' = mean S_i, Sigma' = R'S' Sigma (R'S')^T,
mu' = mu + mean Delta_i.

The paper obtains the per-vertex D from ACAP and does not restate it.  The
reading used here: a per-face deformation gradient D_f = F'_f F_f^-1 with the
frame F = [e1, e2, n / sqrt(|n|)] (e1 = v1 - v0, e2 = v2 - v0, n = e1 x e2),
then D_v = the rest-area-weighted mean of D_f over the faces around v, then
D_v = R_v S_v by polar decomposition (SVD; if det D_v < 0 the smallest
singular direction is flipped so R_v is a proper rotation), r_v = log R_v as
an axis-angle vector with angle in [0, pi].

A second reading (ONE_RING), closer to ACAP's own per-vertex fit: D_v is
the least-squares map of the vertex's one-ring edges, cotangent-weighted,
plus its area-weighted normal:
    D_v = argmin_D  sum_j c_vj |e'_vj - D e_vj|^2 + |n'_v - D n_v|^2
        = (sum_j c_vj e'_vj e_vj^T + n'_v n_v^T)(sum_j c_vj e_vj e_vj^T + n_v n_v^T)^-1
with e_vj = V_j - V_v over the edges at v, c_vj = sum over the faces holding
the edge of max(0, cot(angle opposite the edge) / 2), N_v = sum over the
faces at v of e1 x e2 and n_v = N_v / sqrt(|N_v|) (the normal term keeps a
flat one-ring well posed); primes are the deformed mesh.  Rigid motions and
uniform scalings give D_v = R and s I exactly.

Eq. 13's mean update mu' = mu + mean Delta_i is exact only for translations;
mode FRAME (default) adds (R'S' - I)(mu - P_bar), P_bar = mean P_i, so that a
rigidly moved proxy moves the bound Gaussians rigidly.  Mode LITERAL is Eq. 13
as printed.  Barycentrics: face vertices (v0, v1, v2) get weights
(1 - b1 - b2, b1, b2) where (b1, b2) is the stored binding coordinate.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

from .render import cov3d_fp64, quat_rotmat_fp64

FRAME, LITERAL = 0, 1
FACES, ONE_RING = "faces", "one_ring"  # per-vertex transform readings


def face_frames(V, F):
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    e1 = V[F[:, 1]] - V[F[:, 0]]
    e2 = V[F[:, 2]] - V[F[:, 0]]
    n = np.cross(e1, e2)
    nn = np.linalg.norm(n, axis=1)
    n3 = n / np.sqrt(nn)[:, None]
    return np.stack([e1, e2, n3], -1), 0.5 * nn  # columns e1, e2, n3; area


def vertex_transforms(V, Vd, F, method=FACES):
    """Per-vertex offset Delta [Nv,3], log-rotation r [Nv,3], stretch S [Nv,3,3]."""
    if method == ONE_RING:
        Dv = one_ring_gradients(V, Vd, F)
    else:
        _, area = face_frames(V, F)
        Df = face_gradients(V, Vd, F)
        nv = len(V)
        F = np.asarray(F, np.int64)
        Dv = np.zeros((nv, 3, 3))
        wv = np.zeros(nv)
        for k in range(3):
            np.add.at(Dv, F[:, k], area[:, None, None] * Df)
            np.add.at(wv, F[:, k], area)
        Dv = Dv / wv[:, None, None]
    r, S = polar_log(Dv)
    delta = np.asarray(Vd, np.float64) - np.asarray(V, np.float64)
    return delta, r, S


def face_gradients(V, Vd, F):
    """D_f = F'_f F_f^-1 per face."""
    Fr, _ = face_frames(V, F)
    Fd, _ = face_frames(Vd, F)
    return Fd @ np.linalg.inv(Fr)


def one_ring_gradients(V, Vd, F):
    """D_v of the ONE_RING reading (module docstring), every vertex."""
    V = np.asarray(V, np.float64)
    Vd = np.asarray(Vd, np.float64)
    F = np.asarray(F, np.int64)
    nv = len(V)
    A = np.zeros((nv, 3, 3))
    B = np.zeros((nv, 3, 3))
    P, Q = V[F], Vd[F]
    for k in range(3):
        i, j = (k + 1) % 3, (k + 2) % 3
        u1, u2 = P[:, i] - P[:, k], P[:, j] - P[:, k]
        cot = (u1 * u2).sum(1) / np.linalg.norm(np.cross(u1, u2), axis=1)
        w = np.maximum(0.5 * cot, 0.0)
        e, ed = P[:, j] - P[:, i], Q[:, j] - Q[:, i]
        EE = w[:, None, None] * e[:, :, None] * e[:, None, :]
        DE = w[:, None, None] * ed[:, :, None] * e[:, None, :]
        for v in (i, j):
            np.add.at(A, F[:, v], EE)
            np.add.at(B, F[:, v], DE)
    N = np.zeros((nv, 3))
    Nd = np.zeros((nv, 3))
    nf = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    ndf = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0])
    for k in range(3):
        np.add.at(N, F[:, k], nf)
        np.add.at(Nd, F[:, k], ndf)
    n = N / np.sqrt(np.linalg.norm(N, axis=1))[:, None]
    nd = Nd / np.sqrt(np.linalg.norm(Nd, axis=1))[:, None]
    A += n[:, :, None] * n[:, None, :]
    B += nd[:, :, None] * n[:, None, :]
    return B @ np.linalg.inv(A)


def polar_log(D):
    """D = R S (R proper rotation, S symmetric) by SVD, and r = log R (axis-angle)."""
    U, s, Vt = np.linalg.svd(D)
    neg = np.linalg.det(U @ Vt) < 0
    U[neg, :, 2] *= -1.0
    R = U @ Vt
    S = np.transpose(R, (0, 2, 1)) @ D
    S = 0.5 * (S + np.transpose(S, (0, 2, 1)))
    r = Rotation.from_matrix(R).as_rotvec()
    return r, S


def deform_gaussians(means, quats, scales, face, bary, V, Vd, F, mode=FRAME, cov3d=None, method=FACES, table=None):
    """Eq. 12-13 for every Gaussian.

    face [N,8] int, bary [N,8,2] (weights of face vertices 1 and 2).
    table: the per-vertex (Delta, r, S) of vertex_transforms(V, Vd, F, method)
    when the caller has it already (it depends on the proxy only).
    Returns (mu' [N,3], Sigma' [N,3,3], q' [N,4] (w,x,y,z), w >= 0).
    """
    delta, r, S = table if table is not None else vertex_transforms(V, Vd, F, method)
    Fi = np.asarray(F, np.int64)[np.asarray(face, np.int64)]           # [N,8,3]
    b = np.asarray(bary, np.float64)
    w = np.stack([1.0 - b[..., 0] - b[..., 1], b[..., 0], b[..., 1]], -1)  # [N,8,3]
    Vr = np.asarray(V, np.float64)
    P = np.einsum("nck,nckd->ncd", w, Vr[Fi])                           # bound points
    Di = np.einsum("nck,nckd->ncd", w, delta[Fi])
    ri = np.einsum("nck,nckd->ncd", w, r[Fi])
    Si = np.einsum("nck,nckde->ncde", w, S[Fi])
    rbar = ri.mean(1)
    Sbar = Si.mean(1)
    dbar = Di.mean(1)
    pbar = P.mean(1)
    Rp = Rotation.from_rotvec(rbar).as_matrix()
    A = Rp @ Sbar
    mu = np.asarray(means, np.float64)
    if mode == FRAME:
        mu2 = mu + dbar + np.einsum("nij,nj->ni", A - np.eye(3), mu - pbar)
    else:
        mu2 = mu + dbar
    Sig = np.asarray(cov3d, np.float64) if cov3d is not None else cov3d_fp64(quats, scales)
    Sig2 = A @ Sig @ np.transpose(A, (0, 2, 1))
    q = np.asarray(quats, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    qr = Rotation.from_rotvec(rbar) * Rotation.from_quat(q[:, [1, 2, 3, 0]])
    xyzw = qr.as_quat()
    q2 = xyzw[:, [3, 0, 1, 2]]
    q2 = np.where(q2[:, :1] < 0, -q2, q2)
    return mu2, Sig2, q2


def sym6(S):
    """[N,3,3] -> [N,6] (xx, xy, xz, yy, yz, zz)."""
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], -1)
