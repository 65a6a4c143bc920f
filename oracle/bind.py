"""Brute-force Gaussian-centric binding (test infrastructure only).

Sec. 3.3 "Binding Gaussians to Mesh": from every training camera a ray is cast
towards the Gaussian centre (UniMGS*, mode CENTER) or towards each of the 8
corners of the Gaussian's bounding box (UniMGS, mode BBX); every face the ray
hits is a candidate, and the target is bound to the candidate whose hit point
is nearest to it.  The face index, the barycentric coordinate of the hit
point and the distance are recorded.

Readings where the paper is silent:
  * a ray is the half-line o + t (p - o), t > 0, from the camera centre o
    through the target p and beyond; every hit counts, not only the first;
  * BBX corner i = mu + R_q (+-k s_x, +-k s_y, +-k s_z) with k = 3 (bit 0 of i
    selects the x sign, bit 1 y, bit 2 z; a set bit means +);
  * distance = |t - 1| * |p - o| (the hit point is o + t(p - o));
  * ties: lower camera index, then lower face index;
  * a target that no ray hits falls back to the closest point on the mesh
    (region method for the closest point on a triangle), flagged; mode
    NEAREST uses the closest point for every target.

All arithmetic is canonical float32 (each numpy float32 op is one correctly
rounded IEEE operation, no FMA), so the result is a bit-exact reference.
The ray/triangle test is the Moller-Trumbore formulation.
Barycentric output (b1, b2): weights of face vertices 1 and 2; vertex 0
gets 1 - b1 - b2.
"""
from __future__ import annotations

import numpy as np

from .canonical import camera_center, quat_to_rotmat

F32 = np.float32
BBX, CENTER, NEAREST = 0, 1, 2
FLAG_HIT, FLAG_FALLBACK = 1, 2


def targets(means, quats, scales, mode, k_sigma=3.0):
    """[N,8,3] float32 target points (CENTER repeats mu 8 times)."""
    mu = np.asarray(means, np.float32)
    n = mu.shape[0]
    out = np.zeros((n, 8, 3), np.float32)
    if mode in (CENTER, NEAREST):
        out[:] = mu[:, None, :]
        return out
    r = quat_to_rotmat(quats)
    s = np.asarray(scales, np.float32)
    ks = [F32(k_sigma) * s[:, j] for j in range(3)]
    for i in range(8):
        off = [ks[j] if (i >> j) & 1 else -ks[j] for j in range(3)]
        for a in range(3):
            out[:, i, a] = mu[:, a] + ((r[a][0] * off[0] + r[a][1] * off[1]) + r[a][2] * off[2])
    return out


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]


def ray_hits(o, p, V, F):
    """Moller-Trumbore of the ray o + t(p - o) against all faces.

    o, p: float32 [3]; returns (hit [F] bool, u [F], v [F], dist [F]) in float32.
    """
    V = np.asarray(V, np.float32)
    F = np.asarray(F, np.int64)
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    d = [p[k] - o[k] for k in range(3)]
    with np.errstate(all="ignore"):
        e1 = [B[:, k] - A[:, k] for k in range(3)]
        e2 = [C[:, k] - A[:, k] for k in range(3)]
        pv = _cross(d, e2)
        det = _dot(e1, pv)
        tv = [o[k] - A[:, k] for k in range(3)]
        un = _dot(tv, pv)
        qv = _cross(tv, e1)
        vn = _dot(d, qv)
        tn = _dot(e2, qv)
        u = un / det
        v = vn / det
        t = tn / det
        hit = (det != 0) & (u >= 0) & (v >= 0) & ((u + v) <= F32(1)) & (t > 0) & np.isfinite(t)
        dn = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
        dist = np.abs(t - F32(1)) * dn
    return hit, u.astype(np.float32), v.astype(np.float32), dist.astype(np.float32)


def closest_points(p, V, F):
    """Closest point of every face to p (region method, canonical float32).

    Returns (b1 [F], b2 [F], dist2 [F]); the closest point is
    a + (ab*b1 + ac*b2) with a = vertex 0, ab = v1 - v0, ac = v2 - v0.
    """
    V = np.asarray(V, np.float32)
    F = np.asarray(F, np.int64)
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nf = len(F)
    with np.errstate(all="ignore"):
        ab = [B[:, k] - A[:, k] for k in range(3)]
        ac = [C[:, k] - A[:, k] for k in range(3)]
        ap = [p[k] - A[:, k] for k in range(3)]
        d1 = _dot(ab, ap)
        d2 = _dot(ac, ap)
        bp = [p[k] - B[:, k] for k in range(3)]
        d3 = _dot(ab, bp)
        d4 = _dot(ac, bp)
        cp = [p[k] - C[:, k] for k in range(3)]
        d5 = _dot(ab, cp)
        d6 = _dot(ac, cp)
        vc = d1 * d4 - d3 * d2
        vb = d5 * d2 - d1 * d6
        va = d3 * d6 - d5 * d4
        z = np.zeros(nf, np.float32)
        one = np.ones(nf, np.float32)
        r3 = d1 / (d1 - d3)
        r5 = d2 / (d2 - d6)
        n6 = d4 - d3
        m6 = d5 - d6
        r6 = n6 / (n6 + m6)
        den = (va + vb) + vc
        r7v = vb / den
        r7w = vc / den
        conds = [
            (d1 <= 0) & (d2 <= 0),
            (d3 >= 0) & (d4 <= d3),
            (vc <= 0) & (d1 >= 0) & (d3 <= 0),
            (d6 >= 0) & (d5 <= d6),
            (vb <= 0) & (d2 >= 0) & (d6 <= 0),
            (va <= 0) & (n6 >= 0) & (m6 >= 0),
        ]
        b1 = np.select(conds, [z, one, r3, z, z, one - r6], r7v).astype(np.float32)
        b2 = np.select(conds, [z, z, z, one, r5, r6], r7w).astype(np.float32)
        q = [A[:, k] + (ab[k] * b1 + ac[k] * b2) for k in range(3)]
        dd = [p[k] - q[k] for k in range(3)]
        dist2 = (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2]
    return b1, b2, dist2.astype(np.float32)


def bind(means, quats, scales, V, F, cam_viewmats, mode=BBX, k_sigma=3.0, gaussian_ids=None):
    """Brute-force binding.

    Returns dict face [n,8] int32, bary [n,8,2] float32, dist [n,8] float32,
    flags [n,8] uint8 (FLAG_HIT or FLAG_FALLBACK), for the Gaussians in
    gaussian_ids (all when None).
    """
    means = np.asarray(means, np.float32)
    ids = np.arange(len(means)) if gaussian_ids is None else np.asarray(gaussian_ids)
    tg = targets(means[ids], None if quats is None else np.asarray(quats)[ids],
                 None if scales is None else np.asarray(scales)[ids], mode, k_sigma)
    centres = [camera_center(vm) for vm in cam_viewmats]
    n = len(ids)
    face = np.full((n, 8), -1, np.int32)
    bary = np.zeros((n, 8, 2), np.float32)
    dist = np.zeros((n, 8), np.float32)
    flags = np.zeros((n, 8), np.uint8)
    nf = len(F)
    fidx = np.arange(nf)
    for gi in range(n):
        ncorner = 1 if mode in (CENTER, NEAREST) else 8
        for ci in range(ncorner):
            p = tg[gi, ci]
            best = None
            if mode != NEAREST:
                for cam, o in enumerate(centres):
                    hit, u, v, dd = ray_hits(o, p, V, F)
                    if not hit.any():
                        continue
                    hi = np.nonzero(hit)[0]
                    order = np.lexsort((hi, dd[hi]))
                    j = hi[order[0]]
                    cand = (float(dd[j]), cam, int(j), u[j], v[j], dd[j])
                    if best is None or (cand[0], cand[1], cand[2]) < (best[0], best[1], best[2]):
                        best = cand
            if best is not None:
                face[gi, ci] = best[2]
                bary[gi, ci] = (best[3], best[4])
                dist[gi, ci] = best[5]
                flags[gi, ci] = FLAG_HIT
            else:
                b1, b2, d2 = closest_points(p, V, F)
                order = np.lexsort((fidx, d2))
                j = order[0]
                face[gi, ci] = j
                bary[gi, ci] = (b1[j], b2[j])
                dist[gi, ci] = np.sqrt(d2[j])
                flags[gi, ci] = FLAG_FALLBACK
        if mode in (CENTER, NEAREST):
            face[gi, 1:] = face[gi, 0]
            bary[gi, 1:] = bary[gi, 0]
            dist[gi, 1:] = dist[gi, 0]
            flags[gi, 1:] = flags[gi, 0]
    return dict(face=face, bary=bary, dist=dist, flags=flags)
