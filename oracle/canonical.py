"""Canonical float32 decisions of the rasterizer (test infrastructure only).

Every operation here is a single IEEE-754 binary32 operation rounded to
nearest-even: numpy float32 ufuncs (add, subtract, multiply, divide, sqrt)
are correctly rounded and never fused, so the results are reproducible on any
machine.  These functions fix *which* fragments exist and in which order they
are blended; the fp64 image path in render.py reuses them, so the set and the
order of fragments are identical by construction.

Conventions (the paper leaves all of them open; Sec. 3.2 only says that
triangle fragments join the depth sort of the 3DGS rasterizer):
  * camera: world->camera [R|t], x right, y down, z forward; pixel (x, y) has
    its centre at (x+0.5, y+0.5); u = (fx*X)/Z + cx, v = (fy*Y)/Z + cy.
  * Gaussian footprint: the axis-aligned box of the 3-sigma ellipse of the
    dilated 2D covariance (EWA splatting as in 3DGS, Sec. 3.2 / Eq. 1-2).
  * triangles: vertices snapped to 1/256 px, integer edge functions, top-left
    fill rule, M = 4 samples per pixel (Eq. 4 sets M = 4) at the rotated-grid
    offsets (-2,-6), (6,-2), (-6,2), (2,6) / 16 px.
  * depth of a primitive: the view-space Z of the Gaussian mean, or the
    triangle's centroid Z computed as ((z0 + z1) + z2) / 3.
  * order: ascending (tile, depth bits, unified id); unified ids are Gaussians
    [0, Ng) followed by the triangles of mesh 0, mesh 1, ...
"""
from __future__ import annotations

import numpy as np

F32 = np.float32
SNAP = 256                       # sub-pixel units per pixel
MAX_SCREEN = 16384.0             # triangles with a vertex beyond this are culled
SAMPLE_OFFSETS = np.array([[-32, -96], [96, -32], [-96, 32], [32, 96]], np.int64)  # 1/256 px
DILATION = F32(0.3)
JAC_CLAMP = F32(1.3)
SIGMA_EXTENT = F32(3.0)


def _f(x):
    return np.asarray(x, dtype=np.float32)


def view_transform(viewmat, pts):
    """p_cam = R p + t, each component ((r0*x + r1*y) + r2*z) + t."""
    vm = _f(viewmat)
    p = _f(pts)
    out = []
    for i in range(3):
        out.append(((vm[i, 0] * p[:, 0] + vm[i, 1] * p[:, 1]) + vm[i, 2] * p[:, 2]) + vm[i, 3])
    return out


def camera_center(viewmat):
    """c = -R^T t, each component -((R0i*t0 + R1i*t1) + R2i*t2)."""
    vm = _f(viewmat)
    t = vm[:, 3]
    return np.array([-((vm[0, i] * t[0] + vm[1, i] * t[1]) + vm[2, i] * t[2]) for i in range(3)], np.float32)


def quat_to_rotmat(q):
    """Rotation matrix of the normalised quaternion (w, x, y, z); rows r[i][j]."""
    q = _f(q)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    n = np.sqrt(((w * w + x * x) + y * y) + z * z)
    zero = n == 0
    n = np.where(zero, F32(1), n)
    w = np.where(zero, F32(1), w / n)
    x = np.where(zero, F32(0), x / n)
    y = np.where(zero, F32(0), y / n)
    z = np.where(zero, F32(0), z / n)
    two = F32(2)
    one = F32(1)
    r = [[None] * 3 for _ in range(3)]
    r[0][0] = one - two * (y * y + z * z)
    r[0][1] = two * (x * y - w * z)
    r[0][2] = two * (x * z + w * y)
    r[1][0] = two * (x * y + w * z)
    r[1][1] = one - two * (x * x + z * z)
    r[1][2] = two * (y * z - w * x)
    r[2][0] = two * (x * z - w * y)
    r[2][1] = two * (y * z + w * x)
    r[2][2] = one - two * (x * x + y * y)
    return r


def cov3d_from_quat_scale(q, s):
    """Sigma = (R S)(R S)^T, returned as the 6 entries xx, xy, xz, yy, yz, zz."""
    r = quat_to_rotmat(q)
    s = _f(s)
    M = [[r[i][j] * s[:, j] for j in range(3)] for i in range(3)]

    def e(i, j):
        return (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2]

    return [e(0, 0), e(0, 1), e(0, 2), e(1, 1), e(1, 2), e(2, 2)]


def _sym(c6):
    xx, xy, xz, yy, yz, zz = c6
    return [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]


def project_gaussians(means, quats, scales, cov3d, cam):
    """Canonical projection of Gaussians for one camera.

    Returns a dict of float32/int arrays: valid, u, v, Z, a, b, c (dilated 2D
    covariance), rect (x_lo, x_hi, y_lo, y_hi; inclusive, clipped to the image).
    """
    vm = _f(cam.viewmat)
    fx, fy, cx, cy = F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy)
    W, H = int(cam.width), int(cam.height)
    X, Y, Z = view_transform(vm, means)
    with np.errstate(all="ignore"):
        valid = Z > F32(cam.near)
        u = (fx * X) / Z + cx
        v = (fy * Y) / Z + cy
        if cov3d is not None:
            c6 = [_f(cov3d)[:, k] for k in range(6)]
        else:
            c6 = cov3d_from_quat_scale(quats, scales)
        S = _sym(c6)
        two = F32(2)
        lim_x = JAC_CLAMP * (F32(W) / (two * fx))
        lim_y = JAC_CLAMP * (F32(H) / (two * fy))
        xc = np.minimum(lim_x, np.maximum(-lim_x, X / Z)) * Z
        yc = np.minimum(lim_y, np.maximum(-lim_y, Y / Z)) * Z
        z2 = Z * Z
        j00 = fx / Z
        j11 = fy / Z
        j02 = -((fx * xc) / z2)
        j12 = -((fy * yc) / z2)
        T0 = [j00 * vm[0, k] + j02 * vm[2, k] for k in range(3)]
        T1 = [j11 * vm[1, k] + j12 * vm[2, k] for k in range(3)]
        U0 = [(T0[0] * S[0][k] + T0[1] * S[1][k]) + T0[2] * S[2][k] for k in range(3)]
        U1 = [(T1[0] * S[0][k] + T1[1] * S[1][k]) + T1[2] * S[2][k] for k in range(3)]
        a = (U0[0] * T0[0] + U0[1] * T0[1]) + U0[2] * T0[2]
        b = (U0[0] * T1[0] + U0[1] * T1[1]) + U0[2] * T1[2]
        c = (U1[0] * T1[0] + U1[1] * T1[1]) + U1[2] * T1[2]
        a = a + DILATION
        c = c + DILATION
        det = a * c - b * b
        rx = SIGMA_EXTENT * np.sqrt(a)
        ry = SIGMA_EXTENT * np.sqrt(c)
        half = F32(0.5)
        valid = valid & (det > 0) & np.isfinite(u) & np.isfinite(v) & np.isfinite(rx) & np.isfinite(ry)
        xlo = np.maximum(np.ceil((u - rx) - half), F32(0))
        xhi = np.minimum(np.floor((u + rx) - half), F32(W - 1))
        ylo = np.maximum(np.ceil((v - ry) - half), F32(0))
        yhi = np.minimum(np.floor((v + ry) - half), F32(H - 1))
        valid = valid & (xlo <= xhi) & (ylo <= yhi)
    rect = np.zeros((len(Z), 4), np.int64)
    rect[valid, 0] = xlo[valid].astype(np.int64)
    rect[valid, 1] = xhi[valid].astype(np.int64)
    rect[valid, 2] = ylo[valid].astype(np.int64)
    rect[valid, 3] = yhi[valid].astype(np.int64)
    return dict(valid=valid, u=u, v=v, Z=Z, a=a, b=b, c=c, rect=rect)


def _floordiv(a, b):
    return np.floor_divide(a, b)


def setup_triangles(verts, faces, cam, dilate=0):
    """Canonical triangle setup for one camera.  `dilate` widens the pixel
    rect by that many pixels on every side before clipping (soft-edge
    coverage, where a triangle reaches pixels near but outside its samples).

    Returns dict: valid, sx, sy (int64 [F,3] snapped coords, original vertex
    order), A, B (int64 [F,3]), Cb (int64 [F,3], edge constant with the
    top-left bias folded in), Cu (unbiased constant), rect (int64 [F,4]),
    depth (float32 [F]).  Edge k is the edge opposite vertex k of the
    (orientation-corrected) triangle; covered(p) <=> all_k A_k px + B_k py + Cb_k >= 0.
    """
    vm = _f(cam.viewmat)
    fx, fy, cx, cy = F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy)
    W, H = int(cam.width), int(cam.height)
    X, Y, Z = view_transform(vm, verts)
    with np.errstate(all="ignore"):
        u = (fx * X) / Z + cx
        v = (fy * Y) / Z + cy
        lim = F32(MAX_SCREEN)
        vok = (Z > F32(cam.near)) & np.isfinite(u) & np.isfinite(v) & (np.abs(u) <= lim) & (np.abs(v) <= lim)
        su = np.where(vok, np.rint(F32(SNAP) * u), F32(0)).astype(np.int64)
        sv = np.where(vok, np.rint(F32(SNAP) * v), F32(0)).astype(np.int64)
    f = np.asarray(faces, np.int64)
    valid = vok[f].all(1)
    sx = su[f]
    sy = sv[f]
    Zf = Z[f]
    area = (sx[:, 1] - sx[:, 0]) * (sy[:, 2] - sy[:, 0]) - (sx[:, 2] - sx[:, 0]) * (sy[:, 1] - sy[:, 0])
    valid &= area != 0
    flip = area < 0
    ox = sx.copy()
    oy = sy.copy()
    ox[flip, 1], ox[flip, 2] = sx[flip, 2], sx[flip, 1]
    oy[flip, 1], oy[flip, 2] = sy[flip, 2], sy[flip, 1]
    A = np.zeros_like(ox)
    B = np.zeros_like(ox)
    Cu = np.zeros_like(ox)
    Cb = np.zeros_like(ox)
    for k in range(3):
        a_ = (k + 1) % 3
        b_ = (k + 2) % 3
        A[:, k] = oy[:, a_] - oy[:, b_]
        B[:, k] = ox[:, b_] - ox[:, a_]
        Cu[:, k] = ox[:, a_] * oy[:, b_] - oy[:, a_] * ox[:, b_]
        topleft = (A[:, k] > 0) | ((A[:, k] == 0) & (B[:, k] > 0))
        Cb[:, k] = Cu[:, k] - np.where(topleft, 0, 1)
    xmin, xmax = sx.min(1), sx.max(1)
    ymin, ymax = sy.min(1), sy.max(1)
    xlo = np.maximum(-_floordiv(-(xmin - 224), SNAP) - dilate, 0)
    xhi = np.minimum(_floordiv(xmax - 32, SNAP) + dilate, W - 1)
    ylo = np.maximum(-_floordiv(-(ymin - 224), SNAP) - dilate, 0)
    yhi = np.minimum(_floordiv(ymax - 32, SNAP) + dilate, H - 1)
    valid &= (xlo <= xhi) & (ylo <= yhi)
    rect = np.stack([xlo, xhi, ylo, yhi], 1)
    rect[~valid] = 0
    with np.errstate(all="ignore"):
        depth = ((Zf[:, 0] + Zf[:, 1]) + Zf[:, 2]) / F32(3)
    return dict(valid=valid, sx=sx, sy=sy, A=A, B=B, Cb=Cb, Cu=Cu, rect=rect, depth=depth,
                u=u[f], v=v[f], flip=flip)


def sample_coverage(A, B, Cb, px, py):
    """4-bit coverage mask of pixel (px, py) for triangles with edge data
    A, B, Cb ([K,3] int64).  Bit j is sample j of SAMPLE_OFFSETS."""
    A = np.asarray(A, np.int64)
    B = np.asarray(B, np.int64)
    Cb = np.asarray(Cb, np.int64)
    cxs = np.int64(px) * SNAP + 128
    cys = np.int64(py) * SNAP + 128
    mask = np.zeros(A.shape[0], np.int64)
    for j in range(4):
        sxp = cxs + SAMPLE_OFFSETS[j, 0]
        syp = cys + SAMPLE_OFFSETS[j, 1]
        e = A * sxp + B * syp + Cb
        inside = (e >= 0).all(1)
        mask |= inside.astype(np.int64) << j
    return mask


def centre_coverage(A, B, Cb, px, py):
    """Coverage of the pixel centre alone (used by the DIRECT ablation)."""
    A = np.asarray(A, np.int64)
    B = np.asarray(B, np.int64)
    Cb = np.asarray(Cb, np.int64)
    e = A * (np.int64(px) * SNAP + 128) + B * (np.int64(py) * SNAP + 128) + Cb
    return (e >= 0).all(1)


def depth_bits(z):
    return _f(z).view(np.uint32).astype(np.uint64)


class Primitives:
    """Canonical per-camera decisions for a whole scene (Gaussians + meshes)."""

    def __init__(self, scene, cam_index=0, cov3d=None, dilate=0):
        g = scene.gaussians
        cam = scene.cameras[cam_index]
        self.cam = cam
        self.ng = g.n
        pg = project_gaussians(g.means, g.quats, g.scales, cov3d, cam)
        self.g = pg
        self.tris = []
        rects = [pg["rect"]]
        valids = [pg["valid"]]
        depths = [pg["Z"]]
        off = g.n
        self.mesh_offsets = []
        for m in scene.meshes:
            t = setup_triangles(m.verts, m.faces, cam, dilate)
            self.tris.append(t)
            self.mesh_offsets.append(off)
            off += m.nf
            rects.append(t["rect"])
            valids.append(t["valid"])
            depths.append(t["depth"])
        self.n = off
        self.rect = np.concatenate(rects, 0)
        self.valid = np.concatenate(valids, 0)
        self.depth = np.concatenate(depths, 0).astype(np.float32)
        self.dbits = depth_bits(self.depth)
        # triangle edge data concatenated over meshes, indexed by (id - ng)
        if self.tris:
            # orientation of each triangle: the sign of its snapped integer area
            self.tri_sign = np.concatenate(
                [np.sign((t["sx"][:, 1] - t["sx"][:, 0]) * (t["sy"][:, 2] - t["sy"][:, 0])
                         - (t["sx"][:, 2] - t["sx"][:, 0]) * (t["sy"][:, 1] - t["sy"][:, 0])) for t in self.tris], 0)
            self.A = np.concatenate([t["A"] for t in self.tris], 0)
            self.B = np.concatenate([t["B"] for t in self.tris], 0)
            self.Cb = np.concatenate([t["Cb"] for t in self.tris], 0)
            self.Cu = np.concatenate([t["Cu"] for t in self.tris], 0)
        else:
            self.A = self.B = self.Cb = self.Cu = np.zeros((0, 3), np.int64)
            self.tri_sign = np.zeros(0, np.int64)

    def tile_rects(self, ts):
        r = self.rect
        return np.stack([r[:, 0] // ts, r[:, 1] // ts, r[:, 2] // ts, r[:, 3] // ts], 1)

    def tiles_touched(self, ts):
        tr = self.tile_rects(ts)
        n = (tr[:, 1] - tr[:, 0] + 1) * (tr[:, 3] - tr[:, 2] + 1)
        return np.where(self.valid, n, 0)


def sorted_tile_lists(prims_per_cam, ts):
    """Sorted (tile, depth, id) lists for all cameras.

    Returns (tile_ptr [n_tiles_total+1], ids [K] int64, dbits [K] uint32) where
    tile t of camera c has global index c*tiles_per_cam + ty*tiles_x + tx and
    its list is ids[tile_ptr[t]:tile_ptr[t+1]] in ascending (depth bits, id).
    """
    all_tile = []
    all_id = []
    all_db = []
    tiles_total = 0
    for P in prims_per_cam:
        W, H = P.cam.width, P.cam.height
        tx_n = (W + ts - 1) // ts
        ty_n = (H + ts - 1) // ts
        tr = P.tile_rects(ts)
        ids = np.nonzero(P.valid)[0]
        w = tr[ids, 1] - tr[ids, 0] + 1
        h = tr[ids, 3] - tr[ids, 2] + 1
        cnt = w * h
        rep = np.repeat(np.arange(len(ids)), cnt)
        start = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)
        k = np.arange(int(cnt.sum()), dtype=np.int64) - start[rep]
        tx = tr[ids[rep], 0] + k % w[rep]
        ty = tr[ids[rep], 2] + k // w[rep]
        all_tile.append(tiles_total + ty * tx_n + tx)
        all_id.append(ids[rep].astype(np.int64))
        all_db.append(P.dbits[ids[rep]])
        tiles_total += tx_n * ty_n
    tile = np.concatenate(all_tile) if all_tile else np.zeros(0, np.int64)
    ids = np.concatenate(all_id) if all_id else np.zeros(0, np.int64)
    db = np.concatenate(all_db) if all_db else np.zeros(0, np.uint64)
    order = np.lexsort((ids, db, tile))
    tile, ids, db = tile[order], ids[order], db[order]
    ptr = np.zeros(tiles_total + 1, np.int64)
    np.add.at(ptr, tile + 1, 1)
    ptr = np.cumsum(ptr)
    return ptr, ids, db.astype(np.uint32)
