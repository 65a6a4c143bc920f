"""Hand-built scenes for the pin tests (no method arithmetic here)."""
import numpy as np

from paper_2601_19233_gb300 import scenes as S


def cam(W=32, H=32, fx=None, dist=3.0):
    fx = fx if fx is not None else S.focal_from_fov(W, 60.0)
    return S.front_camera(W, H, fx, dist)


def gaussians(means, scales=None, quats=None, opac=None, colors=None):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = len(means)
    scales = np.full((n, 3), 0.05, np.float32) if scales is None else np.asarray(scales, np.float32).reshape(n, 3)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else np.asarray(quats, np.float32)
    opac = np.full(n, 0.8, np.float32) if opac is None else np.asarray(opac, np.float32).reshape(n)
    colors = np.full((n, 3), 0.5, np.float32) if colors is None else np.asarray(colors, np.float32).reshape(n, 3)
    sh = ((colors - 0.5) / S.SH_C0).astype(np.float32)[:, None, :]
    return S.Gaussians(means, quats, scales, opac, sh, 0)


def no_gaussians():
    return S.Gaussians(np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                       np.zeros((0, 3), np.float32), np.zeros(0, np.float32),
                       np.zeros((0, 1, 3), np.float32), 0)


def screen_quad(camera, z_world, alpha=1.0, color=(0.2, 0.4, 0.6), extent=None, split="diag"):
    """Two triangles forming a quad that covers the whole image, at world depth z."""
    Z = z_world + camera.viewmat[2, 3]
    W, H = camera.width, camera.height
    e = extent if extent is not None else 2.0
    x0 = (-e * W - camera.cx) * Z / camera.fx
    x1 = ((1 + e) * W - camera.cx) * Z / camera.fx
    y0 = (-e * H - camera.cy) * Z / camera.fy
    y1 = ((1 + e) * H - camera.cy) * Z / camera.fy
    V = np.array([[x0, y0, z_world], [x1, y0, z_world], [x1, y1, z_world], [x0, y1, z_world]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    col = np.tile(np.asarray(color, np.float32), (4, 1))
    return S.Mesh(V, F, col, None, np.full(2, alpha, np.float32))


def single_triangle(camera, pix_pts, z_world, alpha=1.0, colors=None):
    """A triangle whose vertices project to the given pixel coordinates."""
    Z = z_world + camera.viewmat[2, 3]
    V = []
    for (u, v) in pix_pts:
        V.append([(u - camera.cx) * Z / camera.fx, (v - camera.cy) * Z / camera.fy, z_world])
    V = np.array(V, np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    col = np.asarray(colors if colors is not None else [[0.9, 0.1, 0.3]] * 3, np.float32)
    return S.Mesh(V, F, col, None, np.array([alpha], np.float32))


def scene(g, meshes, camera, tile=8):
    return S.Scene(g, list(meshes), [camera], tile=tile)


def compare_with_ties(got, ref_rgb, ref_T, tie, alts, tol):
    """GPU RGB+T `got` [..., 4] against the fp64 oracle.  Every pixel is held
    to `tol` per channel: an ordinary pixel against the oracle's composite, a
    tie pixel (a decision within rounding distance of its threshold, which the
    fp32 kernels may take the other way) against the closest of its
    composite_alternatives (`alts`: flat pixel index -> [n_alt, 4]).
    Returns (max error of the ordinary pixels, number of tie pixels, tie
    pixels matching no alternative within tol, max error of the closest
    alternative over the tie pixels)."""
    got = np.asarray(got).reshape(-1, 4)
    ref = np.concatenate([np.asarray(ref_rgb).reshape(-1, 3), np.asarray(ref_T).reshape(-1, 1)], 1)
    tie = np.asarray(tie).reshape(-1)
    err = np.abs(got - ref).max(1)
    e_plain = float(err[~tie].max()) if (~tie).any() else 0.0
    bad, e_tie = 0, 0.0
    for k in np.nonzero(tie)[0]:
        e = float(np.abs(alts[int(k)] - got[k]).max(1).min())
        e_tie = max(e_tie, e)
        bad += e > tol
    return e_plain, int(tie.sum()), bad, e_tie
