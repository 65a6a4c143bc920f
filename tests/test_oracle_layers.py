"""Pins of the oracle's expected depth and separate-pass composite (the
baseline Sec. 4.1 / Fig. 5b compares the single pass against)."""
import numpy as np

from oracle import layers as L
from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H


def test_gaussian_depth_is_the_mean_depth():
    # one Gaussian: wherever it blends, the expected depth is its camera depth
    c = H.cam(24, 24)
    g = H.gaussians([[0.05, -0.03, 0.4]], scales=[[0.3, 0.25, 0.1]], opac=[0.9])
    r = R.render_image(H.scene(g, [], c), t_eps=None)
    z = float(g.means[0, 2]) + float(c.viewmat[2, 3])  # front camera: camera z = world z + distance
    hit = np.isfinite(r["depth"])
    assert hit.sum() > 50
    assert np.abs(r["depth"][hit] - z).max() < 1e-12
    assert np.all(r["wsum"][~hit] == 0.0)


def test_triangle_depth_is_the_ray_plane_depth():
    # a tilted triangle: at pixel centres inside it, the perspective-correct
    # depth equals the depth where the pixel's ray meets the triangle's plane
    c = H.cam(32, 32)
    V = np.array([[-0.9, -0.8, -0.4], [0.9, -0.7, 0.5], [0.1, 0.9, 0.1]], np.float32)
    m = S.Mesh(V, np.array([[0, 1, 2]], np.int32), np.ones((3, 3), np.float32), None, np.ones(1, np.float32))
    sc = H.scene(H.no_gaussians(), [m], c)
    fr = R.Frame(sc)
    Rm, t = c.viewmat[:, :3].astype(np.float64), c.viewmat[:, 3].astype(np.float64)
    P = V.astype(np.float64) @ Rm.T + t
    n = np.cross(P[1] - P[0], P[2] - P[0])
    checked = 0
    for py in range(32):
        for px in range(32):
            frags = fr.fragments_at(px, py)
            if not frags or not frags[0]["centre"]:
                continue
            d = np.array([(px + 0.5 - c.cx) / c.fx, (py + 0.5 - c.cy) / c.fy, 1.0])
            z = np.dot(n, P[0]) / np.dot(n, d)  # camera depth of the ray's hit
            assert abs(frags[0]["z"] - z) < 1e-9 * z
            checked += 1
    assert checked > 100


def _disjoint(gauss_in_front):
    c = H.cam(32, 32)
    rng = np.random.default_rng(3)
    zg = -0.6 if gauss_in_front else 0.8
    means = np.stack([rng.uniform(-0.5, 0.5, 60), rng.uniform(-0.5, 0.5, 60), np.full(60, zg)], 1)
    g = H.gaussians(means, scales=np.full((60, 3), 0.08), opac=rng.uniform(0.3, 0.9, 60),
                    colors=rng.uniform(0, 1, (60, 3)))
    q = H.screen_quad(c, 0.2 if gauss_in_front else -0.7, 0.6, (0.2, 0.7, 0.4))
    t = H.single_triangle(c, [(3.0, 2.0), (30.0, 9.0), (12.0, 29.0)], 0.1 if gauss_in_front else -0.8, 0.5)
    return H.scene(g, [q, t], c), H.scene(g, [], c), H.scene(H.no_gaussians(), [q, t], c)


def test_separate_pass_equals_single_pass_when_layers_do_not_interleave():
    # with every Gaussian in front of every triangle (or every triangle in
    # front), the single pass is the two layers composited over each other
    for front in (True, False):
        full, ga, me = _disjoint(front)
        one = R.render_image(full, t_eps=None, bg=(0.1, 0.2, 0.3))
        a = R.render_image(ga, t_eps=None)
        b = R.render_image(me, t_eps=None)
        rgb, T = L.separate_pass(a, b, bg=(0.1, 0.2, 0.3))
        assert np.abs(rgb - one["rgb"]).max() < 1e-12
        assert np.abs(T - one["T"]).max() < 1e-12
        # and the nearer layer is the one the depth order picks
        both = np.isfinite(a["depth"]) & np.isfinite(b["depth"])
        assert both.sum() > 50
        assert np.all((a["depth"][both] < b["depth"][both]) == front)


def test_separate_pass_fails_nested_transparency():
    # Fig. 5b: Gaussians inside a transparent bowl; the per-pixel depth order
    # of whole layers cannot put them between the bowl's front and back
    # faces, so the separate pass differs visibly from the single pass
    sc, ga, me = S.nested_scene(size=64, n_gauss=1500)
    one = R.render_image(sc, t_eps=None)
    a = R.render_image(ga, t_eps=None)
    b = R.render_image(me, t_eps=None)
    rgb, _ = L.separate_pass(a, b)
    ok = ~one["tie"]
    assert np.abs(rgb - one["rgb"])[ok].max() > 0.05
