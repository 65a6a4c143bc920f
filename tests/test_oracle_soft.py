"""Pins of the soft-edge coverage oracle (an extension beyond the paper:
Eq. 7-9 with the binary sample coverage replaced by a product of edge
sigmoids, so that vertex positions get gradient through coverage).

* the coverage of a sample near one edge of a large triangle is the logistic
  function of its distance to that edge's line, written out from the line
  equation (closed form), for either vertex order;
* as sigma -> 0 the coverage becomes the point-in-triangle test of the
  sample, and the soft composite becomes the binary one;
* the numpy forward equals the torch forward, and the torch gradient equals
  central finite differences of the numpy forward, vertex positions included.
"""
import copy

import numpy as np
import pytest

from oracle import canonical as cn
from oracle import grad as G
from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H


def _samples(px, py):
    return [(px + 0.5 + cn.SAMPLE_OFFSETS[j, 0] / 256.0, py + 0.5 + cn.SAMPLE_OFFSETS[j, 1] / 256.0)
            for j in range(4)]


@pytest.mark.parametrize("flip", [False, True])
def test_coverage_is_the_logistic_of_the_edge_distance(flip):
    # edge on the vertical line x = 10.3, the triangle to its right; the other
    # two edges are ~900 px from the samples (their factors are 1 to 1e-300)
    tu = np.array([10.3, 10.3, 3000.0])
    tv = np.array([-1000.0, 1000.0, 0.0])
    if flip:
        tu, tv = tu[[0, 2, 1]], tv[[0, 2, 1]]
    for sigma in (0.25, 0.5, 1.0):
        for px in (8, 9, 10, 11):
            c = R.soft_coverage(tu[None], tv[None], px, 5, sigma)[0]
            want = [1.0 / (1.0 + np.exp(-(sx - 10.3) / sigma)) for sx, _ in _samples(px, 5)]
            assert np.abs(c - want).max() < 1e-12


def test_coverage_of_a_slanted_edge():
    # edge through (0, 0) and (40, 30): unit normal (-3, 4)/5 points into the
    # triangle (third vertex (0, 400) is on the +normal side)
    tu = np.array([0.0, 40.0, 0.0]) * 20
    tv = np.array([0.0, 30.0, 400.0]) * 20
    sigma = 0.6
    for (px, py) in [(20, 15), (21, 15), (19, 16), (40, 31)]:
        c = R.soft_coverage(tu[None], tv[None], px, py, sigma)[0]
        want = [1.0 / (1.0 + np.exp(-((-3 * sx + 4 * sy) / 5.0) / sigma)) for sx, sy in _samples(px, py)]
        assert np.abs(c - want).max() < 1e-9


def test_degenerate_triangle_covers_nothing():
    c = R.soft_coverage(np.array([[1.0, 5.0, 9.0]]), np.array([[1.0, 5.0, 9.0]]), 4, 4, 0.5)
    assert np.all(c == 0)


def test_small_sigma_is_the_point_in_triangle_test():
    rng = np.random.default_rng(4)
    for _ in range(200):
        tu = rng.uniform(0, 16, 3)
        tv = rng.uniform(0, 16, 3)
        px, py = int(rng.integers(0, 16)), int(rng.integers(0, 16))
        c = R.soft_coverage(tu[None], tv[None], px, py, 1e-4)[0]
        area = (tu[1] - tu[0]) * (tv[2] - tv[0]) - (tu[2] - tu[0]) * (tv[1] - tv[0])
        for j, (sx, sy) in enumerate(_samples(px, py)):
            lam = [(tu[(e + 1) % 3] - sx) * (tv[(e + 2) % 3] - sy) - (tu[(e + 2) % 3] - sx) * (tv[(e + 1) % 3] - sy)
                   for e in range(3)]
            L = [np.hypot(tu[(e + 2) % 3] - tu[(e + 1) % 3], tv[(e + 2) % 3] - tv[(e + 1) % 3]) for e in range(3)]
            dist = min(np.sign(area) * lam[e] / L[e] for e in range(3))
            if abs(dist) < 5e-3:
                continue
            assert c[j] == pytest.approx(1.0 if dist > 0 else 0.0, abs=1e-12)


def test_dilation():
    assert R.soft_dilation(None) == 0
    assert R.soft_dilation(0.5) == 4
    assert R.soft_dilation(0.3) == 3  # ceil(2.4000000953674316)
    assert R.soft_dilation(1.0) == 8


def _scene(seed, valpha=False, W=24, H=20, n=30):
    return S.small_scene(seed, W, H, n, mesh_subdiv=1, sh_degree=1, log_scale_mu=-2.8, with_valpha=valpha,
                         mesh_radius=0.45)


def test_small_sigma_composite_is_the_binary_composite():
    sc = _scene(3)
    hard = R.render_image(sc)
    soft = R.render_image(sc, soft=1e-3)
    d = np.abs(soft["rgb"] - hard["rgb"]).max(-1)
    # only pixels with a sample within ~0.02 px of an edge (or of the 1/256
    # snapping) may differ
    assert (d > 1e-6).mean() < 0.03
    assert np.median(d) < 1e-12


def test_soft_composite_differs_from_binary_at_edges_only():
    sc = _scene(3)
    hard = R.render_image(sc)
    soft = R.render_image(sc, soft=0.5)
    d = np.abs(soft["rgb"] - hard["rgb"]).max(-1)
    assert d.max() > 1e-2           # silhouettes are blurred
    assert (d < 1e-6).mean() > 0.3  # interiors and mesh-free pixels are not


def _to64(sc):
    sc = copy.deepcopy(sc)
    g = sc.gaussians
    for k in ("means", "quats", "scales", "opacities", "sh"):
        setattr(g, k, np.asarray(getattr(g, k), np.float64))
    for m in sc.meshes:
        m.verts = np.asarray(m.verts, np.float64)
        m.vcolor = np.asarray(m.vcolor, np.float64)
        if m.valpha is not None:
            m.valpha = np.asarray(m.valpha, np.float64)
    return sc


@pytest.mark.parametrize("sigma", [0.4])
def test_torch_forward_equals_numpy_forward(sigma):
    sc = _scene(3, valpha=True)
    ref = R.render_image(sc, soft=sigma)
    fr, pix, table = G.decision_table(sc, soft=sigma)
    p = G.leaf_params(sc)
    C, T = G.composite_torch(sc, p, fr, pix, table)
    assert np.abs(C.detach().numpy().reshape(ref["rgb"].shape) - ref["rgb"]).max() < 1e-12
    assert np.abs(T.detach().numpy().reshape(ref["T"].shape) - ref["T"]).max() < 1e-12


def test_fd_vertex_positions_through_coverage():
    sigma = 0.4
    sc = _scene(5, valpha=True, W=18, H=14, n=20)
    rng = np.random.default_rng(7)
    H, W = sc.cameras[0].height, sc.cameras[0].width
    gC = rng.normal(size=(H, W, 3))
    gT = rng.normal(size=(H, W))
    grads, _, _ = G.image_grad(sc, gC, gT, soft=sigma)
    hard, _, _ = G.image_grad(sc, gC, gT)
    ga = grads["verts0"]
    # coverage adds gradient that the binary form does not have
    assert np.abs(ga - hard["verts0"]).max() > 0.1 * np.abs(ga).max()
    h = 1e-6
    L0, sig0 = G.loss_numpy(_to64(sc), gC, gT, soft=sigma)
    scale = np.abs(ga).max()
    checked = 0
    for fi in np.argsort(-np.abs(ga).ravel())[:10]:
        idx = np.unravel_index(fi, ga.shape)
        vals, ok = [], True
        for sgn in (1, -1):
            s2 = _to64(sc)
            s2.meshes[0].verts[idx] += sgn * h
            L, sig = G.loss_numpy(s2, gC, gT, soft=sigma)
            ok = ok and sig == sig0
            vals.append(L)
        if not ok:
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - ga[idx]) <= 1e-5 * scale + 1e-6 * abs(fd), (idx, fd, ga[idx], scale)
        checked += 1
    assert checked >= 7


def test_coverage_is_invariant_to_vertex_order():
    rng = np.random.default_rng(11)
    tu = rng.uniform(0, 20, (50, 3))
    tv = rng.uniform(0, 20, (50, 3))
    for px, py in [(5, 5), (10, 12), (17, 3)]:
        c = R.soft_coverage(tu, tv, px, py, 0.7)
        for perm in ([1, 2, 0], [2, 0, 1], [0, 2, 1], [2, 1, 0]):
            c2 = R.soft_coverage(tu[:, perm], tv[:, perm], px, py, 0.7)
            assert np.abs(c - c2).max() < 1e-12


def test_widened_rects_are_the_binary_rects_plus_the_dilation():
    sc = _scene(3)
    cam = sc.cameras[0]
    for sigma in (0.3, 0.5, 1.0):
        R_ = R.soft_dilation(sigma)
        m = sc.meshes[0]
        hard = cn.setup_triangles(m.verts, m.faces, cam)
        soft = cn.setup_triangles(m.verts, m.faces, cam, R_)
        both = hard["valid"] & soft["valid"]
        h, s = hard["rect"][both], soft["rect"][both]
        assert np.array_equal(s[:, 0], np.maximum(h[:, 0] - R_, 0))
        assert np.array_equal(s[:, 1], np.minimum(h[:, 1] + R_, cam.width - 1))
        assert np.array_equal(s[:, 2], np.maximum(h[:, 2] - R_, 0))
        assert np.array_equal(s[:, 3], np.minimum(h[:, 3] + R_, cam.height - 1))
        # widening only adds triangles (those whose sample rect was empty)
        assert np.all(soft["valid"][hard["valid"]])


# a sliver whose snapped integer area (the setup's orientation) has the
# opposite sign of its unsnapped area
SLIVER = [(5.027790005723492, 10.736210131921993), (14.411724373399148, 12.507311622341327),
          (41.61529358247677, 17.643240721287356)]


def _sliver_scene(pts=SLIVER):
    c = H.cam(48, 32)
    return H.scene(H.no_gaussians(), [H.single_triangle(c, pts, 0.2, 0.7)], c, tile=8)


def test_soft_orientation_is_the_setup_orientation():
    """The orientation sg of the soft coverage is the sign of the snapped
    integer area (the one the setup orders the edges by and the kernels store
    in the triangle record), not the sign of the unsnapped area: exact on both
    sides.  On this sliver (its middle vertex almost on the segment between
    the other two) the two signs disagree, and the coverage along it differs
    with the choice."""
    sc = _sliver_scene()
    P = cn.Primitives(sc, 0, dilate=R.soft_dilation(0.5))
    t = P.tris[0]
    sx, sy = t["sx"][0], t["sy"][0]
    snapped = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sx[2] - sx[0]) * (sy[1] - sy[0])
    fr = R.Frame(sc, 0, soft=0.5)
    vu, vv, _ = fr.V[0]
    f = np.asarray(sc.meshes[0].faces[0], np.int64)
    tu, tv = vu[f][None], vv[f][None]
    unsnapped = (tu[0, 1] - tu[0, 0]) * (tv[0, 2] - tv[0, 0]) - (tu[0, 2] - tu[0, 0]) * (tv[0, 1] - tv[0, 0])
    assert P.tri_sign[0] == np.sign(snapped) and np.sign(snapped) != np.sign(unsnapped)
    px, py = 4, 10  # a pixel on the sliver
    c_setup = R.soft_coverage(tu, tv, px, py, 0.5, P.tri_sign[:1])[0]
    c_fp = R.soft_coverage(tu, tv, px, py, 0.5, np.sign([unsnapped]))[0]
    assert np.abs(c_setup - c_fp).max() > 0.02
    # the fragments the oracle composites take the setup's sign
    frag = [g for g in fr.fragments_at(px, py) if g["kind"] == "t"][0]
    assert np.allclose(frag["cov"], c_setup, rtol=0, atol=1e-15)
