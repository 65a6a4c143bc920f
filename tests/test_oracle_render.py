"""Pins of the oracle composite against what the paper and the mathematics fix."""
import math

import numpy as np
import pytest

from oracle import canonical as cn
from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H


def _img(sc, **kw):
    return R.render_image(sc, **kw)


# -- energy: sum of weights + T_final = 1 (Eq. 7-9 with the entity T update) --

@pytest.mark.parametrize("t_eps", [None, 1e-4])
def test_energy_config0(t_eps):
    sc = S.config0()
    r = _img(sc, t_eps=t_eps)
    assert np.abs(r["wsum"] + r["T"] - 1.0).max() < 1e-12
    assert r["nfrag"].max() > 5


def test_energy_small_scene_valpha():
    sc = S.small_scene(7, 40, 28, 300, mesh_subdiv=2, with_valpha=True)
    r = _img(sc, t_eps=None)
    assert np.abs(r["wsum"] + r["T"] - 1.0).max() < 1e-12
    # every weight non-negative => colour bounded by the max fragment colour
    assert r["rgb"].min() >= 0.0


def _stack_scene(alpha=0.5):
    """Triangle - Gaussian - triangle along the view ray (Fig. 3c)."""
    c = H.cam(16, 16)
    q1 = H.screen_quad(c, -1.0, alpha, (1.0, 0.0, 0.0))
    q2 = H.screen_quad(c, 1.0, alpha, (0.0, 0.0, 1.0))
    m = S.Mesh(np.concatenate([q1.verts, q2.verts]), np.concatenate([q1.faces, q2.faces + 4]),
               np.concatenate([q1.vcolor, q2.vcolor]), None, np.concatenate([q1.falpha, q2.falpha]))
    g = H.gaussians([[0, 0, 0]], scales=[[5, 5, 0.01]], opac=[0.9], colors=[[0, 1, 0]])
    return H.scene(g, [m], c)


def test_entity_all_overflows_full_does_not():
    sc = _stack_scene()
    full = _img(sc, t_eps=None)
    bad = _img(sc, t_eps=None, mode=R.ENTITY_ALL)
    assert np.abs(full["wsum"] + full["T"] - 1).max() < 1e-12
    # ENTITY_ALL gives the rear triangle a transmittance that ignores the Gaussian
    assert (bad["wsum"] + bad["T"] - 1).max() > 0.05


def test_t_product_reading_breaks_energy_in_multi_triangle_entity():
    # the literal product T <- T (1 - O_i alpha_i) of Eq. 6 with O_i from Eq. 8
    # agrees with the entity update for a single triangle, but over-counts the
    # transmittance decay for longer entities (O_i already carries t^j)
    c = H.cam(16, 16)
    qs = [H.screen_quad(c, z, 0.5, (1, 1, 1)) for z in (-1.0, -0.5, 0.0)]
    m3 = S.Mesh(np.concatenate([q.verts for q in qs]), np.concatenate([q.faces + 4 * i for i, q in enumerate(qs)]),
                np.concatenate([q.vcolor for q in qs]), None, np.concatenate([q.falpha for q in qs]))
    big = H.single_triangle(c, [(-500.0, -500.0), (900.0, -500.0), (-500.0, 900.0)], -1.0, 0.5)
    one = H.scene(H.no_gaussians(), [big], c)
    assert np.abs(_img(one, t_eps=None, t_product=True)["T"] - _img(one, t_eps=None)["T"]).max() == 0
    sc = H.scene(H.no_gaussians(), [m3], c)
    full = _img(sc, t_eps=None)
    lit = _img(sc, t_eps=None, t_product=True)
    assert np.abs(full["wsum"] + full["T"] - 1).max() < 1e-12
    assert np.allclose(full["T"], 0.125)
    assert (lit["wsum"] + lit["T"] - 1).min() > 0.1


# -- special cases with closed forms --

def test_single_opaque_full_cover_triangle_exact_colour():
    c = H.cam(24, 20)
    m = H.single_triangle(c, [(-500.0, -500.0), (900.0, -500.0), (-500.0, 900.0)], 0.0, 1.0,
                          colors=[[0.25, 0.5, 0.75]] * 3)
    sc = H.scene(H.no_gaussians(), [m], c)
    r = _img(sc, t_eps=None)
    # exact up to the rounding of the (normalised) barycentric weights
    assert np.abs(r["rgb"] - np.array([0.25, 0.5, 0.75])).max() < 1e-15
    assert np.all(r["T"] == 0.0)
    # two opaque triangles sharing an edge (a quad) still give exactly T = 0
    q = H.screen_quad(c, 0.0, 1.0, (0.25, 0.5, 0.75))
    rq = _img(H.scene(H.no_gaussians(), [q], c), t_eps=None)
    assert np.all(rq["T"] == 0.0)
    assert np.abs(rq["rgb"] - np.array([0.25, 0.5, 0.75])).max() < 1e-15


def test_watertight_quad_counts_each_sample_once():
    # two triangles sharing the diagonal; alpha 0.5: each sample covered by
    # exactly one of them -> every t^j = 0.5 -> T = 0.5 everywhere, C = 0.5 c
    c = H.cam(32, 32)
    m = H.screen_quad(c, 0.0, 0.5, (1.0, 1.0, 1.0), extent=0.0)  # quad = exactly the image
    # shift the quad by a non-grid amount so that the diagonal crosses samples
    m.verts[:, 0] += np.float32(0.0137)
    sc = H.scene(H.no_gaussians(), [m], c)
    r = _img(sc, t_eps=None)
    inner = r["T"][2:-2, 2:-2]
    assert np.all(inner == 0.5)
    assert np.abs(r["rgb"][2:-2, 2:-2] - 0.5).max() < 1e-15


def test_half_coverage_opaque_gives_half_colour():
    # a vertical edge through the pixel centres: samples with x offset > 0 are
    # inside (2 of 4), so O = 1/2 and T = 1/2 (Eq. 7-9, M = 4)
    c = H.cam(16, 16)
    x_edge = 8.5  # pixel 8's centre
    m = H.single_triangle(c, [(x_edge, -100.0), (x_edge + 400.0, 8.0), (x_edge, 200.0)], 0.0, 1.0,
                          colors=[[0.8, 0.6, 0.4]] * 3)
    sc = H.scene(H.no_gaussians(), [m], c)
    r = _img(sc, t_eps=None)
    assert r["T"][8, 8] == 0.5
    assert np.allclose(r["rgb"][8, 8], [0.4, 0.3, 0.2], atol=1e-12)
    assert r["T"][8, 9] == 0.0 and r["T"][8, 7] == 1.0


def test_full_coverage_reduces_to_pixel_alpha_blending():
    # all samples covered -> the entity blend is Eq. 1-2 applied to triangles
    c = H.cam(16, 16)
    qs = [H.screen_quad(c, z, a, col) for z, a, col in
          [(-1.0, 0.3, (1, 0, 0)), (-0.5, 0.6, (0, 1, 0)), (0.5, 0.45, (0, 0, 1))]]
    m = S.Mesh(np.concatenate([q.verts for q in qs]), np.concatenate([q.faces + 4 * i for i, q in enumerate(qs)]),
               np.concatenate([q.vcolor for q in qs]), None, np.concatenate([q.falpha for q in qs]))
    sc = H.scene(H.no_gaussians(), [m], c)
    r = _img(sc, t_eps=None)
    T = 1.0
    C = np.zeros(3)
    for a, col in [(0.3, (1, 0, 0)), (0.6, (0, 1, 0)), (0.45, (0, 0, 1))]:
        C += T * a * np.array(col, float)
        T *= (1 - a)
    a32 = [float(np.float32(x)) for x in (0.3, 0.6, 0.45)]
    T2 = 1.0
    C2 = np.zeros(3)
    for a, col in zip(a32, [(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        C2 += T2 * a * np.array(col, float)
        T2 *= (1 - a)
    assert np.allclose(r["rgb"], C2, atol=1e-12)
    assert np.allclose(r["T"], T2, atol=1e-12)
    d = _img(sc, t_eps=None, mode=R.DIRECT)
    assert np.allclose(d["rgb"], r["rgb"], atol=1e-12)


def test_isotropic_gaussian_closed_form():
    c = H.cam(33, 33)
    sigma, op = 0.03, 0.7
    g = H.gaussians([[0, 0, 0]], scales=[[sigma] * 3], opac=[op], colors=[[0.3, 0.6, 0.9]])
    sc = H.scene(g, [], c)
    G = R.gaussians_fp64(sc.gaussians, c)
    Z = 3.0
    s32 = float(np.float32(sigma))
    var = (c.fx * s32 / Z) ** 2 + 0.3
    assert np.allclose(G["conic"][0], [1 / var, 0, 1 / var], rtol=1e-12)
    assert np.allclose([G["u"][0], G["v"][0]], [16.5, 16.5])
    r = _img(sc, t_eps=None)
    for (x, y) in [(16, 16), (18, 16), (16, 13), (19, 20)]:
        d2 = (x + 0.5 - 16.5) ** 2 + (y + 0.5 - 16.5) ** 2
        a = min(0.99, float(np.float32(op)) * math.exp(-0.5 * d2 / var))
        expect = a * np.array([0.3, 0.6, 0.9]) if a >= 1 / 255 else np.zeros(3)
        assert np.allclose(r["rgb"][y, x], expect, atol=1e-7), (x, y)
    # footprint: 3 sigma of the dilated variance around the centre pixel
    P = cn.Primitives(sc)
    rx = float(np.float32(3) * np.sqrt(np.float32(P.g["a"][0])))
    assert P.rect[0, 0] == math.ceil(16.5 - rx - 0.5)


def test_depth_separated_scene_factorises():
    sc = S.small_scene(11, 37, 29, 200, mesh_subdiv=2, mesh_radius=0.3, mesh_offset=(0.0, 0.0, -2.0))
    both = _img(sc, t_eps=None)
    mesh_only = _img(S.Scene(H.no_gaussians(), sc.meshes, sc.cameras), t_eps=None)
    g_only = _img(S.Scene(sc.gaussians, [], sc.cameras), t_eps=None)
    # mesh entirely in front of every Gaussian (camera at z=-3, mesh around z=-2)
    expect = mesh_only["rgb"] + mesh_only["T"][..., None] * g_only["rgb"]
    assert np.abs(both["rgb"] - expect).max() < 1e-12
    assert np.abs(both["T"] - mesh_only["T"] * g_only["T"]).max() < 1e-12
    assert (mesh_only["T"] < 1).sum() > 20


def test_brute_force_gather_matches_image_gather():
    sc = S.small_scene(3, 32, 32, 40, mesh_subdiv=0, mesh_radius=0.6)
    img = _img(sc)
    pix = [(x, y) for y in range(32) for x in range(32)]
    rgb, T, tie, ws = R.render_pixels(sc, pix)
    assert np.abs(rgb - img["rgb"].reshape(-1, 3)).max() < 1e-15
    assert np.abs(T - img["T"].reshape(-1)).max() < 1e-15


def test_background_uses_final_transmittance():
    sc = S.small_scene(5, 24, 24, 60, mesh_subdiv=1)
    bg = (0.1, 0.7, 0.3)
    a = _img(sc, t_eps=None)
    b = _img(sc, t_eps=None, bg=bg)
    assert np.abs(b["rgb"] - (a["rgb"] + a["T"][..., None] * np.array(bg))).max() < 1e-12


def test_early_termination_bounded():
    sc = S.config0()
    a = _img(sc, t_eps=None)
    b = _img(sc, t_eps=1e-4)
    # blend-then-stop: the dropped remainder is at most T_stop * max colour
    maxc = 1.0 + 2.0  # SH0 colours are U[0,1]; triangle colours U[0,1]
    assert np.abs(a["rgb"] - b["rgb"]).max() <= 1e-4 * maxc
