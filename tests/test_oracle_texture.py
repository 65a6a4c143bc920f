"""Pins of the oracle's texture sampling for textured meshes (c_i from a
texture, the NEXT extension of Sec. 3.2's per-vertex colour)."""
import numpy as np

from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H


def _ramp(tw, th, a, b, c):
    """T[j, i] = a + b u_i + c v_j at the texel centres (u_i = (i+0.5)/tw)."""
    u = (np.arange(tw) + 0.5) / tw
    v = (np.arange(th) + 0.5) / th
    return a[None, None, :] + b[None, None, :] * u[None, :, None] + c[None, None, :] * v[:, None, None]


def test_bilinear_reproduces_affine_textures():
    a, b, c = np.array([0.1, 0.2, 0.3]), np.array([0.5, -0.2, 0.1]), np.array([-0.3, 0.4, 0.2])
    tex = _ramp(17, 11, a, b, c)
    rng = np.random.default_rng(0)
    uv = np.stack([rng.uniform(0.5 / 17, 1 - 0.5 / 17, 200), rng.uniform(0.5 / 11, 1 - 0.5 / 11, 200)], 1)
    got = R.sample_texture(tex, uv)
    assert np.abs(got - (a + uv[:, :1] * b + uv[:, 1:] * c)).max() < 1e-12
    # at texel centres the lookup returns the texel itself; outside, the edge
    assert np.abs(R.sample_texture(tex, np.array([[4.5 / 17, 7.5 / 11]])) - tex[7, 4]).max() < 1e-12
    assert np.abs(R.sample_texture(tex, np.array([[-0.3, 1.7]])) - tex[10, 0]).max() < 1e-12


def test_textured_triangle_colour_is_the_ray_hit_texture_value():
    # a tilted triangle whose uv is an affine function of the world position:
    # with an affine texture, the colour at a pixel centre inside the triangle
    # is that function at the point where the pixel's ray meets the triangle
    c = H.cam(40, 40)
    V = np.array([[-0.9, -0.8, -0.4], [0.9, -0.7, 0.5], [0.1, 0.9, 0.1]], np.float32)
    M = np.array([[0.4, 0.1], [-0.05, 0.35]])
    uv = (V[:, :2].astype(np.float64) @ M.T + 0.5).astype(np.float32)
    a, b, cc = np.array([0.2, 0.3, 0.1]), np.array([0.4, 0.1, -0.2]), np.array([0.1, -0.3, 0.5])
    tex = _ramp(64, 64, a, b, cc).astype(np.float32)
    m = S.Mesh(V, np.array([[0, 1, 2]], np.int32), np.zeros((3, 3), np.float32), None, np.ones(1, np.float32),
               uv=uv, texture=tex)
    sc = H.scene(H.no_gaussians(), [m], c)
    fr = R.Frame(sc)
    Rm, t = c.viewmat[:, :3].astype(np.float64), c.viewmat[:, 3].astype(np.float64)
    P = V.astype(np.float64) @ Rm.T + t
    n = np.cross(P[1] - P[0], P[2] - P[0])
    checked = 0
    for py in range(40):
        for px in range(40):
            frags = fr.fragments_at(px, py)
            if not frags or not frags[0]["centre"]:
                continue
            d = np.array([(px + 0.5 - c.cx) / c.fx, (py + 0.5 - c.cy) / c.fy, 1.0])
            hit_cam = d * (np.dot(n, P[0]) / np.dot(n, d))
            hit = Rm.T @ (hit_cam - t)  # world point
            uvp = M @ hit[:2] + 0.5
            ref = a + uvp[0] * b + uvp[1] * cc
            # uv inside the interior of the texel-centre lattice: no clamping
            assert np.all((uvp > 0.5 / 64) & (uvp < 1 - 0.5 / 64))
            assert np.abs(frags[0]["color"] - ref).max() < 1e-6
            checked += 1
    assert checked > 150
