"""Pins of the oracle binding (Sec. 3.3) against closed forms."""
import numpy as np

from oracle import bind as B
from paper_2601_19233_gb300 import scenes as S


def _plane(half=5.0):
    V = np.array([[-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return V, F


def _cam_at(z):
    c = S.front_camera(64, 64, 50.0, -z)   # front_camera(dist) sits at (0,0,-dist)
    return c


def test_plane_central_projection_closed_form():
    V, F = _plane()
    h = 4.0
    cam = _cam_at(h)  # camera centre (0,0,4)
    rng = np.random.default_rng(0)
    n = 60
    mu = np.c_[rng.uniform(-1, 1, (n, 2)), rng.uniform(-0.5, 0.5, n)].astype(np.float32)
    q = np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32)
    s = np.full((n, 3), 0.01, np.float32)
    out = B.bind(mu, q, s, V, F, [cam.viewmat], mode=B.CENTER)
    o = np.array([0, 0, h])
    p = mu.astype(np.float64)
    t = h / (h - p[:, 2])
    hit = o + t[:, None] * (p - o)
    dist = np.abs(t - 1) * np.linalg.norm(p - o, axis=1)
    assert np.all(out["flags"] == B.FLAG_HIT)
    assert np.allclose(out["dist"][:, 0], dist, rtol=2e-5, atol=1e-6)
    Vd = V.astype(np.float64)
    for i in range(n):
        f = out["face"][i, 0]
        b1, b2 = out["bary"][i, 0]
        P = (1 - b1 - b2) * Vd[F[f, 0]] + b1 * Vd[F[f, 1]] + b2 * Vd[F[f, 2]]
        assert np.allclose(P, hit[i], atol=1e-5)
        # the face containing the hit point: triangle 0 is below the diagonal y = x
        want = 0 if hit[i, 1] < hit[i, 0] else 1
        if abs(hit[i, 1] - hit[i, 0]) > 1e-5:
            assert f == want


def test_bbx_corners_axis_aligned():
    mu = np.array([[0.1, -0.2, 0.3]], np.float32)
    s = np.array([[0.01, 0.02, 0.03]], np.float32)
    q = np.array([[1, 0, 0, 0]], np.float32)
    tg = B.targets(mu, q, s, B.BBX, 3.0)
    ks = np.float32(3.0) * s[0]
    for i in range(8):
        sign = np.array([1 if (i >> j) & 1 else -1 for j in range(3)], np.float32)
        assert np.all(tg[0, i] == mu[0] + sign * ks)


def test_nearest_face_wins_among_layers():
    # two parallel planes; target between them, closer to the far plane: the
    # ray hits both, and the binding takes the hit nearest to the target
    V1, F1 = _plane()
    V2 = V1.copy()
    V2[:, 2] = -1.0
    V = np.concatenate([V1, V2])
    F = np.concatenate([F1, F1 + 4])
    cam = _cam_at(4.0)
    mu = np.array([[0.2, 0.1, -0.8]], np.float32)
    out = B.bind(mu, np.array([[1, 0, 0, 0]], np.float32), np.full((1, 3), 0.01, np.float32), V, F,
                 [cam.viewmat], mode=B.CENTER)
    assert out["face"][0, 0] in (2, 3)


def test_fallback_and_nearest_closest_point():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    # p above the interior: closest point is the orthogonal projection
    p = np.array([0.2, 0.3, 0.5], np.float32)
    b1, b2, d2 = B.closest_points(p, V, F)
    assert np.allclose([b1[0], b2[0]], [0.2, 0.3], atol=1e-7)
    assert np.isclose(d2[0], 0.25, rtol=1e-6)
    # beyond vertex 1: closest point is the vertex
    b1, b2, d2 = B.closest_points(np.array([2, -1, 0], np.float32), V, F)
    assert (b1[0], b2[0]) == (1.0, 0.0)
    # against dense sampling of a random triangle
    rng = np.random.default_rng(1)
    for _ in range(20):
        V = rng.normal(size=(3, 3)).astype(np.float32)
        p = rng.normal(size=3).astype(np.float32) * 2
        b1, b2, d2 = B.closest_points(p, V, F)
        g = np.linspace(0, 1, 301)
        u, v = np.meshgrid(g, g)
        m = (u + v) <= 1
        pts = (1 - u[m] - v[m])[:, None] * V[0] + u[m][:, None] * V[1] + v[m][:, None] * V[2]
        dmin = np.sqrt(((pts - p) ** 2).sum(1)).min()
        assert np.sqrt(d2[0]) <= dmin + 1e-5
        assert dmin - np.sqrt(d2[0]) < 0.02 * np.abs(V).max()
    # a target with no ray hit falls back and is flagged
    cam = _cam_at(4.0)
    out = B.bind(np.array([[5.0, 5.0, 0.5]], np.float32), np.array([[1, 0, 0, 0]], np.float32),
                 np.full((1, 3), 0.01, np.float32), V, F, [cam.viewmat], mode=B.CENTER)
    assert out["flags"][0, 0] == B.FLAG_FALLBACK
    out2 = B.bind(np.array([[5.0, 5.0, 0.5]], np.float32), None, None, V, F, [cam.viewmat], mode=B.NEAREST)
    assert out2["face"][0, 0] == out["face"][0, 0]
    assert np.all(out2["bary"] == out["bary"])


def test_bbx_binding_on_sphere_hits():
    V, F = S.icosphere(2, 1.0)
    rng = np.random.default_rng(2)
    n = 10
    mu = S.shell_points(rng, n, 1.0, 0.01)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    s = np.full((n, 3), 0.02, np.float32)
    cams = S.fibonacci_cameras(6, 3.0)
    out = B.bind(mu, q, s, V, F, [c.viewmat for c in cams], mode=B.BBX)
    assert np.all(out["flags"] == B.FLAG_HIT)
    # the bound point is within the corner's distance to the sphere + facet sag
    tg = B.targets(mu, q, s, B.BBX)
    r = np.linalg.norm(tg.astype(np.float64), axis=-1)
    assert np.all(out["dist"] <= np.abs(r - 1) * 2.5 + 0.05)
