"""Pins of the canonical float32 decisions (coverage, footprints, keys, order)."""
import math
from fractions import Fraction

import numpy as np

from oracle import canonical as cn
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H


def _exact_inside(tri, p):
    """Exact (rational) strict inside / on-edge test of point p in triangle tri."""
    (x0, y0), (x1, y1), (x2, y2) = tri
    def cr(ax, ay, bx, by, px, py):
        return (bx - ax) * (py - ay) - (by - ay) * (px - ax)
    d = [cr(x0, y0, x1, y1, *p), cr(x1, y1, x2, y2, *p), cr(x2, y2, x0, y0, *p)]
    pos = all(v > 0 for v in d) or all(v < 0 for v in d)
    on = any(v == 0 for v in d) and (all(v >= 0 for v in d) or all(v <= 0 for v in d))
    return pos, on


def test_sample_coverage_matches_exact_point_in_triangle():
    rng = np.random.default_rng(0)
    c = H.cam(64, 48)
    checked = 0
    for _ in range(40):
        pts = rng.uniform(-8, 72, size=(3, 2))
        m = H.single_triangle(c, pts, float(rng.uniform(-0.5, 0.5)))
        t = cn.setup_triangles(m.verts, m.faces, c)
        if not t["valid"][0]:
            continue
        tri = [(int(t["sx"][0, k]), int(t["sy"][0, k])) for k in range(3)]
        for _ in range(200):
            px, py = int(rng.integers(0, 64)), int(rng.integers(0, 48))
            mask = int(cn.sample_coverage(t["A"], t["B"], t["Cb"], px, py)[0])
            for j in range(4):
                s = (px * 256 + 128 + int(cn.SAMPLE_OFFSETS[j, 0]), py * 256 + 128 + int(cn.SAMPLE_OFFSETS[j, 1]))
                inside, on = _exact_inside(tri, s)
                if on:
                    continue
                assert ((mask >> j) & 1) == int(inside)
                checked += 1
    assert checked > 10000


def test_top_left_rule_shared_edges_counted_once():
    # a fan of triangles around a vertex placed exactly on a sample: every
    # sample of the covered region belongs to exactly one triangle
    c = H.cam(32, 32)
    centre = (16 + 0.5 + 32 / 256, 16 + 0.5 - 96 / 256)  # exactly sample 0 of pixel (16,16)... shifted
    ang = np.linspace(0, 2 * np.pi, 7)[:-1] + 0.3
    ring = [(centre[0] + 12 * math.cos(a), centre[1] + 12 * math.sin(a)) for a in ang]
    tris = []
    for i in range(6):
        tris.append(H.single_triangle(c, [centre, ring[i], ring[(i + 1) % 6]], 0.0))
    counts = np.zeros((32, 32, 4), np.int64)
    for m in tris:
        t = cn.setup_triangles(m.verts, m.faces, c)
        assert t["valid"][0]
        for py in range(32):
            for px in range(32):
                mask = int(cn.sample_coverage(t["A"], t["B"], t["Cb"], px, py)[0])
                for j in range(4):
                    counts[py, px, j] += (mask >> j) & 1
    assert counts.max() == 1
    assert counts[14:19, 14:19].min() == 1  # interior fully covered, no cracks


def test_snap_is_round_half_even_of_exact_product():
    c = H.cam(40, 40)
    rng = np.random.default_rng(1)
    m = H.single_triangle(c, rng.uniform(0, 40, size=(3, 2)), 0.2)
    t = cn.setup_triangles(m.verts, m.faces, c)
    X, Y, Z = cn.view_transform(c.viewmat, m.verts)
    u = (np.float32(c.fx) * X) / Z + np.float32(c.cx)
    for k in range(3):
        exact = Fraction(float(u[k])) * 256
        assert t["sx"][0, k] == round(exact)  # Python round() is half-even on exact rationals


def test_view_transform_close_to_fp64():
    rng = np.random.default_rng(2)
    p = rng.uniform(-2, 2, size=(1000, 3)).astype(np.float32)
    cams = S.orbit_cameras(4, 3.0, 64, 64, 50.0)
    for cm in cams:
        X, Y, Z = cn.view_transform(cm.viewmat, p)
        ref = p.astype(np.float64) @ cm.viewmat[:, :3].astype(np.float64).T + cm.viewmat[:, 3]
        assert np.abs(Z - ref[:, 2]).max() < 4e-7 * 5
        assert np.abs(X - ref[:, 0]).max() < 4e-7 * 5


def test_axis_aligned_gaussian_footprint_closed_form():
    c = H.cam(64, 64)
    rng = np.random.default_rng(3)
    n = 200
    mu = np.c_[rng.uniform(-0.8, 0.8, (n, 2)), rng.uniform(-0.5, 0.5, n)].astype(np.float32)
    sc = rng.uniform(0.005, 0.08, (n, 3)).astype(np.float32)
    g = H.gaussians(mu, scales=sc)
    pg = cn.project_gaussians(g.means, g.quats, g.scales, None, c)
    m64 = mu.astype(np.float64)
    Z = m64[:, 2] + 3.0
    X, Y = m64[:, 0], m64[:, 1]
    fx = c.fx
    u = fx * X / Z + 32
    v = fx * Y / Z + 32
    s64 = sc.astype(np.float64)
    # J (with no clamp active) applied to an axis-aligned Sigma
    a = (fx / Z) ** 2 * s64[:, 0] ** 2 + (fx * X / Z ** 2) ** 2 * s64[:, 2] ** 2 + 0.3
    cc = (fx / Z) ** 2 * s64[:, 1] ** 2 + (fx * Y / Z ** 2) ** 2 * s64[:, 2] ** 2 + 0.3
    rx, ry = 3 * np.sqrt(a), 3 * np.sqrt(cc)
    xlo = np.ceil(u - rx - 0.5)
    yhi = np.floor(v + ry - 0.5)
    ok = 0
    for i in range(n):
        if not pg["valid"][i]:
            continue
        if abs((u[i] - rx[i] - 0.5) - round(u[i] - rx[i] - 0.5)) < 1e-4:
            continue
        if abs((v[i] + ry[i] - 0.5) - round(v[i] + ry[i] - 0.5)) < 1e-4:
            continue
        assert pg["rect"][i, 0] == max(0, xlo[i])
        assert pg["rect"][i, 3] == min(63, yhi[i])
        ok += 1
    assert ok > 150
    assert np.allclose(pg["a"], a, rtol=1e-5)


def test_tile_lists_cover_fragments_and_are_sorted():
    sc = S.small_scene(21, 45, 37, 400, mesh_subdiv=2)
    ts = 8
    P = cn.Primitives(sc)
    ptr, ids, db = cn.sorted_tile_lists([P], ts)
    tx_n = (45 + ts - 1) // ts
    assert ptr[-1] == P.tiles_touched(ts).sum()
    for t in range(len(ptr) - 1):
        seg_ids = ids[ptr[t]:ptr[t + 1]]
        seg_db = db[ptr[t]:ptr[t + 1]].astype(np.int64)
        key = seg_db * (1 << 32) + seg_ids
        assert np.all(np.diff(key) > 0)
        assert np.all(P.dbits[seg_ids] == seg_db.astype(np.uint64))
    # every primitive appears in exactly the tiles of its pixel rect
    for i in np.nonzero(P.valid)[0][:200]:
        x0, x1, y0, y1 = P.rect[i]
        want = {(y // ts) * tx_n + (x // ts) for x in (x0, x1) for y in (y0, y1)}
        got = {t for t in range(len(ptr) - 1) if i in set(ids[ptr[t]:ptr[t + 1]].tolist())}
        assert want <= got
        assert len(got) == P.tiles_touched(ts)[i]


def test_depth_keys_are_float_bits_and_triangle_centroid():
    sc = S.config0()
    P = cn.Primitives(sc)
    ng = sc.gaussians.n
    Z = cn.view_transform(sc.cameras[0].viewmat, sc.gaussians.means)[2]
    assert np.all(P.dbits[:ng] == Z.view(np.uint32))
    m = sc.meshes[0]
    Zv = (m.verts.astype(np.float64) @ sc.cameras[0].viewmat[:, :3].astype(np.float64).T)[:, 2] + 3.0
    cen = Zv[m.faces].mean(1)
    assert np.abs(P.depth[ng:] - cen).max() < 1e-6
    # ascending float bits order == ascending depth for positive depths
    o1 = np.argsort(P.dbits, kind="stable")
    o2 = np.argsort(P.depth, kind="stable")
    assert np.all(P.depth[o1] == P.depth[o2])
