"""GPU binding (Sec. 3.3) against the brute-force oracle: faces, barycentrics,
distances and flags bit-exact."""
import numpy as np
import pytest
import torch

from oracle import bind as B
from paper_2601_19233_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    return umgs.Context(0)


def _gpu_bind(ctx, g, V, F, cams, mode):
    from paper_2601_19233_gb300 import umgs
    dg = umgs.gaussians_to_device(g)
    face, bary, dist, flags, nfb = umgs.bind(ctx, dg, torch.as_tensor(V).cuda(), torch.as_tensor(F).cuda(), cams,
                                             mode=mode)
    return face.cpu().numpy(), bary.cpu().numpy(), dist.cpu().numpy(), flags.cpu().numpy(), nfb


def _scene(seed, n=150, subdiv=2, far=10):
    rng = np.random.default_rng(seed)
    V, F = S.icosphere(subdiv, 1.0)
    V = (V * np.array([1.0, 0.8, 1.2], np.float32)).astype(np.float32)  # not a sphere: uneven cells
    means = S.shell_points(rng, n, 1.0, 0.08)
    means[:far] = rng.uniform(-3, 3, size=(far, 3)).astype(np.float32)  # some far from the surface
    g = S.make_gaussians(rng, means, -3.5, 0)
    cams = S.fibonacci_cameras(9, 3.0)
    return g, V, F, cams


@pytest.mark.parametrize("mode", [B.BBX, B.CENTER, B.NEAREST])
def test_bind_bit_exact(ctx, mode):
    g, V, F, cams = _scene(7 + mode)
    face, bary, dist, flags, nfb = _gpu_bind(ctx, g, V, F, cams, mode)
    ref = B.bind(g.means, g.quats, g.scales, V, F, [c.viewmat for c in cams], mode=mode)
    assert np.array_equal(flags, ref["flags"])
    assert np.array_equal(face, ref["face"])
    assert np.array_equal(bary.view(np.uint32), ref["bary"].view(np.uint32))
    assert np.array_equal(dist.view(np.uint32), ref["dist"].view(np.uint32))
    assert nfb == int((ref["flags"] == B.FLAG_FALLBACK).sum())
    if mode != B.NEAREST:
        assert (flags == B.FLAG_HIT).mean() > 0.5


def test_plane_closed_form(ctx):
    V = np.array([[-5, -5, 0], [5, -5, 0], [5, 5, 0], [-5, 5, 0]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    cam = S.front_camera(64, 64, 50.0, -4.0)  # centre (0,0,4)
    rng = np.random.default_rng(3)
    n = 64
    mu = np.c_[rng.uniform(-1, 1, (n, 2)), rng.uniform(-0.5, 0.5, n)].astype(np.float32)
    g = S.make_gaussians(rng, mu, -4.0, 0)
    face, bary, dist, flags, _ = _gpu_bind(ctx, g, V, F, [cam], B.CENTER)
    h = 4.0
    p = mu.astype(np.float64)
    t = h / (h - p[:, 2])
    want = np.abs(t - 1) * np.linalg.norm(p - np.array([0, 0, h]), axis=1)
    assert np.all(flags == B.FLAG_HIT)
    assert np.allclose(dist[:, 0], want, rtol=2e-5, atol=1e-6)


def _bind_chunk(args):
    means, quats, scales, V, F, vms = args
    return B.bind(means, quats, scales, V, F, vms, mode=B.BBX)


def test_full_size_sampled(ctx):
    """Bench-size binding (1M Gaussians, 100 cameras, 20,480-face proxy),
    checked bit-exact against brute force on 64 Gaussians (512 targets): 32
    drawn at random and the 32 whose bound points lie closest to a face edge
    (smallest barycentric weight), where a wrong face is likeliest.  The brute
    force runs in a spawned process pool."""
    import multiprocessing as mp
    import os
    sc = S.config1()
    g = sc.gaussians
    face, bary, dist, flags, nfb = _gpu_bind(ctx, g, sc.proxy_verts, sc.proxy_faces, sc.bind_cameras, B.BBX)
    assert face.shape == (g.n, 8) and (face >= 0).all()
    rand = np.random.default_rng(0).choice(g.n, size=32, replace=False)
    w = np.concatenate([bary, 1.0 - bary.sum(-1, keepdims=True)], -1).min(-1).min(-1)
    w[rand] = np.inf
    idx = np.sort(np.concatenate([rand, np.argsort(w)[:32]]))
    vms = [c.viewmat for c in sc.bind_cameras]
    chunks = [c for c in np.array_split(idx, 16) if len(c)]
    with mp.get_context("spawn").Pool(min(len(chunks), os.cpu_count() or 1)) as pool:
        parts = pool.map(_bind_chunk, [(g.means[c], g.quats[c], g.scales[c], sc.proxy_verts, sc.proxy_faces, vms)
                                       for c in chunks])
    ref = {k: np.concatenate([p_[k] for p_ in parts]) for k in ("face", "bary", "dist", "flags")}
    assert np.array_equal(face[idx], ref["face"])
    assert np.array_equal(bary[idx].view(np.uint32), ref["bary"].view(np.uint32))
    assert np.array_equal(dist[idx].view(np.uint32), ref["dist"].view(np.uint32))
    assert np.array_equal(flags[idx], ref["flags"])


def test_bad_face_index_rejected(ctx):
    from paper_2601_19233_gb300 import umgs
    g, V, F, cams = _scene(1, n=10)
    F = F.copy()
    F[5, 2] = len(V) + 1
    with pytest.raises(umgs.UmgsError) as e:
        _gpu_bind(ctx, g, V, F, cams, B.BBX)
    assert e.value.status == 1
