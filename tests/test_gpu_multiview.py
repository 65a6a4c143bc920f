"""Multi-view form: persistent compositor, CUDA-graph capture and autotuning.

The schedule and the graph change how the work is launched, not what is
computed: their outputs must equal the one-CTA-per-tile render bit for bit,
and that render matches the oracle (keys exact, images within 2e-4)."""
import math

import numpy as np
import pytest
import torch

from paper_2601_19233_gb300 import scenes as S
from tests.test_gpu_render import check_image, check_lists, ctx  # noqa: F401

pytestmark = pytest.mark.gpu
# a split render against the whole-tile one: a segment may blend fragments
# after the whole tile fell below t_eps = 1e-4 (colours <= 1), plus rounding
SPLIT_TOL = 1e-4 + 1e-5


def _clustered(seed=2024, n=3000, cams=6, size=96):
    """A small stand-in for the 64-view orbit workload: 70% of the Gaussians
    in 3 blobs (uneven tile load), a torus, cameras on an orbit."""
    rng = np.random.default_rng(seed)
    nb = int(0.7 * n)
    c = rng.uniform(-0.5, 0.5, size=(3, 3))
    blob = c[rng.integers(0, 3, size=nb)] + rng.normal(0, 0.15, size=(nb, 3))
    means = np.concatenate([blob, rng.uniform(-1, 1, size=(n - nb, 3))]).astype(np.float32)
    g = S.make_gaussians(rng, means, -3.5, 3)
    V, F = S.torus(40, 20)
    vcol = rng.uniform(0, 1, size=(len(V), 3)).astype(np.float32)
    fa = np.ones(len(F), np.float32)
    m = rng.uniform(size=len(F)) < 0.3
    fa[m] = rng.uniform(0.2, 0.8, size=int(m.sum())).astype(np.float32)
    fx = S.focal_from_fov(size, 60.0)
    camsl = S.orbit_cameras(cams, 3.0, size, size, fx, lambda k: 20.0 * math.sin(2 * math.pi * k / 16))
    return S.Scene(g, [S.Mesh(V, F, vcol, None, fa)], camsl, tile=16)


def _dev(sc):
    from paper_2601_19233_gb300 import umgs
    return umgs.gaussians_to_device(sc.gaussians), [umgs.mesh_to_device(m) for m in sc.meshes]


def test_persistent_schedules_bit_identical(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = _clustered()
    g, ms = _dev(sc)
    fr = umgs.Frame(ctx)
    base = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16), frame=fr).cpu().numpy()
    check_lists(sc, fr, 16)
    check_image(sc, base)
    for ts in (8, 16, 32):
        ref = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(ts)).cpu().numpy()
        for sched in (1, 2, 4):
            out = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(ts, sched=sched)).cpu().numpy()
            assert np.array_equal(out, ref), (ts, sched)
        assert np.array_equal(ref, base)


def test_graph_replay_matches_render(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = _clustered(7)
    g, ms = _dev(sc)
    opts = umgs.render_opts(16, sched=2)
    ref = umgs.render(ctx, g, ms, sc.cameras, opts).clone()
    out = torch.zeros_like(ref)
    fr = umgs.Frame(ctx)
    gr = umgs.Graph(ctx, fr, g, ms, sc.cameras, opts, out)
    for _ in range(3):
        out.zero_()
        gr.launch()
        gr.check()
        assert torch.equal(out, ref)
    # new input values, same pointers: the replay follows them
    g.means.add_(0.01)
    ref2 = umgs.render(ctx, g, ms, sc.cameras, opts)
    gr.launch()
    gr.check()
    assert torch.equal(out, ref2)
    assert not torch.equal(ref2, ref)


def test_graph_capacity_overflow_is_reported(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = _clustered(9, n=1500)
    g, ms = _dev(sc)
    opts = umgs.render_opts(16)
    out = torch.zeros((len(sc.cameras), 96, 96, 4), device="cuda")
    fr = umgs.Frame(ctx)
    gr = umgs.Graph(ctx, fr, g, ms, sc.cameras, opts, out, key_headroom=1.0)
    gr.launch()
    gr.check()
    g.scales.mul_(6.0)  # much larger footprints: more pairs than the captured capacity
    out.fill_(-1.0)
    gr.launch()
    with pytest.raises(umgs.UmgsError) as e:
        gr.check()
    assert e.value.status == 3
    # no tile was composited: background (black) with T = 1 everywhere
    assert torch.all(out[..., 3] == 1.0) and torch.all(out[..., :3] == 0.0)


def test_autotune_picks_a_valid_config(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = _clustered(11)
    g, ms = _dev(sc)
    out = torch.zeros((len(sc.cameras), 96, 96, 4), device="cuda")
    best, ms_per = umgs.autotune(ctx, g, ms, sc.cameras, umgs.render_opts(16), out)
    assert best.tile_size in (8, 16, 32) and best.sched in (0, 1, 2, 4) and best.split in (0, 512, 1024, 2048)
    assert ms_per > 0
    ref = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16)).cpu().numpy()
    got = umgs.render(ctx, g, ms, sc.cameras, best).cpu().numpy()
    if best.split == 0:
        assert np.array_equal(got, ref)
    else:  # split segments: within t_eps x the largest colour plus rounding
        assert np.abs(got - ref).max() <= SPLIT_TOL


def test_async_render_matches_sync_and_reports_overflow(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = _clustered(13)
    g, ms = _dev(sc)
    fr = umgs.Frame(ctx)
    ref = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16), frame=fr).clone()
    K = fr.counts()[0]
    fa = umgs.Frame(ctx)
    fa.reserve(K + 16)
    aopts = umgs.render_opts(16, asynchronous=True)
    for _ in range(2):
        out = umgs.render(ctx, g, ms, sc.cameras, aopts, frame=fa)
        fa.check()
        assert torch.equal(out, ref)
    assert fa.counts()[0] == -1
    # too small a capacity: reported, and no tile is composited
    fs = umgs.Frame(ctx)
    fs.reserve(K // 2)
    out = umgs.render(ctx, g, ms, sc.cameras, aopts, frame=fs)
    with pytest.raises(umgs.UmgsError) as e:
        fs.check()
    assert e.value.status == 3
    assert torch.all(out[..., 3] == 1.0)
    # asynchronous without a reserved capacity is refused
    with pytest.raises(umgs.UmgsError) as e:
        umgs.render(ctx, g, ms, sc.cameras, aopts, frame=umgs.Frame(ctx))
    assert e.value.status == 1


def _dense(seed, n=20000, cams=2, size=96, mesh_z=None):
    """Dense blobs (tile lists of several thousand records) and, optionally,
    a screen-filling transparent quad at world depth mesh_z (in front of the
    blobs for z < 0 as seen by the first camera, behind them for z > 0)."""
    from tests import helpers as H
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.4, 0.4, size=(3, 3))
    means = (c[rng.integers(0, 3, size=n)] + rng.normal(0, 0.15, size=(n, 3))).astype(np.float32)
    g = S.make_gaussians(rng, means, -3.5, 1)
    g.opacities = (0.05 + 0.2 * g.opacities).astype(np.float32)  # faint: long lists before termination
    fx = S.focal_from_fov(size, 60.0)
    camsl = S.orbit_cameras(cams, 3.0, size, size, fx)
    meshes = []
    if mesh_z is not None:
        front = S.front_camera(size, size, fx)
        meshes = [H.screen_quad(front, mesh_z, 0.4, (0.9, 0.2, 0.1), extent=3.0)]
    return S.Scene(g, meshes, camsl, tile=16)


def _split_tiles(sc, split):
    """Tiles the split planner cuts (oracle lists): longer than `split`, with
    at least `split` Gaussian records in front of the first triangle."""
    from oracle import canonical as cn
    prims = [cn.Primitives(sc, k) for k in range(len(sc.cameras))]
    ptr, ids, _ = cn.sorted_tile_lists(prims, 16)
    ng = sc.gaussians.n
    n = 0
    for t in range(len(ptr) - 1):
        seg = ids[ptr[t]:ptr[t + 1]]
        if len(seg) <= split:
            continue
        tri = np.nonzero(seg >= ng)[0]
        ftri = int(tri[0]) if len(tri) else len(seg)
        n += ftri >= split
    return n


@pytest.mark.parametrize("sched", [0, 2])
def test_work_split_matches_oracle_and_whole_tiles(ctx, sched):
    from paper_2601_19233_gb300 import umgs
    sc = _dense(31)
    assert _split_tiles(sc, 256) >= 4
    g, ms = _dev(sc)
    whole = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, sched=sched)).cpu().numpy()
    for split in (256, 700):
        out = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, sched=sched, split=split)).cpu().numpy()
        d = np.abs(out - whole).max()
        assert d <= SPLIT_TOL, (split, d)
        assert d > 0.0  # the segments were merged (fp association differs)
    check_image(sc, out)


def test_work_split_never_cuts_behind_a_triangle(ctx):
    from paper_2601_19233_gb300 import umgs
    # a transparent quad in front of every blob: each list starts with it, so no tile is cut
    sc = _dense(32, cams=1, mesh_z=-1.5)
    assert _split_tiles(sc, 256) == 0
    g, ms = _dev(sc)
    whole = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16)).cpu().numpy()
    out = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, split=256)).cpu().numpy()
    assert np.array_equal(out, whole)
    # the same quad behind the blobs: the Gaussian prefix is cut, the quad's entity is whole
    sc = _dense(33, cams=1, mesh_z=1.5)
    assert _split_tiles(sc, 256) >= 4
    g, ms = _dev(sc)
    out = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, split=256, sched=1)).cpu().numpy()
    whole = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16)).cpu().numpy()
    assert np.abs(out - whole).max() <= SPLIT_TOL
    check_image(sc, out)


def test_work_split_graph_replay(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = _dense(34)
    g, ms = _dev(sc)
    opts = umgs.render_opts(16, sched=2, split=512)
    ref = umgs.render(ctx, g, ms, sc.cameras, opts).clone()
    out = torch.zeros_like(ref)
    gr = umgs.Graph(ctx, umgs.Frame(ctx), g, ms, sc.cameras, opts, out)
    for _ in range(2):
        out.zero_()
        gr.launch()
        gr.check()
        assert torch.equal(out, ref)


def test_work_split_rejected_with_saved_state(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = _dense(35, n=500)
    g, ms = _dev(sc)
    for opts in (umgs.render_opts(16, save=True, split=512), umgs.render_opts(16, split=100),
                 umgs.render_opts(16, edge_sigma=0.5, split=512)):
        with pytest.raises(umgs.UmgsError) as e:
            umgs.render(ctx, g, ms, sc.cameras, opts, frame=umgs.Frame(ctx))
        assert e.value.status == 1
