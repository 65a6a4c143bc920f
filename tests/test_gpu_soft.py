"""GPU parity of the soft-edge coverage path (UMGS_RENDER_SOFT_EDGE, an
extension beyond the paper) against the oracle, through the C ABI.

Bar: tile lists over the widened triangle rects bit-exact; images within
max-abs 2e-4 of the fp64 oracle (tie pixels excluded, as for the binary
path); gradients, vertex positions through coverage included, within
1e-3 max|g_ref| + 1e-6 of the fp64 autograd oracle.
"""
import numpy as np
import pytest
import torch

from oracle import canonical as cn
from oracle import grad as OG
from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H
from tests.test_gpu_render import check_ref

pytestmark = pytest.mark.gpu
TOL = 2e-4


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    return umgs.Context(0)


def _render(ctx, sc, sigma, tile=16, save=False, t_eps=1e-4):
    from paper_2601_19233_gb300 import umgs
    g = umgs.gaussians_to_device(sc.gaussians) if sc.gaussians.n > 0 else None
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    fr = umgs.Frame(ctx)
    opts = umgs.render_opts(tile, t_eps=t_eps, save=save, edge_sigma=sigma)
    out = umgs.render(ctx, g, ms, sc.cameras, opts, frame=fr)
    torch.cuda.synchronize()
    return out, fr, g, ms


def _check_lists(sc, fr, tile, sigma):
    prims = [cn.Primitives(sc, c, dilate=R.soft_dilation(sigma)) for c in range(len(sc.cameras))]
    ptr, ids, db = cn.sorted_tile_lists(prims, tile)
    gptr, gids, gdb = fr.lists()
    assert np.array_equal(gptr.cpu().numpy(), ptr)
    assert np.array_equal(gids.cpu().numpy().astype(np.int64), ids)
    assert np.array_equal(gdb.cpu().numpy().view(np.uint32), db)
    return len(ids)


@pytest.mark.parametrize("seed,W,H,n,sigma,tile", [(91, 45, 37, 400, 0.5, 16), (92, 36, 28, 300, 1.0, 8),
                                                   (93, 70, 41, 600, 0.25, 32)])
def test_soft_lists_and_image(ctx, seed, W, H, n, sigma, tile):
    sc = S.small_scene(seed, W, H, n, mesh_subdiv=2, sh_degree=1, with_valpha=seed % 2 == 0)
    out, fr, _, _ = _render(ctx, sc, sigma, tile)
    nk = _check_lists(sc, fr, tile, sigma)
    hard = [cn.Primitives(sc, 0)]
    assert nk > cn.sorted_tile_lists(hard, tile)[1].size  # the widened rects reach more tiles
    ref = R.render_image(sc, soft=sigma)
    check_ref(out.cpu().numpy()[0], ref)
    # and it is not the binary-coverage image
    assert np.abs(R.render_image(sc)["rgb"] - ref["rgb"]).max() > 1e-2


def test_soft_tile_sizes_agree(ctx):
    sc = S.small_scene(94, 50, 44, 300, mesh_subdiv=2, sh_degree=0)
    outs = [_render(ctx, sc, 0.7, ts)[0].cpu().numpy() for ts in (8, 16, 32)]
    # same fragments in the same order per pixel: identical up to fp32 rounding
    assert np.abs(outs[0] - outs[1]).max() < 1e-6
    assert np.abs(outs[0] - outs[2]).max() < 1e-6


@pytest.mark.parametrize("seed,W,H,n,sigma,valpha", [(95, 40, 34, 300, 0.6, True), (96, 36, 30, 250, 1.0, False)])
def test_soft_gradients(ctx, seed, W, H, n, sigma, valpha):
    from paper_2601_19233_gb300 import umgs
    sc = S.small_scene(seed, W, H, n, mesh_subdiv=2, sh_degree=1, with_valpha=valpha)
    rng = np.random.default_rng(seed)
    ref_img = R.render_image(sc, soft=sigma)
    gC = rng.normal(size=(H, W, 3))
    gT = rng.normal(size=(H, W))
    gC[ref_img["tie"]] = 0
    gT[ref_img["tie"]] = 0
    ref, _, _ = OG.image_grad(sc, gC, gT, soft=sigma)
    hard_ref, _, _ = OG.image_grad(sc, gC, gT)
    out, fr, g, ms = _render(ctx, sc, sigma, 16, save=True)
    dl = torch.as_tensor(np.concatenate([gC, gT[..., None]], -1)[None].astype(np.float32)).cuda()
    got = umgs.render_backward(ctx, fr, g, ms, dl)
    torch.cuda.synchronize()
    names = ["means", "quats", "scales", "opacities", "sh", "verts0", "vcolor0", "valpha0" if valpha else "falpha0"]
    for k in names:
        r = ref[k]
        gk = got[k].cpu().numpy().reshape(r.shape)
        scale = np.abs(r).max()
        assert np.abs(gk - r).max() <= 1e-3 * scale + 1e-6, (k, np.abs(gk - r).max(), scale)
    # coverage carries gradient to the vertex positions that the binary form has not
    assert np.abs(ref["verts0"] - hard_ref["verts0"]).max() > 0.1 * np.abs(ref["verts0"]).max()


def test_soft_sliver_takes_the_setup_orientation(ctx):
    """A sliver whose snapped integer area and unsnapped area have opposite
    signs: the kernels take the soft coverage's orientation from the triangle
    record (the setup's integer sign), as the oracle does: image and vertex
    gradients match it."""
    from paper_2601_19233_gb300 import umgs
    from tests.test_oracle_soft import SLIVER
    c = H.cam(48, 32)
    g = H.gaussians(np.array([[0.1, 0.05, 0.3]]), scales=np.full((1, 3), 0.08, np.float32), opac=[0.5],
                    colors=[[0.2, 0.8, 0.4]])
    sc = H.scene(g, [H.single_triangle(c, SLIVER, 0.2, 0.7)], c, tile=8)
    out, fr, gd, ms = _render(ctx, sc, 0.5, 8, save=True)
    _check_lists(sc, fr, 8, 0.5)
    ref = R.render_image(sc, soft=0.5)
    check_ref(out.cpu().numpy()[0], ref)
    rng = np.random.default_rng(3)
    gC = rng.normal(size=(32, 48, 3))
    gT = rng.normal(size=(32, 48))
    gC[ref["tie"]] = 0
    gT[ref["tie"]] = 0
    r, _, _ = OG.image_grad(sc, gC, gT, soft=0.5)
    dl = torch.as_tensor(np.concatenate([gC, gT[..., None]], -1)[None].astype(np.float32)).cuda()
    got = umgs.render_backward(ctx, fr, gd, ms, dl)
    torch.cuda.synchronize()
    gk = got["verts0"].cpu().numpy().reshape(r["verts0"].shape)
    assert np.abs(gk - r["verts0"]).max() <= 1e-3 * np.abs(r["verts0"]).max() + 1e-6


def test_soft_invalid_options_rejected(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = S.small_scene(97, 16, 16, 10, mesh_subdiv=1)
    g = umgs.gaussians_to_device(sc.gaussians)
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    bad = [umgs.render_opts(16, edge_sigma=-1.0), umgs.render_opts(16, edge_sigma=17.0),
           umgs.render_opts(16, blend_mode=umgs.BLEND_MSAA_ALL, edge_sigma=0.5),
           umgs.render_opts(16, mixed=True, edge_sigma=0.5), umgs.render_opts(16, t_product=True, edge_sigma=0.5),
           umgs.render_opts(16, sched=1, edge_sigma=0.5)]
    for o in bad:
        with pytest.raises(umgs.UmgsError):
            umgs.render(ctx, g, ms, sc.cameras, o, frame=umgs.Frame(ctx))
