"""GPU backward (umgs_render_backward) against the fp64 autograd oracle.

Tolerance per parameter group: |g - g_ref| <= 1e-3 max|g_ref| + 1e-6 (fp32
accumulation with atomics against fp64).  Upstream gradients are zeroed on
tie pixels (a decision within rounding of a threshold)."""
import numpy as np
import pytest
import torch

from oracle import grad as OG
from oracle import render as R
from paper_2601_19233_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    return umgs.Context(0)


def _run(ctx, sc, seed, tile=None, use_cov3d=False):
    from paper_2601_19233_gb300 import umgs
    cam = sc.cameras[0]
    H, W = cam.height, cam.width
    rng = np.random.default_rng(seed)
    ref_img = R.render_image(sc)
    gC = rng.normal(size=(H, W, 3))
    gT = rng.normal(size=(H, W))
    gC[ref_img["tie"]] = 0
    gT[ref_img["tie"]] = 0
    cov = None
    if use_cov3d:
        from oracle.deform import sym6
        from oracle.render import cov3d_fp64
        cov = sym6(cov3d_fp64(sc.gaussians.quats, sc.gaussians.scales)).astype(np.float32)
    ref, rgb, T = OG.image_grad(sc, gC, gT, cov3d=cov)
    g = umgs.gaussians_to_device(sc.gaussians)
    if use_cov3d:
        g.cov3d = torch.as_tensor(cov).cuda()
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    fr = umgs.Frame(ctx)
    out = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(tile or sc.tile, save=True), frame=fr)
    dl = torch.as_tensor(np.concatenate([gC, gT[..., None]], -1)[None].astype(np.float32)).cuda()
    grads = umgs.render_backward(ctx, fr, g, ms, dl)
    torch.cuda.synchronize()
    return ref, {k: v.cpu().numpy() for k, v in grads.items()}, out.cpu().numpy(), rgb


def _compare(ref, got, names):
    for k in names:
        r = ref[k]
        gk = got[k].reshape(r.shape)
        scale = np.abs(r).max()
        err = np.abs(gk - r).max()
        assert err <= 1e-3 * scale + 1e-6, (k, err, scale)


def test_config0_gradients(ctx):
    sc = S.config0()
    ref, got, out, rgb = _run(ctx, sc, 0)
    _compare(ref, got, ["means", "quats", "scales", "opacities", "sh", "verts0", "vcolor0", "falpha0"])


@pytest.mark.parametrize("seed,W,H,n,deg,valpha", [(71, 45, 37, 500, 3, True), (72, 40, 52, 700, 1, False)])
def test_small_scene_gradients(ctx, seed, W, H, n, deg, valpha):
    sc = S.small_scene(seed, W, H, n, mesh_subdiv=2, sh_degree=deg, with_valpha=valpha)
    ref, got, out, rgb = _run(ctx, sc, seed, tile=16)
    names = ["means", "quats", "scales", "opacities", "sh", "verts0", "vcolor0"]
    names.append("valpha0" if valpha else "falpha0")
    _compare(ref, got, names)


def test_cov3d_input_gradients(ctx):
    sc = S.small_scene(81, 33, 29, 300, mesh_subdiv=1, sh_degree=0)
    ref, got, out, rgb = _run(ctx, sc, 81, tile=8, use_cov3d=True)
    _compare(ref, got, ["means", "cov3d", "opacities", "sh", "verts0", "vcolor0", "falpha0"])


def test_opaque_stack_overflow_rerun(ctx):
    # 12 full-screen opaque-ish quads stacked: more triangle fragments per pixel
    # than the initial saved-state capacity, exercising the re-run path
    from tests import helpers as Hh
    c = Hh.cam(20, 16)
    qs = [Hh.screen_quad(c, z, 0.3, (0.1 * i, 0.5, 1 - 0.05 * i)) for i, z in enumerate(np.linspace(-1.5, 0.8, 12))]
    m = S.Mesh(np.concatenate([q.verts for q in qs]), np.concatenate([q.faces + 4 * i for i, q in enumerate(qs)]),
               np.concatenate([q.vcolor for q in qs]), None, np.concatenate([q.falpha for q in qs]))
    sc = Hh.scene(Hh.no_gaussians(), [m], c)
    ref, got, out, rgb = _run(ctx, sc, 5, tile=8)
    _compare(ref, got, ["verts0", "vcolor0", "falpha0"])


def test_multi_camera_gradients_sum_over_views(ctx):
    # three views of one scene, SH degree 2: the backward sums the per-view
    # gradients, the oracle is run per view and summed
    from paper_2601_19233_gb300 import umgs
    sc = S.small_scene(91, 36, 30, 400, mesh_subdiv=1, sh_degree=2, n_cams=3)
    rng = np.random.default_rng(91)
    dls, ref = [], None
    for c, cam in enumerate(sc.cameras):
        img = R.render_image(sc, c)
        gC = rng.normal(size=(cam.height, cam.width, 3))
        gT = rng.normal(size=(cam.height, cam.width))
        gC[img["tie"]] = 0
        gT[img["tie"]] = 0
        r, _, _ = OG.image_grad(sc, gC, gT, cam_index=c)
        ref = r if ref is None else {k: ref[k] + r[k] for k in ref}
        dls.append(np.concatenate([gC, gT[..., None]], -1))
    g = umgs.gaussians_to_device(sc.gaussians)
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    fr = umgs.Frame(ctx)
    umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, save=True), frame=fr)
    dl = torch.as_tensor(np.stack(dls).astype(np.float32)).cuda()
    got = {k: v.cpu().numpy() for k, v in umgs.render_backward(ctx, fr, g, ms, dl).items()}
    _compare(ref, got, ["means", "quats", "scales", "opacities", "sh", "verts0", "vcolor0", "falpha0"])


def test_bf16_sh_gradients(ctx):
    # SH stored in bf16: the oracle sees the same (bf16-representable) values
    from paper_2601_19233_gb300 import umgs
    sc = S.small_scene(93, 40, 33, 500, mesh_subdiv=1, sh_degree=3)
    sc.gaussians.sh = torch.as_tensor(sc.gaussians.sh).to(torch.bfloat16).to(torch.float32).numpy()
    cam = sc.cameras[0]
    rng = np.random.default_rng(93)
    img = R.render_image(sc)
    gC = rng.normal(size=(cam.height, cam.width, 3))
    gC[img["tie"]] = 0
    ref, _, _ = OG.image_grad(sc, gC, None)
    g = umgs.gaussians_to_device(sc.gaussians, sh_dtype=torch.bfloat16)
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    fr = umgs.Frame(ctx)
    umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, save=True), frame=fr)
    dl = np.zeros((1, cam.height, cam.width, 4), np.float32)
    dl[0, ..., :3] = gC
    got = {k: v.cpu().numpy() for k, v in umgs.render_backward(ctx, fr, g, ms, torch.as_tensor(dl).cuda()).items()}
    assert got["sh"].dtype == np.float32
    _compare(ref, got, ["means", "quats", "scales", "opacities", "sh"])


def test_autograd_function_matches_direct_backward_and_descends(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = S.small_scene(95, 40, 36, 600, mesh_subdiv=1, sh_degree=1)
    g = umgs.gaussians_to_device(sc.gaussians)
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    for t in (g.means, g.quats, g.scales, g.opacities, g.sh, ms[0].verts, ms[0].vcolor):
        t.requires_grad_(True)
    w = torch.randn((1, 36, 40, 4), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    out = umgs.render_autograd(ctx, g, ms, sc.cameras)
    (out * w).sum().backward()
    fr = umgs.Frame(ctx)
    umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, save=True), frame=fr)
    direct = umgs.render_backward(ctx, fr, g, ms, w.contiguous())
    for name, t in (("means", g.means), ("quats", g.quats), ("scales", g.scales), ("opacities", g.opacities),
                    ("sh", g.sh), ("verts0", ms[0].verts), ("vcolor0", ms[0].vcolor)):
        # atomics make the summation order (and the last bits) run-dependent
        d = direct[name]
        assert torch.allclose(t.grad, d, rtol=1e-4, atol=1e-6 * float(d.abs().max()) + 1e-12), name
    # a few gradient steps on the colours lower an L2 loss to a fixed target
    target = umgs.render(ctx, g, ms, sc.cameras).detach() * 0.5
    opt = torch.optim.Adam([g.sh, ms[0].vcolor], lr=2e-2)
    losses = []
    for _ in range(8):
        opt.zero_grad()
        loss = ((umgs.render_autograd(ctx, g, ms, sc.cameras)[..., :3] - target[..., :3]) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.7 * losses[0]
