"""GPU parity of the forward rasterizer against the oracle (through the C ABI).

Bar: tile lists (keys: tile, depth bits, unified id) and their sort order are
bit-exact; images agree with the fp64 oracle within max-abs 2e-4 per channel
(fp32 path).  At "tie" pixels, where a fragment's alpha sits within 1e-6 of
the 1/255 cut or T within 0.1% of the termination threshold, the fp32 kernels
may take that decision the other way: there the image must match one of the
oracle's composites with each such decision taken either way.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import canonical as cn
from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H

pytestmark = pytest.mark.gpu
TOL = 2e-4


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    return umgs.Context(0)


def gpu_render(ctx, sc, tile=None, mode=0, t_eps=1e-4, bg=(0, 0, 0), sh_dtype=torch.float32, frame=True):
    from paper_2601_19233_gb300 import umgs
    g = umgs.gaussians_to_device(sc.gaussians, sh_dtype=sh_dtype) if sc.gaussians.n > 0 else None
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    fr = umgs.Frame(ctx) if frame else None
    opts = umgs.render_opts(tile or sc.tile, mode, t_eps, bg)
    out = umgs.render(ctx, g, ms, sc.cameras, opts, frame=fr)
    torch.cuda.synchronize()
    return out.cpu().numpy(), fr


def check_lists(sc, fr, tile):
    prims = [cn.Primitives(sc, c) for c in range(len(sc.cameras))]
    ptr, ids, db = cn.sorted_tile_lists(prims, tile)
    gptr, gids, gdb = fr.lists()
    gptr = gptr.cpu().numpy()
    gids = gids.cpu().numpy().astype(np.int64)
    gdb = gdb.cpu().numpy().view(np.uint32)
    assert gptr.shape == ptr.shape
    assert np.array_equal(gptr, ptr)
    assert np.array_equal(gids, ids)
    assert np.array_equal(gdb, db)
    return len(ids)


def check_ref(img, ref, tol=TOL, tie_max=0.01):
    """One camera's GPU image [H,W,4] against an oracle render_image result:
    every pixel within tol (tie pixels against their alternatives), and at
    most tie_max of the pixels ties."""
    e, nt, bad, et = H.compare_with_ties(img, ref["rgb"], ref["T"], ref["tie"], ref["alts"], tol)
    assert nt <= tie_max * ref["tie"].size, ("tie pixels", nt, ref["tie"].size)
    assert e <= tol and bad == 0, (e, nt, bad, et)
    return e


def check_image(sc, out, mode=R.FULL, bg=(0, 0, 0), tol=TOL):
    for c in range(len(sc.cameras)):
        check_ref(out[c], R.render_image(sc, c, mode=mode, bg=bg), tol)


def test_config0_lists_and_image(ctx):
    sc = S.config0()
    out, fr = gpu_render(ctx, sc)
    nk = check_lists(sc, fr, sc.tile)
    assert nk > 1000
    check_image(sc, out)


@pytest.mark.parametrize("seed,W,Hh,n,sub,deg", [(31, 45, 37, 700, 2, 1), (32, 70, 53, 1500, 3, 3),
                                                  (33, 17, 90, 300, 1, 2)])
def test_ragged_multi_tile_scenes(ctx, seed, W, Hh, n, sub, deg):
    sc = S.small_scene(seed, W, Hh, n, mesh_subdiv=sub, sh_degree=deg, with_valpha=(seed % 2 == 0))
    out, fr = gpu_render(ctx, sc, tile=16)
    check_lists(sc, fr, 16)
    check_image(sc, out)


@pytest.mark.parametrize("mode", [R.DIRECT, R.MSAA_ALL, R.ENTITY_ALL])
def test_ablation_modes(ctx, mode):
    sc = S.config0()
    out, fr = gpu_render(ctx, sc, mode=mode)
    check_image(sc, out, mode=mode)


def test_t_product_reading(ctx):
    # the literal Eq. 6 transmittance inside entities (flag), against the
    # oracle's t_product reading; differs from FULL only on multi-triangle entities
    from paper_2601_19233_gb300 import umgs
    sc = S.config0()
    g = umgs.gaussians_to_device(sc.gaussians)
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    out = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(sc.tile, t_product=True)).cpu().numpy()
    check_ref(out[0], R.render_image(sc, t_product=True))
    with pytest.raises(umgs.UmgsError):
        umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(sc.tile, t_product=True, save=True))
    with pytest.raises(umgs.UmgsError):
        umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(sc.tile, blend_mode=R.DIRECT, t_product=True))


def test_tile_sizes_bit_identical(ctx):
    sc = S.small_scene(41, 77, 45, 900, mesh_subdiv=2, sh_degree=1)
    outs = []
    for ts in (8, 16, 32):
        o, fr = gpu_render(ctx, sc, tile=ts)
        check_lists(sc, fr, ts)
        outs.append(o)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    check_image(sc, outs[1])


def test_wide_depth_range_takes_the_fourth_depth_pass(ctx):
    # depths from 0.3 to 150: the high halves of the depth keys span more than
    # 255 values, so the depth sort runs its fourth pass (on the digit counts
    # its third pass gathers); lists bit-exact, image within the bar
    rng = np.random.default_rng(77)
    c = H.cam(64, 48)
    n = 900
    Z = np.exp(rng.uniform(np.log(0.3), np.log(150.0), n)).astype(np.float32)
    u, v = rng.uniform(0, 64, n), rng.uniform(0, 48, n)
    means = np.c_[(u - c.cx) * Z / c.fx, (v - c.cy) * Z / c.fy, Z - c.viewmat[2, 3]]
    scales = (np.exp(rng.normal(0.7, 0.4, (n, 3))) * Z[:, None] / c.fx).astype(np.float32)
    g = H.gaussians(means, scales=scales, opac=rng.uniform(0.2, 0.9, n), colors=rng.uniform(0, 1, (n, 3)))
    m = H.single_triangle(c, [(5, 4), (60, 10), (30, 44)], 20.0 - c.viewmat[2, 3], 0.6)
    sc = H.scene(g, [m], c, tile=16)
    k = cn.Primitives(sc, 0).dbits[cn.Primitives(sc, 0).valid]
    assert (int(k.max()) >> 16) - (int(k.min()) >> 16) + 1 > 255
    out, fr = gpu_render(ctx, sc, tile=16)
    check_lists(sc, fr, 16)
    check_image(sc, out)


def test_multi_camera(ctx):
    sc = S.small_scene(51, 48, 40, 800, mesh_subdiv=2, sh_degree=3, n_cams=3)
    out, fr = gpu_render(ctx, sc)
    check_lists(sc, fr, 16)
    check_image(sc, out)


def test_background_and_no_early_exit(ctx):
    sc = S.small_scene(61, 33, 33, 500, mesh_subdiv=1)
    bg = (0.2, 0.5, 0.9)
    out, _ = gpu_render(ctx, sc, bg=bg)
    check_image(sc, out, bg=bg)
    out2, _ = gpu_render(ctx, sc, t_eps=0.0)
    check_ref(out2[0], R.render_image(sc, t_eps=None))


def test_empty_and_degenerate_inputs(ctx):
    c = H.cam(20, 13)
    # nothing at all: background, T = 1
    sc = H.scene(H.no_gaussians(), [], c)
    out, fr = gpu_render(ctx, sc, bg=(0.3, 0.2, 0.1))
    assert np.all(out[0, ..., 3] == 1.0)
    assert np.allclose(out[0, ..., :3], np.float32([0.3, 0.2, 0.1]))
    assert fr.counts()[0] == 0
    # Gaussians behind the camera and a triangle crossing the near plane are culled
    g = H.gaussians([[0, 0, -3.5], [0, 0, -10]])
    tri = S.Mesh(np.array([[0, 0, -5], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.int32),
                 np.ones((3, 3), np.float32), None, None)
    sc2 = H.scene(g, [tri], c)
    out2, fr2 = gpu_render(ctx, sc2)
    assert fr2.counts()[0] == 0
    assert np.all(out2[0, ..., 3] == 1.0)
    # a single opaque full-cover triangle returns its exact colour
    m = H.single_triangle(c, [(-500.0, -500.0), (900.0, -500.0), (-500.0, 900.0)], 0.0, 1.0,
                          colors=[[0.25, 0.5, 0.75]] * 3)
    out3, _ = gpu_render(ctx, H.scene(H.no_gaussians(), [m], c))
    assert np.all(out3[0, ..., 3] == 0.0)
    assert np.abs(out3[0, ..., :3] - np.float32([0.25, 0.5, 0.75])).max() < 1e-6


def test_invalid_arguments_rejected(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = S.config0()
    g = umgs.gaussians_to_device(sc.gaussians)
    with pytest.raises(umgs.UmgsError) as e:
        umgs.render(ctx, g, [], sc.cameras, umgs.render_opts(tile_size=12))
    assert e.value.status == 1
    bad = S.Mesh(sc.meshes[0].verts, sc.meshes[0].faces.copy(), sc.meshes[0].vcolor, None, None)
    bad.faces[3, 1] = 10 ** 6
    with pytest.raises(umgs.UmgsError) as e:
        umgs.render(ctx, g, [umgs.mesh_to_device(bad)], sc.cameras)
    assert e.value.status == 1


def _offset_view(t):
    """A float32 copy of t whose data starts 4 bytes past a 16-byte boundary."""
    buf = torch.empty(t.numel() + 1, dtype=torch.float32, device=t.device)
    v = buf[1:].view(t.shape)
    v.copy_(t)
    assert v.data_ptr() % 16 == 4
    return v


def test_misaligned_arrays_rejected_on_the_host(ctx):
    """The kernels move the image, the SH rows of degree 1 and 3, the upstream
    gradient and the backward's quaternions as 16-byte words: a pointer off
    that boundary is refused before anything is launched."""
    from paper_2601_19233_gb300 import umgs
    sc = S.config0()
    cam = sc.cameras[0]
    g = umgs.gaussians_to_device(sc.gaussians)
    n = g.n
    sh3 = torch.zeros((n, 16, 3), device="cuda")
    n0 = umgs.kernel_launches()
    with pytest.raises(umgs.UmgsError) as e:
        umgs.render(ctx, g, [], sc.cameras, out=_offset_view(torch.zeros((1, cam.height, cam.width, 4), device="cuda")))
    assert e.value.status == 1 and "out_rgbt" in str(e.value)
    for sh, deg in ((sh3, 3), (sh3[:, :4].contiguous(), 1)):
        g3 = umgs.DevGaussians(g.means, g.quats, g.scales, g.opacities, _offset_view(sh), deg)
        with pytest.raises(umgs.UmgsError) as e:
            umgs.render(ctx, g3, [], sc.cameras)
        assert e.value.status == 1 and "sh" in str(e.value)
    assert umgs.kernel_launches() == n0
    # rows of degree 0 and 2 are read as single values: any float boundary does
    for deg in (0, 2):
        K = (deg + 1) ** 2
        sh = torch.zeros((n, K, 3), device="cuda")
        sh[:, 0] = g.sh[:, 0]
        g0 = umgs.DevGaussians(g.means, g.quats, g.scales, g.opacities, _offset_view(sh), deg)
        out = umgs.render(ctx, g0, [], sc.cameras)
        ref = umgs.render(ctx, umgs.DevGaussians(g.means, g.quats, g.scales, g.opacities, sh, deg), [], sc.cameras)
        assert torch.equal(out, ref)
    fr = umgs.Frame(ctx)
    out = umgs.render(ctx, g, [], sc.cameras, umgs.render_opts(sc.tile, save=True), frame=fr)
    dl_bad, q_bad, dl = _offset_view(torch.zeros_like(out)), _offset_view(g.quats), torch.zeros_like(out)
    n0 = umgs.kernel_launches()
    with pytest.raises(umgs.UmgsError) as e:
        umgs.render_backward(ctx, fr, g, [], dl_bad)
    assert e.value.status == 1 and "dL_drgbt" in str(e.value)
    gq = umgs.DevGaussians(g.means, q_bad, g.scales, g.opacities, g.sh, g.sh_degree)
    with pytest.raises(umgs.UmgsError) as e:
        umgs.render_backward(ctx, fr, gq, [], dl)
    assert e.value.status == 1 and "quats" in str(e.value)
    assert umgs.kernel_launches() == n0


def test_evaluation_count_matches_oracle(ctx):
    sc = S.config0()
    out, fr = gpu_render(ctx, sc)
    total, per_pix = R.evaluation_count(sc)
    ref = R.render_image(sc)
    got = fr.evaluations()
    # termination ties may move the cut by a few entries on a tie pixel
    assert abs(got - total) <= int(ref["tie"].sum()) * int(per_pix.max())
    assert total > 10000


def test_kernel_launch_counter(ctx):
    # every render launches the projection, shading, triangle setup, the
    # binning kernels and the compositor; the library counts them
    from paper_2601_19233_gb300 import umgs
    sc = S.config0()
    gpu_render(ctx, sc)
    n0 = umgs.kernel_launches()
    gpu_render(ctx, sc)
    n1 = umgs.kernel_launches()
    assert 15 <= n1 - n0 <= 60


def test_maximum_image_width(ctx):
    # 32768 px wide (the largest size the 16-bit packed rects hold) and a
    # ragged 6 px high: Gaussians and a triangle at both horizontal ends and
    # across the 16-bit boundary of the tile index
    W, Hh = 32768, 6
    c = H.cam(W, Hh, fx=W / 2.0)
    Z = 3.0
    xs = [3.0, 40.0, 16380.0, 16390.0, 32700.0, 32766.5]
    means = [[(x - c.cx) * Z / c.fx, (3.0 - c.cy) * Z / c.fy, 0.0] for x in xs]
    g = H.gaussians(means, scales=np.full((len(xs), 3), 0.0006, np.float32),
                    colors=np.linspace(0.1, 0.9, 3 * len(xs)).reshape(-1, 3))
    tri = H.single_triangle(c, [(32740.0, -2.0), (32767.9, 7.5), (32730.0, 8.0)], -0.2, 0.7)
    tri2 = H.single_triangle(c, [(-1.0, 0.5), (12.0, 1.0), (2.0, 7.0)], 0.3, 1.0)
    sc = H.scene(g, [tri, tri2], c, tile=16)
    out, fr = gpu_render(ctx, sc, tile=16)
    check_lists(sc, fr, 16)
    check_image(sc, out)


def test_primitive_count_limits_rejected(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = S.config0()
    g = umgs.gaussians_to_device(sc.gaussians)
    cg = g.c()
    cg.n = 1 << 40  # more primitives than unified 32-bit ids can name
    out = torch.empty((1, 128, 128, 4), device="cuda")
    cams = (umgs.CCamera * 1)(umgs.camera_struct(sc.cameras[0]))
    opts = umgs.render_opts(8)
    st = umgs.lib().umgs_render(ctx._h, ctypes.byref(cg), None, 0, cams, 1, ctypes.byref(opts),
                                umgs._ptr(out), None, None)
    assert st == 1


def test_region_count_limit_rejected(ctx):
    # 9 views of 32768 x 32768 with 8-pixel tiles: 9 x 512 x 1024 regions of
    # 8 x 4 tiles, more than the 2^22 that (region, id) keys can name; the
    # call fails before launching or allocating anything
    from paper_2601_19233_gb300 import umgs
    sc = S.config0()
    g = umgs.gaussians_to_device(sc.gaussians)
    big = H.cam(32768, 32768, fx=16384.0)
    out = torch.empty((1, 4), device="cuda")
    cams = (umgs.CCamera * 9)(*[umgs.camera_struct(big)] * 9)
    opts = umgs.render_opts(8)
    n0 = umgs.kernel_launches()
    st = umgs.lib().umgs_render(ctx._h, ctypes.byref(g.c()), None, 0, cams, 9, ctypes.byref(opts),
                                umgs._ptr(out), None, None)
    assert st == 1 and b"regions" in umgs.lib().umgs_last_error(ctx._h)
    assert umgs.kernel_launches() == n0


def test_wide_records_fill_unstaged(ctx):
    # 2,200 wide Gaussians (3 sigma = 36 px) over a 128 x 32 image with 8-pixel
    # tiles (two regions of 8 x 4 tiles): each pair of a region covers most of
    # its 32 tiles, so a chunk of 2,048 (region, id) pairs carries ~60k list
    # entries, more than the fill stages in shared memory, and writes them
    # directly; lists bit-exact, image against the oracle
    c0 = H.cam(128, 32, fx=100.0)
    rng = np.random.default_rng(21)
    n = 2200
    Z = 3.0
    u = rng.uniform(28.0, 100.0, n)
    v = rng.uniform(12.0, 20.0, n)
    means = np.stack([(u - c0.cx) * Z / c0.fx, (v - c0.cy) * Z / c0.fy, rng.uniform(-0.3, 0.3, n)], 1)
    scales = np.full((n, 3), 12.0 * Z / c0.fx, np.float32)
    g = H.gaussians(means, scales=scales, opac=np.full(n, 0.05, np.float32),
                    colors=rng.uniform(0.1, 0.9, (n, 3)))
    sc = H.scene(g, [], c0, tile=8)
    # no early termination (hundreds of fragments per pixel would put many
    # pixels next to the t_eps threshold)
    out, fr = gpu_render(ctx, sc, tile=8, t_eps=-1.0)
    k = check_lists(sc, fr, 8)
    assert k > 2048 * 20
    # (~2,000 fragments per pixel: 9% of the pixels hold an alpha within 1e-6 of 1/255)
    check_ref(out[0], R.render_image(sc, 0, t_eps=None), tie_max=0.15)
