"""Mixed-precision form: bf16 SH coefficients and fp16 Gaussian records with
fp32 accumulation.  Keys and order stay bit-exact (the footprint decisions
are fp32); the image error against the fp64 oracle is bounded and reported."""
import numpy as np
import pytest
import torch

from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests.test_gpu_render import check_lists, check_ref, ctx  # noqa: F401

pytestmark = pytest.mark.gpu


def _render(ctx, sc, mixed, sh_dtype):
    from paper_2601_19233_gb300 import umgs
    g = umgs.gaussians_to_device(sc.gaussians, sh_dtype=sh_dtype)
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    fr = umgs.Frame(ctx)
    out = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, mixed=mixed), frame=fr)
    torch.cuda.synchronize()
    return out.cpu().numpy(), fr


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return 10 * np.log10(1.0 / max(mse, 1e-20))


@pytest.mark.parametrize("seed", [91, 92])
def test_mixed_precision_error_bounded(ctx, seed):
    sc = S.small_scene(seed, 70, 55, 1500, mesh_subdiv=2, sh_degree=3)
    out, fr = _render(ctx, sc, True, torch.bfloat16)
    check_lists(sc, fr, 16)
    ref = R.render_image(sc)
    check_ref(out[0], ref, tol=2e-2)
    ok = ~ref["tie"]
    err = np.abs(out[0, ..., :3] - ref["rgb"])[ok]
    assert np.percentile(err, 99.9) < 1e-2
    assert psnr(out[0, ..., :3][ok], ref["rgb"][ok]) > 45.0
    # fp16 records alone (fp32 SH): smaller error
    out2, _ = _render(ctx, sc, True, torch.float32)
    check_ref(out2[0], ref, tol=1e-2)


def test_bf16_sh_with_fp32_records(ctx):
    sc = S.small_scene(93, 40, 40, 800, mesh_subdiv=1, sh_degree=3)
    out, fr = _render(ctx, sc, False, torch.bfloat16)
    # the oracle evaluated on the bf16-rounded coefficients agrees to fp32 tolerance
    sc2 = S.small_scene(93, 40, 40, 800, mesh_subdiv=1, sh_degree=3)
    sc2.gaussians.sh = torch.as_tensor(sc2.gaussians.sh).to(torch.bfloat16).float().numpy()
    check_ref(out[0], R.render_image(sc2))
