"""umgs_deform_noalloc: the deformation entry point for callers that cannot
allocate device memory (their allocator owns the device, or they cannot pay
for cudaMalloc's synchronisation).  It must give what umgs_deform gives, call
after call, while keeping its scratch in a fixed device array.

This file is collected last on purpose: it runs after every other test and
also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2601_19233_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _inputs(seed, n=4000, subdiv=3):
    rng = np.random.default_rng(seed)
    V, F = S.icosphere(subdiv, 1.0)
    g = S.make_gaussians(rng, S.shell_points(rng, n, 1.0, 0.05), -4.0, 0)
    face = rng.integers(0, len(F), size=(n, 8)).astype(np.int32)
    b = rng.uniform(0, 1, size=(n, 8, 2))
    b = np.where(b.sum(-1, keepdims=True) > 1, 1 - b, b).astype(np.float32)
    Vd = S.displace(V, S.sinusoid_params(np.random.default_rng(seed + 1)), seed)
    return V, Vd, F, g, face, b


def test_noalloc_matches_context_deform_twice():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    ctx = umgs.Context(0)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    for call, seed in enumerate((11, 12)):  # two calls in a row, different inputs
        V, Vd, F, g, face, b = _inputs(seed)
        dg = umgs.gaussians_to_device(g)
        args = (t(face), t(b), t(V), t(Vd.astype(np.float32)), t(F))
        ref = umgs.deform(ctx, dg, *args)
        ctx.sync()
        n = g.n
        out = (torch.full((n, 3), float("nan"), device="cuda"), torch.full((n, 6), float("nan"), device="cuda"),
               torch.full((n, 4), float("nan"), device="cuda"))
        umgs.deform_noalloc(dg, *args, out=out)
        torch.cuda.synchronize()
        for a, r in zip(out, ref):
            a, r = a.cpu().numpy(), r.cpu().numpy()
            assert np.isfinite(a).all(), call
            scale = max(1.0, float(np.abs(r).max()))
            assert np.abs(a - r).max() <= 1e-5 * scale, call


def test_noalloc_rejects_oversized_proxy():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    nv = umgs.NOALLOC_MAX_PROXY_VERTICES + 1
    V = torch.zeros((nv, 3), device="cuda")
    F = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    g = umgs.DevGaussians(torch.zeros((1, 3), device="cuda"), torch.zeros((1, 4), device="cuda"),
                          torch.ones((1, 3), device="cuda"), torch.ones(1, device="cuda"),
                          torch.zeros((1, 1, 3), device="cuda"), 0)
    face = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    bary = torch.zeros((1, 8, 2), device="cuda")
    out = (torch.empty((1, 3), device="cuda"), torch.empty((1, 6), device="cuda"), None)
    with pytest.raises(umgs.UmgsError) as e:
        umgs.deform_noalloc(g, face, bary, V, V, F, out=out)
    assert e.value.status == 3
