"""umgs_spatial_order: the Morton order of the Gaussians' means (a layout
tool), and the binding's and the deformation's independence of the order
the model is stored in (Sec. 3.3 and Eq. 12-13 act per Gaussian: a permuted
model binds and deforms to the permuted result)."""
import numpy as np
import pytest
import torch

from paper_2601_19233_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    return umgs.Context(0)


def _spread10(v):
    v = v.astype(np.uint64) & 0x3ff
    out = np.zeros_like(v)
    for b in range(10):
        out |= ((v >> b) & 1) << (3 * b)
    return out


def morton_codes(means):
    """The code the header states, in float32 with the same operations."""
    means = np.asarray(means, np.float32)
    code = np.zeros(len(means), np.uint64)
    for a in range(3):
        x = means[:, a]
        fin = np.isfinite(x)
        lo, hi = np.float32(x[fin].min()), np.float32(x[fin].max())
        scale = np.float32(1024.0) / np.maximum(np.float32(hi - lo), np.float32(1e-30))
        with np.errstate(invalid="ignore"):
            u = np.fmin(np.fmax((x - lo) * scale, np.float32(0)), np.float32(1023))
        code |= _spread10(u.astype(np.uint32)) << a
    return code


@pytest.mark.parametrize("n", [1, 777, 100_003])
def test_spatial_order_is_the_morton_order(ctx, n):
    from paper_2601_19233_gb300 import umgs
    rng = np.random.default_rng(n)
    means = rng.normal(0, 1, (n, 3)).astype(np.float32)
    if n > 10:
        means[3, 1] = np.nan  # a non-finite coordinate counts as the low bound
        means[5] = means[9]   # equal codes keep index order
    perm = umgs.spatial_order(ctx, torch.as_tensor(means).cuda()).cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(n))
    c = morton_codes(means)[perm]
    assert np.all(c[1:] >= c[:-1])
    tie = c[1:] == c[:-1]
    assert np.all(perm[1:][tie] > perm[:-1][tie])


def test_zero_extent_gives_the_identity(ctx):
    from paper_2601_19233_gb300 import umgs
    means = torch.ones((300, 3), device="cuda")
    assert np.array_equal(umgs.spatial_order(ctx, means).cpu().numpy(), np.arange(300))


def test_permuted_model_deforms_to_the_permuted_result(ctx):
    from paper_2601_19233_gb300 import umgs
    rng = np.random.default_rng(5)
    V, F = S.icosphere(3, 1.0)
    V, F = V.astype(np.float32), F.astype(np.int32)
    n = 3000
    g = S.make_gaussians(rng, S.shell_points(rng, n, 1.0, 0.05), -4.0, 1)
    Vd = S.displace(V, S.sinusoid_params(np.random.default_rng(6)), 17).astype(np.float32)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    dg = umgs.gaussians_to_device(g)
    perm = umgs.spatial_order(ctx, dg.means)
    pl = perm.long()
    dp = umgs.DevGaussians(dg.means[pl].contiguous(), dg.quats[pl].contiguous(), dg.scales[pl].contiguous(),
                           dg.opacities[pl].contiguous(), dg.sh[pl].contiguous(), dg.sh_degree)
    cams = S.fibonacci_cameras(40, 3.0)
    outs, binds = [], []
    for m in (dg, dp):
        face, bary, _, _, _ = umgs.bind(ctx, m, t(V), t(F), cams, mode=umgs.BIND_BBX)
        binds.append((face.cpu().numpy(), bary.cpu().numpy()))
        off, ent = umgs.binding_csr(ctx, face, bary, t(F), len(V))
        outs.append([x.cpu().numpy() for x in umgs.deform_csr(ctx, m, off, ent, t(V), t(Vd), t(F))])
    p = perm.cpu().numpy().astype(np.int64)
    # the binding acts per Gaussian: bit for bit
    assert np.array_equal(binds[0][0][p], binds[1][0]) and np.array_equal(binds[0][1][p], binds[1][1])
    # the deformation too, but the per-vertex table it rebuilds every call is
    # summed with float atomics (area-weighted face gradients): two calls
    # round apart in the last bits
    (m0, c0, q0), (m1, c1, q1) = outs
    assert np.abs(m0[p] - m1).max() < 2e-6
    assert (np.abs(c0[p] - c1) / np.abs(c1).max(1, keepdims=True)).max() < 2e-5
    assert np.abs(np.abs((q0[p] * q1).sum(1)) - 1).max() < 2e-6
