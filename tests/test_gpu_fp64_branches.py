"""The two fp64 branches of the GPU path, forced and checked against the oracle.

* Near-singular projected covariances (EWA projection, Sec. 3.2): a conic
  whose 2x2 determinant is below a*c/128 is inverted in fp64.  Long, thin
  needle Gaussians seen obliquely reach that branch; their keys must stay
  bit-exact and their images within 2e-4 of the fp64 oracle, and the frame's
  fp64 conic counter reports how many (camera, Gaussian) records took it.
* Sliver proxy faces (per-face deformation gradient, Sec. 3.3): a rest frame
  with |e1 x e2| < 1e-3 |e1||e2| is inverted in fp64.  A proxy with an
  isolated sliver triangle, Gaussians bound to it, must deform like the fp64
  oracle (mu' within 1e-5, Sigma' within 1e-4 relative), and the context's
  fp64 face counter reports the sliver.
"""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import deform as D
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H
from tests.test_gpu_render import check_image, check_lists, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    return umgs.Context(0)


def _needles(seed, n_needle=60, n_plain=300, size=192):
    """Needles of 0.6-1.2 world units (35-70 px at this focal length) with a
    1e-4 cross-section in random 3D directions, between ordinary Gaussians."""
    rng = np.random.default_rng(seed)
    c = H.cam(size, size)
    mu = np.c_[rng.uniform(-0.6, 0.6, (n_needle + n_plain, 2)), rng.uniform(-0.3, 0.3, n_needle + n_plain)]
    sc = np.exp(rng.normal(-3.5, 0.4, (n_needle + n_plain, 3)))
    sc[:n_needle] = np.c_[rng.uniform(0.6, 1.2, n_needle), np.full((n_needle, 2), 1e-4)]
    q = Rotation.random(n_needle + n_plain, random_state=seed).as_quat()[:, [3, 0, 1, 2]]
    op = rng.uniform(0.3, 0.95, n_needle + n_plain)
    col = rng.uniform(0, 1, (n_needle + n_plain, 3))
    g = H.gaussians(mu, scales=sc, quats=q, opac=op, colors=col)
    m = H.single_triangle(c, [(20, 30), (170, 60), (90, 170)], 0.4, 0.6)
    return H.scene(g, [m], c, tile=16)


@pytest.mark.parametrize("seed", [41, 42])
def test_needle_gaussians_take_the_fp64_conic_branch(ctx, seed):
    sc = _needles(seed)
    out, fr = gpu_render(ctx, sc, tile=16)
    check_lists(sc, fr, 16)
    check_image(sc, out)
    st = fr.stats()
    # the oracle's fp64 Sigma_2D of these needles is that near-singular too
    assert st["fp64_conics"] >= 10, st


def _sliver_problem(seed=0, n=2000):
    rng = np.random.default_rng(seed)
    V, F = S.icosphere(2, 1.0)
    nv = len(V)
    # an isolated sliver: sin(angle at the first vertex) = 2.5e-4 / 0.5 = 5e-4
    sl = np.array([[2.0, 0.0, 0.0], [3.0, 0.0, 0.0], [2.5, 2.5e-4, 0.0]], np.float32)
    V = np.concatenate([V, sl]).astype(np.float32)
    F = np.concatenate([F, [[nv, nv + 1, nv + 2]]]).astype(np.int32)
    means = np.concatenate([S.shell_points(rng, n // 2, 1.0, 0.05),
                            sl.mean(0) + rng.normal(0, 0.05, (n - n // 2, 3)).astype(np.float32)])
    g = S.make_gaussians(rng, means.astype(np.float32), -4.0, 0)
    face = rng.integers(0, len(F) - 1, size=(n, 8)).astype(np.int32)
    face[n // 2:] = len(F) - 1  # the second half is bound to the sliver only
    b = rng.uniform(0, 1, size=(n, 8, 2))
    b = np.where(b.sum(-1, keepdims=True) > 1, 1 - b, b).astype(np.float32)
    # a smooth displacement plus a rotation of the sliver about its centre
    Vd = S.displace(V, S.sinusoid_params(np.random.default_rng(seed + 1)), 23).astype(np.float64)
    Rm = Rotation.from_rotvec([0.2, -0.1, 0.3]).as_matrix()
    c0 = sl.mean(0)
    Vd[nv:] = (V[nv:] - c0) @ Rm.T + c0 + np.array([0.01, 0.02, -0.01])
    return V, Vd.astype(np.float32), F, g, face, b


def test_sliver_proxy_face_takes_the_fp64_inverse(ctx):
    from paper_2601_19233_gb300 import umgs
    V, Vd, F, g, face, b = _sliver_problem(3)
    dg = umgs.gaussians_to_device(g)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    m, c, q = umgs.deform(ctx, dg, t(face), t(b), t(V), t(Vd), t(F))
    ctx.sync()
    assert umgs.deform_fp64_faces(ctx) == 1
    m, c = m.cpu().numpy(), c.cpu().numpy()
    mr, Sr, _ = D.deform_gaussians(g.means, g.quats, g.scales, face, b, V, Vd, F)
    assert np.abs(m - mr).max() < 1e-5
    ref = D.sym6(Sr)
    assert (np.abs(c - ref) / np.abs(ref).max(1, keepdims=True)).max() < 1e-4
    # the sliver's vertices have that one face only: their transform is the
    # face's deformation gradient (here a rotation) itself
    tab = umgs.deform_vertex_table(ctx, len(V)).cpu().numpy()
    delta, r, Sv = D.vertex_transforms(V, Vd, F)
    assert np.abs(tab[-3:, 3:6] - r[-3:]).max() < 2e-5
    assert np.abs(tab[-3:, 6:] - D.sym6(Sv[-3:])).max() < 2e-5
    # a sliver-free proxy takes no fp64 inverse
    Vs, Fs = S.icosphere(2, 1.0)
    n = 100
    umgs.deform(ctx, umgs.gaussians_to_device(S.make_gaussians(np.random.default_rng(1), S.shell_points(
        np.random.default_rng(2), n), -4.0, 0)), t(np.zeros((n, 8), np.int32)), t(np.full((n, 8, 2), 0.25, np.float32)),
        t(Vs.astype(np.float32)), t(Vs.astype(np.float32)), t(Fs.astype(np.int32)))
    assert umgs.deform_fp64_faces(ctx) == 0
