"""GPU parity of the deformation transfer (Eq. 12-13) against the fp64 oracle."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import deform as D
from oracle.render import cov3d_fp64
from paper_2601_19233_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_19233_gb300 import build, umgs
    build.build()
    return umgs.Context(0)


def _problem(seed=0, n=5000, subdiv=3):
    rng = np.random.default_rng(seed)
    V, F = S.icosphere(subdiv, 1.0)
    g = S.make_gaussians(rng, S.shell_points(rng, n, 1.0, 0.05), -4.0, 0)
    face = rng.integers(0, len(F), size=(n, 8)).astype(np.int32)
    b = rng.uniform(0, 1, size=(n, 8, 2))
    b = np.where(b.sum(-1, keepdims=True) > 1, 1 - b, b).astype(np.float32)
    return V, F, g, face, b


def _run(ctx, V, Vd, F, g, face, b, mode=0, cov3d=None):
    from paper_2601_19233_gb300 import umgs
    dg = umgs.gaussians_to_device(g)
    if cov3d is not None:
        dg.cov3d = torch.as_tensor(cov3d.astype(np.float32)).cuda()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    m, c, q = umgs.deform(ctx, dg, t(face), t(b), t(V.astype(np.float32)), t(Vd.astype(np.float32)), t(F), mode=mode)
    ctx.sync()
    return m.cpu().numpy(), c.cpu().numpy(), q.cpu().numpy()


def _cov_err(c6, Sig):
    ref = D.sym6(Sig)
    scale = np.abs(ref).max(1, keepdims=True)
    return (np.abs(c6 - ref) / scale).max()


def _quat_err(q, qref):
    d = np.minimum(np.abs(q - qref).max(1), np.abs(q + qref).max(1))
    return d.max()


@pytest.mark.parametrize("mode", [D.FRAME, D.LITERAL])
def test_smooth_deformation_matches_oracle(ctx, mode):
    V, F, g, face, b = _problem(1)
    Vd = S.displace(V, S.sinusoid_params(np.random.default_rng(5)), 17)
    m, c, q = _run(ctx, V, Vd, F, g, face, b, mode)
    mr, Sr, qr = D.deform_gaussians(g.means, g.quats, g.scales, face, b, V, Vd, F, mode=mode)
    assert np.abs(m - mr).max() < 1e-5
    assert _cov_err(c, Sr) < 1e-4
    assert _quat_err(q, qr) < 1e-5


def test_vertex_table_matches_oracle(ctx):
    from paper_2601_19233_gb300 import umgs
    V, F, g, face, b = _problem(2)
    Vd = S.displace(V, S.sinusoid_params(np.random.default_rng(6)), 40)
    _run(ctx, V, Vd, F, g, face, b)
    tab = umgs.deform_vertex_table(ctx, len(V)).cpu().numpy()
    delta, r, Sv = D.vertex_transforms(V, Vd, F)
    assert np.abs(tab[:, :3] - delta).max() < 1e-6
    assert np.abs(tab[:, 3:6] - r).max() < 2e-5
    assert np.abs(tab[:, 6:] - D.sym6(Sv)).max() < 2e-5


def test_rigid_motion_moves_gaussians_rigidly(ctx):
    V, F, g, face, b = _problem(3)
    Rm = Rotation.random(random_state=3).as_matrix()
    t = np.array([0.3, -0.1, 0.2])
    Vd = V.astype(np.float64) @ Rm.T + t
    m, c, q = _run(ctx, V, Vd, F, g, face, b)
    assert np.abs(m - (g.means.astype(np.float64) @ Rm.T + t)).max() < 1e-5
    Sig = cov3d_fp64(g.quats, g.scales)
    assert _cov_err(c, Rm @ Sig @ Rm.T) < 1e-5


def test_identity_and_cov3d_input(ctx):
    V, F, g, face, b = _problem(4, n=2000)
    Sig = cov3d_fp64(g.quats, g.scales)
    m, c, q = _run(ctx, V, V, F, g, face, b, cov3d=D.sym6(Sig))
    assert np.abs(m - g.means).max() < 1e-6
    assert _cov_err(c, Sig) < 1e-5


def test_out_of_range_face_is_reported(ctx):
    from paper_2601_19233_gb300 import umgs
    V, F, g, face, b = _problem(5, n=100)
    face = face.copy()
    face[7, 3] = len(F) + 5
    with pytest.raises(umgs.UmgsError) as e:
        _run(ctx, V, V, F, g, face, b)
    assert e.value.status == 1
    ctx.sync()  # status cleared


def test_compact_binding_and_deformation(ctx):
    from paper_2601_19233_gb300 import umgs
    V, F, g, face, b = _problem(3)
    Vd = S.displace(V, S.sinusoid_params(np.random.default_rng(8)), 23)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    tf = t(F)
    cnt, ent = umgs.binding_compact(ctx, t(face), t(b), tf, len(V))
    cnt, ent = cnt.cpu().numpy(), ent.cpu().numpy()
    # the compact form is the binding regrouped: distinct vertices, weights summing
    # (1/8) x the barycentric weights of each vertex over the 8 points
    for i in (0, 17, 4999):
        wv = {}
        for p in range(8):
            w3 = (1.0 - b[i, p, 0] - b[i, p, 1], b[i, p, 0], b[i, p, 1])
            for k in range(3):
                v = int(F[face[i, p], k])
                wv[v] = wv.get(v, 0.0) + 0.125 * float(w3[k])
        assert cnt[i] == len(wv)
        got = {int(ent[i, j, 0]): float(ent[i, j, 1:2].view(np.float32)[0]) for j in range(cnt[i])}
        assert set(got) == set(wv)
        assert max(abs(got[v] - wv[v]) for v in wv) < 1e-6
    assert np.all((cnt >= 1) & (cnt <= 24))
    for mode in (D.FRAME, D.LITERAL):
        m0, c0, q0 = _run(ctx, V, Vd, F, g, face, b, mode)
        dg = umgs.gaussians_to_device(g)
        m1, c1, q1 = umgs.deform_compact(ctx, dg, t(cnt), t(ent), t(V.astype(np.float32)),
                                         t(Vd.astype(np.float32)), tf, mode=mode)
        m1, c1, q1 = m1.cpu().numpy(), c1.cpu().numpy(), q1.cpu().numpy()
        assert np.abs(m1 - m0).max() < 2e-6
        assert (np.abs(c1 - c0) / np.abs(c0).max(1, keepdims=True)).max() < 2e-5
        assert _quat_err(q1, q0) < 2e-6
        mr, Sr, qr = D.deform_gaussians(g.means, g.quats, g.scales, face, b, V, Vd, F, mode=mode)
        assert np.abs(m1 - mr).max() < 1e-5
        assert _cov_err(c1, Sr) < 1e-4


def test_compact_binding_bad_index(ctx):
    from paper_2601_19233_gb300 import umgs
    V, F, g, face, b = _problem(4, n=64)
    face[5, 3] = len(F) + 7
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    cnt, ent = umgs.binding_compact(ctx, t(face), t(b), t(F), len(V))
    assert int(cnt[5]) == -1 and int((cnt >= 1).sum()) == 63
    m, c, q = umgs.deform_compact(ctx, umgs.gaussians_to_device(g), cnt, ent, t(V.astype(np.float32)),
                                  t(V.astype(np.float32)), t(F))
    with pytest.raises(umgs.UmgsError):
        ctx.sync()
    m = m.cpu().numpy()
    assert np.all(np.isnan(m[5])) and np.all(np.isfinite(np.delete(m, 5, axis=0)))


@pytest.mark.parametrize("mode", [D.FRAME, D.LITERAL])
def test_one_ring_transform_matches_oracle(ctx, mode):
    # UMGS_DEFORM_ONE_RING: the per-vertex table from the cotangent-weighted
    # one-ring least squares, then the same Eq. 12-13
    from paper_2601_19233_gb300 import umgs
    V, F, g, face, b = _problem(7)
    Vd = S.displace(V, S.sinusoid_params(np.random.default_rng(8)), 23)
    m, c, q = _run(ctx, V, Vd, F, g, face, b, mode | umgs.DEFORM_ONE_RING)
    tab = umgs.deform_vertex_table(ctx, len(V)).cpu().numpy()
    delta, r, Sv = D.vertex_transforms(V, Vd, F, D.ONE_RING)
    assert np.abs(tab[:, :3] - delta).max() < 1e-6
    assert np.abs(tab[:, 3:6] - r).max() < 2e-5
    assert np.abs(tab[:, 6:] - D.sym6(Sv)).max() < 2e-5
    mr, Sr, qr = D.deform_gaussians(g.means, g.quats, g.scales, face, b, V, Vd, F, mode=mode, method=D.ONE_RING)
    assert np.abs(m - mr).max() < 1e-5
    assert _cov_err(c, Sr) < 1e-4
    assert _quat_err(q, qr) < 1e-5
    # the two readings differ on a smooth non-rigid deformation
    _, r_f, S_f = D.vertex_transforms(V, Vd, F)
    assert np.abs(D.sym6(S_f) - D.sym6(Sv)).max() > 1e-3


def test_one_ring_rigid_and_noalloc_rejects(ctx):
    from paper_2601_19233_gb300 import umgs
    V, F, g, face, b = _problem(9)
    Rm = Rotation.random(random_state=9).as_matrix()
    t = np.array([-0.2, 0.1, 0.3])
    Vd = V.astype(np.float64) @ Rm.T + t
    m, c, q = _run(ctx, V, Vd, F, g, face, b, umgs.DEFORM_ONE_RING)
    assert np.abs(m - (g.means.astype(np.float64) @ Rm.T + t)).max() < 1e-5
    Sig = cov3d_fp64(g.quats, g.scales)
    assert _cov_err(c, Rm @ Sig @ Rm.T) < 1e-5
    with pytest.raises(umgs.UmgsError):  # unknown mode bits
        _run(ctx, V, Vd, F, g, face, b, 2)
    # the allocation-free entry point keeps the per-face reading only
    dg = umgs.gaussians_to_device(g)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    out = (torch.empty((g.n, 3), device="cuda"), torch.empty((g.n, 6), device="cuda"), None)
    with pytest.raises(umgs.UmgsError):
        umgs.deform_noalloc(dg, t(face), t(b), t(V.astype(np.float32)), t(Vd.astype(np.float32)), t(F), out,
                            mode=umgs.DEFORM_ONE_RING)


def test_csr_binding_and_deformation(ctx):
    """The CSR form holds the padded compact rows packed: the same distinct
    vertices and weights per Gaussian (runs padded to an even length with a
    zero weight), and the deformation through it agrees with the padded
    form's."""
    from paper_2601_19233_gb300 import umgs
    V, F, g, face, b = _problem(4)
    face[7, 3] = len(F) + 5  # an out-of-range face: entries (-1, 0) and a NaN output
    Vd = S.displace(V, S.sinusoid_params(np.random.default_rng(9)), 31)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    tf = t(F)
    cnt, ent = umgs.binding_compact(ctx, t(face), t(b), tf, len(V))
    off, csr = umgs.binding_csr(ctx, t(face), t(b), tf, len(V))
    cnt, ent, off, csr = cnt.cpu().numpy(), ent.cpu().numpy(), off.cpu().numpy(), csr.cpu().numpy()
    assert off[0] == 0 and np.all(np.diff(off) % 2 == 0) and off[-1] == len(csr)
    for i in range(len(cnt)):
        run = csr[off[i]:off[i + 1]]
        if cnt[i] < 0:
            assert i == 7 and np.array_equal(run, [[-1, 0], [-1, 0]])
            continue
        assert len(run) == cnt[i] + (cnt[i] & 1)
        assert np.array_equal(run[:cnt[i]], ent[i, :cnt[i]])
        if cnt[i] & 1:
            assert run[-1, 0] == run[0, 0] and run[-1, 1] == 0
    dg = umgs.gaussians_to_device(g)
    for mode in (D.FRAME, D.LITERAL):
        m0, c0, q0 = umgs.deform_compact(ctx, dg, t(cnt), t(ent), t(V.astype(np.float32)),
                                         t(Vd.astype(np.float32)), tf, mode=mode)
        m1, c1, q1 = umgs.deform_csr(ctx, dg, t(off), t(csr), t(V.astype(np.float32)),
                                     t(Vd.astype(np.float32)), tf, mode=mode)
        m0, m1, c0, c1 = m0.cpu().numpy(), m1.cpu().numpy(), c0.cpu().numpy(), c1.cpu().numpy()
        ok = np.ones(len(m0), bool)
        ok[7] = False
        assert np.isnan(m1[7]).all()
        # the same sums (the padding adds 0 x a row); the two kernel builds may round apart
        assert np.abs(m1[ok] - m0[ok]).max() < 2e-6
        assert (np.abs(c1[ok] - c0[ok]) / np.abs(c0[ok]).max(1, keepdims=True)).max() < 2e-5
        assert _quat_err(q1.cpu().numpy()[ok], q0.cpu().numpy()[ok]) < 2e-6
    with pytest.raises(umgs.UmgsError):
        ctx.sync()  # the bad index is reported
