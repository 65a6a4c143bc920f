"""Pins of the oracle deformation transfer (Eq. 12-13 with the per-face frame reading)."""
import numpy as np
import pytest
from scipy.linalg import polar
from scipy.spatial.transform import Rotation

from oracle import deform as D
from oracle.render import cov3d_fp64
from paper_2601_19233_gb300 import scenes as S


def _setup(seed=0, n=300):
    rng = np.random.default_rng(seed)
    V, F = S.icosphere(2, 1.0)
    mu = (rng.normal(size=(n, 3)) * 0.3).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    s = np.exp(rng.normal(-3, 0.4, size=(n, 3))).astype(np.float32)
    face = rng.integers(0, len(F), size=(n, 8)).astype(np.int32)
    b = rng.uniform(0, 1, size=(n, 8, 2))
    b = np.where(b.sum(-1, keepdims=True) > 1, 1 - b, b).astype(np.float32)
    return V, F, mu, q, s, face, b


def _rot(seed=5):
    return Rotation.random(random_state=seed).as_matrix()


def test_identity_motion():
    V, F, mu, q, s, face, b = _setup()
    mu2, Sig2, q2 = D.deform_gaussians(mu, q, s, face, b, V, V, F)
    assert np.abs(mu2 - mu).max() < 1e-12
    assert np.abs(Sig2 - cov3d_fp64(q, s)).max() < 1e-15
    qn = q / np.linalg.norm(q, axis=1, keepdims=True)
    qn = np.where(qn[:, :1] < 0, -qn, qn)
    assert np.abs(q2 - qn).max() < 1e-7


@pytest.mark.parametrize("mode", [D.FRAME, D.LITERAL])
def test_translation(mode):
    V, F, mu, q, s, face, b = _setup(1)
    t = np.array([0.3, -0.2, 0.7])
    mu2, Sig2, _ = D.deform_gaussians(mu, q, s, face, b, V, V + t, F, mode=mode)
    assert np.abs(mu2 - (mu + t)).max() < 1e-12
    assert np.abs(Sig2 - cov3d_fp64(q, s)).max() < 1e-15


def test_rigid_motion_frame_mode_is_rigid():
    V, F, mu, q, s, face, b = _setup(2)
    Rm, t = _rot(), np.array([0.1, 0.5, -0.3])
    Vd = V.astype(np.float64) @ Rm.T + t
    mu2, Sig2, q2 = D.deform_gaussians(mu, q, s, face, b, V, Vd, F)
    assert np.abs(mu2 - (mu.astype(np.float64) @ Rm.T + t)).max() < 1e-12
    Sig = cov3d_fp64(q, s)
    assert np.abs(Sig2 - Rm @ Sig @ Rm.T).max() < 1e-14
    qr = Rotation.from_matrix(Rm) * Rotation.from_quat(q[:, [1, 2, 3, 0]].astype(np.float64))
    ref = qr.as_quat()[:, [3, 0, 1, 2]]
    ref = np.where(ref[:, :1] < 0, -ref, ref)
    assert np.abs(q2 - ref).max() < 1e-9


def test_rigid_motion_literal_mode_closed_form():
    V, F, mu, q, s, face, b = _setup(3)
    Rm, t = _rot(7), np.array([0.2, 0.0, 0.1])
    Vd = V.astype(np.float64) @ Rm.T + t
    mu2, _, _ = D.deform_gaussians(mu, q, s, face, b, V, Vd, F, mode=D.LITERAL)
    Fi = F[face]
    w = np.stack([1 - b[..., 0].astype(np.float64) - b[..., 1], b[..., 0], b[..., 1]], -1)
    P = np.einsum("nck,nckd->ncd", w, V.astype(np.float64)[Fi]).mean(1)
    assert np.abs(mu2 - (mu + P @ (Rm - np.eye(3)).T + t)).max() < 1e-12


def test_uniform_scale():
    V, F, mu, q, s, face, b = _setup(4)
    k = 1.7
    mu2, Sig2, _ = D.deform_gaussians(mu, q, s, face, b, V, V.astype(np.float64) * k, F)
    assert np.abs(mu2 - k * mu.astype(np.float64)).max() < 1e-12
    assert np.abs(Sig2 - k * k * cov3d_fp64(q, s)).max() < 1e-14


def test_polar_matches_library():
    rng = np.random.default_rng(9)
    M = np.eye(3) + 0.4 * rng.normal(size=(200, 3, 3))
    r, Sv = D.polar_log(M)
    Rm = Rotation.from_rotvec(r).as_matrix()
    for k in range(200):
        Rl, Sl = polar(M[k])  # M = Rl Sl with Rl orthogonal
        if np.linalg.det(M[k]) > 0:
            assert np.abs(Rm[k] - Rl).max() < 1e-9
            assert np.abs(Sv[k] - Sl).max() < 1e-9
        assert abs(np.linalg.det(Rm[k]) - 1) < 1e-12
        assert np.abs(Rm[k] @ Sv[k] - M[k]).max() < 1e-12
        assert np.abs(Sv[k] - Sv[k].T).max() < 1e-15
    assert np.all(np.linalg.norm(r, axis=1) <= np.pi + 1e-12)


def test_face_gradient_maps_edges_and_scaled_normal():
    V, F = S.icosphere(1, 1.0)
    rng = np.random.default_rng(10)
    Vd = V.astype(np.float64) + 0.1 * rng.normal(size=V.shape)
    Df = D.face_gradients(V, Vd, F)
    V = V.astype(np.float64)
    for f in range(len(F)):
        a, b, c = F[f]
        e1, e2 = V[b] - V[a], V[c] - V[a]
        d1, d2 = Vd[b] - Vd[a], Vd[c] - Vd[a]
        n, nd = np.cross(e1, e2), np.cross(d1, d2)
        assert np.allclose(Df[f] @ e1, d1, atol=1e-12)
        assert np.allclose(Df[f] @ e2, d2, atol=1e-12)
        assert np.allclose(Df[f] @ (n / np.sqrt(np.linalg.norm(n))), nd / np.sqrt(np.linalg.norm(nd)), atol=1e-12)


def test_similarity_gives_scaled_rotation_per_vertex():
    V, F = S.icosphere(1, 1.0)
    Rm, k = _rot(11), 1.3
    delta, r, Sv = D.vertex_transforms(V, V.astype(np.float64) @ (k * Rm).T, F)
    assert np.abs(Rotation.from_rotvec(r).as_matrix() - Rm).max() < 1e-12
    assert np.abs(Sv - k * np.eye(3)).max() < 1e-12


# -- the ONE_RING per-vertex reading (cotangent-weighted one-ring least squares) --

def test_one_ring_similarity_gives_scaled_rotation():
    # rigid motions and uniform scalings are reproduced exactly: e' = kR e and
    # n' = kR n make the normal equations B = kR A
    V, F = S.icosphere(2, 1.0)
    Rm, k = _rot(12), 0.7
    Vd = V.astype(np.float64) @ (k * Rm).T + np.array([0.3, -0.2, 0.5])
    delta, r, Sv = D.vertex_transforms(V, Vd, F, D.ONE_RING)
    assert np.abs(Rotation.from_rotvec(r).as_matrix() - Rm).max() < 1e-12
    assert np.abs(Sv - k * np.eye(3)).max() < 1e-12


def test_one_ring_is_the_weighted_least_squares_fit():
    # against the stacked least-squares problem solved directly per vertex
    # (rows sqrt(c) e -> sqrt(c) e' for every face edge at v, plus n -> n'),
    # built here from the mesh without the normal-equation algebra
    V, F = S.icosphere(1, 1.0)
    rng = np.random.default_rng(13)
    V = V.astype(np.float64)
    Vd = V + 0.15 * rng.normal(size=V.shape)
    Dv = D.one_ring_gradients(V, Vd, F)
    for v in range(len(V)):
        rows, rhs = [], []
        nsum, ndsum = np.zeros(3), np.zeros(3)
        for f in np.nonzero((F == v).any(1))[0]:
            tri = F[f]
            nsum += np.cross(V[tri[1]] - V[tri[0]], V[tri[2]] - V[tri[0]])
            ndsum += np.cross(Vd[tri[1]] - Vd[tri[0]], Vd[tri[2]] - Vd[tri[0]])
            for k in range(3):  # edge (tri[k+1], tri[k+2]) opposite corner k
                i, j = tri[(k + 1) % 3], tri[(k + 2) % 3]
                if v not in (i, j):
                    continue
                a, b = V[i] - V[tri[k]], V[j] - V[tri[k]]
                c = max(0.0, 0.5 * np.dot(a, b) / np.linalg.norm(np.cross(a, b)))
                o = j if v == i else i
                rows.append(np.sqrt(c) * (V[o] - V[v]))
                rhs.append(np.sqrt(c) * (Vd[o] - Vd[v]))
        rows.append(nsum / np.sqrt(np.linalg.norm(nsum)))
        rhs.append(ndsum / np.sqrt(np.linalg.norm(ndsum)))
        X, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)  # rows @ X = rhs, X = D^T
        assert np.abs(X.T - Dv[v]).max() < 1e-10


def test_one_ring_deformation_of_gaussians_rigid():
    V, F, mu, q, s, face, b = _setup(21)
    Rm = _rot(22)
    t = np.array([0.1, 0.4, -0.3])
    Vd = V.astype(np.float64) @ Rm.T + t
    mu2, Sig2, q2 = D.deform_gaussians(mu, q, s, face, b, V, Vd, F, method=D.ONE_RING)
    assert np.abs(mu2 - (mu.astype(np.float64) @ Rm.T + t)).max() < 1e-10
    Sig = cov3d_fp64(q, s)
    assert np.abs(Sig2 - Rm @ Sig @ Rm.T).max() < 1e-12
