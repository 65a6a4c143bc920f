"""Pins of the oracle's rotations and of the EWA projection with rotated cameras.

Every Gaussian covariance the oracle uses is built from a quaternion
(Sigma = R_q diag(s^2) R_q^T) and projected through the camera rotation
(Sigma_2D = J W Sigma W^T J^T + 0.3 I, the EWA splatting of Sec. 3.2 /
Eq. 1-2 inherited from 3DGS).  These tests fix both against definitions
that share nothing with the oracle's formulas:

  * the rotation of a unit quaternion is checked against hand-written
    matrices of quarter and half turns, against Rodrigues' formula for an
    axis-angle pair, against the quaternion sandwich q v q* evaluated with the
    Hamilton product, and against scipy's Rotation;
  * the projected covariance is checked against the Jacobian of the pinhole
    map world -> pixel taken by central finite differences of the projection
    itself, for rolled and yawed cameras and rotated, anisotropic Gaussians,
    and against closed forms for needles on the optical axis;
  * the Gaussian's pixel rect is the axis-aligned box of its 3-sigma ellipse,
    u +- 3 sqrt(Sigma_2D[0,0]), v +- 3 sqrt(Sigma_2D[1,1]), rounded to the
    pixel centres inside it.
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import canonical as cn
from oracle import grad as OG
from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H

SQ = math.sqrt(0.5)

# (quaternion (w, x, y, z), rotation matrix) written out by hand: a rotation
# by theta about a unit axis n has q = (cos(theta/2), sin(theta/2) n), and a
# quarter turn about x sends y to z and z to -y (right-handed).
HAND = [
    ((SQ, SQ, 0, 0), [[1, 0, 0], [0, 0, -1], [0, 1, 0]]),     # +90 deg about x
    ((SQ, 0, SQ, 0), [[0, 0, 1], [0, 1, 0], [-1, 0, 0]]),     # +90 deg about y
    ((SQ, 0, 0, SQ), [[0, -1, 0], [1, 0, 0], [0, 0, 1]]),     # +90 deg about z
    ((SQ, -SQ, 0, 0), [[1, 0, 0], [0, 0, 1], [0, -1, 0]]),    # -90 deg about x
    ((0, 1, 0, 0), [[1, 0, 0], [0, -1, 0], [0, 0, -1]]),      # 180 deg about x
    ((0, 0, 1, 0), [[-1, 0, 0], [0, 1, 0], [0, 0, -1]]),      # 180 deg about y
    ((0, 0, 0, 1), [[-1, 0, 0], [0, -1, 0], [0, 0, 1]]),      # 180 deg about z
    ((1, 0, 0, 0), [[1, 0, 0], [0, 1, 0], [0, 0, 1]]),        # identity
]


def _canonical_matrix(q):
    r = cn.quat_to_rotmat(np.asarray(q, np.float32).reshape(-1, 4))
    return np.array([[np.asarray(r[i][j], np.float64) for j in range(3)] for i in range(3)]).transpose(2, 0, 1)


def _torch_matrix(q):
    return OG.quat_rotmat_torch(torch.as_tensor(np.asarray(q, np.float64).reshape(-1, 4))).numpy()


ROTMATS = {
    "fp64": lambda q: R.quat_rotmat_fp64(np.asarray(q, np.float64).reshape(-1, 4)),
    "canonical_f32": _canonical_matrix,
    "torch_fp64": _torch_matrix,
}
TOL = {"fp64": 1e-14, "canonical_f32": 2e-7, "torch_fp64": 1e-14}


def _rodrigues(axis, theta):
    n = np.asarray(axis, np.float64)
    n = n / np.linalg.norm(n)
    K = np.array([[0, -n[2], n[1]], [n[2], 0, -n[0]], [-n[1], n[0], 0]])
    return np.eye(3) + math.sin(theta) * K + (1 - math.cos(theta)) * (K @ K)


def _hamilton(p, q):
    pw, pv = p[0], np.asarray(p[1:])
    qw, qv = q[0], np.asarray(q[1:])
    return np.r_[pw * qw - pv @ qv, pw * qv + qw * pv + np.cross(pv, qv)]


@pytest.mark.parametrize("impl", list(ROTMATS))
def test_quarter_and_half_turns(impl):
    for q, M in HAND:
        got = ROTMATS[impl](q)[0]
        assert np.abs(got - np.asarray(M, np.float64)).max() <= TOL[impl], (q, got)


@pytest.mark.parametrize("impl", list(ROTMATS))
def test_rodrigues_axis_angle(impl):
    rng = np.random.default_rng(11)
    for _ in range(20):
        axis = rng.normal(size=3)
        theta = float(rng.uniform(-math.pi, math.pi))
        n = axis / np.linalg.norm(axis)
        q = np.r_[math.cos(theta / 2), math.sin(theta / 2) * n]
        got = ROTMATS[impl](q)[0]
        assert np.abs(got - _rodrigues(axis, theta)).max() <= 10 * TOL[impl] + 1e-15


@pytest.mark.parametrize("impl", list(ROTMATS))
def test_quaternion_sandwich_and_scipy(impl):
    # R v = q (0, v) q*, and scipy's Rotation (scalar-last quaternions); the
    # quaternions are not normalised: every implementation normalises first
    rng = np.random.default_rng(12)
    qs = rng.normal(size=(64, 4)) * rng.uniform(0.2, 3.0, size=(64, 1))
    Ms = ROTMATS[impl](qs)
    ref = Rotation.from_quat(qs[:, [1, 2, 3, 0]]).as_matrix()
    assert np.abs(Ms - ref).max() <= 10 * TOL[impl] + 1e-15
    for q, M in zip(qs, Ms):
        qn = q / np.linalg.norm(q)
        v = rng.normal(size=3)
        rv = _hamilton(_hamilton(qn, np.r_[0.0, v]), qn * np.array([1, -1, -1, -1]))
        assert abs(rv[0]) < 1e-12
        assert np.abs(M @ v - rv[1:]).max() <= 10 * TOL[impl] * np.abs(v).max() + 1e-13


def test_covariance_is_rotated_diagonal():
    # Sigma = R diag(s^2) R^T: the columns of R are the principal axes with
    # variances s^2 (eigen-decomposition), for both oracle paths
    rng = np.random.default_rng(13)
    qs = rng.normal(size=(32, 4))
    sc = rng.uniform(0.01, 0.2, size=(32, 3))
    Sig = R.cov3d_fp64(qs, sc)
    Rs = Rotation.from_quat(qs[:, [1, 2, 3, 0]]).as_matrix()
    for i in range(32):
        for k in range(3):
            axis = Rs[i][:, k]
            assert np.abs(Sig[i] @ axis - sc[i, k] ** 2 * axis).max() < 1e-15
    c6 = cn.cov3d_from_quat_scale(qs.astype(np.float32), sc.astype(np.float32))
    full = np.stack([np.asarray(c, np.float64) for c in c6], -1)
    want = np.stack([Sig[:, 0, 0], Sig[:, 0, 1], Sig[:, 0, 2], Sig[:, 1, 1], Sig[:, 1, 2], Sig[:, 2, 2]], -1)
    assert np.abs(full - want).max() < 1e-6 * np.abs(want).max()


# ---------------------------------------------------------------------------
# EWA projection with rotated cameras

def _camera(Rw, t, W=96, H=72, fx=80.0):
    vm = np.zeros((3, 4), np.float32)
    vm[:, :3] = Rw
    vm[:, 3] = t
    return S.Camera(vm, fx, fx, W / 2.0, H / 2.0, W, H, 0.2)


def _pixel_of(cam, p):
    """The pinhole map world point -> (u, v) in fp64, written out directly."""
    vm = np.asarray(cam.viewmat, np.float64)
    X, Y, Z = vm[:, :3] @ p + vm[:, 3]
    return np.array([cam.fx * X / Z + cam.cx, cam.fy * Y / Z + cam.cy])


def _fd_jacobian(cam, p, h=1e-6):
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (_pixel_of(cam, p + e) - _pixel_of(cam, p - e)) / (2 * h)
    return J


def _sigma2d_from_conic(conic):
    A, B, C = conic
    return np.linalg.inv(np.array([[A, B], [B, C]]))


def _yaw_pitch_roll(yaw, pitch, roll):
    return Rotation.from_euler("yxz", [yaw, pitch, roll]).as_matrix()


def test_needle_on_axis_rolled_camera_swaps_a_and_c():
    # a camera rolled 90 deg about its view axis maps world x to camera y:
    # an axis-aligned needle on the optical axis has its a and c swapped
    fx, Z = 80.0, 3.0
    sx, sy, sz = 0.4, 0.01, 0.02
    g = H.gaussians([[0, 0, 0]], scales=[[sx, sy, sz]])
    sx, sy, sz = (float(x) for x in g.scales[0])  # the stored float32 values
    roll = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], np.float64)   # camera x = -world y, camera y = world x
    plain = R.gaussians_fp64(g, _camera(np.eye(3), [0, 0, Z], fx=fx))
    rolled = R.gaussians_fp64(g, _camera(roll, [0, 0, Z], fx=fx))
    k = (fx / Z) ** 2
    want_plain = np.diag([k * sx * sx + 0.3, k * sy * sy + 0.3])
    want_rolled = np.diag([k * sy * sy + 0.3, k * sx * sx + 0.3])
    assert np.abs(_sigma2d_from_conic(plain["conic"][0]) - want_plain).max() < 1e-12 * k
    assert np.abs(_sigma2d_from_conic(rolled["conic"][0]) - want_rolled).max() < 1e-12 * k
    for cam, want in ((_camera(np.eye(3), [0, 0, Z], fx=fx), want_plain), (_camera(roll, [0, 0, Z], fx=fx), want_rolled)):
        pg = cn.project_gaussians(g.means, g.quats, g.scales, None, cam)
        assert abs(float(pg["a"][0]) - want[0, 0]) < 1e-5 * want[0, 0]
        assert abs(float(pg["c"][0]) - want[1, 1]) < 1e-5 * want[1, 1]
        assert abs(float(pg["b"][0])) < 1e-5


def test_needle_on_axis_yawed_camera_closed_form():
    # camera yawed by phi about its y axis, Gaussian at the origin on the
    # optical axis: Sigma_cam[0,0] = cos^2 phi sx^2 + sin^2 phi sz^2
    fx, Z, phi = 80.0, 3.0, 0.6
    sx, sy, sz = 0.02, 0.05, 0.3
    Ry = np.array([[math.cos(phi), 0, math.sin(phi)], [0, 1, 0], [-math.sin(phi), 0, math.cos(phi)]])
    g = H.gaussians([[0, 0, 0]], scales=[[sx, sy, sz]])
    sx, sy, sz = (float(x) for x in g.scales[0])
    cam = _camera(Ry, [0, 0, Z], fx=fx)
    cp, sp = float(cam.viewmat[0, 0]), float(cam.viewmat[0, 2])  # the stored float32 cos and sin
    k = (fx / Z) ** 2
    a = k * (cp * cp * sx * sx + sp * sp * sz * sz) + 0.3
    c = k * sy * sy + 0.3
    got = _sigma2d_from_conic(R.gaussians_fp64(g, cam)["conic"][0])
    assert np.abs(got - np.diag([a, c])).max() < 1e-11 * k
    pg = cn.project_gaussians(g.means, g.quats, g.scales, None, cam)
    assert abs(float(pg["a"][0]) - a) < 1e-5 * a and abs(float(pg["c"][0]) - c) < 1e-5 * c


def _rotated_scene(seed, n=40):
    """Cameras at distance 3 looking at the origin (look_at), then turned by a
    random roll about the view axis and a small yaw and pitch; Gaussians near
    the origin with random quaternions and anisotropic scales."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(4):
        eye = rng.normal(size=3)
        base = S.look_at(3.0 * eye / np.linalg.norm(eye), np.zeros(3), 96, 72, 80.0)
        turn = _yaw_pitch_roll(rng.uniform(-0.15, 0.15), rng.uniform(-0.15, 0.15), rng.uniform(-math.pi, math.pi))
        Rw = turn @ np.asarray(base.viewmat[:, :3], np.float64)
        t = turn @ np.asarray(base.viewmat[:, 3], np.float64)
        cams.append(_camera(Rw, t))
    means = rng.uniform(-0.3, 0.3, size=(n, 3))
    quats = rng.normal(size=(n, 4))
    scales = np.exp(rng.normal(-3.0, 0.7, size=(n, 3)))
    g = H.gaussians(means, scales=scales, quats=quats)
    return g, cams


def test_projected_covariance_equals_pinhole_jacobian_rotated_cameras():
    # Sigma_2D - 0.3 I = J_pi Sigma J_pi^T with J_pi the Jacobian of the pinhole
    # map world -> pixel at the mean, here taken by finite differences of the
    # map itself; Sigma from scipy's rotation of the quaternion.  Any sign,
    # index or transpose error in J, in the camera rotation W or in R_q fails.
    g, cams = _rotated_scene(21)
    Rq = Rotation.from_quat(np.asarray(g.quats, np.float64)[:, [1, 2, 3, 0]]).as_matrix()
    Sig = Rq @ (np.asarray(g.scales, np.float64)[:, :, None] ** 2 * np.transpose(Rq, (0, 2, 1)))
    checked = 0
    for cam in cams:
        fp = R.gaussians_fp64(g, cam)
        pg = cn.project_gaussians(g.means, g.quats, g.scales, None, cam)
        for i in range(g.n):
            p = np.asarray(g.means[i], np.float64)
            Xc = np.asarray(cam.viewmat, np.float64)[:, :3] @ p + np.asarray(cam.viewmat, np.float64)[:, 3]
            # the Jacobian clamp of 3DGS (1.3 tan(fov/2)) must be inactive here
            if abs(Xc[0] / Xc[2]) > 1.2 * cam.width / (2 * cam.fx) or abs(Xc[1] / Xc[2]) > 1.2 * cam.height / (2 * cam.fy):
                continue
            J = _fd_jacobian(cam, p)
            want = J @ Sig[i] @ J.T + 0.3 * np.eye(2)
            got = _sigma2d_from_conic(fp["conic"][i])
            assert np.abs(got - want).max() < 1e-6 * np.abs(want).max(), (i, got, want)
            uv = _pixel_of(cam, p)
            assert abs(fp["u"][i] - uv[0]) < 1e-9 and abs(fp["v"][i] - uv[1]) < 1e-9
            # canonical fp32 path: same covariance to fp32 accuracy
            got32 = np.array([[pg["a"][i], pg["b"][i]], [pg["b"][i], pg["c"][i]]], np.float64)
            assert np.abs(got32 - want).max() < 2e-5 * np.abs(want).max()
            checked += 1
    assert checked > 100


def test_gaussian_rect_is_box_of_three_sigma_ellipse():
    # the pixel rect of a Gaussian holds the pixel centres (x + 0.5, y + 0.5)
    # with |x + 0.5 - u| <= 3 sqrt(Sigma_2D[0,0]) and |y + 0.5 - v| <= 3 sqrt(Sigma_2D[1,1]),
    # clipped to the image: the axis-aligned bounding box of the ellipse
    # d^T Sigma_2D^-1 d <= 9 (not the circle of radius 3 sqrt(lambda_max)),
    # with Sigma_2D from the pinhole Jacobian as above
    g, cams = _rotated_scene(22, n=60)
    Rq = Rotation.from_quat(np.asarray(g.quats, np.float64)[:, [1, 2, 3, 0]]).as_matrix()
    Sig = Rq @ (np.asarray(g.scales, np.float64)[:, :, None] ** 2 * np.transpose(Rq, (0, 2, 1)))
    checked = anisotropic = 0
    for cam in cams:
        pg = cn.project_gaussians(g.means, g.quats, g.scales, None, cam)
        for i in range(g.n):
            if not pg["valid"][i]:
                continue
            p = np.asarray(g.means[i], np.float64)
            Xc = np.asarray(cam.viewmat, np.float64)[:, :3] @ p + np.asarray(cam.viewmat, np.float64)[:, 3]
            if abs(Xc[0] / Xc[2]) > 1.2 * cam.width / (2 * cam.fx) or abs(Xc[1] / Xc[2]) > 1.2 * cam.height / (2 * cam.fy):
                continue
            J = _fd_jacobian(cam, p)
            S2 = J @ Sig[i] @ J.T + 0.3 * np.eye(2)
            u, v = _pixel_of(cam, p)
            rx, ry = 3 * math.sqrt(S2[0, 0]), 3 * math.sqrt(S2[1, 1])
            edges = [u - rx - 0.5, u + rx - 0.5, v - ry - 0.5, v + ry - 0.5]
            if min(abs(e - round(e)) for e in edges) < 1e-3:
                continue  # a box edge within rounding of a pixel centre
            want = [max(0, math.ceil(edges[0])), min(cam.width - 1, math.floor(edges[1])),
                    max(0, math.ceil(edges[2])), min(cam.height - 1, math.floor(edges[3]))]
            if want[0] > want[1] or want[2] > want[3]:
                continue
            assert list(pg["rect"][i]) == want, (i, pg["rect"][i], want)
            lam = np.linalg.eigvalsh(S2)
            if lam[1] > 2 * lam[0]:
                # the lambda_max circle would be strictly wider on the minor axis
                r = 3 * math.sqrt(lam[1])
                if min(rx, ry) < r - 1.0:
                    anisotropic += 1
            checked += 1
    assert checked > 100
    assert anisotropic > 20
