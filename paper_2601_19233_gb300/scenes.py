"""Seeded synthetic scene generators.

This module only draws inputs: Gaussians, triangle meshes, proxy meshes,
cameras and per-frame proxy displacements, as float32/int32 numpy arrays.
It holds none of the rendering, binding or deformation arithmetic, so both
the CUDA path and the CPU oracle can consume its output without sharing any
method code.

Workload shapes follow the paper's setting (Sec. 4): scenes of a few hundred
thousand to millions of Gaussians, proxy meshes of ~20-50K faces, render
meshes of 60K-2M faces and 800x800 to 4K views.  The datasets themselves
(NeRF-Synthetic, MipNeRF360) are not used; these generators stand in for them.

Camera convention: pinhole, world->camera [R|t], OpenCV axes (x right,
y down, z forward), fx = fy = (W/2)/tan(fovx/2), cx = W/2, cy = H/2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SH_C0 = 0.28209479177387814  # only used to express a target colour as a DC coefficient


@dataclass
class Camera:
    viewmat: np.ndarray  # float32 [3,4]  world -> camera [R|t]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2

    def center(self) -> np.ndarray:
        R = self.viewmat[:, :3].astype(np.float64)
        t = self.viewmat[:, 3].astype(np.float64)
        return -R.T @ t


@dataclass
class Gaussians:
    means: np.ndarray      # f32 [N,3]
    quats: np.ndarray      # f32 [N,4] (w,x,y,z), not necessarily normalised
    scales: np.ndarray     # f32 [N,3] activated standard deviations
    opacities: np.ndarray  # f32 [N]   activated, in (0,1)
    sh: np.ndarray         # f32 [N,K,3], K = (deg+1)^2
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


@dataclass
class Mesh:
    verts: np.ndarray            # f32 [V,3]
    faces: np.ndarray            # i32 [F,3]
    vcolor: np.ndarray           # f32 [V,3]
    valpha: np.ndarray | None = None  # f32 [V]
    falpha: np.ndarray | None = None  # f32 [F] (overrides valpha)
    uv: np.ndarray | None = None       # f32 [V,2] texture coordinates (with `texture`)
    texture: np.ndarray | None = None  # f32 [TH,TW,3] RGB; when given, c_i is sampled from it

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nf(self) -> int:
        return int(self.faces.shape[0])


@dataclass
class Scene:
    gaussians: Gaussians
    meshes: list
    cameras: list
    tile: int = 16
    proxy_verts: np.ndarray | None = None
    proxy_faces: np.ndarray | None = None
    bind_cameras: list = field(default_factory=list)
    extra: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# cameras

def focal_from_fov(width: int, fovx_deg: float) -> float:
    return (width / 2.0) / math.tan(math.radians(fovx_deg) / 2.0)


def look_at(eye, target, width, height, fx, near=0.2, down=(0.0, 1.0, 0.0)) -> Camera:
    """Camera at `eye` looking at `target`; world `down` maps to screen +y."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    w = np.asarray(down, np.float64)
    r = np.cross(w, f)
    if np.linalg.norm(r) < 1e-6:
        r = np.cross(np.array([0.0, 0.0, 1.0]), f)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], 0)
    t = -R @ eye
    vm = np.concatenate([R, t[:, None]], 1).astype(np.float32)
    return Camera(vm, float(fx), float(fx), width / 2.0, height / 2.0, int(width), int(height), float(near))


def front_camera(width, height, fx, dist=3.0, near=0.2) -> Camera:
    """R = I, t = (0,0,dist): camera at (0,0,-dist) looking down +z at the origin."""
    vm = np.zeros((3, 4), np.float32)
    vm[:, :3] = np.eye(3, dtype=np.float32)
    vm[2, 3] = dist
    return Camera(vm, float(fx), float(fx), width / 2.0, height / 2.0, int(width), int(height), float(near))


def orbit_cameras(n, radius, width, height, fx, elev_deg_fn=None, near=0.2):
    cams = []
    for k in range(n):
        az = 2.0 * math.pi * k / n
        el = math.radians(elev_deg_fn(k) if elev_deg_fn else 0.0)
        eye = radius * np.array([math.cos(el) * math.sin(az), -math.sin(el), -math.cos(el) * math.cos(az)])
        cams.append(look_at(eye, (0, 0, 0), width, height, fx, near))
    return cams


def fibonacci_cameras(n, radius, width=512, height=512, fovx_deg=60.0, near=0.2):
    ga = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    fx = focal_from_fov(width, fovx_deg)
    for i in range(n):
        z = 1.0 - 2.0 * (i + 0.5) / n
        rr = math.sqrt(max(0.0, 1.0 - z * z))
        phi = i * ga
        eye = radius * np.array([rr * math.cos(phi), rr * math.sin(phi), z])
        cams.append(look_at(eye, (0, 0, 0), width, height, fx, near))
    return cams


# ----------------------------------------------------------------------------
# meshes

def icosphere(subdiv: int, radius: float = 1.0):
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = (np.array(verts) * radius).astype(np.float32)
    F = np.array(faces, np.int32)
    return V, F


def torus(a: int, b: int, major: float = 1.0, minor: float = 0.3):
    """(a x b) quad grid on a torus around the y axis, 2 triangles per quad."""
    i = np.arange(a)
    j = np.arange(b)
    uu, vv = np.meshgrid(2 * np.pi * i / a, 2 * np.pi * j / b, indexing="ij")
    x = (major + minor * np.cos(vv)) * np.cos(uu)
    y = minor * np.sin(vv)
    z = (major + minor * np.cos(vv)) * np.sin(uu)
    V = np.stack([x, y, z], -1).reshape(-1, 3).astype(np.float32)
    idx = lambda ii, jj: (ii % a) * b + (jj % b)
    I, J = np.meshgrid(i, j, indexing="ij")
    I = I.ravel()
    J = J.ravel()
    q0, q1, q2, q3 = idx(I, J), idx(I + 1, J), idx(I + 1, J + 1), idx(I, J + 1)
    F = np.concatenate([np.stack([q0, q1, q2], -1), np.stack([q0, q2, q3], -1)], 0).astype(np.int32)
    # interleave so that the two halves of a quad are adjacent ids
    F = F.reshape(2, -1, 3).transpose(1, 0, 2).reshape(-1, 3)
    return V, F


# ----------------------------------------------------------------------------
# Gaussians

def random_quats(rng, n):
    return rng.normal(size=(n, 4)).astype(np.float32)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def shell_points(rng, n, radius=1.0, noise=0.02):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius + rng.normal(0.0, noise, size=(n, 1))
    return (d * r).astype(np.float32)


def make_gaussians(rng, means, log_scale_mu, sh_degree, sh_sigma=0.2, dc_colors=None):
    n = means.shape[0]
    scales = np.exp(rng.normal(log_scale_mu, 0.5, size=(n, 3))).astype(np.float32)
    quats = random_quats(rng, n)
    opac = sigmoid(rng.normal(0.0, 1.0, size=n)).astype(np.float32)
    K = (sh_degree + 1) ** 2
    if dc_colors is not None:
        sh = np.zeros((n, K, 3), np.float32)
        sh[:, 0, :] = (dc_colors - 0.5) / SH_C0
        if K > 1:
            sh[:, 1:, :] = rng.normal(0.0, sh_sigma, size=(n, K - 1, 3))
    else:
        sh = rng.normal(0.0, sh_sigma, size=(n, K, 3)).astype(np.float32)
    return Gaussians(means.astype(np.float32), quats, scales, opac, sh.astype(np.float32), sh_degree)


# ----------------------------------------------------------------------------
# proxy displacement (smooth, bounded by amplitude)

def sinusoid_params(rng, k=8):
    a = rng.normal(size=(k, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    nvec = rng.normal(size=(k, 3))
    nvec /= np.linalg.norm(nvec, axis=1, keepdims=True)
    omega = rng.uniform(1.0, 4.0, size=k)
    phi = rng.uniform(0.0, 2 * np.pi, size=k)
    return dict(a=a, n=nvec, omega=omega, phi=phi)


def displace(verts, params, frame, amplitude=0.1, period=100):
    a, nvec, om, ph = params["a"], params["n"], params["omega"], params["phi"]
    k = a.shape[0]
    v = verts.astype(np.float64)
    arg = om[None, :] * (v @ nvec.T) + ph[None, :] + 2 * np.pi * frame / period
    d = (np.sin(arg)[:, :, None] * a[None, :, :]).sum(1) * (amplitude / k)
    return (v + d).astype(np.float32)


# ----------------------------------------------------------------------------
# configurations

def config0(seed=1000):
    """128x128, 2,000 Gaussians (SH0), icosphere subdiv-2 mesh (320 faces)."""
    rng = np.random.default_rng(seed)
    W = H = 128
    fx = focal_from_fov(W, 60.0)
    cam = front_camera(W, H, fx, 3.0)
    n = 2000
    means = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    g = make_gaussians(rng, means, -4.0, 0, dc_colors=None)
    cols = rng.uniform(0, 1, size=(n, 3))
    g.sh[:, 0, :] = ((cols - 0.5) / SH_C0).astype(np.float32)
    V, F = icosphere(2, 0.5)
    vcol = rng.uniform(0, 1, size=(V.shape[0], 3)).astype(np.float32)
    falpha = np.ones(F.shape[0], np.float32)
    half = rng.permutation(F.shape[0])[: F.shape[0] // 2]
    falpha[half] = 0.5
    mesh = Mesh(V, F, vcol, None, falpha)
    return Scene(g, [mesh], [cam], tile=8)


def small_scene(seed, W, H, n_gauss, mesh_subdiv=1, sh_degree=0, log_scale_mu=-3.5,
                n_cams=1, with_valpha=False, transparent_frac=0.5, mesh_radius=0.5,
                mesh_offset=(0.0, 0.0, 0.0)):
    """A small scene with ragged image size for parity at multi-tile scale."""
    rng = np.random.default_rng(seed)
    fx = focal_from_fov(W, 60.0)
    if n_cams == 1:
        cams = [front_camera(W, H, fx, 3.0)]
    else:
        cams = orbit_cameras(n_cams, 3.0, W, H, fx, lambda k: 20.0 * math.sin(2 * math.pi * k / 16))
    means = rng.uniform(-1, 1, size=(n_gauss, 3)).astype(np.float32)
    g = make_gaussians(rng, means, log_scale_mu, sh_degree)
    meshes = []
    if mesh_subdiv >= 0:
        V, F = icosphere(mesh_subdiv, mesh_radius)
        V = V + np.asarray(mesh_offset, np.float32)
        vcol = rng.uniform(0, 1, size=(V.shape[0], 3)).astype(np.float32)
        falpha = None
        valpha = None
        if with_valpha:
            valpha = rng.uniform(0.2, 1.0, size=V.shape[0]).astype(np.float32)
        else:
            falpha = np.ones(F.shape[0], np.float32)
            m = rng.uniform(size=F.shape[0]) < transparent_frac
            falpha[m] = rng.uniform(0.2, 0.8, size=int(m.sum())).astype(np.float32)
        meshes.append(Mesh(V, F, vcol, valpha, falpha))
    return Scene(g, meshes, cams, tile=16)


def config1(seed=1001, n_gauss=1_000_000, torus_ab=(400, 250), width=1920, height=1080,
            proxy_subdiv=5, n_bind_cams=100):
    """1080p: 1M Gaussians SH3 on a noisy unit-sphere shell, a 200k-face torus
    (30% of faces alpha U[0.2,0.8]) intersecting it, a 20,480-face proxy."""
    rng = np.random.default_rng(seed)
    fx = focal_from_fov(width, 60.0)
    cam = front_camera(width, height, fx, 3.0)
    means = shell_points(rng, n_gauss, 1.0, 0.02)
    g = make_gaussians(rng, means, -5.0, 3, sh_sigma=0.2)
    V, F = torus(*torus_ab)
    vcol = rng.uniform(0, 1, size=(V.shape[0], 3)).astype(np.float32)
    falpha = np.ones(F.shape[0], np.float32)
    m = rng.uniform(size=F.shape[0]) < 0.3
    falpha[m] = rng.uniform(0.2, 0.8, size=int(m.sum())).astype(np.float32)
    PV, PF = icosphere(proxy_subdiv, 1.0)
    sc = Scene(g, [Mesh(V, F, vcol, None, falpha)], [cam], tile=16, proxy_verts=PV, proxy_faces=PF,
               bind_cameras=fibonacci_cameras(n_bind_cams, 3.0))
    sc.extra["sinusoids"] = sinusoid_params(rng)
    return sc


def config2(seed=1002, n_gauss=500_000, torus_ab=(250, 200), n_cams=64, size=800):
    """64 orbit cameras at 800x800; 70% of Gaussians in 3 blobs (uneven tile load)."""
    rng = np.random.default_rng(seed)
    fx = focal_from_fov(size, 60.0)
    cams = orbit_cameras(n_cams, 3.0, size, size, fx, lambda k: 20.0 * math.sin(2 * math.pi * k / 16))
    nb = int(0.7 * n_gauss)
    centres = rng.uniform(-0.5, 0.5, size=(3, 3))
    which = rng.integers(0, 3, size=nb)
    blob = centres[which] + rng.normal(0.0, 0.15, size=(nb, 3))
    uni = rng.uniform(-1, 1, size=(n_gauss - nb, 3))
    means = np.concatenate([blob, uni], 0).astype(np.float32)
    g = make_gaussians(rng, means, -5.0, 3)
    V, F = torus(*torus_ab)
    vcol = rng.uniform(0, 1, size=(V.shape[0], 3)).astype(np.float32)
    falpha = np.ones(F.shape[0], np.float32)
    m = rng.uniform(size=F.shape[0]) < 0.3
    falpha[m] = rng.uniform(0.2, 0.8, size=int(m.sum())).astype(np.float32)
    return Scene(g, [Mesh(V, F, vcol, None, falpha)], cams, tile=16)


def config3(seed=1003, n_gauss=300_000, torus_ab=(250, 100), n_cams=8, size=512):
    """8 views at 512x512, 300k Gaussians SH3 on a shell + 50k-face torus."""
    rng = np.random.default_rng(seed)
    fx = focal_from_fov(size, 60.0)
    cams = orbit_cameras(n_cams, 3.0, size, size, fx, lambda k: 20.0 * math.sin(2 * math.pi * k / 16))
    means = shell_points(rng, n_gauss, 1.0, 0.02)
    g = make_gaussians(rng, means, -5.0, 3)
    V, F = torus(*torus_ab)
    vcol = rng.uniform(0, 1, size=(V.shape[0], 3)).astype(np.float32)
    falpha = np.ones(F.shape[0], np.float32)
    m = rng.uniform(size=F.shape[0]) < 0.3
    falpha[m] = rng.uniform(0.2, 0.8, size=int(m.sum())).astype(np.float32)
    return Scene(g, [Mesh(V, F, vcol, None, falpha)], cams, tile=16)


def config4(seed=1004, n_gauss=6_000_000, torus_ab=(1000, 1000), width=3840, height=2160):
    """4K, 6M Gaussians SH3 on a shell + 2M-face torus (30% transparent)."""
    rng = np.random.default_rng(seed)
    fx = focal_from_fov(width, 60.0)
    cam = front_camera(width, height, fx, 3.0)
    means = shell_points(rng, n_gauss, 1.0, 0.02)
    g = make_gaussians(rng, means, -5.5, 3)
    V, F = torus(*torus_ab)
    vcol = rng.uniform(0, 1, size=(V.shape[0], 3)).astype(np.float32)
    falpha = np.ones(F.shape[0], np.float32)
    m = rng.uniform(size=F.shape[0]) < 0.3
    falpha[m] = rng.uniform(0.2, 0.8, size=int(m.sum())).astype(np.float32)
    return Scene(g, [Mesh(V, F, vcol, None, falpha)], [cam], tile=16)


def closeup_scene(seed=1006, size=512, n_gauss=400_000):
    """A close-up of a dense, faint cluster (the load imbalance the per-tile
    work split is for): 400k Gaussians of opacity 0.001-0.003 and projected
    sigma ~1.3 px packed into a 64 x 64 pixel square at the image centre, so
    that 16 tiles hold ~40k records each and no pixel reaches T < 1e-4, the
    rest of the image nearly empty; a small opaque icosphere beside it."""
    rng = np.random.default_rng(seed)
    fx = focal_from_fov(size, 60.0)
    cam = front_camera(size, size, fx, 3.0)
    half = 32.0 * 3.0 / fx  # 32 px at depth 3
    means = np.c_[rng.uniform(-half, half, (n_gauss, 2)), rng.uniform(-0.05, 0.05, n_gauss)].astype(np.float32)
    g = make_gaussians(rng, means, math.log(1.3 * 3.0 / fx), 0)
    g.opacities[:] = rng.uniform(0.001, 0.003, size=n_gauss).astype(np.float32)
    Vs, Fs = icosphere(2, 0.1)
    Vs = (Vs + np.array([0.6, 0.0, 0.0], np.float32)).astype(np.float32)
    vcol = rng.uniform(0, 1, size=(Vs.shape[0], 3)).astype(np.float32)
    return Scene(g, [Mesh(Vs, Fs, vcol, None, np.ones(Fs.shape[0], np.float32))], [cam], tile=16)


def nested_scene(seed=1005, size=256, n_gauss=30_000, bowl_subdiv=3, bowl_alpha=0.35, n_cams=1):
    """Nested transparency (the setting of Sec. 4.1, Fig. 5b): a Gaussian
    object (three overlapping coloured boxes of points, 0.5 across) and an
    opaque mesh sphere beside it, both enclosed by a transparent sphere
    ("bowl", radius 0.8, face alpha `bowl_alpha`, bluish).  Returns
    (scene, gaussian_layer, mesh_layer): the full scene and the two
    representations as scenes of their own (for the separate-pass baseline)."""
    rng = np.random.default_rng(seed)
    fx = focal_from_fov(size, 60.0)
    if n_cams == 1:
        cams = [front_camera(size, size, fx, 3.0)]
    else:
        cams = orbit_cameras(n_cams, 3.0, size, size, fx, lambda k: 15.0 * math.sin(2 * math.pi * k / 8))
    centres = np.array([[-0.15, 0.05, 0.0], [0.05, -0.1, 0.1], [0.0, 0.15, -0.1]])
    cols = np.array([[0.9, 0.2, 0.1], [0.95, 0.8, 0.1], [0.2, 0.5, 0.9]])
    which = rng.integers(0, 3, size=n_gauss)
    means = (centres[which] + rng.uniform(-0.12, 0.12, size=(n_gauss, 3))).astype(np.float32)
    means[:, 0] -= 0.15
    g = make_gaussians(rng, means, -4.0, 0, dc_colors=cols[which])
    g.opacities[:] = rng.uniform(0.6, 0.95, size=n_gauss).astype(np.float32)
    Vb, Fb = icosphere(bowl_subdiv, 0.8)
    bowl = Mesh(Vb, Fb, np.tile(np.array([[0.55, 0.75, 1.0]], np.float32), (Vb.shape[0], 1)), None,
                np.full(Fb.shape[0], bowl_alpha, np.float32))
    Vs, Fs = icosphere(2, 0.18)
    Vs = (Vs + np.array([0.38, 0.1, 0.05], np.float32)).astype(np.float32)
    ball = Mesh(Vs, Fs, rng.uniform(0.2, 0.4, size=(Vs.shape[0], 3)).astype(np.float32) + np.float32([0.5, 0.0, 0.3]),
                None, np.ones(Fs.shape[0], np.float32))
    empty = Gaussians(np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32), np.zeros((0, 3), np.float32),
                      np.zeros(0, np.float32), np.zeros((0, 1, 3), np.float32), 0)
    scene = Scene(g, [ball, bowl], cams, tile=16)
    return scene, Scene(g, [], cams, tile=16), Scene(empty, [ball, bowl], cams, tile=16)
