"""Pins of the gradient oracle: its torch forward equals the numpy forward,
its SH basis equals the general-definition basis, and its autograd gradient
equals central finite differences of the numpy forward."""
import copy

import numpy as np
import pytest
import torch

from oracle import grad as G
from oracle import render as R
from oracle.sh import sh_basis
from paper_2601_19233_gb300 import scenes as S


def _scene(seed, valpha, W=24, H=20, n=30, deg=1):
    sc = S.small_scene(seed, W, H, n, mesh_subdiv=1, sh_degree=deg, log_scale_mu=-2.8, with_valpha=valpha,
                       mesh_radius=0.45)
    return sc


def _to64(sc):
    sc = copy.deepcopy(sc)
    g = sc.gaussians
    for k in ("means", "quats", "scales", "opacities", "sh"):
        setattr(g, k, np.asarray(getattr(g, k), np.float64))
    for m in sc.meshes:
        m.verts = np.asarray(m.verts, np.float64)
        m.vcolor = np.asarray(m.vcolor, np.float64)
        if m.valpha is not None:
            m.valpha = np.asarray(m.valpha, np.float64)
        if m.falpha is not None:
            m.falpha = np.asarray(m.falpha, np.float64)
    return sc


def test_sh_torch_matches_definition():
    d = np.random.default_rng(0).normal(size=(200, 3))
    a = G.sh_basis_torch(torch.as_tensor(d), 3).numpy()
    assert np.abs(a - sh_basis(d, 3)).max() < 1e-12


@pytest.mark.parametrize("valpha", [False, True])
def test_torch_forward_equals_numpy_forward(valpha):
    sc = _scene(3, valpha)
    ref = R.render_image(sc)
    fr, pix, table = G.decision_table(sc)
    p = G.leaf_params(sc)
    C, T = G.composite_torch(sc, p, fr, pix, table)
    assert np.abs(C.detach().numpy().reshape(ref["rgb"].shape) - ref["rgb"]).max() < 1e-12
    assert np.abs(T.detach().numpy().reshape(ref["T"].shape) - ref["T"]).max() < 1e-12
    assert sum(len(r) for r in table) > 100


def _fd_check(sc, names_to_check, rng, nsamp=12, h=1e-6):
    H, W = sc.cameras[0].height, sc.cameras[0].width
    gC = rng.normal(size=(H, W, 3))
    gT = rng.normal(size=(H, W))
    grads, _, _ = G.image_grad(sc, gC, gT)
    sc64 = _to64(sc)
    L0, sig0 = G.loss_numpy(sc64, gC, gT)
    checked = 0
    for name in names_to_check:
        ga = grads[name]
        scale = np.abs(ga).max()
        flat = np.argsort(-np.abs(ga).ravel())[: nsamp // 2]
        flat = np.concatenate([flat, rng.choice(ga.size, size=nsamp // 2, replace=False)])
        for fi in flat:
            idx = np.unravel_index(fi, ga.shape)
            if "alpha" in name:
                x0 = float(_get(_to64(sc), name)[idx])
                if x0 <= h or x0 >= 1 - h:  # alpha clamp kink: one-sided derivative only
                    continue
            vals = []
            ok = True
            for sgn in (1, -1):
                s2 = _to64(sc)
                arr = _get(s2, name)
                arr[idx] += sgn * h
                L, sig = G.loss_numpy(s2, gC, gT)
                ok = ok and sig == sig0
                vals.append(L)
            if not ok:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - ga[idx]) <= 1e-5 * scale + 1e-6 * abs(fd), (name, idx, fd, ga[idx], scale)
            checked += 1
    return checked


def _get(sc, name):
    g = sc.gaussians
    if name in ("means", "quats", "scales", "opacities", "sh"):
        return getattr(g, name)
    base, mi = name[:-1], int(name[-1])
    m = sc.meshes[mi]
    return {"verts": m.verts, "vcolor": m.vcolor, "valpha": m.valpha, "falpha": m.falpha}[base]


def test_fd_gaussians_and_vertex_alpha():
    sc = _scene(5, True)
    n = _fd_check(sc, ["means", "quats", "scales", "opacities", "sh", "verts0", "vcolor0", "valpha0"],
                  np.random.default_rng(1))
    assert n >= 60


def test_fd_face_alpha():
    sc = _scene(6, False)
    n = _fd_check(sc, ["falpha0", "verts0", "means", "sh"], np.random.default_rng(2))
    assert n >= 30
