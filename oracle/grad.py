"""fp64 gradient of the composite (test infrastructure only).

The image is a piecewise-smooth function of the scene parameters: the
fragment sets, sample coverages, depth order, 1/255 cuts and the
termination point (the "decisions") are piecewise constant, and between
them the colour is a smooth function (Sec. 3.2, Eq. 1-2, 7-9).  This module
re-states the forward in plain PyTorch CPU fp64 ops with the decisions of
the numpy oracle held fixed, and differentiates it with autograd, giving
the exact gradient of L = sum_pixels (g . C + h T) with respect to
  Gaussians: means, quats, scales, opacities, SH coefficients (or cov3d),
  meshes:    vertex positions, vertex colours, vertex / face alpha.
Vertex positions receive gradient through attribute interpolation only
(coverage is piecewise constant), and with soft-edge coverage (soft=sigma)
also through the coverage c^j of every sample.  The torch forward is pinned against the
numpy forward, and the gradient against central finite differences of the
numpy forward (see tests/test_oracle_grad.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

from . import render as R
from .canonical import SAMPLE_OFFSETS as cn_offsets

DT = torch.float64


def sh_basis_torch(d: torch.Tensor, degree: int) -> torch.Tensor:
    """Real SH (Condon-Shortley phase), index l*l + (m + l), as polynomials:
    Y_l^{+-m} = sqrt(2) K_l^m (-1)^m P_l^(m)(z) Re/Im((x + i y)^m)."""
    n = torch.linalg.norm(d, dim=1, keepdim=True)
    d = d / n
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    cols = [None] * (degree + 1) ** 2
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, degree + 1):
        r0, i0 = re[-1], im[-1]
        re.append(r0 * x - i0 * y)
        im.append(r0 * y + i0 * x)
    for l in range(degree + 1):
        pl = npleg.leg2poly([0] * l + [1])  # power-series coefficients of P_l
        for m in range(l + 1):
            q = nppoly.polyder(pl, m) if m > 0 else pl
            val = torch.zeros_like(z)
            for c in q[::-1]:
                val = val * z + float(c)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            s = (-1.0) ** m
            if m == 0:
                cols[l * l + l] = K * val
            else:
                cols[l * l + l + m] = math.sqrt(2.0) * K * s * val * re[m]
                cols[l * l + l - m] = math.sqrt(2.0) * K * s * val * im[m]
    return torch.stack(cols, 1)


def quat_rotmat_torch(q):
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def gaussians_torch(p, cam, sh_degree):
    """u, v, conic (A, B, C), opacity, rgb of every Gaussian (fp64, differentiable)."""
    vm = torch.as_tensor(np.asarray(cam.viewmat, np.float64))
    Rm, t = vm[:, :3], vm[:, 3]
    mu = p["means"]
    pc = mu @ Rm.T + t
    X, Y, Z = pc[:, 0], pc[:, 1], pc[:, 2]
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    u = fx * X / Z + cx
    v = fy * Y / Z + cy
    if p.get("cov3d") is not None:
        c = p["cov3d"]
        S = torch.stack([torch.stack([c[:, 0], c[:, 1], c[:, 2]], -1),
                         torch.stack([c[:, 1], c[:, 3], c[:, 4]], -1),
                         torch.stack([c[:, 2], c[:, 4], c[:, 5]], -1)], -2)
    else:
        Rq = quat_rotmat_torch(p["quats"])
        M = Rq * p["scales"][:, None, :]
        S = M @ M.transpose(1, 2)
    lim_x = 1.3 * (cam.width / (2.0 * fx))
    lim_y = 1.3 * (cam.height / (2.0 * fy))
    xc = torch.clamp(X / Z, -lim_x, lim_x) * Z
    yc = torch.clamp(Y / Z, -lim_y, lim_y) * Z
    zero = torch.zeros_like(Z)
    J = torch.stack([torch.stack([fx / Z, zero, -fx * xc / (Z * Z)], -1),
                     torch.stack([zero, fy / Z, -fy * yc / (Z * Z)], -1)], -2)
    T = J @ Rm
    S2 = T @ S @ T.transpose(1, 2)
    a = S2[:, 0, 0] + 0.3
    b = S2[:, 0, 1]
    c2 = S2[:, 1, 1] + 0.3
    det = a * c2 - b * b
    conic = torch.stack([c2 / det, -b / det, a / det], -1)
    campos = torch.as_tensor(-(np.asarray(cam.viewmat, np.float64)[:, :3].T @ np.asarray(cam.viewmat, np.float64)[:, 3]))
    K = (sh_degree + 1) ** 2
    Y = sh_basis_torch(mu - campos, sh_degree)
    rgb = torch.clamp(torch.einsum("nk,nkc->nc", Y, p["sh"][:, :K, :]) + 0.5, min=0.0)
    return u, v, conic, p["opacities"], rgb


def vertices_torch(verts, cam):
    vm = torch.as_tensor(np.asarray(cam.viewmat, np.float64))
    pc = verts @ vm[:, :3].T + vm[:, 3]
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    return u, v, pc[:, 2]


def decision_table(scene, cam_index=0, t_eps=R.T_EPS, pixels=None, soft=None):
    """Per pixel: ordered contributing fragments [(id, kind, mask)] up to the
    termination point, from the numpy oracle (FULL mode)."""
    fr = R.Frame(scene, cam_index, soft=soft)
    cam = fr.cam
    if pixels is None:
        pixels = [(x, y) for y in range(cam.height) for x in range(cam.width)]
    table = []
    for (x, y) in pixels:
        frags = fr.fragments_at(int(x), int(y))
        res = R.composite(frags, R.FULL, t_eps)
        used = {i for i, _ in res["weights"]}
        row = [(f["id"], f["kind"], f.get("mask", 0)) for f in frags[:res["n"]] if f["id"] in used]
        table.append(row)
    return fr, pixels, table


def leaf_params(scene, with_cov3d=None):
    """fp64 leaf tensors (requires_grad) of every differentiable input."""
    g = scene.gaussians
    t = lambda a: torch.tensor(np.asarray(a, np.float64), dtype=DT, requires_grad=True)
    p = {"means": t(g.means), "opacities": t(g.opacities), "sh": t(g.sh)}
    if with_cov3d is not None:
        p["cov3d"] = t(with_cov3d)
    else:
        p["quats"] = t(g.quats)
        p["scales"] = t(g.scales)
    for mi, m in enumerate(scene.meshes):
        p["verts%d" % mi] = t(m.verts)
        p["vcolor%d" % mi] = t(m.vcolor)
        if m.falpha is not None:
            p["falpha%d" % mi] = t(m.falpha)
        elif m.valpha is not None:
            p["valpha%d" % mi] = t(m.valpha)
    return p


def composite_torch(scene, p, fr, pixels, table, bg=(0.0, 0.0, 0.0)):
    """Differentiable FULL-mode composite of the given pixels with the
    decision table fixed (with fr.soft set, triangle coverage is the
    differentiable soft-edge coverage of render.soft_coverage).  Returns
    (C [P,3], T [P])."""
    cam = fr.cam
    ng = fr.ng
    P = len(pixels)
    L = max([len(r) for r in table] + [1])
    u, v, conic, opac, rgb = gaussians_torch(p, cam, scene.gaussians.sh_degree)
    kind = np.zeros((P, L), np.int64)
    gid = np.zeros((P, L), np.int64)
    mask = np.zeros((P, L), np.int64)
    for k, row in enumerate(table):
        for j, (i, kd, m) in enumerate(row):
            kind[k, j] = 1 if kd == "g" else 2
            gid[k, j] = i
            mask[k, j] = m
    px = torch.tensor([x + 0.5 for x, _ in pixels], dtype=DT)[:, None].expand(P, L)
    py = torch.tensor([y + 0.5 for _, y in pixels], dtype=DT)[:, None].expand(P, L)
    kind_t = torch.as_tensor(kind)
    # Gaussian alpha and colour per (pixel, slot)
    if ng > 0:
        gi = torch.as_tensor(np.where(kind == 1, gid, 0))
        dx = px - u[gi]
        dy = py - v[gi]
        A, B, C = conic[gi, 0], conic[gi, 1], conic[gi, 2]
        power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
        ga = torch.clamp(opac[gi] * torch.exp(power), max=R.ALPHA_MAX)
        gc = rgb[gi]
    else:  # no Gaussians: no slot is a Gaussian slot
        ga = torch.zeros((P, L), dtype=DT)
        gc = torch.zeros((P, L, 3), dtype=DT)
    # triangle alpha and colour per (pixel, slot)
    ta = torch.zeros((P, L), dtype=DT)
    tc = torch.zeros((P, L, 3), dtype=DT)
    o = torch.stack([torch.as_tensor((mask >> j) & 1, dtype=DT) for j in range(4)], -1)  # [P,L,4]
    for mi, m in enumerate(scene.meshes):
        off = fr.P.mesh_offsets[mi]
        sel = (kind == 2) & (gid >= off) & (gid < off + m.nf)
        if not sel.any():
            continue
        fid = torch.as_tensor(np.where(sel, gid - off, 0))
        F = torch.as_tensor(np.asarray(m.faces, np.int64))[fid]  # [P,L,3]
        vu, vv, vz = vertices_torch(p["verts%d" % mi], cam)
        U_, V_, Z_ = vu[F], vv[F], vz[F]
        lam = []
        for k in range(3):
            a, b = (k + 1) % 3, (k + 2) % 3
            lam.append((U_[..., a] - px) * (V_[..., b] - py) - (U_[..., b] - px) * (V_[..., a] - py))
        lam = torch.stack(lam, -1)
        area = lam.sum(-1, keepdim=True)
        lam = torch.where(area != 0, lam / torch.where(area == 0, torch.ones_like(area), area),
                          torch.full_like(lam, 1.0 / 3.0))
        lam = torch.clamp(lam, min=0.0)
        w = lam / Z_
        s = w.sum(-1, keepdim=True)
        w = torch.where(s > 0, w / torch.where(s > 0, s, torch.ones_like(s)), torch.full_like(w, 1.0 / 3.0))
        col = torch.einsum("plk,plkc->plc", w, p["vcolor%d" % mi][F])
        if ("falpha%d" % mi) in p:
            al = p["falpha%d" % mi][fid]
        elif ("valpha%d" % mi) in p:
            al = (w * p["valpha%d" % mi][F]).sum(-1)
        else:
            al = torch.ones((P, L), dtype=DT)
        al = torch.clamp(al, 0.0, 1.0)
        selt = torch.as_tensor(sel)
        ta = torch.where(selt, al, ta)
        tc = torch.where(selt[..., None], col, tc)
        if fr.soft:
            # the triangle's orientation: the sign of its snapped integer area
            # (render.soft_coverage), a constant of the decision table
            tl = np.where(sel, gid - fr.P.ng, 0)
            sg = torch.as_tensor(np.where(sel, fr.P.tri_sign[tl], 0), dtype=DT)
            cov = []
            for j in range(4):
                sx = px + float(cn_offsets[j, 0]) / 256.0
                sy = py + float(cn_offsets[j, 1]) / 256.0
                c = torch.ones_like(px)
                for e in range(3):
                    a, b = (e + 1) % 3, (e + 2) % 3
                    lam_e = (U_[..., a] - sx) * (V_[..., b] - sy) - (U_[..., b] - sx) * (V_[..., a] - sy)
                    Le = torch.sqrt((U_[..., b] - U_[..., a]) ** 2 + (V_[..., b] - V_[..., a]) ** 2)
                    c = c * torch.sigmoid(sg * lam_e / Le / fr.soft)
                cov.append(torch.where(sg != 0, c, torch.zeros_like(c)))
            o = torch.where(selt[..., None], torch.stack(cov, -1), o)
    Cacc = torch.zeros((P, 3), dtype=DT)
    T = torch.ones(P, dtype=DT)
    Tin = torch.ones(P, dtype=DT)
    t4 = torch.ones((P, 4), dtype=DT)
    in_ent = torch.zeros(P, dtype=torch.bool)
    for j in range(L):
        isg = kind_t[:, j] == 1
        ist = kind_t[:, j] == 2
        # Gaussian step
        a = ga[:, j]
        Cg = Cacc + (T * a)[:, None] * gc[:, j]
        Tg = T * (1 - a)
        # triangle step
        start = ist & ~in_ent
        Tin2 = torch.where(start, T, Tin)
        t42 = torch.where(start[:, None], torch.ones_like(t4), t4)
        oj = o[:, j]
        at = ta[:, j]
        O = (oj * t42).sum(-1) / 4.0
        Ct = Cacc + (Tin2 * O * at)[:, None] * tc[:, j]
        t43 = t42 * (1 - oj * at[:, None])
        Tt = Tin2 * t43.sum(-1) / 4.0
        Cacc = torch.where(isg[:, None], Cg, torch.where(ist[:, None], Ct, Cacc))
        T = torch.where(isg, Tg, torch.where(ist, Tt, T))
        Tin = torch.where(ist, Tin2, Tin)
        t4 = torch.where(ist[:, None], t43, t4)
        in_ent = torch.where(isg, torch.zeros_like(in_ent), torch.where(ist, torch.ones_like(in_ent), in_ent))
    Cout = Cacc + T[:, None] * torch.as_tensor(np.asarray(bg, np.float64))
    return Cout, T


def image_grad(scene, dL_drgb, dL_dT=None, cam_index=0, cov3d=None, bg=(0.0, 0.0, 0.0), t_eps=R.T_EPS,
               soft=None):
    """Gradient of L = sum(dL_drgb . rgb) + sum(dL_dT * T) over the full image.
    Returns (grads dict of numpy fp64 arrays, rgb [H,W,3], T [H,W])."""
    fr, pixels, table = decision_table(scene, cam_index, t_eps, soft=soft)
    p = leaf_params(scene, cov3d)
    C, T = composite_torch(scene, p, fr, pixels, table, bg)
    H, W = fr.cam.height, fr.cam.width
    gC = torch.as_tensor(np.asarray(dL_drgb, np.float64).reshape(-1, 3))
    L = (C * gC).sum()
    if dL_dT is not None:
        L = L + (T * torch.as_tensor(np.asarray(dL_dT, np.float64).reshape(-1))).sum()
    names = list(p.keys())
    gr = torch.autograd.grad(L, [p[k] for k in names], allow_unused=True)
    out = {k: (np.zeros(p[k].shape) if g is None else g.numpy()) for k, g in zip(names, gr)}
    return out, C.detach().numpy().reshape(H, W, 3), T.detach().numpy().reshape(H, W)


def loss_numpy(scene, dL_drgb, dL_dT=None, cam_index=0, bg=(0.0, 0.0, 0.0), t_eps=R.T_EPS, soft=None):
    """L evaluated by the numpy forward oracle (decisions recomputed), plus a
    decision signature for finite-difference checks."""
    r = R.render_image(scene, cam_index, bg=bg, t_eps=t_eps, soft=soft)
    L = float((r["rgb"] * np.asarray(dL_drgb, np.float64)).sum())
    if dL_dT is not None:
        L += float((r["T"] * np.asarray(dL_dT, np.float64)).sum())
    sig = hash((r["sig"],)) if "sig" in r else None
    return L, sig
