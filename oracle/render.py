"""fp64 per-pixel composite of triangles and Gaussians (test infrastructure only).

For every pixel the oracle gathers all fragments that cover it, from all
primitives, orders them by (depth bits, unified id) and composites them.  The
fragment set and the order are the canonical float32 decisions of
canonical.py; everything else (Gaussian alpha, colours, attribute
interpolation, blending) is fp64.

Composite (blend mode FULL, Sec. 3.2):
  * a Gaussian fragment (Eq. 1-2): alpha = min(0.99, o * exp(-1/2 d^T conic d))
    with d = pixel centre - projected mean; it is a fragment only when
    alpha >= 1/255.  C += T*alpha*c, T <- T*(1-alpha).
  * a triangle fragment covers >= 1 of the M = 4 samples.  A maximal run of
    triangle fragments with no Gaussian fragment between them is one entity
    (the depth-adjacent grouping of Sec. 3.2).  At the entity start
    T_in = T and t^j = 1 (Eq. 7).  For triangle i of the entity:
    O_i = (1/4) sum_j o_i^j t^j (Eq. 8); C += T_in*O_i*alpha_i*c_i (Eq. 9);
    t^j <- t^j (1 - o_i^j alpha_i) (Eq. 7); T <- T_in*(1/4) sum_j t^j.
    The last update is the reading of "T is still updated for later blending"
    that keeps sum(weights) + T_final = 1; the literal product form
    T <- T*(1 - O_i alpha_i) of Eq. 6 is available as t_product=True.
  * background (Eq. 10-11, read as an opaque background): C += T_final*bg.
  * optional early termination: after blending a fragment, stop once T < t_eps.

Ablation modes of Fig. 3 / Fig. 4:
  DIRECT      triangles are single fragments covered at the pixel centre (no AA).
  MSAA_ALL    Eq. 5-6: a triangle is a pixel-level fragment of alpha O_i*alpha_i
              with O_i = (1/M) sum_j o_i^j.
  ENTITY_ALL  all triangles of the pixel form one entity even with Gaussians
              between them (the colour-overflow case of Fig. 3c).

Soft-edge coverage (an extension beyond the paper, FULL mode only; parity
pinned in tests/test_oracle_soft.py): the binary sample coverage o_i^j of
Eq. 7-8 is replaced by c_i^j = prod_e sigmoid(d_e(s_j) / sigma), d_e the
signed distance (pixels, positive inside) from sample s_j to edge e of the
unsnapped projected triangle, so that the composite is differentiable in the
vertex positions through coverage.  A triangle is a fragment of every pixel
of its pixel rect widened by ceil(8 sigma) pixels; Eq. 7-9 are unchanged with
c in place of o (they reduce to the binary form when every c is 0 or 1).

Tie decisions (test reading; pinned in tests/test_oracle_ties.py): a
Gaussian's alpha within 1e-6 of 1/255, or T within 0.1% of t_eps, is a
decision the fp32 kernels may take the other way.  The composite flags them,
and composite_alternatives composites the pixel with each taken either way.
"""
from __future__ import annotations

import numpy as np

from . import canonical as cn
from .sh import sh_to_rgb

FULL, DIRECT, MSAA_ALL, ENTITY_ALL = 0, 1, 2, 3
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_EPS = 1e-4


# ----------------------------------------------------------------------------
# fp64 per-primitive quantities

def gaussians_fp64(g, cam, cov3d=None):
    """fp64 projected mean (u, v), conic (A, B, C) and colour of every Gaussian."""
    vm = np.asarray(cam.viewmat, np.float64)
    R, t = vm[:, :3], vm[:, 3]
    mu = np.asarray(g.means, np.float64)
    p = mu @ R.T + t
    X, Y, Z = p[:, 0], p[:, 1], p[:, 2]
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    with np.errstate(all="ignore"):
        u = fx * X / Z + cx
        v = fy * Y / Z + cy
        if cov3d is not None:
            c = np.asarray(cov3d, np.float64)
            S = np.stack([np.stack([c[:, 0], c[:, 1], c[:, 2]], -1),
                          np.stack([c[:, 1], c[:, 3], c[:, 4]], -1),
                          np.stack([c[:, 2], c[:, 4], c[:, 5]], -1)], -2)
        else:
            S = cov3d_fp64(g.quats, g.scales)
        lim_x = 1.3 * (cam.width / (2.0 * fx))
        lim_y = 1.3 * (cam.height / (2.0 * fy))
        xc = np.clip(X / Z, -lim_x, lim_x) * Z
        yc = np.clip(Y / Z, -lim_y, lim_y) * Z
        J = np.zeros((len(Z), 2, 3))
        J[:, 0, 0] = fx / Z
        J[:, 0, 2] = -fx * xc / (Z * Z)
        J[:, 1, 1] = fy / Z
        J[:, 1, 2] = -fy * yc / (Z * Z)
        T = J @ R
        S2 = T @ S @ np.transpose(T, (0, 2, 1))
        a = S2[:, 0, 0] + 0.3
        b = S2[:, 0, 1]
        c2 = S2[:, 1, 1] + 0.3
        det = a * c2 - b * b
        conic = np.stack([c2 / det, -b / det, a / det], -1)
    campos = -R.T @ t
    rgb = sh_to_rgb(g.sh, mu - campos, g.sh_degree)
    return dict(u=u, v=v, conic=conic, opacity=np.asarray(g.opacities, np.float64), rgb=rgb, Z=Z)


def quat_rotmat_fp64(q):
    q = np.asarray(q, np.float64)
    n = np.linalg.norm(q, axis=1, keepdims=True)
    n = np.where(n == 0, 1.0, n)
    q = q / n
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)
    return R


def cov3d_fp64(quats, scales):
    R = quat_rotmat_fp64(quats)
    M = R * np.asarray(scales, np.float64)[:, None, :]
    return M @ np.transpose(M, (0, 2, 1))


def vertices_fp64(mesh, cam):
    vm = np.asarray(cam.viewmat, np.float64)
    p = np.asarray(mesh.verts, np.float64) @ vm[:, :3].T + vm[:, 3]
    with np.errstate(all="ignore"):
        u = cam.fx * p[:, 0] / p[:, 2] + cam.cx
        v = cam.fy * p[:, 1] / p[:, 2] + cam.cy
    return u, v, p[:, 2]


def soft_dilation(sigma):
    """Pixels by which a triangle's rect is widened for soft-edge coverage."""
    return int(np.ceil(8.0 * float(np.float32(sigma)))) if sigma else 0


def soft_coverage(tu, tv, px, py, sigma, sg=None):
    """Soft coverage c^j (j = 0..3, the samples of canonical.SAMPLE_OFFSETS)
    of pixel (px, py) by triangles with unsnapped screen vertices tu, tv
    ([K,3] fp64, original vertex order): c^j = prod_e sigmoid(d_e / sigma),
    d_e = s * lambda_e / |P_b - P_a| for the edge (a, b) = (e+1, e+2) opposite
    vertex e, lambda_e(x) = (u_a - x)(v_b - y) - (u_b - x)(v_a - y) twice the
    signed area of (x, P_a, P_b) and s the triangle's orientation: `sg` [K],
    the sign of its snapped integer area (canonical.Primitives.tri_sign, the
    orientation the setup uses), or, when not given, the sign of the
    unsnapped area.  A triangle of zero area covers nothing.  Returns [K,4]."""
    tu = np.asarray(tu, np.float64).reshape(-1, 3)
    tv = np.asarray(tv, np.float64).reshape(-1, 3)
    if sg is None:
        area = (tu[:, 1] - tu[:, 0]) * (tv[:, 2] - tv[:, 0]) - (tu[:, 2] - tu[:, 0]) * (tv[:, 1] - tv[:, 0])
        sg = np.sign(area)
    sg = np.asarray(sg, np.float64).reshape(-1)
    out = np.ones((tu.shape[0], 4))
    for j in range(4):
        sx = px + 0.5 + cn.SAMPLE_OFFSETS[j, 0] / 256.0
        sy = py + 0.5 + cn.SAMPLE_OFFSETS[j, 1] / 256.0
        for e in range(3):
            a, b = (e + 1) % 3, (e + 2) % 3
            lam = (tu[:, a] - sx) * (tv[:, b] - sy) - (tu[:, b] - sx) * (tv[:, a] - sy)
            L = np.hypot(tu[:, b] - tu[:, a], tv[:, b] - tv[:, a])
            with np.errstate(all="ignore"):
                d = np.where(L > 0, sg * lam / np.where(L > 0, L, 1.0), 0.0)
            with np.errstate(over="ignore"):  # exp overflow -> factor 0, as the limit
                out[:, j] *= 1.0 / (1.0 + np.exp(-d / sigma))
    out[sg == 0] = 0.0
    return out


def triangle_attributes(mesh, fid, vu, vv, vz, px, py):
    """Colour and alpha of faces `fid` at the centre of pixel (px, py).

    Screen-space barycentrics of the pixel centre w.r.t. the unsnapped
    projected triangle, clamped at 0, then perspective-corrected with 1/Z and
    normalised; colour and alpha are interpolated from the vertices (alpha is
    the per-face value when given) and alpha is clamped to [0, 1].
    A textured mesh (uv and texture given) takes its colour from the texture
    at the same perspective-correct interpolation of the vertex uv
    (sample_texture).  Returns (colour, alpha, weights); triangle_depth gives
    the depth there.
    """
    f = np.asarray(mesh.faces, np.int64)[fid]
    u = vu[f]
    v = vv[f]
    z = vz[f]
    qx, qy = px + 0.5, py + 0.5
    lam = np.zeros(u.shape)
    for k in range(3):
        a, b = (k + 1) % 3, (k + 2) % 3
        lam[:, k] = (u[:, a] - qx) * (v[:, b] - qy) - (u[:, b] - qx) * (v[:, a] - qy)
    area = lam.sum(1, keepdims=True)
    lam = np.where(area != 0, lam / np.where(area == 0, 1.0, area), 1.0 / 3.0)
    lam = np.maximum(lam, 0.0)
    w = lam / z
    s = w.sum(1, keepdims=True)
    w = np.where(s > 0, w / np.where(s > 0, s, 1.0), 1.0 / 3.0)
    if getattr(mesh, "texture", None) is not None:
        uv = np.einsum("fk,fkc->fc", w, np.asarray(mesh.uv, np.float64)[f])
        col = sample_texture(np.asarray(mesh.texture, np.float64), uv)
    else:
        col = np.einsum("fk,fkc->fc", w, np.asarray(mesh.vcolor, np.float64)[f])
    if mesh.falpha is not None:
        alpha = np.asarray(mesh.falpha, np.float64)[fid]
    elif mesh.valpha is not None:
        alpha = (w * np.asarray(mesh.valpha, np.float64)[f]).sum(1)
    else:
        alpha = np.ones(len(fid))
    return col, np.clip(alpha, 0.0, 1.0), w


def sample_texture(tex, uv):
    """Bilinear texture lookup with clamp-to-edge addressing: texel (i, j)
    (column i, row j) of a [TH,TW,3] texture sits at uv ((i+0.5)/TW,
    (j+0.5)/TH); the four texels around uv are weighted by their distance."""
    th, tw = tex.shape[:2]
    x = uv[:, 0] * tw - 0.5
    y = uv[:, 1] * th - 0.5
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = (x - x0)[:, None], (y - y0)[:, None]
    ix0 = np.clip(x0, 0, tw - 1).astype(np.int64)
    ix1 = np.clip(x0 + 1, 0, tw - 1).astype(np.int64)
    iy0 = np.clip(y0, 0, th - 1).astype(np.int64)
    iy1 = np.clip(y0 + 1, 0, th - 1).astype(np.int64)
    top = (1 - fx) * tex[iy0, ix0] + fx * tex[iy0, ix1]
    bot = (1 - fx) * tex[iy1, ix0] + fx * tex[iy1, ix1]
    return (1 - fy) * top + fy * bot


def triangle_depth(mesh, fid, vu, vv, vz, px, py):
    """Camera depth of faces `fid` at the centre of pixel (px, py): with the
    same clamped screen barycentrics l_m as triangle_attributes, the
    perspective-correct z = (sum_m l_m) / (sum_m l_m / z_m); 3 / sum_m 1/z_m
    when every l_m is 0."""
    f = np.asarray(mesh.faces, np.int64)[fid]
    u, v, z = vu[f], vv[f], vz[f]
    qx, qy = px + 0.5, py + 0.5
    lam = np.zeros(u.shape)
    for k in range(3):
        a, b = (k + 1) % 3, (k + 2) % 3
        lam[:, k] = (u[:, a] - qx) * (v[:, b] - qy) - (u[:, b] - qx) * (v[:, a] - qy)
    area = lam.sum(1, keepdims=True)
    lam = np.where(area != 0, lam / np.where(area == 0, 1.0, area), 1.0 / 3.0)
    lam = np.maximum(lam, 0.0)
    s = (lam / z).sum(1)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(s > 0, lam.sum(1) / np.where(s > 0, s, 1.0), 3.0 / (1.0 / z).sum(1))


# ----------------------------------------------------------------------------
# scene evaluation context for one camera

class Frame:
    """Canonical decisions + fp64 quantities of a scene seen by one camera."""

    def __init__(self, scene, cam_index=0, cov3d=None, soft=None):
        self.scene = scene
        self.cam = scene.cameras[cam_index]
        self.soft = soft  # soft-edge width sigma (pixels), or None for binary coverage
        self.P = cn.Primitives(scene, cam_index, cov3d, soft_dilation(soft))
        self.G = gaussians_fp64(scene.gaussians, self.cam, cov3d)
        self.V = [vertices_fp64(m, self.cam) for m in scene.meshes]
        self.ng = scene.gaussians.n

    def mesh_of(self, tid):
        """(mesh index, face index) of triangle unified id tid."""
        for mi, off in enumerate(self.P.mesh_offsets):
            nf = self.scene.meshes[mi].nf
            if off <= tid < off + nf:
                return mi, tid - off
        raise IndexError(tid)

    def fragments_at(self, px, py, candidates=None):
        """All fragments of pixel (px, py), sorted by (depth bits, id).

        Each fragment is a dict: id, kind ('g'|'t'), alpha (Gaussian alpha
        before the 1/255 test, or triangle alpha), color (3), z (camera depth
        of a Gaussian's mean, or of the triangle at the pixel centre), mask
        (triangle sample bits), centre (triangle centre coverage).
        """
        P = self.P
        if candidates is None:
            r = P.rect
            candidates = np.nonzero(P.valid & (r[:, 0] <= px) & (r[:, 1] >= px) & (r[:, 2] <= py) & (r[:, 3] >= py))[0]
        candidates = np.asarray(candidates, np.int64)
        frags = []
        gi = candidates[candidates < self.ng]
        if len(gi):
            G = self.G
            dx = (px + 0.5) - G["u"][gi]
            dy = (py + 0.5) - G["v"][gi]
            A, B, C = G["conic"][gi, 0], G["conic"][gi, 1], G["conic"][gi, 2]
            power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
            alpha = np.minimum(ALPHA_MAX, G["opacity"][gi] * np.exp(power))
            for k, i in enumerate(gi):
                frags.append(dict(id=int(i), kind="g", alpha=float(alpha[k]), color=G["rgb"][i], z=float(G["Z"][i])))
        ti = candidates[candidates >= self.ng]
        if len(ti):
            loc = ti - self.ng
            mask = cn.sample_coverage(P.A[loc], P.B[loc], P.Cb[loc], px, py)
            cen = cn.centre_coverage(P.A[loc], P.B[loc], P.Cb[loc], px, py)
            for k, tid in enumerate(ti):
                if mask[k] == 0 and not cen[k] and not self.soft:
                    continue
                mi, fi = self.mesh_of(int(tid))
                vu, vv, vz = self.V[mi]
                col, alpha, _ = triangle_attributes(self.scene.meshes[mi], np.array([fi]), vu, vv, vz, px, py)
                zt = triangle_depth(self.scene.meshes[mi], np.array([fi]), vu, vv, vz, px, py)
                f = dict(id=int(tid), kind="t", alpha=float(alpha[0]), color=col[0], z=float(zt[0]),
                         mask=int(mask[k]), centre=bool(cen[k]))
                if self.soft:
                    fv = np.asarray(self.scene.meshes[mi].faces, np.int64)[fi]
                    f["cov"] = soft_coverage(vu[fv], vv[fv], px, py, self.soft, P.tri_sign[loc[k]:loc[k] + 1])[0]
                frags.append(f)
        frags.sort(key=lambda f: (int(P.dbits[f["id"]]), f["id"]))
        return frags


# ----------------------------------------------------------------------------
# the composite itself

def composite(frags, mode=FULL, t_eps=T_EPS, t_product=False, bg=(0.0, 0.0, 0.0), choices=None):
    """Composite a depth-ordered fragment list of one pixel.

    Returns dict: color (3, background included), T (final transmittance),
    weights (list of (id, weight)), depth (sum_i w_i z_i / sum_i w_i over the
    blended fragments, +inf when none), tie (True when a decision sits within
    rounding distance of a threshold: |alpha - 1/255| < 1e-6 or
    |T - t_eps| < 1e-3 t_eps), n (fragments consumed), decisions (the outcome
    taken at each such tie decision, in order: True = the Gaussian is blended
    / the pixel stops).  choices: outcomes to take at the first len(choices)
    tie decisions instead of the fp64 comparison (composite_alternatives).
    """
    C = np.zeros(3)
    T = 1.0
    in_ent = False
    T_in = 1.0
    t = np.ones(4)
    g_since = 1.0
    weights = []
    tie = False
    n = 0
    taken = []

    def decide(outcome):
        if choices is not None and len(taken) < len(choices):
            outcome = bool(choices[len(taken)])
        taken.append(outcome)
        return outcome

    for f in frags:
        n += 1
        if f["kind"] == "g":
            a = f["alpha"]
            keep = a >= ALPHA_MIN
            if abs(a - ALPHA_MIN) < 1e-6:
                tie = True
                keep = decide(keep)
            if not keep:
                continue
            w = T * a
            C += w * f["color"]
            weights.append((f["id"], w))
            T = T * (1.0 - a)
            if mode == ENTITY_ALL:
                g_since *= (1.0 - a)
            else:
                in_ent = False
        else:
            a = f["alpha"]
            if mode == DIRECT:
                if not f["centre"]:
                    continue
                w = T * a
                C += w * f["color"]
                weights.append((f["id"], w))
                T = T * (1.0 - a)
            elif mode == MSAA_ALL:
                m = f["mask"]
                if m == 0:
                    continue
                O = sum((m >> j) & 1 for j in range(4)) / 4.0
                w = T * O * a
                C += w * f["color"]
                weights.append((f["id"], w))
                T = T * (1.0 - O * a)
            else:
                m = f["mask"]
                if "cov" in f:  # soft-edge coverage: a fragment wherever its widened rect holds the pixel
                    assert mode == FULL and not t_product
                    o = np.asarray(f["cov"], np.float64)
                elif m == 0:
                    continue
                else:
                    o = np.array([(m >> j) & 1 for j in range(4)], np.float64)
                if not in_ent:
                    T_in = T
                    t = np.ones(4)
                    g_since = 1.0
                    in_ent = True
                O = float((o * t).sum()) / 4.0
                w = T_in * O * a
                C += w * f["color"]
                weights.append((f["id"], w))
                t = t * (1.0 - o * a)
                if t_product:
                    T = T * (1.0 - O * a)
                elif mode == ENTITY_ALL:
                    T = T_in * float(t.sum()) / 4.0 * g_since
                else:
                    T = T_in * float(t.sum()) / 4.0
        if t_eps is not None:
            stop = T < t_eps
            if abs(T - t_eps) < 1e-3 * t_eps:
                tie = True
                stop = decide(stop)
            if stop:
                break
    C = C + T * np.asarray(bg, np.float64)
    # expected depth of the blended fragments: sum w z / sum w (+inf if none)
    zmap = {f["id"]: f.get("z", np.nan) for f in frags}
    wsum = sum(w for _, w in weights)
    depth = sum(w * zmap[i] for i, w in weights) / wsum if wsum > 0 else np.inf
    return dict(color=C, T=T, weights=weights, tie=tie, n=n, depth=depth, decisions=taken)


def composite_alternatives(frags, mode=FULL, t_eps=T_EPS, t_product=False, bg=(0.0, 0.0, 0.0), max_runs=64):
    """Every result the composite of one pixel can have when each tie
    decision (a fragment's alpha within rounding distance of 1/255, or T of
    t_eps) may go either way: a decision taken in fp32 by the kernels can land
    on the other side of the threshold than the fp64 one here.  Depth-first
    over the decision outcomes (a flipped decision can change which decisions
    follow it); at most max_runs composites.  Returns [n_alt, 4] (RGB, T),
    the fp64 outcome first."""
    out = []
    stack = [[]]
    while stack and len(out) < max_runs:
        c = stack.pop()
        r = composite(frags, mode, t_eps, t_product, bg, choices=c)
        out.append(np.r_[r["color"], r["T"]])
        d = r["decisions"]
        for i in range(len(c), len(d)):
            stack.append(d[:i] + [not d[i]])
    return np.array(out)


def render_pixels(scene, pixels, cam_index=0, mode=FULL, t_eps=T_EPS, t_product=False,
                  bg=(0.0, 0.0, 0.0), cov3d=None, frame=None, soft=None, alts=None):
    """Composite an explicit list of pixels [(x, y), ...] by brute-force gather
    over all primitives.  Returns (rgb [K,3], T [K], tie [K], wsum [K]).
    alts: a dict that receives, for every tie pixel k, its
    composite_alternatives [n_alt, 4]."""
    fr = frame or Frame(scene, cam_index, cov3d, soft)
    K = len(pixels)
    rgb = np.zeros((K, 3))
    T = np.zeros(K)
    tie = np.zeros(K, bool)
    wsum = np.zeros(K)
    for k, (x, y) in enumerate(pixels):
        frags = fr.fragments_at(int(x), int(y))
        r = composite(frags, mode, t_eps, t_product, bg)
        rgb[k] = r["color"]
        T[k] = r["T"]
        tie[k] = r["tie"]
        wsum[k] = sum(w for _, w in r["weights"])
        if alts is not None and r["tie"]:
            alts[k] = composite_alternatives(frags, mode, t_eps, t_product, bg)
    return rgb, T, tie, wsum


def render_image(scene, cam_index=0, mode=FULL, t_eps=T_EPS, t_product=False,
                 bg=(0.0, 0.0, 0.0), cov3d=None, frame=None, soft=None, window=None):
    """Full image by primitive-major gather: every (primitive, pixel-in-rect)
    pair is evaluated, pairs are grouped per pixel, ordered by (depth bits,
    id) and composited.  Returns dict rgb [H,W,3], T [H,W], tie [H,W],
    wsum [H,W], nfrag [H,W], depth [H,W] (expected depth, +inf where nothing
    blends), alts (for every tie pixel, by flat index y*W + x, its
    composite_alternatives [n_alt, 4]).  soft: soft-edge width sigma in pixels (FULL mode only).
    window: (x0, x1, y0, y1), inclusive: only the pixels of that rectangle are
    composited (the rect of every primitive is cut to it); the others keep
    the background and T = 1."""
    fr = frame or Frame(scene, cam_index, cov3d, soft)
    P = fr.P
    W, H = fr.cam.width, fr.cam.height
    ids = np.nonzero(P.valid)[0]
    r = P.rect[ids]
    if window is not None:
        x0, x1, y0, y1 = (int(v) for v in window)
        r = np.stack([np.maximum(r[:, 0], x0), np.minimum(r[:, 1], x1),
                      np.maximum(r[:, 2], y0), np.minimum(r[:, 3], y1)], 1)
        keep = (r[:, 0] <= r[:, 1]) & (r[:, 2] <= r[:, 3])
        ids, r = ids[keep], r[keep]
    w = r[:, 1] - r[:, 0] + 1
    h = r[:, 3] - r[:, 2] + 1
    cnt = w * h
    rep = np.repeat(np.arange(len(ids)), cnt)
    start = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)
    k = np.arange(int(cnt.sum()), dtype=np.int64) - start[rep]
    pid = ids[rep]
    pxs = r[rep, 0] + k % w[rep]
    pys = r[rep, 2] + k // w[rep]
    order = np.lexsort((pid, P.dbits[pid], pys * W + pxs))
    pid, pxs, pys = pid[order], pxs[order], pys[order]
    pix = pys * W + pxs
    out_rgb = np.zeros((H * W, 3))
    out_T = np.ones(H * W)
    out_tie = np.zeros(H * W, bool)
    out_ws = np.zeros(H * W)
    out_n = np.zeros(H * W, np.int64)
    out_d = np.full(H * W, np.inf)
    sig = []
    alts = {}
    bgv = np.asarray(bg, np.float64)
    out_rgb[:] = bgv
    bounds = np.nonzero(np.diff(np.concatenate([[-1], pix, [-2]])))[0]
    for s, e in zip(bounds[:-1], bounds[1:]):
        p = int(pix[s])
        frags = fr.fragments_at(p % W, p // W, candidates=pid[s:e])
        res = composite(frags, mode, t_eps, t_product, bg)
        out_rgb[p] = res["color"]
        out_T[p] = res["T"]
        out_tie[p] = res["tie"]
        if res["tie"]:
            alts[p] = composite_alternatives(frags, mode, t_eps, t_product, bg)
        out_ws[p] = sum(x for _, x in res["weights"])
        out_n[p] = len(frags)
        out_d[p] = res["depth"]
        sig.append((p, res["n"], tuple(i for i, _ in res["weights"]),
                    tuple(f.get("mask", -1) for f in frags[:res["n"]])))
    return dict(rgb=out_rgb.reshape(H, W, 3), T=out_T.reshape(H, W), tie=out_tie.reshape(H, W),
                wsum=out_ws.reshape(H, W), nfrag=out_n.reshape(H, W), depth=out_d.reshape(H, W),
                sig=hash(tuple(sig)), alts=alts)


def evaluation_count(scene, cam_index=0, mode=FULL, t_eps=T_EPS, frame=None):
    """Algorithmic work of the compositor: for every pixel, the number of
    entries of its depth-ordered candidate list (Gaussians whose pixel rect
    holds the pixel, triangles whose pixel rect holds it) up to and including
    the fragment after which T < t_eps (all of them when it never drops).
    Returns (total, per-pixel counts [H,W])."""
    fr = frame or Frame(scene, cam_index)
    P = fr.P
    W, H = fr.cam.width, fr.cam.height
    counts = np.zeros((H, W), np.int64)
    r = P.rect
    for y in range(H):
        for x in range(W):
            cand = np.nonzero(P.valid & (r[:, 0] <= x) & (r[:, 1] >= x) & (r[:, 2] <= y) & (r[:, 3] >= y))[0]
            if len(cand) == 0:
                continue
            order = np.lexsort((cand, P.dbits[cand]))
            cand = cand[order]
            frags = {f["id"]: f for f in fr.fragments_at(x, y, candidates=cand)}
            res = composite([frags[i] for i in cand if i in frags], mode, t_eps)
            # position (in the candidate list) of the last consumed fragment
            consumed = [f for f in cand if f in frags][:res["n"]]
            if res["T"] < t_eps and consumed:
                counts[y, x] = int(np.nonzero(cand == consumed[-1])[0][0]) + 1
            else:
                counts[y, x] = len(cand)
    return int(counts.sum()), counts
