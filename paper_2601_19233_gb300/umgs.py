"""Thin Python binding of libumgs (ctypes).  Argument marshalling only: every
step of rendering, binding and deformation runs in the CUDA library.

PyTorch provides device memory and the current CUDA stream; tensors are
passed as raw device pointers.  If the library is missing the import of the
entry points raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libumgs.so")

OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CAPACITY", 4: "CUDA", 5: "TIMEOUT",
          6: "NOT_IMPLEMENTED"}
BLEND_FULL, BLEND_DIRECT, BLEND_MSAA_ALL, BLEND_ENTITY_ALL = 0, 1, 2, 3
F32, BF16 = 0, 1
BIND_BBX, BIND_CENTER, BIND_NEAREST = 0, 1, 2
RENDER_SAVE_BACKWARD = 1
RENDER_MIXED = 2
RENDER_T_PRODUCT = 4
RENDER_ASYNC = 8
RENDER_DEPTH = 16
RENDER_SOFT_EDGE = 32
DEFORM_FRAME, DEFORM_LITERAL, DEFORM_ONE_RING = 0, 1, 16


class UmgsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("umgs %s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class CGaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("quats", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("cov3d", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("sh_dtype", ctypes.c_int32)]


class CMesh(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("faces", ctypes.c_void_p), ("vcolor", ctypes.c_void_p),
                ("valpha", ctypes.c_void_p), ("falpha", ctypes.c_void_p), ("nv", ctypes.c_int64),
                ("nf", ctypes.c_int64), ("uv", ctypes.c_void_p), ("texture", ctypes.c_void_p),
                ("tex_w", ctypes.c_int32), ("tex_h", ctypes.c_int32)]


class CCamera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_z", ctypes.c_float)]


class CGaussianGrads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("quats", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("cov3d", ctypes.c_void_p)]


class CMeshGrads(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("vcolor", ctypes.c_void_p), ("valpha", ctypes.c_void_p),
                ("falpha", ctypes.c_void_p)]


class CFrameStats(ctypes.Structure):
    _fields_ = [("gaussian_evals", ctypes.c_int64), ("triangle_evals", ctypes.c_int64),
                ("fp64_conics", ctypes.c_int64), ("list_entries", ctypes.c_int64)]


class CRenderOpts(ctypes.Structure):
    _fields_ = [("tile_size", ctypes.c_int32), ("blend_mode", ctypes.c_int32), ("t_eps", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("flags", ctypes.c_int32), ("sched", ctypes.c_int32),
                ("edge_sigma", ctypes.c_float), ("split", ctypes.c_int32)]


_lib = None


def lib():
    """Load libumgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libumgs.so not found at %s: run __graft_entry__.build() "
                               "(there is no CPU fallback)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.umgs_ctx_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
        L.umgs_ctx_destroy.argtypes = [vp]
        L.umgs_last_error.argtypes = [vp]
        L.umgs_last_error.restype = ctypes.c_char_p
        L.umgs_default_render_opts.argtypes = [ctypes.POINTER(CRenderOpts)]
        L.umgs_frame_create.argtypes = [vp, ctypes.POINTER(vp)]
        L.umgs_frame_destroy.argtypes = [vp]
        L.umgs_render.argtypes = [vp, ctypes.POINTER(CGaussians), ctypes.POINTER(CMesh), i32,
                                  ctypes.POINTER(CCamera), i32, ctypes.POINTER(CRenderOpts), vp, vp, vp]
        L.umgs_frame_counts.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.umgs_frame_lists.argtypes = [vp, vp, vp, vp, vp]
        L.umgs_frame_evaluations.argtypes = [vp, ctypes.POINTER(i64), vp]
        L.umgs_frame_evaluations.restype = ctypes.c_int
        L.umgs_frame_stats_read.argtypes = [vp, ctypes.POINTER(CFrameStats), vp]
        L.umgs_frame_stats_read.restype = ctypes.c_int
        L.umgs_deform_fp64_faces.argtypes = [vp, ctypes.POINTER(i64), vp]
        L.umgs_deform_fp64_faces.restype = ctypes.c_int
        L.umgs_ctx_sync.argtypes = [vp, vp]
        L.umgs_deform.argtypes = [vp, ctypes.POINTER(CGaussians), vp, vp, vp, vp, vp, i64, i64, i32, vp, vp, vp, vp]
        L.umgs_deform_vertex_table.argtypes = [vp, vp, i64, vp]
        L.umgs_bind.argtypes = [vp, ctypes.POINTER(CGaussians), vp, vp, i64, i64, ctypes.POINTER(CCamera), i32, i32,
                                ctypes.c_float, vp, vp, vp, vp, ctypes.POINTER(i64), vp]
        L.umgs_bind.restype = ctypes.c_int
        L.umgs_render_backward.argtypes = [vp, vp, ctypes.POINTER(CGaussians), ctypes.POINTER(CMesh), i32, vp,
                                           ctypes.POINTER(CGaussianGrads), ctypes.POINTER(CMeshGrads), vp]
        L.umgs_render_backward.restype = ctypes.c_int
        L.umgs_deform_noalloc.argtypes = [ctypes.POINTER(CGaussians), vp, vp, vp, vp, vp, i64, i64, i32, vp, vp,
                                          vp, vp]
        L.umgs_deform_noalloc.restype = ctypes.c_int
        L.umgs_render_graph_create.argtypes = [vp, vp, ctypes.POINTER(CGaussians), ctypes.POINTER(CMesh), i32,
                                               ctypes.POINTER(CCamera), i32, ctypes.POINTER(CRenderOpts), vp,
                                               ctypes.c_float, ctypes.POINTER(vp), vp]
        L.umgs_graph_launch.argtypes = [vp, vp]
        L.umgs_graph_check.argtypes = [vp, vp]
        L.umgs_graph_destroy.argtypes = [vp]
        L.umgs_autotune.argtypes = [vp, ctypes.POINTER(CGaussians), ctypes.POINTER(CMesh), i32,
                                    ctypes.POINTER(CCamera), i32, ctypes.POINTER(CRenderOpts), vp,
                                    ctypes.POINTER(ctypes.c_double), vp]
        for name in ("umgs_render_graph_create", "umgs_graph_launch", "umgs_graph_check", "umgs_autotune"):
            getattr(L, name).restype = ctypes.c_int
        L.umgs_profile_enable.argtypes = [vp, i32]
        L.umgs_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        L.umgs_binding_compact.argtypes = [vp, vp, vp, i64, vp, i64, i64, vp, vp, vp]
        L.umgs_binding_compact.restype = ctypes.c_int
        L.umgs_deform_compact.argtypes = [vp, ctypes.POINTER(CGaussians), vp, vp, vp, vp, vp, i64, i64, i32, vp, vp,
                                          vp, vp]
        L.umgs_deform_compact.restype = ctypes.c_int
        L.umgs_binding_csr.argtypes = [vp, vp, vp, i64, vp, i64, i64, vp, vp, i64, ctypes.POINTER(i64), vp]
        L.umgs_binding_csr.restype = ctypes.c_int
        L.umgs_deform_csr.argtypes = [vp, ctypes.POINTER(CGaussians), vp, vp, vp, vp, vp, i64, i64, i32, vp, vp,
                                      vp, vp]
        L.umgs_deform_csr.restype = ctypes.c_int
        L.umgs_spatial_order.argtypes = [vp, vp, i64, vp, vp]
        L.umgs_spatial_order.restype = ctypes.c_int
        L.umgs_frame_reserve.argtypes = [vp, i64]
        L.umgs_frame_reserve.restype = ctypes.c_int
        L.umgs_frame_check.argtypes = [vp, vp]
        L.umgs_frame_check.restype = ctypes.c_int
        L.umgs_frame_depth.argtypes = [vp, vp, vp]
        L.umgs_frame_depth.restype = ctypes.c_int
        L.umgs_composite_layers.argtypes = [vp, vp, vp, vp, vp, i64, ctypes.POINTER(ctypes.c_float), vp, vp]
        L.umgs_composite_layers.restype = ctypes.c_int
        L.umgs_kernel_launches.argtypes = []
        L.umgs_kernel_launches.restype = ctypes.c_longlong
        for name in ("umgs_profile_enable", "umgs_profile_read", "umgs_ctx_create", "umgs_frame_create", "umgs_render", "umgs_frame_counts",
                     "umgs_frame_lists", "umgs_ctx_sync", "umgs_deform", "umgs_deform_vertex_table"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "tensor must be a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A libumgs context on one device (owns workspace)."""

    def __init__(self, device=0):
        self._h = ctypes.c_void_p()
        self.device = device
        st = lib().umgs_ctx_create(ctypes.byref(self._h), int(device))
        if st != OK:
            raise UmgsError(st, "umgs_ctx_create(device=%d)" % device)

    def check(self, st, what):
        if st != OK:
            msg = lib().umgs_last_error(self._h)
            raise UmgsError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def sync(self, stream=None):
        """umgs_ctx_sync: synchronise and raise deferred device-side errors."""
        self.check(lib().umgs_ctx_sync(self._h, _stream(stream)), "umgs_ctx_sync")

    def close(self):
        if self._h:
            lib().umgs_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Frame:
    """Saved state of one render (sorted lists, records, per-pixel state)."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        self._h = ctypes.c_void_p()
        ctx.check(lib().umgs_frame_create(ctx._h, ctypes.byref(self._h)), "umgs_frame_create")

    def counts(self):
        k, t = ctypes.c_int64(), ctypes.c_int64()
        self.ctx.check(lib().umgs_frame_counts(self._h, ctypes.byref(k), ctypes.byref(t)), "umgs_frame_counts")
        return k.value, t.value

    def reserve(self, key_capacity: int):
        """umgs_frame_reserve: pair capacity of asynchronous renders into this frame."""
        self.ctx.check(lib().umgs_frame_reserve(self._h, ctypes.c_int64(int(key_capacity))), "umgs_frame_reserve")

    def check(self, stream=None):
        """umgs_frame_check: raises on a pair-capacity overflow or bad face index of an asynchronous render."""
        self.ctx.check(lib().umgs_frame_check(self._h, _stream(stream)), "umgs_frame_check")

    def evaluations(self):
        """(pixel, fragment) evaluations of the last render (synchronises)."""
        v = ctypes.c_int64()
        self.ctx.check(lib().umgs_frame_evaluations(self._h, ctypes.byref(v), _stream()), "umgs_frame_evaluations")
        return v.value

    def stats(self):
        """umgs_frame_stats_read: dict of gaussian_evals, triangle_evals, fp64_conics, list_entries (synchronises)."""
        st = CFrameStats()
        self.ctx.check(lib().umgs_frame_stats_read(self._h, ctypes.byref(st), _stream()), "umgs_frame_stats_read")
        return {f: int(getattr(st, f)) for f, _ in CFrameStats._fields_}

    def lists(self):
        """(tile_ptr int64 [T+1], ids int32 [K], dbits int32 [K] (uint32 bits)) on the device."""
        k, t = self.counts()
        dev = torch.device("cuda", self.ctx.device)
        ptr = torch.empty(t + 1, dtype=torch.int64, device=dev)
        ids = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
        db = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
        self.ctx.check(lib().umgs_frame_lists(self._h, _ptr(ptr), _ptr(ids), _ptr(db), _stream()),
                       "umgs_frame_lists")
        return ptr, ids[:k], db[:k]

    def depth(self, ncams, height, width):
        """umgs_frame_depth: expected depth [ncams, H, W] float32 on the device (+inf where nothing blends)."""
        out = torch.empty((ncams, height, width), dtype=torch.float32, device=torch.device("cuda", self.ctx.device))
        self.ctx.check(lib().umgs_frame_depth(self._h, _ptr(out), _stream()), "umgs_frame_depth")
        return out

    def __del__(self):
        try:
            if self._h:
                lib().umgs_frame_destroy(self._h)
        except Exception:
            pass


# ----------------------------------------------------------------------------
# device-side scene containers (plain tensors)

@dataclass
class DevGaussians:
    means: torch.Tensor
    quats: torch.Tensor
    scales: torch.Tensor
    opacities: torch.Tensor
    sh: torch.Tensor
    sh_degree: int
    cov3d: torch.Tensor | None = None

    @property
    def n(self):
        return int(self.means.shape[0])

    def c(self):
        dtype = BF16 if self.sh.dtype == torch.bfloat16 else F32
        return CGaussians(_ptr(self.means), _ptr(self.quats), _ptr(self.scales), _ptr(self.opacities),
                          _ptr(self.sh), _ptr(self.cov3d), self.n, int(self.sh_degree), dtype)


@dataclass
class DevMesh:
    verts: torch.Tensor
    faces: torch.Tensor
    vcolor: torch.Tensor
    valpha: torch.Tensor | None = None
    falpha: torch.Tensor | None = None
    uv: torch.Tensor | None = None       # [nv,2] texture coordinates
    texture: torch.Tensor | None = None  # [TH,TW,3] RGB

    def c(self):
        th, tw = (int(self.texture.shape[0]), int(self.texture.shape[1])) if self.texture is not None else (0, 0)
        return CMesh(_ptr(self.verts), _ptr(self.faces), _ptr(self.vcolor), _ptr(self.valpha), _ptr(self.falpha),
                     int(self.verts.shape[0]), int(self.faces.shape[0]), _ptr(self.uv), _ptr(self.texture), tw, th)


def camera_struct(cam) -> CCamera:
    c = CCamera()
    vm = np.asarray(cam.viewmat, np.float32).reshape(12)
    for k in range(12):
        c.viewmat[k] = float(vm[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.near_z = int(cam.width), int(cam.height), float(cam.near)
    return c


def _t(a, device, dtype=None):
    if a is None:
        return None
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device).contiguous()


def gaussians_to_device(g, device="cuda", sh_dtype=torch.float32) -> DevGaussians:
    return DevGaussians(_t(g.means, device), _t(g.quats, device), _t(g.scales, device), _t(g.opacities, device),
                        _t(g.sh, device, sh_dtype), g.sh_degree)


def mesh_to_device(m, device="cuda") -> DevMesh:
    return DevMesh(_t(m.verts, device), _t(m.faces.astype(np.int32), device), _t(m.vcolor, device),
                   _t(m.valpha, device), _t(m.falpha, device), _t(getattr(m, "uv", None), device),
                   _t(getattr(m, "texture", None), device))


def render_opts(tile_size=16, blend_mode=BLEND_FULL, t_eps=1e-4, bg=(0.0, 0.0, 0.0), save=False,
                mixed=False, sched=0, t_product=False, asynchronous=False, depth=False,
                edge_sigma=None, split=0) -> CRenderOpts:
    """edge_sigma: soft-edge triangle coverage of that width in pixels
    (UMGS_RENDER_SOFT_EDGE), or None for the binary sample coverage.
    split: per-tile work split (segments of that many records), 0 = off."""
    o = CRenderOpts()
    lib().umgs_default_render_opts(ctypes.byref(o))
    o.sched = int(sched)
    o.split = int(split)
    o.flags = ((RENDER_SAVE_BACKWARD if save else 0) | (RENDER_MIXED if mixed else 0)
               | (RENDER_T_PRODUCT if t_product else 0) | (RENDER_ASYNC if asynchronous else 0)
               | (RENDER_DEPTH if depth else 0) | (RENDER_SOFT_EDGE if edge_sigma else 0))
    o.edge_sigma = float(edge_sigma or 0.0)
    o.tile_size = int(tile_size)
    o.blend_mode = int(blend_mode)
    o.t_eps = float(t_eps)
    for k in range(3):
        o.bg[k] = float(bg[k])
    return o


def render(ctx: Context, gaussians: DevGaussians | None, meshes, cameras, opts: CRenderOpts | None = None,
           out: torch.Tensor | None = None, frame: Frame | None = None, stream=None) -> torch.Tensor:
    """umgs_render: returns [ncams, H, W, 4] float32 (RGB, T) on the device."""
    cams = (CCamera * len(cameras))(*[camera_struct(c) for c in cameras])
    H, W = int(cameras[0].height), int(cameras[0].width)
    dev = torch.device("cuda", ctx.device)
    if out is None:
        out = torch.empty((len(cameras), H, W, 4), dtype=torch.float32, device=dev)
    cm = (CMesh * max(1, len(meshes)))(*[m.c() for m in meshes]) if meshes else None
    cg = gaussians.c() if gaussians is not None else None
    st = lib().umgs_render(ctx._h, ctypes.byref(cg) if cg is not None else None, cm, len(meshes), cams,
                           len(cameras), ctypes.byref(opts) if opts is not None else None, _ptr(out),
                           frame._h if frame is not None else None, _stream(stream))
    ctx.check(st, "umgs_render")
    return out


def deform(ctx: Context, rest: DevGaussians, face: torch.Tensor, bary: torch.Tensor, proxy_v: torch.Tensor,
           proxy_vd: torch.Tensor, proxy_f: torch.Tensor, mode=DEFORM_FRAME, out=None, with_quats=True,
           stream=None):
    """umgs_deform: returns (means' [n,3], cov3d' [n,6], quats' [n,4] or None)."""
    n = rest.n
    dev = torch.device("cuda", ctx.device)
    if out is None:
        out = (torch.empty((n, 3), dtype=torch.float32, device=dev),
               torch.empty((n, 6), dtype=torch.float32, device=dev),
               torch.empty((n, 4), dtype=torch.float32, device=dev) if with_quats else None)
    cg = rest.c()
    st = lib().umgs_deform(ctx._h, ctypes.byref(cg), _ptr(face), _ptr(bary), _ptr(proxy_v), _ptr(proxy_vd),
                           _ptr(proxy_f), int(proxy_v.shape[0]), int(proxy_f.shape[0]), int(mode), _ptr(out[0]),
                           _ptr(out[1]), _ptr(out[2]), _stream(stream))
    ctx.check(st, "umgs_deform")
    return out


def binding_compact(ctx: Context, face: torch.Tensor, bary: torch.Tensor, proxy_f: torch.Tensor, nv: int,
                    stream=None):
    """umgs_binding_compact: (count int32 [n], entries int32 [n,24,2]) on the device."""
    n = int(face.shape[0])
    dev = torch.device("cuda", ctx.device)
    count = torch.empty((n,), dtype=torch.int32, device=dev)
    entries = torch.empty((n, 24, 2), dtype=torch.int32, device=dev)
    ctx.check(lib().umgs_binding_compact(ctx._h, _ptr(face), _ptr(bary), n, _ptr(proxy_f), int(nv),
                                         int(proxy_f.shape[0]), _ptr(count), _ptr(entries), _stream(stream)),
              "umgs_binding_compact")
    return count, entries


def deform_compact(ctx: Context, rest: DevGaussians, count: torch.Tensor, entries: torch.Tensor,
                   proxy_v: torch.Tensor, proxy_vd: torch.Tensor, proxy_f: torch.Tensor, mode=DEFORM_FRAME,
                   out=None, with_quats=True, stream=None):
    """umgs_deform_compact: umgs_deform over a compact binding; returns (means', cov3d', quats' or None)."""
    n = rest.n
    dev = torch.device("cuda", ctx.device)
    if out is None:
        out = (torch.empty((n, 3), dtype=torch.float32, device=dev),
               torch.empty((n, 6), dtype=torch.float32, device=dev),
               torch.empty((n, 4), dtype=torch.float32, device=dev) if with_quats else None)
    cg = rest.c()
    st = lib().umgs_deform_compact(ctx._h, ctypes.byref(cg), _ptr(count), _ptr(entries), _ptr(proxy_v),
                                   _ptr(proxy_vd), _ptr(proxy_f), int(proxy_v.shape[0]), int(proxy_f.shape[0]),
                                   int(mode), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _stream(stream))
    ctx.check(st, "umgs_deform_compact")
    return out


def binding_csr(ctx: Context, face: torch.Tensor, bary: torch.Tensor, proxy_f: torch.Tensor, nv: int, stream=None):
    """umgs_binding_csr: (offsets int32 [n+1], entries int32 [total,2]) on the device."""
    n = int(face.shape[0])
    dev = torch.device("cuda", ctx.device)
    offsets = torch.empty((n + 1,), dtype=torch.int32, device=dev)
    total = ctypes.c_int64(0)
    st = lib().umgs_binding_csr(ctx._h, _ptr(face), _ptr(bary), n, _ptr(proxy_f), int(nv), int(proxy_f.shape[0]),
                                _ptr(offsets), None, 0, ctypes.byref(total), _stream(stream))
    if st not in (OK, 3):  # CAPACITY: the size query
        ctx.check(st, "umgs_binding_csr")
    entries = torch.empty((max(1, total.value), 2), dtype=torch.int32, device=dev)
    ctx.check(lib().umgs_binding_csr(ctx._h, _ptr(face), _ptr(bary), n, _ptr(proxy_f), int(nv),
                                     int(proxy_f.shape[0]), _ptr(offsets), _ptr(entries), int(entries.shape[0]),
                                     ctypes.byref(total), _stream(stream)), "umgs_binding_csr")
    return offsets, entries


def spatial_order(ctx: Context, means: torch.Tensor, stream=None) -> torch.Tensor:
    """umgs_spatial_order: int32 [n] permutation (Morton order of the means)."""
    assert means.dtype == torch.float32 and means.dim() == 2 and means.shape[1] == 3, "means must be float32 [n,3]"
    n = int(means.shape[0])
    perm = torch.empty((n,), dtype=torch.int32, device=torch.device("cuda", ctx.device))
    ctx.check(lib().umgs_spatial_order(ctx._h, _ptr(means), n, _ptr(perm), _stream(stream)), "umgs_spatial_order")
    return perm


def deform_csr(ctx: Context, rest: DevGaussians, offsets: torch.Tensor, entries: torch.Tensor,
               proxy_v: torch.Tensor, proxy_vd: torch.Tensor, proxy_f: torch.Tensor, mode=DEFORM_FRAME,
               out=None, with_quats=True, stream=None):
    """umgs_deform_csr: umgs_deform over the CSR binding; returns (means', cov3d', quats' or None)."""
    n = rest.n
    dev = torch.device("cuda", ctx.device)
    if out is None:
        out = (torch.empty((n, 3), dtype=torch.float32, device=dev),
               torch.empty((n, 6), dtype=torch.float32, device=dev),
               torch.empty((n, 4), dtype=torch.float32, device=dev) if with_quats else None)
    cg = rest.c()
    st = lib().umgs_deform_csr(ctx._h, ctypes.byref(cg), _ptr(offsets), _ptr(entries), _ptr(proxy_v),
                               _ptr(proxy_vd), _ptr(proxy_f), int(proxy_v.shape[0]), int(proxy_f.shape[0]),
                               int(mode), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _stream(stream))
    ctx.check(st, "umgs_deform_csr")
    return out


NOALLOC_MAX_PROXY_VERTICES = 32768


def deform_noalloc(rest: DevGaussians, face, bary, proxy_v, proxy_vd, proxy_f, out, mode=DEFORM_FRAME,
                   stream=None):
    """umgs_deform_noalloc: the deformation for callers that cannot allocate
    device memory.  `out` = (means [n,3], cov3d [n,6], quats [n,4] or None),
    all preallocated by the caller; nothing is allocated on the device.
    Runs on the current device; see include/umgs.h for the shared-scratch rules.

    The C entry point cannot see the sizes of the buffers it is given, so the
    shapes, dtypes, devices and layouts are checked here (ValueError)."""
    n = rest.n
    dev = torch.device("cuda", torch.cuda.current_device())

    def need(t, shape, dtype, what):
        if t is None or tuple(t.shape) != shape or t.dtype != dtype or t.device != dev or not t.is_contiguous():
            got = "None" if t is None else "%s %s on %s%s" % (tuple(t.shape), t.dtype, t.device,
                                                               "" if t.is_contiguous() else " (not contiguous)")
            raise ValueError("deform_noalloc: %s must be a contiguous %s tensor of shape %s on %s, got %s"
                             % (what, dtype, shape, dev, got))

    nv, nf = int(proxy_v.shape[0]), int(proxy_f.shape[0])
    need(face, (n, 8), torch.int32, "face")
    need(bary, (n, 8, 2), torch.float32, "bary")
    need(proxy_v, (nv, 3), torch.float32, "proxy_v")
    need(proxy_vd, (nv, 3), torch.float32, "proxy_vd")
    need(proxy_f, (nf, 3), torch.int32, "proxy_f")
    if len(out) != 3:
        raise ValueError("deform_noalloc: out must be (means, cov3d, quats or None)")
    need(out[0], (n, 3), torch.float32, "out[0] (means)")
    need(out[1], (n, 6), torch.float32, "out[1] (cov3d)")
    if out[2] is not None:
        need(out[2], (n, 4), torch.float32, "out[2] (quats)")
    for name in ("means", "quats", "scales", "opacities"):
        t = getattr(rest, name)
        if t.device != dev:
            raise ValueError("deform_noalloc: rest.%s is on %s, not the current device %s" % (name, t.device, dev))
    cg = rest.c()
    st = lib().umgs_deform_noalloc(ctypes.byref(cg), _ptr(face), _ptr(bary), _ptr(proxy_v), _ptr(proxy_vd),
                                   _ptr(proxy_f), int(proxy_v.shape[0]), int(proxy_f.shape[0]), int(mode),
                                   _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _stream(stream))
    if st != OK:
        raise UmgsError(st, "umgs_deform_noalloc")
    return out


def deform_fp64_faces(ctx: Context, stream=None) -> int:
    """umgs_deform_fp64_faces: proxy faces of the last deformation inverted in fp64 (slivers)."""
    v = ctypes.c_int64()
    ctx.check(lib().umgs_deform_fp64_faces(ctx._h, ctypes.byref(v), _stream(stream)), "umgs_deform_fp64_faces")
    return int(v.value)


def deform_vertex_table(ctx: Context, nv: int, stream=None) -> torch.Tensor:
    t = torch.empty((nv, 12), dtype=torch.float32, device=torch.device("cuda", ctx.device))
    ctx.check(lib().umgs_deform_vertex_table(ctx._h, _ptr(t), int(nv), _stream(stream)), "umgs_deform_vertex_table")
    return t


NUM_STAGES = 16


def profile_enable(ctx: Context, on=True):
    ctx.check(lib().umgs_profile_enable(ctx._h, 1 if on else 0), "umgs_profile_enable")


def composite_layers(ctx: Context, a_rgbt, a_depth, b_rgbt, b_depth, bg=(0.0, 0.0, 0.0), out=None, stream=None):
    """umgs_composite_layers: separate-pass baseline, the nearer of two layers over the other, then bg."""
    if out is None:
        out = torch.empty_like(a_rgbt)
    npix = a_rgbt.numel() // 4
    assert a_depth.numel() == npix and b_depth.numel() == npix and b_rgbt.numel() == 4 * npix
    cbg = (ctypes.c_float * 3)(*[float(x) for x in bg])
    ctx.check(lib().umgs_composite_layers(ctx._h, _ptr(a_rgbt), _ptr(a_depth), _ptr(b_rgbt), _ptr(b_depth), npix,
                                          cbg, _ptr(out), _stream(stream)), "umgs_composite_layers")
    return out


def kernel_launches() -> int:
    """umgs_kernel_launches: kernels launched by the library in this process so far."""
    return int(lib().umgs_kernel_launches())


def profile_read(ctx: Context):
    """(ms [16], launches [16]) summed per stage since the last read."""
    ms = (ctypes.c_double * NUM_STAGES)()
    n = (ctypes.c_int64 * NUM_STAGES)()
    ctx.check(lib().umgs_profile_read(ctx._h, ms, n), "umgs_profile_read")
    return list(ms), list(n)


def bind(ctx: Context, g: DevGaussians, proxy_v: torch.Tensor, proxy_f: torch.Tensor, cameras, mode=BIND_BBX,
         k_sigma=3.0, stream=None):
    """umgs_bind: returns (face [n,8] i32, bary [n,8,2], dist [n,8], flags [n,8] u8, num_fallback)."""
    n = g.n
    dev = torch.device("cuda", ctx.device)
    face = torch.empty((n, 8), dtype=torch.int32, device=dev)
    bary = torch.empty((n, 8, 2), dtype=torch.float32, device=dev)
    dist = torch.empty((n, 8), dtype=torch.float32, device=dev)
    flags = torch.empty((n, 8), dtype=torch.uint8, device=dev)
    cams = (CCamera * max(1, len(cameras)))(*[camera_struct(c) for c in cameras])
    nfb = ctypes.c_int64(0)
    cg = g.c()
    st = lib().umgs_bind(ctx._h, ctypes.byref(cg), _ptr(proxy_v), _ptr(proxy_f), int(proxy_v.shape[0]),
                         int(proxy_f.shape[0]), cams, len(cameras), int(mode), float(k_sigma), _ptr(face), _ptr(bary),
                         _ptr(dist), _ptr(flags), ctypes.byref(nfb), _stream(stream))
    ctx.check(st, "umgs_bind")
    return face, bary, dist, flags, nfb.value


def render_backward(ctx: Context, frame: Frame, gaussians: DevGaussians | None, meshes, dL_drgbt: torch.Tensor,
                    stream=None):
    """umgs_render_backward: returns dict of gradient tensors (Gaussian and per-mesh)."""
    dev = torch.device("cuda", ctx.device)
    out = {}
    cg = None
    gg = CGaussianGrads()
    if gaussians is not None and gaussians.n > 0:
        n = gaussians.n
        out["means"] = torch.empty((n, 3), device=dev)
        out["opacities"] = torch.empty((n,), device=dev)
        out["sh"] = torch.empty(tuple(gaussians.sh.shape), device=dev, dtype=torch.float32)
        if gaussians.cov3d is not None:
            out["cov3d"] = torch.empty((n, 6), device=dev)
        else:
            out["quats"] = torch.empty((n, 4), device=dev)
            out["scales"] = torch.empty((n, 3), device=dev)
        gg = CGaussianGrads(_ptr(out["means"]), _ptr(out.get("quats")), _ptr(out.get("scales")),
                            _ptr(out["opacities"]), _ptr(out["sh"]), _ptr(out.get("cov3d")))
        cg = gaussians.c()
    mgs = []
    for mi, m in enumerate(meshes):
        out["verts%d" % mi] = torch.empty_like(m.verts)
        out["vcolor%d" % mi] = torch.empty_like(m.vcolor)
        fa = va = None
        if m.falpha is not None:
            fa = out["falpha%d" % mi] = torch.empty_like(m.falpha)
        elif m.valpha is not None:
            va = out["valpha%d" % mi] = torch.empty_like(m.valpha)
        mgs.append(CMeshGrads(_ptr(out["verts%d" % mi]), _ptr(out["vcolor%d" % mi]), _ptr(va), _ptr(fa)))
    cm = (CMesh * max(1, len(meshes)))(*[m.c() for m in meshes]) if meshes else None
    cmg = (CMeshGrads * max(1, len(mgs)))(*mgs) if mgs else None
    st = lib().umgs_render_backward(ctx._h, frame._h, ctypes.byref(cg) if cg is not None else None, cm, len(meshes),
                                    _ptr(dL_drgbt.contiguous()), ctypes.byref(gg), cmg, _stream(stream))
    ctx.check(st, "umgs_render_backward")
    return out


class _RenderFunction(torch.autograd.Function):
    """umgs_render (saved state) forward, umgs_render_backward backward.
    Differentiable inputs: the Gaussian tensors (means, quats, scales,
    opacities, SH, cov3d) and per mesh (verts, vcolor, valpha, falpha)."""

    @staticmethod
    def forward(fctx, ctx, frame, cameras, opts, gaussians, meshes, *tensors):
        out = render(ctx, gaussians, meshes, cameras, opts, frame=frame)
        fctx.state = (ctx, frame, gaussians, meshes)
        fctx.dtypes = [t.dtype if t is not None else None for t in tensors]
        return out

    @staticmethod
    def backward(fctx, dout):
        ctx, frame, g, meshes = fctx.state
        grads = render_backward(ctx, frame, g, meshes, dout.contiguous())
        names = ["means", "quats", "scales", "opacities", "sh", "cov3d"]
        for mi in range(len(meshes)):
            names += ["verts%d" % mi, "vcolor%d" % mi, "valpha%d" % mi, "falpha%d" % mi]
        out = []
        for name, dt in zip(names, fctx.dtypes):
            gr = grads.get(name)
            out.append(gr.to(dt) if (gr is not None and dt is not None) else None)
        return (None,) * 6 + tuple(out)


def render_autograd(ctx: Context, gaussians: DevGaussians | None, meshes, cameras, opts: CRenderOpts | None = None,
                    frame: Frame | None = None) -> torch.Tensor:
    """Differentiable render: [ncams, H, W, 4] (RGB, T) whose backward runs
    umgs_render_backward.  Each call keeps its state in its own Frame (pass
    one to reuse its buffers; it must not be re-rendered before backward).
    FULL blending, fp32 records only (the backward's scope)."""
    o = CRenderOpts()
    if opts is None:
        o = render_opts(16, save=True)
    else:
        ctypes.memmove(ctypes.byref(o), ctypes.byref(opts), ctypes.sizeof(CRenderOpts))
        o.flags |= RENDER_SAVE_BACKWARD
    frame = frame or Frame(ctx)
    g = gaussians
    ts = [g.means, g.quats, g.scales, g.opacities, g.sh, g.cov3d] if g is not None else [None] * 6
    for m in meshes:
        ts += [m.verts, m.vcolor, m.valpha, m.falpha]
    return _RenderFunction.apply(ctx, frame, cameras, o, gaussians, meshes, *ts)


class Graph:
    """umgs_render_graph_*: a render captured in a CUDA graph (see include/umgs.h)."""

    def __init__(self, ctx: Context, frame: Frame, gaussians, meshes, cameras, opts, out, key_headroom=1.25,
                 stream=None):
        self.ctx, self.frame, self.out = ctx, frame, out
        self._keep = (gaussians, meshes)
        self._cams = (CCamera * len(cameras))(*[camera_struct(c) for c in cameras])
        self._cm = (CMesh * max(1, len(meshes)))(*[m.c() for m in meshes]) if meshes else None
        self._cg = gaussians.c() if gaussians is not None else None
        self._opts = opts
        self._h = ctypes.c_void_p()
        st = lib().umgs_render_graph_create(ctx._h, frame._h, ctypes.byref(self._cg) if self._cg else None, self._cm,
                                            len(meshes), self._cams, len(cameras), ctypes.byref(opts), _ptr(out),
                                            float(key_headroom), ctypes.byref(self._h), _stream(stream))
        ctx.check(st, "umgs_render_graph_create")

    def launch(self, stream=None):
        self.ctx.check(lib().umgs_graph_launch(self._h, _stream(stream)), "umgs_graph_launch")

    def check(self, stream=None):
        self.ctx.check(lib().umgs_graph_check(self._h, _stream(stream)), "umgs_graph_check")

    def __del__(self):
        try:
            if self._h:
                lib().umgs_graph_destroy(self._h)
        except Exception:
            pass


def autotune(ctx: Context, gaussians, meshes, cameras, opts: CRenderOpts, out, stream=None):
    """umgs_autotune: returns (best opts, ms per render)."""
    cams = (CCamera * len(cameras))(*[camera_struct(c) for c in cameras])
    cm = (CMesh * max(1, len(meshes)))(*[m.c() for m in meshes]) if meshes else None
    cg = gaussians.c() if gaussians is not None else None
    o = CRenderOpts()
    ctypes.memmove(ctypes.byref(o), ctypes.byref(opts), ctypes.sizeof(CRenderOpts))
    ms = ctypes.c_double()
    st = lib().umgs_autotune(ctx._h, ctypes.byref(cg) if cg else None, cm, len(meshes), cams, len(cameras),
                             ctypes.byref(o), _ptr(out), ctypes.byref(ms), _stream(stream))
    ctx.check(st, "umgs_autotune")
    return o, ms.value
