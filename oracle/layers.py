"""Separate-pass baseline in fp64 (test infrastructure only).

Sec. 4.1 (Fig. 5b) compares the single pass against the separate-pass
scheme of earlier hybrid renderers: Gaussians and meshes are rasterised
apart and their images are composited pixel by pixel according to depth.
This module writes that scheme out: each layer is an oracle render with a
zero background and its expected depth (oracle.render.render_image), the
nearer layer goes over the farther one (the first layer on equal depths),
and the background is added behind both:

    C = C_f + T_f C_b + T_f T_b bg,   T = T_f T_b.
"""
from __future__ import annotations

import numpy as np


def separate_pass(a, b, bg=(0.0, 0.0, 0.0)):
    """a, b: dicts with rgb [H,W,3], T [H,W], depth [H,W] (layers rendered
    on a zero background).  Returns (rgb [H,W,3], T [H,W])."""
    a_front = ~(b["depth"] < a["depth"])
    f_rgb = np.where(a_front[..., None], a["rgb"], b["rgb"])
    k_rgb = np.where(a_front[..., None], b["rgb"], a["rgb"])
    f_T = np.where(a_front, a["T"], b["T"])
    k_T = np.where(a_front, b["T"], a["T"])
    T = f_T * k_T
    rgb = f_rgb + f_T[..., None] * k_rgb + T[..., None] * np.asarray(bg, np.float64)
    return rgb, T
