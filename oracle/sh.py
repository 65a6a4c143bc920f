"""Real spherical harmonics from their general definition (test infrastructure only).

The paper renders Gaussians with the 3DGS colour model (Sec. 3.2 builds on
the 3DGS rasterizer): view-dependent colour is a degree-<=3 real spherical
harmonic expansion evaluated at the unit direction from the camera centre to
the Gaussian mean, plus 0.5, clamped below at 0.

Basis: Y_l^m for l = 0..deg, m = -l..l, flat index l*l + (m + l), with the
Condon-Shortley phase included in the associated Legendre functions
(scipy.special.lpmv carries it):
    Y_l^0  = K_l^0 P_l^0(cos t)
    Y_l^m  = sqrt(2) K_l^m cos(m p) P_l^m(cos t)        m > 0
    Y_l^-m = sqrt(2) K_l^m sin(m p) P_l^m(cos t)        m > 0
    K_l^m  = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!)
This is the basis of the 3DGS colour model (e.g. Y_1^{-1} = -c*y,
Y_1^0 = c*z, Y_1^1 = -c*x with c = sqrt(3/(4 pi))).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import lpmv


def sh_basis(dirs: np.ndarray, degree: int) -> np.ndarray:
    """fp64 [N, (degree+1)^2] basis values at unit directions dirs [N,3]."""
    d = np.asarray(dirs, np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    ct = np.clip(d[:, 2], -1.0, 1.0)
    ph = np.arctan2(d[:, 1], d[:, 0])
    out = np.zeros((d.shape[0], (degree + 1) ** 2), np.float64)
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            P = lpmv(am, l, ct)
            if m == 0:
                y = K * P
            elif m > 0:
                y = math.sqrt(2.0) * K * np.cos(am * ph) * P
            else:
                y = math.sqrt(2.0) * K * np.sin(am * ph) * P
            out[:, l * l + (m + l)] = y
    return out


def sh_to_rgb(sh: np.ndarray, dirs: np.ndarray, degree: int) -> np.ndarray:
    """max(0, sum_k sh[n,k,:] Y_k(dir_n) + 0.5), fp64 [N,3]."""
    K = (degree + 1) ** 2
    Y = sh_basis(dirs, degree)
    c = np.einsum("nk,nkc->nc", Y, np.asarray(sh, np.float64)[:, :K, :])
    return np.maximum(c + 0.5, 0.0)
