"""Pins of the oracle's real spherical harmonics."""
import math

import numpy as np

from oracle.sh import sh_basis, sh_to_rgb


def test_orthonormal_on_sphere():
    # Gauss-Legendre in cos(theta) x uniform phi integrates these polynomials exactly
    x, w = np.polynomial.legendre.leggauss(16)
    phi = np.arange(32) * 2 * np.pi / 32
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wt = (w[:, None] * np.full(32, 2 * np.pi / 32)[None, :]).reshape(-1)
    Y = sh_basis(d, 3)
    G = (Y * wt[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_low_order_closed_forms():
    rng = np.random.default_rng(0)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x, y, z = d.T
    Y = sh_basis(d, 2)
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y[:, 0], c0)
    assert np.allclose(Y[:, 1], -c1 * y)
    assert np.allclose(Y[:, 2], c1 * z)
    assert np.allclose(Y[:, 3], -c1 * x)
    k = 0.5 * math.sqrt(15 / math.pi)
    assert np.allclose(Y[:, 4], k * x * y)
    assert np.allclose(Y[:, 5], -k * y * z)
    assert np.allclose(Y[:, 6], 0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1))
    assert np.allclose(Y[:, 7], -k * x * z)
    assert np.allclose(Y[:, 8], 0.5 * k * (x * x - y * y))


def test_rgb_offset_and_clamp():
    d = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    sh = np.zeros((2, 1, 3))
    sh[0, 0] = [1.0, -5.0, 0.0]
    rgb = sh_to_rgb(sh, d, 0)
    c0 = 0.5 / math.sqrt(math.pi)
    assert np.allclose(rgb[0], [c0 + 0.5, 0.0, 0.5])
    assert np.allclose(rgb[1], [0.5, 0.5, 0.5])
