"""Pins of the oracle's grid and spherical harmonics (Sec. 4.2, 5.4).

Each check ties the oracle to something other than itself: exact quadrature of
polynomials, scipy's associated Legendre functions, orthonormality by
quadrature, the known VSH norms, and the fact that a uniform vector field is a
pure W_1 mode (grad of a linear function)."""
from math import factorial, pi

import numpy as np
import pytest
from scipy import special

from oracle import sph


@pytest.mark.parametrize("p", [4, 6, 8])
def test_grid_weights_and_polynomial_exactness(p):
    th, ph, nrm, w = sph.unit_grid(p)
    assert len(w) == (p + 1) * (2 * p + 2)
    assert abs(w.sum() - 4 * pi) < 1e-13
    # int over the unit sphere of x^a y^b z^c for a+b+c <= 2p+1 (exact values)
    def exact(a, b, c):
        if a % 2 or b % 2 or c % 2:
            return 0.0
        g = lambda k: special.gamma((k + 1) / 2)
        return 2 * g(a) * g(b) * g(c) / special.gamma((a + b + c + 3) / 2)
    x, y, z = nrm.T
    for a in range(0, 2 * p + 2, 3):
        for b in range(0, 2 * p + 2 - a, 2):
            for c in range(0, 2 * p + 2 - a - b, 3):
                got = np.sum(w * x ** a * y ** b * z ** c)
                assert abs(got - exact(a, b, c)) < 1e-13, (a, b, c)


def test_sphere_area_scales():
    X, N, W = sph.sphere_nodes([[1, 2, 3], [0, 0, 0]], [0.5, 2.0], 6)
    P = sph.nodes_per_sphere(6)
    assert abs(W[:P].sum() - 4 * pi * 0.25) < 1e-13
    assert abs(W[P:].sum() - 4 * pi * 4.0) < 1e-12
    assert np.allclose(np.linalg.norm(X[:P] - [1, 2, 3], axis=1), 0.5)


def test_legendre_matches_scipy():
    t = np.linspace(-0.99, 0.99, 17)
    for n in range(0, 11):
        for m in range(-n, n + 1):
            ref = special.lpmv(m, n, t)        # Condon-Shortley phase included
            got = sph.assoc_legendre(n, m, t)
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * factorial(n + abs(m))), (n, m)


def test_ylm_matches_scipy_and_derivatives():
    th = np.array([0.3, 1.1, 2.0, 2.9])
    ph = np.array([0.1, 2.0, -1.3, 4.0])
    h = 1e-6
    for n in range(0, 9):
        for m in range(-n, n + 1):
            y = sph.ylm_parts(n, m, th, ph)
            assert np.allclose(y["Y"], special.sph_harm_y(n, m, th, ph), atol=1e-14)
            yp = sph.ylm_parts(n, m, th + h, ph)
            ym = sph.ylm_parts(n, m, th - h, ph)
            assert np.allclose((yp["Y"] - ym["Y"]) / (2 * h), y["Yt"], atol=1e-8)
            assert np.allclose((yp["Yt"] - ym["Yt"]) / (2 * h), y["Ytt"], atol=1e-7)
            if m:
                assert np.allclose(y["Ys"] * np.sin(th), y["Y"], atol=1e-14)
                assert np.allclose((yp["Ys"] - ym["Ys"]) / (2 * h), y["Yts"], atol=1e-7)


@pytest.mark.parametrize("p", [4, 8])
def test_vsh_gram_is_diagonal_with_known_norms(p):
    th, ph, nrm, w = sph.unit_grid(p)
    rows, norms = [], []
    for n, m in sph.modes(p):
        V, W, X = sph.vsh(n, m, th, ph)
        for B, nn in zip((V, W, X), sph.vsh_norm2(n)):
            if n == 0 and nn == 0:
                assert np.abs(B).max() < 1e-14      # W_0^0 = X_0^0 = 0
                continue
            rows.append(B)
            norms.append(nn)
    B = np.array(rows)
    G = np.einsum("kpi,lpi,p->kl", B, np.conj(B), w)
    assert np.abs(G - np.diag(norms)).max() < 1e-12
    # the closed forms used for the norms
    for n in range(1, p + 1):
        assert sph.vsh_norm2(n) == ((n + 1) * (2 * n + 1), n * (2 * n + 1), n * (n + 1))


def test_analysis_synthesis_roundtrip_and_uniform_field():
    p = 6
    rng = np.random.default_rng(3)
    th, ph, nrm, w = sph.unit_grid(p)
    coef = sph.analysis(rng.standard_normal((len(w), 3)), p)
    band = sph.grid_synthesis(coef, p)
    coef2 = sph.analysis(band, p)
    for k in coef:
        assert np.allclose(coef[k], coef2[k], atol=1e-13)
    assert np.allclose(sph.grid_synthesis(coef2, p), band, atol=1e-13)
    # a uniform field is a pure W_1 mode (W_1 = grad of a linear function)
    ez = np.tile([0.0, 0.0, 1.0], (len(w), 1))
    c = sph.analysis(ez, p)
    for (n, m), (v, wv, x) in c.items():
        if (n, m) == (1, 0):
            assert abs(wv) > 0.1 and abs(v) < 1e-14 and abs(x) < 1e-14
        else:
            assert max(abs(v), abs(wv), abs(x)) < 1e-14
    assert np.allclose(sph.grid_synthesis(c, p), ez, atol=1e-14)
