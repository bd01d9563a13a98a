"""Sphere grid, scalar and vector spherical harmonics -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Paper: Yan et al., arXiv 1909.06623.
  * Grid -- Sec. 5.4 and Sec. 6.5: (p+1) Gauss-Legendre rings in cos(theta) times
    a uniform grid in phi.  Reading: (p+1) x (2p+2) nodes, the count that gives
    the 486 traction unknowns per sphere quoted at p = 8 in Sec. 6.5 (3 x 162);
    Sec. 5.1 and 5.4 also print (p+1)(2p+1), which that count contradicts.
  * Y_n^m and P_n^m -- Sec. 4.2, written exactly as the paper defines them:
    orthonormal Y with the (-1)^m (Condon-Shortley) factor inside P_n^m, which
    is built here from its Rodrigues formula by exact polynomial
    differentiation (numpy.polynomial), and P_n^{-m} from the stated relation.
  * VSH -- Sec. 4.2, eq. rhoshexp: G = grad_Gamma Y, V = G - (n+1) Y e_r,
    W = G + n Y e_r, X = e_r x G; coefficients are <rho, conj(basis)> over the
    sphere, and the expansion divides them by |basis|^2.

Grid node order on each sphere: ring k (ascending cos(theta) = GL node t_k)
major, azimuth l minor: node = k * (2p+2) + l, phi_l = 2 pi l / (2p+2).
"""
from functools import lru_cache
from math import factorial, pi, sqrt

import numpy as np
from numpy.polynomial import Polynomial


# ----------------------------------------------------------------------------
# grid (Sec. 5.4)
# ----------------------------------------------------------------------------
def gauss_legendre(p):
    """(p+1) Gauss-Legendre nodes t_k (ascending) and weights on [-1, 1]."""
    t, w = np.polynomial.legendre.leggauss(p + 1)
    return t, w


def unit_grid(p):
    """Nodes of the unit sphere: theta, phi, unit normals (P x 3), weights.

    Weight of node (k, l) = w_k^GL * 2 pi / (2p+2); the weights sum to 4 pi.
    """
    t, wgl = gauss_legendre(p)
    nphi = 2 * p + 2
    phi1 = 2.0 * pi * np.arange(nphi) / nphi
    theta = np.repeat(np.arccos(t), nphi)
    phi = np.tile(phi1, p + 1)
    w = np.repeat(wgl, nphi) * (2.0 * pi / nphi)
    nrm = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi),
                    np.cos(theta)], axis=1)
    return theta, phi, nrm, w


def nodes_per_sphere(p):
    return (p + 1) * (2 * p + 2)


def sphere_nodes(centers, radii, p):
    """All surface nodes x = c + a n, normals n and weights a^2 w (Sec. 5.4)."""
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    radii = np.asarray(radii, dtype=np.float64).reshape(-1)
    _, _, nrm, w = unit_grid(p)
    X = centers[:, None, :] + radii[:, None, None] * nrm[None, :, :]
    Nr = np.broadcast_to(nrm[None], X.shape).copy()
    W = radii[:, None] ** 2 * w[None, :]
    return X.reshape(-1, 3), Nr.reshape(-1, 3), W.reshape(-1)


# ----------------------------------------------------------------------------
# P_n^m and Y_n^m (Sec. 4.2)
# ----------------------------------------------------------------------------
@lru_cache(maxsize=None)
def _rodrigues_Q(n, m):
    """Q_n^m(t) = d^{n+m}/dt^{n+m} (t^2 - 1)^n / (2^n n!), for 0 <= m <= n.

    With it, P_n^m(t) = (-1)^m (1 - t^2)^{m/2} Q_n^m(t): the paper's definition.
    """
    base = Polynomial([-1.0, 0.0, 1.0]) ** n
    return base.deriv(n + m) / (2.0 ** n * factorial(n))


@lru_cache(maxsize=None)
def _rodrigues_Q_derivs(n, m):
    Q = _rodrigues_Q(n, m)
    return Q, Q.deriv(1), Q.deriv(2)


def assoc_legendre(n, m, t):
    """P_n^m(t) for -n <= m <= n, Condon-Shortley phase included (Sec. 4.2)."""
    t = np.asarray(t, dtype=np.float64)
    if m < 0:
        mm = -m
        return ((-1) ** mm * factorial(n - mm) / factorial(n + mm)
                * assoc_legendre(n, mm, t))
    return (-1) ** m * (1.0 - t * t) ** (0.5 * m) * _rodrigues_Q(n, m)(t)


def norm_nm(n, m):
    """sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!)."""
    return sqrt((2 * n + 1) / (4.0 * pi) * factorial(n - m) / factorial(n + m))


_YCACHE = {}


def ylm_parts(n, m, theta, phi):
    """Memoised front end of _ylm_parts for small angle sets (grids reused by
    every operator application); the values are those of _ylm_parts."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    if theta.size > 4096:
        return _ylm_parts(n, m, theta, phi)
    key = (n, m, theta.tobytes(), phi.tobytes())
    hit = _YCACHE.get(key)
    if hit is None:
        if len(_YCACHE) > 200000:
            _YCACHE.clear()
        hit = _YCACHE[key] = _ylm_parts(n, m, theta, phi)
    return hit


def _ylm_parts(n, m, theta, phi):
    """Y_n^m and the angular pieces the VSH and their gradients need.

    Returns a dict of complex arrays:
      Y        Y_n^m(theta, phi)
      Yt       dY/dtheta
      Ytt      d^2Y/dtheta^2
      Ys       Y / sin(theta)                 (finite at the poles for m != 0)
      Yts      dY/dtheta / sin - cos Y / sin^2 (= d/dtheta (Y / sin))
    For m < 0 the relation Y_n^{-m} = (-1)^m conj(Y_n^m), which follows from the
    paper's P_n^{-m} relation, is applied to every piece (d/dtheta is real).
    """
    if m < 0:
        pos = _ylm_parts(n, -m, theta, phi)
        sgn = (-1) ** (-m)
        return {k: sgn * np.conj(v) for k, v in pos.items()}
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    s, t = np.sin(theta), np.cos(theta)
    Q, Q1, Q2 = _rodrigues_Q_derivs(n, m)
    q, q1, q2 = Q(t), Q1(t), Q2(t)
    c = norm_nm(n, m) * (-1) ** m
    E = np.exp(1j * m * phi)

    def spow(k):
        # s**k with the convention that a zero coefficient kills it (k may be < 0)
        return s ** k if k >= 0 else 1.0 / s ** (-k)

    Y = c * spow(m) * q * E
    Yt = c * ((m * spow(m - 1) * t * q if m >= 1 else 0.0) - spow(m + 1) * q1) * E
    Ytt = c * ((m * (m - 1) * spow(m - 2) * t * t * q if m >= 2 else 0.0)
               - m * spow(m) * q - (2 * m + 1) * spow(m) * t * q1
               + spow(m + 2) * q2) * E
    if m >= 1:
        # Y/s = c s^{m-1} q E;  d/dtheta (Y/s) = c [(m-1) s^{m-2} t q - s^m q'] E
        Ys = c * spow(m - 1) * q * E
        Yts = c * (((m - 1) * spow(m - 2) * t * q if m >= 2 else 0.0)
                   - spow(m) * q1) * E
    else:
        Ys = Y / s
        Yts = Yt / s - t * Y / (s * s)
    return {"Y": Y, "Yt": Yt, "Ytt": Ytt, "Ys": Ys, "Yts": Yts}


# ----------------------------------------------------------------------------
# VSH basis (Sec. 4.2, eq. rhoshexp)
# ----------------------------------------------------------------------------
def frame(theta, phi):
    """Cartesian components of e_r, e_theta, e_phi (each ... x 3)."""
    s, t = np.sin(theta), np.cos(theta)
    cp, sp = np.cos(phi), np.sin(phi)
    er = np.stack([s * cp, s * sp, t], axis=-1)
    et = np.stack([t * cp, t * sp, -s], axis=-1)
    ep = np.stack([-sp, cp, np.zeros_like(phi)], axis=-1)
    return er, et, ep


def vsh(n, m, theta, phi):
    """V_n^m, W_n^m, X_n^m on the unit sphere as complex Cartesian vectors.

    G = grad_Gamma Y = dY/dtheta e_theta + (1/sin) dY/dphi e_phi, with
    dY/dphi = i m Y; V = G - (n+1) Y e_r; W = G + n Y e_r; X = e_r x G.
    """
    yp = ylm_parts(n, m, theta, phi)
    er, et, ep = frame(theta, phi)
    Gt = yp["Yt"]
    Gp = 1j * m * yp["Ys"] if m != 0 else np.zeros_like(Gt)
    G = Gt[..., None] * et + Gp[..., None] * ep
    Yr = yp["Y"][..., None] * er
    V = G - (n + 1) * Yr
    W = G + n * Yr
    X = Gt[..., None] * ep - Gp[..., None] * et  # e_r x e_theta = e_phi, e_r x e_phi = -e_theta
    return V, W, X


def vsh_norm2(n):
    """|V|^2, |W|^2, |X|^2 on the unit sphere (derived from the orthonormal Y)."""
    return (n + 1) * (2 * n + 1), n * (2 * n + 1), n * (n + 1)


def modes(p):
    """All (n, m) with 0 <= n <= p, -n <= m <= n."""
    return [(n, m) for n in range(p + 1) for m in range(-n, n + 1)]


@lru_cache(maxsize=None)
def _grid_vsh(p):
    theta, phi, _, w = unit_grid(p)
    out = {}
    for n, m in modes(p):
        out[(n, m)] = vsh(n, m, theta, phi)
    return out


def analysis(sig, p):
    """VSH expansion coefficients of a vector field on one unit sphere's grid.

    sig: (P, 3) real grid values.  Returns a dict (n, m) -> (sV, sW, sX) with
    s = <sig, conj(basis)> / |basis|^2, the factors that multiply V, W, X in
    eq. rhoshexp.  The inner product is the grid quadrature (Sec. 5.4).
    """
    _, _, _, w = unit_grid(p)
    B = _grid_vsh(p)
    out = {}
    for (n, m), (V, W, X) in B.items():
        nv, nw, nx = vsh_norm2(n)
        hv = np.sum(w[:, None] * sig * np.conj(V))
        hw = np.sum(w[:, None] * sig * np.conj(W))
        hx = np.sum(w[:, None] * sig * np.conj(X))
        out[(n, m)] = (hv / nv, hw / nw if nw else 0.0, hx / nx if nx else 0.0)
    return out


def synthesis(coef, p, theta, phi):
    """Real vector field sum_{n,m} sV V + sW W + sX X at directions (theta, phi)."""
    theta = np.asarray(theta, dtype=np.float64)
    acc = np.zeros(theta.shape + (3,), dtype=np.complex128)
    for (n, m), (sv, sw, sx) in coef.items():
        V, W, X = vsh(n, m, theta, phi)
        acc += sv * V + sw * W + sx * X
    return acc.real


def grid_synthesis(coef, p):
    theta, phi, _, _ = unit_grid(p)
    return synthesis(coef, p, theta, phi)
