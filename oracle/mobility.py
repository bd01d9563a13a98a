"""Mobility solve U = M F by the indirect boundary-integral formulation -- oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Yan et al., arXiv 1909.06623, Sec. 4.1.
  * rho_j(x) = F_j/|Gamma_j| + tau_j^{-1} T_j x (x - c_j).  Reading: tau_j is
    the tensor int (|y-c|^2 I - (y-c)(y-c)^T) dS = (8 pi/3) a^4 I for a sphere,
    the one that makes int (x-c) x rho dS = T (the paper calls it a "moment of
    inertia tensor" and cites it without a formula).
  * eq. rigidbodyrho: (I/2 + K + L)[zeta] = -(I/2 + K)[rho] on every surface,
    with L_j[z](x) = |Gamma_j|^{-1} int z + tau_j^{-1} (int (y-c_j) x z) x (x-c_j).
  * eq. velS: u = S[rho + zeta]; U_j, Omega_j by averaging u over Gamma_j:
    U_j = |Gamma_j|^{-1} int u,  Omega_j = tau_j^{-1} int (x - c_j) x u.
  * GMRES (Sec. 4.1, 5.1): the paper gives no variant.  Reading: unrestarted
    GMRES with modified Gram-Schmidt and Givens rotations, zero initial guess,
    stop when ||r|| / ||b|| < tol, zeta = 0 when b = 0.
  * Sign: rho = +F/|Gamma| with a positive mobility (U parallel to F for one
    sphere), pinned by the single-sphere drag U = F/(6 pi a), Omega = T/(8 pi a^3)
    quoted in Sec. 6.1.
"""
from math import pi

import numpy as np

from .layer import Suspension


def tau(a):
    """(8 pi / 3) a^4: the scalar of tau = tau I for a sphere of radius a."""
    return 8.0 * pi / 3.0 * a ** 4


def rho_from_FT(sus, FT):
    """rho on every node from per-sphere force/torque FT (N x 6)."""
    FT = np.asarray(FT, dtype=np.float64).reshape(sus.N, 6)
    F = FT[sus.sph_of, :3]
    T = FT[sus.sph_of, 3:]
    a = sus.a[sus.sph_of]
    rel = sus.X - sus.c[sus.sph_of]
    return F / (4 * pi * a ** 2)[:, None] + np.cross(T, rel) / tau(a)[:, None]


def sphere_moments(sus, z):
    """Per sphere: int z dS and int (y - c) x z dS by the grid quadrature."""
    rel = sus.X - sus.c[sus.sph_of]
    f = np.zeros((sus.N, 3))
    t = np.zeros((sus.N, 3))
    np.add.at(f, sus.sph_of, sus.W[:, None] * z)
    np.add.at(t, sus.sph_of, sus.W[:, None] * np.cross(rel, z))
    return f, t


def apply_L(sus, z):
    f, t = sphere_moments(sus, z)
    a = sus.a[sus.sph_of]
    rel = sus.X - sus.c[sus.sph_of]
    return (f[sus.sph_of] / (4 * pi * a ** 2)[:, None]
            + np.cross(t[sus.sph_of] / tau(a)[:, None], rel))


def apply_A(sus, z):
    """(I/2 + K + L)[z]: the left-hand side of eq. rigidbodyrho."""
    return 0.5 * z + sus.apply("K", z) + apply_L(sus, z)


def gmres(matvec, b, tol, maxit):
    """Unrestarted GMRES(MGS, Givens), x0 = 0.  Returns x, iterations, rel. res."""
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0
    n = b.size
    Q = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = nb
    Q[0] = b.ravel() / nb
    k = 0
    res = 1.0
    for k in range(1, maxit + 1):
        w = matvec(Q[k - 1].reshape(b.shape)).ravel()
        for j in range(k):
            H[j, k - 1] = Q[j] @ w
            w = w - H[j, k - 1] * Q[j]
        H[k, k - 1] = np.linalg.norm(w)
        if H[k, k - 1] > 0:
            Q[k] = w / H[k, k - 1]
        for j in range(k - 1):
            h0, h1 = H[j, k - 1], H[j + 1, k - 1]
            H[j, k - 1] = cs[j] * h0 + sn[j] * h1
            H[j + 1, k - 1] = -sn[j] * h0 + cs[j] * h1
        h0, h1 = H[k - 1, k - 1], H[k, k - 1]
        den = np.hypot(h0, h1)
        cs[k - 1], sn[k - 1] = h0 / den, h1 / den
        H[k - 1, k - 1] = den
        H[k, k - 1] = 0.0
        g[k] = -sn[k - 1] * g[k - 1]
        g[k - 1] = cs[k - 1] * g[k - 1]
        res = abs(g[k]) / nb
        if res < tol:
            break
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    x = (Q[:k].T @ y).reshape(b.shape)
    return x, k, res


def extract_velocity(sus, u):
    """U_j = int u / |Gamma_j|, Omega_j = tau_j^{-1} int (x - c_j) x u."""
    f, t = sphere_moments(sus, u)
    U = f / (4 * pi * sus.a ** 2)[:, None]
    Om = t / tau(sus.a)[:, None]
    return np.concatenate([U, Om], axis=1)


def mobility_apply(sus, FT, tol=1e-12, maxit=200, return_info=False):
    """U/Omega (N x 6) for force/torque FT (N x 6): Sec. 4.1 step by step."""
    rho = rho_from_FT(sus, FT)
    b = -(0.5 * rho + sus.apply("K", rho))
    zeta, its, res = gmres(lambda z: apply_A(sus, z), b, tol, maxit)
    u = sus.apply("S", rho + zeta)
    UO = extract_velocity(sus, u)
    if return_info:
        return UO, {"gmres_iters": its, "gmres_res": res, "zeta": zeta, "rho": rho}
    return UO
