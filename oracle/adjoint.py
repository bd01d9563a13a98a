"""Gradients of a velocity loss through the mobility solve -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no adjoint; the gradient is the derivative of the discrete map of
Sec. 4.1 (U = M F for given centres), so the oracle computes it from its own
forward solve:
  * loss L = sum_i |U_i|^2 (velocities and angular velocities of every sphere);
  * dL/dF exactly as 2 M^T U with M assembled column by column (6N mobility
    solves; small N only);
  * dL/dF and dL/dc by central finite differences of the forward solve
    (any N that the oracle can solve; c = sphere centres, radii fixed).
Finite differences must not move a pair across the near-pair threshold
beta (a_i + a_j): callers choose coordinates and steps that keep every pair at
least 10 h away from it (see near_margin).
"""
import numpy as np

from . import mobility
from .layer import Suspension


def loss(centers, radii, FT, p, beta=1.75, tol=1e-13):
    UO = mobility.mobility_apply(Suspension(centers, radii, p, beta), FT, tol, 400)
    return float(np.sum(UO * UO)), UO


def mobility_matrix(centers, radii, p, beta=1.75, tol=1e-13):
    sus = Suspension(centers, radii, p, beta)
    N = sus.N
    M = np.zeros((6 * N, 6 * N))
    for k in range(6 * N):
        e = np.zeros(6 * N)
        e[k] = 1.0
        M[:, k] = mobility.mobility_apply(sus, e.reshape(N, 6), tol, 400).ravel()
    return M


def grad_F_exact(centers, radii, FT, p, beta=1.75):
    """dL/dF = 2 M^T U with the assembled discrete mobility."""
    M = mobility_matrix(centers, radii, p, beta)
    U = M @ np.asarray(FT, dtype=np.float64).ravel()
    return (2.0 * M.T @ U).reshape(-1, 6)


def grad_fd(centers, radii, FT, p, coords, h=1e-6, beta=1.75):
    """Central differences of L.  coords: list of ('F', i, k) or ('c', i, k)."""
    out = []
    for kind, i, k in coords:
        vals = []
        for s in (+1, -1):
            C = np.array(centers, dtype=np.float64, copy=True)
            F = np.array(FT, dtype=np.float64, copy=True)
            if kind == "F":
                F[i, k] += s * h
            else:
                C[i, k] += s * h
            vals.append(loss(C, radii, F, p, beta)[0])
        out.append((vals[0] - vals[1]) / (2 * h))
    return np.array(out)


def near_margin(centers, radii, beta=1.75):
    """Smallest | |c_i - c_j| - beta (a_i + a_j) | over all pairs."""
    c = np.asarray(centers, dtype=np.float64)
    a = np.asarray(radii, dtype=np.float64)
    m = np.inf
    for i in range(len(a)):
        d = np.linalg.norm(c - c[i], axis=1)
        t = np.abs(d - beta * (a + a[i]))
        t[i] = np.inf
        m = min(m, float(t.min()))
    return m
