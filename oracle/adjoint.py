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

The collision-resolved step of Sec. 3.2 (U = U_nc + M D gamma) is
differentiated in F_ext on its active set (collision_grad_F), assuming strict
complementarity; step_loss gives the same L through the full oracle step for
finite differences.
"""
import numpy as np

from . import lcp, mobility
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


# ----------------------------------------------------------------------------
# the collision step (Sec. 3.2) differentiated on the active set
# ----------------------------------------------------------------------------
def D_matrix(N, ij, nrm):
    """Dense 6N x n_c contact Jacobian of eq. Dmatdef (columns -n on i, +n on j)."""
    D = np.zeros((6 * N, len(ij)))
    for l, (i, j) in enumerate(ij):
        D[6 * i:6 * i + 3, l] = -nrm[l]
        D[6 * j:6 * j + 3, l] = nrm[l]
    return D


def collision_grad_F(M, D, gamma, ubar, active_tol=0.0):
    """dL/dF_ext of U = M F + M D gamma(F) for one collision-resolved step.

    On the active set A = {gamma > active_tol} (strict complementarity: the
    inactive constraints keep g > 0 under a small change of F), the LCP gives
    gamma_A = -(D_A^T M D_A)^{-1} (Phi_A / dt + D_A^T M F), so
        dU/dF = M - M D_A (D_A^T M D_A)^{-1} D_A^T M,
        dL/dF = (dU/dF)^T ubar = v - M^T D_A lam,
        v = M^T ubar,  (D_A^T M D_A)^T lam = D_A^T v.
    M (6N x 6N) is the assembled discrete mobility, D the contact Jacobian."""
    A = np.asarray(gamma) > active_tol
    v = M.T @ np.asarray(ubar, dtype=np.float64).ravel()
    if not A.any():
        return v.reshape(-1, 6), A
    DA = D[:, A]
    MAA = DA.T @ M @ DA
    lam = np.linalg.solve(MAA.T, DA.T @ v)
    return (v - M.T @ (DA @ lam)).reshape(-1, 6), A


def step_loss(centers, radii, FT, dt, p, *, delta=0.1, a_c_scale=1.0, beta=1.75,
              identity=False):
    """L = sum |U|^2 of one collision-resolved step (oracle, tight tolerances)."""
    if identity:
        out = lcp.resolve_collisions_identity(centers, radii, FT, dt, delta=delta,
                                              a_c_scale=a_c_scale, bbpgd_tol=1e-13)
    else:
        out = lcp.resolve_collisions(centers, radii, FT, dt, p, beta=beta, delta=delta,
                                     a_c_scale=a_c_scale, gmres_tol=1e-13, bbpgd_tol=1e-12)
    return float(np.sum(out["U"] ** 2)), out


def collision_grad_c_contacts(M, D, gamma, ubar, U, centers, ij, nrm, dt, active_tol=0.0):
    """The part of dL/dc (sphere centres) of one collision step that comes
    through the contact geometry: Phi_l = |c_j - c_i| - R_i - R_j and
    n_l = (c_j - c_i)/|c_j - c_i| in D, on the active set (strict
    complementarity, contact and near sets fixed).  With
    mu = (D_A^T M D_A)^{-T} D_A^T M^T ubar and w = dL/dF = M^T (ubar - D_A mu),
    differentiating gamma_A = -(D_A^T M D_A)^{-1} (Phi_A/dt + D_A^T M F) and
    U = M (F + D_A gamma_A) gives, per active contact l,
        v_l = (I - n n^T) t_l / |c_j - c_i| - (mu_l / dt) n_l,
        t_l = gamma_l (w_j - w_i) - mu_l (U_j - U_i)   (force parts),
    added to dL/dc_j and subtracted from dL/dc_i.  The remaining part is
    (ubar - D_A mu)^T (dM/dc) (F + D_A gamma_A); it vanishes for the identity
    mobility.  Returns (dL/dc contact part (N x 3), mu (n_c, zero off A))."""
    A = np.asarray(gamma) > active_tol
    N = len(centers)
    ub = np.asarray(ubar, dtype=np.float64).ravel()
    mu = np.zeros(len(gamma))
    g = np.zeros((N, 3))
    if not A.any():
        return g, mu
    DA = D[:, A]
    MAA = DA.T @ M @ DA
    mu[A] = np.linalg.solve(MAA.T, DA.T @ (M.T @ ub))
    w = (M.T @ (ub - D @ mu)).reshape(N, 6)
    Uf = np.asarray(U).reshape(N, 6)
    C = np.asarray(centers, dtype=np.float64)
    for l in np.nonzero(A)[0]:
        i, j = ij[l]
        n = np.asarray(nrm[l])
        d = np.linalg.norm(C[j] - C[i])
        t = gamma[l] * (w[j, :3] - w[i, :3]) - mu[l] * (Uf[j, :3] - Uf[i, :3])
        v = (t - n * (n @ t)) / d - (mu[l] / dt) * n
        g[j] += v
        g[i] -= v
    return g, mu
