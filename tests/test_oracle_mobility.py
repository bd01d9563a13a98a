"""Pins of the oracle's mobility solve (Sec. 2, 4.1).

* single sphere: U = F/(6 pi a), Omega = T/(8 pi a^3) (the Stokes drag the
  paper compares against in Sec. 6.1), to round-off;
* two distant spheres: the pair mobility tends to the Rotne-Prager-Yamakawa
  form, exact to O((a/d)^4);
* symmetry and positive definiteness of the discrete mobility (Sec. 2) to the
  discretisation level, improving spectrally with p;
* exact equivariance under the rotation by 2 pi/(2p+2) about z, which maps the
  grid onto itself;
* the GMRES routine against a dense solve;
* eq. rigidbodyrho rearranged for mu = rho + zeta (the form the CUDA path
  solves) gives the same density and velocities;
* randomly oriented sphere grids (Sec. 5.4): identity orientations change
  nothing, one sphere keeps its exact drag, a global rotation of centres,
  grids and forces rotates the velocities exactly, and the velocities differ
  from the unrotated grids' only at the discretisation level."""
from math import pi

import numpy as np
import pytest

from oracle import mobility
from oracle.layer import Suspension
from paper_1909_06623_gb300 import workloads


@pytest.mark.parametrize("a", [1.0, 0.55])
def test_single_sphere_drag(a):
    sus = Suspension([[0.3, -0.1, 2.0]], [a], 6)
    FT = np.array([[0.3, -1.0, 0.5, 0.2, 0.7, -0.4]])
    UO = mobility.mobility_apply(sus, FT)
    assert np.abs(UO[0, :3] - FT[0, :3] / (6 * pi * a)).max() < 1e-14 / a
    assert np.abs(UO[0, 3:] - FT[0, 3:] / (8 * pi * a ** 3)).max() < 1e-14 / a ** 3


def test_far_pair_matches_rpy():
    d = 20.0
    sus = Suspension([[0, 0, 0], [0, d * 0.6, d * 0.8]], [1.0, 1.0], 6)
    FT = np.zeros((2, 6))
    FT[0, :3] = [0.3, 0.5, -1.0]
    UO = mobility.mobility_apply(sus, FT)
    dh = np.array([0, 0.6, 0.8])
    M12 = ((1 + 2 / (3 * d * d)) * np.eye(3) + (1 - 2 / (d * d)) * np.outer(dh, dh)) / (8 * pi * d)
    ref = M12 @ FT[0, :3]
    assert np.abs(UO[1, :3] - ref).max() < 2e-6 * np.abs(ref).max()


def _mobility_matrix(c, a, p):
    sus = Suspension(c, a, p)
    N = len(a)
    M = np.zeros((6 * N, 6 * N))
    for k in range(6 * N):
        FT = np.zeros(6 * N)
        FT[k] = 1.0
        M[:, k] = mobility.mobility_apply(sus, FT.reshape(N, 6), 1e-13).ravel()
    return M


def test_mobility_symmetric_positive_definite():
    c = np.array([[0, 0, 0], [2.6, 0.2, 0.0], [0.8, 2.5, 0.6]])
    a = np.array([1.0, 0.8, 0.9])
    asym = []
    for p in (4, 6):
        M = _mobility_matrix(c, a, p)
        asym.append(np.abs(M - M.T).max() / np.abs(M).max())
        assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    assert asym[1] < asym[0] / 5 and asym[1] < 1e-3


def test_grid_rotation_equivariance():
    p = 4
    ang = 2 * pi / (2 * p + 2)
    Rz = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]])
    c = np.array([[0, 0, 0], [2.3, 0.4, 0.3]])
    a = np.array([1.0, 0.9])
    FT = np.array([[0.2, -0.5, 1.0, 0.1, 0.0, 0.3], [-0.4, 0.1, 0.2, 0.0, 0.2, 0.0]])
    U1 = mobility.mobility_apply(Suspension(c, a, p), FT, 1e-13)
    FT2 = np.concatenate([FT[:, :3] @ Rz.T, FT[:, 3:] @ Rz.T], axis=1)
    U2 = mobility.mobility_apply(Suspension(c @ Rz.T, a, p), FT2, 1e-13)
    U1r = np.concatenate([U1[:, :3] @ Rz.T, U1[:, 3:] @ Rz.T], axis=1)
    assert np.abs(U1r - U2).max() < 1e-11


def test_gmres_against_dense_solve():
    rng = np.random.default_rng(0)
    A = np.eye(40) + 0.3 * rng.standard_normal((40, 40)) / np.sqrt(40)
    b = rng.standard_normal(40)
    x, its, res = mobility.gmres(lambda v: A @ v, b, 1e-13, 40)
    assert res < 1e-13 and np.abs(x - np.linalg.solve(A, b)).max() < 1e-11
    x0, its0, _ = mobility.gmres(lambda v: A @ v, np.zeros(40), 1e-13, 40)
    assert its0 == 0 and not x0.any()


def test_gradient_wrt_force_exact_vs_fd():
    """dL/dF = 2 M^T U (assembled mobility) agrees with central differences of
    the loss L = sum |U|^2; M^T differs from M by the discretisation level."""
    from oracle import adjoint
    c = np.array([[0.0, 0.0, 0.0], [2.4, 0.3, 0.0]])
    a = np.array([1.0, 0.8])
    FT = np.array([[0.3, -0.5, 1.0, 0.1, 0.0, 0.2], [-0.2, 0.4, 0.1, 0.0, 0.3, 0.0]])
    p = 4
    g = adjoint.grad_F_exact(c, a, FT, p)
    coords = [("F", 0, 0), ("F", 1, 2), ("F", 0, 4)]
    fd = adjoint.grad_fd(c, a, FT, p, coords, h=1e-4)
    ref = np.array([g[i, k] for _, i, k in coords])
    assert np.abs(fd - ref).max() < 1e-7 * np.abs(g).max()   # L is quadratic in F


def test_rearranged_unknown_gives_the_same_solve():
    """eq. rigidbodyrho solved for mu = rho + zeta: (I/2 + K + L)[mu] = L[rho],
    since (I/2 + K + L)[rho] - (I/2 + K)[rho] = L[rho].  The CUDA path solves
    this form (its right-hand side needs no traction application); with the
    oracle's operators both forms give the same density and velocities."""
    rng = np.random.default_rng(11)
    C = np.array([[0.0, 0.0, 0.0], [2.3, 0.4, -0.2], [0.3, 2.6, 0.5]])
    R = np.array([1.0, 0.8, 0.9])
    sus = Suspension(C, R, 3)
    FT = rng.standard_normal((3, 6))
    rho = mobility.rho_from_FT(sus, FT)
    A = lambda z: mobility.apply_A(sus, z.reshape(-1, 3)).reshape(-1)
    b_zeta = -(0.5 * rho + sus.apply("K", rho)).reshape(-1)
    b_mu = mobility.apply_L(sus, rho).reshape(-1)
    zeta, _, _ = mobility.gmres(A, b_zeta, 1e-14, 300)
    mu, _, _ = mobility.gmres(A, b_mu, 1e-14, 300)
    assert np.abs(mu - (rho.reshape(-1) + zeta)).max() < 1e-11 * np.abs(mu).max()
    U_zeta = mobility.extract_velocity(sus, sus.apply("S", rho + zeta.reshape(-1, 3)))
    U_mu = mobility.extract_velocity(sus, sus.apply("S", mu.reshape(-1, 3)))
    assert np.abs(U_mu - U_zeta).max() < 1e-11 * np.abs(U_zeta).max()
    assert np.abs(U_zeta - mobility.mobility_apply(sus, FT, tol=1e-14)).max() < 1e-11 * np.abs(U_zeta).max()


def _rot6(U, R):
    return np.concatenate([U[:, :3] @ R.T, U[:, 3:] @ R.T], axis=1)


def test_random_grid_orientations():
    p = 4
    c = np.array([[0.0, 0.0, 0.0], [2.4, 0.5, -0.3], [0.2, 2.5, 0.6]])
    a = np.array([1.0, 0.8, 0.9])
    FT = np.array([[0.2, -0.5, 1.0, 0.1, 0.0, 0.3], [-0.4, 0.1, 0.2, 0.0, 0.2, 0.0],
                   [0.3, 0.3, -0.6, 0.1, -0.2, 0.4]])
    Q = workloads.random_rotations(5, 3)
    assert np.abs(np.einsum("nij,nkj->nik", Q, Q) - np.eye(3)).max() < 1e-14
    assert np.allclose(np.linalg.det(Q), 1.0)
    U0 = mobility.mobility_apply(Suspension(c, a, p), FT, 1e-13)
    # identity orientations: the same arithmetic
    Ui = mobility.mobility_apply(Suspension(c, a, p, rotations=np.tile(np.eye(3), (3, 1, 1))), FT, 1e-13)
    assert np.abs(Ui - U0).max() < 1e-14
    # one sphere: exact drag in any orientation
    U1 = mobility.mobility_apply(Suspension(c[:1], a[:1], p, rotations=Q[:1]), FT[:1], 1e-14)
    assert np.abs(U1[0, :3] - FT[0, :3] / (6 * pi)).max() < 1e-14
    assert np.abs(U1[0, 3:] - FT[0, 3:] / (8 * pi)).max() < 1e-14
    # global rotation of centres, grids and forces
    UQ = mobility.mobility_apply(Suspension(c, a, p, rotations=Q), FT, 1e-13)
    R = workloads.random_rotations(6, 1)[0]
    UR = mobility.mobility_apply(Suspension(c @ R.T, a, p, rotations=np.einsum("ij,njk->nik", R, Q)),
                                 _rot6(FT, R), 1e-13)
    assert np.abs(UR - _rot6(UQ, R)).max() < 1e-11 * np.abs(UQ).max()
    # orientation changes the result only through the discretisation
    assert 1e-9 < np.abs(UQ - U0).max() < 1e-3 * np.abs(U0).max()
