"""Pins of the oracle's gradient of the collision-resolved step (Sec. 3.2)
in the external forces, on the active set of the LCP.

* identity mobility (M = I): the formula against central differences of the
  full step (contacts, BBPGD, update) in every force / torque coordinate;
* directions the active constraints absorb: a loss gradient dL/dU = D_A y
  (a change of U along the active normals) gives dL/dF = 0, for the identity
  and for the assembled boundary-integral mobility;
* boundary-integral mobility (p = 4, five spheres, three active contacts):
  the formula with the assembled M against central differences of the full
  oracle step in sampled coordinates."""
import os

import numpy as np
import pytest

from oracle import adjoint, lcp
from paper_1909_06623_gb300 import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def chain(seed, n=5):
    w = workloads.contact_chain(seed, n)
    return w.centers, w.radii, w.FT


def strict(out, margin=1e-3):
    """Active gammas and inactive residuals well away from zero."""
    gam, g = out["gamma"], out["g"]
    act = gam > 0
    return act.any() and np.all(gam[act] > margin) and np.all(g[~act] > margin)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_identity_collision_gradient_fd(seed):
    c, a, F = chain(seed)
    dt = 1e-3
    L0, out = adjoint.step_loss(c, a, F, dt, 0, identity=True)
    assert strict(out)
    N = len(a)
    D = adjoint.D_matrix(N, out["ij"], out["normals"])
    grad, A = adjoint.collision_grad_F(np.eye(6 * N), D, out["gamma"], 2.0 * out["U"])
    h = 1e-6 * np.abs(F).max()
    fd = np.zeros_like(F)
    for i in range(N):
        for k in range(6):
            Fp, Fm = F.copy(), F.copy()
            Fp[i, k] += h
            Fm[i, k] -= h
            fd[i, k] = (adjoint.step_loss(c, a, Fp, dt, 0, identity=True)[0]
                        - adjoint.step_loss(c, a, Fm, dt, 0, identity=True)[0]) / (2 * h)
    assert np.abs(grad - fd).max() < 1e-6 * np.abs(fd).max()
    # torques never meet a sphere contact: their gradient is 2 U_omega = 2 T
    assert np.allclose(grad[:, 3:], 2.0 * F[:, 3:], rtol=1e-12)


def test_active_directions_have_no_gradient():
    c, a, F = chain(4)
    out = adjoint.step_loss(c, a, F, 1e-3, 0, identity=True)[1]
    N = len(a)
    D = adjoint.D_matrix(N, out["ij"], out["normals"])
    A = out["gamma"] > 0
    y = np.random.default_rng(0).standard_normal(A.sum())
    grad, _ = adjoint.collision_grad_F(np.eye(6 * N), D, out["gamma"], D[:, A] @ y)
    assert np.abs(grad).max() < 1e-12 * np.abs(D[:, A] @ y).max()


@pytest.fixture(scope="module")
def bie_case():
    """Stored oracle outputs (tests/golden/make_golden.py collision_grad): the
    assembled mobility M of five spheres at p = 4, the step's contacts and
    gamma, and central differences of the full oracle step."""
    d = np.load(os.path.join(HERE, "golden", "collision_grad_p4.npz"))
    D = adjoint.D_matrix(len(d["radii"]), d["ij"], d["normals"])
    return dict(d=d, M=d["M"], D=D)


def test_bie_active_directions_have_no_gradient(bie_case):
    d, M, D = bie_case["d"], bie_case["M"], bie_case["D"]
    A = d["gamma"] > 0
    assert A.sum() == 3
    y = np.array([1.0, -2.0, 0.5])
    grad, _ = adjoint.collision_grad_F(M, D, d["gamma"], D[:, A] @ y)
    assert np.abs(grad).max() < 1e-9 * np.abs(M.T @ (D[:, A] @ y)).max()


def test_bie_collision_gradient_fd(bie_case):
    d = bie_case["d"]
    out = {"gamma": d["gamma"], "g": d["g"]}
    assert strict(out, margin=1e-2)
    grad, _ = adjoint.collision_grad_F(bie_case["M"], bie_case["D"], d["gamma"], 2.0 * d["U"])
    for (i, k), fd in zip(d["coords"], d["fd"]):
        assert abs(grad[i, k] - fd) < 1e-6 * np.abs(grad).max(), (i, k, grad[i, k], fd)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_identity_collision_gradient_centres_fd(seed):
    """Identity mobility: dL/dc of the step comes only from the contact
    geometry (Phi and the normals in D); central differences of the full
    oracle step in every centre coordinate."""
    c, a, F = chain(seed)
    dt = 1e-3
    L0, out = adjoint.step_loss(c, a, F, dt, 0, identity=True)
    assert strict(out)
    N = len(a)
    D = adjoint.D_matrix(N, out["ij"], out["normals"])
    grad, _ = adjoint.collision_grad_c_contacts(np.eye(6 * N), D, out["gamma"], 2.0 * out["U"], out["U"],
                                                c, out["ij"], out["normals"], dt)
    h = 1e-7
    fd = np.zeros((N, 3))
    for i in range(N):
        for k in range(3):
            cp, cm = c.copy(), c.copy()
            cp[i, k] += h
            cm[i, k] -= h
            fd[i, k] = (adjoint.step_loss(cp, a, F, dt, 0, identity=True)[0]
                        - adjoint.step_loss(cm, a, F, dt, 0, identity=True)[0]) / (2 * h)
    assert np.abs(grad - fd).max() < 1e-5 * np.abs(fd).max()
    # translation invariance: the gradient sums to zero over the spheres
    assert np.abs(grad.sum(axis=0)).max() < 1e-9 * np.abs(grad).max()
