"""Pins of the oracle's contact set, D, and BBPGD (Sec. 3, Algorithm 1).

* contacts: a hand-checkable example, and agreement with scipy's k-d tree pair
  query on a random suspension;
* D and D^T are adjoint (eq. Dtranspose) and D^T U is the rate of change of Phi;
* BBPGD against exact LCP solutions by active-set enumeration (unique for SPD
  M, Sec. 3.3.2), complementarity at convergence, the absolute error bound of
  eq. abserrcqp, and the scalar-LCP fact of Sec. 6.2 (one GD step solves it);
* the full collision-resolved step against enumeration with the explicitly
  assembled M = D^T M D (n_c = 3 contacts, p = 4);
* the comparison solvers of Sec. 3.3.1 (APGD, minimum-map Newton) against
  enumeration and against Algorithm 1."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import lcp, mobility
from oracle.layer import Suspension
from paper_1909_06623_gb300 import workloads


def test_contacts_hand_example():
    c = np.array([[0, 0, 0], [2.05, 0, 0], [0, 0, 2.2], [10, 10, 10]])
    a = np.array([1.0, 1.0, 1.0, 0.5])
    ij, phi, nrm = lcp.build_contacts(c, a, 0.1)
    assert ij.tolist() == [[0, 1]]
    assert abs(phi[0] - 0.05) < 1e-15 and np.allclose(nrm[0], [1, 0, 0])
    ij, phi, nrm = lcp.build_contacts(c, a, 0.25)
    assert ij.tolist() == [[0, 1], [0, 2]]
    ij, phi, _ = lcp.build_contacts(c, a, 0.0, a_c_scale=1.05)
    assert ij.tolist() == [[0, 1], [0, 2], [1, 2]][:len(ij)] and abs(phi[0] + 0.05) < 1e-15


def test_contacts_match_kdtree():
    w = workloads.tiny(7, 60, 4, phi=0.3)
    ij, phi, nrm = lcp.build_contacts(w.centers, w.radii, 0.2)
    pairs = cKDTree(w.centers).query_pairs(2 * w.radii.max() + 0.2, output_type="ndarray")
    keep = []
    for i, j in pairs:
        i, j = min(i, j), max(i, j)
        if np.linalg.norm(w.centers[i] - w.centers[j]) - w.radii[i] - w.radii[j] <= 0.2:
            keep.append((i, j))
    assert sorted(keep) == [tuple(x) for x in ij.tolist()]
    assert np.allclose(np.linalg.norm(nrm, axis=1), 1.0)


def test_D_adjoint_and_phi_rate():
    rng = np.random.default_rng(1)
    w = workloads.tiny(3, 30, 4, phi=0.3)
    ij, phi, nrm = lcp.build_contacts(w.centers, w.radii, 0.3)
    gam = rng.random(len(ij))
    U = rng.standard_normal((30, 6))
    assert abs(np.sum(lcp.D_apply(30, ij, nrm, gam) * U) - gam @ lcp.DT_apply(ij, nrm, U)) < 1e-12
    h = 1e-7
    c2 = w.centers + h * U[:, :3]
    d2 = np.linalg.norm(c2[ij[:, 1]] - c2[ij[:, 0]], axis=1) - w.radii[ij[:, 0]] - w.radii[ij[:, 1]]
    assert np.abs((d2 - phi) / h - lcp.DT_apply(ij, nrm, U)).max() < 1e-5


@pytest.mark.parametrize("seed", range(6))
def test_bbpgd_matches_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = 1 + seed % 6
    B = rng.standard_normal((n, n))
    M = B @ B.T + 0.5 * np.eye(n)
    q = rng.standard_normal(n)
    exact = lcp.lcp_enumerate(M, q)
    for variant in (1, 2):
        gam, g, info = lcp.bbpgd(lambda x: M @ x, q, 1e-12, variant=variant)
        assert info["status"] == "ok"
        assert np.abs(gam - exact).max() < 1e-10
        assert gam.min() >= 0 and g.min() >= -1e-12 and abs(gam @ g) < 1e-10
        ev = np.linalg.eigvalsh(M)
        bound = (ev.max() + 1) / ev.min() * info["phi"]      # eq. abserrcqp
        assert np.linalg.norm(gam - exact) <= bound + 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_bbpgd_initial_guess_reaches_enumerated_solution(seed):
    """Algorithm 1 takes gamma_0 as input: from the exact solution it stops
    after the single evaluation of g_0 (no GD step), from a perturbed one it
    converges to the same LCP solution (unique for SPD M, Sec. 3.3.2)."""
    rng = np.random.default_rng(100 + seed)
    n = 2 + seed % 5
    B = rng.standard_normal((n, n))
    M = B @ B.T + 0.5 * np.eye(n)
    q = rng.standard_normal(n)
    exact = lcp.lcp_enumerate(M, q)
    if not np.any(exact):
        q[0] = -abs(q[0]) - 1.0
        exact = lcp.lcp_enumerate(M, q)
    gam, g, info = lcp.bbpgd(lambda x: M @ x, q, 1e-9, gamma0=exact)
    assert info["iters"] == 0 and info["mvops"] == 1 and np.array_equal(gam, exact)
    g0 = np.maximum(exact + 0.3 * rng.standard_normal(n), 0.0)
    if not np.any(g0):
        g0[0] = 1.0
    gam, g, info = lcp.bbpgd(lambda x: M @ x, q, 1e-12, gamma0=g0, safeguard=True)
    assert info["status"] == "ok" and info["mvops"] == info["iters"] + 2
    assert np.abs(gam - exact).max() < 1e-10


def test_scalar_lcp_one_step_and_trivial_cases():
    gam, g, info = lcp.bbpgd(lambda x: 2.0 * x, np.array([-3.0]), 1e-12)
    assert info["iters"] == 1 and info["mvops"] == 2 and abs(gam[0] - 1.5) < 1e-15
    gam, g, info = lcp.bbpgd(lambda x: 2.0 * x, np.array([3.0]), 1e-12)
    assert info["iters"] == 0 and info["mvops"] == 0 and gam[0] == 0.0


def test_collision_step_against_enumeration():
    c = np.array([[0, 0, 0], [2.02, 0, 0], [1.0, 1.76, 0.0], [5.0, 0.3, 0.2]])
    a = np.ones(4)
    FT = np.zeros((4, 6))
    FT[:, :3] = 20.0 * np.array([[1.0, 0.3, 0.0], [-1.0, 0.2, 0.0], [0.0, -1.0, 0.1], [-0.5, 0, 0]])
    dt = 0.05
    out = lcp.resolve_collisions(c, a, FT, dt, 4, gmres_tol=1e-13, bbpgd_tol=1e-11)
    ij, nrm = out["ij"], out["normals"]
    assert len(ij) == 3 and out["info"]["n_active"] >= 1
    sus = Suspension(c, a, 4)
    M = np.zeros((3, 3))
    for l in range(3):
        e = np.zeros(3)
        e[l] = 1.0
        M[:, l] = lcp.DT_apply(ij, nrm, mobility.mobility_apply(sus, lcp.D_apply(4, ij, nrm, e), 1e-13))
    exact = lcp.lcp_enumerate(M, out["q"])
    assert np.abs(out["gamma"] - exact).max() < 1e-7 * max(1.0, np.abs(exact).max())
    g = out["g"]
    assert out["gamma"].min() >= 0 and g.min() > -1e-10
    assert abs(out["gamma"] @ g) < 1e-9
    # after the step, the linearised gaps are non-negative
    lin = out["phi"] + dt * lcp.DT_apply(ij, nrm, out["U"])
    assert lin.min() > -1e-9


def test_bbpgd_breakdown_and_safeguard():
    """Algorithm 1 defines no step when s^T y <= 0.  A matrix whose symmetric
    part is indefinite produces that; the literal reading stops ("breakdown"),
    the safeguard keeps the previous step length and carries on."""
    M = np.array([[1.0, 0.0], [0.0, -0.3]])
    q = np.array([-1.0, -1.0])
    gam, g, info = lcp.bbpgd(lambda x: M @ x, q, 1e-12, jmax=50)
    assert info["status"] == "breakdown"
    gam, g, info = lcp.bbpgd(lambda x: M @ x, q, 1e-12, jmax=50, safeguard=True)
    assert info["safeguards"] >= 1 and info["status"] in ("ok", "not_converged")


# ---------------------------------------------------------------------------
# large contact sets: per-sphere rows, vectorised D / D^T, identity mobility
# ---------------------------------------------------------------------------
def test_contact_rows_bit_exact():
    w = workloads.jittered_lattice(11, 343, jitter=0.15)
    ij, phi, nrm = lcp.build_contacts(w.centers, w.radii, 0.1, 1.05)
    assert len(ij) > 100
    for i in range(w.N):
        j, ph, nr = lcp.contacts_of_sphere(w.centers, w.radii, i, 0.1, 1.05)
        sel = ij[:, 0] == i
        assert np.array_equal(j, ij[sel, 1])
        assert ph.tobytes() == phi[sel].tobytes() and nr.tobytes() == nrm[sel].tobytes()


def test_vectorised_D_products():
    rng = np.random.default_rng(5)
    w = workloads.jittered_lattice(12, 216, jitter=0.2)
    ij, phi, nrm = lcp.build_contacts(w.centers, w.radii, 0.1, 1.05)
    gam = rng.random(len(ij))
    U = rng.standard_normal((w.N, 6))
    assert np.abs(lcp.D_apply_vec(w.N, ij, nrm, gam) - lcp.D_apply(w.N, ij, nrm, gam)).max() < 1e-14
    assert np.abs(lcp.DT_apply_vec(ij, nrm, U) - lcp.DT_apply(ij, nrm, U)).max() < 1e-14
    assert abs(np.sum(lcp.D_apply_vec(w.N, ij, nrm, gam) * U) - gam @ lcp.DT_apply_vec(ij, nrm, U)) < 1e-11


def test_identity_step_head_on_pair():
    # two spheres overlapping along x, no external force: M = D^T D = 2, so
    # gamma = -Phi / (2 dt) and one step separates them to exactly Phi = 0
    c = np.array([[0.0, 0.0, 0.0], [1.9, 0.0, 0.0]])
    a = np.array([1.0, 1.0])
    dt = 1e-3
    out = lcp.resolve_collisions_identity(c, a, np.zeros((2, 6)), dt, delta=0.1, bbpgd_tol=1e-12)
    assert out["ij"].tolist() == [[0, 1]]
    assert abs(out["gamma"][0] - 0.1 / (2 * dt)) < 1e-9
    cn = out["centers_new"]
    assert abs(np.linalg.norm(cn[1] - cn[0]) - 2.0) < 1e-13
    # approaching at speed 2f with a gap: gamma = max(0, -(Phi/dt - 2 f) / 2)
    c2 = np.array([[0.0, 0.0, 0.0], [2.05, 0.0, 0.0]])
    F = np.zeros((2, 6))
    F[0, 0], F[1, 0] = 100.0, -100.0
    out = lcp.resolve_collisions_identity(c2, a, F, dt, delta=0.1, bbpgd_tol=1e-12)
    assert abs(out["gamma"][0] - (200.0 - 0.05 / dt) / 2) < 1e-9
    cn = out["centers_new"]
    assert abs(np.linalg.norm(cn[1] - cn[0]) - 2.0) < 1e-13
    # separating pair: no force needed
    out = lcp.resolve_collisions_identity(c2, a, -F, dt, delta=0.1, bbpgd_tol=1e-12)
    assert out["gamma"][0] == 0.0 and out["info"]["iters"] == 0


@pytest.mark.parametrize("seed", range(3))
def test_identity_step_matches_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    # a short chain of touching unit spheres along a wobbly line
    n = 5
    c = np.zeros((n, 3))
    for k in range(1, n):
        d = np.array([1.0, 0.2 * rng.standard_normal(), 0.2 * rng.standard_normal()])
        c[k] = c[k - 1] + (1.95 + 0.1 * rng.random()) * d / np.linalg.norm(d)
    a = np.ones(n)
    F = rng.standard_normal((n, 6)) * 50
    dt = 1e-3
    out = lcp.resolve_collisions_identity(c, a, F, dt, delta=0.1, bbpgd_tol=1e-12)
    ij, nrm, q = out["ij"], out["normals"], out["q"]
    nc = len(q)
    assert nc >= n - 1
    M = np.zeros((nc, nc))
    for k in range(nc):
        e = np.zeros(nc)
        e[k] = 1.0
        M[:, k] = lcp.DT_apply(ij, nrm, lcp.D_apply(n, ij, nrm, e))
    ref = lcp.lcp_enumerate(M, q)
    assert np.abs(out["gamma"] - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())
    g = M @ out["gamma"] + q
    assert out["gamma"].min() >= 0 and g.min() > -1e-9 and abs(out["gamma"] @ g) < 1e-6
    # U = F_ext + D gamma
    U = F + lcp.D_apply(n, ij, nrm, out["gamma"])
    assert np.abs(out["U"] - U).max() < 1e-9


def test_jittered_lattice_statistics():
    w = workloads.jittered_lattice(13, 8000)
    pairs = cKDTree(w.centers).query_pairs(2 * 1.05 + 0.1, output_type="ndarray")
    d = np.linalg.norm(w.centers[pairs[:, 0]] - w.centers[pairs[:, 1]], axis=1)
    phi = d - 1.05 * (w.radii[pairs[:, 0]] + w.radii[pairs[:, 1]])
    nc = np.sum(phi <= 0.1)
    assert 0.7 < nc / w.N < 1.3
    assert 0.4 < np.sum(phi < 0) / nc < 0.8
    vol = np.sum(4 / 3 * np.pi * w.radii ** 3)
    L = np.ptp(w.centers, axis=0) + 2 * 1.0
    assert 0.25 < vol / np.prod(L) < 0.4


# ---------------------------------------------------------------------------
# failure rule (keep_best): smallest-residual iterate, growth guard
# ---------------------------------------------------------------------------
def _spd_lcp(seed, n=24):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    M = A @ A.T / n + 0.05 * np.eye(n)
    return M, rng.standard_normal(n)


def test_bbpgd_keep_best_returns_smallest_residual():
    """Capped where BB's residual is not monotone: the returned residual is
    the minimum over the recorded iterates (gamma_0 included), the returned
    pair (gamma, g) has that residual, and it is the iterate an uncapped run
    reaches at that index (bit for bit); without the rule the last iterate is
    returned."""
    found = 0
    for seed in range(20):
        M, q = _spd_lcp(seed)
        mop = lambda g: M @ g
        _, _, full = lcp.bbpgd(mop, q, 1e-12, jmax=500)
        h = full["history"]
        bad = [j for j in range(1, len(h)) if h[j] > min(h[:j])]
        if not bad:
            continue
        j = bad[0]
        gam, g, info = lcp.bbpgd(mop, q, 1e-12, jmax=j, keep_best=True)
        assert info["status"] == "not_converged" and info["iters"] == j
        assert info["phi"] == min(info["history"]) < info["history"][-1]
        assert np.array_equal(g, M @ gam + q)
        assert lcp.minmap(gam, g) == info["phi"]
        gb, _, ib = lcp.bbpgd(mop, q, 1e-12, jmax=info["best"])
        assert ib["iters"] == info["best"] and np.array_equal(gb, gam)
        gl, _, il = lcp.bbpgd(mop, q, 1e-12, jmax=j)
        assert il["phi"] == h[j] and not np.array_equal(gl, gam)
        found += 1
    assert found >= 3


def test_bbpgd_growth_guard():
    """An indefinite M (a negative diagonal entry) makes the projected steps
    grow without bound; with the safeguard the loop would run to j_max and
    overflow, the growth guard stops it with breakdown once the residual
    reaches 1e6 times the initial one and returns the best iterate."""
    M = np.array([[2.0, 0.0], [0.0, -0.5]])
    q = np.array([-1.0, -1.0])
    with np.errstate(over="ignore", invalid="ignore"):
        _, _, free = lcp.bbpgd(lambda g: M @ g, q, 1e-10, jmax=200, safeguard=True)
    assert free["status"] == "not_converged" and not free["phi"] < 1e12
    gam, g, info = lcp.bbpgd(lambda g: M @ g, q, 1e-10, jmax=200, safeguard=True,
                             keep_best=True)
    h = info["history"]
    assert info["status"] == "breakdown" and info["iters"] < 200
    assert h[-1] >= lcp.GROWTH_LIMIT * h[0] and all(x < lcp.GROWTH_LIMIT * h[0] for x in h[:-1])
    assert info["phi"] == min(h) and lcp.minmap(gam, g) == info["phi"]


def test_dense_packings_touch_at_the_collision_radius():
    """Dense workloads (volume fraction above random sequential addition) are
    compressed at the collision radius a_c = 1.05 a: no pair overlaps there
    (Phi >= 0, the state the collision solver maintains) and many pairs
    touch, as in a sediment; the contact set at delta = 0.1 has about two
    pairs per sphere."""
    w = workloads.config5(500, 4)
    ij, phi, _ = lcp.build_contacts(w.centers, w.radii, 0.1, a_c_scale=1.05)
    assert phi.min() >= 0.0
    assert np.sum(phi < 1e-6) > 0.2 * len(w.radii)
    assert 1.0 < len(phi) / len(w.radii) < 4.0


# ---------------------------------------------------------------------------
# particle-wall constraints (Sec. 3.3.3): columns of D on one particle only
# ---------------------------------------------------------------------------
WALLS = np.array([[0.0, 0.0, 1.0, 0.0],      # floor z = 0, fluid above
                  [-1.0, 0.0, 0.0, -10.0]])  # side wall x = 10, fluid at x < 10


def test_wall_contacts_hand_example():
    c = np.array([[0.0, 0.0, 1.05], [3.0, 0.0, 1.2], [8.95, 4.0, 5.0], [8.9, 8.0, 1.02]])
    a = np.ones(4)
    ij, phi, nrm = lcp.build_wall_contacts(c, a, WALLS, 0.1)
    assert ij.tolist() == [[-1, 0], [-2, 2], [-1, 3], [-2, 3]]
    assert np.allclose(phi, [0.05, 0.05, 0.02, 0.1], atol=1e-14)
    assert np.array_equal(nrm, WALLS[[0, 1, 0, 1], :3])
    # D and D^T with a wall column: +gamma n on the sphere alone, n . U_i
    gam = np.array([1.0, 2.0, 3.0, 4.0])
    FT = lcp.D_apply(4, ij, nrm, gam)
    assert np.allclose(FT[:, :3], [[0, 0, 1], [0, 0, 0], [-2, 0, 0], [-4, 0, 3]])
    U = np.arange(24, dtype=float).reshape(4, 6)
    assert np.allclose(lcp.DT_apply(ij, nrm, U), [2.0, -12.0, 20.0, -18.0])
    # adjointness <D g, U> = <g, D^T U>
    assert abs(np.sum(FT[:, :3] * U[:, :3]) - gam @ lcp.DT_apply(ij, nrm, U)) < 1e-12


def test_sphere_onto_wall_lands_on_contact():
    """One sphere pushed into the floor: the LCP is scalar, gamma =
    -(Phi/dt + n.U_nc) / (n.M n), and the step ends exactly on contact.
    Identity mobility (n.M n = 1) and the boundary-integral mobility of one
    sphere (exact drag: n.M n = 1/(6 pi a))."""
    dt, f = 1e-2, 40.0
    c = np.array([[0.3, -0.2, 1.0 * 1.05 + 0.07]])
    a = np.array([1.0])
    FT = np.array([[0.5, 0.0, -f, 0.0, 0.0, 0.0]])
    out = lcp.resolve_collisions_identity(c, a, FT, dt, delta=0.1, a_c_scale=1.05, walls=WALLS[:1],
                                          bbpgd_tol=1e-13)
    assert abs(out["gamma"][0] - (f - 0.07 / dt)) < 1e-10
    assert abs(out["centers_new"][0, 2] - 1.05) < 1e-12
    f = 400.0                       # the fluid slows the sphere: f / (6 pi) > Phi / dt
    FT[0, 2] = -f
    out = lcp.resolve_collisions(c, a, FT, dt, 4, delta=0.1, a_c_scale=1.05, walls=WALLS[:1],
                                 gmres_tol=1e-13, bbpgd_tol=1e-12)
    U_nc = out["U_nc"][0, 2]
    assert abs(U_nc + f / (6 * np.pi)) < 1e-12
    assert abs(out["gamma"][0] - (-(0.07 / dt + U_nc) * 6 * np.pi)) < 1e-9
    assert abs(out["centers_new"][0, 2] - 1.05) < 1e-12
    assert abs(out["centers_new"][0, 0] - (0.3 + 0.5 / (6 * np.pi) * dt)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_identity_step_with_walls_matches_enumeration(seed):
    """Spheres pressed into a corner (floor and side wall) and into each
    other: Algorithm 1 on pair and wall constraints together equals the
    enumerated LCP solution with the assembled M = D^T D."""
    rng = np.random.default_rng(seed)
    c = np.array([[8.85, 0.0, 1.02], [6.75, 0.1, 1.0], [8.9, 2.1, 1.1], [7.8, 1.0, 2.9]])
    c = c + 0.01 * rng.standard_normal(c.shape)
    a = np.ones(4)
    FT = np.zeros((4, 6))
    FT[:, :3] = 30.0 * np.array([1.0, 0.2, -1.0]) + 5.0 * rng.standard_normal((4, 3))
    dt = 1e-2
    out = lcp.resolve_collisions_identity(c, a, FT, dt, delta=0.2, walls=WALLS, bbpgd_tol=1e-12)
    ij, nrm, q = out["ij"], out["normals"], out["q"]
    assert (ij[:, 0] < 0).sum() >= 3 and (ij[:, 0] >= 0).sum() >= 2
    nc = len(q)
    Dm = np.stack([lcp.D_apply(4, ij, nrm, np.eye(nc)[l])[:, :3].ravel() for l in range(nc)], axis=1)
    M = Dm.T @ Dm
    ref = lcp.lcp_enumerate(M, q)
    assert np.abs(out["gamma"] - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())
    assert (out["gamma"] > 0).sum() >= 2


# ---------------------------------------------------------------------------
# comparison solvers (Sec. 3.3.1): APGD and the alternating BB step
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(4))
def test_apgd_and_alternating_bb_match_enumeration(seed):
    """APGD (Nesterov with an adaptive Lipschitz estimate) and Algorithm 1
    with BB1/BB2 alternating reach the enumerated LCP solution of a random
    SPD problem; APGD spends more products of M per iteration (its
    sufficient-decrease checks), the reason the paper prefers BBPGD."""
    rng = np.random.default_rng(100 + seed)
    n = 6
    A = rng.standard_normal((n, n))
    M = A @ A.T + 0.5 * np.eye(n)
    q = rng.standard_normal(n) * 3
    ref = lcp.lcp_enumerate(M, q)
    mop = lambda x: M @ x
    ga, _, ia = lcp.apgd(mop, q, 1e-11, jmax=20000)
    gb, _, ib = lcp.bbpgd(mop, q, 1e-11, jmax=20000, variant=3, safeguard=True)
    for gam in (ga, gb):
        assert np.abs(gam - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())
    assert ia["status"] == "ok" and ib["status"] == "ok"
    assert ia["mvops"] > ia["iters"]


def test_apgd_identity_step_matches_bbpgd():
    """The identity-mobility collision step solved by APGD equals the one
    solved by Algorithm 1 (a jittered lattice with active contacts)."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.jittered_lattice(7, 125)
    kw = dict(delta=0.1, a_c_scale=1.05, bbpgd_tol=1e-12, bbpgd_max=50000)
    a = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, solver="apgd", **kw)
    b = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, **kw)
    assert b["info"]["n_active"] > 5
    assert np.abs(a["gamma"] - b["gamma"]).max() < 1e-8 * np.abs(b["gamma"]).max()
    assert np.abs(a["U"] - b["U"]).max() < 1e-8 * np.abs(b["U"]).max()


@pytest.mark.parametrize("seed", range(8))
def test_minmap_newton_matches_enumeration(seed):
    """Minimum-map Newton (Sec. 3.3.1) reaches the enumerated solution of a
    random SPD LCP, H = min(gamma, g) = 0 to rounding, in a few Newton steps;
    info counts every product of M."""
    rng = np.random.default_rng(100 + seed)
    n = 3 + seed
    A = rng.standard_normal((n, n))
    M = A @ A.T + 0.5 * np.eye(n)
    q = rng.standard_normal(n) * 3
    ref = lcp.lcp_enumerate(M, q)
    calls = [0]

    def mop(x):
        calls[0] += 1
        return M @ x

    gam, g, info = lcp.minmap_newton(mop, q, 1e-12, jmax=100)
    assert info["status"] == "ok" and info["phi"] < 1e-12
    assert np.abs(gam - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    assert np.abs(g - (M @ gam + q)).max() < 1e-11 * max(1.0, np.abs(q).max())
    assert info["mvops"] == calls[0] and info["cg_iters"] <= info["mvops"]
    assert info["iters"] <= 10


def test_minmap_newton_decoupled_and_trivial_cases():
    """M = m I decouples the LCP into gamma_l = max(0, -q_l / m): the first
    Newton step (F = {q < 0}, one CG step on a multiple of the identity)
    lands on it; q >= 0 needs no step and no product."""
    q = np.array([-3.0, 2.0, -0.5, 0.0, -7.0])
    gam, g, info = lcp.minmap_newton(lambda x: 2.0 * x, q, 1e-14)
    assert info["iters"] == 1 and info["mvops"] == 1 and info["status"] == "ok"
    assert np.array_equal(gam, np.maximum(0.0, -q / 2.0))
    gam, g, info = lcp.minmap_newton(lambda x: 2.0 * x, np.array([3.0, 0.5]), 1e-14)
    assert info["iters"] == 0 and info["mvops"] == 0 and not np.any(gam)


def test_minmap_newton_collision_steps():
    """The collision step with Newton as the LCP solver: the identity-mobility
    step equals Algorithm 1's (jittered lattice with active contacts), and the
    boundary-integral step (p = 4, three contacts) equals the enumerated
    solution of its assembled M = D^T M D."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.jittered_lattice(7, 125)
    kw = dict(delta=0.1, a_c_scale=1.05, bbpgd_tol=1e-12, bbpgd_max=50000)
    a = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, solver="newton", **kw)
    b = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, **kw)
    assert a["info"]["status"] == "ok" and b["info"]["n_active"] > 5
    assert a["info"]["iters"] < b["info"]["iters"] / 4
    assert np.abs(a["gamma"] - b["gamma"]).max() < 1e-10 * np.abs(b["gamma"]).max()
    assert np.abs(a["U"] - b["U"]).max() < 1e-10 * np.abs(b["U"]).max()
    c = np.array([[0, 0, 0], [2.02, 0, 0], [1.0, 1.76, 0.0], [5.0, 0.3, 0.2]])
    FT = np.zeros((4, 6))
    FT[:, :3] = 20.0 * np.array([[1.0, 0.3, 0.0], [-1.0, 0.2, 0.0], [0.0, -1.0, 0.1], [-0.5, 0, 0]])
    out = lcp.resolve_collisions(c, np.ones(4), FT, 0.05, 4, gmres_tol=1e-13, bbpgd_tol=1e-11,
                                 solver="newton")
    ij, nrm = out["ij"], out["normals"]
    sus = Suspension(c, np.ones(4), 4)
    M = np.zeros((3, 3))
    for l in range(3):
        e = np.zeros(3)
        e[l] = 1.0
        M[:, l] = lcp.DT_apply(ij, nrm, mobility.mobility_apply(sus, lcp.D_apply(4, ij, nrm, e), 1e-13))
    exact = lcp.lcp_enumerate(M, out["q"])
    assert out["info"]["status"] == "ok" and out["info"]["n_active"] >= 1
    assert np.abs(out["gamma"] - exact).max() < 1e-7 * max(1.0, np.abs(exact).max())


def test_rotor_workloads():
    """Sec. 7 workloads: the rotor cluster's radii follow the log-normal law
    with mean 1 and standard deviation 0.3 and start collision-free at the
    collision radius 1.1 a; the monolayer lies in z = 0 with no overlap at
    a_c and many pairs touching; both carry the torque (0, 0, 1) only."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.rotor_cluster(N=600)
    assert abs(w.radii.mean() - 1.0) < 0.05 and abs(w.radii.std() - 0.3) < 0.05
    _, phi, _ = lcp.build_contacts(w.centers, w.radii, 0.0, 1.1, 0.3)
    assert len(phi) > 0 and phi.min() >= 0.0
    assert np.all(w.FT[:, :5] == 0) and np.all(w.FT[:, 5] == 1.0) and w.dt == 1.0
    m = workloads.rotor_monolayer(N=300)
    assert np.all(m.centers[:, 2] == 0.0)
    _, phi, _ = lcp.build_contacts(m.centers, m.radii, 0.0, 1.1, 0.3)
    assert phi.min() >= 0.0 and np.sum(phi < 1e-6) > 0.5 * len(m.radii)
    assert np.all(m.FT[:, 5] == 1.0) and m.dt == 0.5
