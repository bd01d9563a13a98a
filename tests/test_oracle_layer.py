"""Pins of the oracle's layer potentials (Sec. 4.1, 4.2).

* The VSH exterior field (eq. ssgext) and its traction against direct
  quadrature of the Stokeslet / traction kernel on a finely upsampled grid at
  well-separated targets -- an independent route to the same integrals.
* A planted mistake (eq. ssgext's rho^W term in f^V as printed, (n+1)/(4n+2))
  fails that comparison: the pin catches the reading it decides.
* grad u against finite differences; div u = 0; the Stokes momentum balance
  grad p = lap u by finite differences of the oracle's own gradient.
* Self parts: the single-sphere facts the paper relies on (rigid modes in the
  null space of I/2 + K, Sec. 4.1), K[e_z] = -e_z/2 on the unit sphere (direct
  integral: int r r^T / |r|^3 dS over the sphere gives (4 pi/3) I), and the
  per-degree multipliers solved from the single-layer jump conditions.
"""
from math import pi

import numpy as np
import pytest

from oracle import layer, sph


def _band_limited(p, seed):
    rng = np.random.default_rng(seed)
    th, ph, nrm, w = sph.unit_grid(p)
    return sph.grid_synthesis(sph.analysis(rng.standard_normal((len(w), 3)), p), p)


def _brute(op, coef, p, center, a, xt, nt, q=40):
    thq, phq, nrmq, wq = sph.unit_grid(q)
    sigq = sph.synthesis(coef, p, thq, phq)
    return layer.far_sum(op, xt, nt, np.zeros(len(xt), int), center + a * nrmq, a * a * wq,
                         sigq, np.ones(len(wq), int), lambda i: np.array([], int))


def _targets(rng, R, center, a, k=6):
    d = rng.standard_normal((k, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    nt = rng.standard_normal((k, 3))
    nt /= np.linalg.norm(nt, axis=1)[:, None]
    return center + a * R * d, nt


@pytest.mark.parametrize("p", [4, 6])
def test_exterior_field_matches_quadrature(p):
    rng = np.random.default_rng(11)
    coef = sph.analysis(_band_limited(p, 1), p)
    for center, a in ((np.zeros(3), 1.0), (np.array([1.0, -2.0, 0.5]), 0.6)):
        for R in (2.5, 3.5, 6.0):
            xt, nt = _targets(rng, R, center, a)
            u, t = layer.vsh_field(coef, p, center, a, xt, nt)
            ub = _brute("S", coef, p, center, a, xt, nt)
            tb = _brute("K", coef, p, center, a, xt, nt)
            assert np.abs(u - ub).max() <= 1e-12 * np.abs(ub).max()
            assert np.abs(t - tb).max() <= 1e-12 * np.abs(tb).max()


def test_printed_fV_coefficient_is_caught(monkeypatch):
    """eq. ssgext printed with (n+1)/(4n+2) in f^V: the quadrature pin fails."""
    p = 4
    coef = sph.analysis(_band_limited(p, 2), p)
    orig = layer.radial_factors

    def printed(n, c, r):
        fV, fW, fX, g, dfV, dfW, dfX = orig(n, c, r)
        extra = c[1] / (2.0 * (2 * n + 1))        # ((n+1) - n)/(4n+2) * sW
        rp2, rp0 = r ** -(n + 2.0), r ** -(n + 0.0)
        return (fV + extra * (rp2 - rp0), fW, fX, g,
                dfV + extra * (-(n + 2) * rp2 + n * rp0) / r, dfW, dfX)

    monkeypatch.setattr(layer, "radial_factors", printed)
    rng = np.random.default_rng(5)
    xt, nt = _targets(rng, 3.0, np.zeros(3), 1.0)
    u, _ = layer.vsh_field(coef, p, np.zeros(3), 1.0, xt, nt)
    ub = _brute("S", coef, p, np.zeros(3), 1.0, xt, nt)
    assert np.abs(u - ub).max() > 1e-4 * np.abs(ub).max()


def test_gradient_divergence_and_momentum():
    p = 6
    coef = sph.analysis(_band_limited(p, 3), p)
    x0 = np.array([[1.2, -0.4, 0.6], [0.2, 0.9, -1.5]])
    u0, p0, g0 = layer.exterior_unit(coef, p, x0)
    h = 1e-5
    gfd = np.zeros_like(g0)
    pgrad = np.zeros((len(x0), 3))
    lap = np.zeros((len(x0), 3))
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        up, pp, gp = layer.exterior_unit(coef, p, x0 + e)
        um, pm, gm = layer.exterior_unit(coef, p, x0 - e)
        gfd[:, i, :] = (up - um) / (2 * h)
        pgrad[:, i] = (pp - pm) / (2 * h)
        lap += (gp[:, i, :] - gm[:, i, :]) / (2 * h)      # d_i (d_i u_j)
    scale = np.abs(g0).max()
    assert np.abs(gfd - g0).max() < 1e-8 * scale
    assert np.abs(np.trace(g0, axis1=1, axis2=2)).max() < 1e-13 * scale
    assert np.abs(pgrad - lap).max() < 1e-6 * np.abs(lap).max()


def test_polar_targets_use_rotated_frame_consistently():
    p = 6
    coef = sph.analysis(_band_limited(p, 4), p)
    # inside the guard the rotated frame is used; the direct-frame formulas are
    # still accurate at sin(theta) = 1e-3 and must agree with it
    xb = np.array([[0.99e-3 * 1.6, 0.0, 1.6], [0.0, -0.5e-3 * 2.1, -2.1]])
    ub, pb, gb = layer.exterior_unit(coef, p, xb)
    ud, pd, gd = layer._exterior_unit_frame(coef, p, xb)
    assert np.abs(ub - ud).max() < 1e-10
    assert np.abs(pb - pd).max() < 1e-10
    assert np.abs(gb - gd).max() < 1e-8
    # exactly on the axis
    u0, p0, g0 = layer.exterior_unit(coef, p, np.array([[0.0, 0.0, -1.3]]))
    u1, p1, g1 = layer.exterior_unit(coef, p, np.array([[1e-7, 0.0, -1.3]]))
    assert np.abs(u0 - u1).max() < 1e-6 and np.abs(g0 - g1).max() < 1e-5


def _mode_field(p, n, m, kind):
    th, ph, nrm, w = sph.unit_grid(p)
    V, W, X = sph.vsh(n, m, th, ph)
    B = {"V": V, "W": W, "X": X}[kind]
    return B


@pytest.mark.parametrize("p", [4, 8])
def test_self_multipliers_from_jump_conditions(p):
    """S_self and K_self act per degree n with the multipliers that follow from
    the single-layer jump conditions (S continuous, traction jump = -density)."""
    S = {"V": lambda n: n / ((2 * n + 1) * (2 * n + 3)),
         "W": lambda n: (n + 1) / ((2 * n - 1) * (2 * n + 1)),
         "X": lambda n: 1 / (2 * n + 1)}
    K = {"V": lambda n: 0.5 - 2 * n * (n + 2) / ((2 * n + 1) * (2 * n + 3)),
         "W": lambda n: 0.5 - (2 * n * n + 1) / ((2 * n - 1) * (2 * n + 1)),
         "X": lambda n: 0.5 - (n + 2) / (2 * n + 1)}
    for n in range(0, p + 1):
        for m in (0, n):
            for kind in ("V", "W", "X"):
                if n == 0 and kind != "V":
                    continue
                B = _mode_field(p, n, m, kind)
                for part in (B.real, B.imag):
                    if np.abs(part).max() < 1e-12:
                        continue
                    ss, ks = layer.self_terms(part, p, 1.0)
                    assert np.abs(ss - S[kind](n) * part).max() < 1e-12, (n, m, kind)
                    assert np.abs(ks - K[kind](n) * part).max() < 1e-12, (n, m, kind)
                    s2, _ = layer.self_terms(part, p, 0.7)
                    assert np.abs(s2 - 0.7 * ss).max() < 1e-12


def test_single_sphere_facts():
    p = 6
    th, ph, nrm, w = sph.unit_grid(p)
    ez = np.tile([0.0, 0.0, 1.0], (len(w), 1))
    ss, ks = layer.self_terms(ez, p, 1.0)
    assert np.abs(ks + 0.5 * ez).max() < 1e-13          # K[e_z] = -e_z/2
    assert np.abs(ss - 2.0 / 3.0 * ez).max() < 1e-13     # translation: U = F/(6 pi a)
    rot = np.cross([0.3, -0.2, 0.9], nrm)
    ss, ks = layer.self_terms(rot, p, 1.0)
    assert np.abs(0.5 * rot + ks).max() < 1e-13          # rigid rotation in the null space
    assert np.abs(ss - rot / 3.0).max() < 1e-13          # Omega = T/(8 pi a^3)
    _, ks = layer.self_terms(nrm, p, 1.0)
    assert np.abs(0.5 * nrm + ks - nrm).max() < 1e-13    # uniform normal density


def test_kernel_formulas():
    r = np.array([[0.3, -1.2, 0.7]])
    d = np.linalg.norm(r)
    G = layer.stokeslet(r)[0]
    assert np.allclose(G, (np.eye(3) / d + np.outer(r[0], r[0]) / d ** 3) / (8 * pi))
    T = layer.traction_kernel(r)[0]
    # T is the stress of the Stokeslet: T_ijk = -delta_ij p_k... in symmetric form
    # check against finite-difference stress of G with pressure r_k/(4 pi |r|^3)
    h = 1e-6
    dG = np.zeros((3, 3, 3))            # dG[l, i, k] = d_l G_ik
    for l in range(3):
        e = np.zeros(3)
        e[l] = h
        dG[l] = (layer.stokeslet(r + e)[0] - layer.stokeslet(r - e)[0]) / (2 * h)
    pk = r[0] / (4 * pi * d ** 3)
    # sigma_il for point force e_k: -p_k delta_il + d_l G_ik + d_i G_lk
    S = np.zeros((3, 3, 3))
    for k in range(3):
        for i in range(3):
            for l in range(3):
                S[i, k, l] = -pk[k] * (i == l) + dG[l, i, k] + dG[i, l, k]
    assert np.allclose(S, T, atol=1e-8)


# ---------------------------------------------------------------------------
# near-pair lists (Sec. 4.2): j is near i when |c_i - c_j| < beta (R_i + R_j)
# ---------------------------------------------------------------------------
def test_near_lists_threshold_hand_example():
    """Spheres placed on the threshold beta (R_i + R_j), beta = 1.75, each
    against sphere 0 (a = 1 at the origin) along its own axis, far from the
    others.  Along an axis the centre distance is exactly the coordinate
    (sqrt(fl(x * x)) = |x| in binary floating point).
      1: a = 0.5 at exactly 1.75 * 1.5 = 2.625          -> not near (strict <)
      2: a = 0.5 at 2.625 (1 - 1e-12)                    -> near
      3: a = 1   at 3.5 (1 + 1e-12)                      -> not near
      4: a = 0.6 at 1.5 * 1.75 * 1.6: inside beta times the sum of the
         diameters, outside beta times the sum of the radii -> not near
      5: a = 0.6 at 2.8 (1 - 1e-12) on -y                -> near"""
    beta = 1.75
    C = np.array([[0.0, 0.0, 0.0],
                  [2.625, 0.0, 0.0],
                  [0.0, 2.625 * (1 - 1e-12), 0.0],
                  [0.0, 0.0, 3.5 * (1 + 1e-12)],
                  [-1.5 * 1.75 * 1.6, 0.0, 0.0],
                  [0.0, -2.8 * (1 - 1e-12), 0.0]])
    R = np.array([1.0, 0.5, 0.5, 1.0, 0.6, 0.6])
    near = layer.near_lists(C, R, beta)
    assert [list(x) for x in near] == [[2, 5], [], [0], [], [], [0]]


def test_near_lists_match_kdtree_brute_force():
    """Random polydisperse suspension: the lists equal those from a k-d tree
    pair query (candidates within beta * 2 max a) filtered with an independent
    distance routine (math.dist), both directions, no self pairs, ascending."""
    import math

    from scipy.spatial import cKDTree

    from paper_1909_06623_gb300 import workloads
    C, R, _ = workloads.random_suspension(1234, 400, 0.30, pair_frac=0.05)
    beta = 1.75
    near = layer.near_lists(C, R, beta)
    ref = [set() for _ in range(len(R))]
    margins = []
    for i, j in cKDTree(C).query_pairs(beta * 2 * R.max()):
        d = math.dist(C[i], C[j])
        lim = beta * (R[i] + R[j])
        margins.append(abs(d - lim) / lim)
        if d < lim:
            ref[i].add(j)
            ref[j].add(i)
    assert min(margins) > 1e-9      # no pair sits on the threshold
    for i in range(len(R)):
        assert list(near[i]) == sorted(ref[i])
    total = sum(len(x) for x in near)
    assert 5 * len(R) < total < 30 * len(R)   # about 15 per sphere at this packing


def test_crowded_shell_workload():
    """The crowded-shell parity case: gaps to the large sphere within the
    stated range, no overlaps, every small sphere's surface within 1.5 large
    radii of its centre (so all of its nodes are close items of the large
    source), and near lists (beta = 1.75) pairing the large sphere with every
    small one and no two small ones."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.crowded_shell(4)
    C, R = w.centers, w.radii
    assert R[0] == 4.0 and np.all(R[1:] == 0.5) and len(R) == 25
    gap_big = np.linalg.norm(C[1:], axis=1) - R[0] - R[1:]
    assert gap_big.min() >= 0.02 and gap_big.max() <= 0.3
    d = np.linalg.norm(C[:, None] - C[None], axis=-1) - R[:, None] - R[None]
    np.fill_diagonal(d, np.inf)
    assert d.min() > 0
    assert np.all(np.linalg.norm(C[1:], axis=1) + R[1:] < 1.5 * R[0])
    near = layer.near_lists(C, R, 1.75)
    assert np.array_equal(near[0], np.arange(1, 25))
    assert all(np.array_equal(near[i], [0]) for i in range(1, 25))
