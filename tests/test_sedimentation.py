"""Multi-step workloads (Sec. 6.3) and the relative contact threshold (Sec. 3.2).

CPU (oracle pins):
* the pair threshold delta + delta_rel (a_i + a_j) -- the paper sets the
  threshold to 30% of the sum of the radii -- against a hand example at the
  boundary and against scipy's k-d tree pair query with the condition written
  as d <= (a_c_scale + delta_rel)(a_i + a_j) + delta;
* the oracle's per-sphere rows equal its pair loop with the relative threshold;
* the sedimenting-cluster workload: N spheres in the cluster ball at the stated
  volume fraction, collision-free at the collision radius, deterministic.

GPU (parity):
* cell-list and all-pairs searches against the oracle, bit for bit, with the
  relative threshold;
* sps_simulate (steps in place) against the oracle's step applied repeatedly
  (FP64, small cluster), and the mixed path against the FP64 path on a larger
  cluster.
"""
import pathlib

import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree

from oracle import lcp
from paper_1909_06623_gb300 import workloads

GOLDEN = pathlib.Path(__file__).parent / "golden"

# --------------------------------------------------------------------------- CPU
def test_relative_threshold_hand_example():
    a = np.array([0.6, 0.9])
    acs = 1.05
    for delta in (0.0, 0.1):
        thr = delta + 0.3 * (a[0] + a[1])
        for eps, inside in ((-1e-9, True), (1e-9, False)):
            d = acs * a[0] + acs * a[1] + thr + eps
            c = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
            ij, phi, _ = lcp.build_contacts(c, a, delta, acs, delta_rel=0.3)
            assert (len(ij) == 1) == inside
            # the absolute threshold alone never includes this pair
            assert len(lcp.build_contacts(c, a, delta, acs)[0]) == 0


def test_relative_threshold_matches_kdtree():
    w = workloads.tiny(41, 300, 2, phi=0.3)
    acs, delta, drel = 1.05, 0.02, 0.3
    ij, phi, nrm = lcp.build_contacts(w.centers, w.radii, delta, acs, delta_rel=drel)
    C, a = w.centers, w.radii
    pairs = cKDTree(C).query_pairs(2 * (acs + drel) * a.max() + delta, output_type="ndarray")
    keep = []
    for i, j in pairs:
        i, j = min(i, j), max(i, j)
        if np.linalg.norm(C[i] - C[j]) <= (acs + drel) * (a[i] + a[j]) + delta:
            keep.append((i, j))
    keep = sorted(keep)
    assert len(keep) > 100
    assert ij.tolist() == [list(p) for p in keep]
    # the relative part uses the sphere radii: the collision radii would add
    # pairs here
    ij_c = lcp.build_contacts(C, a * acs, delta, 1.0, delta_rel=drel)[0]
    assert len(ij_c) > len(ij)


def test_relative_threshold_rows_equal_pair_loop():
    w = workloads.tiny(42, 200, 2, phi=0.3)
    ij, phi, nrm = lcp.build_contacts(w.centers, w.radii, 0.0, 1.05, delta_rel=0.3)
    rows = []
    for i in range(w.N):
        js, ph, nr = lcp.contacts_of_sphere(w.centers, w.radii, i, 0.0, 1.05, delta_rel=0.3)
        rows += [(i, j, p_, tuple(n_)) for j, p_, n_ in zip(js, ph, nr)]
    assert [(r[0], r[1]) for r in rows] == [tuple(x) for x in ij.tolist()]
    assert np.array([r[2] for r in rows]).tobytes() == phi.tobytes()
    assert np.array([r[3] for r in rows]).tobytes() == nrm.tobytes()


def test_sedimenting_cluster_workload():
    w = workloads.sedimenting_cluster(N=300)
    w2 = workloads.sedimenting_cluster(N=300)
    assert np.array_equal(w.centers, w2.centers)
    assert w.N == 300 and np.all(w.radii == 1.0)
    Rb = (300 / 0.20) ** (1 / 3)
    assert np.linalg.norm(w.centers, axis=1).max() <= Rb - 1.0 + 1e-12
    d = np.linalg.norm(w.centers[:, None] - w.centers[None], axis=-1) + 1e9 * np.eye(w.N)
    assert d.min() > 2 * 1.05                   # collision-free at a_c = 1.05 a
    assert np.all(w.FT[:, 2] == -1.0) and np.all(w.FT[:, [0, 1, 3, 4, 5]] == 0.0)
    assert abs(w.dt - 0.05) < 1e-15 and w.params["delta_rel"] == 0.3
    # the relative threshold finds the cluster's neighbour pairs
    ij = lcp.build_contacts(w.centers, w.radii, 0.0, 1.05, delta_rel=0.3)[0]
    assert len(ij) > w.N


# --------------------------------------------------------------------------- GPU
@pytest.fixture(scope="module")
def sps():
    from paper_1909_06623_gb300 import build
    build.build()
    import paper_1909_06623_gb300 as m
    return m


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.gpu
@pytest.mark.parametrize("delta", [0.0, 0.05])
def test_gpu_relative_threshold_bit_exact(sps, delta):
    layouts = [workloads.jittered_lattice(43, 3000, jitter=0.2), workloads.tiny(44, 400, 2, phi=0.3),
               workloads.sedimenting_cluster(N=500)]
    for w in layouts:
        ref = lcp.build_contacts(w.centers, w.radii, delta, 1.05, delta_rel=0.3)
        got = []
        for search in (sps.SPS_SEARCH_CELLS, sps.SPS_SEARCH_ALL_PAIRS):
            ctx = sps.Context(p=2, delta=delta, delta_rel=0.3, a_c_scale=1.05, contact_search=search)
            nc = ctx.build_contacts(dev(w.centers), dev(w.radii))
            assert nc == len(ref[0]), w.name
            ij, phi, nrm = ctx.get_contacts()
            got.append((ij.cpu().numpy(), phi.cpu().numpy(), nrm.cpu().numpy()))
        for g in got:
            assert np.array_equal(g[0], ref[0]), w.name
            assert g[1].tobytes() == ref[1].tobytes() and g[2].tobytes() == ref[2].tobytes(), w.name


@pytest.mark.gpu
def test_gpu_simulate_matches_oracle_steps(sps):
    """Two steps in place against the oracle's step applied twice (stored by
    tests/golden/make_golden.py sed_steps; both steps have active contacts)."""
    d = np.load(GOLDEN / "sed_steps_p4.npz")
    assert np.all(d["n_active"] > 0)
    ctx = sps.Context(p=int(d["p"]), delta=0.0, delta_rel=0.3, a_c_scale=1.05, gmres_tol=1e-13,
                      gmres_max=300, bbpgd_tol=1e-12, bbpgd_max=20000)
    pos = dev(d["centers"])
    pos, UO, stats = ctx.simulate(pos, dev(d["radii"]), dev(d["FT"]), float(d["dt"]), 2)
    assert len(stats) == 2 and all(s["status"] == 0 for s in stats)
    assert [s["n_active"] for s in stats] == d["n_active"].tolist()
    traj = d["traj"]
    disp = np.abs(traj[-1] - traj[0]).max()
    assert np.abs(pos.cpu().numpy() - traj[-1]).max() <= 1e-10 * disp
    assert np.abs(UO.cpu().numpy() - d["U"][-1]).max() <= 1e-10 * np.abs(d["U"][-1]).max()


@pytest.mark.gpu
def test_gpu_simulate_mixed_vs_fp64(sps):
    w = workloads.sedimenting_cluster(N=200)
    kw = dict(p=6, delta=0.0, delta_rel=0.3, a_c_scale=1.05, bbpgd_tol=1e-8, bbpgd_max=5000,
              bb_safeguard=1)
    out = {}
    for prec, tol in ((0, 1e-10), (1, 1e-7)):
        ctx = sps.Context(precision=prec, gmres_tol=tol, gmres_max=300, **kw)
        pos = dev(w.centers)
        pos, UO, stats = ctx.simulate(pos, dev(w.radii), dev(w.FT), w.dt, 3)
        assert [s["status"] for s in stats] == [0, 0, 0]
        assert stats[-1]["n_contacts"] > w.N
        out[prec] = (pos.cpu().numpy(), UO.cpu().numpy())
    disp = np.abs(out[0][0] - w.centers).max()
    assert np.abs(out[1][0] - out[0][0]).max() <= 1e-5 * disp
    assert np.abs(out[1][1] - out[0][1]).max() <= 1e-5 * np.abs(out[0][1]).max()


@pytest.mark.gpu
def test_gpu_bb_warm_start_matches_oracle_steps(sps):
    """Algorithm 1 started from the previous step's gamma (bb_warm = 1): the
    second step's LCP solution still matches the oracle's step (which starts
    from gamma_0 = 0) to the FP64 tolerance."""
    d = np.load(GOLDEN / "sed_steps_p4.npz")
    ctx = sps.Context(p=int(d["p"]), delta=0.0, delta_rel=0.3, a_c_scale=1.05, gmres_tol=1e-13,
                      gmres_max=300, bbpgd_tol=1e-12, bbpgd_max=20000, bb_warm=1)
    pos = dev(d["centers"])
    pos, UO, stats = ctx.simulate(pos, dev(d["radii"]), dev(d["FT"]), float(d["dt"]), 2)
    assert all(s["status"] == 0 for s in stats)
    # step 2 started from a nonzero gamma_0: g_0 = M gamma_0 + q costs one
    # evaluation of M gamma (and the step length one more if it iterates)
    s2 = stats[1]
    assert (s2["bbpgd_iters"] == 0 and s2["mvops"] == 1) or s2["mvops"] == s2["bbpgd_iters"] + 2
    traj = d["traj"]
    disp = np.abs(traj[-1] - traj[0]).max()
    assert np.abs(pos.cpu().numpy() - traj[-1]).max() <= 1e-10 * disp
    assert np.abs(UO.cpu().numpy() - d["U"][-1]).max() <= 1e-10 * np.abs(d["U"][-1]).max()


@pytest.mark.gpu
def test_gpu_bb_warm_start_config2_mixed(sps):
    """Config 2 (1,000 spheres, p = 6, mixed): after the benchmark's three
    warm-up steps (which resolve the initial overlaps at the collision
    radius), three steps from gamma_0 = 0 and three from the previous step's
    gamma reach the same velocities within the mixed-path tolerance, the
    warm-started steps with fewer BBPGD iterations.  With bb_warm = 2 (the
    previous step's last step length as alpha_0) the same, with no more
    products of M beyond the iterations than bb_warm = 1 takes."""
    w = workloads.config2()
    # the benchmark's solver settings (eps_tol = 1e-5: the mixed operator's
    # rounding keeps the min-map residual from settling much below that)
    kw = dict(p=6, delta=0.1, a_c_scale=1.05, gmres_tol=1e-6, gmres_max=150, bbpgd_tol=1e-5,
              bbpgd_max=100, bb_safeguard=1, precision=1)
    ctx = sps.Context(bb_warm=0, **kw)
    pos, rad, FT = dev(w.centers), dev(w.radii), dev(w.FT)
    pos_out = torch.empty_like(pos)
    for _ in range(3):
        ctx.resolve_collisions(pos, rad, FT, w.dt, pos_out=pos_out, allow=(4, 5))
        pos.copy_(pos_out)
    start = pos.clone()
    out = {}
    for warm in (0, 1, 2):
        c = sps.Context(bb_warm=warm, **kw)
        p, UO, stats = c.simulate(start.clone(), rad, FT, w.dt, 3)
        assert all(s["status"] == 0 for s in stats)
        out[warm] = (p.cpu().numpy(), UO.cpu().numpy(), stats)
    U0 = out[0][1]
    disp = np.abs(out[0][0] - start.cpu().numpy()).max()
    for warm in (1, 2):
        assert np.abs(out[warm][1] - U0).max() <= 1e-5 * np.abs(U0).max()
        assert np.abs(out[warm][0] - out[0][0]).max() <= 1e-5 * disp
    it0 = sum(s["bbpgd_iters"] for s in out[0][2][1:])
    it1 = sum(s["bbpgd_iters"] for s in out[1][2][1:])
    assert it1 < it0
    extra = {warm: sum(s["mvops"] - s["bbpgd_iters"] for s in out[warm][2][1:]) for warm in (1, 2)}
    assert extra[2] <= extra[1]
