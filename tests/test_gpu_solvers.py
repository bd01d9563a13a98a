"""The comparison LCP solvers of Sec. 3.3.1 on the CUDA path: APGD
(lcp_solver = 1), minimum-map Newton (lcp_solver = 2) and Algorithm 1 with
BB1/BB2 alternating (bb_variant = 3).  All must reach the LCP solution the
oracle finds (enumeration-pinned BBPGD), within what eps_tol leaves: 1e-8
relative."""
import os

import numpy as np
import pytest
import torch

from oracle import lcp

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")


@pytest.fixture(scope="module")
def sps():
    from paper_1909_06623_gb300 import build
    build.build()
    import paper_1909_06623_gb300 as m
    return m


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def relerr(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("solver,variant", [(1, 1), (0, 3)])
def test_identity_step_comparison_solvers(sps, solver, variant):
    from paper_1909_06623_gb300 import workloads
    w = workloads.jittered_lattice(7, 343)
    ref = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, delta=0.1, a_c_scale=1.05,
                                          bbpgd_tol=1e-12, bbpgd_max=50000)
    assert ref["info"]["n_active"] > 10
    ctx = sps.Context(p=2, delta=0.1, a_c_scale=1.05, mobility=sps.SPS_MOB_IDENTITY, bbpgd_tol=1e-12,
                      bbpgd_max=50000, lcp_solver=solver, bb_variant=variant, bb_safeguard=1)
    gam, U, _ = ctx.resolve_collisions(dev(w.centers), dev(w.radii), dev(w.FT), w.dt)
    assert ctx.last_stats["status"] == 0
    assert relerr(gam.cpu().numpy(), ref["gamma"]) < 1e-8
    assert relerr(U.cpu().numpy(), ref["U"]) < 1e-8
    if solver == 1:      # APGD evaluates M more than once per iteration
        assert ctx.last_stats["mvops"] > ctx.last_stats["bbpgd_iters"]


def test_apgd_boundary_integral_step(sps):
    """The five-sphere active step (p = 4, FP64) solved by APGD: the stored
    oracle step's gamma and velocities (BBPGD to 1e-12) within 1e-8."""
    d = np.load(os.path.join(GOLD, "active_step_p4.npz"))
    ctx = sps.Context(p=int(d["p"]), delta=0.1, a_c_scale=1.05, gmres_tol=1e-13, gmres_max=300,
                      bbpgd_tol=1e-12, bbpgd_max=5000, lcp_solver=1)
    gam, U, _ = ctx.resolve_collisions(dev(d["centers"]), dev(d["radii"]), dev(d["FT"]), float(d["dt"]))
    assert ctx.last_stats["status"] == 0
    assert relerr(gam.cpu().numpy(), d["gamma"]) < 1e-8
    assert relerr(U.cpu().numpy(), d["U"]) < 1e-8


@pytest.mark.parametrize("N,seed", [(343, 7), (1000, 8)])
def test_identity_step_minmap_newton(sps, N, seed):
    """Newton on the identity-mobility step: the LCP solution of the oracle's
    Algorithm 1 (1e-12) within 1e-8, in as many Newton steps as the oracle's
    Newton (+-1: the CG iterates differ in rounding) and far fewer than
    Algorithm 1's iterations."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.jittered_lattice(seed, N)
    kw = dict(delta=0.1, a_c_scale=1.05, bbpgd_tol=1e-12, bbpgd_max=50000)
    ref = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, **kw)
    nt = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, solver="newton", **kw)
    assert ref["info"]["n_active"] > 10 and nt["info"]["status"] == "ok"
    ctx = sps.Context(p=2, delta=0.1, a_c_scale=1.05, mobility=sps.SPS_MOB_IDENTITY, bbpgd_tol=1e-12,
                      bbpgd_max=100, lcp_solver=2)
    gam, U, pos_out = ctx.resolve_collisions(dev(w.centers), dev(w.radii), dev(w.FT), w.dt)
    st = ctx.last_stats
    assert st["status"] == 0 and st["final_phi"] < 1e-12
    assert abs(st["bbpgd_iters"] - nt["info"]["iters"]) <= 1
    assert st["bbpgd_iters"] < ref["info"]["iters"] / 4
    assert relerr(gam.cpu().numpy(), ref["gamma"]) < 1e-8
    assert relerr(U.cpu().numpy(), ref["U"]) < 1e-8
    assert np.abs(pos_out.cpu().numpy() - ref["centers_new"]).max() < 1e-10 * np.abs(w.centers).max()


def test_minmap_newton_boundary_integral_step(sps):
    """The five-sphere active step (p = 4, FP64) solved by minimum-map Newton:
    the stored oracle step's gamma and velocities (BBPGD to 1e-12) within 1e-8,
    with every product of M a mobility solve."""
    d = np.load(os.path.join(GOLD, "active_step_p4.npz"))
    ctx = sps.Context(p=int(d["p"]), delta=0.1, a_c_scale=1.05, gmres_tol=1e-13, gmres_max=300,
                      bbpgd_tol=1e-12, bbpgd_max=100, lcp_solver=2)
    gam, U, _ = ctx.resolve_collisions(dev(d["centers"]), dev(d["radii"]), dev(d["FT"]), float(d["dt"]))
    st = ctx.last_stats
    assert st["status"] == 0
    assert relerr(gam.cpu().numpy(), d["gamma"]) < 1e-8
    assert relerr(U.cpu().numpy(), d["U"]) < 1e-8
    # U_nc, the products of M (mvops) and the solve of the returned iterate
    assert st["mobility_solves"] == st["mvops"] + 2
