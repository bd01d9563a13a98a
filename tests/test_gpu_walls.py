"""Particle-wall constraints (Sec. 3.3.3) on the CUDA path against the oracle.

A wall is a plane n.x = d (unit normal into the fluid); each sphere near it
adds a column of D on that sphere alone.  Contacts are compared to the bit
(pair rows first, then wall rows (-1 - w, i)); steps within 1e-10 (FP64 and
identity mobility).  Stored oracle values: tests/golden/walls_p4.npz."""
import os

import numpy as np
import pytest
import torch

from oracle import lcp

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
WALLS = np.array([[0.0, 0.0, 1.0, 0.0], [-1.0, 0.0, 0.0, -10.0]])


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


def _corner(seed):
    rng = np.random.default_rng(seed)
    c = np.array([[8.85, 0.0, 1.02], [6.75, 0.1, 1.0], [8.9, 2.1, 1.1], [7.8, 1.0, 2.9]])
    c = c + 0.01 * rng.standard_normal(c.shape)
    FT = np.zeros((4, 6))
    FT[:, :3] = 30.0 * np.array([1.0, 0.2, -1.0]) + 5.0 * rng.standard_normal((4, 3))
    return c, np.ones(4), FT


@pytest.mark.parametrize("search", [1, 2])
def test_wall_contacts_bit_exact(sps, search):
    """All-pairs and cell-list searches, with walls: the oracle's list to the
    bit (a random box of 600 spheres between two walls, delta = 0.3)."""
    rng = np.random.default_rng(11)
    C = rng.random((600, 3)) * np.array([10.0, 10.0, 12.0])
    R = 0.4 + 0.3 * rng.random(600)
    W = np.array([[0.0, 0.0, 1.0, 0.0], [0.0, 0.0, -1.0, -12.0], [-1.0, 0.0, 0.0, -10.0]])
    ctx = sps.Context(p=2, delta=0.3, a_c_scale=1.05, delta_rel=0.1, contact_search=search)
    ctx.set_walls(W)
    nc = ctx.build_contacts(dev(C), dev(R))
    pij, pphi, pn = lcp.build_contacts(C, R, 0.3, 1.05, 0.1)
    wij, wphi, wn = lcp.build_wall_contacts(C, R, W, 0.3, 1.05, 0.1)
    ij, phi, nrm = ctx.get_contacts()
    assert nc == len(pij) + len(wij) and len(wij) > 50
    assert np.array_equal(ij.cpu().numpy(), np.concatenate([pij, wij]))
    ref_phi = np.concatenate([pphi, wphi])
    assert np.array_equal(phi.cpu().numpy().view(np.uint64), ref_phi.view(np.uint64))
    assert np.array_equal(nrm.cpu().numpy(), np.concatenate([pn, wn]))
    # D and D^T with wall columns against the oracle's
    g = rng.random(nc)
    U = rng.standard_normal((600, 6))
    ijn = np.concatenate([pij, wij])
    nn = np.concatenate([pn, wn])
    assert relerr(ctx.contact_force(dev(g), 600).cpu().numpy(), lcp.D_apply(600, ijn, nn, g)) < 1e-14
    assert relerr(ctx.contact_rate(dev(U)).cpu().numpy(), lcp.DT_apply(ijn, nn, U)) < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_identity_step_with_walls(sps, seed):
    c, a, FT = _corner(seed)
    ref = lcp.resolve_collisions_identity(c, a, FT, 1e-2, delta=0.2, walls=WALLS, bbpgd_tol=1e-13)
    ctx = sps.Context(p=2, delta=0.2, mobility=sps.SPS_MOB_IDENTITY, bbpgd_tol=1e-13)
    ctx.set_walls(WALLS)
    gam, U, pn = ctx.resolve_collisions(dev(c), dev(a), dev(FT), 1e-2)
    assert relerr(gam.cpu().numpy(), ref["gamma"]) < 1e-10
    assert relerr(U.cpu().numpy(), ref["U"]) < 1e-10


def test_bie_step_onto_floor_matches_oracle(sps):
    d = np.load(os.path.join(GOLD, "active_step_p4.npz"))
    w = np.load(os.path.join(GOLD, "walls_p4.npz"))
    assert (w["ij"][:, 0] < 0).sum() >= 1 and w["n_active"] >= 3
    for precision, tol, gtol, btol in ((0, 1e-10, 1e-13, 1e-12), (1, 1e-5, 1e-9, 1e-6)):
        ctx = sps.Context(p=int(d["p"]), delta=0.1, a_c_scale=1.05, gmres_tol=gtol, gmres_max=300,
                          bbpgd_tol=btol, warm_start=0, precision=precision)
        ctx.set_walls(w["walls"])
        gam, U, pn = ctx.resolve_collisions(dev(d["centers"]), dev(d["radii"]), dev(w["FT"]),
                                            float(d["dt"]))
        ij, _, _ = ctx.get_contacts()
        assert np.array_equal(ij.cpu().numpy(), w["ij"])
        assert relerr(gam.cpu().numpy(), w["gamma"]) < tol, precision
        assert relerr(U.cpu().numpy(), w["U"]) < tol, precision


def test_single_sphere_lands_on_floor(sps):
    """One sphere driven into the floor, boundary-integral mobility: the LCP
    is scalar and the step ends exactly on contact (Phi = 0 at a_c)."""
    dt, f = 1e-2, 400.0
    c = np.array([[0.3, -0.2, 1.05 + 0.07]])
    FT = np.array([[0.5, 0.0, -f, 0.0, 0.0, 0.0]])
    ctx = sps.Context(p=4, delta=0.1, a_c_scale=1.05, gmres_tol=1e-13, bbpgd_tol=1e-12)
    ctx.set_walls(WALLS[:1])
    gam, U, pn = ctx.resolve_collisions(dev(c), dev([1.0]), dev(FT), dt)
    assert abs(gam.item() - (0.07 / dt - f / (6 * np.pi)) * -6 * np.pi) < 1e-9
    assert abs(pn[0, 2].item() - 1.05) < 1e-12


def test_warm_start_over_steps_with_walls(sps):
    """Algorithm 1 from the previous step's gamma (bb_warm) with wall rows in
    the list: the same steps as from gamma_0 = 0, within eps_tol."""
    c, a, FT = _corner(5)
    out = {}
    for warm in (0, 1):
        ctx = sps.Context(p=2, delta=0.2, mobility=sps.SPS_MOB_IDENTITY, bbpgd_tol=1e-12, bb_warm=warm)
        ctx.set_walls(WALLS)
        pos = dev(c)
        for _ in range(3):
            _, U, po = ctx.resolve_collisions(pos, dev(a), dev(FT), 1e-2)
            pos = po.clone()
        out[warm] = pos.cpu().numpy()
    assert np.abs(out[0] - out[1]).max() < 1e-9
