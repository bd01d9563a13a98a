"""GPU parity of the contact search and the identity-mobility collision step.

* The cell-list search and the all-pairs search against the oracle's pair
  loop (Sec. 3.2), bit for bit (indices, Phi and normal bits), on lattices,
  random suspensions and degenerate layouts (one cell, a flat layer, two far
  clusters, a single sphere, no contacts).
* At the size the contact benchmark times (2 x 10^7 spheres), sampled rows
  against the oracle's per-sphere row, and the invariants of the list.
* The identity-mobility step (U = F, M = D^T D) against the oracle's step
  with the same mobility: gamma, U and the new centres <= 1e-10 relative; at
  full size, the complementarity of the BBPGD result (Algorithm 1, eq.
  mmapnorm) checked with the oracle's D products on the GPU's contact list.
"""
import functools

import numpy as np
import pytest
import torch

from oracle import lcp
from paper_1909_06623_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
N_BENCH = 20_000_000


@pytest.fixture(scope="module")
def sps():
    from paper_1909_06623_gb300 import build
    build.build()
    import paper_1909_06623_gb300 as m
    return m


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def gpu_contacts(sps, C, R, search, delta=0.1, acs=1.05):
    ctx = sps.Context(p=2, delta=delta, a_c_scale=acs, contact_search=search)
    nc = ctx.build_contacts(dev(C), dev(R))
    if nc == 0:
        return np.zeros((0, 2), np.int32), np.zeros(0), np.zeros((0, 3))
    ij, phi, nrm = ctx.get_contacts()
    return ij.cpu().numpy(), phi.cpu().numpy(), nrm.cpu().numpy()


def same_bits(a, b):
    return (a[0].shape == b[0].shape and np.array_equal(a[0], b[0])
            and a[1].tobytes() == b[1].tobytes() and a[2].tobytes() == b[2].tobytes())


@functools.lru_cache(maxsize=1)
def layouts():
    out = []
    w = workloads.jittered_lattice(21, 3000)
    out.append(("lattice3000", w.centers, w.radii))
    w = workloads.tiny(22, 400, 2, phi=0.3)
    out.append(("random400", w.centers, w.radii))
    rng = np.random.default_rng(23)
    # every sphere in one cell (box smaller than a cell side)
    out.append(("one_cell", rng.random((300, 3)) * 2.0, 0.5 + 0.5 * rng.random(300)))
    # a flat layer: no extent in z
    C = np.concatenate([rng.random((900, 2)) * 40.0, np.zeros((900, 1))], axis=1)
    out.append(("flat", C, 0.5 + 0.5 * rng.random(900)))
    # two clusters 1e6 apart (cell count capped, coarse cells)
    C = rng.random((600, 3)) * 12.0
    C[300:] += 1e6
    out.append(("far_clusters", C, 0.5 + 0.5 * rng.random(600)))
    # no contacts at all
    C = np.stack(np.meshgrid(*[np.arange(8.0) * 5.0] * 3), -1).reshape(-1, 3)
    out.append(("sparse", C, np.ones(len(C))))
    out.append(("single", np.array([[1.0, 2.0, 3.0]]), np.array([0.7])))
    return out


@pytest.mark.parametrize("case", range(7))
def test_cell_list_matches_all_pairs_and_oracle(sps, case):
    name, C, R = layouts()[case]
    ref = lcp.build_contacts(C, R, 0.1, 1.05)
    cells = gpu_contacts(sps, C, R, sps.SPS_SEARCH_CELLS)
    pairs = gpu_contacts(sps, C, R, sps.SPS_SEARCH_ALL_PAIRS)
    assert same_bits(cells, pairs), name
    assert np.array_equal(cells[0], ref[0]), name
    assert cells[1].tobytes() == ref[1].tobytes(), name
    assert cells[2].tobytes() == ref[2].tobytes(), name


def test_cell_list_delta_zero_and_large(sps):
    w = workloads.jittered_lattice(24, 1000, jitter=0.2)
    for delta in (0.0, 1.5):
        ref = lcp.build_contacts(w.centers, w.radii, delta, 1.05)
        got = gpu_contacts(sps, w.centers, w.radii, sps.SPS_SEARCH_CELLS, delta=delta)
        assert np.array_equal(got[0], ref[0]) and got[1].tobytes() == ref[1].tobytes()


@pytest.fixture(scope="module")
def bench_case(sps):
    """The contact benchmark's input at full size, with one identity step."""
    w = workloads.jittered_lattice(workloads.SEED_BASE + 6, N_BENCH)
    tol = 1e-4 * np.sqrt(w.N)
    ctx = sps.Context(p=2, delta=0.1, a_c_scale=1.05, mobility=sps.SPS_MOB_IDENTITY,
                      bbpgd_tol=tol, bbpgd_max=1000)
    pos, rad, FT = dev(w.centers), dev(w.radii), dev(w.FT)
    gam, UO, pos_out = ctx.resolve_collisions(pos, rad, FT, w.dt, gamma_cap=4 * w.N)
    st = dict(ctx.last_stats)
    ij, phi, nrm = ctx.get_contacts()
    out = dict(w=w, tol=tol, st=st, gamma=gam.cpu().numpy(), U=UO.cpu().numpy(),
               pos_out=pos_out.cpu().numpy(), ij=ij.cpu().numpy(), phi=phi.cpu().numpy(),
               nrm=nrm.cpu().numpy())
    del ctx, pos, rad, FT, gam, UO, pos_out, ij, phi, nrm
    torch.cuda.empty_cache()
    return out


def test_cell_list_full_size_sampled_rows(bench_case):
    w, ij, phi, nrm = bench_case["w"], bench_case["ij"], bench_case["phi"], bench_case["nrm"]
    nc = len(phi)
    assert 0.7 * w.N < nc < 1.3 * w.N
    # invariants: i < j, rows sorted by (i, j), Phi <= delta, unit normals
    assert np.all(ij[:, 0] < ij[:, 1])
    key = ij[:, 0].astype(np.int64) * w.N + ij[:, 1]
    assert np.all(np.diff(key) > 0)
    assert np.all(phi <= 0.1)
    assert np.abs(np.linalg.norm(nrm, axis=1) - 1.0).max() < 1e-14
    starts = np.searchsorted(ij[:, 0], np.arange(w.N + 1))
    rng = np.random.default_rng(5)
    for i in list(rng.choice(w.N, 24, replace=False)) + [0, w.N - 1]:
        j, ph, nr = lcp.contacts_of_sphere(w.centers, w.radii, int(i), 0.1, 1.05)
        a, b = starts[i], starts[i + 1]
        assert np.array_equal(ij[a:b, 1], j)
        assert phi[a:b].tobytes() == ph.tobytes() and nrm[a:b].tobytes() == nr.tobytes()


def test_identity_step_full_size_complementarity(bench_case):
    w, st = bench_case["w"], bench_case["st"]
    ij, nrm, phi, gam = bench_case["ij"], bench_case["nrm"], bench_case["phi"], bench_case["gamma"]
    assert st["status"] == 0 and st["n_contacts"] == len(gam) and st["bbpgd_iters"] > 0
    q = phi / w.dt + lcp.DT_apply_vec(ij, nrm, w.FT)
    Fc = lcp.D_apply_vec(w.N, ij, nrm, gam)
    g = lcp.DT_apply_vec(ij, nrm, Fc) + q
    assert gam.min() >= 0.0
    # min-map residual below the tolerance (eq. mmapnorm), up to the rounding
    # of the different summation order
    mm = np.linalg.norm(np.minimum(gam, g))
    assert mm < bench_case["tol"] * (1 + 1e-6) + 1e-9 * np.linalg.norm(q)
    assert abs(mm - st["final_phi"]) < 1e-6 * np.linalg.norm(q)
    U = w.FT + Fc
    scale = np.abs(U).max()
    assert np.abs(bench_case["U"] - U).max() < TOL64 * scale
    assert np.abs(bench_case["pos_out"] - (w.centers + w.dt * U[:, :3])).max() < 1e-12 * np.abs(w.centers).max()
    assert st["n_active"] == int(np.sum(gam > 0))


@pytest.mark.parametrize("N,seed,search", [(512, 31, 1), (3375, 32, 2)])
def test_identity_step_matches_oracle(sps, N, seed, search):
    w = workloads.jittered_lattice(seed, N)
    ref = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, delta=0.1, a_c_scale=1.05,
                                          bbpgd_tol=1e-10, bbpgd_max=5000)
    assert ref["info"]["status"] == "ok"
    ctx = sps.Context(p=2, delta=0.1, a_c_scale=1.05, mobility=sps.SPS_MOB_IDENTITY,
                      bbpgd_tol=1e-10, bbpgd_max=5000, contact_search=search)
    gam, UO, pos_out = ctx.resolve_collisions(dev(w.centers), dev(w.radii), dev(w.FT), w.dt)
    st = ctx.last_stats
    assert st["n_contacts"] == len(ref["q"])
    gs = np.abs(ref["gamma"]).max()
    assert np.abs(gam.cpu().numpy() - ref["gamma"]).max() < TOL64 * gs
    U = UO.cpu().numpy()
    assert np.abs(U - ref["U"]).max() < TOL64 * np.abs(ref["U"]).max()
    assert np.abs(pos_out.cpu().numpy() - ref["centers_new"]).max() < 1e-13 * np.abs(w.centers).max()
    assert st["n_active"] == ref["info"]["n_active"]


@pytest.mark.parametrize("scale", [1e-30, 1e-12, 1e30])
def test_identity_step_scale_equivariance(sps, scale):
    """Algorithm 1 with the identity mobility is equivariant under F -> sF,
    dt -> dt/s, eps_tol -> s eps_tol: gamma and U scale by s and the positions
    move alike.  FP64 against the oracle at s = 1, 1e-10."""
    w = workloads.jittered_lattice(31, 512)
    ref = lcp.resolve_collisions_identity(w.centers, w.radii, w.FT, w.dt, delta=0.1, a_c_scale=1.05,
                                          bbpgd_tol=1e-10, bbpgd_max=5000)
    ctx = sps.Context(p=2, delta=0.1, a_c_scale=1.05, mobility=sps.SPS_MOB_IDENTITY,
                      bbpgd_tol=1e-10 * scale, bbpgd_max=5000)
    gam, UO, pos_out = ctx.resolve_collisions(dev(w.centers), dev(w.radii), dev(scale * w.FT),
                                              w.dt / scale)
    assert ctx.last_stats["status"] == 0
    assert ctx.last_stats["n_active"] == ref["info"]["n_active"]
    gs = np.abs(ref["gamma"]).max()
    assert np.abs(gam.cpu().numpy() / scale - ref["gamma"]).max() < TOL64 * gs
    assert np.abs(UO.cpu().numpy() / scale - ref["U"]).max() < TOL64 * np.abs(ref["U"]).max()
    assert np.abs(pos_out.cpu().numpy() - ref["centers_new"]).max() < 1e-12 * np.abs(w.centers).max()


def test_identity_mobility_apply_and_adjoint(sps):
    w = workloads.jittered_lattice(33, 64)
    ctx = sps.Context(p=2, mobility=sps.SPS_MOB_IDENTITY)
    pos, rad, FT = dev(w.centers), dev(w.radii), dev(w.FT)
    U = ctx.mobility_apply(pos, rad, FT)
    assert torch.equal(U, FT)
    gU = torch.randn(64, 6, dtype=torch.float64, device="cuda")
    U2, gF, gx = ctx.mobility_adjoint(pos, rad, FT, gU)
    assert torch.equal(U2, FT) and torch.equal(gF, gU) and float(gx.abs().max()) == 0.0


def test_identity_rejects_bad_inputs(sps):
    w = workloads.jittered_lattice(34, 27)
    ctx = sps.Context(p=2, mobility=sps.SPS_MOB_IDENTITY)
    R = w.radii.copy()
    R[3] = -1.0
    with pytest.raises(sps.SPSError):
        ctx.resolve_collisions(dev(w.centers), dev(R), dev(w.FT), 1e-3)
    C = w.centers.copy()
    C[5, 1] = np.nan
    with pytest.raises(sps.SPSError):
        ctx.resolve_collisions(dev(C), dev(w.radii), dev(w.FT), 1e-3)
