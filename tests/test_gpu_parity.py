"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated by the workloads this library is built for): contacts and
indices bit-exact; FP64 path <= 1e-10 relative (max-norm over the compared
array, relative to its largest entry); mixed path <= 1e-5 relative.  The
oracle values come from tests/golden/*.npz (written by make_golden.py, which
calls only oracle/) or are computed live for small cases."""
import os
from math import pi

import numpy as np
import pytest
import torch

from oracle import lcp, mobility, sph
from oracle.layer import Suspension
from paper_1909_06623_gb300 import workloads

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
TOL64 = 1e-10
TOLMX = 1e-5


@pytest.fixture(scope="module")
def sps():
    from paper_1909_06623_gb300 import build
    build.build()
    import paper_1909_06623_gb300 as m
    return m


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def planes(a):  # (NP, 3) -> (3, NP) device
    return dev(np.ascontiguousarray(np.asarray(a).T))


def relerr(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


def load(name):
    return np.load(os.path.join(GOLD, name), allow_pickle=False)


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
def test_nodes_match_oracle(sps):
    d = load("tiny_layers.npz")
    C, R, p = d["c1_centers"], d["c1_radii"], int(d["c1_p"])
    ctx = sps.Context(p=p)
    ctx.set_geometry(dev(C), dev(R))
    X, Nr, W = ctx.nodes()
    Xo, No, Wo = sph.sphere_nodes(C, R, p)
    assert np.abs(X.cpu().numpy().T - Xo).max() < 1e-14 * np.abs(Xo).max() * 10
    assert np.abs(Nr.cpu().numpy().T - No).max() < 1e-14
    assert np.abs(W.cpu().numpy() - Wo).max() < 1e-14


@pytest.mark.parametrize("name", ["cfg2_sample.npz", "tiny_layers.npz"])
def test_near_lists_match_oracle(sps, name):
    """Near pairs (Sec. 4.2), exact: per-sphere counts against the oracle's
    stored counts (config 2) and the whole CSR against the oracle's lists."""
    from oracle.layer import near_lists
    d = load(name)
    if name == "tiny_layers.npz":
        C, R, p = d["c1_centers"], d["c1_radii"], int(d["c1_p"])
    else:
        C, R, p = d["centers"], d["radii"], int(d["p"])
    ctx = sps.Context(p=p, beta=1.75)
    ctx.set_geometry(dev(C), dev(R))
    ptr, idx = ctx.near_lists()
    ptr, idx = ptr.cpu().numpy(), idx.cpu().numpy()
    ref = near_lists(C, R, 1.75)
    counts = np.diff(ptr)
    assert np.array_equal(counts, [len(x) for x in ref])
    if "near_count" in d.files:
        assert np.array_equal(counts, d["near_count"])
    assert np.array_equal(idx, np.concatenate(ref).astype(np.int32))
    assert ctx.geometry_counts()[0] == len(idx)


@pytest.mark.parametrize("name,acs", [("cfg2_sample.npz", 1.0), ("cfg1_step.npz", 1.0),
                                      ("active_step_p4.npz", 1.05)])
def test_contacts_bit_exact(sps, name, acs):
    d = load(name)
    ctx = sps.Context(p=4, delta=0.1, a_c_scale=acs)
    nc = ctx.build_contacts(dev(d["centers"]), dev(d["radii"]))
    assert nc == len(d["ij"])
    ij, phi, nrm = ctx.get_contacts()
    assert np.array_equal(ij.cpu().numpy(), d["ij"])
    assert np.array_equal(phi.cpu().numpy().view(np.uint64), d["phi"].view(np.uint64))
    assert np.array_equal(nrm.cpu().numpy().view(np.uint64), d["normals"].view(np.uint64))


def test_contacts_large_delta_and_edges(sps):
    rng = np.random.default_rng(5)
    C = rng.random((300, 3)) * 12
    R = 0.3 + 0.4 * rng.random(300)          # overlaps allowed
    ctx = sps.Context(p=2, delta=0.7)
    nc = ctx.build_contacts(dev(C), dev(R))
    ij, phi, nrm = lcp.build_contacts(C, R, 0.7)
    g_ij, g_phi, g_n = ctx.get_contacts()
    assert nc == len(ij) and np.array_equal(g_ij.cpu().numpy(), ij)
    assert np.array_equal(g_phi.cpu().numpy(), phi) and np.array_equal(g_n.cpu().numpy(), nrm)
    # one sphere: empty list
    assert ctx.build_contacts(dev(C[:1]), dev(R[:1])) == 0


def test_D_and_DT_match_oracle(sps):
    d = load("active_step_p4.npz")
    C, R = d["centers"], d["radii"]
    ctx = sps.Context(p=4, delta=0.3, a_c_scale=1.05)
    ctx.build_contacts(dev(C), dev(R))
    ij, phi, nrm = lcp.build_contacts(C, R, 0.3, 1.05)
    rng = np.random.default_rng(0)
    gam = rng.random(len(ij))
    U = rng.standard_normal((len(R), 6))
    FT = ctx.contact_force(dev(gam), len(R)).cpu().numpy()
    assert relerr(FT, lcp.D_apply(len(R), ij, nrm, gam)) < 1e-15
    rate = ctx.contact_rate(dev(U)).cpu().numpy()
    assert relerr(rate, lcp.DT_apply(ij, nrm, U)) < 1e-14


# ---------------------------------------------------------------------------
# layer operators
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["c1", "c2", "c3"])
@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOLMX), (2, TOL64)])
def test_layer_operators_tiny(sps, case, precision, tol):
    d = load("tiny_layers.npz")
    C, R, p, sig = d[f"{case}_centers"], d[f"{case}_radii"], int(d[f"{case}_p"]), d[f"{case}_sigma"]
    ctx = sps.Context(p=p, precision=precision)
    ctx.set_geometry(dev(C), dev(R))
    s = planes(sig)
    for op, key in ((sps.SPS_OP_S, "S"), (sps.SPS_OP_K, "K"), (sps.SPS_OP_A, "A")):
        out = ctx.layer_apply(op, s).cpu().numpy().T
        assert relerr(out, d[f"{case}_{key}"]) < tol, (case, key)


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOLMX), (2, TOL64)])
def test_layer_operators_crowded_close_items(sps, precision, tol):
    """One sphere of radius 4 ringed by 24 of radius 0.5 at gaps 0.04-0.3
    (p = 4): every node of the small spheres lies within 1.5 radii of the
    large one, so that source has 1,200 close items, more than the 1,024 a
    near-field CTA lists (the mixed path then finds them again by the same
    test).  S, K and I/2 + K + L against the oracle on every node."""
    d = load("crowded_p4.npz")
    C, R, p = d["centers"], d["radii"], int(d["p"])
    P = (p + 1) * (2 * p + 2)
    dist = np.linalg.norm(C[1:], axis=1)
    assert np.all(dist + R[1:] < 1.5 * R[0]) and (len(R) - 1) * P > 1024
    ctx = sps.Context(p=p, precision=precision)
    ctx.set_geometry(dev(C), dev(R))
    s = planes(d["sigma"])
    for op, key in ((sps.SPS_OP_S, "S"), (sps.SPS_OP_K, "K"), (sps.SPS_OP_A, "A")):
        out = ctx.layer_apply(op, s).cpu().numpy().T
        assert relerr(out, d[key]) < tol, key


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOLMX), (2, TOL64)])
def test_layer_operators_cfg2_sampled(sps, precision, tol):
    """Full-size geometry (1,000 spheres, p = 6) in the launch shape the bench
    uses; the oracle evaluated S, K and I/2+K+L on a sample of target spheres."""
    d = load("cfg2_sample.npz")
    p = int(d["p"])
    P = (p + 1) * (2 * p + 2)
    ctx = sps.Context(p=p, precision=precision)
    ctx.set_geometry(dev(d["centers"]), dev(d["radii"]))
    s = planes(d["sigma"])
    sl = np.concatenate([np.arange(i * P, (i + 1) * P) for i in d["targets"]])
    for op, key in ((sps.SPS_OP_S, "S"), (sps.SPS_OP_K, "K"), (sps.SPS_OP_A, "A")):
        out = ctx.layer_apply(op, s).cpu().numpy().T[sl]
        assert relerr(out, d[key]) < tol, key


@pytest.mark.parametrize("name", ["tiny_layers.npz", "cfg2_sample.npz"])
def test_double_float_far_field_matches_fp64(sps, name):
    """SPS_FP64_DW (far-field pair terms in double-float on the FP32 pipe)
    against the native FP64 kernels on every node: the same operator to
    1e-13 of its largest value (the FP64 path itself meets the oracle at
    1e-10); the FP32 far field of the mixed path is ~3e-7 away."""
    d = load(name)
    if name == "tiny_layers.npz":
        C, R, p = d["c3_centers"], d["c3_radii"], int(d["c3_p"])
    else:
        C, R, p = d["centers"], d["radii"], int(d["p"])
    P = (p + 1) * (2 * p + 2)
    sig = planes(np.random.default_rng(3).standard_normal((len(R) * P, 3)))
    out = {}
    for prec in (0, 2):
        ctx = sps.Context(p=p, precision=prec)
        ctx.set_geometry(dev(C), dev(R))
        out[prec] = [ctx.layer_apply(op, sig).cpu().numpy() for op in (sps.SPS_OP_S, sps.SPS_OP_K)]
    for a, b in zip(out[2], out[0]):
        assert relerr(a, b) < 1e-13


@pytest.mark.parametrize("p", [3, 6, 8])
def test_tensor_core_transforms(sps, p):
    """The mixed path's VSH analysis and self synthesis run on the tensor
    cores (three-term BF16 split, FP32 accumulation).  One sphere isolates the
    self term (no far or near pairs); 200 spheres span two 128-sphere tiles
    with a ragged tail; p = 8 takes two N tiles (270 and 486 rows).  Both are
    compared with the oracle: the self term alone within 5e-6 (FP32-class: a
    two-term split would leave 2^-16 = 1.5e-5), the full operator within the
    mixed-path tolerance."""
    rng = np.random.default_rng(40 + p)
    P = (p + 1) * (2 * p + 2)
    cases = [(np.zeros((1, 3)), np.array([0.8]), 5e-6)]
    w = workloads.tiny(40 + p, 200, p, phi=0.05)
    cases.append((w.centers, w.radii, TOLMX))
    for C, R, tol in cases:
        ctx = sps.Context(p=p, precision=1)
        ctx.set_geometry(dev(C), dev(R))
        sig = rng.standard_normal((len(R) * P, 3))
        if len(R) > 1:
            tg = [0, 77, 128, 199]
            sus = Suspension(C, R, p)
            sl = np.concatenate([np.arange(i * P, (i + 1) * P) for i in tg])
        else:
            tg, sus, sl = None, Suspension(C, R, p), slice(None)
        for op, key in ((sps.SPS_OP_S, "S"), (sps.SPS_OP_K, "K")):
            out = ctx.layer_apply(op, planes(sig)).cpu().numpy().T[sl]
            ref = np.asarray(sus.apply(key, sig, targets=tg)).reshape(-1, 3)[sl]
            assert relerr(out, ref) < tol, (p, len(R), key)


# ---------------------------------------------------------------------------
# mobility
# ---------------------------------------------------------------------------
def test_single_sphere_drag(sps):
    ctx = sps.Context(p=6, gmres_tol=1e-13)
    FT = np.array([[0.3, -1.0, 0.5, 0.2, 0.7, -0.4]])
    for a in (1.0, 0.6):
        U = ctx.mobility_apply(dev([[1.0, 2.0, -3.0]]), dev([a]), dev(FT)).cpu().numpy()
        assert np.abs(U[0, :3] - FT[0, :3] / (6 * pi * a)).max() < 1e-13
        assert np.abs(U[0, 3:] - FT[0, 3:] / (8 * pi * a ** 3)).max() < 1e-13 / a ** 3


@pytest.mark.parametrize("case", ["c1", "c2", "c3"])
def test_mobility_tiny_fp64(sps, case):
    d = load("tiny_layers.npz")
    C, R, p = d[f"{case}_centers"], d[f"{case}_radii"], int(d[f"{case}_p"])
    ctx = sps.Context(p=p, gmres_tol=1e-13, gmres_max=300)
    U = ctx.mobility_apply(dev(C), dev(R), dev(d[f"{case}_FT"])).cpu().numpy()
    assert relerr(U, d[f"{case}_U"]) < TOL64


@pytest.mark.parametrize("case", ["c1", "c3"])
def test_mobility_tiny_mixed(sps, case):
    d = load("tiny_layers.npz")
    C, R, p = d[f"{case}_centers"], d[f"{case}_radii"], int(d[f"{case}_p"])
    ctx = sps.Context(p=p, gmres_tol=1e-9, gmres_max=300, precision=1)
    U = ctx.mobility_apply(dev(C), dev(R), dev(d[f"{case}_FT"])).cpu().numpy()
    assert relerr(U, d[f"{case}_U"]) < TOLMX
    # refinement against an FP64-accurate residual recovers the FP64 answer,
    # with that residual's far field in double-float (ir_dw = 1) or in FP64
    for ir_dw in (1, 0):
        ctx = sps.Context(p=p, gmres_tol=1e-7, gmres_max=300, precision=1, ir_tol=1e-13, ir_dw=ir_dw)
        U = ctx.mobility_apply(dev(C), dev(R), dev(d[f"{case}_FT"])).cpu().numpy()
        assert relerr(U, d[f"{case}_U"]) < 1e-10, ir_dw
        assert ctx.last_stats["ir_sweeps"] >= 1


def test_zero_force_and_nonfinite(sps):
    ctx = sps.Context(p=4)
    C = dev([[0, 0, 0], [3.0, 0, 0]])
    R = dev([1.0, 1.0])
    U = ctx.mobility_apply(C, R, dev(np.zeros((2, 6)))).cpu().numpy()
    assert not U.any() and ctx.last_stats["gmres_iters"] == 0
    bad = np.zeros((2, 6))
    bad[0, 0] = np.nan
    with pytest.raises(sps.SPSError) as e:
        ctx.mobility_apply(C, R, dev(bad))
    assert e.value.code == 8


# ---------------------------------------------------------------------------
# collision-resolved step
# ---------------------------------------------------------------------------
def _check_step(d, gamma, U, pos_new, tol):
    q = d["q"]
    gref = d["gamma"]
    if np.abs(gref).max() > 0:
        assert relerr(gamma, gref) < tol
    else:
        assert np.abs(gamma).max() <= tol * max(np.abs(q).max(), 1.0)
    assert relerr(U, d["U"]) < tol
    assert np.abs(pos_new - d["centers_new"]).max() < tol * np.abs(d["U"]).max() * float(d["dt"]) + 1e-15


@pytest.mark.parametrize("name,acs", [("cfg1_step.npz", 1.0), ("active_step_p4.npz", 1.05)])
def test_step_fp64(sps, name, acs):
    d = load(name)
    p = int(d["p"])
    # cold GMRES starts, as in the oracle: the BBPGD iterates then follow the
    # oracle's path (near-touching spheres at p = 4 make M only approximately SPD)
    ctx = sps.Context(p=p, delta=0.1, a_c_scale=acs, gmres_tol=1e-13, gmres_max=300,
                      bbpgd_tol=1e-12, warm_start=0)
    gam, U, pn = ctx.resolve_collisions(dev(d["centers"]), dev(d["radii"]), dev(d["FT"]),
                                        float(d["dt"]))
    st = ctx.last_stats
    assert st["n_contacts"] == len(d["ij"]) and st["n_active"] == int(d["n_active"])
    assert st["bbpgd_iters"] == int(d["bbpgd_iters"])
    _check_step(d, gam.cpu().numpy(), U.cpu().numpy(), pn.cpu().numpy(), TOL64)


@pytest.mark.parametrize("jmax", [2, 7])
def test_capped_step_returns_oracle_best_iterate(sps, jmax):
    """Algorithm 1 capped at j_max = 2 and 7 on the five-sphere active step:
    the library ends with NOT_CONVERGED and returns the iterate of smallest
    min-map residual with its own M D gamma, which is not the last iterate
    at either cap; the oracle's failure rule (keep_best) gives the same
    gamma and U (FP64 path, 1e-10)."""
    d = load("active_step_p4.npz")
    c = load("capped_step_p4.npz")
    assert int(c[f"best_{jmax}"]) < jmax
    ctx = sps.Context(p=int(d["p"]), delta=0.1, a_c_scale=1.05, gmres_tol=1e-13, gmres_max=300,
                      bbpgd_tol=1e-12, bbpgd_max=jmax, warm_start=0)
    gam, U, _ = ctx.resolve_collisions(dev(d["centers"]), dev(d["radii"]), dev(d["FT"]),
                                       float(d["dt"]), allow=(4,))
    st = ctx.last_stats
    assert st["status"] == 4 and st["bbpgd_iters"] == jmax
    assert abs(st["final_phi"] - float(c[f"phi_{jmax}"])) <= 1e-10 * float(c[f"phi_{jmax}"])
    assert relerr(gam.cpu().numpy(), c[f"gamma_{jmax}"]) < TOL64
    assert relerr(U.cpu().numpy(), c[f"U_{jmax}"]) < TOL64


def test_step_mixed_and_host_api(sps):
    d = load("active_step_p4.npz")
    p = int(d["p"])
    # an FP32 far field puts ~1e-7 relative noise on M gamma: eps_tol 1e-6 is reachable
    kw = dict(p=p, delta=0.1, a_c_scale=1.05, gmres_tol=1e-9, gmres_max=300, bbpgd_tol=1e-6,
              precision=1, warm_start=0)
    ctx = sps.Context(**kw)
    gam, U, pn = ctx.resolve_collisions(dev(d["centers"]), dev(d["radii"]), dev(d["FT"]),
                                        float(d["dt"]))
    _check_step(d, gam.cpu().numpy(), U.cpu().numpy(), pn.cpu().numpy(), TOLMX)
    n = len(d["radii"])
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).pin_memory()
    g_h = torch.zeros(64, dtype=torch.float64).pin_memory()
    U_h = torch.zeros(n, 6, dtype=torch.float64).pin_memory()
    p_h = torch.zeros(n, 3, dtype=torch.float64).pin_memory()
    nc = ctx.resolve_collisions_host(pin(d["centers"]), pin(d["radii"]), pin(d["FT"]),
                                     float(d["dt"]), g_h, U_h, p_h)
    assert nc == len(d["ij"])
    assert np.array_equal(g_h[:nc].numpy(), gam.cpu().numpy())
    assert np.array_equal(U_h.numpy(), U.cpu().numpy())


def test_step_capacity_and_single_sphere(sps):
    d = load("active_step_p4.npz")
    ctx = sps.Context(p=4, delta=0.1, a_c_scale=1.05)
    with pytest.raises(sps.SPSError) as e:
        ctx.resolve_collisions(dev(d["centers"]), dev(d["radii"]), dev(d["FT"]), 0.05, gamma_cap=2)
    assert e.value.code == 6
    gam, U, pn = ctx.resolve_collisions(dev([[0.0, 0, 0]]), dev([1.0]),
                                        dev([[0, 0, -1.0, 0, 0, 0]]), 0.1)
    assert len(gam) == 0
    assert abs(U[0, 2].item() + 1 / (6 * pi)) < 1e-12


def test_warm_start_matches_cold(sps):
    """GMRES warm starts (previous solution as initial guess) change only the
    Krylov path: the converged step agrees with the cold-start step."""
    d = load("tiny_layers.npz")
    C, R, p = d["c1_centers"], d["c1_radii"], int(d["c1_p"])
    FT = 5.0 * d["c1_FT"]
    out = {}
    for warm in (0, 1):
        ctx = sps.Context(p=p, delta=0.3, a_c_scale=1.02, gmres_tol=1e-12, gmres_max=300,
                          bbpgd_tol=1e-10, warm_start=warm, bb_safeguard=1)
        pos = dev(C)
        for k in range(2):                 # second step: U_nc warm-started from step 1
            gam, U, pn = ctx.resolve_collisions(pos, dev(R), dev(FT), 0.05)
            pos = pn.clone()
        out[warm] = (gam.cpu().numpy(), U.cpu().numpy(), ctx.last_stats)
    assert relerr(out[1][1], out[0][1]) < 1e-8
    if np.abs(out[0][0]).max() > 0:
        assert relerr(out[1][0], out[0][0]) < 1e-6
    assert out[1][2]["gmres_iters"] < out[0][2]["gmres_iters"]


def test_bbpgd_cap_returns_consistent_best_iterate(sps):
    """With the BBPGD cap hit (NOT_CONVERGED) the step returns the iterate of
    smallest min-map residual together with its own M D gamma: U - U_nc equals
    the mobility of D gamma, and the reported residual is that of gamma."""
    d = load("active_step_p4.npz")
    p = int(d["p"])
    ctx = sps.Context(p=p, delta=0.1, a_c_scale=1.05, gmres_tol=1e-12, gmres_max=300, bbpgd_tol=1e-12,
                      bbpgd_max=3, warm_start=0)
    C, R, FT = dev(d["centers"]), dev(d["radii"]), dev(d["FT"])
    gam, U, _ = ctx.resolve_collisions(C, R, FT, float(d["dt"]), allow=(4,))
    st = dict(ctx.last_stats)
    assert st["status"] == 4 and st["bbpgd_iters"] == 3
    n = len(d["radii"])
    Fc = ctx.contact_force(gam.contiguous(), n)
    Uc = ctx.mobility_apply(C, R, Fc)
    Unc = ctx.mobility_apply(C, R, FT)
    assert relerr((U - Unc).cpu().numpy(), Uc.cpu().numpy()) < 1e-9
    q = d["phi"] / float(d["dt"]) + ctx.contact_rate(Unc).cpu().numpy()
    g = ctx.contact_rate(Uc).cpu().numpy() + q
    phi = np.linalg.norm(np.minimum(gam.cpu().numpy(), g))
    assert abs(phi - st["final_phi"]) < 1e-8 * max(phi, 1.0)
