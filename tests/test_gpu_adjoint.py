"""GPU adjoint of the mobility solve, through the C ABI.

* transpose identities <w, Op v> = <Op^T w, v> for S, K and I/2+K+L (tiny
  polydisperse cases with close pairs and the full 1,000-sphere geometry);
* dL/dF for L = sum |U|^2 against the oracle's exact 2 M^T U (assembled
  mobility) and against central differences of the GPU forward solve;
* dL/dc (sphere centres) against central differences of the GPU and of the
  oracle forward solve, on coordinates whose near pairs stay away from the
  beta (a_i + a_j) threshold.
Tolerance for gradients: 1e-4 relative (FP64 path), as stated for the adjoint.
"""
import os

import numpy as np
import pytest
import torch

from oracle import adjoint as oadj

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


def _transpose_gap(ctx, sps, op, NP, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    v = torch.randn(3, NP, dtype=torch.float64, device="cuda", generator=g)
    w = torch.randn(3, NP, dtype=torch.float64, device="cuda", generator=g)
    Av = ctx.layer_apply(op, v)
    ATw = ctx.layer_apply_transpose(op, w)
    lhs = torch.sum(w * Av).item()
    rhs = torch.sum(ATw * v).item()
    scale = (torch.linalg.norm(w) * torch.linalg.norm(Av)).item()
    return abs(lhs - rhs) / scale


@pytest.mark.parametrize("case", ["c1", "c2", "c3"])
def test_transpose_identities_tiny(sps, case):
    d = np.load(os.path.join(GOLD, "tiny_layers.npz"))
    C, R, p = d[f"{case}_centers"], d[f"{case}_radii"], int(d[f"{case}_p"])
    ctx = sps.Context(p=p)
    ctx.set_geometry(dev(C), dev(R))
    NP = len(R) * (p + 1) * (2 * p + 2)
    for op in (sps.SPS_OP_S, sps.SPS_OP_K, sps.SPS_OP_A):
        assert _transpose_gap(ctx, sps, op, NP, 3 + op) < 1e-13, op


def test_transpose_identities_cfg2(sps):
    d = np.load(os.path.join(GOLD, "cfg2_sample.npz"))
    p = int(d["p"])
    ctx = sps.Context(p=p)
    ctx.set_geometry(dev(d["centers"]), dev(d["radii"]))
    NP = len(d["radii"]) * (p + 1) * (2 * p + 2)
    for op in (sps.SPS_OP_S, sps.SPS_OP_K, sps.SPS_OP_A):
        assert _transpose_gap(ctx, sps, op, NP, 11 + op) < 1e-12, op


def _case3():
    C = np.array([[0.0, 0.0, 0.0], [2.3, 0.4, 0.1], [0.6, 2.2, -0.5]])
    R = np.array([1.0, 0.8, 0.9])
    FT = np.array([[0.3, -0.5, 1.0, 0.1, 0.0, 0.2], [-0.2, 0.4, 0.1, 0.0, 0.3, 0.0],
                   [0.1, 0.1, -0.6, -0.2, 0.0, 0.1]])
    return C, R, FT


def test_force_gradient_matches_oracle_exact(sps):
    C, R, FT = _case3()
    p = 4
    ref = oadj.grad_F_exact(C, R, FT, p)
    ctx = sps.Context(p=p, gmres_tol=1e-13, gmres_max=400)
    U = ctx.mobility_apply(dev(C), dev(R), dev(FT))
    _, gF, _ = ctx.mobility_adjoint(dev(C), dev(R), dev(FT), 2.0 * U, want_pos=False)
    g = gF.cpu().numpy()
    assert np.abs(g - ref).max() < 1e-9 * np.abs(ref).max()


def test_force_gradient_fd_polydisperse(sps):
    """A larger case with close pairs: dL/dF against central differences of the
    GPU forward solve (L is quadratic in F, so differences are exact up to
    rounding)."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.tiny(21, 12, 5, phi=0.15, n_pairs=2, gap=0.01)
    ctx = sps.Context(p=5, gmres_tol=1e-13, gmres_max=400)
    pos, rad, FT = dev(w.centers), dev(w.radii), dev(w.FT)
    U = ctx.mobility_apply(pos, rad, FT)
    _, gF, _ = ctx.mobility_adjoint(pos, rad, FT, 2.0 * U, want_pos=False)
    h = 1e-3
    for i, k in ((0, 0), (3, 2), (7, 4), (11, 5)):
        vals = []
        for s in (1, -1):
            F2 = FT.clone()
            F2[i, k] += s * h
            Ui = ctx.mobility_apply(pos, rad, F2)
            vals.append(torch.sum(Ui * Ui).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gF[i, k].item()) < 1e-7 * gF.abs().max().item(), (i, k)


def _fd_gpu(ctx, pos, rad, FT, i, k, h):
    vals = []
    for s in (1, -1):
        p2 = pos.clone()
        p2[i, k] += s * h
        U = ctx.mobility_apply(p2, rad, FT)
        vals.append(torch.sum(U * U).item())
    return (vals[0] - vals[1]) / (2 * h)


def test_centre_gradient_fd_gpu(sps):
    """dL/dc against central differences of the GPU FP64 forward solve on a
    polydisperse case with near pairs (no pair within 10 h of the beta
    threshold, so the near lists are the same at c +- h)."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.tiny(21, 12, 5, phi=0.15, n_pairs=2, gap=0.01)
    h = 1e-5
    assert oadj.near_margin(w.centers, w.radii) > 20 * h
    ctx = sps.Context(p=5, gmres_tol=1e-13, gmres_max=400)
    pos, rad, FT = dev(w.centers), dev(w.radii), dev(w.FT)
    U = ctx.mobility_apply(pos, rad, FT)
    _, gF, gx = ctx.mobility_adjoint(pos, rad, FT, 2.0 * U)
    scale = gx.abs().max().item()
    for i, k in ((0, 0), (2, 1), (5, 2), (8, 0), (11, 1)):
        fd = _fd_gpu(ctx, pos, rad, FT, i, k, h)
        assert abs(fd - gx[i, k].item()) < 1e-4 * scale, (i, k, fd, gx[i, k].item())
    # translation invariance: the centre gradients sum to zero
    assert gx.sum(dim=0).abs().max().item() < 1e-9 * scale


def test_centre_gradient_matches_oracle_fd(sps):
    C, R, FT = _case3()
    p = 4
    h = 1e-5
    assert oadj.near_margin(C, R) > 20 * h
    coords = [("c", 0, 0), ("c", 1, 1), ("c", 2, 2)]
    ref = oadj.grad_fd(C, R, FT, p, coords, h=h)
    ctx = sps.Context(p=p, gmres_tol=1e-13, gmres_max=400)
    U = ctx.mobility_apply(dev(C), dev(R), dev(FT))
    _, _, gx = ctx.mobility_adjoint(dev(C), dev(R), dev(FT), 2.0 * U)
    got = np.array([gx[i, k].item() for _, i, k in coords])
    assert np.abs(got - ref).max() < 1e-4 * np.abs(gx.cpu().numpy()).max()


def test_autograd_function(sps):
    """torch.autograd through MobilityFunction equals the direct adjoint call."""
    C, R, FT = _case3()
    ctx = sps.Context(p=4, gmres_tol=1e-13, gmres_max=400)
    pos = dev(C).requires_grad_(True)
    F = dev(FT).requires_grad_(True)
    U = sps.mobility(pos, dev(R), F, ctx)
    L = (U * U).sum()
    L.backward()
    U2 = ctx.mobility_apply(dev(C), dev(R), dev(FT))
    _, gF, gx = ctx.mobility_adjoint(dev(C), dev(R), dev(FT), 2.0 * U2)
    assert torch.allclose(F.grad, gF, rtol=1e-10, atol=1e-14)
    assert torch.allclose(pos.grad, gx, rtol=1e-10, atol=1e-14)


def test_mixed_adjoint_close_to_fp64(sps):
    """The mixed-precision adjoint (FP32 transposed far sums, FP64 near and
    Krylov) agrees with the FP64 adjoint to the mixed-path tolerance."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.tiny(21, 12, 5, phi=0.15, n_pairs=2, gap=0.01)
    pos, rad, FT = dev(w.centers), dev(w.radii), dev(w.FT)
    out = {}
    for prec, tol in ((0, 1e-13), (1, 1e-9)):
        ctx = sps.Context(p=5, gmres_tol=tol, gmres_max=400, precision=prec)
        U = ctx.mobility_apply(pos, rad, FT)
        out[prec] = ctx.mobility_adjoint(pos, rad, FT, 2.0 * U)
        if prec == 1:
            NP = len(w.radii) * 72
            ctx.set_geometry(pos, rad)
            for op in (sps.SPS_OP_S, sps.SPS_OP_K, sps.SPS_OP_A):
                assert _transpose_gap(ctx, sps, op, NP, 5 + op) < 2e-6, op
    for k in (1, 2):
        a, b = out[1][k], out[0][k]
        assert ((a - b).abs().max() / b.abs().max()).item() < 1e-4


def test_cfg4_gradient_finite_differences(sps):
    """1,000 unit spheres at volume fraction 0.25, p = 6, L = sum |U|^2.
    Gradients dL/dF and dL/dc: the mixed-precision adjoint (FP32 transposed
    far sums) against the FP64-class adjoint (double-float forward far field,
    FP64 transposed sums and adjoint GMRES), and both against central
    differences (h = 1e-6) on 32 seeded coordinates (16 forces, 16 centre
    components whose near pairs stay 100 h away from the beta threshold).
    The 64 forward solves of the differences run on the mixed path refined to
    a relative FP64-accurate residual of 1e-12 (double-float far field).
    Bar: 1e-4 of the gradient's largest entry."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.config4()
    pos, rad, FT = dev(w.centers), dev(w.radii), dev(w.FT)
    cdw = sps.Context(p=6, gmres_tol=1e-12, gmres_max=400, precision=sps.SPS_FP64_DW)
    U = cdw.mobility_apply(pos, rad, FT)
    _, gF, gx = cdw.mobility_adjoint(pos, rad, FT, 2.0 * U)
    cmx = sps.Context(p=6, gmres_tol=1e-8, gmres_max=400, precision=1)
    Um = cmx.mobility_apply(pos, rad, FT)
    _, gFm, gxm = cmx.mobility_adjoint(pos, rad, FT, 2.0 * Um)
    mixed_vs_dw = [((a - b).abs().max() / b.abs().max()).item() for a, b in ((gFm, gF), (gxm, gx))]
    assert max(mixed_vs_dw) < 1e-4, mixed_vs_dw
    rng = np.random.default_rng(workloads.SEED_BASE + 40)
    h = 1e-6
    coords = [("F", int(i), int(k)) for i, k in zip(rng.choice(w.N, 16), rng.integers(0, 6, 16))]
    picked = 0
    for i in rng.permutation(w.N):
        d = np.linalg.norm(w.centers - w.centers[i], axis=1)
        t = np.abs(d - 1.75 * (w.radii + w.radii[i]))
        t[i] = np.inf
        if t.min() > 100 * h:
            coords.append(("c", int(i), int(rng.integers(0, 3))))
            picked += 1
        if picked == 16:
            break
    cfd = sps.Context(p=6, gmres_tol=1e-7, gmres_max=400, precision=1, ir_tol=1e-12, ir_max=12)
    errs, errs_m = [], []
    for kind, i, k in coords:
        vals = []
        for sgn in (1, -1):
            p2, F2 = pos.clone(), FT.clone()
            if kind == "F":
                F2[i, k] += sgn * h
            else:
                p2[i, k] += sgn * h
            Ui = cfd.mobility_apply(p2, rad, F2)
            assert cfd.last_stats["gmres_res_max"] < 1e-12
            vals.append(torch.sum(Ui * Ui).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        g, gm = (gF, gFm) if kind == "F" else (gx, gxm)
        errs.append(abs(fd - g[i, k].item()) / g.abs().max().item())
        errs_m.append(abs(fd - gm[i, k].item()) / gm.abs().max().item())
    print(f"cfg4: mixed vs FP64-class adjoint {max(mixed_vs_dw):.2e}; central differences vs "
          f"FP64-class adjoint {max(errs):.2e}, vs mixed adjoint {max(errs_m):.2e}")
    assert max(errs) < 1e-4 and max(errs_m) < 1e-4


# ---------------------------------------------------------------------------
# the collision-resolved step, differentiated in F_ext on the active set
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_collision_adjoint_identity(sps, seed):
    """Identity mobility: GPU dL/dF against the oracle's active-set formula
    with M = I (on the oracle's own step) and central differences of the
    oracle step (pinned in tests/test_oracle_adjoint_lcp.py)."""
    from oracle import adjoint as oadj
    from paper_1909_06623_gb300 import workloads
    w = workloads.contact_chain(seed)
    L0, out = oadj.step_loss(w.centers, w.radii, w.FT, w.dt, 0, identity=True)
    N = w.N
    D = oadj.D_matrix(N, out["ij"], out["normals"])
    ref, A = oadj.collision_grad_F(np.eye(6 * N), D, out["gamma"], 2.0 * out["U"])
    ctx = sps.Context(p=2, delta=0.1, mobility=sps.SPS_MOB_IDENTITY, bbpgd_tol=1e-12, gmres_tol=1e-12)
    U, gF, gx = ctx.collision_adjoint(dev(w.centers), dev(w.radii), dev(w.FT), w.dt,
                                      dev(2.0 * out["U"]), want_pos=True)
    st = ctx.last_stats
    assert st["n_active"] == int(A.sum())
    assert np.abs(U.cpu().numpy() - out["U"]).max() < 1e-10 * np.abs(out["U"]).max()
    assert np.abs(gF.cpu().numpy() - ref).max() < 1e-9 * np.abs(ref).max()
    # centres: the identity mobility does not depend on them, so only the
    # contact geometry contributes (pinned against central differences)
    refx, _ = oadj.collision_grad_c_contacts(np.eye(6 * N), D, out["gamma"], 2.0 * out["U"], out["U"],
                                             w.centers, out["ij"], out["normals"], w.dt)
    assert np.abs(gx.cpu().numpy() - refx).max() < 1e-9 * np.abs(refx).max()


@pytest.fixture(scope="module")
def collision_golden():
    d = np.load(os.path.join(GOLD, "collision_grad_p4.npz"))
    return d


@pytest.mark.parametrize("precision,tol", [(0, 1e-4), (1, 1e-4)])
def test_collision_adjoint_bie(sps, collision_golden, precision, tol):
    """Five spheres at p = 4 with three active contacts: GPU dL/dF (L = sum
    |U|^2, dL/dU = 2U of the GPU step) against the oracle's active-set formula
    with its assembled mobility and against central differences of the full
    oracle step, 1e-4 relative (the adjoint bar)."""
    from oracle import adjoint as oadj
    d = collision_golden
    N = len(d["radii"])
    D = oadj.D_matrix(N, d["ij"], d["normals"])
    ref, A = oadj.collision_grad_F(d["M"], D, d["gamma"], 2.0 * d["U"])
    ctx = sps.Context(p=int(d["p"]), delta=0.1, a_c_scale=float(d["a_c_scale"]),
                      gmres_tol=1e-13 if precision == 0 else 1e-9, gmres_max=300,
                      bbpgd_tol=1e-12 if precision == 0 else 1e-6, precision=precision, warm_start=0)
    pos, rad, FT = dev(d["centers"]), dev(d["radii"]), dev(d["FT"])
    U, _, _ = ctx.collision_adjoint(pos, rad, FT, float(d["dt"]), dev(2.0 * d["U"]))
    U, gF, gx = ctx.collision_adjoint(pos, rad, FT, float(d["dt"]), 2.0 * U, want_pos=True)
    assert ctx.last_stats["n_active"] == int(A.sum())
    g = gF.cpu().numpy()
    assert np.abs(g - ref).max() < tol * np.abs(ref).max()
    for (i, k), fd in zip(d["coords"], d["fd"]):
        assert abs(g[i, k] - fd) < tol * np.abs(ref).max(), (i, k)
    # centres: central differences of the full oracle step
    dc = np.load(os.path.join(GOLD, "collision_grad_c_p4.npz"))
    gxx = gx.cpu().numpy()
    scale = np.abs(dc["fd"]).max()
    for (i, k), fd in zip(dc["coords"], dc["fd"]):
        assert abs(gxx[i, k] - fd) < tol * scale, (i, k, gxx[i, k], fd)
    assert np.abs(gxx.sum(axis=0)).max() < 1e-6 * np.abs(gxx).max()   # translation invariance


def test_collision_step_autograd(sps):
    """torch.autograd through the collision step matches the adjoint calls."""
    from paper_1909_06623_gb300 import workloads
    w = workloads.contact_chain(2)
    ctx = sps.Context(p=2, delta=0.1, mobility=sps.SPS_MOB_IDENTITY, bbpgd_tol=1e-12, gmres_tol=1e-12)
    pos = dev(w.centers).requires_grad_(True)
    FT = dev(w.FT).requires_grad_(True)
    U = sps.collision_step(pos, dev(w.radii), FT, w.dt, ctx)
    (U * U).sum().backward()
    U2, gF, gx = ctx.collision_adjoint(dev(w.centers), dev(w.radii), dev(w.FT), w.dt, 2.0 * U.detach(),
                                       want_pos=True)
    assert torch.allclose(FT.grad, gF, rtol=1e-12, atol=0)
    assert torch.allclose(pos.grad, gx, rtol=1e-12, atol=0)
