"""Randomly oriented sphere grids (Sec. 5.4) on the CUDA path, against the
FP64 oracle's Suspension(rotations=Q).

Node k of sphere i sits at c_i + a_i Q_i n_k; the VSH self and near terms work
in each sphere's frame.  Stored oracle values: tests/golden/rotated_p4.npz
(make_golden.py, oracle only).  Tolerances as everywhere: FP64 and the
double-float path 1e-10, mixed 1e-5 (max-norm relative to the largest entry)."""
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")


@pytest.fixture(scope="module")
def sps():
    from paper_1909_06623_gb300 import build
    build.build()
    import paper_1909_06623_gb300 as m
    return m


@pytest.fixture(scope="module")
def gold():
    return np.load(os.path.join(GOLD, "rotated_p4.npz"))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def relerr(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


def _case(gold, c):
    return (gold[f"{c}_centers"], gold[f"{c}_radii"], int(gold[f"{c}_p"]), gold[f"{c}_Q"])


@pytest.mark.parametrize("c", ["c1", "c3"])
def test_oriented_nodes_match_oracle(sps, gold, c):
    C, R, p, Q = _case(gold, c)
    ctx = sps.Context(p=p)
    ctx.set_orientation(dev(Q))
    ctx.set_geometry(dev(C), dev(R))
    X, Nr, _ = ctx.nodes()
    assert relerr(X.cpu().numpy().T, gold[f"{c}_X"]) < 1e-14
    nrm = (gold[f"{c}_X"] - np.repeat(C, len(X[0]) // len(R), axis=0)) / np.repeat(R, len(X[0]) // len(R))[:, None]
    assert np.abs(Nr.cpu().numpy().T - nrm).max() < 1e-13


@pytest.mark.parametrize("c", ["c1", "c3"])
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5), (2, 1e-10)])
def test_oriented_layer_operators_match_oracle(sps, gold, c, precision, tol):
    C, R, p, Q = _case(gold, c)
    ctx = sps.Context(p=p, precision=precision)
    ctx.set_orientation(dev(Q))
    ctx.set_geometry(dev(C), dev(R))
    s = dev(gold[f"{c}_sigma"].T)
    for op, key in ((sps.SPS_OP_S, "S"), (sps.SPS_OP_K, "K"), (sps.SPS_OP_A, "A")):
        out = ctx.layer_apply(op, s).cpu().numpy().T
        assert relerr(out, gold[f"{c}_{key}"]) < tol, (c, key, precision)


@pytest.mark.parametrize("c", ["c1", "c3"])
def test_oriented_mobility_matches_oracle(sps, gold, c):
    C, R, p, Q = _case(gold, c)
    for precision, tol, gtol in ((0, 1e-10, 1e-13), (1, 1e-5, 1e-9)):
        ctx = sps.Context(p=p, precision=precision, gmres_tol=gtol, gmres_max=300)
        ctx.set_orientation(dev(Q))
        U = ctx.mobility_apply(dev(C), dev(R), dev(gold[f"{c}_FT"])).cpu().numpy()
        assert relerr(U, gold[f"{c}_U"]) < tol, precision


def test_identity_orientation_changes_nothing(sps, gold):
    """Identity rotations reproduce the unrotated operators to the bit (their
    zero products vanish exactly), in FP64 and in the mixed path."""
    C, R, p, _ = _case(gold, "c1")
    s = dev(gold["c1_sigma"].T)
    eye = dev(np.tile(np.eye(3), (len(R), 1, 1)))
    for precision in (0, 1):
        outs = []
        for Q in (None, eye):
            ctx = sps.Context(p=p, precision=precision)
            if Q is not None:
                ctx.set_orientation(Q)
            ctx.set_geometry(dev(C), dev(R))
            outs.append([ctx.layer_apply(op, s) for op in (sps.SPS_OP_S, sps.SPS_OP_K)])
        for a, b in zip(*outs):
            assert torch.equal(a, b), precision


def test_oriented_collision_step_and_simulate(sps, gold):
    """The five-sphere active step with randomly oriented grids against the
    oracle step (FP64, 1e-10); sps_simulate keeps the orientation from step
    to step (two steps equal two single steps on a fresh context)."""
    d = np.load(os.path.join(GOLD, "active_step_p4.npz"))
    Q = dev(gold["step_Q"])
    kw = dict(p=int(d["p"]), delta=0.1, a_c_scale=1.05, gmres_tol=1e-13, gmres_max=300,
              bbpgd_tol=1e-12, warm_start=0)
    ctx = sps.Context(**kw)
    ctx.set_orientation(Q)
    gam, U, pn = ctx.resolve_collisions(dev(d["centers"]), dev(d["radii"]), dev(d["FT"]),
                                        float(d["dt"]))
    assert ctx.last_stats["n_active"] == int(gold["step_n_active"])
    assert relerr(gam.cpu().numpy(), gold["step_gamma"]) < 1e-10
    assert relerr(U.cpu().numpy(), gold["step_U"]) < 1e-10
    disp = gold["step_centers_new"] - d["centers"]
    assert np.abs((pn.cpu().numpy() - d["centers"]) - disp).max() < 1e-10 * np.abs(disp).max()
    # two steps through sps_simulate vs two single steps
    pos = dev(d["centers"])
    c2 = sps.Context(**kw)
    c2.set_orientation(Q)
    _, U2, st = c2.simulate(pos, dev(d["radii"]), dev(d["FT"]), float(d["dt"]), 2)
    assert len(st) == 2
    c3 = sps.Context(**kw)
    c3.set_orientation(Q)
    p1 = dev(d["centers"])
    for _ in range(2):
        _, U3, po = c3.resolve_collisions(p1, dev(d["radii"]), dev(d["FT"]), float(d["dt"]))
        p1 = po.clone()
    assert relerr(U2.cpu().numpy(), U3.cpu().numpy()) < 1e-12
    assert relerr(pos.cpu().numpy(), p1.cpu().numpy()) < 1e-14


def test_orientation_argument_checks(sps, gold):
    C, R, p, Q = _case(gold, "c1")
    ctx = sps.Context(p=p)
    bad = Q.copy()
    bad[0, 0, 0] += 1e-6
    with pytest.raises(sps.SPSError):
        ctx.set_orientation(dev(bad))
    refl = Q.copy()
    refl[1] = -refl[1]
    with pytest.raises(sps.SPSError):
        ctx.set_orientation(dev(refl))
    ctx.set_orientation(dev(Q))
    with pytest.raises(sps.SPSError):              # another sphere count
        ctx.set_geometry(dev(C[:-1]), dev(R[:-1]))
    with pytest.raises(sps.SPSError):              # no adjoint of oriented grids
        ctx.mobility_adjoint(dev(C), dev(R), dev(gold["c1_FT"]), dev(gold["c1_FT"]))
    ctx.set_orientation(None)
    ctx.set_geometry(dev(C[:-1]), dev(R[:-1]))
