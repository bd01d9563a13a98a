"""Writes the oracle reference files used by the GPU parity tests.

Calls only the CPU oracle (oracle/) and the seeded input generators
(paper_1909_06623_gb300.workloads); every stored expected value is an oracle
output.  Each file also stores its inputs, so the tests feed the CUDA path
exactly what the oracle saw.

    python tests/golden/make_golden.py            # all files
    python tests/golden/make_golden.py cfg1       # one file
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import adjoint, lcp, mobility, sph  # noqa: E402
from oracle.layer import Suspension  # noqa: E402
from paper_1909_06623_gb300 import workloads  # noqa: E402


def _step(name, C, R, FT, dt, p, **kw):
    out = lcp.resolve_collisions(C, R, FT, dt, p, **kw)
    info = out["info"]
    np.savez_compressed(
        os.path.join(HERE, name + ".npz"), centers=C, radii=R, FT=FT, dt=dt, p=p,
        params=np.array([kw.get("beta", 1.75), kw.get("delta", 0.1), kw.get("a_c_scale", 1.0),
                         kw["gmres_tol"], kw["bbpgd_tol"]]),
        ij=out["ij"], phi=out["phi"], normals=out["normals"], gamma=out["gamma"], q=out["q"],
        U=out["U"], U_nc=out["U_nc"], centers_new=out["centers_new"],
        n_active=info["n_active"], bbpgd_iters=info["iters"])
    print(name, info)


def cfg1():
    """Config 1: 8 unit spheres, p = 8, one step (FP64 parity)."""
    w = workloads.config1()
    _step("cfg1_step", w.centers, w.radii, w.FT, w.dt, w.p, delta=0.1, gmres_tol=1e-13,
          bbpgd_tol=1e-12)


def active():
    """Five spheres pushed together: several active contacts, p = 4."""
    C = np.array([[0, 0, 0], [2.02, 0.1, 0], [1.0, 1.78, 0.05], [4.1, 0.3, 0.2],
                  [1.1, 0.6, 1.85]])
    R = np.array([1.0, 1.0, 0.95, 1.0, 0.8])
    FT = np.zeros((5, 6))
    FT[:, :3] = 20.0 * np.array([[1.0, 0.3, 0.2], [-1.0, 0.2, 0.0], [0.0, -1.0, 0.1],
                                 [-0.9, 0, 0], [0.1, 0.0, -1.0]])
    FT[:, 3:] = [[0.5, 0, 0], [0, 0, 0], [0, 0.3, 0], [0, 0, 0], [0, 0, -0.4]]
    _step("active_step_p4", C, R, FT, 0.05, 4, delta=0.1, a_c_scale=1.05, gmres_tol=1e-13,
          bbpgd_tol=1e-12)


def capped():
    """The five-sphere active step with Algorithm 1 capped at j_max = 2 and 7
    under the failure rule (keep_best): at both caps the last iterate is not
    the one of smallest residual (residuals 2.47, 0.968, 1.002, ...; iterate
    6 at 3.6e-3, iterate 7 at 6.8e-3)."""
    d = np.load(os.path.join(HERE, "active_step_p4.npz"))
    out = {}
    for jmax in (2, 7):
        r = lcp.resolve_collisions(d["centers"], d["radii"], d["FT"], float(d["dt"]), int(d["p"]),
                                   delta=0.1, a_c_scale=1.05, gmres_tol=1e-13, bbpgd_tol=1e-12,
                                   bbpgd_max=jmax, keep_best=True)
        out[f"gamma_{jmax}"] = r["gamma"]
        out[f"U_{jmax}"] = r["U"]
        out[f"best_{jmax}"] = r["info"]["best"]
        out[f"phi_{jmax}"] = r["info"]["phi"]
        out[f"history_{jmax}"] = np.array(r["info"]["history"])
        print("capped", jmax, r["info"]["status"], r["info"]["best"], r["info"]["history"])
    np.savez_compressed(os.path.join(HERE, "capped_step_p4.npz"), **out)


def cfg2_sample():
    """Config 2 geometry (1,000 spheres, p = 6): contacts, near lists and the
    layer operators S, K, I/2+K+L of a seeded random density on a sample of
    target spheres (the oracle evaluates only those)."""
    w = workloads.config2()
    sus = Suspension(w.centers, w.radii, w.p)
    rng = np.random.default_rng(workloads.SEED_BASE + 20)
    sig = rng.standard_normal((sus.N * sus.P, 3))
    nn = np.array([len(x) for x in sus.near])
    # targets: the sphere with most near neighbours, two close-pair members, random ones
    ij, phi, nrm = lcp.build_contacts(w.centers, w.radii, 0.1)
    tg = [int(np.argmax(nn)), int(ij[np.argmin(phi), 0]), int(ij[np.argmin(phi), 1])]
    tg += [int(x) for x in rng.choice(sus.N, 5, replace=False)]
    tg = sorted(set(tg))
    t0 = time.time()
    S = sus.apply("S", sig, targets=tg)
    K = sus.apply("K", sig, targets=tg)
    A = 0.5 * sig + K + mobility.apply_L(sus, sig)
    sl = np.concatenate([np.arange(i * sus.P, (i + 1) * sus.P) for i in tg])
    np.savez_compressed(os.path.join(HERE, "cfg2_sample.npz"), centers=w.centers, radii=w.radii,
                        FT=w.FT, p=w.p, sigma=sig, targets=np.array(tg), S=S[sl], K=K[sl],
                        A=A[sl], ij=ij, phi=phi, normals=nrm,
                        near_count=nn)
    print("cfg2_sample", tg, f"{time.time() - t0:.1f}s")


def tiny_layers():
    """Small polydisperse cases (p = 3, 4, 5) with close pairs: full operators."""
    out = {}
    for seed, N, p in ((1, 6, 4), (2, 9, 3), (3, 5, 5)):
        w = workloads.tiny(seed, N, p, phi=0.08, gap=5e-3)
        sus = Suspension(w.centers, w.radii, p)
        rng = np.random.default_rng(seed + 100)
        sig = rng.standard_normal((sus.N * sus.P, 3))
        out[f"c{seed}_centers"] = w.centers
        out[f"c{seed}_radii"] = w.radii
        out[f"c{seed}_p"] = p
        out[f"c{seed}_sigma"] = sig
        out[f"c{seed}_S"] = sus.apply("S", sig)
        out[f"c{seed}_K"] = sus.apply("K", sig)
        out[f"c{seed}_A"] = 0.5 * sig + out[f"c{seed}_K"] + mobility.apply_L(sus, sig)
        out[f"c{seed}_FT"] = w.FT
        out[f"c{seed}_U"] = mobility.mobility_apply(sus, w.FT, 1e-13, 300)
    np.savez_compressed(os.path.join(HERE, "tiny_layers.npz"), **out)
    print("tiny_layers")



def crowded():
    """One sphere of radius 4 ringed by 24 of radius 0.5 (p = 4): the large
    source has 1,200 close items.  Full operators S, K, I/2 + K + L."""
    t0 = time.time()
    w = workloads.crowded_shell(4)
    sus = Suspension(w.centers, w.radii, w.p)
    sig = np.random.default_rng(404).standard_normal((sus.N * sus.P, 3))
    K = sus.apply("K", sig)
    np.savez_compressed(os.path.join(HERE, "crowded_p4.npz"), centers=w.centers, radii=w.radii,
                        p=w.p, sigma=sig, S=sus.apply("S", sig), K=K,
                        A=0.5 * sig + K + mobility.apply_L(sus, sig))
    print("crowded", f"{time.time() - t0:.1f}s")


def rotated():
    """Randomly oriented grids (Sec. 5.4, rotations from the seeded generator):
    the tiny cases' operators and mobility, and the five-sphere active step,
    all evaluated by the oracle's Suspension(rotations=Q)."""
    out = {}
    for seed, N, p in ((1, 6, 4), (3, 5, 5)):
        w = workloads.tiny(seed, N, p, phi=0.08, gap=5e-3)
        Q = workloads.random_rotations(workloads.SEED_BASE + 50 + seed, N)
        sus = Suspension(w.centers, w.radii, p, rotations=Q)
        rng = np.random.default_rng(seed + 100)
        sig = rng.standard_normal((sus.N * sus.P, 3))
        out[f"c{seed}_centers"] = w.centers
        out[f"c{seed}_radii"] = w.radii
        out[f"c{seed}_p"] = p
        out[f"c{seed}_Q"] = Q
        out[f"c{seed}_sigma"] = sig
        out[f"c{seed}_X"] = sus.X
        out[f"c{seed}_S"] = sus.apply("S", sig)
        out[f"c{seed}_K"] = sus.apply("K", sig)
        out[f"c{seed}_A"] = 0.5 * sig + out[f"c{seed}_K"] + mobility.apply_L(sus, sig)
        out[f"c{seed}_FT"] = w.FT
        out[f"c{seed}_U"] = mobility.mobility_apply(sus, w.FT, 1e-13, 300)
    d = np.load(os.path.join(HERE, "active_step_p4.npz"))
    Q = workloads.random_rotations(workloads.SEED_BASE + 57, len(d["radii"]))
    r = lcp.resolve_collisions(d["centers"], d["radii"], d["FT"], float(d["dt"]), int(d["p"]),
                               delta=0.1, a_c_scale=1.05, gmres_tol=1e-13, bbpgd_tol=1e-12,
                               rotations=Q)
    out.update(step_Q=Q, step_gamma=r["gamma"], step_U=r["U"], step_centers_new=r["centers_new"],
               step_bbpgd_iters=r["info"]["iters"], step_n_active=r["info"]["n_active"])
    np.savez_compressed(os.path.join(HERE, "rotated_p4.npz"), **out)
    print("rotated", r["info"])


def walls():
    """The five-sphere active step (p = 4) pressed onto a floor z = -1.1 by an
    extra downward force (Sec. 3.3.3 particle-wall constraints), and a
    corner of a floor and a side wall with the identity mobility."""
    d = np.load(os.path.join(HERE, "active_step_p4.npz"))
    W = np.array([[0.0, 0.0, 1.0, -1.1]])
    FT = d["FT"].copy()
    FT[:, 2] -= 30.0
    r = lcp.resolve_collisions(d["centers"], d["radii"], FT, float(d["dt"]), int(d["p"]), delta=0.1,
                               a_c_scale=1.05, gmres_tol=1e-13, bbpgd_tol=1e-12, walls=W)
    out = dict(walls=W, FT=FT, ij=r["ij"], phi=r["phi"], normals=r["normals"], gamma=r["gamma"],
               U=r["U"], centers_new=r["centers_new"], n_active=r["info"]["n_active"],
               bbpgd_iters=r["info"]["iters"])
    print("walls", r["info"], r["ij"].tolist(), r["gamma"])
    np.savez_compressed(os.path.join(HERE, "walls_p4.npz"), **out)


def collision_grad():
    """The five-sphere active step (p = 4): the assembled mobility, the step's
    contacts and gamma, and central differences (h = 1e-5 max|F|) of
    L = sum |U|^2 through the full oracle step in six force / torque
    coordinates, for the active-set gradient of the step."""
    d = np.load(os.path.join(HERE, "active_step_p4.npz"))
    C, R, FT, dt, p = d["centers"], d["radii"], d["FT"], float(d["dt"]), int(d["p"])
    L0, out = adjoint.step_loss(C, R, FT, dt, p, a_c_scale=1.05)
    M = adjoint.mobility_matrix(C, R, p)
    coords = np.array([(0, 0), (1, 1), (2, 1), (3, 2), (4, 0), (4, 4)])
    h = 1e-5 * np.abs(FT).max()
    fd = []
    for i, k in coords:
        Fp, Fm = FT.copy(), FT.copy()
        Fp[i, k] += h
        Fm[i, k] -= h
        fd.append((adjoint.step_loss(C, R, Fp, dt, p, a_c_scale=1.05)[0]
                   - adjoint.step_loss(C, R, Fm, dt, p, a_c_scale=1.05)[0]) / (2 * h))
        print("fd", i, k, fd[-1], flush=True)
    np.savez_compressed(os.path.join(HERE, "collision_grad_p4.npz"), centers=C, radii=R, FT=FT,
                        dt=dt, p=p, a_c_scale=1.05, M=M, ij=out["ij"], normals=out["normals"],
                        gamma=out["gamma"], g=out["g"], U=out["U"], loss=L0, coords=coords,
                        h=h, fd=np.array(fd))


def collision_grad_c():
    """The same step: central differences (h = 1e-6) of L = sum |U|^2 through
    the full oracle step in six centre coordinates (every pair stays at least
    10 h from the near-pair and contact thresholds)."""
    d = np.load(os.path.join(HERE, "active_step_p4.npz"))
    C, R, FT, dt, p = d["centers"], d["radii"], d["FT"], float(d["dt"]), int(d["p"])
    h = 1e-6
    assert adjoint.near_margin(C, R) > 10 * h
    coords = np.array([(0, 0), (1, 1), (2, 2), (3, 0), (4, 1), (4, 2)])
    fd = []
    for i, k in coords:
        Cp, Cm = C.copy(), C.copy()
        Cp[i, k] += h
        Cm[i, k] -= h
        fd.append((adjoint.step_loss(Cp, R, FT, dt, p, a_c_scale=1.05)[0]
                   - adjoint.step_loss(Cm, R, FT, dt, p, a_c_scale=1.05)[0]) / (2 * h))
        print("fd", i, k, fd[-1], flush=True)
    np.savez_compressed(os.path.join(HERE, "collision_grad_c_p4.npz"), coords=coords, h=h,
                        fd=np.array(fd))


def sed_steps():
    """Two collision-resolved steps of a 10-sphere sedimenting cluster (Sec.
    6.3 geometry, p = 4, threshold 30% of the sum of the radii, a_c = 1.05 a)
    with strong random forces added to gravity and dt = 0.5, so that both
    steps have active contacts; the oracle's step applied twice."""
    w = workloads.sedimenting_cluster(N=10, phi=0.25, p=4)
    rng = np.random.default_rng(workloads.SEED_BASE + 60)
    FT = w.FT.copy()
    FT[:, :3] += 20.0 * rng.standard_normal((w.N, 3))
    dt, kw = 0.5, dict(delta=0.0, delta_rel=0.3, a_c_scale=1.05, gmres_tol=1e-13,
                       bbpgd_tol=1e-12, bbpgd_max=20000)
    C = w.centers.copy()
    traj, Us, active = [C], [], []
    for _ in range(2):
        out = lcp.resolve_collisions(C, w.radii, FT, dt, 4, **kw)
        print("sed_steps", out["info"])
        C = out["centers_new"]
        traj.append(C)
        Us.append(out["U"])
        active.append(out["info"]["n_active"])
    np.savez_compressed(os.path.join(HERE, "sed_steps_p4.npz"), centers=w.centers, radii=w.radii,
                        FT=FT, dt=dt, p=4, traj=np.array(traj), U=np.array(Us),
                        n_active=np.array(active))


ALL = {"cfg1": cfg1, "active": active, "capped": capped, "rotated": rotated, "walls": walls, "cfg2": cfg2_sample, "tiny": tiny_layers,
       "crowded": crowded,
       "collision_grad": collision_grad, "collision_grad_c": collision_grad_c,
       "sed_steps": sed_steps}

if __name__ == "__main__":
    for k in (sys.argv[1:] or ALL):
        ALL[k]()
