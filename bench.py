"""Benchmark: collision-resolved time steps of a 1,000-sphere suspension.

Workload (default): 1,000 spheres, radii uniform in [0.5, 1], volume fraction
0.30, 5% of pairs pre-placed at gaps U(1e-4, 1e-2), order p = 6 (98 nodes per
sphere, 98,000 nodes), F ~ N(0,1), T ~ N(0,0.1), dt = 1e-3, mixed precision
(FP32 far field with compensated sums, FP64 Krylov / BBPGD / near and self
quadrature).  One "step" = one call of sps_resolve_collisions: the U_nc
mobility solve, the contact set, BBPGD (each iteration a mobility solve) and the
Euler update; positions advance step after step.

Also (unless --no-contact-bench) one identity-mobility collision step on a
large jittered lattice (2 x 10^7 spheres, volume fraction 0.35, a ~ U[0.5,1],
a_c = 1.05 a, delta = 0.1): the contact search, D, D^T and Algorithm 1 with
U = F, where no N-body sum runs; its kernels are HBM-bound and are reported
against the measured HBM bandwidth ("contact_bbpgd_microbench").

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("collision-resolved steps/s and layer-potential interactions/s vs FP64 GPU, "
          "% roofline")
FLOPS_PER_PAIR = {"K": 30, "S": 29}   # algorithmic FP32 operations per pair term
# dram__bytes_read.sum + dram__bytes_write.sum of one k_far32<K> launch at the
# 1,000-sphere p = 6 workload, from an ncu capture of the current kernel
# (None whenever the kernel changes until it is captured again)
FAR_K_TRAFFIC_BYTES = 3630848 + 76800
SMS, LANES = 152, 128
N_PHASES = 13
PHASES = ["far_K", "far_S", "far_aux", "near_K", "near_S", "self_vsh", "krylov", "contact",
          "bbpgd", "geometry", "bb_D", "bb_DT", "far_dw"]
CONTACT_N = 20_000_000


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        d = {}
    mhz = float(d.get("sm_max_mhz", 2070.0))
    return {"fp32_tflops": SMS * LANES * 2 * mhz * 1e6 / 1e12, "sm_max_mhz": mhz,
            "hbm_gbs": d.get("hbm_gbs", 6800.0), "source": "measured" if d else "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def workload(name):
    from paper_1909_06623_gb300 import workloads
    if name == "cfg2":
        return workloads.config2()
    if name == "cfg3":
        return workloads.config3()
    if name == "cfg4":
        return workloads.config4()
    if name.startswith("cfg5"):
        _, N, p = name.split("_")
        return workloads.config5(int(N), int(p))
    if name == "sed":
        return workloads.sedimenting_cluster()
    if name.startswith("rotor_mono"):        # rotor_mono_<N>: monolayer disk (Sec. 7.2)
        return workloads.rotor_monolayer(N=int(name.split("_")[-1]))
    if name.startswith("rotor"):             # rotor_<N>: spherical rotor cluster (Sec. 7.1)
        return workloads.rotor_cluster(N=int(name.split("_")[-1]))
    raise ValueError(name)


PRECISION = {"fp64": 0, "mixed": 1, "fp64dw": 2}


def ctx_params(precision, bb_warm=2, bbpgd_tol=1e-6):
    """Solver settings of the benchmark step.  Collision radius a_c = 1.05 a is
    the paper's choice at p = 6 (Sec. 6.1).  eps_tol = 1e-6 (the paper runs
    1e-3 to 1e-5, Sec. 6.2) keeps gamma within 1e-5 of a tightly solved
    FP64-accurate step (at 1e-5 the gap is 4.5e-5, set by eps_tol, not by the
    arithmetic).  The GMRES tolerance and the BBPGD cap are this benchmark's.
    bb_warm = 1 starts Algorithm 1 from the previous step's gamma, 2 also from
    its last step length (no product M g_0 for alpha_0; the paper's runs:
    gamma_0 = 0, --bb-warm 0)."""
    return dict(p=6, delta=0.1, beta=1.75, a_c_scale=1.05,
                gmres_tol=1e-6 if precision == "mixed" else 1e-8, gmres_max=150,
                bbpgd_tol=bbpgd_tol, bbpgd_max=100, bb_safeguard=1, warm_start=1, bb_warm=bb_warm,
                precision=PRECISION[precision])


# ---------------------------------------------------------------------------
# oracle (CPU) leg: a bounded sample of one layer-operator application
# ---------------------------------------------------------------------------
# layer-operator applications per config-2 step of the oracle's own algorithm
# (eq. rigidbodyrho in zeta with its traction right-hand side, gamma_0 = 0,
# GMRES from the previous solve's density), counted on the GPU path run in
# that form; both CPU legs scale a one-application sample by it
ORACLE_APPLIES_PER_STEP = 185.0


_SUS = {}


def _oracle_worker(job):
    """One process of the oracle sample: the traction operator K on its share
    of the target spheres (seconds spent in the operator).  The geometry is
    built once per process and workload."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    centers, radii, p, seed, targets = job
    from oracle.layer import Suspension
    key = (len(radii), p, float(centers[0, 0]), float(centers[-1, 2]))
    if key not in _SUS:
        _SUS.clear()
        _SUS[key] = Suspension(centers, radii, p)
    sus = _SUS[key]
    sig = np.random.default_rng(seed).standard_normal((sus.N * sus.P, 3))
    t0 = time.perf_counter()
    sus.apply("K", sig, targets=list(targets))
    return time.perf_counter() - t0


def oracle_sample(w, n_targets=3, seed=0, cores=1, pool=None):
    """Times the FP64 oracle's traction operator K (self + near + all-pairs
    far field) on n_targets target spheres per core and scales it to one full
    application.  cores > 1 runs one spawned process per core, each on its own
    targets, and takes the wall time of the parallel section.  Returns
    (seconds per full application, wall seconds of the sample, targets)."""
    rng = np.random.default_rng(seed)
    tg = rng.choice(w.N, min(w.N, n_targets * cores), replace=False)
    if cores == 1:
        dt = _oracle_worker((w.centers, w.radii, w.p, seed, tg))
        return dt * w.N / len(tg), dt, len(tg)
    import multiprocessing as mp
    jobs = [(w.centers, w.radii, w.p, seed, part) for part in np.array_split(tg, cores)]
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores)
    try:
        if own:
            pool.map(_oracle_worker, jobs)           # start-up: imports, geometry
        t0 = time.perf_counter()
        pool.map(_oracle_worker, jobs)
        dt = time.perf_counter() - t0
    finally:
        if own:
            pool.close()
            pool.join()
    return dt * w.N / len(tg), dt, len(tg)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def matvecs_per_step_estimate(stats_list):
    """Layer-operator applications per step, counted by the library (every
    GMRES iteration, warm-start residual, right-hand side and velocity)."""
    if not stats_list:
        return 60.0
    return float(np.mean([s["layer_applies"] for s in stats_list]))


# ---------------------------------------------------------------------------
def run_reference(args, w):
    steps, warm = args.steps, args.warmup
    import multiprocessing as mp
    cores = host_cores()
    times = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for k in range(warm + steps):
            # each worker builds the geometry on its first job (a warm-up step)
            full, sample, ntg = oracle_sample(w, seed=k, cores=cores, pool=pool)
            if k >= warm:
                times.append(full)
    mv = args.ref_matvecs_per_step
    step_s = float(np.mean(times)) * mv
    val = 1.0 / step_s
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": warm, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "N": w.N, "p": w.p,
                                            "l2": "cpu"},
            "cpu_baseline": {"value": val, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": (f"FP64 numpy oracle on {cores} host cores (one process "
                                        f"each): traction operator K on {ntg} of {w.N} target "
                                        f"spheres per step (all-pairs far field + VSH near/self), "
                                        f"scaled x{w.N}/{ntg} to one application and x{mv:.0f} "
                                        f"applications per step (the oracle's algorithm)")},
            "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def replica_throughput(total_s, steps, world, device):
    """Whole-job steps/s of `world` independent replicas that each timed
    `steps` steps in total_s seconds: the job lasts as long as its slowest
    replica (max over ranks), so value = world * steps / that time.  Returns
    (value, max time).  Collective: one all-reduce of a scalar (NCCL on the
    GPU run, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    if world > 1:
        t = torch.tensor([total_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return world * steps / total_s, total_s


def run_gpu(args, w):
    import torch
    import torch.distributed as dist
    import paper_1909_06623_gb300 as sps

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    prm = ctx_params(args.precision, args.bb_warm, args.bbpgd_tol)
    if w.name.startswith("sed") or w.name.startswith("rotor"):
        # the paper's own settings for its Sec. 6.3 / 7 workloads: threshold
        # 30% of the sum of the radii, eps_tol, collision radius
        prm.update({k: w.params[k] for k in ("delta", "delta_rel", "bbpgd_tol", "a_c_scale")
                    if k in w.params})
    if w.name.startswith("cfg3"):
        # 4,000 spheres at volume fraction 0.40: every mobility solve refined
        # to an FP64-accurate relative residual of 1e-10, eps_tol = 1e-8
        prm.update(ir_tol=w.params["ir_tol"], ir_max=12, bbpgd_tol=w.params["bbpgd_tol"],
                   bbpgd_max=100)
    ctx = sps.Context(stream=stream, **prm)
    pos = dev(w.centers)
    rad = dev(w.radii)
    FT = dev(w.FT)
    gam = torch.empty(16 * w.N, dtype=torch.float64, device="cuda")
    UO = torch.empty(w.N, 6, dtype=torch.float64, device="cuda")
    pos_out = torch.empty_like(pos)
    allow = (4, 5)        # NOT_CONVERGED / BREAKDOWN are reported, not fatal

    def step(p_in):
        ctx.resolve_collisions(p_in, rad, FT, w.dt, gamma=gam, UO=UO, pos_out=pos_out,
                               gamma_cap=gam.numel(), allow=allow)
        return ctx.last_stats

    for _ in range(args.warmup):
        step(pos)
        pos.copy_(pos_out)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    sps._lib.load().sps_profile(ctx.h, 1)
    pos_t0 = pos.clone()                     # the e2e leg replays from here
    torch.cuda.nvtx.range_push("timed")      # ncu --nvtx-include "timed/" captures this region
    for k in range(args.steps):
        if k == args.steps - 1:
            pos_last = pos.clone()         # the FP64 check reruns this step
        flush.zero_()                      # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        stats.append(dict(step(pos)))
        ev[k][1].record(stream)
        pos.copy_(pos_out)
        if args.progress:                  # one line per step on stderr (survives a killed run)
            torch.cuda.synchronize()
            st_ = stats[-1]
            print(json.dumps({"step": k, "ms": ev[k][0].elapsed_time(ev[k][1]), "status": st_["status"],
                              "bbpgd_iters": st_["bbpgd_iters"], "gmres_iters": st_["gmres_iters"],
                              "n_contacts": st_["n_contacts"], "n_active": st_["n_active"],
                              "final_phi": st_["final_phi"], "ir_sweeps": st_["ir_sweeps"],
                              "layer_applies": st_["layer_applies"]}), file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    nc_last = stats[-1]["n_contacts"]
    gam_last, U_last = gam[:nc_last].clone(), UO.clone()
    ph_ms = (ctypes.c_double * N_PHASES)()
    ph_n = (ctypes.c_longlong * N_PHASES)()
    sps._lib.load().sps_profile_read(ctx.h, ph_ms, ph_n)
    sps._lib.load().sps_profile(ctx.h, 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, total_s = replica_throughput(sum(step_ms) / 1e3, args.steps, world, "cuda")

    # dominant kernel: far-field traction N-body (phase 0)
    N, P = w.N, (w.p + 1) * (2 * w.p + 2)
    NP = N * P
    n_near = stats[-1]["n_near_pairs"]
    pairs = NP * NP - P * P * (N + n_near)
    farK_ms, farK_n = ph_ms[0], ph_n[0]
    farS_ms, farS_n = ph_ms[1], ph_n[1]
    avgK = farK_ms / max(farK_n, 1)
    pk = peaks()
    achieved = FLOPS_PER_PAIR["K"] * pairs / (avgK * 1e-3) / 1e12
    interactions = pairs * (farK_n + farS_n) / total_s
    phase_report = {nm: {"ms": round(ph_ms[i], 3), "launches": int(ph_n[i])}
                    for i, nm in enumerate(PHASES)}
    launches = int(sum(s["kernel_launches"] for s in stats))

    # e2e: same step through the host-buffer entry point (copies inside)
    e2e = None
    if args.e2e_steps > 0:
        hpos = torch.as_tensor(w.centers, dtype=torch.float64).pin_memory()
        hrad = torch.as_tensor(w.radii, dtype=torch.float64).pin_memory()
        hFT = torch.as_tensor(w.FT, dtype=torch.float64).pin_memory()
        hg = torch.empty(16 * N, dtype=torch.float64).pin_memory()
        hU = torch.empty(N, 6, dtype=torch.float64).pin_memory()
        hp = torch.empty(N, 3, dtype=torch.float64).pin_memory()
        # replay the timed region's trajectory: one untimed host step from its
        # first positions, then the timed host steps (its steps 2, 3, ...)
        hpos.copy_(pos_t0.cpu())
        ctx.resolve_collisions_host(hpos, hrad, hFT, w.dt, hg, hU, hp, allow=allow)
        hpos.copy_(hp)
        # re-run timing cleanly (per-call wall time, flush outside)
        e2e_times = []
        for _ in range(args.e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            nc = ctx.resolve_collisions_host(hpos, hrad, hFT, w.dt, hg, hU, hp, allow=allow)
            e2e_times.append(time.perf_counter() - t1)
            hpos.copy_(hp)
        e2e_total = sum(e2e_times)
        e2e = {"value": args.e2e_steps / e2e_total, "unit": "steps/s",
               "h2d_bytes_per_step": int(8 * (3 * N + N + 6 * N)),
               "d2h_bytes_per_step": int(8 * (6 * N + 3 * N + nc)),
               "steps": args.e2e_steps,
               "replays": "steps 2.. of the timed region (positions restored, one untimed host step)"}

    # the last timed step again from the same positions (gamma_0 = 0):
    #  - on the plain FP64 path at this benchmark's eps_tol (GMRES 1e-10): a
    #    measured FP64 step rate;
    #  - as a tight FP64-accurate reference (double-float far field, FP64
    #    elsewhere; GMRES 1e-12, eps_tol 1e-9): the error of the mixed step
    #    (relative 2-norms, the paper's eps_2), which includes its eps_tol.
    def rerun(prm_over, label):
        c = sps.Context(stream=stream, **prm_over)
        g_, U_, p_ = torch.empty_like(gam), torch.empty_like(UO), torch.empty_like(pos)
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.resolve_collisions(pos_last, rad, FT, w.dt, gamma=g_, UO=U_, pos_out=p_,
                             gamma_cap=g_.numel(), allow=allow)
        e1.record(stream)
        torch.cuda.synchronize()
        st_ = dict(c.last_stats)
        c.close()
        ms_ = e0.elapsed_time(e1)
        rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        same = st_["n_contacts"] == nc_last
        return {"label": label, "steps_per_s": 1e3 / ms_, "ms": ms_,
                "gmres_tol": prm_over["gmres_tol"], "bbpgd_tol": prm_over["bbpgd_tol"],
                "status": st_["status"], "bbpgd_iters": st_["bbpgd_iters"],
                "gmres_iters": st_["gmres_iters"], "layer_applies": st_["layer_applies"],
                "err": {"U": rel(U_last, U_), "gamma": rel(gam_last, g_[:nc_last]) if same and nc_last else None}}

    fp64_step, ref_step = None, None
    if w.name.startswith("cfg2"):
        if not args.no_fp64_step:
            prm64 = dict(prm, precision=0, gmres_tol=1e-10, bb_warm=0)
            fp64_step = rerun(prm64, "plain FP64 path, this benchmark's eps_tol")
            fp64_step["mixed_speedup"] = fp64_step["ms"] / step_ms[-1]
            prm_ref = dict(prm, precision=2, gmres_tol=1e-12, gmres_max=300, bbpgd_tol=1e-9,
                           bbpgd_max=1000, bb_warm=0)
            ref_step = rerun(prm_ref, "FP64-accurate reference (double-float far field), tight tolerances")
    err_vs_fp64 = None
    if ref_step:
        err_vs_fp64 = dict(ref_step["err"], norm="relative 2-norm over all spheres / contacts",
                           step=f"timed step {args.steps} from the same positions",
                           reference="FP64-accurate path (double-float far field, FP64 near/self/"
                                     "Krylov/BBPGD), GMRES 1e-12, eps_tol 1e-9, gamma_0 = 0")
        if fp64_step:
            err_vs_fp64["vs_plain_fp64_same_eps_tol"] = fp64_step["err"]

    # the paper's initial guess gamma_0 = 0 on the same trajectory: a few
    # steps from the timed region's first positions with a fresh context
    gamma0_leg = None
    if args.gamma0_steps > 0 and args.bb_warm and w.name.startswith("cfg2"):
        cz = sps.Context(stream=stream, **dict(prm, bb_warm=0))
        pz = pos_t0.clone()
        tz = []
        for k in range(args.gamma0_steps + 1):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cz.resolve_collisions(pz, rad, FT, w.dt, gamma=gam, UO=UO, pos_out=pos_out,
                                  gamma_cap=gam.numel(), allow=allow)
            e1.record(stream)
            pz.copy_(pos_out)
            torch.cuda.synchronize()
            if k > 0:                     # the first step only warms the context
                tz.append((e0.elapsed_time(e1), dict(cz.last_stats)))
        cz.close()
        gamma0_leg = {"steps_per_s": 1e3 * len(tz) / sum(t for t, _ in tz),
                      "steps": len(tz), "bbpgd_iters": [st["bbpgd_iters"] for _, st in tz],
                      "gmres_iters": [st["gmres_iters"] for _, st in tz],
                      "note": "Algorithm 1 from gamma_0 = 0 (the paper's runs), steps 2.. of "
                              "the timed region replayed with a fresh context"}

    # FP64 vs mixed: one traction-operator application each, same geometry
    mv = {}
    for prec in ("fp64", "mixed", "fp64dw"):
        c2 = sps.Context(stream=stream, **ctx_params(prec))
        c2.set_geometry(pos, rad)
        sig = torch.randn(3, NP, dtype=torch.float64, device="cuda")
        out = torch.empty_like(sig)
        c2.layer_apply(sps.SPS_OP_K, sig, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = {"fp64": 1, "mixed": 5, "fp64dw": 2}[prec]
        e0.record(stream)
        for _ in range(reps):
            c2.layer_apply(sps.SPS_OP_K, sig, out)
        e1.record(stream)
        torch.cuda.synchronize()
        mv[prec] = e0.elapsed_time(e1) / reps
        c2.close()
    mvps = matvecs_per_step_estimate(stats)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        # config 2: the oracle algorithm's count; elsewhere this run's count
        mvo = args.ref_matvecs_per_step if w.name.startswith("cfg2") else mvps
        full, sample, ntg = oracle_sample(w, cores=cores)
        full1, sample1, ntg1 = oracle_sample(w, cores=1)
        cpu = {"value": 1.0 / (full * mvo), "unit": "steps/s", "cores": cores, "kind": "oracle",
               "sample": (f"FP64 numpy oracle on {cores} host cores (one process each): traction "
                          f"operator K on {ntg} of {N} target spheres ({sample:.1f} s wall), "
                          f"scaled x{N}/{ntg} to one application and x{mvo:.0f} applications "
                          f"per step ({'the oracle algorithm' if w.name.startswith('cfg2') else 'this run'})"),
               "one_core": {"value": 1.0 / (full1 * mvo), "cores": 1,
                            "sample": f"K on {ntg1} target spheres ({sample1:.1f} s)"}}

    contact = None
    if rank == 0 and not args.no_contact_bench:
        del flush
        torch.cuda.empty_cache()
        contact = run_contacts(args, args.contact_n, local)

    if rank == 0:
        last = stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": w.name, "N": N, "p": w.p, "nodes": NP, "precision": args.precision,
                       "gmres_tol": ctx.prm.gmres_tol, "bbpgd_tol": ctx.prm.bbpgd_tol,
                       "ir_tol": ctx.prm.ir_tol,
                       "delta": ctx.prm.delta, "delta_rel": ctx.prm.delta_rel,
                       "bbpgd_gamma0": {0: "zero", 1: "previous step",
                                        2: "previous step (gamma and step length)"}[ctx.prm.bb_warm],
                       "a_c_scale": ctx.prm.a_c_scale, "bbpgd_max": ctx.prm.bbpgd_max,
                       "dt": w.dt, "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "interactions_per_s": interactions,
            "roofline": {"bound": "alu", "kernel": "k_far32<K> (far-field traction N-body)",
                         "achieved": achieved, "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / pk["fp32_tflops"],
                         "traffic": FAR_K_TRAFFIC_BYTES if w.name.startswith("cfg2") else None,
                         "flops_per_pair": FLOPS_PER_PAIR["K"], "pairs_per_launch": pairs,
                         "avg_launch_ms": avgK,
                         "peak_note": (f"152 SMs x 128 FP32 lanes x 2 x {pk['sm_max_mhz']:.0f} MHz "
                                       f"(sm_max_mhz {pk['source']})")},
            "fp64_gpu": {"traction_matvec_ms": mv["fp64"], "mixed_traction_matvec_ms": mv["mixed"],
                         "fp64dw_traction_matvec_ms": mv["fp64dw"],
                         "mixed_speedup_matvec": mv["fp64"] / mv["mixed"],
                         "matvecs_per_step": mvps,
                         "step": fp64_step, "reference_step": ref_step},
            "err_vs_fp64": err_vs_fp64,
            "gamma0_zero": gamma0_leg,
            "solver": {"gmres_iters_per_step": float(np.mean([s["gmres_iters"] for s in stats])),
                       "layer_applies_per_step": float(np.mean([s["layer_applies"] for s in stats])),
                       "mobility_solves_per_step": float(np.mean([s["mobility_solves"] for s in stats])),
                       "bbpgd_iters": [s["bbpgd_iters"] for s in stats],
                       "n_contacts": last["n_contacts"], "n_active": last["n_active"],
                       "n_near_pairs": n_near, "status": [s["status"] for s in stats],
                       "final_phi": [s["final_phi"] for s in stats],
                       "bb_safeguards": [s["bb_safeguards"] for s in stats],
                       "gmres_res_max": last["gmres_res_max"],
                       "ir_sweeps": [s["ir_sweeps"] for s in stats]},
            "phases_ms": phase_report,
            "step_ms": step_ms,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "contact_bbpgd_microbench": contact,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# contact / BBPGD microbenchmark (identity mobility, HBM-bound)
# ---------------------------------------------------------------------------
def contact_bytes(N, nc):
    """Algorithmic bytes of one launch of each BBPGD pass of the identity
    mobility: every array element the pass must touch, once (FP64 values 8 B,
    indices 4 B).
      per-sphere pass (F = D gamma_n): per contact its two incidence entries
        (8), gamma_n and n (32); per sphere its incidence offset (4) and force (24);
      per-contact pass (D^T F + q and the statistics): per contact i, j (8),
        n (24), q, gamma_n, gamma, g (32) and g_new (8); per sphere its force (24)."""
    return {"bb_D": 40 * nc + 28 * N, "bb_DT": 72 * nc + 24 * N}


def contact_bytes_per_end(N, nc):
    """The same launches counted per contact END, the survey's D gamma formula
    (gamma 8, n 24 and an index 4 read for each of the two ends of a contact,
    48 B written per sphere), and D^T U as 2 x 24 + 24 + 8 read and 8 written
    per contact with U read per end (the 8 written is g_new); the per-contact
    statistics add q, gamma_n, gamma and g (32).  Counts gamma and n twice
    per contact, so it reads higher than contact_bytes."""
    return {"bb_D": 72 * nc + 48 * N, "bb_DT": (2 * 24 + 24 + 8 + 8 + 32) * nc}


def contact_fp64_flops(nc, bb_variant=1):
    """FP64 operations (an FMA counts 2) of the same launches: the per-sphere
    pass does 3 FMA per contact end; the per-contact pass 3 subtractions and 3
    FMA for D^T F + q, 2 subtractions and 3 FMA (4 for BB2) for the
    statistics (the min of the min-map residual runs on the integer units)."""
    return {"bb_D": 12 * nc, "bb_DT": (17 + 2 * (bb_variant == 2)) * nc}


FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (nominal), the recipe's figure


def run_contacts(args, N, gpu_index, standalone=False):
    import torch
    import paper_1909_06623_gb300 as sps
    from paper_1909_06623_gb300 import workloads
    w = workloads.jittered_lattice(workloads.SEED_BASE + 6, N)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    tol = 1e-4 * np.sqrt(N)
    ctx = sps.Context(stream=stream, p=2, delta=0.1, a_c_scale=1.05, mobility=sps.SPS_MOB_IDENTITY,
                      bbpgd_tol=tol, bbpgd_max=1000, bb_safeguard=1)
    pos, rad, FT = dev(w.centers), dev(w.radii), dev(w.FT)
    gam = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    UO = torch.empty(N, 6, dtype=torch.float64, device="cuda")
    pos_out = torch.empty_like(pos)

    def step():
        ctx.resolve_collisions(pos, rad, FT, w.dt, gamma=gam, UO=UO, pos_out=pos_out,
                               gamma_cap=gam.numel(), allow=(4, 5))
        return dict(ctx.last_stats)

    for _ in range(args.warmup):
        step()
        pos.copy_(pos_out)
    torch.cuda.synchronize()
    lib = sps._lib.load()
    clocks = ClockSampler(gpu_index)
    clocks.start()
    lib.sps_profile(ctx.h, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    for k in range(args.steps):
        ev[k][0].record(stream)
        stats.append(step())
        ev[k][1].record(stream)
        pos.copy_(pos_out)
    torch.cuda.synchronize()
    ph_ms = (ctypes.c_double * N_PHASES)()
    ph_n = (ctypes.c_longlong * N_PHASES)()
    lib.sps_profile_read(ctx.h, ph_ms, ph_n)
    lib.sps_profile(ctx.h, 0)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    nc = stats[-1]["n_contacts"]
    pk = peaks()
    by = contact_bytes(N, nc)
    by_end = contact_bytes_per_end(N, nc)
    roof = []
    fl = contact_fp64_flops(nc)
    for nm, kern in (("bb_D", "k_bb_gather"), ("bb_DT", "k_bb_ident_DT")):
        i = PHASES.index(nm)
        avg = ph_ms[i] / max(ph_n[i], 1)
        ach = by[nm] / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        f64 = fl[nm] / (avg * 1e-3) / 1e12 if avg > 0 else 0.0
        roof.append({"kernel": kern, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "bytes_per_launch": by[nm],
                     "avg_launch_ms": avg, "launches": int(ph_n[i]), "traffic": None,
                     "peak_note": f"measured STREAM copy ({pk['source']})",
                     "per_end_count": {"bytes_per_launch": by_end[nm],
                                       "achieved": by_end[nm] / (avg * 1e-3) / 1e9 if avg > 0 else 0.0,
                                       "frac": (by_end[nm] / (avg * 1e-3) / 1e9 / pk["hbm_gbs"]
                                                if avg > 0 else 0.0)},
                     "fp64": {"flops_per_launch": fl[nm], "achieved_tflops": f64,
                              "peak_tflops": FP64_PEAK_TFLOPS, "frac": f64 / FP64_PEAK_TFLOPS}})
    out = {"workload": w.name, "N": N, "n_contacts": nc,
           "n_active": stats[-1]["n_active"], "bbpgd_tol": tol,
           "bbpgd_iters": [s["bbpgd_iters"] for s in stats],
           "status": [s["status"] for s in stats],
           "ms_per_step": float(np.mean(step_ms)), "step_ms": step_ms,
           "steps_per_s": 1e3 / float(np.mean(step_ms)),
           "contact_updates_per_s": nc * float(np.mean([s["bbpgd_iters"] for s in stats])) /
           (float(np.mean(step_ms)) * 1e-3),
           "phases_ms": {nm: {"ms": round(ph_ms[i], 3), "launches": int(ph_n[i])}
                         for i, nm in enumerate(PHASES) if ph_n[i]},
           "roofline": roof,
           "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
           "clocks": clk,
           "l2": "inputs larger than L2 (positions and radii alone 640 MB), no flush",
           "data": "synthetic jittered lattice (contact statistics of the random suspensions)"}
    ctx.close()
    if standalone:
        print(json.dumps({"contact_bbpgd_microbench": out}), flush=True)
    return out


def run_sweep(args):
    """Sweep of the layer operator over suspension size and order (spheres
    a ~ U[0.5, 1] at volume fraction 0.35 with close pairs): per (N, p) one
    traction-operator application in mixed precision (far-field pair rate and
    fraction of FP32 peak), the FP64 application where it takes under ~2 s,
    and one full collision-resolved step in mixed precision for N <= 2000."""
    import torch
    import paper_1909_06623_gb300 as sps
    from paper_1909_06623_gb300 import workloads
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    lib = sps._lib.load()
    pk = peaks()
    rows = []
    for N in (500, 2000, 4000, 8000):
        for p in (4, 6, 8):
            try:
                row = sweep_point(N, p, dev, stream, lib, pk)
            except Exception as e:          # keep sweeping; the row records the failure
                row = {"workload": f"cfg5_N{N}_p{p}", "N": N, "p": p, "error": str(e)[:300]}
            rows.append(row)
            print(json.dumps(row), flush=True)
    print(json.dumps({"sweep": rows, "peak_fp32_tflops": pk["fp32_tflops"]}), flush=True)


def sweep_point(N, p, dev, stream, lib, pk):
    """One (N, p) point of run_sweep."""
    import torch
    import paper_1909_06623_gb300 as sps
    from paper_1909_06623_gb300 import workloads
    w = workloads.config5(N, p)
    P = (p + 1) * (2 * p + 2)
    NP = N * P
    row = {"workload": w.name, "N": N, "p": p, "nodes": NP}
    for prec in ("mixed", "fp64"):
        # one step after one warm-up step: gamma_0 = 0 (the warm-up step's
        # gamma resolves the initial overlaps and is no guess for the next)
        prm = ctx_params(prec, bb_warm=0)
        prm["p"] = p
        ctx = sps.Context(stream=stream, **prm)
        ctx.set_geometry(dev(w.centers), dev(w.radii))
        if prec == "fp64" and NP * NP > 1.2e10:
            row["fp64_K_ms"] = None
            ctx.close()
            continue
        sig = torch.randn(3, NP, dtype=torch.float64, device="cuda")
        out = torch.empty_like(sig)
        ctx.layer_apply(sps.SPS_OP_K, sig, out)
        reps = 3 if prec == "mixed" else 1
        torch.cuda.synchronize()
        lib.sps_profile(ctx.h, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.layer_apply(sps.SPS_OP_K, sig, out)
        e1.record(stream)
        torch.cuda.synchronize()
        ph_ms = (ctypes.c_double * N_PHASES)()
        ph_n = (ctypes.c_longlong * N_PHASES)()
        lib.sps_profile_read(ctx.h, ph_ms, ph_n)
        lib.sps_profile(ctx.h, 0)
        op_ms = e0.elapsed_time(e1) / reps
        row[f"{prec}_K_ms"] = op_ms
        if prec == "mixed":
            # far pairs: all node pairs minus self and near spheres
            near, close = ctx.geometry_counts()
            pairs = NP * NP - P * P * (N + near)
            farK = ph_ms[0] / max(ph_n[0], 1)
            ach = FLOPS_PER_PAIR["K"] * pairs / (farK * 1e-3) / 1e12
            row.update(far_pairs=pairs, near_pairs=near, close_entries=close, far_K_ms=farK,
                       far_K_tflops=ach, far_K_frac=ach / pk["fp32_tflops"],
                       interactions_per_s=pairs / (farK * 1e-3))
            if N <= 2000:
                FT = dev(w.FT)
                pos = dev(w.centers)
                rad = dev(w.radii)
                g = torch.empty(16 * N, dtype=torch.float64, device="cuda")
                U = torch.empty(N, 6, dtype=torch.float64, device="cuda")
                po = torch.empty_like(pos)
                ctx.resolve_collisions(pos, rad, FT, w.dt, gamma=g, UO=U, pos_out=po,
                                       gamma_cap=g.numel(), allow=(4, 5))
                pos.copy_(po)
                torch.cuda.synchronize()
                e0.record(stream)
                ctx.resolve_collisions(pos, rad, FT, w.dt, gamma=g, UO=U, pos_out=po,
                                       gamma_cap=g.numel(), allow=(4, 5))
                e1.record(stream)
                torch.cuda.synchronize()
                stt = ctx.last_stats
                row.update(step_ms=e0.elapsed_time(e1), step_gmres_iters=stt["gmres_iters"],
                           step_bbpgd_iters=stt["bbpgd_iters"], step_contacts=stt["n_contacts"],
                           step_status=stt["status"])
        ctx.close()
    if row.get("fp64_K_ms") and row.get("mixed_K_ms"):
        row["mixed_speedup_K"] = row["fp64_K_ms"] / row["mixed_K_ms"]
    return row


def run_single_op(args, w):
    """One layer-operator application on the workload's geometry (a small,
    self-contained case for kernel captures)."""
    import torch
    import paper_1909_06623_gb300 as sps
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    ctx = sps.Context(**ctx_params(args.precision))
    ctx.set_geometry(dev(w.centers), dev(w.radii))
    torch.manual_seed(0)
    sig = torch.randn(3, w.N * ctx.P, dtype=torch.float64, device="cuda")
    op = {"K": sps.SPS_OP_K, "S": sps.SPS_OP_S, "A": sps.SPS_OP_A}[args.single_op]
    out = ctx.layer_apply(op, sig)
    torch.cuda.synchronize()
    print(json.dumps({"single_op": args.single_op, "max_abs": out.abs().max().item()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cfg2")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp64dw"])
    ap.add_argument("--bbpgd-tol", type=float, default=1e-6,
                    help="eps_tol of Algorithm 1 (absolute min-map residual)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-matvecs-per-step", type=float, default=ORACLE_APPLIES_PER_STEP,
                    help="layer-operator applications per config-2 step for the oracle's "
                         "algorithm (the paper's formulation: zeta with its traction "
                         "right-hand side, gamma_0 = 0, GMRES from the previous solve's "
                         "density; measured on the GPU path in that form)")
    ap.add_argument("--single-op", choices=["K", "S", "A"], default=None,
                    help="apply one layer operator on the workload geometry and exit")
    ap.add_argument("--no-contact-bench", action="store_true")
    ap.add_argument("--progress", action="store_true",
                    help="print one JSON line per timed step to stderr as it completes")
    ap.add_argument("--no-fp64-step", action="store_true",
                    help="skip the FP64 and FP64-accurate reruns of the last timed step "
                         "(FP64 rate and error against FP64)")
    ap.add_argument("--gamma0-steps", type=int, default=3,
                    help="steps of the gamma_0 = 0 comparison leg (0: skip)")
    ap.add_argument("--bb-warm", type=int, default=2, choices=[0, 1, 2],
                    help="1: Algorithm 1 starts from the previous step's gamma; 2: also from its "
                         "last step length; 0: gamma_0 = 0")
    ap.add_argument("--contact-n", type=int, default=CONTACT_N)
    ap.add_argument("--contact-only", action="store_true",
                    help="run only the identity-mobility contact benchmark")
    ap.add_argument("--sweep", action="store_true",
                    help="operator / step sweep over N in {500..8000} and p in {4, 6, 8}")
    args = ap.parse_args()
    if args.sweep:
        run_sweep(args)
        return
    if args.contact_only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        run_contacts(args, args.contact_n, int(os.environ.get("LOCAL_RANK", "0")), standalone=True)
        return
    w = workload(args.workload)
    if args.single_op:
        run_single_op(args, w)
        return
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args, w)
        return
    run_gpu(args, w)


if __name__ == "__main__":
    main()
