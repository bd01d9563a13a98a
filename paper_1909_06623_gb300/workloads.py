"""Seeded synthetic suspensions shaped like the paper's workloads.

Input generation only: sphere centres, radii, forces and torques.  This module
holds none of the method's arithmetic and is the one piece of code that both the
CUDA path (bench, tests) and the CPU oracle's tests consume.

Shapes follow the paper's test problems (Yan et al., arXiv 1909.06623, Sec. 6):
random non-overlapping spheres in a free-space cube at a target volume
fraction, radii uniform in [0.5, 1] (Sec. 6.5 draws log-normal radii; the
uniform law is the one the workloads below fix), a few pairs pre-placed close to
contact so that collisions and near-singular quadrature are exercised.

Placement is random sequential addition (largest sphere first) with a minimum
gap between every two spheres; volume fractions above what that reaches are
made by compressing an addition at a lower fraction and pushing overlapping
pairs apart (a geometric relaxation, no hydrodynamics).
"""
from dataclasses import dataclass, field
from math import pi

import numpy as np

SEED_BASE = 1909066230


@dataclass
class Workload:
    name: str
    centers: np.ndarray          # N x 3 float64
    radii: np.ndarray            # N float64
    FT: np.ndarray               # N x 6 float64 (force, torque)
    p: int
    dt: float
    steps: int
    params: dict = field(default_factory=dict)

    @property
    def N(self):
        return len(self.radii)


def _cell_key(c, h):
    return tuple(np.floor(c / h).astype(np.int64))


class _Grid:
    """Uniform cell grid for overlap queries during placement."""

    def __init__(self, h):
        self.h = h
        self.cells = {}

    def add(self, k, c):
        self.cells.setdefault(_cell_key(c, self.h), []).append(k)

    def remove(self, k, c):
        self.cells[_cell_key(c, self.h)].remove(k)

    def around(self, c):
        i, j, l = _cell_key(c, self.h)
        out = []
        for a in (i - 1, i, i + 1):
            for b in (j - 1, j, j + 1):
                for d in (l - 1, l, l + 1):
                    out.extend(self.cells.get((a, b, d), ()))
        return out


def _fits(k, c, r, C, R, grid, gap, skip=()):
    for j in grid.around(c):
        if j == k or j in skip:
            continue
        if np.linalg.norm(C[j] - c) < R[j] + r + gap:
            return False
    return True


def rsa(rng, radii, L, gap, max_tries=200000):
    """Random sequential addition in [0, L]^3, largest first, all gaps > gap."""
    N = len(radii)
    order = np.argsort(-radii, kind="stable")
    C = np.full((N, 3), np.nan)
    grid = _Grid(2.0 * radii.max() + gap)
    for k in order:
        r = radii[k]
        for _ in range(max_tries):
            c = r + rng.random(3) * (L - 2 * r)
            if _fits(k, c, r, C, radii, grid, gap):
                C[k] = c
                grid.add(k, c)
                break
        else:
            raise RuntimeError("random sequential addition jammed")
    return C


def place_close_pairs(rng, C, R, n_pairs, gap_lo, gap_hi, min_gap, L=None,
                      direction=None):
    """Re-place n_pairs disjoint partners at a small gap from their mates."""
    N = len(R)
    grid = _Grid(2.0 * R.max() + min_gap)
    for k in range(N):
        grid.add(k, C[k])
    used = set()
    pairs = []
    perm = rng.permutation(N)
    idx = 0
    while len(pairs) < n_pairs and idx + 1 < N:
        i, j = int(perm[idx]), int(perm[idx + 1])
        idx += 2
        for _ in range(200):
            u = direction if direction is not None else rng.standard_normal(3)
            u = np.asarray(u, dtype=np.float64) / np.linalg.norm(u)
            g = gap_lo if gap_hi == gap_lo else gap_lo + (gap_hi - gap_lo) * rng.random()
            c = C[i] + u * (R[i] + R[j] + g)
            if L is not None and (np.any(c < R[j]) or np.any(c > L - R[j])):
                continue
            if _fits(j, c, R[j], C, R, grid, min_gap, skip={i}):
                grid.remove(j, C[j])
                C[j] = c
                grid.add(j, c)
                pairs.append((i, j))
                used.update((i, j))
                break
    return C, pairs


def compress(C, R, phi_from, phi_to, gap, sweeps=400, dim=3):
    """Scale the packing about its centre in 40 steps and, after each, push
    overlapping pairs apart (all pairs of a sweep at once) until every gap
    exceeds gap.  dim = 2: phi is an area fraction and the points stay in
    their plane (z = const)."""
    from scipy.spatial import cKDTree
    C = C.copy()
    mid = C.mean(axis=0)
    steps = 40
    f = ((phi_from / phi_to) ** (1.0 / dim)) ** (1.0 / steps)
    reach = 2.0 * R.max() + gap
    for _ in range(steps):
        C = mid + (C - mid) * f
        for _ in range(sweeps):
            pr = cKDTree(C).query_pairs(reach, output_type="ndarray")
            if len(pr) == 0:
                break
            i, j = pr[:, 0], pr[:, 1]
            d = C[j] - C[i]
            dist = np.sqrt(np.einsum("kc,kc->k", d, d))
            need = R[i] + R[j] + gap
            m = dist < need
            if not m.any():
                break
            push = (0.5 * (need[m] - dist[m]) * 1.0001 + 1e-12) / dist[m]
            step = d[m] * push[:, None]
            np.add.at(C, i[m], -step)
            np.add.at(C, j[m], step)
        else:
            raise RuntimeError("compression did not converge")
    return C


def box_side(radii, phi):
    return (np.sum(4.0 / 3.0 * pi * radii ** 3) / phi) ** (1.0 / 3.0)


def random_suspension(seed, N, phi, a_lo=0.5, a_hi=1.0, pair_frac=0.05,
                      gap_lo=1e-4, gap_hi=1e-2, min_gap=2e-2, collision_scale=None):
    """Polydisperse random suspension at volume fraction phi plus close pairs.

    collision_scale (dense packings, phi > 0.33): place and compress with the
    collision radii a_c = collision_scale * a and min_gap measured between
    collision spheres, so that no pair overlaps at the collision radius (the
    state the collision solver keeps: Phi >= 0); phi stays the volume
    fraction of the true spheres."""
    rng = np.random.default_rng(seed)
    R = a_lo + (a_hi - a_lo) * rng.random(N) if a_hi > a_lo else np.full(N, a_lo)
    L = box_side(R, phi)
    if phi <= 0.33:
        C = rsa(rng, R, L, min_gap)
    elif collision_scale is not None:
        Rc = collision_scale * R
        phic = phi * collision_scale ** 3
        L0 = box_side(Rc, 0.30)
        C = compress(rsa(rng, Rc, L0, min_gap), Rc, 0.30, phic, min_gap)
    else:
        L0 = box_side(R, 0.30)
        C = compress(rsa(rng, R, L0, min_gap), R, 0.30, phi, min_gap)
    n_pairs = int(round(pair_frac * N / 1.0)) // 1
    n_pairs = min(n_pairs, N // 2)
    if n_pairs:
        C, _ = place_close_pairs(rng, C, R, n_pairs, gap_lo, gap_hi, min_gap)
    return C, R, rng


def small_cluster(seed, N=8, a=1.0, side=8.0, min_gap=0.05, close_gap=1e-3,
                  n_close=2):
    """N equal spheres in a cube of given side, all gaps > min_gap, then n_close
    pairs re-placed along +z at gap close_gap."""
    rng = np.random.default_rng(seed)
    R = np.full(N, a)
    # centres uniform in [0, side]^3 (spheres may poke out of the cube)
    C = np.full((N, 3), np.nan)
    grid = _Grid(2 * a + min_gap)
    for k in range(N):
        for _ in range(100000):
            c = rng.random(3) * side
            if _fits(k, c, a, C, R, grid, min_gap):
                C[k] = c
                grid.add(k, c)
                break
        else:
            raise RuntimeError("placement failed")
    C, pairs = place_close_pairs(rng, C, R, n_close, close_gap, close_gap, min_gap,
                                 direction=(0.0, 0.0, 1.0))
    if len(pairs) != n_close:
        raise RuntimeError("could not place the close pairs")
    return C, R, rng


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------
def config1():
    """8 unit spheres, p = 8, F = (0,0,-1), one step dt = 1e-3 (FP64 parity)."""
    C, R, _ = small_cluster(SEED_BASE + 1)
    FT = np.zeros((8, 6))
    FT[:, 2] = -1.0
    return Workload("cfg1_N8_p8", C, R, FT, p=8, dt=1e-3, steps=1,
                    params=dict(delta=0.1, gmres_tol=1e-12, bbpgd_tol=1e-10))


def config2(N=1000, seed=SEED_BASE + 2):
    """1,000 spheres a ~ U[0.5,1], volume fraction 0.30, 5% close pairs, p = 6,
    F ~ N(0,1), T ~ N(0,0.1), 20 steps of dt = 1e-3."""
    C, R, rng = random_suspension(seed, N, 0.30)
    FT = np.concatenate([rng.standard_normal((N, 3)),
                         0.1 * rng.standard_normal((N, 3))], axis=1)
    return Workload(f"cfg2_N{N}_p6_phi0.30", C, R, FT, p=6, dt=1e-3, steps=20,
                    params=dict(delta=0.1, gmres_tol=1e-8, bbpgd_tol=1e-6))


def config3(N=4000, seed=SEED_BASE + 3, a_c_scale=1.05):
    """4,000 spheres a ~ U[0.5,1] at volume fraction 0.40, p = 6, gravity
    F = (0,0,-(a/0.75)^3), 10 steps of dt = 5e-4.  Packed at the collision
    radius a_c = 1.05 a with no gap (a dense sediment: many pairs touching at
    a_c, none overlapping)."""
    C, R, _ = random_suspension(seed, N, 0.40, pair_frac=0.0, min_gap=0.0,
                                collision_scale=a_c_scale)
    FT = np.zeros((N, 6))
    FT[:, 2] = -(R / 0.75) ** 3
    return Workload(f"cfg3_N{N}_p6_phi0.40", C, R, FT, p=6, dt=5e-4, steps=10,
                    params=dict(delta=0.1, ir_tol=1e-10, bbpgd_tol=1e-8))


def config4(N=1000, seed=SEED_BASE + 4):
    """1,000 unit spheres at volume fraction 0.25, p = 6, F ~ N(0,1)."""
    C, R, rng = random_suspension(seed, N, 0.25, a_lo=1.0, a_hi=1.0, pair_frac=0.0)
    FT = np.concatenate([rng.standard_normal((N, 3)), np.zeros((N, 3))], axis=1)
    return Workload(f"cfg4_N{N}_p6_phi0.25", C, R, FT, p=6, dt=1e-3, steps=1,
                    params=dict(delta=0.1))


def config5(N, p, seed=None, a_c_scale=1.05):
    """Sweep point: N spheres a ~ U[0.5,1] at volume fraction 0.35, order p,
    packed at the collision radius a_c = 1.05 a with no gap (no pre-placed
    close pairs; no pair overlaps at a_c)."""
    seed = SEED_BASE + 5 + 17 * N + p if seed is None else seed
    C, R, rng = random_suspension(seed, N, 0.35, pair_frac=0.0, min_gap=0.0,
                                  collision_scale=a_c_scale)
    FT = np.concatenate([rng.standard_normal((N, 3)),
                         0.1 * rng.standard_normal((N, 3))], axis=1)
    return Workload(f"cfg5_N{N}_p{p}_phi0.35", C, R, FT, p=p, dt=1e-3, steps=1,
                    params=dict(delta=0.1))


def tiny(seed, N, p, phi=0.2, a_lo=0.5, a_hi=1.0, n_pairs=1, gap=1e-2):
    """Small random case for parity tests (a few spheres, one close pair)."""
    rng = np.random.default_rng(seed)
    R = a_lo + (a_hi - a_lo) * rng.random(N)
    L = box_side(R, phi)
    C = rsa(rng, R, L, 0.05)
    if n_pairs:
        C, _ = place_close_pairs(rng, C, R, n_pairs, gap, gap, 0.05)
    FT = np.concatenate([rng.standard_normal((N, 3)),
                         0.1 * rng.standard_normal((N, 3))], axis=1)
    return Workload(f"tiny_N{N}_p{p}_s{seed}", C, R, FT, p=p, dt=1e-3, steps=1)


def crowded_shell(seed, n_small=24, a_big=4.0, a_small=0.5, gap_lo=0.02, gap_hi=0.3, p=4):
    """One large sphere at the origin ringed by n_small small ones at gaps
    U[gap_lo, gap_hi] from its surface, directions on a Fibonacci lattice of
    the sphere, each turned by a seeded random angle about the axis.  Every
    small sphere's nodes lie within 1.5 large-sphere radii of its centre, so
    the large source has n_small * (p + 1)(2p + 2) close items: a parity case
    for near-field paths that hold a bounded number of close items."""
    rng = np.random.default_rng(seed)
    k = np.arange(n_small) + 0.5
    z = 1.0 - 2.0 * k / n_small
    th = np.pi * (1.0 + 5.0 ** 0.5) * k + 2 * np.pi * rng.random()
    u = np.stack([np.sqrt(1 - z * z) * np.cos(th), np.sqrt(1 - z * z) * np.sin(th), z], axis=1)
    dist = a_big + a_small + gap_lo + (gap_hi - gap_lo) * rng.random(n_small)
    C = np.concatenate([np.zeros((1, 3)), u * dist[:, None]])
    R = np.concatenate([[a_big], np.full(n_small, a_small)])
    FT = np.concatenate([rng.standard_normal((n_small + 1, 3)),
                         0.1 * rng.standard_normal((n_small + 1, 3))], axis=1)
    return Workload(f"crowded_shell_n{n_small}_p{p}_s{seed}", C, R, FT, p=p, dt=1e-3, steps=1)


def jittered_lattice(seed, N, phi=0.35, a_lo=0.5, a_hi=1.0, jitter=0.1):
    """Large contact workload: N spheres, a ~ U[a_lo, a_hi], centres on a
    simple-cubic lattice whose spacing s gives volume fraction phi, each moved
    by U(-jitter s, jitter s) per coordinate.  Spheres are numbered in lattice
    order (x fastest), so neighbours have nearby indices.  With a_c = 1.05 a
    and delta = 0.1 this has about one contact per sphere, about 60% of them
    overlapping, as the random suspensions at volume fraction 0.30-0.35 do.
    F ~ N(0, 1), T ~ N(0, 0.1^2) per sphere."""
    rng = np.random.default_rng(seed)
    R = a_lo + (a_hi - a_lo) * rng.random(N)
    mean_vol = 4.0 / 3.0 * pi * (a_hi ** 4 - a_lo ** 4) / (4.0 * (a_hi - a_lo)) \
        if a_hi > a_lo else 4.0 / 3.0 * pi * a_lo ** 3
    s = (mean_vol / phi) ** (1.0 / 3.0)
    n = int(np.ceil(N ** (1.0 / 3.0)))
    k = np.arange(N, dtype=np.int64)
    site = np.stack([k % n, (k // n) % n, k // (n * n)], axis=1).astype(np.float64)
    C = site * s + rng.uniform(-jitter * s, jitter * s, (N, 3))
    FT = np.concatenate([rng.standard_normal((N, 3)),
                         0.1 * rng.standard_normal((N, 3))], axis=1)
    return Workload(f"lattice_N{N}_phi{phi:.2f}", C, R, FT, p=0, dt=1e-3, steps=1,
                    params=dict(delta=0.1, a_c_scale=1.05))


def contact_chain(seed, n=5):
    """n unit spheres in a wobbly chain, neighbours within U(1.96, 2.02) of
    touching, squeezed by opposing x-forces: every neighbour pair is a contact,
    most of them active.  F ~ 80 N(0, 1) plus a linear squeeze."""
    rng = np.random.default_rng(seed)
    c = np.zeros((n, 3))
    for k in range(1, n):
        d = np.array([1.0, 0.3 * rng.standard_normal(), 0.3 * rng.standard_normal()])
        c[k] = c[k - 1] + (1.96 + 0.06 * rng.random()) * d / np.linalg.norm(d)
    F = 80.0 * rng.standard_normal((n, 6))
    F[:, 0] += np.linspace(60.0, -60.0, n)
    return Workload(f"chain_n{n}_s{seed}", c, np.ones(n), F, p=0, dt=1e-3, steps=1,
                    params=dict(delta=0.1))


def sedimenting_cluster(seed=SEED_BASE + 6, N=1000, phi=0.20, a=1.0, a_c_scale=1.05, p=6,
                        steps=20):
    """The sedimentation test of Sec. 6.3: N monodisperse spheres of radius a in
    a dense spherical cluster of volume fraction phi in unbounded fluid, every
    sphere pulled by the same force F = (0, 0, -1) (no torque), collision radius
    a_c = 1.05 a, dt = 0.05 eta a^2 / F, p = 6, BBPGD tolerance 1e-4, contact
    threshold 30% of the sum of the radii (Sec. 3.2).  The cluster radius is
    a (N / phi)^(1/3); centres by random sequential addition inside it with
    every gap above 2 (a_c - a) + 0.02 a, so the start is collision-free."""
    rng = np.random.default_rng(seed)
    R = np.full(N, float(a))
    Rb = a * (N / phi) ** (1.0 / 3.0)
    gap = 2.0 * (a_c_scale - 1.0) * a + 0.02 * a
    C = np.full((N, 3), np.nan)
    grid = _Grid(2.0 * a + gap)
    for k in range(N):
        for _ in range(200000):
            v = rng.standard_normal(3)
            c = v / np.linalg.norm(v) * (Rb - a) * rng.random() ** (1.0 / 3.0)
            if _fits(k, c, a, C, R, grid, gap):
                C[k] = c
                grid.add(k, c)
                break
        else:
            raise RuntimeError("random sequential addition jammed")
    FT = np.zeros((N, 6))
    FT[:, 2] = -1.0
    return Workload(f"sed_cluster_N{N}_phi{phi:.2f}", C, R, FT, p=p, dt=0.05 * a * a, steps=steps,
                    params=dict(delta=0.0, delta_rel=0.3, a_c_scale=a_c_scale, bbpgd_tol=1e-4))


def random_rotations(seed, N):
    """N rotation matrices drawn uniformly from SO(3) (unit quaternions from
    normalised 4-d Gaussian vectors): the random orientation of each sphere's
    grid (Sec. 5.4).  N x 3 x 3 float64."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((N, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def _lognormal_radii(rng, N, mean=1.0, sd=0.3):
    """Radii with a log-normal law of the given mean and standard deviation
    (Sec. 7.1 prints the law's parameters as mu = a, sigma = 0.3 a; read here
    as the radius distribution's mean and standard deviation)."""
    s2 = np.log(1.0 + (sd / mean) ** 2)
    return rng.lognormal(np.log(mean) - 0.5 * s2, np.sqrt(s2), N)


def rotor_cluster(seed=SEED_BASE + 7, N=10000, phi=0.10, a_c_scale=1.1, p=6, steps=10):
    """Sec. 7.1: a spherical cluster of N polydisperse rotors (log-normal radii,
    mean 1, sd 0.3) at volume fraction phi in unbounded fluid, the same torque
    T = (0, 0, 1) on every sphere and no force, collision radius 1.1 a,
    dt = 1.0 eta a^3 / T, eps_tol = 1e-5, p = 6, contact threshold 30% of the
    sum of the radii.  Centres by random sequential addition in a ball at
    the collision radius with no gap (collision-free start)."""
    rng = np.random.default_rng(seed)
    R = _lognormal_radii(rng, N)
    Rc = a_c_scale * R
    Rb = (np.sum(R ** 3) / phi) ** (1.0 / 3.0)
    order = np.argsort(-R, kind="stable")
    C = np.full((N, 3), np.nan)
    grid = _Grid(2.0 * Rc.max())
    for k in order:
        for _ in range(200000):
            v = rng.standard_normal(3)
            c = v / np.linalg.norm(v) * (Rb - R[k]) * rng.random() ** (1.0 / 3.0)
            if _fits(k, c, Rc[k], C, Rc, grid, 0.0):
                C[k] = c
                grid.add(k, c)
                break
        else:
            raise RuntimeError("random sequential addition jammed")
    FT = np.zeros((N, 6))
    FT[:, 5] = 1.0
    return Workload(f"rotor_cluster_N{N}_phi{phi:.2f}", C, R, FT, p=p, dt=1.0, steps=steps,
                    params=dict(delta=0.0, delta_rel=0.3, a_c_scale=a_c_scale, bbpgd_tol=1e-5))


def rotor_monolayer(seed=SEED_BASE + 8, N=20000, area=0.60, a_c_scale=1.1, p=6, steps=10):
    """Sec. 7.2: a disk of N monodisperse rotors (a = 1) confined to the plane
    z = 0 at area fraction 0.60 (about 0.73 at the collision radius 1.1 a),
    torque T = (0, 0, 1) perpendicular to the disk, dt = 0.5 eta a^3 / T,
    eps_tol = 1e-5, p = 6, contact threshold 30% of the sum of the radii.
    Random sequential addition in a disk at area fraction 0.45 of the
    collision disks, then in-plane compression at the collision radius with
    no gap (no overlap at a_c; many pairs touch)."""
    rng = np.random.default_rng(seed)
    R = np.ones(N)
    ac = a_c_scale
    Rd0 = ac * np.sqrt(N / 0.45)
    C = np.full((N, 3), np.nan)
    grid = _Grid(2.0 * ac)
    Rcs = np.full(N, ac)
    for k in range(N):
        for _ in range(200000):
            r = (Rd0 - ac) * np.sqrt(rng.random())
            t = 2 * pi * rng.random()
            c = np.array([r * np.cos(t), r * np.sin(t), 0.0])
            if _fits(k, c, ac, C, Rcs, grid, 0.0):
                C[k] = c
                grid.add(k, c)
                break
        else:
            raise RuntimeError("random sequential addition jammed")
    C = compress(C, Rcs, 0.45, area * ac * ac, 0.0, sweeps=4000, dim=2)
    C[:, 2] = 0.0
    FT = np.zeros((N, 6))
    FT[:, 5] = 1.0
    return Workload(f"rotor_monolayer_N{N}_area{area:.2f}", C, R, FT, p=p, dt=0.5, steps=steps,
                    params=dict(delta=0.0, delta_rel=0.3, a_c_scale=a_c_scale, bbpgd_tol=1e-5))
