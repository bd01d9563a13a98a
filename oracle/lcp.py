"""Contacts, the sparse contact Jacobian D, BBPGD and one Euler step -- oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Yan et al., arXiv 1909.06623.
  * Sec. 3.2: the constraint set A(C, delta) = {pairs with Phi <= delta}.
    Phi_ij = |c_i - c_j| - R_i - R_j for spheres, with R the collision radius
    a_c (Sec. 6.1 sets a_c slightly above a).  Readings: delta is an absolute
    distance (the workloads quote "contact cutoff 0.1").  The paper's own
    choice, 30% of the sum of the radii, is the option delta_rel: the pair's
    threshold is delta + delta_rel (a_i + a_j), a the sphere radii (not the
    collision radii), evaluated in that order; pairs i < j sorted by (i, j);
    d^2 = (dx dx + dy dy) + dz dz evaluated without fused multiply-add, so the
    list is reproducible to the bit.
  * eq. Dmatdef / Dtranspose: column D_l carries -n_l on sphere i's force and
    +n_l on sphere j's force (no torque for spheres), n_l = (c_j - c_i)/|c_j - c_i|,
    so D^T U = n_l . (U_j - U_i) = dPhi/dt.
  * eq. lcp:LCPdef: M = D^T M D, q = Phi/dt + D^T U_nc.
  * Algorithm 1 (BBPGD) with the min-map residual of eq. mmapnorm and the BB1
    step (BB2 optional; variant 3 alternates BB1 on odd and BB2 on even
    steps, the alternation the paper mentions for Algorithm 1).
  * APGD (Sec. 3.3.1 cites it as the comparison method, no listing): Nesterov's
    accelerated projected gradient with an adaptive Lipschitz estimate
    (Mazhar et al. 2015): the gradient at the extrapolated point y is formed
    with its own product M y, the step 1/L is halved until the sufficient-
    decrease test f(x) <= f(y) + g(y).(x - y) + L/2 |x - y|^2 holds, the momentum
    restarts when g(x).(x - x_old) > 0, L shrinks by 0.9 after each accepted
    step, L_0 from |M (e - 0)| / |e| for the vector of ones e, stop on the
    min-map residual of eq. mmapnorm at the new iterate.  Readings where the algorithm is silent: gamma_0 = 0,
    whose product M gamma_0 = 0 needs no mobility solve; a non-positive s^T y
    (or y^T y for BB2) stops with status "breakdown", or, with safeguard=True,
    keeps the previous step length and continues (the discrete mobility is
    symmetric only to discretisation accuracy, so s^T M s can turn
    non-positive for nearly touching spheres at low order p); j_max caps the
    loop.
  * Failure rule (keep_best=True; Algorithm 1 says nothing about a loop that
    ends without meeting eps_tol): a residual at or above GROWTH_LIMIT times
    max(phi_0, eps_tol) stops with "breakdown" (an indefinite discrete M makes
    the projected steps grow without bound), and whenever the loop stops
    without meeting eps_tol (breakdown, growth or j_max) the iterate of
    smallest residual among gamma_0, gamma_1, ... is returned (the earliest
    on ties).  Off by default.
  * Walls (Sec. 3.3.3, "Extensions"): a boundary does not enter the
    mobility; each particle-boundary pair adds a column to D with nonzero
    entries on that particle only.  A wall here is a plane n.x = d with unit
    normal n pointing into the fluid: Phi = (n.c_i - d) - R_i, in the set
    when Phi <= delta + delta_rel a_i (the wall has no radius; a reading),
    column +n on sphere i (the wall acts as a static first body, so
    D^T U = n.U_i).  Wall contacts follow the pair contacts, sorted by
    (sphere, wall), recorded as (-1 - w, i).
  * Minimum-map Newton (Sec. 3.3.1 names it, after Niebe and Erleben 2015,
    as the second-order alternative it rejects; no listing): a root of
    H(gamma) = min(gamma, g) (eq. mmapnorm) by Newton steps J Delta = -H with
    J the element of the generalised Jacobian taking row l of M where
    g_l < gamma_l (the set F) and row l of the identity elsewhere.  Readings
    where the paper is silent: the step splits into Delta_l = -gamma_l off F
    and M_FF Delta_F = -(g + M [0; Delta_off F])_F, solved "iteratively" by
    conjugate gradients from 0 to relative residual NEWTON_CG_TOL (at most
    NEWTON_CG_MAX products); M Delta is the sum of those products with the CG
    coefficients, so g(gamma + t Delta) = g + t M Delta costs no further
    product; t = 1, halved (at most NEWTON_HALVINGS times, else "breakdown")
    until the Armijo test |H(gamma + t Delta)|^2 <= (1 - 2 sigma t) |H(gamma)|^2,
    sigma = NEWTON_SIGMA; gamma_0 = 0; stop on eq. mmapnorm below eps_tol.
    gamma may end with entries down to -eps_tol (H is zero at the root, not
    the projection).
  * eq. time-step: C^{k+1} = C^k + (U_nc + M D gamma) dt, positions only
    (spheres are isotropic; the grid keeps its lab-frame orientation).
"""
import itertools

import numpy as np

from . import mobility
from .layer import Suspension


def build_contacts(centers, radii, delta, a_c_scale=1.0, delta_rel=0.0):
    """Contact list (Sec. 3.2): ij (n_c x 2, i < j), Phi (n_c), normals (n_c x 3)."""
    c = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    a = np.asarray(radii, dtype=np.float64).reshape(-1)
    R = a * a_c_scale
    ij, ph, nr = [], [], []
    N = len(R)
    for i in range(N):
        for j in range(i + 1, N):
            dx = c[j, 0] - c[i, 0]
            dy = c[j, 1] - c[i, 1]
            dz = c[j, 2] - c[i, 2]
            # numpy float64 scalars: every operation rounded separately (no FMA)
            d2 = (dx * dx + dy * dy) + dz * dz
            d = np.sqrt(d2)
            phi = (d - R[i]) - R[j]
            if phi <= delta + delta_rel * (a[i] + a[j]):
                ij.append((i, j))
                ph.append(phi)
                nr.append((dx / d, dy / d, dz / d))
    return (np.array(ij, dtype=np.int32).reshape(-1, 2),
            np.array(ph, dtype=np.float64), np.array(nr, dtype=np.float64).reshape(-1, 3))


def build_wall_contacts(centers, radii, walls, delta, a_c_scale=1.0, delta_rel=0.0):
    """Particle-wall contacts (Sec. 3.3.3): for every sphere i (ascending) and
    wall w (ascending) with Phi = (n_w . c_i - d_w) - R_i <= delta +
    delta_rel a_i.  walls: W x 4 rows (n_x, n_y, n_z, d), n a unit normal
    into the fluid.  Returns ij rows (-1 - w, i), Phi, normals n_w."""
    c = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    a = np.asarray(radii, dtype=np.float64).reshape(-1)
    W = np.asarray(walls, dtype=np.float64).reshape(-1, 4)
    ij, ph, nr = [], [], []
    for i in range(len(a)):
        for w in range(len(W)):
            n = W[w, :3]
            # every operation rounded separately, in this order
            h = (n[0] * c[i, 0] + n[1] * c[i, 1]) + n[2] * c[i, 2]
            phi = (h - W[w, 3]) - a[i] * a_c_scale
            if phi <= delta + delta_rel * a[i]:
                ij.append((-1 - w, i))
                ph.append(phi)
                nr.append(tuple(n))
    return (np.array(ij, dtype=np.int32).reshape(-1, 2),
            np.array(ph, dtype=np.float64), np.array(nr, dtype=np.float64).reshape(-1, 3))


def D_apply(N, ij, nrm, gamma):
    """F_c = D gamma (N x 6, torques zero), eq. Dmatdef; a wall contact
    (first index negative) acts on its sphere only."""
    FT = np.zeros((N, 6))
    for l, (i, j) in enumerate(ij):
        if i >= 0:
            FT[i, :3] -= gamma[l] * nrm[l]
        FT[j, :3] += gamma[l] * nrm[l]
    return FT


def DT_apply(ij, nrm, UO):
    """(D^T U)_l = n_l . (U_j - U_i), eq. Dtranspose (a wall does not move)."""
    return np.array([nrm[l] @ (UO[j, :3] - (UO[i, :3] if i >= 0 else 0.0))
                     for l, (i, j) in enumerate(ij)])


def minmap(gamma, g):
    """phi(gamma, g) = || min(gamma, g) ||_2, eq. mmapnorm."""
    return float(np.linalg.norm(np.minimum(gamma, g)))


GROWTH_LIMIT = 1e6


def bbpgd(Mop, q, tol, jmax=10000, variant=1, safeguard=False, gamma0=None, keep_best=False):
    """Algorithm 1.  Mop(gamma) -> M gamma.  gamma0: the algorithm's initial
    guess (default 0, the paper's choice, whose product M gamma_0 = 0 needs no
    evaluation).  keep_best: the failure rule of the module docstring.
    Returns gamma, g, info; info["history"] lists the residual of every
    iterate (gamma_0 first) and info["best"] the index of the one returned."""
    q = np.asarray(q, dtype=np.float64)
    mv = 0
    if gamma0 is None or not np.any(gamma0):
        gamma = np.zeros_like(q)
        g = q.copy()                               # M gamma_0 = 0 for gamma_0 = 0
    else:
        gamma = np.asarray(gamma0, dtype=np.float64).copy()
        g = Mop(gamma) + q
        mv += 1
    phi0 = minmap(gamma, g)
    info = {"iters": 0, "mvops": mv, "status": "ok", "phi": phi0, "safeguards": 0,
            "history": [phi0], "best": 0}
    if phi0 < tol:
        return gamma, g, info
    Mg = Mop(g)
    mv += 1
    gMg = g @ Mg
    if not gMg > 0:
        info.update(status="breakdown", mvops=mv)
        return gamma, g, info
    alpha = (g @ g) / gMg
    best = (phi0, 0, gamma, g)
    limit = GROWTH_LIMIT * max(phi0, tol)

    def stop(status):
        info["status"] = status
        if keep_best and best[1] != info["iters"]:
            info.update(phi=best[0], best=best[1])
            return best[2], best[3], info
        return gamma, g, info

    for j in range(1, jmax + 1):
        gamma_new = np.maximum(gamma - alpha * g, 0.0)
        g_new = Mop(gamma_new) + q
        mv += 1
        phi = minmap(gamma_new, g_new)
        s = gamma_new - gamma
        y = g_new - g
        gamma, g = gamma_new, g_new
        info.update(iters=j, mvops=mv, phi=phi, best=j)
        info["history"].append(phi)
        if phi < tol:
            return gamma, g, info
        if phi < best[0]:
            best = (phi, j, gamma, g)
        if keep_best and not phi < limit:
            return stop("breakdown")
        sy = s @ y
        yy = y @ y
        ok = sy > 0 if variant == 1 else (sy > 0 and yy > 0)
        if not ok:
            if not safeguard:
                return stop("breakdown")
            info["safeguards"] += 1          # keep the previous step length
            continue
        bb1 = variant == 1 or (variant == 3 and j % 2 == 1)
        alpha = (s @ s) / sy if bb1 else sy / yy
    return stop("not_converged")


def apgd(Mop, q, tol, jmax=10000):
    """APGD for the CQP of eq. CQPdef (see the module docstring).  Mop(x) ->
    M x.  f(x) = x.M x / 2 + q.x.  Returns gamma, g, info (info["mvops"]
    counts the evaluations of M, the expensive part)."""
    q = np.asarray(q, dtype=np.float64)
    n = len(q)
    mv = 0
    gam = np.zeros(n)
    g0 = q.copy()                                   # M 0 + q
    info = {"iters": 0, "mvops": 0, "status": "ok", "phi": minmap(gam, g0)}
    if info["phi"] < tol:
        return gam, g0, info
    e = np.ones(n)
    L = np.linalg.norm(Mop(e)) / np.linalg.norm(e)
    mv += 1
    t = 1.0 / L
    y, theta = gam.copy(), 1.0
    Mgam = np.zeros(n)
    for k in range(1, jmax + 1):
        My = Mop(y) if np.any(y) else np.zeros(n)   # the gradient at the extrapolated point
        mv += int(np.any(y))
        gy = My + q
        for _ in range(200):                        # doubling L: bounded by the largest eigenvalue
            x = np.maximum(y - t * gy, 0.0)
            Mx = Mop(x)
            mv += 1
            d = x - y
            # f(x) <= f(y) + g(y).d + L/2 |d|^2, written for the quadratic f as
            # d.M d <= L |d|^2 (exact; free of the cancellation in f(x) - f(y))
            if d @ (Mx - My) <= L * (d @ d):
                break
            L *= 2.0
            t = 1.0 / L
        gx = Mx + q
        phi = minmap(x, gx)
        info.update(iters=k, mvops=mv, phi=phi)
        if phi < tol:
            return x, gx, info
        theta_new = 0.5 * (-theta * theta + theta * np.sqrt(theta * theta + 4.0))
        beta = theta * (1.0 - theta) / (theta * theta + theta_new)
        y_new = x + beta * (x - gam)
        if gx @ (x - gam) > 0:                      # restart the momentum
            y_new, theta_new = x.copy(), 1.0
        gam, Mgam, y, theta = x, Mx, y_new, theta_new
        L *= 0.9
        t = 1.0 / L
    info["status"] = "not_converged"
    return gam, Mgam + q, info


NEWTON_CG_TOL = 1e-3     # relative residual of the CG solve of each Newton system
NEWTON_CG_MAX = 200
NEWTON_SIGMA = 1e-4      # Armijo constant of the line search on theta = |H|^2 / 2
NEWTON_HALVINGS = 30


def minmap_newton(Mop, q, tol, jmax=100):
    """Minimum-map Newton for the LCP of eq. lcp:LCPdef (see the module
    docstring): a root of H(gamma) = min(gamma, g), g = M gamma + q.  Mop(x) ->
    M x.  Returns gamma, g, info (info["mvops"] counts products of M,
    info["cg_iters"] the CG iterations over all Newton steps)."""
    q = np.asarray(q, dtype=np.float64)
    n = len(q)
    gam = np.zeros(n)
    g = q.copy()                                    # M 0 + q
    phi = minmap(gam, g)
    info = {"iters": 0, "mvops": 0, "cg_iters": 0, "status": "ok", "phi": phi}
    if phi < tol:
        return gam, g, info
    mv = cg = 0
    for k in range(1, jmax + 1):
        # Jacobian of H: row l of M where H_l = g_l (g_l < gamma_l, the set F),
        # row l of the identity elsewhere (ties included)
        free = g < gam
        dC = np.where(free, 0.0, -gam)              # identity rows: Delta_l = -gamma_l
        MdC = np.zeros(n)
        if np.any(dC):
            MdC = Mop(dC)
            mv += 1
        # M_FF Delta_F = -(g + M dC)_F by CG from 0; the unmasked products of
        # the search directions add up to M [Delta_F; 0]
        b = np.where(free, -g - MdC, 0.0)
        x, MxF = np.zeros(n), np.zeros(n)
        r = b.copy()
        pd = r.copy()
        rr = r @ r
        bnorm = np.sqrt(rr)
        for _ in range(NEWTON_CG_MAX):
            if np.sqrt(rr) <= NEWTON_CG_TOL * bnorm:
                break
            Mp = Mop(pd)
            mv += 1
            cg += 1
            Ap = np.where(free, Mp, 0.0)
            pAp = pd @ Ap
            if not pAp > 0:
                break
            a = rr / pAp
            x += a * pd
            MxF += a * Mp
            r -= a * Ap
            rr_new = r @ r
            pd = r + (rr_new / rr) * pd
            rr = rr_new
        d = x + dC
        Md = MxF + MdC
        # Armijo backtracking on theta: the exact Newton direction has
        # directional derivative -2 theta, so accept theta(t) <= (1 - 2 sigma t) theta(0)
        theta0 = 0.5 * phi * phi
        t, accepted = 1.0, False
        for _ in range(NEWTON_HALVINGS + 1):
            gam_t, g_t = gam + t * d, g + t * Md
            phi_t = minmap(gam_t, g_t)
            if 0.5 * phi_t * phi_t <= (1.0 - 2.0 * NEWTON_SIGMA * t) * theta0:
                accepted = True
                break
            t *= 0.5
        info.update(mvops=mv, cg_iters=cg)
        if not accepted:
            info["status"] = "breakdown"
            return gam, g, info
        gam, g, phi = gam_t, g_t, phi_t
        info.update(iters=k, phi=phi)
        if phi < tol:
            return gam, g, info
    info["status"] = "not_converged"
    return gam, g, info


def lcp_enumerate(Mmat, q):
    """Exact LCP solution by trying every active set (small n_c only).

    M SPD gives a unique solution (Sec. 3.3.2): the set S with
    gamma_S = -M_SS^{-1} q_S >= 0 and (M gamma + q)_{not S} >= 0.
    """
    n = len(q)
    best = None
    for k in range(n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            gam = np.zeros(n)
            if S:
                gam[S] = np.linalg.solve(Mmat[np.ix_(S, S)], -q[S])
            w = Mmat @ gam + q
            rest = [i for i in range(n) if i not in S]
            if np.all(gam[S] >= -1e-12) and np.all(w[rest] >= -1e-12):
                best = gam
                return best
    return best


def _all_contacts(centers, radii, delta, a_c_scale, delta_rel, walls):
    ij, phi, nrm = build_contacts(centers, radii, delta, a_c_scale, delta_rel)
    if walls is None or len(walls) == 0:
        return ij, phi, nrm
    wij, wphi, wn = build_wall_contacts(centers, radii, walls, delta, a_c_scale, delta_rel)
    return np.concatenate([ij, wij]), np.concatenate([phi, wphi]), np.concatenate([nrm, wn])


def resolve_collisions(centers, radii, FT_ext, dt, p, *, beta=1.75, delta=0.1,
                       a_c_scale=1.0, gmres_tol=1e-12, gmres_max=200,
                       bbpgd_tol=1e-10, bbpgd_max=10000, variant=1, safeguard=False,
                       delta_rel=0.0, rotations=None, keep_best=False, walls=None,
                       solver="bbpgd"):
    """One collision-resolved Euler step (Sec. 3.2, four-step procedure).

    1. U_nc = M F_ext; 2. contacts and D; 3. BBPGD for gamma with
    M gamma = D^T M D gamma; 4. U = U_nc + M D gamma, c += U dt.
    keep_best: the failure rule of bbpgd; U then uses M D gamma of the
    iterate returned.  walls: optional W x 4 planes (see build_wall_contacts).
    Returns dict with gamma, ij, phi, normals, U (N x 6), centers_new, info.
    """
    sus = Suspension(centers, radii, p, beta, rotations)
    U_nc, inf0 = mobility.mobility_apply(sus, FT_ext, gmres_tol, gmres_max, return_info=True)
    ij, phi0, nrm = _all_contacts(centers, radii, delta, a_c_scale, delta_rel, walls)
    q = phi0 / dt + DT_apply(ij, nrm, U_nc)
    state = {"U_c": np.zeros_like(U_nc), "solves": 1, "gmres": inf0["gmres_iters"]}

    def Mop(gam):
        UO, inf = mobility.mobility_apply(sus, D_apply(sus.N, ij, nrm, gam),
                                          gmres_tol, gmres_max, return_info=True)
        state["U_c"] = UO
        state["U_c_of"].append(UO)
        state["solves"] += 1
        state["gmres"] += inf["gmres_iters"]
        return DT_apply(ij, nrm, UO)

    state["U_c_of"] = []
    if solver in ("apgd", "newton"):
        if solver == "apgd":
            gamma, g, info = apgd(Mop, q, bbpgd_tol, bbpgd_max)
        else:
            gamma, g, info = minmap_newton(Mop, q, bbpgd_tol, bbpgd_max)
        info["best"] = info["iters"]
        # U_c of the returned iterate: one more solve (the products of APGD
        # and Newton are not products of the iterates)
        U_c = (mobility.mobility_apply(sus, D_apply(sus.N, ij, nrm, gamma), gmres_tol, gmres_max)
               if np.any(gamma) else np.zeros_like(U_nc))
    else:
        gamma, g, info = bbpgd(Mop, q, bbpgd_tol, bbpgd_max, variant, safeguard, keep_best=keep_best)
    if solver in ("apgd", "newton"):
        pass
    elif info["iters"] == 0 or info["best"] == 0:
        U_c = np.zeros_like(U_nc)       # gamma = gamma_0 = 0
    else:
        # the solve of the returned iterate: Mop's calls are M g_0, then one
        # per iterate gamma_1, gamma_2, ...
        U_c = state["U_c_of"][info["best"]]
    U = U_nc + U_c
    cnew = np.asarray(centers, dtype=np.float64) + U[:, :3] * dt
    info.update(solves=state["solves"], gmres_iters=state["gmres"], n_contacts=len(q),
                n_active=int(np.sum(gamma > 0)))
    return {"gamma": gamma, "g": g, "q": q, "ij": ij, "phi": phi0, "normals": nrm,
            "U": U, "U_nc": U_nc, "centers_new": cnew, "info": info}


# ----------------------------------------------------------------------------
# Large contact sets: one sphere's row, vectorised D / D^T, identity mobility
# ----------------------------------------------------------------------------
def contacts_of_sphere(centers, radii, i, delta, a_c_scale=1.0, delta_rel=0.0):
    """Row i of the contact set of Sec. 3.2: every j > i with Phi_ij <= delta.

    The same arithmetic as build_contacts, element-wise over all j at once
    (numpy rounds each array operation separately, so the values agree to the
    bit).  Returns (j ascending, Phi, normals)."""
    c = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    a = np.asarray(radii, dtype=np.float64).reshape(-1)
    cj = c[i + 1:]
    dx = cj[:, 0] - c[i, 0]
    dy = cj[:, 1] - c[i, 1]
    dz = cj[:, 2] - c[i, 2]
    d = np.sqrt((dx * dx + dy * dy) + dz * dz)
    phi = (d - a[i] * a_c_scale) - a[i + 1:] * a_c_scale
    k = np.nonzero(phi <= delta + delta_rel * (a[i] + a[i + 1:]))[0]
    nrm = np.stack([dx[k] / d[k], dy[k] / d[k], dz[k] / d[k]], axis=1)
    return (k + i + 1).astype(np.int64), phi[k], nrm


def D_apply_vec(N, ij, nrm, gamma):
    """D gamma of eq. Dmatdef for large contact sets (unbuffered scatter-add);
    sphere pairs only (no wall contacts)."""
    assert np.all(np.asarray(ij)[:, 0] >= 0)
    FT = np.zeros((N, 6))
    f = np.asarray(gamma, dtype=np.float64)[:, None] * np.asarray(nrm, dtype=np.float64)
    for c in range(3):
        np.add.at(FT[:, c], ij[:, 0], -f[:, c])
        np.add.at(FT[:, c], ij[:, 1], f[:, c])
    return FT


def DT_apply_vec(ij, nrm, UO):
    """D^T U of eq. Dtranspose for large contact sets (sphere pairs only)."""
    assert np.all(np.asarray(ij)[:, 0] >= 0)
    dU = UO[ij[:, 1], :3] - UO[ij[:, 0], :3]
    return np.einsum("lc,lc->l", nrm, dU)


def resolve_collisions_identity(centers, radii, FT_ext, dt, *, delta=0.1, a_c_scale=1.0,
                                bbpgd_tol=1e-10, bbpgd_max=10000, variant=1, safeguard=False,
                                delta_rel=0.0, walls=None, solver="bbpgd"):
    """The collision step of Sec. 3.2 with the mobility replaced by the
    identity (U = F, Omega = T).  No fluid: M = D^T D is the constraint Gram
    matrix, which isolates contacts, D products and Algorithm 1 at sizes where
    no N-body sum could run.  Returns the same dict as resolve_collisions."""
    C = np.asarray(centers, dtype=np.float64)
    FT_ext = np.asarray(FT_ext, dtype=np.float64).reshape(-1, 6)
    N = len(C)
    ij, phi0, nrm = _all_contacts(C, radii, delta, a_c_scale, delta_rel, walls)
    U_nc = FT_ext.copy()
    q = phi0 / dt + DT_apply(ij, nrm, U_nc)
    state = {"U_c": np.zeros_like(U_nc)}

    def Mop(gam):
        state["U_c"] = D_apply(N, ij, nrm, gam)
        return DT_apply(ij, nrm, state["U_c"])

    if solver in ("apgd", "newton"):
        if solver == "apgd":
            gamma, g, info = apgd(Mop, q, bbpgd_tol, bbpgd_max)
        else:
            gamma, g, info = minmap_newton(Mop, q, bbpgd_tol, bbpgd_max)
        U_c = D_apply(N, ij, nrm, gamma)
    else:
        gamma, g, info = bbpgd(Mop, q, bbpgd_tol, bbpgd_max, variant, safeguard)
        U_c = np.zeros_like(U_nc) if info["iters"] == 0 else state["U_c"]
    U = U_nc + U_c
    info.update(n_contacts=len(q), n_active=int(np.sum(gamma > 0)))
    return {"gamma": gamma, "g": g, "q": q, "ij": ij, "phi": phi0, "normals": nrm,
            "U": U, "U_nc": U_nc, "centers_new": C + U[:, :3] * dt, "info": info}
