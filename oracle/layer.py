"""Stokes layer potentials on spheres -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Yan et al., arXiv 1909.06623.
  * Kernels and operators -- Sec. 4.1: Stokeslet G_ij = (delta_ij/|r| +
    r_i r_j/|r|^3)/(8 pi), traction kernel T_ijk = -3 r_i r_j r_k/(4 pi |r|^5),
    viscosity 1; single layer S[rho](x) = int G(x-y) rho(y) dS_y and traction
    operator K[rho](x) = int T(x-y) n(x) rho(y) dS_y.  T is symmetric in all
    three indices, so K[rho]_i(x) = -3/(4 pi) int (r.rho)(r.n(x)) r_i/|r|^5.
  * Far field -- Sec. 5.1: plain quadrature over the surface nodes of every
    other sphere (the paper evaluates the same sums with KIFMM).
  * Near and self field -- Sec. 4.2 and 5.4: the VSH coefficients of a sphere's
    density give its exterior single-layer velocity and pressure (eq. ssgshexp,
    ssgext); the traction is (-p I + grad u + grad u^T) n (Sec. 4.2), with grad u
    taken from the closed-form expansion.  Near pairs: centre distance below
    beta (R_i + R_j) (Sec. 4.2).

Readings of the paper taken here:
  * eq. ssgext, f^V: the rho^W term is printed with (n+1)/(4n+2).  Solving
    the Stokes equations with the single-layer jump conditions gives n/(4n+2)
    (the on-surface value r = 1 is the same either way, the off-surface field
    is not).  This module uses n/(4n+2); tests pin it against direct quadrature
    of the Stokeslet at well-separated targets.
  * Near pairs are excluded from the far quadrature and their VSH value is
    added instead (Sec. 4.2 says the VSH value replaces the inaccurate one).
  * The traction operator's self part is the on-surface principal value:
    K_self[s] = t_ext(s) + P(s)/2, where t_ext is the exterior traction of the
    sphere's own single layer at r -> 1+ and P(s) = synthesis(analysis(s)) is
    the band-limited part of s; the 1/2 I of eq. rigidbodyrho acts on the grid
    values themselves.
  * grad u is written in the spherical frame of the source sphere with the
    textbook formulas for the gradient of a vector field; targets closer than
    sin(theta) < 1e-3 to that frame's polar axis are evaluated in a frame
    rotated by 90 degrees about the x axis (the density is re-expanded there).
"""
from math import pi

import numpy as np

from . import sph

POLE_GUARD = 1e-3


# ----------------------------------------------------------------------------
# kernels and far-field quadrature (Sec. 4.1, 5.1)
# ----------------------------------------------------------------------------
def stokeslet(r):
    """G(r) for r (..., 3) -> (..., 3, 3)."""
    d = np.sqrt(np.sum(r * r, axis=-1))
    eye = np.eye(3)
    return (eye / d[..., None, None]
            + r[..., :, None] * r[..., None, :] / d[..., None, None] ** 3) / (8 * pi)


def traction_kernel(r):
    """T(r) for r (..., 3) -> (..., 3, 3, 3)."""
    d = np.sqrt(np.sum(r * r, axis=-1))
    return (-3.0 / (4 * pi) * r[..., :, None, None] * r[..., None, :, None]
            * r[..., None, None, :] / d[..., None, None, None] ** 5)


def near_lists(centers, radii, beta):
    """near[i] = sorted j != i with |c_i - c_j| < beta (R_i + R_j) (Sec. 4.2)."""
    c = np.asarray(centers, dtype=np.float64)
    a = np.asarray(radii, dtype=np.float64)
    out = []
    for i in range(len(a)):
        d = np.sqrt(np.sum((c - c[i]) ** 2, axis=1))
        m = d < beta * (a + a[i])
        m[i] = False
        out.append(np.nonzero(m)[0])
    return out


def far_sum(op, Xt, Nt, sph_t, Xs, Ws, Ss, sph_s, excl, chunk=2048):
    """Direct quadrature over source nodes whose sphere is not excluded.

    op 'S': u(x) = sum_y w_y G(x - y) sigma(y)
    op 'K': t(x) = sum_y w_y T(x - y) : sigma(y) n(x)
    excl(i) -> set of source spheres skipped for target sphere i.
    """
    out = np.zeros_like(Xt)
    # targets per pass: each pass holds a few (targets x sources) arrays, so
    # the chunk shrinks with the source count (the per-target sums do not change)
    chunk = max(1, min(chunk, int(4e6 // max(len(Xs), 1))))
    for i0 in range(0, len(Xt), chunk):
        i1 = min(i0 + chunk, len(Xt))
        r = Xt[i0:i1, None, :] - Xs[None, :, :]
        mask = np.ones((i1 - i0, len(Xs)), dtype=bool)
        for ii in range(i0, i1):
            ex = excl(sph_t[ii])
            if len(ex):
                mask[ii - i0] = ~np.isin(sph_s, ex)
        ws = np.where(mask, Ws[None, :], 0.0)
        d2 = np.sum(r * r, axis=-1)
        d2 = np.where(mask, d2, 1.0)
        inv = 1.0 / np.sqrt(d2)
        rs = np.sum(r * Ss[None, :, :], axis=-1)
        if op == "S":
            term = (Ss[None, :, :] * inv[..., None]
                    + r * (rs * inv ** 3)[..., None]) / (8 * pi)
        else:
            rn = np.sum(r * Nt[i0:i1, None, :], axis=-1)
            term = (-3.0 / (4 * pi)) * r * (rs * rn * inv ** 5)[..., None]
        out[i0:i1] = np.sum(ws[..., None] * term, axis=1)
    return out


# ----------------------------------------------------------------------------
# exterior single-layer field of one unit sphere (Sec. 4.2, eq. ssgext)
# ----------------------------------------------------------------------------
def radial_factors(n, coef_nm, r):
    """f^V, f^W, f^X, g and their r-derivatives for one (n, m) (eq. ssgext).

    coef_nm = (sV, sW, sX), the multipliers of V, W, X in eq. rhoshexp.
    """
    sV, sW, sX = coef_nm
    rp2, rp1, rp0 = r ** -(n + 2.0), r ** -(n + 1.0), r ** -(n + 0.0)
    A1 = n * sV / ((2 * n + 1) * (2 * n + 3))
    A2 = n * sW / (2.0 * (2 * n + 1))          # printed as (n+1)/(4n+2): see module doc
    B = (n + 1) * sW / ((2 * n + 1) * (2 * n - 1))
    C = sX / (2 * n + 1)
    fV = A1 * rp2 + A2 * (rp2 - rp0)
    fW = B * rp0
    fX = C * rp1
    g = n * sW * rp1
    dfV = -(n + 2) * A1 * rp2 / r + A2 * (-(n + 2) * rp2 + n * rp0) / r
    dfW = -n * B * rp0 / r
    dfX = -(n + 1) * C * rp1 / r
    return fV, fW, fX, g, dfV, dfW, dfX


def _exterior_unit_frame(coef, p, xt):
    """u, p, grad u (grad_ij = d_i u_j) of the unit sphere's single layer at xt.

    xt: (M, 3) points outside the unit sphere centred at the origin, none near
    the polar axis.  Spherical-frame formulas, rotated to Cartesian.
    """
    r = np.sqrt(np.sum(xt * xt, axis=1))
    theta = np.arccos(np.clip(xt[:, 2] / r, -1.0, 1.0))
    phi = np.arctan2(xt[:, 1], xt[:, 0])
    s, t = np.sin(theta), np.cos(theta)
    M = len(r)
    z = lambda: np.zeros(M, dtype=np.complex128)
    ur, ut, uf = z(), z(), z()
    dr_ur, dr_ut, dr_uf = z(), z(), z()
    dt_ur, dt_ut, dt_uf = z(), z(), z()
    dp_ur, dp_ut, dp_uf = z(), z(), z()
    pres = z()
    for (n, m), cf in coef.items():
        if n == 0:
            continue  # W_0 = X_0 = 0 and f^V carries a factor n: no exterior field
        fV, fW, fX, g, dfV, dfW, dfX = radial_factors(n, cf, r)
        y = sph.ylm_parts(n, m, theta, phi)
        Y, Yt, Ytt, Ys, Yts = y["Y"], y["Yt"], y["Ytt"], y["Ys"], y["Yts"]
        im = 1j * m
        rad, drad = n * fW - (n + 1) * fV, n * dfW - (n + 1) * dfV
        tan, dtan = fV + fW, dfV + dfW
        ur += rad * Y
        ut += tan * Yt - fX * im * Ys
        uf += tan * im * Ys + fX * Yt
        dr_ur += drad * Y
        dr_ut += dtan * Yt - dfX * im * Ys
        dr_uf += dtan * im * Ys + dfX * Yt
        dt_ur += rad * Yt
        dt_ut += tan * Ytt - fX * im * Yts
        dt_uf += tan * im * Yts + fX * Ytt
        dp_ur += rad * im * Y
        dp_ut += tan * im * Yt + fX * m * m * Ys
        dp_uf += -tan * m * m * Ys + fX * im * Yt
        pres += g * Y
    cot = t / s
    Gs = np.zeros((M, 3, 3), dtype=np.complex128)
    Gs[:, 0, 0], Gs[:, 0, 1], Gs[:, 0, 2] = dr_ur, dr_ut, dr_uf
    Gs[:, 1, 0] = (dt_ur - ut) / r
    Gs[:, 1, 1] = (dt_ut + ur) / r
    Gs[:, 1, 2] = dt_uf / r
    Gs[:, 2, 0] = (dp_ur / s - uf) / r
    Gs[:, 2, 1] = (dp_ut / s - uf * cot) / r
    Gs[:, 2, 2] = (dp_uf / s + ur + ut * cot) / r
    er, et, ep = sph.frame(theta, phi)
    R = np.stack([er, et, ep], axis=2)  # columns are the local basis vectors
    u = (R @ np.stack([ur, ut, uf], axis=1)[..., None])[..., 0]
    gradu = R @ Gs @ np.transpose(R, (0, 2, 1))
    for name, v in (("u", u), ("p", pres), ("grad u", gradu)):
        scale = max(1.0, float(np.max(np.abs(v))))
        assert np.max(np.abs(v.imag)) <= 1e-9 * scale, name
    return u.real, pres.real, gradu.real


_ROT = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])


def _rotated_coef(coef, p):
    """Coefficients of s'(y) = R^T s(R y): the density seen from the rotated frame."""
    theta, phi, nrm, _ = sph.unit_grid(p)
    yr = nrm @ _ROT.T                                  # R y for every grid node
    th = np.arccos(np.clip(yr[:, 2], -1.0, 1.0))
    ph = np.arctan2(yr[:, 1], yr[:, 0])
    vals = sph.synthesis(coef, p, th, ph)              # s(R y)
    return sph.analysis(vals @ _ROT, p)                # R^T s(R y)


def exterior_unit(coef, p, xt):
    """u, p, grad u of the unit sphere's single layer; pole-safe dispatch."""
    xt = np.asarray(xt, dtype=np.float64).reshape(-1, 3)
    r = np.sqrt(np.sum(xt * xt, axis=1))
    sinth = np.sqrt(xt[:, 0] ** 2 + xt[:, 1] ** 2) / r
    polar = sinth < POLE_GUARD
    u = np.zeros_like(xt)
    pr = np.zeros(len(xt))
    g = np.zeros((len(xt), 3, 3))
    if np.any(~polar):
        u[~polar], pr[~polar], g[~polar] = _exterior_unit_frame(coef, p, xt[~polar])
    if np.any(polar):
        cr = _rotated_coef(coef, p)
        xr = xt[polar] @ _ROT                          # R^T x
        ur, prr, gr = _exterior_unit_frame(cr, p, xr)
        u[polar] = ur @ _ROT.T
        pr[polar] = prr
        g[polar] = _ROT @ gr @ _ROT.T
    return u, pr, g


def traction(pres, gradu, n):
    """t = (-p I + grad u + grad u^T) n (Sec. 4.2)."""
    sym = gradu + np.transpose(gradu, (0, 2, 1))
    return -pres[:, None] * n + np.einsum("mij,mj->mi", sym, n)


def vsh_field(coef, p, center, radius, xt, normals=None):
    """S[sigma](x) and (optionally) its traction with target normals, for the
    single layer of one sphere of given centre and radius (scaled from the unit
    sphere: S_a[s](x) = a S_1[s](x~), traction is scale free, x~ = (x - c)/a)."""
    xt = (np.asarray(xt, dtype=np.float64) - center) / radius
    u, pr, g = exterior_unit(coef, p, xt)
    u = radius * u
    if normals is None:
        return u, None
    return u, traction(pr, g, normals)


# ----------------------------------------------------------------------------
# self part (Sec. 4.2, 5.4)
# ----------------------------------------------------------------------------
def self_terms(sig_sphere, p, radius):
    """S_self[s] and K_self[s] on one sphere's own grid.

    S_self = a * u_ext(r = 1);  K_self = t_ext(r -> 1+) + synthesis(analysis(s))/2
    (the on-surface principal value; see the module docstring).
    """
    coef = sph.analysis(sig_sphere, p)
    _, _, nrm, _ = sph.unit_grid(p)
    u, pr, g = exterior_unit(coef, p, nrm)
    tplus = traction(pr, g, nrm)
    proj = sph.grid_synthesis(coef, p)
    return radius * u, tplus + 0.5 * proj


# ----------------------------------------------------------------------------
# full layer operators on a suspension
# ----------------------------------------------------------------------------
class Suspension:
    """Geometry of N spheres of order p: nodes, normals, weights, near lists.

    rotations (optional, N x 3 x 3 orthogonal): the orientation Q_i of each
    sphere's grid (Sec. 5.4 orients every sphere's grid at random).  Node k of
    sphere i sits at c_i + a_i Q_i n_k; the sphere's VSH expansions live in its
    own frame, so densities are rotated into it (components Q_i^T s) before
    the analysis and fields evaluated from it are rotated back (Q_i u).
    Without rotations every Q_i is the identity."""

    def __init__(self, centers, radii, p, beta=1.75, rotations=None):
        self.c = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
        self.a = np.asarray(radii, dtype=np.float64).reshape(-1)
        self.p = p
        self.N = len(self.a)
        self.P = sph.nodes_per_sphere(p)
        self.beta = beta
        self.Q = None if rotations is None else np.asarray(rotations, dtype=np.float64).reshape(-1, 3, 3)
        self.X, self.Nrm, self.W = sph.sphere_nodes(self.c, self.a, p)
        if self.Q is not None:
            # rotate each sphere's unit grid: n_k -> Q_i n_k (rows: n_k^T Q_i^T)
            nrm = self.Nrm.reshape(self.N, self.P, 3)
            nrm = np.einsum("ikj,imj->ikm", nrm, self.Q)
            self.Nrm = nrm.reshape(-1, 3)
            self.X = (self.c[:, None, :] + self.a[:, None, None] * nrm).reshape(-1, 3)
        self.sph_of = np.repeat(np.arange(self.N), self.P)
        self.near = near_lists(self.c, self.a, beta)

    def to_local(self, j, v):
        """Vectors (rows) from the lab frame into sphere j's grid frame."""
        return v if self.Q is None else v @ self.Q[j]

    def to_lab(self, j, v):
        """Vectors (rows) from sphere j's grid frame into the lab frame."""
        return v if self.Q is None else v @ self.Q[j].T

    def nodes(self, i):
        return slice(i * self.P, (i + 1) * self.P)

    def apply(self, op, sig, targets=None):
        """S[sig] ('S') or K[sig] ('K') at the nodes: self + near + far.

        sig: (N*P, 3).  targets: optional list of sphere indices to evaluate
        (others are left zero) -- used for sampled parity at large N.
        """
        tg = range(self.N) if targets is None else targets
        out = np.zeros_like(self.X)
        coefs = {}

        def coef_of(j):
            if j not in coefs:
                coefs[j] = sph.analysis(self.to_local(j, sig[self.nodes(j)]), self.p)
            return coefs[j]

        for i in tg:
            sl = self.nodes(i)
            # self (in sphere i's grid frame)
            ss, ks = self_terms(self.to_local(i, sig[sl]), self.p, self.a[i])
            acc = self.to_lab(i, ss if op == "S" else ks).copy()
            # near: targets and normals in sphere j's frame, fields back
            for j in self.near[i]:
                xt = self.c[j] + self.to_local(j, self.X[sl] - self.c[j])
                nt = None if op == "S" else self.to_local(j, self.Nrm[sl])
                u, t = vsh_field(coef_of(j), self.p, self.c[j], self.a[j], xt, nt)
                acc += self.to_lab(j, u if op == "S" else t)
            out[sl] = acc
        # far
        tmask = np.zeros(self.N, dtype=bool)
        tmask[list(tg)] = True
        tn = tmask[self.sph_of]
        excl = lambda i: np.concatenate([[i], self.near[i]])
        out[tn] += far_sum(op, self.X[tn], self.Nrm[tn], self.sph_of[tn],
                           self.X, self.W, sig, self.sph_of, excl)
        return out
