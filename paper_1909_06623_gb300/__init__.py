"""GB300-native collision-resolving Stokes suspensions of rigid spheres.

Python front end of libsps.so (C ABI in include/sps.h).  Method: Yan, Corona,
Malhotra, Veerapaneni & Shelley, arXiv 1909.06623 -- BBPGD collision
resolution (Algorithm 1) around an indirect boundary-integral mobility solve
(Sec. 4) with VSH self / near-singular quadrature and an all-pairs far field.

The functions mirror the C entry points (same names without the ``sps_``
prefix on the methods of :class:`Context`); they only marshal arguments:
torch tensors provide device memory and the CUDA stream.
"""
import ctypes

import torch

from . import _lib
from ._lib import (SPS_FP64, SPS_FP64_DW, SPS_MIXED, SPS_MOB_BIE, SPS_MOB_IDENTITY, SPS_OP_A, SPS_OP_K,
                   SPS_OP_S, SPS_SEARCH_ALL_PAIRS, SPS_SEARCH_AUTO, SPS_SEARCH_CELLS, SPSError,
                   sps_params, sps_stats)

__all__ = ["Context", "SPSError", "SPS_FP64", "SPS_MIXED", "SPS_FP64_DW", "SPS_OP_S", "SPS_OP_K", "SPS_OP_A",
           "SPS_MOB_BIE", "SPS_MOB_IDENTITY", "SPS_SEARCH_AUTO", "SPS_SEARCH_ALL_PAIRS",
           "SPS_SEARCH_CELLS",
           "default_params", "unit_tables", "nodes_per_sphere", "MobilityFunction", "mobility",
           "CollisionStepFunction", "collision_step"]


def nodes_per_sphere(p):
    return (p + 1) * (2 * p + 2)


def default_params(**kw):
    lib = _lib.load()
    prm = sps_params()
    lib.sps_default_params(ctypes.byref(prm))
    for k, v in kw.items():
        if not hasattr(prm, k):
            raise KeyError(k)
        setattr(prm, k, v)
    return prm


def _ptr(t, dtype=torch.float64, device=True):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if device and not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not device and t.is_cuda:
        raise TypeError("expected a CPU tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def unit_tables(p):
    """Host-only: unit nodes (3 x P), weights (P), analysis (6NC x 3P), synthesis (3P x 6NC)."""
    import numpy as np
    lib = _lib.load()
    P = nodes_per_sphere(p)
    NC = (p + 1) * (p + 2) // 2
    nodes = np.zeros(3 * P)
    w = np.zeros(P)
    A = np.zeros(6 * NC * 3 * P)
    S = np.zeros(3 * P * 6 * NC)
    rc = lib.sps_unit_tables(p, nodes.ctypes.data, w.ctypes.data, A.ctypes.data, S.ctypes.data)
    if rc:
        raise SPSError(rc, "sps_unit_tables")
    return nodes.reshape(3, P), w, A.reshape(6 * NC, 3 * P), S.reshape(3 * P, 6 * NC)


class Context:
    """Owns an sps_ctx (device scratch, contact list) bound to a CUDA stream."""

    def __init__(self, stream=None, **params):
        self.lib = _lib.load()
        self.prm = default_params(**params)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.sps_create(ctypes.byref(self.prm), ctypes.c_void_p(stream.cuda_stream),
                                 ctypes.byref(h))
        if rc:
            raise SPSError(rc, "sps_create")
        self.h = h
        self.last_stats = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.sps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            raise SPSError(rc, self.lib.sps_last_error(self.h).decode())
        return rc

    @property
    def P(self):
        return nodes_per_sphere(self.prm.p)

    # ---- geometry and operators -------------------------------------------------
    def set_geometry(self, pos, radii):
        n = radii.numel()
        self._check(self.lib.sps_set_geometry(self.h, n, _ptr(pos), _ptr(radii)))
        self.n = n

    def set_orientation(self, Q):
        """Per-sphere grid rotations Q (n x 3 x 3 CUDA float64 tensor), or
        None for identity grids (sps_set_orientation)."""
        if Q is None:
            self._check(self.lib.sps_set_orientation(self.h, 0, None))
            return
        Q = Q.reshape(-1, 9).contiguous()
        self._check(self.lib.sps_set_orientation(self.h, Q.shape[0], _ptr(Q)))

    def set_walls(self, walls):
        """Planar walls: rows (n_x, n_y, n_z, d) of the planes n . x = d, unit
        normals into the fluid (sps_set_walls); None or empty removes them."""
        import numpy as np
        if walls is None or len(walls) == 0:
            self._check(self.lib.sps_set_walls(self.h, 0, None))
            return
        w = np.ascontiguousarray(np.asarray(walls, dtype=np.float64).reshape(-1, 4))
        self._check(self.lib.sps_set_walls(self.h, len(w), w.ctypes.data_as(ctypes.c_void_p)))

    def geometry_counts(self):
        """(directed near pairs, close near entries) of the current geometry."""
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.sps_geometry_counts(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def near_lists(self):
        """(near_ptr (N+1), near_idx) of the current geometry, int32 device tensors."""
        nn, _ = self.geometry_counts()
        ptr = torch.empty(self.n + 1, dtype=torch.int32, device="cuda")
        idx = torch.empty(max(nn, 1), dtype=torch.int32, device="cuda")
        self._check(self.lib.sps_near_lists(self.h, _ptr(ptr, torch.int32), _ptr(idx, torch.int32)))
        return ptr, idx[:nn]

    def nodes(self):
        NP = self.n * self.P
        X = torch.empty(3, NP, dtype=torch.float64, device="cuda")
        Nr = torch.empty_like(X)
        W = torch.empty(NP, dtype=torch.float64, device="cuda")
        np_out = ctypes.c_int()
        self._check(self.lib.sps_nodes(self.h, _ptr(X), _ptr(Nr), _ptr(W), ctypes.byref(np_out)))
        return X, Nr, W

    def layer_apply(self, op, sigma, out=None):
        if out is None:
            out = torch.empty_like(sigma)
        self._check(self.lib.sps_layer_apply(self.h, int(op), _ptr(sigma), _ptr(out)))
        return out

    def layer_apply_transpose(self, op, v, out=None):
        if out is None:
            out = torch.empty_like(v)
        self._check(self.lib.sps_layer_apply_transpose(self.h, int(op), _ptr(v), _ptr(out)))
        return out

    def mobility_adjoint(self, pos, radii, FT, dL_dU, want_pos=True, allow_not_converged=False):
        """(U, dL/dFT, dL/dpos or None) for a loss whose gradient in U is dL_dU."""
        n = radii.numel()
        UO = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        gF = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        gx = torch.empty(n, 3, dtype=torch.float64, device="cuda") if want_pos else None
        st = sps_stats()
        rc = self.lib.sps_mobility_adjoint(self.h, n, _ptr(pos), _ptr(radii), _ptr(FT),
                                           _ptr(dL_dU.contiguous()), _ptr(UO), _ptr(gF), _ptr(gx),
                                           ctypes.byref(st))
        self._check(rc, allow=(4,) if allow_not_converged else ())
        self.last_stats = st.as_dict()
        return UO, gF, gx

    def collision_adjoint(self, pos, radii, FT_ext, dt, dL_dU, want_pos=False, allow=()):
        """(U, dL/dF_ext, dL/dpos or None) of one collision-resolved step
        (positions are not advanced)."""
        n = radii.numel()
        UO = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        gF = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        gx = torch.empty(n, 3, dtype=torch.float64, device="cuda") if want_pos else None
        st = sps_stats()
        rc = self.lib.sps_collision_adjoint(self.h, n, _ptr(pos), _ptr(radii), _ptr(FT_ext), float(dt),
                                            _ptr(dL_dU.contiguous()), _ptr(UO), _ptr(gF), _ptr(gx),
                                            ctypes.byref(st))
        self._check(rc, allow=allow)
        self.last_stats = st.as_dict()
        self.n_c = st.n_contacts
        return UO, gF, gx

    def build_contacts(self, pos, radii):
        nc = ctypes.c_int()
        self._check(self.lib.sps_build_contacts(self.h, radii.numel(), _ptr(pos), _ptr(radii),
                                                ctypes.byref(nc)))
        self.n_c = nc.value
        return nc.value

    def get_contacts(self):
        nc = getattr(self, "n_c", 0)
        ij = torch.empty(max(nc, 1), 2, dtype=torch.int32, device="cuda")
        phi = torch.empty(max(nc, 1), dtype=torch.float64, device="cuda")
        nrm = torch.empty(max(nc, 1), 3, dtype=torch.float64, device="cuda")
        self._check(self.lib.sps_get_contacts(self.h, _ptr(ij, torch.int32), _ptr(phi), _ptr(nrm)))
        return ij[:nc], phi[:nc], nrm[:nc]

    def contact_force(self, gamma, n):
        FT = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        self._check(self.lib.sps_contact_force(self.h, _ptr(gamma), _ptr(FT)))
        return FT

    def contact_rate(self, UO):
        out = torch.empty(max(self.n_c, 1), dtype=torch.float64, device="cuda")
        self._check(self.lib.sps_contact_rate(self.h, _ptr(UO), _ptr(out)))
        return out[: self.n_c]

    # ---- solves --------------------------------------------------------------------
    def mobility_apply(self, pos, radii, FT, UO=None, allow_not_converged=False):
        n = radii.numel()
        if UO is None:
            UO = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        st = sps_stats()
        rc = self.lib.sps_mobility_apply(self.h, n, _ptr(pos), _ptr(radii), _ptr(FT), _ptr(UO),
                                         ctypes.byref(st))
        self._check(rc, allow=(4,) if allow_not_converged else ())
        self.last_stats = st.as_dict()
        return UO

    def resolve_collisions(self, pos, radii, FT_ext, dt, gamma=None, UO=None, pos_out=None,
                           gamma_cap=None, allow=()):
        n = radii.numel()
        if gamma_cap is None:
            gamma_cap = 16 * n
        if gamma is None:
            gamma = torch.empty(max(gamma_cap, 1), dtype=torch.float64, device="cuda")
        if UO is None:
            UO = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        if pos_out is None:
            pos_out = torch.empty(n, 3, dtype=torch.float64, device="cuda")
        st = sps_stats()
        rc = self.lib.sps_resolve_collisions(self.h, n, _ptr(pos), _ptr(radii), _ptr(FT_ext),
                                             float(dt), _ptr(gamma), int(gamma_cap), _ptr(UO),
                                             _ptr(pos_out), ctypes.byref(st))
        self._check(rc, allow=allow)
        self.last_stats = st.as_dict()
        self.n_c = st.n_contacts          # the contact list stays in the context
        return gamma[: st.n_contacts], UO, pos_out

    def simulate(self, pos, radii, FT_ext, dt, steps, UO=None, allow=()):
        """`steps` collision-resolved steps (sps_simulate); pos (n x 3, CUDA,
        float64) is advanced in place.  Returns (pos, UO of the last step,
        list of per-step stats dicts)."""
        n = radii.numel()
        if UO is None:
            UO = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        stats = (sps_stats * max(steps, 1))()
        done = ctypes.c_int()
        rc = self.lib.sps_simulate(self.h, n, _ptr(pos), _ptr(radii), _ptr(FT_ext), float(dt),
                                   int(steps), _ptr(UO), stats, ctypes.byref(done))
        self._check(rc, allow=allow)
        out = [stats[k].as_dict() for k in range(done.value)]
        if out:
            self.last_stats = out[-1]
            self.n_c = out[-1]["n_contacts"]
        return pos, UO, out

    def resolve_collisions_host(self, pos, radii, FT_ext, dt, gamma, UO, pos_out, allow=()):
        """Same step on host (CPU, ideally pinned) tensors; copies happen inside."""
        n = radii.numel()
        nc = ctypes.c_int()
        st = sps_stats()
        rc = self.lib.sps_resolve_collisions_host(
            self.h, n, _ptr(pos, device=False), _ptr(radii, device=False),
            _ptr(FT_ext, device=False), float(dt), _ptr(gamma, device=False), gamma.numel(),
            _ptr(UO, device=False), _ptr(pos_out, device=False), ctypes.byref(nc),
            ctypes.byref(st))
        self._check(rc, allow=allow)
        self.last_stats = st.as_dict()
        self.n_c = nc.value
        return nc.value


class MobilityFunction(torch.autograd.Function):
    """U = M(pos) FT as a differentiable function of forces/torques and centres.

    forward: sps_mobility_apply; backward: sps_mobility_adjoint (exact gradient
    of the discrete map; radii and near lists are held fixed, so the gradient
    in pos is that of the current piece of a piecewise-smooth map).
    """

    @staticmethod
    def forward(fctx, pos, radii, FT, ctx):
        U = ctx.mobility_apply(pos.detach().contiguous(), radii.detach().contiguous(),
                               FT.detach().contiguous())
        fctx.save_for_backward(pos, radii, FT)
        fctx.sps = ctx
        return U

    @staticmethod
    def backward(fctx, gU):
        pos, radii, FT = fctx.saved_tensors
        want_pos = fctx.needs_input_grad[0]
        _, gF, gx = fctx.sps.mobility_adjoint(pos.detach().contiguous(), radii.detach().contiguous(),
                                              FT.detach().contiguous(), gU.contiguous(),
                                              want_pos=want_pos)
        return (gx if want_pos else None), None, (gF if fctx.needs_input_grad[2] else None), None


def mobility(pos, radii, FT, ctx):
    """Differentiable U = M F (see MobilityFunction)."""
    return MobilityFunction.apply(pos, radii, FT, ctx)


class CollisionStepFunction(torch.autograd.Function):
    """U of one collision-resolved step (Sec. 3.2) as a differentiable function
    of the external forces/torques and the centres.

    forward: sps_collision_adjoint's forward step; backward: its adjoint on the
    active set of the LCP (contact, active and near sets held fixed)."""

    @staticmethod
    def forward(fctx, pos, radii, FT, dt, ctx):
        U, _, _ = ctx.collision_adjoint(pos.detach().contiguous(), radii.detach().contiguous(),
                                        FT.detach().contiguous(), dt,
                                        torch.zeros_like(FT, dtype=torch.float64).contiguous())
        fctx.save_for_backward(pos, radii, FT)
        fctx.sps = ctx
        fctx.dt = dt
        return U

    @staticmethod
    def backward(fctx, gU):
        pos, radii, FT = fctx.saved_tensors
        want_pos = fctx.needs_input_grad[0]
        _, gF, gx = fctx.sps.collision_adjoint(pos.detach().contiguous(), radii.detach().contiguous(),
                                               FT.detach().contiguous(), fctx.dt, gU.contiguous(),
                                               want_pos=want_pos)
        return (gx if want_pos else None), None, (gF if fctx.needs_input_grad[2] else None), None, None


def collision_step(pos, radii, FT, dt, ctx):
    """Differentiable U of one collision-resolved step (see CollisionStepFunction)."""
    return CollisionStepFunction.apply(pos, radii, FT, dt, ctx)
