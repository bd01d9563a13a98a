"""The allocation-free contact builder (sps_build_contacts_noalloc).

Some callers cannot allocate device memory when they need the contact list:
code inside a host whose own memory pool has reserved the device (a framework's
caching allocator, an MPS client with a hard memory limit), where a cudaMalloc
outside that pool fails, and stepping loops that must never allocate mid-step.
For them the library keeps the builder's scratch in a fixed device array.
This test calls that entry point through the C ABI and checks it against the
ordinary entry point (sps_build_contacts + sps_get_contacts, delta_rel = 0),
bit for bit, on two calls in a row with different inputs (the shared array
must not carry state between calls).
The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(lib, pos, rad, acs, delta, cap):
    ij = torch.zeros(max(cap, 1), 2, dtype=torch.int32, device="cuda")
    phi = torch.zeros(max(cap, 1), dtype=torch.float64, device="cuda")
    nrm = torch.zeros(max(cap, 1), 3, dtype=torch.float64, device="cuda")
    nc = ctypes.c_int(-1)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.sps_build_contacts_noalloc(
        rad.numel(), ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(rad.data_ptr()),
        float(acs), float(delta), int(cap), ctypes.c_void_p(ij.data_ptr()),
        ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(nrm.data_ptr()), ctypes.byref(nc),
        ctypes.c_void_p(stream))
    return rc, nc.value, ij[: max(nc.value, 0)], phi[: max(nc.value, 0)], nrm[: max(nc.value, 0)]


def test_noalloc_contacts_match_context_builder():
    from paper_1909_06623_gb300 import build, workloads
    build.build()
    import paper_1909_06623_gb300 as sps
    lib = sps._lib.load()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")

    w = workloads.config2()
    rng = np.random.default_rng(7)
    cases = [(w.centers, w.radii, 1.05, 0.1),
             (w.centers + 0.02 * rng.standard_normal(w.centers.shape), w.radii, 1.0, 0.3)]
    for C, R, acs, delta in cases:          # two calls in a row, different inputs
        pos, rad = dev(C), dev(R)
        ctx = sps.Context(p=2, a_c_scale=acs, delta=delta)
        n_ref = ctx.build_contacts(pos, rad)
        ij_ref, phi_ref, nrm_ref = ctx.get_contacts()
        rc, nc, ij, phi, nrm = _noalloc(lib, pos, rad, acs, delta, 8 * len(R))
        assert rc == 0 and nc == n_ref > 0
        assert torch.equal(ij, ij_ref)
        assert torch.equal(phi.view(torch.int64), phi_ref.view(torch.int64))
        assert torch.equal(nrm.view(torch.int64), nrm_ref.view(torch.int64))
        # too small an output: the count is reported, nothing is written
        rc, nc2, _, _, _ = _noalloc(lib, pos, rad, acs, delta, n_ref - 1)
        assert rc == 6 and nc2 == n_ref
