"""The allocation-free energy measurement (sv_energy_noalloc) against the
context-based sv_expect_energy, through the C ABI.

This entry point exists for callers that cannot allocate device memory;
it keeps its scratch in a fixed library array.  Two calls in a row must
both agree with the allocating path, which also checks that the shared
scratch is cleared between calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2111_08044_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,precision", [(14, "c64"), (13, "c64"), (11, "c128")])
def test_noalloc_energy_matches_context_energy(svlib, L, precision):
    import torch
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params

    cfg = inputs.ChainConfig(L=L, seed=21, edge_field_weight=0.75)
    with FloquetSimulator(L, precision=precision) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        sim.evolve(3)
        e_ref, n_ref = sim.energy()
        p, keep = capi.make_params(**chain_params(cfg))
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=sim.state.device)
        prec = capi.SV_C128 if precision == "c128" else capi.SV_C64
        for _ in range(2):
            out.fill_(float("nan"))
            rc = svlib.sv_energy_noalloc(ctypes.c_void_p(sim.state.data_ptr()), L, prec,
                                         ctypes.byref(p),
                                         ctypes.cast(out.data_ptr(), capi._dp),
                                         ctypes.c_void_p(sim.stream.cuda_stream))
            assert rc == capi.SV_OK
            torch.cuda.synchronize()
            e, n = out.tolist()
            tol = 1e-9 if precision == "c64" else 1e-12
            assert abs(e - e_ref) < tol, (e, e_ref)
            assert abs(n - n_ref) < tol, (n, n_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(svlib):
    import torch
    p, _ = capi.make_params()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    buf = torch.zeros(8, dtype=torch.complex64, device="cuda")
    rc = svlib.sv_energy_noalloc(ctypes.c_void_p(buf.data_ptr()), 35, capi.SV_C64,
                                 ctypes.byref(p), ctypes.cast(out.data_ptr(), capi._dp), None)
    assert rc == capi.SV_EINVAL
    rc = svlib.sv_energy_noalloc(ctypes.c_void_p(buf.data_ptr()), 34, capi.SV_C128,
                                 ctypes.byref(p), ctypes.cast(out.data_ptr(), capi._dp), None)
    assert rc == capi.SV_EINVAL
    rc = svlib.sv_energy_noalloc(None, 8, capi.SV_C64, ctypes.byref(p),
                                 ctypes.cast(out.data_ptr(), capi._dp), None)
    assert rc == capi.SV_EINVAL
