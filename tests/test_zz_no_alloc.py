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


def _noalloc(svlib, sim, L, prec, p, out):
    import torch
    out.fill_(float("nan"))
    rc = svlib.sv_energy_noalloc(ctypes.c_void_p(sim.state.data_ptr()), L, prec,
                                 ctypes.byref(p), ctypes.cast(out.data_ptr(), capi._dp),
                                 ctypes.c_void_p(sim.stream.cuda_stream))
    assert rc == capi.SV_OK
    torch.cuda.synchronize()
    return out.tolist()


def _run(svlib, L, precision, seed=21, calls=2):
    import torch
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params

    cfg = inputs.ChainConfig(L=L, seed=seed, edge_field_weight=0.75)
    with FloquetSimulator(L, precision=precision) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        sim.evolve(3)
        e_ref, n_ref = sim.energy()
        p, keep = capi.make_params(**chain_params(cfg))
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=sim.state.device)
        prec = capi.SV_C128 if precision == "c128" else capi.SV_C64
        tol = 1e-9 if precision == "c64" else 1e-12
        for _ in range(calls):
            e, n = _noalloc(svlib, sim, L, prec, p, out)
            assert abs(e - e_ref) < tol, (L, precision, e, e_ref)
            assert abs(n - n_ref) < tol, (L, precision, n, n_ref)


@pytest.mark.parametrize("L,precision", [(14, "c64"), (13, "c64"), (11, "c128"),
                                         (2, "c64"), (2, "c128"), (3, "c64"), (3, "c128")])
def test_noalloc_energy_matches_context_energy(svlib, L, precision):
    """L = 2: one pass carries both edge sites and no bulk field; L = 3: one
    bulk site beside the odd chain's last-site pass."""
    _run(svlib, L, precision)


def test_noalloc_scratch_is_cleared_between_sizes(svlib):
    """A larger chain fills more scratch slices than a smaller one reads; the
    smaller chain's call right after must not see them."""
    _run(svlib, 16, "c64", seed=5, calls=1)
    _run(svlib, 12, "c64", seed=6, calls=2)
    _run(svlib, 15, "c128", seed=7, calls=1)
    _run(svlib, 5, "c128", seed=8, calls=2)


def test_noalloc_rejects_what_it_cannot_measure(svlib):
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
    # general bond terms: the observable is sum_b H_b, not the Ising H0
    hb = inputs.gue_bond_terms(2, seed=3)
    pg, keep = capi.make_params(h_bonds=hb, K=1, theta=0.0)
    rc = svlib.sv_energy_noalloc(ctypes.c_void_p(buf.data_ptr()), 3, capi.SV_C64,
                                 ctypes.byref(pg), ctypes.cast(out.data_ptr(), capi._dp), None)
    assert rc == capi.SV_EINVAL
