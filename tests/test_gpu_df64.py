"""The double-float check mode (SV_DF64): each real number is a pair of
FP32 values hi + lo, about 48 significant bits, computed on the FP32 pipe.

Element-by-element parity with the FP64 oracle is in test_gpu_plain.py
(every kernel variant, both layer orders).  Here: it follows the complex128
mode over hundreds of periods at L = 20 (the two check modes of the error
study, Sec. V), its norm does not drift, its complex128 read-out and
write-in, checkpoints, and the calls it does not have."""
import ctypes

import numpy as np
import pytest

from paper_2111_08044_gb300 import capi, inputs
from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params

pytestmark = pytest.mark.gpu


def _run(L, precision, periods, seed=4):
    cfg = inputs.ChainConfig(L=L, seed=seed)
    with FloquetSimulator(L, precision=precision) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        e, n = sim.evolve(periods)
        psi = sim.host_state()
    return e, n, psi


def _words(t):
    """The buffer's raw 64-bit words (the double-float pairs as held)."""
    import torch
    return torch.view_as_real(t).view(torch.int64).clone()


def test_df64_follows_c128_over_200_periods(svlib):
    """Both check modes drift in norm by about +6e-14 per period (the FP64
    gate tables' own unitarity defect, the same every period), so their
    norms part by a few 1e-12 over 200 periods; the energy densities agree
    to 1e-13."""
    e1, n1, p1 = _run(20, "c128", 200)
    e2, n2, p2 = _run(20, "df64", 200)
    assert np.max(np.abs(e1 - e2)) < 1e-12
    assert np.max(np.abs(n1 - n2)) < 2e-11
    assert np.linalg.norm(p1 - p2) < 1e-10


@pytest.mark.parametrize("L", [14, 17])
def test_df64_norm_drift_is_that_of_c128(svlib, L):
    """Measured: +4.9e-14 and +6.0e-14 per period at L = 14, 17 (the
    complex128 mode: about +6e-14); the complex64 forms' bound is 5e-9."""
    _, n, _ = _run(L, "df64", 400, seed=6)
    t = np.arange(1, n.size + 1, dtype=np.float64)
    slope = float(np.polyfit(t, n, 1)[0])
    assert abs(slope) < 3e-13, slope
    assert abs(n[-1] - 1.0) < 1e-10


def test_df64_state_write_and_read(svlib):
    import torch
    L = 12
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(1 << L) + 1j * rng.standard_normal(1 << L)
    psi /= np.linalg.norm(psi)
    with FloquetSimulator(L, precision="df64") as sim:
        sim.init_product_state(inputs.ChainConfig(L=L).spinors())
        sim.set_host_state(psi, period=7)
        back = sim.host_state()
        dev = sim.state_c128().cpu().numpy()
        assert sim.period == 7
    # hi = nearest float, lo = nearest float to the remainder
    for part in (np.real, np.imag):
        assert np.all(np.abs(part(back) - part(psi)) <= 2.0 ** -48 * np.abs(part(psi)))
    np.testing.assert_array_equal(dev, back)
    assert dev.dtype == np.complex128 and isinstance(sim.state, torch.Tensor)


def test_df64_checkpoint_resume_is_bitwise(svlib, tmp_path):
    cfg = inputs.ChainConfig(L=15, seed=8)
    path = str(tmp_path / "df.ckpt").encode()
    with FloquetSimulator(cfg.L, precision="df64") as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        sim.evolve(5)
        capi.check(svlib.sv_save(sim._ctx, path), sim._ctx, "sv_save")
        e_ref, _ = sim.evolve(4)
        raw_ref = _words(sim.state)
    L, prec, per = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    assert svlib.sv_checkpoint_info(path, ctypes.byref(L), ctypes.byref(prec),
                                    ctypes.byref(per)) == capi.SV_OK
    assert (L.value, prec.value, per.value) == (cfg.L, capi.SV_DF64, 5)
    with FloquetSimulator(cfg.L, precision="df64") as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        capi.check(svlib.sv_load(sim._ctx, path), sim._ctx, "sv_load")
        assert sim.period == 5
        e, _ = sim.evolve(4)
        assert bool((_words(sim.state) == raw_ref).all())
    np.testing.assert_array_equal(e, e_ref)


def test_df64_refuses_what_it_does_not_have(svlib):
    cfg = inputs.ChainConfig(L=10, seed=1)
    with FloquetSimulator(cfg.L, precision="df64") as sim:
        sim.init_product_state(cfg.spinors())
        for mode in (capi.SV_MODE_BLOCK, capi.SV_MODE_MULTIGATE):
            p, keep = capi.make_params(**chain_params(cfg, mode=mode))
            assert svlib.sv_build_floquet(sim._ctx, ctypes.byref(p)) == capi.SV_EUNSUPPORTED
        sim.build(**chain_params(cfg))
        d = ctypes.c_double()
        assert svlib.sv_energy_moments(sim._ctx, ctypes.byref(d), ctypes.byref(d),
                                       ctypes.byref(d)) == capi.SV_EUNSUPPORTED
        sp = np.ascontiguousarray(cfg.spinors())
        assert svlib.sv_overlap_product(sim._ctx, sp.ctypes.data_as(capi._dp), ctypes.byref(d),
                                        ctypes.byref(d)) == capi.SV_EUNSUPPORTED
        pairs = np.zeros((cfg.L // 2, 8))
        pairs[:, 0] = 1.0
        assert svlib.sv_init_pairs(sim._ctx, cfg.L, pairs.ctypes.data_as(capi._dp)) == \
            capi.SV_EUNSUPPORTED
        e, n = sim.energy()
        assert abs(n - 1.0) < 1e-13
