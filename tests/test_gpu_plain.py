"""GPU parity of the plain (per-gate) form against the FP64 oracle, through
the C ABI.  Tolerances: complex64 energy density <= 1e-5 absolute and state
infidelity <= 1e-5 per 1000 periods; complex128 and double-float check
modes 1e-11."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sim(L, precision="c64"):
    from paper_2111_08044_gb300.sim import FloquetSimulator
    return FloquetSimulator(L, precision=precision)


def _infidelity(a, b):
    a = a.astype(np.complex128)
    b = b.astype(np.complex128)
    ov = np.vdot(a, b)
    return 1.0 - abs(ov) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


@pytest.mark.parametrize("precision,tol", [("c64", 1e-5), ("c128", 1e-11), ("df64", 1e-11)])
def test_small_preset_100_periods(svlib, precision, tol):
    from paper_2111_08044_gb300.sim import chain_params
    cfg = inputs.preset("small")
    psi_o, e0_o, e_o, n_o = orc.run_chain(cfg)
    with _sim(cfg.L, precision) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        e0, n0 = sim.energy()
        e, n = sim.evolve(cfg.periods)
        psi = sim.host_state()
        assert sim.period == cfg.periods
    assert abs(e0 - e0_o) < tol
    np.testing.assert_allclose(e, e_o, atol=tol, rtol=0)
    # complex64: the norm may drift by rounding of the gates (no systematic
    # bias is left after unitarity-aware FP32 rounding); complex128 holds it
    np.testing.assert_allclose(n, n_o, atol=tol, rtol=0)
    assert _infidelity(psi, psi_o) < tol
    np.testing.assert_allclose(psi, psi_o, atol=10 * tol, rtol=0)


CASES = [(L, fl, ew) for L in (2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 14)
         for fl, ew in ((0, 0.5), (1, 1.0))]


@pytest.mark.parametrize("L,first,ew", CASES)
@pytest.mark.parametrize("precision", ["c64", "c128", "df64"])
def test_state_after_three_periods(svlib, L, first, ew, precision):
    """Every kernel variant (tiny chain, low bonds with shuffles, high bonds)
    and both layer orders against the oracle, element by element."""
    from paper_2111_08044_gb300.sim import chain_params
    cfg = inputs.ChainConfig(L=L, J=1.05, hx=0.83, hz=0.37, T=0.61, K=3, theta=0.29,
                             edge_field_weight=ew, first_layer=first, periods=3, seed=40 + L)
    psi_o, e0_o, e_o, n_o = orc.run_chain(cfg)
    with _sim(L, precision) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        e, n = sim.evolve(cfg.periods)
        psi = sim.host_state()
    # df64: about 2^-47 of the terms per complex multiply-add, against the
    # FP64 mode's 2^-53
    tol = {"c64": 2e-6, "c128": 1e-13, "df64": 5e-13}[precision]
    err = np.linalg.norm(psi.astype(np.complex128) - psi_o)
    assert err < tol * 4, err
    etol = 2e-6 if precision == "c64" else 1e-12
    np.testing.assert_allclose(e, e_o, atol=etol, rtol=0)
    np.testing.assert_allclose(n, n_o, atol=etol, rtol=0)


@pytest.mark.parametrize("precision", ["c64", "c128", "df64"])
def test_initial_state_and_energy(svlib, precision):
    cfg = inputs.ChainConfig(L=13, seed=9)
    psi_o = orc.product_state(cfg.spinors())
    _, hobs = orc.chain_inputs(cfg)
    e_o, _ = orc.energy(psi_o, hobs)
    from paper_2111_08044_gb300.sim import chain_params
    with _sim(cfg.L, precision) as sim:
        sim.init_product_state(cfg.spinors())
        psi = sim.host_state()
        sim.build(**chain_params(cfg))
        e, n = sim.energy()
    tol = 1e-6 if precision == "c64" else 1e-13
    np.testing.assert_allclose(psi, psi_o, atol=tol, rtol=0)
    assert abs(e - e_o / cfg.L) < tol
    assert abs(n - 1.0) < tol


def test_renormalize_and_state_roundtrip(svlib):
    from paper_2111_08044_gb300.sim import chain_params
    cfg = inputs.ChainConfig(L=10, seed=2)
    with _sim(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        sim.evolve(5)
        psi = sim.host_state()
        sim.set_host_state(psi * 1.5, period=5)
        n_before = sim.renormalize()
        assert abs(n_before - 2.25) < 1e-5
        _, n = sim.energy()
        assert abs(n - 1.0) < 1e-6
        assert sim.period == 5
        np.testing.assert_allclose(sim.host_state(), psi, atol=1e-6, rtol=0)


@pytest.mark.parametrize("precision", ["c128", "df64"])
def test_per_period_parameters(svlib, precision):
    """Per-period kick angle and field (plain form) against the oracle."""
    from paper_2111_08044_gb300.sim import chain_params
    P = 6
    rng = np.random.default_rng(1)
    cfg = inputs.ChainConfig(L=9, periods=P, seed=5, theta_p=rng.uniform(0.1, 0.5, P),
                             hx_p=rng.uniform(0.6, 1.0, P))
    psi_o, _, e_o, _ = orc.run_chain(cfg)
    with _sim(cfg.L, precision) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        e, _ = sim.evolve(P)
        psi = sim.host_state()
        with pytest.raises(Exception):
            sim.evolve(1)  # beyond the per-period table
    np.testing.assert_allclose(e, e_o, atol=1e-12, rtol=0)
    np.testing.assert_allclose(psi, psi_o, atol=1e-12, rtol=0)


def test_folded_renormalisation_plain(svlib):
    """renorm_every folds a rescale into the first gate pass of a period."""
    from paper_2111_08044_gb300.sim import chain_params
    cfg = inputs.ChainConfig(L=11, periods=20, seed=12)
    _, _, e_o, _ = orc.run_chain(cfg)
    with _sim(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        psi0 = sim.host_state()
        sim.set_host_state(psi0 * 1.1, period=0)
        sim.build(**chain_params(cfg, renorm_every=2))
        e, n = sim.evolve(cfg.periods)
    np.testing.assert_allclose(e, e_o, atol=1e-5, rtol=0)
    assert abs(n[0] - 1.21) < 1e-5 and abs(n[1] - 1.21) < 1e-5  # no rescale before period 2
    assert np.all(np.abs(n[1::2][1:] - 1.0) < 1e-5)  # rescaled at periods 2, 4, ...


def test_call_order_errors(svlib):
    from paper_2111_08044_gb300 import capi
    with _sim(8) as sim:
        with pytest.raises(capi.SvError) as ei:
            sim.evolve(1)
        assert ei.value.code == capi.SV_ESTATE
        with pytest.raises(capi.SvError) as ei:
            sim.build()
        assert ei.value.code == capi.SV_ESTATE
        sim.init_product_state(inputs.random_product_spinors(8, 1))
        with pytest.raises(capi.SvError) as ei:
            sim.build(K=0)
        assert ei.value.code == capi.SV_EINVAL
        with pytest.raises(capi.SvError) as ei:
            sim.init_product_state(np.zeros((8, 4)))
        assert ei.value.code == capi.SV_EINVAL
