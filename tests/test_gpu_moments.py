"""GPU energy moments (E and sigma_E, Eq. 10-11), product-state overlaps and
inverse periods (the echo of Sec. V), through the C ABI: against the FP64
oracle at sizes it runs in seconds, and at the full L = 30 against the
product-state closed form and the echo's own invariants."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs
from tests.test_oracle_moments import _product_state_moments

pytestmark = pytest.mark.gpu

BLOCK = dict(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3)


def _oracle_state(cfg, periods):
    hdrive, hobs = orc.chain_inputs(cfg)
    psi = orc.product_state(cfg.spinors())
    orc.evolve(psi, periods, hdrive, cfg.tau, cfg.theta, cfg.K, cfg.first_layer, hobs)
    return psi, hobs


@pytest.mark.parametrize("precision,tol", [("c128", 1e-11), ("c64", 2e-6)])
def test_energy_moments_match_oracle(svlib, precision, tol):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=12, seed=6)
    with FloquetSimulator(cfg.L, precision=precision) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        sim.evolve(3)
        E, s, n = sim.energy_moments()
        ov = sim.overlap_product(cfg.spinors())
    psi, hobs = _oracle_state(cfg, 3)
    Eo, so, no = orc.energy_moments(psi, hobs)
    assert abs(E - Eo) < tol * cfg.L, (E, Eo)
    assert abs(s - so) < tol * cfg.L, (s, so)
    assert abs(n - no) < tol
    ovo = np.vdot(orc.product_state(cfg.spinors()), psi)
    assert abs(ov - ovo) < tol, (ov, ovo)


def test_energy_moments_full_size_product_state(svlib):
    """L = 30 (8 GiB): E and sigma_E of the product initial state against the
    closed form from two- and three-site local algebra."""
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=30, seed=4)
    sp = cfg.spinors()
    with FloquetSimulator(cfg.L) as sim:
        sim.init_product_state(sp)
        sim.build(**chain_params(cfg, **BLOCK))
        E, s, n = sim.energy_moments()
        ov = sim.overlap_product(sp)
    hb = orc.ising_bond_hamiltonians(cfg.L, cfg.J, cfg.hx, cfg.hz, cfg.edge_field_weight)
    Ec, sc = _product_state_moments(sp, hb)
    assert abs(n - 1.0) < 1e-5
    assert abs(E - Ec) < 1e-5 * cfg.L, (E, Ec)
    assert abs(s - sc) < 1e-5 * cfg.L, (s, sc)
    assert abs(ov - 1.0) < 1e-5


@pytest.mark.parametrize("L,mode", [(10, "plain"), (16, "block")])
def test_inverse_period_matches_oracle(svlib, L, mode):
    """One inverse period applied to an evolved state equals the oracle's
    U_F^dagger applied to the same state."""
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=L, seed=8)
    extra = BLOCK if mode == "block" else {}
    prec = "c64" if mode == "block" else "c128"
    with FloquetSimulator(L, precision=prec) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg, **extra))
        sim.evolve(2)
        before = sim.host_state().astype(np.complex128)
        sim.build(**chain_params(cfg, inverse=1, **extra))
        e, n = sim.evolve(1)
        after = sim.host_state().astype(np.complex128)
    hb = orc.ising_bond_hamiltonians(L, cfg.J, cfg.hx, cfg.hz, cfg.edge_field_weight)
    ref = before.copy()
    orc.period(ref, orc.bond_gates(hb, cfg.tau), orc.kick_gates(L, cfg.theta), cfg.K,
               cfg.first_layer, inverse=True)
    tol = 1e-12 if prec == "c128" else 2e-5
    assert np.linalg.norm(after - ref) < tol
    Eo, _ = orc.energy(ref, hb)
    assert abs(e[0] - Eo / L) < (1e-12 if prec == "c128" else 1e-5)


@pytest.mark.parametrize("L,periods,mode", [(20, 20, "block"), (30, 3, "block"), (12, 8, "plain")])
def test_echo_returns_to_the_start(svlib, L, periods, mode):
    """P periods forward, then P inverse periods: the overlap with the
    starting product state returns to 1 (the echo of Sec. V), and the
    energies of the way back retrace those of the way out."""
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=L, seed=9)
    sp = cfg.spinors()
    extra = BLOCK if mode == "block" else {}
    with FloquetSimulator(L) as sim:
        sim.init_product_state(sp)
        sim.build(**chain_params(cfg, **extra))
        ef, _ = sim.evolve(periods)
        moved = abs(sim.overlap_product(sp))
        sim.build(**chain_params(cfg, inverse=1, **extra))
        eb, nb = sim.evolve(periods)
        ov = sim.overlap_product(sp)
    assert moved < 0.999  # the state did move away
    assert abs(1.0 - ov) < 1e-5 * periods, ov
    # after k inverse periods the state is back at forward period P - k
    np.testing.assert_allclose(eb[:-1], ef[::-1][1:], atol=1e-5, rtol=0)
    e0 = inputs.ChainConfig(L=L, seed=9)
    hb = orc.ising_bond_hamiltonians(L, e0.J, e0.hx, e0.hz, e0.edge_field_weight)
    E0, _ = _product_state_moments(sp, hb)
    assert abs(eb[-1] - E0 / L) < 1e-5
