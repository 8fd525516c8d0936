"""GPU parity of the multi-gate form (SV_MODE_MULTIGATE: many gates of the
period applied per pass to a shared-memory tile, Eq. 2 gate by gate)
against the FP64 oracle, through the C ABI: states element by element and
the energy density of every period."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


def _run(cfg, periods, **over):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    with FloquetSimulator(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg, mode=capi.SV_MODE_MULTIGATE, **over))
        e, n = sim.evolve(periods)
        return e, n, sim.host_state(), sim.pass_info()


@pytest.mark.parametrize("L,first,ew", [(2, 0, 0.5), (5, 1, 1.0), (10, 0, 0.5), (13, 1, 0.5),
                                        (14, 0, 0.5), (17, 1, 1.0), (20, 0, 0.5), (22, 1, 0.5)])
def test_multigate_matches_oracle(svlib, L, first, ew):
    """L <= 13: the whole chain is one tile, one pass a period; L > 13:
    windows of 9 sites over tiles of 2^13 amplitudes, including windows
    that start below site 4 (tile = the 13 lowest bits) and above it."""
    cfg = inputs.ChainConfig(L=L, periods=4, seed=70 + L, first_layer=first,
                             edge_field_weight=ew)
    psi_o, _, e_o, n_o = orc.run_chain(cfg)
    e, n, psi, info = _run(cfg, cfg.periods)
    passes, gates, _ = info
    assert gates == 4 * (L - 1)
    if L <= 13:
        assert passes == 1
    err = np.linalg.norm(psi.astype(np.complex128) - psi_o)
    assert err < 2e-7 * np.sqrt(cfg.periods * gates) + 1e-6, (L, err)
    np.testing.assert_allclose(e, e_o, atol=1e-6, rtol=0)
    np.testing.assert_allclose(n, n_o, atol=1e-6, rtol=0)


def test_multigate_per_period_drive_and_renormalisation(svlib):
    L, P = 16, 5
    base = inputs.ChainConfig(L=L, periods=P, seed=5)
    rng = np.random.default_rng(3)
    cfg = inputs.ChainConfig(L=L, periods=P, seed=5, theta_p=0.3 + 0.05 * rng.standard_normal(P),
                             hx_p=0.9 + 0.05 * rng.standard_normal(P))
    psi_o, _, e_o, _ = orc.run_chain(cfg)
    e, n, psi, _ = _run(cfg, P)
    np.testing.assert_allclose(e, e_o, atol=1e-6, rtol=0)
    assert 1 - abs(np.vdot(psi.astype(np.complex128), psi_o)) ** 2 < 1e-10
    # folded renormalisation: same energies, norm back at 1 every period
    e2, n2, _, _ = _run(base, P, renorm_every=1)
    _, _, e_b, _ = orc.run_chain(base)
    np.testing.assert_allclose(e2, e_b, atol=1e-6, rtol=0)
    assert np.all(np.abs(n2 - 1.0) < 1e-6)


def test_multigate_inverse_period_is_the_echo(svlib):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=18, seed=9)
    with FloquetSimulator(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg, mode=capi.SV_MODE_MULTIGATE))
        sim.evolve(10)
        sim.build(**chain_params(cfg, mode=capi.SV_MODE_MULTIGATE, inverse=1))
        sim.evolve(10)
        ov = sim.overlap_product(cfg.spinors())
    assert abs(1.0 - ov) < 1e-5


def test_multigate_refuses_complex128(svlib):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=8, seed=1)
    with FloquetSimulator(cfg.L, precision="c128") as sim:
        sim.init_product_state(cfg.spinors())
        with pytest.raises(capi.SvError):
            sim.build(**chain_params(cfg, mode=capi.SV_MODE_MULTIGATE))
