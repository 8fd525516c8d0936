"""GPU parity of the block form (fused n-site unitaries, relabel folded into
each pass) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


def _run_block(cfg, n, split, periods, expect_tc=None):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    with FloquetSimulator(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg, mode=capi.SV_MODE_BLOCK, block_n=n, split=split))
        if expect_tc is not None:
            assert sim.form_info() == (expect_tc, n)
        e, nn = sim.evolve(periods)
        return e, nn, sim.host_state(), sim.pass_info()


BLOCK_CASES = [(8, 3), (8, 4), (10, 5), (12, 6), (12, 7), (13, 6), (14, 5), (16, 6),
               (17, 7)]


@pytest.mark.parametrize("L,n", BLOCK_CASES)
def test_simt_block_form_matches_oracle(svlib, L, n):
    cfg = inputs.ChainConfig(L=L, periods=4, seed=60 + L)
    psi_o, _, e_o, n_o = orc.run_chain(cfg)
    e, nn, psi, info = _run_block(cfg, n, capi.SV_SPLIT_FP32, cfg.periods, expect_tc=False)
    assert info[0] >= 1
    err = np.linalg.norm(psi.astype(np.complex128) - psi_o)
    assert err < 1e-5, err
    np.testing.assert_allclose(e, e_o, atol=2e-6, rtol=0)
    np.testing.assert_allclose(nn, n_o, atol=2e-6, rtol=0)


def test_block_small_preset_100_periods(svlib):
    cfg = inputs.preset("small")
    psi_o, _, e_o, _ = orc.run_chain(cfg)
    e, nn, psi, _ = _run_block(cfg, 6, capi.SV_SPLIT_BF16X3, cfg.periods)
    np.testing.assert_allclose(e, e_o, atol=1e-5, rtol=0)
    ov = np.vdot(psi.astype(np.complex128), psi_o)
    assert 1 - abs(ov) ** 2 < 1e-5


def _infidelity(a, b):
    a = a.astype(np.complex128)
    b = b.astype(np.complex128)
    return 1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


@pytest.mark.parametrize("L", [13, 14, 16, 20])
def test_tensor_core_block_form_matches_oracle(svlib, L):
    """tcgen05 block passes (exact level-0 digit products on bf16 tensor
    cores) against the oracle, element by element and in energy."""
    cfg = inputs.ChainConfig(L=L, periods=3, seed=80 + L)
    psi_o, _, e_o, n_o = orc.run_chain(cfg)
    e, nn, psi, info = _run_block(cfg, 6, capi.SV_SPLIT_BF16X3, cfg.periods, expect_tc=True)
    assert _infidelity(psi, psi_o) < 1e-8
    # Each pass rounds the state to 2^-23 of every row's largest amplitude
    # (one exponent per row of 64): up to ~1e-6 of the state norm per pass,
    # accumulating as a random walk over the passes.
    err = np.linalg.norm(psi.astype(np.complex128) - psi_o)
    assert err < 4e-6 * np.sqrt(cfg.periods * info[0]), err
    np.testing.assert_allclose(e, e_o, atol=2e-6, rtol=0)
    np.testing.assert_allclose(nn, n_o, atol=5e-6, rtol=0)


@pytest.mark.parametrize("L", [14, 17])
def test_tensor_core_100_periods_with_renormalisation(svlib, L):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=L, periods=100, seed=90 + L)
    psi_o, _, e_o, _ = orc.run_chain(cfg)
    with FloquetSimulator(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg, mode=capi.SV_MODE_BLOCK, block_n=6,
                                 split=capi.SV_SPLIT_BF16X3, renorm_every=1))
        assert sim.form_info() == (True, 6)
        e, nn = sim.evolve(cfg.periods)
        psi = sim.host_state()
    np.testing.assert_allclose(e, e_o, atol=1e-5, rtol=0)
    assert np.all(np.abs(nn - 1.0) < 2e-5)  # one period of drift at most
    assert _infidelity(psi, psi_o) < 1e-5


@pytest.mark.parametrize("L,first,ew,periods", [(15, 1, 1.0, 3), (21, 0, 1.0, 2), (23, 0, 0.5, 2),
                                                (26, 1, 0.5, 1)])
def test_tensor_core_variants_match_oracle(svlib, L, first, ew, periods):
    """Odd L, the other layer order and whole edge fields; at L = 23 (and
    L = 16 above) one pass writes through a reordered staging tile (a 4-D or
    5-D store view); at L = 26 the CTAs run 54 tiles each (a ragged tail over
    152 SMs), so the pass instances specialised on what they measure are
    checked element by element.  Most of these plans start their periods off
    site 0, so every evolution here also runs the relabel into the period
    layout and the last period's hand-back to the natural layout."""
    cfg = inputs.ChainConfig(L=L, periods=periods, seed=90 + L, first_layer=first,
                             edge_field_weight=ew)
    psi_o, _, e_o, n_o = orc.run_chain(cfg)
    e, nn, psi, info = _run_block(cfg, 6, capi.SV_SPLIT_BF16X3, cfg.periods, expect_tc=True)
    assert _infidelity(psi, psi_o) < 1e-8
    err = np.linalg.norm(psi.astype(np.complex128) - psi_o)
    assert err < 4e-6 * np.sqrt(cfg.periods * info[0]), err
    np.testing.assert_allclose(e, e_o, atol=2e-6, rtol=0)
    np.testing.assert_allclose(nn, n_o, atol=5e-6, rtol=0)


@pytest.mark.parametrize("L", [16, 22])
def test_kept_period_layout_matches_natural_layout(svlib, L):
    """sv_set_layout_policy(1): one period per sv_evolve call with the state
    kept in the plan's period layout between calls (no relabel pass per
    call).  Energies, the measured energy and the final state (brought back
    to the natural layout by the state copy) agree with evolving in one
    call; the only difference is one more rounding by a relabel pass."""
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=L, seed=40 + L)
    kw = chain_params(cfg, mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3)
    P = 6
    with FloquetSimulator(L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**kw)
        e_ref, n_ref = sim.evolve(P)
        psi_ref = sim.host_state()
    with FloquetSimulator(L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**kw)
        sim.keep_period_layout(True)
        e = np.concatenate([sim.evolve(1)[0] for _ in range(P)])
        e_meas, _ = sim.energy()        # restores the natural layout first
        psi = sim.host_state()
        e_more, _ = sim.evolve(2)       # and evolves on from there
    np.testing.assert_allclose(e, e_ref, atol=1e-7, rtol=0)
    assert abs(e_meas - e_ref[-1]) < 1e-6
    err = np.linalg.norm(psi.astype(np.complex128) - psi_ref.astype(np.complex128))
    assert err < 1e-6, err
    assert np.all(np.isfinite(e_more))
