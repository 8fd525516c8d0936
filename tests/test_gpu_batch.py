"""Batched evolution of independent chains (uneven L, per-chain couplings)
through the batch calls of the C ABI, every form against the FP64 oracle
chain by chain."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

FORMS = [capi.SV_BATCH_PLAIN, capi.SV_BATCH_BLOCK_SIMT, capi.SV_BATCH_BLOCK_TC,
         capi.SV_BATCH_RESIDENT, capi.SV_BATCH_MULTIGATE, capi.SV_BATCH_AUTO]


def _chains(Ls, seed):
    cs = inputs.batch_preset(n_chains=len(Ls), seed=seed, Lmin=2, Lmax=2, periods=8)
    # keep each chain's drawn couplings and state seed, set its length
    return [inputs.ChainConfig(L=L, J=c.J, hx=c.hx, hz=c.hz, theta=c.theta, periods=8,
                               seed=c.seed) for L, c in zip(Ls, cs)]


@pytest.mark.parametrize("form", FORMS)
def test_batch_forms_match_oracle(svlib, form):
    from paper_2111_08044_gb300.sim import FloquetBatch
    Ls = [6, 9, 12, 13, 14, 14, 15, 17]
    chains = _chains(Ls, seed=7)
    P = 8
    with FloquetBatch(chains, form=form) as b:
        forms = b.forms()
        widths = b.widths()
        e, n = b.evolve(P)
        states = [b.chain_state(c) for c in range(len(chains))]
    for c, cfg in enumerate(chains):
        # a forced form a chain cannot use falls back to the plain form
        if form >= 0:
            fits = {capi.SV_BATCH_PLAIN: True, capi.SV_BATCH_BLOCK_SIMT: cfg.L >= 6,
                    capi.SV_BATCH_BLOCK_TC: cfg.L >= 13,
                    capi.SV_BATCH_RESIDENT: cfg.L <= 14,
                    capi.SV_BATCH_MULTIGATE: True}[form]
            assert forms[c] == (form if fits else capi.SV_BATCH_PLAIN)
        # the block forms' width: 6 when forced, 5..7 when the autotuner chose
        if forms[c] in (capi.SV_BATCH_BLOCK_TC, capi.SV_BATCH_BLOCK_SIMT):
            assert widths[c] == 6 if form >= 0 else 5 <= widths[c] <= 7
        else:
            assert widths[c] == 0
        psi_o, _, e_o, n_o = orc.run_chain(cfg, periods=P)
        np.testing.assert_allclose(e[c], e_o, atol=1e-5, rtol=0, err_msg=f"chain {c} L={cfg.L}")
        np.testing.assert_allclose(n[c], n_o, atol=1e-5, rtol=0)
        # FP32 gate tables repeat every period, so their rounding (about
        # 1e-7 of the state per pass) can add up coherently over the passes
        err = np.linalg.norm(states[c].astype(np.complex128) - psi_o)
        assert err < 2e-7 * P * 4 * (cfg.L - 1) + 1e-5, (c, cfg.L, forms[c], err)


def test_tensor_core_groups_match_oracle(svlib):
    """Tensor-core chains of one L run as a group: each pass of all of them
    is one launch over all their tiles, a CTA taking a contiguous range that
    can span two chains (operand reload, coefficients and partial sums per
    chain).  Five chains of L = 20 (640 tiles on 152 CTAs, 3 of them
    spanning two chains) and ten of L = 19 (640 tiles, 6 CTAs spanning),
    interleaved, each with its own couplings and state, over 20 periods
    (the 16-period graph and single periods) against the oracle."""
    from paper_2111_08044_gb300.sim import FloquetBatch
    Ls = [20, 19, 19] * 5
    chains = _chains(Ls, seed=11)
    P = 20
    with FloquetBatch(chains, form=capi.SV_BATCH_BLOCK_TC) as b:
        assert list(b.forms()) == [capi.SV_BATCH_BLOCK_TC] * len(chains)
        e, n = b.evolve(P)
        states = [b.chain_state(c) for c in range(len(chains))]
    for c, cfg in enumerate(chains):
        psi_o, _, e_o, n_o = orc.run_chain(cfg, periods=P)
        np.testing.assert_allclose(e[c], e_o, atol=1e-5, rtol=0, err_msg=f"chain {c} L={cfg.L}")
        np.testing.assert_allclose(n[c], n_o, atol=1e-5, rtol=0)
        err = np.linalg.norm(states[c].astype(np.complex128) - psi_o)
        assert err < 1e-4, (c, cfg.L, err)


def test_batch_continues_across_calls(svlib):
    """Two evolve calls equal one; more periods than one graph run holds."""
    from paper_2111_08044_gb300.sim import FloquetBatch
    chains = _chains([8, 14, 16], seed=9)
    with FloquetBatch(chains, form=capi.SV_BATCH_AUTO) as b:
        e1, _ = b.evolve(5)
        e2, _ = b.evolve(20)
    e = np.concatenate([e1, e2], axis=1)
    for c, cfg in enumerate(chains):
        _, _, e_o, _ = orc.run_chain(cfg, periods=25)
        np.testing.assert_allclose(e[c], e_o, atol=1e-5, rtol=0)


def test_batch_preset_shape(svlib):
    """The 512-chain preset (L 14..22) builds, autotunes and runs."""
    from paper_2111_08044_gb300.sim import FloquetBatch
    chains = inputs.batch_preset(512)
    with FloquetBatch(chains) as b:
        forms = b.forms()
        e, n = b.evolve(2)
    assert e.shape == (512, 2)
    assert np.all(np.isfinite(e)) and np.all(np.abs(n - 1.0) < 1e-5)
    Ls = np.array([c.L for c in chains])
    assert np.all(forms[Ls > 14] != capi.SV_BATCH_RESIDENT)
    # spot-check two chains against the oracle
    for c in (int(np.argmin(Ls)), 7):
        _, _, e_o, _ = orc.run_chain(chains[c], periods=2)
        np.testing.assert_allclose(e[c], e_o, atol=1e-5, rtol=0)
