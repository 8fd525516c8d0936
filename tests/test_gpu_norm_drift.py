"""Norm drift of every complex64 form over many periods.

The exact evolution is unitary, so the norm stays 1 (Sec. III.A).  In
single precision each period's rounding moves it a little; what must not
happen is a drift with a repeating sign, which adds up linearly in the
number of periods (the paper's long f32 runs, Sec. V).  Two such drifts were
found and removed: the plain gate's FMA chain started from a bare product
with a fixed table entry (about -1.3e-9 per gate), and the block passes'
operands were rounded entry by entry (a defect U^H U - I of the same sign
every period, about -1e-7 per period at L = 26).  Here the slope of the
norm over the periods is bounded well below those rates for every form.
"""
import numpy as np
import pytest

from paper_2111_08044_gb300 import capi, inputs
from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params

pytestmark = pytest.mark.gpu

PERIODS = 200
# per-period slope bound; the drifts removed were 4e-8 .. 1.2e-7 per period
# at these lengths, the random walk of the rounding is ~1e-10 per period
SLOPE = 5e-9

FORMS = {
    "plain": dict(mode=capi.SV_MODE_PLAIN),
    "block_simt": dict(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_FP32),
    "block_tc": dict(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3),
    "multigate": dict(mode=capi.SV_MODE_MULTIGATE),
}


def _slope(norms):
    t = np.arange(1, len(norms) + 1, dtype=np.float64)
    return float(np.polyfit(t, norms, 1)[0])


@pytest.mark.parametrize("L", [14, 17, 20])
@pytest.mark.parametrize("form", list(FORMS))
def test_norm_drift_per_period(svlib, form, L):
    cfg = inputs.ChainConfig(L=L, seed=3)
    with FloquetSimulator(L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg, **FORMS[form]))
        if form == "block_tc":
            tc, _ = sim.form_info()
            assert tc == 1
        _, n = sim.evolve(PERIODS)
    s = _slope(n)
    assert abs(s) < SLOPE, (form, L, s, n[-1] - 1.0)
    assert abs(n[-1] - 1.0) < 2 * SLOPE * PERIODS


def test_norm_drift_resident_batch(svlib):
    """The batch's shared-memory resident form (L <= 14) uses the plain
    gate's hi + lo tables with its own FMA chain."""
    from paper_2111_08044_gb300.sim import FloquetBatch
    chains = [inputs.ChainConfig(L=L, seed=20 + k) for k, L in enumerate([10, 12, 14, 14])]
    with FloquetBatch(chains, form=capi.SV_BATCH_RESIDENT) as b:
        assert list(b.forms()) == [capi.SV_BATCH_RESIDENT] * len(chains)
        _, n = b.evolve(PERIODS)
    for c in range(len(chains)):
        s = _slope(n[c])
        assert abs(s) < SLOPE, (chains[c].L, s)
