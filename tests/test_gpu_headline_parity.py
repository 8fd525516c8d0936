"""Element-by-element parity at the bench workload's size.

One period of the L = 30 chain (Sec. III.A: K Trotter steps of the two
brickwork layers, then the kick) in the plain and tensor-core block forms,
every one of the 2^30 amplitudes compared with the FP64 oracle run on the
host in the same test, plus the period's energy density.  At L = 30 the
tensor-core form's period is 16 passes starting at the window of site 2:
the evolution runs the relabel pass into that layout, the period, and the
last pass's variant that hands back the natural layout, so a wrong store
of any subset of amplitudes in any of them fails here, not only through an
energy.

The oracle's state is 16 GiB (FP64); on a host with less than 96 GiB of
memory the test runs at L = 28 instead (still 2^15 tiles, 216 tiles per
CTA)."""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

CHUNK = 1 << 24


def _host_bytes():
    try:
        return os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError, AttributeError):
        return 0


L_HEAD = 30 if _host_bytes() >= (96 << 30) else 28


@pytest.fixture(scope="module")
def oracle_one_period():
    cfg = inputs.ChainConfig(L=L_HEAD, seed=4)
    psi = orc.product_state(cfg.spinors())
    hdrive, hobs = orc.chain_inputs(cfg)
    e, n = orc.evolve(psi, 1, hdrive, cfg.tau, cfg.theta, cfg.K, cfg.first_layer, hobs)
    yield cfg, psi, float(e[0])
    del psi


def _compare(psi, psi_o):
    """Chunked comparison (no state-sized temporaries): the largest
    amplitude error, the L2 error, the largest reference amplitude and the
    infidelity."""
    d2 = n_o = n_g = 0.0
    dmax = amax = 0.0
    ov = 0.0 + 0.0j
    for s in range(0, psi_o.size, CHUNK):
        g = psi[s:s + CHUNK].astype(np.complex128)
        o = psi_o[s:s + CHUNK]
        d = np.abs(g - o)
        dmax = max(dmax, float(d.max()))
        amax = max(amax, float(np.abs(o).max()))
        d2 += float(np.dot(d, d))
        n_o += float(np.vdot(o, o).real)
        n_g += float(np.vdot(g, g).real)
        ov += complex(np.vdot(o, g))
    return dmax, np.sqrt(d2), amax, 1.0 - abs(ov) ** 2 / (n_o * n_g)


@pytest.mark.parametrize("form", ["block_tc", "plain"])
def test_one_period_every_amplitude_at_bench_size(svlib, oracle_one_period, form):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg, psi_o, e_o = oracle_one_period
    kw = chain_params(cfg)
    if form == "block_tc":
        kw.update(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3)
    with FloquetSimulator(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**kw)
        if form == "block_tc":
            assert sim.form_info() == (True, 6)
        passes = sim.pass_info()[0]
        e, n = sim.evolve(1)
        psi = sim.host_state()
    dmax, d2, amax, infid = _compare(psi, psi_o)
    del psi
    # Tensor-core form: each pass rounds an amplitude to 2^-24 of its row's
    # largest one (digits at the row's exponent) plus the FP32 store, a
    # random walk over the passes; plain form: each of the 116 gate passes
    # rounds to FP32 (gate tables exact to ~2^-48).  Bounded per amplitude
    # relative to the largest amplitude, and in L2 against the unit norm.
    per_pass = 2.0 ** -23
    assert dmax < 2 * per_pass * np.sqrt(passes) * amax * 8, (form, dmax, amax)
    assert d2 < 4e-6 * np.sqrt(passes), (form, d2)
    assert infid < 1e-8, (form, infid)
    assert abs(e[0] - e_o) < 1e-6, (form, e[0], e_o)
    assert abs(n[0] - 1.0) < 1e-6, (form, n[0])
