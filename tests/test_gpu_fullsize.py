"""Full-size parity of the complex64 forms, at the bench workload's L = 30 and
the in-place L = 34 state (128 GiB), through properties the FP64 oracle or
the mathematics fix at any size:

* one period with J != 0: after one period (K Trotter steps of two
  brickwork layers) <h_b> of a product state depends only on sites within
  2K of the bond, so the full-chain energy density is the sum over bonds of
  oracle runs on sub-chains that cover each bond's light cone;
* J = 0: every site precesses independently, so the energy density after
  any number of periods has a closed form."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


def _gpu_energies(cfg, mode, periods):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    kw = chain_params(cfg)
    if mode == "block":
        kw.update(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3)
    with FloquetSimulator(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**kw)
        if mode == "block":
            assert sim.form_info() == (True, 6)
        e, n = sim.evolve(periods)
    return e, n


def _light_cone_energy(cfg):
    """Energy density after one period from per-bond oracle runs on
    sub-chains [lo, hi] covering sites b - 2K - 1 .. b + 2K + 2 (lo even, so
    the sub-chain keeps the chain's layer parity; its bonds carry the
    full chain's bond Hamiltonians)."""
    L, K = cfg.L, cfg.K
    hfull = orc.ising_bond_hamiltonians(L, cfg.J, cfg.hx, cfg.hz, cfg.edge_field_weight)
    sp = cfg.spinors()
    reach = 2 * K + 1
    total = 0.0
    for b in range(L - 1):
        lo = max(0, b - reach)
        lo -= lo % 2
        hi = min(L - 1, b + 1 + reach)
        ls = hi - lo + 1
        psi = orc.product_state(sp[lo:hi + 1])
        hdrive = np.ascontiguousarray(hfull[lo:hi])
        hobs = np.zeros_like(hdrive)
        hobs[b - lo] = hfull[b]
        e, n = orc.evolve(psi, 1, hdrive, cfg.tau, cfg.theta, K, cfg.first_layer, hobs)
        # evolve reports <psi|h_b|psi> / (ls <psi|psi>)
        total += e[0] * ls
    return total / L


@pytest.mark.parametrize("mode", ["block", "plain"])
def test_light_cone_energy_L30_one_period(svlib, mode):
    cfg = inputs.ChainConfig(L=30, seed=4)
    e, n = _gpu_energies(cfg, mode, 1)
    ref = _light_cone_energy(cfg)
    assert abs(e[0] - ref) < 1e-5, (e[0], ref)
    assert abs(n[0] - 1.0) < 1e-5


def _rotate(v, n, alpha):
    c, s = math.cos(2 * alpha), math.sin(2 * alpha)
    return v * c + np.cross(n, v) * s + n * np.dot(n, v) * (1 - c)


def _j0_closed_form(cfg, periods):
    L = cfg.L
    angles = inputs.bloch_angles(inputs.SplitMix64(cfg.seed), L)
    w = np.ones(L)
    w[0] = w[-1] = cfg.edge_field_weight
    vecs = [np.array([math.sin(a[0]) * math.cos(a[1]), math.sin(a[0]) * math.sin(a[1]),
                      math.cos(a[0])]) for a in angles]
    hn = math.hypot(cfg.hx, cfg.hz)
    nf = np.array([cfg.hx / hn, 0.0, cfg.hz / hn])
    out = []
    for _ in range(periods):
        for i in range(L):
            vecs[i] = _rotate(vecs[i], nf, cfg.T * w[i] * hn)
            vecs[i] = _rotate(vecs[i], np.array([1.0, 0.0, 0.0]), cfg.theta)
        out.append(sum(w[i] * (cfg.hx * vecs[i][0] + cfg.hz * vecs[i][2]) for i in range(L)) / L)
    return np.array(out)


@pytest.mark.parametrize("L,mode,periods", [(30, "block", 3), (30, "plain", 2), (34, "block", 2)])
def test_j0_closed_form_full_size(svlib, L, mode, periods):
    """L = 34 runs in place: one 128 GiB state buffer, no second copy."""
    cfg = inputs.ChainConfig(L=L, J=0.0, seed=5)
    e, n = _gpu_energies(cfg, mode, periods)
    np.testing.assert_allclose(e, _j0_closed_form(cfg, periods), atol=1e-5, rtol=0)
    assert np.all(np.abs(n - 1.0) < 1e-5)


def test_tensor_core_pass_is_deterministic_L30(svlib):
    """Two runs of the same L = 30 evolution give bit-identical energies and
    norms.  Every buffer the tensor-core pass hands between roles (input ring
    slots, TMEM operands and accumulators, the staging tile) is released only
    after its readers are done, including the proxy fence between the
    converters' reads of a ring slot and the next TMA load into it; a missing
    hand-over shows up here as run-to-run differences."""
    cfg = inputs.ChainConfig(L=30, seed=4)
    e1, n1 = _gpu_energies(cfg, "block", 3)
    e2, n2 = _gpu_energies(cfg, "block", 3)
    assert np.array_equal(e1, e2), (e1, e2)
    assert np.array_equal(n1, n2), (n1, n2)
    assert np.all(np.abs(n1 - 1.0) < 3e-6), n1
