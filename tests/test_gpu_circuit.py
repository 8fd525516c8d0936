"""The paper's own random Floquet circuit on the GPU (Sec. III.A, Eq. 9):
GUE bond terms, gates exp(-i H_k T) with the paper's even bonds first, the
dimer-product initial state, and E / sigma_E measured on demand, through the
C ABI against the FP64 oracle; at L = 30 against a light-cone sum of oracle
runs on sub-chains."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

BLOCK = dict(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3)


def _gpu(cfg, periods, precision, extra):
    from paper_2111_08044_gb300.sim import FloquetSimulator
    with FloquetSimulator(cfg.L, precision=precision) as sim:
        sim.init_pairs(cfg.pair_states())
        sim.build(**dict(cfg.build_kwargs(), **extra))
        e, n = sim.evolve(periods)
        moments = sim.energy_moments()
        dens = sim.energy()
        psi = sim.host_state().astype(np.complex128)
    return e, n, moments, dens, psi


def _oracle(cfg, periods):
    h = cfg.h_bonds()
    psi = orc.pair_product_state(cfg.pair_states())
    orc.evolve(psi, periods, h, cfg.T, 0.0, 1, 1, h)
    return psi, orc.energy_moments(psi, h)


@pytest.mark.parametrize("L,precision,mode,tol", [(10, "c128", "plain", 1e-12),
                                                  (12, "c64", "plain", 2e-5),
                                                  (16, "c64", "block", 3e-5)])
def test_circuit_matches_oracle(svlib, L, precision, mode, tol):
    cfg = inputs.CircuitConfig(L=L, omega=6.0, seed=11)
    e, n, (E, s, nn), (dens, n2), psi = _gpu(cfg, 3, precision, BLOCK if mode == "block" else {})
    ref, (Eo, so, no) = _oracle(cfg, 3)
    assert np.linalg.norm(psi - ref) < tol
    mt = 1e-11 if precision == "c128" else 2e-6
    assert abs(E - Eo) < mt * L and abs(s - so) < mt * L and abs(nn - no) < mt
    assert abs(dens - Eo / L) < mt
    # a general chain is not measured per period
    assert np.all(np.isnan(e)) and np.all(np.isnan(n))


@pytest.mark.parametrize("precision,tol", [("c128", 1e-14), ("c64", 2e-7)])
def test_pair_state_and_overlap(svlib, precision, tol):
    from paper_2111_08044_gb300.sim import FloquetSimulator
    cfg = inputs.CircuitConfig(L=14, seed=3)
    ps = cfg.pair_states()
    with FloquetSimulator(cfg.L, precision=precision) as sim:
        sim.init_pairs(ps)
        psi = sim.host_state().astype(np.complex128)
        ov0 = sim.overlap_pairs(ps)
        sim.build(**cfg.build_kwargs())
        sim.evolve(2)
        ov2 = sim.overlap_pairs(ps)
        psi2 = sim.host_state().astype(np.complex128)
    ref = orc.pair_product_state(ps)
    np.testing.assert_allclose(psi, ref, atol=tol, rtol=0)
    assert abs(ov0 - 1.0) < 10 * tol
    assert abs(ov2 - np.vdot(ref, psi2)) < 10 * tol


def test_circuit_echo(svlib):
    """10 periods forward and 10 inverse periods back in the block form
    return to the dimer-product state (the echo of Sec. V)."""
    from paper_2111_08044_gb300.sim import FloquetSimulator
    cfg = inputs.CircuitConfig(L=20, omega=6.0, seed=11)
    ps = cfg.pair_states()
    with FloquetSimulator(cfg.L) as sim:
        sim.init_pairs(ps)
        sim.build(**dict(cfg.build_kwargs(), **BLOCK))
        sim.evolve(10, record=False)
        moved = abs(sim.overlap_pairs(ps))
        sim.build(**dict(cfg.build_kwargs(), inverse=1, **BLOCK))
        sim.evolve(10, record=False)
        ov = sim.overlap_pairs(ps)
    assert moved < 0.99
    assert abs(1.0 - ov) < 1e-4, ov


def _light_cone_energy(cfg):
    """E after one period as a sum over bonds of oracle runs on sub-chains:
    the two layers spread H_b over sites b-2..b+3 and the initial pairs then
    take in at most one more site on each side, so a sub-chain from b-3
    (rounded down to even, keeping pairs and layer parity) to b+4 holds
    every amplitude <H_b> depends on."""
    L = cfg.L
    h = cfg.h_bonds()
    ps = cfg.pair_states()
    total = 0.0
    for b in range(L - 1):
        lo = max(0, b - 3)
        lo -= lo % 2
        hi = min(L - 1, b + 4)
        if (hi - lo) % 2 == 0:
            hi += 1
        psi = orc.pair_product_state(ps[lo // 2:(hi + 1) // 2])
        hsub = np.ascontiguousarray(h[lo:hi])
        hobs = np.zeros_like(hsub)
        hobs[b - lo] = h[b]
        orc.evolve(psi, 1, hsub, cfg.T, 0.0, 1, 1, hobs)
        e, n = orc.energy(psi, hobs)
        total += e / n
    return total


def test_circuit_full_size_light_cone(svlib):
    """L = 30 (8 GiB), block form: E after one period against the light-cone
    sum of oracle runs."""
    cfg = inputs.CircuitConfig(L=30, omega=6.0, seed=11)
    from paper_2111_08044_gb300.sim import FloquetSimulator
    with FloquetSimulator(cfg.L) as sim:
        sim.init_pairs(cfg.pair_states())
        sim.build(**dict(cfg.build_kwargs(), **BLOCK))
        E0, s0, _ = sim.energy_moments()
        sim.evolve(1, record=False)
        E, s, nn = sim.energy_moments()
    ref = _light_cone_energy(cfg)
    assert abs(E - ref) < 1e-5 * cfg.L, (E, ref)
    assert abs(nn - 1.0) < 1e-5
    assert s > 0 and s0 > 0
