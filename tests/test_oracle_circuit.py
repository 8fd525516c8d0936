"""The paper's own random Floquet circuit (Sec. III.A): GUE bond terms,
gates exp(-i H_k T), the layer of the paper's even bonds first, and the
dimer-product initial state of Eq. 9.  Pins of the seeded inputs, of the
oracle's pair product state, of the oracle's evolution of this circuit
against dense layer exponentials, and of the library's host gates."""
import ctypes
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs
from tests import dense_reference as dr


def test_gue_bond_terms():
    h = inputs.gue_bond_terms(40, 5)
    assert np.allclose(h, h.conj().transpose(0, 2, 1), atol=0)
    assert np.max(np.abs(np.trace(h, axis1=1, axis2=2))) < 1e-14
    np.testing.assert_allclose(np.linalg.norm(h, axis=(1, 2)), math.sqrt(2), atol=1e-14)
    # one long list: the first terms do not depend on how many are drawn
    np.testing.assert_array_equal(inputs.gue_bond_terms(7, 5), h[:7])
    assert not np.allclose(inputs.gue_bond_terms(7, 6), h[:7])
    # the entries are not degenerate (a GUE draw has a spread spectrum)
    w = np.linalg.eigvalsh(h[0])
    assert np.min(np.diff(w)) > 1e-3


def test_pair_ground_states_are_ground_states():
    h = inputs.gue_bond_terms(9, 3)
    ps = inputs.pair_ground_states(h, 10)
    for k in range(5):
        e0 = np.linalg.eigvalsh(h[2 * k])[0]
        v = ps[k]
        assert abs(np.linalg.norm(v) - 1) < 1e-14
        np.testing.assert_allclose(h[2 * k] @ v, e0 * v, atol=1e-13)


def test_pair_product_state_against_kron():
    """Against the Kronecker order (site L-1) x ... x (site 0): within a
    pair the higher site comes first, so the local index r = 2 b_2k +
    b_2k+1 is read with its two bits swapped."""
    rng = np.random.default_rng(1)
    pairs = rng.normal(size=(3, 4)) + 1j * rng.normal(size=(3, 4))
    psi = orc.pair_product_state(pairs)
    ref = np.array([1.0 + 0j])
    for k in range(2, -1, -1):
        phi = pairs[k] / np.linalg.norm(pairs[k])
        ref = np.kron(ref, phi[[0, 2, 1, 3]])
    np.testing.assert_allclose(psi, ref, atol=1e-15)


@pytest.mark.parametrize("L", [6, 8])
def test_circuit_period_against_dense(L):
    """The oracle's period with K = 1, the 0-based odd bonds first and no
    kick equals U_F = exp(-i T H_even) exp(-i T H_odd) (0-based parities),
    the paper's product of layer exponentials."""
    cfg = inputs.CircuitConfig(L=L, omega=5.0, seed=2)
    h = cfg.h_bonds()
    psi = orc.pair_product_state(cfg.pair_states())
    dense_psi = psi.copy()
    terms = [dr.two_site_op(L, b, h[b]) for b in range(L - 1)]
    H_odd = sum(terms[b] for b in range(1, L - 1, 2))
    H_even = sum(terms[b] for b in range(0, L - 1, 2))
    UF = sla.expm(-1j * cfg.T * H_even) @ sla.expm(-1j * cfg.T * H_odd)
    for _ in range(3):
        dense_psi = UF @ dense_psi
    e, n = orc.evolve(psi, 3, h, cfg.T, 0.0, 1, 1, h)
    np.testing.assert_allclose(psi, dense_psi, atol=1e-12)
    Hbar = sum(terms)
    E = np.vdot(dense_psi, Hbar @ dense_psi).real
    assert abs(e[-1] - E / L) < 1e-12
    Eo, so, no = orc.energy_moments(psi, h)
    s = math.sqrt(np.vdot(Hbar @ dense_psi, Hbar @ dense_psi).real - E * E)
    assert abs(Eo - E) < 1e-12 and abs(so - s) < 1e-12


def test_host_gates_of_custom_bonds(svlib):
    """sv_host_period_gates with h_bonds: exp(-i (T/K) H_b) against scipy's
    expm, in the circuit's layer order."""
    L = 7
    cfg = inputs.CircuitConfig(L=L, omega=7.0, seed=4)
    h = cfg.h_bonds()
    p, keep = capi.make_params(**cfg.build_kwargs())
    n = ctypes.c_int(0)
    assert svlib.sv_host_period_gates(L, ctypes.byref(p), ctypes.byref(n), None, None) == 0
    bonds = np.zeros(n.value, dtype=np.int32)
    mats = np.zeros((n.value, 4, 4), dtype=np.complex128)
    assert svlib.sv_host_period_gates(L, ctypes.byref(p), ctypes.byref(n),
                                      bonds.ctypes.data_as(capi._ip),
                                      mats.ctypes.data_as(capi._dp)) == 0
    np.testing.assert_array_equal(bonds, [1, 3, 5, 0, 2, 4])
    for b, m in zip(bonds, mats):
        np.testing.assert_allclose(m, sla.expm(-1j * cfg.T * h[b]), atol=1e-13)
    # a non-Hermitian term is refused
    bad = h.copy()
    bad[2, 0, 1] += 0.5
    p2, keep2 = capi.make_params(**dict(cfg.build_kwargs(), h_bonds=bad))
    assert svlib.sv_host_period_gates(L, ctypes.byref(p2), ctypes.byref(n), None, None) == capi.SV_EINVAL


def test_sigma_infinite_temperature_against_dense():
    from paper_2111_08044_gb300.paper_model import sigma_infinite_temperature
    L = 7
    h = inputs.gue_bond_terms(L - 1, 11)
    H = sum(dr.two_site_op(L, b, h[b]) for b in range(L - 1))
    assert abs(np.trace(H)) < 1e-12
    assert abs(sigma_infinite_temperature(h) - math.sqrt(np.trace(H @ H).real / 2 ** L)) < 1e-13
