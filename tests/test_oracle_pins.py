"""Pins of the FP64 oracle to things other than itself (no GPU).

Each test fixes the oracle against mathematics the paper's method reduces to:
dense exponentials of each layer (Eq. 4, Eq. 5), closed forms, invariants
(unitarity, the echo of Sec. V), symmetry and brute force at tiny L.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as orc
from paper_2111_08044_gb300 import inputs
from tests import dense_reference as dr


def _dense_case(L, J, hx, hz, ew, tau, theta, K, first_layer, periods, seed):
    sp = inputs.random_product_spinors(L, seed)
    bond_dense = [dr.ising_bond_dense(L, b, J, hx, hz, ew) for b in range(L - 1)]
    U = dr.floquet_dense(bond_dense, L, tau, theta, K, first_layer)
    H0 = sum(bond_dense)
    psi_d = dr.product_state_dense(sp)
    e_dense = []
    for _ in range(periods):
        psi_d = U @ psi_d
        e_dense.append(np.vdot(psi_d, H0 @ psi_d).real / L)
    psi_o = orc.product_state(sp)
    hb = orc.ising_bond_hamiltonians(L, J, hx, hz, ew)
    e_or, n_or = orc.evolve(psi_o, periods, hb, tau, theta, K, first_layer, hb)
    return psi_d, np.array(e_dense), psi_o, e_or, n_or


@pytest.mark.parametrize("L", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("first_layer", [0, 1])
def test_T1_oracle_matches_dense_exponential(L, first_layer):
    rng = np.random.default_rng(100 + L)
    J, hx, hz = rng.uniform(0.5, 1.5, 3)
    ew = 0.5 if L % 2 == 0 else 1.0
    psi_d, e_d, psi_o, e_o, n_o = _dense_case(L, J, hx, hz, ew, 0.13, 0.37, 3,
                                              first_layer, 4, seed=L)
    np.testing.assert_allclose(psi_o, psi_d, atol=1e-12, rtol=0)
    np.testing.assert_allclose(e_o, e_d, atol=1e-12, rtol=0)
    np.testing.assert_allclose(n_o, 1.0, atol=1e-13)


def test_T1_dense_L10_default_circuit():
    cfg = inputs.ChainConfig(L=10, periods=3)
    psi_d, e_d, psi_o, e_o, _ = _dense_case(cfg.L, cfg.J, cfg.hx, cfg.hz,
                                            cfg.edge_field_weight, cfg.tau, cfg.theta,
                                            cfg.K, 0, cfg.periods, seed=7)
    np.testing.assert_allclose(psi_o, psi_d, atol=1e-12, rtol=0)
    np.testing.assert_allclose(e_o, e_d, atol=1e-12, rtol=0)


def _rotate(v, n, alpha):
    """Bloch vector under exp(-i alpha n.sigma): rotation by 2 alpha about n."""
    c, s = math.cos(2 * alpha), math.sin(2 * alpha)
    return v * c + np.cross(n, v) * s + n * np.dot(n, v) * (1 - c)


@pytest.mark.parametrize("L,ew", [(8, 0.5), (9, 0.5), (7, 1.0), (2, 0.5)])
def test_T2_J0_closed_form_precession(L, ew):
    hx, hz, T, K, theta, P = 0.9, 0.4, 0.5, 4, 0.3, 6
    angles = inputs.bloch_angles(inputs.SplitMix64(11), L)
    sp = inputs.spinors_from_angles(angles)
    # per-site field weight: interior sites 1, end sites ew (one bond each)
    w = np.ones(L)
    w[0] = w[-1] = ew
    if L == 2:
        w[:] = ew
    vecs = [np.array([math.sin(a[0]) * math.cos(a[1]), math.sin(a[0]) * math.sin(a[1]),
                      math.cos(a[0])]) for a in angles]
    hnorm = math.hypot(hx, hz)
    nfield = np.array([hx / hnorm, 0.0, hz / hnorm])
    e_closed = []
    for _ in range(P):
        for i in range(L):
            vecs[i] = _rotate(vecs[i], nfield, T * w[i] * hnorm)
            vecs[i] = _rotate(vecs[i], np.array([1.0, 0, 0]), theta)
        e_closed.append(sum(w[i] * (hx * vecs[i][0] + hz * vecs[i][2]) for i in range(L)) / L)
    psi = orc.product_state(sp)
    hb = orc.ising_bond_hamiltonians(L, 0.0, hx, hz, ew)
    e_o, n_o = orc.evolve(psi, P, hb, T / K, theta, K, 0, hb)
    np.testing.assert_allclose(e_o, e_closed, atol=1e-12, rtol=0)


def test_T3_norm_preserved_small_preset():
    cfg = inputs.preset("small")
    _, _, e, n = orc.run_chain(cfg)
    # 44 gate applications per period, each unitary to ~1e-16 in FP64
    assert np.all(np.abs(n - 1.0) < 1e-11)
    assert np.all(np.isfinite(e))


@pytest.mark.parametrize("L,ew", [(6, 0.5), (7, 1.0), (12, 0.5)])
def test_T4_product_state_energy_closed_form(L, ew):
    J, hx, hz = 1.1, 0.7, 0.45
    angles = inputs.bloch_angles(inputs.SplitMix64(5 + L), L)
    x = np.sin(angles[:, 0]) * np.cos(angles[:, 1])
    z = np.cos(angles[:, 0])
    e = 0.0
    for b in range(L - 1):
        wl = ew if b == 0 else 0.5
        wr = ew if b + 1 == L - 1 else 0.5
        e += J * z[b] * z[b + 1] + hx * (wl * x[b] + wr * x[b + 1]) + hz * (wl * z[b] + wr * z[b + 1])
    psi = orc.product_state(inputs.spinors_from_angles(angles))
    e_o, n_o = orc.energy(psi, orc.ising_bond_hamiltonians(L, J, hx, hz, ew))
    assert abs(e_o - e) < 1e-12
    assert abs(n_o - 1.0) < 1e-13


@pytest.mark.parametrize("first_layer", [0, 1])
def test_T5_echo_returns_initial_state(first_layer):
    cfg = inputs.ChainConfig(L=11, first_layer=first_layer)
    psi0 = orc.product_state(cfg.spinors())
    psi = psi0.copy()
    hb = orc.ising_bond_hamiltonians(cfg.L, cfg.J, cfg.hx, cfg.hz)
    gates = orc.bond_gates(hb, cfg.tau)
    kick = orc.kick_gates(cfg.L, cfg.theta)
    for _ in range(20):
        orc.period(psi, gates, kick, cfg.K, first_layer)
    assert abs(np.vdot(psi0, psi)) < 0.999  # it did move
    for _ in range(20):
        orc.period(psi, gates, kick, cfg.K, first_layer, inverse=True)
    assert abs(1 - np.vdot(psi0, psi)) < 1e-12


def test_T6_reflection_symmetry_even_L():
    L = 10
    cfg = inputs.ChainConfig(L=L, periods=8)
    sp = cfg.spinors()
    _, e0a, ea, _ = orc.run_chain(cfg, spinors=sp)
    _, e0b, eb, _ = orc.run_chain(cfg, spinors=np.ascontiguousarray(sp[::-1]))
    assert abs(e0a - e0b) < 1e-13
    np.testing.assert_allclose(ea, eb, atol=1e-12, rtol=0)


def _gue4(rng):
    a = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    h = (a + a.conj().T) / 2
    h -= np.trace(h) / 4 * np.eye(4)
    return h * (math.sqrt(2) / np.linalg.norm(h))


@pytest.mark.parametrize("L", [3, 4, 6])
def test_T7_non_symmetric_gates_pin_index_convention(L):
    rng = np.random.default_rng(L)
    hb = np.stack([_gue4(rng) for _ in range(L - 1)])
    # the gates must not be symmetric for this test to mean anything
    g0 = orc.expm_herm(hb[0], 0.3)
    assert np.abs(g0 - g0.T).max() > 1e-3
    bond_dense = [dr.two_site_op(L, b, hb[b]) for b in range(L - 1)]
    tau, theta, K = 0.3, 0.2, 2
    U = dr.floquet_dense(bond_dense, L, tau, theta, K, 1)
    sp = inputs.random_product_spinors(L, 99)
    psi_d = U @ U @ dr.product_state_dense(sp)
    psi_o = orc.product_state(sp)
    e_o, _ = orc.evolve(psi_o, 2, hb, tau, theta, K, 1, hb)
    np.testing.assert_allclose(psi_o, psi_d, atol=1e-12, rtol=0)
    H0 = sum(bond_dense)
    assert abs(e_o[-1] - np.vdot(psi_d, H0 @ psi_d).real / L) < 1e-12


def test_expm_against_scipy_and_kick_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(5):
        h = _gue4(rng) * rng.uniform(0.1, 4.0)
        tau = rng.uniform(0.05, 2.0)
        np.testing.assert_allclose(orc.expm_herm(h, tau), sla.expm(-1j * tau * h),
                                   atol=1e-13, rtol=0)
    th = 0.3
    k = orc.kick_gates(1, th)[0]
    np.testing.assert_allclose(k, math.cos(th) * np.eye(2) - 1j * math.sin(th) * dr.X,
                               atol=1e-15, rtol=0)


def test_product_state_matches_kron():
    sp = inputs.random_product_spinors(7, 21)
    np.testing.assert_allclose(orc.product_state(sp), dr.product_state_dense(sp),
                               atol=1e-15, rtol=0)


@pytest.mark.parametrize("L,P", [(6, 3), (5, 2)])
def test_adjoint_matches_central_differences(L, P):
    rng = np.random.default_rng(L)
    J, hz, ew, tau, K = 1.0, 0.4, 0.5, 0.125, 4
    theta = rng.uniform(0.2, 0.4, P)
    hx = rng.uniform(0.7, 1.1, P)
    sp = inputs.random_product_spinors(L, 31)
    hobs = orc.ising_bond_hamiltonians(L, J, 0.9, hz, ew)

    def drive(hxv):
        return np.stack([orc.ising_bond_hamiltonians(L, J, h, hz, ew) for h in hxv])

    def f(th, hxv):
        psi = orc.product_state(sp)
        e, _ = orc.evolve(psi, P, drive(hxv), tau, th, K, 0, hobs)
        return e[-1]

    dh = np.stack([orc.ising_dh_dhx(L, ew)] * P)
    psi = orc.product_state(sp)
    gt, gh, efin = orc.adjoint(psi, drive(hx), dh, tau, theta, K, 0, hobs)
    assert abs(efin - f(theta, hx)) < 1e-13
    eps = 1e-5
    for p in range(P):
        d = np.zeros(P)
        d[p] = eps
        fd_t = (f(theta + d, hx) - f(theta - d, hx)) / (2 * eps)
        fd_h = (f(theta, hx + d) - f(theta, hx - d)) / (2 * eps)
        assert abs(gt[p] - fd_t) < 1e-8 * max(1.0, abs(fd_t))
        assert abs(gh[p] - fd_h) < 1e-8 * max(1.0, abs(fd_h))
