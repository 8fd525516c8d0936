"""Pins of the oracle's energy moments (E and sigma_E, Eq. 10 and Eq. 11) and
of its echo (Sec. V), against references that share no code with it:
dense Kronecker-product matrices, a closed form for product states from
two- and three-site local algebra, an eigenstate, and the exact return of an
FP64 echo."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import inputs
from tests import dense_reference as dr


def _dense_moments(psi, L, cfg):
    H = sum(dr.ising_bond_dense(L, b, cfg.J, cfg.hx, cfg.hz, cfg.edge_field_weight)
            for b in range(L - 1))
    n = np.vdot(psi, psi).real
    hp = H @ psi
    E = np.vdot(psi, hp).real / n
    var = np.vdot(hp, hp).real / n - E * E
    return E, np.sqrt(var), n


@pytest.mark.parametrize("L,ew", [(5, 0.5), (8, 1.0)])
def test_moments_match_dense(L, ew):
    cfg = inputs.ChainConfig(L=L, seed=3, edge_field_weight=ew)
    rng = np.random.default_rng(L)
    psi = rng.normal(size=1 << L) + 1j * rng.normal(size=1 << L)
    hb = orc.ising_bond_hamiltonians(L, cfg.J, cfg.hx, cfg.hz, cfg.edge_field_weight)
    E, s, n = orc.energy_moments(psi, hb)
    Ed, sd, nd = _dense_moments(psi, L, cfg)
    assert abs(n - nd) < 1e-10 * nd
    assert abs(E - Ed) < 1e-11 * max(1.0, abs(Ed))
    assert abs(s - sd) < 1e-11 * max(1.0, sd)


def _product_state_moments(spinors, hb):
    """E and sigma_E of a product state: the bonds' local expectations, and
    a variance that only adjacent bonds (sharing one site) add covariance to."""
    v = [np.array([s[0] + 1j * s[1], s[2] + 1j * s[3]]) for s in spinors]
    v = [x / np.linalg.norm(x) for x in v]
    L = len(v)
    mean, sq = [], []
    for b in range(L - 1):
        u = np.kron(v[b], v[b + 1])  # local index 2 b_b + b_{b+1}
        hu = hb[b] @ u
        mean.append(np.vdot(u, hu).real)
        sq.append(np.vdot(hu, hu).real)
    var = sum(sq[b] - mean[b] ** 2 for b in range(L - 1))
    I2 = np.eye(2)
    for b in range(L - 2):
        w = np.kron(np.kron(v[b], v[b + 1]), v[b + 2])
        A = np.kron(hb[b], I2)       # bond (b, b+1): the two high bits
        B = np.kron(I2, hb[b + 1])   # bond (b+1, b+2): the two low bits
        ab = np.vdot(w, A @ (B @ w))
        var += 2.0 * (ab.real - mean[b] * mean[b + 1])
    return sum(mean), np.sqrt(var)


@pytest.mark.parametrize("L", [10, 14, 18])
def test_moments_product_state_closed_form(L):
    cfg = inputs.ChainConfig(L=L, seed=7)
    sp = cfg.spinors()
    psi = orc.product_state(sp)
    hb = orc.ising_bond_hamiltonians(L, cfg.J, cfg.hx, cfg.hz, cfg.edge_field_weight)
    E, s, n = orc.energy_moments(psi, hb)
    Ec, sc = _product_state_moments(sp, hb)
    assert abs(n - 1.0) < 1e-12
    assert abs(E - Ec) < 1e-12 * L
    assert abs(s - sc) < 1e-12 * L


def test_moments_zero_variance_for_an_eigenstate():
    """With no transverse field H0 is diagonal, so a basis state has no
    energy spread; its energy is the classical Ising energy."""
    L = 9
    hb = orc.ising_bond_hamiltonians(L, 1.3, 0.0, 0.7, 0.5)
    x = 0b101100110
    psi = np.zeros(1 << L, dtype=np.complex128)
    psi[x] = 1.0
    E, s, n = orc.energy_moments(psi, hb)
    z = [1 - 2 * ((x >> i) & 1) for i in range(L)]
    Ez = sum(1.3 * z[i] * z[i + 1] for i in range(L - 1))
    Ez += sum(0.7 * (0.5 * z[b] + 0.5 * z[b + 1]) for b in range(L - 1))
    assert s < 1e-7 and abs(E - Ez) < 1e-12


@pytest.mark.parametrize("first_layer", [0, 1])
def test_echo_returns_to_the_start_in_fp64(first_layer):
    cfg = inputs.ChainConfig(L=10, seed=2, first_layer=first_layer)
    psi = orc.product_state(cfg.spinors())
    psi0 = psi.copy()
    hb = orc.ising_bond_hamiltonians(cfg.L, cfg.J, cfg.hx, cfg.hz, cfg.edge_field_weight)
    ov = orc.echo(psi, 30, hb, cfg.tau, cfg.theta, cfg.K, first_layer)
    assert abs(1.0 - ov) < 1e-12
    assert np.linalg.norm(psi - psi0) < 1e-11
