"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds no arithmetic of the simulation method: it only draws
random numbers (SplitMix64, Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) and turns Bloch angles into
single-site spinors, which is how a product initial state is handed to
``sv_init``.  Everything downstream of the spinors (the tensor product, the
gates, the energy) is computed separately by the oracle and by the library.

Workload presets mirror the driven-chain workloads the paper's method is
exercised on (Sec. III: open chain, Floquet period T, energy density
recorded once per period).  Every preset is synthetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace
from typing import List, Optional

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream (published constants of the 2014 paper)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on the closed range [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1))


def bloch_angles(rng: SplitMix64, L: int) -> np.ndarray:
    """Per-site (theta, phi): theta ~ U[0, pi], phi ~ U[0, 2 pi), drawn
    site by site, theta before phi."""
    out = np.empty((L, 2), dtype=np.float64)
    for i in range(L):
        out[i, 0] = math.pi * rng.uniform()
        out[i, 1] = 2.0 * math.pi * rng.uniform()
    return out


def spinors_from_angles(angles: np.ndarray) -> np.ndarray:
    """(L, 4) float64 rows (re a, im a, re b, im b) with a = cos(theta/2) the
    |0> (spin-up) component and b = exp(i phi) sin(theta/2) the |1>
    component."""
    th, ph = angles[:, 0], angles[:, 1]
    a = np.cos(th / 2)
    s = np.sin(th / 2)
    return np.stack([a, np.zeros_like(a), np.cos(ph) * s, np.sin(ph) * s], axis=1)


def random_product_spinors(L: int, seed: int) -> np.ndarray:
    return spinors_from_angles(bloch_angles(SplitMix64(seed), L))


@dataclass
class ChainConfig:
    """One driven open chain: the Ising-type Trotter circuit family.

    Per period: ``K`` Trotter steps, each an even-bond layer then an
    odd-bond layer (``first_layer`` = parity of the bonds applied first) of
    gates exp(-i tau h_b) with tau = T / K, then the kick exp(-i theta sum X).
    """

    L: int
    J: float = 1.0
    hx: float = 0.9
    hz: float = 0.4
    T: float = 0.5
    K: int = 4
    theta: float = 0.3
    edge_field_weight: float = 0.5
    first_layer: int = 0
    periods: int = 100
    seed: int = 0
    theta_p: Optional[np.ndarray] = None  # per-period kick angles
    hx_p: Optional[np.ndarray] = None  # per-period transverse field
    name: str = ""

    @property
    def tau(self) -> float:
        return self.T / self.K

    def spinors(self) -> np.ndarray:
        return random_product_spinors(self.L, self.seed)

    def two_qubit_gates_per_period(self) -> int:
        return self.K * (self.L - 1)


def preset(name: str) -> ChainConfig:
    """Named synthetic workloads.

    small   L=12, 100 periods (oracle-sized parity case)
    mid     L=26, 1000 periods (512 MiB complex64 state)
    adjoint L=20, 200 periods with per-period (theta_p, hx_p)
    large   L=30 (8 GiB complex64 state), the throughput workload
    huge    L=34 in place (128 GiB complex64 state), 100 periods
    """
    base = dict(J=1.0, hx=0.9, hz=0.4, T=0.5, K=4, theta=0.3)
    if name == "small":
        return ChainConfig(L=12, periods=100, seed=0, name=name, **base)
    if name == "mid":
        return ChainConfig(L=26, periods=1000, seed=1, name=name, **base)
    if name == "adjoint":
        P = 200
        return ChainConfig(L=20, periods=P, seed=3, name=name,
                           theta_p=np.full(P, 0.3), hx_p=np.full(P, 0.9), **base)
    if name == "large":
        return ChainConfig(L=30, periods=10_000, seed=4, name=name, **base)
    if name == "huge":
        return ChainConfig(L=34, periods=100, seed=4, name=name, **base)
    raise KeyError(name)


def batch_preset(n_chains: int = 512, seed: int = 2, Lmin: int = 14,
                 Lmax: int = 22, periods: int = 2000) -> List[ChainConfig]:
    """Independent chains of uneven length with per-chain couplings.

    All chain parameters are drawn first (L, J, hx, hz, theta per chain, in
    that order), then one seed per chain for its product state."""
    rng = SplitMix64(seed)
    chains = []
    for c in range(n_chains):
        L = rng.randint(Lmin, Lmax)
        J = rng.uniform_range(0.8, 1.2)
        hx = rng.uniform_range(0.6, 1.0)
        hz = rng.uniform_range(0.2, 0.6)
        th = rng.uniform_range(0.1, 0.5)
        chains.append(ChainConfig(L=L, J=J, hx=hx, hz=hz, theta=th,
                                  periods=periods, name=f"chain{c}"))
    for c in range(n_chains):
        chains[c] = replace(chains[c], seed=rng.next_u64())
    return chains


# ------------------------------------------------- the paper's random circuit

def _normal_pair(rng: SplitMix64):
    """Two independent standard normals from two uniforms (Box and Muller,
    Ann. Math. Statist. 29 (1958) 610)."""
    u1 = 1.0 - rng.uniform()  # (0, 1]
    u2 = rng.uniform()
    r = math.sqrt(-2.0 * math.log(u1))
    return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)


def gue_bond_terms(n_bonds: int, seed: int, frobenius: float = math.sqrt(2.0)) -> np.ndarray:
    """(n_bonds, 4, 4) complex128 two-site Hamiltonians of the random Floquet
    circuit of Sec. III.A: each a Gaussian-unitary-ensemble sample
    (G + G^dagger) / 2, G with independent complex normal entries, shifted
    to zero trace and scaled to Frobenius norm J = sqrt(2).  Drawn one bond
    after another (entries row by row, each as (re, im)), so the first L - 1
    terms are the same for every L, as the paper uses one long list.  The
    paper's own sample is not available; this is a seeded stand-in."""
    rng = SplitMix64(seed)
    out = np.empty((n_bonds, 4, 4), dtype=np.complex128)
    for b in range(n_bonds):
        g = np.empty((4, 4), dtype=np.complex128)
        for r in range(4):
            for c in range(4):
                re, im = _normal_pair(rng)
                g[r, c] = complex(re, im)
        h = (g + g.conj().T) / 2
        h = h - (np.trace(h).real / 4) * np.eye(4)
        out[b] = h * (frobenius / np.linalg.norm(h))
    return out


def pair_ground_states(h_bonds: np.ndarray, L: int) -> np.ndarray:
    """(L/2, 4): the ground state of each bond term on the site pairs (0, 1),
    (2, 3), ... (the paper's 1-based odd bonds), the dimer-product initial
    state of Eq. 9; local index r = 2 b_2k + b_2k+1 as for the bond terms.
    Each vector's largest entry is made real and positive.  (A 4 x 4
    eigensolver prepares the input here; neither the oracle nor the library
    sees anything but the resulting vectors.)"""
    assert L % 2 == 0 and h_bonds.shape[0] >= L - 1
    out = np.empty((L // 2, 4), dtype=np.complex128)
    for k in range(L // 2):
        w, v = np.linalg.eigh(h_bonds[2 * k])
        g = v[:, 0]
        j = int(np.argmax(np.abs(g)))
        out[k] = g * (abs(g[j]) / g[j])
    return out


@dataclass
class CircuitConfig:
    """The paper's random Floquet circuit (Sec. III.A): L qubits, GUE bond
    terms H_k, gates exp(-i H_k T), the layer of the paper's even bonds
    (0-based odd bonds) first, no kick, drive frequency omega = 2 pi / T,
    started from the dimer-product state of Eq. 9."""
    L: int
    omega: float = 6.0
    seed: int = 11

    @property
    def T(self) -> float:
        return 2.0 * math.pi / self.omega

    def h_bonds(self) -> np.ndarray:
        return gue_bond_terms(self.L - 1, self.seed)

    def pair_states(self) -> np.ndarray:
        return pair_ground_states(self.h_bonds(), self.L)

    def build_kwargs(self) -> dict:
        """Keyword arguments of FloquetSimulator.build (plain form; add
        mode / block_n / split for the block form)."""
        return dict(h_bonds=self.h_bonds(), T=self.T, K=1, first_layer=1, theta=0.0)
