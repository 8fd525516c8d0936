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
