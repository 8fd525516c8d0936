"""The paper's own experiment (Sec. III): the random Floquet circuit of GUE
bond terms, started from the dimer-product state of Eq. 9, with the energy
E(t) = <H_bar> and its spread sigma_E(t) (Eq. 10, Eq. 11) recorded at
log-spaced times for several drive frequencies omega = 2 pi / T.

The sample of bond terms is a seeded stand-in for the paper's (not
available).  The infinite-temperature references are E_inf = 0 (the terms
are traceless) and sigma_inf^2 = tr(H_bar^2) / 2^L, a sum of single-bond and
adjacent-bond traces.

    python -m paper_2111_08044_gb300.paper_model --L 26 --omega 5,6,7,8 --tmax 1e4
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import capi, inputs
from .sim import FloquetSimulator

BLOCK = dict(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3)


def sigma_infinite_temperature(h: np.ndarray) -> float:
    """sqrt(tr(H_bar^2) / 2^L) for H_bar = sum_b h_b with traceless terms:
    each bond adds |h_b|_F^2 / 4, each adjacent pair twice the normalised
    trace of their product on three sites; terms further apart are
    uncorrelated."""
    s = sum(np.vdot(x, x).real / 4.0 for x in h)
    I2 = np.eye(2)
    for b in range(len(h) - 1):
        A = np.kron(h[b], I2)       # sites (b, b+1): the two high bits of three
        B = np.kron(I2, h[b + 1])   # sites (b+1, b+2): the two low bits
        s += 2.0 * np.trace(A @ B).real / 8.0
    return math.sqrt(s)


def run(L: int, omega: float, t_max: float, points: int = 24, seed: int = 11,
        block: bool = True):
    """Rows {t, periods, E, E/L, sigma_E, norm} from the dimer-product state."""
    cfg = inputs.CircuitConfig(L=L, omega=omega, seed=seed)
    n_max = max(1, int(round(t_max / cfg.T)))
    marks = sorted(set(int(round(x)) for x in np.logspace(0, math.log10(n_max), points)))
    rows = []
    with FloquetSimulator(L) as sim:
        sim.init_pairs(cfg.pair_states())
        sim.build(**dict(cfg.build_kwargs(), **(BLOCK if block else {})))
        E, s, n = sim.energy_moments()
        rows.append(dict(t=0.0, periods=0, E=E, E_per_site=E / L, sigma_E=s, norm=n))
        done = 0
        for m in marks:
            sim.evolve(m - done, record=False)
            done = m
            E, s, n = sim.energy_moments()
            rows.append(dict(t=m * cfg.T, periods=m, E=E, E_per_site=E / L, sigma_E=s, norm=n))
    return cfg, rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=26)
    ap.add_argument("--omega", default="5,6,7,8")
    ap.add_argument("--tmax", type=float, default=1e4)
    ap.add_argument("--points", type=int, default=24)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--plain", action="store_true", help="plain per-gate form (default: block)")
    a = ap.parse_args()
    h = inputs.gue_bond_terms(a.L - 1, a.seed)
    ref = dict(L=a.L, E_inf=0.0, sigma_inf=sigma_infinite_temperature(h))
    print(json.dumps(ref), flush=True)
    for w in (float(x) for x in a.omega.split(",")):
        cfg, rows = run(a.L, w, a.tmax, a.points, a.seed, not a.plain)
        for r in rows:
            print(json.dumps(dict(omega=w, T=cfg.T, **r)), flush=True)


if __name__ == "__main__":
    main()
