"""The paper's own experiment (Sec. IV, on the model of Sec. III.A): the
random Floquet circuit of GUE bond terms, started from the dimer-product
state of Eq. 9, with the energy
E(t) = <H_bar> and its spread sigma_E(t) (Eq. 10, Eq. 11) recorded at
log-spaced times for several drive frequencies omega = 2 pi / T, and the
heating rate Gamma = 1/(t_2 - t_1) with E(t_k) = E(0) e^-k, fitted to
Gamma = exp(a omega + b) across the frequencies (Sec. IV).

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


def crossing_time(t, ratio, k: int):
    """The time t_k at which E(t)/E(0) first falls to e^-k (Sec. IV: E
    relaxes from E(0) < 0 towards the infinite-temperature value 0), by
    linear interpolation in log t between the two samples that bracket it
    (the samples are log-spaced); None if the curve never gets there."""
    level = math.exp(-k)
    t = np.asarray(t, dtype=float)
    r = np.asarray(ratio, dtype=float)
    if r[0] <= level:
        return float(t[0])
    for i in range(1, len(t)):
        if r[i] > level:
            continue
        w = (r[i - 1] - level) / (r[i - 1] - r[i])  # r[i - 1] > level >= r[i]
        if t[i - 1] <= 0.0:  # the first sample is t = 0
            return float(t[i - 1] + w * (t[i] - t[i - 1]))
        return float(math.exp(math.log(t[i - 1]) + w * (math.log(t[i]) - math.log(t[i - 1]))))
    return None


def heating_rate(t, energy):
    """Gamma = 1 / (t_2 - t_1), the paper's thermalization rate (Sec. IV),
    from the energy curve E(t) with E(0) = energy[0]; None if E(t) does not
    reach E(0) e^-2 within the run."""
    r = np.asarray(energy, dtype=float) / float(energy[0])
    t1, t2 = crossing_time(t, r, 1), crossing_time(t, r, 2)
    if t1 is None or t2 is None or t2 <= t1:
        return None
    return 1.0 / (t2 - t1)


def fit_rates(omegas, rates):
    """Least-squares fit of log Gamma = a omega + b (the paper's exponential
    suppression of heating in the drive frequency); returns (a, b)."""
    a, b = np.polyfit(np.asarray(omegas, dtype=float), np.log(np.asarray(rates, dtype=float)), 1)
    return float(a), float(b)


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
    got = []
    for w in (float(x) for x in a.omega.split(",")):
        cfg, rows = run(a.L, w, a.tmax, a.points, a.seed, not a.plain)
        for r in rows:
            print(json.dumps(dict(omega=w, T=cfg.T, **r)), flush=True)
        g = heating_rate([r["t"] for r in rows], [r["E"] for r in rows])
        print(json.dumps(dict(omega=w, heating_rate=g)), flush=True)
        if g is not None:
            got.append((w, g))
    if len(got) >= 2:
        fa, fb = fit_rates([w for w, _ in got], [g for _, g in got])
        print(json.dumps(dict(fit="log Gamma = a omega + b", a=fa, b=fb, points=len(got))), flush=True)


if __name__ == "__main__":
    main()
