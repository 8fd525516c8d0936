"""Error accumulation of the complex64 forms over many periods.

The complex64 plain and tensor-core block forms run in lockstep with a
check run of the same circuit: the complex128 mode (FP64 arithmetic) or the
double-float mode df64 (FP32 pairs, about 48 significant bits), which gives
the same reference about four times faster on a GPU whose FP64 rate is a
small fraction of its FP32 rate.  Both agree with the FP64 CPU oracle to
1e-11 wherever the oracle can run, and with each other to about 1e-12 over
thousands of periods (compare them with `--ref df64 --forms c128`).

Every `every` periods the study records, for each complex64 form:
- the largest energy-density error over the chunk;
- the state infidelity 1 - |<psi_ref|psi>|^2 / (|psi_ref|^2 |psi|^2);
- the norm drift.

The infidelity is computed on the device in FP64. This mirrors the paper's
accuracy study of long f32 runs against a reference (Sec. V).

    python -m paper_2111_08044_gb300.accuracy --L 26 --periods 1000 --every 100
    python -m paper_2111_08044_gb300.accuracy --ref df64 --L 30 --periods 1000

The echo mode follows the paper's own accuracy check (Sec. V) instead: from
the product state, P periods forward and P inverse periods back in one form,
then the overlap error |1 - <psi(0)|psi'(0)>| and the relative changes of E
and sigma_E (Eq. 10-11) between psi(0) and psi'(0):

    python -m paper_2111_08044_gb300.accuracy --echo --L 26 --periods 10,100,1000

and on the paper's own random circuit from its dimer state (omega = 8 as in
Sec. V):

    python -m paper_2111_08044_gb300.accuracy --echo --circuit --L 34 --periods 10 --forms block_tc
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import capi, inputs
from .sim import FloquetSimulator, chain_params

FORMS = {
    "plain": dict(mode=capi.SV_MODE_PLAIN),
    "block_tc": dict(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3),
    "block_simt": dict(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_FP32),
}
# check modes, which a study may also compare with its reference
CHECK = ("c128", "df64")


def _infidelity(ref, psi):
    import torch
    a = ref.state_c128()
    b = psi.state_c128()
    ov = torch.vdot(a, b)
    na = torch.vdot(a, a).real
    nb = torch.vdot(b, b).real
    return float(1.0 - (ov.abs() ** 2) / (na * nb))


def study(L=26, periods=1000, every=100, seed=1, forms=("plain", "block_tc"), ref="c128"):
    """Rows of the study, one per `every` periods (a generator: each row is
    available as soon as its periods have run).  `ref` is the check mode
    (c128 or df64); `forms` are complex64 forms or the other check mode."""
    import time
    import torch
    cfg = inputs.ChainConfig(L=L, seed=seed)
    refname = ref
    ref = FloquetSimulator(L, precision=refname)
    ref.init_product_state(cfg.spinors())
    ref.build(**chain_params(cfg))
    sims = {}
    for name in forms:
        s = FloquetSimulator(L, precision=name if name in CHECK else "c64")
        s.init_product_state(cfg.spinors())
        s.build(**chain_params(cfg, **FORMS.get(name, {})))
        sims[name] = s
    t_ref = 0.0
    done = 0
    while done < periods:
        k = min(every, periods - done)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_ref, n_ref = ref.evolve(k)
        t_ref += time.perf_counter() - t0
        done += k
        row = {"period": done, "ref": refname, "energy_ref": float(e_ref[-1]),
               "norm_ref_dev": float(n_ref[-1] - 1), "ref_s_per_period": t_ref / done}
        for name, s in sims.items():
            e, n = s.evolve(k)
            row[name] = {"max_abs_energy_err": float(np.max(np.abs(e - e_ref))),
                         "infidelity": _infidelity(ref, s),
                         "norm_dev": float(n[-1] - 1.0)}
        yield row
    for s in list(sims.values()) + [ref]:
        s.close()


def echo(L=26, periods=(10, 100, 1000), seed=1, form="block_tc", precision="c64",
         circuit=False, omega=8.0):
    """The echo of Sec. V for each P in `periods`: P periods forward and P
    inverse periods back.  The start is the Ising chain's product state, or
    with `circuit` the paper's own random circuit (GUE bonds, drive
    frequency omega) from its dimer-product state, as in Sec. V.  Returns,
    per P, the overlap error |1 - <psi(0)|psi'(0)>| and the relative
    changes of E and sigma_E of psi'(0) against psi(0)."""
    import time
    import torch
    kw = FORMS[form] if precision == "c64" else {}
    if circuit:
        ccfg = inputs.CircuitConfig(L=L, omega=omega, seed=seed)
        start = ccfg.pair_states()
        period_T = ccfg.T

        def prepare(sim, inverse):
            sim.build(**dict(ccfg.build_kwargs(), inverse=inverse, **kw))

        def init(sim):
            sim.init_pairs(start)

        def overlap(sim):
            return sim.overlap_pairs(start)
    else:
        cfg = inputs.ChainConfig(L=L, seed=seed)
        start = cfg.spinors()
        period_T = cfg.T

        def prepare(sim, inverse):
            sim.build(**chain_params(cfg, inverse=inverse, **kw))

        def init(sim):
            sim.init_product_state(start)

        def overlap(sim):
            return sim.overlap_product(start)
    rows = []
    for P in periods:
        with FloquetSimulator(L, precision=precision) as sim:
            init(sim)
            prepare(sim, 0)
            E0, s0, _ = sim.energy_moments()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.evolve(P, record=False)
            torch.cuda.synchronize()
            t_fwd = time.perf_counter() - t0
            prepare(sim, 1)
            sim.evolve(P, record=False)
            ov = overlap(sim)
            E1, s1, n1 = sim.energy_moments()
        rows.append({"L": L, "model": "circuit" if circuit else "ising",
                     "form": form if precision == "c64" else precision, "periods": P,
                     "total_time": 2 * P * period_T, "overlap_error": abs(1.0 - ov),
                     "rel_err_E": abs(E1 - E0) / abs(E0), "rel_err_sigma": abs(s1 - s0) / s0,
                     "norm_dev": n1 - 1.0, "s_per_period_forward": t_fwd / P})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=26)
    ap.add_argument("--periods", default="1000",
                    help="periods (study), or a comma list of P (echo)")
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--forms", default="plain,block_tc")
    ap.add_argument("--ref", default="c128", choices=CHECK, help="check mode of the study")
    ap.add_argument("--echo", action="store_true")
    ap.add_argument("--circuit", action="store_true",
                    help="echo the paper's random circuit from its dimer state")
    ap.add_argument("--omega", type=float, default=8.0, help="drive frequency (--circuit)")
    a = ap.parse_args()
    if a.echo:
        ps = tuple(int(x) for x in a.periods.split(","))
        for form in a.forms.split(","):
            for row in echo(a.L, ps, a.seed, form, circuit=a.circuit, omega=a.omega):
                print(json.dumps(row), flush=True)
        return
    for row in study(a.L, int(a.periods), a.every, a.seed, tuple(a.forms.split(",")), a.ref):
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
