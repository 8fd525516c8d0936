#!/usr/bin/env python
"""Throughput of the Floquet period on GB300: periods/s at L=30, complex64.

One step = one Floquet period of the whole hot path: K=4 Trotter steps of
even/odd brickwork gates plus the folded X kick, and the energy density /
norm measurement of that period.  The tensor-core block form is the headline;
the plain per-gate form is timed beside it.  Inputs: a seeded random product
state of 30 sites (8 GiB state, far larger than L2, so no flush is needed).

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]
    torchrun --nproc-per-node N bench.py --gpus N   (independent replicas)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Floquet periods/s at L=30 c64 (plain vs tensor-core block form), % of roofline"
UNIT = "periods/s"
L_BENCH = 30


def _workload(L: int) -> str:
    size = 8 << L
    human = (f"{size >> 30} GiB" if size >= 1 << 30 else
             f"{size >> 20} MiB" if size >= 1 << 20 else f"{size >> 10} KiB")
    return (f"L={L} open chain, complex64 ({human} state), J=1 hx=0.9 hz=0.4 T=0.5 K=4 "
            "theta=0.3, random product state (seed 4 + rank)")


def _parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--oracle-table", action="store_true",
                    help="time the FP64 oracle at several chain lengths and thread counts")
    ap.add_argument("--L", type=int, default=L_BENCH)
    ap.add_argument("--n", type=int, default=6, help="block width of the fused form")
    ap.add_argument("--split", choices=["bf16x3", "fp32"], default="bf16x3")
    ap.add_argument("--plain-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-breakdown", action="store_true",
                    help="time each L group of the 512-chain batch alone against its HBM bound "
                         "(one JSON line per L) instead of the default line")
    ap.add_argument("--batch-periods", type=int, default=2000,
                    help="periods of the 512-chain batch line (the config's 2000; 0 skips it)")
    return ap.parse_args()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _rank_seed(rank):
    """Seed of this replica's product state: each rank evolves its own chain."""
    return 4 + rank


def _time_form(args, mode, steps, rank, world, local):
    """Device-timed K periods of one form; per-launch CUDA events give the
    dominant kernel's average duration."""
    import numpy as np
    import torch

    from paper_2111_08044_gb300 import capi, inputs
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params

    cfg = inputs.ChainConfig(L=args.L, seed=_rank_seed(rank))
    split = capi.SV_SPLIT_BF16X3 if args.split == "bf16x3" else capi.SV_SPLIT_FP32
    kw = chain_params(cfg)
    if mode == "block":
        kw.update(mode=capi.SV_MODE_BLOCK, block_n=args.n, split=split)
    elif mode == "multigate":
        kw.update(mode=capi.SV_MODE_MULTIGATE)
    sim = FloquetSimulator(cfg.L, device=local)
    sim.init_product_state(cfg.spinors())
    sim.build(**kw)
    passes, gates, launches = sim.pass_info()
    entry = 0
    if mode == "block":
        import ctypes
        p, keep = capi.make_params(**kw)
        cnt = ctypes.c_int(0)
        lib = capi.load()
        lib.sv_host_fusion_plan(cfg.L, ctypes.byref(p), args.n, ctypes.byref(cnt), None, None,
                                None)
        lo = np.zeros(cnt.value, dtype=np.int32)
        lib.sv_host_fusion_plan(cfg.L, ctypes.byref(p), args.n, ctypes.byref(cnt),
                                lo.ctypes.data_as(capi._ip), None, None)
        entry = (int(lo[0]) + 6) // 7  # relabel steps from site 0 to the start
    sim.evolve(args.warmup, record=False)
    torch.cuda.synchronize()
    _barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(sim.stream)
    e, n, ms = sim.evolve_profiled(steps)
    end.record(sim.stream)
    torch.cuda.synchronize()
    _barrier(world)
    elapsed_ms = start.elapsed_time(end)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    pass_ms = ms[:passes]
    bytes_per_pass = 16.0 * (1 << args.L)  # read + write of the c64 state
    avg_pass_s = float(pass_ms.sum()) / (steps * passes) / 1e3
    return {
        "elapsed_ms": elapsed_ms,
        "periods_per_s": steps / (elapsed_ms / 1e3),
        "passes_per_period": passes,
        "gates_per_period": gates,
        "launches_per_period": launches,
        "entry_launches": entry,
        "avg_pass_ms": avg_pass_s * 1e3,
        "pass_gbs": bytes_per_pass / avg_pass_s / 1e9,
        "pass_share": float(pass_ms.sum() / ms.sum()),
        "pass_ms_each": [round(float(x) / steps, 4) for x in pass_ms],
        "energy_last": float(e[-1]),
        "norm_last": float(n[-1]),
    }


def _e2e(args, steps, rank, local):
    """Public API end to end with host buffers: sv_init from host spinors,
    sv_build_floquet from host parameters, then one sv_evolve per period
    reading the period's energy and norm back to the host (with the state
    kept in the period layout between calls, sv_set_layout_policy)."""
    import torch

    from paper_2111_08044_gb300 import capi, inputs
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params

    cfg = inputs.ChainConfig(L=args.L, seed=_rank_seed(rank))
    kw = chain_params(cfg, mode=capi.SV_MODE_BLOCK, block_n=args.n,
                      split=capi.SV_SPLIT_BF16X3 if args.split == "bf16x3" else capi.SV_SPLIT_FP32)
    sim = FloquetSimulator(cfg.L, device=local)
    spinors = cfg.spinors()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.init_product_state(spinors)
    sim.build(**kw)
    # one period per call: keep the state in the plan's period layout between
    # calls instead of relabelling it in and out every call
    sim.keep_period_layout(True)
    for _ in range(steps):
        sim.evolve(1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    h2d = spinors.nbytes + sim.build_bytes()
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return {"value": steps / (t1 - t0), "unit": UNIT,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": 16}


def _batch_hbm_bound_ms(chains, forms, widths, hbm_gbs, run=16):
    """HBM-bound milliseconds per period of the batch: every chain's passes
    of a period, plus its entry relabel once per graph run of `run` periods
    when its plan starts off site 0, each moving 16 B x 2^L (read and write
    of complex64) at the measured copy bandwidth.  Resident chains keep
    their state in shared memory within a run and count nothing.  None when
    a chain runs a form without a host plan view (multi-gate)."""
    import ctypes

    from paper_2111_08044_gb300 import capi
    from paper_2111_08044_gb300.sim import chain_params
    lib = capi.load()
    cache, total = {}, 0.0
    for c, cfg in enumerate(chains):
        f, L = int(forms[c]), cfg.L
        if f == capi.SV_BATCH_RESIDENT:
            continue
        key = (L, f, int(widths[c]))
        if key not in cache:
            if f in (capi.SV_BATCH_BLOCK_SIMT, capi.SV_BATCH_BLOCK_TC):
                p, _keep = capi.make_params(**chain_params(cfg, mode=capi.SV_MODE_BLOCK,
                                                           block_n=int(widths[c]) or 6))
                cnt = ctypes.c_int(0)
                capi.check(lib.sv_host_fusion_plan(L, ctypes.byref(p), int(widths[c]) or 6,
                                                   ctypes.byref(cnt), None, None, None))
                lo = (ctypes.c_int * cnt.value)()
                capi.check(lib.sv_host_fusion_plan(L, ctypes.byref(p), int(widths[c]) or 6,
                                                   ctypes.byref(cnt), lo, None, None))
                cache[key] = cnt.value + (1.0 / run if lo[0] != 0 else 0.0)
            elif f == capi.SV_BATCH_PLAIN:
                p, _keep = capi.make_params(**chain_params(cfg))
                cnt = ctypes.c_int(0)
                capi.check(lib.sv_host_period_gates(L, ctypes.byref(p), ctypes.byref(cnt), None,
                                                    None))
                cache[key] = float(cnt.value)
            else:
                return None
        total += cache[key] * 16.0 * (1 << L) / (hbm_gbs * 1e9)
    return total * 1e3


def _batch(args, local):
    """The 512-chain batch (L 14..22, per-chain couplings): chain-periods/s
    over args.batch_periods periods after a warm-up run of 16, with the
    build and autotuning timed separately."""
    import numpy as np
    import torch

    from paper_2111_08044_gb300 import inputs
    from paper_2111_08044_gb300.sim import FloquetBatch

    chains = inputs.batch_preset(512)
    t0 = time.perf_counter()
    b = FloquetBatch(chains, device=local)
    t_create = time.perf_counter() - t0
    b.evolve(16)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(b.stream)
    e, n = b.evolve(args.batch_periods)
    end.record(b.stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    forms = b.forms()
    widths = b.widths()
    Ls = np.array([c.L for c in chains])
    amps = float(sum(1 << int(L) for L in Ls))
    b.close()
    del b
    torch.cuda.empty_cache()
    hbm_gbs = _peaks()[0]
    bound_ms = _batch_hbm_bound_ms(chains, forms, widths, hbm_gbs)
    ms_period = ms / args.batch_periods
    names = {0: "plain", 1: "block_simt", 2: "block_tc", 3: "resident", 4: "multigate"}
    by_L = {}
    for L in sorted(set(Ls.tolist())):
        c = int(np.nonzero(Ls == L)[0][0])
        by_L[str(L)] = names[int(forms[c])] + (f" n={int(widths[c])}" if widths[c] else "")
    return {
        "workload": "512 chains, L uniform 14..22, J~U[0.8,1.2] hx~U[0.6,1.0] hz~U[0.2,0.6] "
                    "theta~U[0.1,0.5], random product states (seed 2), complex64",
        "chain_periods_per_s": 512 * args.batch_periods / (ms / 1e3),
        "periods": args.batch_periods,
        "ms": ms,
        "create_and_autotune_s": t_create,
        "amplitudes": amps,
        "forms": {names[k]: int((forms == k).sum()) for k in range(5) if (forms == k).any()},
        "form_by_L": by_L,
        "norm_max_dev": float(np.abs(n - 1.0).max()),
        "ms_per_period": ms_period,
        "hbm_bound_ms_per_period": bound_ms,
        "hbm_bound_frac": bound_ms / ms_period if bound_ms else None,
    }


def _cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _oracle_full_periods(L: int, periods: int, seed: int, threads=None):
    """The FP64 oracle on the host cores: `periods` full periods (gates, kick
    and the energy / norm measurement of each period) of the bench circuit
    at chain length L, timed as they stand.  Returns (periods/s, seconds,
    threads used)."""
    from oracle import oracle as orc
    from paper_2111_08044_gb300 import inputs
    if threads is not None:
        orc.set_threads(threads)
    cfg = inputs.ChainConfig(L=L, seed=seed)
    psi = orc.product_state(cfg.spinors())
    hdrive, hobs = orc.chain_inputs(cfg)
    t0 = time.perf_counter()
    orc.evolve(psi, periods, hdrive, cfg.tau, cfg.theta, cfg.K, cfg.first_layer, hobs)
    dt = time.perf_counter() - t0
    used = orc.num_threads()
    del psi
    return periods / dt, dt, used


def _oracle_period_groups(L: int, seed: int):
    """The FP64 oracle's period at chain length L cut into its 2K + 2
    operation groups, in order: each gate layer (every bond of one parity,
    index pairing), the kick (every site), and the energy / norm
    measurement.  Any 2K + 2 consecutive groups do one whole period's work.
    Returns (state, groups)."""
    from oracle import oracle as orc
    from paper_2111_08044_gb300 import inputs
    cfg = inputs.ChainConfig(L=L, seed=seed)
    psi = orc.product_state(cfg.spinors())
    hdrive, hobs = orc.chain_inputs(cfg)
    gates = orc.bond_gates(hdrive, cfg.tau)
    kick = orc.kick_gates(L, cfg.theta)
    groups = []
    for _ in range(cfg.K):
        for layer in range(2):
            parity = cfg.first_layer if layer == 0 else 1 - cfg.first_layer

            def gate_layer(parity=parity):
                for b in range(parity, L - 1, 2):
                    orc.apply_2q(psi, b, gates[b])
            groups.append(gate_layer)

    def kick_all():
        for i in range(L):
            orc.apply_1q(psi, i, kick[i])
    groups.append(kick_all)

    def measure():
        orc.energy(psi, hobs)
    groups.append(measure)
    return psi, groups


# DRAM bytes of one tensor-core block pass, read + write, per launch, from
# an ncu capture of three launches at L = 28 (2 GiB state, 1024 tiles per
# CTA): reads 2147.9 MB (the 2147.5 MB the pass must read), writes 2084.1 MB
# (61 MB of the pass's output still sits in L2 when the kernel ends and is
# written back during the next pass).  Traffic scales with the number of
# tiles, i.e. with 2^L.
TC_TRAFFIC_L28 = 2147.9e6 + 2084.1e6


# FP32 pipe of one GB300: 152 SMs x 128 FMA lanes x 2 flops x 2.07 GHz.
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _mg_fp32_tflops(L, form):
    """Algorithmic FP32 rate of the multi-gate form: each gate costs 32 FMA
    per amplitude (the FP32 table and its residual), 4(L-1) gates a period."""
    flops = 2.0 * 32 * (1 << L) * form["gates_per_period"]
    return flops * form["periods_per_s"] / 1e12


def _traffic(args):
    if args.split != "bf16x3" or args.n != 6:
        return None
    return TC_TRAFFIC_L28 * 2.0 ** (args.L - 28)


def run_reference(args):
    """The oracle as it stands on the host cores, on this bench's config:
    step k runs operation group k (mod 2K + 2) of the L=30 period, so 20
    timed steps after 5 warm-up steps are exactly two whole periods."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    psi, groups = _oracle_period_groups(args.L, seed=_rank_seed(0))
    ng = len(groups)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        groups[k % ng]()
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    from oracle import oracle as orc
    total = sum(times)
    value = (args.steps / ng) / total
    sample = (f"the FP64 oracle (index pairing, OpenMP) at L={args.L}: step k is operation "
              f"group k mod {ng} of the period (8 gate layers, the kick, the energy and norm "
              f"measurement); the {args.steps} timed steps do {args.steps / ng:g} periods' "
              f"work (exactly whole periods when steps is a multiple of {ng}); "
              f"CPU: {_cpu_model()}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    del psi
    print(json.dumps(line), flush=True)
    return 0


def _config(args, world):
    l2 = (f"inputs exceed L2 ({(8 << args.L) >> 20} MiB state per replica); no flush" if (8 << args.L) > (129 << 20)
          else "state fits in L2: not the bench workload")
    return {"workload": _workload(args.L),
            "form": f"block n={args.n} {args.split}",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": l2}


def run_batch_breakdown(args):
    """Each L group of the 512-chain preset run alone in the form the full
    batch gives it (resident at L <= 14, tensor-core groups above): ms per
    period of the group against its HBM bound, one JSON line per L."""
    import numpy as np
    import torch

    from paper_2111_08044_gb300 import capi, inputs
    from paper_2111_08044_gb300.sim import FloquetBatch

    hbm_gbs = _peaks()[0]
    chains = inputs.batch_preset(512)
    periods = 64
    for L in sorted({c.L for c in chains}):
        group = [c for c in chains if c.L == L]
        form = capi.SV_BATCH_RESIDENT if L <= 14 else capi.SV_BATCH_BLOCK_TC
        b = FloquetBatch(group, form=form)
        b.evolve(16)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(b.stream)
        b.evolve(periods)
        end.record(b.stream)
        torch.cuda.synchronize()
        ms = start.elapsed_time(end) / periods
        forms, widths = b.forms(), b.widths()
        b.close()
        del b
        torch.cuda.empty_cache()
        bound = _batch_hbm_bound_ms(group, forms, widths, hbm_gbs)
        print(json.dumps({"batch_breakdown": True, "L": L, "chains": len(group),
                          "form": "resident" if form == capi.SV_BATCH_RESIDENT else "block_tc group",
                          "ms_per_period": ms, "hbm_bound_ms_per_period": bound,
                          "hbm_bound_frac": bound / ms if bound else None}), flush=True)
    return 0


def run_oracle_table(args):
    """The oracle's CPU-baseline table: whole periods at several chain
    lengths, all cores and one thread (one JSON line per entry)."""
    from oracle import oracle as orc
    allc = orc.num_threads()
    plan = [(12, 100, allc), (12, 100, 1), (20, 100, allc), (20, 100, 1), (26, 10, allc),
            (26, 1, 1), (30, 2, allc)]
    for L, periods, th in plan:
        v, dt, used = _oracle_full_periods(L, periods, seed=4, threads=th)
        print(json.dumps({"oracle_table": True, "L": L, "periods": periods, "threads": used,
                          "seconds": dt, "periods_per_s": v,
                          "two_qubit_gates_per_s": v * 4 * (L - 1), "cpu": _cpu_model()}),
              flush=True)
    orc.set_threads(allc)
    return 0


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    from paper_2111_08044_gb300 import capi
    capi.load()
    hbm_peak, bf16_peak, peak_src = _peaks()
    plain_steps = args.plain_steps if args.plain_steps is not None else max(2, args.steps // 3)
    mg_steps = max(2, args.steps // 4)
    clocks = Clocks(local)
    clocks.start()
    block = _time_form(args, "block", args.steps, rank, world, local)
    plain = _time_form(args, "plain", plain_steps, rank, world, local)
    multigate = _time_form(args, "multigate", mg_steps, rank, world, local)
    ck = clocks.stop()
    plain.pop("pass_ms_each", None)  # 116 gate passes: the mean is enough
    t_block = _max_over_ranks(block["elapsed_ms"], world)
    t_plain = _max_over_ranks(plain["elapsed_ms"], world)
    value = world * args.steps / (t_block / 1e3)
    plain_value = world * plain_steps / (t_plain / 1e3)
    e2e = None
    if not args.no_e2e:
        e2e = _e2e(args, args.steps, rank, local)
        e2e["value"] = world * e2e["value"]  # replicas run side by side
    batch = _batch(args, local) if args.batch_periods > 0 else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, used = _oracle_full_periods(args.L, 1, seed=_rank_seed(0))
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"one whole period (gates, kick, energy and norm) of this workload at "
                         f"L={args.L} in FP64 ({dt:.1f} s), no scaling; CPU: {_cpu_model()}"}
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    # plus the relabel launch that begins an evolution whose periods start
    # off site 0 (one per timed call)
    gpl = (block["launches_per_period"] * args.steps + block["entry_launches"]
           + plain["launches_per_period"] * plain_steps
           + multigate["launches_per_period"] * mg_steps)
    achieved = block["pass_gbs"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_block / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (complex64 state; block GEMMs "
        + ("tensor cores on exact bf16 digits, FP32 accumulators" if args.split == "bf16x3" else "FP32") + ", FP64 reductions)",
        "data": "synthetic",
        "config": _config(args, world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": _traffic(args),
                     "kernel": "block pass (one fused unitary + relabel per launch)",
                     "peak_source": peak_src},
        "block": {k: block[k] for k in ("periods_per_s", "passes_per_period",
                                        "gates_per_period", "avg_pass_ms", "pass_gbs",
                                        "pass_share", "energy_last", "pass_ms_each")},
        "plain": dict(plain, periods_per_s=plain_value, steps=plain_steps,
                      roofline_frac=plain["pass_gbs"] / hbm_peak),
        "multigate": dict(multigate, steps=mg_steps,
                          periods_per_s=world * mg_steps / (
                              _max_over_ranks(multigate["elapsed_ms"], world) / 1e3),
                          fp32_tflops=_mg_fp32_tflops(args.L, multigate),
                          fp32_frac_of_pipe=_mg_fp32_tflops(args.L, multigate) / FP32_TFLOPS),
        "two_qubit_gates_per_s": value * block["gates_per_period"] / world * world,
        "gpu_launches": gpl,
        "clocks": ck,
        "batch": batch,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = _parse()
    if args.oracle_table:
        return run_oracle_table(args)
    if args.batch_breakdown:
        return run_batch_breakdown(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
