"""The bench's multi-process path on CPU (gloo, world size 2): rank
discovery from the launcher's environment, the barrier, the max over ranks
that sets the whole-job time, distinct per-rank workloads, and the
reference arm, which only rank 0 runs and prints."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    try:
        os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                          MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        sys.path.insert(0, ROOT)
        import torch.distributed as dist
        import bench
        dist.init_process_group("gloo", rank=rank, world_size=world)
        w, r, local = bench._dist()
        bench._barrier(w)
        m = bench._max_over_ranks(10.0 + 3.0 * r, w)
        out.put((r, w, local, m, bench._rank_seed(r)))
        dist.destroy_process_group()
    except Exception as ex:  # report instead of leaving the parent waiting
        out.put(("error", rank, repr(ex)))


def test_rank_helpers_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    assert all(g[0] != "error" for g in got), got
    got = sorted(got)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    assert all(g[1] == 2 and g[2] == g[0] for g in got)
    # the whole-job time is the slowest rank's on every rank
    assert all(g[3] == 13.0 for g in got)
    # each replica evolves its own chain
    assert got[0][4] != got[1][4]


def test_reference_arm_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--L", "16"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout  # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_groups_make_one_period():
    """The reference arm's steps are the period's operation groups; the
    2K + 2 groups in order do exactly the oracle's whole period."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as orc
    from paper_2111_08044_gb300 import inputs
    L = 10
    psi, groups = bench._oracle_period_groups(L, seed=4)
    cfg = inputs.ChainConfig(L=L, seed=4)
    assert len(groups) == 2 * cfg.K + 2
    ref = orc.product_state(cfg.spinors())
    hdrive, hobs = orc.chain_inputs(cfg)
    for _ in range(2):
        for g in groups:
            g()
        orc.period(ref, orc.bond_gates(hdrive, cfg.tau), orc.kick_gates(L, cfg.theta), cfg.K,
                   cfg.first_layer)
    np.testing.assert_allclose(psi, ref, atol=1e-14, rtol=0)
