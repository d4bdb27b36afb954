"""Multi-process logic of bench.py on CPU (gloo, world size 2): every rank
gets its own shard of parameter vectors, the reported time is the slowest
rank's, and the job throughput counts the units of all ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from paper_2602_19687_gb300 import synth  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.workload("batched_trans", batch=4, seed=bench.shard_seed(rank), n_nu=200)
        ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, world, "cpu")
        out[rank] = (w.theta.copy(), ms_max, bench.job_throughput(4, world, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    (th0, ms0, v0), (th1, ms1, v1) = res[0], res[1]
    assert not np.allclose(th0, th1)                 # distinct shards
    assert ms0 == ms1 == 15.0                        # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 4 / 15e-3)  # units of both ranks / that time


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(1024, 1, 80.0) == pytest.approx(12800.0)


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host and prints
    one JSON line with the contract's keys (its own cpu_baseline and an e2e
    object without host-device bytes)."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"), "--impl",
                        "reference", "--steps", "1", "--warmup", "0", "--workload", "tiny"], capture_output=True,
                       text=True, timeout=600, check=True)
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == bench.host_cores()
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_pooled_oracle_gradient_equals_the_serial_one():
    """The oracle legs split a vector's forward + gradient into one pool task
    per gradient slot; reassembled, it is the oracle's own serial gradient,
    and the error report of identical outputs is zero."""
    from oracle import exoskry_oracle as O
    from paper_2602_19687_gb300 import synth
    key = ("tiny", 3, 42)
    w = synth.workload("tiny", batch=3, seed=42)
    vec = bench.valid_vectors(w, 2)
    nfree = w.theta.shape[1]
    pool, cores = bench.oracle_pool(2)
    try:
        out, wall = bench.oracle_gradients(pool, key, vec, nfree)
    finally:
        pool.close()
        pool.join()
    assert cores == 2 and wall > 0
    mem = O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)
    for b in vec:
        th = w.model.full_theta(w.theta[b])[0]
        k = int(w.kind[b])
        g = O.loglike_gradient(w.model, w.tables, th, k, mem, w.y_obs[k], w.sigma[k], list(w.model.free_idx))
        assert np.array_equal(out[b]["grad"], g)
        assert out[b]["lnl"] == O.loglike(w.model, w.tables, th, k, mem, w.y_obs[k], w.sigma[k])
    gpu = {f: {b: out[b][f] for b in vec} for f in ("spec", "binned", "lnl", "grad")}
    e = bench.bf16_error(gpu, out)
    assert e["vectors"] == len(vec) and e["native"]["max"] == 0 and e["grad"]["max"] == 0
    assert e["lnl_abs"]["max"] == 0
