"""The N > 1 host path of the bench, on CPU with gloo ranks (world size 2).

The path runs replicas: every rank runs the whole workload, and no
collective touches the data path.  The only exchange is the timing
reduction: the job's time is the slowest rank's, and the job's rate is the
pairs of all ranks over that time.  These tests run two gloo ranks on
127.0.0.1 and check that reduction, the rate, that replicas of the oracle
agree bit for bit, and that the reference arm's other ranks exit at once.
The reference arm (the oracle on host cores) also runs here in full and
must print the bench's one JSON line with its contract keys."""
import hashlib
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(__file__))

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    return dist


def _rank_timing(rank, port, q):
    import bench
    dist = _init(rank, port)
    per_rank_seconds = [1.25, 3.5][rank]
    t = bench.max_over_ranks(per_rank_seconds, dist, "cpu")
    rate = bench.job_rate(WORLD, 1000, 4, t)
    dist.barrier()
    q.put((rank, t, rate))
    dist.destroy_process_group()


def _rank_replica(rank, port, q):
    import oracle
    import synth
    import torch
    dist = _init(rank, port)
    img, mask = synth.make(1)
    kw = {k: v for k, v in synth.WORKLOADS[1].params.items() if k != "precision"}
    r = oracle.run(img, mask, **kw)
    h = hashlib.sha256(r.log.tobytes() + r.levels[-1].labels.tobytes()).digest()
    mine = torch.tensor(list(h), dtype=torch.uint8)
    got = [torch.zeros(32, dtype=torch.uint8) for _ in range(WORLD)]
    dist.all_gather(got, mine)
    q.put((rank, [bytes(g.tolist()) for g in got], int(r.stats["pairs"])))
    dist.destroy_process_group()


def _guarded(fn, rank, port, q):
    try:
        fn(rank, port, q)
    except BaseException:
        import traceback
        q.put((rank, "error", traceback.format_exc()))
        raise


def _spawn(fn):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_guarded, args=(fn, r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(WORLD)]
    for p in procs:
        p.join(timeout=60)
    errors = [o[2] for o in out if o[1] == "error"]
    assert not errors, errors[0]
    assert all(p.exitcode == 0 for p in procs)
    return sorted(out)


def test_time_is_max_over_ranks_and_rate_counts_all_ranks():
    out = _spawn(_rank_timing)
    for rank, t, rate in out:
        assert t == 3.5                               # the slowest rank's time on every rank
        assert rate == pytest.approx(WORLD * 1000 * 4 / 3.5)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.job_rate(1, 10, 3, 2.0) == 15.0


def test_replicas_agree_bit_for_bit(orc):
    out = _spawn(_rank_replica)
    (_, h0, p0), (_, h1, p1) = out
    assert h0[0] == h0[1] and h0 == h1
    assert p0 == p1 > 0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       env={k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
