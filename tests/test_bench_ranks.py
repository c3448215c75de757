"""The replica path of bench.py on two CPU ranks (gloo): barrier, max over ranks, whole-job rate, rank-0 output.

Under torchrun every rank solves its own replica and nothing crosses ranks on the data path; the only
cross-rank traffic is a barrier around the timed region and the max of the ranks' times. These tests run that
host logic as two gloo processes, without a GPU.
"""
import json
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


CHILD = r"""
import json, os, sys, time
sys.path.insert(0, os.environ["BENCH_ROOT"])
import bench
world, rank, local = bench.dist()
ranks = bench.Ranks(world, rank, None)
# rank r "takes" (r + 1) * 10 ms per step for 4 steps: the slowest rank sets the time
ranks.barrier()
t = ranks.max((rank + 1) * 0.040)
rate = bench.whole_job_rate(world, 4, t)
ranks.barrier()
ranks.close()
print(json.dumps({"rank": rank, "max_s": t, "rate": rate}), flush=True)
"""


def _launch(code, world, extra_env=None, args=()):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), LOCAL_RANK=str(r),
                   WORLD_SIZE=str(world), BENCH_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        cmd = [sys.executable, "-c", code, *args] if code else [sys.executable, os.path.join(ROOT, "bench.py"), *args]
        procs.append(subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      cwd=ROOT))
    outs = []
    for pr in procs:
        try:
            o, e = pr.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            pr.kill()
            o, e = pr.communicate()
        outs.append((pr.returncode, o, e))
    return outs


def test_two_rank_max_and_whole_job_rate():
    outs = _launch(CHILD, 2)
    for rc, o, e in outs:
        assert rc == 0, e
    lines = [json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs]
    for ln in lines:
        # both ranks agree on the slowest rank's time, and the rate counts both ranks' steps
        assert ln["max_s"] == pytest.approx(0.080)
        assert ln["rate"] == pytest.approx(2 * 4 / 0.080)


def test_single_rank_needs_no_process_group():
    import bench
    r = bench.Ranks(1, 0, None)
    r.barrier()
    assert r.max(1.25) == 1.25
    r.close()
    assert bench.whole_job_rate(1, 30, 1.5) == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of a two-rank reference run exits 0 without work and prints nothing
    outs = _launch(None, 1, args=("--impl", "reference", "--steps", "1", "--warmup", "0",
                                  "--workload", "ar10_n10k"), extra_env={"RANK": "1", "WORLD_SIZE": "2"})
    for rc, o, e in outs:
        assert rc == 0, e
        assert o.strip() == ""


def test_reference_arm_line_on_rank_zero():
    outs = _launch(None, 1, args=("--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "ar10_n10k"))
    rc, o, e = outs[0]
    assert rc == 0, e
    line = json.loads(o.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
