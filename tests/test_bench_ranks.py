"""bench.py with N > 1 replicas, on the CPU (world size 2, gloo): the whole-job
time is the slowest rank's and the pivots are summed over ranks; under
torchrun the reference arm runs on rank 0 alone and prints one line."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_replica_aggregation_gloo(tmp_path):
    p = _torchrun([os.path.join("tests", "rank_worker.py"), str(tmp_path)], 300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.load(open(tmp_path / f"rank{r}.json")) for r in (0, 1)]
    assert [x["rank"] for x in lines] == [0, 1]
    for x in lines:
        assert x["elapsed"] == 2.0 and x["iters"] == 300


def test_reference_arm_rank0_only():
    p = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"], 600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(x) for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
