"""The benchmark's multi-rank path on CPU with gloo, world size 2: process-group set-up, the
barrier and the max-over-ranks reduction of the timing, the per-rank shards of the weak-scaling
workload (no data-path collective), and the reference arm under torchrun (rank 0 alone runs
and prints one line, the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


WORKER = r"""
import hashlib, json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import bench
import torch
import torch.distributed as dist
ws, rank, local = bench.dist_setup()
assert ws == 2 and dist.get_backend() == "gloo"
mech, T, P, Y = bench.make_inputs(rank, n=64)
digest = hashlib.sha256(T.tobytes() + Y.tobytes()).hexdigest()
digests = [None, None]
dist.all_gather_object(digests, digest)
bench.barrier(ws)
mx = bench.max_over_ranks(1.5 + rank, ws, torch.device("cpu"))
out = {"rank": rank, "digests": digests, "max": mx, "shape": list(Y.shape)}
with open(os.path.join(os.environ["OUT_DIR"], f"rank{rank}.json"), "w") as f:
    json.dump(out, f)
dist.destroy_process_group()
"""


def _launch(tmp_path, script_args, extra_env=None, timeout=300):
    env = dict(os.environ)
    env.update({"REPO_ROOT": ROOT, "OUT_DIR": str(tmp_path), "CUDA_VISIBLE_DEVICES": ""})
    if extra_env:
        env.update(extra_env)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}"] + script_args
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_gloo_shards_barrier_and_max(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    r = _launch(tmp_path, [str(script)])
    assert r.returncode == 0, r.stderr[-3000:]
    res = [json.load(open(tmp_path / f"rank{k}.json")) for k in (0, 1)]
    for x in res:
        assert x["max"] == 2.5                    # max over ranks of 1.5 + rank
        assert x["shape"] == [64, 53]
    # every rank evaluates its own cells (different state seeds), none are exchanged
    assert res[0]["digests"] == res[1]["digests"]
    assert res[0]["digests"][0] != res[0]["digests"][1]


def test_reference_arm_under_torchrun(tmp_path):
    r = _launch(tmp_path, ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2",
                           "--warmup", "1", "--ref-seconds", "2"])
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
