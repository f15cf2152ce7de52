"""The multi-rank path of bench.py on CPU: two processes joined by the gloo
backend (127.0.0.1), as torchrun launches the ranks on a multi-GPU node.

Each rank is a replica with its own right-hand sides and SLQ probes; the only
collective is the MAX of the timings (and a barrier), so the test checks that
the reduction returns the largest rank's value on every rank, that rank 0 keeps
the workload's own inputs, and that the other rank's inputs are an independent
block of the same shape."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
WORKER = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_multirank_worker.py")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gloo_timing_and_inputs(tmp_path):
    port = str(_free_port())
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    procs = [subprocess.Popen([sys.executable, WORKER, str(r), "2", port, str(tmp_path)], env=env,
                              stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for r in range(2)]
    for p in procs:
        try:
            out, _ = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("a rank did not finish")
        assert p.returncode == 0, out[-2000:]
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == 2 for x in res)
    # MAX over ranks: 0.5 and 1.0 -> 1.0 on both ranks
    assert res[0]["t_max"] == res[1]["t_max"] == 1.0
    wk = wl.config1()
    assert res[0]["b_first"] == [float(v) for v in np.ravel(wk.B)[:4]]
    assert res[1]["b_shape"] == list(wk.B.shape)
    assert res[1]["b_first"] != res[0]["b_first"]
    assert res[0]["probe_seed"] != res[1]["probe_seed"]
