"""One rank of the two-process gloo test of bench.py's multi-rank logic
(run by tests/test_multirank_cpu.py; not a test module itself).

argv: rank world port outdir.  Writes outdir/r<rank>.json."""
import json
import os
import sys

import numpy as np

rank, world, port, outdir = int(sys.argv[1]), int(sys.argv[2]), sys.argv[3], sys.argv[4]
os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=port, RANK=str(rank),
                  WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

import bench  # noqa: E402
import workloads as wl  # noqa: E402

r, w, local, pg = bench.dist_setup(0)          # gpus = 0: the gloo backend
t_max = bench.max_over_ranks(pg, float(rank + 1) * 0.5, torch.device("cpu"))
bench.barrier(pg)
wk = wl.config1()
B = bench.rank_rhs(wk, rank)
out = {"rank": r, "world": w, "local": local, "t_max": t_max,
       "b_first": [float(v) for v in np.ravel(B)[:4]], "b_shape": list(B.shape),
       "probe_seed": int(bench.rank_probe_seed(wk, rank))}
with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
    json.dump(out, f)
pg.destroy_process_group()
