"""The multi-rank path of bench.py on the host: two gloo ranks (world size 2)
reduce their timings to the whole-job value the way an N-GPU run does (replicas:
the solves of all ranks over the slowest rank's time, zero unless every rank
converged).  No GPU."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir, converged):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench._dist()
    bench._barrier(w)
    value, ms_max = bench._weak_value(w, 3, 1000.0 * (r + 1), converged[r])
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "value": value, "ms_max": ms_max}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("converged", [(True, True), (True, False)])
def test_two_gloo_ranks_reduce_to_the_whole_job_value(tmp_path, converged):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path), converged), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for d in res:
        assert d["world"] == 2 and d["ms_max"] == 2000.0        # the slowest rank
        assert d["value"] == (3 * 2 / 2.0 if all(converged) else 0.0)
