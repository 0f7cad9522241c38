"""The N > 1 path on CPU: two ranks over gloo run the replica host logic the bench uses
(per-rank seeds, a barrier, the maximum of the timed region over ranks, the whole-job
rate). The kernels themselves need a GPU; the data path has no collective, so this is
all the multi-process logic there is."""
import importlib.util
import json
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load():
    spec = importlib.util.spec_from_file_location(
        "mpgpu_replicas", os.path.join(ROOT, "paper_2410_18129_gb300", "replicas.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["mpgpu_replicas"] = mod
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import seeded_inputs as si
    reps = _load()
    info = reps.rank_info()
    reps.init(info, backend="gloo")
    b = si.make_batch(reps.rank_seed(0, info.rank), "batch_2048", 16, 256)
    reps.barrier(info)
    ms = 10.0 + 5.0 * info.rank          # this rank's "timed region"
    ms_max = reps.max_over_ranks(info, ms)
    rate = reps.job_rate(info, 16, ms_max)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"rank": info.rank, "world": info.world, "ms_max": ms_max, "rate": rate,
                   "N0": [int(x) for x in b.N[0]]}, f)
    dist.destroy_process_group()


def test_two_rank_replicas_over_gloo(tmp_path):
    world, port = 2, _free_port()
    tmp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [r["rank"] for r in res] == [0, 1] and all(r["world"] == 2 for r in res)
    assert all(r["ms_max"] == 15.0 for r in res)                 # the slowest rank's time, on every rank
    assert all(abs(r["rate"] - 2 * 16 / 0.015) < 1e-6 for r in res)
    assert res[0]["N0"] != res[1]["N0"]                          # disjoint synthetic inputs per replica


def test_single_process_defaults():
    reps = _load()
    info = reps.rank_info({})
    assert (info.world, info.rank, info.local) == (1, 0, 0)
    reps.init(info)                                             # no process group for one rank
    assert reps.max_over_ranks(info, 3.5) == 3.5
    assert reps.job_rate(info, 1000, 500.0) == 2000.0
    assert reps.rank_seed(7, 3) == 10
    assert np.isclose(reps.job_rate(reps.RankInfo(4, 0, 0), 1000, 500.0), 8000.0)
