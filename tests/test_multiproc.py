"""The bench's N > 1 path on CPU: two ranks over gloo (127.0.0.1).  Replicas share no
data; what the ranks do together is the barrier, the max-over-ranks time, disjoint
seeded query streams per rank, and the reference arm running on rank 0 only."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)

    class Args:
        impl = "ours"
    r, w, local = bench.dist_setup(Args())
    assert (r, w, local) == (rank, world, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    slowest = bench.max_over_ranks(10.0 * (rank + 1), w)
    ids = [q["id"] for q in bench.batch_queries(7, 0, rank)]
    everyone = [None] * w
    dist.all_gather_object(everyone, ids)

    class RefArgs:
        pass
    ref = bench.run_reference(RefArgs(), rank, w) if rank != 0 else "skipped on rank 0"
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "ids": everyone, "ref": ref}, f)


def test_two_ranks_over_gloo(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["slowest"] == 20.0                      # max over ranks, same on each rank
        a, b = r["ids"]
        assert len(a) == len(b) and not set(a) & set(b)  # replicas draw disjoint queries
    assert res[1]["ref"] is None                         # reference arm: rank 0 alone runs
