"""The bench's multi-process plumbing on CPU ranks (gloo, world size 2, 127.0.0.1): the path does
not shard (every rank compresses its own replica), so what runs across ranks is the rendezvous,
the max-over-ranks timing and the barrier; the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    w, r, local = bench.dist_setup()
    got = bench.barrier_max(w, 1.5 + rank)         # each rank's time; every rank sees the max
    bench.barrier(w)
    # the reference arm returns at once on ranks other than 0 (no oracle work)
    args = argparse.Namespace(ref_steps=1, warmup=0, steps=0, gpus=world)
    if rank != 0:
        bench.run_reference(args, w, r)
    import torch.distributed as dist
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{w} {r} {local} {got}\n")


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch.distributed")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in (0, 1):
        w, r, local, got = open(tmp_path / f"rank{rank}.txt").read().split()
        assert (int(w), int(r), int(local)) == (2, rank, rank)
        assert float(got) == 2.5
