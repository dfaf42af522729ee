"""Host logic of the multi-rank benchmark on CPU, world size 2 over gloo:
every rank draws its own batch (weak scaling, no data exchange), the timings
are reduced by their maximum over ranks, the whole-job rate counts every
rank's units, and the CPU reference line is printed by rank 0 alone."""
import contextlib
import io
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import synthetic_inputs as si
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seeds = bench.shard_seeds(rank)
        z = si.messages(seeds["mul"], 2, 8)
        enc = si.enc_seeds(seeds["mul"], 4)
        # per-rank timings, rank 1 slower in the first two phases
        mine = [10.0 + 5 * rank, 20.0 + 1 * rank, 30.0 - 3 * rank]
        reduced = bench.max_over_ranks(mine, dist)
        dist.barrier()
        rates = bench.job_rates(world, 64, 15, 16, 5, *reduced)
        # the reference arm: only rank 0 may print (and only rank 0 does work)
        buf = io.StringIO()
        rc = None
        if rank != 0:
            os.environ["RANK"] = str(rank)
            with contextlib.redirect_stdout(buf):
                rc = bench.run_reference(argparse_ns(steps=1, warmup=0, gpus=world, form="tensor"))
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"seeds": seeds, "z": z.real.tolist(), "enc": enc, "reduced": reduced, "rates": rates,
                       "ref_rc": rc, "ref_out": buf.getvalue()}, f)
    finally:
        dist.destroy_process_group()


def argparse_ns(**kw):
    import argparse
    return argparse.Namespace(**kw)


def test_two_ranks_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(world)]
    # disjoint inputs: seeds, messages and encryption randomness all differ
    for key in ("mul", "boot", "reboot", "uneven"):
        assert r[0]["seeds"][key] != r[1]["seeds"][key]
    assert not np.allclose(r[0]["z"], r[1]["z"])
    assert not set(r[0]["enc"]) & set(r[1]["enc"])
    # the same maximum on every rank
    assert r[0]["reduced"] == r[1]["reduced"] == [15.0, 21.0, 30.0]
    # whole-job rates: both ranks' units over the slowest rank's time
    want = {"hmult_per_s": 2 * 64 * 5 / 0.015, "rotations_per_s": 2 * 64 * 15 * 5 / 0.021,
            "bootstraps_per_s": 2 * 16 * 5 / 0.030}
    for k, v in want.items():
        assert r[0]["rates"][k] == pytest.approx(v)
        assert r[1]["rates"][k] == pytest.approx(v)
    # a non-zero rank of the reference arm exits 0 without work or output
    assert r[1]["ref_rc"] == 0 and r[1]["ref_out"] == ""


def test_single_rank_rates_and_seeds():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    r1 = bench.job_rates(1, 64, 15, 16, 5, 100.0, 200.0, 300.0)
    r4 = bench.job_rates(4, 64, 15, 16, 5, 100.0, 200.0, 300.0)
    for k in r1:
        assert r4[k] == pytest.approx(4 * r1[k])  # weak scaling at equal time
    seeds = [bench.shard_seeds(k) for k in range(8)]
    for key in seeds[0]:
        assert len({s[key] for s in seeds}) == 8
    # the streams of different kinds never coincide across ranks 0..7
    allv = [v for s in seeds for v in s.values()]
    assert len(set(allv)) == len(allv)
