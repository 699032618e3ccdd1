"""Sharding over ranks on CPU: two gloo ranks each filter their own frames (or
requests) with the oracle, with no exchange on the data path; gathered on
rank 0 (test only), the shards reproduce the single-process result exactly."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1103_4881_b300 import shard, synth


def test_frame_range_partitions():
    for n in (0, 1, 5, 64, 300):
        for world in (1, 2, 3, 8):
            got = [shard.frame_range(n, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.frame_range(4, 2, 2)


def test_balance_by_bytes_bound():
    rng = np.random.default_rng(7)
    sizes = rng.integers(1, 1000, 500)
    for world in (2, 3, 8):
        owner = shard.balance_by_bytes(sizes, world)
        load = np.bincount(owner, weights=sizes, minlength=world)
        assert load.max() - load.min() <= sizes.max()
        assert load.sum() == sizes.sum()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        # frames: a small batch of the 3/8 K=8 gradient workload
        w = synth.Workload("t", 7, 40, 64, (3, 8), 8, synth.DS_F32, 2000, "gradient")
        a, b = shard.frame_range(w.frames, world, rank)
        mine = oracle.filter_f64(synth.frames(w, range(a, b)), 3, 8, 8) if b > a else None
        # requests: byte-balanced, uint8 RGB 1/2 K=6 and f32 3/8 K=8 on small frames
        reqs = [synth.Request(k, 0.0, 24 + 8 * (k % 3), 32 + 16 * (k % 4), (1, 2) if k % 2 else (3, 8),
                              6 if k % 2 else 8, synth.DS_U8_RGB if k % 2 else synth.DS_F32) for k in range(11)]
        nb = lambda r: r.height * r.width * synth.CHANNELS[r.dtype]
        served = {}
        for r in shard.shard_requests(reqs, world, rank, nb):
            x = synth.request_frame(r)[None]
            f = oracle.filter_u8 if r.dtype == synth.DS_U8_RGB else oracle.filter_f64
            served[r.rid] = f(x, r.ratio[0], r.ratio[1], r.taps)[0]
        got = [None] * world
        dist.gather_object((a, b, mine, served), got if rank == 0 else None, dst=0)
        if rank == 0:
            full = oracle.filter_f64(synth.frames(w), 3, 8, 8)
            parts = [g[2] for g in sorted(got, key=lambda g: g[0]) if g[2] is not None]
            assert np.array_equal(np.concatenate(parts), full)
            allreq = {}
            for g in got:
                assert not set(g[3]) & set(allreq)
                allreq.update(g[3])
            assert sorted(allreq) == list(range(len(reqs)))
            for r in reqs:
                x = synth.request_frame(r)[None]
                f = oracle.filter_u8 if r.dtype == synth.DS_U8_RGB else oracle.filter_f64
                assert np.array_equal(allreq[r.rid], f(x, r.ratio[0], r.ratio[1], r.taps)[0])
        q.put((rank, "ok"))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_requests():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: "ok", 1: "ok"}, res
    assert all(p.exitcode == 0 for p in procs)
