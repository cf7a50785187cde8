"""The camera-sharded form of the path, on two CPU ranks (gloo).

The array shards by camera: each rank converts its cameras and measures their
band statistics; the only exchange is an all-gather of those statistics
(KB), after which every rank solves the tiny per-chain systems redundantly.
This test runs that exchange with torch.distributed on two gloo ranks and
checks that the sharded estimate equals the unsharded one exactly.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1910_03517_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import core
    wl = synth.tower12(frames=1)
    wl.cams = [synth.Camera(512, 288, position=i) for i in range(6)]
    wl.glare_cams = (2,)
    K = len(wl.cams)
    mine = [k for k in range(K) if k % world == rank]
    fr = synth.frame_set(wl, 0)
    p = core.Params(num_blocks=4)
    n = np.zeros((K, 2, 4, 3), np.int64)
    s = np.zeros((K, 2, 4, 3), np.int64)
    for k in mine:
        rgb, luma = core.convert(wl.cams[k], {a: b.numpy() for a, b in fr[k].items()})
        st = core.strip_stats(rgb, luma, None, p.strip_width, p.num_blocks, p.motion_threshold)
        n[k] = st["n"]
        s[k] = st["sum"]
    # the exchange: all-gather of every rank's statistics (zero elsewhere)
    parts_n = [torch.zeros_like(torch.from_numpy(n)) for _ in range(world)]
    parts_s = [torch.zeros_like(torch.from_numpy(s)) for _ in range(world)]
    dist.all_gather(parts_n, torch.from_numpy(n))
    dist.all_gather(parts_s, torch.from_numpy(s))
    n_all = sum(t.numpy() for t in parts_n)
    s_all = sum(t.numpy() for t in parts_s)
    maps = core.fit_global(wl.cams, n_all.astype(np.uint32), s_all.astype(np.uint64), p)
    np.save(out_path % rank, maps)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_statistics_give_the_unsharded_fit(tmp_path, orc):
    world = 2
    out = str(tmp_path / "maps_%d.npy")
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    wl = synth.tower12(frames=1)
    wl.cams = [synth.Camera(512, 288, position=i) for i in range(6)]
    wl.glare_cams = (2,)
    fr = synth.frame_set(wl, 0)
    ref = orc.ArrayOracle(wl.cams, orc.Params(num_blocks=4)).step(
        [{a: b.numpy() for a, b in f.items()} for f in fr], want_frame_stats=False)["maps_new"]
    for r in range(world):
        got = np.load(out % r)
        assert np.array_equal(got, ref)
