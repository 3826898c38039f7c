"""Multi-rank path on the CPU: two gloo ranks shard the pixels, each inverts its
shard with the oracle, and the gathered result equals one process doing all
pixels (results depend only on pixel ids); the step time is the max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1208_0302_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import genesis_inputs as gi
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = gi.one_line_spec(n_lambda=32)
    npix = 11
    start, count = sharding.strong_range(rank, world, npix)
    truth = gi.draw_truth(npix, seed=3)
    obs = oracle.synth(spec, truth)
    res = oracle.ga_invert(spec, obs[start:start + count], gi.PRIOR_LO, gi.PRIOR_HI,
                           oracle.ga_config(32, 6, seed=1), pixel_id0=start, nthreads=1)
    # gather the (possibly uneven) shards through padded buffers
    pad = torch.zeros((npix, 9), dtype=torch.int32)
    pad[:count] = torch.from_numpy(res["genes"].astype(np.int32))
    bufs = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad)
    got = [bufs[r][:sharding.strong_range(r, world, npix)[1]] for r in range(world)]
    t = sharding.max_over_ranks(1.0 + rank, dist)
    if rank == 0:
        np.save(os.path.join(out_dir, "genes.npy"), torch.cat(got).numpy())
        np.save(os.path.join(out_dir, "tmax.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_ranges_tile_the_map():
    for world in [1, 2, 3, 8]:
        for npix in [0, 1, 7, 65536, 65537]:
            spans = [sharding.strong_range(r, world, npix) for r in range(world)]
            at = 0
            for s, c in spans:
                assert s == at
                at += c
            assert at == npix
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
        assert [sharding.weak_range(r, world, 100)[0] for r in range(world)] == [100 * r for r in range(world)]
    with pytest.raises(ValueError):
        sharding.strong_range(2, 2, 10)


def test_two_gloo_ranks_match_single_process(tmp_path):
    import genesis_inputs as gi
    import oracle
    oracle.build()
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    genes = np.load(tmp_path / "genes.npy")
    spec = gi.one_line_spec(n_lambda=32)
    truth = gi.draw_truth(11, seed=3)
    obs = oracle.synth(spec, truth)
    ref = oracle.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, oracle.ga_config(32, 6, seed=1),
                           pixel_id0=0, nthreads=1)
    assert np.array_equal(genes.astype(np.uint16), ref["genes"])
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.0
