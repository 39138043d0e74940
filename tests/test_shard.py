"""Chain sharding host logic on world-size-2 gloo ranks (CPU, no GPU): disjoint seeds and
the across-rank observable summary equal to the single-process one."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2510_13866_gb300.shard import OBS_FIELDS, chain_seeds, gather_observables, summarize


def _fake_obs(seed, n):
    rng = np.random.default_rng(seed)
    return [{f: float(rng.normal()) for f in OBS_FIELDS} for _ in range(n)]


def _worker(rank, world, port, n, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = chain_seeds(rank, n)
    res = gather_observables(_fake_obs(100 + rank, n))
    out[rank] = (seeds, res)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_gather_matches_single_process():
    n, world = 5, 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), n, out), nprocs=world, join=True)
    seeds0, res0 = out[0]
    seeds1, res1 = out[1]
    assert set(seeds0).isdisjoint(seeds1) and sorted(seeds0 + seeds1) == list(range(2 * n))
    allv = [[o[f] for f in OBS_FIELDS] for o in _fake_obs(100, n) + _fake_obs(101, n)]
    ref = summarize(allv)
    for f in OBS_FIELDS:
        assert np.allclose(res0[f], ref[f]) and np.allclose(res1[f], ref[f])


def test_single_process_summary():
    obs = _fake_obs(3, 4)
    s = gather_observables(obs)
    v = np.array([[o[f] for f in OBS_FIELDS] for o in obs])
    assert np.isclose(s["density"][0], v[:, 0].mean())
    assert np.isclose(s["ekin"][1], v[:, 3].std(ddof=1) / 2.0)
