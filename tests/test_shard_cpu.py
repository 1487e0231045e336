"""Multi-rank path on CPU: world_size-2 gloo ranks shard independent instances
(no data-path collective), each runs its shard with the oracle, and the union
equals the single-process result; the timed region is max-reduced."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1408_5853_gb300 import shard


def test_balanced_shards_cover_everything_once():
    sizes = [64 * 256, 512 * 2048, 100 * 300, 512 * 2048, 70 * 400, 64 * 256, 300 * 900]
    for world in (1, 2, 3, 4):
        parts = shard.balanced_shards(sizes, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import oracle
    from paper_1408_5853_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfgs = inputs.batched_cases(seed=1, n=6)
    for c in cfgs:
        c.update(nr=min(c["nr"], 24), nz=min(c["nz"], 20))
        c["dt"] = 0.5 * oracle.tau_stab(c, 20.0, 100.0)
    mine = shard.balanced_shards([c["nr"] * c["nz"] for c in cfgs], world)[rank]
    for k in mine:
        T, _, _ = oracle.step_n(cfgs[k], inputs.initial_field(cfgs[k], "smooth", seed=k), 5,
                                0.0, cfgs[k]["dt"])
        np.save(os.path.join(out_dir, f"inst{k}.npy"), T)
    t = shard.max_over_ranks(float(rank + 1))
    np.save(os.path.join(out_dir, f"max{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_instances(tmp_path):
    from oracle import oracle
    from paper_1408_5853_gb300 import inputs
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    cfgs = inputs.batched_cases(seed=1, n=6)
    for k, c in enumerate(cfgs):
        c.update(nr=min(c["nr"], 24), nz=min(c["nz"], 20))
        c["dt"] = 0.5 * oracle.tau_stab(c, 20.0, 100.0)
        ref, _, _ = oracle.step_n(c, inputs.initial_field(c, "smooth", seed=k), 5, 0.0, c["dt"])
        got = np.load(tmp_path / f"inst{k}.npy")
        assert np.array_equal(got, ref), k
    for r in range(world):
        assert np.load(tmp_path / f"max{r}.npy")[0] == float(world)
