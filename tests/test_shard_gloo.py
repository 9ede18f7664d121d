"""Multi-rank host logic on CPU (gloo, world size 2): shell sharding and the single all-reduce that assembles a
spectrum reproduce the single-process result exactly (the per-shell work is computed by the oracle here)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2605_27231_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    from oracle import decomposition, sigw, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, L = 8, 1.0
    Phi, _ = synth.phi_tilde(N, L, 1e-2, 0.5, 2 * 2 * np.pi, seed=5, kind="local", F_NL=2.0)
    dec = decomposition.build()

    def compute(my):
        r = sigw.omega(Phi, L, dec, shells=my)
        return {k: r[k] for k in ("omega", "PA", "PB", "Nk")}

    full = shard.spectrum_by_shells(compute, [1, 2, 3, 4], rank, world)
    np.save(os.path.join(out_dir, "rank%d.npy" % rank), full.numpy())
    dist.destroy_process_group()


def test_partition_is_disjoint_and_complete():
    items = list(range(1, 65))
    parts = [shard.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert all(set(a).isdisjoint(b) for i, a in enumerate(parts) for b in parts[i + 1:])
    s0, s1 = shard.seeds_for_rank([1, 2, 3, 4], 0, 2), shard.seeds_for_rank([1, 2, 3, 4], 1, 2)
    assert set(s0).isdisjoint(s1)
    with pytest.raises(ValueError):
        shard.shard(items, 2, 2)


def test_shell_sharding_over_two_gloo_ranks(tmp_path):
    from oracle import decomposition, sigw, synth
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    N, L = 8, 1.0
    Phi, _ = synth.phi_tilde(N, L, 1e-2, 0.5, 2 * 2 * np.pi, seed=5, kind="local", F_NL=2.0)
    ref = sigw.omega(Phi, L, decomposition.build(), shells=[1, 2, 3, 4])
    for r in range(world):
        got = np.load(tmp_path / ("rank%d.npy" % r))
        np.testing.assert_array_equal(got[:, 0], ref["omega"])
        np.testing.assert_array_equal(got[:, 3], ref["Nk"])
