"""Multi-rank path on CPU: two gloo ranks, each solving its share of the
(partial wave, energy) pairs with the oracle, reproduce the single-process
collision strengths -- for the interleaved energy shards (gather), for the
paper's twisted assignment (reduce), and for energy shards with the
outer-region propagation (every energy propagates on its own, so the same
shards hold)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import propagate  # noqa: E402
from paper_1909_07321_gb300 import partition, synth  # noqa: E402

R1 = 22.0


def _coupling(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, 0.3, (2, n, n))
    return 0.5 * (A + A.transpose(0, 2, 1))


def _solve(pw, E, p, prop):
    if prop:
        return propagate.solve_energies(pw, E, _coupling(4, 70 + p), R1)["omega"]
    return oracle.solve_energies(pw, E)["omega"]


def _pws():
    a = synth.random_pw(41, 4, 50, z=1.0, a=18.0)
    b = synth.random_pw(42, 4, 50, z=1.0, a=18.0)
    b["e_thr"] = a["e_thr"].copy()
    b["g"] = 2.5
    c = synth.random_pw(43, 4, 50, z=1.0, a=18.0)
    c["e_thr"] = a["e_thr"].copy()
    c["g"] = 0.5
    return [a, b, c], synth.midpoint_grid(0.02, 2.0, 37)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pws, E = _pws()
    n_tri = pws[0]["n_levels"] * (pws[0]["n_levels"] + 1) // 2
    if mode in ("gather", "gather_propagated"):
        idx = partition.energy_shard(E.size, rank, world)
        local = np.zeros((idx.size, n_tri))
        for p in partition.pw_order(len(pws), rank, world):
            local += _solve(pws[p], E[idx], p, mode == "gather_propagated")
        full = partition.gather_omega(local, E.size, rank, world)
    else:
        part = np.zeros((E.size, n_tri))
        for p in partition.pw_order(len(pws), rank, world):
            idx = partition.twisted_shard(E.size, p, rank, world)
            part[idx] += oracle.solve_energies(pws[p], E[idx])["omega"]
        full = partition.reduce_omega(part)
    if rank == 0:
        np.save(out_path, full)
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["gather", "twisted", "gather_propagated"])
def test_two_ranks_reproduce_single_process(tmp_path, mode):
    import torch.multiprocessing as mp
    out = str(tmp_path / "omega.npy")
    mp.start_processes(_worker, args=(2, _free_port(), mode, out), nprocs=2, join=True,
                       start_method="spawn")
    full = np.load(out)
    pws, E = _pws()
    ref = sum(_solve(pw, E, p, mode == "gather_propagated") for p, pw in enumerate(pws))
    np.testing.assert_allclose(full, ref, rtol=1e-13, atol=1e-300)


def test_shards_cover_each_pair_once():
    for world in (1, 2, 3, 8):
        for n_E in (1, 7, 64):
            got = np.concatenate([partition.energy_shard(n_E, r, world) for r in range(world)])
            assert np.array_equal(np.sort(got), np.arange(n_E))
            for pw in range(5):
                got = np.concatenate([partition.twisted_shard(n_E, pw, r, world) for r in range(world)])
                assert np.array_equal(np.sort(got), np.arange(n_E))
                # a rank never takes two consecutive energies of one partial wave
                for r in range(world):
                    s = partition.twisted_shard(n_E, pw, r, world)
                    if world > 1:
                        assert np.all(np.diff(s) == world)
        orders = [partition.pw_order(5, r, world) for r in range(world)]
        assert all(sorted(o) == list(range(5)) for o in orders)
