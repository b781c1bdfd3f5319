"""The multi-rank host logic of the benchmark on CPU: two gloo ranks on 127.0.0.1.

Each rank of a family of independent functions runs its own part (disjoint seeds, same
size); a single-function workload is a replica on every rank; the job's value is the units
summed over ranks divided by the slowest rank's time.
"""
import os
import socket

import pytest

import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w = W.shard(W.poisson_batched_64(), rank, world)
        ids = sorted(round(float(f["cx"][0]), 12) for f in w.funcs)  # identifies the functions
        rep = W.shard(W.bsh_m60_adaptive_k10(), rank, world)
        n_local = 1000 + 500 * rank
        ms_local = 10.0 + 5.0 * rank
        n_all, ms = bench.reduce_over_ranks(n_local, ms_local, world)
        q.put((rank, len(w.funcs), ids, float(rep.funcs[0]["cx"][0]), n_all, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, n0, s0, rep0, na0, ms0), (_, n1, s1, rep1, na1, ms1) = res[0], res[1]
    assert n0 == n1 == 64                       # same amount of work per rank (weak scaling)
    assert not set(s0) & set(s1)                # different functions on the two ranks
    assert rep0 == rep1                         # single-function workload: a replica per rank
    assert na0 == na1 == 1000 + 1500            # units summed over ranks
    assert ms0 == ms1 == pytest.approx(15.0)    # slowest rank's time


def test_shard_is_identity_for_one_rank():
    w = W.poisson_batched_64()
    assert W.shard(w, 0, 1) is w
    w0 = W.shard(w, 0, 2)
    assert [f["cx"][0] for f in w0.funcs] == [f["cx"][0] for f in w.funcs]  # rank 0 keeps part 0


# ----------------------------------------------------------------- destination partition

def _partition_rank(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1507_01888_gb300 import partition as PT
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys, coeffs = W.random_tree_coeffs(300, 3, 4, seed=5)
        ranges = PT.split_ranges(keys, world)
        lo, hi = ranges[rank]
        own = PT.in_range(keys, lo, hi)
        k_all, c_all = PT.exchange(torch.from_numpy(keys[own].view(np.int64).copy()),
                                   torch.from_numpy(coeffs[own].copy()))
        q.put((rank, k_all.numpy().view(np.uint64).copy(), c_all.numpy().copy(), lo, hi))
    finally:
        dist.destroy_process_group()


def test_partition_exchange_gives_every_rank_the_whole_tree():
    """Three gloo ranks hold disjoint key ranges of a tree; the all-gather gives each the whole
    tree in key order."""
    import numpy as np
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_partition_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    keys, coeffs = W.random_tree_coeffs(300, 3, 4, seed=5)
    for r in range(world):
        assert (res[r][1] == keys).all() and np.array_equal(res[r][2], coeffs)
    # the ranges tile the key space in order
    assert res[0][3] == 0 and res[world - 1][4] == int(np.uint64(0xFFFFFFFFFFFFFFFF))
    for r in range(world - 1):
        assert res[r][4] == res[r + 1][3]


def test_partition_ranges_and_halo_by_brute_force():
    import numpy as np
    from paper_1507_01888_gb300 import partition as PT
    keys, _ = W.random_tree_coeffs(200, 3, 3, seed=7)
    ranges = PT.split_ranges(keys, 4)
    owned = sum(PT.in_range(keys, lo, hi).astype(int) for lo, hi in ranges)
    assert (owned == 1).all()                      # every box owned by exactly one rank
    counts = [int(PT.in_range(keys, lo, hi).sum()) for lo, hi in ranges]
    assert max(counts) - min(counts) <= 1          # balanced by box count
    n, x, y, z = PT._split_key(keys)
    for lo, hi in ranges:
        halo = PT.halo_mask(keys, lo, hi, 1)
        for i in range(len(keys)):                 # brute force: some in-cell neighbour key in range
            nb = 1 << int(n[i])
            want = False
            for lx in (-1, 0, 1):
                for ly in (-1, 0, 1):
                    for lz in (-1, 0, 1):
                        a, b, c = x[i] + lx, y[i] + ly, z[i] + lz
                        if 0 <= a < nb and 0 <= b < nb and 0 <= c < nb:
                            t = (int(n[i]) << 57) | (int(a) << 38) | (int(b) << 19) | int(c)
                            want |= lo <= t < hi
            assert bool(halo[i]) == want


def _lost_rank(rank, world, port, q):
    import datetime
    import time
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1507_01888_gb300 import partition as PT
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    keys, coeffs = W.random_tree_coeffs(100, 2, 3, seed=7)
    lo, hi = PT.split_ranges(keys, world)[rank]
    own = PT.in_range(keys, lo, hi)
    if rank == world - 1:  # this rank leaves between steps, before the exchange, without a word
        q.put((rank, "left", 0.0))
        q.close()
        q.join_thread()  # the message is sent before the process ends
        os._exit(0)
    t0 = time.monotonic()
    try:
        PT.exchange(torch.from_numpy(keys[own].view(np.int64).copy()), torch.from_numpy(coeffs[own].copy()))
        q.put((rank, "completed", time.monotonic() - t0))
    except Exception as e:  # the survivors learn of it on the host: the collective fails
        q.put((rank, type(e).__name__, time.monotonic() - t0))
    q.close()
    q.join_thread()
    os._exit(0)  # no orderly shutdown of a process group that lost a member


def test_exchange_fails_loudly_when_a_rank_is_lost():
    """Failure detection on the host: one of three gloo ranks exits before the halo exchange.
    The others do not hang: their all-gather raises within the process group's timeout."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_lost_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
    assert res[world - 1][1] == "left"
    for r in range(world - 1):
        assert res[r][1] != "completed", res[r]
        assert res[r][2] < 60.0


# ----------------------------------------------------------------- halo-only exchange

def _halo_rank(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1507_01888_gb300 import partition as PT
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys, coeffs = W.random_tree_coeffs(400, 3, 4, seed=9)
        weights = 1.0 + (keys >> np.uint64(57)).astype(float) ** 2  # uneven work per box
        ranges = PT.split_ranges(keys, world, weights)
        plan = PT.HaloPlan(keys, ranges, rank, 1)
        own = torch.from_numpy(coeffs[plan.own].copy())
        got = plan.exchange(own)
        q.put((rank, plan.halo_keys.copy(), got.numpy().copy(), plan.n_received, plan.n_sent, plan.n_halo))
    finally:
        dist.destroy_process_group()


def _run_ranks(target, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_gives_each_rank_exactly_its_halo(world):
    """gloo ranks cut the key space by work; one all-to-all leaves each rank with exactly the
    boxes within |l|_inf <= 1 of its destination range (brute-force halo), in key order, and it
    received only the halo boxes other ranks own (less than the whole tree minus its own part)."""
    import numpy as np
    from paper_1507_01888_gb300 import partition as PT
    res = _run_ranks(_halo_rank, world)
    keys, coeffs = W.random_tree_coeffs(400, 3, 4, seed=9)
    weights = 1.0 + (keys >> np.uint64(57)).astype(float) ** 2
    ranges = PT.split_ranges(keys, world, weights)
    sent = recv = 0
    for r in range(world):
        _, hk, hc, n_recv, n_sent, n_halo = res[r]
        want = PT.halo_mask(keys, *ranges[r], 1)
        assert (hk == keys[want]).all() and np.array_equal(hc, coeffs[want])
        own = PT.in_range(keys, *ranges[r])
        assert n_recv == int((want & ~own).sum()) < len(keys) - int(own.sum())
        sent += n_sent
        recv += n_recv
    assert sent == recv


def test_halo_shrinks_as_ranges_narrow_and_weights_balance_work():
    """Without communication: the largest per-rank halo (and so the bytes a rank receives and
    holds) shrinks as the number of ranks grows, and work-weighted ranges balance the weight
    where box-count ranges do not."""
    import numpy as np
    from paper_1507_01888_gb300 import partition as PT
    keys = np.unique(np.concatenate([W.random_tree_coeffs(150, 3, 3, seed=13)[0],
                                     W.random_tree_coeffs(450, 3, 5, seed=14)[0]]))
    lv = (keys >> np.uint64(57)).astype(int)
    halos = []
    for world in (1, 2, 4):
        ranges = PT.split_ranges(keys, world)
        halos.append(max(PT.HaloPlan(keys, ranges, r, 1).n_halo for r in range(world)))
    assert halos[0] == len(keys) and halos[0] > halos[1] > halos[2]
    w = PT.level_weights(keys, np.bincount(lv, minlength=20), np.bincount(lv, weights=10.0 ** lv, minlength=20))
    by_count = PT.split_ranges(keys, 4)
    by_work = PT.split_ranges(keys, 4, w)
    def spread(ranges):
        loads = [w[PT.in_range(keys, lo, hi)].sum() for lo, hi in ranges]
        return max(loads) / (sum(loads) / len(loads))
    assert spread(by_work) < spread(by_count)
