"""Multi-process paths on CPU: two gloo ranks (world size 2, 127.0.0.1).

The decode itself shards with no collective; what is checked here is the host
logic around it: the stream partition (every stream exactly once, same on
every rank, LPT load bound), the FP64 all-reduce of the zone-scale gradients
(the per-rank sums of the oracle's dL/dA_z over each rank's streams add up to
the single-process sum over all streams) and the max-over-ranks timing rule of
the benchmark.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import siggen

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

from paper_2605_01086_gb300.shard import decode_cost, shard_assignment, shard_streams  # noqa: E402

N_STREAMS = 9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _streams():
    wl = siggen.mixed_10000_logu(n=N_STREAMS, lo=40, hi=5000)
    doms = [oracle.trained_domain(d) for d in range(4)]
    rng = np.random.default_rng(5)
    items = []
    for i in range(wl.n_streams):
        d = doms[int(wl.domains[i])]
        S = int(wl.lengths[i])
        x = siggen.signal(int(wl.domains[i]), int(wl.seeds[i]), S)
        _, _, lv = oracle.encode_stream(x, d)
        g = rng.standard_normal(S)
        items.append((int(wl.domains[i]), S, lv, g))
    return wl, doms, items


def _costs(wl, doms, items):
    """Decode cost of every stream from its length and its encoded word count."""
    nw = []
    for i in range(wl.n_streams):
        x = siggen.signal(int(wl.domains[i]), int(wl.seeds[i]), int(wl.lengths[i]))
        nw.append(oracle.encode_stream(x, doms[int(wl.domains[i])])[0].size)
    return decode_cost(wl.lengths, np.array(nw))


def _grad_of(idx, doms, items):
    gA = np.zeros((4, 3), np.float64)
    for i in idx:
        dom, S, lv, g = items[i]
        gA[dom] += oracle.backward_stream(lv, S, doms[dom], g)[1]
    return gA


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2605_01086_gb300.shard import allreduce_scale_grad, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, doms, items = _streams()
        mine = shard_streams(_costs(wl, doms, items), world, rank)
        every = [None] * world
        dist.all_gather_object(every, [int(i) for i in mine])
        g = torch.from_numpy(_grad_of(mine, doms, items))
        allreduce_scale_grad(g)
        t = max_over_ranks(1.0 + rank)
        q.put((rank, every, g.numpy().copy(), t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_partition_and_scale_gradient():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    wl, doms, items = _streams()
    # both ranks saw the same partition; it covers every stream exactly once
    assert res[0][1] == res[1][1]
    flat = sorted(i for part in res[0][1] for i in part)
    assert flat == list(range(wl.n_streams))
    # all-reduced gradient = single-process gradient over all streams
    full = _grad_of(range(wl.n_streams), doms, items)
    for r in res:
        np.testing.assert_allclose(r[2], full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    assert res[0][2].any()
    # max over ranks
    assert res[0][3] == res[1][3] == 2.0


def test_lpt_partition_bounds():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        n = np.floor(np.exp(rng.uniform(np.log(4096), np.log(4194304), 500))).astype(np.int64)
        loads, parts = shard_assignment(n, world)
        assert sorted(np.concatenate(parts).tolist()) == list(range(n.size))
        assert loads.sum() == n.sum()
        # LPT: the largest load exceeds the mean by at most the largest item
        assert loads.max() <= n.sum() / world + n.max()
        assert all(np.array_equal(shard_streams(n, world, r), parts[r]) for r in range(world))


def test_partition_edge_cases():
    loads, parts = shard_assignment([], 2)
    assert loads.tolist() == [0, 0] and all(p.size == 0 for p in parts)
    loads, parts = shard_assignment([5, 5, 5, 5], 2)
    assert loads.tolist() == [10, 10]
    loads, parts = shard_assignment([7], 3)
    assert loads.tolist() == [7, 0, 0]
    with pytest.raises(ValueError):
        shard_assignment([1, -1], 2)
    with pytest.raises(ValueError):
        shard_assignment([1], 0)


def test_decode_cost_is_bytes_moved():
    # 4 bytes per float32 sample written, 9 bytes per SymLen word read (8 + 1)
    np.testing.assert_array_equal(decode_cost([0, 1, 1000], [0, 1, 70]), [0, 13, 4630])
    with pytest.raises(ValueError):
        decode_cost([1, 2], [1])
    # a stream that compresses worse costs more than one of the same length
    c = decode_cost([4096, 4096], [200, 900])
    assert c[1] > c[0]
    # the partition balances bytes, not samples: two equal-length streams with
    # very different word counts and two short ones
    costs = decode_cost([1000, 1000, 10, 10], [10, 400, 1, 1])
    loads, parts = shard_assignment(costs, 2)
    assert sorted(loads.tolist()) == sorted([int(costs[1]), int(costs[0] + costs[2] + costs[3])])
