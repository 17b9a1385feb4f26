"""Multi-rank host logic on CPU (gloo, world size 2): element-range sharding of one batch
reproduces the unsharded oracle result, and the max-over-ranks timing reduction that
bench.py uses returns the slowest rank."""

import os
import socket

import numpy as np
import pytest

from paper_1405_7470_gb300.shard import element_range, shard_u


def test_ranges_partition_exactly():
    for E in (0, 1, 7, 1000, 1 << 21):
        for world in (1, 2, 3, 8):
            rs = [element_range(E, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == E
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        element_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    D, u = synth.operands(1001, 12, 3, np.float32, seed=3)
    res = {}
    for layout in ("elem", "node"):
        uu = synth.to_node_major(u) if layout == "node" else u
        e0, e1 = element_range(1001, world, rank)
        part = oracle.contract(D, shard_u(uu, layout, e0, e1), layout)
        # gather the parts on every rank (test only: the data path itself has no collective)
        flat = torch.from_numpy(np.ascontiguousarray(part).ravel())
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([flat.numel()]))
        bufs = [torch.zeros(int(n.item()), dtype=torch.float64) for n in sizes]
        mx = max(b.numel() for b in bufs)
        padded = torch.zeros(mx, dtype=torch.float64)
        padded[:flat.numel()] = flat
        outs = [torch.zeros(mx, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(outs, padded)
        pieces = []
        for r, o in enumerate(outs):
            a, b = element_range(1001, world, r)
            shp = (3, b - a, 12) if layout == "elem" else (3, 12, b - a)
            pieces.append(o[: int(sizes[r].item())].numpy().reshape(shp))
        full = np.concatenate(pieces, axis=1 if layout == "elem" else 2)
        res[layout] = bool(np.array_equal(full, oracle.contract(D, uu, layout)))
    t = torch.tensor([1.5 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    res["max_time"] = float(t.item())
    dist.destroy_process_group()
    q.put((rank, res))


def test_two_rank_sharding_matches_oracle():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert results[r]["elem"] and results[r]["node"]
        assert results[r]["max_time"] == 2.5
