"""Level sharding across ranks: the host logic of the multi-GPU path, run as
world_size-2 gloo ranks on the CPU.  Each rank filters its own (domain,
level) pieces with the oracle (the GPU path is the same per slice) and the
pieces are all-gathered; the assembled result must equal the unsharded one
bit for bit, since no recursion crosses a level."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import oracle  # noqa: E402
from paper_1404_5756_gb300 import shard, synth  # noqa: E402


def _domains():
    doms = synth.ragged_domains(3, scale=0.02, max_levels=8)
    # one level-dependent domain: per-level masks and length scales
    d = doms[1]
    nz = d["nz"] = max(d["nz"], 3)
    rng = np.random.default_rng(7)
    d["mask"] = np.stack([np.roll(d["mask"], k, axis=1) for k in range(nz)])
    d["Lx"] = np.stack([d["Lx"] * (1.0 + 0.1 * k) for k in range(nz)]).astype(np.float32)
    d["Ly"] = d["Lx"].copy()
    fields = [rng.standard_normal((2, dd["nz"]) + np.asarray(dd["mask"]).shape[-2:])
              .astype(np.float32) for dd in doms]
    return doms, fields


def _vh(d, x):
    return oracle.vh(x, d["mask"], d["Lx"], d["Ly"])


def test_partition_covers_every_level_once_and_balances():
    doms = [dict(mask=np.ones((n, 2 * n), np.uint8), nz=nz) for n, nz in
            [(10, 7), (3, 40), (25, 1), (8, 13)]]
    plane = {i: 2 * n * n for i, (n, _) in enumerate([(10, 7), (3, 40), (25, 1), (8, 13)])}
    for world in (1, 2, 3, 5, 16):
        parts = shard.partition(doms, world)
        assert len(parts) == world
        seen = {}
        for r, pieces in enumerate(parts):
            for p in pieces:
                for k in range(p.k0, p.k0 + p.nk):
                    assert (p.domain, k) not in seen
                    seen[(p.domain, k)] = r
        assert sorted(seen) == [(i, k) for i, d in enumerate(doms) for k in range(d["nz"])]
        # ranks own consecutive runs of the (domain, level) order
        order = [seen[key] for key in sorted(seen)]
        assert order == sorted(order)
        loads = [sum(p.nk * plane[p.domain] for p in pieces) for pieces in parts]
        assert max(loads) - min(loads) <= 2 * max(plane.values())


def test_sub_domain_cuts_only_level_dependent_inputs():
    m2 = np.ones((4, 5), np.uint8)
    m3 = np.arange(3 * 4 * 5).reshape(3, 4, 5) % 2
    L = np.full((4, 5), 3.0, np.float32)
    s = shard.sub_domain(dict(mask=m3, Lx=L, Ly=L, nz=3), 1, 2)
    assert s["nz"] == 2 and np.array_equal(s["mask"], m3[1:3]) and s["Lx"] is L
    s = shard.sub_domain(dict(mask=m2, Lx=L, Ly=L, nz=3), 2, 1)
    assert s["mask"] is m2 and s["nz"] == 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        doms, fields = _domains()
        subs, parts, pieces = shard.shard(doms, fields, rank, world)
        mine = [(p, _vh(s, x)) for p, s, x in zip(pieces, subs, parts)]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        if rank == 0:
            full = shard.assemble(doms, 2, gathered)
            ok = all(np.array_equal(f, _vh(d, x)) for f, d, x in zip(full, doms, fields))
            q.put(("ok" if ok else "mismatch", sum(len(g) for g in gathered)))
    except Exception as e:  # report to the parent instead of hanging it
        q.put(("error", repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_unsharded_operator():
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank did not finish"
    assert all(p.exitcode == 0 for p in procs)
    status, npieces = q.get(timeout=5)
    assert status == "ok", npieces
    assert npieces >= 3
