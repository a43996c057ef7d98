"""The level-sharded path on the GPU: every rank's pieces (shard.partition)
run as that rank's own Plan, one rank after another on this one GPU, and the
assembled result is compared with the FP64 oracle on the unsharded field.
Ranks share nothing and never wait on one another, so running them in turn
on one device exercises exactly the per-rank code of a multi-GPU run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_1404_5756_gb300 import Options, shard, synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _domains():
    # the regional grid at a few levels (the register kernel's line lengths)
    # and three small ragged domains, one with level-dependent inputs
    w = synth.workload(2, nz=5)
    doms = [dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=w["nz"])]
    fields = [w["x"]]
    extra = synth.ragged_domains(3, scale=0.05, max_levels=6)
    d = extra[1]
    nz = d["nz"] = max(d["nz"], 3)
    d["mask"] = np.stack([np.roll(d["mask"], k, axis=1) for k in range(nz)])
    d["Lx"] = np.stack([d["Lx"] * (1.0 + 0.1 * k) for k in range(nz)]).astype(np.float32)
    d["Ly"] = d["Lx"].copy()
    rng = np.random.default_rng(1404)
    for dd in extra:
        doms.append(dict(mask=dd["mask"], Lx=dd["Lx"], Ly=dd["Ly"], nz=dd["nz"]))
        fields.append(rng.standard_normal((2, dd["nz"]) + np.asarray(dd["mask"]).shape[-2:])
                      .astype(np.float32))
    return doms, fields


@pytest.fixture(scope="module")
def case():
    doms, fields = _domains()
    orc.set_threads(8)
    try:
        ref = {adj: [orc.vh(x.astype(np.float64), d["mask"], np.asarray(d["Lx"], np.float64),
                            np.asarray(d["Ly"], np.float64), adjoint=adj)
                     for d, x in zip(doms, fields)] for adj in (False, True)}
    finally:
        orc.set_threads(1)
    return doms, fields, ref


@pytest.mark.parametrize("world", [1, 2, 3, 5])
@pytest.mark.parametrize("adjoint", [False, True])
def test_sharded_plans_reproduce_the_oracle(case, world, adjoint):
    doms, fields, ref = case
    gathered = []
    for rank in range(world):
        op = shard.RankOperator(doms, rank, world, Options(order=3))
        out = op.apply(op.parts(fields), adjoint=adjoint)
        torch.cuda.synchronize()
        if op.plan is not None:
            assert op.plan.status() == 0
        gathered.append([(p, y.cpu().numpy()) for p, y in out])
        op.close()
    assert sum(len(g) for g in gathered) >= world
    full = shard.assemble(doms, 2, gathered)
    for f, o in zip(full, ref[adjoint]):
        assert f.shape == o.shape
        assert np.abs(f - o).max() <= TOL * np.abs(o).max()


def test_sharding_does_not_change_a_slice(case):
    """A slice's output does not depend on which rank filtered it: the world-1
    and world-3 results agree to FP32 rounding of the same recursion."""
    doms, fields, _ = case
    runs = []
    for world in (1, 3):
        gathered = []
        for rank in range(world):
            op = shard.RankOperator(doms, rank, world, Options(order=1, iters=5))
            gathered.append([(p, y.cpu().numpy()) for p, y in op.apply(op.parts(fields))])
            op.close()
        runs.append(shard.assemble(doms, 2, gathered))
    for a, b in zip(*runs):
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()
