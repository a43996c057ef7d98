"""Input validation and memory safety through the C ABI, without any fault
on the GPU: bad length scales at sea points are refused before any launch,
whatever sits at land points (NaN, Inf) is ignored and land output is
exactly 0, and NaN canary bands around every output region are left
untouched by every kernel path (tile kernel with aligned and unaligned
rows, both lane widths, long-line kernel, multi-domain launch, in place,
host-buffer pipeline).  A bounded device-side wait that gives up is reported
as RF_ETIMEOUT and leaves the context usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1404_5756_gb300 import Options, Plan, _lib, synth  # noqa: E402

pytestmark = pytest.mark.gpu
FILTERS = [(3, 1), (1, 5)]
PAD = 4099          # canary floats on each side (not a multiple of 4: odd alignments too)


def case(seed, ny, nx, land=0.25):
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=(ny, nx)) > land).astype(np.uint8)
    L = rng.uniform(1.0, 20.0, (ny, nx)).astype(np.float32)
    return mask, L


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -2.0, 0.0])
def test_bad_length_scale_at_sea_is_refused(bad):
    mask, L = case(1, 20, 30)
    j, i = np.argwhere(mask == 1)[0]
    for which in ("Lx", "Ly"):
        Lx, Ly = L.copy(), L.copy()
        (Lx if which == "Lx" else Ly)[j, i] = bad
        with pytest.raises(_lib.RFError) as e:
            Plan(dict(mask=mask, Lx=Lx, Ly=Ly, nz=1))
        assert e.value.code == _lib.RF_EINVAL
    # at a land point the same value is ignored
    j, i = np.argwhere(mask == 0)[0]
    Lx = L.copy()
    Lx[j, i] = bad
    plan = Plan(dict(mask=mask, Lx=Lx, Ly=L, nz=1))
    assert plan.status() == 0


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("nx", [130, 4200])
def test_land_input_is_ignored(order, K, nx):
    """NaN and Inf at land points change nothing and land output is 0 (tile
    kernel for 130-point rows, long-line kernel for 4200)."""
    mask, L = case(2 + nx, 24, nx)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 2, 24, nx)).astype(np.float32)
    x[:, :, mask == 0] = 0.0
    dirty = x.copy()
    land = np.argwhere(mask == 0)
    dirty[0, 0, land[::2, 0], land[::2, 1]] = np.nan
    dirty[1, 1, land[1::2, 0], land[1::2, 1]] = np.inf
    plan = Plan(dict(mask=mask, Lx=L, Ly=L, nz=2), Options(order=order, iters=K))
    for adjoint in (False, True):
        run = plan.apply_adjoint if adjoint else plan.apply
        clean = run(torch.from_numpy(x).cuda()).cpu().numpy()
        got = run(torch.from_numpy(dirty).cuda()).cpu().numpy()
        assert np.isfinite(got).all()
        assert np.array_equal(got, clean)
        assert np.all(got[:, :, mask == 0] == 0.0)
    assert plan.status() == 0


def canaried(numel, fill=None):
    """A device buffer of PAD + numel + PAD floats, the pads NaN; returns the
    buffer and the middle view."""
    buf = torch.full((PAD + numel + PAD,), float("nan"), device="cuda")
    mid = buf[PAD:PAD + numel]
    if fill is not None:
        mid.copy_(fill.reshape(-1))
    return buf, mid


def pads_intact(buf):
    a = buf[:PAD].cpu().numpy()
    b = buf[-PAD:].cpu().numpy()
    return bool(np.isnan(a).all() and np.isnan(b).all())


@pytest.mark.parametrize("order,K", FILTERS)
@pytest.mark.parametrize("ny,nx", [(384, 1024), (61, 97), (9, 4200), (700, 33)])
def test_output_canaries_untouched(order, K, ny, nx):
    """Aligned rows (1024), unaligned odd sizes (97 x 61, so no 16-byte row
    copies; the field starts 4099 floats into its buffer), long rows on the
    long-line kernel (4200) and long columns with 32 lanes (700)."""
    mask, L = case(ny * nx, ny, nx)
    rng = np.random.default_rng(4)
    x = torch.from_numpy(rng.standard_normal((2, 2, ny, nx)).astype(np.float32)).cuda()
    plan = Plan(dict(mask=mask, Lx=L, Ly=L, nz=2), Options(order=order, iters=K))
    ref_f, ref_a = plan.apply(x), plan.apply_adjoint(x)
    for adjoint, ref in ((False, ref_f), (True, ref_a)):
        ibuf, xin = canaried(x.numel(), x)
        obuf, out = canaried(x.numel())
        run = plan.apply_adjoint if adjoint else plan.apply
        run(xin.view(x.shape), out=out.view(x.shape))
        torch.cuda.synchronize()
        assert pads_intact(ibuf) and pads_intact(obuf)
        assert torch.equal(out.view(x.shape), ref)
        # in place
        run(xin.view(x.shape), out=xin.view(x.shape))
        torch.cuda.synchronize()
        assert pads_intact(ibuf)
        assert torch.equal(xin.view(x.shape), ref)
    assert plan.status() == 0


def test_multi_domain_canaries_between_domains():
    """Ragged domains packed into one buffer, each behind its own NaN band,
    through the multi-domain launch (and after tuning)."""
    doms = synth.ragged_domains(5, scale=0.1, max_levels=6)
    rng = np.random.default_rng(6)
    specs = [dict(mask=d["mask"], Lx=d["Lx"], Ly=d["Ly"], nz=d["nz"]) for d in doms]
    shapes = [(1, d["nz"], d["ny"], d["nx"]) for d in doms]
    sizes = [int(np.prod(s)) for s in shapes]
    total = sum(sizes) + PAD * (len(sizes) + 1)
    buf = torch.full((total,), float("nan"), device="cuda")
    views, offs, o = [], [], PAD
    for s, n in zip(shapes, sizes):
        v = buf[o:o + n].view(s)
        v.copy_(torch.from_numpy(rng.standard_normal(s).astype(np.float32)))
        views.append(v)
        offs.append(o)
        o += n + PAD
    plan = Plan(specs, Options(order=3))
    refs = [Plan(sp, Options(order=3)).apply(v.clone()) for sp, v in zip(specs, views)]

    def bands_ok():
        b = buf.cpu().numpy()
        ok = np.isnan(b[:PAD]).all()
        for off, n in zip(offs, sizes):
            ok = ok and np.isnan(b[off + n:off + n + PAD]).all()
        return bool(ok)

    for tuned in (False, True):
        if tuned:
            plan.tune_batch(1)
        outs = [torch.full_like(v, float("nan")) for v in views]
        plan.apply(views, out=outs)
        torch.cuda.synchronize()
        assert bands_ok()
        for out, ref in zip(outs, refs):
            assert torch.equal(out, ref)
    plan.apply([v.clone() for v in views], out=views)   # in place over the packed buffer
    torch.cuda.synchronize()
    assert bands_ok()
    assert plan.status() == 0


def test_host_pipeline_canaries():
    w = synth.workload(2, nz=6, nvar=2)
    plan = Plan(dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=6))
    x = torch.from_numpy(w["x"])
    ref = plan.apply(x.cuda()).cpu()
    hbuf = torch.full((PAD + x.numel() + PAD,), float("nan")).pin_memory()
    out = hbuf[PAD:PAD + x.numel()].view(x.shape)
    plan.apply_host(x.pin_memory(), out, nvar=2)
    assert np.isnan(hbuf[:PAD].numpy()).all() and np.isnan(hbuf[-PAD:].numpy()).all()
    assert torch.equal(out, ref)


def test_bounded_wait_that_gives_up_reports_timeout():
    """With a wait bound of 0 polls every register-kernel CTA gives up its
    wait on the coefficient copy at once: it records the timeout, lets the
    copy land and returns.  rf_plan_status then reports RF_ETIMEOUT, and the
    context stays usable: a fresh plan computes the same result as before."""
    w = synth.workload(2, nz=2, nvar=2)
    spec = dict(mask=w["mask"], Lx=w["Lx"], Ly=w["Ly"], nz=2)
    x = torch.from_numpy(w["x"]).cuda()
    ref = Plan(spec).apply(x)
    torch.cuda.synchronize()
    plan = Plan(spec)
    plan.set_wait_limit(0)
    plan.apply(x)
    torch.cuda.synchronize()
    assert plan.status() == _lib.RF_ETIMEOUT
    with pytest.raises(_lib.RFError):
        plan.set_wait_limit(-1)
    again = Plan(spec).apply(x)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)
