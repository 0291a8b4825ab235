"""Batches of uneven boxes: the captured CUDA graph and the eager per-box launches give
the same products (bitwise), equal to each box's own se_mobility_apply to FP32 rounding,
and graph replays stay correct."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1506_08481_b300 import api, inputs, params  # noqa: E402


def test_batch_graph_matches_per_box_products(oracle_mod):
    boxes = inputs.batch_boxes(seed=3, nbox=6, nmin=40, nmax=300)
    ctxs, xs, refs = [], [], []
    rng = np.random.default_rng(0)
    for cfg in boxes:
        sp = params.choose(cfg.L, cfg.N, 1e-6, M_max=64, a_eff=params.effective_radius(cfg.rad), precision=0)
        c = api.Context()
        c.set_params(sp.xi, sp.M, sp.P, sp.rc)
        c.set_option(api.SE_OPT_SHAPE_M, sp.m)
        c.set_config(cfg.pos, cfg.rad, cfg.L)
        x = torch.tensor(rng.standard_normal((cfg.N, 3)), device="cuda", dtype=torch.float32)
        refs.append(c.apply(x).clone())
        ctxs.append(c)
        xs.append(x)
    torch.cuda.synchronize()
    ys = [torch.empty_like(x) for x in xs]
    b = api.Batch(ctxs, nstreams=4)
    first = None
    for use_graph in (False, True, True):           # eager, capture + launch, replay
        for y in ys:
            y.fill_(float("nan"))
        b.apply(xs, ys, use_graph=use_graph)
        torch.cuda.synchronize()
        # a box alone may split its spreading tiles over CTAs (small grids) and so sum in
        # another order than inside a batch: equal to FP32 rounding; the batch's own
        # eager and graph launches are bitwise equal
        for y, r in zip(ys, refs):
            assert float(torch.linalg.norm(y - r) / torch.linalg.norm(r)) <= 1e-6
        if first is None:
            first = [y.clone() for y in ys]
        else:
            for y, f in zip(ys, first):
                assert torch.equal(y, f)
    # new inputs in the same buffers: the replayed graph reads them
    for x in xs:
        x.mul_(-2.0)
    b.apply(xs, ys, use_graph=True)
    torch.cuda.synchronize()
    for y, r in zip(ys, refs):
        assert torch.allclose(y, -2.0 * r, rtol=1e-5, atol=1e-7)
    # the forces-only product of one box against the FP64 oracle
    cfg = boxes[0]
    xx = np.zeros((cfg.N, 12))
    xx[:, :3] = xs[0].double().cpu().numpy()
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, xx, tol=1e-12)[:, :3]
    got = ys[0].double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    b.close()


@pytest.mark.parametrize("ncomp,dtype", [(3, torch.float32), (12, torch.float64), (11, torch.float32)])
def test_persistent_batch_matches_per_box_launches(ncomp, dtype):
    """One persistent launch for every box (se_batch_apply mode 2) against the batch's
    per-box launches: the same stage code on the same data, so the same products (to
    FP32 rounding), on replays and with new inputs in the same buffers.  The boxes mix
    8^3 and 8x8x16 spreading tiles (a 24^3 grid with P = 12 leaves no room for the
    taller tiles), the real-space and the hybrid size modes, uneven N, and a monodisperse box
    (its pair table stores 13 of the 19 coefficients)."""
    boxes = inputs.batch_boxes(seed=5, nbox=7, nmin=40, nmax=400)
    rad = np.ones(300)
    L = inputs.box_side(rad, 0.2)
    boxes[2] = inputs.Config("mono_n300", L, inputs.positions_rsa(rad, L, np.random.default_rng(8)), rad)
    ctxs, xs = [], []
    rng = np.random.default_rng(2)
    for k, cfg in enumerate(boxes):
        sp = params.choose(cfg.L, cfg.N, 1e-6, M_max=64, a_eff=params.effective_radius(cfg.rad), precision=0)
        c = api.Context()
        if k == 0:
            c.set_params(sp.xi, 24, 12, min(sp.rc, 0.45 * cfg.L))
        else:
            c.set_params(sp.xi, sp.M, sp.P, sp.rc)
            c.set_option(api.SE_OPT_SHAPE_M, sp.m)
        c.set_option(api.SE_OPT_SIZE_MODE, 0 if k == 1 else 1)
        c.set_config(cfg.pos, cfg.rad, cfg.L)
        xs.append(torch.tensor(rng.standard_normal((cfg.N, ncomp)), device="cuda", dtype=dtype))
        ctxs.append(c)
    ref = [torch.empty_like(x) for x in xs]
    ys = [torch.empty_like(x) for x in xs]
    b = api.Batch(ctxs, nstreams=4)
    b.apply(xs, ref, use_graph=0)
    torch.cuda.synchronize()

    def close(a, r):
        return float(torch.linalg.norm((a - r).double()) / torch.linalg.norm(r.double())) <= 1e-6

    for rep in range(3):                  # prepare (eager step), then two persistent launches
        for y in ys:
            y.fill_(float("nan"))
        b.apply(xs, ys, use_graph=api.Batch.PERSISTENT)
        b.status()
        for y, r in zip(ys, ref):
            assert torch.isfinite(y).all() and close(y, r), rep
    for x in xs:
        x.mul_(-2.0)
    b.apply(xs, ys, use_graph=api.Batch.PERSISTENT)
    b.status()
    for y, r in zip(ys, ref):
        assert close(y, -2.0 * r)
    b.close()


def test_batch_with_largest_box_vs_oracle(oracle_mod):
    """Boxes of the 64-box workload's kind (bidisperse radii 1 and 1.5 at equal numbers,
    forces only, FP32, parameters the chooser picks on a grid of at most 128^3 as in the
    benchmark: method tolerance 2.5e-7, FP32 floor 1e-6), one of them at the workload's largest size N = 8000 and
    phi = 0.45: the graph and the persistent launch against the FP64 oracle on 256 sampled
    rows of every box, <= 1e-6 in relative 2-norm."""
    rng = np.random.default_rng(40)
    boxes = []
    for n, phi in ((8000, 0.45), (1500, 0.1), (600, 0.3)):
        rad = inputs.radii_bidisperse(n, 1.0, 1.5, 0.5, rng)
        L = inputs.box_side(rad, phi)
        boxes.append(inputs.Config(f"n{n}", L, inputs.positions_dense(rad, L, rng, sweeps=4), rad))
    ctxs, xs = [], []
    for cfg in boxes:
        sp = params.choose(cfg.L, cfg.N, 2.5e-7, M_max=128, a_eff=params.effective_radius(cfg.rad), precision=0,
                           fp32_tol=1e-6)
        c = api.Context()
        c.set_params(sp.xi, sp.M, sp.P, sp.rc)
        c.set_option(api.SE_OPT_SHAPE_M, sp.m)
        c.set_option(api.SE_OPT_SIZE_MODE, 1)
        c.set_config(cfg.pos, cfg.rad, cfg.L)
        ctxs.append(c)
        xs.append(torch.tensor(rng.standard_normal((cfg.N, 3)), device="cuda", dtype=torch.float32))
    refs = []
    for cfg, x in zip(boxes, xs):
        rows = np.sort(rng.choice(cfg.N, 256, replace=False))
        xx = np.zeros((cfg.N, 12))
        xx[:, :3] = x.double().cpu().numpy()
        refs.append((rows, oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, xx, rows=rows, tol=1e-11)[:, :3]))
    ys = [torch.empty_like(x) for x in xs]
    b = api.Batch(ctxs, nstreams=4)
    for mode in (True, True, api.Batch.PERSISTENT, api.Batch.PERSISTENT):
        for y in ys:
            y.fill_(float("nan"))
        b.apply(xs, ys, use_graph=mode)
        b.status()
        for cfg, y, (rows, ref) in zip(boxes, ys, refs):
            e = np.linalg.norm(y.double().cpu().numpy()[rows] - ref) / np.linalg.norm(ref)
            print(f"{cfg.name} mode {int(mode)}: {e:.2e}")
            assert e <= 1e-6, (cfg.name, mode)
    b.close()


def test_persistent_batch_bounded_wait_runs_out():
    """Failure detection without a GPU fault: the injected stall keeps one box's first
    phases from ever counting as finished, so the CTAs that wait for them give up after
    the (shortened) wait limit; the launch returns, se_batch_status reports the failure,
    and once the hook is off the same batch computes the right products again."""
    boxes = inputs.batch_boxes(seed=9, nbox=4, nmin=60, nmax=300)
    ctxs, xs = [], []
    rng = np.random.default_rng(3)
    for cfg in boxes:
        sp = params.choose(cfg.L, cfg.N, 1e-6, M_max=64, a_eff=params.effective_radius(cfg.rad), precision=0)
        c = api.Context()
        c.set_params(sp.xi, sp.M, sp.P, sp.rc)
        c.set_option(api.SE_OPT_SHAPE_M, sp.m)
        c.set_option(api.SE_OPT_SIZE_MODE, 1)
        c.set_config(cfg.pos, cfg.rad, cfg.L)
        ctxs.append(c)
        xs.append(torch.tensor(rng.standard_normal((cfg.N, 3)), device="cuda", dtype=torch.float32))
    ref = [c.apply(x).clone() for c, x in zip(ctxs, xs)]
    ys = [torch.empty_like(x) for x in xs]
    b = api.Batch(ctxs, nstreams=2)
    b.set_wait_limit(0.05)
    b.inject_stall(2)
    import time
    for step in range(2):                 # the eager preparing step, then the persistent launch
        b.apply(xs, ys, use_graph=api.Batch.PERSISTENT)
    t = time.perf_counter()
    with pytest.raises(api.SeError) as e:
        b.status()
    assert e.value.code == api.SE_ERR_CUDA
    assert time.perf_counter() - t < 5.0
    b.status()                            # the failure was reported once and cleared
    b.inject_stall(-1)
    for step in range(2):
        for y in ys:
            y.fill_(float("nan"))
        b.apply(xs, ys, use_graph=api.Batch.PERSISTENT)
        b.status()
        for y, r in zip(ys, ref):
            assert float(torch.linalg.norm(y - r) / torch.linalg.norm(r)) <= 1e-6
    b.close()
