"""Batched persistent launch: requests of k = 1..5 with uneven point counts in
one graph launch give the same |M|^2 as one standalone launch per request
(bit for bit: same per-point code, in either kernel form), and match the
oracle on samples."""
import ctypes

import numpy as np
import pytest

from tests.test_gpu_parity import mixed_tol
from paper_2511_19456_b300 import Batch, Plan, _lib, phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REQS = [(5, 37, 6.0), (1, 3001, 1.0), (3, 999, 3.0), (2, 1, 2.5), (4, 257, 4.0), (1, 64, 8.0),
        (5, 100, 3.0), (3, 0, 2.0), (4, 33, 7.0), (2, 4096, 1.5)]


def make_inputs(seed0=700):
    moms = [torch.from_numpy(ps.points(k, max(n, 1), om, seed0 + i))[:n].contiguous().cuda()
            for i, (k, n, om) in enumerate(REQS)]
    return moms


@pytest.mark.parametrize("form", ["table", "specialised"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_standalone_and_oracle(orc, precision, form):
    plans = {k: Plan(k, precision=precision) for k in range(1, 6)}
    moms = make_inputs()
    batch = Batch([plans[k] for k, _, _ in REQS], [n for _, n, _ in REQS])
    assert batch.info()["kernel_form"] == "specialised"   # a new batch's form
    batch.set_kernel_form(form)
    assert batch.info()["kernel_form"] == form
    outs = batch.eval(moms)
    torch.cuda.synchronize()
    for (k, n, _), m, o in zip(REQS, moms, outs):
        if n == 0:
            continue
        # the batch runs the point code of the standalone plan in the same
        # form: bit for bit
        plans[k].set_kernel_form(form)
        ref = plans[k].eval(m)
        torch.cuda.synchronize()
        assert torch.equal(o, ref), (k, n)
    # oracle on a sample of each request
    for (k, n, _), m, o in zip(REQS, moms, outs):
        if n == 0:
            continue
        idx = np.unique(np.linspace(0, n - 1, min(n, 8)).astype(int))
        mm = m.cpu().numpy()[idx]
        r, kap = orc.m2(mm, kappa=True)
        rel = np.abs(o.cpu().numpy()[idx] / r - 1)
        tol = np.maximum(1e-12, 64 * 2.0 ** -53 * kap) if precision == "fp64" else mixed_tol(k, kap)
        assert np.all(rel <= tol), (k, rel.max())


def test_batch_tune_and_replay():
    plans = {k: Plan(k, precision="mixed") for k in range(1, 6)}
    moms = make_inputs(900)
    batch = Batch([plans[k] for k, _, _ in REQS], [n for _, n, _ in REQS])
    first = [o.clone() for o in batch.eval(moms)]
    ms = batch.tune(moms)
    info = batch.info()
    assert ms > 0 and info["block"] in (64, 128, 256) and info["n_items"] > 0
    assert info["kernel_form"] in ("table", "specialised")
    outs = batch.outputs()
    for _ in range(3):
        batch.eval(moms, outs)
    torch.cuda.synchronize()
    for a, b in zip(first, outs):
        assert torch.equal(a, b)


def test_batch_rejects_bad_requests():
    L = _lib.lib()
    h = ctypes.c_void_p()
    a, b = Plan(2), Plan(3, precision="mixed")
    ph = (ctypes.c_void_p * 2)(a._h.value, b._h.value)
    nn = (ctypes.c_longlong * 2)(10, 10)
    assert L.qed_batch_create(ph, 2, nn, ctypes.byref(h)) == _lib.QED_EINVAL
    f = Plan(2, summed=False, hel=[1, 1, 1, 1, 1])
    ph = (ctypes.c_void_p * 1)(f._h.value)
    assert L.qed_batch_create(ph, 1, nn, ctypes.byref(h)) == _lib.QED_EUNSUPPORTED
    six = Plan(6)
    ph = (ctypes.c_void_p * 1)(six._h.value)
    assert L.qed_batch_create(ph, 1, nn, ctypes.byref(h)) == _lib.QED_EUNSUPPORTED
    nn = (ctypes.c_longlong * 1)(-1)
    ph = (ctypes.c_void_p * 1)(a._h.value)
    assert L.qed_batch_create(ph, 1, nn, ctypes.byref(h)) == _lib.QED_EINVAL


# ---- the seeded stream of the batched configuration itself
def oracle_subset(k):
    """Points of each request compared with the oracle: 4,096 for k <= 4,
    256 at k = 5 (about 1e8 oracle FLOP per point)."""
    return 4096 if k <= 4 else 256


@pytest.fixture(scope="module")
def seeded_stream():
    """The configuration's 64 seeded requests (k = 1..5, 1e3 to 1e6 points,
    omega in [1, 8]), every point from the host generator."""
    reqs = ps.batched_requests()
    return reqs, [ps.points(r["k"], r["n_points"], r["omega"], r["seed"]) for r in reqs]


@pytest.fixture(scope="module")
def seeded_stream_oracle(orc, seeded_stream):
    reqs, moms = seeded_stream
    return [orc.m2(m[:oracle_subset(r["k"])], kappa=True) for r, m in zip(reqs, moms)]


def _static_call(plans, n, moms, outs):
    L = _lib.lib()
    nreq = len(plans)
    ph = (ctypes.c_void_p * nreq)(*[p._h.value for p in plans])
    nn = (ctypes.c_longlong * nreq)(*n)
    pm = (ctypes.c_void_p * nreq)(*[m.data_ptr() for m in moms])
    po = (ctypes.c_void_p * nreq)(*[o.data_ptr() for o in outs])
    return L.qed_batch_eval_static(ph, nreq, nn, pm, po, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("entry", ["qed_batch_eval", "qed_batch_eval_table", "qed_batch_eval_static"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_seeded_batched_stream_vs_oracle(seeded_stream, seeded_stream_oracle, entry, precision):
    """All 64 requests (10.9 M points) in one persistent launch, then each
    request's first points against the oracle at the per-point bounds:
    qed_batch_eval in its tuned (mixed) or default (FP64) form and in the
    table form, and the allocation-free entry point."""
    from tests.test_gpu_parity import check_mixed_median
    reqs, moms = seeded_stream
    plans = {k: Plan(k, precision=precision) for k in range(1, 6)}
    req_plans = [plans[r["k"]] for r in reqs]
    n = [r["n_points"] for r in reqs]
    d = [torch.from_numpy(m).cuda() for m in moms]
    if entry.startswith("qed_batch_eval") and entry != "qed_batch_eval_static":
        batch = Batch(req_plans, n)
        if entry == "qed_batch_eval_table":
            batch.set_kernel_form("table")
        elif precision == "mixed":
            batch.tune(d, batch.outputs())
        outs = batch.eval(d)
    else:
        outs = [torch.full((c,), -1.0, dtype=torch.float64, device="cuda") for c in n]
        assert _static_call(req_plans, n, d, outs) == _lib.QED_OK
    torch.cuda.synchronize()
    rels, kaps = [], []
    for r, o, (ref, kap) in zip(reqs, outs, seeded_stream_oracle):
        got = o[:len(ref)].cpu().numpy()
        rel = np.abs(got / ref - 1.0)
        tol = np.maximum(1e-12, 64 * 2.0 ** -53 * kap) if precision == "fp64" else mixed_tol(r["k"], kap)
        assert np.all(rel <= tol), (r, float(rel.max()))
        assert torch.isfinite(o).all() and (o > 0).all()
        rels.append(rel)
        kaps.append(kap)
    rel, kap = np.concatenate(rels), np.concatenate(kaps)
    print(f"\n{entry} {precision}: {rel.size} oracle points over {len(reqs)} requests, "
          f"median rel {np.median(rel):.3e} max {rel.max():.3e} (kappa max {kap.max():.1f})")
    if precision == "mixed":
        check_mixed_median(rel, kap)


def test_batch_form_rejects_unknown():
    L = _lib.lib()
    batch = Batch([Plan(2)], [10])
    assert L.qed_batch_set_kernel_form(batch._h, 2) == _lib.QED_EINVAL
    assert L.qed_batch_set_kernel_form(None, 0) == _lib.QED_EINVAL
    assert batch.info()["kernel_form"] == "specialised"
