"""Persistent serving kernels (me_server_params.persistent = 1): the e+e-, g g and u ubar
families run on one resident kernel each, fed through a ring of work descriptors in
pinned host memory; gg_ttgg requests stay on the slots.  Each result equals the same
request evaluated alone, and a kernel whose bounded wait for work runs out ends with
ME_ERR_TIMEOUT and is launched again by the next request (the stall is on the host)."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KIND = {"ee_uu": "born", "ee_uug": "real_subtracted", "gg_tt": "born", "gg_ttg": "real_subtracted",
        "gg_ttgg": "born", "uu_ttg": "real_subtracted"}


@pytest.fixture(scope="module")
def me():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_07439_gb300 as m
    return m


def _requests(n, seed, hi=8192):
    reqs = synth.mixed_stream(n, seed, lo=256, hi=hi)
    for r in reqs:
        b = synth.flat_points(r["process"], r["n"], r["seed"])
        r["p"], r["w"] = b.p, b.wgt
    return reqs


def _alone(me, r, precision, **kw):
    # one lane per point, as in the persistent kernels (gg_ttgg, served by the slots: tuned)
    h = me.Handle(r["process"], precision=precision, lanes_per_event=0 if r["process"] == "gg_ttgg" else 1, **kw)
    f = h.born if KIND[r["process"]] == "born" else h.real_subtracted
    return f(r["p"], r["w"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_results_same_alone_and_in_the_mix(me, precision):
    """float64: the persistent kernel runs the per-point code of the one-lane kernels,
    compiled into another kernel (the compiler may fuse other multiply-adds), so the
    weights agree to rounding: Borns to 1e-12, subtracted reals to 1e-11 on 99.9 % of
    the points of a request and 1e-8 on all (their cancellation amplifies the rounding);
    mixed precision: both re-evaluate the flagged points in float64 (whole points here,
    items in the handle), to the mixed-precision tolerance (1e-5 of |W| on 99.9 % of the
    points of each request, 1e-4 on all)."""
    prec = me.ME_PREC_MIXED if precision == "mixed" else me.ME_PREC_FP64
    reqs = _requests(30, 51)
    srv = me.Server(n_slots=2, precision=prec, persistent=True)
    tickets = [srv.submit(r["process"], KIND[r["process"]], r["p"], r["w"]) for r in reqs]
    res = [srv.poll(t, timeout_us=120_000_000) for t in tickets]
    st = srv.stats()
    srv.close()
    for r, out in zip(reqs, res):
        assert out["status"] == me.ME_OK, (r["process"], out["status"])
        ref = _alone(me, r, prec)
        rel = np.abs(out["out"] - ref) / np.abs(ref)
        if prec == me.ME_PREC_FP64 and KIND[r["process"]] == "born":
            assert rel.max() <= 1e-12, (r["process"], rel.max())
        elif prec == me.ME_PREC_FP64:
            assert np.quantile(rel, 0.999) <= 1e-11 and rel.max() <= 1e-8, (r["process"], np.sort(rel)[-3:])
        else:
            assert np.quantile(rel, 0.999) <= 1e-5 and rel.max() <= 1e-4, (r["process"], np.sort(rel)[-3:])
        np.testing.assert_allclose(out["sum_w"], out["out"].sum(), rtol=1e-12)
    n_fam = sum(r["process"] != "gg_ttgg" for r in reqs)
    assert st["persistent_requests"] == n_fam and st["persistent_launches"] >= 1, st


def test_persistent_kernel_idle_timeout_and_relaunch(me):
    """After the last request the host stalls for 0.3 s: the kernels' bounded waits for
    work (1 ms) run out, each ends with ME_ERR_TIMEOUT (counted), the context stays usable,
    and the next request launches its family's kernel again and is served correctly."""
    srv = me.Server(n_slots=1, precision=me.ME_PREC_FP64, persistent=True, persistent_idle_us=1000)
    b = synth.flat_points("gg_ttg", 3000, 61)
    r1 = srv.poll(srv.submit("gg_ttg", "real_subtracted", b.p, b.wgt), timeout_us=60_000_000)
    assert r1["status"] == me.ME_OK
    time.sleep(0.3)  # host-side stall: no work arrives
    st1 = srv.stats()
    assert st1["persistent_idle_timeouts"] >= 1 and st1["persistent_launches"] == 1, st1
    r2 = srv.poll(srv.submit("gg_ttg", "real_subtracted", b.p, b.wgt), timeout_us=60_000_000)
    st2 = srv.stats()
    srv.close()
    assert r2["status"] == me.ME_OK and st2["persistent_launches"] == 2, st2
    np.testing.assert_array_equal(r1["out"], r2["out"])
    ref = _alone(me, {"process": "gg_ttg", "p": b.p, "w": b.wgt}, me.ME_PREC_FP64)
    rel = np.abs(r2["out"] - ref) / np.abs(ref)
    assert np.quantile(rel, 0.999) <= 1e-11 and rel.max() <= 1e-8


def test_persistent_kernels_apply_the_cuts(me):
    """The persistent family kernels evaluate the cuts of every term as the masked
    evaluation does (Algorithm 2): with heavy-quark and thrust-axis cuts on, each request
    equals the same request evaluated alone with the same cuts, exact zeros included."""
    cuts = dict(cut_pt_min=100.0, cut_abs_y_max=1.0, cut_abs_cos_axis_max=0.7)
    reqs = _requests(16, 53)
    srv = me.Server(n_slots=2, precision=me.ME_PREC_FP64, persistent=True, **cuts)
    tickets = [srv.submit(r["process"], KIND[r["process"]], r["p"], r["w"]) for r in reqs]
    res = [srv.poll(t, timeout_us=120_000_000) for t in tickets]
    srv.close()
    zeros = 0
    for r, out in zip(reqs, res):
        assert out["status"] == me.ME_OK
        ref = _alone(me, r, me.ME_PREC_FP64, **cuts)
        z = ref == 0.0
        zeros += int(z.sum())
        assert np.all(out["out"][z] == 0.0), r["process"]
        rel = np.abs(out["out"][~z] - ref[~z]) / np.abs(ref[~z])
        if rel.size:
            assert np.quantile(rel, 0.999) <= 1e-11 and rel.max() <= 1e-8, (r["process"], np.sort(rel)[-3:])
    assert zeros > 0
