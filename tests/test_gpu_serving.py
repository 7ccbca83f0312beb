"""Request loop (me_server_create / me_submit / me_poll): continuous batching of mixed
requests, admission by memory, malformed requests, bounded waits."""
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


def _alone(me, r, precision):
    h = me.Handle(r["process"], precision=precision, lanes_per_event=4)
    f = h.born if KIND[r["process"]] == "born" else h.real_subtracted
    return f(r["p"], r["w"])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_results_same_alone_and_in_the_mix(me, precision):
    prec = me.ME_PREC_MIXED if precision == "mixed" else me.ME_PREC_FP64
    reqs = _requests(24, 31)
    srv = me.Server(n_slots=4, precision=prec, lanes_per_event=4)
    tickets = [srv.submit(r["process"], KIND[r["process"]], r["p"], r["w"]) for r in reqs]
    res = [srv.poll(t, timeout_us=60_000_000) for t in tickets]
    for r, out in zip(reqs, res):
        assert out["status"] == me.ME_OK
        ref = _alone(me, r, prec)
        np.testing.assert_allclose(out["out"], ref, rtol=1e-12, atol=0)
        np.testing.assert_allclose(out["sum_w"], ref.sum(), rtol=1e-12)
        assert out["t_total_us"] >= out["t_queue_us"] >= 0
    srv.close()


def test_admission_under_a_tiny_memory_budget(me):
    """Budget just above the largest request: requests run (mostly) one at a time but all
    complete with the same results."""
    reqs = _requests(10, 41, hi=4096)
    biggest = max(r["n"] * (4 * r["p"].shape[1] + 2) * 8 for r in reqs)
    srv = me.Server(n_slots=4, mem_budget_bytes=biggest + 1, lanes_per_event=4)
    tickets = [srv.submit(r["process"], KIND[r["process"]], r["p"], r["w"]) for r in reqs]
    for r, t in zip(reqs, tickets):
        out = srv.poll(t, timeout_us=60_000_000)
        assert out["status"] == me.ME_OK
        np.testing.assert_allclose(out["out"], _alone(me, r, me.ME_PREC_MIXED), rtol=1e-12)
    srv.close()


def test_malformed_and_oversized_requests(me):
    srv = me.Server(n_slots=2, mem_budget_bytes=1 << 20, max_queue=2, lanes_per_event=4)
    b = synth.flat_points("gg_tt", 64, 3)
    with pytest.raises(me.MEError) as e:
        srv.submit("gg_xx", "born", b.p)
    assert e.value.code == me.ME_ERR_PROCESS
    big = synth.flat_points("gg_tt", 40000, 3)  # 40000 * 18 * 8 B > 1 MiB budget
    with pytest.raises(me.MEError) as e:
        srv.submit("gg_tt", "born", big.p)
    assert e.value.code == me.ME_ERR_BUSY
    with pytest.raises(me.MEError) as e:
        srv.poll(987654321)
    assert e.value.code == me.ME_ERR_ARG
    srv.close()


def test_queue_full_and_bounded_poll(me):
    """A full queue rejects with ME_ERR_BUSY; a zero-timeout poll on unfinished work
    returns ME_ERR_TIMEOUT (host-side wait only) and a later poll returns the result."""
    srv = me.Server(n_slots=1, max_queue=1, lanes_per_event=4)
    b = synth.flat_points("gg_ttgg", 20000, 6)
    t1 = srv.submit("gg_ttgg", "born", b.p)
    rejected = 0
    extra = []
    for _ in range(8):
        try:
            extra.append(srv.submit("gg_ttgg", "born", b.p))
        except me.MEError as e:
            assert e.code == me.ME_ERR_BUSY
            rejected += 1
    assert rejected >= 1
    r = srv.poll(t1, timeout_us=0)
    assert r["status"] in (me.ME_ERR_TIMEOUT, me.ME_OK)
    if r["status"] == me.ME_ERR_TIMEOUT:
        r = srv.poll(t1, timeout_us=120_000_000)
    assert r["status"] == me.ME_OK and r["n"] == b.n
    for t in extra:
        assert srv.poll(t, timeout_us=120_000_000)["status"] == me.ME_OK
    srv.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_graph_replays_match_ordinary_launches(me, precision):
    """After the first request of a (process, kind) on a slot, later ones replay the
    slot's captured CUDA graph (batch size read on the device, momenta at the slot's
    stride); every result equals the same request evaluated alone."""
    prec = me.ME_PREC_MIXED if precision == "mixed" else me.ME_PREC_FP64
    srv = me.Server(n_slots=2, precision=prec, lanes_per_event=4)
    for proc in ("gg_ttg", "gg_ttgg", "ee_uu"):
        kind = KIND[proc]
        sizes = [300, 4096, 1000, 2500, 64, 3000, 777, 4096]
        reqs = [synth.flat_points(proc, m, 50 + i) for i, m in enumerate(sizes)]
        ts = [srv.submit(proc, kind, b.p, b.wgt) for b in reqs]
        for b, t in zip(reqs, ts):
            out = srv.poll(t, timeout_us=60_000_000)
            assert out["status"] == me.ME_OK
            ref = _alone(me, {"process": proc, "p": b.p, "w": b.wgt}, prec)
            np.testing.assert_allclose(out["out"], ref, rtol=1e-12, atol=0)
    st = srv.stats()
    srv.close()
    assert st["plain_runs"] + st["graph_runs"] == 24
    assert st["graph_runs"] >= 24 - 2 * 3 * 2  # at most two ordinary runs per (slot, key)
