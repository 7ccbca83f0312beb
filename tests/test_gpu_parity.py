"""CUDA path (through the C ABI) versus the FP64 oracle on identical seeded points."""
import math

import numpy as np
import pytest

import synth
from oracle import fks, nlo_ee
from oracle import matrix_element as ome
from oracle.matrix_element import to_points
from tests import fp64_arbiter as arb

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def me():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_07439_gb300 as m
    return m


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


TREE_CASES = [("ee_uu", 1), ("ee_uug", 2), ("gg_tt", 3), ("gg_ttg", 4), ("uu_tt", 5), ("uu_ttg", 6),
              ("gg_ttgg", 7)]


@pytest.mark.parametrize("name,seed", TREE_CASES)
def test_tree_fp64_matches_oracle(me, name, seed):
    n = 257 if name != "gg_ttgg" else 67
    b = synth.flat_points(name, n, seed)
    ref = ome.me2(name, to_points(b.p)) * b.wgt
    h = me.Handle(name, precision=me.ME_PREC_FP64)
    got = h.born(_dev(b.p), _dev(b.wgt)).cpu().numpy()
    # <= 1e-12 of the oracle per point, or, where the float64 inputs do not fix the value
    # that well, within the conditioning bound of the extended-precision oracle
    arb.check_fp64(got, lambda q: ome.me2(name, q), to_points(b.p), b.wgt)
    # host pointers give the same numbers
    got_h = h.born(b.p, b.wgt)
    np.testing.assert_array_equal(got_h, got)


@pytest.mark.parametrize("name,seed", TREE_CASES)
def test_tree_mixed_matches_oracle(me, name, seed):
    n = 2000 if name != "gg_ttgg" else 200
    b = synth.flat_points(name, n, seed + 100)
    ref = ome.me2(name, to_points(b.p))
    h = me.Handle(name, precision=me.ME_PREC_MIXED)
    got = h.born(_dev(b.p)).cpu().numpy()
    rel = np.abs(got / ref - 1)
    assert np.quantile(rel, 0.999) <= 1e-5, np.sort(rel)[-5:]
    assert rel.max() < 1e-3


def test_gg_tt_scan_fp64(me):
    b = synth.gg_tt_scan(1031, 3)
    ref = ome.me2("gg_tt", to_points(b.p))
    h = me.Handle("gg_tt")
    np.testing.assert_allclose(h.born(_dev(b.p)).cpu().numpy(), ref, rtol=1e-12)


def _sub_mag(name, k, fp):
    tot, parts = fks.real_subtracted(name, k, fp, detail=True)
    mag = sum(np.abs(p["RS"]) + np.abs(p["RS"] - p["W"]) for p in parts)
    return tot, mag


def _rs(name, fp=fks.FKSParams()):
    """The oracle's subtracted real of `name` as a function of the points (float64 or
    extended precision, following the input)."""
    return lambda q: fks.real_subtracted(name, q, fp)


@pytest.mark.parametrize("name,seed", [("ee_uug", 2), ("gg_ttg", 4), ("uu_ttg", 8)])
@pytest.mark.parametrize("xc,dl", [(0.5, 1.0), (1.0, 2.0), (0.2, 0.7)])
def test_real_subtracted_fp64_flat(me, name, seed, xc, dl):
    b = synth.flat_points(name, 257, seed)
    h = me.Handle(name, precision=me.ME_PREC_FP64, xi_cut=xc, delta=dl)
    got = h.real_subtracted(_dev(b.p)).cpu().numpy()
    arb.check_fp64(got, _rs(name, fks.FKSParams(xc, dl)), to_points(b.p))


@pytest.mark.parametrize("name", ["gg_ttg", "uu_ttg"])
def test_real_subtracted_fp64_approach(me, name):
    b, lab = synth.approach_points(name, 32, 5)
    h = me.Handle(name, precision=me.ME_PREC_FP64)
    got = h.real_subtracted(_dev(b.p)).cpu().numpy()
    st = arb.check_fp64(got, _rs(name), to_points(b.p))
    # the float64 inputs fix the weight (C cond u < 1) on most approach points; the rest
    # (soft-collinear corners, 1 - y or xi at 1e-8) are only required to be finite
    assert st["unresolved"] <= 0.35 * b.n, st


def test_real_subtracted_fp64_approach_fsr(me):
    rng = np.random.default_rng(7)
    n = 200
    xi = 10.0 ** rng.uniform(-8, -1, n)
    y = 1 - 10.0 ** rng.uniform(-8, -1, n)
    p = synth.fsr_emission_points(100.0, rng.uniform(-1, 1, n), rng.uniform(0, 6.28, n), xi, y,
                                  rng.uniform(0, 6.28, n), 2)
    h = me.Handle("ee_uug")
    got = h.real_subtracted(_dev(p)).cpu().numpy()
    st = arb.check_fp64(got, _rs("ee_uug"), to_points(p))
    assert st["arbitrated"] + st["agree_1e-12"] >= 0.25 * n, st


@pytest.mark.parametrize("name,seed", [("ee_uug", 2), ("gg_ttg", 4), ("uu_ttg", 8)])
def test_real_subtracted_mixed(me, name, seed):
    """Mixed precision with FP64 rescue: <= 1e-5 relative on >= 99.9% of points."""
    b = synth.flat_points(name, 4000, seed + 50)
    k = to_points(b.p)
    ref, mag = _sub_mag(name, k, fks.FKSParams())
    h = me.Handle(name, precision=me.ME_PREC_MIXED)
    got = h.real_subtracted(_dev(b.p)).cpu().numpy()
    rel = np.abs(got - ref) / np.abs(ref)
    assert np.quantile(rel, 0.999) <= 1e-5, np.sort(rel)[-8:]
    assert np.all(np.abs(got - ref) <= 1e-4 * mag)
    n_resc = h.last_rescued()
    assert 0 <= n_resc <= b.n
    # integrated result within 1e-6 relative
    assert abs(got.sum() - ref.sum()) <= 1e-6 * np.abs(ref).sum()


@pytest.mark.parametrize("name", ["gg_ttg", "uu_ttg"])
def test_real_subtracted_mixed_approach_rescued(me, name):
    """On soft/collinear approach sequences, points within the thresholds (xi or 1-y
    below 1e-3) are re-evaluated in FP64 and match the oracle to FP64 resolution; the
    rest pass the stability test or are re-evaluated, and meet the mixed-precision target
    (at most 0.2 % of points beyond 1e-5 of the weight, or beyond FP64 resolution where
    that is coarser)."""
    b, lab = synth.approach_points(name, 16, 5)
    k = to_points(b.p)
    h = me.Handle(name, precision=me.ME_PREC_MIXED)
    got = h.real_subtracted(_dev(b.p)).cpu().numpy()
    assert h.last_rescued() >= int(0.8 * b.n)
    near = lab["value"] < 1e-3
    # inside the thresholds the points are re-evaluated in float64: the float64 rule
    arb.check_fp64(got[near], _rs(name), k[near])
    # beyond the thresholds: within 1e-5 of the weight, or, where the float64 inputs fix
    # the weight less well than that, within the conditioning bound (extended oracle)
    far = ~near
    with np.errstate(all="ignore"):
        ref = fks.real_subtracted(name, k[far])
    got_far = got[far]
    off = ~(np.abs(got_far - ref) <= 1e-5 * np.abs(ref))
    idx = np.flatnonzero(off)
    if idx.size:
        fx, cond = arb.extended(_rs(name), k[far][idx])
        with np.errstate(all="ignore"):
            err = (np.abs(got_far[idx] - fx) / np.abs(fx)).astype(float)
        ok = err <= np.maximum(1e-5, arb.C_COND * cond * arb.U)
        off[idx[ok]] = False
    assert np.mean(off) <= 0.002, (int(off.sum()), far.sum())


def test_nbody_nlo(me):
    b = synth.flat_points("ee_uu", 129, 1)
    ref = nlo_ee.nbody_nlo(to_points(b.p), 0.3, 1.5)
    h = me.Handle("ee_uu", xi_cut=0.3, delta=1.5)
    np.testing.assert_allclose(h.nbody_nlo(_dev(b.p)).cpu().numpy(), ref, rtol=1e-12)


def test_accumulators_and_resume(me):
    b = synth.flat_points("gg_tt", 1000, 3)
    h = me.Handle("gg_tt")
    out = h.born(_dev(b.p), _dev(b.wgt)).cpu().numpy()
    s, s2, n = h.accumulators()
    assert n == 1000
    np.testing.assert_allclose([s, s2], [out.sum(), (out * out).sum()], rtol=1e-12)
    h.set_accumulators((1.0, 2.0, 3.0))
    assert h.accumulators() == (1.0, 2.0, 3.0)


def test_edge_cases_and_errors(me):
    h = me.Handle("gg_tt")
    empty = np.zeros((4, 4, 0))
    assert h.born(empty).shape == (0,)
    one = synth.flat_points("gg_tt", 1, 3)
    np.testing.assert_allclose(h.born(one.p), ome.me2("gg_tt", to_points(one.p)), rtol=1e-12)
    with pytest.raises(me.MEError) as e:
        me.Handle("gg_xx")
    assert e.value.code == me.ME_ERR_PROCESS
    with pytest.raises(me.MEError) as e:
        h.real_subtracted(one.p)
    assert e.value.code == me.ME_ERR_PROCESS
    with pytest.raises(me.MEError) as e:
        me.Handle("gg_tt", xi_cut=0.0)
    assert e.value.code == me.ME_ERR_ARG
    with pytest.raises(ValueError):
        h.born(np.zeros((4, 5, 3)))


def test_determinism(me):
    b = synth.flat_points("gg_ttg", 3000, 11)
    h = me.Handle("gg_ttg", precision=me.ME_PREC_MIXED, lanes_per_event=8)
    a1 = h.real_subtracted(_dev(b.p)).cpu().numpy()
    a2 = h.real_subtracted(_dev(b.p)).cpu().numpy()
    np.testing.assert_array_equal(a1, a2)


def test_pinned_host_buffers_read_in_place(me):
    """Pinned host buffers are used in place by the kernels (no staging copy); the results
    equal those from device buffers and from pageable host buffers, bit for bit."""
    b = synth.flat_points("gg_ttg", 5000, 61)
    h = me.Handle("gg_ttg", precision=me.ME_PREC_MIXED, lanes_per_event=1)
    dev = h.real_subtracted(_dev(b.p), _dev(b.wgt)).cpu().numpy()
    pageable = h.real_subtracted(b.p.copy(), b.wgt.copy())
    pp = torch.from_numpy(b.p.copy()).pin_memory()
    pw = torch.from_numpy(b.wgt.copy()).pin_memory()
    po = torch.empty(b.n, dtype=torch.float64).pin_memory()
    h.real_subtracted(pp.numpy(), pw.numpy(), po.numpy())
    np.testing.assert_array_equal(po.numpy(), dev)
    np.testing.assert_array_equal(pageable, dev)


@pytest.mark.parametrize("name,seed", [("gg_ttg", 71), ("uu_ttg", 72), ("ee_uug", 73)])
def test_queued_rescue_equals_separate_launches(me, name, seed):
    """The one-launch kernel that queues its unstable points per block and re-evaluates
    them in float64 gives the results, the rescued count and the accumulators of a
    float32 launch followed by a float64 launch over the compacted list (both one lane
    per point).  Both run the same per-point code, but compiled into different kernels
    the compiler may fuse multiply-adds differently, so the float32 values differ by
    float32 rounding and a point on the stability threshold may be re-evaluated by one
    path only: the two agree to the mixed-precision tolerance (1e-5 of |W| each way).
    Sizes: many tiles per block of the persistent grid with a ragged tail, one partial
    tile, and an empty batch."""
    hq = me.Handle(name, precision=me.ME_PREC_MIXED, queued_rescue=1)
    hs = me.Handle(name, precision=me.ME_PREC_MIXED, lanes_per_event=1)
    for n in (200000 + 77, 50, 0):
        b = synth.flat_points(name, max(n, 1), seed)
        p, w = b.p[:, :, :n], b.wgt[:n]
        hq.set_accumulators((0.0, 0.0, 0.0))
        hs.set_accumulators((0.0, 0.0, 0.0))
        q = hq.real_subtracted(_dev(p), _dev(w)).cpu().numpy()
        s = hs.real_subtracted(_dev(p), _dev(w)).cpu().numpy()
        nq, ns = hq.last_rescued(), hs.last_rescued()
        assert abs(nq - ns) <= max(2, 1e-4 * n)
        if n > 100000:
            assert nq > 1000
        if n:
            rel = np.abs(q - s) / np.maximum(np.abs(s), 1e-300)
            assert np.quantile(rel, 0.999) <= 2e-5 and rel.max() <= 1e-4, np.sort(rel)[-3:]
        aq, as_ = np.asarray(hq.accumulators()), np.asarray(hs.accumulators())
        assert aq[2] == as_[2] == n
        np.testing.assert_allclose(aq[:2], as_[:2], rtol=1e-6, atol=0)


@pytest.mark.parametrize("name,seed", [("gg_ttg", 81), ("uu_ttg", 82), ("ee_uug", 83)])
def test_item_rescue_matches_point_rescue(me, name, seed):
    """The item rescue re-evaluates in float64 only the ingredients (real-emission
    helicity blocks, counterterm Born values) a flagged point's tolerance needs and
    recombines W = sum_i a_i v_i in float64; re-evaluating the flagged points whole is
    the reference.  Same lane layout, so the float32 pass and the flagged points are
    identical: the counts agree exactly, the item path does less float64 work, and the
    weights agree to the mixed-precision tolerance (1e-5 of |W|, 99.9 %; the residual
    float32 error of a flagged point is budgeted at half of that).  A ragged size
    spans many blocks and warps."""
    n = 100003
    b = synth.flat_points(name, n, seed)
    p, w = _dev(b.p), _dev(b.wgt)
    hi = me.Handle(name, precision=me.ME_PREC_MIXED, rescue=me.ME_RESCUE_ITEMS, lanes_per_event=2)
    hp = me.Handle(name, precision=me.ME_PREC_MIXED, rescue=me.ME_RESCUE_POINTS, lanes_per_event=2)
    wi = hi.real_subtracted(p, w).cpu().numpy()
    wp = hp.real_subtracted(p, w).cpu().numpy()
    pts, blocks, borns = hi.last_rescue_work()
    assert pts == hp.last_rescued() > 0
    nb = {"gg_ttg": 4, "uu_ttg": 2, "ee_uug": 2}[name]
    assert 0 < blocks < nb * pts and borns <= pts
    rel = np.abs(wi - wp) / np.abs(wp)
    assert np.quantile(rel, 0.999) <= 1e-5 and rel.max() <= 1e-4, np.sort(rel)[-3:]
    assert abs(wi.sum() - wp.sum()) <= 1e-6 * np.abs(wp).sum()
    # unflagged points are untouched by the rescue: identical bits
    np.testing.assert_array_equal(np.sort(np.flatnonzero(wi != wp)).size <= pts, True)


def test_domain_boundary_points(me):
    """Points on the boundary of the FKS domain (no emitted energy, or the gluon exactly
    along a beam) carry weight 0 in both precisions, as in the oracle; they are not
    re-evaluated, and the accumulators stay finite."""
    xi = np.array([0.3, 0.0, 0.3, 0.3])
    cb = np.array([0.2, 0.2, 1.0, -1.0])
    p = synth.emission_points(1000.0, 173.0, xi, cb, np.full(4, 0.4), np.full(4, 0.3), np.full(4, 1.1))
    with np.errstate(all="ignore"):
        ref = fks.real_subtracted("gg_ttg", to_points(p))
    for prec in (me.ME_PREC_FP64, me.ME_PREC_MIXED):
        h = me.Handle("gg_ttg", precision=prec)
        got = h.real_subtracted(_dev(p)).cpu().numpy()
        assert list(got[1:]) == [0.0, 0.0, 0.0]
        assert abs(got[0] / ref[0] - 1) <= (1e-12 if prec == me.ME_PREC_FP64 else 1e-5)
        acc = h.accumulators()
        assert np.all(np.isfinite(acc)) and acc[2] == 4
        if prec == me.ME_PREC_MIXED:
            assert h.last_rescued() <= 1
