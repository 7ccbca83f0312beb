"""Cuts of each term (Algorithm 2: evaluate every term, zero those whose cuts fail at the
term's own kinematics) and the per-term queues (the variant discussed after Algorithm 2:
queue only the amplitudes whose terms survive), CUDA path versus the oracle with the
same cuts (oracle.cuts).

A cut decision is an integer result taken in float64 on both sides with the same
operations; the counter-event momenta it is taken on are computed by each side with its
own float64 arithmetic, so a point within rounding of a threshold may be decided either
way.  Such points are found by re-running the oracle with every threshold moved by 1e-9
(relative) both ways: where the two differ, the CUDA result must match one of them;
everywhere else it must match the oracle at the nominal cuts."""
import functools

import numpy as np
import pytest

import synth
from oracle import fks, nlo_ee
from oracle.cuts import Cuts, tree_weights
from oracle.matrix_element import to_points
from tests import fp64_arbiter as arb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CUTS = {
    "ee": [Cuts(abs_cos_axis_max=0.6), Cuts(abs_cos_axis_max=0.8, thrust_max=0.9)],
    "heavy": [Cuts(pt_min=150.0), Cuts(pt_min=100.0, abs_y_max=1.0)],
    "heavy4": [Cuts(pt_min=200.0, abs_y_max=1.2)],
}
FAMILY = {"ee_uu": "ee", "ee_uug": "ee", "gg_tt": "heavy", "gg_ttg": "heavy", "uu_tt": "heavy",
          "uu_ttg": "heavy", "gg_ttgg": "heavy4"}
N_REAL = {"ee_uug": 4099, "gg_ttg": 2051, "uu_ttg": 2051}


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


def _params(c: Cuts):
    return dict(cut_pt_min=c.pt_min, cut_abs_y_max=c.abs_y_max, cut_abs_cos_axis_max=c.abs_cos_axis_max,
                cut_thrust_max=c.thrust_max)


def _moved(c: Cuts, eps: float) -> Cuts:
    """Thresholds moved by eps relative: eps > 0 tightens every cut, eps < 0 loosens it."""
    return Cuts(pt_min=c.pt_min * (1 + eps), abs_y_max=c.abs_y_max * (1 - eps),
                abs_cos_axis_max=c.abs_cos_axis_max * (1 - eps) if c.abs_cos_axis_max < 1 else 1.0,
                thrust_max=c.thrust_max * (1 - eps) if c.thrust_max < 1 else 1.0)


@functools.lru_cache(maxsize=None)
def _real_case(name, icut):
    b = synth.fks_points(name, N_REAL[name], 31 + icut)
    k = to_points(b.p)
    c = CUTS[FAMILY[name]][icut]
    ref = fks.real_subtracted(name, k, cuts=c)
    lo = fks.real_subtracted(name, k, cuts=_moved(c, 1e-9))
    hi = fks.real_subtracted(name, k, cuts=_moved(c, -1e-9))
    _, parts = fks.real_subtracted(name, k, detail=True)
    mag = sum(np.abs(p["RS"]) + np.abs(p["RS"] - p["W"]) for p in parts)
    return b, k, c, ref, lo, hi, mag


def _either(got, lo, hi, tol):
    return ((np.abs(got - lo) <= tol * np.maximum(np.abs(lo), 1e-300)) |
            (np.abs(got - hi) <= tol * np.maximum(np.abs(hi), 1e-300)))


@pytest.mark.parametrize("queues", [0, 1])
@pytest.mark.parametrize("icut", [0, 1])
@pytest.mark.parametrize("name", ["ee_uug", "gg_ttg", "uu_ttg"])
def test_real_subtracted_with_cuts_fp64(me, name, icut, queues):
    b, k, c, ref, lo, hi, _ = _real_case(name, icut)
    h = me.Handle(name, precision=me.ME_PREC_FP64, term_queues=queues, **_params(c))
    got = h.real_subtracted(_dev(b.p)).cpu().numpy()
    uniq = lo == hi
    assert uniq.mean() > 0.99
    # every term cut away (or the domain boundary): exactly 0 on both sides
    zero = uniq & (ref == 0.0)
    assert np.all(got[zero] == 0.0)
    assert 0.02 < zero.mean() < 0.9, zero.mean()  # the cuts remove some points, not all
    live = uniq & ~zero
    arb.check_fp64(got[live], lambda q: fks.real_subtracted(name, q, cuts=c), k[live])
    assert np.all(_either(got[~uniq], lo[~uniq], hi[~uniq], 1e-9))


@pytest.mark.parametrize("queues", [0, 1])
@pytest.mark.parametrize("icut", [0, 1])
@pytest.mark.parametrize("name", ["ee_uug", "gg_ttg", "uu_ttg"])
def test_real_subtracted_with_cuts_mixed(me, name, icut, queues):
    """Mixed precision with the float64 item rescue: <= 1e-5 relative on >= 99.9 % of the
    points with a weight, exact zeros where every term is cut away, and the sum within
    1e-6 of sum |W| of the float64 GPU result on the same inputs.  (The sum is compared
    with the float64 path, not the oracle: points sampled within ~1e-6 of a collinear
    limit have weights that their float64 inputs fix only to ~1e-5 -- the float64 path
    and the oracle differ by that much there, within the conditioning bound of the
    float64 parity rule -- and one such point outweighs the rest of the sum's error.)"""
    b, k, c, ref, lo, hi, mag = _real_case(name, icut)
    h = me.Handle(name, precision=me.ME_PREC_MIXED, term_queues=queues, **_params(c))
    got = h.real_subtracted(_dev(b.p)).cpu().numpy()
    h64 = me.Handle(name, precision=me.ME_PREC_FP64, term_queues=queues, **_params(c))
    got64 = h64.real_subtracted(_dev(b.p)).cpu().numpy()
    uniq = lo == hi
    zero = uniq & (ref == 0.0)
    assert np.all(got[zero] == 0.0)
    live = uniq & ~zero
    # within 1e-5 of the weight, or, where the float64 inputs fix the weight less well
    # than that (points the sampler put near a collinear limit), within the conditioning
    # bound of the float64 parity rule against the extended-precision oracle
    g, r, kl = got[live], ref[live], k[live]
    off = ~(np.abs(g - r) <= 1e-5 * np.abs(r))
    idx = np.flatnonzero(off)
    if idx.size:
        fx, cond = arb.extended(lambda q: fks.real_subtracted(name, q, cuts=c), kl[idx])
        with np.errstate(all="ignore"):
            err = (np.abs(g[idx] - fx) / np.abs(fx)).astype(float)
        off[idx[err <= np.maximum(1e-5, arb.C_COND * cond * arb.U)]] = False
    assert np.mean(off) <= 1e-3, (int(off.sum()), live.sum())
    assert np.all(np.abs(g - r) <= 1e-4 * mag[live])
    assert np.all(_either(got[~uniq], lo[~uniq], hi[~uniq], 1e-4))
    assert abs(got.sum() - got64.sum()) <= 1e-6 * np.abs(got64).sum()
    assert 0 <= h.last_rescued() <= b.n


@pytest.mark.parametrize("name", ["ee_uug", "gg_ttg", "uu_ttg"])
def test_queued_terms_match_masked_terms(me, name):
    """Without cuts the per-term queues skip the Born sets of inactive counterterms only:
    float64 results agree with Algorithm 2's masked evaluation to rounding, and mixed
    ones to the mixed-precision target."""
    b = synth.flat_points(name, 3001, 77)
    p = _dev(b.p)
    res = {}
    for prec in (0, 1):
        for q in (0, 1):
            res[prec, q] = me.Handle(name, precision=prec, term_queues=q).real_subtracted(p).cpu().numpy()
    a, q = res[0, 0], res[0, 1]
    nz = a != 0
    assert np.quantile(np.abs(q[nz] / a[nz] - 1), 0.999) <= 1e-12
    assert np.all(q[~nz] == 0)
    rel = np.abs(res[1, 1][nz] / a[nz] - 1)
    assert np.quantile(rel, 0.999) <= 1e-5


TREES = [("ee_uu", 1), ("ee_uug", 2), ("gg_tt", 3), ("uu_tt", 5), ("gg_ttgg", 7)]


@pytest.mark.parametrize("queues", [0, 1])
@pytest.mark.parametrize("name,seed", TREES)
def test_tree_with_cuts(me, name, seed, queues):
    n = 1027 if name != "gg_ttgg" else 131
    b = synth.flat_points(name, n, seed)
    k = to_points(b.p)
    c = CUTS[FAMILY[name]][-1]
    lo, hi = tree_weights(name, k, _moved(c, 1e-9)), tree_weights(name, k, _moved(c, -1e-9))
    uniq = (lo == 0) == (hi == 0)
    ref = tree_weights(name, k, c) * b.wgt
    for prec in (me.ME_PREC_FP64, me.ME_PREC_MIXED):
        h = me.Handle(name, precision=prec, term_queues=queues, **_params(c))
        got = h.born(_dev(b.p), _dev(b.wgt)).cpu().numpy()
        zero = uniq & (ref == 0)
        assert np.all(got[zero] == 0.0)
        live = uniq & ~zero
        if name != "ee_uu":
            assert live.mean() > 0.05 and zero.mean() > 0.05
        else:
            assert live.sum() == 0  # two partons have thrust 1: the thrust cut removes every point
        if prec == me.ME_PREC_FP64 and live.any():
            arb.check_fp64(got[live], lambda q: tree_weights(name, q, c), k[live], b.wgt[live])
        elif live.any():
            rel = np.abs(got[live] / ref[live] - 1)
            assert np.quantile(rel, 0.999) <= 1e-5 and rel.max() < 1e-3


@pytest.mark.parametrize("queues", [0, 1])
def test_nbody_nlo_with_cuts(me, queues):
    b = synth.flat_points("ee_uu", 1029, 1)
    k = to_points(b.p)
    c = Cuts(abs_cos_axis_max=0.5)
    ref = nlo_ee.nbody_nlo(k, 0.3, 1.5, cuts=c)
    h = me.Handle("ee_uu", xi_cut=0.3, delta=1.5, term_queues=queues, **_params(c))
    got = h.nbody_nlo(_dev(b.p)).cpu().numpy()
    lo = nlo_ee.nbody_nlo(k, 0.3, 1.5, cuts=_moved(c, 1e-9))
    hi = nlo_ee.nbody_nlo(k, 0.3, 1.5, cuts=_moved(c, -1e-9))
    uniq = lo == hi
    np.testing.assert_allclose(got[uniq], ref[uniq], rtol=1e-12)
    assert 0.3 < np.mean(ref != 0) < 0.7


def test_edge_cases_with_queues(me):
    # an empty batch, a ragged warp; every term cut away (thrust <= 0.5: three partons
    # have T >= 2/3) gives exact zeros and nothing to rescue; one point and 33 points
    for q in (0, 1):
        h = me.Handle("ee_uug", precision=me.ME_PREC_MIXED, term_queues=q, cut_thrust_max=0.5)
        assert h.real_subtracted(np.zeros((4, 5, 0))).shape == (0,)
        b = synth.flat_points("ee_uug", 33, 3)
        got = h.real_subtracted(_dev(b.p)).cpu().numpy()
        assert np.all(got == 0.0) and h.last_rescued() == 0
        h = me.Handle("gg_ttg", precision=me.ME_PREC_FP64, term_queues=q, cut_pt_min=120.0)
        for n in (1, 33):
            b = synth.flat_points("gg_ttg", n, 4)
            got = h.real_subtracted(_dev(b.p)).cpu().numpy()
            ref = fks.real_subtracted("gg_ttg", to_points(b.p), cuts=Cuts(pt_min=120.0))
            np.testing.assert_allclose(got, ref, rtol=1e-10, atol=0)
    with pytest.raises(me.MEError) as e:
        me.Handle("gg_ttg", cut_pt_min=-1.0)
    assert e.value.code == me.ME_ERR_ARG
    with pytest.raises(me.MEError) as e:
        me.Handle("gg_ttg", term_queues=3)
    assert e.value.code == me.ME_ERR_ARG


def test_served_requests_with_queues(me):
    """The request loop runs the per-term queues and the cuts of its parameters: the
    same numbers as a direct call."""
    c = CUTS["heavy"][1]
    b = synth.flat_points("gg_ttg", 2000, 12)
    direct = me.Handle("gg_ttg", precision=me.ME_PREC_FP64, term_queues=1, **_params(c)).real_subtracted(b.p)
    srv = me.Server(n_slots=2, precision=me.ME_PREC_FP64, term_queues=1, **_params(c))
    try:
        t = srv.submit("gg_ttg", "real_subtracted", b.p)
        r = srv.poll(t, timeout_us=60_000_000)
    finally:
        srv.close()
    assert r["status"] == me.ME_OK
    np.testing.assert_allclose(r["out"], direct, rtol=1e-13, atol=0)


def test_rescue_counts_of_the_queues_and_host_inputs(me):
    """The per-term path reports its float64 Born configurations by kind (their sum is
    the born_sets count of me_last_rescue_work; the masked path reports none), and host
    inputs read in place give the same numbers as device inputs."""
    b = synth.flat_points("gg_ttg", 3001, 78)
    hq = me.Handle("gg_ttg", precision=me.ME_PREC_MIXED, term_queues=1)
    got_dev = hq.real_subtracted(_dev(b.p)).cpu().numpy()
    pts, blocks, configs = hq.last_rescue_work()
    c0, c1 = hq.last_rescue_configs()
    assert pts == hq.last_rescued() > 0 and configs == c0 + c1 > 0 and blocks > 0
    pinned = torch.from_numpy(b.p).pin_memory()
    got_host = hq.real_subtracted(pinned.numpy())
    np.testing.assert_array_equal(got_host, got_dev)
    hm = me.Handle("gg_ttg", precision=me.ME_PREC_MIXED, term_queues=0)
    hm.real_subtracted(_dev(b.p))
    assert hm.last_rescue_configs() == (0, 0)
