"""Device-side phase space (me_generate_flat): Philox4x32-10 + RAMBO on the GPU gives the
same points and weights as the seeded host generator, and the generated points evaluate
like host-generated ones."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SQRT_S = {"ee_uu": 100.0, "ee_uug": 100.0, "gg_tt": 1000.0, "gg_ttg": 1000.0, "gg_ttgg": 2000.0,
          "uu_tt": 1000.0, "uu_ttg": 1000.0}


@pytest.fixture(scope="module")
def me():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_07439_gb300 as m
    return m


@pytest.mark.parametrize("name", list(SQRT_S))
def test_device_points_match_host_generator(me, name):
    n, seed, first, stream = 4099, 4, 12345, 3
    h = me.Handle(name, precision=me.ME_PREC_MIXED)
    p, w = h.generate_flat(n, seed, SQRT_S[name], first_point=first, stream=stream)
    ref = synth.flat_points(name, n, seed, first_point=first, stream=stream)
    got = p.cpu().numpy()
    # momenta to a few ulps of sqrt(s) (device log/sin/cos/sqrt vs the host library),
    # amplified by RAMBO's own conditioning: the boost to the centre of mass divides by
    # M = sqrt(Q^2) of the summed massless vectors, so (Q0/M)^2 magnifies rounding
    nout = p.shape[1] - 2
    u = synth.uniforms(seed, stream, n, 4 * nout, first)
    q0 = -np.log(u[2::4] * u[3::4])
    c = 2.0 * u[0::4] - 1.0
    s_ = np.sqrt(1.0 - c * c)
    f = 2.0 * np.pi * u[1::4]
    Q = np.stack([q0.sum(0), (q0 * s_ * np.cos(f)).sum(0), (q0 * s_ * np.sin(f)).sum(0), (q0 * c).sum(0)])
    cond = Q[0] ** 2 / (Q[0] ** 2 - (Q[1:] ** 2).sum(0))
    tol = 1e-14 * SQRT_S[name] * np.maximum(10.0, cond)
    assert np.all(np.abs(got - ref.p) <= tol[None, None, :])
    np.testing.assert_allclose(w.cpu().numpy(), ref.wgt, rtol=1e-12)


def test_generated_points_evaluate_like_host_points(me):
    n = 20000
    h = me.Handle("gg_ttg", precision=me.ME_PREC_FP64)
    p, w = h.generate_flat(n, 7, 1000.0)
    ref = synth.flat_points("gg_ttg", n, 7)
    a = h.real_subtracted(p, w).cpu().numpy()
    b = h.real_subtracted(torch.from_numpy(ref.p).cuda(), torch.from_numpy(ref.wgt).cuda()).cpu().numpy()
    # the points differ at the 1e-16 level; the weights then agree to far better than the
    # mixed-precision target (subtraction cancellations stay below 1e5 on flat points)
    assert np.quantile(np.abs(a - b) / np.abs(b), 0.999) < 1e-9


def test_bad_arguments(me):
    h = me.Handle("gg_tt", precision=me.ME_PREC_MIXED)
    with pytest.raises(me.MEError):
        h.generate_flat(16, 1, 300.0)  # below the t tbar threshold
    host = np.zeros((4, 4, 8))
    rc = h.lib.me_generate_flat(h.h, 1, 0, 0, 1000.0, 8, host.ctypes.data, None)
    assert rc == me.ME_ERR_ARG  # host memory is rejected


@pytest.mark.parametrize("name", ["ee_uug", "gg_ttg", "uu_ttg"])
def test_fks_points_match_host_generator(me, name):
    """Points generated on the device in FKS-sector variables (me_generate_fks) equal the
    host restatement (synth.fks_points): momenta to a few ulps of sqrt(s), weights to
    1e-12 (device sin/cos/sqrt against the host library; the final-state weight depends
    on the cosines of the gluon with both partons, computed from the momenta)."""
    n, seed, first, stream = 4099, 9, 777, 5
    h = me.Handle(name, precision=me.ME_PREC_MIXED)
    p, w = h.generate_fks(n, seed, SQRT_S[name], first_point=first, stream=stream)
    ref = synth.fks_points(name, n, seed, first_point=first, stream=stream)
    assert np.all(np.abs(p.cpu().numpy() - ref.p) <= 1e-13 * SQRT_S[name])
    # the weight's collinear density 1/sqrt(1 - y_j) is taken at cosines recomputed from
    # the momenta: a rounding of the momenta moves it by ~ 2^-53 / (1 - y_j) relative
    g = ref.p[1:, 4] / np.linalg.norm(ref.p[1:, 4], axis=0)
    omy = np.ones(n)
    for leg in ((2, 3) if name == "ee_uug" else (0, 1)):
        kj = ref.p[1:, leg] / np.linalg.norm(ref.p[1:, leg], axis=0)
        omy = np.minimum(omy, 1.0 - (g * kj).sum(axis=0))
    tol = 1e-12 * np.maximum(10.0, 10.0 / np.maximum(omy, 1e-300))
    rel = np.abs(w.cpu().numpy() / ref.wgt - 1)
    assert np.all(rel <= tol), np.max(rel / tol)


@pytest.mark.parametrize("name,flat_seed", [("ee_uug", 2), ("gg_ttg", 4)])
def test_fks_points_reduce_the_monte_carlo_error(me, name, flat_seed):
    """The same integral (the subtracted real over 2^20 points, mixed precision) from flat
    RAMBO points and from points sampled in FKS variables: the two estimates agree within
    their combined errors, and the FKS-variable sampling has the smaller standard error
    (the soft region sampled flat in xi, the collinear ones with density ~ 1/sqrt(1-y))."""
    n = 1 << 20
    h = me.Handle(name, precision=me.ME_PREC_MIXED)
    res = {}
    for gen in ("flat", "fks"):
        p, w = (h.generate_flat if gen == "flat" else h.generate_fks)(n, flat_seed, SQRT_S[name])
        x = h.real_subtracted(p, w).cpu().numpy()
        res[gen] = (x.mean(), x.std() / np.sqrt(n))
    (mf, ef), (mk, ek) = res["flat"], res["fks"]
    assert abs(mf - mk) <= 4.0 * np.hypot(ef, ek), res
    assert ek < 0.95 * ef, res


def test_fks_points_bad_process(me):
    h = me.Handle("gg_tt", precision=me.ME_PREC_MIXED)
    with pytest.raises(me.MEError) as e:
        h.generate_fks(16, 1, 1000.0)
    assert e.value.code == me.ME_ERR_PROCESS
