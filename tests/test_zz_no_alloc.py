"""The allocation-free entry point gives the same weights as the handle-based entry
point.  It exists for callers that cannot allocate GPU memory: applications whose
device memory belongs to another allocator (a caching pool), code that must not trigger
the device-wide synchronisation of cudaMalloc/cudaFree, and code running where
allocation is not permitted.  Called through the C ABI directly, for all three processes
with FKS sectors in an interleaved order, twice in a row, so that each call runs on the
built-in scratch and tables the previous call (for another process) left behind."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PROCESSES = [("ee_uug", 23), ("gg_ttg", 21), ("uu_ttg", 22)]
# two rounds in different orders: every process follows a different one each time
ORDER = ["gg_ttg", "ee_uug", "uu_ttg", "uu_ttg", "gg_ttg", "ee_uug"]


@pytest.fixture(scope="module")
def me():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_07439_gb300 as m
    return m


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_noalloc_matches_handle_interleaved(me, precision):
    prec = me.ME_PREC_MIXED if precision == "mixed" else me.ME_PREC_FP64
    lib = me.library()
    data, ref = {}, {}
    for name, seed in PROCESSES:
        b = synth.flat_points(name, 4099, seed)
        p = torch.from_numpy(b.p).cuda()
        w = torch.from_numpy(b.wgt).cuda()
        h = me.Handle(name, precision=prec, lanes_per_event=4)
        ref[name] = h.real_subtracted(p, w).cpu().numpy()
        h.close()
        data[name] = (b.n, p, w)
    params = me.default_params(precision=prec, lanes_per_event=4)
    for name in ORDER:
        n, p, w = data[name]
        out = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        rc = lib.me_eval_real_subtracted_noalloc(name.encode(), ctypes.byref(params), p.data_ptr(), w.data_ptr(),
                                                 n, out.data_ptr(), None)
        assert rc == me.ME_OK, lib.me_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        r = ref[name]
        rel = np.abs(got - r) / np.abs(r)
        # the tolerance of the mixed-precision parity tests: 1e-5 relative on 99.9% of
        # points; the same kernels on the same points in float64 agree to rounding
        assert np.all(np.isfinite(got)), name
        assert np.quantile(rel, 0.999) <= 1e-5, (name, np.quantile(rel, 0.999))
        assert np.max(rel) <= (1e-3 if prec == me.ME_PREC_MIXED else 1e-12), (name, np.max(rel))


def test_noalloc_rejects_oversize_and_host_buffers(me):
    lib = me.library()
    params = me.default_params(precision=me.ME_PREC_MIXED)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.me_eval_real_subtracted_noalloc(b"gg_ttg", ctypes.byref(params), x.data_ptr(), None,
                                             (1 << 20) + 1, x.data_ptr(), None)
    assert rc == me.ME_ERR_ARG
    host = np.zeros(4 * 5 * 8)
    rc = lib.me_eval_real_subtracted_noalloc(b"gg_ttg", ctypes.byref(params), host.ctypes.data, None, 8,
                                             x.data_ptr(), None)
    assert rc == me.ME_ERR_ARG
    rc = lib.me_eval_real_subtracted_noalloc(b"gg_tt", ctypes.byref(params), x.data_ptr(), None, 1,
                                             x.data_ptr(), None)
    assert rc == me.ME_ERR_PROCESS


def test_noalloc_keeps_the_callers_current_device(me):
    """The call switches to params->device for its work and switches back afterwards."""
    lib = me.library()
    params = me.default_params(precision=me.ME_PREC_FP64)
    b = synth.flat_points("gg_ttg", 33, 24)
    p = torch.from_numpy(b.p).cuda()
    out = torch.empty(b.n, dtype=torch.float64, device="cuda")
    before = torch.cuda.current_device()
    rc = lib.me_eval_real_subtracted_noalloc(b"gg_ttg", ctypes.byref(params), p.data_ptr(), None, b.n,
                                             out.data_ptr(), None)
    assert rc == me.ME_OK, lib.me_last_error()
    assert torch.cuda.current_device() == before


def test_noalloc_applies_the_cuts(me):
    """The cuts of the parameters reach the allocation-free entry too: with heavy-quark
    cuts its weights equal those of a handle with the same cuts (the masked evaluation),
    exact zeros included."""
    lib = me.library()
    cuts = dict(cut_pt_min=100.0, cut_abs_y_max=1.0)
    b = synth.flat_points("gg_ttg", 2053, 27)
    p = torch.from_numpy(b.p).cuda()
    ref = me.Handle("gg_ttg", precision=me.ME_PREC_FP64, term_queues=0, **cuts).real_subtracted(p).cpu().numpy()
    params = me.default_params(precision=me.ME_PREC_FP64, **cuts)
    out = torch.full((b.n,), np.nan, dtype=torch.float64, device="cuda")
    rc = lib.me_eval_real_subtracted_noalloc(b"gg_ttg", ctypes.byref(params), p.data_ptr(), None, b.n,
                                             out.data_ptr(), None)
    assert rc == me.ME_OK, lib.me_last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    z = ref == 0.0
    assert 0.05 < z.mean() < 0.95 and np.all(got[z] == 0.0)
    rel = np.abs(got[~z] - ref[~z]) / np.abs(ref[~z])
    assert np.quantile(rel, 0.999) <= 1e-11 and rel.max() <= 1e-8
