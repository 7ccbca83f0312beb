"""The algorithmic operation counts behind the bench's roofline fractions (the host
program csrc/me_flops.cu, built with nvcc's host compiler, no GPU): the per-term queues'
Born configurations add up to the Born part of the masked evaluation."""
import pytest


@pytest.fixture(scope="module")
def ops():
    from paper_2503_07439_gb300 import build as b
    return b.op_counts()


def test_counts_are_consistent(ops):
    real, born, sub = ops["born_per_event"], ops["born_per_event"], ops["real_subtracted_per_event"]
    cfg = ops["term_config_per_event"]
    # subtracted real = real-emission |M|^2 + the counterterms' Born values
    for name, b2 in (("ee_uug", "ee_uu"), ("uu_ttg", "uu_tt"), ("gg_ttg", "gg_tt")):
        born_set = sub[name] - real[name]
        assert born_set > born[b2]
        soft, coll = cfg[name]
        if name == "gg_ttg":
            # the masked evaluation computes both sectors' spin-correlated Borns; a
            # collinear configuration of the queues only the active sector's
            assert 0 < born_set - (soft + coll) < born[b2]
        else:
            assert soft + coll == born_set
    # every count is per event of the processes' helicity sums
    nh = {"ee_uu": 16, "ee_uug": 32, "gg_tt": 16, "gg_ttg": 32, "gg_ttgg": 64, "uu_tt": 16, "uu_ttg": 32}
    for name, h in nh.items():
        assert abs(ops["per_helicity"][name] - 2 * born[name] / h) <= 1.0
