"""The helicity blocks of the CUDA path are exact (CPU; no GPU needed).

A host build of the kernels' amplitude templates (csrc/me_blockcheck.cu) evaluates the
colour-summed |M|^2 of every process over all helicities one at a time, and over the
helicity blocks of one member of each flipped pair (doubled: |M(h)|^2 = |M(-h)|^2),
skipping the blocks that vanish by helicity conservation.  The two must agree to
rounding in float64 and float32, and the float64 value must equal the oracle's
Feynman-diagram result on the same points."""
import subprocess

import numpy as np
import pytest

import synth
from oracle import matrix_element as ome

PIDS = {"ee_uu": 0, "ee_uug": 1, "gg_tt": 2, "gg_ttg": 3, "gg_ttgg": 4, "uu_tt": 5, "uu_ttg": 6}


@pytest.fixture(scope="module")
def tool():
    from paper_2503_07439_gb300 import build
    try:
        return build.block_check_tool()
    except (RuntimeError, FileNotFoundError) as e:
        pytest.skip(f"CUDA toolchain unavailable: {e}")


@pytest.mark.parametrize("name", list(PIDS))
def test_blocks_equal_single_helicities_and_oracle(tool, name):
    n = 6 if name == "gg_ttgg" else 40
    b = synth.flat_points(name, n, 23)
    inp = f"{PIDS[name]} {n} {b.p.shape[1]}\n" + " ".join("%.17g" % x for x in b.p.reshape(-1)) + "\n"
    r = subprocess.run([tool], input=inp, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    v = np.array([[float(x) for x in line.split()] for line in r.stdout.split("\n") if line.strip()])
    assert v.shape == (n, 4)
    b64, s64, b32, s32 = v.T
    assert np.max(np.abs(b64 / s64 - 1)) < 1e-14
    assert np.max(np.abs(b32 / s32 - 1)) < 2e-6
    # the kernels' |M|^2 omits the initial spin and colour average
    avg = {"ee_uu": 4, "ee_uug": 4, "gg_tt": 256, "gg_ttg": 256, "gg_ttgg": 512, "uu_tt": 36, "uu_ttg": 36}[name]
    ref = ome.me2(name, ome.to_points(b.p))
    assert np.max(np.abs(b64 / avg / ref - 1)) < 1e-10
