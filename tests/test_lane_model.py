"""Host model of the packed lane words of the D->C Hungarian against the oracle.

The device kernel keeps, per column, a packed key, a word with the matched row
and that row's potential, and a 64-scaled column potential, all modulo 2^32,
with a sentinel column outside the LAP (Sec. 4.1: one Hungarian LAP per
concentration).  tests/lane_model.c performs the same word arithmetic on
arrays and is compared here with the oracle's Hungarian method on random
tiles with two dead columns (widths 3-64) and full LAPs (sizes 1-63), values
from heavy ties up to the largest entry the packed keys take: duals,
assignment, steps and relaxations equal; on arbitrary 32-bit entries every
run stops.  The GPU parity tests check the kernel itself.
"""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def model(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("lane_model") / "lane_model")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-o", exe, os.path.join(HERE, "lane_model.c"),
                           os.path.join(ROOT, "oracle", "rlt2_oracle.c"), "-lm"])
    return exe


@pytest.mark.parametrize("seed", [1, 2])
def test_lane_words_equal_oracle(model, seed):
    out = subprocess.run([model, "20000", str(seed)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "disagree 0, unbounded 0" in out.stdout, out.stdout
