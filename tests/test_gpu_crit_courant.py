"""The GPU schemes' critical Courant numbers (found by simulation, as the
paper's Sec. 4.7 does) agree with the oracle's Bloch-wave analysis, computed
here on the CPU with the same growth criterion, and with the paper's Table
crit-Cr (3D, k = 1), read from tests/golden/crit_courant_3d.txt."""
import pytest

import crit_courant as cc
from oracle import LSRK54_A, LSRK54_B
from test_oracle_crit_courant import golden
from test_oracle_timestep import stability_poly

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bloch_k1():
    b = cc.Bloch(1)
    g = stability_poly(LSRK54_A, LSRK54_B)
    lsrk = cc.bisect(lambda c: b.lsrk_stable(c, g), lo=0.05, hi=1.0, tol=2e-3)
    ader = cc.bisect(lambda c: b.ader_stable(c), lo=0.05, hi=0.4, tol=2e-3)
    return lsrk, ader


def test_crit_courant_k1_matches_oracle_and_paper(bloch_k1):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03981_gb300 import crit_courant
    lsrk = crit_courant.critical(1, "lsrk", N=4, steps=1000)
    ader = crit_courant.critical(1, "ader", N=4, steps=1000)
    o_lsrk, o_ader = bloch_k1
    assert abs(lsrk - o_lsrk) < 0.01, (lsrk, o_lsrk)
    assert abs(ader - o_ader) < 0.01, (ader, o_ader)
    paper = golden()[1]
    assert abs(ader - paper[2]) <= 0.15 * paper[2], (ader, paper)
    assert 0.8 * paper[0] <= lsrk <= 1.02 * paper[0], (lsrk, paper)
