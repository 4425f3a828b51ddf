"""The GPU schemes' critical Courant numbers (found by simulation, as the
paper's Sec. 4.7 does) agree with the oracle's Bloch-wave analysis and with
the paper's Table crit-Cr (3D, k = 1)."""
import pytest

pytestmark = pytest.mark.gpu


def test_crit_courant_k1_matches_oracle_and_paper():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03981_gb300 import crit_courant
    lsrk = crit_courant.critical(1, "lsrk", N=4, steps=1000)
    ader = crit_courant.critical(1, "ader", N=4, steps=1000)
    # oracle Bloch analysis (same criterion): 0.259 / 0.112; paper: 0.28 / 0.13
    assert abs(lsrk - 0.259) < 0.03, lsrk
    assert abs(ader - 0.112) < 0.02, ader
