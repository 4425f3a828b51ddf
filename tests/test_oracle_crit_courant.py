"""Pin against the paper's printed critical Courant numbers (Table crit-Cr,
Sec. 4.7, 3D Cartesian mesh), stored in tests/golden/crit_courant_3d.txt.

ADER (Eq. (6) with Algorithm 3) is compared at 15%.  The paper's LSRK4(5) is
a different 2R scheme from the 2N scheme built here, so LSRK is held to the
ballpark (20%, and below the paper's value since the 2N scheme's stability
region is smaller).
"""
import os

import numpy as np
import pytest

from oracle import LSRK54_A, LSRK54_B
import crit_courant as cc
from test_oracle_timestep import stability_poly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "crit_courant_3d.txt")


def golden():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, a, b, c = line.split()
            rows[int(k)] = (float(a), float(b), float(c))
    return rows


@pytest.fixture(scope="module", params=[1, 4])
def bloch(request):
    return cc.Bloch(request.param)


def test_lsrk_crit_courant_ballpark(bloch):
    ref = golden()[bloch.k][0]
    g = stability_poly(LSRK54_A, LSRK54_B)
    cr = cc.bisect(lambda c: bloch.lsrk_stable(c, g), lo=0.05, hi=1.0, tol=2e-3)
    assert 0.8 * ref <= cr <= 1.02 * ref, (bloch.k, cr, ref)


def test_ader_crit_courant(bloch):
    ref = golden()[bloch.k][2]
    cr = cc.bisect(lambda c: bloch.ader_stable(c), lo=0.05, hi=0.4, tol=4e-3)
    assert abs(cr - ref) <= 0.15 * ref, (bloch.k, cr, ref)
