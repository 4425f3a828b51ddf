"""The paper's operation-count model (Sec. 4.1) as restated in opcount.py,
checked against what the paper states about it."""
from paper_1805_03981_gb300 import opcount


def test_c_tensorial_even_odd_halves_the_plain_product():
    # the even-odd decomposition cuts a 1D matrix-vector product of (k+1)^2
    # multiply-adds (2 (k+1)^2 operations) to about one half
    for k in range(3, 13):
        plain = 2 * (k + 1) ** 2
        assert 0.45 < opcount.c_tensorial(k, 1) / plain < 0.75, k
    # one kernel on a delta-dimensional domain runs over (k+1)^(delta-1) lines
    for k in range(1, 13):
        assert opcount.c_tensorial(k, 3) == opcount.c_tensorial(k, 1) * (k + 1) ** 2


def test_ader_fewer_operations_than_five_stage_rk():
    # "ADER involves fewer arithmetic operations for all considered
    # polynomial degrees k in {1..12} for both d = 2, 3" (Sec. 4.1)
    for d in (2, 3):
        for k in range(1, 13):
            ops = opcount.paper_scheme_ops(k, d)
            assert ops["ader"] < ops["rk"], (d, k)


def test_predictor_share_grows_with_degree():
    # the predictor carries the extra dependency on k: its share of an ADER
    # step grows with the degree
    shares = [opcount.paper_scheme_ops(k)["tck"] / opcount.paper_scheme_ops(k)["ader"] for k in range(1, 13)]
    assert all(b > a for a, b in zip(shares, shares[1:]))


def test_predictor_without_basis_change_costs_more():
    """Alg. 1 (projection in the GL basis for every derivative) costs more
    than Alg. 2 with the on-the-fly basis change, which costs more than
    Alg. 2 with degree reduction every second derivative (Secs. 3.2-3.3),
    and the gap widens with the degree."""
    ratios = []
    for n in range(2, 9):
        a1, a2, a23 = (opcount.tck_flops_alg1(n), opcount.tck_flops(n, 0, "gl"), opcount.tck_flops(n, 2, "g"))
        assert a1 > a2 > a23, n
        ratios.append(a1 / a23)
    assert all(b > a for a, b in zip(ratios, ratios[1:]))


def test_bench_roofline_counts():
    """The algorithmic counts behind the bench's roofline figures: the LSRK
    stage of the default workload (curved pulse 32^3, k=5, FP64,
    Gauss-point states) moves 1.87 GB and 2.59 GFLOP per launch (four state
    vectors, the per-point geometry, connectivity; the operator with the
    stage update, walls on the cube's boundary faces), and that of the
    FP32 plane wave 64^3 at k=4 (affine compact data) 2.16 GB and 10.2 GFLOP."""
    E = 32 ** 3
    assert opcount.bytes_per_element("lsrk_stage", 6, 8, 2, affine=False) * E == 1869742080
    assert round(opcount.flops_per_element("lsrk_stage", 6, 2, 1.0 - 1.0 / 32, "g", False) * E) == 2586968064
    E = 64 ** 3
    assert opcount.bytes_per_element("lsrk_stage", 5, 4, 2, affine=True) * E == 2156920832
    assert round(opcount.flops_per_element("lsrk_stage", 5, 2, 1.0, "g", True) * E) == 10243276800
