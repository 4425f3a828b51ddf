"""Host logic of the autotuner's table: lookup by precision, degree and
size class, and what apply sets on a solver (no GPU: a stand-in solver
records the calls)."""
from paper_1805_03981_gb300 import _lib, autotune


class FakeSolver:
    def __init__(self, prec, k, E, affine):
        self.prec, self.k, self.E, self._affine = prec, k, E, affine
        self.calls = []

    def set_tiling(self, op, tck):
        self.calls.append(("tiling", op, tck))

    def tiling(self):
        return [c for c in self.calls if c[0] == "tiling"][-1][1:]

    def set_predictor_kernel(self, kind):
        self.calls.append(("pred", kind))

    def is_affine(self):
        return self._affine


TABLE = {"fp32": {"4": {"small": {"epb_op": 3, "epb_tck": 2, "pred": "columns"},
                        "large": {"epb_op": 5, "epb_tck": 4, "pred": "lines"}}},
         "fp64": {"4": {"small": {"epb_op": 1, "epb_tck": 1}}}}   # a table without the form


def test_lookup_by_size_class_and_missing_entries():
    assert autotune.lookup(TABLE, "fp32", 4, 100) == (3, 2, "columns")
    assert autotune.lookup(TABLE, "fp32", 4, autotune.SMALL_LIMIT + 1) == (5, 4, "lines")
    assert autotune.lookup(TABLE, "fp64", 4, 10) == (1, 1, None)
    assert autotune.lookup(TABLE, "fp32", 5, 10) is None
    assert autotune.lookup(None, "fp32", 4, 10) is None


def test_apply_sets_tiling_and_form_except_on_affine_solvers():
    s = FakeSolver(_lib.DG_FP32, 4, 100, affine=False)
    assert autotune.apply(s, TABLE) == (3, 2)
    assert ("pred", _lib.PRED_COLUMNS) in s.calls
    s = FakeSolver(_lib.DG_FP32, 4, 10 ** 5, affine=False)
    autotune.apply(s, TABLE)
    assert ("pred", _lib.PRED_LINES) in s.calls
    s = FakeSolver(_lib.DG_FP32, 4, 100, affine=True)           # keeps the interleaved default
    autotune.apply(s, TABLE)
    assert [c for c in s.calls if c[0] == "pred"] == []
    s = FakeSolver(_lib.DG_FP64, 4, 100, affine=False)          # old table: tiling only
    autotune.apply(s, TABLE)
    assert s.calls == [("tiling", 1, 1)]
