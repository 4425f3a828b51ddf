"""Autotuner for the tiling of the kernels and the form of the predictor.

For each precision, degree k and size class it builds a seeded synthetic
instance (curved cube, variable coefficients) with Gauss-point states (the
kernels the steppers, batches and the server run), measures every candidate
number of elements per thread block with dg_tune (device time per launch of
the LSRK-stage operator, the ADER-update operator and the predictor), the
predictor in both its line and its column form, and records the fastest.
The table is a JSON file keyed by GPU name; solvers created later pick
their tiling, and on curved or variable-coefficient meshes their predictor
form, from it with ``apply`` (on affine meshes with constant coefficients
the default interleaved form stays).  Tiling never changes results; the
two predictor forms take the same sums in another order, so the form
changes them at rounding level only.

    python -m paper_1805_03981_gb300.autotune [--out PATH] [--prec fp32,fp64] [--k 1-7]
"""
import argparse
import json
import os

CANDIDATES = [1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32]
SIZE_CLASSES = {"small": 4, "large": 12}       # elements per axis of the tuning mesh
SMALL_LIMIT = 4096                              # meshes up to this many elements use "small"
DEFAULT_PATH = os.environ.get("DG_AUTOTUNE_CACHE",
                              os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json"))


def gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def size_class(n_elem):
    return "small" if n_elem <= SMALL_LIMIT else "large"


def tune(precs=("fp32", "fp64"), ks=range(1, 8), reps=3, seed=7):
    import synth
    from . import _lib
    out = {}
    for pname in precs:
        prec = _lib.DG_FP64 if pname == "fp64" else _lib.DG_FP32
        for k in ks:
            for cls, N in SIZE_CLASSES.items():
                cfg = synth.configs.random_instance(seed, N=N, k=k, nsteps=1)
                s = _lib.Solver(cfg["mesh"], k, prec, 1.0, cfg["rho"], cfg["c"])
                s.set_basis(_lib.BASIS_G)
                res = {}
                runs = [(_lib.KIND_LSRK, "lsrk", None), (_lib.KIND_ADER, "ader", None),
                        (_lib.KIND_TCK, "tck_lines", _lib.PRED_LINES), (_lib.KIND_TCK, "tck_columns", _lib.PRED_COLUMNS)]
                for kind, name, pred in runs:
                    if pred is not None:
                        s.set_predictor_kernel(pred)
                    ms = s.tune(kind, CANDIDATES, reps)
                    ok = [(m, c) for m, c in zip(ms, CANDIDATES) if m > 0]
                    best = min(ok)
                    res[name] = {"epb": best[1], "ms": best[0],
                                 "all": {str(c): round(m, 5) for m, c in ok}}
                # the operator serves both LSRK and ADER: favour LSRK's choice
                res["epb_op"] = res["lsrk"]["epb"]
                form = "columns" if res["tck_columns"]["ms"] < res["tck_lines"]["ms"] else "lines"
                res["tck"] = dict(res["tck_" + form], pred=form)
                res["epb_tck"] = res["tck"]["epb"]
                res["pred"] = form
                out.setdefault(pname, {}).setdefault(str(k), {})[cls] = res
                s.close()
    return out


def save(table, path=DEFAULT_PATH):
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[gpu_name()] = table
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    return path


def load(path=DEFAULT_PATH):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    return data.get(gpu_name())


def lookup(table, prec_name, k, n_elem):
    """(epb_op, epb_tck, predictor form or None) for this case, or None."""
    try:
        r = table[prec_name][str(k)][size_class(n_elem)]
        return r["epb_op"], r["epb_tck"], r.get("pred")
    except (KeyError, TypeError):
        return None


def apply(solver, table):
    """Set the solver's tiling, and its predictor form unless its elements
    are affine with constant coefficients, from the table; returns the
    tiling used."""
    from . import _lib
    pname = "fp64" if solver.prec == _lib.DG_FP64 else "fp32"
    t = lookup(table, pname, solver.k, solver.E) if table else None
    if t:
        solver.set_tiling(t[0], t[1])
        if t[2] and not solver.is_affine():
            solver.set_predictor_kernel(_lib.PRED_COLUMNS if t[2] == "columns" else _lib.PRED_LINES)
    return solver.tiling()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--prec", default="fp32,fp64")
    ap.add_argument("--k", default="1-7")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    lo, hi = (int(x) for x in a.k.split("-")) if "-" in a.k else (int(a.k), int(a.k))
    table = tune(a.prec.split(","), range(lo, hi + 1), a.reps)
    print(save(table, a.out))
    print(json.dumps({p: {k: {c: (v["epb_op"], v["epb_tck"], v["pred"]) for c, v in kk.items()}
                          for k, kk in t.items()} for p, t in table.items()}))


if __name__ == "__main__":
    main()
