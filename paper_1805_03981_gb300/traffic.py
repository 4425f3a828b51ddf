"""Measured DRAM traffic per kernel launch, recorded from ncu.

The traffic of a launch is ``dram__bytes_read.sum + dram__bytes_write.sum``
(one ncu pass, ``--clock-control none``).  A table of these figures lives in
``profiles/dram_traffic.txt``; each row names the workload, the precision,
the size, the degree, the storage basis, the kernel kind and that kernel's
elements per block it was taken on, and the table carries a SHA-256 digest of
the kernel sources and build script it was taken with (DIGEST_FILES).  ``lookup`` returns a
figure only when the digest of the sources as they are now equals the
table's and a row matches the launch configuration exactly: once a kernel
changes, its old counters no longer describe it.

Recording (the ncu CSV comes from ``ncu --metrics
dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
--print-units base --csv``)::

    python -m paper_1805_03981_gb300.traffic --csv launches.csv \\
        --workload curved_pulse --prec fp64 --size 32 --k 5 --basis g \\
        --tiling 5,5 --measured-size 24 --command "<the ncu command line>"

``--measured-size`` records a capture taken on a smaller mesh of the same
recipe (so that ncu holds a few GB at most) for the full size: every kernel
here moves a fixed number of bytes per element, so the bytes (and times)
scale by the ratio of element counts, (size / measured size)^3.
"""
import argparse
import csv
import hashlib
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
TABLE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
COLUMNS = ("workload", "prec", "size", "k", "basis", "kernel", "elements_per_block",
           "launches", "read_bytes", "write_bytes", "traffic_bytes", "avg_us")
NKEY = 7

# epilogue template argument of the operator kernels -> kernel kind
_EPI_KIND = {0: "operator", 1: "lsrk_stage", 2: "ader_update", 3: "lsrk_stage"}


# The sources that determine the code of the recorded kernels (the 3D operator
# and predictor launched one solve at a time) and the layout of their
# per-element data: the kernel bodies, their instantiation units, the 1D
# tables and strides (tables.h) and the build flags.  The geometry set-up
# (setup.cu) only fills values into layouts fixed there, so it is not part
# of the digest.  The launch configuration that matters is part of each row
# (elements per block).
DIGEST_FILES = ("dg_kernels.cuh", "kern_inst.cuh", "kern_f64_lo.cu", "kern_f64_hi.cu", "kern_f32_lo.cu",
                "kern_f32_hi.cu", "kern_tck_odd_f64.cu", "kern_tck_odd_f32.cu", "tckc.cuh",
                "kern_tckc_f64_lo.cu", "kern_tckc_f64_hi.cu", "kern_tckc_f32_lo.cu", "kern_tckc_f32_hi.cu",
                "tckn.cuh", "kern_tckn.cu", "tcki.cuh", "kern_tcki_f32.cu", "kern_lsrk2r_f64.cu",
                "kern_lsrk2r_f32.cu", "tables.h", "tables.cpp")


def sources_digest():
    """SHA-256 over the kernel-determining sources (DIGEST_FILES) and build.py."""
    h = hashlib.sha256()
    csrc = os.path.join(PKG, "csrc")
    files = [os.path.join(csrc, f) for f in DIGEST_FILES]
    files.append(os.path.join(PKG, "build.py"))
    for path in files:
        h.update(os.path.basename(path).encode())
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_kind(name):
    """Kind of a demangled kernel name, or None for kernels outside the path's kinds."""
    m = re.search(r"\b(op|opg|opga)_kernel<\s*\d+\s*,\s*\w+\s*,\s*(\d+)\s*>", name)
    if m:
        return _EPI_KIND.get(int(m.group(2)))
    if re.search(r"\btck[cni]?_kernel<", name):
        return "tck"
    return None


def parse_ncu_csv(path):
    """Per kernel kind: launches, mean read / write bytes and mean duration (us)."""
    launches = {}
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        kind = kernel_kind(row.get("Kernel Name", ""))
        if kind is None:
            continue
        rec = launches.setdefault((kind, row["ID"]), {})
        value = float(row["Metric Value"].replace(",", ""))
        unit = row.get("Metric Unit", "")
        scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9,
                 "ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3}.get(unit)
        if scale is None:
            raise ValueError("unexpected metric unit %r in %s" % (unit, path))
        rec[row["Metric Name"]] = value * scale
    out = {}
    for (kind, _), rec in launches.items():
        agg = out.setdefault(kind, [0, 0.0, 0.0, 0.0])
        agg[0] += 1
        agg[1] += rec["dram__bytes_read.sum"]
        agg[2] += rec["dram__bytes_write.sum"]
        agg[3] += rec.get("gpu__time_duration.sum", 0.0)
    return {kind: {"launches": n, "read_bytes": r / n, "write_bytes": w / n,
                   "traffic_bytes": (r + w) / n, "avg_us": t / n}
            for kind, (n, r, w, t) in out.items()}


def read_table(path=TABLE):
    """(digest, header comment lines, rows as dicts) of the traffic table."""
    if not os.path.exists(path):
        return None, [], []
    digest, comments, rows = None, [], []
    with open(path) as f:
        for ln in f:
            ln = ln.rstrip("\n")
            if ln.startswith("# sources_sha256:"):
                digest = ln.split(":", 1)[1].strip()
            elif ln.startswith("#") or not ln.strip():
                comments.append(ln)
            else:
                rows.append(dict(zip(COLUMNS, ln.split())))
    return digest, comments, rows


def _key(row):
    return tuple(str(row[c]) for c in COLUMNS[:NKEY])


def _epb(kernel, tiling):
    """Elements per block of a kernel kind under an (operator, predictor) tiling."""
    return tiling[1] if kernel == "tck" else tiling[0]


def lookup(workload, prec, size, k, basis, tiling, kernel, path=TABLE):
    """Traffic bytes per launch recorded for exactly this configuration and
    the current sources, else None."""
    digest, _, rows = read_table(path)
    if digest is None or digest != sources_digest():
        return None
    want = (workload, prec, str(size), str(k), basis, kernel, str(_epb(kernel, tiling)))
    for row in rows:
        if _key(row) == want:
            return float(row["traffic_bytes"])
    return None


def record(csv_path, workload, prec, size, k, basis, tiling, command, path=TABLE, measured_size=None):
    """Merge the kinds measured in one ncu CSV into the table.  Rows recorded
    with other sources are dropped, as they no longer describe the kernels.
    measured_size: the capture's mesh size when smaller than size (the
    figures are scaled by the ratio of element counts)."""
    digest = sources_digest()
    old_digest, comments, rows = read_table(path)
    if old_digest != digest:
        rows, comments = [], []
    measured = parse_ncu_csv(csv_path)
    if not measured:
        raise ValueError("no launches of the path's kernels in %s" % csv_path)
    if measured_size and measured_size != size:
        f = (float(size) / measured_size) ** 3
        for m in measured.values():
            for key in ("read_bytes", "write_bytes", "traffic_bytes", "avg_us"):
                m[key] *= f
        command = "%s   [taken at size %d, scaled by (%d/%d)^3]" % (command, measured_size, size, measured_size)
    for kind, m in sorted(measured.items()):
        row = {"workload": workload, "prec": prec, "size": size, "k": k, "basis": basis,
               "kernel": kind, "elements_per_block": _epb(kind, tiling),
               "launches": m["launches"], "read_bytes": "%.0f" % m["read_bytes"],
               "write_bytes": "%.0f" % m["write_bytes"],
               "traffic_bytes": "%.0f" % m["traffic_bytes"], "avg_us": "%.1f" % m["avg_us"]}
        rows = [r for r in rows if _key(r) != _key(row)]
        rows.append(row)
    cmd_line = "# command: " + command
    comments = [c for c in comments if c.startswith("# command:") and c != cmd_line]
    with open(path, "w") as f:
        f.write("# DRAM traffic per launch: dram__bytes_read.sum + dram__bytes_write.sum (bytes),\n"
                "# mean over the captured launches of each kind; avg_us is ncu's gpu__time_duration\n"
                "# (serialised, cold-cache).  One ncu pass, --clock-control none.\n")
        f.write("# sources_sha256: %s\n" % digest)
        for c in comments:
            f.write(c + "\n")
        f.write(cmd_line + "\n")
        f.write("# columns: " + " ".join(COLUMNS) + "\n")
        for r in sorted(rows, key=_key):
            f.write(" ".join(str(r[c]) for c in COLUMNS) + "\n")
    return measured


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--csv", required=True)
    ap.add_argument("--workload", required=True)
    ap.add_argument("--prec", required=True, choices=["fp64", "fp32"])
    ap.add_argument("--size", type=int, required=True)
    ap.add_argument("--k", type=int, required=True)
    ap.add_argument("--basis", required=True, choices=["g", "gl"])
    ap.add_argument("--tiling", required=True, help="op,tck elements per block")
    ap.add_argument("--command", required=True)
    ap.add_argument("--measured-size", type=int, default=0)
    ap.add_argument("--out", default=TABLE)
    a = ap.parse_args()
    tiling = tuple(int(x) for x in a.tiling.split(","))
    for kind, m in sorted(record(a.csv, a.workload, a.prec, a.size, a.k, a.basis, tiling,
                                 a.command, a.out, a.measured_size or None).items()):
        print("%-12s launches %3d  traffic %.4g B/launch  avg %.1f us"
              % (kind, m["launches"], m["traffic_bytes"], m["avg_us"]))


if __name__ == "__main__":
    main()
