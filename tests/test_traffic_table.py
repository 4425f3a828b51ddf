"""The ncu traffic table: parsing, recording and the source-digest guard.

The table feeds ``roofline.traffic`` of the bench line; a figure must only
come back for the exact launch configuration and the sources it was taken
with.
"""
import os

from paper_1805_03981_gb300 import traffic

HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
          '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
          '"Metric Value"\n')


def _row(i, name, metric, unit, value):
    return ('"%d","1","python3.12","h","%s","1","7","(180, 1, 1)","(100, 1, 1)","0","10.3",'
            '"Command line profiler metrics","%s","%s","%s"\n' % (i, name, metric, unit, value))


def _csv(tmp_path):
    lines = ["==PROF== Connected to process 1\n", HEADER]
    launches = [
        (0, "void opg_kernel<6, double, 1>(OpParams)", 1000, 500, 2000),
        (1, "void opg_kernel<6, double, 1>(OpParams)", 3000, 500, 4000),
        (2, "void opg_kernel<6, double, 2>(OpParams)", 800, 400, 1500),
        (3, "void tck_kernel<6, double, 2>(TckParams)", 600, 200, 3000),
        (4, "void basis_kernel<6, double>(void *, int, int)", 9, 9, 9),
    ]
    for i, name, rd, wr, ns in launches:
        lines.append(_row(i, name, "dram__bytes_read.sum", "byte", "{:,}".format(rd)))
        lines.append(_row(i, name, "dram__bytes_write.sum", "byte", wr))
        lines.append(_row(i, name, "gpu__time_duration.sum", "ns", ns))
    path = tmp_path / "launches.csv"
    path.write_text("".join(lines))
    return str(path)


def test_kernel_kinds():
    assert traffic.kernel_kind("void opg_kernel<6, double, 1>(OpParams)") == "lsrk_stage"
    assert traffic.kernel_kind("void op_kernel<4, float, 2>(OpParams)") == "ader_update"
    assert traffic.kernel_kind("void opga_kernel<5, float, 0>(OpParams)") == "operator"
    assert traffic.kernel_kind("void tck_kernel<6, double, 2>(TckParams)") == "tck"
    assert traffic.kernel_kind("void basis_kernel<6, double>(void *, int, int)") is None


def test_parse_means_per_kind(tmp_path):
    m = traffic.parse_ncu_csv(_csv(tmp_path))
    assert set(m) == {"lsrk_stage", "ader_update", "tck"}
    assert m["lsrk_stage"]["launches"] == 2
    assert m["lsrk_stage"]["read_bytes"] == 2000
    assert m["lsrk_stage"]["traffic_bytes"] == 2500
    assert m["lsrk_stage"]["avg_us"] == 3.0
    assert m["tck"]["traffic_bytes"] == 800


def test_record_and_lookup(tmp_path):
    table = str(tmp_path / "dram_traffic.txt")
    traffic.record(_csv(tmp_path), "curved_pulse", "fp64", 32, 5, "g", (5, 4), "ncu ...", table)
    look = lambda kernel, tiling: traffic.lookup("curved_pulse", "fp64", 32, 5, "g", tiling, kernel, table)
    assert look("lsrk_stage", (5, 4)) == 2500
    assert look("tck", (5, 4)) == 800
    # each kind is keyed on its own kernel's elements per block
    assert look("lsrk_stage", (5, 9)) == 2500
    assert look("tck", (9, 4)) == 800
    assert look("lsrk_stage", (6, 4)) is None
    assert traffic.lookup("curved_pulse", "fp32", 32, 5, "g", (5, 4), "lsrk_stage", table) is None
    # a second capture at another tiling adds rows and keeps the first
    traffic.record(_csv(tmp_path), "curved_pulse", "fp64", 32, 5, "g", (6, 6), "ncu -x", table)
    assert look("lsrk_stage", (6, 6)) == 2500 and look("lsrk_stage", (5, 5)) == 2500
    text = open(table).read()
    assert "# command: ncu ..." in text and "# command: ncu -x" in text


def test_digest_guard(tmp_path):
    table = str(tmp_path / "dram_traffic.txt")
    traffic.record(_csv(tmp_path), "curved_pulse", "fp64", 32, 5, "g", (5, 5), "ncu", table)
    text = open(table).read()
    digest = traffic.sources_digest()
    assert digest in text
    with open(table, "w") as f:
        f.write(text.replace(digest, "0" * 64))
    assert traffic.lookup("curved_pulse", "fp64", 32, 5, "g", (5, 5), "lsrk_stage", table) is None


def test_missing_table_gives_none(tmp_path):
    assert traffic.lookup("curved_pulse", "fp64", 32, 5, "g", (5, 5), "lsrk_stage",
                          str(tmp_path / "absent.txt")) is None
    assert os.path.basename(traffic.TABLE) == "dram_traffic.txt"
