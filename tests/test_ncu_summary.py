"""Host logic of the ncu helpers: launch-list summary and the DRAM traffic record that
bench.py reports next to the roofline (no GPU; small ncu-format CSV files written here)."""
import csv
import json

import pytest

import ncu_summary as ns


def _write(path, rows):
    with open(path, "w", newline="") as fh:
        fh.write("==PROF== Connected to process 1\n")
        csv.writer(fh, quoting=csv.QUOTE_ALL).writerows(rows)


K1 = "void wdb::(anonymous namespace)::tile_kernel<float, (int)2, (bool)0>(wdb::TileArgs, const T1 *, T1 *, E)"
K2 = "void wdb::(anonymous namespace)::tile_kernel<float, (int)3, (bool)0>(wdb::TileArgs, const T1 *, T1 *, E)"
K4 = "void wdb::(anonymous namespace)::tile_kernel<float, (int)4, (bool)0>(wdb::TileArgs, const T1 *, T1 *, E)"


def _metrics_log(path):
    head = ["ID", "Process ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]
    rows = [head]
    # a kernel that must not be taken for kernel 1 or 2, then two launches of each
    for lid, (k, rd, wr, t) in enumerate([(K4, 1, 1, 1), (K1, 1000, 24, 45000), (K2, 2000, 0, 59.5),
                                          (K1, 9, 9, 9), (K2, 9, 9, 9)]):
        rows.append([str(lid), "1", k, "dram__bytes_read.sum", "Kbyte", str(rd)])
        rows.append([str(lid), "1", k, "dram__bytes_write.sum", "byte", str(wr)])
        rows.append([str(lid), "1", k, "gpu__time_duration.sum", "ns" if k == K1 else "us", str(t)])
    _write(path, rows)


def test_fista_dram_first_launch_and_units(tmp_path):
    p = tmp_path / "log.csv"
    _metrics_log(p)
    got = ns.fista_dram(str(p))
    assert set(got) == {"k1_residual", "k2_step"}
    assert got["k1_residual"]["dram__bytes_read.sum"] == 1e6       # Kbyte -> bytes
    assert got["k1_residual"]["dram__bytes_write.sum"] == 24
    assert got["k1_residual"]["gpu__time_duration.sum"] == pytest.approx(45.0)   # ns -> us
    assert got["k2_step"]["dram__bytes_read.sum"] == 2e6
    assert got["k2_step"]["gpu__time_duration.sum"] == pytest.approx(59.5)
    assert got["k1_residual"]["kernel"] == "tile_kernel<float, 2, 0>"


def test_launch_summary_counts_time_rows_only(tmp_path):
    # a metrics log with three metrics per launch: launches and shares come from the
    # duration rows alone, in their own units
    p = tmp_path / "log.csv"
    _metrics_log(p)
    out = ns.summarise(str(p))
    assert "5 launches" in out
    shares = sorted(float(ln.split()[-1].rstrip("%")) for ln in out.splitlines()[2:])
    total = 1000 + 45009 + 68500          # ns: K4 1 us, K1 45000 + 9 ns, K2 59.5 + 9 us
    assert shares == pytest.approx(sorted([100 * 1000 / total, 100 * 45009 / total, 100 * 68500 / total]), abs=0.05)


def test_fista_dram_raw_page(tmp_path):
    p = tmp_path / "raw.csv"
    head = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum"]
    units = ["", "", "Mbyte", "Mbyte", "usecond"]
    _write(p, [head, units, ["0", K1, "80.5", "29", "470.1"], ["1", K2, "185", "79", "485"]])
    got = ns.fista_dram(str(p))
    assert got["k1_residual"]["dram__bytes_read.sum"] == pytest.approx(80.5e6)
    assert got["k2_step"]["dram__bytes_write.sum"] == pytest.approx(79e6)
    assert got["k2_step"]["gpu__time_duration.sum"] == pytest.approx(485)


def test_write_traffic_record_and_source_hash(tmp_path):
    p = tmp_path / "log.csv"
    _metrics_log(p)
    rec = tmp_path / "traffic.json"
    ns.write_traffic(str(p), "1024", "profiles/x.md", str(rec))
    r = json.loads(rec.read_text())
    e = r["1024"]["k1_residual"]
    assert e["dram_bytes_per_launch"] == 1000024
    assert e["sources"] == ns.TILE_SOURCES
    assert e["sources_sha256"] == ns.kernel_sources_sha256(ns.TILE_SOURCES)
    # the hash covers the file names and contents in sorted order
    assert ns.kernel_sources_sha256(list(reversed(ns.TILE_SOURCES))) == e["sources_sha256"]
    assert ns.kernel_sources_sha256(ns.TILE_SOURCES[:-1]) != e["sources_sha256"]


def test_launch_list_summary(tmp_path):
    p = tmp_path / "launches.csv"
    head = ["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]
    rows = [head, ["0", K1, "gpu__time_duration.sum", "usecond", "30"],
            ["1", K2, "gpu__time_duration.sum", "nsecond", "10000"],
            ["2", K1, "gpu__time_duration.sum", "usecond", "60"]]
    _write(p, rows)
    out = ns.summarise(str(p))
    lines = out.splitlines()
    assert "3 launches, 100.0 us" in lines[0]
    k1 = next(l for l in lines if "tile_kernel<float, (int)2" in l or "tile_kernel<float, 2" in l)
    assert k1.split()[-3:] == ["2", "90.0", "90.0%"]
