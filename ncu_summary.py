"""ncu output helpers.

Summarise a launch list (--metrics gpu__time_duration.sum --csv) per kernel: launches,
total device time and share, split by NVTX range when ncu recorded one:

    python -m ncu_summary launches.csv

Record the DRAM bytes per launch of the FISTA kernels (circulant or row-varying) from a capture that holds
dram__bytes_read.sum and dram__bytes_write.sum (the first launch of each kernel), with the
hash of the sources they were compiled from, in profiles/traffic.json (bench.py reports the
record only while the sources still hash the same):

    ncu -i capture.ncu-rep --page raw --csv > raw.csv      (or an ncu --csv metrics log)
    python -m ncu_summary traffic raw.csv 4096 profiles/tile_kernels_4096_full.md
"""
from __future__ import annotations

import csv
import hashlib
import json
import os
import re
import sys
from collections import defaultdict

CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1512_08401_gb300", "csrc")
TILE_SOURCES = ["tile.cu", "tile.cuh", "device_util.cuh", "layout_types.h", "wdb_internal.h"]
VROW_SOURCES = ["vtheta.cu", "vtheta.h", "device_util.cuh", "layout_types.h", "wdb_internal.h"]
# name prefixes of the FISTA kernels: tile_kernel<float, EPI, ...> (circulant Theta_K) and
# vrow_kernel<float, EPI> (row-varying Theta_K)
FISTA_KERNELS = {"k1_residual": "tile_kernel<float, 2", "k2_step": "tile_kernel<float, 3",
                 "vk1_residual": "vrow_kernel<float, 1", "vk2_step": "vrow_kernel<float, 2"}
KERNEL_SOURCES = {"k1_residual": TILE_SOURCES, "k2_step": TILE_SOURCES,
                  "vk1_residual": VROW_SOURCES, "vk2_step": VROW_SOURCES}


def kernel_sources_sha256(files) -> str:
    """sha256 over the given csrc files (the sources a kernel is compiled from)."""
    h = hashlib.sha256()
    for f in sorted(files):
        h.update(f.encode())
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()


def short(name: str) -> str:
    # template casts and anonymous namespaces first, then the parameter list
    n = re.sub(r"\((unsigned )?(int|bool|long|char)\)|\(anonymous namespace\)::", "", name)
    n = re.sub(r"\(.*", "", n)
    n = re.sub(r"^void ", "", n)
    n = re.sub(r"wdb::(\(anonymous namespace\)|_GLOBAL__N__\w+)::", "", n)
    return n[:90]


def summarise(path: str) -> str:
    rows = list(csv.reader(line for line in open(path) if not line.startswith("==")))
    head = rows[0]
    ki = head.index("Kernel Name")
    vi = head.index("Metric Value")
    ui = head.index("Metric Unit")
    ri = next((i for i, h in enumerate(head) if h.startswith("NVTX") or h == "thread_domain:push_pop_ranges"), None)
    mi = head.index("Metric Name") if "Metric Name" in head else None
    tot = defaultdict(float)
    cnt = defaultdict(int)
    for r in rows[1:]:
        if len(r) <= max(ki, vi):
            continue
        if mi is not None and r[mi] != "gpu__time_duration.sum":
            continue   # other metrics of the same launch
        v = float(r[vi].replace(",", ""))
        unit = r[ui]
        ns = v * {"nsecond": 1, "ns": 1, "usecond": 1e3, "us": 1e3, "msecond": 1e6, "ms": 1e6, "second": 1e9,
                  "s": 1e9}.get(unit, 1)
        rng = r[ri] if ri is not None else ""
        key = (rng, short(r[ki]))
        tot[key] += ns
        cnt[key] += 1
    out = []
    for rng in sorted({k[0] for k in tot}):
        keys = [k for k in tot if k[0] == rng]
        s = sum(tot[k] for k in keys)
        out.append(f"range {rng or '(all)'}: {sum(cnt[k] for k in keys)} launches, {s / 1e3:.1f} us")
        out.append(f"  {'kernel':90s} {'launches':>8s} {'total us':>10s} {'share':>6s}")
        for k in sorted(keys, key=lambda k: -tot[k]):
            out.append(f"  {k[1]:90s} {cnt[k]:8d} {tot[k] / 1e3:10.1f} {100 * tot[k] / s:5.1f}%")
    return "\n".join(out)


def _kernel_label(name: str) -> str:
    n = name.replace("(int)", "").replace("(bool)", "")
    n = re.sub(r"(wdb::)?(\(anonymous namespace\)|_GLOBAL__N__\w+|unnamed>)::", "", n)
    return short(n)


# to bytes and microseconds
_UNIT = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-3, "usecond": 1, "msecond": 1e3,
         "ns": 1e-3, "us": 1, "ms": 1e3}


def fista_dram(path: str) -> dict:
    """DRAM bytes and duration of the first launch of each FISTA kernel in an ncu CSV: either
    a raw page (one row per launch, one column per metric) or a --csv metrics log (one row
    per launch and metric)."""
    rows = list(csv.reader(line for line in open(path) if not line.startswith("==")))
    head = rows[0]
    per = defaultdict(dict)   # (launch id, kernel) -> metric -> value
    if "Metric Name" in head:
        ki, ni, vi = head.index("Kernel Name"), head.index("Metric Name"), head.index("Metric Value")
        ii, ui = head.index("ID"), head.index("Metric Unit")
        for r in rows[1:]:
            if len(r) > max(ki, ni, vi, ui):
                per[(int(r[ii]), r[ki])][r[ni]] = float(r[vi].replace(",", "")) * _UNIT.get(r[ui], 1)
    else:
        ki, ii = head.index("Kernel Name"), head.index("ID")
        cols = {m: head.index(m) for m in ("dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum")
                if m in head}
        units = rows[1]
        for r in rows[2:]:
            if len(r) > ki:
                d = {}
                for m, c in cols.items():
                    v = float(r[c].replace(",", ""))
                    d[m] = v * _UNIT.get(units[c], 1)
                per[(int(r[ii]), r[ki])] = d
    out = {}
    for (lid, kname), d in sorted(per.items()):
        label = _kernel_label(kname)
        for key, want in FISTA_KERNELS.items():
            if key not in out and re.search(re.escape(want) + r"[,>]", label):
                out[key] = dict(d, kernel=label)
    return out


def write_traffic(csv_path: str, workload: str, profile: str, record: str) -> dict:
    """Update `record` (profiles/traffic.json) for `workload` from the capture in `csv_path`."""
    got = fista_dram(csv_path)
    rec = json.load(open(record)) if os.path.exists(record) else {}
    rec.setdefault("_about", "DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the "
                             "FISTA kernels from ncu captures; valid while the listed sources hash to "
                             "sources_sha256.")
    ent = rec.setdefault(workload, {})
    for key, d in got.items():
        rd, wr = d.get("dram__bytes_read.sum", 0.0), d.get("dram__bytes_write.sum", 0.0)
        src = KERNEL_SOURCES[key]
        ent[key] = {"kernel": d["kernel"], "dram_bytes_per_launch": int(round(rd + wr)),
                    "dram_read": int(round(rd)), "dram_write": int(round(wr)),
                    "duration_us_under_ncu": round(d.get("gpu__time_duration.sum", 0.0), 2),
                    "sources": src, "sources_sha256": kernel_sources_sha256(src), "profile": profile}
    with open(record, "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    return got


if __name__ == "__main__":
    if len(sys.argv) >= 2 and sys.argv[1] == "traffic":
        root = os.path.dirname(os.path.abspath(__file__))
        print(json.dumps(write_traffic(sys.argv[2], sys.argv[3], sys.argv[4],
                                       os.path.join(root, "profiles", "traffic.json")), indent=1))
    else:
        print(summarise(sys.argv[1]))
