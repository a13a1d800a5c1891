"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel:
launches, total device time and share, split by NVTX range when ncu recorded one.

    python -m paper_1512_08401_gb300.ncu_summary launches.csv
"""
from __future__ import annotations

import csv
import re
import sys
from collections import defaultdict


def short(name: str) -> str:
    n = re.sub(r"\(.*", "", name)
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
    tot = defaultdict(float)
    cnt = defaultdict(int)
    for r in rows[1:]:
        if len(r) <= max(ki, vi):
            continue
        v = float(r[vi].replace(",", ""))
        unit = r[ui]
        ns = v * {"nsecond": 1, "usecond": 1e3, "msecond": 1e6, "second": 1e9}.get(unit, 1)
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


if __name__ == "__main__":
    print(summarise(sys.argv[1]))
