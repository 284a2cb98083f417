"""Summarise an ncu launch list (``--metrics gpu__time_duration.sum --csv --log-file F``):
launches, total device time and share per kernel, largest first.

    python -m paper_2607_12138_b300.ncu_launches launches.csv [top]
"""
from __future__ import annotations

import collections
import csv
import re
import sys

_SCALE = {"ns": 1, "nsecond": 1, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6, "s": 1e9, "second": 1e9}


def summarise(path: str, top: int = 30) -> str:
    with open(path) as f:
        lines = [ln for ln in f if not ln.startswith("==")]
    rows = list(csv.reader(lines))
    hdr = rows[0]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    agg = collections.defaultdict(lambda: [0, 0.0])
    for row in rows[1:]:
        name = re.sub(r"\(BlockArgs.*|\(TcArgs.*|\(.*", "", row[ki]).strip()
        ns = float(row[vi].replace(",", "")) * _SCALE[row[ui]]
        agg[name][0] += 1
        agg[name][1] += ns
    tot = sum(a[1] for a in agg.values())
    out = [f"{'launches':>8} {'total ms':>10} {'share':>7}  kernel"]
    for k, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1])[:top]:
        out.append(f"{c:8d} {t / 1e6:10.3f} {100 * t / tot:6.2f}%  {k[:120]}")
    out.append(f"total {tot / 1e6:.3f} ms over {sum(a[0] for a in agg.values())} launches")
    return "\n".join(out)


if __name__ == "__main__":
    print(summarise(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 30))
