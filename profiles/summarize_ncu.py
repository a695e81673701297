"""Summarise an ncu CSV launch list (gpu__time_duration.sum per launch) into
per-kernel launch counts, total time and share.

    python profiles/summarize_ncu.py launches.csv
"""
import collections
import csv
import re
import sys


def kernel_name(full):
    s = full.replace("(anonymous namespace)", "").replace("<unnamed>", "")
    s = re.sub(r"\(.*$", "", s)               # drop the argument list
    s = re.sub(r"^void\s+", "", s.strip())
    base = s.split("<")[0]
    targs = s[len(base):]
    return base.split("::")[-1] + targs


def summarize(path):
    rows = list(csv.reader(open(path)))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hdr]
    ki, mi, vi, ui = (h.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    scale = {"nsecond": 1e-3, "ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3,
             "second": 1e6, "s": 1e6}
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hdr + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        a = agg[kernel_name(r[ki])]
        a[0] += 1
        a[1] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
    tot = sum(v[1] for v in agg.values())
    out = [f"{'kernel':34s} {'launches':>8s} {'total_us':>10s} {'share':>6s}"]
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append(f"{k:34s} {n:8d} {t:10.1f} {100 * t / tot:5.1f}%")
    return "\n".join(out)


if __name__ == "__main__":
    print(summarize(sys.argv[1]))
