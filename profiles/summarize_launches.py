"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel.

Usage: python profiles/summarize_launches.py launches.csv
Prints launches, total device time and share per kernel name.
"""
import collections
import csv
import sys

SCALE = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}


def kernel_name(raw):
    s = raw.replace("void ", "").replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
    s = s.split("(")[0]
    return s.split("<")[0].strip()


def main(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr = rows[hi]
    ki, mi, vi, ui = (hdr.index("Kernel Name"), hdr.index("Metric Name"),
                      hdr.index("Metric Value"), hdr.index("Metric Unit"))
    tot = collections.defaultdict(float)
    cnt = collections.Counter()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = kernel_name(r[ki])
        tot[name] += float(r[vi].replace(",", "")) * SCALE.get(r[ui], 1.0)
        cnt[name] += 1
    T = sum(tot.values())
    print(f"{'kernel':44s} {'launches':>8s} {'total_us':>11s} {'share':>7s}")
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        print(f"{k[:44]:44s} {cnt[k]:8d} {v:11.1f} {100 * v / T:6.1f}%")
    print(f"{'total':44s} {sum(cnt.values()):8d} {T:11.1f}")


if __name__ == "__main__":
    main(sys.argv[1])
