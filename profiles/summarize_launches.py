"""Summarise an ncu launch list (``--metrics gpu__time_duration.sum --csv``) per kernel:
launches, total device time and share.  Usage: python profiles/summarize_launches.py launches.csv"""
import collections
import csv
import re
import sys


def kernel_key(name: str) -> str:
    name = re.sub(r"^void ", "", name)
    base = name.split("(")[0]
    if "<" in base and not base.startswith("(anonymous"):
        head, _, tail = base.partition("<")
        return head + "<" + tail.split(",")[0].rstrip(">") + ">"
    return re.sub(r"^\(anonymous namespace\)::", "", base)


def main(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ki, vi, mi = h.index("Kernel Name"), h.index("Metric Value"), h.index("Metric Name")
    agg = collections.OrderedDict()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        k = kernel_key(r[ki])
        a = agg.setdefault(k, [0, 0.0])
        a[0] += 1
        a[1] += float(r[vi].replace(",", ""))
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':58s} {'launches':>8s} {'total us':>12s} {'share':>7s}")
    for k, v in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k[:58]:58s} {v[0]:8d} {v[1] / 1e3:12.1f} {100 * v[1] / tot:6.2f}%")
    print(f"{'total':58s} {sum(v[0] for v in agg.values()):8d} {tot / 1e3:12.1f}")


if __name__ == "__main__":
    main(sys.argv[1])
