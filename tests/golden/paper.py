"""Reader for tests/golden/paper_reported.txt (values printed in the paper)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_reported.txt")


def reported():
    out = {}
    with open(_PATH) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split()[:2]
            out[key] = float(val)
    return out
