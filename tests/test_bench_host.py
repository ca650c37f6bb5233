"""Host-side bookkeeping of bench.py (no GPU): the stored ncu traffic is reported only
for the kernel sources and the look-ahead setting it was captured with, the algorithmic
byte count of the tensor-core update adds up panel by panel, and the whole-job
throughput of one rank is its solves over its device time."""
import json
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_carry_their_capture_keys():
    d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    assert "trail_tc@lookahead0" in d and "trail_tc@lookahead1" in d
    for key, e in d.items():
        cls, mode = key.split("@lookahead")
        assert cls in bench.KERNEL_SRC
        assert e["lookahead"] == int(mode)
        assert e["bytes_per_launch"] > 0 and len(e["src_sha"]) == 16


def test_source_hash_covers_every_file_of_the_class(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2602_10541_gb300" / "csrc"
    csrc.mkdir(parents=True)
    names = bench.KERNEL_SRC["trail_tc"]
    for n in names:
        shutil.copy(os.path.join(ROOT, "paper_2602_10541_gb300", "csrc", n), csrc / n)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._src_sha(names)
    assert bench._src_sha(names) == h0
    for n in names:                      # a change in any source or header moves the hash
        p = csrc / n
        text = p.read_text()
        p.write_text(text + "\n// edited\n")
        assert bench._src_sha(names) != h0
        p.write_text(text)
    assert bench._src_sha(names) == h0


@pytest.mark.parametrize("m,n,nb", [(100, 40, 32), (64, 64, 32), (300, 97, 16)])
def test_update_bytes_add_up_per_panel(m, n, nb):
    # element by element: every trailing element of C (right-hand side column included)
    # is read twice and written once, every element of V read once, and the operand
    # image of V written as 32 hi/lo pairs per row
    want = 0.0
    for k in range(0, n, nb):
        c = min(nb, n - k)
        for _row in range(k, m):
            want += 12.0 * (n + 1 - (k + c)) + 4.0 * c + 8.0 * 32
    unit, got = bench._algorithmic("trail_tc", m, n, m, nb, 1, 2, 4)
    assert unit == "bytes" and got == pytest.approx(want, rel=1e-15)


def test_single_rank_throughput_is_solves_over_device_time():
    value, total = bench._job_throughput(2500.0, 20, 1)
    assert total == 2500.0 and value == pytest.approx(8.0)
