"""Host-side bookkeeping of bench.py (no GPU): the stored ncu traffic is reported only
for the kernel sources and workload it was captured with, the algorithmic work of the
two-level schedule adds up to the one-level schedule's plus the rows above the inner
panels, the whole-job throughput of one rank is its solves over its device time, and the
autotuner's launch table is read with defaults for keys it lacks."""
import json
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_carry_their_capture_keys():
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        pytest.skip("no ncu traffic on record")
    d = json.load(open(path))
    for cls, e in d.items():
        assert cls in bench.KERNEL_SRC
        assert len(e["src_sha"]) == 16
        # the record's own launches: bytes over flops, and the algorithmic floor (the
        # Y pass reads each FP32 entry of [V | C] once: 4 bytes per 6 * 2 * nbk flops)
        assert e["bytes_per_tensor_flop"] == pytest.approx(sum(e["dram_bytes"]) / sum(e["bf16_tensor_flops"]))
        assert e["bytes_per_tensor_flop"] > 0.5 * 4.0 / (6 * 2 * bench.BLK)


def test_block_launch_count_matches_the_blocks_with_trailing_columns():
    assert bench._block_launches(4096, 1) == 2 * 32
    assert bench._block_launches(300, 1) == 2 * 3
    assert bench._block_launches(256, 0) == 2 * 1


def test_source_hash_covers_every_file_of_the_class(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2602_10541_gb300" / "csrc"
    csrc.mkdir(parents=True)
    names = bench.KERNEL_SRC["block_y"]
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


@pytest.mark.parametrize("m,n,nb", [(1000, 300, 32), (700, 256, 16), (500, 130, 32), (400, 64, 32)])
def test_two_level_work_adds_up(m, n, nb):
    """One level: panel kp updates every column right of it with its rows kp.. (4 (m-kp)
    nb n_c flops).  Two levels: inside the block the same, and the outer update applies
    the whole block with the block's rows k.. to the columns right of the block, so it
    also multiplies the zeros above each inner panel's diagonal: the difference is
    exactly sum over inner panels of 4 (kp - k) nb n_right."""
    nrhs = 1
    one = sum(4.0 * (m - kp) * min(nb, n - kp) * (n + nrhs - (kp + min(nb, n - kp)))
              for kp in range(0, n, nb))
    y, u = bench._blocked_flops(m, n, nrhs)
    gram = sum(2.0 * (m - k) * min(128, n - k) * min(128, n - k) for k in range(0, n, 128)
               if n + nrhs > k + min(128, n - k))
    two = (y - gram) + u + bench._inner_flops(m, n, nb)
    extra = 0.0
    for k in range(0, n, 128):
        nbk = min(128, n - k)
        for kp in range(k, k + nbk, nb):
            extra += 4.0 * (kp - k) * min(nb, n - kp) * (n + nrhs - (k + nbk))
    assert two == pytest.approx(one + extra, rel=1e-14)
    unit, amount = bench._algorithmic("block_u", m, n, m, nb, 1, 2, 4)
    assert unit == "flops" and amount == pytest.approx(bench.SPLIT_PRODUCTS * u)


def test_oracle_sample_ratio_is_the_qr_work_ratio():
    s = bench.WORKLOADS["poisson5d"]["cpu_sample"]
    r = bench._scale_ratio("poisson5d", s)
    assert r == pytest.approx((32768 + 4096) * 4096 ** 2 / ((s["n_int"] + s["n_bc"]) * s["n_feat"] ** 2))
    assert bench._scale_ratio("helmholtz2d", None) == 1.0


def test_single_rank_throughput_is_solves_over_device_time():
    value, total = bench._job_throughput(2500.0, 20, 1)
    assert total == 2500.0 and value == pytest.approx(8.0)


def test_tuned_launch_fills_keys_the_table_lacks(tmp_path, monkeypatch):
    """pipeline.tuned() takes the recorded launch shape and falls back to the default for
    any key the table does not hold (a table written before a key existed)."""
    import json
    from paper_2602_10541_gb300 import pipeline as pl
    table = tmp_path / "tuning.json"
    table.write_text(json.dumps({"inverse_eval": {"threads": 512, "ctas_per_sm": 2, "ms": 1.0}}))
    real_join = os.path.join
    pkg = os.path.dirname(os.path.abspath(pl.__file__))
    monkeypatch.setattr(os.path, "join",
                        lambda *a: str(table) if a == (pkg, "tuning.json") else real_join(*a))
    got = pl.tuned("inverse_eval", {"threads": 256, "ctas_per_sm": 1, "cluster": 1})
    assert got == {"threads": 512, "ctas_per_sm": 2, "cluster": 1}
    assert pl.tuned("other_kernel", {"a": 1}) == {"a": 1}


def test_tuner_candidates_cover_every_launch_shape():
    from paper_2602_10541_gb300 import tune
    shapes = {(c["threads"], c["ctas_per_sm"], c["cluster"]) for c in tune.CANDIDATES}
    assert shapes == {(t, k, c) for t in (256, 512) for k in (1, 2) for c in (1, 2, 4)}


def test_inverse_evaluation_work_of_both_plans():
    """The thin-Q plan's FMAs per instance are 2 n_int n + n^2 (two passes over the
    interior rows of Q and two substitutions); the reflector plan's are 4 m_aug n.  For
    the batched configuration's largest instance the thin plan does 2.5x less."""
    shapes = [(8192, 1024, 2048), (1024, 128, 512)]
    thin = bench._inverse_eval_fma(shapes, True)
    refl = bench._inverse_eval_fma(shapes, False)
    assert thin == 2 * 8192 * 2048 + 2048 ** 2 + 2 * 1024 * 512 + 512 ** 2
    assert refl == 4 * (8192 + 1024 + 2048) * 2048 + 4 * (1024 + 128 + 512) * 512
    big_t, big_r = bench._inverse_eval_fma(shapes[:1], True), bench._inverse_eval_fma(shapes[:1], False)
    assert 2.4 < big_r / big_t < 2.6
