"""bench.py's reference arm (the FP64 oracle on the host cores): one JSON
line with the keys of the benchmark contract, and silence on ranks other
than 0 under a multi-process launch."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, timeout=240):
    env = dict(os.environ, **(extra_env or {}))
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


@pytest.mark.timeout(300)
def test_reference_arm_prints_one_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "Gupd/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["vs_baseline"] is None and d["dtype"] == "f64" and d["data"].startswith("synthetic")
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_equal_psnr_compares_like_with_like():
    """The learned-prox comparison picks, among solves that reach the
    target PSNR, the fastest of each side with the same kind of TV prox:
    cold-started proxes on both sides for `speedup`, warm-started ones
    allowed on both for `speedup_vs_any_tv`; solves below the target never
    count, and without a learned solve at the target there is no result."""
    from paper_1306_1392_b300.train_prox import equal_psnr
    r = lambda v, k, ms, ps: {"variant": v, "n_iter": k, "s_per_slice": ms * 1e-3, "psnr_mean": ps}
    rows = [r("tv", 200, 7.0, 30.0), r("tv", 125, 4.0, 30.1), r("tv", 100, 3.0, 29.9),    # 100: below target
            r("fbp+tv", 150, 5.0, 30.2), r("tv-warm-dual15", 100, 3.2, 30.0),
            r("tv-warm-dual5", 80, 2.0, 29.8),                                          # below target
            r("tv+ista4", 28, 1.25, 30.1), r("tv+ista2", 25, 1.0, 29.5),                  # ista2: below target
            r("tv-warm-dual10+ista4", 28, 1.0, 30.05), r("ista", 5, 0.5, 24.0)]
    e = equal_psnr(rows, 30.0, 7.0e-3)
    assert (e["tv_variant"], e["tv_n_iter"]) == ("tv", 125)
    assert (e["pnp_variant"], e["pnp_n_iter"]) == ("tv+ista4", 28)
    assert abs(e["speedup"] - 4.0 / 1.25) < 1e-12
    assert (e["any_tv_variant"], e["any_pnp_variant"]) == ("tv-warm-dual15", "tv-warm-dual10+ista4")
    assert abs(e["speedup_vs_any_tv"] - 3.2 / 1.0) < 1e-12
    assert abs(e["speedup_vs_tv_from_zero"] - 7.0 / 1.25) < 1e-12
    assert equal_psnr([x for x in rows if "ista" not in x["variant"]], 30.0, 7.0e-3) is None
