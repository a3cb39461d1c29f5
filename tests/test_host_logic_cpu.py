"""Host-side logic that needs no GPU: the autotuner's choice and cache (with
a fake timer standing in for the device), and the benchmark's reference arm
(the oracle on the host cores) printing its one JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_size_class_is_a_log2_bucket():
    from paper_2504_04411_gb300 import autotune
    assert autotune.size_class(2_073_600, 2_000_000, 0.01) == autotune.size_class(2_000_000, 2_100_000, 0.0101)
    assert autotune.size_class(2_073_600, 2_000_000, 0.01) != autotune.size_class(4_000_000, 2_000_000, 0.01)


def test_tune_picks_the_fastest_and_caches(tmp_path, monkeypatch):
    from paper_2504_04411_gb300 import autotune

    class PH:
        class pos:
            shape = (1000, 3)

    class HP:
        class pos:
            shape = (5000, 3)

    fake = {(0, 0.5): 3.0, (0, 0.6): 2.5, (0, 2.0 / 3.0): 2.6, (0, 0.75): 2.7, (0, 1.0): 3.3, (1, 0.5): 4.0,
            (1, 1.0): 4.1, (4, 0.5): 9.0, (4, 1.0): 8.0}
    assert set(fake) == set(autotune.CANDIDATES)
    calls = []

    def timer(hp, batches, r0, mapping, cell_factor, params=None):
        calls.append((mapping, cell_factor))
        return fake[(mapping, cell_factor)]

    monkeypatch.setattr(autotune, "time_config", timer)
    cache = str(tmp_path / "tune.json")
    got = autotune.tune(HP, [PH, PH], 0.01, cache=cache)
    assert (got["mapping"], got["cell_factor"]) == (0, 0.6)
    assert sorted(calls) == sorted(fake)
    calls.clear()
    again = autotune.tune(HP, [PH, PH], 0.01, cache=cache)     # from the cache: no timing
    assert (again["mapping"], again["cell_factor"]) == (0, 0.6) and not calls
    assert json.load(open(cache))[got["key"]]["mapping"] == 0


def test_tune_batch_picks_traversal_then_tile(tmp_path, monkeypatch):
    from paper_2504_04411_gb300 import autotune

    class S:
        nh, J, r0 = 1000, 10_000, 0.01

    def timer(scenes, hps, photon_lists, mapping, cf, tile):
        return {64: 2.0, 128: 1.5, 256: 1.8}[tile] + (0.0 if (mapping, cf) == (0, 0.75) else 1.0)

    monkeypatch.setattr(autotune, "_time_batch", timer)
    got = autotune.tune_batch([S] * 4, None, [None, None], cache=str(tmp_path / "t.json"))
    assert got["mapping"] == 0 and got["cell_factors"] == [0.75] * 4 and got["tile"] == 128


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "pairs/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["steps"] == 2 and d["warmup"] == 1
