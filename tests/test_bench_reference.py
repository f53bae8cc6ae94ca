"""The reference arm of bench.py (the oracle on the host cores) on a small grid: one JSON line
with the contract's keys, exactly K timed steps after W warm-ups; ranks other than 0 print
nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--grid", "16",
                          "--steps", "3", "--warmup", "2"], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    return [l for l in out.stdout.splitlines() if l.strip()]


def test_reference_line():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 2
    assert d["value"] > 0 and d["unit"] == d["e2e"]["unit"] == d["cpu_baseline"]["unit"]
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert abs(d["ms_per_step"] - 1000.0 * 8 / d["value"]) <= 1e-6 * d["ms_per_step"]


def test_reference_other_ranks_are_silent():
    assert _run({"RANK": "1"}) == []
