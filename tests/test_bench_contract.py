"""bench.py's reference arm on the CPU: one JSON line with the keys the
benchmark contract fixes (the GPU arm's line is checked on a GB300)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["value"] > 0
    assert d["config"]["workload"] == "wator_2048x2048" and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_profile_commands_run_committed_files():
    """Every ncu command in profiles/ keeps the GPU clocks as they are
    (--clock-control none) and runs bench.py with options it still has."""
    import re
    bench = open(os.path.join(ROOT, "bench.py")).read()
    pdir = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(pdir)):
        text = open(os.path.join(pdir, f)).read().replace("\\\n", " ").replace('\\"', "'")
        cmds = re.findall(r"(?m)^\s*(ncu\s+--.*)$", text) + re.findall(r'"command":\s*"(ncu [^"]*)"', text)
        assert cmds, f
        for c in cmds:
            assert "--clock-control none" in c, (f, c)
            tail = c.split("python bench.py", 1)
            if len(tail) == 2:
                for opt in re.findall(r"(--[a-z][a-z0-9-]*)", tail[1]):
                    assert '"%s"' % opt in bench, (f, opt)
