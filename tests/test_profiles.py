"""The ncu summaries under profiles/ name the command that made them; every
such command must run committed files only: `bench.py` with flags it
accepts.  Also the GEMM-family traffic record parses, and carries the
source hash `bench.py` checks before it reports `roofline.traffic`.  CPU
only."""
import glob
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_flags():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                         capture_output=True, text=True, timeout=120, cwd=ROOT).stdout
    return set(re.findall(r"(--[a-z0-9][a-z0-9-]*)", out))


def _commands(text):
    # a command may continue over lines ending in a backslash
    joined = re.sub(r"\\\n\s*", " ", text)
    return [ln.strip() for ln in joined.splitlines() if "python bench.py" in ln]


def test_profile_commands_use_committed_bench_flags():
    flags = _bench_flags()
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    seen = 0
    for f in files:
        text = open(f).read()
        for cmd in _commands(text):
            tail = cmd.split("python bench.py", 1)[1]
            for flag in re.findall(r"(--[a-z0-9][a-z0-9-]*)", tail):
                assert flag in flags, (os.path.basename(f), flag)
            seen += 1
            assert "--clock-control none" in cmd or not cmd.startswith("ncu"), (f, cmd)
        # the commands are the indented (code) lines that start with ncu
        for cmd in re.findall(r"^ {4}ncu .*", re.sub(r"\\\n\s*", " ", text), re.M):
            assert "--clock-control none" in cmd, (os.path.basename(f), cmd)
    assert seen > 0


def test_gemm_traffic_record_parses():
    sys.path.insert(0, ROOT)
    import bench
    txt = open(bench.TRAFFIC_FILE).read()
    assert re.search(r"bytes_per_flop:\s*[0-9.]+", txt)
    sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    assert sha is not None
    bpf, src = bench.gemm_traffic_per_flop()
    # a record for the current sources, or null with the stated reason
    assert (bpf is not None and bpf > 0) or src == "kernel changed since the capture"
