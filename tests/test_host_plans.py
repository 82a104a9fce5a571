"""Host logic: the plan builder's formatted operations, executed on the CPU
in FP64 by tests/host/plan_emulator.cpp (which links the product's
acr_plan.cpp and acr_structure.cpp), reproduce exact results on operands
whose result fits the block structure, merged plans equal separate ones
(and every plan keeps its GEMM stages' 64-column-output groups first, as
the launcher's kernel split assumes), and the apply's per-chunk index lists
reproduce H x and H^T x.  No GPU involved."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1712_08872_gb300", "csrc")


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_emulator")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "plan_emulator.cpp"),
                    os.path.join(CSRC, "acr_plan.cpp"), os.path.join(CSRC, "acr_structure.cpp"),
                    "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("n,eta,leaf", [(16, 2.0, 16), (16, 2.0, 32), (16, 1.0, 16),
                                        (32, 2.0, 64)])
def test_plans_reproduce_exact_operations(emulator, n, eta, leaf):
    r = subprocess.run([emulator, str(n), str(eta), str(leaf)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count(" ok") == 8, r.stdout
