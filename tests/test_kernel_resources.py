"""Resource budgets of the tensor-core product kernels, from the assembler's
own report (`nvcc -Xptxas -v`, CPU only): each kernel is designed around a
number of resident CTAs per SM, so its registers must fit the SM's 64 K
registers at that residency, and none may spill.

  k_tasks_tc      256 threads, 3 CTAs per SM  -> <= 85 registers
  k_tasks_tc_ws   192 threads, 1 CTA per SM   -> <= 255
  k_tasks_sw<,16> 128 threads, 4 CTAs per SM  -> <= 128
  k_tasks_sw<,32> 128 threads, 2 CTAs per SM  -> <= 255
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2305_05581_gb300", "csrc", "tc.cu")
OBJ = os.path.join(ROOT, "_build", "tc_resources.o")

BUDGET = {  # kernel (mangled-name stem) -> largest register count
    "k_tasks_tcILi": 85,
    "k_tasks_tc_wsILi": 255,
    "k_tasks_swILi0ELi16E": 128, "k_tasks_swILi1ELi16E": 128,
    "k_tasks_swILi0ELi32E": 255, "k_tasks_swILi1ELi32E": 255,
}


@pytest.fixture(scope="module")
def report():
    from paper_2305_05581_gb300 import build as b
    nv = b.nvcc()
    if not (os.path.exists(nv) or shutil.which(nv)):
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(OBJ), exist_ok=True)
    r = subprocess.run([nv] + b.ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I",
                                        os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c", SRC, "-o", OBJ],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    kernels = {}
    name = None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
            kernels[name] = {}
            continue
        if name is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            kernels[name]["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            kernels[name]["regs"] = int(m.group(1))
    return kernels


@pytest.mark.parametrize("stem", sorted(BUDGET))
def test_registers_fit_the_designed_residency(report, stem):
    hits = {n: k for n, k in report.items() if re.search(r"\d" + stem + r"|[^_a-z]" + stem, n) and
            (stem != "k_tasks_tcILi" or "k_tasks_tc_ws" not in n)}
    assert hits, f"no kernel {stem} in the report"
    for n, k in hits.items():
        assert k.get("regs", 999) <= BUDGET[stem], (n, k)
        assert k.get("spill", 1) == 0, (n, k)
