"""Host-side planning of the tensor-core products (routing of output blocks
to the small-block warp kernels or the tcgen05 tile kernel, chunks, split-K
pieces and their partial tiles, the launch checks), on seeded synthetic work
lists: tests/hostcheck/plancheck.cu includes the planning code of tc.cu as it
is, is compiled here with nvcc and makes no CUDA call (CPU only)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2305_05581_gb300")
LIB = os.path.join(PKG, "libtns.so")
EXE = os.path.join(ROOT, "_build", "plancheck")


@pytest.fixture(scope="module")
def plancheck():
    from paper_2305_05581_gb300 import build as b
    nv = b.nvcc()
    if not (os.path.exists(nv) or shutil.which(nv)):
        pytest.skip("nvcc not available")
    if not os.path.exists(LIB):
        b.build()
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    subprocess.check_call([nv] + b.ARCH + ["-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", EXE,
                                           os.path.join(ROOT, "tests", "hostcheck", "plancheck.cu"), "-L", PKG,
                                           "-ltns", "-Xlinker", "-rpath", "-Xlinker", PKG])
    return EXE


def test_plan_routing_chunks_splits_and_checks(plancheck):
    r = subprocess.run([plancheck], capture_output=True, text=True, timeout=600)
    out = r.stdout
    assert r.returncode == 0 and out.strip().endswith("ALL OK"), out[-2000:] + r.stderr[-2000:]
    lines = [l for l in out.splitlines() if l.startswith("ok ")]
    assert len(lines) == 24  # 3 seeds x 4 routing limits x 2 precisions
    # every route is exercised: each kernel gets blocks under some limit, none under limit 0
    assert any(" 0 on the 32-state" not in l for l in lines)
    assert all("0 blocks on the 16-state kernel, 0 on the 32-state kernel" in l for l in lines if "limit 0 " in l)
    assert all(" 0 on the tile kernel" not in l for l in lines)
    # long product lists are cut into split-K pieces under every limit
    assert all(not l.endswith(" 0 split tiles") for l in lines)
