"""Checkpoint / restart of a sweep on the GPU: a context restored from a
checkpoint taken mid-sweep continues the sweep with the same energies as the
context that wrote it (FP64 products, fixed schedule: bitwise)."""
import os

import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx():
    from paper_2305_05581_gb300 import Context
    os.environ["TNS_AUTOTUNE"] = "0"
    try:
        return Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    finally:
        del os.environ["TNS_AUTOTUNE"]


def test_restart_continues_the_sweep(tmp_path):
    from paper_2305_05581_gb300 import TNS_FP64
    N, n, s2, D = 8, 8, 0, 48
    h, v = synth.integrals(N, 3.0, 0)
    a = _ctx()
    a.load_integrals(h, v)
    a.mps_init(N, n, s2, D, seed=3)
    for k in range(0, 4):
        a.step(k, True, D, tol=1e-9, max_iter=100, precision=TNS_FP64)
    path = str(tmp_path / "sweep.ckpt")
    a.checkpoint_save(path, site=4, left_to_right=True)
    rest = [(4, True), (5, True), (6, False), (5, False)]
    ea = [a.step(k, d, D, tol=1e-9, max_iter=100, precision=TNS_FP64).energy for k, d in rest]
    b = _ctx()
    site, ltr = b.checkpoint_load(path)
    assert (site, ltr) == (4, True)
    eb = [b.step(k, d, D, tol=1e-9, max_iter=100, precision=TNS_FP64).energy for k, d in rest]
    assert ea == eb
    a.close()
    b.close()
