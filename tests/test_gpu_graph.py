"""Batched form: online schedule autotuning and CUDA-graph replay of the
H_eff*psi launch sequence.  Every schedule variant computes the same products
(only the split-K summation order differs); the graph replay of a schedule is
bitwise identical to its direct launches."""
import os

import numpy as np
import pytest

import synth
from oracle import dmrg as O3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_05581_gb300 import (Context, DEFAULT_LIB, TNS_BF16X3, TNS_FP64,  # noqa: E402
                                    blocks_to_vector)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(DEFAULT_LIB):
        from paper_2305_05581_gb300 import build as b
        b.build()


def _ctx(**env):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return Context(device=0, stream=torch.cuda.current_stream().cuda_stream)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


CASE = (10, 10, 0, 90, 4)


def _load(ctx, seed=21):
    N, n, s2, D, k = CASE
    h, v = synth.integrals(N, 3.0, seed)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=seed)
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    return h, v, bonds, sites


def _apply(ctx, x, nvec, prec, times):
    k = CASE[4]
    out = []
    for _ in range(times):
        y = torch.empty_like(x)
        ctx.heff_apply_ptr(k, x.data_ptr(), y.data_ptr(), nvec, prec)
        out.append(y)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec,tol", [(TNS_FP64, 1e-13), (TNS_BF16X3, 2e-5)])
@pytest.mark.parametrize("nvec", [1, 4])
def test_autotuned_graph_replays_match_fixed_schedule(prec, tol, nvec):
    ref_ctx = _ctx(TNS_AUTOTUNE="0", TNS_GRAPHS="0")
    _load(ref_ctx)
    _, length = ref_ctx.psi_layout(CASE[4])
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(nvec * length, device="cuda", dtype=torch.float64, generator=g)
    ref = _apply(ref_ctx, x, nvec, prec, 1)[0]
    ctx = _ctx()
    _load(ctx)
    # tuning products (one untimed, then two timed samples of each variant:
    # three split-K schedules, and for the tensor-core form also the
    # persistent kernel), then capture and replays of the chosen schedule
    ntune = 1 + 2 * (3 if prec == TNS_FP64 else 4)
    ys = _apply(ctx, x, nvec, prec, ntune + 4)
    scale = float(torch.linalg.norm(ref))
    for y in ys:
        assert float(torch.linalg.norm(y - ref)) <= tol * scale
    for y in ys[ntune + 1:]:
        assert torch.equal(y, ys[ntune])


@pytest.mark.parametrize("prec", [TNS_FP64, TNS_BF16X3])
def test_graph_replay_is_bitwise_equal_to_direct_launch(prec):
    direct = _ctx(TNS_AUTOTUNE="0", TNS_GRAPHS="0")
    graphed = _ctx(TNS_AUTOTUNE="0")
    _load(direct)
    _load(graphed)
    _, length = direct.psi_layout(CASE[4])
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(2 * length, device="cuda", dtype=torch.float64, generator=g)
    a = _apply(direct, x, 2, prec, 2)
    b = _apply(graphed, x, 2, prec, 3)
    assert torch.equal(a[0], a[1])
    for y in b:
        assert torch.equal(y, a[0])


def test_graph_replay_matches_oracle():
    ctx = _ctx()
    h, v, bonds, sites = _load(ctx, seed=8)
    N, n, s2, D, k = CASE
    desc, length = ctx.psi_layout(k)
    keys = synth.psi_keys(bonds, N, n, s2, k)
    X = synth.random_psi(keys, seed=2)[0]
    x = torch.tensor(blocks_to_vector(desc, length, X), device="cuda")
    ys = _apply(ctx, x, 1, TNS_FP64, 6)
    ref = blocks_to_vector(desc, length, O3.DenseHeff(O3.Integrals(h, v), bonds, sites, k, n, s2).apply(X))
    for y in ys:
        assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", [TNS_FP64, TNS_BF16X3])
def test_tuned_schedule_is_cached_by_shape(prec):
    """A work list of the same shape (the step's list rebuilt) takes the cached
    schedule without tuning again, and its products equal the tuned list's."""
    N, n, s2, D, k = CASE
    ctx = _ctx()
    _load(ctx)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(length, device="cuda", dtype=torch.float64, generator=g)
    y = torch.empty_like(x)
    for _ in range(12):  # one untimed product, two timed samples of every variant, then the graph
        ctx.heff_apply_ptr(k, x.data_ptr(), y.data_ptr(), 1, prec)
    st0 = ctx.schedule_stats()
    assert st0["tuned"] == 1 and st0["cache_hits"] == 0
    ctx.build_env(k)  # a new work list of the same shape
    y2 = torch.empty_like(x)
    ctx.heff_apply_ptr(k, x.data_ptr(), y2.data_ptr(), 1, prec)
    torch.cuda.synchronize()
    st1 = ctx.schedule_stats()
    assert st1["tuned"] == 1 and st1["cache_hits"] == 1
    assert torch.equal(y, y2)  # same schedule, same summation order
    ctx.close()
