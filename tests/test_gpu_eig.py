"""Truncation hand-off on the GPU: the batched symmetric eigensolver against
LAPACK (numpy.linalg.eigvalsh) and the truncated two-site wavefunction of a
step against the global top-D singular triplets of its sector matrices."""
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_05581_gb300 import Context, DEFAULT_LIB, TNS_FP64, vector_to_blocks  # noqa: E402

SITE_QN = [(0, 0), (1, 1), (1, -1), (2, 0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(DEFAULT_LIB):
        from paper_2305_05581_gb300 import build as b
        b.build()


def _ctx():
    return Context(device=0, stream=torch.cuda.current_stream().cuda_stream)


def _matrices(rng):
    mats = []
    for n in (1, 2, 3, 5, 17, 64, 127, 300):
        a = rng.standard_normal((n, n))
        mats.append(a + a.T)
    n = 90
    mats.append(np.zeros((n, n)))                                    # all-zero
    mats.append(np.eye(n))                                           # fully degenerate
    mats.append(np.diag(rng.standard_normal(n)))                     # already diagonal
    m = rng.standard_normal((n, 3))
    mats.append(m @ m.T)                                             # rank 3, PSD
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat([2.0, 1.0, 1e-3, 0.0], [10, 30, 20, 30])
    mats.append((q * lam) @ q.T)                                     # clustered eigenvalues
    lam = 10.0 ** (-np.arange(n) / 6.0)
    mats.append((q * lam) @ q.T)                                     # graded density-matrix-like
    a = rng.standard_normal((1000, 1000))
    mats.append(a @ a.T / 1000.0)                                    # large PSD
    return mats


def test_sym_eig_matches_lapack():
    rng = np.random.default_rng(11)
    mats = _matrices(rng)
    sizes = [m.shape[0] for m in mats]
    packed = np.concatenate([m.ravel() for m in mats])
    A = torch.tensor(packed, device="cuda", dtype=torch.float64)
    Z = torch.empty_like(A)
    w = torch.empty(sum(sizes), device="cuda", dtype=torch.float64)
    ctx = _ctx()
    ctx.sym_eig_ptr(sizes, A.data_ptr(), Z.data_ptr(), w.data_ptr())
    torch.cuda.synchronize()
    Zh, wh = Z.cpu().numpy(), w.cpu().numpy()
    o = ow = 0
    for m in mats:
        n = m.shape[0]
        z = Zh[o:o + n * n].reshape(n, n)  # row p = eigenvector p
        lam = wh[ow:ow + n]
        o += n * n
        ow += n
        scale = max(1.0, np.abs(m).max()) * n
        ref = np.linalg.eigvalsh(m)
        assert np.max(np.abs(np.sort(lam) - ref)) <= 1e-14 * scale
        assert np.max(np.abs(z @ z.T - np.eye(n))) <= 1e-14 * n
        assert np.max(np.abs(m @ z.T - z.T * lam)) <= 1e-14 * scale


def test_sym_eig_rejects_oversize():
    ctx = _ctx()
    A = torch.zeros(1, device="cuda", dtype=torch.float64)
    with pytest.raises(Exception):
        ctx.sym_eig_ptr([5000], A.data_ptr(), A.data_ptr(), A.data_ptr())


def _sector_matrices(blocks):
    """Middle-bond sector q -> (matrix, row keys, col keys) with rows (q_l, s1), cols (s2, q_r)."""
    rows, cols = {}, {}
    for (ql, s1, s2, qr), b in blocks.items():
        q = (ql[0] + SITE_QN[s1][0], ql[1] + SITE_QN[s1][1])
        rows.setdefault(q, {})[(ql, s1)] = b.shape[0]
        cols.setdefault(q, {})[(s2, qr)] = b.shape[1]
    out = {}
    for q in rows:
        ro, co = {}, {}
        r = c = 0
        for key in sorted(rows[q]):
            ro[key] = r
            r += rows[q][key]
        for key in sorted(cols[q]):
            co[key] = c
            c += cols[q][key]
        out[q] = (np.zeros((r, c)), ro, co)
    for (ql, s1, s2, qr), b in blocks.items():
        q = (ql[0] + SITE_QN[s1][0], ql[1] + SITE_QN[s1][1])
        M, ro, co = out[q]
        r0, c0 = ro[(ql, s1)], co[(s2, qr)]
        M[r0:r0 + b.shape[0], c0:c0 + b.shape[1]] = b
    return out


@pytest.mark.parametrize("ltr", [True, False])
@pytest.mark.parametrize("N,n,s2,D,k,Dcut", [(8, 8, 0, 40, 3, 10), (10, 9, 1, 60, 4, 25)])
def test_truncated_wavefunction_is_global_top_d(N, n, s2, D, k, Dcut, ltr):
    h, v = synth.integrals(N, 3.0, 40 + N)
    bonds, sites = synth.random_mps(N, n, s2, D, center=k, seed=k)
    ctx = _ctx()
    ctx.load_integrals(h, v)
    ctx.mps_import(N, n, s2, D, bonds, sites)
    ctx.build_env(k)
    desc, length = ctx.psi_layout(k)
    psi = np.zeros(length)
    st = ctx.step(k, ltr, Dcut, tol=1e-10, max_iter=200, precision=TNS_FP64, cutoff=0.0,
                  psi_host_ptr=psi.ctypes.data)
    trunc = np.zeros(length)
    ctx.psi_guess(k, trunc.ctypes.data)
    # reference: per-sector SVD of the converged psi, global top-Dcut
    secs = _sector_matrices(vector_to_blocks(desc, psi))
    allsv = sorted(((s, q, i) for q, (M, _, _) in secs.items()
                    for i, s in enumerate(np.linalg.svd(M, compute_uv=False))), key=lambda t: -t[0])
    kept = allsv[:Dcut]
    gap = allsv[Dcut - 1][0] - allsv[Dcut][0] if len(allsv) > Dcut else 1.0
    assert gap > 1e-6, "test case needs a gap at the cut"
    disc = sum(s * s for s, _, _ in allsv[Dcut:])
    assert abs(st.discarded - disc) <= 1e-12 + 1e-10 * disc
    nkeep = {}
    for _, q, _ in kept:
        nkeep[q] = nkeep.get(q, 0) + 1
    got = _sector_matrices(vector_to_blocks(desc, trunc))
    for q, (M, _, _) in secs.items():
        u, s, vt = np.linalg.svd(M, full_matrices=False)
        r = nkeep.get(q, 0)
        ref = (u[:, :r] * s[:r]) @ vt[:r]
        G = got[q][0] if q in got else np.zeros_like(M)
        assert np.max(np.abs(G - ref)) <= 1e-10
