"""The eigen-solver over the whole GPU and streaming snapshots (stats_finalize_warm).

Every snapshot is compared with the oracle on the same rows: the two-pass covariance of
the rows accumulated so far and the oracle's cyclic Jacobi on it.  Inputs come from a
seeded host generator (rows of X = Z L^T + mu with a known population covariance
L L^T = Q diag(1/k) Q^T); both sides read the same host rows.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2604_23826_gb300")
from paper_2604_23826_gb300 import inputs  # noqa: E402


def _device_cols(X):
    d = torch.as_tensor(X, device="cuda")
    return d, [d[j] for j in range(X.shape[0])]


def _check_pairs(an, M, ev_tol=1e-11, vec_tol=1e-8, orth_tol=1e-12):
    """Eigenpairs of an (evals descending, rows of evecs) against the oracle's Jacobi on M."""
    ev, V = O.jacobi(M)
    scale = np.abs(ev).max()
    assert np.abs(an.evals - ev).max() <= ev_tol * scale
    assert abs(an.evals.sum() - np.trace(M)) <= ev_tol * abs(np.trace(M))
    gaps = np.abs(np.diff(ev))
    for k in range(len(ev)):
        sep = min(gaps[k - 1] if k > 0 else np.inf, gaps[k] if k < len(gaps) else np.inf)
        if sep > 1e-6 * scale:
            assert np.abs(an.evecs[k] - V[k]).max() <= vec_tol, k
    pa = len(ev)
    assert np.abs(an.evecs @ an.evecs.T - np.eye(pa)).max() <= orth_tol
    R = an.evecs @ M @ an.evecs.T - np.diag(an.evals)
    assert np.abs(R).max() <= 1e-12 * scale


@pytest.mark.parametrize("p", [24, 25, 64, 129, 256])
def test_grid_solver_against_oracle(p):
    """Widths from the smallest that takes the grid-wide solver, odd ones (zero-padded to even
    order) and the widest; covariance and correlation eigenpairs."""
    n = 20_000
    L, mu = inputs.wide_factor(11 + p, p)
    X = inputs.gen_correlated_host(n, L, mu, seed=p)
    _, cols = _device_cols(X)
    cov = O.cov_twopass_columns(list(X))
    corr = O.corr_from_cov(cov)
    with G.stats_init(G.Config([G.STATS_F64] * p, G.STATS_FP64_SHIFTED, [0] * p)) as ctx:
        G.stats_accumulate(ctx, cols, n)
        an = G.stats_finalize_warm(ctx, 0)
        anc = G.stats_finalize_warm(ctx, 1)
    assert np.abs(an.cov - cov).max() <= 1e-13 * np.abs(cov).max()
    assert an.sweeps > 0 and anc.sweeps > 0
    _check_pairs(an, cov)
    _check_pairs(anc, corr)


def test_grid_solver_matches_one_block_solver():
    """stats_finalize (grid-wide solver at this width) against stats_finalize_batched (the
    one-block solver inside the finalize kernel) on the same context."""
    p, n = 96, 30_000
    L, mu = inputs.wide_factor(3, p)
    X = inputs.gen_correlated_host(n, L, mu, seed=9)
    _, cols = _device_cols(X)
    with G.stats_init(G.Config([G.STATS_F64] * p, G.STATS_FP64_SHIFTED, [0] * p)) as ctx:
        G.stats_accumulate(ctx, cols, n)
        a = G.stats_finalize(ctx)
        (b,) = G.stats_finalize_batched([ctx])
    assert np.array_equal(a.cov, b.cov)
    scale = np.abs(b.evals).max()
    assert np.abs(a.evals - b.evals).max() <= 1e-13 * scale
    gaps = np.abs(np.diff(b.evals))
    for k in range(p):
        sep = min(gaps[k - 1] if k > 0 else np.inf, gaps[k] if k < len(gaps) else np.inf)
        if sep > 1e-6 * scale:
            assert np.abs(a.evecs[k] - b.evecs[k]).max() <= 1e-9, k


def test_grid_solver_repeated_eigenvalues():
    """Duplicated and constant columns: a zero eigenvalue of multiplicity 9 (cov), compared as a
    subspace; the remaining eigenpairs against the oracle."""
    p0, n = 24, 10_000
    L, mu = inputs.wide_factor(5, p0)
    X0 = inputs.gen_correlated_host(n, L, mu, seed=5)
    X = np.concatenate([X0, X0[:6], np.full((3, n), 2.5)], axis=0)  # p = 33
    p = X.shape[0]
    _, cols = _device_cols(X)
    cov = O.cov_twopass_columns(list(X))
    with G.stats_init(G.Config([G.STATS_F64] * p, G.STATS_FP64_SHIFTED, [0] * p)) as ctx:
        G.stats_accumulate(ctx, cols, n)
        an = G.stats_finalize_warm(ctx, 0)
    ev, V = O.jacobi(cov)
    scale = ev.max()
    assert np.abs(an.evals - ev).max() <= 1e-11 * scale
    assert np.all(np.abs(an.evals[-9:]) <= 1e-12 * scale)
    P_gpu = an.evecs[-9:].T @ an.evecs[-9:]
    P_ref = V[-9:].T @ V[-9:]
    assert np.abs(P_gpu - P_ref).max() <= 1e-8
    assert np.abs(an.evecs @ an.evecs.T - np.eye(p)).max() <= 1e-12
    for k in range(p - 9):
        if min(abs(ev[k] - ev[k - 1]) if k else np.inf, abs(ev[k] - ev[k + 1])) > 1e-6 * scale:
            assert np.abs(an.evecs[k] - V[k]).max() <= 1e-8


@pytest.mark.parametrize("p,mode", [(32, G.STATS_FP64_SHIFTED), (256, G.STATS_FP64_SHIFTED),
                                    (64, G.STATS_BF16X4)])
def test_streaming_snapshots_against_oracle(p, mode):
    """A table streamed in chunks, a snapshot after each: every snapshot equals the oracle on the
    rows so far; seeded snapshots take fewer sweeps than a cold solve of the same matrix."""
    n_chunk, chunks = 25_000, 4
    L, mu = inputs.wide_factor(21, p)
    dt = G.STATS_F32 if mode in (G.STATS_BF16X3, G.STATS_BF16X4) else G.STATS_F64
    cfg = G.Config([dt] * p, mode, [0] * p)
    with G.StreamingAnalysis(cfg) as sa:
        keep = []
        for c in range(chunks):
            X = inputs.gen_correlated_host(n_chunk, L, mu, seed=17, row0=c * n_chunk)
            if dt == G.STATS_F32:
                X = X.astype(np.float32)
            d, cols = _device_cols(X)
            keep.append(d)
            sa.update(cols, n_chunk)
            an = sa.snapshot()
            rows = np.concatenate([k.cpu().numpy() for k in keep], axis=1)
            cov = O.cov_twopass_columns([r.astype(np.float64) for r in rows])
            cold = G.stats_finalize_warm(sa.ctx, 0)
            assert np.array_equal(an.cov, cold.cov)
            tol = 1e-13 if dt == G.STATS_F64 else 2e-6
            assert np.linalg.norm(an.cov - cov) <= tol * np.linalg.norm(cov)
            if dt == G.STATS_F64:
                _check_pairs(an, cov)
            else:  # eigenvalues move by at most the covariance error (Weyl)
                ev, _ = O.jacobi(cov)
                assert np.abs(an.evals - ev).max() <= tol * np.linalg.norm(cov)
            # the eigen-solve itself, on the snapshot's own matrix: an orthonormal diagonalising basis
            scale = np.abs(an.evals).max()
            assert np.abs(an.evecs @ an.cov @ an.evecs.T - np.diag(an.evals)).max() <= 1e-12 * scale
            assert np.abs(an.evecs @ an.evecs.T - np.eye(p)).max() <= 1e-12
            # seeded and cold solves agree to the solver's backward error, O(p eps) of the norm
            assert np.abs(an.evals - cold.evals).max() <= 2e-15 * p * np.abs(cold.evals).max()
            if c > 0:
                assert an.sweeps < cold.sweeps, (c, an.sweeps, cold.sweeps)


def test_bad_seed_is_ignored():
    """A seed that is not orthonormal (or not finite) gives exactly the cold result."""
    p, n = 40, 8_000
    L, mu = inputs.wide_factor(2, p)
    X = inputs.gen_correlated_host(n, L, mu, seed=2)
    _, cols = _device_cols(X)
    with G.stats_init(G.Config([G.STATS_F64] * p, G.STATS_FP64_SHIFTED, [0] * p)) as ctx:
        G.stats_accumulate(ctx, cols, n)
        cold = G.stats_finalize_warm(ctx, 0)
        rnd = np.random.default_rng(0).standard_normal((p, p))
        nan = cold.evecs.copy()
        nan[3, 5] = np.nan
        near = cold.evecs * (1 + 1e-7)
        for seed in (rnd, nan, near):
            an = G.stats_finalize_warm(ctx, 0, seed)
            assert np.array_equal(an.evals, cold.evals) and np.array_equal(an.evecs, cold.evecs)
            assert an.sweeps == cold.sweeps
        # the exact previous result is accepted: it is already diagonalising
        again = G.stats_finalize_warm(ctx, 0, cold.evecs)
        assert again.sweeps <= 2
        _check_pairs(again, cold.cov, ev_tol=1e-13)
        with pytest.raises(ValueError):
            G.stats_finalize_warm(ctx, 0, np.eye(p - 1))


def test_small_width_seeded_and_undefined_pca():
    """p_a below the grid threshold with a seed still takes the grid-wide solver; a zero
    variance with pca_on = 1 leaves the eigenpairs undefined (NaN, sweeps -1)."""
    n = 5_000
    L, mu = inputs.wide_factor(8, 6)
    X = inputs.gen_correlated_host(n, L, mu, seed=8)
    _, cols = _device_cols(X)
    with G.stats_init(G.Config([G.STATS_F64] * 6, G.STATS_FP64_SHIFTED, [0] * 6)) as ctx:
        G.stats_accumulate(ctx, cols, n)
        cold = G.stats_finalize(ctx)
        an = G.stats_finalize_warm(ctx, 0, cold.evecs)
        assert an.sweeps >= 0
        _check_pairs(an, O.cov_twopass_columns(list(X)))
    Xz = X.copy()
    Xz[2] = 1.0
    _, cols = _device_cols(Xz)
    with G.stats_init(G.Config([G.STATS_F64] * 6, G.STATS_FP64_SHIFTED, [0] * 6)) as ctx:
        G.stats_accumulate(ctx, cols, n)
        an = G.stats_finalize_warm(ctx, 1, cold.evecs)
        assert an.sweeps == -1 and np.all(np.isnan(an.evals))


def test_correlated_generator_validation():
    """The paper's suggested check with known dependencies: rows of X = Z L^T + mu with
    population covariance Q diag(1/k) Q^T.  As the stream grows, the snapshot's leading
    eigenvalues approach 1/k within a few standard errors (sqrt(2/n) relative) and its
    leading eigenvectors approach Q's columns."""
    p, n_chunk, chunks = 32, 200_000, 5
    rng = np.random.default_rng(4)
    q, r = np.linalg.qr(rng.standard_normal((p, p)))
    q = q * np.sign(np.diag(r))
    L, mu = inputs.wide_factor(4, p)   # the same Q (seed 4, p = 32) as drawn above
    assert np.allclose(L @ L.T, (q / np.arange(1, p + 1)) @ q.T, atol=1e-12)
    cfg = G.Config([G.STATS_F32] * p, G.STATS_BF16X3, [0] * p)
    errs = []
    with G.StreamingAnalysis(cfg) as sa:
        for c in range(chunks):
            X = inputs.gen_correlated_host(n_chunk, L, mu, seed=40, row0=c * n_chunk).astype(np.float32)
            d, cols = _device_cols(X)
            sa.update(cols, n_chunk)
            torch.cuda.synchronize()
            del d
            an = sa.snapshot()
            n = (c + 1) * n_chunk
            k = np.arange(1, 6)
            rel = np.abs(an.evals[:5] * k - 1.0)
            assert np.all(rel <= 6 * np.sqrt(2.0 / n)), (n, rel)
            errs.append(1.0 - abs(float(an.evecs[0] @ q[:, 0])))
            assert errs[-1] <= 50.0 / n, (n, errs[-1])
    assert errs[-1] < errs[0]
