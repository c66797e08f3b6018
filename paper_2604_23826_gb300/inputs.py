"""Seeded synthetic inputs for the FP32 workloads (no statistics are computed here).

Two recipes, shared by the benchmark and the GPU tests:

* many independent tables: table t has n_t rows, n_t log-uniform on [1e3, 1e7], and
  p_t columns, p_t uniform on {8, 16, 32, 64}; column j is N(mu_j, sigma_j^2) in FP32
  with mu_j ~ U[1e3, 1e5] and sigma_j ~ U[0.1, 10] (a mean-to-spread ratio up to 1e6);
* one wide correlated table: X = Z L^T + mu with Z ~ N(0, 1) FP32, p = 256,
  L = chol(Q diag(1/k) Q^T) for a Haar-random Q (population eigenvalues exactly 1/k),
  mu_j ~ U[0, 1e3].

Shapes and parameters come from numpy's seeded generator; the Gaussian draws on the
device from torch's seeded device generator.  Tables are stored column-major
([p, n] tensors), so each column is one contiguous device array.
"""
from __future__ import annotations

import math

import numpy as np


def many_tables_shapes(seed: int, ntables: int, n_lo: float = 1e3, n_hi: float = 1e7):
    """(n_t, p_t, mu_t, sigma_t) for each table, from numpy's generator seeded `seed`."""
    rng = np.random.default_rng(seed)
    ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), ntables))).astype(np.int64)
    ps = rng.choice(np.array([8, 16, 32, 64]), ntables)
    params = []
    for t in range(ntables):
        mu = rng.uniform(1e3, 1e5, int(ps[t]))
        sd = rng.uniform(0.1, 10.0, int(ps[t]))
        params.append((int(ns[t]), int(ps[t]), mu, sd))
    return params


def check_sample(params, small_max: float = 1e6, n_small=None, n_large: int = 64):
    """Indices of the many-tables workload picked for a check against the CPU oracle.

    Every table of at most small_max rows (or n_small of them) and n_large of the larger
    tables; a subset is stratified by row count (evenly spaced ranks in order of n, so the
    whole range of sizes is represented), and the result is in table order."""
    def spread(idx, k):
        idx = sorted(idx, key=lambda t: (params[t][0], t))
        if k is None or k >= len(idx):
            return idx
        return [idx[int(round(i * (len(idx) - 1) / max(1, k - 1)))] for i in range(k)]
    small = [t for t, (n, _, _, _) in enumerate(params) if n <= small_max]
    large = [t for t, (n, _, _, _) in enumerate(params) if n > small_max]
    return sorted(set(spread(small, n_small)) | set(spread(large, n_large)))


def gen_table(torch, n: int, p: int, mu, sd, seed: int, device, out=None):
    """[p, n] float32 on `device`: row j ~ N(mu_j, sd_j^2) (FP32 after the affine map)."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    x = out if out is not None else torch.empty((p, n), dtype=torch.float32, device=device)
    x.normal_(0.0, 1.0, generator=g)
    x.mul_(torch.as_tensor(np.asarray(sd, dtype=np.float32), device=device)[:, None])
    x.add_(torch.as_tensor(np.asarray(mu, dtype=np.float32), device=device)[:, None])
    return x


def waves(params, max_bytes: int):
    """Split tables (in order) into groups whose FP32 bytes stay within max_bytes."""
    out, cur, size = [], [], 0
    for t, (n, p, _, _) in enumerate(params):
        b = 4 * n * p
        if cur and size + b > max_bytes:
            out.append(cur)
            cur, size = [], 0
        cur.append(t)
        size += b
    if cur:
        out.append(cur)
    return out


def wide_factor(seed: int, p: int = 256):
    """(L, mu): L = chol(Q diag(1/k) Q^T), Q Haar-random (QR of a Gaussian, signs fixed)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((p, p)))
    q = q * np.sign(np.diag(r))
    cov = (q * (1.0 / np.arange(1, p + 1))) @ q.T
    L = np.linalg.cholesky(cov)
    mu = rng.uniform(0.0, 1e3, p)
    return L, mu


def gen_wide(torch, n: int, L, mu, seed: int, device, chunk: int = 1 << 22, out=None):
    """[p, n] float32: X = Z L^T + mu, drawn in row chunks (Z chunk [rows, p] from a seeded generator)."""
    p = L.shape[0]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    x = out if out is not None else torch.empty((p, n), dtype=torch.float32, device=device)
    Lt = torch.as_tensor(L.T.astype(np.float32), device=device)
    m = torch.as_tensor(np.asarray(mu, dtype=np.float32), device=device)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        z = torch.randn((r1 - r0, p), generator=g, device=device, dtype=torch.float32)
        y = torch.addmm(m, z, Lt)
        x[:, r0:r1].copy_(y.t())
        del z, y
    return x


def gen_correlated_host(n: int, L, mu, seed: int, row0: int = 0, block: int = 1 << 16):
    """[p, n] float64 on the host: rows row0 .. row0 + n - 1 of X = Z L^T + mu, Z ~ N(0, 1).

    Row block b (rows b*block .. (b+1)*block - 1 of the whole table) draws its Z from numpy's
    generator seeded (seed, b), so any row range is reproducible without drawing the rows
    before it, and chunks of a stream equal the same rows of one long table."""
    L = np.asarray(L, dtype=np.float64)
    p = L.shape[0]
    out = np.empty((p, n), dtype=np.float64)
    r = row0
    while r < row0 + n:
        b = r // block
        z = np.random.default_rng([seed, b]).standard_normal((block, p))
        lo = r - b * block
        hi = min(block, row0 + n - b * block)
        out[:, r - row0:r - row0 + hi - lo] = (z[lo:hi] @ L.T + mu).T
        r = b * block + hi
    return out
