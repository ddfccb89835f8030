"""Seeded synthetic sparse matrices shaped like the paper's workloads.

The paper's data (MovieLens, AMiner, SNAP; Sec. 4) are not available, so these
generators stand in for them: tall CSR matrices with log-normal row degrees,
Zipf-distributed column popularity (a few very hot columns, a long tail), and
tf-idf-like values.  This module holds no frPCA arithmetic; it only creates
inputs, and both the CUDA path's tests/benchmark and the CPU oracle read them.

Recipe of ``powerlaw_csr(m, n, deg_mean, zipf_s, values, seed)``:
  1. row degree d_i = clamp(round(LogNormal(mu, 1.0)), 1, n) with
     mu = ln(deg_mean) - 1/2, so E[d] ~ deg_mean;
  2. column ranks drawn from P(r) proportional to (r+1)^-s, r in [0, n), without
     replacement inside a row (duplicates redrawn), then mapped through a
     seeded random permutation of [0, n) so hot columns are scattered; rows
     are sorted; rows are drawn in blocks of 65,536, each block from its own
     Philox stream (threads build blocks in parallel; the matrix does not
     depend on their number);
  3. values: "tfidf": log(1 + c) * log(m / df_j), c ~ Poisson(2) conditioned on
     c >= 1, df_j the column count; "binary_tfidf": log(m / df_j); "uniform":
     U(0, 1).  A column present in every row gets value 0 (kept as a
     structural zero).
All randomness comes from numpy's Philox generator keyed by (seed, purpose).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class CSR:
    m: int
    n: int
    indptr: np.ndarray   # int64, m + 1
    indices: np.ndarray  # int32, nnz, sorted and unique within a row
    data: np.ndarray     # float32 or float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def astype(self, dtype) -> "CSR":
        return CSR(self.m, self.n, self.indptr, self.indices, self.data.astype(dtype))

    def to_dense(self) -> np.ndarray:
        A = np.zeros((self.m, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.m), np.diff(self.indptr))
        A[rows, self.indices] = self.data
        return A

    def row_ids(self) -> np.ndarray:
        return np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.indptr))


def _rng(seed: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([seed, purpose], dtype=np.uint64)))


def from_coo(m: int, n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """CSR from distinct (row, col) pairs in any order."""
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=indptr[1:])
    return CSR(m, n, indptr, cols.astype(np.int32), np.ascontiguousarray(vals))


def from_dense(A: np.ndarray, keep_zeros: bool = False) -> CSR:
    m, n = A.shape
    if keep_zeros:
        rows, cols = np.divmod(np.arange(m * n), n)
    else:
        rows, cols = np.nonzero(A)
    return from_coo(m, n, rows.astype(np.int64), cols.astype(np.int64), A[rows, cols].astype(np.float64))


def uniform_csr(m: int, n: int, nnz: int, seed: int = 1, dtype=np.float64) -> CSR:
    """Exactly ``nnz`` distinct positions drawn uniformly, values U(0, 1)."""
    rng = _rng(seed, 1)
    lin = np.sort(rng.choice(m * n, size=nnz, replace=False))
    rows, cols = np.divmod(lin, n)
    vals = _rng(seed, 2).random(nnz)
    return from_coo(m, n, rows, cols, vals.astype(dtype))


def _zipf_cdf(n: int, s: float) -> np.ndarray:
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


# Rows are generated in fixed blocks, each from its own Philox stream, so the
# matrix does not depend on how many threads build it.
_ROW_BLOCK = 1 << 16


def _block_rng(seed: int, purpose: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([seed, (purpose << 32) | block], dtype=np.uint64)))


def _powerlaw_block(b, r0, r1, indptr, n, cdf, perm, seed, cols_out):
    """Columns of rows r0 .. r1-1: Zipf ranks without repeats inside a row,
    mapped through perm, sorted within each row; written into cols_out."""
    rng = _block_rng(seed, 11, b)
    p0, p1 = int(indptr[r0]), int(indptr[r1])
    cnt = p1 - p0
    if cnt == 0:
        return

    def draw(k):
        r = np.searchsorted(cdf, rng.random(k), side="right")
        return np.minimum(r, n - 1).astype(np.int64)

    rows = np.repeat(np.arange(r1 - r0, dtype=np.int64), np.diff(indptr[r0:r1 + 1]))
    key = rows * n + draw(cnt)
    # Redraw repeated (row, rank) pairs until every row's ranks are distinct.
    while True:
        key.sort()
        dup = np.flatnonzero(key[1:] == key[:-1]) + 1
        if dup.size == 0:
            break
        key[dup] = (key[dup] // n) * n + draw(dup.size)
    key = rows * n + perm[key % n]
    key.sort()
    cols_out[p0:p1] = (key % n).astype(np.int32)


def powerlaw_csr(m: int, n: int, deg_mean: float, zipf_s: float, values: str = "tfidf",
                 seed: int = 1, dtype=np.float32, sigma_ln: float = 1.0, threads: int | None = None) -> CSR:
    import concurrent.futures
    import os

    rng_deg, rng_perm = _rng(seed, 10), _rng(seed, 12)
    mu = np.log(deg_mean) - 0.5 * sigma_ln ** 2
    deg = np.clip(np.rint(rng_deg.lognormal(mu, sigma_ln, size=m)), 1, n).astype(np.int64)
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(deg, out=indptr[1:])
    nnz = int(indptr[-1])
    cdf = _zipf_cdf(n, zipf_s)
    perm = rng_perm.permutation(n).astype(np.int64)
    cols = np.empty(nnz, dtype=np.int32)
    blocks = [(b, r0, min(m, r0 + _ROW_BLOCK)) for b, r0 in enumerate(range(0, m, _ROW_BLOCK))]
    workers = threads or min(16, os.cpu_count() or 1)
    if workers > 1 and len(blocks) > 1:
        with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(lambda t: _powerlaw_block(*t, indptr, n, cdf, perm, seed, cols), blocks))
    else:
        for t in blocks:
            _powerlaw_block(*t, indptr, n, cdf, perm, seed, cols)
    df = np.bincount(cols, minlength=n).astype(np.float64)
    idf = np.log(m / np.maximum(df, 1.0))
    if values == "tfidf":
        vals = np.empty(nnz, dtype=np.float64)
        for b, r0, r1 in blocks:
            p0, p1 = int(indptr[r0]), int(indptr[r1])
            rng_val = _block_rng(seed, 13, b)
            c = rng_val.poisson(2.0, size=p1 - p0)
            zero = np.flatnonzero(c == 0)
            while zero.size:
                c[zero] = rng_val.poisson(2.0, size=zero.size)
                zero = zero[c[zero] == 0]
            vals[p0:p1] = np.log1p(c.astype(np.float64)) * idf[cols[p0:p1]]
    elif values == "binary_tfidf":
        vals = idf[cols]
    elif values == "uniform":
        vals = np.empty(nnz, dtype=np.float64)
        for b, r0, r1 in blocks:
            p0, p1 = int(indptr[r0]), int(indptr[r1])
            vals[p0:p1] = _block_rng(seed, 13, b).random(p1 - p0)
    else:
        raise ValueError(values)
    return CSR(m, n, indptr, cols, vals.astype(dtype))


def gaussian_block(R: int, c: int, seed: int, purpose: int = 20, dtype=np.float64) -> np.ndarray:
    """Dense N(0,1) block for loss terms and test operands (not the method's randn)."""
    return _rng(seed, purpose).standard_normal((R, c)).astype(dtype)


# The workloads named by the benchmark configuration, by what they are.
WORKLOADS = {
    "uniform_2000x1000_nnz20000": dict(kind="uniform", m=2000, n=1000, nnz=20000, k=10, l=20, q=3, dtype="f64"),
    "powerlaw_200000x50000_deg100": dict(kind="powerlaw", m=200_000, n=50_000, deg_mean=100, zipf_s=1.1,
                                         values="tfidf", k=100, l=120, q=5, dtype="f32"),
    "powerlaw_1000000x200000_deg100": dict(kind="powerlaw", m=1_000_000, n=200_000, deg_mean=100, zipf_s=1.1,
                                           values="tfidf", k=100, l=120, q=5, dtype="f32"),
    "powerlaw_100000x20000_deg50": dict(kind="powerlaw", m=100_000, n=20_000, deg_mean=50, zipf_s=1.1,
                                        values="tfidf", k=32, l=48, q=4, dtype="f32"),
    "powerlaw_12000000x320000_deg40": dict(kind="powerlaw", m=12_000_000, n=320_000, deg_mean=40, zipf_s=1.05,
                                           values="binary_tfidf", k=100, l=120, q=5, dtype="f32"),
    # Stand-ins for the matrices of the shape comparison (Table 3): an
    # AMiner-sized 647,789 x 323,896 matrix with 16 entries per row (Matrix 4's
    # density), its first 107,966 columns (as Matrix 7 is cut from Matrix 6)
    # and its first 107,966 rows (as Matrix 8); k = 100, s = 5, q = 11.
    "powerlaw_647789x323896_deg16": dict(kind="powerlaw", m=647_789, n=323_896, deg_mean=16, zipf_s=1.05,
                                         values="tfidf", k=100, l=105, q=11, dtype="f32"),
    "powerlaw_647789x107966_cols": dict(kind="slice", base="powerlaw_647789x323896_deg16", m=647_789, n=107_966,
                                        k=100, l=105, q=11, dtype="f32"),
    "powerlaw_107966x323896_rows": dict(kind="slice", base="powerlaw_647789x323896_deg16", m=107_966, n=323_896,
                                        k=100, l=105, q=11, dtype="f32"),
}


def leading_block(A: CSR, m: int, n: int) -> CSR:
    """The first m rows and first n columns of A (entries keep their values)."""
    indptr = A.indptr[: m + 1]
    cols = A.indices[: indptr[-1]]
    vals = A.data[: indptr[-1]]
    keep = cols < n
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(indptr))[keep]
    out_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=out_ptr[1:])
    return CSR(m, n, out_ptr, np.ascontiguousarray(cols[keep]), np.ascontiguousarray(vals[keep]))


def make_workload(name: str, seed: int = 1, dtype=None) -> CSR:
    w = WORKLOADS[name]
    dt = dtype or (np.float64 if w["dtype"] == "f64" else np.float32)
    if w["kind"] == "uniform":
        return uniform_csr(w["m"], w["n"], w["nnz"], seed=seed, dtype=dt)
    if w["kind"] == "slice":
        return leading_block(make_workload(w["base"], seed=seed, dtype=dt), w["m"], w["n"])
    return powerlaw_csr(w["m"], w["n"], w["deg_mean"], w["zipf_s"], w["values"], seed=seed, dtype=dt)
