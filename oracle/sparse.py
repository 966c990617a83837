"""ORACLE -- test infrastructure only: sparse matrix-vector products and the
conjugate-gradient solver (Sec. 3.2.6), in binary64.

A matrix is CSR: rowptr (nrows + 1, int64), col (int32), val.

* `spmv(rowptr, col, val, x)`: y_i = sum_k val[k] * x[col[k]] over row i, and
  sum_k |val[k] * x[col[k]]| (for error bounds), by the definition.
* `cg(rowptr, col, val, b, x0, rtol, maxit)`: conjugate gradients
  (Hestenes-Stiefel): r = b - A x, p = r, rs = r.r; repeat while
  ||r|| > rtol ||b|| and fewer than maxit steps: q = A p, alpha = rs / p.q,
  x += alpha p, r -= alpha q, rs' = r.r, p = r + (rs' / rs) p, rs = rs'.
  Returns (x, steps, [||r_k||]).
"""
from __future__ import annotations

import numpy as np


def _rows(rowptr):
    return np.repeat(np.arange(rowptr.size - 1, dtype=np.int64), np.diff(rowptr))


def spmv(rowptr, col, val, x):
    rowptr = np.asarray(rowptr, np.int64)
    prod = np.asarray(val, np.float64) * np.asarray(x, np.float64)[np.asarray(col, np.int64)]
    rows = _rows(rowptr)
    n = rowptr.size - 1
    return (np.bincount(rows, weights=prod, minlength=n),
            np.bincount(rows, weights=np.abs(prod), minlength=n))


def cg(rowptr, col, val, b, x0, rtol, maxit, directions=False):
    b = np.asarray(b, np.float64)
    x = np.array(x0, np.float64)
    r = b - spmv(rowptr, col, val, x)[0]
    p = r.copy()
    rs = float(r @ r)
    tol2 = rtol * rtol * float(b @ b)
    hist = [np.sqrt(rs)]
    dirs = [p.copy()] if directions else None
    k = 0
    while rs > tol2 and k < maxit:
        q = spmv(rowptr, col, val, p)[0]
        pq = float(p @ q)
        if pq == 0:
            break
        alpha = rs / pq
        x += alpha * p
        r -= alpha * q
        rs_new = float(r @ r)
        p = r + (rs_new / rs) * p
        rs = rs_new
        k += 1
        hist.append(np.sqrt(rs))
        if directions:
            dirs.append(p.copy())
    if directions:
        return x, k, hist, dirs
    return x, k, hist
