"""LWE matrix products mod q = 2^32 (oracle; test infrastructure only).

Algorithm "ZipPIR", Response: b = D^T qu_0 mod q. In the row-major R x C
orientation used by the library (R answers, C query entries), this is
ans[r] = sum_c D[r, c] q[c] mod 2^32: the plain definition, written out.

Algorithm "ZipPIR" caption: the global hint is H = -D^T A. The library returns the
positive product H+ = D A mod 2^32; the compression uses (-H+) mod 2^32.

numpy uint64 is exact here: a product is below 2^8 * 2^32 = 2^40, and a chunk of
at most 2^16 of them sums below 2^56, so nothing wraps before the explicit
reduction mod 2^32.
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
_CHUNK = 1 << 16


def matvec_mod_q(D: np.ndarray, q: np.ndarray) -> np.ndarray:
    """ans = D q mod 2^32 for D (R x C, entries < 2^8) and q (C,) u32. Returns u32 (R,)."""
    D = np.asarray(D)
    q = np.asarray(q, dtype=np.uint64)
    R, C = D.shape
    acc = np.zeros(R, dtype=np.uint64)
    for c0 in range(0, C, _CHUNK):
        part = D[:, c0:c0 + _CHUNK].astype(np.uint64) @ q[c0:c0 + _CHUNK]
        acc = (acc + (part & MASK32)) & MASK32
    return acc.astype(np.uint32)


def matmat_mod_q(D: np.ndarray, X: np.ndarray) -> np.ndarray:
    """D X mod 2^32 for D (R x C, entries < 2^8) and X (C x k) u32. Returns u32 (R, k).

    Used for batched answers (X = Q^T) and for the global hint H+ = D A.
    """
    D = np.asarray(D)
    X = np.asarray(X, dtype=np.uint64)
    R, C = D.shape
    acc = np.zeros((R, X.shape[1]), dtype=np.uint64)
    for c0 in range(0, C, _CHUNK):
        part = D[:, c0:c0 + _CHUNK].astype(np.uint64) @ X[c0:c0 + _CHUNK]
        acc = (acc + (part & MASK32)) & MASK32
    return acc.astype(np.uint32)


def hint_plus(D: np.ndarray, A: np.ndarray) -> np.ndarray:
    """H+ = D A mod 2^32 (R x n)."""
    return matmat_mod_q(D, A)


def hint_neg(D: np.ndarray, A: np.ndarray) -> np.ndarray:
    """The paper's hint H = -D A mod 2^32 (Algorithm "ZipPIR" caption)."""
    Hp = hint_plus(D, A).astype(np.uint64)
    return ((np.uint64(1 << 32) - Hp) & MASK32).astype(np.uint32)
