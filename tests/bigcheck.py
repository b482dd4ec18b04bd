"""Checks of full-size GPU results that the oracle cannot recompute whole within a test's
time (test infrastructure, like the oracle it calls).

* ``rows_product``: D[rows] X mod 2^32 by the oracle's ``lwe.matmat_mod_q``, in row
  blocks spread over the host cores (numpy releases the GIL inside its integer matrix
  products, so threads run in parallel).
* ``left_projection`` and ``freivalds``: a randomized check of a whole product M = D N
  mod 2^32 (Freivalds): with W an R x T matrix of uniform u32, W^T M must equal
  (W^T D) N mod 2^32. U = W^T D is one pass of the oracle's products over D, shared by
  every product checked against the same D. For an error matrix E = M - D N whose nonzero
  column has an entry of 2-adic valuation v (and none lower), each column of W misses it
  with probability exactly 2^-(32 - v), so T columns miss it with probability
  2^-T(32 - v): at most 2^-T, and at most 2^-2T unless every error in that column is a
  multiple of 2^31.

Products of u32 values mod 2^32 are taken in numpy uint64: the products and sums wrap mod
2^64, and since 2^32 divides 2^64 the result mod 2^32 is exact.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from oracle import lwe


def host_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def mod32_matmul(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """X Y mod 2^32 for u32 matrices (uint64 wrap-around, exact mod 2^32)."""
    return (X.astype(np.uint64) @ Y.astype(np.uint64)).astype(np.uint32)


def _split(n: int, parts: int) -> list[tuple[int, int]]:
    step = max(1, -(-n // parts))
    return [(a, min(n, a + step)) for a in range(0, n, step)]


def mod32_matmul_par(X: np.ndarray, Y: np.ndarray, along: str = "k") -> np.ndarray:
    """X Y mod 2^32 with the work split over the host cores: along the inner dimension
    (partial products summed mod 2^32) or along the rows of X."""
    nt = host_threads()
    with ThreadPoolExecutor(nt) as ex:
        if along == "rows":
            parts = list(ex.map(lambda ab: mod32_matmul(X[ab[0]:ab[1]], Y), _split(X.shape[0], nt)))
            return np.concatenate(parts, axis=0)
        parts = list(ex.map(lambda ab: mod32_matmul(X[:, ab[0]:ab[1]], Y[ab[0]:ab[1]]),
                            _split(X.shape[1], 4 * nt)))
    acc = np.zeros(parts[0].shape, dtype=np.uint64)
    for p in parts:
        acc += p
    return (acc & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def rows_product(Drows: np.ndarray, X: np.ndarray, block: int = 16, fn=lwe.matmat_mod_q) -> np.ndarray:
    """Drows X mod 2^32 (Drows: r x C bytes, X: C x k u32) by the oracle's matmat_mod_q (or
    another row-wise oracle product ``fn``, such as lwe.hint_neg) in row blocks run on all
    host cores."""
    blocks = [(a, min(Drows.shape[0], a + block)) for a in range(0, Drows.shape[0], block)]
    with ThreadPoolExecutor(host_threads()) as ex:
        parts = list(ex.map(lambda ab: fn(Drows[ab[0]:ab[1]], X), blocks))
    return np.concatenate(parts, axis=0)


def left_projection(D: np.ndarray, C: int, W: np.ndarray, cols: int = 256,
                    width: int = 8) -> np.ndarray:
    """U = W^T D[:, :C] mod 2^32 (T x C) for D (R x >= C bytes) and W (R x T u32): the
    oracle's matmat_mod_q on column blocks of D (as D^T blocks, C x R bytes), at most
    ``width`` columns of W at a time (numpy's integer products slow down on wide operands)."""
    R, T = W.shape
    U = np.zeros((T, C), dtype=np.uint32)

    def block(c0):
        c1 = min(C, c0 + cols)
        Dt = np.ascontiguousarray(D[:, c0:c1].T)
        for t0 in range(0, T, width):
            U[t0:t0 + width, c0:c1] = lwe.matmat_mod_q(Dt, W[:, t0:t0 + width]).T

    with ThreadPoolExecutor(host_threads()) as ex:
        list(ex.map(block, range(0, C, cols)))
    return U


def freivalds(W: np.ndarray, U: np.ndarray, M: np.ndarray, N: np.ndarray) -> np.ndarray:
    """Columns j of M (R x k) that fail W^T M[:, j] = U N[:, j] mod 2^32, with U = W^T D
    and N (C x k): an empty array when M = D N passes."""
    left = mod32_matmul_par(W.T, M)            # T x k
    right = mod32_matmul_par(U, N)             # T x k
    return np.nonzero(np.any(left != right, axis=0))[0]
