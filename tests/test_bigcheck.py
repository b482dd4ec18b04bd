"""Pins of the full-size check helpers (tests/bigcheck.py) on small inputs, on the CPU: the
parallel products equal the oracle's plain ones, and the randomized product check passes a
correct product and catches planted errors (one wrong entry, an error of 2^31, a wrong
block of rows)."""
import numpy as np

import bigcheck
import synth
from oracle import lwe


def _setup(R=300, C=257, k=5, seed=1):
    D = synth.database(R, C, seed)
    N = synth.uniform_queries(k, C, seed + 1).T.copy()     # C x k
    return D, N, lwe.matmat_mod_q(D, N)                    # M = D N mod 2^32 (R x k)


def test_parallel_products_equal_the_oracle():
    D, N, M = _setup()
    rows = [0, 3, 299, 150]
    assert np.array_equal(bigcheck.rows_product(D[rows], N, block=2), M[rows])
    W = synth.uniform_queries(16, 300, 9).T.copy()         # R x T
    U = bigcheck.left_projection(D, 257, W, cols=64, width=5)
    want = np.zeros((16, 257), dtype=np.uint64)            # brute force, mod 2^32
    for t in range(16):
        for r in range(300):
            want[t] = (want[t] + np.uint64(W[r, t]) * D[r].astype(np.uint64)) & np.uint64(0xFFFFFFFF)
    assert np.array_equal(U, want.astype(np.uint32))
    X = synth.uniform_queries(40, 77, 3)
    Y = synth.uniform_queries(33, 77, 4).T
    ref = (X.astype(object) @ Y.astype(object)) % 2**32
    assert np.array_equal(bigcheck.mod32_matmul_par(X, Y), ref.astype(np.uint32))
    assert np.array_equal(bigcheck.mod32_matmul_par(X, Y, along="rows"), ref.astype(np.uint32))


def test_freivalds_passes_and_catches_planted_errors():
    D, N, M = _setup()
    W = synth.uniform_queries(16, 300, 11).T.copy()
    U = bigcheck.left_projection(D, 257, W)
    assert bigcheck.freivalds(W, U, M, N).size == 0
    bad = M.copy()
    bad[7, 2] += np.uint32(1)
    assert list(bigcheck.freivalds(W, U, bad, N)) == [2]
    bad = M.copy()
    bad[123, 4] ^= np.uint32(1 << 31)                      # the hardest error: valuation 31
    assert list(bigcheck.freivalds(W, U, bad, N)) == [4]
    bad = M.copy()
    bad[128:256, 0] = bad[0:128, 0]                        # a wrong tile of 128 rows
    assert list(bigcheck.freivalds(W, U, bad, N)) == [0]
