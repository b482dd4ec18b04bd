"""ZipPIR server Response and client (oracle; test infrastructure only).

Follows Algorithm "ZipPIR" (Sec. 4.2) with the extensions the paper's final
construction uses (Sec. 4.3, "Batched compression for smaller responses",
"Lowering offline communication costs"; Sec. 4.4 says the first three extensions
are in it). In the row-major orientation of the library:

  D      R x C database, entries in Z_p            (paper: db^T, d1 = R, d0 = C)
  A      C x n public LWE matrix
  H+     D A mod q;  Hneg = -H+ mod q               (paper's hint H = -db^T A)
  qu     C-vector:  A sk + e + Delta u_{i0} mod q    (Query)
  ans    D qu mod q                                  (Response, first product)
  b'     b'[r'] = sum_{j<ell} gamma^j ans[r' ell + j]       (batched compression,
  H'     H'[r', i] = sum_{j<ell} gamma^j Hneg[r' ell + j, i]  Algorithm "Batch
                                                             Compression", Sec. 3.3)
  t      t[r'] = (b'[r'] + sum_i H'[r', i] cko[i]) mod m     (Response, second product)
  k      k[r'] = PaillierMatMul_m(H', ck_r)[r']               (Hint)
  mu     (t + Dec(k)) mod m = b' + H' sk  exactly             (proof of Thm. 2, App. D)
  slots  mu_j = floor(mu / gamma^j) mod gamma;  f = round((mu_j mod q) p / q) mod p

Readings (where the paper is silent or loose):
  * rows past R in the last packed row are zero (the paper's d1' = floor(d1/gamma)
    would drop them);
  * slot j of packed row r' holds answer row r' ell + j (j = 0 least significant);
  * rounding ties go up: round(v p / q) = floor((2 v p + q) / (2 q));
  * the discrete Gaussian is sampled on [-10 sigma, 10 sigma] with probabilities
    proportional to exp(-x^2 / (2 sigma^2)) (client side only);
  * the query secret is uniform in Z_q (default) or binary (the algorithm's own
    choice); the packing scale follows the secret.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import chacha20, lwe, paillier
from .params import Params, Q

# Nonces (domain tags) of the ChaCha20 expansions: the ASCII tag, zero-padded to 12 bytes.
NONCE_A = b"A" + bytes(11)
NONCE_CKR = b"ckr" + bytes(9)


def expand_matrix(key: bytes, rows: int, cols: int, nonce: bytes = NONCE_A) -> np.ndarray:
    """The public matrix A (rows x cols u32) from a 32-byte seed: entry (r, c) is keystream
    word r cols + c (block counter from 0). A is uniform in Z_q^{rows x cols} with q = 2^32,
    so the words are used as they are (Sec. 2.1.1)."""
    w = chacha20.keystream_words(key, nonce, 0, rows * cols)
    return np.array(w, dtype=np.uint32).reshape(rows, cols)


def expand_ck_r(key: bytes, pk: paillier.PublicKey, key_bits: int, count: int,
                nonce: bytes = NONCE_CKR, counter0: int = 0) -> list[int]:
    """ck_r from a 32-byte seed (Sec. 4.3, offline communication): element i is the
    integer of 2 key_bits + 128 bits in keystream words [W i, W (i + 1)), W = (2 key_bits +
    128) / 32, little-endian, reduced mod m^2, so that its distance from uniform on
    Z_{m^2} is below 2^-128."""
    W = (2 * key_bits + 128) // 32
    w = chacha20.keystream_words(key, nonce, counter0, W * count)
    m2 = pk.m2
    out = []
    for i in range(count):
        v = 0
        for x in reversed(w[W * i:W * (i + 1)]):
            v = (v << 32) | x
        out.append(v % m2)
    return out


# ----------------------------------------------------------------------------- packing
def pack(values, params: Params) -> list[int]:
    """b'[r'] = sum_{j<ell} gamma^j values[r' ell + j]  (Algorithm "Batch Compression")."""
    vals = [int(v) for v in values]
    ell, g = params.ell, params.gamma
    out = []
    for r0 in range(0, len(vals), ell):
        acc = 0
        for j, v in enumerate(vals[r0:r0 + ell]):
            acc += v * g ** j
        out.append(acc)
    return out


def unpack(mu: int, params: Params) -> list[int]:
    """mu_j = floor(mu / gamma^j) mod gamma for j < ell  (ModifiedBatchedLWEDecrypt)."""
    g = params.gamma
    return [(mu // g ** j) % g for j in range(params.ell)]


def packed_hint_row(Hneg: np.ndarray, rp: int, params: Params) -> list[int]:
    """H'[rp, :] = sum_j gamma^j Hneg[rp ell + j, :] (rows past R are zero)."""
    ell, g = params.ell, params.gamma
    R, n = Hneg.shape
    row = [0] * n
    for j in range(ell):
        r = rp * ell + j
        if r >= R:
            break
        gj = g ** j
        hr = Hneg[r]
        for i in range(n):
            row[i] += int(hr[i]) * gj
    return row


# ----------------------------------------------------------------------------- server
def compress_rows(ans: np.ndarray, Hneg: np.ndarray, cko, m: int, params: Params,
                  packed_rows=None) -> list[int]:
    """t[r'] = (b'[r'] + sum_i H'[r', i] cko[i]) mod m  (Algorithm "ZipPIR", Response).

    ``ans`` is the full answer vector (R,), ``Hneg`` the R x n negated hint,
    ``cko`` the n offsets (each < m). Returns t for ``packed_rows`` (default: all).
    """
    R = len(ans)
    d1p = params.d1p(R)
    rows = range(d1p) if packed_rows is None else packed_rows
    ell = params.ell
    out = []
    for rp in rows:
        bp = pack(ans[rp * ell:min(R, (rp + 1) * ell)], params)[0]
        hrow = packed_hint_row(Hneg, rp, params)
        acc = bp
        for i, c in enumerate(cko):
            acc += hrow[i] * int(c)
        out.append(acc % m)
    return out


def response(D: np.ndarray, qu: np.ndarray, Hneg: np.ndarray, cko, m: int,
             params: Params) -> tuple[np.ndarray, list[int]]:
    """The full server Response: (ans, t)."""
    ans = lwe.matvec_mod_q(D, qu)
    return ans, compress_rows(ans, Hneg, cko, m, params)


# ----------------------------------------------------------------------------- client
def discrete_gaussian(count: int, sigma: float, g: np.random.Generator) -> np.ndarray:
    """Errors e ~ chi: discrete Gaussian on [-10 sigma, 10 sigma] (int64)."""
    bound = int(np.ceil(10 * sigma))
    xs = np.arange(-bound, bound + 1)
    w = np.exp(-(xs.astype(np.float64) ** 2) / (2.0 * sigma * sigma))
    return g.choice(xs, size=count, p=w / w.sum()).astype(np.int64)


@dataclass
class Client:
    params: Params
    pk: paillier.PublicKey
    sk: paillier.SecretKey
    ck_r: list[int] = field(default_factory=list)   # random compression-key part, in Z_{m^2}
    pt_r: list[int] = field(default_factory=list)   # Dec(ck_r)


def setup(params: Params, seed: int, sample_ck_r: bool = True) -> Client:
    """Setup: Paillier keys, ck_r sampled uniformly from Z_{m^2} by a seeded PRG
    (Sec. 4.3, "Lowering offline communication costs"), pt_r = Dec(ck_r).

    With ``sample_ck_r=False`` the client draws pt_r uniformly from Z_m and keeps
    no ck_r: the distribution H1 of the security proof (App. D), equal to Dec of a
    uniform ck_r up to the negligible chance of an invalid ciphertext. It skips n
    Paillier decryptions on instances whose hint k is replaced by
    ``dec_k_shortcut``.
    """
    pk, sk = paillier.keygen(params.key_bits, seed)
    g = np.random.Generator(np.random.PCG64([int(seed), 202]))
    if not sample_ck_r:
        nb = pk.m.bit_length() + 128
        pt_r = [paillier._rand_bits(g, nb) % pk.m for _ in range(params.n)]
        return Client(params, pk, sk, [], pt_r)
    m2 = pk.m2
    nb = m2.bit_length() + 128
    ck_r = [paillier._rand_bits(g, nb) % m2 for _ in range(params.n)]
    pt_r = [paillier.decrypt(sk, c) for c in ck_r]
    return Client(params, pk, sk, ck_r, pt_r)


@dataclass
class Query:
    cko: list[int]        # compression-key offsets, each in Z_m
    qu: np.ndarray        # u32 (C,)
    lwe_sk: np.ndarray    # the query's LWE secret (uint64 values < q)
    i0: int


def query(client: Client, A: np.ndarray, i0: int, seed: int) -> Query:
    """Query: fresh LWE secret, cko = (sk - pt_r) mod m, qu = A sk + e + Delta u_{i0} mod q."""
    P = client.params
    C, n = A.shape
    assert n == P.n
    g = np.random.Generator(np.random.PCG64([int(seed), 303]))
    if P.secret == "uniform":
        s = g.integers(0, Q, size=n, dtype=np.uint64)
    else:
        s = g.integers(0, 2, size=n, dtype=np.uint64)
    m = client.pk.m
    cko = [(int(s[i]) - client.pt_r[i]) % m for i in range(n)]
    e = discrete_gaussian(C, P.sigma, g)
    # A s mod 2^32: uint64 arithmetic wraps mod 2^64, which is exact mod 2^32.
    As = (A.astype(np.uint64) @ s) & np.uint64(0xFFFFFFFF)
    u = np.zeros(C, dtype=np.uint64)
    u[i0] = P.delta
    qu = (As + e.astype(np.uint64) + u) & np.uint64(0xFFFFFFFF)   # e < 0 wraps mod 2^64
    return Query(cko, qu.astype(np.uint32), s, i0)


def paillier_matmul_rows(client: Client, Hneg: np.ndarray, packed_rows) -> list[int]:
    """Hint: k[r'] = PaillierMatMul_m(H', ck_r)[r'] = prod_i ck_r[i]^{H'[r', i]} mod m^2."""
    pk = client.pk
    out = []
    for rp in packed_rows:
        hrow = packed_hint_row(Hneg, rp, client.params)
        acc = 1
        for i, h in enumerate(hrow):
            acc = paillier.add(pk, acc, paillier.smul(pk, h, client.ck_r[i]))
        out.append(acc)
    return out


def combine(pk: paillier.PublicKey, k: list[int], t: list[int]) -> list[int]:
    """Combined response k (+) t (Sec. 4.3, last extension): the homomorphic sum of the
    hint ciphertext k[r'] and t[r'] encrypted with randomness 1, one ciphertext per packed
    row, so that Dec(k (+) t) = Dec(k) + t mod m."""
    return [paillier.add(pk, kk, paillier.encrypt(pk, tt, 1)) for kk, tt in zip(k, t)]


def dec_k_shortcut(client: Client, Hneg: np.ndarray, packed_rows) -> list[int]:
    """Dec(k[r']) through the homomorphic identity Dec(k[r']) = H'[r', :] . pt_r mod m.

    A stand-in for decrypting the real per-client hint k on instances where
    computing k (n modular exponentiations per packed row) is too slow; the real
    path is ``paillier_matmul_rows`` followed by ``paillier.decrypt``.
    """
    m = client.pk.m
    out = []
    for rp in packed_rows:
        hrow = packed_hint_row(Hneg, rp, client.params)
        out.append(sum(h * p for h, p in zip(hrow, client.pt_r)) % m)
    return out


def extract(client: Client, dec_k: list[int], t: list[int], R: int) -> np.ndarray:
    """Extract: mu = (t + Dec(k)) mod m, unpack the slots, round each to Z_p.

    Returns the recovered record (R,) as uint8 (p <= 256) or int64.
    """
    P = client.params
    m = client.pk.m
    out = []
    for rp, (tv, dk) in enumerate(zip(t, dec_k)):
        mu = (tv + dk) % m
        for j, mj in enumerate(unpack(mu, P)):
            if rp * P.ell + j >= R:
                break
            v = mj % Q
            out.append(((2 * v * P.p + Q) // (2 * Q)) % P.p)
    dt = np.uint8 if P.p <= 256 else np.int64
    return np.array(out, dtype=dt)
