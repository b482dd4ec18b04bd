"""Compression of LWE ciphertexts and RLWE coefficients into Paillier ciphertexts
(Sec. 3), oracle / test infrastructure only.

Plain Python integers. The additive scheme is Paillier with g = m + 1
(`oracle.paillier`); its homomorphic addition is multiplication mod m^2 and the
plaintext multiplication a (x) c is c^a mod m^2.

  LWE         ct = (a, b), a in Z_q^n, b = <a, s> + Delta mu + e mod q, Delta = round(q / p)
  LWECompress x = Enc(b; 1) (+) sum_i ((q - a[i]) mod q) (x) ck[i],  ck[i] = Enc(s[i])
              (Algorithm "LWE compression"): Dec(x) = b + sum_i ((q - a[i]) mod q) s[i]
              < q + n q^2 <= m, and Dec(x) mod q = b - <a, s> mod q
  Batched     x = sum_j gamma^j (x) x_j, gamma = q + n q^2 (binary s: q + n q), ell slots
              with gamma^ell < m (Algorithm "Batch Compression")
  Fast        the same x from the expanded key eck[j][i] = 2^j (x) ck[i] (Algorithm "Batch
              compression of LWE ciphertexts using precomputed powers")
  RLWE        coefficient k of the phase B - A S in Z_q[X]/(X^N + 1) (Algorithm
              "Compressing Extracted RLWE Coefficient", App. B)
  Packed key  t slots of delta per Paillier ciphertext, unpacked by the server with
              plaintext multiplications by powers of delta (App. "LWECompress Using Packed
              Compression Keys")

Readings: the initial x = b of the algorithms is b encrypted with randomness 1, i.e.
1 + b m mod m^2; the exponent of a coefficient is (q - a) mod q (so a = 0 gives 0);
rounding ties go up (round(v / Delta) = floor((2 v + Delta) / (2 Delta))); q may be
2^64 (the Concrete parameter sets) or any modulus below it.
"""
from __future__ import annotations

import numpy as np

from . import paillier


def delta_of(q: int, p: int) -> int:
    """Delta = round(q / p), ties up."""
    return (2 * q + p) // (2 * p)


def round_div(v: int, d: int) -> int:
    """round(v / d) for v >= 0, ties up."""
    return (2 * v + d) // (2 * d)


def gamma_of(q: int, n: int, binary: bool) -> int:
    """Slot scale of batched compression: q + n q^2, or q + n q for binary secrets."""
    return q + n * q * q if not binary else q + n * q


def max_slots(m: int, gamma: int) -> int:
    """Largest ell with gamma^ell < m (the condition of the batched correctness theorem)."""
    ell = 0
    while gamma ** (ell + 1) < m:
        ell += 1
    return ell


# ----------------------------------------------------------------------------- LWE
def lwe_keygen(n: int, q: int, binary: bool, g: np.random.Generator) -> list[int]:
    if binary:
        return [int(x) for x in g.integers(0, 2, size=n)]
    return [int.from_bytes(g.bytes(8), "little") % q for _ in range(n)]


def lwe_encrypt(s: list[int], mu: int, q: int, p: int, g: np.random.Generator,
                sigma: float = 3.2) -> tuple[list[int], int]:
    """b = <a, s> + Delta mu + e mod q with a uniform and e a rounded Gaussian (client side;
    the noise distribution does not enter compression)."""
    a = [int.from_bytes(g.bytes(8), "little") % q for _ in range(len(s))]
    e = int(np.rint(g.normal(0.0, sigma)))
    b = (sum(ai * si for ai, si in zip(a, s)) + delta_of(q, p) * mu + e) % q
    return a, b


def lwe_phase(s: list[int], a: list[int], b: int, q: int) -> int:
    """mu* = b - <a, s> mod q."""
    return (b - sum(ai * si for ai, si in zip(a, s))) % q


def lwe_decrypt(s: list[int], a: list[int], b: int, q: int, p: int) -> int:
    return round_div(lwe_phase(s, a, b, q), delta_of(q, p)) % p


def compression_key(pk: paillier.PublicKey, s: list[int], g: np.random.Generator,
                    shared_randomness: bool = False) -> list[int]:
    """ck[i] = Enc(s[i]) with fresh randomness; with ``shared_randomness`` every entry uses
    the same r (valid ciphertexts that decrypt alike, one r^m instead of n: for tests of
    large n only, not a secure key)."""
    m, m2 = pk.m, pk.m2
    draw = lambda: int.from_bytes(g.bytes(pk.m.bit_length() // 8 + 8), "little") % (m - 2) + 2
    if shared_randomness:
        rho = pow(draw(), m, m2)
        return [(1 + (si % m) * m) * rho % m2 for si in s]
    return [paillier.encrypt(pk, si, draw()) for si in s]


def trivial(pk: paillier.PublicKey, x: int) -> int:
    """x encrypted with randomness 1: (1 + m)^x = 1 + x m mod m^2."""
    return (1 + x * pk.m) % pk.m2


def lwe_compress(pk: paillier.PublicKey, ck: list[int], a: list[int], b: int, q: int) -> int:
    """Algorithm "LWE compression": x = b; x <- x (+) ((q - a[i]) (x) ck[i]) for every i."""
    x = trivial(pk, b)
    for ai, c in zip(a, ck):
        x = paillier.add(pk, x, paillier.smul(pk, (q - ai) % q, c))
    return x


def modified_lwe_decrypt(sk: paillier.SecretKey, x: int, q: int, p: int) -> int:
    """mu** = Dec(x) mod q, then round(mu** / Delta)."""
    return round_div(paillier.decrypt(sk, x) % q, delta_of(q, p)) % p


def expand_compression_key(pk: paillier.PublicKey, ck: list[int], t: int) -> list[list[int]]:
    """eck[0] = ck, eck[j + 1][i] = eck[j][i] (+) eck[j][i]  (so eck[j][i] = 2^j (x) ck[i])."""
    eck = [list(ck)]
    for _ in range(t - 1):
        eck.append([paillier.add(pk, c, c) for c in eck[-1]])
    return eck


def fast_lwe_compress(pk: paillier.PublicKey, eck: list[list[int]], a: list[int], b: int, q: int) -> int:
    """x = b; for every i and every set bit j of (q - a[i]) mod q: x <- x (+) eck[j][i]."""
    t = len(eck)
    x = trivial(pk, b)
    for i, ai in enumerate(a):
        e = (q - ai) % q
        assert e < (1 << t)
        for j in range(t):
            if (e >> j) & 1:
                x = paillier.add(pk, x, eck[j][i])
    return x


def batched_lwe_compress(pk: paillier.PublicKey, ck: list[int], cts, q: int, gamma: int) -> int:
    """Algorithm "Batch Compression": x = sum_j gamma^j (x) LWECompress(ck, c_j), starting
    from the encryption of 0 with randomness 1."""
    x = 1
    for j, (a, b) in enumerate(cts):
        xj = lwe_compress(pk, ck, a, b, q)
        x = paillier.add(pk, x, paillier.smul(pk, gamma ** j, xj))
    return x


def modified_batched_decrypt(sk: paillier.SecretKey, x: int, q: int, p: int, gamma: int,
                             ell: int) -> list[int]:
    """mu_j** = floor(Dec(x) / gamma^j) mod gamma, then round((mu_j** mod q) / Delta)."""
    mu = paillier.decrypt(sk, x)
    d = delta_of(q, p)
    return [round_div((mu // gamma ** j) % gamma % q, d) % p for j in range(ell)]


def rescale(a: list[int], b: int, q: int, r: int) -> tuple[list[int], int]:
    """Modulus switching before compression (Sec. 3.3, "Rescaling for Compression"): every
    coefficient x of (a, b) becomes round(x r / q) mod r, ties up, i.e.
    floor((x r + floor(q / 2)) / q) mod r. The ciphertext then lives modulo r < q; the
    paper states (proof not in its text) that it still decrypts for binary keys when the
    noise stays below Delta / 4."""
    f = lambda x: ((x * r + q // 2) // q) % r
    return [f(x) for x in a], f(b)


# ----------------------------------------------------------------------------- RLWE
def negacyclic_mul(A: list[int], S: list[int], q: int) -> list[int]:
    """A S in Z_q[X]/(X^N + 1): X^N = -1, so the term A[j] S[i] lands on X^(i + j) with sign
    + when i + j < N and on X^(i + j - N) with sign - otherwise."""
    N = len(A)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            if i + j < N:
                out[i + j] += A[j] * S[i]
            else:
                out[i + j - N] -= A[j] * S[i]
    return [v % q for v in out]


def rlwe_encrypt(S: list[int], mu: list[int], q: int, p: int, g: np.random.Generator,
                 sigma: float = 3.2) -> tuple[list[int], list[int]]:
    """B = A S + Delta mu + E mod q (Algorithm "Encryption and Decryption of E_RLWE")."""
    N = len(S)
    A = [int.from_bytes(g.bytes(8), "little") % q for _ in range(N)]
    E = [int(v) for v in np.rint(g.normal(0.0, sigma, size=N))]
    AS = negacyclic_mul(A, S, q)
    d = delta_of(q, p)
    return A, [(AS[k] + d * mu[k] + E[k]) % q for k in range(N)]


def rlwe_decrypt(S: list[int], A: list[int], B: list[int], q: int, p: int) -> list[int]:
    AS = negacyclic_mul(A, S, q)
    d = delta_of(q, p)
    return [round_div((B[k] - AS[k]) % q, d) % p for k in range(len(B))]


def rlwe_compress_coefficient(pk: paillier.PublicKey, ck: list[int], A: list[int], B: list[int],
                              k: int, q: int) -> int:
    """Algorithm "Compressing Extracted RLWE Coefficient": x = B[k];
    x <- x (+) ((q - A[k - i]) mod q) (x) ck[i] for i <= k, and x <- x (+) A[N + k - i] (x) ck[i]
    for i > k."""
    N = len(A)
    x = trivial(pk, B[k])
    for i in range(k + 1):
        x = paillier.add(pk, x, paillier.smul(pk, (q - A[k - i]) % q, ck[i]))
    for i in range(k + 1, N):
        x = paillier.add(pk, x, paillier.smul(pk, A[N + k - i], ck[i]))
    return x


# ----------------------------------------------------------------------------- packed keys
def packed_slots(m: int, delta: int) -> int:
    """t = floor(0.5 log2 m / log2 delta), taken as the largest t with delta^(2t) <= m."""
    t = 0
    while delta ** (2 * (t + 1)) <= m:
        t += 1
    return t


def generate_packed_key(pk: paillier.PublicKey, s: list[int], delta: int, t: int,
                        g: np.random.Generator) -> list[int]:
    """pck_i = Enc(delta^-(t-1) sum_{j<t} s[i t + j] delta^j mod m), i < ceil(n / t)."""
    m = pk.m
    dinv = pow(pow(delta, t - 1, m), -1, m)
    out = []
    for i in range((len(s) + t - 1) // t):
        v = sum(s[i * t + j] * delta ** j for j in range(t) if i * t + j < len(s))
        r = int.from_bytes(g.bytes(m.bit_length() // 8 + 8), "little") % (m - 2) + 2
        out.append(paillier.encrypt(pk, dinv * v % m, r))
    return out


def unpack_compression_key(pk: paillier.PublicKey, pck: list[int], delta: int, t: int, n: int) -> list[int]:
    """ck[i t + j] = delta^(t-1-j) (x) pck[i]."""
    return [paillier.smul(pk, delta ** (t - 1 - j), pck[i])
            for i in range(len(pck)) for j in range(t) if i * t + j < n]


def modified_lwe_decrypt_packed(sk: paillier.SecretKey, x: int, q: int, p: int, delta: int,
                                t: int) -> int:
    """y = delta^(t-1) Dec(x) mod m; mu** = floor(y / delta^(t-1)) mod q; round(mu** / Delta)."""
    m = sk.m
    y = pow(delta, t - 1) * paillier.decrypt(sk, x) % m
    mu = (y // delta ** (t - 1)) % q
    return round_div(mu, delta_of(q, p)) % p
