"""Pins of the LWE/RLWE compression oracle (Sec. 3, App. B, packed-key appendix) against
what the paper's theorems fix: a compressed ciphertext decrypts to the LWE (or RLWE
coefficient) decryption of what it compressed, the batched form to every slot, the
packed key to the same message; the fast form equals the plain one; the negacyclic
product equals a polynomial product folded by X^N = -1 computed by numpy."""
import numpy as np
import pytest

from oracle import lwecompress as lc
from oracle import paillier

Q64 = 1 << 64
Q27 = 134217689  # a prime below 2^27 (checked below)


@pytest.fixture(scope="module")
def keys():
    return paillier.keygen(512, 77)


def _cts(s, q, p, count, g):
    mus = [int(g.integers(0, p)) for _ in range(count)]
    return mus, [lc.lwe_encrypt(s, mu, q, p, g) for mu in mus]


def test_q27_is_prime():
    sympy = pytest.importorskip("sympy")
    assert sympy.isprime(Q27) and Q27 < 2 ** 27


@pytest.mark.parametrize("n,q,p,binary", [(16, Q64, 16, False), (24, 1 << 11, 4, False),
                                          (12, Q27, 8, True), (20, Q64, 2, True)])
def test_lwe_compress_correct(keys, n, q, p, binary):
    """Theorem "Correctness" (Sec. 3.1): Dec(x) = b + sum_i ((q - a_i) mod q) s_i < q + n q^2
    exactly, its residue mod q is the LWE phase, and the modified decryption gives the
    message."""
    pk, sk = keys
    g = np.random.default_rng(n)
    s = lc.lwe_keygen(n, q, binary, g)
    ck = lc.compression_key(pk, s, g)
    mus, cts = _cts(s, q, p, 3, g)
    for mu, (a, b) in zip(mus, cts):
        x = lc.lwe_compress(pk, ck, a, b, q)
        dec = paillier.decrypt(sk, x)
        assert dec == b + sum(((q - ai) % q) * si for ai, si in zip(a, s))
        assert dec < lc.gamma_of(q, n, binary)
        assert dec % q == lc.lwe_phase(s, a, b, q)
        assert lc.modified_lwe_decrypt(sk, x, q, p) == lc.lwe_decrypt(s, a, b, q, p) == mu


def test_shared_randomness_key_decrypts(keys):
    """The test-speed compression key (one r for every entry) decrypts to s."""
    pk, sk = keys
    g = np.random.default_rng(4)
    s = lc.lwe_keygen(6, Q64, False, g)
    ck = lc.compression_key(pk, s, g, shared_randomness=True)
    assert [paillier.decrypt(sk, c) for c in ck] == s
    assert len(set(ck)) == len(set(s))


def test_fast_equals_plain_compress(keys):
    """Algorithm "Batch compression ... using precomputed powers": the expanded key gives
    the same ciphertext, bit for bit; a = 0 (exponent 0) included."""
    pk, sk = keys
    g = np.random.default_rng(5)
    n, q = 10, Q64
    s = lc.lwe_keygen(n, q, False, g)
    ck = lc.compression_key(pk, s, g)
    eck = lc.expand_compression_key(pk, ck, 64)
    assert eck[5][3] == pow(ck[3], 32, pk.m2)
    _, cts = _cts(s, q, 16, 2, g)
    cts.append(([0] * n, 7))
    for a, b in cts:
        assert lc.fast_lwe_compress(pk, eck, a, b, q) == lc.lwe_compress(pk, ck, a, b, q)


@pytest.mark.parametrize("binary", [False, True])
def test_batched_compress_correct(keys, binary):
    """Theorem "Correctness" (Sec. 3.3): with gamma^ell < m every slot decrypts; ell is the
    largest such count."""
    pk, sk = keys
    g = np.random.default_rng(9 + binary)
    n, q, p = 16, 1 << 32, 16
    gamma = lc.gamma_of(q, n, binary)
    ell = lc.max_slots(pk.m, gamma)
    assert gamma ** ell < pk.m <= gamma ** (ell + 1)
    s = lc.lwe_keygen(n, q, binary, g)
    ck = lc.compression_key(pk, s, g)
    mus, cts = _cts(s, q, p, ell, g)
    x = lc.batched_lwe_compress(pk, ck, cts, q, gamma)
    assert lc.modified_batched_decrypt(sk, x, q, p, gamma, ell) == mus


def test_negacyclic_product_matches_numpy():
    g = np.random.default_rng(1)
    N, q = 16, Q27
    A = [int(v) for v in g.integers(0, q, size=N)]
    S = [int(v) for v in g.integers(0, q, size=N)]
    full = np.convolve(np.array(A, dtype=object), np.array(S, dtype=object))
    folded = [(full[k] - (full[k + N] if k + N < len(full) else 0)) % q for k in range(N)]
    assert lc.negacyclic_mul(A, S, q) == folded
    # X^(N-1) * X = X^N = -1
    e1 = [0] * N
    e1[1] = 1
    top = [0] * N
    top[N - 1] = 1
    assert lc.negacyclic_mul(top, e1, q) == [q - 1] + [0] * (N - 1)


@pytest.mark.parametrize("q,binary", [(Q27, False), (Q64, True)])
def test_rlwe_coefficient_compress_correct(keys, q, binary):
    """Theorem "Correctness" (App. B): the compressed coefficient k decrypts to coefficient
    k of the RLWE decryption (first, middle and last coefficient)."""
    pk, sk = keys
    g = np.random.default_rng(3)
    N, p = 16, 8
    S = lc.lwe_keygen(N, q, binary, g)
    ck = lc.compression_key(pk, S, g)
    mu = [int(v) for v in g.integers(0, p, size=N)]
    A, B = lc.rlwe_encrypt(S, mu, q, p, g)
    assert lc.rlwe_decrypt(S, A, B, q, p) == mu
    for k in (0, 5, N - 1):
        x = lc.rlwe_compress_coefficient(pk, ck, A, B, k, q)
        assert lc.modified_lwe_decrypt(sk, x, q, p) == mu[k]


@pytest.mark.parametrize("binary", [False, True])
def test_packed_key_correct(keys, binary):
    """Packed compression keys: unpacking and compressing, then the packed-key decryption,
    gives the message; t is the largest count with delta^(2t) <= m, and a ragged last
    packed ciphertext (n not a multiple of t) works."""
    pk, sk = keys
    g = np.random.default_rng(21 + binary)
    q, p = 1 << 16, 16
    n = 7
    delta = lc.gamma_of(q, n, binary)
    t = lc.packed_slots(pk.m, delta)
    assert t >= 2 and delta ** (2 * t) <= pk.m < delta ** (2 * t + 2)
    s = lc.lwe_keygen(n, q, binary, g)
    pck = lc.generate_packed_key(pk, s, delta, t, g)
    assert len(pck) == -(-n // t)
    ck = lc.unpack_compression_key(pk, pck, delta, t, n)
    mus, cts = _cts(s, q, p, 3, g)
    for mu, (a, b) in zip(mus, cts):
        x = lc.lwe_compress(pk, ck, a, b, q)
        assert lc.modified_lwe_decrypt_packed(sk, x, q, p, delta, t) == mu


def test_planted_sign_mistake_fails(keys):
    """Compressing with a[i] instead of (q - a[i]) mod q gives b + <a, s>, which does not
    decrypt (the pins above would catch the dropped negation)."""
    pk, sk = keys
    g = np.random.default_rng(30)
    n, q, p = 16, Q64, 16
    s = lc.lwe_keygen(n, q, False, g)
    ck = lc.compression_key(pk, s, g)
    mus, cts = _cts(s, q, p, 6, g)
    wrong = 0
    for mu, (a, b) in zip(mus, cts):
        x = lc.trivial(pk, b)
        for ai, c in zip(a, ck):
            x = paillier.add(pk, x, paillier.smul(pk, ai, c))
        wrong += lc.modified_lwe_decrypt(sk, x, q, p) != mu
    assert wrong >= 4


@pytest.mark.parametrize("q,r", [(Q64, 1 << 20), (Q27, 1 << 11), (1 << 32, 12289)])
def test_rescale_rounding(q, r):
    """Rounding to nearest with ties up, against the doubled-numerator form
    floor((2 x r + q) / (2 q)), and for q = 2^64, r = 2^20 against the shift form
    (x + 2^43) >> 44; edge values 0, q - 1 and the neighbours of every tie."""
    g = np.random.default_rng(r)
    xs = [0, 1, q - 1, q // 2, q // 2 - 1] + [int.from_bytes(g.bytes(8), "little") % q for _ in range(200)]
    ties = [(2 * k + 1) * q // (2 * r) for k in range(5)]
    xs += ties + [t + 1 for t in ties] + [t - 1 for t in ties if t > 0]
    a2, b2 = lc.rescale(xs, xs[7], q, r)
    assert a2 == [((2 * x * r + q) // (2 * q)) % r for x in xs]
    assert b2 == a2[7]
    if (q, r) == (Q64, 1 << 20):
        assert a2 == [((x + (1 << 43)) >> 44) % r for x in xs]


def test_rescale_then_compress_decrypts(keys):
    """Binary secret, small noise: (a, b) mod 2^64 rescaled to r = 2^20 still decrypts
    (the rounding adds at most (n + 1) / 2 to the phase), and so does its compression
    modulo r."""
    pk, sk = keys
    g = np.random.default_rng(12)
    n, q, r, p = 64, Q64, 1 << 20, 16
    s = lc.lwe_keygen(n, q, True, g)
    ck = lc.compression_key(pk, s, g)
    for mu in (0, 5, 15):
        a, b = lc.lwe_encrypt(s, mu, q, p, g)
        a2, b2 = lc.rescale(a, b, q, r)
        assert lc.lwe_decrypt(s, a2, b2, r, p) == mu
        assert lc.modified_lwe_decrypt(sk, lc.lwe_compress(pk, ck, a2, b2, r), r, p) == mu


def test_sizes_match_the_papers_table():
    """The printed sizes of the single-compression table (tests/golden/lwe_compress_sizes.txt):
    a compressed ciphertext is one Paillier ciphertext, 2 log2 m bits = 768 bytes at 3072
    bits (the library's 2L words); an uncompressed LWE ciphertext is (n + 1) log2 q bits and
    an RLWE one (A from a seed) N log2 q bits; the reduction is 1 - compressed/uncompressed.
    LWE rows agree to the printed precision; the RLWE sizes are printed 0.01 KB above
    N log2 q / 8 bytes in three rows, so they get that much slack."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "lwe_compress_sizes.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 8
    key_bits = 3072
    for kind, n, lq, comp, kb, red in rows:
        n, lq, comp, kb, red = int(n), int(lq), int(comp), float(kb), float(red)
        assert comp == 2 * key_bits // 8 == 4 * (2 * key_bits // 32)
        bits = (n + 1) * lq if kind == "lwe" else n * lq
        size = bits / 8
        slack = 0.006 if kind == "lwe" else 0.016
        assert abs(size / 1000 - kb) < slack, (kind, n, lq)
        assert abs(100 * (1 - comp / size) - red) < (0.011 if kind == "lwe" else 0.03), (kind, n, lq)
