"""Pins for the oracle (CPU only): each test checks the oracle against something other
than itself -- brute force on tiny inputs, closed forms, an independent library
primality test, the Paillier laws, the correctness theorem of ZipPIR (record
recovery) and the identity in its proof (App. D)."""
import numpy as np
import pytest

import synth
from oracle import lwe, paillier, zippir
from oracle.params import Params, Q


# ----------------------------------------------------------------------------- LWE products
def brute_matvec(D, q):
    R, C = D.shape
    return [sum(int(D[r, c]) * int(q[c]) for c in range(C)) % Q for r in range(R)]


@pytest.mark.parametrize("R,C,seed", [(8, 8, 1), (8, 8, 2), (1, 1, 3), (7, 31, 4), (31, 7, 5), (8, 33, 6)])
def test_matvec_brute_force(R, C, seed):
    D = synth.database(R, C, seed)
    q = synth.uniform_queries(1, C, seed)[0]
    assert lwe.matvec_mod_q(D, q).tolist() == brute_matvec(D, q)


def test_matvec_closed_forms():
    D = synth.database(16, 40, 9)
    for i in (0, 17, 39):
        e = np.zeros(40, dtype=np.uint32)
        e[i] = 1
        assert np.array_equal(lwe.matvec_mod_q(D, e), D[:, i].astype(np.uint32))
    # all-maximal entries: every row is 255 * (2^32 - 1) * C = -255 C mod 2^32
    for C in (1, 1025, 131072):
        Dm = np.full((3, C), 255, dtype=np.uint8)
        qm = np.full(C, 0xFFFFFFFF, dtype=np.uint32)
        assert lwe.matvec_mod_q(Dm, qm).tolist() == [(-255 * C) % Q] * 3


def test_matvec_linear():
    D = synth.database(20, 300, 3)
    Qs = synth.uniform_queries(2, 300, 3)
    s = ((Qs[0].astype(np.uint64) + Qs[1]) & 0xFFFFFFFF).astype(np.uint32)
    lhs = lwe.matvec_mod_q(D, s).astype(np.uint64)
    rhs = (lwe.matvec_mod_q(D, Qs[0]).astype(np.uint64) + lwe.matvec_mod_q(D, Qs[1])) & 0xFFFFFFFF
    assert np.array_equal(lhs, rhs)


def test_hint_brute_force_and_sign():
    D = synth.database(6, 9, 4)
    A = synth.seed_matrix(9, 5, 4)
    Hp = lwe.hint_plus(D, A)
    for r in range(6):
        for i in range(5):
            assert int(Hp[r, i]) == sum(int(D[r, c]) * int(A[c, i]) for c in range(9)) % Q
    Hn = lwe.hint_neg(D, A)
    assert np.all(((Hp.astype(np.uint64) + Hn) & 0xFFFFFFFF) == 0)
    # matmat on columns equals matvec on each column
    for i in range(5):
        assert np.array_equal(lwe.matmat_mod_q(D, A)[:, i], lwe.matvec_mod_q(D, A[:, i]))


# ----------------------------------------------------------------------------- parameters
@pytest.mark.parametrize("secret,bits", [("uniform", 2048), ("binary", 2048), ("uniform", 3072)])
def test_slots_worst_case(secret, bits):
    """ell slots of the largest possible slot value fit below 2^(bits-1); ell+1 do not."""
    P = Params(n=1024, key_bits=bits, secret=secret)
    smax = 1 if secret == "binary" else Q - 1
    slot_max = (Q - 1) + P.n * (Q - 1) * smax          # b + H sk, Sec. 3.1 bound
    assert slot_max < P.gamma
    top = sum(slot_max * P.gamma ** j for j in range(P.ell))
    assert top < 2 ** (bits - 1)
    assert P.gamma ** (P.ell + 1) >= 2 ** (bits - 1)
    # round-trip of the worst case through the slot decoder
    assert zippir.unpack(top, P) == [slot_max] * P.ell


@pytest.mark.parametrize("secret,scale,ell", [("uniform", "proven", 27), ("binary", "proven", 48),
                                               ("uniform", "overlap", 31), ("binary", "overlap", 63)])
def test_slot_counts(secret, scale, ell):
    """Slots per packed row at n = 1024, 2048 bits: ell slots of the largest slot value
    (b + H sk < q + n q^2, or q + n q) fit below 2^2047 at the scale's gamma; one more slot
    of the bound does not (the overlap scale's slots overlap: gamma < bound)."""
    P = Params(n=1024, key_bits=2048, secret=secret, scale=scale)
    assert P.ell == ell
    smax = 1 if secret == "binary" else Q - 1
    slot_max = (Q - 1) + P.n * (Q - 1) * smax
    bound = Q + P.n * Q * (Q if secret == "uniform" else 1)
    assert slot_max < bound
    assert P.gamma == (bound if scale == "proven" else (Q * Q if secret == "uniform" else Q))
    assert sum(slot_max * P.gamma ** j for j in range(ell)) < 2 ** 2047
    assert sum((bound - 1) * P.gamma ** j for j in range(ell + 1)) >= 2 ** 2047


@pytest.mark.parametrize("seed,secret", [(4, "uniform"), (5, "binary")])
def test_e2e_overlap_scale(seed, secret):
    """Overlap scale (Sec. 3.3.3): with the real hint k, Extract still returns column i0;
    the slots overlap (gamma below the slot bound), so this is checked by recovery (the
    paper defers its proof)."""
    R, C, n = 130, 48, 8
    P = Params(n=n, key_bits=2048, secret=secret, scale="overlap")
    assert P.gamma < P.slot_bound
    D = synth.database(R, C, seed)
    A = synth.seed_matrix(C, n, seed)
    Hn = lwe.hint_neg(D, A)
    cl = zippir.setup(P, seed + 100, sample_ck_r=True)
    i0 = (11 * seed) % C
    qy = zippir.query(cl, A, i0, seed + 200)
    ans, t = zippir.response(D, qy.qu, Hn, qy.cko, cl.pk.m, P)
    rows = range(P.d1p(R))
    k = zippir.paillier_matmul_rows(cl, Hn, rows)
    dec_k = [paillier.decrypt(cl.sk, kk) for kk in k]
    assert dec_k == zippir.dec_k_shortcut(cl, Hn, rows)
    rec = zippir.extract(cl, dec_k, t, R)
    assert np.array_equal(rec, D[:, i0])


def test_e2e_overlap_tiny_config():
    """1024 x 1024, n = 1024, uniform secret at the overlap scale (31 slots)."""
    R = C = n = 1024
    P = Params(n=n, key_bits=2048, secret="uniform", scale="overlap")
    D = synth.database(R, C, 9)
    A = synth.seed_matrix(C, n, 9)
    Hn = lwe.hint_neg(D, A)
    cl = zippir.setup(P, 109, sample_ck_r=False)
    qy = zippir.query(cl, A, 77, 309)
    ans, t = zippir.response(D, qy.qu, Hn, qy.cko, cl.pk.m, P)
    assert len(t) == -(-R // 31)
    rows = list(range(len(t)))
    rec = zippir.extract(cl, zippir.dec_k_shortcut(cl, Hn, rows), t, R)
    assert np.array_equal(rec, D[:, 77])


def test_pack_unpack_roundtrip():
    P = Params(n=1024, key_bits=2048)
    g = synth.rng(5)
    for _ in range(5):
        vals = [int(x) for x in g.integers(0, 2**62, size=P.ell, dtype=np.uint64)]
        assert zippir.unpack(zippir.pack(vals, P)[0], P) == vals
    assert P.d1p(1024) == 38 and P.d1p(32768) == 1214 and P.d1p(27) == 1 and P.d1p(28) == 2


# ----------------------------------------------------------------------------- Paillier
@pytest.fixture(scope="module")
def key2048():
    return paillier.keygen(2048, 11)


def test_keygen_primes(key2048):
    sympy = pytest.importorskip("sympy")
    pk, sk = key2048
    assert pk.m.bit_length() == 2048
    assert sk.p1 * sk.p2 == pk.m
    assert sympy.isprime(sk.p1) and sympy.isprime(sk.p2)


def test_paillier_laws(key2048):
    pk, sk = key2048
    m, m2 = pk.m, pk.m2
    g = synth.rng(12)
    xs = [0, 1, m - 1] + synth.uniform_below(m, 2, 12)
    for x in xs:
        r = synth.uniform_below(m, 1, int(x % 1000) + 13)[0] | 1
        assert paillier.decrypt(sk, paillier.encrypt(pk, x, r)) == x
    # Enc(x; 1) = (1 + m)^x = 1 + x m mod m^2 (binomial theorem)
    x = xs[3]
    assert paillier.encrypt(pk, x, 1) == (1 + x * m) % m2 == pow(1 + m, x, m2)
    # homomorphisms, also on arbitrary elements of Z_{m^2}^* (Sec. 4.1)
    c1, c2 = synth.uniform_below(m2, 2, 14)
    a = int(g.integers(0, 2**62))
    d1, d2 = paillier.decrypt(sk, c1), paillier.decrypt(sk, c2)
    assert paillier.decrypt(sk, paillier.add(pk, c1, c2)) == (d1 + d2) % m
    assert paillier.decrypt(sk, paillier.smul(pk, a, c1)) == a * d1 % m


# ----------------------------------------------------------------------------- ZipPIR end to end
def _instance(R, C, n, secret, seed, sample_ck_r):
    P = Params(n=n, key_bits=2048, secret=secret)
    D = synth.database(R, C, seed)
    A = synth.seed_matrix(C, n, seed)
    Hn = lwe.hint_neg(D, A)
    cl = zippir.setup(P, seed + 100, sample_ck_r=sample_ck_r)
    return P, D, A, Hn, cl


@pytest.mark.parametrize("seed,secret", [(1, "uniform"), (2, "uniform"), (3, "binary")])
def test_e2e_real_hint(seed, secret):
    """Correctness theorem (Thm. 2): with the real per-client hint k = PaillierMatMul(H', ck_r),
    Extract returns column i0 of the database."""
    R, C, n = 60, 48, 8
    P, D, A, Hn, cl = _instance(R, C, n, secret, seed, True)
    i0 = (7 * seed) % C
    qy = zippir.query(cl, A, i0, seed + 200)
    ans, t = zippir.response(D, qy.qu, Hn, qy.cko, cl.pk.m, P)
    rows = range(P.d1p(R))
    k = zippir.paillier_matmul_rows(cl, Hn, rows)
    dec_k = [paillier.decrypt(cl.sk, kk) for kk in k]
    assert dec_k == zippir.dec_k_shortcut(cl, Hn, rows)
    rec = zippir.extract(cl, dec_k, t, R)
    assert np.array_equal(rec, D[:, i0])


@pytest.mark.parametrize("seed,secret", [(1, "uniform"), (3, "binary")])
def test_e2e_combined_response(seed, secret):
    """k (+) t (Sec. 4.3): one decryption per packed row gives mu = Dec(k) + t mod m directly,
    and Extract on those mu returns column i0; the ciphertext equals k (1 + t m) mod m^2."""
    R, C, n = 60, 48, 8
    P, D, A, Hn, cl = _instance(R, C, n, secret, seed, True)
    i0 = (5 * seed + 3) % C
    qy = zippir.query(cl, A, i0, seed + 300)
    ans, t = zippir.response(D, qy.qu, Hn, qy.cko, cl.pk.m, P)
    rows = range(P.d1p(R))
    k = zippir.paillier_matmul_rows(cl, Hn, rows)
    kt = zippir.combine(cl.pk, k, t)
    m, m2 = cl.pk.m, cl.pk.m2
    assert kt == [kk * (1 + tt * m) % m2 for kk, tt in zip(k, t)]
    mus = [paillier.decrypt(cl.sk, c) for c in kt]
    assert mus == [(paillier.decrypt(cl.sk, kk) + tt) % m for kk, tt in zip(k, t)]
    rec = zippir.extract(cl, [0] * len(mus), mus, R)
    assert np.array_equal(rec, D[:, i0])


def _proof_identity(P, cl, Hn, qy, ans, t, rows):
    """(t + H' pt_r) mod m == b' + H' sk exactly, and b' + H' sk < m (App. D)."""
    m = cl.pk.m
    for rp in rows:
        hrow = zippir.packed_hint_row(Hn, rp, P)
        bp = zippir.pack(ans[rp * P.ell:(rp + 1) * P.ell], P)[0]
        rhs = bp + sum(h * int(s) for h, s in zip(hrow, qy.lwe_sk))
        lhs = (t[rp] + sum(h * p for h, p in zip(hrow, cl.pt_r))) % m
        assert rhs < m
        assert lhs == rhs


@pytest.mark.parametrize("seed", [4, 5])
def test_e2e_tiny_config(seed):
    """Tiny end-to-end PIR at the 1024 x 1024, n = 1024, 2048-bit size: recovery and
    the proof identity on every packed row."""
    R = C = n = 1024
    P, D, A, Hn, cl = _instance(R, C, n, "uniform", seed, False)
    i0 = 389 * seed % C
    qy = zippir.query(cl, A, i0, seed + 300)
    ans, t = zippir.response(D, qy.qu, Hn, qy.cko, cl.pk.m, P)
    assert len(t) == 38
    rows = list(range(38))
    rec = zippir.extract(cl, zippir.dec_k_shortcut(cl, Hn, rows), t, R)
    assert np.array_equal(rec, D[:, i0])
    _proof_identity(P, cl, Hn, qy, ans, t, rows[:3] + rows[-2:])


def test_planted_mistakes_break_recovery():
    """A wrong hint sign or a wrong slot order each make recovery fail,
    so the e2e pins above would catch those mistakes in the oracle."""
    R, C, n = 90, 64, 16
    P, D, A, Hn, cl = _instance(R, C, n, "uniform", 21, False)
    qy = zippir.query(cl, A, 5, 22)
    m = cl.pk.m
    rows = range(P.d1p(R))
    ans = lwe.matvec_mod_q(D, qy.qu)
    good = zippir.compress_rows(ans, Hn, qy.cko, m, P)
    assert np.array_equal(zippir.extract(cl, zippir.dec_k_shortcut(cl, Hn, rows), good, R), D[:, 5])
    # wrong sign: use H+ in place of -H+
    Hp = lwe.hint_plus(D, A)
    bad = zippir.compress_rows(ans, Hp, qy.cko, m, P)
    assert not np.array_equal(zippir.extract(cl, zippir.dec_k_shortcut(cl, Hp, rows), bad, R), D[:, 5])
    # wrong slot order: reverse the answers inside each packed row on the server only
    ell = P.ell
    rev = ans.copy()
    for r0 in range(0, R, ell):
        rev[r0:r0 + ell] = ans[r0:r0 + ell][::-1]
    bad = zippir.compress_rows(rev, Hn, qy.cko, m, P)
    assert not np.array_equal(zippir.extract(cl, zippir.dec_k_shortcut(cl, Hn, rows), bad, R), D[:, 5])


def test_sizes():
    """Response sizes (Sec. 4.4): t is d1' log m bits, the per-client hint 2 d1' log m bits."""
    P = Params(n=1024, key_bits=2048)
    d1p = P.d1p(32768)
    assert d1p * 2048 // 8 == 1214 * 256
    assert 2 * d1p * 2048 // 8 == 621568


def test_chacha20_keystream_matches_library():
    """The oracle's ChaCha20 (RFC 8439 block function) against the `cryptography` package's
    ChaCha20 keystream, for several keys, nonces and block counters and a ragged length."""
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    from oracle import chacha20
    g = np.random.default_rng(8439)
    for trial in range(4):
        key = g.bytes(32)
        nonce = g.bytes(12)
        ctr = int(g.integers(0, 2**31))
        nwords = 16 * trial + 7
        enc = ciphers.Cipher(ciphers.algorithms.ChaCha20(key, ctr.to_bytes(4, "little") + nonce),
                             mode=None).encryptor()
        ks = enc.update(b"\0" * (4 * nwords))
        want = [int.from_bytes(ks[4 * i:4 * i + 4], "little") for i in range(nwords)]
        assert chacha20.keystream_words(key, nonce, ctr, nwords) == want


def test_seed_expansions_match_library():
    """A and ck_r expanded from seeds: the oracle's words against the `cryptography`
    package's ChaCha20 byte stream, read independently (little-endian words; 528-byte
    integers reduced mod m^2)."""
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    from oracle import paillier, zippir
    key = bytes(range(7, 39))

    def stream(nonce, nbytes, ctr=0):
        enc = ciphers.Cipher(ciphers.algorithms.ChaCha20(key, ctr.to_bytes(4, "little") + nonce),
                             mode=None).encryptor()
        return enc.update(b"\0" * nbytes)

    A = zippir.expand_matrix(key, 5, 7)
    ks = stream(zippir.NONCE_A, 4 * 35)
    assert A.dtype == np.uint32 and A.shape == (5, 7)
    assert A[3, 4] == int.from_bytes(ks[4 * 25:4 * 26], "little")
    assert A.tobytes() == ks  # row-major little-endian words
    pk, _ = paillier.keygen(512, 3)
    ck = zippir.expand_ck_r(key, pk, 512, 6, counter0=5)
    ks = stream(zippir.NONCE_CKR, 6 * 144, ctr=5)
    assert ck == [int.from_bytes(ks[144 * i:144 * (i + 1)], "little") % pk.m2 for i in range(6)]
    assert all(0 <= c < pk.m2 for c in ck)
