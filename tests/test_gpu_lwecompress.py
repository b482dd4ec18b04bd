"""GPU parity of the standalone compression of LWE ciphertexts and RLWE coefficients
(Sec. 3, App. B, the packed-key appendix) against the oracle, through the C ABI, for 2048-
and 3072-bit keys. Paillier ciphertexts are compared bit for bit; decryptions check the
correctness theorems end to end."""
import numpy as np
import pytest

import synth
from oracle import lwecompress as lc
from oracle import paillier

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q64 = 1 << 64
Q27 = 134217689


@pytest.fixture(scope="module")
def zp():
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as m
    return m


@pytest.fixture(scope="module")
def keys():
    return {2048: paillier.keygen(2048, 5), 3072: paillier.keygen(3072, 6)}


def u64_dev(vals):
    return torch.from_numpy(np.array(vals, dtype=np.uint64).reshape(np.shape(vals)).view(np.int64)).cuda()


def ct_dev(vals, L):
    return torch.from_numpy(synth.ints_to_limbs(vals, 2 * L).view(np.int32)).cuda()


def ct_host(t):
    return synth.limbs_to_ints(t.cpu().numpy().view(np.uint32))


def _setup(zp, keys, bits, n, q, binary, seed, T):
    pk, sk = keys[bits]
    g = np.random.default_rng(seed)
    s = lc.lwe_keygen(n, q, binary, g)
    ck = lc.compression_key(pk, s, g, shared_randomness=bits == 3072 or n > 64)
    comp = zp.LweCompressor(0, bits, pk.m)
    comp.set_key(ct_dev(ck, bits // 32), T)
    return pk, sk, g, s, ck, comp


@pytest.mark.parametrize("bits", [2048, 3072])
@pytest.mark.parametrize("q,p", [(Q64, 16), (1 << 11, 4), (Q27, 8)])
def test_lwe_compress_parity(zp, keys, bits, q, p):
    n = 24
    pk, sk, g, s, ck, comp = _setup(zp, keys, bits, n, q, False, q % 1000 + bits, (q - 1).bit_length())
    mus = [int(g.integers(0, p)) for _ in range(5)]
    cts = [lc.lwe_encrypt(s, mu, q, p, g) for mu in mus]
    cts.append(([0] * n, 0))          # all exponents 0 and b = 0: x = 1
    cts.append(([1] * n, q - 1))      # exponents q - 1
    X = ct_host(comp.compress(u64_dev([a for a, _ in cts]), u64_dev([b for _, b in cts]), q))
    assert X == [lc.lwe_compress(pk, ck, a, b, q) for a, b in cts]
    assert X[5] == 1
    assert [lc.modified_lwe_decrypt(sk, x, q, p) for x in X[:5]] == mus


@pytest.mark.parametrize("mode", ["horner", "folded", "auto"])
def test_batched_compress_parity(zp, keys, mode):
    """Groups of ell (the largest count the theorem allows) and a ragged last group; the
    Horner and folded forms give the oracle's ciphertext and every slot decrypts."""
    n, q, p = 16, 1 << 32, 16
    pk, sk = keys[2048]
    gamma = lc.gamma_of(q, n, False)
    ell = lc.max_slots(pk.m, gamma)
    T = ((q - 1) * sum(gamma ** j for j in range(ell))).bit_length()
    pk, sk, g, s, ck, comp = _setup(zp, keys, 2048, n, q, False, 40, T)
    count = 2 * ell + 3
    mus = [int(g.integers(0, p)) for _ in range(count)]
    cts = [lc.lwe_encrypt(s, mu, q, p, g) for mu in mus]
    X = ct_host(comp.compress(u64_dev([a for a, _ in cts]), u64_dev([b for _, b in cts]), q, ell=ell,
                              gamma=gamma, mode=mode))
    assert len(X) == 3
    for gi in range(3):
        grp = cts[gi * ell:(gi + 1) * ell]
        assert X[gi] == lc.batched_lwe_compress(pk, ck, grp, q, gamma)
        assert lc.modified_batched_decrypt(sk, X[gi], q, p, gamma, len(grp)) == mus[gi * ell:(gi + 1) * ell]


def test_batched_3072_binary(zp, keys):
    """3072-bit key, binary secret (gamma = q + n q), q = 2^64, both forms."""
    n, q, p = 12, Q64, 4
    pk, sk = keys[3072]
    gamma = lc.gamma_of(q, n, True)
    ell = 9
    T = ((q - 1) * sum(gamma ** j for j in range(ell))).bit_length()
    pk, sk, g, s, ck, comp = _setup(zp, keys, 3072, n, q, True, 41, T)
    mus = [int(g.integers(0, p)) for _ in range(ell)]
    cts = [lc.lwe_encrypt(s, mu, q, p, g) for mu in mus]
    want = lc.batched_lwe_compress(pk, ck, cts, q, gamma)
    for mode in ("horner", "folded"):
        X = ct_host(comp.compress(u64_dev([a for a, _ in cts]), u64_dev([b for _, b in cts]), q, ell=ell,
                                  gamma=gamma, mode=mode))
        assert X == [want]
    assert lc.modified_batched_decrypt(sk, want, q, p, gamma, ell) == mus


@pytest.mark.parametrize("bits,q", [(2048, Q27), (3072, Q64)])
def test_rlwe_coefficient_parity(zp, keys, bits, q):
    """Extraction of coefficients 0, 7 and N - 1 and their compression equal the oracle's
    RLWECompressCoefficient; each decrypts to its coefficient."""
    N, p = 32, 8
    pk, sk, g, S, ck, comp = _setup(zp, keys, bits, N, q, False, 50, (q - 1).bit_length())
    mu = [int(v) for v in g.integers(0, p, size=N)]
    A, B = lc.rlwe_encrypt(S, mu, q, p, g)
    ks = [0, 7, N - 1]
    Ao, Bo = comp.rlwe_extract(u64_dev(A), u64_dev(B), q, ks)
    a_got = Ao.cpu().numpy().view(np.uint64)
    for c, k in enumerate(ks):
        want = [A[k - i] if i <= k else (q - A[N + k - i]) % q for i in range(N)]
        assert [int(v) for v in a_got[c]] == want
    assert [int(v) for v in Bo.cpu().numpy().view(np.uint64)] == [B[k] for k in ks]
    X = ct_host(comp.compress(Ao, Bo, q))
    for c, k in enumerate(ks):
        assert X[c] == lc.rlwe_compress_coefficient(pk, ck, A, B, k, q)
        assert lc.modified_lwe_decrypt(sk, X[c], q, p) == mu[k]


@pytest.mark.parametrize("binary", [False, True])
def test_unpack_key_parity(zp, keys, binary):
    """Packed keys (n not a multiple of t) unpack to the oracle's ck, and compression with
    them decrypts through the packed-key decryption."""
    pk, sk = keys[3072]
    q, p, n = Q64, 16, 23
    delta = lc.gamma_of(q, n, binary)
    t = lc.packed_slots(pk.m, delta)
    g = np.random.default_rng(60 + binary)
    s = lc.lwe_keygen(n, q, binary, g)
    pck = lc.generate_packed_key(pk, s, delta, t, g)
    comp = zp.LweCompressor(0, 3072, pk.m)
    ck = comp.unpack_key(ct_dev(pck, 96), n, t, delta)
    want = lc.unpack_compression_key(pk, pck, delta, t, n)
    assert ct_host(ck) == want
    assert len(pck) >= 2  # a ragged last packed ciphertext
    comp.set_key(ck, 64)
    mu = 11
    a, b = lc.lwe_encrypt(s, mu, q, p, g)
    X = ct_host(comp.compress(u64_dev([a]), u64_dev([b]), q))
    assert X == [lc.lwe_compress(pk, want, a, b, q)]
    assert lc.modified_lwe_decrypt_packed(sk, X[0], q, p, delta, t) == mu


def test_paper_parameter_set_630_q64(zp, keys):
    """The first parameter set of the single-compression evaluation: n = 630, q = 2^64,
    3072-bit key; one ciphertext against the oracle and decrypted."""
    n, q, p = 630, Q64, 16
    pk, sk, g, s, ck, comp = _setup(zp, keys, 3072, n, q, False, 70, 64)
    a, b = lc.lwe_encrypt(s, 9, q, p, g)
    X = ct_host(comp.compress(u64_dev([a]), u64_dev([b]), q))
    assert X == [lc.lwe_compress(pk, ck, a, b, q)]
    assert lc.modified_lwe_decrypt(sk, X[0], q, p) == 9


def test_invalid_arguments(zp, keys):
    pk, sk = keys[2048]
    comp = zp.LweCompressor(0, 2048, pk.m)
    A = u64_dev([[1] * 8])
    B = u64_dev([3])
    with pytest.raises(zp.ZipPIRError):
        comp.n = 8
        comp.compress(A, B, Q27)  # no key yet
    with pytest.raises(zp.ZipPIRError):
        zp.LweCompressor(0, 1024, pk.m)
    pk, sk, g, s, ck, comp = _setup(zp, keys, 2048, 8, Q27, False, 80, 20)
    with pytest.raises(zp.ZipPIRError):
        comp.compress(A, B, Q27)  # T = 20 < 27 bits of q - 1
    pk, sk, g, s, ck, comp = _setup(zp, keys, 2048, 8, Q27, False, 81, 27)
    with pytest.raises(zp.ZipPIRError):
        comp.compress(u64_dev([[1] * 8] * 200), u64_dev([3] * 200), Q27, ell=200,
                      gamma=lc.gamma_of(Q27, 8, False))  # gamma^ell far above m
    with pytest.raises(zp.ZipPIRError):
        comp.rlwe_extract(u64_dev([1] * 8), u64_dev([2] * 8), Q27, [8])


@pytest.mark.parametrize("q,r", [(Q64, 1 << 20), (Q27, 1 << 11), (1 << 32, 12289)])
def test_rescale_parity(zp, q, r):
    """Modulus switching on the GPU equals the oracle's rounding, edge values included."""
    g = np.random.default_rng(r)
    count, n = 6, 37
    A = [[int.from_bytes(g.bytes(8), "little") % q for _ in range(n)] for _ in range(count)]
    A[0][:5] = [0, 1, q - 1, q // 2, q // 2 - 1]
    A[1][:3] = [(2 * k + 1) * q // (2 * r) for k in range(3)]  # ties
    B = [int.from_bytes(g.bytes(8), "little") % q for _ in range(count)]
    Ao, Bo = zp.lc_rescale(u64_dev(A), u64_dev(B), q, r)
    got_a = [[int(v) for v in row] for row in Ao.cpu().numpy().view(np.uint64)]
    got_b = [int(v) for v in Bo.cpu().numpy().view(np.uint64)]
    for j in range(count):
        wa, wb = lc.rescale(A[j], B[j], q, r)
        assert got_a[j] == wa and got_b[j] == wb


def test_rescale_then_compress_on_gpu(zp, keys):
    """Binary secret, q = 2^64 rescaled to 2^20 on the GPU, then compressed modulo 2^20 on
    the GPU: the oracle's ciphertext, and the messages decrypt."""
    n, q, r, p = 32, Q64, 1 << 20, 16
    pk, sk, g, s, ck, comp = _setup(zp, keys, 2048, n, q, True, 90, 20)
    mus = [int(g.integers(0, p)) for _ in range(4)]
    cts = [lc.lwe_encrypt(s, mu, q, p, g) for mu in mus]
    Ao, Bo = zp.lc_rescale(u64_dev([a for a, _ in cts]), u64_dev([b for _, b in cts]), q, r)
    X = ct_host(comp.compress(Ao, Bo, r))
    for j, (a, b) in enumerate(cts):
        a2, b2 = lc.rescale(a, b, q, r)
        assert X[j] == lc.lwe_compress(pk, ck, a2, b2, r)
        assert lc.modified_lwe_decrypt(sk, X[j], r, p) == mus[j]
