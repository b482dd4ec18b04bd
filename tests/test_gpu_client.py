"""GPU parity of the client-side pieces: the ChaCha20 keystream that expands A and ck_r
from seeds, and the batched modular exponentiation mod m^2 that Paillier's decryption and
encryption rest on, against the oracle and Python's integers, through the C ABI.
Bit-exact."""
import numpy as np
import pytest

import synth
from oracle import chacha20, paillier, zippir
from oracle.params import Params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zp():
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as m
    return m


@pytest.mark.parametrize("nwords,counter0", [(1, 0), (15, 1), (16, 7), (17, 2**31),
                                             (1000, 12345), (4099, 2**32 - 257)])
def test_chacha20_keystream_parity(zp, nwords, counter0):
    """Ragged lengths (partial last block), counters up to the last block before the 32-bit
    counter wraps, and a misaligned destination for the ragged tail."""
    g = np.random.default_rng(nwords)
    key, nonce = g.bytes(32), g.bytes(12)
    want = np.array(chacha20.keystream_words(key, nonce, counter0, nwords), dtype=np.uint32)
    out = torch.full((nwords,), -1, dtype=torch.int32, device="cuda")
    zp.prg_chacha20(key, nonce, counter0, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)
    big = torch.full((nwords + 1,), -1, dtype=torch.int32, device="cuda")
    zp.prg_chacha20(key, nonce, counter0, big[1:])  # 4-byte offset: the unaligned store path
    got = big.cpu().numpy().view(np.uint32)
    assert got[0] == 0xFFFFFFFF and np.array_equal(got[1:], want)


def test_chacha20_counter_wrap_rejected(zp):
    out = torch.empty(33, dtype=torch.int32, device="cuda")
    with pytest.raises(zp.ZipPIRError):
        zp.prg_chacha20(bytes(32), bytes(12), 2**32 - 2, out)  # 3 blocks from 2^32 - 2


def test_chacha20_expands_seed_matrix_words(zp):
    """A large expansion (1 Mi words) against the oracle on sampled blocks: the first,
    the last and a spread of blocks in between."""
    key, nonce = bytes(range(32)), bytes(range(100, 112))
    nwords = 1 << 20
    out = torch.empty(nwords, dtype=torch.int32, device="cuda")
    zp.prg_chacha20(key, nonce, 1, out)
    got = out.cpu().numpy().view(np.uint32)
    for blk in [0, 1, 4095, 30000, nwords // 16 - 1]:
        assert list(got[16 * blk:16 * blk + 16]) == chacha20.block(key, 1 + blk, nonce)


def _client(zp, seed):
    P = Params(n=8, key_bits=2048, secret="uniform")
    cl = zippir.setup(P, seed, sample_ck_r=False)
    ctx = zp.Context(0, n=8, key_bits=2048)
    return cl, ctx, ctx.register_client(cl.pk.m)


def _dev(vals, L):
    return torch.from_numpy(synth.ints_to_limbs(vals, 2 * L).view(np.int32)).cuda()


@pytest.mark.parametrize("count", [1, 5, 64])
def test_powm_parity(zp, count):
    cl, ctx, gcl = _client(zp, 500 + count)
    m2 = cl.pk.m2
    g = np.random.default_rng(count)
    bases = [int.from_bytes(g.bytes(520), "little") % m2 for _ in range(count)]
    bases[0] = m2 - 1
    for e in [0, 1, 2, 3, 2**31 + 1, int.from_bytes(g.bytes(256), "little"), cl.pk.m]:
        got = synth.limbs_to_ints(gcl.powm(_dev(bases, ctx.L), e).cpu().numpy().view(np.uint32))
        assert got == [pow(b, e, m2) for b in bases], e


def test_powm_decrypts(zp):
    """u = c^lambda mod m^2 on the GPU; L(u) mu mod m recovers each plaintext, including
    0 and m - 1."""
    cl, ctx, gcl = _client(zp, 77)
    m = cl.pk.m
    g = np.random.default_rng(77)
    xs = [0, 1, m - 1] + [int.from_bytes(g.bytes(256), "little") % m for _ in range(13)]
    cs = [paillier.encrypt(cl.pk, x, int.from_bytes(g.bytes(256), "little") % (m - 2) + 2) for x in xs]
    u = synth.limbs_to_ints(gcl.powm(_dev(cs, ctx.L), cl.sk.lam).cpu().numpy().view(np.uint32))
    assert [(ui - 1) // m * cl.sk.mu % m for ui in u] == xs


def test_powm_invalid_arguments(zp):
    cl, ctx, gcl = _client(zp, 9)
    b = _dev([3], ctx.L)
    with pytest.raises(zp.ZipPIRError):
        gcl.powm(b, 1 << (32 * 128))  # 129 exponent words
    with pytest.raises(zp.ZipPIRError):
        gcl.powm(torch.empty(2 * 2 * ctx.L + 1, dtype=torch.int32, device="cuda")[1:].view(2, -1), 5)


@pytest.mark.parametrize("count,counter0", [(1, 0), (5, 3), (64, 1000)])
def test_expand_ckr_parity(zp, count, counter0):
    """ck_r from a seed: consecutive elements start at every word offset within a block
    (132 i mod 16 in {0, 4, 8, 12})."""
    cl, ctx, gcl = _client(zp, 600 + count)
    key = bytes(range(count, count + 32))
    got = synth.limbs_to_ints(gcl.expand_ckr(key, count, counter0=counter0).cpu().numpy().view(np.uint32))
    assert got == zippir.expand_ck_r(key, cl.pk, 2048, count, counter0=counter0)


def test_expand_ckr_small_modulus_needs_four_subtractions(zp):
    """m = 2^2047 + 1 (odd, 2048 bits, m^2 just above 2^4094): the reduction of a value
    below 2^4096 + m^2 takes up to four subtractions of m^2; powm under the same m."""
    from oracle import paillier as pl
    m = (1 << 2047) + 1
    ctx = zp.Context(0, n=8, key_bits=2048)
    gcl = ctx.register_client(m)
    key = bytes(32)
    got = synth.limbs_to_ints(gcl.expand_ckr(key, 40).cpu().numpy().view(np.uint32))
    assert got == zippir.expand_ck_r(key, pl.PublicKey(m), 2048, 40)
    b = got[:8]
    out = synth.limbs_to_ints(gcl.powm(_dev(b, ctx.L), 65537).cpu().numpy().view(np.uint32))
    assert out == [pow(x, 65537, m * m) for x in b]


def test_expand_ckr_rejects_counter_wrap(zp):
    cl, ctx, gcl = _client(zp, 3)
    with pytest.raises(zp.ZipPIRError):
        gcl.expand_ckr(bytes(32), 16, counter0=2**32 - 100)  # needs 132 blocks


def test_decrypt_parity(zp):
    """Dec on the GPU equals the oracle's for random plaintexts, 0, 1 and m - 1, and for
    the client's ck_r (pt_r = Dec(ck_r))."""
    P = Params(n=8, key_bits=2048, secret="uniform")
    cl = zippir.setup(P, 900, sample_ck_r=True)
    ctx = zp.Context(0, n=8, key_bits=2048)
    gcl = ctx.register_client(cl.pk.m)
    m = cl.pk.m
    g = np.random.default_rng(900)
    xs = [0, 1, m - 1] + [int.from_bytes(g.bytes(256), "little") % m for _ in range(9)]
    cs = [paillier.encrypt(cl.pk, x, int.from_bytes(g.bytes(256), "little") % (m - 2) + 2) for x in xs]
    got = synth.limbs_to_ints(gcl.decrypt(_dev(cs, ctx.L), cl.sk.lam, cl.sk.mu).cpu().numpy().view(np.uint32))
    assert got == xs
    pt = synth.limbs_to_ints(gcl.decrypt(_dev(cl.ck_r, ctx.L), cl.sk.lam, cl.sk.mu).cpu().numpy().view(np.uint32))
    assert pt == cl.pt_r


def test_seeded_client_end_to_end(zp):
    """The whole client side from seeds on the GPU: A from its seed feeds the hint, ck_r
    from its seed feeds k, Dec(k) on the GPU equals H' pt_r mod m (the homomorphic
    identity of the hint), with pt_r = Dec(ck_r) also from the GPU; all against the oracle."""
    from oracle import lwe
    R, C, n = 60, 48, 8
    P = Params(n=n, key_bits=2048, secret="uniform")
    D = synth.database(R, C, 5)
    keyA, keyC = bytes(range(32)), bytes(range(32, 64))
    A = zippir.expand_matrix(keyA, C, n)
    cl0 = zippir.setup(P, 55, sample_ck_r=False)
    ctx = zp.Context(0, n=n, key_bits=2048)
    gcl = ctx.register_client(cl0.pk.m)
    dA = torch.empty((C, n), dtype=torch.int32, device="cuda")
    zp.prg_chacha20(keyA, zippir.NONCE_A, 0, dA)
    assert np.array_equal(dA.cpu().numpy().view(np.uint32), A)
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    dD = torch.from_numpy(buf).cuda()
    db = zp.Database(ctx, dD, R, C, ld)
    db.gen_hint(dA)
    ckr = gcl.expand_ckr(keyC, n)
    ck_r = zippir.expand_ck_r(keyC, cl0.pk, 2048, n)
    pt_r = synth.limbs_to_ints(gcl.decrypt(ckr, cl0.sk.lam, cl0.sk.mu).cpu().numpy().view(np.uint32))
    assert pt_r == [paillier.decrypt(cl0.sk, c) for c in ck_r]
    k = db.client_hint(gcl, ckr)
    deck = synth.limbs_to_ints(gcl.decrypt(k, cl0.sk.lam, cl0.sk.mu).cpu().numpy().view(np.uint32))
    cl = zippir.Client(P, cl0.pk, cl0.sk, ck_r, pt_r)
    Hn = lwe.hint_neg(D, A)
    assert deck == zippir.dec_k_shortcut(cl, Hn, range(db.d1p))


def test_decrypt_invalid_arguments(zp):
    cl, ctx, gcl = _client(zp, 10)
    c = _dev([5, 6], ctx.L)
    with pytest.raises(zp.ZipPIRError):
        gcl.decrypt(torch.empty(2 * 2 * ctx.L + 1, dtype=torch.int32, device="cuda")[1:].view(2, -1),
                    cl.sk.lam, cl.sk.mu)
    out = gcl.decrypt(c[:0], cl.sk.lam, cl.sk.mu)  # count 0: nothing to do
    assert out.shape[0] == 0
