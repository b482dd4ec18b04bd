"""GPU parity of the RNS compression of large batches (Sec. 5.2: H'.ck_o modulo word-size
primes, one reduction at the end) against the oracle, through the C ABI. Exact integers:
bit-exact comparisons."""
import numpy as np
import pytest

import synth
from oracle import lwe, paillier, zippir
from oracle.params import Params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zp():
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as m
    return m


def u32_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def u32_host(t):
    return t.cpu().numpy().view(np.uint32)


def _db(zp, c, D):
    R, C = D.shape
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    dD = torch.from_numpy(buf).cuda()
    return zp.Database(c, dD, R, C, ld), dD


@pytest.mark.parametrize("R,C,n,B,secret", [(60, 32, 8, 1, "uniform"), (100, 48, 64, 3, "uniform"),
                                            (333, 64, 64, 17, "uniform"), (95, 40, 16, 5, "binary"),
                                            (200, 64, 1000, 2, "uniform"), (700, 64, 1024, 40, "uniform")])
@pytest.mark.parametrize("fp16", [False, True])
def test_rns_compress_parity(zp, R, C, n, B, secret, fp16):
    """Forced RNS path: t equals the oracle's (b' + H'.cko) mod m for every query and packed
    row, each query with its own client modulus, ragged last packed row; with the fp16 copy
    of the residue planes (A operand through TMA) as well."""
    P = Params(n=n, key_bits=2048, secret=secret)
    c = zp.Context(0, n=n, secret=secret)
    c.set_option("compress_path", "rns")
    D = synth.database(R, C, R + n)
    A = synth.seed_matrix(C, n, n + 1)
    Hn = lwe.hint_neg(D, A)
    db, dD = _db(zp, c, D)
    db.gen_hint(u32_dev(A))
    if fp16:
        db.prepare_fp16()  # the RNS planes are built by the first batch, their fp16 copy with them
    ms = [synth.random_odd_modulus(2048, 50 + b) for b in range(B)]
    cls = [c.register_client(m) for m in ms]
    ckos = [synth.uniform_below(ms[b], n, 60 + b) for b in range(B)]
    ans = synth.uniform_queries(B, R, 70)
    T = db.compress(cls, u32_dev(ans), u32_dev(np.stack([synth.ints_to_limbs(x, 64) for x in ckos])))
    got = u32_host(T)
    for b in range(B):
        assert synth.limbs_to_ints(got[b]) == zippir.compress_rows(ans[b], Hn, ckos[b], ms[b], P)
    assert c.device_status() == 0


@pytest.mark.parametrize("R,B", [(1080, 8), (2100, 17), (3600, 6)])
@pytest.mark.parametrize("fp16", [False, True])
def test_rns_several_m_tiles_per_prime(zp, R, B, fp16):
    """n = 1024 and d1' = 40 / 78 / 134 packed rows, i.e. two / three / five 32-packed-row M
    tiles per prime (the tile index g > 0 of the grouped product) and, at d1' = 134, two
    128-row M tiles of the CRT product (the second ragged); the last packed row ragged at R =
    2100 and 3600: every packed row of every query equals the oracle's t, on the byte planes
    and on their fp16 copy."""
    n, C = 1024, 64
    P = Params(n=n, key_bits=2048)
    assert P.d1p(R) > 32
    c = zp.Context(0, n=n)
    c.set_option("compress_path", "rns")
    D = synth.database(R, C, R + 7)
    A = synth.seed_matrix(C, n, R + 8)
    Hn = lwe.hint_neg(D, A)
    db, dD = _db(zp, c, D)
    db.gen_hint(u32_dev(A))
    if fp16:
        db.prepare_fp16()
    ms = [synth.random_odd_modulus(2048, 150 + b) for b in range(B)]
    cls = [c.register_client(m) for m in ms]
    ckos = [synth.uniform_below(ms[b], n, 160 + b) for b in range(B)]
    ans = synth.uniform_queries(B, R, 170)
    T = db.compress(cls, u32_dev(ans), u32_dev(np.stack([synth.ints_to_limbs(x, 64) for x in ckos])))
    got = u32_host(T)
    assert got.shape[1] == P.d1p(R)
    for b in range(B):
        assert synth.limbs_to_ints(got[b]) == zippir.compress_rows(ans[b], Hn, ckos[b], ms[b], P)
    assert c.device_status() == 0


@pytest.mark.parametrize("fp16", [False, True])
def test_rns_edge_values(zp, fp16):
    """cko at 0 and m - 1 and answers at 2^32 - 1 (the largest residue products and CRT sums)."""
    R, C, n = 60, 32, 64
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    c.set_option("compress_path", "rns")
    D = synth.database(R, C, 8)
    A = synth.seed_matrix(C, n, 8)
    Hn = lwe.hint_neg(D, A)
    db, dD = _db(zp, c, D)
    db.gen_hint(u32_dev(A))
    if fp16:
        db.prepare_rns()
        db.prepare_fp16()  # planes first, then the fp16 copies of D and of the planes
    pk, _ = paillier.keygen(2048, 77)
    m = pk.m
    cl = c.register_client(m)
    ans = np.full(R, 0xFFFFFFFF, dtype=np.uint32)
    for cko in ([m - 1] * n, [0] * n, [m - 1 if i % 2 else 0 for i in range(n)]):
        T = db.compress([cl], u32_dev(ans[None, :]), u32_dev(synth.ints_to_limbs(cko, 64)[None]))
        assert synth.limbs_to_ints(u32_host(T)[0]) == zippir.compress_rows(ans, Hn, cko, m, P)


def test_rns_auto_threshold_equals_tc_and_updates(zp):
    """Automatic choice: 20 queries (>= rns_min_batch, default 8) take the RNS path and agree with
    the tensor-core byte-plane path bit for bit; after row updates and hint regeneration
    the RNS planes of the touched packed rows follow and t matches the oracle."""
    R, C, n, B = 150, 64, 32, 20
    P = Params(n=n, key_bits=2048)
    D = synth.database(R, C, 5)
    A = synth.seed_matrix(C, n, 6)
    ms = [synth.random_odd_modulus(2048, 80 + b % 3) for b in range(B)]
    ckos = [synth.uniform_below(ms[b], n, 90 + b) for b in range(B)]
    ckod = u32_dev(np.stack([synth.ints_to_limbs(x, 64) for x in ckos]))
    ans = synth.uniform_queries(B, R, 91)
    outs = []
    for path in ("auto", "tc"):
        c = zp.Context(0, n=n)
        c.set_option("compress_path", path)
        assert zp.zp_get_overlap(c) >= 0
        db, dD = _db(zp, c, D)
        db.gen_hint(u32_dev(A))
        if path == "auto":
            db.prepare_fp16()  # regeneration below must keep the fp16 residue planes current
        cls = [c.register_client(m) for m in ms]
        outs.append(u32_host(db.compress(cls, u32_dev(ans), ckod)))
        if path == "auto":
            rows = np.array([0, 1, 77, 149], dtype=np.uint32)
            new = synth.database(len(rows), C, 123)
            db.update_rows(rows, torch.from_numpy(new).cuda())
            db.gen_hint(u32_dev(A), rows=rows)
            D2 = D.copy()
            D2[rows] = new
            Hn2 = lwe.hint_neg(D2, A)
            T2 = u32_host(db.compress(cls, u32_dev(ans), ckod))
            for b in (0, 7, 19):
                assert synth.limbs_to_ints(T2[b]) == zippir.compress_rows(ans[b], Hn2, ckos[b], ms[b], P)
    assert np.array_equal(outs[0], outs[1])


def test_prepare_rns(zp):
    """zp_db_prepare_rns builds the residue planes up front (the serving loop's setup); it
    needs the hint first, and the batch that follows gives the oracle's t."""
    R, C, n, B = 70, 32, 16, 9
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    D = synth.database(R, C, 44)
    A = synth.seed_matrix(C, n, 45)
    Hn = lwe.hint_neg(D, A)
    db, dD = _db(zp, c, D)
    with pytest.raises(zp.ZipPIRError):
        db.prepare_rns()
    db.gen_hint(u32_dev(A))
    db.prepare_rns()
    m = synth.random_odd_modulus(2048, 46)
    cl = c.register_client(m)
    ckos = [synth.uniform_below(m, n, 47 + b) for b in range(B)]
    ans = synth.uniform_queries(B, R, 48)
    T = u32_host(db.compress([cl] * B, u32_dev(ans), u32_dev(np.stack([synth.ints_to_limbs(x, 64) for x in ckos]))))
    for b in (0, B - 1):
        assert synth.limbs_to_ints(T[b]) == zippir.compress_rows(ans[b], Hn, ckos[b], m, P)


def test_batched_respond_overlap_on_and_off(zp):
    """zp_respond of a batch on the tensor cores with its compression products beside the
    answers on the internal stream ("batch_overlap" 1) and one after the other (0): the same
    bits, and t and the answers equal the oracle's (d1' = 78, n = 1024, ragged n % 128 = 0)."""
    R, C, n, B = 2100, 256, 1024, 12
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    D = synth.database(R, C, 321)
    A = synth.seed_matrix(C, n, 322)
    Hn = lwe.hint_neg(D, A)
    db, dD = _db(zp, c, D)
    db.gen_hint(u32_dev(A))
    ms = [synth.random_odd_modulus(2048, 330 + b) for b in range(B)]
    cls = [c.register_client(m) for m in ms]
    ckos = [synth.uniform_below(ms[b], n, 340 + b) for b in range(B)]
    Q = synth.uniform_queries(B, C, 350)
    CKO = u32_dev(np.stack([synth.ints_to_limbs(x, 64) for x in ckos]))
    outs = []
    for ov in (1, 0):
        c.set_option("batch_overlap", ov)
        ans, T = db.respond(cls, u32_dev(Q), CKO)
        outs.append((u32_host(ans), u32_host(T)))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    ans_h, T_h = outs[0]
    assert np.array_equal(ans_h, lwe.matmat_mod_q(D, Q.T).T)
    for b in (0, 5, B - 1):
        assert synth.limbs_to_ints(T_h[b]) == zippir.compress_rows(ans_h[b], Hn, ckos[b], ms[b], P)
    assert c.device_status() == 0
