"""GPU parity of the online Response against the oracle, through the C ABI.

Everything is exact integer work, so every comparison is bit-exact."""
import numpy as np
import pytest

import synth
from oracle import lwe, zippir
from oracle.params import Params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zp():
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(zp):
    return zp.Context(0, n=1024, key_bits=2048, secret="uniform")


def to_dev_db(zp, D):
    R, C = D.shape
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    return torch.from_numpy(buf).cuda(), ld


def u32_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def u32_host(t):
    return t.cpu().numpy().view(np.uint32)


SHAPES = [(1, 1), (7, 7), (8, 8), (31, 1025), (1024, 1024), (1025, 31), (64, 257), (130, 4096),
          (333, 9999), (2049, 700)]


@pytest.mark.parametrize("R,C", SHAPES)
def test_gemv_parity(zp, ctx, R, C):
    D = synth.database(R, C, R * 7 + C)
    q = synth.uniform_queries(1, C, R + C)[0]
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(ctx, dD, R, C, ld)
    got = u32_host(db.answer(u32_dev(q[None, :])))[0]
    assert np.array_equal(got, lwe.matvec_mod_q(D, q))
    db.close()


def test_gemv_closed_forms(zp, ctx):
    R, C = 300, 70000
    D = np.full((R, C), 255, dtype=np.uint8)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(ctx, dD, R, C, ld)
    q = np.full(C, 0xFFFFFFFF, dtype=np.uint32)
    got = u32_host(db.answer(u32_dev(q[None, :])))[0]
    assert np.all(got == np.uint32((-255 * C) % 2**32))
    # unit query: column i
    D2 = synth.database(R, C, 5)
    dD2, _ = to_dev_db(zp, D2)
    db2 = zp.Database(ctx, dD2, R, C, ld)
    for i in (0, 12345, C - 1):
        e = np.zeros(C, dtype=np.uint32)
        e[i] = 1
        got = u32_host(db2.answer(u32_dev(e[None, :])))[0]
        assert np.array_equal(got, D2[:, i].astype(np.uint32))
    db.close()
    db2.close()


@pytest.mark.parametrize("R,C,B", [(1, 1, 2), (7, 300, 3), (64, 256, 4), (65, 257, 2),
                                   (333, 9999, 3), (2049, 700, 4), (130, 4096, 4), (1, 1, 5),
                                   (31, 300, 6), (33, 257, 7), (333, 9999, 8), (2049, 700, 5),
                                   (4096, 4096, 8)])
def test_multi_query_gemv_parity(zp, ctx, R, C, B):
    """Two to four queries share one pass of the dp4a GEMV over D (ragged row blocks and
    column tiles, stream-K splits across CTAs); five to eight, at the boundary, take the
    tensor cores."""
    D = synth.database(R, C, 11 * B + R)
    Q = synth.uniform_queries(B, C, 13 * B + C)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(ctx, dD, R, C, ld)
    got = u32_host(db.answer(u32_dev(Q)))
    assert np.array_equal(got, lwe.matmat_mod_q(D, Q.T).T)
    db.close()


def test_multi_query_gemv_closed_form_and_tc(zp):
    """All-255 database against all-ones queries gives -255 C mod 2^32 in every entry (4
    queries on the GEMV, 8 on the tensor cores); the tensor-core path forced for the same
    batch agrees on random data."""
    R, C = 300, 70000
    D = np.full((R, C), 255, dtype=np.uint8)
    Q = np.full((4, C), 0xFFFFFFFF, dtype=np.uint32)
    Q[1] = 1
    Q8 = np.full((8, C), 0xFFFFFFFF, dtype=np.uint32)
    Q8[5] = 1
    c = zp.Context(0, n=64)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    got = u32_host(db.answer(u32_dev(Q)))
    assert np.all(got[[0, 2, 3]] == np.uint32((-255 * C) % 2**32))
    assert np.all(got[1] == np.uint32(255 * C))
    got8 = u32_host(db.answer(u32_dev(Q8)))
    assert np.all(got8[[0, 1, 2, 3, 4, 6, 7]] == np.uint32((-255 * C) % 2**32))
    assert np.all(got8[5] == np.uint32(255 * C))
    db.close()
    D2 = synth.database(R, 3000, 17)
    Q2 = synth.uniform_queries(3, 3000, 18)
    dD2, ld2 = to_dev_db(zp, D2)
    db2 = zp.Database(c, dD2, R, 3000, ld2)
    a_gemv = u32_host(db2.answer(u32_dev(Q2)))
    c.set_option("answer_path", "tc")
    a_tc = u32_host(db2.answer(u32_dev(Q2)))
    assert np.array_equal(a_gemv, a_tc)
    assert np.array_equal(a_gemv, lwe.matmat_mod_q(D2, Q2.T).T)
    db2.close()
    c.close()


@pytest.mark.parametrize("R,C,B", [(64, 64, 2), (100, 333, 5), (1024, 1024, 8), (257, 2000, 33),
                                   (1000, 4097, 17), (130, 1030, 64), (300, 3000, 65),
                                   (129, 700, 100)])
def test_batched_answer_parity(zp, ctx, R, C, B):
    """Batched answers (two queries: dp4a GEMV; five and more: tensor cores with byte planes,
    centred fp16, chunked exact sums)."""
    D = synth.database(R, C, B)
    Q = synth.uniform_queries(B, C, B + 1)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(ctx, dD, R, C, ld)
    got = u32_host(db.answer(u32_dev(Q)))
    assert np.array_equal(got, lwe.matmat_mod_q(D, Q.T).T)
    db.close()


@pytest.mark.parametrize("R,C,B", [(100, 333, 5), (1024, 1024, 8), (257, 2000, 33), (1000, 4097, 17),
                                   (130, 1030, 64), (300, 3000, 65), (129, 700, 100)])
def test_batched_answer_fp16_copy(zp, ctx, R, C, B):
    """The resident fp16 copy of D as the A operand (TMA straight into the tensor-core
    pipeline, no converters): the same bits as the oracle, ragged R and C (its padding holds
    the centred value of a zero byte), and after row updates the copy follows D."""
    D = synth.database(R, C, B + 7)
    Q = synth.uniform_queries(B, C, B + 8)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(ctx, dD, R, C, ld)
    db.prepare_fp16()
    got = u32_host(db.answer(u32_dev(Q)))
    assert np.array_equal(got, lwe.matmat_mod_q(D, Q.T).T)
    rows = np.array([0, R // 2, R - 1], dtype=np.uint32)
    new = synth.database(len(rows), C, B + 9)
    db.update_rows(rows, torch.from_numpy(new).cuda())
    D2 = D.copy()
    D2[rows] = new
    got = u32_host(db.answer(u32_dev(Q)))
    assert np.array_equal(got, lwe.matmat_mod_q(D2, Q.T).T)
    ctx.set_option("answer_fp16", 0)  # the byte path on the same database agrees
    try:
        assert np.array_equal(u32_host(db.answer(u32_dev(Q))), got)
    finally:
        ctx.set_option("answer_fp16", 1)
    db.close()


@pytest.mark.parametrize("dval,qval", [(0, 0), (255, 0xFFFFFFFF), (0, 0xFFFFFFFF), (255, 0),
                                       ("alt", 0xFF00FF00)])
@pytest.mark.parametrize("fp16", [False, True])
def test_batched_answer_extremes(zp, ctx, dval, qval, fp16):
    """Centred products at their extremes: |A'B'| = 2^14 for every term, so each 1024-long
    chunk sum sits exactly at the fp32 exactness limit 2^24."""
    R, C, B = 256, 3072, 20
    if dval == "alt":
        D = np.tile(np.array([0, 255], dtype=np.uint8), (R, C // 2))
    else:
        D = np.full((R, C), dval, dtype=np.uint8)
    Q = np.full((B, C), qval, dtype=np.uint32)
    Q[1::2] = ~Q[1::2]
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(ctx, dD, R, C, ld)
    if fp16:
        db.prepare_fp16()
    got = u32_host(db.answer(u32_dev(Q)))
    assert np.array_equal(got, lwe.matmat_mod_q(D, Q.T).T)
    db.close()


# K positions of the one small term, inside a 1024-long chunk: its first and last term,
# inside a K = 16 MMA step (5, 1029), at step boundaries (15, 16, 17), mid-chunk (511) and
# the start of the second chunk (1024) and the last K position (2047)
ODD_POS = [0, 5, 15, 16, 17, 511, 1023, 1024, 1029, 2047]


@pytest.mark.parametrize("fp16", [False, True])
def test_batched_answer_accumulator_keeps_24_bits(zp, ctx, fp16):
    """Every fp32 partial sum of a K chunk keeps all 24 bits: in a row, all centred products
    are 2^14 (bytes 0 x 0) except a few of -128 and one of +-1 (a database byte 129 or 127
    times a query plane byte 0x81 or 0x7F) at a varying K position, so the chunk sum lands on
    an odd value just below 2^24 (1023 2^14 +- 1 - 128 k). An accumulator with fewer bits
    would drop the odd term; the result must equal the oracle's bits."""
    R, C, B = 2 * len(ODD_POS) * 8, 2048, 8
    D = np.zeros((R, C), dtype=np.uint8)
    for r in range(R):
        D[r, ODD_POS[r % len(ODD_POS)]] = 129 if (r // len(ODD_POS)) % 2 == 0 else 127
    Q = np.zeros((B, C), dtype=np.uint32)
    for b in range(B):
        Q[b, ODD_POS] = 0x81 if b < B // 2 else 0x7F   # plane 0 only; planes 1-3 stay 0
    Q[B - 1, ODD_POS[3]] |= 0x81000000                 # one plane-3 byte as well
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(ctx, dD, R, C, ld)
    if fp16:
        db.prepare_fp16()
    ctx.set_option("answer_path", "tc")
    try:
        got = u32_host(db.answer(u32_dev(Q)))
        got1 = u32_host(db.answer(u32_dev(Q[:1])))      # a single query on the tensor cores
    finally:
        ctx.set_option("answer_path", "auto")
    want = lwe.matmat_mod_q(D, Q.T).T
    assert np.array_equal(got, want)
    assert np.array_equal(got1, want[:1])
    db.close()


def test_compression_products_accumulator_keeps_24_bits(zp):
    """The same 24-bit check for the compression products V = H.cko (byte planes of the
    negated hint times the bytes of cko, n = 1024 = one K chunk): H row r is zero but for
    H[r, j_r] = 129 or 127 (the plane-0 byte), cko[i] = 0x81 for i in the set of positions,
    so plane 0 x byte 0 of cko sums 2^14 terms with -128s and one +-1 to an odd value below
    2^24. t must equal the oracle's."""
    n = 1024
    P = Params(n=n, key_bits=2048)
    pos = [p for p in ODD_POS if p < n]
    R = 4 * len(pos)
    C = R                                   # D = identity: H+ row r = row r of A
    c = zp.Context(0, n=n)
    D = np.eye(R, C, dtype=np.uint8)
    A = np.zeros((C, n), dtype=np.uint32)
    for r in range(R):
        hneg = 129 if (r // len(pos)) % 2 == 0 else 127
        A[r, pos[r % len(pos)]] = (-hneg) % 2**32    # H+ = D.A; the negated hint is hneg
    Hn = lwe.hint_neg(D, A)
    assert Hn[0, pos[0]] == 129 and Hn[len(pos), pos[0]] == 127
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    m = synth.random_odd_modulus(2048, 31)
    cl = c.register_client(m)
    cko = [0] * n
    for p in pos:
        cko[p] = 0x81
    ans = synth.uniform_queries(1, R, 32)[0]
    for path in ("tc", "rns", "simt"):           # byte planes; residues; CUDA cores
        c.set_option("compress_path", path)
        T = db.compress([cl], u32_dev(ans[None, :]), u32_dev(synth.ints_to_limbs(cko, 64)[None]))
        assert synth.limbs_to_ints(u32_host(T)[0]) == zippir.compress_rows(ans, Hn, cko, m, P)
    assert c.device_status() == 0
    db.close()
    c.close()


@pytest.mark.parametrize("path", ["simt", "tc"])
def test_single_query_other_paths(zp, path):
    """The CUDA-core and tensor-core kernels also serve B = 1 and agree with the GEMV."""
    c = zp.Context(0, n=64)
    c.set_option("answer_path", path)
    R, C = 700, 1500
    D = synth.database(R, C, 3)
    q = synth.uniform_queries(1, C, 4)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    assert np.array_equal(u32_host(db.answer(u32_dev(q)))[0], lwe.matvec_mod_q(D, q[0]))
    db.close()
    c.close()


@pytest.mark.parametrize("R,C,n,path", [(40, 30, 16, "auto"), (300, 200, 64, "auto"),
                                        (1024, 1024, 1024, "auto"), (300, 200, 64, "simt"),
                                        (513, 1100, 96, "auto"), (70, 5000, 40, "auto")])
def test_hint_parity(zp, R, C, n, path):
    c = zp.Context(0, n=n)
    c.set_option("answer_path", path)
    D = synth.database(R, C, n)
    A = synth.seed_matrix(C, n, n)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    H = torch.empty((R, n), dtype=torch.int32, device="cuda")
    db.gen_hint(u32_dev(A), H)
    assert np.array_equal(u32_host(H), lwe.hint_plus(D, A))
    db.close()
    c.close()


def _e2e(zp, R, C, n, secret, seed, B=1, scale="proven", path=None):
    P = Params(n=n, key_bits=2048, secret=secret, scale=scale)
    c = zp.Context(0, n=n, secret=secret, scale=scale)
    if path:
        c.set_option("compress_path", path)
    D = synth.database(R, C, seed)
    A = synth.seed_matrix(C, n, seed)
    Hn = lwe.hint_neg(D, A)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    assert db.ell == P.ell and db.d1p == P.d1p(R)
    db.gen_hint(u32_dev(A))
    clients, qs = [], []
    for b in range(B):
        cl = zippir.setup(P, seed * 100 + b, sample_ck_r=False)
        qy = zippir.query(cl, A, (seed * 31 + 7 * b) % C, seed * 100 + b + 50)
        clients.append(cl)
        qs.append(qy)
    handles = [c.register_client(cl.pk.m) for cl in clients]
    Q = u32_dev(np.stack([qy.qu for qy in qs]))
    CKO = u32_dev(np.stack([synth.ints_to_limbs(qy.cko, 64) for qy in qs]))
    ans, T = db.respond(handles, Q, CKO)
    ans, T = u32_host(ans), u32_host(T)
    for b in range(B):
        want_ans = lwe.matvec_mod_q(D, qs[b].qu)
        assert np.array_equal(ans[b], want_ans)
        want_t = zippir.compress_rows(want_ans, Hn, qs[b].cko, clients[b].pk.m, P)
        got_t = synth.limbs_to_ints(T[b])
        assert got_t == want_t
        rows = range(P.d1p(R))
        rec = zippir.extract(clients[b], zippir.dec_k_shortcut(clients[b], Hn, rows), got_t, R)
        assert np.array_equal(rec, D[:, qs[b].i0])
    db.close()
    c.close()


def test_e2e_tiny_config(zp):
    """1024 x 1024 database, n = 1024, 2048-bit key: ans and t bit-identical to the oracle,
    and the client recovers its record from the GPU's response."""
    _e2e(zp, 1024, 1024, 1024, "uniform", 1)


@pytest.mark.parametrize("R,C,n,secret,seed,B", [
    (27, 16, 32, "uniform", 2, 1), (28, 40, 32, "uniform", 3, 2), (100, 64, 48, "binary", 4, 1),
    (500, 300, 128, "uniform", 5, 3), (49, 33, 1024, "binary", 6, 1)])
def test_e2e_ragged(zp, R, C, n, secret, seed, B):
    _e2e(zp, R, C, n, secret, seed, B)


@pytest.mark.parametrize("R,C,n,secret,seed,B,path", [
    (1024, 1024, 1024, "uniform", 11, 1, None), (700, 256, 1024, "binary", 12, 2, None),
    (300, 64, 64, "uniform", 13, 8, "rns"), (200, 96, 32, "binary", 14, 3, "simt")])
def test_e2e_overlap_scale(zp, R, C, n, secret, seed, B, path):
    """Overlap scale (Sec. 3.3.3): gamma = q^2 (uniform) or q (binary), 31 / 63 slots per
    packed row at n = 1024; t bit-identical to the oracle on the tensor-core, RNS and
    CUDA-core paths, and the record is recovered."""
    if n == 1024:
        assert Params(n=n, secret=secret, scale="overlap").ell == (31 if secret == "uniform" else 63)
    _e2e(zp, R, C, n, secret, seed, B, scale="overlap", path=path)


def test_compress_edge_values(zp):
    """cko at its extremes (0 and m - 1) and answers at 2^32 - 1."""
    R, C, n = 60, 32, 64
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    D = synth.database(R, C, 8)
    A = synth.seed_matrix(C, n, 8)
    Hn = lwe.hint_neg(D, A)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    from oracle import paillier
    pk, _ = paillier.keygen(2048, 77)
    m = pk.m
    cl = c.register_client(m)
    ans = np.full(R, 0xFFFFFFFF, dtype=np.uint32)
    for cko in ([m - 1] * n, [0] * n, [m - 1 if i % 2 else 0 for i in range(n)]):
        T = db.compress([cl], u32_dev(ans[None, :]), u32_dev(synth.ints_to_limbs(cko, 64)[None]))
        assert synth.limbs_to_ints(u32_host(T)[0]) == zippir.compress_rows(ans, Hn, cko, m, P)
    db.close()
    c.close()


def test_update_rows_and_regenerate(zp):
    R, C, n = 200, 96, 32
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    D = synth.database(R, C, 9)
    A = synth.seed_matrix(C, n, 9)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    H = torch.empty((R, n), dtype=torch.int32, device="cuda")
    db.gen_hint(u32_dev(A), H)
    rows = np.array([3, 77, 199], dtype=np.uint32)
    new = synth.database(3, C, 10)
    db.update_rows(rows, torch.from_numpy(new).cuda())
    assert db.stale_rows() == 3
    from oracle import paillier
    pk, _ = paillier.keygen(2048, 5)
    cl = c.register_client(pk.m)
    q = synth.uniform_queries(1, C, 11)
    cko = synth.uniform_below(pk.m, n, 12)
    with pytest.raises(zp.ZipPIRError) as ei:
        db.respond([cl], u32_dev(q), u32_dev(synth.ints_to_limbs(cko, 64)[None]))
    assert ei.value.code == zp.ZP_ESTATE
    db.gen_hint(u32_dev(A), H, rows=rows)
    assert db.stale_rows() == 0
    D2 = D.copy()
    D2[rows] = new
    assert np.array_equal(u32_host(H), lwe.hint_plus(D2, A))
    ans, T = db.respond([cl], u32_dev(q), u32_dev(synth.ints_to_limbs(cko, 64)[None]))
    want_ans = lwe.matvec_mod_q(D2, q[0])
    assert np.array_equal(u32_host(ans)[0], want_ans)
    assert synth.limbs_to_ints(u32_host(T)[0]) == zippir.compress_rows(
        want_ans, lwe.hint_neg(D2, A), cko, pk.m, P)
    db.close()
    c.close()


def test_respond_host_matches_device(zp):
    R, C, n = 300, 256, 64
    c = zp.Context(0, n=n)
    D = synth.database(R, C, 13)
    A = synth.seed_matrix(C, n, 13)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    m = synth.random_odd_modulus(2048, 14)
    cl = c.register_client(m)
    q = synth.uniform_queries(2, C, 15)
    cko = np.stack([synth.ints_to_limbs(synth.uniform_below(m, n, 16 + b), 64) for b in range(2)])
    ans_d, T_d = db.respond([cl, cl], u32_dev(q), u32_dev(cko))
    hans = np.empty((2, R), dtype=np.uint32)
    T_h = db.respond_host([cl, cl], q, cko, hAns=hans)
    assert np.array_equal(T_h, u32_host(T_d)) and np.array_equal(hans, u32_host(ans_d))
    db.close()
    c.close()


@pytest.mark.parametrize("B", [1, 9])
def test_respond_host_after_device_calls(zp, B):
    """zp_respond_host after device-buffer calls have sized the products' scratch (n = 1024,
    the single-query overlap path and the RNS path of nine queries): its inputs must not share
    a buffer with the kernels' operands, and t equals the oracle's."""
    R, C, n = 2100, 512, 1024
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    D = synth.database(R, C, 21)
    A = synth.seed_matrix(C, n, 22)
    Hn = lwe.hint_neg(D, A)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    ms = [synth.random_odd_modulus(2048, 23 + b) for b in range(B)]
    cls = [c.register_client(m) for m in ms]
    q = synth.uniform_queries(B, C, 24)
    ckos = [synth.uniform_below(ms[b], n, 25 + b) for b in range(B)]
    cko = np.stack([synth.ints_to_limbs(x, 64) for x in ckos])
    for _ in range(2):
        ans_d, T_d = db.respond(cls, u32_dev(q), u32_dev(cko))
    hans = np.empty((B, R), dtype=np.uint32)
    for _ in range(2):
        T_h = db.respond_host(cls, q, cko, hAns=hans)
        assert np.array_equal(T_h, u32_host(T_d)) and np.array_equal(hans, u32_host(ans_d))
    for b in (0, B - 1):
        assert synth.limbs_to_ints(T_h[b]) == zippir.compress_rows(hans[b], Hn, ckos[b], ms[b], P)
    db.close()
    c.close()


def test_invalid_arguments_fail_loudly(zp, ctx):
    D = synth.database(10, 16, 1)
    dD, ld = to_dev_db(zp, D)
    with pytest.raises(zp.ZipPIRError):
        zp.zp_setup_db(ctx.handle, dD.data_ptr() + 1, 10, 16, 16)   # misaligned
    with pytest.raises(zp.ZipPIRError):
        zp.zp_setup_db(ctx.handle, dD.data_ptr(), 10, 16, 8)        # pitch < C
    db = zp.Database(ctx, dD, 10, 16, ld)
    with pytest.raises(zp.ZipPIRError) as ei:                      # no hint yet
        db.compress([ctx.register_client(synth.random_odd_modulus(2048, 1))],
                    torch.zeros((1, 10), dtype=torch.int32, device="cuda"),
                    torch.zeros((1, 1024 * 64), dtype=torch.int32, device="cuda"))
    assert ei.value.code == zp.ZP_ESTATE
    with pytest.raises(zp.ZipPIRError):
        ctx.register_client(2**2047)          # even
    with pytest.raises(zp.ZipPIRError):
        ctx.register_client(2**2046 + 1)      # too short
    assert ctx.device_status() == 0
    db.close()


@pytest.mark.parametrize("n", [64, 1000, 1024])
def test_compress_tc_equals_simt(zp, n):
    """The tensor-core and CUDA-core compression products give identical t."""
    R, C = 333, 128
    D = synth.database(R, C, n)
    A = synth.seed_matrix(C, n, n)
    dD, ld = to_dev_db(zp, D)
    m = synth.random_odd_modulus(2048, n)
    cko = u32_dev(np.stack([synth.ints_to_limbs(synth.uniform_below(m, n, 7 + b), 64) for b in range(3)]))
    ans = u32_dev(synth.uniform_queries(3, R, 9))
    outs = []
    for path in ("simt", "tc"):
        c = zp.Context(0, n=n)
        c.set_option("compress_path", path)
        db = zp.Database(c, dD, R, C, ld)
        db.gen_hint(u32_dev(A))
        cl = c.register_client(m)
        outs.append(u32_host(db.compress([cl, cl, cl], ans, cko)))
        db.close()
        cl.close()
        c.close()
    assert np.array_equal(outs[0], outs[1])


def test_compress_zero_database(zp):
    """D = 0 gives H = 0: every hint byte centres to -128 and, with cko = 0, each product sum
    is exactly 2^24 before the correction; t must equal b' mod m."""
    R, C, n = 100, 64, 1024
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    D = np.zeros((R, C), dtype=np.uint8)
    A = synth.seed_matrix(C, n, 1)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    m = synth.random_odd_modulus(2048, 3)
    cl = c.register_client(m)
    ans = synth.uniform_queries(1, R, 4)
    for cko in ([0] * n, [m - 1] * n):
        T = db.compress([cl], u32_dev(ans), u32_dev(synth.ints_to_limbs(cko, 64)[None]))
        assert synth.limbs_to_ints(u32_host(T)[0]) == zippir.compress_rows(
            ans[0], np.zeros((R, n), dtype=np.uint32), cko, m, P)
    db.close()
    c.close()


@pytest.mark.parametrize("overlap", [0, 40, 100])
def test_respond_overlap_identical(zp, overlap):
    """With the compression products running concurrently on a subset of SMs, the single-query
    Response is identical to the oracle (and to the sequential one)."""
    R, C, n = 2000, 3000, 1024
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    c.set_option("overlap_sms", overlap)
    D = synth.database(R, C, 21)
    A = synth.seed_matrix(C, n, 21)
    Hn = lwe.hint_neg(D, A)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    m = synth.random_odd_modulus(2048, 22)
    cl = c.register_client(m)
    q = synth.uniform_queries(1, C, 23)
    cko = synth.uniform_below(m, n, 24)
    for rep in range(2):
        ans, T = db.respond([cl], u32_dev(q), u32_dev(synth.ints_to_limbs(cko, 64)[None]))
        want = lwe.matvec_mod_q(D, q[0])
        assert np.array_equal(u32_host(ans)[0], want)
        assert synth.limbs_to_ints(u32_host(T)[0]) == zippir.compress_rows(want, Hn, cko, m, P)
    assert c.device_status() == 0
    db.close()
    c.close()


@pytest.mark.parametrize("secret,n", [("uniform", 1024), ("binary", 48)])
def test_respond_pack_split(zp, secret, n):
    """One query with its products beside the answer: the V part of the packing reduced on
    the internal stream and (b' + Y) mod m after the join ("pack_split" 1) gives the same bits
    as packing everything after the join (0) and the oracle's t; ragged last packed row, two
    calls in a row, for both secrets (binary: ell = 54, X up to 4077 bits before the fold)."""
    R, C = 2000, 1000
    P = Params(n=n, key_bits=2048, secret=secret)
    c = zp.Context(0, n=n, secret=secret)
    c.set_option("overlap_sms", 40)
    D = synth.database(R, C, 31)
    A = synth.seed_matrix(C, n, 32)
    Hn = lwe.hint_neg(D, A)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    m = synth.random_odd_modulus(2048, 33)
    cl = c.register_client(m)
    outs = []
    for split in (1, 0, 1):
        c.set_option("pack_split", split)
        q = synth.uniform_queries(1, C, 34 + len(outs))
        cko = synth.uniform_below(m, n, 35)
        ans, T = db.respond([cl], u32_dev(q), u32_dev(synth.ints_to_limbs(cko, 64)[None]))
        want = lwe.matvec_mod_q(D, q[0])
        assert np.array_equal(u32_host(ans)[0], want)
        t = synth.limbs_to_ints(u32_host(T)[0])
        assert t == zippir.compress_rows(want, Hn, cko, m, P)
        outs.append(t)
    assert c.device_status() == 0
    db.close()
    c.close()


def test_split_compress_api(zp):
    """zp_compress_products + zp_compress_finish equal zp_compress; a finish whose batch
    does not match the products is refused."""
    R, C, n = 300, 200, 128
    c = zp.Context(0, n=n)
    D = synth.database(R, C, 31)
    A = synth.seed_matrix(C, n, 31)
    dD, ld = to_dev_db(zp, D)
    db = zp.Database(c, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    m = synth.random_odd_modulus(2048, 32)
    cl = c.register_client(m)
    cko = u32_dev(np.stack([synth.ints_to_limbs(synth.uniform_below(m, n, 33 + b), 64) for b in range(2)]))
    ans = u32_dev(synth.uniform_queries(2, R, 34))
    ref = db.compress([cl, cl], ans, cko)
    st = torch.cuda.current_stream().cuda_stream
    T = torch.empty_like(ref)
    zp.zp_compress_products(db.handle, cko.data_ptr(), 2, st)
    zp.zp_compress_finish(db.handle, [cl, cl], ans.data_ptr(), 2, T.data_ptr(), st)
    assert torch.equal(T, ref)
    with pytest.raises(zp.ZipPIRError) as ei:
        zp.zp_compress_finish(db.handle, [cl], ans.data_ptr(), 1, T.data_ptr(), st)
    assert ei.value.code == zp.ZP_ESTATE
    db.close()
    c.close()
