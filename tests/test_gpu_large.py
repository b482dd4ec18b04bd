"""Full-size parity on the 8 GiB database (65536 x 131072, n = 1024): answers for batches of
1, 8 and 128 queries, the hint and the compressed answer, checked against the oracle on
sampled outputs (whole rows of the answer, whole rows of the hint, whole packed rows of t,
including the ragged last packed row)."""
import numpy as np
import pytest

import synth
from oracle import lwe, zippir
from oracle.params import Params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R, C, n = 65536, 131072, 1024


@pytest.fixture(scope="module")
def big():
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as zp
    ctx = zp.Context(0, n=n)
    ld = zp.db_pitch(C)
    D = synth.device_database(R, C, 5, "cuda", ld=ld)
    A = synth.device_uniform_u32((C, n), 6, "cuda")
    db = zp.Database(ctx, D, R, C, ld)
    H = torch.empty((R, n), dtype=torch.int32, device="cuda")
    db.gen_hint(A, H)
    torch.cuda.synchronize()
    A_h = A.cpu().numpy().view(np.uint32)
    yield zp, ctx, db, D, A_h, H
    db.close()
    ctx.close()


def _rows(D, rows):
    return D[rows].cpu().numpy()[:, :C]


@pytest.mark.parametrize("B", [1, 8, 128])
def test_answers_sampled(big, B):
    zp, ctx, db, D, A_h, H = big
    Q = synth.device_uniform_u32((B, C), 100 + B, "cuda")
    ans = db.answer(Q)
    torch.cuda.synchronize()
    rows = [0, 1, 4097, 33333, R - 1]
    Dr = _rows(D, rows)
    Qh = Q.cpu().numpy().view(np.uint32)
    got = ans.cpu().numpy().view(np.uint32)
    for b in sorted({0, B // 2, B - 1}):
        assert np.array_equal(got[b, rows], lwe.matvec_mod_q(Dr, Qh[b]))
    assert ctx.device_status() == 0


def test_hint_sampled(big):
    zp, ctx, db, D, A_h, H = big
    rows = [0, 777, R - 1]
    want = lwe.hint_plus(_rows(D, rows), A_h)
    assert np.array_equal(H[rows].cpu().numpy().view(np.uint32), want)


def test_compress_sampled_packed_rows(big):
    zp, ctx, db, D, A_h, H = big
    P = Params(n=n, key_bits=2048)
    ell = P.ell
    m = synth.random_odd_modulus(2048, 9)
    cl = ctx.register_client(m)
    cko = synth.uniform_below(m, n, 10)
    q = synth.device_uniform_u32((1, C), 11, "cuda")
    ans, T = db.respond([cl], q, torch.from_numpy(synth.ints_to_limbs(cko, 64).view(np.int32)[None]).cuda())
    torch.cuda.synchronize()
    ans_h = ans.cpu().numpy().view(np.uint32)[0]
    T_h = T.cpu().numpy().view(np.uint32)[0]
    d1p = P.d1p(R)
    assert T_h.shape[0] == d1p
    for rp in (0, d1p - 1):                      # the last packed row is ragged (R % ell rows)
        r0, r1 = rp * ell, min(R, (rp + 1) * ell)
        rows = list(range(r0, r1))
        Dr = _rows(D, rows)
        ans_o = lwe.matvec_mod_q(Dr, q.cpu().numpy().view(np.uint32)[0])
        assert np.array_equal(ans_h[r0:r1], ans_o)
        Hn = lwe.hint_neg(Dr, A_h)               # rows r0..r1 of -D.A
        full_ans = np.zeros(ell, dtype=np.uint32)
        full_ans[:r1 - r0] = ans_o
        Hpad = np.zeros((ell, n), dtype=np.uint32)
        Hpad[:r1 - r0] = Hn
        # the oracle on this packed row alone: rows past R are zero
        t = zippir.compress_rows(full_ans[:r1 - r0], Hpad[:r1 - r0], cko, m, P, packed_rows=[0])
        assert synth.limbs_to_ints(T_h[rp:rp + 1]) == t
    assert ctx.device_status() == 0


def test_fp16_copy_answers_and_hint_randomized_check(big):
    """Batches of 8 and 128 queries answered from the resident fp16 copy of D (the operand the
    8 GiB benchmark workloads use) give the byte path's bits; every answer of both batches and
    every entry of the hint H+ = D.A pass the randomized product check against the oracle
    (tests/bigcheck.py: 16 projections W^T D of the whole database by the oracle's products,
    a miss probability of at most 2^-16 per wrong column, 2^-32 unless its errors are all
    multiples of 2^31); sampled rows are recomputed by the oracle directly."""
    import bigcheck
    zp, ctx, db, D, A_h, H = big
    Qs = {B: synth.device_uniform_u32((B, C), 200 + B, "cuda") for B in (8, 128)}
    by_bytes = {B: db.answer(Q) for B, Q in Qs.items()}
    db.prepare_fp16()
    by_fp16 = {B: db.answer(Q) for B, Q in Qs.items()}
    torch.cuda.synchronize()
    for B in Qs:
        assert torch.equal(by_fp16[B], by_bytes[B])
    assert ctx.device_status() == 0
    Dh = D.cpu().numpy()
    W = synth.uniform_queries(16, R, 210).T.copy()        # R x 16
    U = bigcheck.left_projection(Dh, C, W)
    rows = [0, 1, 4097, 33333, R - 1]
    for B, Q in Qs.items():
        Qh = Q.cpu().numpy().view(np.uint32)
        got = by_fp16[B].cpu().numpy().view(np.uint32)
        bad = bigcheck.freivalds(W, U, np.ascontiguousarray(got.T), np.ascontiguousarray(Qh.T))
        assert bad.size == 0, "B=%d: queries with wrong answers %s" % (B, bad[:10])
        want = bigcheck.rows_product(np.ascontiguousarray(Dh[rows, :C]), np.ascontiguousarray(Qh.T))
        assert np.array_equal(got[:, rows], want.T)
    Hh = H.cpu().numpy().view(np.uint32)
    bad = bigcheck.freivalds(W, U, Hh, A_h)
    assert bad.size == 0, "hint columns with wrong entries: %s" % bad[:10]
