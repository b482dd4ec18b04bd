"""Full-size parity of the batched Response as it is benchmarked: a 1 GiB database (32768 x
32768 bytes), n = 1024, 64 queries of 64 clients with their own 2048-bit moduli, answers
from the resident fp16 copy of D on the tensor cores, compression in the residue number
system from the fp16 copy of the residue planes of H' (d1' = 1214 packed rows, 38 M tiles
per prime). Checked against the oracle:

* every one of the 64 x 32768 answers, by the randomized product check of
  tests/bigcheck.py (16 projections of D by the oracle's products);
* all 64 answers on eight rows, and whole packed rows r' = 0, 1, 31, 32, 33, 607, 1212,
  1213 of t for all 64 clients (tiles g = 0, 1 and the last, ragged, packed row), each
  recomputed by the oracle from its rows of D and of the hint.
"""
import numpy as np
import pytest

import bigcheck
import synth
from oracle import lwe, zippir
from oracle.params import Params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = C = 32768
n, B = 1024, 64


@pytest.fixture(scope="module")
def run():
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as zp
    ctx = zp.Context(0, n=n)
    ld = zp.db_pitch(C)
    D = synth.device_database(R, C, 31, "cuda", ld=ld)
    A = synth.device_uniform_u32((C, n), 32, "cuda")
    db = zp.Database(ctx, D, R, C, ld)
    db.gen_hint(A)
    db.prepare_fp16()
    moduli = [synth.random_odd_modulus(2048, 300 + b) for b in range(B)]
    cls = [ctx.register_client(m) for m in moduli]
    ckos = [synth.uniform_below(moduli[b], n, 400 + b) for b in range(B)]
    CKO = torch.from_numpy(np.stack([synth.ints_to_limbs(x, 64) for x in ckos]).view(np.int32)).cuda()
    Q = synth.device_uniform_u32((B, C), 33, "cuda")
    launches0 = ctx.kernel_launches()
    ans, T = db.respond(cls, Q, CKO)
    torch.cuda.synchronize()
    assert ctx.kernel_launches() > launches0
    assert ctx.device_status() == 0
    out = {
        "D": D.cpu().numpy(), "A": A.cpu().numpy().view(np.uint32), "Q": Q.cpu().numpy().view(np.uint32),
        "ans": ans.cpu().numpy().view(np.uint32), "T": T.cpu().numpy().view(np.uint32),
        "moduli": moduli, "ckos": ckos,
    }
    yield out
    for c in cls:
        c.close()
    db.close()
    ctx.close()


def test_all_answers_randomized_check(run):
    D, Q, ans = run["D"], run["Q"], run["ans"]
    W = synth.uniform_queries(16, R, 34).T.copy()          # R x 16
    U = bigcheck.left_projection(D, C, W)
    bad = bigcheck.freivalds(W, U, np.ascontiguousarray(ans.T), np.ascontiguousarray(Q.T))
    assert bad.size == 0, "queries with wrong answers: %s" % bad[:10]


def test_answers_on_rows(run):
    D, Q, ans = run["D"], run["Q"], run["ans"]
    rows = [0, 1, 127, 128, 4095, 16384, R - 2, R - 1]
    want = bigcheck.rows_product(D[rows, :C], np.ascontiguousarray(Q.T))   # 8 x 64
    assert np.array_equal(ans[:, rows], want.T)


def test_packed_rows_all_clients(run):
    D, A, Q, ans, T = run["D"], run["A"], run["Q"], run["ans"], run["T"]
    P = Params(n=n, key_bits=2048)
    ell, d1p = P.ell, P.d1p(R)
    assert T.shape == (B, d1p, 64) and d1p == 1214
    QT = np.ascontiguousarray(Q.T)
    for rp in (0, 1, 31, 32, 33, 607, d1p - 2, d1p - 1):
        r0, r1 = rp * ell, min(R, (rp + 1) * ell)
        Dr = np.ascontiguousarray(D[r0:r1, :C])
        ans_o = bigcheck.rows_product(Dr, QT)              # (r1 - r0) x 64
        assert np.array_equal(ans[:, r0:r1], ans_o.T)
        Hn = bigcheck.rows_product(Dr, A, block=1, fn=lwe.hint_neg)   # rows of -D.A
        for b in range(B):
            t = zippir.compress_rows(ans_o[:, b], Hn, run["ckos"][b], run["moduli"][b], P,
                                     packed_rows=[0])
            assert synth.limbs_to_ints(T[b, rp:rp + 1]) == t, (rp, b)
