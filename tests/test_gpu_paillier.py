"""GPU parity of the per-client hint k = PaillierMatMul(H', ck_r) and of the combined
response k (+) t (Sec. 4.3) against the oracle, through the C ABI. Exact integers:
every comparison is bit-exact."""
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


def _setup(zp, R, C, n, secret, seed, scale="proven"):
    P = Params(n=n, key_bits=2048, secret=secret, scale=scale)
    D = synth.database(R, C, seed)
    A = synth.seed_matrix(C, n, seed)
    Hn = lwe.hint_neg(D, A)
    cl = zippir.setup(P, seed + 100, sample_ck_r=True)
    ctx = zp.Context(0, n=n, key_bits=2048, secret=secret, scale=scale)
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    dD = torch.from_numpy(buf).cuda()
    db = zp.Database(ctx, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    gcl = ctx.register_client(cl.pk.m)
    ckr = u32_dev(synth.ints_to_limbs(cl.ck_r, 2 * ctx.L))
    return P, D, A, Hn, cl, ctx, db, gcl, ckr, dD


@pytest.mark.parametrize("R,C,n,secret,seed,scale", [
    (60, 48, 8, "uniform", 1, "proven"), (200, 64, 16, "uniform", 2, "proven"),
    (100, 40, 12, "binary", 3, "proven"), (100, 40, 8, "uniform", 4, "overlap"),
    (140, 40, 8, "binary", 5, "overlap")])
def test_client_hint_parity(zp, R, C, n, secret, seed, scale):
    """k on the GPU equals prod_i ck_r[i]^{H'[r', i]} mod m^2 for every packed row,
    including the ragged last one (proven and overlap scales)."""
    P, D, A, Hn, cl, ctx, db, gcl, ckr, dD = _setup(zp, R, C, n, secret, seed, scale)
    k = db.client_hint(gcl, ckr)
    got = synth.limbs_to_ints(u32_host(k))
    want = zippir.paillier_matmul_rows(cl, Hn, range(db.d1p))
    assert got == want
    assert ctx.device_status() == 0


def test_client_hint_subset_and_update(zp):
    """Recomputing listed packed rows after a row update: the listed rows change to the
    new k, the other rows are left as they were."""
    R, C, n = 90, 32, 8
    P, D, A, Hn, cl, ctx, db, gcl, ckr, dD = _setup(zp, R, C, n, "uniform", 7)
    k = db.client_hint(gcl, ckr)
    before = synth.limbs_to_ints(u32_host(k))
    rows = np.array([3, 60], dtype=np.uint32)  # packed rows 0 and 2 (ell = 27)
    new = synth.database(len(rows), C, 99)
    db.update_rows(rows, torch.from_numpy(new).cuda())
    db.gen_hint(u32_dev(A), rows=rows)
    D2 = D.copy()
    D2[rows] = new
    Hn2 = lwe.hint_neg(D2, A)
    db.client_hint(gcl, ckr, out=k, packed_rows=[0, 2])
    after = synth.limbs_to_ints(u32_host(k))
    assert after[1] == before[1]
    assert [after[0], after[2]] == zippir.paillier_matmul_rows(cl, Hn2, [0, 2])


@pytest.mark.parametrize("secret,seed", [("uniform", 11), ("binary", 12)])
def test_combined_response_recovers_record(zp, secret, seed):
    """k (+) t from the GPU equals the oracle's, and one Paillier decryption per packed row
    gives mu = Dec(k) + t mod m, from which Extract recovers column i0."""
    R, C, n = 120, 48, 8
    P, D, A, Hn, cl, ctx, db, gcl, ckr, dD = _setup(zp, R, C, n, secret, seed)
    i0 = 17
    qy = zippir.query(cl, A, i0, seed + 5)
    k = db.client_hint(gcl, ckr)
    cko = u32_dev(synth.ints_to_limbs(qy.cko, ctx.L)[None])
    _, T = db.respond([gcl], u32_dev(qy.qu[None]), cko)
    out = db.combine([gcl], k[None].contiguous(), T)
    got = synth.limbs_to_ints(u32_host(out)[0])
    t = synth.limbs_to_ints(u32_host(T)[0])
    want = zippir.combine(cl.pk, synth.limbs_to_ints(u32_host(k)), t)
    assert got == want
    mus = [paillier.decrypt(cl.sk, c) for c in got]
    rec = zippir.extract(cl, [0] * len(mus), mus, R)
    assert np.array_equal(rec, D[:, i0])


def test_combine_batch_of_clients(zp):
    """A batch of queries from different clients: each (query, packed row) uses its own
    client's m^2; edge values t = 0 and t = m - 1 and k = 1."""
    R, C, n = 60, 32, 8
    P, D, A, Hn, cl, ctx, db, gcl, ckr, dD = _setup(zp, R, C, n, "uniform", 21)
    cl2 = zippir.setup(P, 321, sample_ck_r=False)
    gcl2 = ctx.register_client(cl2.pk.m)
    d1p = db.d1p
    g = np.random.default_rng(5)
    ks, ts = [], []
    for c in (cl, cl2):
        m, m2 = c.pk.m, c.pk.m2
        kk = [1] + [int.from_bytes(g.bytes(520), "little") % m2 for _ in range(d1p - 1)]
        tt = [0, m - 1] + [int.from_bytes(g.bytes(260), "little") % m for _ in range(d1p - 2)]
        ks.append(kk)
        ts.append(tt)
    K = u32_dev(np.stack([synth.ints_to_limbs(kk, 2 * ctx.L) for kk in ks]))
    T = u32_dev(np.stack([synth.ints_to_limbs(tt, ctx.L) for tt in ts]))
    out = u32_host(db.combine([gcl, gcl2], K, T))
    for b, c in enumerate((cl, cl2)):
        assert synth.limbs_to_ints(out[b]) == zippir.combine(c.pk, ks[b], ts[b])


def test_client_hint_full_size_row(zp):
    """n = 1024 (the paper's LWE dimension), 2048-bit key: one packed row against the oracle.
    ck_r is drawn uniformly from Z_{m^2} without the client's decryptions (k does not use
    them), which keeps the oracle's side to the n modular exponentiations of that row."""
    R, C, n = 54, 64, 1024
    P = Params(n=n, key_bits=2048, secret="uniform")
    D = synth.database(R, C, 31)
    A = synth.seed_matrix(C, n, 31)
    Hn = lwe.hint_neg(D, A)
    cl0 = zippir.setup(P, 131, sample_ck_r=False)
    m2 = cl0.pk.m2
    g = np.random.default_rng(31)
    ck_r = [int.from_bytes(g.bytes(528), "little") % m2 for _ in range(n)]
    cl = zippir.Client(P, cl0.pk, cl0.sk, ck_r, [])
    ctx = zp.Context(0, n=n, key_bits=2048, secret="uniform")
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    dD = torch.from_numpy(buf).cuda()
    db = zp.Database(ctx, dD, R, C, ld)
    db.gen_hint(u32_dev(A))
    gcl = ctx.register_client(cl.pk.m)
    k = db.client_hint(gcl, u32_dev(synth.ints_to_limbs(ck_r, 2 * ctx.L)))
    got = synth.limbs_to_ints(u32_host(k))
    assert got[1] == zippir.paillier_matmul_rows(cl, Hn, [1])[0]


def test_client_hint_invalid_arguments(zp):
    R, C, n = 60, 32, 8
    P, D, A, Hn, cl, ctx, db, gcl, ckr, dD = _setup(zp, R, C, n, "uniform", 41)
    with pytest.raises(zp.ZipPIRError):
        db.client_hint(gcl, ckr, packed_rows=[db.d1p])
    other = zp.Context(0, n=n)
    ocl = other.register_client(cl.pk.m)
    with pytest.raises(zp.ZipPIRError):
        db.client_hint(ocl, ckr)
