"""The autotuner measures and sets the batch thresholds, the SM split, the GEMV
configurations, the tile widths of the tensor-core answers and RNS products, the operand
copy and the batch overlap; every choice it can make gives the oracle's bits."""
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


def u32_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def test_autotune_then_exact(zp):
    R, C, n = 4096, 4096, 64
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    D = synth.database(R, C, 12)
    A = synth.seed_matrix(C, n, 13)
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    db = zp.Database(c, torch.from_numpy(buf).cuda(), R, C, ld)
    db.gen_hint(u32_dev(A))
    db.prepare_fp16()
    got = db.autotune()
    assert 1 <= got["gemv_max_batch"] <= 4
    assert got["rns_min_batch"] in (0, 2, 4, 6, 8, 12, 16)
    assert 0 <= got["overlap_sms"] < 200
    assert got["gemv_cfg_alone"] in (1, 2) and got["gemv_cfg_shared"] in (1, 2)
    assert got["answer_bt_16"] == 16 and got["answer_bt_32"] in (16, 32)
    assert got["answer_bt_64"] in (16, 32, 64) and got["answer_bt_128"] in (16, 32, 64)
    assert got["answer_fp16"] in (0, 1)
    assert got["rns_bt_16"] == 16 and got["rns_bt_128"] in (16, 32, 64)
    assert got["batch_overlap"] in (0, 1)
    for k, v in got.items():
        assert zp.zp_get_option_value(c, k) == v
    assert c.device_status() == 0
    Hn = lwe.hint_neg(D, A)
    for B in (1, 3, 9, 20, 64, 100):
        Q = synth.uniform_queries(B, C, 20 + B)
        ans = db.answer(u32_dev(Q))
        assert np.array_equal(ans.cpu().numpy().view(np.uint32), lwe.matmat_mod_q(D, Q.T).T)
        m = synth.random_odd_modulus(2048, 30 + B)
        cl = c.register_client(m)
        ckos = [synth.uniform_below(m, n, 40 + b) for b in range(B)]
        T = db.compress([cl] * B, ans, u32_dev(np.stack([synth.ints_to_limbs(x, 64) for x in ckos])))
        Th = T.cpu().numpy().view(np.uint32)
        a_h = ans.cpu().numpy().view(np.uint32)
        for b in (0, B - 1):
            assert synth.limbs_to_ints(Th[b]) == zippir.compress_rows(a_h[b], Hn, ckos[b], m, P)


@pytest.mark.parametrize("B", [16, 32, 64, 128])
def test_every_tile_width_exact(zp, B):
    """Every tile width the tuner can choose for a batch class, for the answers (byte and
    fp16 operands) and for the RNS products, gives the oracle's bits."""
    R, C, n = 300, 512, 64
    P = Params(n=n, key_bits=2048)
    c = zp.Context(0, n=n)
    c.set_option("compress_path", "rns")
    D = synth.database(R, C, 70 + B)
    A = synth.seed_matrix(C, n, 71 + B)
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    db = zp.Database(c, torch.from_numpy(buf).cuda(), R, C, ld)
    db.gen_hint(u32_dev(A))
    Hn = lwe.hint_neg(D, A)
    Q = synth.uniform_queries(B, C, 72 + B)
    want = lwe.matmat_mod_q(D, Q.T).T
    m = synth.random_odd_modulus(2048, 73 + B)
    cl = c.register_client(m)
    ckos = [synth.uniform_below(m, n, 74 + b) for b in range(B)]
    CKO = u32_dev(np.stack([synth.ints_to_limbs(x, 64) for x in ckos]))
    cls_name = str(B)
    first = None
    for fp16 in (False, True):
        if fp16:
            db.prepare_fp16()
        for bt in (16, 32, 64):
            if bt > min(B, 64):
                continue
            c.set_option("answer_bt_" + cls_name, bt)
            c.set_option("rns_bt_" + cls_name, bt)
            ans = db.answer(u32_dev(Q))
            a_h = ans.cpu().numpy().view(np.uint32)
            assert np.array_equal(a_h, want), (fp16, bt)
            T = db.compress([cl] * B, ans, CKO).cpu().numpy().view(np.uint32)
            if first is None:
                first = T
                for b in (0, B - 1):
                    assert synth.limbs_to_ints(T[b]) == zippir.compress_rows(a_h[b], Hn, ckos[b], m, P)
            assert np.array_equal(T, first), (fp16, bt)
    with pytest.raises(zp.ZipPIRError):
        c.set_option("answer_bt_16", 32)
    assert c.device_status() == 0
