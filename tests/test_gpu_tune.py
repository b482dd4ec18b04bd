"""The autotuner measures and sets the batch thresholds and the SM split; every path it
can pick gives the oracle's bits."""
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
    got = db.autotune()
    assert 1 <= got["gemv_max_batch"] <= 4
    assert got["rns_min_batch"] in (0, 2, 4, 6, 8, 12, 16)
    assert 0 <= got["overlap_sms"] < 200
    for k, v in got.items():
        assert zp.zp_get_option_value(c, k) == v
    assert c.device_status() == 0
    Hn = lwe.hint_neg(D, A)
    for B in (3, 9):
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
