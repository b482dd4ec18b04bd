"""Failure detection on the GPU without a fault: a bounded wait that nothing satisfies gives
up after its limit, reports it in the context's status word, and leaves the context usable."""
import time

import numpy as np
import pytest

import synth
from oracle import lwe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zp():
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as m
    return m


def test_bounded_wait_times_out_and_context_survives(zp):
    c = zp.Context(0, n=64)
    assert c.device_status() == 0
    t0 = time.perf_counter()
    c.selftest_wait(4_000_000)  # about 2 ms at 2 GHz
    status = c.device_status()  # synchronises
    assert status & 0x4
    assert time.perf_counter() - t0 < 5.0
    assert c.device_status() == 0  # cleared by the read
    # the context keeps working: an answer on the same context is exact
    R, C = 300, 1000
    D = synth.database(R, C, 3)
    q = synth.uniform_queries(1, C, 4)
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    db = zp.Database(c, torch.from_numpy(buf).cuda(), R, C, ld)
    got = db.answer(torch.from_numpy(q.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)[0]
    assert np.array_equal(got, lwe.matvec_mod_q(D, q[0]))
    assert c.device_status() == 0
    with pytest.raises(zp.ZipPIRError):
        c.selftest_wait(1 << 40)
    db.close()
    c.close()
