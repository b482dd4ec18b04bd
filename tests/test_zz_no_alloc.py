"""zp_answer_noalloc: the single-query answer for callers that cannot allocate device
memory (serving threads that must not block on the allocator, plug-ins inside a host whose
memory manager owns all of HBM). Its scratch is a fixed array compiled into the library;
these tests compare it, through the C ABI, with zp_answer on the same database, on two
calls in a row, at a ragged size and at the largest size the array holds, and check its
size limit."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _db(zp, ctx, R, C, seed):
    D = synth.database(R, C, seed)
    ld = zp.db_pitch(C)
    buf = np.zeros((R, ld), dtype=np.uint8)
    buf[:, :C] = D
    dD = torch.from_numpy(buf).cuda()
    return zp.Database(ctx, dD, R, C, ld), dD


@pytest.mark.parametrize("R,C", [(3001, 70001), (129, 1 << 18)])
def test_noalloc_matches_answer_twice(R, C):
    """Two calls in a row (the second finds the first one's planes in the array) give
    zp_answer's bits: a ragged size, and C = 262144, where the planes fill the array."""
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as zp
    lib = zp.load_library()
    ctx = zp.Context(0, n=64)
    db, dD = _db(zp, ctx, R, C, 5)
    stream = torch.cuda.current_stream().cuda_stream
    dev0 = torch.cuda.current_device()
    for call in range(2):
        q = synth.uniform_queries(1, C, 10 + call)
        dq = torch.from_numpy(q.view(np.int32)).cuda()
        ref = db.answer(dq)
        out = torch.full((1, R), -1, dtype=torch.int32, device="cuda")
        rc = lib.zp_answer_noalloc(db.handle, dq.data_ptr(), out.data_ptr(), stream)
        assert rc == 0, zp.last_error()
        assert torch.cuda.current_device() == dev0
        torch.cuda.synchronize()
        assert torch.equal(out, ref)          # integer results: exact
    assert ctx.device_status() == 0
    db.close()
    ctx.close()


def test_noalloc_rejects_too_many_columns():
    import paper_2603_09190_gb300 as zp
    lib = zp.load_library()
    ctx = zp.Context(0, n=64)
    C = (1 << 18) + 16
    db, dD = _db(zp, ctx, 1, C, 6)
    dq = torch.zeros((1, C), dtype=torch.int32, device="cuda")
    out = torch.zeros((1, 1), dtype=torch.int32, device="cuda")
    rc = lib.zp_answer_noalloc(db.handle, dq.data_ptr(), out.data_ptr(), None)
    assert rc == zp.ZP_EINVAL and "262144" in zp.last_error()
    db.close()
    ctx.close()
