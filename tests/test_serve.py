"""Serving loop: scheduling logic with a fake backend (CPU), and on the GPU the identity of
every result alone and in a mix of concurrent batches over several databases."""
import numpy as np
import pytest

from paper_2603_09190_gb300.serve import Request, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """Batches finish `dur` clock units after launch; records every launch and update."""

    def __init__(self, clock, dur=1.0, db_bytes=100, per_query=10):
        self.clock, self.dur = clock, dur
        self._db_bytes, self.per_query = db_bytes, per_query
        self.launches, self.updates, self.busy = [], [], {}

    def db_bytes(self, name):
        return self._db_bytes

    def batch_bytes(self, name, B):
        return B * self.per_query

    def launch(self, name, reqs, slot=0):
        self.launches.append((self.clock(), name, [r.rid for r in reqs], slot))
        self.busy[name] = max(self.busy.get(name, -1), self.clock() + self.dur)
        return (name, self.clock() + self.dur)

    def poll(self, h):
        return self.clock() >= h[1]

    def finish(self, h, reqs):
        for r in reqs:
            r.T = np.array([r.rid], dtype=np.uint32)

    def idle(self, name):
        return self.clock() >= self.busy.get(name, -1)

    def apply_updates(self, name, rows, new_rows):
        self.updates.append((self.clock(), name, list(rows)))


def _req(rid, db, t):
    return Request(rid, db, "c%d" % (rid % 3), np.zeros(4, np.uint32), np.zeros((2, 2), np.uint32), t)


def test_continuous_batching_and_overlap():
    """One slot per database: requests that arrive while its batch runs form the next one;
    batches of different databases overlap."""
    clk = FakeClock()
    be = FakeBackend(clk)
    srv = Server(be, hbm_budget=10_000, max_batch=8, clock=clk, slots=1)
    srv.add_database("a", 10, 10)
    srv.add_database("b", 10, 10)
    srv.submit(_req(0, "a", 0.0))
    srv.step()                                   # batch [0] starts on a
    for rid in range(1, 6):                      # arrive while a is busy
        clk.t = 0.1 * rid
        srv.submit(_req(rid, "a", clk.t))
        srv.submit(_req(100 + rid, "b", clk.t))
        srv.step()
    # b started as soon as its first request came; a's new arrivals wait for the slot
    assert [l[1] for l in be.launches] == ["a", "b"]
    clk.t = 1.0
    srv.step()                                   # a finishes, the waiting requests form one batch
    assert be.launches[-1][1] == "a" and be.launches[-1][2] == [1, 2, 3, 4, 5]
    for _ in range(100):                         # let the fake clock run until drained
        if not srv.pending():
            break
        clk.t += 1.0
        srv.step()
    assert not srv.pending()
    assert sorted(r.rid for r in srv.done) == sorted([0, 1, 2, 3, 4, 5] + [101, 102, 103, 104, 105])
    for r in srv.done:
        assert r.T[0] == r.rid and r.t_done >= r.t_launch >= r.t_arrival


def test_same_database_batches_overlap():
    """Two slots per database: a second batch of the same database starts while the first
    runs, a third waits for a free slot, and every result comes back."""
    clk = FakeClock()
    be = FakeBackend(clk)
    srv = Server(be, hbm_budget=10_000, max_batch=8, clock=clk, slots=2)
    srv.add_database("a", 10, 10)
    for rid in range(3):
        srv.submit(_req(rid, "a", 0.0))
    srv.step()
    clk.t = 0.2
    for rid in (3, 4):
        srv.submit(_req(rid, "a", 0.2))
    srv.step()
    assert [(l[0], l[2], l[3]) for l in be.launches] == [(0.0, [0, 1, 2], 0), (0.2, [3, 4], 1)]
    assert srv.max_same_db == 2
    clk.t = 0.5
    srv.submit(_req(5, "a", 0.5))
    srv.step()
    assert len(be.launches) == 2                  # both slots busy: 5 waits
    clk.t = 1.0
    srv.step()                                    # the first batch ends; 5 takes its slot
    assert be.launches[-1] == (1.0, "a", [5], 0)
    while srv.pending():
        clk.t += 1.0
        srv.step()
    assert sorted(r.rid for r in srv.done) == list(range(6))
    for r in srv.done:
        assert r.T[0] == r.rid and r.t_done >= r.t_launch >= r.t_arrival
    assert srv.report(0.0, clk.t)["max_batches_of_one_db_in_flight"] == 2


def test_hbm_budget_limits_batches():
    clk = FakeClock()
    be = FakeBackend(clk, db_bytes=100, per_query=10)
    srv = Server(be, hbm_budget=100 + 100 + 45, max_batch=64, clock=clk)
    srv.add_database("a", 1, 1)
    srv.add_database("b", 1, 1)
    with pytest.raises(MemoryError):
        srv.add_database("c", 1, 1)
    for rid in range(20):
        srv.submit(_req(rid, "a", 0.0))
        srv.submit(_req(50 + rid, "b", 0.0))
    srv.step()
    # 45 bytes left: a gets 4 queries (halving 20 -> 10 -> 5... until it fits), b what remains
    sizes = [len(l[2]) for l in be.launches]
    assert sum(s * 10 for s in sizes) <= 45
    assert srv.inflight_bytes <= 45
    while srv.pending():
        clk.t += 1.0
        srv.step()
        assert srv.inflight_bytes <= 45
    assert len(srv.done) == 40


def test_updates_applied_only_when_idle():
    clk = FakeClock()
    be = FakeBackend(clk)
    srv = Server(be, hbm_budget=10_000, clock=clk)
    srv.add_database("a", 10, 10)
    srv.submit(_req(0, "a", 0.0))
    srv.step()
    srv.update_rows("a", [3, 4], None)
    srv.submit(_req(1, "a", 0.0))
    clk.t = 0.5
    srv.step()
    assert be.updates == []                      # batch still running
    clk.t = 1.0
    srv.step()                                   # finish, then update, then next batch
    assert be.updates == [(1.0, "a", [3, 4])]
    assert be.launches[-1][2] == [1] and be.launches[-1][0] == 1.0
    assert srv.regenerations == 1


@pytest.mark.gpu
def test_results_identical_alone_and_in_mix():
    torch = pytest.importorskip("torch")
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as zp
    import synth
    from oracle import lwe, zippir
    from oracle.params import Params
    from paper_2603_09190_gb300.serve import ZipBackend

    n = 256
    ctx = zp.Context(0, n=n)
    be = ZipBackend(ctx, max_batch=16, slots=2)
    shapes = {"small": (600, 700), "mid": (1500, 1100), "wide": (300, 4000)}
    host = {}
    for i, (name, (R, C)) in enumerate(shapes.items()):
        D = synth.database(R, C, 40 + i)
        A = synth.seed_matrix(C, n, 40 + i)
        ld = zp.db_pitch(C)
        buf = np.zeros((R, ld), dtype=np.uint8)
        buf[:, :C] = D
        dD = torch.from_numpy(buf).cuda()
        db = zp.Database(ctx, dD, R, C, ld)
        dA = torch.from_numpy(A.view(np.int32)).cuda()
        db.gen_hint(dA)
        be.add_database(name, db, dA)
        host[name] = (D, A, dD)
    moduli = {"c%d" % k: synth.random_odd_modulus(2048, 500 + k) for k in range(5)}
    for cid, m in moduli.items():
        be.add_client(cid, m)
    rng = synth.rng(9)
    reqs = []
    for rid in range(40):
        name = list(shapes)[int(rng.integers(0, 3))]
        cid = "c%d" % int(rng.integers(0, 5))
        R, C = shapes[name]
        q = rng.integers(0, 2**32, size=C, dtype=np.uint64).astype(np.uint32)
        cko = synth.ints_to_limbs(synth.uniform_below(moduli[cid], n, 1000 + rid), 64)
        reqs.append((rid, name, cid, q, cko))

    max_same_db = [0]

    def serve(batch_all):
        # batches of at most 8: a database with more requests fills both of its slots
        srv = Server(be, hbm_budget=40 << 30, max_batch=8, slots=2)
        for name, (R, C) in shapes.items():
            srv.add_database(name, R, C)
        out = {}
        if batch_all:
            for rid, name, cid, q, cko in reqs:
                srv.submit(Request(rid, name, cid, q, cko))
            srv.run_until_idle()
            assert srv.batches < len(reqs)       # requests were really batched together
            max_same_db[0] = srv.max_same_db
        else:
            for rid, name, cid, q, cko in reqs:
                srv.submit(Request(rid, name, cid, q, cko))
                srv.run_until_idle()
        for r in srv.done:
            out[r.rid] = (r.T, r.ans)
        return out

    alone = serve(False)
    mix = serve(True)
    assert alone.keys() == mix.keys() == set(range(40))
    for rid in range(40):
        assert np.array_equal(alone[rid][0], mix[rid][0]) and np.array_equal(alone[rid][1], mix[rid][1])
    assert max_same_db[0] >= 2                   # batches of one database overlapped
    # and the results are the oracle's
    P = Params(n=n)
    for rid, name, cid, q, cko in reqs[:4]:
        D, A, _ = host[name]
        want = lwe.matvec_mod_q(D, q)
        assert np.array_equal(mix[rid][1], want)
        t = zippir.compress_rows(want, lwe.hint_neg(D, A), synth.limbs_to_ints(cko), moduli[cid], P)
        assert synth.limbs_to_ints(mix[rid][0]) == t
    assert ctx.device_status() == 0
