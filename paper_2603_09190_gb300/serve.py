"""Serving loop for the ZipPIR online Response: continuous batching over several resident
databases on one GPU.

Requests (one query of one client against one database) arrive at any time. Each
database has `slots` handles (the database and views of it, zp_db_view: each with its own
working buffers and CUDA stream), so up to `slots` batches of one database are in flight at
once; requests that arrive while they run wait in the database's queue and form the next
batch, launched as soon as a slot and the HBM budget allow -- batches of the same and of
different databases overlap on the device. Per-client state (the registered Paillier
modulus and its Barrett constant) stays resident. Database updates are queued; a database
with pending updates takes no new batch until its batches in flight have finished, then the
updates are applied and the stale hint rows regenerated (Sec. 6, "Database updates") before
its next batch.

The scheduling logic is plain Python over a small backend interface, so it is tested on
the CPU with a fake backend; `ZipBackend` drives the real library.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    db: str
    client: str
    q: np.ndarray            # u32 (C,)
    cko: np.ndarray          # u32 (n, L)
    t_arrival: float = 0.0
    t_launch: float = 0.0
    t_done: float = 0.0
    T: np.ndarray | None = None     # u32 (d1', L): the compressed answer
    ans: np.ndarray | None = None   # u32 (R,): the plain LWE answer

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class _Batch:
    handle: object                   # backend handle of the running batch
    reqs: list
    nbytes: int
    slot: int


@dataclass
class _DbState:
    name: str
    R: int
    C: int
    slots: int
    queue: collections.deque = field(default_factory=collections.deque)
    inflight: list = field(default_factory=list)   # _Batch of the batches on the device
    updates: list = field(default_factory=list)    # (rows, new_rows) waiting for idle time
    scanned_bytes: int = 0

    def free_slot(self) -> int | None:
        used = {b.slot for b in self.inflight}
        for s in range(self.slots):
            if s not in used:
                return s
        return None


class Server:
    """Continuous-batching scheduler.

    backend: object with
      db_bytes(name) -> int                       resident bytes of a database (D + hint state)
      batch_bytes(name, B) -> int                 device bytes one batch of B queries needs
      launch(name, requests, slot) -> handle      asynchronous Response of a batch on slot
                                                  (0 <= slot < slots) of the database
      poll(handle) -> bool                        batch finished?
      finish(handle, requests) -> None            fills T / ans of the requests
      apply_updates(name, rows, new_rows) -> None asynchronous row update + hint regeneration
      idle(name) -> bool                          no device work pending for the database
    slots: batches of one database that may be in flight at once (the backend holds that
    many handles per database).
    """

    def __init__(self, backend, hbm_budget: int, max_batch: int = 64, clock=time.perf_counter,
                 slots: int = 2):
        self.backend = backend
        self.hbm_budget = int(hbm_budget)
        self.max_batch = int(max_batch)
        self.slots = int(slots)
        self.max_same_db = 0             # most batches of one database seen in flight at once
        self.clock = clock
        self.dbs: dict[str, _DbState] = {}
        self.resident = 0
        self.inflight_bytes = 0
        self.done: list[Request] = []
        self.lock = threading.Lock()
        self.regenerations = 0
        self.batches = 0

    # ------------------------------------------------------------------ setup
    def add_database(self, name: str, R: int, C: int):
        need = self.backend.db_bytes(name)
        if self.resident + need > self.hbm_budget:
            raise MemoryError("database %s (%d bytes) does not fit the HBM budget" % (name, need))
        self.resident += need
        self.dbs[name] = _DbState(name, R, C, self.slots)

    # ------------------------------------------------------------------ traffic
    def submit(self, req: Request):
        with self.lock:
            req.t_arrival = req.t_arrival or self.clock()
            self.dbs[req.db].queue.append(req)

    def update_rows(self, db: str, rows, new_rows):
        with self.lock:
            self.dbs[db].updates.append((np.asarray(rows, dtype=np.uint32), new_rows))

    def pending(self) -> int:
        return sum(len(d.queue) + sum(len(b.reqs) for b in d.inflight) + len(d.updates)
                   for d in self.dbs.values())

    # ------------------------------------------------------------------ progress
    def step(self) -> int:
        """Completes finished batches, applies updates of idle databases, launches new
        batches within the budget. Returns the number of requests completed."""
        completed = 0
        with self.lock:
            for d in self.dbs.values():
                for bt in [b for b in d.inflight if self.backend.poll(b.handle)]:
                    self.backend.finish(bt.handle, bt.reqs)
                    now = self.clock()
                    for r in bt.reqs:
                        r.t_done = now
                    self.done.extend(bt.reqs)
                    completed += len(bt.reqs)
                    d.scanned_bytes += len(bt.reqs) * d.R * d.C
                    self.inflight_bytes -= bt.nbytes
                    d.inflight.remove(bt)
            # idle time: apply queued updates and regenerate the stale hint rows (a database
            # with updates pending takes no new batch until its batches in flight are done)
            for d in self.dbs.values():
                if not d.inflight and d.updates and self.backend.idle(d.name):
                    for rows, new_rows in d.updates:
                        self.backend.apply_updates(d.name, rows, new_rows)
                        self.regenerations += 1
                    d.updates = []
            # admit: oldest head-of-queue first, as slots and memory allow
            blocked = set()              # databases whose smallest batch does not fit now
            while True:
                ready = [d for d in self.dbs.values() if d.queue and not d.updates and
                         d.name not in blocked and d.free_slot() is not None]
                if not ready:
                    break
                d = min(ready, key=lambda x: x.queue[0].t_arrival)
                B = min(len(d.queue), self.max_batch)
                while B > 0:
                    need = self.backend.batch_bytes(d.name, B)
                    if self.resident + self.inflight_bytes + need <= self.hbm_budget:
                        break
                    B //= 2
                if B == 0:
                    blocked.add(d.name)
                    continue
                reqs = [d.queue.popleft() for _ in range(B)]
                now = self.clock()
                for r in reqs:
                    r.t_launch = now
                slot = d.free_slot()
                nbytes = self.backend.batch_bytes(d.name, B)
                d.inflight.append(_Batch(self.backend.launch(d.name, reqs, slot), reqs, nbytes, slot))
                self.inflight_bytes += nbytes
                self.batches += 1
                self.max_same_db = max(self.max_same_db, len(d.inflight))
        return completed

    def run_until_idle(self, timeout: float = 600.0):
        t0 = time.perf_counter()
        while self.pending():
            if self.step() == 0:
                time.sleep(0.0002)
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError("serving loop did not drain")

    # ------------------------------------------------------------------ metrics
    def report(self, t_begin: float, t_end: float) -> dict:
        lat = np.array([r.latency for r in self.done]) * 1e3
        scanned = sum(d.scanned_bytes for d in self.dbs.values())
        span = max(t_end - t_begin, 1e-9)
        return {"requests": len(self.done), "qps": len(self.done) / span,
                "db_gb_s": scanned / span / 1e9,
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "batches": self.batches, "mean_batch": len(self.done) / max(self.batches, 1),
                "hint_regenerations": self.regenerations,
                "max_batches_of_one_db_in_flight": self.max_same_db}


class ZipBackend:
    """Backend on the real library: per database, `slots` handles (the database and views of
    it, each with its own library scratch), each with a CUDA stream and pinned staging and
    device buffers sized for the largest batch."""

    def __init__(self, ctx, max_batch: int = 64, slots: int = 2):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.max_batch = max_batch
        self.slots = slots
        self.d = {}          # name -> dict(db, A, per-slot handles/streams/buffers)
        self.clients = {}    # client id -> Client

    def add_client(self, cid, m: int):
        self.clients[cid] = self.ctx.register_client(m)

    def add_database(self, name, db, A):
        torch = self.torch
        Bm, C, R, L, n = self.max_batch, db.C, db.R, db.L, self.ctx.n
        dev = db.D.device
        if Bm >= 8 and n <= 1024:
            db.prepare_rns()  # large batches compress in RNS: build its tables now, not mid-run
        if Bm > 4:
            db.prepare_fp16()  # batches of five and more answer from the fp16 copy of D
        slots = []
        for s in range(self.slots):
            slots.append({
                "db": db if s == 0 else db.view(), "stream": torch.cuda.Stream(dev),
                "hQ": torch.empty((Bm, C), dtype=torch.int32, pin_memory=True),
                "hK": torch.empty((Bm, n, L), dtype=torch.int32, pin_memory=True),
                "hT": torch.empty((Bm, db.d1p, L), dtype=torch.int32, pin_memory=True),
                "hA": torch.empty((Bm, R), dtype=torch.int32, pin_memory=True),
                "Q": torch.empty((Bm, C), dtype=torch.int32, device=dev),
                "K": torch.empty((Bm, n, L), dtype=torch.int32, device=dev),
                "T": torch.empty((Bm, db.d1p, L), dtype=torch.int32, device=dev),
                "ans": torch.empty((Bm, R), dtype=torch.int32, device=dev),
            })
        self.d[name] = {"db": db, "A": A, "slots": slots}

    def db_bytes(self, name):
        x = self.d[name]
        db = x["db"]
        n = self.ctx.n
        Rp = (db.R + 31) // 32 * 32
        Rq = (db.d1p + 31) // 32 * 32
        rns = 153 * 4 * Rq * (math.ceil(n / 16) * 16 + 4) if self.max_batch >= 8 and n <= 1024 else 0
        d16 = 2 * db.R * ((db.C + 127) // 128 * 128) if self.max_batch > 4 else 0
        if self.max_batch >= 8 and n <= 1024:
            d16 += 2 * 153 * 4 * Rq * ((n + 127) // 128 * 128)  # fp16 copy of the RNS planes
        bufs = sum(t.numel() * t.element_size() for sl in x["slots"] for k, t in sl.items()
                   if k in ("Q", "K", "T", "ans"))
        return db.R * db.ld + db.R * n * 8 + 4 * Rp * math.ceil(n / 16) * 16 + rns + d16 + bufs

    def batch_bytes(self, name, B):
        db = self.d[name]["db"]
        n = self.ctx.n
        Kp = (db.C + 63) // 64 * 64
        Rp = (db.R + 31) // 32 * 32
        Rq = (db.d1p + 31) // 32 * 32
        # library scratch of one batch (per handle): compression products or residues, the
        # fp16 operand planes, the CRT buffers of the RNS path
        return B * Rp * 67 * 4 + B * 256 * ((n + 63) // 64 * 64) * 2 + \
            ((B + 63) // 64) * 256 * Kp * 2 + B * Rq * (4 * 160 + 67 * 4 + 16)

    def launch(self, name, reqs, slot=0):
        import paper_2603_09190_gb300 as zp
        torch = self.torch
        x = self.d[name]["slots"][slot]
        db, st = x["db"], x["stream"]
        B = len(reqs)
        hQ, hK = x["hQ"].numpy().view(np.uint32), x["hK"].numpy().view(np.uint32)
        for i, r in enumerate(reqs):
            hQ[i] = r.q
            hK[i] = r.cko
        st.wait_stream(torch.cuda.current_stream(db.D.device))
        with torch.cuda.stream(st):
            x["Q"][:B].copy_(x["hQ"][:B], non_blocking=True)
            x["K"][:B].copy_(x["hK"][:B], non_blocking=True)
            zp.zp_respond(db.handle, [self.clients[r.client] for r in reqs], x["Q"].data_ptr(),
                          x["K"].data_ptr(), B, x["ans"].data_ptr(), x["T"].data_ptr(),
                          st.cuda_stream)
            x["hT"][:B].copy_(x["T"][:B], non_blocking=True)
            x["hA"][:B].copy_(x["ans"][:B], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return (ev, B, name, slot)

    def poll(self, handle):
        return handle[0].query()

    def finish(self, handle, reqs):
        ev, B, name, slot = handle
        ev.synchronize()
        x = self.d[name]["slots"][slot]
        hT, hA = x["hT"].numpy().view(np.uint32), x["hA"].numpy().view(np.uint32)
        for i, r in enumerate(reqs):
            r.T = hT[i].copy()
            r.ans = hA[i].copy()

    def idle(self, name):
        return all(sl["stream"].query() for sl in self.d[name]["slots"])

    def apply_updates(self, name, rows, new_rows):
        torch = self.torch
        x = self.d[name]
        db, st = x["db"], x["slots"][0]["stream"]
        with torch.cuda.stream(st):
            db.update_rows(rows, new_rows, stream=st)
            db.gen_hint(x["A"], rows=rows, stream=st)
        # the views' next batches must see the new rows: their streams wait for the update
        ev = torch.cuda.Event()
        ev.record(st)
        for sl in x["slots"][1:]:
            sl["stream"].wait_event(ev)

    def close(self):
        for x in self.d.values():
            for sl in x["slots"][1:]:
                sl["db"].close()
