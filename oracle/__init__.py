"""Oracle for the ZipPIR online server phase (arXiv 2603.09190).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct CPU
implementation of what the server computes and of the client around it. It may
be imported only by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU
baseline leg of ``bench.py``. The CUDA library and its Python binding never
import, link or call it, and it shares no code with them: integers are exact
(numpy uint64 with explicit reduction mod 2^32, Python ints for Paillier), and
every function cites the part of the paper it follows.

Modules:
  params   -- scheme parameters: q, p, Delta, the packing scale gamma, slots ell
  lwe      -- ans = D.q mod 2^32 and the global hint H = D.A mod 2^32
  paillier -- key generation, Enc/Dec, homomorphic add / plaintext multiply
  zippir   -- packing, the server Response (ans, t) and the client
              Setup / Query / Extract, PaillierMatMul for the per-client hint

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (brute force, closed forms, library primes, the
correctness theorem, the proof identity). Nothing is "parity unpinned".
"""
from . import params, lwe, paillier, zippir  # noqa: F401
