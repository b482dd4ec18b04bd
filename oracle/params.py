"""Scheme parameters (oracle; test infrastructure only).

Sec. 2.1.1 (LWE): ciphertext modulus q, plaintext modulus p, Delta = round(q/p).
Sec. 3.3 (Algorithm "Batch Compression", its caption and correctness theorem):
the packing scale gamma must bound every slot value; with a uniform secret in
Z_q the slot value b + sum_i (q - a_i) sk_i is below q + n q^2, with a binary
secret below q + n q (Sec. 3.3.3). The theorem needs m > gamma^ell.

Reading taken where the paper is loose (Sec. 4.4 gives ell through a ceiling
formula with the smaller, overlap scale): ell is the largest integer with
gamma^ell < 2^(key_bits - 1). Every key of ``key_bits`` bits has
m >= 2^(key_bits - 1), so the theorem's m > gamma^ell holds for all clients with
keys of that size and the packed hint is the same for all of them.

Overlap scale (Sec. 3.3.3, "Better compression with a smaller scale"; its proof is
not in the paper): gamma = q^2 (uniform secret) or q (binary), so that neighbouring
slots overlap; the slot values still lie below the proven bound gamma_p = q + n q^2
(or q + n q). Reading: ell is the largest integer with
(gamma_p - 1) sum_{j<ell} gamma^j < 2^(key_bits - 1), the largest packed value, which
for gamma = gamma_p is the rule above. Recovery then needs the noise plus the spill of
the slot below (at most about n) to stay under Delta / 2; checked by end-to-end recovery.
"""
from __future__ import annotations

from dataclasses import dataclass

Q_BITS = 32
Q = 1 << Q_BITS


@dataclass(frozen=True)
class Params:
    n: int = 1024            # LWE dimension
    key_bits: int = 2048     # Paillier modulus size (bits of m)
    secret: str = "uniform"  # "uniform" (sk in Z_q^n) or "binary" (sk in {0,1}^n)
    p: int = 256             # plaintext modulus (database entries in Z_p)
    sigma: float = 6.4       # error standard deviation (Sec. 5.2)
    scale: str = "proven"    # "proven" (gamma = slot bound) or "overlap" (Sec. 3.3.3)

    @property
    def q(self) -> int:
        return Q

    @property
    def delta(self) -> int:
        # Delta = round(q / p), Sec. 2.1.1
        return (Q + self.p // 2) // self.p

    @property
    def slot_bound(self) -> int:
        # every slot value is below q + n q^2 (uniform secret, Sec. 3.3) or q + n q (binary,
        # Sec. 3.3.3)
        if self.secret == "uniform":
            return Q + self.n * Q * Q
        if self.secret == "binary":
            return Q + self.n * Q
        raise ValueError("secret must be 'uniform' or 'binary'")

    @property
    def gamma(self) -> int:
        if self.scale == "proven":
            return self.slot_bound
        if self.scale == "overlap":
            return Q * Q if self.secret == "uniform" else Q
        raise ValueError("scale must be 'proven' or 'overlap'")

    @property
    def ell(self) -> int:
        # largest ell whose largest packed value (slot_bound - 1) sum_{j<ell} gamma^j is
        # below 2^(key_bits-1); for the proven scale: gamma^ell < 2^(key_bits-1) (batched
        # correctness theorem, Sec. 3.3)
        g, top = self.gamma, self.slot_bound - 1
        bound = 1 << (self.key_bits - 1)
        ell, acc = 0, 0
        while top * (acc + g ** ell) < bound:
            acc += g ** ell
            ell += 1
        if ell == 0:
            raise ValueError("key too small for one slot")
        return ell

    def d1p(self, R: int) -> int:
        # number of packed rows: ceil(R / ell); the last one is zero-padded
        return -(-R // self.ell)
