"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side tests/bench.

This module holds no arithmetic of the ZipPIR method. It only draws random inputs
(database bytes, the public LWE matrix A, query vectors, compression-key offsets,
moduli for throughput runs) from seeded generators, and converts Python integers
to and from little-endian 32-bit limb arrays (pure marshalling).

Generators: numpy ``Generator(PCG64(seed))`` on the host, which gives identical
streams on x86 and Arm, and ``torch.Generator`` on a CUDA device for inputs too
large to draw on the host (GiB-sized databases). The paper leaves its PRG open
("a cryptographically secure PRG", Sec. 2.1.1 and Sec. 4.3); the choice here only
fixes reproducibility of synthetic inputs.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "database", "seed_matrix", "uniform_queries", "uniform_below",
    "random_odd_modulus", "ints_to_limbs", "limbs_to_ints", "device_database",
    "device_uniform_u32",
]


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Deterministic host generator for (seed, stream)."""
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def database(R: int, C: int, seed: int, p: int = 256, ld: int | None = None) -> np.ndarray:
    """R x C database of entries uniform in [0, p), dtype uint8, row-major.

    With ``ld`` (row pitch in bytes, >= C) the returned array is R x ld with the
    padding columns filled by 0xA5, a value no test may depend on.
    """
    g = rng(seed, 1)
    D = g.integers(0, p, size=(R, C), dtype=np.uint16).astype(np.uint8)
    if ld is None or ld == C:
        return D
    out = np.full((R, ld), 0xA5, dtype=np.uint8)
    out[:, :C] = D
    return out


def seed_matrix(C: int, n: int, seed: int) -> np.ndarray:
    """The public LWE matrix A, C x n, uniform u32 (expanded from a seed, Sec. 2.1.1)."""
    return rng(seed, 2).integers(0, 2**32, size=(C, n), dtype=np.uint64).astype(np.uint32)


def uniform_queries(B: int, C: int, seed: int) -> np.ndarray:
    """B x C uniform u32 query vectors (statistically identical to LWE queries)."""
    return rng(seed, 3).integers(0, 2**32, size=(B, C), dtype=np.uint64).astype(np.uint32)


def _uniform_bits(g: np.random.Generator, bits: int) -> int:
    words = (bits + 31) // 32
    w = g.integers(0, 2**32, size=words, dtype=np.uint64)
    v = 0
    for i in range(words - 1, -1, -1):
        v = (v << 32) | int(w[i])
    return v & ((1 << bits) - 1)


def uniform_below(bound: int, count: int, seed: int, stream: int = 4) -> list[int]:
    """``count`` integers uniform in [0, bound) (64 extra bits, then reduced)."""
    g = rng(seed, stream)
    nb = bound.bit_length() + 64
    return [_uniform_bits(g, nb) % bound for _ in range(count)]


def random_odd_modulus(bits: int, seed: int) -> int:
    """An odd integer of exactly ``bits`` bits.

    Throughput runs use it in place of a Paillier modulus: the server's work in
    the compression step does not depend on the factorisation of m.
    """
    g = rng(seed, 5)
    v = _uniform_bits(g, bits)
    return v | (1 << (bits - 1)) | 1


def ints_to_limbs(values, L: int) -> np.ndarray:
    """Python ints (each < 2^(32L)) -> array (len, L) of little-endian u32 limbs."""
    vals = list(values)
    out = np.zeros((len(vals), L), dtype=np.uint32)
    for r, v in enumerate(vals):
        v = int(v)
        if v < 0 or v.bit_length() > 32 * L:
            raise ValueError("value does not fit in %d limbs" % L)
        b = v.to_bytes(4 * L, "little")
        out[r] = np.frombuffer(b, dtype="<u4")
    return out


def limbs_to_ints(arr: np.ndarray) -> list[int]:
    """Array (..., L) of little-endian u32 limbs -> flat list of Python ints."""
    a = np.ascontiguousarray(arr, dtype="<u4").reshape(-1, arr.shape[-1])
    return [int.from_bytes(row.tobytes(), "little") for row in a]


def device_database(R: int, C: int, seed: int, device, ld: int | None = None, p: int = 256):
    """R x C uniform [0, p) uint8 database drawn directly on ``device`` (torch).

    Returns a tensor of shape (R, ld) whose first C columns are the database; the
    pitch columns are zero. Used for GiB-sized inputs.
    """
    import torch
    ld = C if ld is None else ld
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + 1)
    out = torch.empty((R, ld), dtype=torch.uint8, device=device)
    chunk = max(1, (1 << 28) // max(ld, 1))
    for r0 in range(0, R, chunk):
        r1 = min(R, r0 + chunk)
        blk = torch.randint(0, p, (r1 - r0, C), generator=g, device=device, dtype=torch.int32)
        out[r0:r1, :C] = blk.to(torch.uint8)
        if ld > C:
            out[r0:r1, C:] = 0
    return out


def device_uniform_u32(shape, seed: int, device):
    """Uniform u32 values drawn on ``device``, returned as an int32 tensor (bit pattern)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + 7)
    lo = torch.randint(0, 1 << 16, shape, generator=g, device=device, dtype=torch.int64)
    hi = torch.randint(0, 1 << 16, shape, generator=g, device=device, dtype=torch.int64)
    v = (hi << 16) | lo
    return (v - ((v >> 31) << 32)).to(torch.int32)
