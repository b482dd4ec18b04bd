"""CPU checks of two arithmetic shortcuts the CUDA kernels take, restated here in Python
integers (no GPU, no oracle involvement):

* k_mod_packed reduces the residue-number-system sums V < 2^2087 mod a 2048-bit m with the
  quotient estimated from the top words alone, q_e = floor(V_t mu_t / 2^127) with V_t =
  floor(V / 2^1984), mu_t = floor(mu / 2^1985) and mu = floor(2^4096 / m) (the Barrett constant
  of Handbook of Applied Cryptography Alg. 14.42). The kernel needs q - 2 <= q_e <= q.
* k_crt_prep transposes bytes among groups of four lanes with two rounds of shuffles and
  byte permutations; the selectors must give lane 4 g + a the plane-a bytes of the group.
"""
import random

M64 = (1 << 64) - 1


def quotient_estimate(V: int, mu: int) -> int:
    w = [(V >> (32 * i)) & 0xFFFFFFFF for i in range(67)]
    u = [(mu >> (32 * i)) & 0xFFFFFFFF for i in range(66)]
    vh, vl = (w[65] << 32) | w[64], (w[63] << 32) | w[62]
    mut = ((u[64] << 63) | (u[63] << 31) | (u[62] >> 1)) & M64
    a1 = (vl * mut) >> 64
    b0, b1 = (vh * mut) & M64, (vh * mut) >> 64
    s1 = a1 + b0
    s2 = (b1 + (s1 >> 64)) & M64
    s1 &= M64
    return ((s2 << 1) | (s1 >> 63)) & M64


def test_quotient_estimate_bound():
    rnd = random.Random(2603)
    for it in range(20000):
        if it % 5 == 0:
            m = (1 << 2048) - 1 - 2 * rnd.getrandbits(20)        # near the top
        elif it % 7 == 0:
            m = (1 << 2047) + 1 + 2 * rnd.getrandbits(10)        # near the bottom
        else:
            m = (1 << 2047) | rnd.getrandbits(2047) | 1
        mu = (1 << 4096) // m
        top = rnd.choice([2087, 2086, 2080, 2048, 2047, 1000, 64])
        V = (1 << 2087) - 1 if it % 11 == 0 else rnd.getrandbits(top)
        q, qe = V // m, quotient_estimate(V, mu)
        assert q - 2 <= qe <= q
        assert qe < 1 << 40


def byte_perm(x: int, y: int, s: int) -> int:
    """The CUDA __byte_perm selector semantics: bytes 0-3 from x, 4-7 from y."""
    b = [(x >> (8 * i)) & 255 for i in range(4)] + [(y >> (8 * i)) & 255 for i in range(4)]
    return sum(b[(s >> (4 * n)) & 7] << (8 * n) for n in range(4))


def test_byte_transpose_selectors():
    rnd = random.Random(9190)
    for _ in range(200):
        x = [rnd.getrandbits(32) for _ in range(32)]
        w1 = [byte_perm(x[l], x[l ^ 1], 0x3715) if l & 1 else byte_perm(x[l], x[l ^ 1], 0x6240)
              for l in range(32)]
        w2 = [byte_perm(w1[l ^ 2], w1[l], 0x7632) if l & 2 else byte_perm(w1[l], w1[l ^ 2], 0x5410)
              for l in range(32)]
        for l in range(32):
            a, g = l & 3, l >> 2
            assert w2[l] == sum(((x[4 * g + i] >> (8 * a)) & 255) << (8 * i) for i in range(4))
