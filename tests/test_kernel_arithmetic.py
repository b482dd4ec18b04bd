"""CPU checks of arithmetic shortcuts the CUDA kernels take, restated here in Python
integers (no GPU; the packing parameters come from oracle.params):

* k_mod_packed reduces the residue-number-system sums V < 2^2087 mod a 2048-bit m with the
  quotient estimated from the top words alone, q_e = floor(V_t mu_t / 2^127) with V_t =
  floor(V / 2^1984), mu_t = floor(mu / 2^1985) and mu = floor(2^4096 / m) (the Barrett constant
  of Handbook of Applied Cryptography Alg. 14.42). The kernel needs q - 2 <= q_e <= q.
* k_crt_prep transposes bytes among groups of four lanes with two rounds of shuffles and
  byte permutations; the selectors must give lane 4 g + a the plane-a bytes of the group.
* k_gemm_tc<CRT> sums the base-256 digits of V with the byte planes along K and the
  constants' rows shifted per plane, then undoes the centring per valid (plane, digit).
* k_pack_ans gathers b' = sum_j ans_j gamma^j from per-lane 96-bit column sums and adds Y
  with one conditional subtraction of m.
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


def _crt_epilogue_words(A, B, Kp):
    """The CRT product as k_gemm_tc<CRT> computes it: centred bytes (value - 128; padding
    bytes zero), plane a of A against the B rows shifted by a (rows outside 0..255 read as a
    centred zero), fp32-exact digit sums S_t; then per word the row term (128 x the plane
    row sums of the valid planes), the column term (128 colsum[t - a] - 16384 Kp per valid
    plane) and one carry chain over two halves of 144 columns (words 0..35, then 36..67)."""
    import numpy as np
    KC = A.shape[1]
    Ap = np.full((4, Kp), -128, np.int64)
    Ap[:, :KC] = A - 128
    Bp = np.full((Kp, 256), -128, np.int64)
    Bp[:KC] = B - 128
    S = np.zeros(288, np.int64)
    for a in range(4):
        Bs = np.zeros((Kp, 288), np.int64)
        Bs[:, a:a + 256] = Bp
        S += Ap[a] @ Bs
    assert np.abs(S).max() <= 1 << 24                      # exact in the fp32 accumulator
    rs, cs = [int(x) for x in A.sum(1)], [int(x) for x in B.sum(0)]
    r4 = 128 * sum(rs)
    rw_lo = 128 * (rs[0] + ((rs[0] + rs[1]) << 8) + ((rs[0] + rs[1] + rs[2]) << 16)) + (r4 << 24)
    rw_hi = 128 * ((rs[1] + rs[2] + rs[3]) + ((rs[2] + rs[3]) << 8) + (rs[3] << 16))
    words, carry = [], 0
    for hh in range(2):
        for wi in range(36 if hh == 0 else 32):
            w = 36 * hh + wi
            cw = 0
            for j in range(4):
                t = 4 * w + j
                cw += sum(128 * cs[t - a] - 16384 * Kp for a in range(4) if 0 <= t - a < 256) << (8 * j)
            sv = carry + cw + (rw_lo if w == 0 else (r4 * 0x01010101 if w < 64 else (rw_hi if w == 64 else 0)))
            for j in range(4):
                sv += int(S[144 * hh + 4 * wi + j]) << (8 * j)
            assert 0 <= sv < 1 << 62
            words.append(sv & 0xFFFFFFFF)
            carry = sv >> 32
    assert carry == 0 and words[67] == 0
    return sum(x << (32 * i) for i, x in enumerate(words[:67]))


def test_crt_product_epilogue_model():
    """The digit sums with the planes along K and the centring terms give V = sum_a 2^(8a)
    (plane a of A) . (the 256-byte constants of B) exactly, for K = 181 (ell = 27, planes
    padded to 192) and 208 (ell = 54, padded to 256), random and extreme bytes."""
    import numpy as np
    rng = np.random.default_rng(2603)
    for KC, Kp in ((181, 192), (208, 256)):
        for kind in ("random", "max", "zero"):
            if kind == "random":
                A, B = rng.integers(0, 256, (4, KC)), rng.integers(0, 256, (KC, 256))
            elif kind == "max":
                A, B = np.full((4, KC), 255), np.full((KC, 256), 255)
            else:
                A, B = np.zeros((4, KC), np.int64), np.zeros((KC, 256), np.int64)
            consts = [sum(int(B[k, c]) << (8 * c) for c in range(256)) for k in range(KC)]
            want = sum(sum(int(A[a, k]) * consts[k] for k in range(KC)) << (8 * a) for a in range(4))
            assert _crt_epilogue_words(A, B, Kp) == want


def _pack_ans_model(ans, gam, Y, m):
    """k_pack_ans: lane l sums columns 2l and 2l + 1 of sum_j ans_j gamma^j as 96-bit
    (lo, mid, hi); word 2l = lo(2l) + mid(2l - 1) + hi(2l - 2), word 2l + 1 = lo(2l + 1) +
    mid(2l) + hi(2l - 1); Y added; carry out of word 63 or w >= m: subtract m mod 2^2048."""
    M32 = (1 << 32) - 1
    col = [sum(a * ((g >> (32 * w)) & M32) for a, g in zip(ans, gam)) for w in range(64)]
    assert all(c < 1 << 96 for c in col)
    assert (col[63] >> 32) == 0 and (col[62] >> 64) == 0   # lane 31's dropped parts
    lo = [c & M32 for c in col]
    mid = [(c >> 32) & M32 for c in col]
    hi = [c >> 64 for c in col]
    v = [lo[w] + (mid[w - 1] if w >= 1 else 0) + (hi[w - 2] if w >= 2 else 0) + ((Y >> (32 * w)) & M32)
         for w in range(64)]
    X = sum(x << (32 * i) for i, x in enumerate(v))
    w, top = X & ((1 << 2048) - 1), X >> 2048
    if top or w >= m:
        w = (w - m) % (1 << 2048)
    return w


def test_pack_answers_model():
    """(b' + Y) mod m for both secrets' gamma and ell (ell = 27 and 54), ragged last packed
    rows, all-ones answers and Y = m - 1: b' < m by the choice of ell, so one subtraction."""
    from oracle.params import Params
    rnd = random.Random(48)
    for secret, n in (("uniform", 1024), ("binary", 48)):
        P = Params(n=n, key_bits=2048, secret=secret)
        for it in range(60):
            m = (1 << 2047) | rnd.getrandbits(2047) | 1
            nrows = P.ell if it % 4 else rnd.randint(1, P.ell)
            ans = [rnd.getrandbits(32) if it % 3 else (1 << 32) - 1 for _ in range(nrows)]
            gam = [P.gamma ** j for j in range(nrows)]
            Y = rnd.randrange(m) if it % 5 else m - 1
            bp = sum(a * g for a, g in zip(ans, gam))
            assert bp < m
            assert _pack_ans_model(ans, gam, Y, m) == (bp + Y) % m
