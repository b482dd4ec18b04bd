"""Paillier cryptosystem over Python ints (oracle; test infrastructure only).

Sec. 2.1.2: plaintexts in Z_m, m = P1 * P2, ciphertexts in Z_{m^2}; addition of
plaintexts is ciphertext multiplication, multiplication by a plaintext is
exponentiation. The paper does not fix the variant; this uses g = m + 1 and
lambda = lcm(P1 - 1, P2 - 1), mu = lambda^{-1} mod m (textbook Paillier, 1999).
Any valid variant decrypts to the same plaintexts, which is all the protocol uses.

Key generation: two primes of key_bits/2 bits with the top two bits set, so that
m has exactly key_bits bits; primality by Miller-Rabin with bases drawn from the
seeded generator.
"""
from __future__ import annotations

from dataclasses import dataclass
from math import gcd

import numpy as np

_SMALL_PRIMES = [p for p in range(3, 2000) if all(p % d for d in range(2, int(p ** 0.5) + 1))]


def _rand_bits(g: np.random.Generator, bits: int) -> int:
    words = (bits + 31) // 32
    w = g.integers(0, 2**32, size=words, dtype=np.uint64)
    v = 0
    for x in w[::-1]:
        v = (v << 32) | int(x)
    return v & ((1 << bits) - 1)


def is_probable_prime(nv: int, g: np.random.Generator, rounds: int = 40) -> bool:
    """Miller-Rabin with ``rounds`` random bases."""
    if nv < 2:
        return False
    if nv in (2, 3):
        return True
    if nv % 2 == 0:
        return False
    for sp in _SMALL_PRIMES:
        if nv == sp:
            return True
        if nv % sp == 0:
            return False
    d, s = nv - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for _ in range(rounds):
        a = 2 + _rand_bits(g, nv.bit_length() + 32) % (nv - 3)
        x = pow(a, d, nv)
        if x in (1, nv - 1):
            continue
        for _ in range(s - 1):
            x = x * x % nv
            if x == nv - 1:
                break
        else:
            return False
    return True


def gen_prime(bits: int, g: np.random.Generator) -> int:
    """Random prime of exactly ``bits`` bits with its two top bits set."""
    while True:
        c = _rand_bits(g, bits) | (3 << (bits - 2)) | 1
        if is_probable_prime(c, g):
            return c


@dataclass(frozen=True)
class PublicKey:
    m: int

    @property
    def m2(self) -> int:
        return self.m * self.m


@dataclass(frozen=True)
class SecretKey:
    m: int
    lam: int
    mu: int
    p1: int = 0
    p2: int = 0


def keygen(key_bits: int, seed: int) -> tuple[PublicKey, SecretKey]:
    """Paillier key pair with an m of exactly ``key_bits`` bits (Algorithm "ZipPIR", Setup)."""
    g = np.random.Generator(np.random.PCG64([int(seed), 101]))
    half = key_bits // 2
    while True:
        P1 = gen_prime(half, g)
        P2 = gen_prime(key_bits - half, g)
        if P1 == P2:
            continue
        m = P1 * P2
        if m.bit_length() != key_bits or gcd(m, (P1 - 1) * (P2 - 1)) != 1:
            continue
        lam = (P1 - 1) * (P2 - 1) // gcd(P1 - 1, P2 - 1)
        mu = pow(lam, -1, m)
        return PublicKey(m), SecretKey(m, lam, mu, P1, P2)


def encrypt(pk: PublicKey, x: int, r: int) -> int:
    """Enc(x; r) = g^x r^m mod m^2 with g = m + 1, so g^x = 1 + x m mod m^2."""
    m, m2 = pk.m, pk.m2
    return (1 + (x % m) * m) * pow(r, m, m2) % m2


def decrypt(sk: SecretKey, c: int) -> int:
    """Dec(c) = L(c^lambda mod m^2) mu mod m, with L(u) = (u - 1) / m."""
    m, m2 = sk.m, sk.m * sk.m
    u = pow(c, sk.lam, m2)
    return (u - 1) // m * sk.mu % m


def add(pk: PublicKey, c1: int, c2: int) -> int:
    """Homomorphic addition (the paper's circled plus): c1 c2 mod m^2."""
    return c1 * c2 % pk.m2


def smul(pk: PublicKey, a: int, c: int) -> int:
    """Plaintext multiplication (the paper's circled times): c^a mod m^2."""
    return pow(c, a, pk.m2)
