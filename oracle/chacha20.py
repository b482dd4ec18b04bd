"""ChaCha20 keystream (RFC 8439, Sec. 2.3: the block function), oracle / test
infrastructure only.

The paper expands the public matrix A and the clients' random ck_r from short seeds with
a secure PRG that it does not name (Sec. 2.1.1, Sec. 4.3); ChaCha20 is the reading
taken. Plain Python integers, one block at a time.
"""
from __future__ import annotations

MASK = 0xFFFFFFFF
SIGMA = (0x61707865, 0x3320646E, 0x79622D32, 0x6B206574)  # "expand 32-byte k"


def _rotl(x: int, r: int) -> int:
    return ((x << r) | (x >> (32 - r))) & MASK


def _quarter(s: list[int], a: int, b: int, c: int, d: int) -> None:
    s[a] = (s[a] + s[b]) & MASK
    s[d] = _rotl(s[d] ^ s[a], 16)
    s[c] = (s[c] + s[d]) & MASK
    s[b] = _rotl(s[b] ^ s[c], 12)
    s[a] = (s[a] + s[b]) & MASK
    s[d] = _rotl(s[d] ^ s[a], 8)
    s[c] = (s[c] + s[d]) & MASK
    s[b] = _rotl(s[b] ^ s[c], 7)


def block(key: bytes, counter: int, nonce: bytes) -> list[int]:
    """The 16 output words of the block function for a 32-byte key, a 32-bit block
    counter and a 12-byte nonce: 20 rounds (10 column + diagonal double rounds) of the
    state constants | key | counter | nonce, plus the initial state."""
    assert len(key) == 32 and len(nonce) == 12 and 0 <= counter <= MASK
    k = [int.from_bytes(key[4 * i:4 * i + 4], "little") for i in range(8)]
    nw = [int.from_bytes(nonce[4 * i:4 * i + 4], "little") for i in range(3)]
    init = list(SIGMA) + k + [counter] + nw
    s = list(init)
    for _ in range(10):
        _quarter(s, 0, 4, 8, 12)
        _quarter(s, 1, 5, 9, 13)
        _quarter(s, 2, 6, 10, 14)
        _quarter(s, 3, 7, 11, 15)
        _quarter(s, 0, 5, 10, 15)
        _quarter(s, 1, 6, 11, 12)
        _quarter(s, 2, 7, 8, 13)
        _quarter(s, 3, 4, 9, 14)
    return [(s[i] + init[i]) & MASK for i in range(16)]


def keystream_words(key: bytes, nonce: bytes, counter0: int, nwords: int) -> list[int]:
    """nwords 32-bit words of keystream: the words of blocks counter0, counter0 + 1, ..."""
    out: list[int] = []
    c = counter0
    while len(out) < nwords:
        out.extend(block(key, c, nonce))
        c += 1
    return out[:nwords]
