// zp_chacha.cuh -- the ChaCha20 block function (RFC 8439, Sec. 2.3), the PRG that expands
// the public matrix A and the clients' ck_r from 32-byte seeds (the paper asks for a
// cryptographically secure PRG without naming one). Words are little-endian.
#pragma once

#include <stdint.h>

namespace {

struct ChachaKey {
  uint32_t k[8];  // the 32-byte key
  uint32_t n[3];  // the 12-byte nonce
};

__host__ __forceinline__ ChachaKey chacha_key_from_bytes(const uint8_t* key, const uint8_t* nonce) {
  ChachaKey c;
  for (int i = 0; i < 8; ++i)
    c.k[i] = (uint32_t)key[4 * i] | ((uint32_t)key[4 * i + 1] << 8) |
             ((uint32_t)key[4 * i + 2] << 16) | ((uint32_t)key[4 * i + 3] << 24);
  for (int i = 0; i < 3; ++i)
    c.n[i] = (uint32_t)nonce[4 * i] | ((uint32_t)nonce[4 * i + 1] << 8) |
             ((uint32_t)nonce[4 * i + 2] << 16) | ((uint32_t)nonce[4 * i + 3] << 24);
  return c;
}

__device__ __forceinline__ uint32_t chacha_rotl(uint32_t x, int r) { return __funnelshift_l(x, x, r); }

#define ZP_CHACHA_QR(a, b, c, d) \
  a += b;                        \
  d = chacha_rotl(d ^ a, 16);    \
  c += d;                        \
  b = chacha_rotl(b ^ c, 12);    \
  a += b;                        \
  d = chacha_rotl(d ^ a, 8);     \
  c += d;                        \
  b = chacha_rotl(b ^ c, 7);

// out = the 16 words of block `counter`: 20 rounds (10 column + diagonal double rounds) of
// the state constants | key | counter | nonce, plus the initial state.
__device__ __forceinline__ void chacha20_block(const ChachaKey& key, uint32_t counter,
                                               uint32_t (&out)[16]) {
  const uint32_t init[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                             key.k[0], key.k[1], key.k[2], key.k[3], key.k[4], key.k[5],
                             key.k[6], key.k[7], counter, key.n[0], key.n[1], key.n[2]};
  uint32_t x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = init[i];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    ZP_CHACHA_QR(x[0], x[4], x[8], x[12])
    ZP_CHACHA_QR(x[1], x[5], x[9], x[13])
    ZP_CHACHA_QR(x[2], x[6], x[10], x[14])
    ZP_CHACHA_QR(x[3], x[7], x[11], x[15])
    ZP_CHACHA_QR(x[0], x[5], x[10], x[15])
    ZP_CHACHA_QR(x[1], x[6], x[11], x[12])
    ZP_CHACHA_QR(x[2], x[7], x[8], x[13])
    ZP_CHACHA_QR(x[3], x[4], x[9], x[14])
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i] = x[i] + init[i];
}
#undef ZP_CHACHA_QR

}  // namespace
