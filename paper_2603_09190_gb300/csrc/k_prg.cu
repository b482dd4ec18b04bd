// k_prg.cu -- ChaCha20 keystream on the GPU (RFC 8439, Sec. 2.3: the block function), the
// PRG that expands the public matrix A and the clients' ck_r from 32-byte seeds (the paper
// names no PRG: Sec. 2.1.1 and Sec. 4.3 ask for a cryptographically secure one). One thread
// per 64-byte block: 20 rounds (10 column + diagonal double rounds) of the state
// constants | key | block counter | nonce, plus the initial state, written as 16 words.
#include "zp_internal.cuh"

namespace {

struct ChachaKey {
  uint32_t k[8];
  uint32_t n[3];
};

__device__ __forceinline__ uint32_t rotl32(uint32_t x, int r) { return __funnelshift_l(x, x, r); }

#define ZP_QR(a, b, c, d)      \
  a += b;                      \
  d = rotl32(d ^ a, 16);       \
  c += d;                      \
  b = rotl32(b ^ c, 12);       \
  a += b;                      \
  d = rotl32(d ^ a, 8);        \
  c += d;                      \
  b = rotl32(b ^ c, 7);

__global__ void __launch_bounds__(256) k_chacha20(ChachaKey key, uint32_t counter0,
                                                  uint32_t* __restrict__ out, uint64_t nwords) {
  const uint64_t blk = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blk * 16 >= nwords) return;
  const uint32_t init[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                             key.k[0], key.k[1], key.k[2], key.k[3], key.k[4], key.k[5],
                             key.k[6], key.k[7], counter0 + (uint32_t)blk, key.n[0], key.n[1],
                             key.n[2]};
  uint32_t x0 = init[0], x1 = init[1], x2 = init[2], x3 = init[3], x4 = init[4], x5 = init[5],
           x6 = init[6], x7 = init[7], x8 = init[8], x9 = init[9], x10 = init[10],
           x11 = init[11], x12 = init[12], x13 = init[13], x14 = init[14], x15 = init[15];
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    ZP_QR(x0, x4, x8, x12)
    ZP_QR(x1, x5, x9, x13)
    ZP_QR(x2, x6, x10, x14)
    ZP_QR(x3, x7, x11, x15)
    ZP_QR(x0, x5, x10, x15)
    ZP_QR(x1, x6, x11, x12)
    ZP_QR(x2, x7, x8, x13)
    ZP_QR(x3, x4, x9, x14)
  }
  const uint32_t w[16] = {x0 + init[0],   x1 + init[1],   x2 + init[2],   x3 + init[3],
                          x4 + init[4],   x5 + init[5],   x6 + init[6],   x7 + init[7],
                          x8 + init[8],   x9 + init[9],   x10 + init[10], x11 + init[11],
                          x12 + init[12], x13 + init[13], x14 + init[14], x15 + init[15]};
  uint32_t* dst = out + blk * 16;
  if (blk * 16 + 16 <= nwords && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      reinterpret_cast<uint4*>(dst)[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (blk * 16 + i < nwords) dst[i] = w[i];
  }
}
#undef ZP_QR

}  // namespace

extern "C" int zp_prg_chacha20(const uint8_t* hKey, const uint8_t* hNonce, uint32_t counter0,
                               uint32_t* dOut, uint64_t nwords, void* stream) {
  if (!hKey || !hNonce || (!dOut && nwords)) return zp_set_error(ZP_EINVAL, "zp_prg_chacha20: null argument");
  if (nwords == 0) return ZP_OK;
  const uint64_t blocks = (nwords + 15) / 16;
  if ((uint64_t)counter0 + blocks - 1 > 0xFFFFFFFFull)
    return zp_set_error(ZP_EINVAL, "zp_prg_chacha20: the 32-bit block counter would wrap");
  ChachaKey k;
  for (int i = 0; i < 8; ++i)
    k.k[i] = (uint32_t)hKey[4 * i] | ((uint32_t)hKey[4 * i + 1] << 8) |
             ((uint32_t)hKey[4 * i + 2] << 16) | ((uint32_t)hKey[4 * i + 3] << 24);
  for (int i = 0; i < 3; ++i)
    k.n[i] = (uint32_t)hNonce[4 * i] | ((uint32_t)hNonce[4 * i + 1] << 8) |
             ((uint32_t)hNonce[4 * i + 2] << 16) | ((uint32_t)hNonce[4 * i + 3] << 24);
  zp_clear_pending_error();
  k_chacha20<<<(unsigned)((blocks + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      k, counter0, dOut, nwords);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}
