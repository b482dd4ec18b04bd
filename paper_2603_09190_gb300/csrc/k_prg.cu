// k_prg.cu -- ChaCha20 keystream on the GPU: one thread per 64-byte block.
#include "zp_chacha.cuh"
#include "zp_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) k_chacha20(ChachaKey key, uint32_t counter0,
                                                  uint32_t* __restrict__ out, uint64_t nwords) {
  const uint64_t blk = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blk * 16 >= nwords) return;
  uint32_t w[16];
  chacha20_block(key, counter0 + (uint32_t)blk, w);
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

}  // namespace

extern "C" int zp_prg_chacha20(const uint8_t* hKey, const uint8_t* hNonce, uint32_t counter0,
                               uint32_t* dOut, uint64_t nwords, void* stream) {
  if (!hKey || !hNonce || (!dOut && nwords)) return zp_set_error(ZP_EINVAL, "zp_prg_chacha20: null argument");
  if (nwords == 0) return ZP_OK;
  const uint64_t blocks = (nwords + 15) / 16;
  if ((uint64_t)counter0 + blocks - 1 > 0xFFFFFFFFull)
    return zp_set_error(ZP_EINVAL, "zp_prg_chacha20: the 32-bit block counter would wrap");
  const ChachaKey k = chacha_key_from_bytes(hKey, hNonce);
  zp_clear_pending_error();
  k_chacha20<<<(unsigned)((blocks + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      k, counter0, dOut, nwords);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}
