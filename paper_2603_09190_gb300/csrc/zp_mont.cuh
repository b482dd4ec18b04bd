// zp_mont.cuh -- Montgomery products modulo an odd N of 32 WPL words held by one warp
// (words [WPL lane, WPL lane + WPL) in lane): N = m^2 of a Paillier key of 16 WPL words,
// so WPL = 4 for 2048-bit keys and 6 for 3072-bit keys.
//
// r = a b 2^(-1024 WPL) mod N (Montgomery, Math. Comp. 1985) in the coarsely integrated
// operand scanning form (CIOS; Koc, Acar, Kaliski, IEEE Micro 1996). Each of the 32 WPL
// steps adds a_i b and u N (u = t_0 (-N)^{-1} mod 2^32, which zeroes word 0) and shifts
// the sum down one word; the word sums stay lazily unnormalised in 64-bit lane
// accumulators (below 2^42 for WPL <= 8), so a step needs no carry chain across lanes:
// three shuffles (a_i, u, the shifted word). One normalisation and one conditional
// subtraction of N at the end give the result below N.
#pragma once

#include "zp_warpint.cuh"

namespace {

template <int WPL>
struct ModN {
  uint32_t n[WPL];  // this lane's words of N
  uint32_t ninv;    // -N^{-1} mod 2^32
};

// src 16-byte aligned (WPL = 4) or 8-byte aligned (WPL = 6)
template <int WPL>
__device__ __forceinline__ void load_lane_words(const uint32_t* __restrict__ src, uint32_t (&w)[WPL]) {
  if constexpr (WPL % 4 == 0) {
#pragma unroll
    for (int q = 0; q < WPL / 4; ++q) {
      const uint4 v = reinterpret_cast<const uint4*>(src + WPL * lane_id())[q];
      w[4 * q] = v.x;
      w[4 * q + 1] = v.y;
      w[4 * q + 2] = v.z;
      w[4 * q + 3] = v.w;
    }
  } else {
    static_assert(WPL % 2 == 0, "WPL must be even");
#pragma unroll
    for (int q = 0; q < WPL / 2; ++q) {
      const uint2 v = reinterpret_cast<const uint2*>(src + WPL * lane_id())[q];
      w[2 * q] = v.x;
      w[2 * q + 1] = v.y;
    }
  }
}

template <int WPL>
__device__ __forceinline__ void store_lane_words(uint32_t* __restrict__ dst, const uint32_t (&w)[WPL]) {
  if constexpr (WPL % 4 == 0) {
#pragma unroll
    for (int q = 0; q < WPL / 4; ++q)
      reinterpret_cast<uint4*>(dst + WPL * lane_id())[q] =
          make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < WPL / 2; ++q)
      reinterpret_cast<uint2*>(dst + WPL * lane_id())[q] = make_uint2(w[2 * q], w[2 * q + 1]);
  }
}

template <int WPL>
__device__ __forceinline__ ModN<WPL> load_modn(const uint32_t* __restrict__ n, uint32_t ninv) {
  ModN<WPL> M;
  load_lane_words<WPL>(n, M.n);
  M.ninv = ninv;
  return M;
}

// r = a b 2^(-1024 WPL) mod N, for a < 2^(1024 WPL) and b < N (r may alias a or b).
template <int WPL>
__device__ __forceinline__ void mont_mul(const ModN<WPL>& M, const uint32_t (&a)[WPL],
                                         const uint32_t (&b)[WPL], uint32_t (&r)[WPL]) {
  const uint32_t lane = lane_id();
  uint64_t acc[WPL];
#pragma unroll
  for (int k = 0; k < WPL; ++k) acc[k] = 0;
#pragma unroll 1
  for (int src = 0; src < 32; ++src) {
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
      const uint32_t ai = __shfl_sync(0xffffffffu, a[s], src);  // word WPL src + s of a
      uint32_t ph[WPL];
#pragma unroll
      for (int k = 0; k < WPL; ++k) {
        const uint64_t p = (uint64_t)ai * b[k];
        acc[k] += (uint32_t)p;
        ph[k] = (uint32_t)(p >> 32);
      }
#pragma unroll
      for (int k = 1; k < WPL; ++k) acc[k] += ph[k - 1];
      // u makes word 0 vanish mod 2^32 (word 0 lives in lane 0)
      const uint32_t u = __shfl_sync(0xffffffffu, (uint32_t)acc[0] * M.ninv, 0);
      uint32_t qh[WPL];
#pragma unroll
      for (int k = 0; k < WPL; ++k) {
        const uint64_t q = (uint64_t)u * M.n[k];
        acc[k] += (uint32_t)q;
        qh[k] = (uint32_t)(q >> 32);
      }
#pragma unroll
      for (int k = 1; k < WPL; ++k) acc[k] += qh[k - 1];
      // divide by 2^32: every word moves down one place; word 0 keeps only its carry
      const uint64_t from_next = __shfl_down_sync(0xffffffffu, acc[0], 1);
      const uint64_t c0 = lane == 0 ? (acc[0] >> 32) : 0ull;
      acc[0] = acc[1] + c0;
#pragma unroll
      for (int k = 1; k < WPL - 1; ++k) acc[k] = acc[k + 1];
      // the high halves of the top words belong to the next lane's word 0, which is now
      // this lane's top word
      acc[WPL - 1] = (lane == 31 ? 0ull : from_next) + ph[WPL - 1] + qh[WPL - 1];
    }
  }
  uint32_t w[WPL];
  const uint32_t top = warp_normalize_top<WPL>(acc, w);  // the sum is below 2 N
  if (top != 0 || warp_geq<WPL>(w, M.n)) warp_sub<WPL>(w, M.n);
#pragma unroll
  for (int k = 0; k < WPL; ++k) r[k] = w[k];
}

// x <- x^e (Montgomery form) by left-to-right square-and-multiply; e = the ew words of
// e_words (warp-uniform), e > 0.
template <int WPL>
__device__ __forceinline__ void mont_pow_words(const ModN<WPL>& M, uint32_t (&x)[WPL],
                                               const uint32_t* e_words, int ew) {
  int top = -1;
  for (int w = ew - 1; w >= 0 && top < 0; --w)
    if (e_words[w]) top = 32 * w + 31 - __clz(e_words[w]);
  uint32_t y[WPL];
#pragma unroll
  for (int k = 0; k < WPL; ++k) y[k] = x[k];
  for (int bit = top - 1; bit >= 0; --bit) {
    mont_mul<WPL>(M, y, y, y);
    if ((e_words[bit >> 5] >> (bit & 31)) & 1u) mont_mul<WPL>(M, y, x, y);
  }
#pragma unroll
  for (int k = 0; k < WPL; ++k) x[k] = y[k];
}

}  // namespace
