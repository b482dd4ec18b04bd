// zp_warpint.cuh -- big integers spread over the 32 lanes of a warp: an integer of
// WPL*32 words is held with words [WPL*lane, WPL*lane + WPL) in lane (little-endian).
// Carries and borrows cross lanes in one step: the lanes that generate one (G) and the
// lanes that would pass one on (P) are ballots, and the carry into every lane is read off
// the single integer addition G + (G | P) (the carry-lookahead identity).
#pragma once

#include "zp_internal.cuh"

namespace {

// Adds per-word 64-bit column values v (each < 2^62) into normalized 32-bit words w.
template <int WPL>
__device__ __forceinline__ void warp_normalize(const uint64_t (&v)[WPL], uint32_t (&w)[WPL]) {
  const uint32_t lane = lane_id();
  uint64_t c = 0;
#pragma unroll
  for (int t = 0; t < WPL; ++t) {
    const uint64_t s = v[t] + c;
    w[t] = (uint32_t)s;
    c = s >> 32;
  }
  uint64_t cin = __shfl_up_sync(0xffffffffu, c, 1);
  if (lane == 0) cin = 0;
  uint32_t cc;
  {
    const uint64_t s = (uint64_t)w[0] + cin;
    w[0] = (uint32_t)s;
    cc = (uint32_t)(s >> 32);
  }
#pragma unroll
  for (int t = 1; t < WPL; ++t) {
    const uint64_t s = (uint64_t)w[t] + cc;
    w[t] = (uint32_t)s;
    cc = (uint32_t)(s >> 32);
  }
  uint32_t all = 0xFFFFFFFFu;
#pragma unroll
  for (int t = 0; t < WPL; ++t) all &= w[t];
  const uint32_t G = __ballot_sync(0xffffffffu, cc != 0);
  const uint32_t P = __ballot_sync(0xffffffffu, all == 0xFFFFFFFFu);
  const uint32_t K = (uint32_t)((uint64_t)G + (uint64_t)(G | P)) ^ P;  // carry into each lane
  if ((K >> lane) & 1u) {
    uint32_t c1 = 1;
#pragma unroll
    for (int t = 0; t < WPL; ++t) {
      const uint64_t s = (uint64_t)w[t] + c1;
      w[t] = (uint32_t)s;
      c1 = (uint32_t)(s >> 32);
    }
  }
}

// a -= b over the warp (mod 2^(32*32*WPL)).
template <int WPL>
__device__ __forceinline__ void warp_sub(uint32_t (&a)[WPL], const uint32_t (&b)[WPL]) {
  const uint32_t lane = lane_id();
  uint32_t br = 0;
#pragma unroll
  for (int t = 0; t < WPL; ++t) {
    const uint64_t s = (uint64_t)a[t] - b[t] - br;
    a[t] = (uint32_t)s;
    br = (uint32_t)(s >> 63);
  }
  uint32_t any = 0;
#pragma unroll
  for (int t = 0; t < WPL; ++t) any |= a[t];
  const uint32_t G = __ballot_sync(0xffffffffu, br != 0);
  const uint32_t P = __ballot_sync(0xffffffffu, any == 0);
  const uint32_t K = (uint32_t)((uint64_t)G + (uint64_t)(G | P)) ^ P;  // borrow into each lane
  if ((K >> lane) & 1u) {
    uint32_t b1 = 1;
#pragma unroll
    for (int t = 0; t < WPL; ++t) {
      const uint64_t s = (uint64_t)a[t] - b1;
      a[t] = (uint32_t)s;
      b1 = (uint32_t)(s >> 63);
    }
  }
}

// a >= b over the warp.
template <int WPL>
__device__ __forceinline__ bool warp_geq(const uint32_t (&a)[WPL], const uint32_t (&b)[WPL]) {
  int cmp = 0;
#pragma unroll
  for (int t = WPL - 1; t >= 0; --t)
    if (cmp == 0 && a[t] != b[t]) cmp = a[t] > b[t] ? 1 : -1;
  const uint32_t GT = __ballot_sync(0xffffffffu, cmp > 0);
  const uint32_t LT = __ballot_sync(0xffffffffu, cmp < 0);
  if ((GT | LT) == 0) return true;
  const int top = 31 - __clz(GT | LT);
  return (GT >> top) & 1u;
}

// As warp_normalize, and returns the carry out of the top word (the words above the
// WPL*32 held ones).
template <int WPL>
__device__ __forceinline__ uint32_t warp_normalize_top(const uint64_t (&v)[WPL], uint32_t (&w)[WPL]) {
  const uint32_t lane = lane_id();
  uint64_t c = 0;
#pragma unroll
  for (int t = 0; t < WPL; ++t) {
    const uint64_t s = v[t] + c;
    w[t] = (uint32_t)s;
    c = s >> 32;
  }
  const uint64_t c_top = __shfl_sync(0xffffffffu, c, 31);  // the top lane's carry leaves the warp
  uint64_t cin = __shfl_up_sync(0xffffffffu, c, 1);
  if (lane == 0) cin = 0;
  uint32_t cc;
  {
    const uint64_t s = (uint64_t)w[0] + cin;
    w[0] = (uint32_t)s;
    cc = (uint32_t)(s >> 32);
  }
#pragma unroll
  for (int t = 1; t < WPL; ++t) {
    const uint64_t s = (uint64_t)w[t] + cc;
    w[t] = (uint32_t)s;
    cc = (uint32_t)(s >> 32);
  }
  uint32_t all = 0xFFFFFFFFu;
#pragma unroll
  for (int t = 0; t < WPL; ++t) all &= w[t];
  const uint32_t G = __ballot_sync(0xffffffffu, cc != 0);
  const uint32_t P = __ballot_sync(0xffffffffu, all == 0xFFFFFFFFu);
  const uint64_t S = (uint64_t)G + (uint64_t)(G | P);
  const uint32_t K = (uint32_t)S ^ P;  // carry into each lane
  if ((K >> lane) & 1u) {
    uint32_t c1 = 1;
#pragma unroll
    for (int t = 0; t < WPL; ++t) {
      const uint64_t s = (uint64_t)w[t] + c1;
      w[t] = (uint32_t)s;
      c1 = (uint32_t)(s >> 32);
    }
  }
  return (uint32_t)c_top + (uint32_t)(S >> 32);
}

}  // namespace
