// zp_bigint_host.h -- small host-side multi-precision helpers (little-endian 32-bit words)
// for the constants of the Montgomery arithmetic and the bounds checked before launches.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace zp_host {

using Big = std::vector<uint32_t>;

inline void trim(Big& a) {
  while (a.size() > 1 && a.back() == 0) a.pop_back();
}

inline Big from_u64(uint64_t v) {
  Big r{(uint32_t)v, (uint32_t)(v >> 32)};
  trim(r);
  return r;
}

inline uint32_t bits(const Big& a) {
  for (size_t i = a.size(); i-- > 0;)
    if (a[i]) return (uint32_t)(32 * i + 32 - __builtin_clz(a[i]));
  return 0;
}

// schoolbook product
inline Big mul(const Big& a, const Big& b) {
  Big r(a.size() + b.size(), 0);
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); ++j) {
      const uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    r[i + b.size()] = (uint32_t)carry;
  }
  trim(r);
  return r;
}

inline Big add(const Big& a, const Big& b) {
  Big r(std::max(a.size(), b.size()) + 1, 0);
  uint64_t c = 0;
  for (size_t i = 0; i < r.size(); ++i) {
    c += (uint64_t)(i < a.size() ? a[i] : 0) + (i < b.size() ? b[i] : 0);
    r[i] = (uint32_t)c;
    c >>= 32;
  }
  trim(r);
  return r;
}

// -1, 0, 1 for a < b, a == b, a > b
inline int cmp(const Big& a, const Big& b) {
  const size_t n = std::max(a.size(), b.size());
  for (size_t i = n; i-- > 0;) {
    const uint32_t x = i < a.size() ? a[i] : 0, y = i < b.size() ? b[i] : 0;
    if (x != y) return x < y ? -1 : 1;
  }
  return 0;
}

// 2^k mod N (N has nw words, N odd > 1) by doubling with a conditional subtraction
inline Big pow2_mod(uint32_t k, const Big& N) {
  const size_t nw = N.size();
  Big r(nw + 1, 0);
  r[0] = 1;
  for (uint32_t it = 0; it < k; ++it) {
    uint32_t carry = 0;
    for (size_t w = 0; w <= nw; ++w) {
      const uint32_t nc = r[w] >> 31;
      r[w] = (r[w] << 1) | carry;
      carry = nc;
    }
    bool ge = true;
    for (size_t w = nw + 1; w-- > 0;) {
      const uint32_t mw = w < nw ? N[w] : 0u;
      if (r[w] != mw) {
        ge = r[w] > mw;
        break;
      }
    }
    if (ge) {
      uint64_t br = 0;
      for (size_t w = 0; w <= nw; ++w) {
        const uint64_t s = (uint64_t)r[w] - (w < nw ? N[w] : 0u) - br;
        r[w] = (uint32_t)s;
        br = (s >> 63) & 1u;
      }
    }
  }
  r.resize(nw);
  return r;
}

// -(n0)^{-1} mod 2^32 for odd n0 (Newton's iteration doubles the correct bits)
inline uint32_t neg_inv32(uint32_t n0) {
  uint32_t inv = n0;
  for (int it = 0; it < 5; ++it) inv *= 2u - n0 * inv;
  return 0u - inv;
}

}  // namespace zp_host
