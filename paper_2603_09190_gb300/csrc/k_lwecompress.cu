// k_lwecompress.cu -- compression of LWE ciphertexts (and extracted RLWE coefficients) into
// Paillier ciphertexts on the GPU (Sec. 3; App. B; the packed-key appendix), for 2048- and
// 3072-bit keys.
//
// With ck[i] = Enc(s[i]) and g = m + 1, LWECompress gives
//     x = (1 + b m) prod_i ck[i]^{(q - a[i]) mod q}  mod m^2,
// and batched compression of ell ciphertexts x = prod_j x_j^{gamma^j}. Both are computed as
//     x = (1 + b' m) prod_i ck[i]^{E_i}  mod m^2,
//     E_i = sum_j gamma^j ((q - a_j[i]) mod q),  b' = sum_j gamma^j b_j,
// the same element of Z*_{m^2} ((1 + b m)^{gamma^j} = 1 + gamma^j b m mod m^2), either
//  * folded: E_i and b' as above, one exponent of up to key_bits bits per base, or
//  * Horner: every x_j with its own exponents (< q), then X <- X^gamma x_j per group,
//    which does less work but has a sequential chain of ell |gamma| squarings per group.
// The exponentiations use the expanded key eck[i][k] = ck[i]^{2^k} (Montgomery form,
// Algorithm "Batch compression ... using precomputed powers"): the product over the set
// bits of E_i of eck[i][k]. Work items are (group, base, chunk of exponent words), one warp
// each; their partial products are multiplied pairwise, one level per launch, and the
// group's factor 1 + b' m is applied last.
#include "zp_bigint_host.h"
#include "zp_internal.cuh"
#include "zp_mont.cuh"

struct zp_lc {
  int device;
  uint32_t key_bits, L;  // m has L words, m^2 has 2L
  uint32_t ninv;
  uint32_t *d_m, *d_m2, *d_r1, *d_r2;
  std::vector<uint32_t> h_m;
  // expanded key
  uint32_t n, T;
  uint32_t* d_eck;  // n x T x 2L words
  zp_scratch s_e, s_pa, s_pb, s_x, s_k;
};

namespace {

constexpr int LC_EW_MAX = 98;  // exponent words (key_bits / 32 + 2)

template <int WPL>
struct LcConsts {
  const uint32_t* m2;
  const uint32_t* r1;
  const uint32_t* r2;
  const uint32_t* m;
  uint32_t ninv;
};

template <int WPL>
__device__ __forceinline__ ModN<WPL> lc_mod(const LcConsts<WPL>& c) {
  return load_modn<WPL>(c.m2, c.ninv);
}

struct SmallWords {
  uint32_t w[8];
};

// eck[i][k] = ck[i]^{2^k} R mod m^2 for k < T: one warp per base.
template <int WPL>
__global__ void __launch_bounds__(128) k_lc_square_chain(const uint32_t* __restrict__ ck, uint32_t n,
                                                         uint32_t T, LcConsts<WPL> c,
                                                         uint32_t* __restrict__ eck) {
  constexpr int MW = 32 * WPL;
  const uint32_t i = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (i >= n) return;
  const ModN<WPL> M = lc_mod(c);
  uint32_t x[WPL], r2[WPL];
  load_lane_words<WPL>(ck + (uint64_t)i * MW, x);
  load_lane_words<WPL>(c.r2, r2);
  mont_mul<WPL>(M, x, r2, x);
  uint32_t* dst = eck + (uint64_t)i * T * MW;
  store_lane_words<WPL>(dst, x);
  for (uint32_t k = 1; k < T; ++k) {
    mont_mul<WPL>(M, x, x, x);
    store_lane_words<WPL>(dst + (uint64_t)k * MW, x);
  }
}

// Exponents: one thread per (group g, column i <= n). Column i < n gets
// E = sum_j gamma^j ((q - a_j[i]) mod q), column n gets b' = sum_j gamma^j b_j, over the
// ciphertexts j < ell_g of the group (Horner: E <- E gamma + e_j). q = 0 stands for 2^64.
__global__ void __launch_bounds__(128) k_lc_exponents(const uint64_t* __restrict__ A,
                                                      const uint64_t* __restrict__ B, uint32_t count,
                                                      uint32_t n, uint64_t q, uint32_t ell,
                                                      SmallWords gam, uint32_t gw, uint32_t EW,
                                                      uint32_t* __restrict__ E) {
  const uint32_t G = (count + ell - 1) / ell;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (uint64_t)G * (n + 1)) return;
  const uint32_t g = (uint32_t)(tid / (n + 1)), i = (uint32_t)(tid % (n + 1));
  const uint32_t j0 = g * ell;
  const uint32_t lg = count - j0 < ell ? count - j0 : ell;
  uint32_t e[LC_EW_MAX], t[LC_EW_MAX];
  for (uint32_t w = 0; w < EW; ++w) e[w] = 0;
  uint32_t cw = 0;  // words in use
  for (int j = (int)lg - 1; j >= 0; --j) {
    const uint32_t ct = j0 + (uint32_t)j;
    uint64_t v;
    if (i < n) {
      const uint64_t a = A[(uint64_t)ct * n + i];
      v = a == 0 ? 0ull : q - a;
    } else {
      v = B[ct];
    }
    // e <- e gamma + v
    const uint32_t nw = cw + gw + 2 < EW ? cw + gw + 2 : EW;
    for (uint32_t w = 0; w < nw; ++w) t[w] = 0;
    for (uint32_t u = 0; u < cw; ++u) {
      uint64_t carry = 0;
      for (uint32_t k = 0; k < gw && u + k < nw; ++k) {
        const uint64_t s = (uint64_t)e[u] * gam.w[k] + t[u + k] + carry;
        t[u + k] = (uint32_t)s;
        carry = s >> 32;
      }
      for (uint32_t w = u + gw; carry && w < nw; ++w) {
        const uint64_t s = (uint64_t)t[w] + carry;
        t[w] = (uint32_t)s;
        carry = s >> 32;
      }
    }
    uint64_t carry = v;
    for (uint32_t w = 0; w < nw; ++w) {
      const uint64_t s = (uint64_t)t[w] + (uint32_t)carry;
      t[w] = (uint32_t)s;
      carry = (carry >> 32) + (s >> 32);
    }
    cw = 0;
    for (uint32_t w = 0; w < nw; ++w) {
      e[w] = t[w];
      if (t[w]) cw = w + 1;
    }
  }
  uint32_t* dst = E + tid * EW;
  for (uint32_t w = 0; w < EW; ++w) dst[w] = e[w];
}

// Partial products: item (g, i, r) multiplies eck[i][32 w + bit] over the set bits of
// exponent words w in [r WR, (r + 1) WR) of E[g][i]; an item with no set bit gives R mod m^2.
template <int WPL>
__global__ void __launch_bounds__(128) k_lc_products(const uint32_t* __restrict__ E, uint32_t EW,
                                                     uint32_t n, uint32_t G, uint32_t WR, uint32_t NR,
                                                     const uint32_t* __restrict__ eck, uint32_t T,
                                                     LcConsts<WPL> c, uint32_t* __restrict__ part) {
  constexpr int MW = 32 * WPL;
  const uint64_t idx = (uint64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (idx >= (uint64_t)G * n * NR) return;
  const uint32_t r = (uint32_t)(idx % NR);
  const uint64_t gi = idx / NR;
  const uint32_t i = (uint32_t)(gi % n), g = (uint32_t)(gi / n);
  const ModN<WPL> M = lc_mod(c);
  const uint32_t* er = E + ((uint64_t)g * (n + 1) + i) * EW;
  const uint32_t* tab = eck + (uint64_t)i * T * MW;
  uint32_t acc[WPL], f[WPL];
  bool first = true;
  const uint32_t w1 = (r + 1) * WR < EW ? (r + 1) * WR : EW;
  for (uint32_t w = r * WR; w < w1; ++w) {
    uint32_t ew = __ldg(er + w);
    while (ew) {
      const uint32_t k = 32 * w + __ffs(ew) - 1;
      ew &= ew - 1;
      if (k >= T) continue;  // only for inputs outside [0, q): never read past the table
      if (first) {
        load_lane_words<WPL>(tab + (uint64_t)k * MW, acc);
        first = false;
      } else {
        load_lane_words<WPL>(tab + (uint64_t)k * MW, f);
        mont_mul<WPL>(M, acc, f, acc);
      }
    }
  }
  if (first) load_lane_words<WPL>(c.r1, acc);
  store_lane_words<WPL>(part + idx * MW, acc);
}

// out[g][k] = in[g][2k] in[g][2k + 1] (Montgomery), or in[g][2k] for the odd last one.
template <int WPL>
__global__ void __launch_bounds__(128) k_lc_tree(const uint32_t* __restrict__ in, uint32_t S,
                                                 uint32_t G, LcConsts<WPL> c, uint32_t* __restrict__ out) {
  constexpr int MW = 32 * WPL;
  const uint32_t So = (S + 1) / 2;
  const uint64_t idx = (uint64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (idx >= (uint64_t)G * So) return;
  const uint32_t g = (uint32_t)(idx / So), k = (uint32_t)(idx % So);
  uint32_t a[WPL];
  load_lane_words<WPL>(in + ((uint64_t)g * S + 2 * k) * MW, a);
  if (2 * k + 1 < S) {
    const ModN<WPL> M = lc_mod(c);
    uint32_t b[WPL];
    load_lane_words<WPL>(in + ((uint64_t)g * S + 2 * k + 1) * MW, b);
    mont_mul<WPL>(M, a, b, a);
  }
  store_lane_words<WPL>(out + idx * MW, a);
}

// x_g = P_g (1 + b'_g m): P_g in Montgomery form, b'_g = column n of the exponents. The
// result stays in Montgomery form (Horner groups) or leaves it.
template <int WPL>
__global__ void __launch_bounds__(128) k_lc_finish(const uint32_t* __restrict__ P, const uint32_t* __restrict__ E,
                                                   uint32_t EW, uint32_t n, uint32_t G, LcConsts<WPL> c,
                                                   int to_plain, uint32_t* __restrict__ out) {
  constexpr int MW = 32 * WPL, L = 16 * WPL;
  __shared__ uint32_t sb[4][LC_EW_MAX], sm[4][L];
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t g = blockIdx.x * 4 + warp;
  if (g >= G) return;
  const uint32_t* bp = E + ((uint64_t)g * (n + 1) + n) * EW;
  for (uint32_t x = lane; x < EW; x += 32) sb[warp][x] = bp[x];
  for (uint32_t x = lane; x < (uint32_t)L; x += 32) sm[warp][x] = c.m[x];
  __syncwarp();
  // word x of b' m: sum_{i + j = x} b'_i m_j; high halves carry into word x + 1
  uint64_t acc[WPL], hi[WPL];
#pragma unroll
  for (int kk = 0; kk < WPL; ++kk) {
    acc[kk] = 0;
    hi[kk] = 0;
    const int x = (int)lane * WPL + kk;
    const int i0 = x - (L - 1) > 0 ? x - (L - 1) : 0;
    const int i1 = x < (int)EW - 1 ? x : (int)EW - 1;
    for (int i = i0; i <= i1; ++i) {
      const uint64_t p = (uint64_t)sb[warp][i] * sm[warp][x - i];
      acc[kk] += (uint32_t)p;
      hi[kk] += p >> 32;
    }
  }
#pragma unroll
  for (int kk = 1; kk < WPL; ++kk) acc[kk] += hi[kk - 1];
  const uint64_t sp_in = __shfl_up_sync(0xffffffffu, hi[WPL - 1], 1);
  if (lane > 0) acc[0] += sp_in;
  if (lane == 0) acc[0] += 1;
  uint32_t gv[WPL];
  warp_normalize<WPL>(acc, gv);  // 1 + b' m < m^2 (b' < m)
  const ModN<WPL> M = lc_mod(c);
  uint32_t r2[WPL], p[WPL];
  load_lane_words<WPL>(c.r2, r2);
  mont_mul<WPL>(M, gv, r2, gv);  // Montgomery form
  load_lane_words<WPL>(P + (uint64_t)g * MW, p);
  mont_mul<WPL>(M, p, gv, p);
  if (to_plain) {
    uint32_t one[WPL];
#pragma unroll
    for (int k = 0; k < WPL; ++k) one[k] = (lane == 0 && k == 0) ? 1u : 0u;
    mont_mul<WPL>(M, p, one, p);
  }
  store_lane_words<WPL>(out + (uint64_t)g * MW, p);
}

// Horner over the slots of each group: X = x_{ell_g - 1}; X <- X^gamma x_j for j = ell_g - 2
// down to 0; out = X (leaving Montgomery form). One warp per group.
template <int WPL>
__global__ void __launch_bounds__(128) k_lc_horner(const uint32_t* __restrict__ X, uint32_t count,
                                                   uint32_t ell, SmallWords gam, uint32_t gw,
                                                   LcConsts<WPL> c, uint32_t* __restrict__ out) {
  constexpr int MW = 32 * WPL;
  __shared__ uint32_t sg[8];
  if (threadIdx.x < 8) sg[threadIdx.x] = gam.w[threadIdx.x];
  __syncthreads();
  const uint32_t g = blockIdx.x * 4 + (threadIdx.x >> 5);
  const uint32_t G = (count + ell - 1) / ell;
  if (g >= G) return;
  const uint32_t j0 = g * ell;
  const uint32_t lg = count - j0 < ell ? count - j0 : ell;
  const ModN<WPL> M = lc_mod(c);
  uint32_t acc[WPL], f[WPL];
  load_lane_words<WPL>(X + (uint64_t)(j0 + lg - 1) * MW, acc);
  for (int j = (int)lg - 2; j >= 0; --j) {
    mont_pow_words<WPL>(M, acc, sg, (int)gw);
    load_lane_words<WPL>(X + (uint64_t)(j0 + j) * MW, f);
    mont_mul<WPL>(M, acc, f, acc);
  }
  uint32_t one[WPL];
#pragma unroll
  for (int k = 0; k < WPL; ++k) one[k] = (lane_id() == 0 && k == 0) ? 1u : 0u;
  mont_mul<WPL>(M, acc, one, acc);
  store_lane_words<WPL>(out + (uint64_t)g * MW, acc);
}

// Unpacking of a packed compression key: ck[i t + t - 1] = pck[i] and
// ck[i t + j] = ck[i t + j + 1]^delta, i.e. delta^(t-1-j) (x) pck[i]; indices >= n are not
// written. One warp per packed ciphertext.
template <int WPL>
__global__ void __launch_bounds__(128) k_lc_unpack(const uint32_t* __restrict__ pck, uint32_t npk,
                                                   uint32_t n, uint32_t t, SmallWords del, uint32_t dw,
                                                   LcConsts<WPL> c, uint32_t* __restrict__ ck) {
  constexpr int MW = 32 * WPL;
  __shared__ uint32_t sd[8];
  if (threadIdx.x < 8) sd[threadIdx.x] = del.w[threadIdx.x];
  __syncthreads();
  const uint32_t i = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (i >= npk) return;
  const ModN<WPL> M = lc_mod(c);
  uint32_t x[WPL], y[WPL], r2[WPL], one[WPL];
#pragma unroll
  for (int k = 0; k < WPL; ++k) one[k] = (lane_id() == 0 && k == 0) ? 1u : 0u;
  load_lane_words<WPL>(pck + (uint64_t)i * MW, x);
  const uint64_t top = (uint64_t)i * t + t - 1;
  if (top < n) store_lane_words<WPL>(ck + top * MW, x);
  load_lane_words<WPL>(c.r2, r2);
  mont_mul<WPL>(M, x, r2, x);
  for (int j = (int)t - 2; j >= 0; --j) {
    mont_pow_words<WPL>(M, x, sd, (int)dw);
    const uint64_t idx = (uint64_t)i * t + (uint32_t)j;
    if (idx < n) {
      mont_mul<WPL>(M, x, one, y);
      store_lane_words<WPL>(ck + idx * MW, y);
    }
  }
}

// Sample extraction of RLWE coefficient k (App. B): the LWE ciphertext (a', B[k]) with
// a'[i] = A[k - i] for i <= k and a'[i] = (q - A[N + k - i]) mod q for i > k, so that
// (q - a'[i]) mod q is the exponent of ck[i] in Algorithm "Compressing Extracted RLWE
// Coefficient". grid (ceil(N / 256), count).
__global__ void __launch_bounds__(256) k_lc_rlwe_extract(const uint64_t* __restrict__ A,
                                                         const uint64_t* __restrict__ Bp, uint32_t N,
                                                         uint64_t q, const uint32_t* __restrict__ K,
                                                         uint64_t* __restrict__ Aout,
                                                         uint64_t* __restrict__ Bout) {
  const uint32_t c = blockIdx.y;
  const uint32_t i = blockIdx.x * 256 + threadIdx.x;
  const uint32_t k = K[c];
  if (i < N) {
    uint64_t v;
    if (i <= k) {
      v = A[k - i];
    } else {
      const uint64_t a = A[N + k - i];
      v = a == 0 ? 0ull : q - a;
    }
    Aout[(uint64_t)c * N + i] = v;
  }
  if (i == 0) Bout[c] = Bp[k];
}

// Modulus switching of LWE coefficients: x -> floor((x r + floor(q / 2)) / q) mod r (round
// to nearest, ties up), q = 0 standing for 2^64. x r + floor(q / 2) < 2^128 for x < q <= 2^64
// and r < q. One thread per coefficient (count x n of A, then the count of B).
__global__ void __launch_bounds__(256) k_lc_rescale(const uint64_t* __restrict__ A,
                                                    const uint64_t* __restrict__ B, uint64_t nA,
                                                    uint64_t nB, uint64_t q, uint64_t r,
                                                    uint64_t* __restrict__ Ao, uint64_t* __restrict__ Bo) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nA + nB) return;
  const uint64_t x = i < nA ? A[i] : B[i - nA];
  const unsigned __int128 half = q == 0 ? ((unsigned __int128)1 << 63) : (unsigned __int128)(q / 2);
  const unsigned __int128 num = (unsigned __int128)x * r + half;
  const uint64_t quo = q == 0 ? (uint64_t)(num >> 64) : (uint64_t)(num / q);
  const uint64_t v = quo % r;
  if (i < nA)
    Ao[i] = v;
  else
    Bo[i - nA] = v;
}

template <int WPL>
LcConsts<WPL> lc_consts(const zp_lc* lc) {
  LcConsts<WPL> c;
  c.m2 = lc->d_m2;
  c.r1 = lc->d_r1;
  c.r2 = lc->d_r2;
  c.m = lc->d_m;
  c.ninv = lc->ninv;
  return c;
}

SmallWords small_words(const uint32_t* h, uint32_t nw) {
  SmallWords s{};
  for (uint32_t i = 0; i < nw && i < 8; ++i) s.w[i] = h[i];
  return s;
}

template <int WPL>
int lc_set_key(zp_lc* lc, const uint32_t* dCk, cudaStream_t st) {
  zp_clear_pending_error();
  k_lc_square_chain<WPL><<<(lc->n + 3) / 4, 128, 0, st>>>(dCk, lc->n, lc->T, lc_consts<WPL>(lc), lc->d_eck);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

template <int WPL>
int lc_unpack(zp_lc* lc, const uint32_t* dPck, uint32_t npk, uint32_t n, uint32_t t, SmallWords d,
              uint32_t dw, uint32_t* dCk, cudaStream_t st) {
  zp_clear_pending_error();
  k_lc_unpack<WPL><<<(npk + 3) / 4, 128, 0, st>>>(dPck, npk, n, t, d, dw, lc_consts<WPL>(lc), dCk);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

// Products, tree and finish for the G groups whose exponents start at E; the result (G x
// 2L) goes to out, in Montgomery form unless to_plain. Groups are processed in chunks of at
// most 2^20 work items (the partial products of a chunk are held at once).
template <int WPL>
int lc_products(zp_lc* lc, const uint32_t* E, uint32_t G, uint32_t EW, int to_plain, uint32_t* out,
                cudaStream_t st) {
  constexpr int MW = 32 * WPL;
  const uint32_t n = lc->n;
  // about 64 Ki work items when the work allows: the exponent words per item grow with it
  const uint64_t words = (uint64_t)G * n * EW;
  uint32_t WR = (uint32_t)((words + 65535) / 65536);
  if (WR < 1) WR = 1;
  if (WR > EW) WR = EW;
  const uint32_t NR = (EW + WR - 1) / WR;
  const uint32_t S0 = n * NR;  // partial products per group
  const uint32_t Gc = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(G, (1ull << 20) / S0));
  int rc = zp_scratch_reserve(&lc->s_pa, (size_t)Gc * S0 * MW * 4);
  if (!rc) rc = zp_scratch_reserve(&lc->s_pb, (size_t)Gc * ((S0 + 1) / 2) * MW * 4);
  if (rc) return rc;
  const LcConsts<WPL> c = lc_consts<WPL>(lc);
  for (uint32_t g0 = 0; g0 < G; g0 += Gc) {
    const uint32_t Gn = G - g0 < Gc ? G - g0 : Gc;
    uint32_t* pa = static_cast<uint32_t*>(lc->s_pa.p);
    uint32_t* pb = static_cast<uint32_t*>(lc->s_pb.p);
    const uint32_t* Eg = E + (uint64_t)g0 * (n + 1) * EW;
    const uint64_t items = (uint64_t)Gn * S0;
    zp_clear_pending_error();
    k_lc_products<WPL><<<(unsigned)((items + 3) / 4), 128, 0, st>>>(Eg, EW, n, Gn, WR, NR, lc->d_eck,
                                                                    lc->T, c, pa);
    ZP_CUDA(cudaGetLastError());
    uint32_t S = S0;
    while (S > 1) {
      const uint32_t So = (S + 1) / 2;
      k_lc_tree<WPL><<<(unsigned)(((uint64_t)Gn * So + 3) / 4), 128, 0, st>>>(pa, S, Gn, c, pb);
      ZP_CUDA(cudaGetLastError());
      std::swap(pa, pb);
      S = So;
    }
    k_lc_finish<WPL><<<(Gn + 3) / 4, 128, 0, st>>>(pa, Eg, EW, n, Gn, c, to_plain, out + (uint64_t)g0 * MW);
    ZP_CUDA(cudaGetLastError());
  }
  return ZP_OK;
}

template <int WPL>
int lc_compress(zp_lc* lc, const uint64_t* dA, const uint64_t* dB, uint32_t count, uint64_t q,
                uint32_t ell, SmallWords gam, uint32_t gw, bool folded, uint32_t EW, uint32_t* dX,
                cudaStream_t st) {
  constexpr int MW = 32 * WPL;
  const uint32_t n = lc->n;
  const uint32_t fold = folded ? ell : 1;     // ciphertexts per exponent group
  const uint32_t G = (count + fold - 1) / fold;
  int rc = zp_scratch_reserve(&lc->s_e, (size_t)G * (n + 1) * EW * 4);
  if (rc) return rc;
  zp_clear_pending_error();
  const uint64_t threads = (uint64_t)G * (n + 1);
  k_lc_exponents<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(
      dA, dB, count, n, q, fold, gam, gw, EW, static_cast<uint32_t*>(lc->s_e.p));
  ZP_CUDA(cudaGetLastError());
  const uint32_t* E = static_cast<const uint32_t*>(lc->s_e.p);
  if (folded || ell == 1) {
    rc = lc_products<WPL>(lc, E, G, EW, 1, dX, st);
  } else {
    rc = zp_scratch_reserve(&lc->s_x, (size_t)count * MW * 4);
    if (rc) return rc;
    uint32_t* X = static_cast<uint32_t*>(lc->s_x.p);
    rc = lc_products<WPL>(lc, E, G, EW, 0, X, st);
    if (rc) return rc;
    const uint32_t Gh = (count + ell - 1) / ell;
    k_lc_horner<WPL><<<(Gh + 3) / 4, 128, 0, st>>>(X, count, ell, gam, gw, lc_consts<WPL>(lc), dX);
    ZP_CUDA(cudaGetLastError());
  }
  return rc;
}

}  // namespace

// ---------------------------------------------------------------------------------
extern "C" int zp_lc_create(int device, uint32_t key_bits, const uint32_t* hM, zp_lc** out) {
  using namespace zp_host;
  try {
    if (!hM || !out) return zp_set_error(ZP_EINVAL, "zp_lc_create: null argument");
    *out = nullptr;
    if (key_bits != 2048 && key_bits != 3072)
      return zp_set_error(ZP_EUNSUPPORTED, "zp_lc_create: key_bits=%u (2048 or 3072)", key_bits);
    const uint32_t L = key_bits / 32;
    Big m(hM, hM + L);
    if ((m[0] & 1u) == 0 || bits(m) != key_bits)
      return zp_set_error(ZP_EINVAL, "zp_lc_create: m must be odd with exactly %u bits", key_bits);
    Big m2 = mul(m, m);
    m2.resize(2 * L, 0);
    const Big r1 = pow2_mod(64 * L, m2), r2 = pow2_mod(128 * L, m2);
    ZP_ON_DEVICE(device);
    zp_lc* lc = new zp_lc();
    lc->device = device;
    lc->key_bits = key_bits;
    lc->L = L;
    lc->ninv = neg_inv32(m2[0]);
    lc->h_m = m;
    lc->d_m = lc->d_m2 = lc->d_r1 = lc->d_r2 = lc->d_eck = nullptr;
    lc->n = lc->T = 0;
    auto fail = [lc](int code, const char* what) {
      for (uint32_t* p : {lc->d_m, lc->d_m2, lc->d_r1, lc->d_r2})
        if (p) cudaFree(p);
      delete lc;
      return zp_set_error(code, "zp_lc_create: %s", what);
    };
    if (cudaMalloc(&lc->d_m, L * 4) != cudaSuccess || cudaMalloc(&lc->d_m2, 8 * L) != cudaSuccess ||
        cudaMalloc(&lc->d_r1, 8 * L) != cudaSuccess || cudaMalloc(&lc->d_r2, 8 * L) != cudaSuccess)
      return fail(ZP_ENOMEM, "cudaMalloc");
    cudaError_t e = cudaMemcpy(lc->d_m, m.data(), L * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(lc->d_m2, m2.data(), 8 * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(lc->d_r1, r1.data(), 8 * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(lc->d_r2, r2.data(), 8 * L, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(ZP_ECUDA, "copy constants");
    *out = lc;
    return ZP_OK;
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_lc_create: host allocation");
  }
}

extern "C" int zp_lc_destroy(zp_lc* lc) {
  if (!lc) return ZP_OK;
  zp_device_scope _zp_scope(lc->device);
  cudaDeviceSynchronize();
  for (uint32_t* p : {lc->d_m, lc->d_m2, lc->d_r1, lc->d_r2, lc->d_eck})
    if (p) cudaFree(p);
  for (zp_scratch* s : {&lc->s_e, &lc->s_pa, &lc->s_pb, &lc->s_x, &lc->s_k})
    if (s->p) cudaFree(s->p);
  delete lc;
  return ZP_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

extern "C" int zp_lc_set_key(zp_lc* lc, const uint32_t* dCk, uint32_t n, uint32_t T, void* stream) {
  if (!lc || !dCk) return zp_set_error(ZP_EINVAL, "zp_lc_set_key: null argument");
  if (n == 0 || n > (1u << 20)) return zp_set_error(ZP_EINVAL, "zp_lc_set_key: n=%u out of [1, 2^20]", n);
  if (T == 0 || T > lc->key_bits)
    return zp_set_error(ZP_EINVAL, "zp_lc_set_key: T=%u out of [1, %u]", T, lc->key_bits);
  if (!aligned16(dCk)) return zp_set_error(ZP_EINVAL, "zp_lc_set_key: dCk must be 16-byte aligned");
  ZP_ON_DEVICE(lc->device);
  const size_t bytes = (size_t)n * T * 8 * lc->L;
  if (lc->d_eck && (size_t)lc->n * lc->T * 8 * lc->L != bytes) {
    cudaFree(lc->d_eck);
    lc->d_eck = nullptr;
  }
  if (!lc->d_eck && cudaMalloc(&lc->d_eck, bytes) != cudaSuccess) {
    lc->d_eck = nullptr;
    lc->n = lc->T = 0;
    return zp_set_error(ZP_ENOMEM, "zp_lc_set_key: cudaMalloc(%zu bytes) for the expanded key", bytes);
  }
  lc->n = n;
  lc->T = T;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return lc->L == 64 ? lc_set_key<4>(lc, dCk, st) : lc_set_key<6>(lc, dCk, st);
}

extern "C" int zp_lc_unpack_key(zp_lc* lc, const uint32_t* dPck, uint32_t n, uint32_t t,
                                const uint32_t* hDelta, uint32_t deltaWords, uint32_t* dCk, void* stream) {
  using namespace zp_host;
  if (!lc || !dPck || !hDelta || !dCk) return zp_set_error(ZP_EINVAL, "zp_lc_unpack_key: null argument");
  if (n == 0 || t == 0) return zp_set_error(ZP_EINVAL, "zp_lc_unpack_key: n and t must be positive");
  if (deltaWords == 0 || deltaWords > 8)
    return zp_set_error(ZP_EINVAL, "zp_lc_unpack_key: deltaWords=%u out of [1, 8]", deltaWords);
  const Big d(hDelta, hDelta + deltaWords);
  if (bits(d) < 2) return zp_set_error(ZP_EINVAL, "zp_lc_unpack_key: delta must be at least 2");
  if (!aligned16(dPck) || !aligned16(dCk))
    return zp_set_error(ZP_EINVAL, "zp_lc_unpack_key: dPck and dCk must be 16-byte aligned");
  ZP_ON_DEVICE(lc->device);
  const uint32_t npk = (n + t - 1) / t;
  const SmallWords sd = small_words(hDelta, deltaWords);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return lc->L == 64 ? lc_unpack<4>(lc, dPck, npk, n, t, sd, deltaWords, dCk, st)
                     : lc_unpack<6>(lc, dPck, npk, n, t, sd, deltaWords, dCk, st);
}

extern "C" int zp_lc_compress(zp_lc* lc, const uint64_t* dA, const uint64_t* dB, uint32_t count,
                              uint64_t q, uint32_t ell, const uint32_t* hGamma, uint32_t gammaWords,
                              int mode, uint32_t* dX, void* stream) {
  using namespace zp_host;
  try {
    if (!lc || !dA || !dB || !dX) return zp_set_error(ZP_EINVAL, "zp_lc_compress: null argument");
    if (!lc->d_eck) return zp_set_error(ZP_ESTATE, "zp_lc_compress: no key (call zp_lc_set_key)");
    if (count == 0) return ZP_OK;
    if (q == 1) return zp_set_error(ZP_EINVAL, "zp_lc_compress: q must be at least 2 (0 stands for 2^64)");
    if (ell == 0) return zp_set_error(ZP_EINVAL, "zp_lc_compress: ell must be positive");
    if (mode < 0 || mode > 2) return zp_set_error(ZP_EINVAL, "zp_lc_compress: mode=%d out of [0, 2]", mode);
    if (ell > 1 && (!hGamma || gammaWords == 0 || gammaWords > 8))
      return zp_set_error(ZP_EINVAL, "zp_lc_compress: gamma needs 1 to 8 words when ell > 1");
    if (!aligned16(dX)) return zp_set_error(ZP_EINVAL, "zp_lc_compress: dX must be 16-byte aligned");
    const Big qm1 = q == 0 ? Big{0xFFFFFFFFu, 0xFFFFFFFFu} : from_u64(q - 1);
    const uint32_t tq = bits(qm1);
    Big gam = ell > 1 ? Big(hGamma, hGamma + gammaWords) : Big{1};
    trim(gam);
    if (ell > 1 && cmp(gam, qm1) <= 0)
      return zp_set_error(ZP_EINVAL, "zp_lc_compress: gamma must exceed q - 1");
    // the largest exponent: (q - 1) sum_{j < ell} gamma^j, below m for the slots to decrypt
    const uint32_t lmax = ell < count ? ell : count;
    Big emax{0};
    for (uint32_t j = 0; j < lmax; ++j) emax = add(mul(emax, gam), qm1);
    if (cmp(emax, lc->h_m) >= 0)
      return zp_set_error(ZP_EINVAL, "zp_lc_compress: (q - 1) sum_j gamma^j must be below m (ell=%u too large)", ell);
    const uint32_t ebits = bits(emax);
    bool folded;
    if (lmax == 1) {
      folded = true;  // one ciphertext per group: both forms coincide
    } else if (mode == 1) {
      folded = false;
    } else if (mode == 2) {
      folded = true;
    } else {
      // folded does n ebits / 2 products per group; Horner ell n tq / 2 per group plus a
      // sequential tail of about 1.5 ell |gamma| products per group
      const double G = (double)((count + ell - 1) / ell);
      const double folded_work = G * lc->n * ebits / 2.0;
      const double horner_work = (double)count * lc->n * tq / 2.0;
      const double tail = 1.5 * ell * bits(gam);
      folded = ebits <= lc->T && folded_work < horner_work + tail * 500.0;
    }
    if (folded && ebits > lc->T)
      return zp_set_error(ZP_EINVAL, "zp_lc_compress: the expanded key has %u powers, folded exponents need %u",
                          lc->T, ebits);
    if (!folded && tq > lc->T)
      return zp_set_error(ZP_EINVAL, "zp_lc_compress: the expanded key has %u powers, q needs %u", lc->T, tq);
    const uint32_t EW = folded ? (ebits + 31) / 32 + 1 : (tq + 31) / 32 + 1;
    if (EW > (uint32_t)LC_EW_MAX) return zp_set_error(ZP_EINVAL, "zp_lc_compress: exponents too wide");
    ZP_ON_DEVICE(lc->device);
    const SmallWords sg = small_words(gam.data(), (uint32_t)gam.size());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return lc->L == 64 ? lc_compress<4>(lc, dA, dB, count, q, ell, sg, (uint32_t)gam.size(), folded, EW, dX, st)
                       : lc_compress<6>(lc, dA, dB, count, q, ell, sg, (uint32_t)gam.size(), folded, EW, dX, st);
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_lc_compress: host allocation");
  }
}

extern "C" int zp_lc_rlwe_extract(zp_lc* lc, const uint64_t* dA, const uint64_t* dB, uint32_t N, uint64_t q,
                                  const uint32_t* hK, uint32_t count, uint64_t* dAout, uint64_t* dBout,
                                  void* stream) {
  if (!lc || !dA || !dB || !hK || !dAout || !dBout)
    return zp_set_error(ZP_EINVAL, "zp_lc_rlwe_extract: null argument");
  if (N == 0) return zp_set_error(ZP_EINVAL, "zp_lc_rlwe_extract: N must be positive");
  if (count == 0) return ZP_OK;
  if (count > 65535) return zp_set_error(ZP_EINVAL, "zp_lc_rlwe_extract: count=%u above 65535", count);
  for (uint32_t c = 0; c < count; ++c)
    if (hK[c] >= N) return zp_set_error(ZP_EINVAL, "zp_lc_rlwe_extract: coefficient %u >= N=%u", hK[c], N);
  ZP_ON_DEVICE(lc->device);
  int rc = zp_scratch_reserve(&lc->s_k, (size_t)count * 4);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* dK = static_cast<uint32_t*>(lc->s_k.p);
  ZP_CUDA(cudaMemcpyAsync(dK, hK, (size_t)count * 4, cudaMemcpyHostToDevice, st));
  zp_clear_pending_error();
  dim3 grid((N + 255) / 256, count);
  k_lc_rlwe_extract<<<grid, 256, 0, st>>>(dA, dB, N, q, dK, dAout, dBout);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

extern "C" int zp_lc_rescale(const uint64_t* dA, const uint64_t* dB, uint32_t count, uint32_t n,
                             uint64_t q, uint64_t r, uint64_t* dAout, uint64_t* dBout, void* stream) {
  if (!dA || !dB || !dAout || !dBout) return zp_set_error(ZP_EINVAL, "zp_lc_rescale: null argument");
  if (r < 2) return zp_set_error(ZP_EINVAL, "zp_lc_rescale: r must be at least 2");
  if (q != 0 && r >= q) return zp_set_error(ZP_EINVAL, "zp_lc_rescale: r must be below q");
  if (count == 0) return ZP_OK;
  const uint64_t nA = (uint64_t)count * n, total = nA + count;
  zp_clear_pending_error();
  k_lc_rescale<<<(unsigned)((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      dA, dB, nA, count, q, r, dAout, dBout);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}
