// k_paillier.cu -- Paillier arithmetic mod m^2 for the per-client hint, the combined
// response and the client-side pieces (ck_r from a seed, exponentiation, decryption).
//
//  * the per-client hint (Algorithm "ZipPIR", Setup, and Sec. 4.3 "Lowering offline
//    communication costs": k = PaillierMatMul(H', ck_r)):
//        k[r'] = prod_i ck_r[i]^{H'[r', i]} mod m^2,  H'[r', i] = sum_j gamma^j Hneg[r' ell + j, i].
//    The exponent splits by slot: k[r'] = prod_j K_{r' ell + j}^{gamma^j} with the per-row
//    products K_r = prod_i ck_r[i]^{Hneg[r, i]} (32-bit exponents). K_r is a product of
//    the precomputed squares ck_r[i]^{2^e} selected by the bits of Hneg[r, i]; the slots
//    are then combined by Horner, X <- X^gamma * K_{r' ell + j}, exponentiation by gamma
//    (< 2^96) by left-to-right square-and-multiply.
//  * the combined response (Sec. 4.3, last extension): k (+) t = k (1 + t m) mod m^2, the
//    homomorphic addition of t encrypted with randomness 1, so that Dec(k (+) t) =
//    Dec(k) + t mod m.
//  * client side: ck_r expanded from a ChaCha20 seed and reduced mod m^2, x^e mod m^2 for
//    a shared exponent, and decryption by one exponentiation to lambda mu followed by an
//    exact division by m.
//
// All products mod m^2 are the Montgomery products of zp_mont.cuh with R = 2^(64 L), one
// warp per product, 4 words per lane.
#include "zp_internal.cuh"
#include "zp_chacha.cuh"
#include "zp_mont.cuh"

namespace {

constexpr int MW = 2 * ZP_MAX_L;  // words of m^2
constexpr int MWPL = MW / 32;     // words per lane

using ModM2 = ModN<MWPL>;

// x <- x^gamma (Montgomery form), gamma = g[0] + g[1] 2^32 + g[2] 2^64 > 0.
__device__ void mont_pow_gamma(const ModM2& M, uint32_t (&x)[MWPL], uint32_t g0, uint32_t g1,
                               uint32_t g2) {
  int top = g2 ? 95 - __clz(g2) : (g1 ? 63 - __clz(g1) : 31 - __clz(g0));
  uint32_t y[MWPL];
#pragma unroll
  for (int k = 0; k < MWPL; ++k) y[k] = x[k];
  for (int bit = top - 1; bit >= 0; --bit) {
    mont_mul(M, y, y, y);
    const uint32_t word = bit >= 64 ? g2 : (bit >= 32 ? g1 : g0);
    if ((word >> (bit & 31)) & 1u) mont_mul(M, y, x, y);
  }
#pragma unroll
  for (int k = 0; k < MWPL; ++k) x[k] = y[k];
}

struct M2Consts {
  const uint32_t* m2;  // 2L words
  const uint32_t* r1;  // 2^(64L) mod m^2 (Montgomery form of 1)
  const uint32_t* r2;  // 2^(128L) mod m^2
  const uint32_t* m;   // L words (combine only)
  uint32_t ninv;
};

__device__ __forceinline__ ModM2 load_mod(const M2Consts& c) {
  ModM2 M;
  load_lane_words(c.m2, M.n);
  M.ninv = c.ninv;
  return M;
}

// ---------------------------------------------------------------------------------
// Squares table P[i][e] = (ck_r[i])^(2^e) in Montgomery form, e < 32: one warp per base.
__global__ void __launch_bounds__(128) k_square_table(const uint32_t* __restrict__ ckr, uint32_t n,
                                                      M2Consts c, uint32_t* __restrict__ P) {
  const uint32_t i = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (i >= n) return;
  const ModM2 M = load_mod(c);
  uint32_t x[MWPL], r2[MWPL];
  load_lane_words(ckr + (uint64_t)i * MW, x);
  load_lane_words(c.r2, r2);
  mont_mul(M, x, r2, x);  // to Montgomery form
  uint32_t* dst = P + (uint64_t)i * 32 * MW;
  store_lane_words(dst, x);
  for (int e = 1; e < 32; ++e) {
    mont_mul(M, x, x, x);
    store_lane_words(dst + (uint64_t)e * MW, x);
  }
}

// Per-row products K_r = prod_i P[i][bits of Hneg[r][i]] (Montgomery form), one warp per
// row of the listed packed rows (slots j < ell; rows past R give the Montgomery one).
// A CTA's RW warps share each base's 32 squares through shared memory.
constexpr int RW = 16;
__global__ void __launch_bounds__(RW * 32) k_row_products(const uint32_t* __restrict__ hneg,
                                                          uint32_t n, uint32_t R, uint32_t ell,
                                                          const uint32_t* __restrict__ prows,
                                                          uint32_t nprows, M2Consts c,
                                                          const uint32_t* __restrict__ P,
                                                          uint32_t* __restrict__ K) {
  __shared__ __align__(16) uint32_t tab[32 * MW];  // the 32 squares of one base (16 KiB)
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t slot = blockIdx.x * RW + warp;    // index into (listed packed row, j)
  const uint32_t total = nprows * ell;
  uint32_t row = 0xFFFFFFFFu;
  if (slot < total) {
    const uint32_t rp = prows ? prows[slot / ell] : slot / ell;
    row = rp * ell + slot % ell;
  }
  const bool valid = row < R;
  const ModM2 M = load_mod(c);
  uint32_t acc[MWPL];
  load_lane_words(c.r1, acc);
  const uint32_t* hrow = hneg + (uint64_t)(valid ? row : 0) * n;
  for (uint32_t i = 0; i < n; ++i) {
    __syncthreads();  // everyone is done with the previous base's squares
    const uint4* src = reinterpret_cast<const uint4*>(P + (uint64_t)i * 32 * MW);
    for (uint32_t x = threadIdx.x; x < 32 * MW / 4; x += RW * 32)
      reinterpret_cast<uint4*>(tab)[x] = __ldg(src + x);
    __syncthreads();
    uint32_t h = valid ? __ldg(hrow + i) : 0u;
    while (h) {
      const int e = __ffs(h) - 1;
      h &= h - 1;
      uint32_t f[MWPL];
      const uint4 v = reinterpret_cast<const uint4*>(tab + e * MW)[lane_id()];
      f[0] = v.x;
      f[1] = v.y;
      f[2] = v.z;
      f[3] = v.w;
      mont_mul(M, acc, f, acc);
    }
  }
  if (slot < total) store_lane_words(K + (uint64_t)slot * MW, acc);
}

// k[r'] = prod_j K_{r' ell + j}^{gamma^j} by Horner, converted out of Montgomery form: one
// warp per listed packed row.
__global__ void __launch_bounds__(128) k_pack_hint(const uint32_t* __restrict__ K, uint32_t ell,
                                                   const uint32_t* __restrict__ prows,
                                                   uint32_t nprows, M2Consts c, uint32_t g0,
                                                   uint32_t g1, uint32_t g2,
                                                   uint32_t* __restrict__ kout) {
  const uint32_t idx = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (idx >= nprows) return;
  const ModM2 M = load_mod(c);
  const uint32_t* Kp = K + (uint64_t)idx * ell * MW;
  uint32_t x[MWPL];
  load_lane_words(Kp + (uint64_t)(ell - 1) * MW, x);
  for (int j = (int)ell - 2; j >= 0; --j) {
    mont_pow_gamma(M, x, g0, g1, g2);
    uint32_t f[MWPL];
    load_lane_words(Kp + (uint64_t)j * MW, f);
    mont_mul(M, x, f, x);
  }
  uint32_t one[MWPL] = {lane_id() == 0 ? 1u : 0u, 0u, 0u, 0u};
  mont_mul(M, x, one, x);  // out of Montgomery form
  const uint32_t rp = prows ? prows[idx] : idx;
  store_lane_words(kout + (uint64_t)rp * MW, x);
}

// out[b][r'] = k[b][r'] (1 + t[b][r'] m_b) mod m_b^2: one warp per (query, packed row).
__global__ void __launch_bounds__(128) k_combine(const uint32_t* __restrict__ k,
                                                 const uint32_t* __restrict__ T, uint32_t B,
                                                 uint32_t d1p, const M2Consts* __restrict__ cl,
                                                 uint32_t* __restrict__ out) {
  __shared__ uint32_t tm[4][2][ZP_MAX_L];
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t idx = blockIdx.x * 4 + warp;
  if (idx >= B * d1p) return;
  const uint32_t b = idx / d1p;
  const M2Consts c = cl[b];
  const uint32_t* t = T + (uint64_t)idx * ZP_MAX_L;
  for (int x = lane; x < ZP_MAX_L; x += 32) {
    tm[warp][0][x] = t[x];
    tm[warp][1][x] = c.m[x];
  }
  __syncwarp();
  // g = 1 + t m: word x of t m is sum_{i + j = x} t_i m_j; low halves go to word x, high
  // halves to word x + 1 (for this lane's top word: the next lane's first word)
  uint64_t acc[MWPL] = {0, 0, 0, 0}, hi[MWPL] = {0, 0, 0, 0};
#pragma unroll
  for (int kk = 0; kk < MWPL; ++kk) {
    const int x = (int)lane * MWPL + kk;
    const int i0 = x - (ZP_MAX_L - 1) > 0 ? x - (ZP_MAX_L - 1) : 0;
    const int i1 = x < ZP_MAX_L - 1 ? x : ZP_MAX_L - 1;
    for (int i = i0; i <= i1; ++i) {
      const uint64_t p = (uint64_t)tm[warp][0][i] * tm[warp][1][x - i];
      acc[kk] += (uint32_t)p;
      hi[kk] += p >> 32;
    }
  }
  acc[1] += hi[0];
  acc[2] += hi[1];
  acc[3] += hi[2];
  const uint64_t sp_in = __shfl_up_sync(0xffffffffu, hi[3], 1);
  if (lane > 0) acc[0] += sp_in;
  if (lane == 0) acc[0] += 1;
  uint32_t g[MWPL];
  warp_normalize<MWPL>(acc, g);  // t m + 1 < m^2
  const ModM2 M = load_mod(c);
  uint32_t kv[MWPL], r2[MWPL];
  load_lane_words(k + (uint64_t)idx * MW, kv);
  load_lane_words(c.r2, r2);
  mont_mul(M, kv, r2, kv);  // k R mod m^2
  mont_mul(M, kv, g, kv);   // k g mod m^2
  store_lane_words(out + (uint64_t)idx * MW, kv);
}

// An exponent of up to 128 words, passed by value.
struct PowExp {
  uint32_t w[128];
};

// y = x^e (both in Montgomery form) by left-to-right binary exponentiation; e = 0 gives
// the Montgomery form of 1.
__device__ __forceinline__ void mont_powm(const ModM2& M, const M2Consts& c, const uint32_t (&x)[MWPL],
                                          const PowExp& e, uint32_t ew, uint32_t (&y)[MWPL]) {
  int top = -1;  // highest set bit of e (warp-uniform)
  for (int w = (int)ew - 1; w >= 0 && top < 0; --w)
    if (e.w[w]) top = 32 * w + 31 - __clz(e.w[w]);
  if (top < 0) {
    load_lane_words(c.r1, y);
    return;
  }
#pragma unroll
  for (int k = 0; k < MWPL; ++k) y[k] = x[k];
  for (int bit = top - 1; bit >= 0; --bit) {
    mont_mul(M, y, y, y);
    if ((e.w[bit >> 5] >> (bit & 31)) & 1u) mont_mul(M, y, x, y);
  }
}

// out[i] = base[i]^e mod m^2 for a shared exponent of ew words: the core of Paillier's
// decryption and of its randomness factor r^m. One warp per base.
__global__ void __launch_bounds__(128) k_powm(const uint32_t* __restrict__ base, PowExp e,
                                              uint32_t ew, uint32_t count, M2Consts c,
                                              uint32_t* __restrict__ out) {
  const uint32_t idx = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (idx >= count) return;
  const ModM2 M = load_mod(c);
  uint32_t x[MWPL], y[MWPL], r2[MWPL];
  load_lane_words(base + (uint64_t)idx * MW, x);
  load_lane_words(c.r2, r2);
  mont_mul(M, x, r2, x);  // to Montgomery form
  mont_powm(M, c, x, e, ew, y);
  uint32_t one[MWPL] = {lane_id() == 0 ? 1u : 0u, 0u, 0u, 0u};
  mont_mul(M, y, one, y);
  store_lane_words(out + (uint64_t)idx * MW, y);
}

// Paillier decryption (g = m + 1): with e = lambda mu, v = c^e mod m^2 = 1 + m Dec(c) (c^lambda
// = 1 + m lambda Dec(c) mod m^2 and lambda mu = 1 mod m), and Dec(c) = (v - 1) / m, an exact
// division computed as the low L words of (v - 1) m^{-1} mod 2^(32 L) (m is odd and the
// quotient is below m < 2^(32 L)). One warp per ciphertext; out is count x L words.
struct MinvArg {
  uint32_t w[ZP_MAX_L];  // m^{-1} mod 2^(32 L)
};
__global__ void __launch_bounds__(128) k_decrypt(const uint32_t* __restrict__ cts, PowExp e,
                                                 uint32_t ew, MinvArg minv, uint32_t count,
                                                 M2Consts c, uint32_t* __restrict__ out) {
  __shared__ uint32_t sv[4][ZP_MAX_L];
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t idx = blockIdx.x * 4 + warp;
  if (idx >= count) return;
  const ModM2 M = load_mod(c);
  uint32_t x[MWPL], y[MWPL], r2[MWPL];
  load_lane_words(cts + (uint64_t)idx * MW, x);
  load_lane_words(c.r2, r2);
  mont_mul(M, x, r2, x);
  mont_powm(M, c, x, e, ew, y);
  uint32_t one[MWPL] = {lane == 0 ? 1u : 0u, 0u, 0u, 0u};
  mont_mul(M, y, one, y);  // v
  warp_sub<MWPL>(y, one);  // v - 1
  if (lane < ZP_MAX_L / MWPL) {
#pragma unroll
    for (int k = 0; k < MWPL; ++k) sv[warp][lane * MWPL + k] = y[k];
  }
  __syncwarp();
  // word xw of the product: sum_{i + j = xw} v_i minv_j; the high halves carry into word xw + 1
  uint64_t acc[MWPL] = {0, 0, 0, 0}, hi[MWPL] = {0, 0, 0, 0};
#pragma unroll
  for (int kk = 0; kk < MWPL; ++kk) {
    const int xw = (int)lane * MWPL + kk;
    if (xw < ZP_MAX_L)
      for (int i = 0; i <= xw; ++i) {
        const uint64_t p = (uint64_t)sv[warp][i] * minv.w[xw - i];
        acc[kk] += (uint32_t)p;
        hi[kk] += p >> 32;
      }
  }
  acc[1] += hi[0];
  acc[2] += hi[1];
  acc[3] += hi[2];
  const uint64_t sp_in = __shfl_up_sync(0xffffffffu, hi[3], 1);
  if (lane > 0) acc[0] += sp_in;
  uint32_t q[MWPL];
  warp_normalize<MWPL>(acc, q);  // words >= L are discarded (mod 2^(32 L))
  if (lane < ZP_MAX_L / MWPL)
    *reinterpret_cast<uint4*>(out + (uint64_t)idx * ZP_MAX_L + MWPL * lane) = make_uint4(q[0], q[1], q[2], q[3]);
}

// ck_r[i] = (the 2L + 4 keystream words [(2L + 4) i, (2L + 4)(i + 1)) of ChaCha20, read as a
// little-endian integer) mod m^2: a value of 2 key_bits + 128 bits whose residue is
// statistically uniform in Z_{m^2}. One warp per element: lanes 0..8 make the (at most 9)
// blocks that cover the element's words, then x = x_lo + 2^(64 L) x_hi is reduced as
// (x_lo + (x_hi R mod m^2)) mod m^2, x_hi R mod m^2 = MontMul(x_hi, R^2).
constexpr int CKR_W = 2 * ZP_MAX_L + 4;
__global__ void __launch_bounds__(128) k_expand_ckr(ChachaKey key, uint32_t counter0,
                                                    uint32_t count, M2Consts c,
                                                    uint32_t* __restrict__ out) {
  __shared__ uint32_t ks[4][9 * 16];
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t idx = blockIdx.x * 4 + warp;
  if (idx >= count) return;
  const uint64_t w0 = (uint64_t)idx * CKR_W;
  const uint32_t o = (uint32_t)(w0 & 15u);
  if (lane < 9) {
    uint32_t b[16];
    chacha20_block(key, counter0 + (uint32_t)(w0 >> 4) + lane, b);
#pragma unroll
    for (int t = 0; t < 16; ++t) ks[warp][16 * lane + t] = b[t];
  }
  __syncwarp();
  uint32_t xl[MWPL], xh[MWPL] = {0, 0, 0, 0}, r2[MWPL];
#pragma unroll
  for (int k = 0; k < MWPL; ++k) xl[k] = ks[warp][o + MWPL * lane + k];
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) xh[k] = ks[warp][o + MW + k];
  }
  const ModM2 M = load_mod(c);
  load_lane_words(c.r2, r2);
  mont_mul(M, xh, r2, xh);  // x_hi R mod m^2
  uint64_t acc[MWPL];
#pragma unroll
  for (int k = 0; k < MWPL; ++k) acc[k] = (uint64_t)xl[k] + xh[k];
  uint32_t w[MWPL];
  uint32_t top = warp_normalize_top<MWPL>(acc, w);
  // the sum is below 2^(64 L) + m^2 <= 5 m^2 (m^2 >= 2^(64 L - 2)): at most four subtractions
  for (int it = 0; it < 5; ++it) {
    const bool ge = warp_geq<MWPL>(w, M.n);
    if (!top && !ge) break;
    warp_sub<MWPL>(w, M.n);
    top = top && ge;
  }
  store_lane_words(out + (uint64_t)idx * MW, w);
}

}  // namespace

// ---------------------------------------------------------------------------------
static M2Consts client_consts(const zp_client* cl) {
  M2Consts c;
  c.m2 = cl->d_m2;
  c.r1 = cl->d_r1;
  c.r2 = cl->d_r2;
  c.m = cl->d_m;
  c.ninv = cl->m2inv;
  return c;
}

int zp_launch_client_hint(zp_db* db, const zp_client* cl, const uint32_t* dCkr, uint32_t* dK,
                          const uint32_t* dRows, uint32_t nprows, cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  const uint32_t n = ctx->P.n, ell = ctx->ell;
  const size_t p_bytes = (size_t)n * 32 * MW * 4;
  const size_t k_bytes = (size_t)nprows * ell * MW * 4;
  int rc = zp_scratch_reserve(&db->s_ptab, p_bytes);
  if (!rc) rc = zp_scratch_reserve(&db->s_krows, k_bytes);
  if (rc) return rc;
  uint32_t* P = static_cast<uint32_t*>(db->s_ptab.p);
  uint32_t* Kr = static_cast<uint32_t*>(db->s_krows.p);
  const M2Consts c = client_consts(cl);
  zp_clear_pending_error();
  ctx->launches += 3;
  k_square_table<<<(n + 3) / 4, 128, 0, st>>>(dCkr, n, c, P);
  ZP_CUDA(cudaGetLastError());
  const uint32_t slots = nprows * ell;
  k_row_products<<<(slots + RW - 1) / RW, RW * 32, 0, st>>>(db->d_hneg, n, db->R, ell, dRows,
                                                            nprows, c, P, Kr);
  ZP_CUDA(cudaGetLastError());
  k_pack_hint<<<(nprows + 3) / 4, 128, 0, st>>>(Kr, ell, dRows, nprows, c, ctx->gamma_w[0],
                                                ctx->gamma_w[1], ctx->gamma_w[2], dK);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

int zp_launch_combine(zp_db* db, zp_client* const* clients, const uint32_t* dK, const uint32_t* dT,
                      uint32_t B, uint32_t* dOut, cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  int rc = zp_scratch_reserve(&db->s_m2consts, (size_t)B * sizeof(M2Consts));
  if (rc) return rc;
  std::vector<M2Consts> h(B);
  for (uint32_t b = 0; b < B; ++b) h[b] = client_consts(clients[b]);
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  ZP_CUDA(cudaMemcpyAsync(db->s_m2consts.p, h.data(), B * sizeof(M2Consts), cudaMemcpyHostToDevice, st));
  const uint64_t warps = (uint64_t)B * db->d1p;
  zp_clear_pending_error();
  ctx->launches++;
  k_combine<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(
      dK, dT, B, db->d1p, static_cast<const M2Consts*>(db->s_m2consts.p), dOut);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

extern "C" int zp_client_powm(const zp_client* cl, const uint32_t* dBase, const uint32_t* hExp,
                              uint32_t expWords, uint32_t* dOut, uint32_t count, void* stream) {
  if (!cl || !hExp || ((!dBase || !dOut) && count))
    return zp_set_error(ZP_EINVAL, "zp_client_powm: null argument");
  if (expWords == 0 || expWords > 128)
    return zp_set_error(ZP_EINVAL, "zp_client_powm: expWords=%u out of [1, 128]", expWords);
  if ((reinterpret_cast<uintptr_t>(dBase) | reinterpret_cast<uintptr_t>(dOut)) & 15u)
    return zp_set_error(ZP_EINVAL, "zp_client_powm: dBase and dOut must be 16-byte aligned");
  if (count == 0) return ZP_OK;
  ZP_ON_DEVICE(cl->device);
  PowExp e{};
  for (uint32_t i = 0; i < expWords; ++i) e.w[i] = hExp[i];
  zp_clear_pending_error();
  cl->ctx->launches++;
  k_powm<<<(count + 3) / 4, 128, 0, static_cast<cudaStream_t>(stream)>>>(dBase, e, expWords, count,
                                                                          client_consts(cl), dOut);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

int zp_launch_decrypt(const zp_client* cl, const uint32_t* e, uint32_t ew, const uint32_t* minv,
                      const uint32_t* dC, uint32_t* dOut, uint32_t count, cudaStream_t st) {
  PowExp pe{};
  for (uint32_t i = 0; i < ew; ++i) pe.w[i] = e[i];
  MinvArg mi;
  for (int i = 0; i < ZP_MAX_L; ++i) mi.w[i] = minv[i];
  zp_clear_pending_error();
  cl->ctx->launches++;
  k_decrypt<<<(count + 3) / 4, 128, 0, st>>>(dC, pe, ew, mi, count, client_consts(cl), dOut);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

extern "C" int zp_client_expand_ckr(const zp_client* cl, const uint8_t* hKey, const uint8_t* hNonce,
                                    uint32_t counter0, uint32_t* dOut, uint32_t count, void* stream) {
  if (!cl || !hKey || !hNonce || (!dOut && count))
    return zp_set_error(ZP_EINVAL, "zp_client_expand_ckr: null argument");
  if (reinterpret_cast<uintptr_t>(dOut) & 15u)
    return zp_set_error(ZP_EINVAL, "zp_client_expand_ckr: dOut must be 16-byte aligned");
  if (count == 0) return ZP_OK;
  const uint64_t last_block = ((uint64_t)count * CKR_W - 1) / 16 + 1;  // lanes may make one more
  if ((uint64_t)counter0 + last_block > 0xFFFFFFFFull)
    return zp_set_error(ZP_EINVAL, "zp_client_expand_ckr: the 32-bit block counter would wrap");
  ZP_ON_DEVICE(cl->device);
  const ChachaKey k = chacha_key_from_bytes(hKey, hNonce);
  zp_clear_pending_error();
  cl->ctx->launches++;
  k_expand_ckr<<<(count + 3) / 4, 128, 0, static_cast<cudaStream_t>(stream)>>>(k, counter0, count,
                                                                               client_consts(cl), dOut);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}
