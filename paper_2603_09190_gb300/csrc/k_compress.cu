// k_compress.cu -- answer compression (Algorithm "ZipPIR", Response, second line, with
// the batched packing of Sec. 3.3 / Sec. 4.3):
//   t[b][r'] = ( sum_{j<ell} gamma^j ( ans[b][r' ell + j] + V[b][r' ell + j] ) ) mod m_b,
//   V[b][row] = sum_{i<n} H[row][i] * cko[b][i]           (exact, < 2^(32 L + 42)),
// with H = -D.A mod 2^32. Since H'[r', i] = sum_j gamma^j H[r' ell + j][i], this equals
// (b'[r'] + sum_i H'[r', i] cko[i]) mod m without ever forming the ~2000-bit packed
// hint: the wide products are taken per answer row and packed afterwards.
//
// Three kernels:
//  * k_vmul_simt: V on CUDA cores, one thread per (row, limb of cko), 96-bit
//    column accumulators, then one carry-propagation pass per row;
//  * k_pack_reduce: one warp per (query, packed row): the ell rows of V are staged
//    in shared memory, then Horner evaluation
//    X = (..((W_{ell-1}) gamma + W_{ell-2}) gamma + ..) gamma + W_0 with
//    W_j = ans + V of row r' ell + j (X < 2^4096) in registers; the high words of X are
//    folded with the client's table of 2^(32 w) mod m (Z = X mod 2^(32 L) + sum_w X_w
//    (2^(32 w) mod m) < 2^2087, Z == X mod m), then Barrett reduction mod m (Barrett,
//    CRYPTO '86; the quotient-estimate form of the Handbook of Applied Cryptography, Alg.
//    14.42) with the per-client constant mu = floor(2^(64 L) / m) on 2-3 quotient words.
//    Big integers live in shared memory; products are summed per output column in
//    96-bit accumulators and carries are resolved across the warp with a
//    generate/propagate ballot (one integer addition over the 32 lane flags);
//  * k_mod_packed (the residue-number-system path of large batches): the packed rows'
//    CRT sums V < 2^2087 mod m, the quotient (< 2^40) estimated from the top words of V and
//    of mu, one product q m and at most two subtractions.
#include <atomic>

#include "zp_internal.cuh"
#include "zp_warpint.cuh"

namespace {

constexpr int VW = ZP_VW;  // words of V per row

// ------------------------------------------------------------------ 96-bit MAC
__device__ __forceinline__ void mac96(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t a,
                                      uint32_t b) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(c0), "+r"(c1), "+r"(c2)
      : "r"(a), "r"(b));
}

// ------------------------------------------------------------------ V on CUDA cores
// grid (ceil(R/4), B), block 256 = 4 rows x 64 limbs.
__global__ void __launch_bounds__(256)
    k_vmul_simt(const uint32_t* __restrict__ hneg, uint32_t R, uint32_t Rp, uint32_t n,
                const uint32_t* __restrict__ cko, uint32_t* __restrict__ V) {
  __shared__ uint32_t S[4][ZP_MAX_L][3];
  const uint32_t b = blockIdx.y;
  const uint32_t rr = threadIdx.x >> 6, l = threadIdx.x & 63;
  const uint32_t row = blockIdx.x * 4 + rr;
  uint32_t c0 = 0, c1 = 0, c2 = 0;
  if (row < R) {
    const uint32_t* h = hneg + (uint64_t)row * n;
    const uint32_t* ck = cko + (uint64_t)b * n * ZP_MAX_L + l;
    for (uint32_t i = 0; i < n; ++i) mac96(c0, c1, c2, __ldg(h + i), __ldg(ck + (uint64_t)i * ZP_MAX_L));
  }
  S[rr][l][0] = c0;
  S[rr][l][1] = c1;
  S[rr][l][2] = c2;
  __syncthreads();
  if (l == 0 && row < R) {
    // word w = S[w].lo + S[w-1].mid + S[w-2].hi + carry
    uint32_t* out = V + ((uint64_t)b * Rp + row) * VW;
    uint64_t carry = 0;
    for (int w = 0; w < VW; ++w) {
      uint64_t s = carry;
      if (w < ZP_MAX_L) s += S[rr][w][0];
      if (w >= 1 && w - 1 < ZP_MAX_L) s += S[rr][w - 1][1];
      if (w >= 2 && w - 2 < ZP_MAX_L) s += S[rr][w - 2][2];
      out[w] = (uint32_t)s;
      carry = s >> 32;
    }
  }
}

// Column sums of the product a (na words) x b (nb words) for output words [w_lo, nw):
// col[w] = sum_{i+j=w} a[i] b[j] as three 32-bit words (exact: < 2^96); columns below
// w_lo are set to zero. Lanes take output words in a strided pattern, which balances the
// triangular column lengths.
__device__ __forceinline__ void warp_mul_cols(const uint32_t* a, int na, const uint32_t* b, int nb,
                                              uint32_t (*col)[3], int nw, int w_lo = 0) {
  for (int w = (int)lane_id(); w < nw; w += 32) {
    uint32_t c0 = 0, c1 = 0, c2 = 0;
    if (w < w_lo) {
      col[w][0] = col[w][1] = col[w][2] = 0u;
      continue;
    }
    const int i0 = w - (nb - 1) > 0 ? w - (nb - 1) : 0;
    const int i1 = w < na - 1 ? w : na - 1;
    // two independent carry chains (even and odd terms) for instruction-level parallelism
    uint32_t d0 = 0, d1 = 0, d2 = 0;
    int i = i0;
    for (; i + 1 <= i1; i += 2) {
      mac96(c0, c1, c2, a[i], b[w - i]);
      mac96(d0, d1, d2, a[i + 1], b[w - i - 1]);
    }
    if (i <= i1) mac96(c0, c1, c2, a[i], b[w - i]);
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, %5;"
        : "+r"(c0), "+r"(c1), "+r"(c2)
        : "r"(d0), "r"(d1), "r"(d2));
    col[w][0] = c0;
    col[w][1] = c1;
    col[w][2] = c2;
  }
}

// Gathers normalized words [0, WPL*32) of a product whose columns [0, nw) are in col.
template <int WPL>
__device__ __forceinline__ void warp_cols_to_words(const uint32_t (*col)[3], int nw,
                                                   uint32_t (&w)[WPL]) {
  const uint32_t lane = lane_id();
  uint64_t v[WPL];
#pragma unroll
  for (int t = 0; t < WPL; ++t) {
    const int x = (int)lane * WPL + t;
    uint64_t s = 0;
    if (x < nw) s += col[x][0];
    if (x >= 1 && x - 1 < nw) s += col[x - 1][1];
    if (x >= 2 && x - 2 < nw) s += col[x - 2][2];
    v[t] = s;
  }
  warp_normalize<WPL>(v, w);
}

struct PackBarrett {
  uint32_t X[ZP_XW];        // the packed sum before reduction (< 2^4096)
  uint32_t ans[64];         // the ell (< 64) answers of the packed row
  uint32_t col[160][3];     // product columns
  uint32_t q1[ZP_MAX_L + 1];
  uint32_t q3[ZP_MAX_L + 1];
  uint32_t m[ZP_MAX_L + 1];
  uint32_t mu[ZP_MAX_L + 1];
};

constexpr int PACK_WARPS = 4;

struct ClientPtrs {
  const uint32_t* m;
  const uint32_t* mu;
  const uint32_t* mkm;  // RNS: M_k mod m (ZP_RNS_K x L), then m - (M mod m)
  const uint32_t* pw;   // 2^(32 w) mod m, w = L .. 2L - 1
};

// grid (ceil(d1p / PACK_WARPS), B), block PACK_WARPS warps, dynamic shared memory
// PACK_WARPS x (PackBarrett + ell x VW words). Requires L == ZP_MAX_L.
// V is [b][Rp][VW] words, the exact products V[row] = H[row,:] . cko[b] of every answer
// row, packed with the answers (W_j = ans + V). ans = NULL packs V alone: T then holds Y =
// (sum_j gamma^j V_j) mod m, which k_pack_ans completes once the answers exist.
__global__ void __launch_bounds__(PACK_WARPS * 32)
    k_pack_reduce(const uint32_t* __restrict__ ans, const uint32_t* __restrict__ V, uint32_t R,
                  uint32_t Rp, uint32_t ell, uint32_t d1p, uint32_t g1, uint32_t g2,
                  const ClientPtrs* __restrict__ cl, uint32_t* __restrict__ T) {
  extern __shared__ __align__(16) uint32_t pack_smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t b = blockIdx.y;
  const uint32_t rp = blockIdx.x * PACK_WARPS + warp;
  if (rp >= d1p) return;
  const uint32_t per_warp = (uint32_t)(sizeof(PackBarrett) / 4) + ell * VW;
  PackBarrett& S = *reinterpret_cast<PackBarrett*>(pack_smem + warp * per_warp);
  uint32_t* Vs = pack_smem + warp * per_warp + sizeof(PackBarrett) / 4;  // ell x VW
  constexpr int L = ZP_MAX_L;

  // ---- stage the rows r' ell .. r' ell + ell - 1 of V (contiguous) and the client constants
  const uint32_t row0 = rp * ell;
  const uint32_t nrows = R - row0 < ell ? R - row0 : ell;
  const uint32_t* src = V + ((uint64_t)b * Rp + row0) * VW;
  {
    // sixteen loads in flight per lane before the stores (the rows come from L2)
    const uint32_t tot = nrows * VW;
    for (uint32_t base = 0; base < tot; base += 32 * 16) {
      uint32_t v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const uint32_t idx = base + 32u * u + lane;
        v[u] = idx < tot ? __ldg(src + idx) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const uint32_t idx = base + 32u * u + lane;
        if (idx < tot) Vs[idx] = v[u];
      }
    }
  }
  for (int x = lane; x < L + 1; x += 32) {
    S.m[x] = x < L ? cl[b].m[x] : 0u;
    S.mu[x] = cl[b].mu[x];
  }
  const uint32_t* ansb = ans ? ans + (uint64_t)b * R + row0 : nullptr;
  for (uint32_t j = lane; j < nrows; j += 32) S.ans[j] = ans ? __ldg(ansb + j) : 0u;
  __syncwarp();

  // ---- Horner: X <- X gamma + W_j (j = ell-1 .. 0), gamma = g1 2^32 + g2 2^64,
  // W_j = ans[row] + V[row]. X is kept with lazy carries: four 64-bit words per lane
  // (words 4 lane .. 4 lane + 3), each below 2^33, so one step needs a local carry
  // pass and one shuffle instead of a full carry resolution.
  uint64_t xv[4] = {0, 0, 0, 0};
  for (int j = (int)nrows - 1; j >= 0; --j) {
    const uint64_t pm1 = __shfl_up_sync(0xffffffffu, xv[3], 1);  // word 4 lane - 1
    const uint64_t pm2 = __shfl_up_sync(0xffffffffu, xv[2], 1);  // word 4 lane - 2
    const uint64_t xm1 = lane ? pm1 : 0, xm2 = lane ? pm2 : 0;
    const uint32_t* Wj = Vs + (uint32_t)j * VW;
    uint64_t v[4];
    v[0] = (uint64_t)g1 * xm1 + (uint64_t)g2 * xm2;
    v[1] = (uint64_t)g1 * xv[0] + (uint64_t)g2 * xm1;
    v[2] = (uint64_t)g1 * xv[1] + (uint64_t)g2 * xv[0];
    v[3] = (uint64_t)g1 * xv[2] + (uint64_t)g2 * xv[1];
    {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const uint32_t x = lane * 4 + t;
        if (x < VW) v[t] += Wj[x];
      }
    }
    if (lane == 0) v[0] += S.ans[j];
    uint64_t c = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint64_t sum = v[t] + c;
      xv[t] = sum & 0xFFFFFFFFull;
      c = sum >> 32;
    }
    const uint64_t cin = __shfl_up_sync(0xffffffffu, c, 1);
    if (lane) xv[0] += cin;
  }
  // final carry resolution, then X to shared memory
  {
    uint32_t w[4];
    warp_normalize<4>(xv, w);
#pragma unroll
    for (int t = 0; t < 4; ++t) S.X[lane * 4 + t] = w[t];
  }
  __syncwarp();
  {
    // X < 2^(64 L) (2L words; 4077 bits for the binary secret at n = 48): fold its high words
    // with the client's table, Z = (X mod 2^(32 L)) + sum_{w = L}^{2L - 1} X_w (2^(32 w) mod m)
    // == X (mod m), Z < 2^2087, so the Barrett reduction below works on 2-3 quotient words.
    // Lane l sums the columns 2l, 2l+1 (96-bit accumulators; the L table rows are coalesced
    // loads).
    const uint32_t* pw = cl[b].pw;
    uint32_t a0 = S.X[2 * lane], a1 = 0, a2 = 0, b0 = S.X[2 * lane + 1], b1 = 0, b2 = 0;
#pragma unroll 8
    for (int w = L; w < 2 * L; ++w) {
      const uint32_t x = S.X[w];
      const uint2 t = __ldg(reinterpret_cast<const uint2*>(pw + (size_t)(w - L) * L) + lane);
      mac96(a0, a1, a2, x, t.x);
      mac96(b0, b1, b2, x, t.y);
    }
    S.col[2 * lane][0] = a0;
    S.col[2 * lane][1] = a1;
    S.col[2 * lane][2] = a2;
    S.col[2 * lane + 1][0] = b0;
    S.col[2 * lane + 1][1] = b1;
    S.col[2 * lane + 1][2] = b2;
    __syncwarp();
    uint32_t zw[3];  // words 3 lane .. 3 lane + 2 of Z
    warp_cols_to_words<3>(S.col, L, zw);  // the L columns above (words up to L + 1)
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 3; ++t) S.X[lane * 3 + t] = zw[t];
    S.X[96 + lane] = 0u;
  }
  __syncwarp();

  // ---- Barrett: q1 = floor(X / b^(L-1)), q3 = floor(q1 mu / b^(L+1)),
  //      r = (X mod b^(L+1)) - (q3 m mod b^(L+1)), then r -= m while r >= m.
  for (int x = lane; x < L + 1; x += 32) S.q1[x] = S.X[L - 1 + x];
  __syncwarp();
  // significant words of an (L+1)-word integer in shared memory (q1 and q3 are short when X
  // is far below b^(2L), as the RNS sums are: < 2^2083)
  auto sig_words = [&](const uint32_t* a) {
    int top = -1;
    for (int x = lane; x < L + 1; x += 32)
      if (a[x]) top = x;
#pragma unroll
    for (int o = 16; o; o >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
    return top + 1 > 1 ? top + 1 : 1;
  };
  const int n1 = sig_words(S.q1);
  // Only the columns from L - 1 up are summed (Handbook of Applied Cryptography, Note
  // 14.44): the dropped lower part is below L b^L, so the quotient estimate below is at
  // most one short of floor(q1 mu / b^(L+1)), r stays below 4m, and the correction loop's
  // three subtractions still end with r < m.
  warp_mul_cols(S.q1, n1, S.mu, L + 1, S.col, 2 * L + 1, L - 1);
  __syncwarp();
  {
    uint32_t w[5];  // words 0..159 of q1 * mu; q3 = words L+1 .. 2L+1
    warp_cols_to_words<5>(S.col, 2 * L + 1, w);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const int x = (int)lane * 5 + t;
      if (x >= L + 1 && x < 2 * L + 2) S.q3[x - (L + 1)] = w[t];
    }
  }
  __syncwarp();
  warp_mul_cols(S.q3, sig_words(S.q3), S.m, L, S.col, L + 1);
  __syncwarp();
  uint32_t r[3], r2[3], mm[3];
  warp_cols_to_words<3>(S.col, L + 1, r2);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int x = (int)lane * 3 + t;
    r2[t] = x < L + 1 ? r2[t] : 0u;
    r[t] = x < L + 1 ? S.X[x] : 0u;
    mm[t] = x < L ? S.m[x] : 0u;
  }
  warp_sub<3>(r, r2);
#pragma unroll
  for (int t = 0; t < 3; ++t)
    if ((int)lane * 3 + t >= L + 1) r[t] = 0u;  // mod b^(L+1)
  for (int it = 0; it < 3; ++it) {
    if (!warp_geq<3>(r, mm)) break;
    warp_sub<3>(r, mm);
  }
  uint32_t* out = T + ((uint64_t)b * d1p + rp) * L;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int x = (int)lane * 3 + t;
    if (x < L) out[x] = r[t];
  }
}

// The second half of a split packing (one query answered by the GEMV while its products run
// beside it): t = (b' + Y) mod m with b' = sum_{j<ell} gamma^j ans[r' ell + j] and Y = (sum_j
// gamma^j V_j) mod m from k_pack_reduce (ans = NULL) on the products' stream. The context
// picks ell with (bound - 1) sum_{j<ell} gamma^j < 2^(key_bits - 1) (the batching bound), and
// every answer is below 2^32 <= bound - 1, so b' < 2^(key_bits - 1) <= m: b' + Y < 2m and one
// conditional subtraction of m ends the reduction (a carry out of word L - 1 counts as >= m).
// b' is summed column by column from the context's table of gamma^j (ell rows of L words):
// lane l keeps the 96-bit sums of words 2l and 2l + 1, with the table rows fetched nine at a
// time ahead of their multiply-adds; the columns are then gathered into 32-bit words with one
// carry resolution (every term is nonnegative and b' < 2^(32 L - 1), so the parts of lane 31
// above word L - 1 are zero). One warp per (query, packed row).
constexpr uint32_t PACKA_WARPS = 8;
__global__ void __launch_bounds__(PACKA_WARPS * 32)
    k_pack_ans(const uint32_t* __restrict__ ans, uint32_t R, uint32_t ell, uint32_t d1p,
               const uint32_t* __restrict__ gam, const uint32_t* __restrict__ Y,
               const ClientPtrs* __restrict__ cl, uint32_t* __restrict__ T) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t rp = blockIdx.x * PACKA_WARPS + (threadIdx.x >> 5), b = blockIdx.y;
  if (rp >= d1p) return;
  constexpr int L = ZP_MAX_L;
  static_assert(L == 64, "two words per lane");
  const uint32_t row0 = rp * ell;
  const uint32_t nrows = R - row0 < ell ? R - row0 : ell;
  const uint32_t* ansb = ans + (uint64_t)b * R + row0;
  const uint32_t an0 = lane < nrows ? __ldg(ansb + lane) : 0u;  // ell <= 64
  const uint32_t an1 = lane + 32 < nrows ? __ldg(ansb + lane + 32) : 0u;
  const uint2 y = __ldg(reinterpret_cast<const uint2*>(Y + ((uint64_t)b * d1p + rp) * L) + lane);
  const uint2 mv = __ldg(reinterpret_cast<const uint2*>(cl[b].m) + lane);
  uint32_t c0 = 0, c1 = 0, c2 = 0, d0 = 0, d1 = 0, d2 = 0;
  const uint2* g2 = reinterpret_cast<const uint2*>(gam) + lane;
  constexpr uint32_t U = 9;
  for (uint32_t j0 = 0; j0 < nrows; j0 += U) {
    uint2 t[U];
#pragma unroll
    for (uint32_t u = 0; u < U; ++u)
      t[u] = j0 + u < nrows ? __ldg(g2 + (size_t)(j0 + u) * (L / 2)) : make_uint2(0u, 0u);
#pragma unroll
    for (uint32_t u = 0; u < U; ++u) {
      const uint32_t j = j0 + u;
      const uint32_t aj = __shfl_sync(0xffffffffu, j < 32 ? an0 : an1, j & 31);
      mac96(c0, c1, c2, aj, t[u].x);
      mac96(d0, d1, d2, aj, t[u].y);
    }
  }
  const uint32_t pm = __shfl_up_sync(0xffffffffu, d1, 1), ph = __shfl_up_sync(0xffffffffu, c2, 1),
                 ph1 = __shfl_up_sync(0xffffffffu, d2, 1);
  uint64_t v[2];
  v[0] = (uint64_t)c0 + (lane ? (uint64_t)pm + ph : 0u) + y.x;
  v[1] = (uint64_t)d0 + c1 + (lane ? (uint64_t)ph1 : 0u) + y.y;
  uint32_t w[2];
  const uint32_t top = warp_normalize_top<2>(v, w);
  const uint32_t mm[2] = {mv.x, mv.y};
  if (top || warp_geq<2>(w, mm)) warp_sub<2>(w, mm);
  reinterpret_cast<uint2*>(T + ((uint64_t)b * d1p + rp) * L)[lane] = make_uint2(w[0], w[1]);
}


// Residue-number-system path, last step (Sec. 5.2: one reduction mod m at the end): T = V mod
// m for the CRT sums V < 2^2087 (ZP_VW words, [b][Rq][ZP_VW]) of the packed rows. The
// quotient q = floor(V / m) is below 2^40 and comes from the top words alone: with the
// client's Barrett constant mu = floor(2^4096 / m), mu_t = floor(mu / 2^1985) (64 bits) and
// V_t = floor(V / 2^1984) (< 2^103), q_e = floor(V_t mu_t / 2^127) is at most q (every factor
// is rounded down) and at least q - 2 (the dropped parts are below V / 2^2111 + mu / 2^2112
// < 2^-23 of a unit, plus the floors), so r = V - q_e m is below 3m and two conditional
// subtractions of m end below m. One warp per (query, packed row); lane l holds words 3 l ..
// 3 l + 2. Requires L == ZP_MAX_L == 64.
constexpr uint32_t MODP_WARPS = 8;
__global__ void __launch_bounds__(MODP_WARPS * 32)
    k_mod_packed(const uint32_t* __restrict__ V, uint32_t Rq, uint32_t d1p,
                 const ClientPtrs* __restrict__ cl, uint32_t* __restrict__ T) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t rp = blockIdx.x * MODP_WARPS + (threadIdx.x >> 5), b = blockIdx.y;
  if (rp >= d1p) return;
  constexpr int L = ZP_MAX_L;
  static_assert(L == 64 && ZP_VW <= 96, "2048-bit moduli, V within the warp's 96 words");
  const uint32_t* Vr = V + ((uint64_t)b * Rq + rp) * ZP_VW;
  const uint32_t* m = cl[b].m;
  const uint32_t* mu = cl[b].mu;
  uint32_t v[3], mm[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const uint32_t x = 3 * lane + t;
    v[t] = x < (uint32_t)ZP_VW ? __ldg(Vr + x) : 0u;
    mm[t] = x < (uint32_t)L ? __ldg(m + x) : 0u;
  }
  // V_t = words 62..65 of V (lanes 20 and 21), mu_t from words 62..64 of mu
  const uint32_t w62 = __shfl_sync(0xffffffffu, v[2], 20), w63 = __shfl_sync(0xffffffffu, v[0], 21);
  const uint32_t w64 = __shfl_sync(0xffffffffu, v[1], 21), w65 = __shfl_sync(0xffffffffu, v[2], 21);
  const uint64_t mut = ((uint64_t)__ldg(mu + 64) << 63) | ((uint64_t)__ldg(mu + 63) << 31) |
                       (uint64_t)(__ldg(mu + 62) >> 1);
  const uint64_t vh = ((uint64_t)w65 << 32) | w64, vl = ((uint64_t)w63 << 32) | w62;
  // bits 127.. of (vh 2^64 + vl) mu_t
  const uint64_t a1 = __umul64hi(vl, mut), b0 = vh * mut, b1 = __umul64hi(vh, mut);
  const uint64_t s1 = a1 + b0, s2 = b1 + (s1 < a1 ? 1u : 0u);
  const uint64_t q = (s2 << 1) | (s1 >> 63);  // < 2^40
  const uint32_t ql = (uint32_t)q, qh = (uint32_t)(q >> 32);
  // q m as 64-bit columns (each < 2^41): word j gets lo(ql m_j) + hi(ql m_{j-1}) + qh m_{j-1}
  const uint32_t mprev = __shfl_up_sync(0xffffffffu, mm[2], 1);
  uint64_t col[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const uint32_t mj1 = t ? mm[t - 1] : (lane ? mprev : 0u);
    col[t] = (((uint64_t)ql * mm[t]) & 0xFFFFFFFFull) + (((uint64_t)ql * mj1) >> 32) +
             (uint64_t)qh * mj1;
  }
  uint32_t qm[3];
  warp_normalize<3>(col, qm);
  warp_sub<3>(v, qm);
  for (int it = 0; it < 2; ++it) {
    if (!warp_geq<3>(v, mm)) break;
    warp_sub<3>(v, mm);
  }
  uint32_t* out = T + ((uint64_t)b * d1p + rp) * L;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const uint32_t x = 3 * lane + t;
    if (x < (uint32_t)L) out[x] = v[t];
  }
}

// Residue-number-system path, step 1 of the reduction (Sec. 5.2): from the residues
// X[b][k][r'] = H'[r', :] . cko[b] mod p_k (row pitch Rq), y_k = X_k (M/p_k)^{-1} mod p_k
// and alpha = floor(sum_k y_k / p_k), so that H'.cko = sum_k y_k M/p_k - alpha M. The sum is taken in
// 64.64 fixed point with integer arithmetic only: S = sum_k y_k floor(2^64 / p_k) (128-bit
// accumulators) is below 2^64 sum_k y_k / p_k by less than 153 2^27 < 2^34.3 units, and
// H'.cko < M 2^-26 puts the fractional part of sum_k y_k / p_k in [0, 2^-26), so
// floor((S + 2^35) / 2^64) = alpha exactly. y_k = X_k inv_k mod p_k by two pseudo-Mersenne
// folds (p = 2^27 - dl, dl < 2^12). Written as the byte planes of the CRT product's A
// operand: row b Rq + r' holds, at byte a kpl + k (kpl = ypitch / 4, a multiple of 64), byte
// a of y_k in column k < ZP_RNS_K and of alpha in column ZP_RNS_K; columns ZP_RNS_K + 1 + j
// (j < ell) hold the answers ans[b][r' ell + j] (zero past R), which the CRT product weighs by
// gamma^j: the packed answer b'; columns past that and packed rows r' in [d1', Rq) are zero.
// yrs[(4 b + a) Rq + r']: the byte sums of plane a. One warp per (query, packed row < Rq).
constexpr uint32_t CRT_PREP_ROWS = 8;  // warps (packed rows) per block of k_crt_prep
__global__ void k_crt_prep(const uint32_t* __restrict__ X, uint32_t B, uint32_t d1p, uint32_t Rq,
                           const zp_rns_dev* __restrict__ rns, uint8_t* __restrict__ Yp,
                           uint32_t ypitch, uint32_t* __restrict__ yrs,
                           const uint32_t* __restrict__ ans, uint32_t R, uint32_t ell) {
  // A block is CRT_PREP_ROWS warps on consecutive packed rows of one query (Rq is a multiple
  // of 32): their residues X[b][k][rp0 ..] come in as one 32-byte sector per prime, through
  // shared memory (pitch 9: the warps' column reads are conflict-free).
  __shared__ uint32_t xs[ZP_RNS_K * (CRT_PREP_ROWS + 1)];
  const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t wid0 = (uint64_t)blockIdx.x * CRT_PREP_ROWS;
  if (wid0 >= (uint64_t)B * Rq) return;  // whole blocks only
  const uint32_t b = (uint32_t)(wid / Rq), rp = (uint32_t)(wid % Rq);
  {
    const uint32_t b0 = (uint32_t)(wid0 / Rq), rp0 = (uint32_t)(wid0 % Rq);
    const uint32_t* X0 = X + (uint64_t)b0 * ZP_RNS_K * Rq + rp0;  // X[b][k][rp], row pitch Rq
    for (uint32_t i = threadIdx.x; i < ZP_RNS_K * CRT_PREP_ROWS; i += blockDim.x) {
      const uint32_t k = i / CRT_PREP_ROWS, j = i % CRT_PREP_ROWS;
      xs[k * (CRT_PREP_ROWS + 1) + j] = rp0 + j < d1p ? __ldg(X0 + (uint64_t)k * Rq + j) : 0u;
    }
    __syncthreads();
  }
  constexpr int QK = (ZP_RNS_K + 1 + 64 + 31) / 32;  // residues, alpha, up to 64 answers
  uint32_t y[QK];
  uint64_t s_lo = 0, s_hi = 0;  // 128-bit sum of y_k floor(2^64 / p_k)
#pragma unroll
  for (int q = 0; q < QK; ++q) {
    const uint32_t k = lane + 32u * q;
    y[q] = 0u;
    if (rp < d1p && k < ZP_RNS_K) {
      const uint32_t p = rns->p[k], dl = (1u << 27) - p;
      const uint64_t x = (uint64_t)xs[k * (CRT_PREP_ROWS + 1) + w] * rns->inv[k];  // < 2^54
      const uint64_t t1 = (x & 0x7FFFFFFull) + (x >> 27) * dl;             // < 2^40
      uint32_t v = (uint32_t)((t1 & 0x7FFFFFFull) + (t1 >> 27) * dl);       // < 2^27 + 2^25
      if (v >= p) v -= p;
      y[q] = v;
      const uint64_t r = rns->mu[k];  // floor((2^64 - 1) / p) = floor(2^64 / p) (p odd)
      const uint64_t prod = (uint64_t)v * r;  // v < p: v floor(2^64 / p) < 2^64, no high word
      s_lo += prod;
      s_hi += s_lo < prod ? 1u : 0u;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const uint64_t olo = __shfl_xor_sync(0xffffffffu, s_lo, o);
    const uint64_t ohi = __shfl_xor_sync(0xffffffffu, s_hi, o);
    s_lo += olo;
    s_hi += ohi + (s_lo < olo ? 1u : 0u);
  }
  constexpr uint32_t KA = ZP_RNS_K;  // column of alpha
  if (rp < d1p && lane == KA % 32)
    y[KA / 32] = (uint32_t)(s_hi + ((s_lo + (1ull << 35)) < s_lo ? 1u : 0u));
  const uint32_t KE = KA + ell;  // column of answer ell - 1
#pragma unroll
  for (int q = 0; q < QK; ++q) {
    const uint32_t k = lane + 32u * q;
    if (k > KA && k <= KE) {
      const uint64_t r = (uint64_t)rp * ell + (k - KA - 1);
      y[q] = (rp < d1p && r < R) ? __ldg(ans + (uint64_t)b * R + r) : 0u;
    }
  }
  // Byte plane a of column k goes to byte a kpl + k of row b Rq + rp (planes of kpl = ypitch
  // / 4 bytes, the tail of each plane zero). Four lanes (k = 4 g .. 4 g + 3 of a block of 32)
  // trade bytes in two shuffle rounds so that lane 4 g + a holds the four plane-a bytes and
  // stores them as one word; the byte sums per plane are summed over the lanes of the plane.
  const uint32_t kpl = ypitch / 4, pa = lane & 3u;
  uint8_t* dst = Yp + ((uint64_t)b * Rq + rp) * ypitch + (uint64_t)pa * kpl;
  uint32_t sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (32u * q >= kpl) break;
    const uint32_t x = q < QK ? y[q] : 0u;
    const uint32_t p1 = __shfl_xor_sync(0xffffffffu, x, 1);
    const uint32_t w1 = (lane & 1u) ? __byte_perm(x, p1, 0x3715) : __byte_perm(x, p1, 0x6240);
    const uint32_t p2 = __shfl_xor_sync(0xffffffffu, w1, 2);
    const uint32_t w2 = (lane & 2u) ? __byte_perm(p2, w1, 0x7632) : __byte_perm(w1, p2, 0x5410);
    *reinterpret_cast<uint32_t*>(dst + 32u * q + 4u * (lane >> 2)) = w2;
    sum += __dp4a(w2, 0x01010101u, 0u);
  }
  sum += __shfl_xor_sync(0xffffffffu, sum, 4);
  sum += __shfl_xor_sync(0xffffffffu, sum, 8);
  sum += __shfl_xor_sync(0xffffffffu, sum, 16);
  if (lane < 4) yrs[((uint64_t)b * 4 + lane) * Rq + rp] = sum;
}

}  // namespace

int zp_launch_compress_products(zp_db* db, const uint32_t* dCKO, uint32_t B, cudaStream_t st,
                                uint32_t max_ctas) {
  zp_ctx* ctx = db->ctx;
  const uint32_t R = db->R, n = ctx->P.n;
  if ((ctx->compress_path == ZP_PATH_TC || ctx->compress_path == ZP_PATH_RNS) && n > 1024)
    return zp_set_error(ZP_EUNSUPPORTED, "tensor-core compression needs n <= 1024");
  // large batches: residues of H'.cko modulo the RNS primes (the packed hint is read once
  // per batch and there are ell times fewer rows); otherwise exact per-row products V
  const bool rns = n <= 1024 && (reinterpret_cast<uintptr_t>(dCKO) & 15u) == 0 &&
                   (ctx->compress_path == ZP_PATH_RNS ||
                    (ctx->compress_path == ZP_PATH_AUTO && ctx->rns_min_batch &&
                     B >= ctx->rns_min_batch));
  if (rns) {
    int rc = zp_ensure_rns(db, st);
    if (!rc) rc = zp_scratch_reserve(&db->s_v, (size_t)B * ZP_RNS_K * db->Rq * sizeof(uint32_t));
    if (!rc) rc = zp_launch_rns_products(db, dCKO, B, static_cast<uint32_t*>(db->s_v.p), st);
    if (rc) return rc;
    db->v_batch = B;
    db->v_rns = true;
    return ZP_OK;
  }
  const bool tc = ctx->compress_path != ZP_PATH_SIMT && n <= 1024;
  int rc = zp_scratch_reserve(&db->s_v, (size_t)B * db->Rp * VW * sizeof(uint32_t));
  if (rc) return rc;
  uint32_t* V = static_cast<uint32_t*>(db->s_v.p);
  if (tc) {
    rc = zp_launch_vmul_tc(db, dCKO, B, V, st, max_ctas);
    if (rc) return rc;
  } else {
    dim3 grid((R + 3) / 4, B);
    zp_clear_pending_error();
    ctx->launches++;
    k_vmul_simt<<<grid, 256, 0, st>>>(db->d_hneg, R, db->Rp, n, dCKO, V);
    ZP_CUDA(cudaGetLastError());
  }
  db->v_batch = B;
  db->v_rns = false;
  return ZP_OK;
}

// The per-query client constants as a device array (db->s_clients), uploaded on `st` only
// when the list changed, and the pack kernel's shared-memory attribute.
static int upload_clients(zp_db* db, zp_client* const* clients, uint32_t B, cudaStream_t st,
                          ClientPtrs** out) {
  zp_ctx* ctx = db->ctx;
  int rc = zp_scratch_reserve(&db->s_clients, (size_t)B * sizeof(ClientPtrs));
  if (rc) return rc;
  ClientPtrs* dcl = static_cast<ClientPtrs*>(db->s_clients.p);
  // upload the per-query client constants only when the list changed
  bool same = db->cl_cache.size() == 4 * (size_t)B;
  for (uint32_t b = 0; same && b < B; ++b)
    same = db->cl_cache[4 * b] == clients[b]->d_m && db->cl_cache[4 * b + 1] == clients[b]->d_mu &&
           db->cl_cache[4 * b + 2] == clients[b]->d_mkm && db->cl_cache[4 * b + 3] == clients[b]->d_pow;
  if (!same) {
    std::vector<ClientPtrs> h(B);
    db->cl_cache.resize(4 * (size_t)B);
    for (uint32_t b = 0; b < B; ++b) {
      h[b] = ClientPtrs{clients[b]->d_m, clients[b]->d_mu, clients[b]->d_mkm, clients[b]->d_pow};
      db->cl_cache[4 * b] = clients[b]->d_m;
      db->cl_cache[4 * b + 1] = clients[b]->d_mu;
      db->cl_cache[4 * b + 2] = clients[b]->d_mkm;
      db->cl_cache[4 * b + 3] = clients[b]->d_pow;
    }
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    cudaError_t e = cudaMemcpyAsync(dcl, h.data(), B * sizeof(ClientPtrs), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      db->cl_cache.clear();
      return zp_cuda_check(e, "cudaMemcpyAsync(clients)");
    }
  }
  // the attribute is per device; two host threads may both set it, which is harmless
  static std::atomic<bool> attr_dev[64];
  std::atomic<bool>& attr = attr_dev[ctx->device & 63];
  if (!attr) {
    ZP_CUDA(cudaFuncSetAttribute(k_pack_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(PACK_WARPS * (sizeof(PackBarrett) + 64 * VW * 4))));
    attr = true;
  }
  *out = dcl;
  return ZP_OK;
}

int zp_launch_compress_finish(zp_db* db, zp_client* const* clients, const uint32_t* dAns,
                              uint32_t B, uint32_t* dT, cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  if (db->v_batch != B)
    return zp_set_error(ZP_ESTATE, "compression finish for %u queries, products hold %u", B,
                        db->v_batch);
  uint32_t* V = static_cast<uint32_t*>(db->s_v.p);
  ClientPtrs* dcl = nullptr;
  int rc = upload_clients(db, clients, B, st, &dcl);
  if (rc) return rc;
  dim3 grid((db->d1p + PACK_WARPS - 1) / PACK_WARPS, B);
  zp_clear_pending_error();
  ctx->launches++;
  if (db->v_rns) {
    // residues -> y, alpha (byte planes) -> exact CRT sums on the tensor cores -> pack + reduce
    // four planes of K rounded up to 64 bytes (the CRT product takes a plane per K block)
    const uint32_t Rq = db->Rq, ypitch = 4 * ((zp_crt_k(ctx) + 63) / 64 * 64);
    const size_t yp_bytes = (size_t)B * Rq * ypitch, yrs_bytes = (size_t)B * 4 * Rq * 4;
    const size_t vc_bytes = (size_t)B * Rq * VW * 4;
    rc = zp_scratch_reserve(&db->s_crt, yp_bytes + yrs_bytes + vc_bytes + 512);
    if (rc) return rc;
    uint8_t* Yp = static_cast<uint8_t*>(db->s_crt.p);
    uint32_t* yrs = reinterpret_cast<uint32_t*>(Yp + (yp_bytes + 255) / 256 * 256);
    uint32_t* Vc = yrs + (yrs_bytes / 4 + 63) / 64 * 64;
    const uint64_t warps = (uint64_t)B * Rq;
    k_crt_prep<<<(unsigned)(warps / CRT_PREP_ROWS), 32 * CRT_PREP_ROWS, 0, st>>>(
        V, B, db->d1p, Rq, ctx->d_rns, Yp, ypitch, yrs, dAns, db->R, ctx->ell);
    ZP_CUDA(cudaGetLastError());
    // the mkm pointers are the third member of each uploaded ClientPtrs
    rc = zp_launch_crt_products(db, reinterpret_cast<const uint32_t* const*>(dcl) + 2,
                                (uint32_t)(sizeof(ClientPtrs) / sizeof(void*)), B, Yp, ypitch, yrs,
                                Vc, st);
    if (rc) return rc;
    zp_clear_pending_error();
    ctx->launches++;
    k_mod_packed<<<dim3((db->d1p + MODP_WARPS - 1) / MODP_WARPS, B), MODP_WARPS * 32, 0, st>>>(
        Vc, Rq, db->d1p, dcl, dT);
  } else {
    const size_t smem = (size_t)PACK_WARPS * (sizeof(PackBarrett) + (size_t)ctx->ell * VW * 4);
    k_pack_reduce<<<grid, PACK_WARPS * 32, smem, st>>>(dAns, V, db->R, db->Rp, ctx->ell, db->d1p,
                                                       ctx->gamma_w[1], ctx->gamma_w[2], dcl, dT);
  }
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

// Split packing for one query answered beside its products (zp_respond): Y = (sum_j gamma^j
// V_j) mod m on the products' stream, before the answers exist ...
int zp_launch_pack_products(zp_db* db, zp_client* const* clients, uint32_t B, cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  if (db->v_batch != B || db->v_rns)
    return zp_set_error(ZP_ESTATE, "split packing: the products hold another batch");
  ClientPtrs* dcl = nullptr;
  int rc = upload_clients(db, clients, B, st, &dcl);
  if (!rc) rc = zp_scratch_reserve(&db->s_ypack, (size_t)B * db->d1p * ZP_MAX_L * 4);
  if (rc) return rc;
  const size_t smem = (size_t)PACK_WARPS * (sizeof(PackBarrett) + (size_t)ctx->ell * VW * 4);
  zp_clear_pending_error();
  ctx->launches++;
  k_pack_reduce<<<dim3((db->d1p + PACK_WARPS - 1) / PACK_WARPS, B), PACK_WARPS * 32, smem, st>>>(
      nullptr, static_cast<const uint32_t*>(db->s_v.p), db->R, db->Rp, ctx->ell, db->d1p,
      ctx->gamma_w[1], ctx->gamma_w[2], dcl, static_cast<uint32_t*>(db->s_ypack.p));
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

// ... and after the join t = (b' + Y) mod m with the answers (the client array uploaded by
// zp_launch_pack_products, ordered before this launch by the join).
int zp_launch_pack_answers(zp_db* db, const uint32_t* dAns, uint32_t B, uint32_t* dT,
                           cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  zp_clear_pending_error();
  ctx->launches++;
  k_pack_ans<<<dim3((db->d1p + PACKA_WARPS - 1) / PACKA_WARPS, B), PACKA_WARPS * 32, 0, st>>>(
      dAns, db->R, ctx->ell, db->d1p, ctx->d_gam, static_cast<const uint32_t*>(db->s_ypack.p),
      static_cast<const ClientPtrs*>(db->s_clients.p), dT);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}
