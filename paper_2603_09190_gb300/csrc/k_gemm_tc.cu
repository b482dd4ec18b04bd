// k_gemm_tc.cu -- exact integer products of byte matrices on the 5th-generation tensor
// cores (tcgen05.mma kind::f16, fp32 accumulators in tensor memory).
//
//   C[m][n] = sum_k A[m][k] * B[n][k],   A, B with entries in [0, 255].
//
// sm_103a has no integer (kind::i8) tensor-core instruction, so the bytes are fed as
// fp16, which holds every integer of [-2048, 2048] exactly. Both operands are centred,
// A' = A - 128 and B' = B - 128, so that a product is at most 2^14 in magnitude and a
// sum of 1024 of them at most 2^24: every partial sum of a 1024-long K chunk is an
// integer that fp32 represents exactly. The accumulator of each chunk is drained to
// int32, chunks are summed in 32-bit integers, and the centring is undone with
//   sum_k A B = sum_k A'B' + 128 sum_k A + 128 sum_k B - 16384 Kp
// (sums over the zero-padded K range Kp). All integer arithmetic wraps mod 2^32,
// which is exact for the mod-2^32 answers and, for the compression products, never
// wraps because every true value is below 2^31.
//
// Uses (template MODE):
//   MODE_ANS  batched LWE answers, ans[b][r] = sum_c D[r][c] Q[b][c] mod 2^32
//             (Algorithm "ZipPIR", Response, first line): A = D (R x C bytes),
//             B = the 4 byte planes of BT queries (N = 4 BT rows), recombined as
//             sum_a 2^(8a) P_a in the epilogue;
//   MODE_HINT the global hint H+ = D A mod 2^32 (Algorithm "ZipPIR" caption): as
//             MODE_ANS with the columns of A as queries, written row-major R x n;
//   MODE_RES  residues of the compression offsets modulo the RNS primes (Sec. 5.2),
//             cko[b][i] mod p_k = sum_beta byte_beta(cko[b][i]) (2^(8 beta) mod p_k): A = the
//             256 bytes of every cko[b][i] (K = 256), B = the four bytes c of 2^(8 beta) mod
//             p_k for 40 primes per N tile (N = 160); the epilogue folds the four sums S_c
//             of a prime into the residue and writes its bytes as the B operand of MODE_RNS
//             (whose row sums k_fp16_rowsum takes afterwards);
//   MODE_CMP  the compression products V[r] = sum_i H[r][i] cko[i] (Algorithm
//             "ZipPIR", Response, second line): A = the 4 byte planes of the negated
//             hint, rows ordered (32 rows of plane 0, of plane 1, ...), B = the 256
//             bytes of every cko[i] (N = 256), K = n <= 1024; the epilogue turns the
//             256 byte-column sums of a row into a 67-word integer V_a (carry
//             propagation), adds the four planes as V = sum_a V_a 2^(8a) and writes
//             V (67 words per row).
//
// Structure (one CTA per SM, persistent over output tiles of 128 x N):
//   warp 0      TMA producer of A: the A tile as bytes (128 x 64, 8 KiB) into a deep
//               byte ring (its source is HBM);
//   warp 2      TMA producer of B: the B tile as fp16 (N x 64, 128-byte swizzle) into
//               the operand ring;
//   warp 1      allocates 512 TMEM columns (two 256-column accumulators) and one
//               elected lane issues the MMAs (4 x K=16 per K block) and the commits;
//   warps 4-7   epilogue: tcgen05.ld of their 32-lane TMEM quarter, int conversion,
//               chunk accumulation, correction, output;
//   warps 8-11  converters: byte tile -> centred fp16 in the swizzled operand layout.
// Every mbarrier wait is bounded; a wait that gives up raises a CTA-wide abort flag and
// a bit in the context's status word, and every role then leaves its loop.
#include <cuda_fp16.h>

#include <atomic>

#include "zp_internal.cuh"

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int A16_BYTES = BM * BK * 2;       // 16 KiB
constexpr int B_MAX_BYTES = 256 * BK * 2;    // 32 KiB
constexpr int U8_STAGE = BM * 2 * BK;        // 16 KiB: two K blocks of A bytes per copy (128-byte rows)
constexpr int KCHUNK = 16;                   // K blocks per exact fp32 accumulation
constexpr int NTHREADS = 384;
constexpr int STG_PITCH = 67;                // words per staged row (odd: no bank conflicts)
constexpr int STG_BYTES = 4 * 32 * STG_PITCH * 4;

enum { MODE_ANS = 0, MODE_HINT = 1, MODE_CMP = 2, MODE_RNS = 3, MODE_RES = 4, MODE_CRT = 5 };

// Three rings: B (fp16, from L2: deep, it is the largest operand), A as bytes (from
// HBM, L2-prefetched) and A as fp16 (written by the converters just before the MMA).
// A16: A is already centred fp16 in HBM (the resident fp16 copy of D), so TMA fills the
// A ring directly: no byte ring, no converters, and the B stages are sized to the tile (N
// rows). For N <= 128 a stage holds KPS = 2 K blocks (one wait and one commit per two K
// blocks: measured 11-14 % faster); the 256-wide tile keeps four one-block stages (two
// two-block stages were slower).
#ifndef ZP_ANS_SU
#define ZP_ANS_SU 2
#endif
#ifndef ZP_ANS_SB
#define ZP_ANS_SB 4
#endif
#ifndef ZP_ANS_FIT
#define ZP_ANS_FIT 0
#endif
template <int MODE, int BT = 64, bool A16 = false>
struct Cfg {
  static constexpr bool ANS_BYTES = MODE == MODE_ANS && !A16;
  static constexpr int KPS = (A16 && BT < 64) ? 2 : 1;                     // K blocks per stage
  static constexpr int BST = A16 ? KPS * 4 * BT * BK * 2
                                 : ((ANS_BYTES && ZP_ANS_FIT) ? 4 * BT * BK * 2 : B_MAX_BYTES);  // B stage stride
  static constexpr int AST = KPS * A16_BYTES;                              // A stage stride
  // stages (with the RNS epilogue's staging the fp16 RNS ring fills 227 KiB)
  static constexpr int SB = A16 ? (MODE == MODE_RNS ? (BT == 32 ? 3 : 4)
                                                   : (BT == 16 ? 4 : (BT == 32 ? 3 : 4)))
                                : ((MODE == MODE_CMP || MODE == MODE_RNS || MODE == MODE_CRT)
                                       ? 3
                                       : (ANS_BYTES ? ZP_ANS_SB : 4));
  static constexpr int SA = SB;  // the A and B stages of a K block are filled and freed together
  // epilogue warps: with an fp16 A operand the converter warps 8-11 have no conversion to do,
  // so the RNS and residue products (whose epilogues bound them) drain TMEM with eight warps,
  // two per lane quarter, each taking half of the tile's columns
  static constexpr int EPW = (A16 && (MODE == MODE_RNS || MODE == MODE_RES)) ? 8 : 4;
  // stages of two K blocks of A bytes: the ring that hides the HBM latency
  static constexpr int SU_FIT = (224 * 1024 - SB * BST - SA * AST) / U8_STAGE;
  static constexpr int SU = A16 ? 0 : (ANS_BYTES ? (ZP_ANS_SU < SU_FIT ? ZP_ANS_SU : SU_FIT) : 2);
  static constexpr int STG = (MODE == MODE_CMP || MODE == MODE_RNS || MODE == MODE_CRT) ? STG_BYTES : 0;
  static constexpr int SMEM = SB * BST + SA * AST + SU * U8_STAGE + STG + 1024 + 512;
  static_assert(SMEM <= 232448, "shared memory above the per-block limit");
  static_assert(A16 || SU >= 1, "at least one byte stage");
};

struct GemmArgs {
  uint32_t num_m_tiles, num_n_tiles, N, nkb, Kp;
  uint32_t Mvalid;            // ANS/HINT: R (rows of D); CMP: R (answer rows)
  uint32_t Bvalid;            // ANS: queries; HINT: n; CMP: queries
  const uint32_t* rowsumA;    // raw byte sums of A rows
  const uint32_t* colsum;     // ANS/HINT: [b][4] plane sums; CMP: [b][256] byte sums
  uint32_t* out;
  uint64_t out_ld;            // ANS: R; HINT: n
  uint32_t Rp;                // CMP: plane stride (rows) of the output
  uint32_t* status;
  // MODE_RNS: the M tiles of prime k are k * mt_per_prime ..; its B rows start at
  // k * num_n_tiles * N; out[(b ZP_RNS_K + k) Rp + r'] (Rp = Rq)
  uint32_t mt_per_prime, d1p;
  const zp_rns_dev* rns;
  // MODE_CMP: the A rows of N tile nt start at nt * a_rows_per_n (0: one A for every N tile)
  uint32_t a_rows_per_n;
  // MODE_RES: A row b res_n + i = the 256 bytes of cko[b][i]; output = the B operand of the
  // RNS product (res_out, centred fp16, tile width res_bt, res_nnt N tiles, K pitch res_kp)
  uint32_t res_n, res_bt, res_nnt, res_kp;
  __half* res_out;
};

__device__ __forceinline__ uint32_t cvt_rn(uint32_t fbits) {
  return (uint32_t)__float2int_rn(__uint_as_float(fbits));
}

// 16 bytes -> 16 centred fp16 (v - 128), exact: (0x6400 | v) is fp16 1024 + v.
__device__ __forceinline__ void bytes_to_centred_f16(uint32_t w, uint32_t& lo, uint32_t& hi) {
  const __half2 off = __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480));  // 1152
  uint32_t p0 = __byte_perm(w, 0x64646464u, 0x4140);
  uint32_t p1 = __byte_perm(w, 0x64646464u, 0x4342);
  __half2 h0 = __hsub2(*reinterpret_cast<__half2*>(&p0), off);
  __half2 h1 = __hsub2(*reinterpret_cast<__half2*>(&p1), off);
  lo = *reinterpret_cast<uint32_t*>(&h0);
  hi = *reinterpret_cast<uint32_t*>(&h1);
}

// Warp-uniform bounded wait: lane 0 waits, the whole warp takes its verdict (the
// tcgen05.ld that follows must be executed by all 32 lanes).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity,
                                          volatile uint32_t* abort_flag, uint32_t* status) {
  uint32_t ok = 1;
  if ((threadIdx.x & 31) == 0)
    ok = mbar_wait_abortable(bar, parity, abort_flag, status, ZP_DEV_TIMEOUT_GEMM) ? 1u : 0u;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) (void)mbar_try_wait(bar, parity);  // each lane observes the completed phase itself
  return ok != 0;
}

// AND of `pred` over the NT threads of the epilogue warps (named barrier 1).
template <int NT = 128>
__device__ __forceinline__ bool bar_and_epi(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n"
      ".reg .pred p, q;\n"
      "setp.ne.u32 p, %1, 0;\n"
      "bar.red.and.pred q, 1, %2, p;\n"
      "selp.u32 %0, 1, 0, q;\n"
      "}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(NT)
      : "memory");
  return r != 0;
}
// Named barrier 1 over the NT threads of the epilogue warps.
template <int NT = 128>
__device__ __forceinline__ void bar_epi() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Static persistent schedule: CTA c takes tiles c, c + G, c + 2G, .. (G = gridDim.x). MODE_CRT
// tiles come in pairs (the two column halves of one M tile) that one CTA takes back to back,
// so that the epilogue carries the lower half's carry into the upper half in a register:
// tile 2 q + h, CTA c takes pairs c, c + G, ..
template <int MODE>
__device__ __forceinline__ uint32_t first_tile() {
  return MODE == MODE_CRT ? 2u * blockIdx.x : blockIdx.x;
}
template <int MODE>
__device__ __forceinline__ uint32_t next_tile(uint32_t t) {
  return MODE == MODE_CRT ? ((t & 1u) ? t + 2u * gridDim.x - 1u : t + 1u) : t + gridDim.x;
}

template <int MODE, int BT, bool A16 = false>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const GemmArgs args) {
  using C = Cfg<MODE, BT, A16>;
  static_assert(!A16 || MODE == MODE_ANS || MODE == MODE_RNS || MODE == MODE_RES,
                "fp16 A operand: batched answers, RNS and residue products only");
  constexpr int SB = C::SB, SA = C::SA, SU = C::SU;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* b_ring = smem;                                    // SB x 32 KiB (1024-aligned)
  uint8_t* a_ring = b_ring + SB * C::BST;                   // SA x 16 KiB (1024-aligned)
  uint8_t* u8_ring = a_ring + SA * C::AST;                  // SU x 16 KiB (1024-aligned)
  uint32_t* stg = reinterpret_cast<uint32_t*>(u8_ring + SU * U8_STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(u8_ring + SU * U8_STAGE + C::STG);
  uint64_t* u8_full = bars;
  uint64_t* u8_empty = u8_full + SU;
  uint64_t* b_full = u8_empty + SU;     // B tile landed (TMA transaction count)
  uint64_t* b_empty = b_full + SB;      // MMAs reading the B stage are done
  uint64_t* a_ready = b_empty + SB;     // fp16 A tile written by the four converter warps
  uint64_t* a_empty = a_ready + SA;     // MMAs reading the A stage are done
  uint64_t* acc_full = a_empty + SA;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile uint32_t* abort_flag = tmem_holder + 1;

  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t num_tiles = args.num_m_tiles * args.num_n_tiles * (MODE == MODE_CRT ? 2u : 1u);
  const uint32_t N = args.N, nkb = args.nkb;
  constexpr uint32_t KPS = C::KPS;
  const uint32_t nks = nkb / KPS;  // stages per tile (nkb is a multiple of KPS)

  if (threadIdx.x == 0) {
    for (int s = 0; s < SU; ++s) {
      mbar_init(&u8_full[s], 1);
      mbar_init(&u8_empty[s], 4);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(&b_full[s], A16 ? 2 : 5);  // B (TMA) + the four converter warps, or A and B (TMA)
      mbar_init(&b_empty[s], 1);
    }
    for (int s = 0; s < SA; ++s) {
      mbar_init(&a_ready[s], 4);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&acc_full[s], 1);
      mbar_init(&acc_empty[s], C::EPW);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0u;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_holder, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  if (warp == 0) {
    if constexpr (A16) {
    // ------------------------------------------------------------ TMA producer of A (fp16)
    if (lane == 0) {
      prefetch_tmap(&tmA);
      uint32_t cnt = 0;
      bool ok = true;
      // no L2 prefetch ahead of these loads: measured slower (prefetch 4 to 64 K blocks
      // ahead: 3 to 43 % on 1 GiB x 64 queries), the TMA loads alone keep HBM busier
      for (uint32_t tile = first_tile<MODE>(); ok && tile < num_tiles; tile = next_tile<MODE>(tile)) {
        const uint32_t mt = tile / args.num_n_tiles;
        const uint32_t arow = mt * BM + (tile % args.num_n_tiles) * args.a_rows_per_n;
        for (uint32_t ks = 0; ks < nks; ++ks, ++cnt) {
          const uint32_t sb = cnt % SB, rb = cnt / SB;
          if (rb > 0 && !mbar_wait_abortable(&b_empty[sb], (rb - 1) & 1u, abort_flag,
                                             args.status, ZP_DEV_TIMEOUT_GEMM)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&b_full[sb], KPS * A16_BYTES);
          for (uint32_t h = 0; h < KPS; ++h) {
            tma_load_2d(a_ring + sb * C::AST + h * A16_BYTES, &tmA, (int32_t)((ks * KPS + h) * BK),
                        (int32_t)arow, &b_full[sb]);
          }
        }
      }
      // Stay until the copies issued last have landed (bounded, ignores the abort flag).
      const uint32_t f_o = cnt > (uint32_t)SB ? cnt - SB : 0;
      const unsigned long long deadline = clock64() + ZP_WAIT_CYCLES;
      for (uint32_t i = f_o; i < cnt; ++i)
        if (!mbar_wait_until(&b_full[i % SB], (i / SB) & 1u, deadline)) {
          atomicOr(args.status, ZP_DEV_TIMEOUT_GEMM);
          break;
        }
    }
    } else {
    // ------------------------------------------------------------ TMA producer of A (bytes)
    if (lane == 0) {
      prefetch_tmap(&tmA);
      uint32_t cnt = 0;
      bool ok = true;
      // L2 prefetch runs PF K blocks ahead of the loads, so that the loads that fill
      // the byte ring hit L2 instead of waiting for HBM.
      constexpr uint32_t PF = 16;
      // prefetch cursor: (tile, pair of K blocks) PF pairs ahead of the load cursor
      const uint32_t npairs = (nkb + 1) / 2;
      uint32_t pf_tile = first_tile<MODE>(), pf_p = 0;
      // coordinates of the pair p of K blocks of a tile's A. MODE_CRT: row (query b, packed
      // row) = b Rp + mt BM + .., the four planes of Kp bytes one after the other
      auto a_xy = [&](uint32_t t, uint32_t p, int32_t& x, int32_t& y) {
        if constexpr (MODE == MODE_CRT) {
          const uint32_t q = t >> 1, b = q / args.num_m_tiles, mt = q % args.num_m_tiles;
          x = (int32_t)(p * 2 * BK);
          y = (int32_t)(b * args.Rp + mt * BM);
        } else {
          x = (int32_t)(p * 2 * BK);
          y = (int32_t)((t / args.num_n_tiles) * BM + (t % args.num_n_tiles) * args.a_rows_per_n);
        }
      };
      auto pf_step = [&]() {
        if (pf_tile < num_tiles) {
          int32_t x, y;
          a_xy(pf_tile, pf_p, x, y);
          tma_prefetch_l2_2d(&tmA, x, y);
        }
        if (++pf_p == npairs) {
          pf_p = 0;
          pf_tile = next_tile<MODE>(pf_tile);
        }
      };
      for (uint32_t f = 0; f < PF / 2; ++f) pf_step();
      uint32_t su = 0, pu = 0;
      for (uint32_t tile = first_tile<MODE>(); ok && tile < num_tiles; tile = next_tile<MODE>(tile)) {
        for (uint32_t p = 0; p < npairs; ++p, ++cnt) {
          pf_step();
          if (cnt >= (uint32_t)SU && !mbar_wait_abortable(&u8_empty[su], pu ^ 1u, abort_flag,
                                                          args.status, ZP_DEV_TIMEOUT_GEMM)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&u8_full[su], U8_STAGE);
          int32_t ax, ay;
          a_xy(tile, p, ax, ay);
          tma_load_2d(u8_ring + su * U8_STAGE, &tmA, ax, ay, &u8_full[su]);
          if (++su == SU) {
            su = 0;
            pu ^= 1u;
          }
        }
      }
      // Stay until the copies issued last have landed (bounded, ignores the abort flag).
      const uint32_t f_u = cnt > (uint32_t)SU ? cnt - SU : 0;
      const unsigned long long deadline = clock64() + ZP_WAIT_CYCLES;
      for (uint32_t i = f_u; i < cnt; ++i)
        if (!mbar_wait_until(&u8_full[i % SU], (i / SU) & 1u, deadline)) {
          atomicOr(args.status, ZP_DEV_TIMEOUT_GEMM);
          break;
        }
    }
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ TMA producer of B (fp16)
    if (lane == 0) {
      prefetch_tmap(&tmB);
      uint32_t cnt = 0;
      bool ok = true;
      for (uint32_t tile = first_tile<MODE>(); ok && tile < num_tiles; tile = next_tile<MODE>(tile)) {
        const uint32_t nt = tile % args.num_n_tiles;
        // B rows of this tile (RNS: the block of the tile's prime)
        const uint32_t brow0 = nt * N + (MODE == MODE_RNS ? (tile / args.num_n_tiles) /
                                                                args.mt_per_prime *
                                                                args.num_n_tiles * N
                                                          : 0u);
        for (uint32_t ks = 0; ks < nks; ++ks, ++cnt) {
          const uint32_t sb = cnt % SB, rb = cnt / SB;
          if (rb > 0 && !mbar_wait_abortable(&b_empty[sb], (rb - 1) & 1u, abort_flag,
                                             args.status, ZP_DEV_TIMEOUT_GEMM)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&b_full[sb], KPS * N * BK * 2);
          if constexpr (MODE == MODE_CRT) {
            // plane a of the A rows pairs with the constants' bytes shifted up by a columns:
            // B rows N h - a .. of query b (rows outside 0..255 read as zero)
            const uint32_t q = tile >> 1, h = tile & 1u, b = q / args.num_m_tiles;
            const uint32_t a = ks * BK / args.Kp;
            tma_load_3d(b_ring + sb * C::BST, &tmB, (int32_t)(ks * BK - a * args.Kp),
                        (int32_t)(N * h) - (int32_t)a, (int32_t)b, &b_full[sb]);
          } else {
            for (uint32_t h = 0; h < KPS; ++h)
              tma_load_2d(b_ring + sb * C::BST + h * (N * BK * 2), &tmB, (int32_t)((ks * KPS + h) * BK),
                          (int32_t)brow0, &b_full[sb]);
          }
        }
      }
      // Stay until the copies issued last have landed (bounded, ignores the abort flag).
      const uint32_t f_o = cnt > (uint32_t)SB ? cnt - SB : 0;
      const unsigned long long deadline = clock64() + ZP_WAIT_CYCLES;
      for (uint32_t i = f_o; i < cnt; ++i)
        if (!mbar_wait_until(&b_full[i % SB], (i / SB) & 1u, deadline)) {
          atomicOr(args.status, ZP_DEV_TIMEOUT_GEMM);
          break;
        }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // Kept lean: one thread feeds the tensor core, on an SMSP shared with busy warps.
      const uint32_t idesc = idesc_f16_f32(BM, N);
      const uint64_t adesc0 = sdesc_k_sw128(smem_u32(a_ring));
      const uint64_t bdesc0 = sdesc_k_sw128(smem_u32(b_ring));
      uint32_t sb = 0, pb = 0, sa = 0, pa = 0, acc_cnt = 0;
      bool ok = true;
      for (uint32_t tile = first_tile<MODE>(); ok && tile < num_tiles; tile = next_tile<MODE>(tile)) {
        uint32_t d = tmem_base, kin = 0;
        for (uint32_t ks = 0; ks < nks; ++ks) {
          if (kin == 0) {
            const uint32_t a = acc_cnt & 1u, ra = acc_cnt >> 1;
            if (ra > 0 && !mbar_wait_abortable(&acc_empty[a], (ra - 1) & 1u, abort_flag,
                                               args.status, ZP_DEV_TIMEOUT_GEMM)) {
              ok = false;
              break;
            }
            tc_fence_after();
            d = tmem_base + a * 256u;
          }
          if (!mbar_wait_abortable(&b_full[sb], pb, abort_flag, args.status,
                                   ZP_DEV_TIMEOUT_GEMM)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (uint32_t h = 0; h < KPS; ++h) {
            // start-address field += stage offset >> 4 (stays below 2^14: shared memory < 256 KiB)
            const uint64_t ad = adesc0 + (uint64_t)((sa * C::AST + h * A16_BYTES) >> 4);
            const uint64_t bd = bdesc0 + (uint64_t)((sb * C::BST + h * N * BK * 2) >> 4);
            umma_f16(d, ad, bd, idesc, kin);
            umma_f16(d, ad + 2u, bd + 2u, idesc, 1u);
            umma_f16(d, ad + 4u, bd + 4u, idesc, 1u);
            umma_f16(d, ad + 6u, bd + 6u, idesc, 1u);
            ++kin;
          }
          umma_commit(&b_empty[sb]);
          // KCHUNK is a multiple of KPS: a chunk ends with a stage
          if (kin == KCHUNK || ks == nks - 1) {
            umma_commit(&acc_full[acc_cnt & 1u]);
            ++acc_cnt;
            kin = 0;
          }
          if (++sb == SB) {
            sb = 0;
            pb ^= 1u;
          }
          if (++sa == SA) {
            sa = 0;
            pa ^= 1u;
          }
        }
      }
      // every MMA issued has completed before TMEM is released
      umma_commit(mma_done);
      if (!mbar_wait_until(mma_done, 0, clock64() + ZP_WAIT_CYCLES))
        atomicOr(args.status, ZP_DEV_TIMEOUT_GEMM);
    }
    __syncwarp();
  } else if (warp >= 8 && C::EPW == 4) {
    // ------------------------------------------------------------ converters
    if constexpr (!A16) {
    const uint32_t ct = threadIdx.x - 256;  // 0..127
    uint32_t cnt = 0, su = 0, pu = 0;
    bool ok = true;
    for (uint32_t tile = first_tile<MODE>(); ok && tile < num_tiles; tile = next_tile<MODE>(tile)) {
      for (uint32_t kb = 0; kb < nkb; ++kb, ++cnt) {
        const uint32_t h = kb & 1u;  // which K block of the 128-byte byte rows
        const uint32_t sa = cnt % SA, rra = cnt / SA;
        if ((h == 0 && !mbar_wait_abortable(&u8_full[su], pu, abort_flag, args.status,
                                            ZP_DEV_TIMEOUT_GEMM)) ||
            (rra > 0 && !mbar_wait_abortable(&b_empty[sa], (rra - 1) & 1u, abort_flag,
                                             args.status, ZP_DEV_TIMEOUT_GEMM))) {
          ok = false;
          break;
        }
        const uint8_t* src = u8_ring + su * U8_STAGE;
        uint8_t* dst = a_ring + sa * A16_BYTES;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t idx = ct + 128u * i;
          const uint32_t row = (idx & 7u) | ((idx >> 5) << 3), ch = (idx >> 3) & 3u;
          // byte tile: 128-byte rows, 16-byte chunk c stored at chunk c ^ (row % 8)
          const uint4 v = *reinterpret_cast<const uint4*>(
              src + row * 128 + (((4 * h + ch) ^ (row & 7u)) << 4));
          uint4 o0, o1;
          bytes_to_centred_f16(v.x, o0.x, o0.y);
          bytes_to_centred_f16(v.y, o0.z, o0.w);
          bytes_to_centred_f16(v.z, o1.x, o1.y);
          bytes_to_centred_f16(v.w, o1.z, o1.w);
          const uint32_t sw = row & 7u;
          *reinterpret_cast<uint4*>(dst + row * 128 + (((2 * ch) ^ sw) << 4)) = o0;
          *reinterpret_cast<uint4*>(dst + row * 128 + (((2 * ch + 1) ^ sw) << 4)) = o1;
        }
        fence_proxy_async_smem();
        __syncwarp();
        const bool last_of_pair = h == 1 || kb == nkb - 1;
        if (lane == 0) {
          mbar_arrive(&b_full[sa]);
          if (last_of_pair) mbar_arrive(&u8_empty[su]);
        }
        if (last_of_pair && ++su == SU) {
          su = 0;
          pu ^= 1u;
        }
      }
    }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    const uint32_t e = warp & 3u;          // TMEM lane quarter (a warp reads lanes 32 (warp % 4) ..)
    const uint32_t eh = (warp - 4u) >> 2;  // which half of the queries (eight epilogue warps)
    const uint32_t lane_addr = (32u * e) << 16;
    uint32_t acc_cnt = 0;
    bool ok = true;
    const uint32_t nchunks = (nkb + KCHUNK - 1) / KCHUNK;
    int64_t crt_carry = 0;  // MODE_CRT: carry out of the lower column half of this thread's row
    for (uint32_t tile = first_tile<MODE>(); ok && tile < num_tiles; tile = next_tile<MODE>(tile)) {
      const uint32_t nt = tile % args.num_n_tiles, mt = tile / args.num_n_tiles;
      if constexpr (MODE == MODE_RNS) {
        // single chunk (n <= 1024). Row (plane e, packed row 32 g + lane) of prime k: column
        // (c, bl) holds S_c, the exact byte-product sum of plane e of H' mod p and byte c of
        // cko[bl] mod p (< 2^26 once the centring is undone). The thread folds the four
        // columns of a query into x = sum_c S_c (2^(8(e + c)) mod p) < 2^55 with 64-bit
        // multiply-adds, then reduces x below 2^28 by two pseudo-Mersenne folds (p = 2^27 -
        // dl, dl < 2^12: x = lo + hi 2^27 == lo + hi dl); the four planes are added through
        // shared memory and reduced once more to [0, p). With eight epilogue warps, warp
        // half eh takes queries [eh BT / 2, (eh + 1) BT / 2).
        constexpr int EPW = C::EPW, NTE = 32 * EPW;
        constexpr int QH = BT / (EPW / 4);     // queries of this warp
        constexpr int GW = QH < 16 ? QH : 16;  // columns per TMEM load
        const uint32_t q0 = eh * QH;
        const uint32_t a = acc_cnt & 1u, ra = acc_cnt >> 1;
        if (!bar_and_epi<NTE>(warp_wait(&acc_full[a], ra & 1u, abort_flag, args.status))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t k = mt / args.mt_per_prime, g = mt % args.mt_per_prime;
        const uint32_t p = args.rns->p[k], dl = (1u << 27) - p;
        uint32_t w[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = args.rns->pow8[k][e + c];
        // the centring terms: corr_row (this row) times sum_c w[c], and per query the column
        // sums' 128 sum_c cs[c BT + bl] w[c] (lane holds queries q0 + 32 h + lane, fetched by
        // shuffles; the row term is this thread's own and is added after the shuffle)
        const int32_t corr_row =
            (int32_t)(128u * __ldg(args.rowsumA + mt * BM + e * 32 + lane) - 16384u * args.Kp);
        const uint64_t rowterm =
            (uint64_t)((int64_t)corr_row * (int64_t)((uint64_t)w[0] + w[1] + w[2] + w[3]));
        const uint32_t* cs = args.colsum + ((uint64_t)k * args.num_n_tiles + nt) * (4 * BT);
        constexpr int NH = (QH + 31) / 32;
        uint64_t qcs[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          const uint32_t bl = q0 + 32u * h + lane;
          uint64_t q = 0;
          if (32u * h + lane < (uint32_t)QH) {
#pragma unroll
            for (int c = 0; c < 4; ++c) q += (uint64_t)(128u * __ldg(cs + c * BT + bl)) * w[c];
          }
          qcs[h] = q;
        }
        constexpr int PITCH = BT + 1;  // odd: conflict-free
        uint32_t* myst = stg + (e * 32 + lane) * PITCH + q0;
#pragma unroll
        for (int gq = 0; gq < QH / GW; ++gq) {
          uint32_t r[4][GW];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint32_t ta = tmem_base + lane_addr + a * 256u + (uint32_t)(c * BT) + q0 + GW * gq;
            if constexpr (GW == 8) tmem_ld8(ta, r[c]);
            else tmem_ld16(ta, r[c]);
          }
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < GW; ++j) {
            const int bq = GW * gq + j;  // query q0 + bq
            uint64_t x = __shfl_sync(0xffffffffu, qcs[bq / 32], bq % 32) + rowterm;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              x += (uint64_t)((int64_t)__float2int_rn(__uint_as_float(r[c][j])) * (int64_t)w[c]);
            const uint64_t t1 = (x & 0x7FFFFFFull) + (x >> 27) * dl;            // < 2^41
            myst[bq] = (uint32_t)((t1 & 0x7FFFFFFull) + (t1 >> 27) * dl);      // < 2^28
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[a]);
        ++acc_cnt;
        bar_epi<NTE>();
        // out[b][k][rp] (row pitch Rp = Rq): a warp writes the 32 packed rows of one query,
        // one 128-byte line
        for (uint32_t bl = warp - 4u; bl < (uint32_t)BT; bl += EPW) {
          const uint32_t t = lane;
          uint32_t y = 0;  // < 2^30
#pragma unroll
          for (int pl = 0; pl < 4; ++pl) y += stg[(pl * 32 + t) * PITCH + bl];
          y = (y & 0x7FFFFFFu) + (y >> 27) * dl;  // < 2^27 + 7 dl < 2p
          if (y >= p) y -= p;
          const uint32_t b = nt * BT + bl;
          if (b < args.Bvalid) args.out[((uint64_t)b * ZP_RNS_K + k) * args.Rp + g * 32 + t] = y;
        }
        bar_epi<NTE>();
      } else if constexpr (MODE == MODE_RES) {
        // single chunk (K = 256). Row b n + i, column (k, c): S_c = sum_beta byte_beta(cko)
        // byte_c(2^(8 beta) mod p_k) < 2^24 once the centring is undone, so the residue is
        // x = sum_c S_c 2^(8c) < 2^48 folded below p (p = 2^27 - dl, dl < 2^12). Its four
        // bytes go to the rows of the RNS product's B operand (fp16, centred).
        constexpr int NR = 4 * ZP_RES_KPER;  // columns per tile (N)
        const uint32_t a = acc_cnt & 1u, ra = acc_cnt >> 1;
        if (!warp_wait(&acc_full[a], ra & 1u, abort_flag, args.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t row = mt * BM + e * 32 + lane;  // b n + i
        const bool live = row < args.Mvalid;
        const uint32_t b = live ? row / args.res_n : 0u, i = live ? row - b * args.res_n : 0u;
        // output addresses: B row (k nnt + b / bt) 4 bt + c bt + b % bt, column i
        const uint32_t bt = args.res_bt;
        const uint64_t nq = (uint64_t)args.res_nnt * 4 * bt;  // B rows per prime
        const uint64_t kp = args.res_kp;
        __half* outp = args.res_out + ((uint64_t)(b / bt) * 4 * bt + b % bt) * kp + i;
        const uint64_t kstep = nq * kp, cstep = (uint64_t)bt * kp;
        // centring terms: corr_row (this row) in every byte column; per prime j of the tile
        // 128 sum_c cs[4 j + c] 2^(8c) and p_j (lanes hold j = lane and lane + 32, fetched
        // by shuffles; the row term is this thread's own)
        const int64_t corr_row =
            live ? (int64_t)(int32_t)(128u * __ldg(args.rowsumA + row) - 16384u * args.Kp) : 0;
        const uint64_t rowterm = (uint64_t)(corr_row * 0x01010101ll);
        const uint32_t* cs = args.colsum + (uint64_t)nt * NR;
        uint64_t csw[2];
        uint32_t pj[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t j = 32u * h + lane, k = nt * ZP_RES_KPER + j;
          uint64_t q = 0;
          if (j < (uint32_t)ZP_RES_KPER) {
#pragma unroll
            for (int c = 0; c < 4; ++c) q += (uint64_t)(128u * __ldg(cs + 4 * j + c)) << (8 * c);
          }
          csw[h] = q;
          pj[h] = (j < (uint32_t)ZP_RES_KPER && k < ZP_RNS_K) ? args.rns->p[k] : 1u;
        }
        // primes j0 .. j0 + PH - 1 of the tile: all of them, or a half with eight warps
        constexpr int PH = ZP_RES_KPER / (C::EPW / 4);
        static_assert(PH % 4 == 0, "four primes per 16-column TMEM load");
        const uint32_t j0 = eh * PH;
#pragma unroll
        for (int g = 0; g < PH / 4; ++g) {
          uint32_t r[16];
          tmem_ld16(tmem_base + lane_addr + a * 256u + 4u * j0 + 16u * g, r);
          tmem_wait_ld();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t j = j0 + 4 * g + kk;
            const uint32_t k = nt * ZP_RES_KPER + j;
            const uint64_t cj = __shfl_sync(0xffffffffu, (j >> 5) ? csw[1] : csw[0], j & 31);
            const uint32_t p = __shfl_sync(0xffffffffu, (j >> 5) ? pj[1] : pj[0], j & 31);
            if (k >= ZP_RNS_K) continue;  // uniform across the warp
            const uint32_t dl = (1u << 27) - p;
            uint64_t x = cj + rowterm;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              x += (uint64_t)((int64_t)__float2int_rn(__uint_as_float(r[4 * kk + c])) << (8 * c));
            const uint64_t t1 = (x & 0x7FFFFFFull) + (x >> 27) * dl;  // < 2^34
            uint32_t v = (uint32_t)((t1 & 0x7FFFFFFull) + (t1 >> 27) * dl);  // < 2^27 + 2^19 < 2p
            if (v >= p) v -= p;
            if (live) {
              __half* o = outp + (uint64_t)k * kstep;
              uint32_t lo, hi;  // the four bytes as centred fp16 (exact)
              bytes_to_centred_f16(v, lo, hi);
              o[0] = __ushort_as_half((unsigned short)(lo & 0xFFFFu));
              o[cstep] = __ushort_as_half((unsigned short)(lo >> 16));
              o[2 * cstep] = __ushort_as_half((unsigned short)(hi & 0xFFFFu));
              o[3 * cstep] = __ushort_as_half((unsigned short)(hi >> 16));
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[a]);
        ++acc_cnt;
      } else if constexpr (MODE == MODE_CRT) {
        // single chunk (K = 4 Kp <= 1024). Tile (query b, packed rows 128 mt .., half h):
        // thread row = packed row rp; column c of the tile is byte position t = 144 h + c of
        // V = sum_a 2^(8a) (plane a of the A row) . constants, i.e. c_t = sum_{a, k} A_a[k]
        // B[k][t - a] over 0 <= t - a < 256 (the B rows shifted by a read zero outside), exact
        // in fp32. Undoing the centring adds, per valid (a, t), 128 rowsum_a + 128 colsum[t - a]
        // - 16384 Kp. Words w = 36 h .. of V are c_t gathered four at a time with the carry
        // chain in 64-bit; the lower half's final carry stays in crt_carry for the upper half.
        const uint32_t q = tile >> 1, hh = tile & 1u;
        const uint32_t b = q / args.num_m_tiles, mq = q % args.num_m_tiles;
        const uint32_t a = acc_cnt & 1u, ra = acc_cnt >> 1;
        if (!bar_and_epi(warp_wait(&acc_full[a], ra & 1u, abort_flag, args.status))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t rl = e * 32 + lane, rp = mq * BM + rl;
        uint32_t rs[4];
#pragma unroll
        for (int pl = 0; pl < 4; ++pl)
          rs[pl] = rp < args.Rp
                       ? __ldg(args.rowsumA + (uint64_t)b * args.a_rows_per_n + pl * args.Rp + rp)
                       : 0u;
        // row terms: 128 sum_{a valid} rowsum_a per byte column, as 64-bit words
        const int64_t r4 = 128 * (int64_t)(rs[0] + rs[1] + rs[2] + rs[3]);
        const int64_t rw_mid = r4 * 0x01010101ll;
        const int64_t rw_lo = 128 * ((int64_t)rs[0] + ((int64_t)(rs[0] + rs[1]) << 8) +
                                     ((int64_t)(rs[0] + rs[1] + rs[2]) << 16)) + (r4 << 24);
        const int64_t rw_hi = 128 * ((int64_t)(rs[1] + rs[2] + rs[3]) + ((int64_t)(rs[2] + rs[3]) << 8) +
                                     ((int64_t)rs[3] << 16));
        // column terms of words w0 + lane and w0 + 32 + lane (fetched by shuffles)
        const uint32_t w0 = 36u * hh;
        const uint32_t* cs = args.colsum + (uint64_t)b * 256;
        const int64_t kterm = 16384 * (int64_t)args.Kp;
        int64_t cw[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const uint32_t w = w0 + 32u * i + lane;
          int64_t v = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int t = 4 * (int)w + j;
            int64_t ct = 0;
#pragma unroll
            for (int pl = 0; pl < 4; ++pl)
              if (t - pl >= 0 && t - pl < 256) ct += 128 * (int64_t)__ldg(cs + t - pl) - kterm;
            v += ct << (8 * j);
          }
          cw[i] = v;
        }
        if (hh == 0) crt_carry = 0;
        int64_t carry = crt_carry;
        uint32_t* myst = stg + rl * 37;  // 37 words per staged row (odd pitch)
        const uint32_t tcol = tmem_base + lane_addr + a * 256u;
#pragma unroll
        for (int gq = 0; gq < 5; ++gq) {  // words 8 gq .. 8 gq + 7 of the half (the fifth: 4)
          if (gq == 4 && hh) break;
          uint32_t r[32];
          if (gq < 4) tmem_ld32(tcol + 32u * gq, r);
          else tmem_ld16(tcol + 128u, *reinterpret_cast<uint32_t(*)[16]>(r));
          tmem_wait_ld();
#pragma unroll
          for (int wl = 0; wl < 8; ++wl) {
            if (gq == 4 && wl >= 4) break;
            const int wi = 8 * gq + wl;  // word of the half
            const uint32_t w = w0 + wi;
            const uint32_t chi = __shfl_sync(0xffffffffu, (uint32_t)(cw[wi / 32] >> 32), wi % 32);
            const uint32_t clo = __shfl_sync(0xffffffffu, (uint32_t)cw[wi / 32], wi % 32);
            const int64_t c = (int64_t)(((uint64_t)chi << 32) | clo);
            int64_t sv = carry + c + (w == 0 ? rw_lo : (w < 64 ? rw_mid : (w == 64 ? rw_hi : 0)));
#pragma unroll
            for (int j = 0; j < 4; ++j)
              sv += (int64_t)__float2int_rn(__uint_as_float(r[4 * wl + j])) * (int64_t)(1u << (8 * j));
            myst[wi] = (uint32_t)sv;
            carry = sv >> 32;
          }
        }
        crt_carry = carry;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[a]);
        ++acc_cnt;
        bar_epi();
        // rows of this tile out, coalesced: words w0 .. w0 + nw - 1 of V[b][rp]
        const uint32_t nw = hh ? (uint32_t)ZP_VW - 36u : 36u;
        uint32_t* dst = args.out + ((uint64_t)b * args.Rp + (uint64_t)mq * BM) * ZP_VW + w0;
        for (uint32_t row = e; row < BM && mq * BM + row < args.Mvalid; row += 4)
          for (uint32_t wl = lane; wl < nw; wl += 32) dst[(uint64_t)row * ZP_VW + wl] = stg[row * 37 + wl];
        bar_epi();
      } else if constexpr (MODE == MODE_CMP) {
        // single chunk (n <= 1024): byte-column sums -> 67-word integer
        const uint32_t a = acc_cnt & 1u, ra = acc_cnt >> 1;
        // the four epilogue warps agree on the verdict before their named barriers
        if (!bar_and_epi(warp_wait(&acc_full[a], ra & 1u, abort_flag, args.status))) {
          ok = false;
          break;
        }
        tc_fence_after();
        // row of A (plane e of answer row 32 mt + lane; batched A: of N tile nt's rows)
        const uint32_t m = mt * BM + e * 32 + lane + nt * args.a_rows_per_n;
        const uint32_t b = nt;
        const uint32_t corr_row = 128u * __ldg(args.rowsumA + m) - 16384u * args.Kp;
        const uint32_t* cs = args.colsum + (uint64_t)b * 256;
        uint32_t* myst = stg + (e * 32 + lane) * STG_PITCH;
        uint64_t carry = 0;
#pragma unroll 1
        for (int g = 0; g < 8; ++g) {
          uint32_t r[32];
          tmem_ld32(tmem_base + lane_addr + a * 256u + 32u * g, r);
          tmem_wait_ld();
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            uint64_t s = carry;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int col = 32 * g + 4 * w + j;
              const uint32_t p = cvt_rn(r[4 * w + j]) + corr_row + 128u * __ldg(cs + col);
              s += (uint64_t)p << (8 * j);
            }
            myst[8 * g + w] = (uint32_t)s;
            carry = s >> 32;
          }
        }
        myst[64] = (uint32_t)carry;
        myst[65] = (uint32_t)(carry >> 32);
        myst[66] = 0u;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[a]);
        ++acc_cnt;
        // V = sum_a V_a 2^(8a): warp 0 adds the four staged planes of its row (exact,
        // sequential carries), then all four warps copy the 32 rows out coalesced.
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (e == 0) {
          const uint32_t* p1 = stg + (1 * 32 + lane) * STG_PITCH;
          const uint32_t* p2 = stg + (2 * 32 + lane) * STG_PITCH;
          const uint32_t* p3 = stg + (3 * 32 + lane) * STG_PITCH;
          uint64_t c = 0;
          uint32_t q1 = 0, q2 = 0, q3 = 0;  // previous words of planes 1..3
#pragma unroll 4
          for (int w = 0; w < ZP_VW; ++w) {
            const uint32_t w1 = p1[w], w2 = p2[w], w3 = p3[w];
            uint64_t s = c + myst[w];
            s += (w1 << 8) | (q1 >> 24);
            s += (w2 << 16) | (q2 >> 16);
            s += (w3 << 24) | (q3 >> 8);
            myst[w] = (uint32_t)s;
            c = s >> 32;
            q1 = w1;
            q2 = w2;
            q3 = w3;
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        uint32_t* dst = args.out + ((uint64_t)b * args.Rp + (uint64_t)mt * 32) * ZP_VW;
        const uint32_t tid = e * 32 + lane;
        for (uint32_t idx = tid; idx < 32u * ZP_VW; idx += 128) {
          const uint32_t rr = idx / ZP_VW, ww = idx % ZP_VW;
          dst[idx] = stg[rr * STG_PITCH + ww];
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      } else {
        uint32_t acc[BT];
#pragma unroll
        for (int i = 0; i < BT; ++i) acc[i] = 0u;
        for (uint32_t c = 0; c < nchunks; ++c) {
          const uint32_t a = acc_cnt & 1u, ra = acc_cnt >> 1;
          if (!warp_wait(&acc_full[a], ra & 1u, abort_flag, args.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int g = 0; g < (4 * BT) / 32; ++g) {
            uint32_t r[32];
            tmem_ld32(tmem_base + lane_addr + a * 256u + 32u * g, r);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int col = 32 * g + j;
              const int pl = col / BT, bl = col % BT;
              acc[bl] += cvt_rn(r[j]) << (8 * pl);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[a]);
          ++acc_cnt;
        }
        if (!ok) break;
        const uint32_t r = mt * BM + e * 32 + lane;
        if (r < args.Mvalid) {
          const uint32_t rowterm = 128u * __ldg(args.rowsumA + r) * 0x01010101u;
          const uint32_t kterm = 16384u * args.Kp * 0x01010101u;
          if constexpr (MODE == MODE_ANS) {
#pragma unroll
            for (int bl = 0; bl < BT; ++bl) {
              const uint32_t b = nt * BT + bl;
              if (b < args.Bvalid) {
                const uint4 cq = *reinterpret_cast<const uint4*>(args.colsum + (uint64_t)b * 4);
                const uint32_t qterm =
                    128u * (cq.x + (cq.y << 8) + (cq.z << 16) + (cq.w << 24)) - kterm;
                args.out[(uint64_t)b * args.out_ld + r] = acc[bl] + rowterm + qterm;
              }
            }
          } else {
            uint32_t* orow = args.out + (uint64_t)r * args.out_ld + (uint64_t)nt * BT;
#pragma unroll
            for (int bl = 0; bl < BT; ++bl) {
              const uint32_t b = nt * BT + bl;
              if (b < args.Bvalid) {
                const uint4 cq = *reinterpret_cast<const uint4*>(args.colsum + (uint64_t)b * 4);
                const uint32_t qterm =
                    128u * (cq.x + (cq.y << 8) + (cq.z << 16) + (cq.w << 24)) - kterm;
                orow[bl] = acc[bl] + rowterm + qterm;
              }
            }
          }
        }
      }
    }
  }
  // warp 3 has no role
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, 512);
}

// ---------------------------------------------------------------------- operand preparation
// Query byte planes as centred fp16 for MODE_ANS / MODE_HINT. Row (nt*N + a*BT + bl) of
// Qc holds plane a of query b = nt*BT + bl over k < Kp: byte a of Q(b, k) - 128, with
// Q(b, k) = 0 for b >= B or k >= C. colsum[b][a] += sum_k byte a of Q(b, k).
// Variant "rows": Q(b, k) = Q[b*C + k]; one CTA per (query, 2048-wide K range).
__global__ void k_prep_q_rows(const uint32_t* __restrict__ Q, uint32_t B, uint32_t C, uint32_t Kp,
                              uint32_t BT, uint32_t N, __half* __restrict__ Qc,
                              uint32_t* __restrict__ colsum) {
  const uint32_t b = blockIdx.y;
  const uint32_t nt = b / BT, bl = b % BT;
  const uint32_t k0 = blockIdx.x * 2048 + threadIdx.x * 8;
  uint32_t s[4] = {0, 0, 0, 0};
  if (k0 < Kp) {
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t k = k0 + i;
      x[i] = (b < B && k < C) ? Q[(uint64_t)b * C + k] : 0u;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      uint32_t h[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t lo = (x[2 * i] >> (8 * a)) & 0xFFu, hi = (x[2 * i + 1] >> (8 * a)) & 0xFFu;
        s[a] += lo + hi;
        const __half2 hv = __halves2half2(__int2half_rn((int)lo - 128), __int2half_rn((int)hi - 128));
        h[i] = *reinterpret_cast<const uint32_t*>(&hv);
      }
      __half* dst = Qc + ((uint64_t)nt * N + a * BT + bl) * Kp + k0;
      *reinterpret_cast<uint4*>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    uint32_t v = s[a];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && b < B && v) atomicAdd(&colsum[b * 4 + a], v);
  }
}

// Variant "cols": Q(b, k) = A[k*B + b] (the hint's queries are the columns of A).
// CTA: 32 queries x 64 k, transposed through shared memory.
__global__ void k_prep_q_cols(const uint32_t* __restrict__ A, uint32_t B, uint32_t Bpad, uint32_t C,
                              uint32_t Kp, uint32_t BT, uint32_t N, __half* __restrict__ Qc,
                              uint32_t* __restrict__ colsum) {
  __shared__ uint32_t tile[64][33];
  const uint32_t b0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  const uint32_t tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: 8 rows per pass
  for (uint32_t kk = ty; kk < 64; kk += 8) {
    const uint32_t k = k0 + kk, b = b0 + tx;
    tile[kk][tx] = (k < C && b < B) ? A[(uint64_t)k * B + b] : 0u;
  }
  __syncthreads();
  // thread -> (query bq = threadIdx.x / 8, 8-wide k group kg = threadIdx.x % 8)
  const uint32_t bq = threadIdx.x >> 3, kg = threadIdx.x & 7;
  const uint32_t b = b0 + bq;
  const uint32_t nt = b / BT, bl = b % BT;
  const bool row_exists = b < Bpad;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    uint32_t h[4], s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t lo = (tile[kg * 8 + 2 * i][bq] >> (8 * a)) & 0xFFu;
      const uint32_t hi = (tile[kg * 8 + 2 * i + 1][bq] >> (8 * a)) & 0xFFu;
      s += lo + hi;
      const __half2 hv = __halves2half2(__int2half_rn((int)lo - 128), __int2half_rn((int)hi - 128));
      h[i] = *reinterpret_cast<const uint32_t*>(&hv);
    }
    if (row_exists) {
      __half* dst = Qc + ((uint64_t)nt * N + a * BT + bl) * Kp + k0 + kg * 8;
      *reinterpret_cast<uint4*>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
    }
    // reduce s over the 8 k-groups of this query (8 consecutive lanes)
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (kg == 0 && b < B && s) atomicAdd(&colsum[b * 4 + a], s);
  }
}

// Compression operand: row (b*256 + beta) of Bc holds byte beta of cko[b][i] - 128 for
// i < n (raw 0 for n <= i < Kp). colsum[b][beta] += sum_i byte beta of cko[b][i].
// CTA: one query, PREP_IB = 16 offsets (enough CTAs for one query); 256 threads.
// With `srcs` (device array), query b's n values start at srcs[b * src_stride] instead of
// cko + b n ZP_MAX_L (the CRT product reads each client's table in place), and the ntail
// values after them come from `tail` (the same for every query).
constexpr uint32_t PREP_IB = 16;
__global__ void k_prep_cko(const uint32_t* __restrict__ cko, uint32_t n, uint32_t Kp,
                           __half* __restrict__ Bc, uint32_t* __restrict__ colsum,
                           const uint32_t* const* __restrict__ srcs = nullptr,
                           uint32_t src_stride = 0, const uint32_t* __restrict__ tail = nullptr,
                           uint32_t ntail = 0) {
  __shared__ uint32_t tile[PREP_IB][ZP_MAX_L + 1];
  const uint32_t b = blockIdx.y, i0 = blockIdx.x * PREP_IB;
  const uint32_t* src = srcs ? srcs[(uint64_t)b * src_stride] : cko + (uint64_t)b * n * ZP_MAX_L;
  for (uint32_t idx = threadIdx.x; idx < PREP_IB * ZP_MAX_L; idx += blockDim.x) {
    const uint32_t ii = idx / ZP_MAX_L, w = idx % ZP_MAX_L;
    const uint32_t i = i0 + ii;
    tile[ii][w] = i < n ? src[(uint64_t)i * ZP_MAX_L + w]
                        : (i < n + ntail ? tail[(uint64_t)(i - n) * ZP_MAX_L + w] : 0u);
  }
  __syncthreads();
  const uint32_t beta = threadIdx.x;  // 0..255
  const uint32_t w = beta >> 2, sh = 8 * (beta & 3);
  uint32_t s = 0;
  __half* dst = Bc + ((uint64_t)b * 256 + beta) * Kp + i0;
#pragma unroll
  for (int g = 0; g < (int)PREP_IB / 8; ++g) {
    uint32_t h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t lo = (tile[g * 8 + 2 * i][w] >> sh) & 0xFFu;
      const uint32_t hi = (tile[g * 8 + 2 * i + 1][w] >> sh) & 0xFFu;
      s += lo + hi;
      const __half2 hv = __halves2half2(__int2half_rn((int)lo - 128), __int2half_rn((int)hi - 128));
      h[i] = *reinterpret_cast<const uint32_t*>(&hv);
    }
    *reinterpret_cast<uint4*>(dst + g * 8) = make_uint4(h[0], h[1], h[2], h[3]);
  }
  if (s) atomicAdd(&colsum[(uint64_t)b * 256 + beta], s);
}

// per device, mode, tile width and A operand type: the kernel attribute is set (atomic flags:
// two host threads may both set an attribute, which is harmless)
std::atomic<bool> g_attr[64][6][3][2];

template <int MODE, int BT, bool A16 = false>
int launch_gemm(zp_ctx* ctx, const CUtensorMap& tmA, const CUtensorMap& tmB, const GemmArgs& ga,
                cudaStream_t st, uint32_t max_ctas = 0) {
  constexpr int bi = BT == 16 ? 0 : (BT == 32 ? 1 : 2);
  using C = Cfg<MODE, BT, A16>;
  if (!g_attr[ctx->device & 63][MODE][bi][A16]) {
    ZP_CUDA(cudaFuncSetAttribute(k_gemm_tc<MODE, BT, A16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 C::SMEM));
    g_attr[ctx->device & 63][MODE][bi][A16] = true;
  }
  uint32_t tiles = ga.num_m_tiles * ga.num_n_tiles;
  uint32_t grid = tiles < (uint32_t)ctx->num_sms ? tiles : (uint32_t)ctx->num_sms;
  if (max_ctas && grid > max_ctas) grid = max_ctas;
  zp_clear_pending_error();
  ctx->launches++;
  k_gemm_tc<MODE, BT, A16><<<grid, NTHREADS, C::SMEM, st>>>(tmA, tmB, ga);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

}  // namespace

// Queries per N tile for a batch of B queries (N = 4 * BT rows of the B operand).

// Batched product out = D . Q^T (MODE_ANS: out[b][r]) or D . A (MODE_HINT: out[r][i]).
// Q(b, k) = dQ[b*C + k] (rows) or dQ[k*B + b] (cols). D given by its tensor map.
int zp_launch_answer_tc(zp_db* db, const CUtensorMap& tmD, uint32_t Rrows, const uint32_t* dQ,
                        uint32_t B, bool q_cols, uint32_t* dOut, uint64_t out_ld, bool hint,
                        const uint32_t* rowsum, cudaStream_t st, bool a16) {
  zp_ctx* ctx = db->ctx;
  const uint32_t C = db->C;
  // the fp16 A path takes two K blocks per stage: K padded to 128
  const uint32_t Kp = a16 ? (C + 127) / 128 * 128 : (C + 63) / 64 * 64;
  // the hint (columns of A as queries, n of them) keeps the widest tile
  const uint32_t BT = hint ? 64u : zp_pick_bt(ctx->ans_bt, B);
  const uint32_t N = 4 * BT;
  const uint32_t nnt = (B + BT - 1) / BT;
  const size_t qc_bytes = (size_t)nnt * N * Kp * 2;
  const size_t cs_bytes = (size_t)nnt * BT * 4 * 4;
  int rc = zp_scratch_reserve(&db->s_tcq, qc_bytes + cs_bytes + 256);
  if (rc) return rc;
  __half* Qc = static_cast<__half*>(db->s_tcq.p);
  uint32_t* colsum = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(db->s_tcq.p) + qc_bytes);
  ZP_CUDA(cudaMemsetAsync(colsum, 0, cs_bytes, st));
  zp_clear_pending_error();
  ctx->launches++;
  if (!q_cols) {
    dim3 grid((Kp + 2047) / 2048, nnt * BT);
    k_prep_q_rows<<<grid, 256, 0, st>>>(dQ, B, C, Kp, BT, N, Qc, colsum);
  } else {
    dim3 grid(Kp / 64, (nnt * BT + 31) / 32);
    k_prep_q_cols<<<grid, 256, 0, st>>>(dQ, B, nnt * BT, C, Kp, BT, N, Qc, colsum);
  }
  ZP_CUDA(cudaGetLastError());
  CUtensorMap tmB;
  rc = zp_encode_tmap_2d(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Qc, Kp, (uint64_t)nnt * N,
                         (uint64_t)Kp * 2, 64, N, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  GemmArgs ga{};
  ga.num_m_tiles = (Rrows + BM - 1) / BM;
  ga.num_n_tiles = nnt;
  ga.N = N;
  ga.nkb = Kp / BK;
  ga.Kp = Kp;
  ga.Mvalid = Rrows;
  ga.Bvalid = B;
  ga.rowsumA = rowsum;
  ga.colsum = colsum;
  ga.out = dOut;
  ga.out_ld = out_ld;
  ga.status = ctx->d_status;
  if (hint) {
    if (BT == 16) return launch_gemm<MODE_HINT, 16>(ctx, tmD, tmB, ga, st);
    if (BT == 32) return launch_gemm<MODE_HINT, 32>(ctx, tmD, tmB, ga, st);
    return launch_gemm<MODE_HINT, 64>(ctx, tmD, tmB, ga, st);
  }
  if (a16) {
    if (BT == 16) return launch_gemm<MODE_ANS, 16, true>(ctx, tmD, tmB, ga, st);
    if (BT == 32) return launch_gemm<MODE_ANS, 32, true>(ctx, tmD, tmB, ga, st);
    return launch_gemm<MODE_ANS, 64, true>(ctx, tmD, tmB, ga, st);
  }
  if (BT == 16) return launch_gemm<MODE_ANS, 16>(ctx, tmD, tmB, ga, st);
  if (BT == 32) return launch_gemm<MODE_ANS, 32>(ctx, tmD, tmB, ga, st);
  return launch_gemm<MODE_ANS, 64>(ctx, tmD, tmB, ga, st);
}

// The resident fp16 copy of D for the tensor-core answers: row r, column k < Kp (C rounded
// up to 128) holds D[r][k] - 128 (k < C) or -128 (the padding, the centred value of a zero
// byte, as the byte path's out-of-range loads give). dRows lists the rows to write (NULL = all R).
// grid (ceil(Kp / 2048), min(rows, 32768)), rows strided over grid.y; eight columns per thread.
__global__ void k_d16_rows(const uint8_t* __restrict__ D, uint64_t ld, uint32_t C, uint32_t Kp,
                           const uint32_t* __restrict__ dRows, uint32_t nrows,
                           __half* __restrict__ D16) {
  const uint32_t k0 = blockIdx.x * 2048 + threadIdx.x * 8;
  if (k0 >= Kp) return;
  for (uint32_t idx = blockIdx.y; idx < nrows; idx += gridDim.y) {
  const uint32_t r = dRows ? dRows[idx] : idx;
  const uint8_t* src = D + (uint64_t)r * ld;
  uint32_t v[8];
  if (k0 + 8 <= C) {
    const uint2 w = *reinterpret_cast<const uint2*>(src + k0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = (w.x >> (8 * j)) & 0xFFu;
      v[4 + j] = (w.y >> (8 * j)) & 0xFFu;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = k0 + j < C ? src[k0 + j] : 0u;
  }
  uint32_t h[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __half2 x = __halves2half2(__int2half_rn((int)v[2 * j] - 128), __int2half_rn((int)v[2 * j + 1] - 128));
    h[j] = *reinterpret_cast<const uint32_t*>(&x);
  }
  *reinterpret_cast<uint4*>(D16 + (uint64_t)r * Kp + k0) = make_uint4(h[0], h[1], h[2], h[3]);
  }
}

int zp_launch_d16_rows(zp_db* db, const uint32_t* dRows, uint32_t nrows, cudaStream_t st) {
  if (nrows == 0) return ZP_OK;
  const uint32_t Kp = (db->C + 127) / 128 * 128;
  zp_clear_pending_error();
  db->ctx->launches++;
  dim3 grid((Kp + 2047) / 2048, nrows < 32768u ? nrows : 32768u);
  k_d16_rows<<<grid, 256, 0, st>>>(db->dD, db->ld, db->C, Kp, dRows, nrows, static_cast<__half*>(db->d_D16));
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

// Compression products V4[b][a][r][67] = sum_i Hbyte_a[r][i] cko[b][i] (n <= 1024).
int zp_launch_vmul_tc(zp_db* db, const uint32_t* dCKO, uint32_t B, uint32_t* V4, cudaStream_t st,
                      uint32_t max_ctas) {
  zp_ctx* ctx = db->ctx;
  const uint32_t n = ctx->P.n;
  const uint32_t Kp = (n + 63) / 64 * 64;
  const size_t bc_bytes = (size_t)B * 256 * Kp * 2;
  const size_t cs_bytes = (size_t)B * 256 * 4;
  int rc = zp_scratch_reserve(&db->s_cko, bc_bytes + cs_bytes + 256);
  if (rc) return rc;
  __half* Bc = static_cast<__half*>(db->s_cko.p);
  uint32_t* colsum = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(db->s_cko.p) + bc_bytes);
  ZP_CUDA(cudaMemsetAsync(colsum, 0, cs_bytes, st));
  zp_clear_pending_error();
  ctx->launches++;
  k_prep_cko<<<dim3(Kp / PREP_IB, B), 256, 0, st>>>(dCKO, n, Kp, Bc, colsum);
  ZP_CUDA(cudaGetLastError());
  CUtensorMap tmB;
  rc = zp_encode_tmap_2d(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Bc, Kp, (uint64_t)B * 256,
                         (uint64_t)Kp * 2, 64, 256, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  GemmArgs ga{};
  ga.num_m_tiles = db->Rp / 32;
  ga.num_n_tiles = B;
  ga.N = 256;
  ga.nkb = Kp / BK;
  ga.Kp = Kp;
  ga.Mvalid = db->R;
  ga.Bvalid = B;
  ga.rowsumA = db->d_hpl_rowsum;
  ga.colsum = colsum;
  ga.out = V4;
  ga.out_ld = 0;
  ga.Rp = db->Rp;
  ga.status = ctx->d_status;
  return launch_gemm<MODE_CMP, 64>(ctx, db->tmap_hpl, tmB, ga, st, max_ctas);
}

// ---------------------------------------------------------------------------------
// RNS compression products (Sec. 5.2): X[b][k][r'] = H'[r', :] . cko[b] mod p_k for the
// ZP_RNS_K primes, as one grouped tensor-core product: for prime k, the byte planes of
// H' mod p_k (A, built by zp_launch_rns_planes) times the byte planes of cko mod p_k (B).
namespace {

// The 256 bytes of each cko element as centred fp16 (byte - 128, exact), the A operand of
// MODE_RES, and their byte sums. One warp per element; lane l takes bytes 8 l .. 8 l + 7.
__global__ void k_cko_f16(const uint32_t* __restrict__ cko, uint32_t rows, __half* __restrict__ out,
                          uint32_t* __restrict__ rowsum) {
  const uint64_t row = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (row >= rows) return;
  const uint2 w = __ldg(reinterpret_cast<const uint2*>(cko + row * 64) + lane);
  uint4 o;
  bytes_to_centred_f16(w.x, o.x, o.y);
  bytes_to_centred_f16(w.y, o.z, o.w);
  reinterpret_cast<uint4*>(out + row * 256)[lane] = o;
  uint32_t sum = __dp4a(w.x, 0x01010101u, 0u) + __dp4a(w.y, 0x01010101u, 0u);
  sum = __reduce_add_sync(0xffffffffu, sum);
  if (lane == 0) rowsum[row] = sum;
}

// Byte sums of rows of a centred fp16 matrix (value + 128 summed over the row): the row sums
// of the RNS product's B operand, after MODE_RES wrote it. One warp per row; cols % 8 == 0.
__global__ void k_fp16_rowsum(const __half* __restrict__ M, uint64_t rows, uint32_t cols,
                              uint32_t* __restrict__ out) {
  const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (wid >= rows) return;
  const uint4* src = reinterpret_cast<const uint4*>(M + wid * cols);
  int32_t s = 0;
  for (uint32_t c = lane; c < cols / 8; c += 32) {
    const uint4 v = __ldg(src + c);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const __half2 h = *reinterpret_cast<const __half2*>(&w[t]);
      s += __half2int_rn(__low2half(h)) + __half2int_rn(__high2half(h));
    }
  }
  s = (int32_t)__reduce_add_sync(0xffffffffu, (uint32_t)s);
  if (lane == 0) out[wid] = (uint32_t)(s + 128 * (int32_t)cols);
}

// Columns i in [n, Kp) of the B operand of the RNS product: the centred value of a zero byte
// (they enter every sum). grid (ceil(rows / 8)), 256 threads.
__global__ void k_rns_kpad(__half* __restrict__ Bc, uint64_t rows, uint32_t n, uint32_t Kp) {
  const uint32_t w = Kp - n;
  const uint64_t idx0 = (uint64_t)blockIdx.x * 8 * w;
  for (uint32_t t = threadIdx.x; t < 8 * w; t += blockDim.x) {
    const uint64_t r = (idx0 + t) / w;
    if (r < rows) Bc[r * Kp + n + (uint32_t)((idx0 + t) % w)] = __int2half_rn(-128);
  }
}

}  // namespace

int zp_launch_rns_products(zp_db* db, const uint32_t* dCKO, uint32_t B, uint32_t* X, cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  const uint32_t n = ctx->P.n;
  const uint32_t Kp = (n + 127) / 128 * 128;
  const uint32_t BT = zp_pick_bt(ctx->rns_bt, B), N = 4 * BT, nnt = (B + BT - 1) / BT;
  const uint64_t brows = (uint64_t)ZP_RNS_K * nnt * N;
  const size_t bc_bytes = (size_t)brows * Kp * 2;
  const size_t cs_bytes = (size_t)brows * 4;
  const size_t ac_off = (bc_bytes + cs_bytes + (size_t)B * n * 4 + 255) / 256 * 256;
  int rc = zp_scratch_reserve(&db->s_cko, ac_off + (size_t)B * n * 512);
  if (rc) return rc;
  __half* Bc = static_cast<__half*>(db->s_cko.p);
  uint32_t* colsum = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(db->s_cko.p) + bc_bytes);
  __half* Ac = reinterpret_cast<__half*>(static_cast<uint8_t*>(db->s_cko.p) + ac_off);
  // cko mod p_k for every query, offset and prime on the tensor cores (MODE_RES): A = the
  // 256 bytes of each cko[b][i] as centred fp16 (k_cko_f16, with their byte sums), B = the
  // context's table of 2^(8 beta) mod p_k; the epilogue writes the byte planes of the residues
  // into Bc, k_fp16_rowsum their sums into colsum (rows of queries past B hold whatever the
  // buffer held: their columns of the product are discarded)
  rc = zp_ensure_res_table(ctx);
  if (rc) return rc;
  uint32_t* ckrs = colsum + brows;  // byte sums of the cko elements
  zp_clear_pending_error();
  ctx->launches++;
  k_cko_f16<<<(unsigned)(((uint64_t)B * n * 32 + 255) / 256), 256, 0, st>>>(dCKO, B * n, Ac, ckrs);
  ZP_CUDA(cudaGetLastError());
  if (Kp > n) {
    zp_clear_pending_error();
    ctx->launches++;
    k_rns_kpad<<<(unsigned)((brows + 7) / 8), 256, 0, st>>>(Bc, brows, n, Kp);
    ZP_CUDA(cudaGetLastError());
  }
  {
    CUtensorMap tmC;
    rc = zp_encode_tmap_2d(&tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Ac, 256, (uint64_t)B * n, 512, 64,
                           128, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    GemmArgs gr{};
    gr.num_m_tiles = (B * n + BM - 1) / BM;
    gr.num_n_tiles = ZP_RES_NT;
    gr.N = 4 * ZP_RES_KPER;
    gr.nkb = 256 / BK;
    gr.Kp = 256;
    gr.Mvalid = B * n;
    gr.Bvalid = B;
    gr.rowsumA = ckrs;
    gr.colsum = ctx->d_resw_cs;
    gr.status = ctx->d_status;
    gr.rns = ctx->d_rns;
    gr.res_n = n;
    gr.res_bt = BT;
    gr.res_nnt = nnt;
    gr.res_kp = Kp;
    gr.res_out = Bc;
    rc = launch_gemm<MODE_RES, 64, true>(ctx, tmC, ctx->tmap_resw, gr, st);
    if (rc) return rc;
    zp_clear_pending_error();
    ctx->launches++;
    k_fp16_rowsum<<<(unsigned)((brows * 32 + 255) / 256), 256, 0, st>>>(Bc, brows, Kp, colsum);
    ZP_CUDA(cudaGetLastError());
  }
  CUtensorMap tmB;
  rc = zp_encode_tmap_2d(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Bc, Kp, brows, (uint64_t)Kp * 2, 64,
                         N, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  GemmArgs ga{};
  ga.num_m_tiles = ZP_RNS_K * (db->Rq / 32);
  ga.num_n_tiles = nnt;
  ga.N = N;
  ga.nkb = Kp / BK;
  ga.Kp = Kp;
  ga.Mvalid = db->d1p;
  ga.Bvalid = B;
  ga.rowsumA = db->d_rns_rowsum;
  ga.colsum = colsum;
  ga.out = X;
  ga.out_ld = 0;
  ga.status = ctx->d_status;
  ga.mt_per_prime = db->Rq / 32;
  ga.d1p = db->d1p;
  ga.Rp = db->Rq;  // out[b][k][r'], r' < Rq
  ga.rns = ctx->d_rns;
  if (db->d_rns16 && ctx->answer_fp16) {  // the resident fp16 copy of the residue planes
    if (BT == 16) return launch_gemm<MODE_RNS, 16, true>(ctx, db->tmap_rns16, tmB, ga, st);
    if (BT == 32) return launch_gemm<MODE_RNS, 32, true>(ctx, db->tmap_rns16, tmB, ga, st);
    return launch_gemm<MODE_RNS, 64, true>(ctx, db->tmap_rns16, tmB, ga, st);
  }
  if (BT == 16) return launch_gemm<MODE_RNS, 16>(ctx, db->tmap_rns, tmB, ga, st);
  if (BT == 32) return launch_gemm<MODE_RNS, 32>(ctx, db->tmap_rns, tmB, ga, st);
  return launch_gemm<MODE_RNS, 64>(ctx, db->tmap_rns, tmB, ga, st);
}

// ---------------------------------------------------------------------------------
// CRT products of the residue-number-system compression (Sec. 5.2: one reduction mod m at
// the end): V[b][r'] = sum_k y[b][r'][k] (M/p_k mod m_b) + alpha (m_b - (M mod m_b))
// + sum_{j<ell} gamma^j ans[b][r' ell + j], i.e. the Chinese-remainder sum of the residues of
// H'[r', :] . cko[b] plus the packed answer b' (congruent to b' + H'.cko mod m_b, below
// 2^2087), taken exactly on the tensor cores (MODE_CRT): for query b, A = the byte planes of
// its y, alpha and answers (k_crt_prep; packed row r' is row b Rq + r', its plane a at bytes
// a Kp .., K = ZP_RNS_K + 1 + ell per plane), B = the 256 bytes of each of its client's
// constants M/p_k mod m_b (read in place through mkm_ptrs[b * ptr_stride]) followed by those
// of gamma^j (the context's table). The four planes run along K against the constants' bytes
// shifted by a, so one accumulator row is a whole packed row and its 259 byte columns are V's
// base-256 digits before carries; the columns are taken in two halves of 144.
int zp_launch_crt_products(zp_db* db, const uint32_t* const* mkm_ptrs, uint32_t ptr_stride,
                           uint32_t B, const uint8_t* Yp, uint32_t ypitch, const uint32_t* yrs,
                           uint32_t* Vc, cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  // K per plane padded to a K block (the planes lie one after the other in each row of Yp,
  // ypitch = 4 Kp); 4 Kp <= 1024 keeps every partial sum of the fp32 accumulator below 2^24
  const uint32_t KC = zp_crt_k(ctx), Kp = (KC + BK - 1) / BK * BK;
  if (ypitch != 4 * Kp) return zp_set_error(ZP_EINVAL, "CRT product: row pitch %u", ypitch);
  if (4 * Kp > (uint32_t)(KCHUNK * BK)) return zp_set_error(ZP_EINVAL, "CRT product: K %u too large", KC);
  const size_t bm_bytes = (size_t)B * 256 * Kp * 2, cs_bytes = (size_t)B * 256 * 4;
  int rc = zp_scratch_reserve(&db->s_crtb, bm_bytes + cs_bytes + 256);
  if (rc) return rc;
  __half* Bm = static_cast<__half*>(db->s_crtb.p);
  uint32_t* colsum = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(db->s_crtb.p) + bm_bytes);
  ZP_CUDA(cudaMemsetAsync(colsum, 0, cs_bytes, st));
  zp_clear_pending_error();
  ctx->launches++;
  k_prep_cko<<<dim3(Kp / PREP_IB, B), 256, 0, st>>>(nullptr, ZP_RNS_K + 1, Kp, Bm, colsum, mkm_ptrs,
                                                ptr_stride, ctx->d_gam, ctx->ell);
  ZP_CUDA(cudaGetLastError());
  constexpr uint32_t NH = 144;  // columns per half (two halves cover byte positions 0..287)
  CUtensorMap tmA, tmB;
  rc = zp_encode_tmap_2d(&tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, Yp, 4 * Kp, (uint64_t)B * db->Rq, ypitch,
                         128, 128, CU_TENSOR_MAP_SWIZZLE_128B);
  if (!rc)
    rc = zp_encode_tmap_3d(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Bm, Kp, 256, B, (uint64_t)Kp * 2,
                           (uint64_t)256 * Kp * 2, 64, NH, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  GemmArgs ga{};
  ga.num_m_tiles = (db->d1p + BM - 1) / BM;
  ga.num_n_tiles = B;
  ga.N = NH;
  ga.nkb = 4 * Kp / BK;
  ga.Kp = Kp;
  ga.Mvalid = db->d1p;
  ga.Bvalid = B;
  ga.rowsumA = yrs;
  ga.colsum = colsum;
  ga.out = Vc;
  ga.Rp = db->Rq;
  ga.a_rows_per_n = 4 * db->Rq;
  ga.status = ctx->d_status;
  return launch_gemm<MODE_CRT, 64>(ctx, tmA, tmB, ga, st);
}
