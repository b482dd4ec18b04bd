// zp_internal.cuh -- internal declarations shared by the library's translation units:
// handle layouts, error reporting, and sm_103a device helpers (mbarrier, TMA bulk
// copies, tensor maps) written as inline PTX.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/zippir.h"

// ------------------------------------------------------------------ host-side state
#define ZP_MAX_L 64        // limbs of m (key_bits / 32); the library is compiled for 2048-bit keys
#define ZP_VW (ZP_MAX_L + 3)  // words of one exact row product V = H[row,:] . cko (< 2^(32L+42))
#define ZP_XW 128          // words of the packed sum before reduction (< 2^4096)

// device-side status codes (bit flags OR-ed into the context's status word)
#define ZP_DEV_TIMEOUT_GEMV 0x1u
#define ZP_DEV_TIMEOUT_GEMM 0x2u
#define ZP_DEV_TIMEOUT_MISC 0x4u

// kernel-path options (zp_set_option)
#define ZP_PATH_AUTO 0
#define ZP_PATH_SIMT 1
#define ZP_PATH_TC 2
#define ZP_PATH_RNS 3  // compression only: residue number system on the tensor cores

// Residue number system of the batched compression: ZP_RNS_K primes just below 2^27 whose
// product (4131 bits) exceeds every H'.ck_o (< n 2^4095 <= 2^4105) by a margin of 2^26.
#define ZP_RNS_K 153
struct zp_rns_dev {             // device copy, one per context
  uint32_t p[ZP_RNS_K];         // the primes
  uint32_t inv[ZP_RNS_K];       // (M / p)^{-1} mod p, M = prod p
  uint64_t mu[ZP_RNS_K];        // floor((2^64 - 1) / p) (Barrett reduction of 64-bit values)
  double dinv[ZP_RNS_K];        // 1 / p
  uint32_t w32[ZP_RNS_K][ZP_MAX_L];  // 2^(32 w) mod p
  uint32_t gj[ZP_RNS_K][64];    // gamma^j mod p, j < ell
  uint32_t pow8[ZP_RNS_K][8];   // 2^(8 a) mod p, a < 8
};

// Residues of the compression offsets on the tensor cores: the table of the bytes of
// 2^(8 beta) mod p_k (beta < 256), ZP_RES_KPER primes per N tile of the product.
#define ZP_RES_KPER 40
#define ZP_RES_NT ((ZP_RNS_K + ZP_RES_KPER - 1) / ZP_RES_KPER)
#define ZP_RES_ROWS (4 * ZP_RES_KPER * ZP_RES_NT)

struct zp_ctx {
  int device;
  zp_params P;
  int answer_path;     // ZP_PATH_* for batched answers and the hint
  int compress_path;   // ZP_PATH_* for the compression products
  uint32_t overlap_sms;  // SMs given to the compression products while a single-query
                         // answer runs on the others (0: no overlap)
  uint32_t ell;        // slots per packed row
  uint32_t L;          // limbs per element of Z_m
  uint32_t gamma_w[3]; // packing scale gamma, little-endian 32-bit words (gamma < 2^96)
  uint32_t rns_min_batch;  // batches of at least this many queries compress in RNS (0: never)
  uint32_t gemv_max_batch; // batches of at most this many queries (<= 4) answer by the GEMV
  uint32_t answer_fp16;    // tensor-core answers read a database's fp16 copy when it has one
  uint32_t batch_overlap;  // zp_respond runs a batch's compression products beside its answers
  uint32_t pack_split;     // one query: the V part of the packing runs beside the answer
  // tile widths (queries per N tile: 16, 32 or 64) of the tensor-core answers and of the RNS
  // products for batches of <= 16, <= 32, <= 64 and > 64 queries (zp_autotune measures them)
  uint32_t ans_bt[4], rns_bt[4];
  // GEMV configuration on the whole GPU [0] and beside the compression products [1]:
  // 1 = 8 consumer warps x 12 stages of 64 rows, 2 = 16 warps x 6 stages of 128 rows
  uint32_t gemv_cfg[2];
  zp_rns_dev* d_rns;   // RNS constants (device)
  // ZP_RES_ROWS x 256 centred fp16: row 4 k + c, column beta = byte c of 2^(8 beta) mod p_k
  // (zero bytes for k >= ZP_RNS_K), its row byte sums, and its tensor map (built on first use)
  void* d_resw;
  uint32_t* d_resw_cs;
  CUtensorMap tmap_resw;
  uint32_t* d_gam;     // ell x ZP_MAX_L words: gamma^j, j < ell (each < 2^(key_bits - 1))
  std::vector<uint32_t> rns_p;  // the primes (host)
  int num_sms;
  uint32_t* d_status;  // device status word (ZP_DEV_* flags)
  uint64_t launches;   // kernels launched by this context
};

struct zp_client {
  zp_ctx* ctx;
  int device;
  uint32_t L;
  std::vector<uint32_t> h_m;  // L limbs (host copy)
  uint32_t* d_m;   // L limbs
  uint32_t* d_mu;  // L+1 limbs: floor(2^(64 L) / m)  (Barrett constant)
  // Montgomery arithmetic mod m^2 (R = 2^(64 L)): per-client hint k, combined response
  uint32_t* d_m2;  // 2L limbs: m^2
  uint32_t* d_r1;  // 2L limbs: R mod m^2
  uint32_t* d_r2;  // 2L limbs: R^2 mod m^2
  uint32_t m2inv;  // -(m^2)^{-1} mod 2^32
  // CRT of the RNS compression: M_k mod m (ZP_RNS_K x L limbs), then m - (M mod m) (L limbs)
  uint32_t* d_mkm;
  // 2^(32 w) mod m for w = L .. 2L - 1 (L x L limbs): folds the high words of the packed
  // sum before its reduction mod m
  uint32_t* d_pow;
};

struct zp_scratch {
  void* p = nullptr;
  size_t bytes = 0;
};

struct zp_db {
  zp_db* base;        // a view (zp_db_view): the database whose state it shares; else null
  zp_ctx* ctx;
  int device;
  const uint8_t* dD;  // caller-owned, R rows of ld bytes
  uint32_t R, C;
  uint64_t ld;
  uint32_t d1p;
  uint32_t Rp;             // R rounded up to 32 (rows of the hint byte-plane layout)
  uint32_t* d_rowsum;      // R: sum_c D[r][c]
  CUtensorMap tmap_gemv;   // D as a 2-D u8 tensor, box 256 x 64 (GEMV on the whole GPU)
  CUtensorMap tmap_gemv128;  // box 256 x 128 (GEMV beside the compression products)
  CUtensorMap tmap_gemm;   // D as a 2-D u8 tensor, box 64 x 128 (tensor-core products)
  // resident centred fp16 copy of D (R x Kp, Kp = C rounded up to 128; built on request):
  // the A operand of the tensor-core answers without conversion in shared memory
  void* d_D16;
  CUtensorMap tmap_d16;    // box 64 x 128, 128-byte swizzle
  // hint in compression layout (library-owned)
  uint32_t* d_hneg;        // R x n u32: -D.A mod 2^32
  uint8_t* d_hpl;          // 4 Rp x lda bytes: row 128 g + 32 a + t = byte a of d_hneg row 32 g + t
  uint32_t* d_hpl_rowsum;  // 4 Rp: byte sums of d_hpl rows
  uint64_t hpl_ld;         // row pitch of d_hpl (n rounded up to 16)
  CUtensorMap tmap_hpl;    // d_hpl as a 2-D u8 tensor, box 64 x 128
  bool hint_ready;
  uint32_t stale;          // rows updated since the last hint generation
  std::vector<uint8_t> stale_v;  // per-row stale flags (host)
  uint32_t v_batch;        // queries whose products are in s_v (0: none)
  bool v_rns;              // s_v holds RNS residues (else exact row products V)
  // H' modulo the RNS primes as byte planes (lazily built for the first RNS batch):
  // row k 4 Rq + 128 g + 32 a + t = byte a of H'[32 g + t, :] mod p_k, Rq = d1' rounded up to 32
  uint8_t* d_rns_hpl;
  uint32_t* d_rns_rowsum;  // byte sums of its rows
  uint32_t Rq;
  CUtensorMap tmap_rns;    // box 64 x 128
  // their centred fp16 copy (rows x Kp, Kp = n rounded up to 128), built when the database
  // has its fp16 copy of D: the A operand of the RNS products without conversion
  void* d_rns16;
  CUtensorMap tmap_rns16;
  std::vector<const uint32_t*> cl_cache;  // client constants last uploaded to s_clients
  cudaStream_t side;       // internal stream of zp_respond's overlap (lazily created)
  cudaEvent_t ev_fork, ev_join;
  // scratch, grown on demand (never shrunk before zp_db_destroy)
  zp_scratch s_qplanes, s_v, s_q, s_cko, s_ans, s_t, s_clients, s_misc, s_tcq, s_hq, s_hcko;
  zp_scratch s_ptab, s_krows, s_m2consts;  // per-client hint and combined response
  zp_scratch s_prows;                      // packed rows whose RNS planes are rebuilt
  zp_scratch s_crt, s_crtb;                // CRT of the residue-number-system compression
  zp_scratch s_ypack;                      // split packing: (sum_j gamma^j V_j) mod m per packed row
};

// error reporting (thread-local message)
int zp_set_error(int code, const char* fmt, ...);
int zp_cuda_check(cudaError_t e, const char* what);
#define ZP_CUDA(call)                                                 \
  do {                                                                \
    cudaError_t _e = (call);                                          \
    if (_e != cudaSuccess) return zp_cuda_check(_e, #call);           \
  } while (0)

int zp_scratch_reserve(zp_scratch* s, size_t bytes);

// A view reads its database's shared state (hint, planes, fp16 copies, RNS tables) at every
// call: copies the pointers and flags of db->base into the view (no-op for a database).
void zp_view_sync(zp_db* db);

// Makes `dev` the current device for the lifetime of the scope and gives the caller its
// own current device back at the end, so that no entry point changes it as a side effect.
struct zp_device_scope {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit zp_device_scope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev == dev)
      prev = -1;
    else
      err = cudaSetDevice(dev);
  }
  ~zp_device_scope() {
    if (prev >= 0) (void)cudaSetDevice(prev);
  }
  zp_device_scope(const zp_device_scope&) = delete;
  zp_device_scope& operator=(const zp_device_scope&) = delete;
};
#define ZP_ON_DEVICE(dev)                                                         \
  zp_device_scope _zp_scope(dev);                                                 \
  if (_zp_scope.err != cudaSuccess) return zp_cuda_check(_zp_scope.err, "cudaSetDevice")

// Clears a pending runtime error left by an unrelated earlier call, so that the
// check after a launch reports only that launch.
static inline void zp_clear_pending_error() { (void)cudaGetLastError(); }

// tensor-map encoding through the driver entry point (no link-time libcuda dependency)
int zp_encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t dim0,
                      uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1,
                      CUtensorMapSwizzle swz);
// 3-D map: dims (dim0, dim1, dim2), byte strides of dims 1 and 2, box (box0, box1, 1).
int zp_encode_tmap_3d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t dim0,
                      uint64_t dim1, uint64_t dim2, uint64_t stride1_bytes, uint64_t stride2_bytes,
                      uint32_t box0, uint32_t box1, CUtensorMapSwizzle swz);

// ------------------------------------------------------------------ kernel launchers
// (defined in the k_*.cu translation units; all asynchronous on `st`)
// tile width for a batch of B queries from a per-class table (B <= 16, <= 32, <= 64, > 64)
static inline uint32_t zp_pick_bt(const uint32_t (&table)[4], uint32_t B) {
  return table[B <= 16 ? 0 : (B <= 32 ? 1 : (B <= 64 ? 2 : 3))];
}
int zp_launch_rowsum(const zp_db* db, const uint32_t* rows, uint32_t nrows, cudaStream_t st);
int zp_launch_rowsum_buf(zp_ctx* ctx, const uint8_t* M, uint64_t ld, uint32_t rows, uint32_t cols,
                         uint32_t* out, cudaStream_t st);
int zp_launch_copy_rows(const uint8_t* src, uint64_t lds, uint8_t* dst, uint64_t ldd, uint32_t C,
                        const uint32_t* rows, uint32_t cnt, int gather, cudaStream_t st);
int zp_launch_answer_tc(zp_db* db, const CUtensorMap& tmD, uint32_t Rrows, const uint32_t* dQ,
                        uint32_t B, bool q_cols, uint32_t* dOut, uint64_t out_ld, bool hint,
                        const uint32_t* rowsum, cudaStream_t st, bool a16 = false);
// the fp16 copy of the listed rows of D (dRows device, NULL = all R) (k_gemm_tc.cu)
int zp_launch_d16_rows(zp_db* db, const uint32_t* dRows, uint32_t nrows, cudaStream_t st);
int zp_launch_vmul_tc(zp_db* db, const uint32_t* dCKO, uint32_t B, uint32_t* V4, cudaStream_t st,
                      uint32_t max_ctas);
int zp_launch_hint_planes_rowsum(zp_db* db, const uint32_t* rows, uint32_t nrows, cudaStream_t st);
// per-client hint k of the listed packed rows (dRows device, NULL = all d1'), and the
// combined response k (+) t (k_paillier.cu)
int zp_launch_client_hint(zp_db* db, const zp_client* cl, const uint32_t* dCkr, uint32_t* dK,
                          const uint32_t* dRows, uint32_t nprows, cudaStream_t st);
int zp_launch_combine(zp_db* db, zp_client* const* clients, const uint32_t* dK, const uint32_t* dT,
                      uint32_t B, uint32_t* dOut, cudaStream_t st);
// Paillier decryption of count ciphertexts with the exponent e = lambda mu (ew words) and
// minv = m^{-1} mod 2^(32 L) (L words), both host arrays (k_paillier.cu)
int zp_launch_decrypt(const zp_client* cl, const uint32_t* e, uint32_t ew, const uint32_t* minv,
                      const uint32_t* dC, uint32_t* dOut, uint32_t count, cudaStream_t st);
// RNS compression (k_rns.cu, k_gemm_tc.cu): the residue planes of H' for the listed packed
// rows (dRows device, NULL = all), the B operand of ck_o residues, and the residue product
// X[b][k][r'] = H'[r', :] . cko[b] mod p_k (row pitch Rq)
int zp_launch_rns_planes(zp_db* db, const uint32_t* dRows, uint32_t nprows, cudaStream_t st);
// allocates and builds the RNS planes of H' on first use (zp_api.cu)
int zp_ensure_rns(zp_db* db, cudaStream_t st);
// builds the context's table of 2^(8 beta) mod p_k on first use (zp_api.cu)
int zp_ensure_res_table(zp_ctx* c);
// the fp16 copy of the RNS plane rows of the listed packed rows (dRows device; NULL = packed
// rows 0 .. nprows - 1, the padding rows up to Rq included) (k_rns.cu)
int zp_launch_rns16_rows(zp_db* db, const uint32_t* dRows, uint32_t nprows, cudaStream_t st);
// builds the fp16 copy of the RNS planes when the database has both (zp_api.cu)
int zp_ensure_rns16(zp_db* db, cudaStream_t st);
int zp_launch_rns_products(zp_db* db, const uint32_t* dCKO, uint32_t B, uint32_t* X, cudaStream_t st);
// the exact CRT sums V[b][r'] (67 words, Rq rows per query) from the byte planes Yp of y and
// alpha (B x 4 Rq rows of ypitch bytes, row sums yrs) and the clients' constants M/p_k mod m
// read through mkm_ptrs[b * ptr_stride] (k_gemm_tc.cu)
int zp_launch_crt_products(zp_db* db, const uint32_t* const* mkm_ptrs, uint32_t ptr_stride,
                           uint32_t B, const uint8_t* Yp, uint32_t ypitch, const uint32_t* yrs,
                           uint32_t* Vc, cudaStream_t st);
// columns of the CRT product's K: ZP_RNS_K residues, alpha, then the ell answers of b'
static inline uint32_t zp_crt_k(const zp_ctx* c) { return ZP_RNS_K + 1 + c->ell; }
// B in 1..4 queries (dq: B x C, dans: B x R); max_ctas limits the single-query grid.
int zp_launch_gemv(zp_db* db, const uint32_t* dq, uint32_t B, uint32_t* dans, cudaStream_t st,
                   uint32_t max_ctas);
int zp_launch_answer_simt(zp_db* db, const uint32_t* dQ, uint32_t B, uint32_t ldq,
                          uint32_t* dOut, uint64_t out_stride_b, uint64_t out_stride_r,
                          const uint8_t* dDrows, uint32_t Rrows, uint64_t ld, cudaStream_t st);
int zp_launch_hint_post(zp_db* db, const uint32_t* dHplus_compact, const uint32_t* rows,
                        uint32_t nrows, uint32_t* dH, cudaStream_t st);
int zp_launch_compress_products(zp_db* db, const uint32_t* dCKO, uint32_t B, cudaStream_t st,
                                uint32_t max_ctas);
// split packing of one query (zp_respond): Y = (sum_j gamma^j V_j) mod m beside the answer,
// then t = (b' + Y) mod m after the join (k_compress.cu)
int zp_launch_pack_products(zp_db* db, zp_client* const* clients, uint32_t B, cudaStream_t st);
int zp_launch_pack_answers(zp_db* db, const uint32_t* dAns, uint32_t B, uint32_t* dT,
                           cudaStream_t st);
int zp_launch_compress_finish(zp_db* db, zp_client* const* clients, const uint32_t* dAns,
                              uint32_t B, uint32_t* dT, cudaStream_t st);
int zp_launch_update_rows(zp_db* db, const uint32_t* rows, uint32_t k, const uint8_t* dNew,
                          cudaStream_t st);

// ------------------------------------------------------------------ device helpers
#ifdef __CUDACC__

// Bounded waits: a wait that has not completed after this many cycles sets a
// status flag and gives up (about 2 s at GB300 clocks).
#define ZP_WAIT_CYCLES (1ull << 32)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar` to complete. Returns false (and sets `flag` in
// *status) if it has not completed within ZP_WAIT_CYCLES.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t* status, uint32_t flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if ((unsigned long long)(clock64() - t0) > ZP_WAIT_CYCLES) {
      if (status) atomicOr(status, flag);
      return false;
    }
  }
  return true;
}

// 2-D tiled TMA load (tile mode) completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t x,
                                            int32_t y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 3-D tiled TMA load (tile mode) completing on `bar`; coordinates outside the tensor read
// as zero (x must stay a multiple of 16 bytes).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int32_t x,
                                            int32_t y, int32_t z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// 2-D tiled TMA load with an L2 cache-policy hint.
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, int32_t x,
                                                 int32_t y, uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Prefetches a 2-D tile of a tensor into L2 (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_l2_2d(const CUtensorMap* map, int32_t x, int32_t y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Waits for phase `parity` of `bar` until the absolute clock64 deadline; false when it
// passes (used to drain copies in flight before a CTA leaves).
__device__ __forceinline__ bool mbar_wait_until(uint64_t* bar, uint32_t parity,
                                                unsigned long long deadline) {
  while (!mbar_try_wait(bar, parity))
    if ((unsigned long long)clock64() > deadline) return false;
  return true;
}

// ---- bounded waits that also give up when another role of the CTA has aborted
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t* bar, uint32_t parity,
                                                    volatile uint32_t* abort_flag,
                                                    uint32_t* status, uint32_t flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if ((unsigned long long)(clock64() - t0) > ZP_WAIT_CYCLES) {
      *abort_flag = 1u;
      if (status) atomicOr(status, flag);
      return false;
    }
  }
}

// ---- tcgen05 (5th-generation tensor cores, tensor memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, fp16 inputs, fp32 accumulators, one CTA.
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives on `bar` once every tcgen05 operation issued so far by this thread completes.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// 8 / 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
// 32 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Shared-memory matrix descriptor for a K-major operand stored with the 128-byte
// swizzle (8-row atoms of 128-byte rows, atoms 1024 bytes apart). Fields: start
// address >> 4 (bits 0-13), leading-dimension offset >> 4 (bits 16-29; unused for
// this layout, 1), stride-dimension offset >> 4 (bits 32-45: 1024 bytes between
// 8-row groups), descriptor version 1 (bits 46-47), swizzle mode 2 = 128-byte
// (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}
// Instruction descriptor of kind::f16 with fp16 A and B, fp32 accumulators, both
// operands K-major: D format F32 (bits 4-5 = 1), A/B format F16 (bits 7-9, 10-12 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ __forceinline__ uint32_t idesc_f16_f32(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

#endif  // __CUDACC__
