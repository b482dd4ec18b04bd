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
#define ZP_MAX_L 64        // limbs of m (key_bits / 32); this build: 2048-bit keys
#define ZP_VW (ZP_MAX_L + 3)  // words of one exact row product V = H[row,:] . cko (< 2^(32L+42))
#define ZP_XW 128          // words of the packed sum before reduction (< 2^4096)

// device-side status codes (bit flags OR-ed into the context's status word)
#define ZP_DEV_TIMEOUT_GEMV 0x1u
#define ZP_DEV_TIMEOUT_GEMM 0x2u
#define ZP_DEV_TIMEOUT_MISC 0x4u

struct zp_ctx {
  int device;
  zp_params P;
  uint32_t ell;        // slots per packed row
  uint32_t L;          // limbs per element of Z_m
  uint32_t gamma_w[3]; // packing scale gamma, little-endian 32-bit words (gamma < 2^96)
  int num_sms;
  uint32_t* d_status;  // device status word (ZP_DEV_* flags)
  uint64_t launches;   // kernels launched by this context
};

struct zp_client {
  zp_ctx* ctx;
  int device;
  uint32_t L;
  uint32_t* d_m;   // L limbs
  uint32_t* d_mu;  // L+1 limbs: floor(2^(64 L) / m)  (Barrett constant)
};

struct zp_scratch {
  void* p = nullptr;
  size_t bytes = 0;
};

struct zp_db {
  zp_ctx* ctx;
  int device;
  const uint8_t* dD;  // caller-owned, R rows of ld bytes
  uint32_t R, C;
  uint64_t ld;
  uint32_t d1p;
  uint32_t* d_rowsum;      // R: sum_c D[r][c]
  CUtensorMap tmap_gemv;   // D as a 2-D u8 tensor, box 256 x 64
  // hint in compression layout (library-owned)
  uint32_t* d_hneg;        // R x n u32: -D.A mod 2^32
  bool hint_ready;
  uint32_t stale;          // rows updated since the last hint generation
  std::vector<uint8_t> stale_v;  // per-row stale flags (host)
  // scratch, grown on demand (never shrunk before zp_db_destroy)
  zp_scratch s_qplanes, s_v, s_q, s_cko, s_ans, s_t, s_clients, s_misc;
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

// Clears a pending runtime error left by an unrelated earlier call, so that the
// check after a launch reports only that launch.
static inline void zp_clear_pending_error() { (void)cudaGetLastError(); }

// tensor-map encoding through the driver entry point (no link-time libcuda dependency)
int zp_encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t dim0,
                      uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1,
                      CUtensorMapSwizzle swz);

// ------------------------------------------------------------------ kernel launchers
// (defined in the k_*.cu translation units; all asynchronous on `st`)
int zp_launch_rowsum(const zp_db* db, const uint32_t* rows, uint32_t nrows, cudaStream_t st);
int zp_launch_gemv(zp_db* db, const uint32_t* dq, uint32_t* dans, cudaStream_t st);
int zp_launch_answer_simt(zp_db* db, const uint32_t* dQ, uint32_t B, uint32_t ldq,
                          uint32_t* dOut, uint64_t out_stride_b, uint64_t out_stride_r,
                          const uint8_t* dDrows, uint32_t Rrows, uint64_t ld, cudaStream_t st);
int zp_launch_hint_post(zp_db* db, const uint32_t* dHplus_compact, const uint32_t* rows,
                        uint32_t nrows, uint32_t* dH, cudaStream_t st);
int zp_launch_compress(zp_db* db, zp_client* const* clients, const uint32_t* dAns,
                       const uint32_t* dCKO, uint32_t B, uint32_t* dT, cudaStream_t st);
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

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

#endif  // __CUDACC__
