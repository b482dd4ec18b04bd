// k_gemv.cu -- the LWE answer of one to four queries (Algorithm "ZipPIR", Response,
// first line):  ans[b][r] = sum_c D[r][c] * q_b[c]  mod 2^32.
//
// Design (GB300, HBM-bound): D is streamed once through a TMA ring of 64 x 256-byte
// tiles (cp.async.bulk.tensor, L2 evict-first), the query is pre-split into its four
// byte planes q = sum_k 2^(8k) q_k so that one dp4a multiplies four database bytes by
// four plane bytes, and each thread keeps one 32-bit accumulator per (row, plane).
// Accumulators wrap mod 2^32, which is exact because (x mod 2^32) 2^(8k) = x 2^(8k)
// mod 2^32. Work is split "stream-K" style: the tile sequence (row block, column
// tile) is cut into one contiguous range per CTA, so every CTA streams the same
// number of bytes; a CTA adds its partial row sums to ans with atomicAdd, which is
// order-independent under wrap-around, so the result is deterministic. A batch of two to
// four queries is answered in the same single pass over D (BQ query plane sets per tile):
// the pass is HBM-bound for two queries and bound by dp4a issue beyond (about 19 T dp4a/s
// on the whole GPU), still well ahead of the tensor-core path for such small batches.
#include <atomic>
#include <cstdio>
#include <mutex>

#include "zp_internal.cuh"

namespace {

constexpr int TCB = 256;                 // bytes (= columns) per tile row
constexpr int QT_BYTES = 4 * 16 * 16;    // q planes of one column tile: 4 planes x 16 chunks x 16 B

// Two configurations, both with more than 114 KiB of shared memory so that an SM runs
// one GEMV CTA and nothing else (which also keeps the SM split of zp_respond clean):
//   <8 consumer warps, 12 stages of 64 x 256 bytes>   fastest on the whole GPU;
//   <16 consumer warps, 6 stages of 128 x 256 bytes>  larger TMA boxes and more warps,
//     about 40% more bytes per SM per second, used when the GEMV shares the GPU with
//     the compression products.
template <int NCW, int STAGES, int BQ = 1>
struct GemvCfg {
  static constexpr int TR = NCW * 8;  // rows per tile: 2 row groups of 4 rows per warp
  static constexpr int TILE_BYTES = TR * TCB;
  static constexpr int STAGE_BYTES = TILE_BYTES + BQ * QT_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 2 * STAGES * 8 + 16;
};
// rows per tile of the whole-GPU configuration (the tensor map db->tmap_gemv)
constexpr int TR = GemvCfg<8, 12>::TR;
constexpr int CTAS_PER_SM = 1;

// Byte planes of B queries (q_b[c] = q[b * C + c]) for the GEMV tile layout. Word index
//   (((ct * B + b) * 4 + k) * 16 + j) * 4 + w
// packs byte k of q_b[c] for c = ct*256 + j*16 + w*4 + i into bits 8i..8i+7 (i < 4);
// columns >= C give 0. Also zeroes ans[0 .. nans) (the GEMV accumulates into it).
__global__ void k_qplanes(const uint32_t* __restrict__ q, uint32_t C, uint32_t nct, uint32_t B,
                          uint32_t* __restrict__ qp, uint32_t* __restrict__ ans, uint64_t nans) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t total = nct * 256u * B;
  if (tid < total) {
    const uint32_t w = tid & 3u, j = (tid >> 2) & 15u, k = (tid >> 6) & 3u, cb = tid >> 8;
    const uint32_t b = cb % B, ct = cb / B;
    const uint32_t c0 = ct * 256u + j * 16u + w * 4u;
    uint32_t v = 0;
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
      const uint32_t c = c0 + i;
      const uint32_t x = c < C ? q[(uint64_t)b * C + c] : 0u;
      v |= ((x >> (8u * k)) & 0xFFu) << (8u * i);
    }
    qp[tid] = v;
  }
  for (uint64_t r = tid; r < nans; r += (uint64_t)gridDim.x * blockDim.x) ans[r] = 0u;
}

template <int NCW, int STAGES, int BQ = 1>
__global__ void __launch_bounds__((NCW + 1) * 32, 1)
    k_gemv(const __grid_constant__ CUtensorMap tmap, const uint32_t* __restrict__ qp,
           uint32_t* __restrict__ ans, uint32_t R, uint32_t nrb, uint32_t nct,
           uint32_t* status) {
  using G = GemvCfg<NCW, STAGES, BQ>;
  constexpr int TR = G::TR, TILE_BYTES = G::TILE_BYTES, STAGE_BYTES = G::STAGE_BYTES;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(empty + STAGES);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t T = (uint64_t)nrb * nct;
  const uint64_t t_begin = T * blockIdx.x / gridDim.x;
  const uint64_t t_end = T * (blockIdx.x + 1) / gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    *abort_flag = 0u;
    fence_mbar_init();
  }
  __syncthreads();
  if (t_begin >= t_end) return;

  if (warp == NCW) {  // ---------------- producer warp: one elected lane issues copies
    if (lane == 0) {
      prefetch_tmap(&tmap);
      const uint64_t pol = l2_policy_evict_first();
      uint32_t issued = 0;
      for (uint64_t t = t_begin; t < t_end; ++t, ++issued) {
        const uint32_t s = issued % STAGES, round = issued / STAGES;
        if (round > 0 && !mbar_wait_abortable(&empty[s], (round - 1) & 1u, abort_flag, status,
                                              ZP_DEV_TIMEOUT_GEMV))
          break;
        const uint32_t rb = (uint32_t)(t / nct), ct = (uint32_t)(t % nct);
        uint8_t* st = smem + s * STAGE_BYTES;
        mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
        tma_load_2d_hint(st, &tmap, (int32_t)(ct * TCB), (int32_t)(rb * TR), &full[s], pol);
        bulk_load(st + TILE_BYTES, qp + (size_t)ct * 256u * BQ, BQ * QT_BYTES, &full[s]);
      }
      // Stay alive until every copy this thread issued has landed (one bounded deadline).
      const uint32_t first = issued > STAGES ? issued - STAGES : 0;
      const unsigned long long deadline = clock64() + ZP_WAIT_CYCLES;
      for (uint32_t i = first; i < issued; ++i)
        if (!mbar_wait_until(&full[i % STAGES], (i / STAGES) & 1u, deadline)) {
          atomicOr(status, ZP_DEV_TIMEOUT_GEMV);
          break;
        }
    }
    return;
  }

  // ---------------- consumer warps
  const uint32_t j = lane & 15u;                   // 16-byte chunk of the 256-byte tile row
  const uint32_t rg = warp * 2u + (lane >> 4);     // row group: rows 4 rg .. 4 rg + 3
  uint32_t acc[4][BQ][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int b = 0; b < BQ; ++b)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[r][b][k] = 0u;

  auto flush = [&](uint32_t rb) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t row = rb * TR + rg * 4u + (uint32_t)r;
#pragma unroll
      for (int b = 0; b < BQ; ++b) {
        uint32_t v = acc[r][b][0] + (acc[r][b][1] << 8) + (acc[r][b][2] << 16) +
                     (acc[r][b][3] << 24);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (j == 0 && row < R) atomicAdd(&ans[(uint64_t)b * R + row], v);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[r][b][k] = 0u;
      }
    }
  };

  uint32_t cur_rb = (uint32_t)(t_begin / nct);
  uint32_t consumed = 0;
  bool ok = true;
  for (uint64_t t = t_begin; t < t_end; ++t, ++consumed) {
    const uint32_t rb = (uint32_t)(t / nct);
    if (rb != cur_rb) {
      flush(cur_rb);
      cur_rb = rb;
    }
    const uint32_t s = consumed % STAGES, round = consumed / STAGES;
    if (!mbar_wait_abortable(&full[s], round & 1u, abort_flag, status, ZP_DEV_TIMEOUT_GEMV)) {
      ok = false;
      break;
    }
    const uint8_t* st = smem + s * STAGE_BYTES;
    const uint4* qv = reinterpret_cast<const uint4*>(st + TILE_BYTES);
    uint4 qk[BQ][4];
#pragma unroll
    for (int b = 0; b < BQ; ++b)
#pragma unroll
      for (int k = 0; k < 4; ++k) qk[b][k] = qv[(b * 4 + k) * 16 + j];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint4 d = *reinterpret_cast<const uint4*>(st + (rg * 4 + r) * TCB + j * 16);
#pragma unroll
      for (int b = 0; b < BQ; ++b)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint32_t a = acc[r][b][k];
          a = __dp4a(d.x, qk[b][k].x, a);
          a = __dp4a(d.y, qk[b][k].y, a);
          a = __dp4a(d.z, qk[b][k].z, a);
          a = __dp4a(d.w, qk[b][k].w, a);
          acc[r][b][k] = a;
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (ok) flush(cur_rb);
}

// per device: the kernel attributes are set (atomic flags: two host threads may both set
// them, which is harmless)
std::atomic<bool> g_attr_done[64];

}  // namespace

namespace {
// Stage counts of the multi-query configurations (8 consumer warps, 64-row tiles), as
// many 16 KiB + BQ KiB stages as shared memory holds.
template <int BQ>
struct MultiStages {
  static constexpr int value = BQ == 2 ? 12 : 11;
};

template <int BQ>
int launch_gemv_multi(zp_db* db, const uint32_t* qp, uint32_t* dans, uint32_t nct,
                      cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  constexpr int S = MultiStages<BQ>::value;
  using G = GemvCfg<8, S, BQ>;
  static std::atomic<bool> attr_done[64];
  if (!attr_done[ctx->device & 63]) {
    ZP_CUDA(cudaFuncSetAttribute(k_gemv<8, S, BQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 G::SMEM_BYTES));
    attr_done[ctx->device & 63] = true;
  }
  const uint32_t nrbs = (db->R + G::TR - 1) / G::TR;
  const uint64_t T = (uint64_t)nrbs * nct;
  uint64_t grid = (uint64_t)ctx->num_sms * CTAS_PER_SM;
  if (grid > T) grid = T;
  zp_clear_pending_error();
  ctx->launches++;
  k_gemv<8, S, BQ><<<(unsigned)grid, 9 * 32, G::SMEM_BYTES, st>>>(db->tmap_gemv, qp, dans, db->R,
                                                                   nrbs, nct, ctx->d_status);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}
}  // namespace

int zp_launch_gemv(zp_db* db, const uint32_t* dq, uint32_t B, uint32_t* dans, cudaStream_t st,
                   uint32_t max_ctas) {
  zp_ctx* ctx = db->ctx;
  if (B < 1 || B > 4) return zp_set_error(ZP_EINVAL, "zp_launch_gemv: B=%u (1..4)", B);
  const uint32_t nct = (db->C + TCB - 1) / TCB;
  const size_t qp_bytes = (size_t)nct * QT_BYTES * B;
  int rc = zp_scratch_reserve(&db->s_qplanes, qp_bytes);
  if (rc) return rc;
  uint32_t* qp = static_cast<uint32_t*>(db->s_qplanes.p);
  {
    const uint32_t total = nct * 256u * B;
    const uint32_t blocks = (total + 255) / 256;
    zp_clear_pending_error();
    ctx->launches++;
    k_qplanes<<<blocks, 256, 0, st>>>(dq, db->C, nct, B, qp, dans, (uint64_t)B * db->R);
  }
  if (B == 2) return launch_gemv_multi<2>(db, qp, dans, nct, st);
  if (B == 3) return launch_gemv_multi<3>(db, qp, dans, nct, st);
  if (B == 4) return launch_gemv_multi<4>(db, qp, dans, nct, st);
  const bool shared_gpu = max_ctas && max_ctas < (uint32_t)ctx->num_sms;
  const bool wide = ctx->gemv_cfg[shared_gpu ? 1 : 0] == 2;  // 16 warps x 128-row tiles
  if (!g_attr_done[ctx->device & 63]) {
    ZP_CUDA(cudaFuncSetAttribute(k_gemv<8, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 GemvCfg<8, 12>::SMEM_BYTES));
    ZP_CUDA(cudaFuncSetAttribute(k_gemv<16, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 GemvCfg<16, 6>::SMEM_BYTES));
    g_attr_done[ctx->device & 63] = true;
  }
  const uint32_t tr = wide ? GemvCfg<16, 6>::TR : GemvCfg<8, 12>::TR;
  const uint32_t nrbs = (db->R + tr - 1) / tr;
  const uint64_t T = (uint64_t)nrbs * nct;
  uint64_t grid = (uint64_t)ctx->num_sms * CTAS_PER_SM;
  if (max_ctas && grid > max_ctas) grid = max_ctas;
  if (grid > T) grid = T;
  zp_clear_pending_error();
  ctx->launches++;
  if (wide)
    k_gemv<16, 6><<<(unsigned)grid, 17 * 32, GemvCfg<16, 6>::SMEM_BYTES, st>>>(
        db->tmap_gemv128, qp, dans, db->R, nrbs, nct, ctx->d_status);
  else
    k_gemv<8, 12><<<(unsigned)grid, 9 * 32, GemvCfg<8, 12>::SMEM_BYTES, st>>>(
        db->tmap_gemv, qp, dans, db->R, nrbs, nct, ctx->d_status);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

// ---------------------------------------------------------------------------------
// zp_answer_noalloc: the single-query answer for callers that must not allocate
// device memory. Its only scratch, the query byte planes, lives in this file-scope
// device array instead of library-allocated memory; every GPU that loads the
// library holds these 1 MiB until the process exits. In host code the array's name
// is only a host-side stand-in, so its device address is looked up once per device
// (cudaGetSymbolAddress, with that device current) and passed to the kernels.
#define ZP_NOALLOC_MAX_C (1u << 18)  // columns: 1024 tiles x 1 KiB of planes = 1 MiB
static __device__ __align__(256) uint32_t g_noalloc_qplanes[(ZP_NOALLOC_MAX_C / TCB) * 256];

namespace {
std::mutex g_noalloc_mu;
uint32_t* g_noalloc_planes[64] = {nullptr};
}  // namespace

extern "C" int zp_answer_noalloc(zp_db* db, const uint32_t* dQ, uint32_t* dAns, void* stream) {
  if (!db || !dQ || !dAns) return zp_set_error(ZP_EINVAL, "zp_answer_noalloc: null argument");
  zp_view_sync(db);
  if (db->C > ZP_NOALLOC_MAX_C)
    return zp_set_error(ZP_EINVAL,
                        "zp_answer_noalloc: C=%u exceeds the %u columns its static buffer holds",
                        db->C, ZP_NOALLOC_MAX_C);
  const int dev = db->device;
  if (dev < 0 || dev >= 64) return zp_set_error(ZP_EINVAL, "zp_answer_noalloc: device %d", dev);
  ZP_ON_DEVICE(dev);
  uint32_t* qp;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_planes[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_qplanes);
      if (e != cudaSuccess) return zp_cuda_check(e, "zp_answer_noalloc: cudaGetSymbolAddress");
      g_noalloc_planes[dev] = static_cast<uint32_t*>(p);
    }
    qp = g_noalloc_planes[dev];
  }
  zp_ctx* ctx = db->ctx;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t nct = (db->C + TCB - 1) / TCB;
  const uint32_t nrb = (db->R + TR - 1) / TR;
  zp_clear_pending_error();
  ctx->launches++;
  k_qplanes<<<(nct * 256u + 255) / 256, 256, 0, st>>>(dQ, db->C, nct, 1u, qp, dAns, db->R);
  ZP_CUDA(cudaGetLastError());
  if (!g_attr_done[dev & 63]) {
    ZP_CUDA(cudaFuncSetAttribute(k_gemv<8, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 GemvCfg<8, 12>::SMEM_BYTES));
    ZP_CUDA(cudaFuncSetAttribute(k_gemv<16, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 GemvCfg<16, 6>::SMEM_BYTES));
    g_attr_done[dev & 63] = true;
  }
  const uint64_t T = (uint64_t)nrb * nct;
  uint64_t grid = (uint64_t)ctx->num_sms * CTAS_PER_SM;
  if (grid > T) grid = T;
  zp_clear_pending_error();
  ctx->launches++;
  k_gemv<8, 12><<<(unsigned)grid, 9 * 32, GemvCfg<8, 12>::SMEM_BYTES, st>>>(
      db->tmap_gemv, qp, dAns, db->R, nrb, nct, ctx->d_status);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}
