// k_simt.cu -- CUDA-core kernels around the hot path: database row sums, a dp4a
// multi-query product for small batches and for the hint, hint post-processing
// (H = -H+ mod 2^32, scatter of regenerated rows) and database row updates.
#include "zp_internal.cuh"

namespace {

// rowsum[r] = sum_c D[r][c] (exact: at most 255 * 2^20 < 2^28). One warp per row.
__global__ void k_rowsum(const uint8_t* __restrict__ D, uint64_t ld, uint32_t R, uint32_t C,
                         const uint32_t* __restrict__ rows, uint32_t nrows,
                         uint32_t* __restrict__ rowsum) {
  const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t cnt = rows ? nrows : R;
  if (wid >= cnt) return;
  const uint32_t r = rows ? rows[wid] : wid;
  const uint8_t* row = D + (uint64_t)r * ld;
  uint32_t s = 0;
  for (uint32_t c = lane * 16; c < C; c += 32 * 16) {
    if (c + 16 <= C) {
      const uint4 v = *reinterpret_cast<const uint4*>(row + c);
      s = __dp4a(v.x, 0x01010101u, s);
      s = __dp4a(v.y, 0x01010101u, s);
      s = __dp4a(v.z, 0x01010101u, s);
      s = __dp4a(v.w, 0x01010101u, s);
    } else {
      for (uint32_t cc = c; cc < C; ++cc) s += row[cc];
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) rowsum[r] = s;
}

// Multi-query dp4a product on CUDA cores:
//   out[b * osb + r * osr] = sum_c D[r][c] * Q(b, c) mod 2^32,  Q(b, c) = Qp[b * qsb + c * qsc].
// CTA tile: 64 rows x 32 queries, K step 64 bytes. Thread: 2 rows x 4 queries x 4 planes.
constexpr int SB_R = 64, SB_Q = 32, SB_K = 64;
constexpr int DS_PITCH = SB_K / 4 + 1;  // words per smem row (+1 word against bank conflicts)

__global__ void __launch_bounds__(256)
    k_answer_simt(const uint8_t* __restrict__ D, uint64_t ld, uint32_t R, uint32_t C,
                  const uint32_t* __restrict__ Qp, uint64_t qsb, uint64_t qsc, uint32_t B,
                  uint32_t* __restrict__ out, uint64_t osb, uint64_t osr) {
  __shared__ uint32_t Ds[SB_R][DS_PITCH];
  __shared__ uint32_t Qs[4][SB_Q][SB_K / 4];  // plane k, query, word (4 columns)
  const uint32_t tid = threadIdx.x;
  const uint32_t r0 = blockIdx.x * SB_R, b0 = blockIdx.y * SB_Q;
  const uint32_t tr = tid & 31, tq = tid >> 5;  // rows 2tr, 2tr+1; queries 4tq..4tq+3
  uint32_t acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0u;

  for (uint32_t c0 = 0; c0 < C; c0 += SB_K) {
    {  // D tile: 64 rows x 64 bytes; thread loads 16 bytes. Bytes >= C meet zero q planes.
      const uint32_t rr = tid >> 2, ch = tid & 3;
      const uint32_t r = r0 + rr, c = c0 + ch * 16;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (r < R && c < C) v = *reinterpret_cast<const uint4*>(D + (uint64_t)r * ld + c);
      Ds[rr][ch * 4 + 0] = v.x;
      Ds[rr][ch * 4 + 1] = v.y;
      Ds[rr][ch * 4 + 2] = v.z;
      Ds[rr][ch * 4 + 3] = v.w;
    }
    // Q planes: 32 queries x 16 words; thread handles 2 (query, word) pairs
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t pair = tid + h * 256;
      const uint32_t qq = pair >> 4, w = pair & 15;
      const uint32_t b = b0 + qq;
      uint32_t x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t c = c0 + w * 4 + i;
        x[i] = (b < B && c < C) ? Qp[(uint64_t)b * qsb + (uint64_t)c * qsc] : 0u;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t v = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) v |= ((x[i] >> (8 * k)) & 0xFFu) << (8 * i);
        Qs[k][qq][w] = v;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int w = 0; w < SB_K / 4; ++w) {
      const uint32_t d0 = Ds[2 * tr][w], d1 = Ds[2 * tr + 1][w];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t qv = Qs[k][tq * 4 + j][w];
          acc[0][j][k] = __dp4a(d0, qv, acc[0][j][k]);
          acc[1][j][k] = __dp4a(d1, qv, acc[1][j][k]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const uint32_t r = r0 + 2 * tr + i;
    if (r >= R) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t b = b0 + tq * 4 + j;
      if (b >= B) continue;
      const uint32_t v = acc[i][j][0] + (acc[i][j][1] << 8) + (acc[i][j][2] << 16) +
                         (acc[i][j][3] << 24);
      out[(uint64_t)b * osb + (uint64_t)r * osr] = v;
    }
  }
}

// Hint post-processing. src: compact H+ rows (cnt x n). For compact row j the
// database row is rows ? rows[j] : j. Writes H+ into dH (if not null) and
// -H+ mod 2^32 into hneg, both R x n row-major.
__global__ void k_hint_post(const uint32_t* __restrict__ src, uint32_t cnt, uint32_t n,
                            const uint32_t* __restrict__ rows, uint32_t* __restrict__ dH,
                            uint32_t* __restrict__ hneg, uint8_t* __restrict__ hpl,
                            uint64_t hpl_ld) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)cnt * n) return;
  const uint32_t j = (uint32_t)(idx / n), i = (uint32_t)(idx % n);
  const uint32_t r = rows ? rows[j] : j;
  const uint32_t v = src[idx];
  const uint64_t o = (uint64_t)r * n + i;
  if (dH && (rows || dH != src)) dH[o] = v;
  const uint32_t h = 0u - v;
  hneg[o] = h;
  // byte planes: row 128 g + 32 a + t of hpl holds byte a of hint row 32 g + t
  const uint64_t base = (uint64_t)(r >> 5) * 128 + (r & 31);
#pragma unroll
  for (uint32_t a = 0; a < 4; ++a) hpl[(base + 32 * a) * hpl_ld + i] = (uint8_t)(h >> (8 * a));
}

// Byte sums of the 4 plane rows of each listed hint row (all rows if rows == NULL).
__global__ void k_hpl_rowsum(const uint8_t* __restrict__ hpl, uint64_t ld, uint32_t n,
                             const uint32_t* __restrict__ rows, uint32_t cnt,
                             uint32_t* __restrict__ out) {
  const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (wid >= cnt * 4u) return;
  const uint32_t j = wid >> 2, a = wid & 3;
  const uint32_t r = rows ? rows[j] : j;
  const uint64_t m = (uint64_t)(r >> 5) * 128 + 32 * a + (r & 31);
  const uint8_t* row = hpl + m * ld;
  uint32_t s = 0;
  for (uint32_t i = lane; i < n; i += 32) s += row[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[m] = s;
}

// Gather rows of D into a compact buffer (pitch ldc), or scatter new rows into D.
__global__ void k_copy_rows(const uint8_t* __restrict__ src, uint64_t lds, uint8_t* __restrict__ dst,
                            uint64_t ldd, uint32_t C, const uint32_t* __restrict__ rows,
                            uint32_t cnt, int gather) {
  const uint32_t j = blockIdx.x;
  if (j >= cnt) return;
  const uint32_t r = rows[j];
  const uint8_t* s = gather ? src + (uint64_t)r * lds : src + (uint64_t)j * lds;
  uint8_t* d = gather ? dst + (uint64_t)j * ldd : dst + (uint64_t)r * ldd;
  for (uint32_t c = threadIdx.x; c < C; c += blockDim.x) d[c] = s[c];
}

}  // namespace

int zp_launch_rowsum(const zp_db* db, const uint32_t* rows, uint32_t nrows, cudaStream_t st) {
  const uint32_t cnt = rows ? nrows : db->R;
  if (cnt == 0) return ZP_OK;
  const uint32_t blocks = (cnt * 32u + 255u) / 256u;
  zp_clear_pending_error();
  db->ctx->launches++;
  k_rowsum<<<blocks, 256, 0, st>>>(db->dD, db->ld, db->R, db->C, rows, nrows, db->d_rowsum);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

int zp_launch_rowsum_buf(zp_ctx* ctx, const uint8_t* M, uint64_t ld, uint32_t rows, uint32_t cols,
                         uint32_t* out, cudaStream_t st) {
  if (rows == 0) return ZP_OK;
  const uint32_t blocks = (rows * 32u + 255u) / 256u;
  zp_clear_pending_error();
  ctx->launches++;
  k_rowsum<<<blocks, 256, 0, st>>>(M, ld, rows, cols, nullptr, 0, out);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

int zp_launch_hint_planes_rowsum(zp_db* db, const uint32_t* rows, uint32_t nrows, cudaStream_t st) {
  const uint32_t cnt = rows ? nrows : db->R;
  if (cnt == 0) return ZP_OK;
  const uint32_t blocks = (cnt * 4u * 32u + 255u) / 256u;
  zp_clear_pending_error();
  db->ctx->launches++;
  k_hpl_rowsum<<<blocks, 256, 0, st>>>(db->d_hpl, db->hpl_ld, db->ctx->P.n, rows, cnt,
                                        db->d_hpl_rowsum);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

int zp_launch_answer_simt(zp_db* db, const uint32_t* dQ, uint32_t B, uint32_t ldq,
                          uint32_t* dOut, uint64_t out_stride_b, uint64_t out_stride_r,
                          const uint8_t* dDrows, uint32_t Rrows, uint64_t ld, cudaStream_t st) {
  // ldq == 0 means the hint layout: Q(b, c) = A[c][b] with A of width B.
  const uint64_t qsb = ldq ? ldq : 1u;
  const uint64_t qsc = ldq ? 1u : B;
  dim3 grid((Rrows + SB_R - 1) / SB_R, (B + SB_Q - 1) / SB_Q);
  zp_clear_pending_error();
  db->ctx->launches++;
  k_answer_simt<<<grid, 256, 0, st>>>(dDrows, ld, Rrows, db->C, dQ, qsb, qsc, B, dOut,
                                      out_stride_b, out_stride_r);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

int zp_launch_hint_post(zp_db* db, const uint32_t* src, const uint32_t* rows, uint32_t cnt,
                        uint32_t* dH, cudaStream_t st) {
  const uint32_t n = db->ctx->P.n;
  const uint64_t total = (uint64_t)cnt * n;
  if (total == 0) return ZP_OK;
  zp_clear_pending_error();
  db->ctx->launches++;
  k_hint_post<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(src, cnt, n, rows, dH, db->d_hneg,
                                                              db->d_hpl, db->hpl_ld);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

int zp_launch_copy_rows(const uint8_t* src, uint64_t lds, uint8_t* dst, uint64_t ldd, uint32_t C,
                        const uint32_t* rows, uint32_t cnt, int gather, cudaStream_t st) {
  if (cnt == 0) return ZP_OK;
  k_copy_rows<<<cnt, 256, 0, st>>>(src, lds, dst, ldd, C, rows, cnt, gather);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

// ---------------------------------------------------------------------------------
// Failure-detection self-test: one mbarrier wait that nothing satisfies, bounded by
// `cycles` SM clock cycles. It gives up the way every bounded wait of the library does:
// a bit in the context's status word, then return (no trap, no fault).
namespace {
__global__ void k_selftest_wait(unsigned long long cycles, uint32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_until(&bar, 0, clock64() + cycles))
    atomicOr(status, ZP_DEV_TIMEOUT_MISC);
  __syncthreads();
}
}  // namespace

extern "C" int zp_selftest_wait(zp_ctx* c, uint64_t cycles, void* stream) {
  if (!c) return zp_set_error(ZP_EINVAL, "zp_selftest_wait: null argument");
  if (cycles > (1ull << 32))
    return zp_set_error(ZP_EINVAL, "zp_selftest_wait: cycles=%llu above 2^32", (unsigned long long)cycles);
  ZP_ON_DEVICE(c->device);
  zp_clear_pending_error();
  c->launches++;
  k_selftest_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(cycles, c->d_status);
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}
