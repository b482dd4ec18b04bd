// k_rns.cu -- the packed hint H' modulo the RNS primes, the operand of the compression of
// large batches (Sec. 5.2 computes H'.ck_o modulo word-size primes and reduces once at the
// end; Sec. 4.3 "Reusability of the offline phase": H' is shared by all clients).
//
//   H'[r', i] mod p = sum_{j < ell} (gamma^j mod p) Hneg[r' ell + j, i] mod p
//
// for the ZP_RNS_K primes p (< 2^27), stored as the four byte planes of each residue in
// the layout of the tensor-core product: row k 4 Rq + 128 g + 32 a + t holds byte a of
// H'[32 g + t, :] mod p_k. Built once per database (about a second per GiB of database at
// n = 1024) and for the packed rows of updated rows after each hint regeneration.
#include <cuda_fp16.h>

#include "zp_internal.cuh"

namespace {

// x mod p for x < 2^64, p < 2^32, mu = floor((2^64 - 1) / p): the estimate is at most one
// short (Barrett).
__device__ __forceinline__ uint32_t mod_p(uint64_t x, uint32_t p, uint64_t mu) {
  const uint64_t q = __umul64hi(x, mu);
  const uint64_t r = x - q * p;
  return (uint32_t)(r >= p ? r - p : r);
}

constexpr int KG = 32;  // primes per thread

// grid (ceil(n / 128), listed packed rows, ceil(K / KG)); one thread per column.
__global__ void __launch_bounds__(128) k_rns_planes(const uint32_t* __restrict__ hneg, uint32_t n,
                                                    uint32_t R, uint32_t ell,
                                                    const uint32_t* __restrict__ prows, uint32_t Rq,
                                                    const zp_rns_dev* __restrict__ rns,
                                                    uint8_t* __restrict__ planes, uint64_t ld) {
  __shared__ uint32_t sg[KG][64];
  __shared__ uint32_t sp[KG];
  __shared__ uint64_t smu[KG];
  const uint32_t k0 = blockIdx.z * KG;
  const uint32_t kn = ZP_RNS_K - k0 < (uint32_t)KG ? ZP_RNS_K - k0 : (uint32_t)KG;
  for (uint32_t x = threadIdx.x; x < KG * 64; x += blockDim.x) {
    const uint32_t kk = x / 64, j = x % 64;
    sg[kk][j] = kk < kn && j < ell ? rns->gj[k0 + kk][j] : 0u;
  }
  for (uint32_t kk = threadIdx.x; kk < (uint32_t)KG; kk += blockDim.x) {
    sp[kk] = kk < kn ? rns->p[k0 + kk] : 1u;
    smu[kk] = kk < kn ? rns->mu[k0 + kk] : 0ull;
  }
  __syncthreads();
  const uint32_t i = blockIdx.x * 128 + threadIdx.x;
  if (i >= n) return;
  const uint32_t rp = prows ? prows[blockIdx.y] : blockIdx.y;
  uint64_t acc[KG];
#pragma unroll
  for (int kk = 0; kk < KG; ++kk) acc[kk] = 0;
  for (uint32_t j = 0; j < ell; ++j) {
    const uint32_t row = rp * ell + j;
    const uint32_t h = row < R ? __ldg(hneg + (uint64_t)row * n + i) : 0u;
#pragma unroll
    for (int kk = 0; kk < KG; ++kk) acc[kk] += (uint64_t)h * sg[kk][j];  // < 2^59 per term
    if ((j & 15u) == 15u) {  // 16 terms and a residue stay below 2^64
#pragma unroll
      for (int kk = 0; kk < KG; ++kk) acc[kk] = mod_p(acc[kk], sp[kk], smu[kk]);
    }
  }
  const uint64_t rowbase = 128ull * (rp >> 5) + (rp & 31u);
#pragma unroll
  for (int kk = 0; kk < KG; ++kk) {
    if ((uint32_t)kk < kn) {
      const uint32_t v = mod_p(acc[kk], sp[kk], smu[kk]);
      uint8_t* dst = planes + ((uint64_t)(k0 + kk) * 4 * Rq + rowbase) * ld + i;
#pragma unroll
      for (int a = 0; a < 4; ++a) dst[(uint64_t)32 * a * ld] = (uint8_t)(v >> (8 * a));
    }
  }
}

// Byte sums of the plane rows of the listed packed rows: one warp per (prime, packed row, plane).
__global__ void k_rns_rowsum(const uint8_t* __restrict__ planes, uint64_t ld, uint32_t n,
                             const uint32_t* __restrict__ prows, uint32_t nprows, uint32_t Rq,
                             uint32_t* __restrict__ out) {
  const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (wid >= (uint64_t)ZP_RNS_K * nprows * 4) return;
  const uint32_t a = (uint32_t)(wid & 3u);
  const uint32_t idx = (uint32_t)((wid >> 2) % nprows);
  const uint32_t k = (uint32_t)((wid >> 2) / nprows);
  const uint32_t rp = prows ? prows[idx] : idx;
  const uint64_t row = (uint64_t)k * 4 * Rq + 128ull * (rp >> 5) + 32 * a + (rp & 31u);
  const uint8_t* src = planes + row * ld;
  uint32_t s = 0;
  for (uint32_t i = lane; i < n; i += 32) s += src[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[row] = s;
}

// Centred fp16 copy of the plane rows of the listed packed rows: row k 4 Rq + 128 g + 32 a
// + t (rp = 32 g + t) for every prime k and plane a, columns < Kp (n rounded up to 128),
// value byte - 128 (-128 in the padding). grid (ceil(Kp / 2048), nprows, ZP_RNS_K * 4).
__global__ void k_rns16_rows(const uint8_t* __restrict__ planes, uint64_t ld, uint32_t n,
                             uint32_t Kp, const uint32_t* __restrict__ prows, uint32_t Rq,
                             __half* __restrict__ out) {
  const uint32_t k0 = blockIdx.x * 2048 + threadIdx.x * 8;
  if (k0 >= Kp) return;
  const uint32_t rp = prows ? prows[blockIdx.y] : blockIdx.y;
  const uint32_t k = blockIdx.z >> 2, a = blockIdx.z & 3u;
  const uint64_t row = (uint64_t)k * 4 * Rq + 128ull * (rp >> 5) + 32 * a + (rp & 31u);
  const uint8_t* src = planes + row * ld;
  uint32_t h[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t c0 = k0 + 2 * j, c1 = c0 + 1;
    const int v0 = c0 < n ? (int)src[c0] : 0, v1 = c1 < n ? (int)src[c1] : 0;
    const __half2 x = __halves2half2(__int2half_rn(v0 - 128), __int2half_rn(v1 - 128));
    h[j] = *reinterpret_cast<const uint32_t*>(&x);
  }
  *reinterpret_cast<uint4*>(out + row * Kp + k0) = make_uint4(h[0], h[1], h[2], h[3]);
}

}  // namespace

int zp_launch_rns16_rows(zp_db* db, const uint32_t* dRows, uint32_t nprows, cudaStream_t st) {
  if (nprows == 0 || !db->d_rns16) return ZP_OK;
  const uint32_t Kp = (db->ctx->P.n + 127) / 128 * 128;
  zp_clear_pending_error();
  db->ctx->launches++;
  k_rns16_rows<<<dim3((Kp + 2047) / 2048, nprows, ZP_RNS_K * 4), 256, 0, st>>>(
      db->d_rns_hpl, db->hpl_ld, db->ctx->P.n, Kp, dRows, db->Rq, static_cast<__half*>(db->d_rns16));
  ZP_CUDA(cudaGetLastError());
  return ZP_OK;
}

int zp_launch_rns_planes(zp_db* db, const uint32_t* dRows, uint32_t nprows, cudaStream_t st) {
  zp_ctx* ctx = db->ctx;
  if (nprows == 0) return ZP_OK;
  const uint32_t n = ctx->P.n;
  zp_clear_pending_error();
  ctx->launches += 2;
  dim3 grid((n + 127) / 128, nprows, (ZP_RNS_K + KG - 1) / KG);
  k_rns_planes<<<grid, 128, 0, st>>>(db->d_hneg, n, db->R, ctx->ell, dRows, db->Rq, ctx->d_rns,
                                     db->d_rns_hpl, db->hpl_ld);
  ZP_CUDA(cudaGetLastError());
  const uint64_t warps = (uint64_t)ZP_RNS_K * nprows * 4;
  k_rns_rowsum<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
      db->d_rns_hpl, db->hpl_ld, n, dRows, nprows, db->Rq, db->d_rns_rowsum);
  ZP_CUDA(cudaGetLastError());
  return zp_launch_rns16_rows(db, dRows, nprows, st);  // keeps the fp16 copy current, if any
}
