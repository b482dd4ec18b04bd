// zp_api.cu -- host side of the C ABI declared in include/zippir.h: argument
// validation, handle lifetime, per-client constants, scratch management and the
// dispatch to the kernels of the online Response (Algorithm "ZipPIR").
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "zp_internal.cuh"

#define ZP_VERSION_NUM 100  // 0.1.0

static thread_local std::string g_err;

int zp_set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int zp_cuda_check(cudaError_t e, const char* what) {
  return zp_set_error(ZP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int zp_scratch_reserve(zp_scratch* s, size_t bytes) {
  if (bytes <= s->bytes) return ZP_OK;
  if (s->p) {
    cudaError_t e = cudaFree(s->p);
    s->p = nullptr;
    s->bytes = 0;
    if (e != cudaSuccess) return zp_cuda_check(e, "cudaFree(scratch)");
  }
  const size_t want = bytes + bytes / 4 + 256;
  cudaError_t e = cudaMalloc(&s->p, want);
  if (e != cudaSuccess) {
    s->p = nullptr;
    return zp_set_error(ZP_ENOMEM, "cudaMalloc(%zu bytes): %s", want, cudaGetErrorString(e));
  }
  s->bytes = want;
  return ZP_OK;
}

static void scratch_free(zp_scratch* s) {
  if (s->p) cudaFree(s->p);
  s->p = nullptr;
  s->bytes = 0;
}

// ------------------------------------------------------------------ tensor maps
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode_fn() {
  // looked up once; the initialisation of a function-local static is thread-safe
  static const PFN_encodeTiled fn = []() -> PFN_encodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_encodeTiled>(p);
    return nullptr;
  }();
  return fn;
}

int zp_encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t dim0,
                      uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1,
                      CUtensorMapSwizzle swz) {
  PFN_encodeTiled fn = get_encode_fn();
  if (!fn) return zp_set_error(ZP_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
  cuuint64_t dims[2] = {dim0, dim1};
  cuuint64_t strides[1] = {stride1_bytes};
  cuuint32_t box[2] = {box0, box1};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return zp_set_error(ZP_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return ZP_OK;
}

int zp_encode_tmap_3d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t dim0,
                      uint64_t dim1, uint64_t dim2, uint64_t stride1_bytes, uint64_t stride2_bytes,
                      uint32_t box0, uint32_t box1, CUtensorMapSwizzle swz) {
  PFN_encodeTiled fn = get_encode_fn();
  if (!fn) return zp_set_error(ZP_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
  cuuint64_t dims[3] = {dim0, dim1, dim2};
  cuuint64_t strides[2] = {stride1_bytes, stride2_bytes};
  cuuint32_t box[3] = {box0, box1, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return zp_set_error(ZP_ECUDA, "cuTensorMapEncodeTiled (3-D) failed (%d)", (int)r);
  return ZP_OK;
}

// ------------------------------------------------------------------ small host bignum helpers
// little-endian u32 words
static void big_mul_small(std::vector<uint32_t>& a, const uint32_t* g, int gw) {
  std::vector<uint32_t> r(a.size() + gw + 1, 0);
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t carry = 0;
    for (int j = 0; j < gw; ++j) {
      uint64_t t = (uint64_t)a[i] * g[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    size_t k = i + gw;
    while (carry) {
      uint64_t t = (uint64_t)r[k] + carry;
      r[k] = (uint32_t)t;
      carry = t >> 32;
      ++k;
    }
  }
  while (r.size() > 1 && r.back() == 0) r.pop_back();
  a.swap(r);
}

static uint32_t big_bits(const std::vector<uint32_t>& a) {
  for (size_t i = a.size(); i-- > 0;)
    if (a[i]) return (uint32_t)(i * 32 + (32 - __builtin_clz(a[i])));
  return 0;
}

// schoolbook product of little-endian word vectors
static std::vector<uint32_t> big_mul(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  std::vector<uint32_t> r(a.size() + b.size(), 0);
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); ++j) {
      const uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    r[i + b.size()] = (uint32_t)carry;
  }
  return r;
}

// x mod m for x < b^(2L) by Barrett's reduction (HAC Alg. 14.42) with mu = floor(b^(2L) / m),
// b = 2^32 (the host twin of the reduction in k_compress.cu)
static std::vector<uint32_t> big_barrett(std::vector<uint32_t> x, const std::vector<uint32_t>& m,
                                         const std::vector<uint32_t>& mu) {
  const size_t L = m.size();
  x.resize(2 * L, 0);
  std::vector<uint32_t> q1(x.begin() + (L - 1), x.end());               // L+1 words
  std::vector<uint32_t> q2 = big_mul(q1, mu);
  std::vector<uint32_t> q3(q2.begin() + (L + 1), q2.begin() + (2 * L + 2));
  std::vector<uint32_t> r2 = big_mul(q3, m);
  std::vector<uint32_t> r(L + 1);
  uint64_t br = 0;
  for (size_t w = 0; w <= L; ++w) {  // r = x - q3 m mod b^(L+1)
    const uint64_t t = (uint64_t)x[w] - r2[w] - br;
    r[w] = (uint32_t)t;
    br = (t >> 63) & 1u;
  }
  for (;;) {  // at most twice
    bool ge = r[L] != 0;
    if (!ge) {
      ge = true;
      for (size_t w = L; w-- > 0;)
        if (r[w] != m[w]) {
          ge = r[w] > m[w];
          break;
        }
    }
    if (!ge) break;
    br = 0;
    for (size_t w = 0; w <= L; ++w) {
      const uint64_t t = (uint64_t)r[w] - (w < L ? m[w] : 0u) - br;
      r[w] = (uint32_t)t;
      br = (t >> 63) & 1u;
    }
  }
  r.resize(L);
  return r;
}

static uint64_t pow_mod_u64(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1;
  a %= p;
  while (e) {
    if (e & 1) r = (uint64_t)((unsigned __int128)r * a % p);
    a = (uint64_t)((unsigned __int128)a * a % p);
    e >>= 1;
  }
  return r;
}

static bool is_prime_u32(uint32_t x) {  // deterministic Miller-Rabin for 32-bit integers
  if (x < 2) return false;
  for (uint32_t q : {2u, 3u, 5u, 7u, 11u, 13u})
    if (x % q == 0) return x == q;
  uint32_t d = x - 1, sh = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++sh;
  }
  for (uint32_t a : {2u, 7u, 61u}) {
    uint64_t y = pow_mod_u64(a, d, x);
    if (y == 1 || y == x - 1) continue;
    bool comp = true;
    for (uint32_t i = 1; i < sh && comp; ++i) {
      y = y * y % x;
      if (y == x - 1) comp = false;
    }
    if (comp) return false;
  }
  return true;
}

// RNS constants of a context: the ZP_RNS_K largest primes below 2^27 and the tables of
// zp_rns_dev (host copy).
static bool rns_setup(zp_ctx* c, zp_rns_dev& h) {
  std::vector<uint32_t>& P = c->rns_p;
  P.clear();
  for (uint32_t x = (1u << 27) - 1; P.size() < ZP_RNS_K; x -= 2)
    if (is_prime_u32(x)) P.push_back(x);
  // the residue folds of the tensor-core products rely on p = 2^27 - dl with dl < 2^12
  // (the smallest of these primes is 2^27 - 2797)
  if ((1u << 27) - P.back() >= (1u << 12)) return false;
  memset(&h, 0, sizeof(h));
  for (int k = 0; k < ZP_RNS_K; ++k) {
    const uint64_t p = P[k];
    h.p[k] = (uint32_t)p;
    uint64_t mk = 1;  // M / p mod p
    for (int j = 0; j < ZP_RNS_K; ++j)
      if (j != k) mk = mk * (P[j] % p) % p;
    h.inv[k] = (uint32_t)pow_mod_u64(mk, p - 2, p);
    h.mu[k] = ~0ull / p;
    h.dinv[k] = 1.0 / (double)p;
    uint64_t w = 1;
    for (int i = 0; i < ZP_MAX_L; ++i) {
      h.w32[k][i] = (uint32_t)w;
      w = (w << 32) % p;
    }
    const uint64_t g = ((uint64_t)c->gamma_w[0] + ((uint64_t)c->gamma_w[1] << 32) % p +
                        (uint64_t)((((unsigned __int128)c->gamma_w[2]) << 64) % p)) % p;
    uint64_t gj = 1;
    for (int j = 0; j < 64; ++j) {
      h.gj[k][j] = (uint32_t)gj;
      gj = gj * g % p;
    }
    uint64_t p8 = 1 % p;
    for (int a = 0; a < 8; ++a, p8 = (p8 << 8) % p) h.pow8[k][a] = (uint32_t)p8;
  }
  return true;
}

// ------------------------------------------------------------------ context
extern "C" int zp_version(void) { return ZP_VERSION_NUM; }

extern "C" int zp_last_error(char* buf, size_t len) {
  if (buf && len) {
    size_t n = g_err.size() < len - 1 ? g_err.size() : len - 1;
    memcpy(buf, g_err.data(), n);
    buf[n] = 0;
  }
  return (int)g_err.size();
}

extern "C" int zp_init(int device, const zp_params* P, zp_ctx** out) {
  try {
    if (!P || !out) return zp_set_error(ZP_EINVAL, "zp_init: null argument");
    *out = nullptr;
    if (P->n < 1 || P->n > 4096) return zp_set_error(ZP_EINVAL, "zp_init: n=%u out of [1,4096]", P->n);
    if (P->p_bits != 8) return zp_set_error(ZP_EINVAL, "zp_init: p_bits must be 8");
    if (P->secret != ZP_SECRET_UNIFORM && P->secret != ZP_SECRET_BINARY)
      return zp_set_error(ZP_EINVAL, "zp_init: bad secret kind %u", P->secret);
    if (P->scale != ZP_SCALE_PROVEN && P->scale != ZP_SCALE_OVERLAP)
      return zp_set_error(ZP_EINVAL, "zp_init: bad scale %u", P->scale);
    if (P->key_bits != 32 * ZP_MAX_L)
      return zp_set_error(ZP_EUNSUPPORTED, "zp_init: key_bits=%u (compiled for %d)", P->key_bits,
                          32 * ZP_MAX_L);
    ZP_ON_DEVICE(device);
    zp_ctx* c = new zp_ctx();
    c->device = device;
    c->P = *P;
    c->L = P->key_bits / 32;
    // slot bound q + n q^2 (uniform secret) or q + n q (binary secret), q = 2^32; gamma is
    // the bound (proven scale) or q^2 / q (overlap scale)
    uint32_t bound_w[3] = {0, 1, P->n};
    if (P->secret == ZP_SECRET_BINARY) {
      bound_w[1] = 1 + P->n;
      bound_w[2] = 0;
    }
    if (P->scale == ZP_SCALE_PROVEN) {
      for (int k = 0; k < 3; ++k) c->gamma_w[k] = bound_w[k];
    } else {
      c->gamma_w[0] = 0;
      c->gamma_w[1] = P->secret == ZP_SECRET_UNIFORM ? 0u : 1u;
      c->gamma_w[2] = P->secret == ZP_SECRET_UNIFORM ? 1u : 0u;
    }
    // ell = largest count with (bound - 1) sum_{j<ell} gamma^j < 2^(key_bits - 1): the largest
    // packed value stays below every key of key_bits bits (for gamma = bound: gamma^ell <
    // 2^(key_bits - 1))
    {
      std::vector<uint32_t> bm1(bound_w, bound_w + 3);  // bound - 1 (bound >= 2^32)
      for (int k = 0; k < 3; ++k) {
        if (bm1[k]--) break;
      }
      std::vector<uint32_t> pw(1, 1), sum(1, 0);
      uint32_t ell = 0;
      for (;;) {
        std::vector<uint32_t> ns = sum;  // sum + gamma^ell
        ns.resize(std::max(ns.size(), pw.size()) + 1, 0);
        uint64_t cy = 0;
        for (size_t w = 0; w < ns.size(); ++w) {
          cy += (uint64_t)ns[w] + (w < pw.size() ? pw[w] : 0u);
          ns[w] = (uint32_t)cy;
          cy >>= 32;
        }
        std::vector<uint32_t> top = big_mul(ns, bm1);
        if (big_bits(top) > P->key_bits - 1) break;  // top >= 2^(key_bits-1)
        sum.swap(ns);
        big_mul_small(pw, c->gamma_w, 3);
        ++ell;
      }
      if (ell == 0) {
        delete c;
        return zp_set_error(ZP_EINVAL, "zp_init: key too small for one slot");
      }
      if (ell > 64) {
        delete c;
        return zp_set_error(ZP_EUNSUPPORTED, "zp_init: %u slots per packed row (at most 64)", ell);
      }
      c->ell = ell;
    }
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
      delete c;
      return zp_cuda_check(e, "cudaGetDeviceProperties");
    }
    c->num_sms = prop.multiProcessorCount;
    c->launches = 0;
    c->answer_path = ZP_PATH_AUTO;
    c->compress_path = ZP_PATH_AUTO;
    // from 8 queries on the RNS compression is faster (measured at 1 and 8 GiB, n = 1024)
    c->rns_min_batch = 8;
    c->gemv_max_batch = 4;  // one dp4a pass beats the tensor cores up to 4 queries (1 GiB)
    c->answer_fp16 = 1;
    c->batch_overlap = 1;
    c->pack_split = 1;
    for (int i = 0; i < 4; ++i) c->ans_bt[i] = c->rns_bt[i] = 16u << (i < 2 ? i : 2);  // 16, 32, 64, 64
    c->gemv_cfg[0] = 1;  // whole GPU: 8 warps x 12 stages
    c->gemv_cfg[1] = 2;  // beside the products: 16 warps x 6 stages
    {
      zp_rns_dev h;
      if (!rns_setup(c, h)) {
        delete c;
        return zp_set_error(ZP_EUNSUPPORTED, "zp_init: RNS primes too far below 2^27");
      }
      if (cudaMalloc(&c->d_rns, sizeof(zp_rns_dev)) != cudaSuccess) {
        c->d_rns = nullptr;
        delete c;
        return zp_set_error(ZP_ENOMEM, "cudaMalloc(RNS constants)");
      }
      if (cudaMemcpy(c->d_rns, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(c->d_rns);
        delete c;
        return zp_set_error(ZP_ECUDA, "copy of the RNS constants");
      }
    }
    // gamma^j (j < ell) as ZP_MAX_L-word integers: the packing weights of the answers in the
    // CRT product of the residue-number-system compression
    {
      std::vector<uint32_t> tab((size_t)c->ell * ZP_MAX_L, 0), pw(1, 1);
      for (uint32_t j = 0; j < c->ell; ++j) {
        for (size_t w = 0; w < pw.size() && w < ZP_MAX_L; ++w) tab[(size_t)j * ZP_MAX_L + w] = pw[w];
        big_mul_small(pw, c->gamma_w, 3);
      }
      if (cudaMalloc(&c->d_gam, tab.size() * 4) != cudaSuccess ||
          cudaMemcpy(c->d_gam, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        if (c->d_gam) cudaFree(c->d_gam);
        cudaFree(c->d_rns);
        delete c;
        return zp_set_error(ZP_ENOMEM, "zp_init: powers of gamma");
      }
    }
    // default SM split of zp_respond for one query: about 3/8 of the SMs run the
    // compression products beside the GEMV (56 of 152 on GB300)
    c->overlap_sms = c->num_sms >= 64 ? (uint32_t)(c->num_sms * 3 + 4) / 8 : 0u;
    e = cudaMalloc(&c->d_status, sizeof(uint32_t));
    if (e != cudaSuccess) {
      delete c;
      return zp_set_error(ZP_ENOMEM, "cudaMalloc(status)");
    }
    cudaMemset(c->d_status, 0, sizeof(uint32_t));
    *out = c;
    return ZP_OK;
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_init: host allocation failed");
  } catch (...) {
    return zp_set_error(ZP_EINVAL, "zp_init: unexpected exception");
  }
}

extern "C" int zp_ctx_destroy(zp_ctx* c) {
  if (!c) return ZP_OK;
  zp_device_scope _zp_scope(c->device);
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_rns) cudaFree(c->d_rns);
  if (c->d_resw) cudaFree(c->d_resw);
  if (c->d_gam) cudaFree(c->d_gam);
  if (c->d_resw_cs) cudaFree(c->d_resw_cs);
  delete c;
  return ZP_OK;
}

extern "C" int zp_set_option(zp_ctx* c, const char* name, int64_t value) {
  if (!c || !name) return zp_set_error(ZP_EINVAL, "zp_set_option: null argument");
  const std::string k(name);
  if (k == "answer_path" || k == "compress_path") {
    if (value < ZP_PATH_AUTO || value > (k == "compress_path" ? ZP_PATH_RNS : ZP_PATH_TC))
      return zp_set_error(ZP_EINVAL, "zp_set_option: %s=%lld out of range", name, (long long)value);
    (k == "answer_path" ? c->answer_path : c->compress_path) = (int)value;
    return ZP_OK;
  }
  if (k == "overlap_sms") {
    if (value < 0 || value >= c->num_sms)
      return zp_set_error(ZP_EINVAL, "zp_set_option: overlap_sms=%lld out of [0, %d)",
                          (long long)value, c->num_sms);
    c->overlap_sms = (uint32_t)value;
    return ZP_OK;
  }
  if (k == "gemv_max_batch") {
    if (value < 1 || value > 4)
      return zp_set_error(ZP_EINVAL, "zp_set_option: gemv_max_batch=%lld out of [1, 4]", (long long)value);
    c->gemv_max_batch = (uint32_t)value;
    return ZP_OK;
  }
  if (k == "answer_fp16") {
    if (value < 0 || value > 1)
      return zp_set_error(ZP_EINVAL, "zp_set_option: answer_fp16=%lld out of [0, 1]", (long long)value);
    c->answer_fp16 = (uint32_t)value;
    return ZP_OK;
  }
  static const char* bt_names[2][4] = {{"answer_bt_16", "answer_bt_32", "answer_bt_64", "answer_bt_128"},
                                       {"rns_bt_16", "rns_bt_32", "rns_bt_64", "rns_bt_128"}};
  for (int t = 0; t < 2; ++t)
    for (int cl = 0; cl < 4; ++cl)
      if (k == bt_names[t][cl]) {
        // at most the class's largest batch (16, 32, 64 queries; 64 for the class above 64)
        const int64_t most = 16 << (cl < 2 ? cl : 2);
        if ((value != 16 && value != 32 && value != 64) || value > most)
          return zp_set_error(ZP_EINVAL, "zp_set_option: %s=%lld (16, 32 or 64, at most %lld)", name,
                              (long long)value, (long long)most);
        (t ? c->rns_bt : c->ans_bt)[cl] = (uint32_t)value;
        return ZP_OK;
      }
  if (k == "gemv_cfg_alone" || k == "gemv_cfg_shared") {
    if (value != 1 && value != 2)
      return zp_set_error(ZP_EINVAL, "zp_set_option: %s=%lld (1 or 2)", name, (long long)value);
    c->gemv_cfg[k == "gemv_cfg_shared"] = (uint32_t)value;
    return ZP_OK;
  }
  if (k == "pack_split") {
    if (value < 0 || value > 1)
      return zp_set_error(ZP_EINVAL, "zp_set_option: pack_split=%lld out of [0, 1]", (long long)value);
    c->pack_split = (uint32_t)value;
    return ZP_OK;
  }
  if (k == "batch_overlap") {
    if (value < 0 || value > 1)
      return zp_set_error(ZP_EINVAL, "zp_set_option: batch_overlap=%lld out of [0, 1]", (long long)value);
    c->batch_overlap = (uint32_t)value;
    return ZP_OK;
  }
  if (k == "rns_min_batch") {
    if (value < 0 || value > 4096)
      return zp_set_error(ZP_EINVAL, "zp_set_option: rns_min_batch=%lld out of [0, 4096]", (long long)value);
    c->rns_min_batch = (uint32_t)value;
    return ZP_OK;
  }
  return zp_set_error(ZP_EINVAL, "zp_set_option: unknown option '%s'", name);
}

extern "C" int zp_get_option(const zp_ctx* c, const char* name, int64_t* value) {
  if (!c || !name || !value) return zp_set_error(ZP_EINVAL, "zp_get_option: null argument");
  const std::string k(name);
  if (k == "answer_path") *value = c->answer_path;
  else if (k == "compress_path") *value = c->compress_path;
  else if (k == "overlap_sms") *value = c->overlap_sms;
  else if (k == "rns_min_batch") *value = c->rns_min_batch;
  else if (k == "gemv_max_batch") *value = c->gemv_max_batch;
  else if (k == "answer_fp16") *value = c->answer_fp16;
  else if (k == "batch_overlap") *value = c->batch_overlap;
  else if (k == "pack_split") *value = c->pack_split;
  else if (k == "answer_bt_16") *value = c->ans_bt[0];
  else if (k == "answer_bt_32") *value = c->ans_bt[1];
  else if (k == "answer_bt_64") *value = c->ans_bt[2];
  else if (k == "answer_bt_128") *value = c->ans_bt[3];
  else if (k == "rns_bt_16") *value = c->rns_bt[0];
  else if (k == "rns_bt_32") *value = c->rns_bt[1];
  else if (k == "rns_bt_64") *value = c->rns_bt[2];
  else if (k == "rns_bt_128") *value = c->rns_bt[3];
  else if (k == "gemv_cfg_alone") *value = c->gemv_cfg[0];
  else if (k == "gemv_cfg_shared") *value = c->gemv_cfg[1];
  else return zp_set_error(ZP_EINVAL, "zp_get_option: unknown option '%s'", name);
  return ZP_OK;
}

extern "C" int zp_kernel_launches(const zp_ctx* c, uint64_t* count) {
  if (!c || !count) return zp_set_error(ZP_EINVAL, "zp_kernel_launches: null argument");
  *count = c->launches;
  return ZP_OK;
}

extern "C" int zp_device_status(zp_ctx* c, uint32_t* code) {
  if (!c || !code) return zp_set_error(ZP_EINVAL, "zp_device_status: null argument");
  ZP_ON_DEVICE(c->device);
  ZP_CUDA(cudaDeviceSynchronize());
  ZP_CUDA(cudaMemcpy(code, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  ZP_CUDA(cudaMemset(c->d_status, 0, sizeof(uint32_t)));
  return ZP_OK;
}

// ------------------------------------------------------------------ database
extern "C" int zp_setup_db(zp_ctx* c, const uint8_t* dD, uint32_t R, uint32_t C, uint64_t ld,
                           zp_db** out) {
  try {
    if (!c || !dD || !out) return zp_set_error(ZP_EINVAL, "zp_setup_db: null argument");
    *out = nullptr;
    if (R < 1 || R > (1u << 20) || C < 1 || C > (1u << 20))
      return zp_set_error(ZP_EINVAL, "zp_setup_db: R=%u C=%u out of [1, 2^20]", R, C);
    if (ld < C || ld % 16 != 0)
      return zp_set_error(ZP_EINVAL, "zp_setup_db: ld_bytes=%llu must be >= C and a multiple of 16",
                          (unsigned long long)ld);
    if (reinterpret_cast<uintptr_t>(dD) % 16 != 0)
      return zp_set_error(ZP_EINVAL, "zp_setup_db: database pointer not 16-byte aligned");
    ZP_ON_DEVICE(c->device);
    zp_db* db = new zp_db();
    db->ctx = c;
    db->device = c->device;
    db->dD = dD;
    db->R = R;
    db->C = C;
    db->ld = ld;
    db->d1p = (R + c->ell - 1) / c->ell;
    db->Rp = (R + 31) / 32 * 32;
    db->d_hneg = nullptr;
    db->d_hpl = nullptr;
    db->d_hpl_rowsum = nullptr;
    db->hpl_ld = ((uint64_t)c->P.n + 15) / 16 * 16;
    db->hint_ready = false;
    db->stale = 0;
    db->v_batch = 0;
    db->side = nullptr;
    db->ev_fork = db->ev_join = nullptr;
    cudaError_t e = cudaMalloc(&db->d_rowsum, (size_t)R * sizeof(uint32_t));
    if (e != cudaSuccess) {
      delete db;
      return zp_set_error(ZP_ENOMEM, "zp_setup_db: cudaMalloc(rowsum)");
    }
    int rc = zp_encode_tmap_2d(&db->tmap_gemv, CU_TENSOR_MAP_DATA_TYPE_UINT8, dD, C, R, ld, 256, 64,
                               CU_TENSOR_MAP_SWIZZLE_NONE);
    if (!rc)
      rc = zp_encode_tmap_2d(&db->tmap_gemv128, CU_TENSOR_MAP_DATA_TYPE_UINT8, dD, C, R, ld, 256, 128,
                             CU_TENSOR_MAP_SWIZZLE_NONE);
    if (!rc)
      rc = zp_encode_tmap_2d(&db->tmap_gemm, CU_TENSOR_MAP_DATA_TYPE_UINT8, dD, C, R, ld, 128, 128,
                             CU_TENSOR_MAP_SWIZZLE_128B);
    if (!rc) rc = zp_launch_rowsum(db, nullptr, 0, 0);
    if (!rc) {
      e = cudaDeviceSynchronize();
      if (e != cudaSuccess) rc = zp_cuda_check(e, "zp_setup_db: row sums");
    }
    if (rc) {
      cudaFree(db->d_rowsum);
      delete db;
      return rc;
    }
    *out = db;
    return ZP_OK;
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_setup_db: host allocation failed");
  }
}

static std::vector<uint8_t>& stale_flags(zp_db* db) {
  if (db->stale_v.size() != db->R) db->stale_v.assign(db->R, 0);
  return db->stale_v;
}

void zp_view_sync(zp_db* v) {
  const zp_db* b = v->base;
  if (!b) return;
  v->d_D16 = b->d_D16;
  v->tmap_d16 = b->tmap_d16;
  v->d_hneg = b->d_hneg;
  v->d_hpl = b->d_hpl;
  v->d_hpl_rowsum = b->d_hpl_rowsum;
  v->hpl_ld = b->hpl_ld;
  v->tmap_hpl = b->tmap_hpl;
  v->hint_ready = b->hint_ready;
  v->stale = b->stale;
  v->d_rns_hpl = b->d_rns_hpl;
  v->d_rns_rowsum = b->d_rns_rowsum;
  v->Rq = b->Rq;
  v->tmap_rns = b->tmap_rns;
  v->d_rns16 = b->d_rns16;
  v->tmap_rns16 = b->tmap_rns16;
}

extern "C" int zp_db_view(zp_db* db, zp_db** out) {
  try {
    if (!db || !out) return zp_set_error(ZP_EINVAL, "zp_db_view: null argument");
    zp_db* base = db->base ? db->base : db;
    zp_db* v = new zp_db();
    v->base = base;
    v->ctx = base->ctx;
    v->device = base->device;
    v->dD = base->dD;
    v->R = base->R;
    v->C = base->C;
    v->ld = base->ld;
    v->d1p = base->d1p;
    v->Rp = base->Rp;
    v->d_rowsum = base->d_rowsum;
    v->tmap_gemv = base->tmap_gemv;
    v->tmap_gemv128 = base->tmap_gemv128;
    v->tmap_gemm = base->tmap_gemm;
    zp_view_sync(v);
    *out = v;
    return ZP_OK;
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_db_view: host allocation failed");
  }
}

extern "C" int zp_db_info(const zp_db* db, uint32_t* ell, uint32_t* d1p, uint32_t* L) {
  if (!db) return zp_set_error(ZP_EINVAL, "zp_db_info: null db");
  if (ell) *ell = db->ctx->ell;
  if (d1p) *d1p = db->d1p;
  if (L) *L = db->ctx->L;
  return ZP_OK;
}

extern "C" int zp_stale_rows(const zp_db* db, uint32_t* count) {
  if (!db || !count) return zp_set_error(ZP_EINVAL, "zp_stale_rows: null argument");
  *count = db->base ? db->base->stale : db->stale;
  return ZP_OK;
}

extern "C" int zp_db_destroy(zp_db* db) {
  if (!db) return ZP_OK;
  zp_device_scope _zp_scope(db->device);
  cudaDeviceSynchronize();
  if (db->base) {  // a view owns only its scratch, stream and events
    db->d_rowsum = db->d_hneg = db->d_hpl_rowsum = db->d_rns_rowsum = nullptr;
    db->d_hpl = db->d_rns_hpl = nullptr;
    db->d_D16 = db->d_rns16 = nullptr;
  }
  if (db->d_rowsum) cudaFree(db->d_rowsum);
  if (db->d_hneg) cudaFree(db->d_hneg);
  if (db->d_hpl) cudaFree(db->d_hpl);
  if (db->d_hpl_rowsum) cudaFree(db->d_hpl_rowsum);
  if (db->d_rns_hpl) cudaFree(db->d_rns_hpl);
  if (db->d_rns_rowsum) cudaFree(db->d_rns_rowsum);
  if (db->d_D16) cudaFree(db->d_D16);
  if (db->d_rns16) cudaFree(db->d_rns16);
  if (db->side) {
    cudaStreamDestroy(db->side);
    cudaEventDestroy(db->ev_fork);
    cudaEventDestroy(db->ev_join);
  }
  zp_scratch* all[] = {&db->s_qplanes, &db->s_v,   &db->s_q,   &db->s_cko,  &db->s_ans,
                       &db->s_t,       &db->s_clients, &db->s_misc, &db->s_tcq, &db->s_hq,
                       &db->s_hcko, &db->s_ptab, &db->s_krows, &db->s_m2consts, &db->s_prows,
                       &db->s_crt, &db->s_crtb, &db->s_ypack};
  for (zp_scratch* s : all) scratch_free(s);
  delete db;
  return ZP_OK;
}

// host row list -> validated device copy in db->s_misc (first bytes)
static int stage_rows(zp_db* db, const uint32_t* hRows, uint32_t k, size_t extra_bytes,
                      uint32_t** dRows, cudaStream_t st) {
  for (uint32_t j = 0; j < k; ++j)
    if (hRows[j] >= db->R) return zp_set_error(ZP_EINVAL, "row index %u >= R=%u", hRows[j], db->R);
  const size_t rows_bytes = ((size_t)k * 4 + 255) / 256 * 256;
  int rc = zp_scratch_reserve(&db->s_misc, rows_bytes + extra_bytes);
  if (rc) return rc;
  *dRows = static_cast<uint32_t*>(db->s_misc.p);
  ZP_CUDA(cudaMemcpyAsync(*dRows, hRows, (size_t)k * 4, cudaMemcpyHostToDevice, st));
  return ZP_OK;
}

int zp_ensure_rns(zp_db* db, cudaStream_t st) {
  if (db->d_rns_hpl) return ZP_OK;
  if (db->base)
    return zp_set_error(ZP_ESTATE, "RNS tables missing: call zp_db_prepare_rns on the database "
                                   "before its views compress large batches");
  const uint32_t n = db->ctx->P.n;
  db->Rq = (db->d1p + 31) / 32 * 32;
  const uint64_t rows = (uint64_t)ZP_RNS_K * 4 * db->Rq;
  const size_t bytes = (size_t)rows * db->hpl_ld;
  if (cudaMalloc(&db->d_rns_hpl, bytes) != cudaSuccess) {
    db->d_rns_hpl = nullptr;
    return zp_set_error(ZP_ENOMEM, "RNS planes of the hint: cudaMalloc(%zu bytes)", bytes);
  }
  if (cudaMalloc(&db->d_rns_rowsum, (size_t)rows * 4) != cudaSuccess) {
    cudaFree(db->d_rns_hpl);
    db->d_rns_hpl = nullptr;
    db->d_rns_rowsum = nullptr;
    return zp_set_error(ZP_ENOMEM, "RNS planes of the hint: cudaMalloc(row sums)");
  }
  ZP_CUDA(cudaMemsetAsync(db->d_rns_hpl, 0, bytes, st));
  ZP_CUDA(cudaMemsetAsync(db->d_rns_rowsum, 0, (size_t)rows * 4, st));
  int rc = zp_encode_tmap_2d(&db->tmap_rns, CU_TENSOR_MAP_DATA_TYPE_UINT8, db->d_rns_hpl, n, rows,
                             db->hpl_ld, 128, 128, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  rc = zp_launch_rns_planes(db, nullptr, db->d1p, st);
  return rc ? rc : zp_ensure_rns16(db, st);
}

int zp_ensure_res_table(zp_ctx* c) {
  if (c->d_resw) return ZP_OK;
  std::vector<uint16_t> w((size_t)ZP_RES_ROWS * 256);
  std::vector<uint32_t> cs(ZP_RES_ROWS, 0);
  for (int k = 0; k < ZP_RES_KPER * ZP_RES_NT; ++k) {
    uint64_t pw = 1;  // 2^(8 beta) mod p_k
    const uint64_t p = k < ZP_RNS_K ? c->rns_p[k] : 0;
    for (int beta = 0; beta < 256; ++beta) {
      for (int cc = 0; cc < 4; ++cc) {
        const uint32_t byte = p ? (uint32_t)(pw >> (8 * cc)) & 0xFFu : 0u;
        // centred byte - 128 as an fp16 bit pattern (exact: |v| <= 128)
        const int v = (int)byte - 128;
        const uint32_t mag = (uint32_t)(v < 0 ? -v : v);
        uint16_t h = 0;
        if (mag) {
          int ex = 31 - __builtin_clz(mag);
          h = (uint16_t)(((ex + 15) << 10) | ((mag << (10 - ex)) & 0x3FFu));
        }
        if (v < 0) h |= 0x8000u;
        w[(size_t)(4 * k + cc) * 256 + beta] = h;
        cs[4 * k + cc] += byte;
      }
      if (p) pw = (pw << 8) % p;
    }
  }
  void* dw = nullptr;
  uint32_t* dcs = nullptr;
  if (cudaMalloc(&dw, w.size() * 2) != cudaSuccess || cudaMalloc(&dcs, cs.size() * 4) != cudaSuccess) {
    if (dw) cudaFree(dw);
    zp_clear_pending_error();
    return zp_set_error(ZP_ENOMEM, "cudaMalloc(residue table)");
  }
  if (cudaMemcpy(dw, w.data(), w.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dcs, cs.data(), cs.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dw);
    cudaFree(dcs);
    return zp_set_error(ZP_ECUDA, "copy of the residue table");
  }
  int rc = zp_encode_tmap_2d(&c->tmap_resw, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, dw, 256, ZP_RES_ROWS,
                             256 * 2, 64, 4 * ZP_RES_KPER, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) {
    cudaFree(dw);
    cudaFree(dcs);
    return rc;
  }
  c->d_resw = dw;
  c->d_resw_cs = dcs;
  return ZP_OK;
}

int zp_ensure_rns16(zp_db* db, cudaStream_t st) {
  if (db->d_rns16 || !db->d_rns_hpl || !db->d_D16 || db->base) return ZP_OK;
  const uint64_t Kp = (db->ctx->P.n + 127) / 128 * 128;
  const uint64_t rows = (uint64_t)ZP_RNS_K * 4 * db->Rq;
  const size_t bytes = (size_t)rows * Kp * 2;
  if (cudaMalloc(&db->d_rns16, bytes) != cudaSuccess) {
    db->d_rns16 = nullptr;
    zp_clear_pending_error();
    return zp_set_error(ZP_ENOMEM, "fp16 RNS planes: cudaMalloc(%zu bytes)", bytes);
  }
  int rc = zp_encode_tmap_2d(&db->tmap_rns16, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, db->d_rns16, Kp, rows,
                             Kp * 2, 64, 128, CU_TENSOR_MAP_SWIZZLE_128B);
  if (!rc) rc = zp_launch_rns16_rows(db, nullptr, db->Rq, st);  // every row, the padding too
  if (rc) {
    cudaFree(db->d_rns16);
    db->d_rns16 = nullptr;
  }
  return rc;
}

static int alloc_hint_state(zp_db* db) {
  const uint32_t n = db->ctx->P.n;
  if (!db->d_hneg) {
    if (cudaMalloc(&db->d_hneg, (size_t)db->R * n * 4) != cudaSuccess) {
      db->d_hneg = nullptr;
      return zp_set_error(ZP_ENOMEM, "zp_gen_hint: cudaMalloc(hint %zu bytes)", (size_t)db->R * n * 4);
    }
  }
  if (!db->d_hpl) {
    const size_t bytes = (size_t)4 * db->Rp * db->hpl_ld;
    if (cudaMalloc(&db->d_hpl, bytes) != cudaSuccess) {
      db->d_hpl = nullptr;
      return zp_set_error(ZP_ENOMEM, "zp_gen_hint: cudaMalloc(hint planes %zu bytes)", bytes);
    }
    cudaError_t e = cudaMemset(db->d_hpl, 0, bytes);
    if (e != cudaSuccess) return zp_cuda_check(e, "cudaMemset(hint planes)");
    if (cudaMalloc(&db->d_hpl_rowsum, (size_t)4 * db->Rp * 4) != cudaSuccess) {
      db->d_hpl_rowsum = nullptr;
      return zp_set_error(ZP_ENOMEM, "zp_gen_hint: cudaMalloc(plane sums)");
    }
    e = cudaMemset(db->d_hpl_rowsum, 0, (size_t)4 * db->Rp * 4);
    if (e != cudaSuccess) return zp_cuda_check(e, "cudaMemset(plane sums)");
    int rc = zp_encode_tmap_2d(&db->tmap_hpl, CU_TENSOR_MAP_DATA_TYPE_UINT8, db->d_hpl, n,
                               (uint64_t)4 * db->Rp, db->hpl_ld, 128, 128, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
  }
  return ZP_OK;
}

extern "C" int zp_gen_hint(zp_db* db, const uint32_t* dA, uint32_t* dH, const uint32_t* hRows,
                           uint32_t nrows, void* stream) {
  try {
    if (!db || !dA) return zp_set_error(ZP_EINVAL, "zp_gen_hint: null argument");
    if (db->base) return zp_set_error(ZP_EINVAL, "zp_gen_hint: called on a view (call it on its database)");
    if (hRows && (nrows == 0 || nrows > db->R))
      return zp_set_error(ZP_EINVAL, "zp_gen_hint: nrows=%u out of [1, R]", nrows);
    zp_ctx* c = db->ctx;
    ZP_ON_DEVICE(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t n = c->P.n;
    int rc = alloc_hint_state(db);
    if (rc) return rc;
    const bool tc = c->answer_path != ZP_PATH_SIMT;
    std::vector<uint8_t>& stale = stale_flags(db);
    if (!hRows) {
      uint32_t* outp = dH;
      if (!outp) {
        rc = zp_scratch_reserve(&db->s_v, (size_t)db->R * n * 4);
        if (rc) return rc;
        outp = static_cast<uint32_t*>(db->s_v.p);
      }
      rc = tc ? zp_launch_answer_tc(db, db->tmap_gemm, db->R, dA, n, true, outp, n, true,
                                    db->d_rowsum, st)
              : zp_launch_answer_simt(db, dA, n, 0, outp, 1, n, db->dD, db->R, db->ld, st);
      if (!rc) rc = zp_launch_hint_post(db, outp, nullptr, db->R, dH, st);
      if (!rc) rc = zp_launch_hint_planes_rowsum(db, nullptr, 0, st);
      if (!rc && db->d_rns_hpl) rc = zp_launch_rns_planes(db, nullptr, db->d1p, st);
      if (rc) return rc;
      db->hint_ready = true;
      stale.assign(db->R, 0);
      db->stale = 0;
      return ZP_OK;
    }
    const uint64_t ldc = ((uint64_t)db->C + 15) / 16 * 16;
    const size_t gather_bytes = ((size_t)nrows * ldc + 255) / 256 * 256;
    const size_t rs_bytes = ((size_t)nrows * 4 + 255) / 256 * 256;
    const size_t hc_bytes = (size_t)nrows * n * 4;
    uint32_t* dRows = nullptr;
    rc = stage_rows(db, hRows, nrows, gather_bytes + rs_bytes + hc_bytes, &dRows, st);
    if (rc) return rc;
    uint8_t* base = static_cast<uint8_t*>(db->s_misc.p) + ((size_t)nrows * 4 + 255) / 256 * 256;
    uint8_t* dG = base;
    uint32_t* dGsum = reinterpret_cast<uint32_t*>(base + gather_bytes);
    uint32_t* dHc = reinterpret_cast<uint32_t*>(base + gather_bytes + rs_bytes);
    zp_clear_pending_error();
    c->launches++;
    rc = zp_launch_copy_rows(db->dD, db->ld, dG, ldc, db->C, dRows, nrows, 1, st);
    if (rc) return rc;
    if (tc) {
      CUtensorMap tmG;
      rc = zp_encode_tmap_2d(&tmG, CU_TENSOR_MAP_DATA_TYPE_UINT8, dG, db->C, nrows, ldc, 128, 128,
                             CU_TENSOR_MAP_SWIZZLE_128B);
      if (!rc) rc = zp_launch_rowsum_buf(c, dG, ldc, nrows, db->C, dGsum, st);
      if (!rc) rc = zp_launch_answer_tc(db, tmG, nrows, dA, n, true, dHc, n, true, dGsum, st);
    } else {
      rc = zp_launch_answer_simt(db, dA, n, 0, dHc, 1, n, dG, nrows, ldc, st);
    }
    if (!rc) rc = zp_launch_hint_post(db, dHc, dRows, nrows, dH, st);
    if (!rc) rc = zp_launch_hint_planes_rowsum(db, dRows, nrows, st);
    if (!rc && db->d_rns_hpl) {  // keep the RNS planes of H' in step: their packed rows
      std::vector<uint32_t> pr(hRows, hRows + nrows);
      for (uint32_t& r : pr) r /= c->ell;
      std::sort(pr.begin(), pr.end());
      pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
      rc = zp_scratch_reserve(&db->s_prows, pr.size() * 4);
      if (!rc) {
        // pageable source: the copy is staged before cudaMemcpyAsync returns
        cudaError_t e = cudaMemcpyAsync(db->s_prows.p, pr.data(), pr.size() * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return zp_cuda_check(e, "cudaMemcpyAsync(packed rows)");
        rc = zp_launch_rns_planes(db, static_cast<const uint32_t*>(db->s_prows.p), (uint32_t)pr.size(), st);
      }
    }
    if (rc) return rc;
    for (uint32_t j = 0; j < nrows; ++j) {
      if (stale[hRows[j]]) {
        stale[hRows[j]] = 0;
        --db->stale;
      }
    }
    return ZP_OK;
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_gen_hint: host allocation failed");
  }
}

extern "C" int zp_update_rows(zp_db* db, const uint32_t* hRows, uint32_t k, const uint8_t* dNew,
                              void* stream) {
  try {
    if (!db || !hRows || !dNew) return zp_set_error(ZP_EINVAL, "zp_update_rows: null argument");
    if (db->base) return zp_set_error(ZP_EINVAL, "zp_update_rows: called on a view (call it on its database)");
    if (k == 0 || k > db->R) return zp_set_error(ZP_EINVAL, "zp_update_rows: k=%u out of [1, R]", k);
    ZP_ON_DEVICE(db->ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t* dRows = nullptr;
    int rc = stage_rows(db, hRows, k, 0, &dRows, st);
    if (rc) return rc;
    zp_clear_pending_error();
    db->ctx->launches++;
    rc = zp_launch_copy_rows(dNew, db->C, const_cast<uint8_t*>(db->dD), db->ld, db->C, dRows, k, 0, st);
    if (!rc) rc = zp_launch_rowsum(db, dRows, k, st);
    if (!rc && db->d_D16) rc = zp_launch_d16_rows(db, dRows, k, st);
    if (rc) return rc;
    std::vector<uint8_t>& stale = stale_flags(db);
    for (uint32_t j = 0; j < k; ++j) {
      if (!stale[hRows[j]]) {
        stale[hRows[j]] = 1;
        ++db->stale;
      }
    }
    return ZP_OK;
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_update_rows: host allocation failed");
  }
}

// ------------------------------------------------------------------ online Response
extern "C" int zp_answer(zp_db* db, const uint32_t* dQ, uint32_t B, uint32_t* dAns, void* stream) {
  if (!db || !dQ || !dAns) return zp_set_error(ZP_EINVAL, "zp_answer: null argument");
  zp_view_sync(db);
  if (B < 1 || B > 4096) return zp_set_error(ZP_EINVAL, "zp_answer: B=%u out of [1, 4096]", B);
  ZP_ON_DEVICE(db->ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  zp_ctx* c = db->ctx;
  // One to four queries: one pass of the dp4a GEMV over D (HBM- or dp4a-bound, ahead of
  // the tensor cores for such batches); more: the tensor-core GEMM.
  if (B <= c->gemv_max_batch && c->answer_path != ZP_PATH_SIMT && c->answer_path != ZP_PATH_TC)
    return zp_launch_gemv(db, dQ, B, dAns, st,
                          B == 1 && c->overlap_sms ? (uint32_t)c->num_sms - c->overlap_sms : 0u);
  if (c->answer_path == ZP_PATH_SIMT)
    return zp_launch_answer_simt(db, dQ, B, db->C, dAns, db->R, 1, db->dD, db->R, db->ld, st);
  const bool a16 = db->d_D16 && c->answer_fp16;
  return zp_launch_answer_tc(db, a16 ? db->tmap_d16 : db->tmap_gemm, db->R, dQ, B, false, dAns, db->R,
                             false, db->d_rowsum, st, a16);
}

extern "C" int zp_register_client(zp_ctx* c, const uint32_t* hM, uint32_t L, zp_client** out) {
  try {
    if (!c || !hM || !out) return zp_set_error(ZP_EINVAL, "zp_register_client: null argument");
    *out = nullptr;
    if (L != c->L) return zp_set_error(ZP_EINVAL, "zp_register_client: L=%u, expected %u", L, c->L);
    std::vector<uint32_t> m(hM, hM + L);
    if ((m[0] & 1u) == 0) return zp_set_error(ZP_EINVAL, "zp_register_client: m must be odd");
    if (big_bits(m) != c->P.key_bits)
      return zp_set_error(ZP_EINVAL, "zp_register_client: m has %u bits, expected %u", big_bits(m),
                          c->P.key_bits);
    // mu = floor(2^(64 L) / m) by binary long division (L+1 words)
    std::vector<uint32_t> mu(L + 1, 0), r(L + 1, 0);
    const uint32_t nbits = 64 * L + 1;
    for (int64_t i = nbits - 1; i >= 0; --i) {
      // r = 2 r + bit(i), bit(i) = 1 only for i = 64 L
      uint32_t carry = (i == (int64_t)(64 * L)) ? 1u : 0u;
      for (uint32_t w = 0; w < L + 1; ++w) {
        const uint32_t nc = r[w] >> 31;
        r[w] = (r[w] << 1) | carry;
        carry = nc;
      }
      // compare r >= m
      bool ge = true;
      for (int64_t w = L; w >= 0; --w) {
        const uint32_t mw = w < (int64_t)L ? m[w] : 0u;
        if (r[w] != mw) {
          ge = r[w] > mw;
          break;
        }
      }
      if (ge) {
        uint64_t br = 0;
        for (uint32_t w = 0; w < L + 1; ++w) {
          const uint64_t s = (uint64_t)r[w] - (w < L ? m[w] : 0u) - br;
          r[w] = (uint32_t)s;
          br = (s >> 63) & 1u;
        }
        if (i / 32 < (int64_t)(L + 1)) mu[i / 32] |= 1u << (i % 32);
      }
    }
    // Montgomery constants mod m^2 (R = 2^(64 L)): m^2, R mod m^2, R^2 mod m^2 and
    // -(m^2)^{-1} mod 2^32 (Newton's iteration x <- x (2 - a x) doubles the correct bits)
    const uint32_t L2 = 2 * L;
    std::vector<uint32_t> m2(L2, 0);
    for (uint32_t i = 0; i < L; ++i) {
      uint64_t carry = 0;
      for (uint32_t j = 0; j < L; ++j) {
        const uint64_t s = (uint64_t)m[i] * m[j] + m2[i + j] + carry;
        m2[i + j] = (uint32_t)s;
        carry = s >> 32;
      }
      m2[i + L] = (uint32_t)carry;
    }
    uint32_t inv = m2[0];
    for (int it = 0; it < 5; ++it) inv *= 2u - m2[0] * inv;
    const uint32_t m2inv = 0u - inv;
    // 2^k mod m^2 by doubling with a conditional subtraction (values stay below m^2)
    auto pow2_mod = [&](uint32_t k) {
      std::vector<uint32_t> r(L2 + 1, 0);
      r[0] = 1;
      for (uint32_t it = 0; it < k; ++it) {
        uint32_t carry = 0;
        for (uint32_t w = 0; w <= L2; ++w) {
          const uint32_t nc = r[w] >> 31;
          r[w] = (r[w] << 1) | carry;
          carry = nc;
        }
        bool ge = true;
        for (int64_t w = L2; w >= 0; --w) {
          const uint32_t mw = w < (int64_t)L2 ? m2[w] : 0u;
          if (r[w] != mw) {
            ge = r[w] > mw;
            break;
          }
        }
        if (ge) {
          uint64_t br = 0;
          for (uint32_t w = 0; w <= L2; ++w) {
            const uint64_t s = (uint64_t)r[w] - (w < L2 ? m2[w] : 0u) - br;
            r[w] = (uint32_t)s;
            br = (s >> 63) & 1u;
          }
        }
      }
      r.resize(L2);
      return r;
    };
    const std::vector<uint32_t> r1 = pow2_mod(32 * L2), r2 = pow2_mod(64 * L2);
    // CRT constants of the RNS compression: M/p_k mod m from prefix and suffix products of
    // the primes (Barrett reductions with mu), then m - (M mod m)
    std::vector<uint32_t> mkm((size_t)(ZP_RNS_K + 1) * L, 0);
    {
      const std::vector<uint32_t>& P = c->rns_p;
      std::vector<std::vector<uint32_t>> pre(ZP_RNS_K + 1), suf(ZP_RNS_K + 1);
      pre[0].assign(L, 0);
      pre[0][0] = 1;
      suf[ZP_RNS_K] = pre[0];
      for (int k = 0; k < ZP_RNS_K; ++k) pre[k + 1] = big_barrett(big_mul(pre[k], {P[k]}), m, mu);
      for (int k = ZP_RNS_K - 1; k >= 0; --k) suf[k] = big_barrett(big_mul(suf[k + 1], {P[k]}), m, mu);
      for (int k = 0; k < ZP_RNS_K; ++k) {
        const std::vector<uint32_t> v = big_barrett(big_mul(pre[k], suf[k + 1]), m, mu);
        std::copy(v.begin(), v.end(), mkm.begin() + (size_t)k * L);
      }
      uint64_t br = 0;  // m - (M mod m), M mod m = pre[K] (nonzero: m has no 27-bit factor)
      for (uint32_t w = 0; w < L; ++w) {
        const uint64_t t = (uint64_t)m[w] - pre[ZP_RNS_K][w] - br;
        mkm[(size_t)ZP_RNS_K * L + w] = (uint32_t)t;
        br = (t >> 63) & 1u;
      }
    }
    // 2^(32 w) mod m, w = L .. 2L - 1 (each from the previous one times 2^32)
    std::vector<uint32_t> pw((size_t)L * L, 0);
    {
      std::vector<uint32_t> x(L + 1, 0);
      x[L] = 1;  // 2^(32 L)
      std::vector<uint32_t> t = big_barrett(x, m, mu);
      for (uint32_t w = 0; w < L; ++w) {
        t.resize(L, 0);
        std::copy(t.begin(), t.end(), pw.begin() + (size_t)w * L);
        std::vector<uint32_t> sh(L + 1, 0);
        std::copy(t.begin(), t.end(), sh.begin() + 1);
        t = big_barrett(sh, m, mu);
      }
    }
    ZP_ON_DEVICE(c->device);
    zp_client* cl = new zp_client();
    cl->ctx = c;
    cl->device = c->device;
    cl->L = L;
    cl->d_m = cl->d_mu = cl->d_m2 = cl->d_r1 = cl->d_r2 = cl->d_mkm = cl->d_pow = nullptr;
    cl->m2inv = m2inv;
    cl->h_m = m;
    auto free_all = [cl]() {
      for (uint32_t* p : {cl->d_m, cl->d_mu, cl->d_m2, cl->d_r1, cl->d_r2, cl->d_mkm, cl->d_pow})
        if (p) cudaFree(p);
    };
    if (cudaMalloc(&cl->d_m, L * 4) != cudaSuccess || cudaMalloc(&cl->d_mu, (L + 1) * 4) != cudaSuccess ||
        cudaMalloc(&cl->d_m2, L2 * 4) != cudaSuccess || cudaMalloc(&cl->d_r1, L2 * 4) != cudaSuccess ||
        cudaMalloc(&cl->d_r2, L2 * 4) != cudaSuccess || cudaMalloc(&cl->d_mkm, mkm.size() * 4) != cudaSuccess ||
        cudaMalloc(&cl->d_pow, pw.size() * 4) != cudaSuccess) {
      free_all();
      delete cl;
      return zp_set_error(ZP_ENOMEM, "zp_register_client: cudaMalloc");
    }
    cudaError_t e = cudaMemcpy(cl->d_m, m.data(), L * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cl->d_mu, mu.data(), (L + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cl->d_m2, m2.data(), L2 * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cl->d_r1, r1.data(), L2 * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cl->d_r2, r2.data(), L2 * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cl->d_mkm, mkm.data(), mkm.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cl->d_pow, pw.data(), pw.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_all();
      delete cl;
      return zp_cuda_check(e, "zp_register_client: copy constants");
    }
    *out = cl;
    return ZP_OK;
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_register_client: host allocation failed");
  }
}

extern "C" int zp_client_destroy(zp_client* cl) {
  if (!cl) return ZP_OK;
  zp_device_scope _zp_scope(cl->device);
  cudaDeviceSynchronize();
  for (uint32_t* p : {cl->d_m, cl->d_mu, cl->d_m2, cl->d_r1, cl->d_r2, cl->d_mkm, cl->d_pow})
    if (p) cudaFree(p);
  delete cl;
  return ZP_OK;
}

static int check_compress_args(zp_db* db, zp_client* const* clients, uint32_t B) {
  if (!clients) return zp_set_error(ZP_EINVAL, "zp_compress: null clients");
  if (B < 1 || B > 4096) return zp_set_error(ZP_EINVAL, "zp_compress: B=%u out of [1, 4096]", B);
  if (!db->hint_ready) return zp_set_error(ZP_ESTATE, "zp_compress: no hint (call zp_gen_hint)");
  if (db->stale) return zp_set_error(ZP_ESTATE, "zp_compress: %u hint rows stale after updates", db->stale);
  for (uint32_t b = 0; b < B; ++b) {
    if (!clients[b]) return zp_set_error(ZP_EINVAL, "zp_compress: clients[%u] is null", b);
    if (clients[b]->ctx != db->ctx) return zp_set_error(ZP_EINVAL, "zp_compress: client %u from another context", b);
  }
  return ZP_OK;
}

extern "C" int zp_compress(zp_db* db, zp_client* const* clients, const uint32_t* dAns,
                           const uint32_t* dCKO, uint32_t B, uint32_t* dT, void* stream) {
  try {
    if (!db || !dAns || !dCKO || !dT) return zp_set_error(ZP_EINVAL, "zp_compress: null argument");
    zp_view_sync(db);
    int rc = check_compress_args(db, clients, B);
    if (rc) return rc;
    ZP_ON_DEVICE(db->ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = zp_launch_compress_products(db, dCKO, B, st, 0);
    if (rc) return rc;
    return zp_launch_compress_finish(db, clients, dAns, B, dT, st);
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_compress: host allocation failed");
  }
}

extern "C" int zp_compress_products(zp_db* db, const uint32_t* dCKO, uint32_t B, void* stream) {
  try {
    if (!db || !dCKO) return zp_set_error(ZP_EINVAL, "zp_compress_products: null argument");
    zp_view_sync(db);
    if (B < 1 || B > 4096) return zp_set_error(ZP_EINVAL, "zp_compress_products: B=%u out of [1, 4096]", B);
    if (!db->hint_ready) return zp_set_error(ZP_ESTATE, "zp_compress_products: no hint (call zp_gen_hint)");
    if (db->stale) return zp_set_error(ZP_ESTATE, "zp_compress_products: %u hint rows stale", db->stale);
    ZP_ON_DEVICE(db->ctx->device);
    // only a single query's products share the GPU with an answer
    return zp_launch_compress_products(db, dCKO, B, static_cast<cudaStream_t>(stream),
                                       B == 1 ? db->ctx->overlap_sms : 0u);
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_compress_products: host allocation failed");
  }
}

extern "C" int zp_compress_finish(zp_db* db, zp_client* const* clients, const uint32_t* dAns,
                                  uint32_t B, uint32_t* dT, void* stream) {
  try {
    if (!db || !dAns || !dT) return zp_set_error(ZP_EINVAL, "zp_compress_finish: null argument");
    zp_view_sync(db);
    int rc = check_compress_args(db, clients, B);
    if (rc) return rc;
    ZP_ON_DEVICE(db->ctx->device);
    return zp_launch_compress_finish(db, clients, dAns, B, dT, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_compress_finish: host allocation failed");
  }
}

static int ensure_side_stream(zp_db* db) {
  if (db->side) return ZP_OK;
  ZP_CUDA(cudaStreamCreateWithFlags(&db->side, cudaStreamNonBlocking));
  ZP_CUDA(cudaEventCreateWithFlags(&db->ev_fork, cudaEventDisableTiming));
  ZP_CUDA(cudaEventCreateWithFlags(&db->ev_join, cudaEventDisableTiming));
  return ZP_OK;
}

extern "C" int zp_respond(zp_db* db, zp_client* const* clients, const uint32_t* dQ,
                          const uint32_t* dCKO, uint32_t B, uint32_t* dAns, uint32_t* dT,
                          void* stream) {
  try {
    if (!db || !dQ || !dCKO || !dAns || !dT) return zp_set_error(ZP_EINVAL, "zp_respond: null argument");
    zp_view_sync(db);
    int rc = check_compress_args(db, clients, B);
    if (rc) return rc;
    zp_ctx* c = db->ctx;
    ZP_ON_DEVICE(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool overlap = B == 1 && c->overlap_sms > 0 && c->answer_path == ZP_PATH_AUTO &&
                         c->compress_path != ZP_PATH_SIMT && c->P.n <= 1024;
    // a batch answered on the tensor cores: its compression products (which do not read the
    // answers) run on the internal stream beside it and take the SMs its last wave leaves idle
    const bool overlap_batch = B > 1 && c->batch_overlap && B > c->gemv_max_batch &&
                               c->answer_path != ZP_PATH_SIMT;
    if (overlap_batch) {
      rc = ensure_side_stream(db);
      if (rc) return rc;
      ZP_CUDA(cudaEventRecord(db->ev_fork, st));
      ZP_CUDA(cudaStreamWaitEvent(db->side, db->ev_fork, 0));
      rc = zp_launch_compress_products(db, dCKO, B, db->side, 0);
      if (rc) return rc;
      rc = zp_answer(db, dQ, B, dAns, stream);
      if (rc) return rc;
      ZP_CUDA(cudaEventRecord(db->ev_join, db->side));
      ZP_CUDA(cudaStreamWaitEvent(st, db->ev_join, 0));
      return zp_launch_compress_finish(db, clients, dAns, B, dT, st);
    }
    if (!overlap) {
      rc = zp_answer(db, dQ, B, dAns, stream);
      if (rc) return rc;
      return zp_compress(db, clients, dAns, dCKO, B, dT, stream);
    }
    // The products V = H.cko do not depend on the answer: they run on `overlap_sms` SMs
    // of an internal stream while the HBM-bound GEMV streams the database on the rest.
    rc = ensure_side_stream(db);
    if (rc) return rc;
    ZP_CUDA(cudaEventRecord(db->ev_fork, st));
    ZP_CUDA(cudaStreamWaitEvent(db->side, db->ev_fork, 0));
    rc = zp_launch_compress_products(db, dCKO, B, db->side, c->overlap_sms);
    if (rc) return rc;
    // "pack_split": the Horner over V, its fold and reduction need no answer either, so they
    // follow the products on the internal stream; after the join only b' + Y remains
    const bool split = c->pack_split && !db->v_rns;
    if (split) {
      rc = zp_launch_pack_products(db, clients, B, db->side);
      if (rc) return rc;
    }
    rc = zp_launch_gemv(db, dQ, 1u, dAns, st, (uint32_t)c->num_sms - c->overlap_sms);
    if (rc) return rc;
    ZP_CUDA(cudaEventRecord(db->ev_join, db->side));
    ZP_CUDA(cudaStreamWaitEvent(st, db->ev_join, 0));
    if (split) return zp_launch_pack_answers(db, dAns, B, dT, st);
    return zp_launch_compress_finish(db, clients, dAns, B, dT, st);
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_respond: host allocation failed");
  }
}

extern "C" int zp_client_hint(zp_db* db, const zp_client* cl, const uint32_t* dCkr, uint32_t* dK,
                              const uint32_t* hPackedRows, uint32_t nrows, void* stream) {
  try {
    if (!db || !cl || !dCkr || !dK) return zp_set_error(ZP_EINVAL, "zp_client_hint: null argument");
    zp_view_sync(db);
    if (cl->ctx != db->ctx) return zp_set_error(ZP_EINVAL, "zp_client_hint: client from another context");
    if (!db->hint_ready) return zp_set_error(ZP_ESTATE, "zp_client_hint: no hint (call zp_gen_hint)");
    if (db->stale) return zp_set_error(ZP_ESTATE, "zp_client_hint: %u hint rows stale after updates", db->stale);
    if ((reinterpret_cast<uintptr_t>(dCkr) | reinterpret_cast<uintptr_t>(dK)) & 15u)
      return zp_set_error(ZP_EINVAL, "zp_client_hint: dCkr and dK must be 16-byte aligned");
    ZP_ON_DEVICE(db->ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t* dRows = nullptr;
    uint32_t np = db->d1p;
    if (hPackedRows) {
      if (nrows == 0) return ZP_OK;
      for (uint32_t j = 0; j < nrows; ++j)
        if (hPackedRows[j] >= db->d1p)
          return zp_set_error(ZP_EINVAL, "zp_client_hint: packed row %u >= d1'=%u", hPackedRows[j], db->d1p);
      int rc = zp_scratch_reserve(&db->s_misc, (size_t)nrows * 4);
      if (rc) return rc;
      ZP_CUDA(cudaMemcpyAsync(db->s_misc.p, hPackedRows, (size_t)nrows * 4, cudaMemcpyHostToDevice, st));
      dRows = static_cast<const uint32_t*>(db->s_misc.p);
      np = nrows;
    }
    return zp_launch_client_hint(db, cl, dCkr, dK, dRows, np, st);
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_client_hint: host allocation failed");
  }
}

// ------------------------------------------------------------------ autotuner
// Measures on `db` (zero-filled test inputs: the kernels' time does not depend on the
// values) and sets the context's batch thresholds and the SM split to the fastest choices.
extern "C" int zp_autotune(zp_db* db, void* stream, int64_t* chosen) {
  try {
    if (!db) return zp_set_error(ZP_EINVAL, "zp_autotune: null argument");
    if (db->base) return zp_set_error(ZP_EINVAL, "zp_autotune: called on a view (call it on its database)");
    zp_ctx* c = db->ctx;
    ZP_ON_DEVICE(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t BQ = 128, n = c->P.n, L = c->L;
    const int saved_answer = c->answer_path, saved_compress = c->compress_path;
    const uint32_t saved_overlap = c->overlap_sms, saved_gemv = c->gemv_max_batch,
                   saved_rns = c->rns_min_batch, saved_fp16 = c->answer_fp16,
                   saved_bo = c->batch_overlap, saved_split = c->pack_split;
    uint32_t saved_abt[4], saved_rbt[4], saved_gcfg[2];
    for (int i = 0; i < 4; ++i) saved_abt[i] = c->ans_bt[i], saved_rbt[i] = c->rns_bt[i];
    for (int i = 0; i < 2; ++i) saved_gcfg[i] = c->gemv_cfg[i];
    uint32_t *dQ = nullptr, *dAns = nullptr, *dCKO = nullptr, *dT = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    zp_client* cl = nullptr;
    auto cleanup = [&]() {
      for (uint32_t* p : {dQ, dAns, dCKO, dT})
        if (p) cudaFree(p);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (cl) zp_client_destroy(cl);
      c->answer_path = saved_answer;
      c->compress_path = saved_compress;
    };
    auto fail = [&](int rc) {
      cleanup();
      c->overlap_sms = saved_overlap;
      c->gemv_max_batch = saved_gemv;
      c->rns_min_batch = saved_rns;
      c->answer_fp16 = saved_fp16;
      c->batch_overlap = saved_bo;
      c->pack_split = saved_split;
      for (int i = 0; i < 4; ++i) c->ans_bt[i] = saved_abt[i], c->rns_bt[i] = saved_rbt[i];
      for (int i = 0; i < 2; ++i) c->gemv_cfg[i] = saved_gcfg[i];
      return rc;
    };
    if (cudaMalloc(&dQ, (size_t)BQ * db->C * 4) != cudaSuccess ||
        cudaMalloc(&dAns, (size_t)BQ * db->R * 4) != cudaSuccess ||
        cudaMalloc(&dCKO, (size_t)BQ * n * L * 4) != cudaSuccess ||
        cudaMalloc(&dT, (size_t)BQ * db->d1p * L * 4) != cudaSuccess)
      return fail(zp_set_error(ZP_ENOMEM, "zp_autotune: test buffers"));
    if (cudaMemsetAsync(dQ, 0, (size_t)BQ * db->C * 4, st) != cudaSuccess ||
        cudaMemsetAsync(dCKO, 0, (size_t)BQ * n * L * 4, st) != cudaSuccess ||
        cudaMemsetAsync(dAns, 0, (size_t)BQ * db->R * 4, st) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return fail(zp_set_error(ZP_ECUDA, "zp_autotune: setup"));
    // mean of 5 runs after one warm-up; a failing run aborts the tuning
    int err = ZP_OK;
    auto time_ms = [&](auto&& fn) {
      float ms = 0.f;
      if (err) return 1e30f;
      if ((err = fn())) return 1e30f;
      cudaEventRecord(e0, st);
      for (int i = 0; i < 5 && !err; ++i) err = fn();
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      return err ? 1e30f : ms / 5.f;
    };
    // (1) answers: one dp4a pass against the tensor cores, 2..4 queries
    uint32_t gemv_max = 1;
    for (uint32_t B = 2; B <= 4; ++B) {
      c->answer_path = ZP_PATH_AUTO;
      c->gemv_max_batch = 4;
      const float g = time_ms([&] { return zp_answer(db, dQ, B, dAns, stream); });
      c->answer_path = ZP_PATH_TC;
      const float t = time_ms([&] { return zp_answer(db, dQ, B, dAns, stream); });
      if (err) return fail(err);
      if (g > t) break;
      gemv_max = B;
    }
    c->answer_path = saved_answer;
    c->gemv_max_batch = gemv_max;
    // (2) compression: byte planes against RNS (needs the hint and n <= 1024)
    uint32_t rns_min = c->rns_min_batch;
    if (db->hint_ready && !db->stale && n <= 1024 && saved_compress == ZP_PATH_AUTO) {
      std::vector<uint32_t> m(L, 0);  // a fixed odd modulus of key_bits bits
      m[0] = 1;
      m[L - 1] = 0xC0000000u;
      int rc = zp_register_client(c, m.data(), L, &cl);
      if (rc) return fail(rc);
      std::vector<zp_client*> cls(BQ, cl);
      rns_min = 0;
      for (uint32_t B : {2u, 4u, 6u, 8u, 12u, 16u}) {
        c->compress_path = ZP_PATH_TC;
        const float bp = time_ms([&] { return zp_compress(db, cls.data(), dAns, dCKO, B, dT, stream); });
        c->compress_path = ZP_PATH_RNS;
        const float rn = time_ms([&] { return zp_compress(db, cls.data(), dAns, dCKO, B, dT, stream); });
        if (err) return fail(err);
        if (rn < bp) {
          rns_min = B;
          break;
        }
      }
      c->compress_path = saved_compress;
    }
    c->rns_min_batch = rns_min;
    // (3) the GEMV configuration of a single-query answer alone on the whole GPU
    {
      c->overlap_sms = 0;
      float best = 1e30f;
      uint32_t best_cfg = saved_gcfg[0];
      for (uint32_t cfg = 1; cfg <= 2; ++cfg) {
        c->gemv_cfg[0] = cfg;
        const float t = time_ms([&] { return zp_answer(db, dQ, 1, dAns, stream); });
        if (err) return fail(err);
        if (t < best) best = t, best_cfg = cfg;
      }
      c->gemv_cfg[0] = best_cfg;
      c->overlap_sms = saved_overlap;
    }
    // (4) the SM split of the single-query Response, the GEMV configuration beside the
    // compression products and whether the packing of V runs beside the answer too
    if (cl && c->num_sms >= 64) {
      float best = 1e30f;
      uint32_t best_ov = 0, best_cfg = saved_gcfg[1], best_split = saved_split;
      for (uint32_t split = 0; split <= 1; ++split) {
        c->pack_split = split;
        for (uint32_t cfg = 1; cfg <= 2; ++cfg) {
          c->gemv_cfg[1] = cfg;
          for (uint32_t frac = 0; frac <= 8; ++frac) {  // 0 and 24% .. 52% of the SMs
            if (frac == 0 && (cfg == 2 || split)) continue;  // no split: whole-GPU configuration
            const uint32_t ov = frac == 0 ? 0u : (uint32_t)(c->num_sms * (20 + 4 * frac) / 100);
            c->overlap_sms = ov;
            const float r = time_ms([&] {
              return zp_respond(db, &cl, dQ, dCKO, 1, dAns, dT, stream);
            });
            if (err) return fail(err);
            if (r < best) best = r, best_ov = ov, best_cfg = cfg, best_split = split;
          }
        }
      }
      // refine the split around the best in steps of 2 SMs
      if (best_ov) {
        c->gemv_cfg[1] = best_cfg;
        c->pack_split = best_split;
        const uint32_t center = best_ov;
        for (int d : {-4, -2, 2, 4}) {
          const int ov = (int)center + d;
          if (ov < 8 || ov > (int)c->num_sms - 8) continue;
          c->overlap_sms = (uint32_t)ov;
          const float r = time_ms([&] {
            return zp_respond(db, &cl, dQ, dCKO, 1, dAns, dT, stream);
          });
          if (err) return fail(err);
          if (r < best) best = r, best_ov = (uint32_t)ov;
        }
      }
      c->overlap_sms = best_ov;
      c->gemv_cfg[1] = best_cfg;
      c->pack_split = best_split;
    }
    // (5) tile widths of the tensor-core answers per batch class (16, 32, 64 queries), and
    // the operand (the fp16 copy of D against its bytes) when the copy exists
    if (c->answer_path != ZP_PATH_SIMT) {
      const int saved_path = c->answer_path;
      c->answer_path = ZP_PATH_TC;
      for (int cls_i = 0; cls_i < 4; ++cls_i) {
        const uint32_t B = 16u << cls_i;  // 16, 32, 64, 128 queries
        float best = 1e30f;
        uint32_t best_bt = c->ans_bt[cls_i];
        for (uint32_t bt = 16; bt <= B && bt <= 64; bt *= 2) {
          c->ans_bt[cls_i] = bt;
          const float t = time_ms([&] { return zp_answer(db, dQ, B, dAns, stream); });
          if (err) return fail(err);
          if (t < best) best = t, best_bt = bt;
        }
        c->ans_bt[cls_i] = best_bt;
      }
      if (db->d_D16) {
        float tf[2];
        for (uint32_t f16 = 0; f16 <= 1; ++f16) {
          c->answer_fp16 = f16;
          tf[f16] = time_ms([&] { return zp_answer(db, dQ, BQ, dAns, stream); });
          if (err) return fail(err);
        }
        c->answer_fp16 = tf[1] <= tf[0] ? 1u : 0u;
      }
      c->answer_path = saved_path;
    }
    // (6) tile widths of the RNS products per batch class, and whether a batch's products run
    // beside its answers in zp_respond
    if (cl && saved_compress == ZP_PATH_AUTO && rns_min && db->d_rns_hpl) {
      std::vector<zp_client*> cls(BQ, cl);
      c->compress_path = ZP_PATH_RNS;
      for (int cls_i = 0; cls_i < 4; ++cls_i) {
        const uint32_t B = 16u << cls_i;
        float best = 1e30f;
        uint32_t best_bt = c->rns_bt[cls_i];
        for (uint32_t bt = 16; bt <= B && bt <= 64; bt *= 2) {
          c->rns_bt[cls_i] = bt;
          const float t = time_ms([&] { return zp_compress(db, cls.data(), dAns, dCKO, B, dT, stream); });
          if (err) return fail(err);
          if (t < best) best = t, best_bt = bt;
        }
        c->rns_bt[cls_i] = best_bt;
      }
      c->compress_path = saved_compress;
      float tb[2];
      for (uint32_t bo = 0; bo <= 1; ++bo) {
        c->batch_overlap = bo;
        tb[bo] = time_ms([&] { return zp_respond(db, cls.data(), dQ, dCKO, BQ, dAns, dT, stream); });
        if (err) return fail(err);
      }
      c->batch_overlap = tb[1] <= tb[0] ? 1u : 0u;
    }
    cleanup();
    if (chosen) {
      chosen[0] = c->gemv_max_batch;
      chosen[1] = c->rns_min_batch;
      chosen[2] = c->overlap_sms;
    }
    return ZP_OK;
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_autotune: host allocation failed");
  }
}

extern "C" int zp_db_prepare_fp16(zp_db* db, void* stream) {
  if (!db) return zp_set_error(ZP_EINVAL, "zp_db_prepare_fp16: null argument");
  if (db->base) return zp_set_error(ZP_EINVAL, "zp_db_prepare_fp16: called on a view (call it on its database)");
  if (db->d_D16) return ZP_OK;
  ZP_ON_DEVICE(db->ctx->device);
  const uint64_t Kp = (db->C + 127) / 128 * 128;  // two K blocks per stage of the fp16 path
  const size_t bytes = (size_t)db->R * Kp * 2;
  if (cudaMalloc(&db->d_D16, bytes) != cudaSuccess) {
    db->d_D16 = nullptr;
    zp_clear_pending_error();
    return zp_set_error(ZP_ENOMEM, "zp_db_prepare_fp16: cudaMalloc(%zu bytes)", bytes);
  }
  int rc = zp_encode_tmap_2d(&db->tmap_d16, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, db->d_D16, Kp, db->R, Kp * 2,
                             64, 128, CU_TENSOR_MAP_SWIZZLE_128B);
  if (!rc) rc = zp_launch_d16_rows(db, nullptr, db->R, static_cast<cudaStream_t>(stream));
  if (rc) {
    cudaFree(db->d_D16);
    db->d_D16 = nullptr;
    return rc;
  }
  return zp_ensure_rns16(db, static_cast<cudaStream_t>(stream));  // if the RNS planes exist
}

extern "C" int zp_db_prepare_rns(zp_db* db, void* stream) {
  if (!db) return zp_set_error(ZP_EINVAL, "zp_db_prepare_rns: null argument");
  if (db->base) return zp_set_error(ZP_EINVAL, "zp_db_prepare_rns: called on a view (call it on its database)");
  if (!db->hint_ready) return zp_set_error(ZP_ESTATE, "zp_db_prepare_rns: no hint (call zp_gen_hint)");
  if (db->stale) return zp_set_error(ZP_ESTATE, "zp_db_prepare_rns: %u hint rows stale after updates", db->stale);
  if (db->ctx->P.n > 1024) return zp_set_error(ZP_EUNSUPPORTED, "zp_db_prepare_rns: needs n <= 1024");
  ZP_ON_DEVICE(db->ctx->device);
  return zp_ensure_rns(db, static_cast<cudaStream_t>(stream));
}

extern "C" int zp_client_decrypt(const zp_client* cl, const uint32_t* hLam, const uint32_t* hMu,
                                 const uint32_t* dC, uint32_t* dOut, uint32_t count, void* stream) {
  try {
    if (!cl || !hLam || !hMu || ((!dC || !dOut) && count))
      return zp_set_error(ZP_EINVAL, "zp_client_decrypt: null argument");
    if ((reinterpret_cast<uintptr_t>(dC) | reinterpret_cast<uintptr_t>(dOut)) & 15u)
      return zp_set_error(ZP_EINVAL, "zp_client_decrypt: dC and dOut must be 16-byte aligned");
    if (count == 0) return ZP_OK;
    const uint32_t L = cl->L;
    const std::vector<uint32_t>& m = cl->h_m;
    // e = lambda mu (< m^2: 2L words)
    std::vector<uint32_t> e = big_mul(std::vector<uint32_t>(hLam, hLam + L),
                                      std::vector<uint32_t>(hMu, hMu + L));
    while (e.size() > 1 && e.back() == 0) e.pop_back();
    // m^{-1} mod 2^(32 L) by Newton's iteration x <- x (2 - m x), from the inverse mod 2^32
    std::vector<uint32_t> x(L, 0);
    uint32_t inv = m[0];
    for (int it = 0; it < 5; ++it) inv *= 2u - m[0] * inv;
    x[0] = inv;
    for (uint32_t prec = 32; prec < 32 * L; prec *= 2) {
      std::vector<uint32_t> t = big_mul(m, x);
      t.resize(L);
      uint64_t br = 0;  // t = 2 - t mod 2^(32 L)
      for (uint32_t w = 0; w < L; ++w) {
        const uint64_t s = (uint64_t)(w == 0 ? 2u : 0u) - t[w] - br;
        t[w] = (uint32_t)s;
        br = (s >> 63) & 1u;
      }
      x = big_mul(x, t);
      x.resize(L);
    }
    ZP_ON_DEVICE(cl->device);
    return zp_launch_decrypt(cl, e.data(), (uint32_t)e.size(), x.data(), dC, dOut, count,
                             static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_client_decrypt: host allocation");
  }
}

extern "C" int zp_combine(zp_db* db, zp_client* const* clients, const uint32_t* dK, const uint32_t* dT,
                          uint32_t B, uint32_t* dOut, void* stream) {
  try {
    if (!db || !clients || !dK || !dT || !dOut) return zp_set_error(ZP_EINVAL, "zp_combine: null argument");
    zp_view_sync(db);
    if (B < 1 || B > 4096) return zp_set_error(ZP_EINVAL, "zp_combine: B=%u out of [1, 4096]", B);
    for (uint32_t b = 0; b < B; ++b) {
      if (!clients[b]) return zp_set_error(ZP_EINVAL, "zp_combine: clients[%u] is null", b);
      if (clients[b]->ctx != db->ctx) return zp_set_error(ZP_EINVAL, "zp_combine: client %u from another context", b);
    }
    if ((reinterpret_cast<uintptr_t>(dK) | reinterpret_cast<uintptr_t>(dT) | reinterpret_cast<uintptr_t>(dOut)) & 15u)
      return zp_set_error(ZP_EINVAL, "zp_combine: dK, dT and dOut must be 16-byte aligned");
    ZP_ON_DEVICE(db->ctx->device);
    return zp_launch_combine(db, clients, dK, dT, B, dOut, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return zp_set_error(ZP_ENOMEM, "zp_combine: host allocation failed");
  }
}

extern "C" int zp_respond_host(zp_db* db, zp_client* const* clients, const uint32_t* hQ,
                               const uint32_t* hCKO, uint32_t B, uint32_t* hT, uint32_t* hAns,
                               void* stream) {
  if (!db || !hQ || !hCKO || !hT) return zp_set_error(ZP_EINVAL, "zp_respond_host: null argument");
  zp_view_sync(db);
  int rc = check_compress_args(db, clients, B);
  if (rc) return rc;
  zp_ctx* c = db->ctx;
  ZP_ON_DEVICE(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t qb = (size_t)B * db->C * 4, cb = (size_t)B * c->P.n * c->L * 4;
  const size_t ab = (size_t)B * db->R * 4, tb = (size_t)B * db->d1p * c->L * 4;
  // the inputs go to buffers of their own: the kernels' operand scratch (s_cko, s_q, ...)
  // is rewritten by zp_respond while it reads its inputs
  if ((rc = zp_scratch_reserve(&db->s_hq, qb)) || (rc = zp_scratch_reserve(&db->s_hcko, cb)) ||
      (rc = zp_scratch_reserve(&db->s_ans, ab)) || (rc = zp_scratch_reserve(&db->s_t, tb)))
    return rc;
  ZP_CUDA(cudaMemcpyAsync(db->s_hq.p, hQ, qb, cudaMemcpyHostToDevice, st));
  ZP_CUDA(cudaMemcpyAsync(db->s_hcko.p, hCKO, cb, cudaMemcpyHostToDevice, st));
  rc = zp_respond(db, clients, static_cast<uint32_t*>(db->s_hq.p), static_cast<uint32_t*>(db->s_hcko.p),
                  B, static_cast<uint32_t*>(db->s_ans.p), static_cast<uint32_t*>(db->s_t.p), stream);
  if (rc) return rc;
  ZP_CUDA(cudaMemcpyAsync(hT, db->s_t.p, tb, cudaMemcpyDeviceToHost, st));
  if (hAns) ZP_CUDA(cudaMemcpyAsync(hAns, db->s_ans.p, ab, cudaMemcpyDeviceToHost, st));
  ZP_CUDA(cudaStreamSynchronize(st));
  return ZP_OK;
}
