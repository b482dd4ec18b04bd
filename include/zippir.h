/*
 * zippir.h -- C ABI of the GB300 (sm_103a) library for the online server phase of
 * ZipPIR (arXiv 2603.09190): the LWE answer ans = D.q mod 2^32 and the per-query
 * LWE-to-Paillier answer compression t = (b' + H'.cko) mod m.
 *
 * Orientation. The database D is R x C, row-major, entries in Z_p (p = 256, one
 * byte each). The paper writes Response as b = db^T qu_0 with db of shape
 * d0 x d1; here D = db^T, so R = d1 (answer length) and C = d0 (query length).
 * A record is column i0 of D.
 *
 * Conventions for every entry point:
 *  - Return value: ZP_OK (0) or a negative ZP_E* code; zp_last_error() gives a
 *    message for the calling thread. No C++ exception crosses this boundary.
 *  - Pointers named d* are DEVICE pointers on the context's device, h* are HOST
 *    pointers. The caller owns every buffer it passes; the library never frees
 *    them and keeps only the database pointer (non-owning) between calls, so the
 *    database must stay alive and unchanged (except through zp_update_rows) until
 *    zp_db_destroy. The library owns its internal state (the negated hint in its
 *    compression layout, row sums, per-client constants, scratch) and frees it in
 *    the matching *_destroy.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Stream-taking calls
 *    are asynchronous: they validate arguments on the host, return an error before
 *    launching anything if validation fails, and otherwise enqueue work on
 *    `stream`. Device buffers must not be reused by the caller before that work
 *    completes. The *_host entry points synchronise `stream` before returning.
 *  - A context must outlive the databases and clients created from it; databases
 *    and clients may be destroyed before or after one another.
 *  - All arithmetic is exact integer arithmetic; results are bit-identical to the
 *    definitions cited at each call.
 *  - Every entry point runs on its handle's device and gives the caller's current
 *    device back before it returns.
 */
#ifndef ZIPPIR_H
#define ZIPPIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum zp_status {
  ZP_OK = 0,
  ZP_EINVAL = -1,      /* bad argument: null pointer, size, alignment, value range */
  ZP_ENOMEM = -2,      /* device or host allocation failed */
  ZP_ECUDA = -3,       /* a CUDA runtime/driver call failed */
  ZP_ETIMEOUT = -4,    /* a bounded device-side wait gave up (kernel returned early) */
  ZP_ESTATE = -5,      /* call out of order, e.g. zp_compress before zp_gen_hint */
  ZP_EUNSUPPORTED = -6 /* parameters the compiled library does not implement */
};

enum zp_secret {
  ZP_SECRET_UNIFORM = 0, /* LWE secret uniform in Z_q: packing scale gamma = q + n q^2 (Sec. 3.3) */
  ZP_SECRET_BINARY = 1   /* LWE secret in {0,1}:     packing scale gamma = q + n q   (Sec. 3.3.3) */
};

enum zp_scale {
  ZP_SCALE_PROVEN = 0, /* gamma = the slot bound above (the batched correctness theorem) */
  ZP_SCALE_OVERLAP = 1 /* gamma = q^2 (uniform) or q (binary): neighbouring slots overlap,
                          which the modified decryption tolerates while the noise stays below
                          Delta / 4 (Sec. 3.3.3, "Better compression with a smaller scale") */
};

typedef struct zp_params {
  uint32_t n;        /* LWE dimension (1 <= n <= 4096) */
  uint32_t key_bits; /* bits of every client's Paillier modulus m; 2048 (compile-time limit) */
  uint32_t secret;   /* enum zp_secret */
  uint32_t p_bits;   /* log2 of the plaintext modulus p; must be 8 (one byte per entry) */
  uint32_t scale;    /* enum zp_scale. Slots per packed row: ell = the largest count with
                        (bound - 1) sum_{j<ell} gamma^j < 2^(key_bits - 1), bound = q + n q^2
                        (uniform) or q + n q (binary): 27 / 48 proven, 31 / 63 overlap at
                        2048 bits and n = 1024 */
} zp_params;

typedef struct zp_ctx zp_ctx;       /* one device, one parameter set */
typedef struct zp_db zp_db;         /* one resident database and its hint */
typedef struct zp_client zp_client; /* one client's public Paillier modulus and constants */
typedef struct zp_lc zp_lc;         /* standalone LWE compression: a Paillier modulus and an expanded key */

/* Library ABI version (major*10000 + minor*100 + patch). */
int zp_version(void);

/* Copies the calling thread's last error message (NUL-terminated, truncated to len).
 * Returns the message length. */
int zp_last_error(char* buf, size_t len);

/* Creates a context on CUDA device `device` for parameters *P.
 * Derived slot count (batched compression theorem, Sec. 3.3): ell is the largest
 * integer with gamma^ell < 2^(key_bits-1), so m > gamma^ell for every key of
 * key_bits bits and the packed hint is the same for all clients.
 * Errors: ZP_EINVAL (P null, n out of range, p_bits != 8), ZP_EUNSUPPORTED
 * (key_bits != 2048), ZP_ECUDA (device unusable). */
int zp_init(int device, const zp_params* P, zp_ctx** out);
int zp_ctx_destroy(zp_ctx* ctx);

/* Registers the database D (Algorithm "ZipPIR", db in Z_p^{d0 x d1}; here R x C).
 * dD: device pointer to R rows of ld_bytes bytes; row r holds D[r, 0..C-1], bytes
 * C..ld_bytes-1 are ignored. dD must be 16-byte aligned and ld_bytes a multiple of
 * 16 with ld_bytes >= C. 1 <= R <= 2^20, 1 <= C <= 2^20.
 * The library computes per-row sums of D (R x 4 bytes, library-owned) and keeps dD.
 * Errors: ZP_EINVAL, ZP_ENOMEM, ZP_ECUDA. Synchronous. */
int zp_setup_db(zp_ctx* ctx, const uint8_t* dD, uint32_t R, uint32_t C, uint64_t ld_bytes,
                zp_db** out);

/* A second handle on the database db (the paper has no counterpart): the view shares
 * everything db holds (D, its fp16 copy, the hint and its byte planes, the RNS tables) and
 * owns only its own working buffers, internal stream and events, so that several batches of
 * one database can be in flight at once, each on its own handle and stream (a serving loop
 * that overlaps same-database batches). The view reads db's current state at every call.
 * Calls that change that state (zp_gen_hint, zp_update_rows, zp_db_prepare_fp16,
 * zp_db_prepare_rns, zp_autotune) are refused on a view (ZP_EINVAL) and must be made on db,
 * ordered on the GPU after the views' work that reads the old state; a view compresses large
 * batches in RNS only after zp_db_prepare_rns(db) (ZP_ESTATE otherwise). Calls on db and its
 * views from different host threads need the caller's own lock. Given a view, the new view
 * shares the same database. Destroy views (zp_db_destroy) before db; destroying a view frees
 * only what it owns. Errors: ZP_EINVAL, ZP_ENOMEM. */
int zp_db_view(zp_db* db, zp_db** out);

/* Reports the packing of this database: slots per Paillier plaintext (ell), packed
 * rows d1' = ceil(R / ell), and 32-bit limbs per element of Z_m (L = key_bits/32). */
int zp_db_info(const zp_db* db, uint32_t* ell, uint32_t* d1p, uint32_t* L);
int zp_db_destroy(zp_db* db);

/* Global hint (Algorithm "ZipPIR" caption; reused by all clients, Sec. 4.3
 * "Reusability of the offline phase"): H+ = D.A mod 2^32, written to dH.
 * dA: C x n u32, row-major (the public LWE matrix). dH: R x n u32, row-major,
 * output; may be NULL if the caller does not want H+.
 * The library also stores the paper's H = -H+ mod 2^32 in its compression layout;
 * zp_compress needs it. hRows: NULL to compute every row, else a HOST array of
 * nrows distinct row indices < R whose hint rows are recomputed (the idle-time
 * regeneration after zp_update_rows, Sec. 6 "Database updates"); other rows of dH
 * are left untouched. hRows is read before the call returns. The same dA must be
 * passed on every call for one database. Asynchronous on `stream`.
 * Errors: ZP_EINVAL (null dA, bad row index), ZP_ENOMEM, ZP_ECUDA. */
int zp_gen_hint(zp_db* db, const uint32_t* dA, uint32_t* dH, const uint32_t* hRows,
                uint32_t nrows, void* stream);

/* LWE answer (Algorithm "ZipPIR", Response, first line): for each of B queries,
 * ans[b][r] = sum_c D[r][c] * Q[b][c] mod 2^32.
 * dQ: B x C u32 row-major (query b at dQ + b*C). dAns: B x R u32 row-major output.
 * 1 <= B <= 4096. Asynchronous on `stream`. Errors: ZP_EINVAL, ZP_ENOMEM, ZP_ECUDA. */
int zp_answer(zp_db* db, const uint32_t* dQ, uint32_t B, uint32_t* dAns, void* stream);

/* Single-query answer that allocates no device memory (the paper has no
 * counterpart; it serves callers of this library that cannot allocate). Same result
 * as zp_answer with B = 1: ans[r] = sum_c D[r][c] * q[c] mod 2^32, dQ: C u32, dAns:
 * R u32 (device). Some callers may not call cudaMalloc at all: latency-critical serving
 * threads that must never block on the device allocator (cudaMalloc can synchronise the
 * device), and plug-ins running inside a host whose memory manager owns every byte of HBM
 * and hands out none. zp_answer grows library scratch on demand; this entry
 * point instead keeps its scratch (the query byte planes) in a 1 MiB array compiled
 * into the library, which every GPU that loads the library holds until the process
 * exits. Limit: C <= 262144 columns (ZP_EINVAL above it, before any work). The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture. All calls on a device share the array,
 * so calls that overlap on the GPU (different streams, no ordering) race and give
 * wrong answers; calls ordered on one stream are safe, and each call rewrites every
 * plane it reads and zeroes dAns itself. Asynchronous on `stream`. Like every entry point,
 * it leaves the caller's current device as it found it.
 * Errors: ZP_EINVAL, ZP_ECUDA. */
int zp_answer_noalloc(zp_db* db, const uint32_t* dQ, uint32_t* dAns, void* stream);

/* Registers a client's public Paillier modulus m (Algorithm "ZipPIR", Setup: the
 * client sends m). hM: HOST array of L = key_bits/32 little-endian u32 limbs; m
 * must be odd with exactly key_bits bits. The library derives the Barrett constant
 * floor(2^(64 L) / m) and copies both to the device. Synchronous.
 * Errors: ZP_EINVAL (null, wrong L, m even or of the wrong size), ZP_ENOMEM, ZP_ECUDA. */
int zp_register_client(zp_ctx* ctx, const uint32_t* hM, uint32_t L, zp_client** out);
int zp_client_destroy(zp_client* cl);

/* Answer compression (Algorithm "ZipPIR", Response, second line, with batched
 * compression, Sec. 4.3): for each query b of client clients[b] with modulus m_b,
 *   t[b][r'] = ( sum_{j<ell} gamma^j * ( ans[b][r' ell + j]
 *                                       + sum_{i<n} H[r' ell + j][i] * cko[b][i] ) ) mod m_b
 * for r' < d1', where H = -D.A mod 2^32 (from zp_gen_hint) and answer rows
 * >= R count as zero. This equals (b' + H'.cko) mod m with the packed answer b'
 * and packed hint H'.
 * dAns: B x R u32 (from zp_answer). dCKO: B x n x L u32 limbs, little-endian, each
 * value < m_b (precondition; a value >= m_b gives the same result as its residue
 * only if it is < 2^(32 L)). dT: B x d1' x L u32 output, little-endian limbs.
 * Asynchronous on `stream`. Errors: ZP_EINVAL, ZP_ESTATE (no hint yet, or rows
 * updated since the last zp_gen_hint), ZP_ENOMEM, ZP_ECUDA. */
int zp_compress(zp_db* db, zp_client* const* clients, const uint32_t* dAns,
                const uint32_t* dCKO, uint32_t B, uint32_t* dT, void* stream);

/* The two halves of zp_compress, for callers that schedule them themselves.
 * zp_compress_products computes, for each query b, the exact row products
 * V[b][r] = sum_i H[r][i] * cko[b][i] (no dependence on the answers) into library
 * scratch; zp_compress_finish packs ans + V and reduces mod m_b into dT, exactly as
 * zp_compress. The products of one call are consumed by the next finish call with the
 * same B (ZP_ESTATE otherwise); both must be ordered on the caller's streams (the
 * finish after the products). For B = 1 with the "overlap_sms" option set, the products
 * use only that many SMs so that they can run concurrently with a single-query
 * zp_answer (which then leaves those SMs free).
 * Errors as zp_compress. */
int zp_compress_products(zp_db* db, const uint32_t* dCKO, uint32_t B, void* stream);
int zp_compress_finish(zp_db* db, zp_client* const* clients, const uint32_t* dAns, uint32_t B,
                       uint32_t* dT, void* stream);

/* The whole online Response for B queries on DEVICE buffers: zp_answer into dAns,
 * then zp_compress into dT. Asynchronous on `stream`. For one query with the
 * "overlap_sms" option set, the compression products run on an internal stream
 * (forked from and joined back to `stream` with events) on overlap_sms SMs while the
 * answer streams the database on the remaining SMs; for a batch answered on the tensor
 * cores ("batch_overlap"), they run on that stream beside the answers on whatever SMs are
 * free. */
int zp_respond(zp_db* db, zp_client* const* clients, const uint32_t* dQ, const uint32_t* dCKO,
               uint32_t B, uint32_t* dAns, uint32_t* dT, void* stream);

/* The whole online Response on HOST buffers: copies hQ (B x C u32) and hCKO
 * (B x n x L u32) to library-owned device buffers, runs zp_respond, copies the
 * compressed answers to hT (B x d1' x L u32) and, if hAns is not NULL, the plain
 * answers to hAns (B x R u32), then synchronises `stream`. Host buffers may be
 * pageable or pinned (pinned is faster). Errors as zp_respond. */
int zp_respond_host(zp_db* db, zp_client* const* clients, const uint32_t* hQ,
                    const uint32_t* hCKO, uint32_t B, uint32_t* hT, uint32_t* hAns,
                    void* stream);

/* Database update (Sec. 6, "Database updates"): overwrites rows hRows[0..k-1]
 * (HOST array of distinct indices < R, read before the call returns) of the
 * caller's database buffer with dNewRows (k x C bytes, row-major, pitch C),
 * updates the row sums and marks those hint rows stale. zp_compress returns
 * ZP_ESTATE until zp_gen_hint has recomputed every stale row (for example with
 * the same row list). Asynchronous on `stream`.
 * Errors: ZP_EINVAL, ZP_ENOMEM, ZP_ECUDA. */
int zp_update_rows(zp_db* db, const uint32_t* hRows, uint32_t k, const uint8_t* dNewRows,
                   void* stream);

/* Per-client hint (Algorithm "ZipPIR", Setup; Sec. 4.3 "Lowering offline communication
 * costs", k = PaillierMatMul(H', ck_r)), offline:
 *   k[r'] = prod_i ck_r[i]^{H'[r', i]} mod m^2,  H'[r', i] = sum_j gamma^j Hneg[r' ell + j, i]
 * (Hneg = -D.A mod 2^32, rows past R zero). The client decrypts k to H'.pt_r, the term
 * t leaves out. dCkr: n x 2L u32 (ck_r[i] < m^2, 2L little-endian limbs), 16-byte
 * aligned. dK: d1' x 2L u32 output, 16-byte aligned. hPackedRows: NULL for every packed
 * row, else a HOST array of nrows packed-row indices < d1' (the rows to recompute after
 * zp_update_rows and zp_gen_hint of their answer rows; other rows of dK are untouched),
 * read before the call returns. Needs the global hint and no stale rows. Work: about n
 * (popcount of a 32-bit exponent) Montgomery products mod m^2 per answer row plus
 * ell x 75 per packed row. Asynchronous on `stream`.
 * Errors: ZP_EINVAL, ZP_ESTATE (no hint or stale rows), ZP_ENOMEM, ZP_ECUDA. */
int zp_client_hint(zp_db* db, const zp_client* cl, const uint32_t* dCkr, uint32_t* dK,
                   const uint32_t* hPackedRows, uint32_t nrows, void* stream);

/* Autotuner: measures on `db` (zero-filled test buffers it allocates and frees; the
 * kernels' time does not depend on the values) and sets the context options to the fastest
 * choices:
 *  - "gemv_max_batch": the one-pass GEMV against the tensor-core GEMM for 2..4 queries;
 *  - "rns_min_batch": the byte-plane against the RNS compression for 2..16 queries (when the
 *    hint is ready, n <= 1024 and "compress_path" is auto; this builds the RNS tables);
 *  - "gemv_cfg_alone": the GEMV configuration of a single-query answer on the whole GPU;
 *  - "overlap_sms" and "gemv_cfg_shared": the SM split of the single-query zp_respond (0 and
 *    24%..52% of the SMs) and the GEMV configuration beside the compression products;
 *  - "answer_bt_16/32/64/128": the tile width (16, 32 or 64 queries) of the tensor-core
 *    answers for batches of 16, 32, 64 and 128 queries, and "answer_fp16" (the fp16 copy of D
 *    against its bytes, when the copy exists);
 *  - "rns_bt_16/32/64/128" and "batch_overlap": the tile width of the RNS products and
 *    whether a batch's products run beside its answers (when the RNS path was measured);
 *  - "pack_split": measured with the single-query SM split.
 * chosen (may be NULL): receives the first three values ("gemv_max_batch", "rns_min_batch",
 * "overlap_sms"); zp_get_option reads the others. Synchronous on `stream`; about a second
 * at 1 GiB. Errors: ZP_EINVAL, ZP_ENOMEM, ZP_ECUDA (the options are left as they were). */
int zp_autotune(zp_db* db, void* stream, int64_t* chosen);

/* Builds now the residues of H' modulo the RNS primes that the compression of large
 * batches uses (see "compress_path"), which the first such batch would otherwise build:
 * a serving loop calls it at setup so that no request waits for it. About 0.75 GB of
 * device memory per GiB of database at n = 1024. Asynchronous on `stream`.
 * Errors: ZP_EINVAL, ZP_ESTATE (no hint or stale rows), ZP_EUNSUPPORTED (n > 1024),
 * ZP_ENOMEM, ZP_ECUDA. */
int zp_db_prepare_rns(zp_db* db, void* stream);

/* Combined response (Sec. 4.3, last extension): out[b][r'] = k[b][r'] (1 + t[b][r'] m_b)
 * mod m_b^2, the homomorphic sum of the hint and t (encrypted with randomness 1), so that
 * Dec(out) = Dec(k) + t mod m: one ciphertext per packed row instead of (k, t).
 * dK: B x d1' x 2L u32 (k of query b's client, each < m_b^2); dT: B x d1' x L u32 (from
 * zp_compress); dOut: B x d1' x 2L u32 output. All 16-byte aligned. clients: B client
 * handles. Asynchronous on `stream`. Errors: ZP_EINVAL, ZP_ENOMEM, ZP_ECUDA. */
int zp_combine(zp_db* db, zp_client* const* clients, const uint32_t* dK, const uint32_t* dT,
               uint32_t B, uint32_t* dOut, void* stream);

/* Number of hint rows marked stale by zp_update_rows and not yet regenerated. */
int zp_stale_rows(const zp_db* db, uint32_t* count);

/* Selects kernel variants for this context (tuning and cross-checking):
 *   "answer_path":   0 auto (one pass of the dp4a GEMV for one to four queries,
 *                    tensor cores for larger batches and the hint), 1 CUDA-core dp4a
 *                    tiled kernels for every batch and the hint, 2 tensor cores also
 *                    for one to four queries;
 *   "compress_path": 0 auto (tensor cores when n <= 1024: byte planes of H for small
 *                    batches, residues modulo 153 primes below 2^27 from "rns_min_batch"
 *                    queries on), 1 CUDA-core products, 2 tensor-core byte planes, 3 RNS
 *                    (2 and 3: ZP_EUNSUPPORTED at call time if n > 1024). The RNS path
 *                    (Sec. 5.2: H'.ck_o modulo word-size primes, one reduction mod m at the
 *                    end by the Chinese remainder theorem) builds H' modulo the primes on
 *                    its first use for a database (about 0.75 GB per GiB of database at
 *                    n = 1024, milliseconds of GPU time) and keeps it in step with
 *                    zp_gen_hint; it needs a 16-byte aligned dCKO (else byte planes run);
 *   "rns_min_batch": smallest batch compressed in RNS under "auto" (default 8; 0 never);
 *   "gemv_max_batch": largest batch (1..4) answered by one GEMV pass under "auto"
 *                    (default 4; zp_autotune measures both);
 *   "overlap_sms":   the number of SMs on which the compression products of a single
 *                    query run while the answer uses the other SMs (zp_respond,
 *                    zp_compress_products, single-query zp_answer); 0 = no overlap.
 *                    Default: about 3/8 of the SMs (56 of 152) on GPUs with >= 64 SMs.
 *   "answer_bt_16", "answer_bt_32", "answer_bt_64", "answer_bt_128": queries per N tile
 *                    (16, 32 or 64; at most 16 / 32 / 64 / 64) of the tensor-core answers for
 *                    batches of <= 16, <= 32, <= 64 and more queries (defaults 16, 32, 64,
 *                    64); "rns_bt_16", ...: the same for the RNS products;
 *   "gemv_cfg_alone", "gemv_cfg_shared": the GEMV configuration on the whole GPU and beside
 *                    the compression products: 1 = 8 consumer warps x 12 stages of 64-row
 *                    tiles (default alone), 2 = 16 warps x 6 stages of 128-row tiles
 *                    (default shared);
 *   "batch_overlap": 1 (default) zp_respond runs the compression products of a batch
 *                    answered on the tensor cores on an internal stream beside the answers
 *                    (they do not read the answers), 0 one after the other;
 *   "pack_split":    1 (default) for one query zp_respond also packs and reduces the
 *                    products' part Y = (sum_j gamma^j V_j) mod m on the internal stream,
 *                    beside the answer, and after the join computes only (b' + Y) mod m
 *                    (one conditional subtraction: b' < m by the choice of ell); 0 packs
 *                    and reduces everything after the join.
 * Every variant computes the same exact result. Errors: ZP_EINVAL (unknown name or value). */
int zp_set_option(zp_ctx* ctx, const char* name, int64_t value);
/* Reads an option set by zp_set_option (or its default). Errors: ZP_EINVAL. */
int zp_get_option(const zp_ctx* ctx, const char* name, int64_t* value);

/* Number of kernels this context has launched so far (all entry points). */
int zp_kernel_launches(const zp_ctx* ctx, uint64_t* count);

/* Device-side error word of the context: nonzero after a kernel gave up a bounded
 * wait (its code says which). Reading it synchronises the device. The word is
 * cleared by the read. */
int zp_device_status(zp_ctx* ctx, uint32_t* code);

/* Resident fp16 copy of the database for batched answers: allocates R x Kp fp16 (Kp = C
 * rounded up to 128; twice the bytes of D) and fills it with D - 128 (centred, exact).
 * From then on the tensor-core answers (batches above gemv_max_batch) read it as their A
 * operand through TMA, with no byte-to-fp16 conversion in shared memory; zp_update_rows
 * keeps it current. With it, the residue planes of H' used by the RNS compression (when
 * built, by zp_db_prepare_rns or the first large batch) also get an fp16 copy (twice their
 * bytes), kept current by hint regeneration. Option "answer_fp16" (zp_set_option, default
 * 1) turns the use of both off (0) or on (1). Asynchronous on `stream`.
 * Errors: ZP_EINVAL, ZP_ENOMEM, ZP_ECUDA. */
int zp_db_prepare_fp16(zp_db* db, void* stream);

/* ChaCha20 keystream (RFC 8439 block function) on the GPU: dOut[0 .. nwords) receives the
 * little-endian 32-bit words of blocks counter0, counter0 + 1, ... for the 32-byte key hKey
 * and the 12-byte nonce hNonce (both HOST, read before the call returns). The PRG that
 * expands the public matrix A (Sec. 2.1.1) and ck_r (Sec. 4.3) from short seeds, for
 * servers that keep only the seed; the paper names no PRG, ChaCha20 is this library's
 * choice. Runs on the current device. Asynchronous on `stream`.
 * Errors: ZP_EINVAL (null argument, 32-bit block counter would wrap), ZP_ECUDA. */
int zp_prg_chacha20(const uint8_t* hKey, const uint8_t* hNonce, uint32_t counter0,
                    uint32_t* dOut, uint64_t nwords, void* stream);

/* Batched modular exponentiation mod m^2 of a client (Montgomery products, one warp per
 * base): dOut[i] = dBase[i]^e mod m^2 for i < count, e = the expWords (1..128) little-endian
 * words of the HOST array hExp. dBase, dOut: count x 2L u32, 16-byte aligned, each base
 * < m^2. The core of Paillier's decryption (e = lambda: Dec(c) = ((c^lambda mod m^2) - 1)/m
 * * mu mod m) and of its encryption's randomness factor (e = m), for client-side load
 * generation. Asynchronous on `stream`. Errors: ZP_EINVAL, ZP_ECUDA. */
int zp_client_powm(const zp_client* cl, const uint32_t* dBase, const uint32_t* hExp,
                   uint32_t expWords, uint32_t* dOut, uint32_t count, void* stream);

/* ck_r expanded from a seed on the GPU: dOut[i] (2L u32, i < count, 16-byte aligned)
 * = the keystream words [(2L+4) i, (2L+4)(i+1)) of zp_prg_chacha20(hKey, hNonce,
 * counter0), read as a little-endian integer of 2 key_bits + 128 bits, mod m^2 of the
 * client: statistically uniform in Z_{m^2} (Sec. 4.3: the client expands ck_r from a
 * short seed so that only the seed is sent offline). Asynchronous on `stream`.
 * Errors: ZP_EINVAL (null, misaligned, 32-bit block counter would wrap), ZP_ECUDA. */
int zp_client_expand_ckr(const zp_client* cl, const uint8_t* hKey, const uint8_t* hNonce,
                         uint32_t counter0, uint32_t* dOut, uint32_t count, void* stream);

/* Batched Paillier decryption (g = m + 1) on the GPU: dOut[i] (L u32) = Dec(dC[i]) =
 * ((dC[i]^(lambda mu) mod m^2) - 1) / m for i < count; dC is count x 2L u32, each in
 * Z*_{m^2}; hLam, hMu: the client's secret lambda and mu = lambda^{-1} mod m (HOST, L
 * words each, read before the call returns). The client-side decryptions of the protocol
 * (pt_r = Dec(ck_r) at setup, Dec(k) at extraction). dC, dOut 16-byte aligned.
 * Asynchronous on `stream`. Errors: ZP_EINVAL, ZP_ENOMEM, ZP_ECUDA. */
int zp_client_decrypt(const zp_client* cl, const uint32_t* hLam, const uint32_t* hMu,
                      const uint32_t* dC, uint32_t* dOut, uint32_t count, void* stream);

/* Failure-detection self-test: launches one kernel whose mbarrier wait nothing
 * satisfies, bounded by `cycles` SM clock cycles (at most 2^32, about 2 s). When the wait
 * gives up, the kernel sets bit 0x4 (a timeout outside the answer and product kernels) of
 * the status word and returns: the path every bounded wait of the library takes, so that
 * a wait that cannot complete costs its limit and an error code, never a hung or faulted
 * device. The context stays usable. Asynchronous on `stream`. Errors: ZP_EINVAL, ZP_ECUDA. */
int zp_selftest_wait(zp_ctx* ctx, uint64_t cycles, void* stream);

/* ---- Standalone compression of LWE ciphertexts and RLWE coefficients (Sec. 3, App. B) ----
 *
 * A Paillier modulus m (g = m + 1) of 2048 or 3072 bits and a compression key
 * ck[i] = Enc(s[i]) (i < n) of an LWE (or RLWE) secret s. LWECompress of ct = (a, b)
 * (Algorithm "LWE compression") is
 *     x = (1 + b m) prod_i ck[i]^{(q - a[i]) mod q}  mod m^2,
 * so that Dec(x) = b + sum_i ((q - a[i]) mod q) s[i] < q + n q^2 and Dec(x) mod q is the LWE
 * phase b - <a, s> mod q; batched compression (Algorithm "Batch Compression") of ell
 * ciphertexts is x = prod_j x_j^{gamma^j} (gamma = q + n q^2, or q + n q for binary s, and
 * gamma^ell < m). Integers mod q are u64 (q <= 2^64; q = 0 stands for 2^64), each below q;
 * Paillier ciphertexts are 2L u32 little-endian words (L = key_bits / 32), 16-byte aligned.
 * Deterministic: the result is bit-identical to the definition. */

/* m: HOST, key_bits / 32 words, odd, exactly key_bits bits (2048 or 3072). Runs on `device`.
 * Errors: ZP_EINVAL, ZP_EUNSUPPORTED (other key sizes), ZP_ENOMEM, ZP_ECUDA. */
int zp_lc_create(int device, uint32_t key_bits, const uint32_t* hM, zp_lc** out);
int zp_lc_destroy(zp_lc* lc);

/* Expanded key (Algorithm "Batch compression ... using precomputed powers"): from dCk (n x 2L
 * u32, each < m^2, device) the library keeps eck[i][k] = ck[i]^{2^k} mod m^2 for k < T (n T
 * 2L words of device memory, owned by lc). T must cover the exponents used: bits(q - 1)
 * for one ciphertext at a time, bits((q - 1) sum_{j < ell} gamma^j) (<= key_bits) for the
 * folded batched form. dCk may be freed once the call's stream work is done.
 * Errors: ZP_EINVAL (n = 0 or > 2^20, T = 0 or > key_bits, misaligned), ZP_ENOMEM, ZP_ECUDA. */
int zp_lc_set_key(zp_lc* lc, const uint32_t* dCk, uint32_t n, uint32_t T, void* stream);

/* Packed compression keys (appendix "LWECompress Using Packed Compression Keys"): from
 * ceil(n / t) packed ciphertexts dPck, dCk[i t + j] = dPck[i]^{delta^(t-1-j)} mod m^2 for
 * i t + j < n (by repeated exponentiation by delta). delta: HOST, deltaWords (1..8) words,
 * at least 2. dCk: n x 2L u32. Errors: ZP_EINVAL, ZP_ECUDA. */
int zp_lc_unpack_key(zp_lc* lc, const uint32_t* dPck, uint32_t n, uint32_t t,
                     const uint32_t* hDelta, uint32_t deltaWords, uint32_t* dCk, void* stream);

/* Compression of count ciphertexts: dA count x n u64 (row j = a of ciphertext j), dB count
 * u64, both device. ell = 1: dX[j] = LWECompress(ck, ct_j) (count x 2L u32). ell > 1: the
 * ciphertexts in groups of ell consecutive ones (the last group may be shorter), dX[g] =
 * prod_{j < ell_g} x_{g ell + j}^{gamma^j} (ceil(count / ell) x 2L u32); gamma: HOST,
 * gammaWords (1..8) words, > q - 1. mode: 0 auto, 1 Horner (per-ciphertext products, then
 * X <- X^gamma x_j per group), 2 folded (one exponent sum_j gamma^j e_j per base and group;
 * needs T >= its bits); both give the same bits. Requires (q - 1) sum_{j<ell} gamma^j < m.
 * Asynchronous on `stream` (scratch held by lc). Errors: ZP_EINVAL, ZP_ESTATE (no key),
 * ZP_ENOMEM, ZP_ECUDA. */
int zp_lc_compress(zp_lc* lc, const uint64_t* dA, const uint64_t* dB, uint32_t count, uint64_t q,
                   uint32_t ell, const uint32_t* hGamma, uint32_t gammaWords, int mode, uint32_t* dX,
                   void* stream);

/* Rescaling (modulus switching, Sec. 3.3 "Rescaling for Compression") of count LWE
 * ciphertexts from q to r (2 <= r < q; q = 0 stands for 2^64): every coefficient x of dA
 * (count x n u64) and dB (count u64) becomes round(x r / q) mod r, ties up
 * (floor((x r + floor(q / 2)) / q) mod r), written to dAout / dBout (same shapes; may
 * alias the inputs). Compressing the result with modulus r uses smaller exponents; the
 * paper states that decryption survives for binary keys with noise below Delta / 4.
 * Runs on the current device. Asynchronous on `stream`. Errors: ZP_EINVAL, ZP_ECUDA. */
int zp_lc_rescale(const uint64_t* dA, const uint64_t* dB, uint32_t count, uint32_t n, uint64_t q,
                  uint64_t r, uint64_t* dAout, uint64_t* dBout, void* stream);

/* Sample extraction of RLWE coefficients (App. B, Algorithm "Compressing Extracted RLWE
 * Coefficient"): for the RLWE ciphertext (A, B) over Z_q[X]/(X^N + 1) (dA, dB: N u64,
 * device) and coefficient indices hK[c] < N (HOST, count <= 65535), the LWE ciphertext
 * dAout[c] (N u64), dBout[c] = B[k] with a'[i] = A[k - i] (i <= k) and (q - A[N + k - i]) mod q
 * (i > k), whose compression by zp_lc_compress is RLWECompressCoefficient(ck, C, k).
 * Errors: ZP_EINVAL (k >= N, count too large), ZP_ENOMEM, ZP_ECUDA. */
int zp_lc_rlwe_extract(zp_lc* lc, const uint64_t* dA, const uint64_t* dB, uint32_t N, uint64_t q,
                       const uint32_t* hK, uint32_t count, uint64_t* dAout, uint64_t* dBout, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ZIPPIR_H */
