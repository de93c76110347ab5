/*
 * ppst.h -- C ABI of the GB300 RNS-CKKS evaluator for PP-STAT's encrypted
 * statistics (Z-score, coefficient of variation, skewness, kurtosis, Pearson
 * correlation) computed with CryptoInvSqrt: a Chebyshev initial guess refined
 * by Newton steps, with pre-normalisation scaling.
 *
 * The calls follow the paper's client/server statement (Sec. 4): the client
 * generates keys and encrypts columns with the public key; the server runs the
 * statistics (Sec. 6) on ciphertexts with the evaluation keys; the client
 * decrypts. Here both sides live in one process on one GPU; the secret key is
 * kept on the host except for the duration of keygen / decrypt.
 *
 * Conventions for every call:
 *  - Return value: PPST_OK (0) on success, a negative PPST_E_* code on error.
 *    The message of the last error of a context is ppst_last_error(ctx).
 *    On error, output handles are left NULL and nothing is leaked.
 *  - Handles are opaque, owned by the library, released with ppst_free()
 *    (any handle type; NULL is ignored). A handle must not outlive its ctx.
 *  - Host buffers (double*, uint64_t*, int64_t*) are owned by the caller, are
 *    read or written only during the call, and need no alignment beyond their
 *    type's.
 *  - Device memory comes from the ppst_allocator given at ctx creation (or
 *    cudaMalloc when none is given); all GPU work of a context is issued on
 *    the CUDA stream given at creation. Calls that return device-resident
 *    results (keygen, encrypt, query, ciphertext ops) may return before the
 *    GPU work finishes; calls that write host buffers synchronise the stream.
 *  - A context is not thread-safe; use one context per host thread.
 *  - Ciphertext limbs are uint64 residues, limb-major: limb i of a polynomial
 *    is N consecutive words modulo prime i of the chain (q_0 .. q_level).
 *    Import/export buffers are in the coefficient domain.
 */
#ifndef PPST_H
#define PPST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPST_OK 0
#define PPST_E_ARG (-1)      /* bad handle, size or option                       */
#define PPST_E_DEPTH (-2)    /* the modulus chain is exhausted (level < 0)       */
#define PPST_E_SCALE (-3)    /* Add/Sub of scales differing by >= 2^-20 (rel.)   */
#define PPST_E_OOM (-4)      /* the allocator returned NULL                      */
#define PPST_E_BUDGET (-5)   /* serving: the request does not fit the HBM budget */
#define PPST_E_CUDA (-6)     /* a CUDA runtime call failed                       */
#define PPST_E_TIMEOUT (-7)  /* serving: ppst_wait timed out                     */
#define PPST_E_STATE (-8)    /* object in the wrong state (e.g. missing key)     */

typedef struct ppst_ctx ppst_ctx;     /* parameters, tables, stream, memory pool   */
typedef struct ppst_sk ppst_sk;       /* secret key (host)                          */
typedef struct ppst_evk ppst_evk;     /* public, relinearisation, Galois keys (GPU) */
typedef struct ppst_ct ppst_ct;       /* one ciphertext (GPU, evaluation domain)    */
typedef struct ppst_col ppst_col;     /* encrypted column: ceil(n / (N/2)) cts + n  */
typedef struct ppst_res ppst_res;     /* encrypted statistic result + depth report  */
typedef struct ppst_server ppst_server; /* continuous-batching request loop        */
typedef struct ppst_plan ppst_plan;     /* a query captured as a CUDA graph         */

/* Parameter set (the paper fixes only N, Delta and logPQ, Sec. 7.1). Prime
 * chain rule: every prime is 1 mod 2N; q_0 is the largest prime below
 * 2^q0_bits; the n_p special primes are the next primes below 2^p_bits
 * (skipping q_0); q_1 .. q_{n_q-1} are the primes nearest 2^q_bits, taken
 * alternately above (odd index) and below (even index). Key switching uses
 * dnum digits of alpha = ceil(n_q / dnum) consecutive primes. */
typedef struct {
    uint32_t log_n;      /* N = 2^log_n, 10 <= log_n <= 16                 */
    uint32_t n_q;        /* L + 1 primes in Q, 2 <= n_q <= 60              */
    uint32_t n_p;        /* K special primes, 1 <= n_p <= 16               */
    uint32_t dnum;       /* number of key-switching digits, 1 <= dnum <= n_q */
    uint32_t q0_bits;    /* bit bound of q_0, <= 61                        */
    uint32_t q_bits;     /* target size of q_1 .. q_L, <= 60               */
    uint32_t p_bits;     /* bit bound of the special primes, <= 61         */
    double log_scale;    /* Delta = 2^log_scale                            */
    double sigma;        /* discrete Gaussian width (0 -> 3.2)             */
    uint32_t gauss_bound;/* truncation |e| <= bound (0 -> 19)              */
} ppst_params;

/* Device memory provider. alloc returns a device pointer of at least `bytes`
 * (256-byte aligned) usable on `stream`, or NULL; release returns it. Called
 * rarely: the library keeps freed buffers in its own size-bucketed pool. */
typedef struct {
    void *(*alloc)(void *user, size_t bytes, void *stream);
    void (*release)(void *user, void *ptr, size_t bytes, void *stream);
    void *user;
} ppst_allocator;

typedef enum {
    PPST_ZSCORE = 0, /* Alg. 4: vector result, one ciphertext per input ct  */
    PPST_CV = 1,     /* Alg. 6 for a positive mean (no Sign): scalar        */
    PPST_SKEW = 2,   /* third-moment mirror of Alg. 5: scalar               */
    PPST_KURT = 3,   /* Alg. 5 (plain, not excess, kurtosis): scalar        */
    PPST_PCC = 4,    /* Sec. 6.5, two columns: scalar                       */
    PPST_CV_SIGNED = 5 /* Alg. 6 with Sign, a mean of either sign: scalar.
                        * Sign(mu) = mu * CryptoInvSqrt(mu^2, B^2), and the
                        * inverse of the sign-corrected mean is that same root
                        * (1/|mu|): one level more than PPST_CV. Needs
                        * |Mean| / B in (0, 1] besides Var / B^2 in (0, 2]. */
} ppst_stat;

/* Per-query options. B_x, B_y: pre-normalisation bounds (Sec. 6.1, Eq. 2):
 * Variance(x, B) = Var / B^2 and Mean(x, B) = Mean / B must lie in (0, 2]
 * (the caller's responsibility: it cannot be checked on encrypted data).
 * cheb_log2deg k: Chebyshev degree 2^k - 1 (Alg. 3; 2 <= k <= 10).
 * newton_steps t: Newton iterations of Alg. 2 (0 <= t <= 10). */
typedef struct {
    double B_x, B_y;
    int32_t cheb_log2deg;
    int32_t newton_steps;
} ppst_qopts;

/* Depth report of a result: level of the inputs, level of the output, the
 * depth used (their difference), the output scale and ciphertext count. */
typedef struct {
    int32_t level_in, level_out, depth_used;
    double scale;
    uint32_t n_cts;
} ppst_report;

/* ---- context -------------------------------------------------------------
 * Builds the prime chain, the transform and base-conversion tables on the GPU.
 * `stream` is a cudaStream_t (NULL = the legacy default stream). `alloc` may
 * be NULL. Errors: PPST_E_ARG (parameters out of range), PPST_E_CUDA, OOM. */
int ppst_ctx_create(const ppst_params *params, const ppst_allocator *alloc, void *stream,
                    ppst_ctx **out);
const char *ppst_last_error(const ppst_ctx *ctx);
/* Tile of the key-switching inner product (no counterpart in the paper): the
 * transform chunks each block owns, 4 (default), 8 or 16 (PPST_E_ARG
 * otherwise). Changes speed only, never results; the autotuner measures it. */
int ppst_ctx_set_tile(ppst_ctx *ctx, uint32_t inner_sub);
/* Block shape of the transform passes (no counterpart in the paper): a pass
 * over few limbs runs 8 or 4 sub-transforms per block instead of 16 (and the
 * inner product a smaller tile than ppst_ctx_set_tile's) whenever 16 would give
 * a grid of fewer than `min_blocks` blocks (default 228 = 1.5 x 152 SMs; 0: always
 * 16; 2^20: always 4). Changes speed only, never results. PPST_E_ARG above 2^20. */
int ppst_ctx_set_pass_blocks(ppst_ctx *ctx, uint32_t min_blocks);
/* Thread shape of the key-switching inner product (no counterpart in the
 * paper): its transform pass keeps 16 or 8 words per thread (8: one warp per
 * 256-point chunk, three butterfly rounds; used at N = 2^15 and 2^16 only, 16
 * elsewhere). flags: bit 0 (8 words only) accumulates the key products exactly
 * in 128 bits and reduces once per word; bit 1 (8 words only) exchanges the
 * transform's words between the rounds by warp shuffles instead of through
 * shared memory; bit 2 runs ModDown's CHUNKS transform pass with 8 words per
 * thread as well, bit 3 ModUp's COLS pass when its grid is small (fewer than
 * 456 blocks of the 16-word form: low levels), bit 4 the first inverse pass
 * (the tensor product's, the automorphism's and the plain inverse
 * transforms') (N = 2^15, 2^16). Default: 8 words, flags 29 (all but the
 * shuffle exchanges: the fastest measured at N = 2^16). Speed only, never
 * results. PPST_E_ARG for other values. */
int ppst_ctx_set_inner_shape(ppst_ctx *ctx, uint32_t words_per_thread, uint32_t flags);
/* Failure-detection self-test (no counterpart in the paper): launches one block
 * that waits on a shared-memory barrier nothing completes, bounded by timeout_us
 * (1 .. 10^6); like the kernels with asynchronous copies, it records the timeout
 * in the context's error word and returns. The launch itself returns PPST_OK; the
 * next synchronising call (ppst_sync, a decryption, an export) returns
 * PPST_E_CUDA and clears the word; the context stays usable. */
int ppst_selftest_wait(ppst_ctx *ctx, uint32_t timeout_us);
/* The prime chain of the context (Sec. 7.1 fixes only its total size; the
 * rule that picks the primes is the library's): primes_out[0 .. n_q + n_p) =
 * q_0 .. q_L, p_0 .. p_{K-1}; *n_primes = n_q + n_p. Writes at most `cap`
 * primes (primes_out may be NULL to query the count). */
int ppst_ctx_primes(const ppst_ctx *ctx, uint64_t *primes_out, size_t cap, uint32_t *n_primes);
/* Block until all GPU work issued on the context's stream has finished. */
int ppst_sync(ppst_ctx *ctx);
/* Bytes currently held by the context's memory pool (in use + cached). */
int ppst_mem_info(const ppst_ctx *ctx, size_t *in_use, size_t *cached);

/* ---- keys (client side, Sec. 4 item 1) -------------------------------------
 * Secret s: ternary; public key (-a s + e, a) over Q; relinearisation key
 * (s^2 -> s) and Galois keys (s(X^(5^r)) -> s) for the rotations listed
 * (NULL / 0: all powers of two 1 .. N/4, which rotate-and-sum needs). All
 * randomness comes from ChaCha20 (RFC 8439) keyed by SplitMix64(seed).
 * Errors: PPST_E_ARG, PPST_E_OOM, PPST_E_CUDA. */
int ppst_keygen(ppst_ctx *ctx, uint64_t seed, const int32_t *rotations, size_t n_rot,
                ppst_sk **sk_out, ppst_evk **evk_out);
/* s as N signed coefficients in {-1, 0, 1} (cap >= N). */
int ppst_sk_export(const ppst_ctx *ctx, const ppst_sk *sk, int64_t *s_out, size_t cap);
/* Digit `digit` of a switching key, coefficient domain, rows q_0..q_L, p_0..p_{K-1}
 * ([n_q + n_p][N] each). which = -1: relinearisation key; otherwise the
 * Galois key of rotation `which`. Synchronises. */
int ppst_evk_export(ppst_ctx *ctx, const ppst_evk *evk, int32_t which, uint32_t digit,
                    uint64_t *b_out, uint64_t *a_out);

/* ---- encryption / decryption (client side, Sec. 4 items 1 and 3) ----------
 * A column of n reals: ceil(n / (N/2)) ciphertexts at the top level and scale
 * Delta, slot j of ciphertext i holding x[i N/2 + j] (zero padded).
 * Ciphertext i uses encryption stream (seed, i). |x| must stay below 2^12 at
 * Delta = 2^50 (E_ARG otherwise). */
int ppst_encrypt_column(ppst_ctx *ctx, const ppst_evk *evk, const double *x, size_t n,
                        uint64_t seed, ppst_col **out);
/* Encrypt a plaintext given as N signed integer coefficients (already scaled),
 * with stream (seed, index): the ciphertext the client would send. */
int ppst_encrypt_ints(ppst_ctx *ctx, const ppst_evk *evk, const int64_t *m, uint64_t seed,
                      uint32_t index, double scale, ppst_ct **out);
/* Decrypt a statistic result: scalars give 1 value (slot 0); Z-score gives the
 * column's n values. Writes min(cap, count) values; *n_out = count. */
int ppst_decrypt(ppst_ctx *ctx, const ppst_sk *sk, const ppst_res *res, double *out, size_t cap,
                 size_t *n_out, ppst_report *report);
/* Decrypt one ciphertext to its N/2 slot values (cap >= N/2). */
int ppst_decrypt_ct(ppst_ctx *ctx, const ppst_sk *sk, const ppst_ct *ct, double *out, size_t cap);

/* ---- statistics (server side, Sec. 6) --------------------------------------
 * Runs the statistic on the context's stream. y is used by PPST_PCC only (same
 * row count as x). Errors: PPST_E_ARG, PPST_E_DEPTH (chain too short for the
 * options), PPST_E_STATE (a needed Galois key is missing), OOM, CUDA. */
int ppst_query(ppst_ctx *ctx, const ppst_evk *evk, ppst_stat stat, const ppst_col *x,
               const ppst_col *y, const ppst_qopts *opts, ppst_res **out);
/* Run `count` independent queries as one batch: every evaluator op of the
 * batch is issued for all queries together (one launch per op step, keys read
 * once per batch). Results are identical to ppst_query's. */
int ppst_query_batch(ppst_ctx *ctx, const ppst_evk *evk, size_t count, const ppst_stat *stats,
                     const ppst_col *const *xs, const ppst_col *const *ys,
                     const ppst_qopts *opts, ppst_res **outs);
/* Number of result ciphertexts and a view of one of them (owned by the result). */
int ppst_res_count(const ppst_res *res, uint32_t *n_cts);
int ppst_res_ct(const ppst_res *res, uint32_t i, const ppst_ct **ct_out);

/* ---- columns built from ciphertexts ----------------------------------------
 * A column of n_rows values held by n_cts ciphertexts (copied). */
int ppst_col_from_cts(ppst_ctx *ctx, const ppst_ct *const *cts, size_t n_cts, size_t n_rows,
                      ppst_col **out);
/* Row and ciphertext counts of a column, and a view of its i-th ciphertext
 * (owned by the column). */
int ppst_col_info(const ppst_col *col, size_t *n_rows, uint32_t *n_cts);
int ppst_col_ct(const ppst_col *col, uint32_t i, const ppst_ct **ct_out);

/* ---- ciphertext ops (Add/Mul/Rot of Sec. 3.1) -------------------------------
 * import/export: coefficient-domain limbs, c0 and c1 each [level + 1][N].
 * Export synchronises. */
int ppst_ct_import(ppst_ctx *ctx, const uint64_t *c0, const uint64_t *c1, uint32_t level,
                   double scale, ppst_ct **out);
int ppst_ct_export(ppst_ctx *ctx, const ppst_ct *ct, uint64_t *c0, uint64_t *c1,
                   uint32_t *level, double *scale);
int ppst_ct_level(const ppst_ct *ct, uint32_t *level, double *scale);
/* Mul(C): tensor, relinearise (hybrid key switch), add, rescale. */
int ppst_hmult(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, const ppst_ct *b,
               ppst_ct **out);
/* Mul(C) that allocates no device memory (the paper has no counterpart: this
 * serves callers that must not allocate once running, e.g. a host whose own
 * allocator already holds all free HBM, or a latency-critical serving thread
 * that cannot take cudaMalloc's device synchronisation). Same result as
 * ppst_hmult, written into `out`, a ciphertext the caller already owns (any
 * level; its contents, level and scale are replaced; it must not be a or b).
 * Every temporary lives in one static 32 MiB device array that each GPU
 * loading the library holds until exit; parameter sets needing more return
 * PPST_E_ARG (N = 2^12 with 20 primes fits; N = 2^16 does not). Creating a
 * context looks up the array's address on its device, which is when the
 * driver commits the array's memory there; the kernels a call launches load
 * on their first launch, so make one call before the free memory is handed to
 * another allocator. Calls share the array: calls whose GPU work overlaps
 * race. It calls no device allocator: not cudaMalloc/cudaFree, not the
 * context's pool, not the ppst_allocator. On an error `out` is unchanged. */
int ppst_hmult_noalloc(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, const ppst_ct *b,
                       ppst_ct *out);
/* Rot: slot j of the result = slot j + r of the input (Galois key needed). */
int ppst_rotate(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, int32_t r, ppst_ct **out);
/* Batched Mul(C) and Rot (Sec. 3.1; batching has no counterpart in the paper):
 * n = 1 .. 16 independent operations whose key switches share one launch
 * sequence, so each switching-key tile is read from HBM once for the batch.
 * hmult_batch: out[i] = a[i] * b[i]; every pair must have the same level
 * min(level(a[i]), level(b[i])). rotate_batch: out[i] = Rot(a[i], r); every
 * a[i] at one level. `out` has room for n handles; on error every out[i] is
 * NULL. Results are bit-identical to n single calls. Errors: PPST_E_ARG
 * (n out of range, levels differ, bad handle), PPST_E_DEPTH, PPST_E_STATE
 * (missing key), PPST_E_OOM, PPST_E_CUDA. */
int ppst_hmult_batch(ppst_ctx *ctx, const ppst_evk *evk, size_t n, const ppst_ct *const *a,
                     const ppst_ct *const *b, ppst_ct **out);
int ppst_rotate_batch(ppst_ctx *ctx, const ppst_evk *evk, size_t n, const ppst_ct *const *a, int32_t r,
                      ppst_ct **out);
/* Rotate-and-sum over all N/2 slots (every slot = the total). */
int ppst_rotsum(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, ppst_ct **out);
int ppst_rescale(ppst_ctx *ctx, const ppst_ct *a, ppst_ct **out);
int ppst_add(ppst_ctx *ctx, const ppst_ct *a, const ppst_ct *b, ppst_ct **out);
int ppst_sub(ppst_ctx *ctx, const ppst_ct *a, const ppst_ct *b, ppst_ct **out);
/* Add(P): round(c * scale) (ties away from zero) added to every slot. */
int ppst_add_const(ppst_ctx *ctx, const ppst_ct *a, double c, ppst_ct **out);
/* Mul(P) then rescale: integer round(k * q_l), k = c (target <= 0) or
 * c * (target / scale); the result's scale is target (or the input scale). */
int ppst_mul_const(ppst_ctx *ctx, const ppst_ct *a, double c, double target, ppst_ct **out);
int ppst_mul_int(ppst_ctx *ctx, const ppst_ct *a, int64_t k, ppst_ct **out);
/* sum_k c_k a_k for 1..32 ciphertexts at one level: integer weights
 * round(c_k (target / scale_k) q_l) (exact, ties away from zero), one rescale;
 * the result's scale is `target`. The Chebyshev leaf sums of Alg. 3. */
int ppst_lin_comb(ppst_ctx *ctx, const ppst_ct *const *cts, const double *coeffs, size_t n, double target,
                  ppst_ct **out);
/* Keep limbs 0..level. */
int ppst_drop(ppst_ctx *ctx, const ppst_ct *a, uint32_t level, ppst_ct **out);
/* CryptoInvSqrt(v, C) (Sec. 5: Alg. 2 with n = 2, Alg. 3, Eq. 1, Eq. 3) on
 * every slot: the degree 2^cheb_log2deg - 1 Chebyshev interpolant of
 * 1 / (sqrt(C) sqrt(u + 1)) at u = v - 1, then newton_steps Newton steps
 * y <- 1.5 y - (x' y) y^2, x' = v C / 2. Approximates 1 / sqrt(C v) for v in
 * (0, 2]; outside that domain the result is meaningless (not detectable on
 * encrypted data). cheb_log2deg in [2, 10], newton_steps in [0, 10], C > 0.
 * Uses cheb_log2deg + 1 + 2 newton_steps levels (cheb_log2deg >= 3);
 * PPST_E_DEPTH when the input's level is too low. */
int ppst_inv_sqrt(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *v, double C, int32_t cheb_log2deg,
                  int32_t newton_steps, ppst_ct **out);

/* ---- prepared queries ---------------------------------------------------------
 * ppst_query_prepare runs the statistic program once (which sizes a private
 * key-switch workspace), then captures it as a CUDA graph; each ppst_plan_run
 * replays the graph (one launch on the context's stream) and returns a new
 * result, identical to ppst_query's for the same inputs. The plan keeps its
 * columns' device buffers alive and holds its own workspace and intermediates
 * until ppst_free(plan). Errors as ppst_query; PPST_E_STATE if the program
 * needed a new device allocation during the capture. */
int ppst_query_prepare(ppst_ctx *ctx, const ppst_evk *evk, ppst_stat stat, const ppst_col *x, const ppst_col *y,
                       const ppst_qopts *opts, ppst_plan **out);
int ppst_plan_run(ppst_plan *plan, ppst_res **out);

/* ---- serving (continuous batching) -----------------------------------------
 * A request loop on its own host threads (GPU work on the context's stream):
 * keys stay resident, queries are admitted while their estimated working sets,
 * plus the results finished but not yet handed over by ppst_wait, fit
 * `hbm_budget` bytes (and at most `max_batch` run together); their ops are
 * batched step by step, and results are handed back by ticket. Admission
 * follows arrival order, except that a query which does not fit may be passed
 * by later ones that do until it has waited 500 ms; from then on nothing
 * passes it. hbm_budget = 0: the device memory free at creation (cudaMemGetInfo:
 * keys and columns already resident are not free) plus the context pool's
 * cached buffers, less 5 % of the device (PPST_E_BUDGET if nothing is left).
 * The paper's server runs one query at a time (Sec. 4); the loop is this
 * library's. */
typedef struct {
    size_t budget;    /* bytes the loop may use                             */
    size_t reserved;  /* working-set estimates of the queries running       */
    size_t held;      /* results finished and not yet taken by ppst_wait    */
    uint32_t running; /* queries running                                    */
    uint32_t queued;  /* queries waiting for admission                      */
} ppst_server_stats;
int ppst_server_create(ppst_ctx *ctx, const ppst_evk *evk, size_t hbm_budget, uint32_t max_batch,
                       ppst_server **out);
int ppst_server_info(ppst_server *srv, ppst_server_stats *out);
/* The admission estimate of a query (working set, result bytes), as submit
 * computes it; PPST_E_ARG for an invalid query. */
int ppst_server_estimate(ppst_server *srv, ppst_stat stat, const ppst_col *x, const ppst_col *y,
                         size_t *working, size_t *result);
/* Enqueue a query; returns immediately with a ticket. PPST_E_BUDGET if the
 * query alone (working set and result) can never fit the budget. */
int ppst_submit(ppst_server *srv, ppst_stat stat, const ppst_col *x, const ppst_col *y,
                const ppst_qopts *opts, uint64_t *ticket);
/* Wait for a ticket (timeout_ms < 0: forever). PPST_E_TIMEOUT on timeout (the
 * ticket stays valid). On success the result is handed over to the caller. */
int ppst_wait(ppst_server *srv, uint64_t ticket, int32_t timeout_ms, ppst_res **out);
/* Latency of a finished ticket, in seconds from submit to result ready. */
int ppst_ticket_latency(ppst_server *srv, uint64_t ticket, double *seconds);

/* ---- kernel timing ----------------------------------------------------------
 * While profiling is on, every launch of the named kernel class (NULL or "":
 * every class) is bracketed by CUDA events on the context's stream. Classes:
 * ntt_cols_fwd, ntt_chunks_fwd, ntt_chunks_inv, ntt_cols_inv (transform
 * passes), modup_cols, inner_chunks, moddown_top, moddown_cols, moddown_chunks
 * (fused key switching), modup, inner_product, moddown_conv, moddown_final
 * (unfused key switching), rescale_cols, rescale_chunks, tensor, automorph,
 * lincomb, elementwise, copy. ppst_prof_read synchronises, returns the launch
 * count, summed device time and summed algorithmic traffic of one class, and
 * forgets them; the traffic is counted in limbs of N words (8N bytes each), as
 * the limbs a kernel must read once plus the limbs it writes (`units`), and as
 * the limbs of the operation's own operands it moves (`method_units`, may be
 * NULL): the input and output ciphertexts and the switching key, each counted
 * once per batched launch, not the intermediates the fused kernels exchange
 * (HMult + key switch at the top level, dnum = 6: 4 x 24 input limbs for the
 * tensor product, 6 x 2 x 28 key limbs for the inner product, 2 x 23 output
 * limbs for the last ModDown pass). ppst_prof_classes
 * writes the recorded class names, comma separated. ppst_launch_count: kernels
 * this context has launched so far (always counted, profiling on or off). */
int ppst_prof_start(ppst_ctx *ctx, const char *kernel_class);
int ppst_prof_stop(ppst_ctx *ctx);
int ppst_prof_read(ppst_ctx *ctx, const char *kernel_class, uint64_t *launches, double *total_ms,
                   uint64_t *units, uint64_t *method_units);
int ppst_prof_classes(ppst_ctx *ctx, char *buf, size_t cap);
int ppst_launch_count(const ppst_ctx *ctx, uint64_t *launches);

/* Release any handle (ctx last). NULL is ignored. */
void ppst_free(void *handle);

#ifdef __cplusplus
}
#endif
#endif /* PPST_H */
