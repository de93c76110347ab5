// ctx.cuh -- context, handles and internal entry points of the library.
#pragma once
#include <atomic>
#include <complex>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ppst.h"
#include "common.cuh"

namespace ppst {

// handle tags (first word of every handle, checked by the C ABI)
enum Tag : uint32_t {
    TAG_CTX = 0x50435458u, TAG_SK = 0x50534b30u, TAG_EVK = 0x5045564bu, TAG_CT = 0x50435430u,
    TAG_COL = 0x50434f4cu, TAG_RES = 0x50524553u, TAG_SRV = 0x50535256u, TAG_PLAN = 0x504c414eu,
    TAG_DEAD = 0xdeadbeefu
};

struct Error {
    int code;
    std::string msg;
};

// size-bucketed device memory pool on top of the user's allocator
struct Pool {
    ppst_allocator user{};
    bool has_user = false;
    cudaStream_t stream = nullptr;
    std::unordered_map<size_t, std::vector<void *>> free_;
    size_t in_use = 0, cached = 0;
    std::recursive_mutex mu;  // batched queries release ciphertexts from their own threads
    // graph capture: `recording` notes every buffer handed out; `frozen` turns a
    // request that the free lists cannot serve into PPST_E_STATE (no allocator
    // call while a stream is being captured)
    bool recording = false, frozen = false;
    std::vector<std::pair<void *, size_t>> ledger;
    void *get(size_t bytes);
    void put(void *p, size_t bytes);
    bool withdraw(void *p, size_t bytes);  // take a free buffer out of circulation
    void trim();
};

struct Ctx;

// Ciphertexts are immutable once written: every op writes a new buffer, so a
// lower-level view (a "drop") can share its parent's buffer.
struct CtObj {
    uint32_t tag = TAG_CT;
    Ctx *ctx = nullptr;
    std::shared_ptr<uint64_t> buf;  // owner of the device buffer (shared by views)
    uint64_t *d = nullptr;  // [2][L+1][N], evaluation (NTT) domain, limbs 0..level valid
    int level = 0;
    double scale = 1.0;
    uint64_t *c0() const;
    uint64_t *c1() const;
};

struct Swk {
    uint64_t *d = nullptr;  // [dnum][2][L+1+K][N], evaluation domain, Montgomery form (x 2^64)
};

struct SkObj {
    uint32_t tag = TAG_SK;
    Ctx *ctx = nullptr;
    std::vector<int64_t> s;
};

struct EvkObj {
    uint32_t tag = TAG_EVK;
    Ctx *ctx = nullptr;
    uint64_t *pk = nullptr;  // [2][L+1][N] evaluation domain, standard form
    Swk relin;
    std::map<int, Swk> rot;  // rotation amount (mod N/2) -> Galois key
    uint64_t seed = 0;
};

struct ColObj {
    uint32_t tag = TAG_COL;
    Ctx *ctx = nullptr;
    std::vector<CtObj *> cts;
    size_t n = 0;
};

struct ResObj {
    uint32_t tag = TAG_RES;
    Ctx *ctx = nullptr;
    std::vector<CtObj *> cts;
    int stat = 0;
    size_t n = 0;
    int level_in = 0;
};

// offsets of the per-digit base-conversion tables of one level, by value in launches
struct DigitOffs {
    uint64_t off[MAXL];
};

// per (level l, limb i) constants of the fused ModDown + rescale
struct MdC {
    Tw pinv;    // P^-1 mod q_i
    Tw qlinv;   // q_l^-1 mod q_i (i < l)
    Tw pq;      // P^-1 q_l^-1 mod q_i
    uint64_t qmod, pad;  // q_l mod q_i
};

// per-kernel-class timing with CUDA events on the launching stream
struct ProfRec {
    cudaEvent_t b, e;
    uint64_t units;   // work units of the launch (limbs for transforms and elementwise kernels)
    uint64_t munits;  // limbs of the op's own inputs and outputs (ciphertexts, keys) the launch moves
};
struct Prof {
    bool on = false;
    std::string only;  // "" = every class
    std::vector<cudaEvent_t> spare;
    std::map<std::string, std::vector<ProfRec>> rec;
    std::atomic<uint64_t> launches{0};  // kernel launches issued by this context (always counted)
    cudaEvent_t take();
};

struct Ctx {
    uint32_t tag = TAG_CTX;
    uint32_t pass_min_blocks = 228;  // transform passes: smaller blocks below this grid size (1.5 x 152 SMs)
    Prof prof;
    ppst_params prm{};
    int logN = 0, N = 0, S = 0, L = 0, K = 0, dnum = 0, alpha = 0, np = 0;
    double scale = 1.0, sigma = 3.2;
    int gbound = 19;
    std::vector<uint64_t> primes;  // q_0..q_L, p_0..p_{K-1}
    std::vector<PrimeC> hpc;       // host copy of the per-prime constants
    std::vector<uint64_t> psi;
    std::vector<std::complex<double>> twist;  // zeta^i, zeta = e^(i pi / N): decoding (host)
    PrimeC *d_pc = nullptr;
    Tw *d_twf = nullptr, *d_twi = nullptr;  // [prime][N]: psi^brv(k), psi^-brv(k) with Shoup companions
    uint64_t *d_cdt = nullptr;  // discrete Gaussian CDT
    std::vector<uint64_t> cdt;
    // key-switching tables (device), offsets per (level, digit)
    uint64_t *d_ks = nullptr;
    std::vector<std::vector<size_t>> modup_off;  // [level][digit] -> offset of hatinv (a) | hatinv_sh (a) | hatM (a x ext)
    size_t moddown_off = 0;                      // hatinvP (K) | hatinvP_sh (K) | hatMP (K x (L+1))
    ConstVec pinv;                               // P^-1 mod q_i, Shoup
    std::vector<ConstVec> resc;                  // [level]: q_l^-1 mod q_i, Shoup (i < l)
    std::vector<ConstVec> resc_qmodv;            // [level]: q_l mod q_i (i < l)
    std::vector<ConstVec> pmod;                  // [0]: P mod q_t for all primes (gadget), Shoup
    // fused key switching: N^-1 (Q_j/q_i)^-1 per (level, limb); N^-1 (P/p_m)^-1 per P row of both
    // accumulators; ModDown + rescale constants per (level, limb)
    Tw *d_modup_outmul = nullptr;
    std::vector<size_t> modup_outmul_off;
    Tw *d_md_outmul = nullptr;
    Tw *d_md_outmul_top = nullptr;  // per level l: N^-1 mod q_l, then the K entries of d_md_outmul
    MdC *d_md_const = nullptr;
    std::vector<MdC> md_const;
    cudaStream_t stream = nullptr;
    // error word that kernels with bounded waits set on a timeout: pinned,
    // mapped host memory, readable without synchronising the stream
    volatile int *h_err = nullptr;
    int *d_err = nullptr;
    Pool pool;
    Error err{0, ""};
    std::mutex err_mu;  // server threads may record errors concurrently
    // Held while GPU work is issued (each ABI call; each scheduling round of a
    // server), so that a server and direct calls never share the workspace at once.
    std::recursive_mutex exec_mu;
    // workspace (allocated on first key switch)
    // (each with a leading item dimension of ws_items for batched key switching)
    uint64_t *ws_d2 = nullptr;   // [L+1][N]
    uint64_t *ws_d2n = nullptr;  // [L+1][N] key-switch input kept in the evaluation domain
    uint64_t *ws_ext = nullptr;  // [dnum][L+1+K][N]
    uint64_t *ws_acc = nullptr;  // [2][L+1+K][N]
    uint64_t *ws_conv = nullptr; // [2][L+1][N]
    uint64_t *ws_top = nullptr;  // [2][N]
    int ws_items = 0;
    size_t ws_bytes = 0;
    int inner_sub = 4;  // chunks per block of the key inner product (4, 8 or 16; autotuned)
    int inner_words = 8;     // words per thread of the inner product's transform (8 is used at N >= 2^15 only)
    bool inner_lazy = true;  // 8 words: accumulate the key products in 128 bits, reduce once
    bool inner_shfl = false; // 8 words: the transform's exchanges by warp shuffles instead of shared memory
    int md_words = 8;        // words per thread of ModDown's last (CHUNKS) pass: 8 (used at N >= 2^15) or 16
    int modup_words = 8;     // ModUp's COLS pass: 8 words per thread on small grids (N >= 2^15), or always 16
    int inv_words = 8;       // words per thread of the first inverse pass (tensor, automorphism, plain
                             // inverse transforms): 8 (used at N >= 2^15) or 16

    size_t ct_words() const { return (size_t)2 * (L + 1) * N; }
    size_t ext_rows() const { return (size_t)(L + 1 + K); }
    int ndigits(int level) const { return (level + 1 + alpha - 1) / alpha; }
    void clear_err()
    {
        std::lock_guard<std::mutex> lk(err_mu);
        err = Error{0, ""};
    }
    int fail(int code, const std::string &m)
    {
        std::lock_guard<std::mutex> lk(err_mu);
        err.code = code;
        err.msg = m;
        return code;
    }
};

inline uint64_t *CtObj::c0() const { return d; }
inline uint64_t *CtObj::c1() const { return d + (size_t)(ctx->L + 1) * ctx->N; }

// C++ exception used inside the library, converted to an error code at the ABI
struct PpstError {
    int code;
    std::string msg;
};
[[noreturn]] void throw_err(int code, const std::string &m);
void cuda_check(cudaError_t e, const char *what);
#define PPST_CUDA(x) ::ppst::cuda_check((x), #x)
void check_launch(const char *what);

// brackets the launches of one kernel class with events when profiling is on
struct ProfScope {
    Ctx &c;
    const char *cls;
    uint64_t units, munits;
    cudaEvent_t b = nullptr;
    ProfScope(Ctx &cc, const char *k, uint64_t u = 0, uint64_t mu = 0);
    ~ProfScope();
};

// ---- host math (host_math.cu) ----
uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q);
uint64_t h_powmod(uint64_t b, uint64_t e, uint64_t q);
uint64_t h_invmod(uint64_t a, uint64_t q);
uint64_t h_shoup(uint64_t w, uint64_t q);  // floor(w 2^64 / q)
bool h_is_prime(uint64_t n);
// exact round-half-away of a double to a signed 128-bit integer (|x| < 2^126)
__int128 h_round_away(double x);
// exact round-half-away of (k * m), k double, m integer < 2^62
__int128 h_round_mul(double k, uint64_t m);
uint64_t h_mod_i128(__int128 v, uint64_t q);

// ---- context (context.cu) ----
Ctx *ctx_create(const ppst_params &p, const ppst_allocator *alloc, cudaStream_t stream);
void ctx_destroy(Ctx *c);
void ensure_workspace(Ctx &c, int items = 1);  // key-switch workspace for `items` ciphertexts
CtObj *ct_new(Ctx &c, int level, double scale);
void ct_free(CtObj *ct);
CtObj *ct_clone(const CtObj &a);             // a view of the same buffer and level
CtObj *ct_view(const CtObj &a, int level);   // a view of limbs 0..level

// ---- NTT (ntt.cu) ----
void ntt_fwd(Ctx &c, const LimbMap &m);
void ntt_inv(Ctx &c, const LimbMap &m);
// inverse NTT whose final N^-1 is replaced by outmul[b] (N^-1 times a per-limb constant)
void ntt_inv_mul(Ctx &c, const LimbMap &m, const Tw *outmul);
// the last (COLS) pass only, for limbs whose CHUNKS pass ran fused into another kernel
void ntt_inv_cols_mul(Ctx &c, const LimbMap &m, const Tw *outmul);
// rescale of a (level l) into out given limb l of both polynomials in the coefficient
// domain (top, [2][N]) and per-limb multipliers mq_i (m_i q_l^-1); z: scratch [2][L+1][N]
void ks_rescale(Ctx &c, const CtObj &a, const uint64_t *top, uint64_t *z, const ConstVec &mq, CtObj &out);
LimbMap map_ct(const Ctx &c, uint64_t *d, int level);  // both polys of a ciphertext buffer
LimbMap map_poly(const Ctx &c, uint64_t *d, int level); // one poly, limbs 0..level

// ---- kernels (kernels.cu) ----
void k_add(Ctx &c, const CtObj &a, const CtObj &b, CtObj &out, bool sub);
void k_neg(Ctx &c, const CtObj &a, CtObj &out);
void k_mul_scalar_ct(Ctx &c, const CtObj &a, const ConstVec &cv, CtObj &out);
void k_add_scalar_c0(Ctx &c, const CtObj &a, const ConstVec &cv, CtObj &out);
void k_tensor(Ctx &c, const CtObj &a, const CtObj &b, int level, uint64_t *d0, uint64_t *d1, uint64_t *d2);
// the same, d2 written to two buffers
void k_tensor2(Ctx &c, const CtObj &a, const CtObj &b, int level, uint64_t *d0, uint64_t *d1, uint64_t *d2,
               uint64_t *d2b);
void k_modup(Ctx &c, const uint64_t *d2coef, int level, uint64_t *ext);
void k_inner_product(Ctx &c, const uint64_t *ext, const Swk &key, int level, uint64_t *acc);
void k_moddown(Ctx &c, uint64_t *acc, int level, const uint64_t *add0, const uint64_t *add1, uint64_t *out0,
               uint64_t *out1);
void k_rescale(Ctx &c, const CtObj &a, CtObj &out);
// rescale of (a times the per-limb constants mul), without materialising the product
void k_rescale_mul(Ctx &c, const CtObj &a, const ConstVec *mul, CtObj &out);
struct LinArgs {
    static constexpr int MAXT = 32;
    const uint64_t *p[MAXT];
    __int128 m[MAXT];
    int n;
};
void k_lincomb(Ctx &c, const LinArgs &args, int level, CtObj &out);
void k_automorph(Ctx &c, const uint64_t *in, int level, uint64_t galois, uint64_t *out, size_t poly_stride,
                 int npoly);
void k_copy(Ctx &c, uint64_t *dst, const uint64_t *src, size_t words);
void k_sample_uniform(Ctx &c, uint64_t seed, uint32_t purpose, uint32_t index, const LimbMap &m);
void k_sample_small(Ctx &c, uint64_t seed, uint32_t purpose, uint32_t index, bool gauss, int64_t *out);
void k_small_to_rns(Ctx &c, const int64_t *v, const LimbMap &m);
void k_swk_combine(Ctx &c, uint64_t *b, const uint64_t *a, const uint64_t *e, const uint64_t *s,
                   const uint64_t *snew, int digit_lo, int digit_hi);
void k_pk_combine(Ctx &c, uint64_t *b, const uint64_t *a, const uint64_t *e, const uint64_t *s);
void k_enc_combine(Ctx &c, const uint64_t *pk, const uint64_t *u, const uint64_t *e0, const uint64_t *e1,
                   const uint64_t *m, CtObj &out);
void k_dec_combine(Ctx &c, const CtObj &ct, const uint64_t *s, uint64_t *m);
void k_to_mont(Ctx &c, uint64_t *d, const LimbMap &m, bool to);
void k_pointwise_sq(Ctx &c, const uint64_t *a, uint64_t *out, const LimbMap &m);

// ---- evaluator (eval.cu) ----
CtObj *ev_add(Ctx &c, const CtObj &a, const CtObj &b, bool sub);
CtObj *ev_add_const(Ctx &c, const CtObj &a, double x);
CtObj *ev_mul_int(Ctx &c, const CtObj &a, int64_t k);
CtObj *ev_mul_const(Ctx &c, const CtObj &a, double x, double target);  // target <= 0: keep scale
CtObj *ev_rescale(Ctx &c, const CtObj &a);
// sum_k c_k a_k with integer weights round(c_k (target / scale_k) q_l) and one rescale
CtObj *ev_lin_comb(Ctx &c, const std::vector<const CtObj *> &cts, const std::vector<double> &coeffs, double target);
CtObj *ev_hmult(Ctx &c, const EvkObj &k, const CtObj &a, const CtObj &b);
CtObj *ev_rotate(Ctx &c, const EvkObj &k, const CtObj &a, int r);
// up to 16 independent HMults / rotations in one pass of launches (pairs at one level)
// device address of the allocation-free HMult's static scratch array on the
// current device (looked up once per device; noalloc.cu)
uint64_t *noalloc_scratch_on_current_device();
std::vector<CtObj *> ev_hmult_batch(Ctx &c, const EvkObj &k, const std::vector<const CtObj *> &as,
                                    const std::vector<const CtObj *> &bs);
std::vector<CtObj *> ev_rotate_batch(Ctx &c, const EvkObj &k, const std::vector<const CtObj *> &as, int r);
CtObj *ev_rotsum(Ctx &c, const EvkObj &k, const CtObj &a);
CtObj *ev_drop(Ctx &c, const CtObj &a, int level);
uint64_t galois_elt(const Ctx &c, int r);

// ---- keys, encryption, encoding (keys.cu) ----
void keygen(Ctx &c, uint64_t seed, const std::vector<int> &rots, SkObj *&sk, EvkObj *&evk);
CtObj *encrypt_ints(Ctx &c, const EvkObj &k, const int64_t *m, uint64_t seed, uint32_t index, double scale);
void encode(const Ctx &c, const double *z, size_t n, double scale, std::vector<int64_t> &m);
// slots of a ciphertext; want = 1: slot 0 only (the others are left 0)
void decrypt_to_slots(Ctx &c, const SkObj &sk, const CtObj &ct, std::vector<double> &slots, int want = 0);
void export_ct(Ctx &c, const CtObj &ct, uint64_t *c0, uint64_t *c1);
CtObj *import_ct(Ctx &c, const uint64_t *c0, const uint64_t *c1, int level, double scale);
void export_swk(Ctx &c, const Swk &k, int digit, uint64_t *b, uint64_t *a);

// ---- statistics (stats.cu) ----
struct QueryIn {
    int stat;
    const ColObj *x, *y;
    ppst_qopts o;
};
void run_queries(Ctx &c, const EvkObj &k, const std::vector<QueryIn> &qs, std::vector<ResObj *> &out);
void validate_query(const Ctx &c, const QueryIn &q);  // PPST_E_ARG on a malformed query
CtObj *ev_inv_sqrt(Ctx &c, const EvkObj &k, const CtObj &v, double C, int cheb_log2deg, int newton_steps);
// PPST_E_CUDA if a kernel reported a timed-out wait (the word is then cleared);
// call once the work in question has completed
void check_device_error(Ctx &c);
// launches one block whose bounded barrier wait runs out after timeout_us (ks.cu)
void wait_selftest(Ctx &c, uint32_t timeout_us);

// ---- serving and prepared queries (stats.cu) ----
struct Server;
void server_destroy(Server *s);
struct Plan;
void plan_destroy(Plan *p);

}  // namespace ppst
