// capi.cu -- the extern "C" boundary (include/ppst.h).
#include <cmath>
#include <cstring>
#include <new>

#include "ctx.cuh"

using namespace ppst;

namespace {

template <class F>
int guard(Ctx *c, F &&f)
{
    try {
        std::unique_lock<std::recursive_mutex> lk;
        if (c) lk = std::unique_lock<std::recursive_mutex>(c->exec_mu);
        f();
        if (c) c->clear_err();
        return PPST_OK;
    } catch (const PpstError &e) {
        if (c) c->fail(e.code, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        if (c) c->fail(PPST_E_OOM, "host allocation failed");
        return PPST_E_OOM;
    } catch (...) {
        if (c) c->fail(PPST_E_ARG, "unexpected error");
        return PPST_E_ARG;
    }
}

template <class T>
bool ok(const T *h, uint32_t tag)
{
    return h && h->tag == tag;
}

#define REQ(cond, msg)                                  \
    do {                                                \
        if (!(cond)) throw_err(PPST_E_ARG, (msg));      \
    } while (0)

const ppst_qopts default_opts = {1.0, 1.0, 7, 3};

void check_opts(const ppst_qopts &o, int stat)
{
    REQ(o.cheb_log2deg >= 2 && o.cheb_log2deg <= 10, "cheb_log2deg out of range [2, 10]");
    REQ(o.newton_steps >= 0 && o.newton_steps <= 10, "newton_steps out of range [0, 10]");
    REQ(o.B_x > 0 && std::isfinite(o.B_x), "B_x must be positive");
    if (stat == PPST_PCC) REQ(o.B_y > 0 && std::isfinite(o.B_y), "B_y must be positive");
}

}  // namespace

namespace ppst {
void validate_query(const Ctx &cc, const QueryIn &q)
{
    const Ctx *c = &cc;
    REQ(q.stat >= PPST_ZSCORE && q.stat <= PPST_CV_SIGNED, "unknown statistic");
    REQ(ok(q.x, TAG_COL) && q.x->ctx == c, "bad column");
    if (q.stat == PPST_PCC) {
        REQ(ok(q.y, TAG_COL) && q.y->ctx == c && q.y->n == q.x->n && q.y->cts.size() == q.x->cts.size(),
            "PCC needs a second column of the same length");
        REQ(q.y->cts[0]->level == q.x->cts[0]->level, "PCC columns at different levels");
    }
    for (const CtObj *ct : q.x->cts) REQ(ct->level == q.x->cts[0]->level, "column ciphertexts at mixed levels");
    check_opts(q.o, q.stat);
}
}  // namespace ppst

extern "C" {

int ppst_ctx_create(const ppst_params *params, const ppst_allocator *alloc, void *stream, ppst_ctx **out)
{
    if (!out) return PPST_E_ARG;
    *out = nullptr;
    if (!params) return PPST_E_ARG;
    try {
        *out = (ppst_ctx *)ctx_create(*params, alloc, (cudaStream_t)stream);
        return PPST_OK;
    } catch (const PpstError &e) {
        return e.code;
    } catch (...) {
        return PPST_E_OOM;
    }
}

const char *ppst_last_error(const ppst_ctx *ctx)
{
    const Ctx *c = (const Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return "invalid context";
    return c->err.msg.c_str();
}

int ppst_ctx_set_tile(ppst_ctx *ctx, uint32_t inner_sub)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        REQ(inner_sub == 4 || inner_sub == 8 || inner_sub == 16, "inner_sub must be 4, 8 or 16");
        c->inner_sub = (int)inner_sub;
    });
}

int ppst_ctx_set_inner_shape(ppst_ctx *ctx, uint32_t words_per_thread, uint32_t flags)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        REQ(words_per_thread == 8 || words_per_thread == 16, "words_per_thread must be 8 or 16");
        REQ(flags <= 31 && ((flags & 3) == 0 || words_per_thread == 8), "flags 1, 2 need 8 words per thread");
        c->inner_words = (int)words_per_thread;
        c->inner_lazy = (flags & 1) != 0;
        c->inner_shfl = (flags & 2) != 0;
        c->md_words = (flags & 4) ? 8 : 16;
        c->modup_words = (flags & 8) ? 8 : 16;
        c->inv_words = (flags & 16) ? 8 : 16;
    });
}

int ppst_ctx_set_pass_blocks(ppst_ctx *ctx, uint32_t min_blocks)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        REQ(min_blocks <= (1u << 20), "min_blocks out of range [0, 2^20]");
        c->pass_min_blocks = min_blocks;
    });
}

int ppst_selftest_wait(ppst_ctx *ctx, uint32_t timeout_us)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        REQ(timeout_us >= 1 && timeout_us <= 1000000, "timeout_us out of range [1, 10^6]");
        wait_selftest(*c, timeout_us);
    });
}

int ppst_ctx_primes(const ppst_ctx *ctx, uint64_t *primes_out, size_t cap, uint32_t *n_primes)
{
    const Ctx *c = (const Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (n_primes) *n_primes = (uint32_t)c->primes.size();
    for (size_t i = 0; primes_out && i < cap && i < c->primes.size(); i++) primes_out[i] = c->primes[i];
    return PPST_OK;
}

int ppst_sync(ppst_ctx *ctx)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        PPST_CUDA(cudaStreamSynchronize(c->stream));
        check_device_error(*c);
    });
}

int ppst_mem_info(const ppst_ctx *ctx, size_t *in_use, size_t *cached)
{
    const Ctx *c = (const Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (in_use) *in_use = c->pool.in_use;
    if (cached) *cached = c->pool.cached;
    return PPST_OK;
}

int ppst_keygen(ppst_ctx *ctx, uint64_t seed, const int32_t *rotations, size_t n_rot, ppst_sk **sk_out,
                ppst_evk **evk_out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!sk_out || !evk_out) return c->fail(PPST_E_ARG, "null output");
    *sk_out = nullptr;
    *evk_out = nullptr;
    return guard(c, [&] {
        std::vector<int> rots;
        if (rotations && n_rot) {
            for (size_t i = 0; i < n_rot; i++) rots.push_back(rotations[i]);
        } else {
            for (int i = 0; (1 << i) < c->S; i++) rots.push_back(1 << i);
        }
        SkObj *sk;
        EvkObj *evk;
        keygen(*c, seed, rots, sk, evk);
        *sk_out = (ppst_sk *)sk;
        *evk_out = (ppst_evk *)evk;
    });
}

int ppst_sk_export(const ppst_ctx *ctx, const ppst_sk *sk, int64_t *s_out, size_t cap)
{
    const Ctx *c = (const Ctx *)ctx;
    const SkObj *s = (const SkObj *)sk;
    if (!ok(c, TAG_CTX) || !ok(s, TAG_SK) || !s_out || cap < (size_t)c->N) return PPST_E_ARG;
    std::memcpy(s_out, s->s.data(), (size_t)c->N * 8);
    return PPST_OK;
}

int ppst_evk_export(ppst_ctx *ctx, const ppst_evk *evk, int32_t which, uint32_t digit, uint64_t *b_out,
                    uint64_t *a_out)
{
    Ctx *c = (Ctx *)ctx;
    const EvkObj *k = (const EvkObj *)evk;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        REQ(ok(k, TAG_EVK) && b_out && a_out && (int)digit < c->dnum, "bad arguments");
        const Swk *s = nullptr;
        if (which < 0) {
            s = &k->relin;
        } else {
            const int rr = which % c->S;
            auto it = k->rot.find(rr);
            if (it == k->rot.end()) throw_err(PPST_E_STATE, "no Galois key for that rotation");
            s = &it->second;
        }
        export_swk(*c, *s, (int)digit, b_out, a_out);
    });
}

int ppst_encrypt_column(ppst_ctx *ctx, const ppst_evk *evk, const double *x, size_t n, uint64_t seed, ppst_col **out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!out) return c->fail(PPST_E_ARG, "null output");
    *out = nullptr;
    return guard(c, [&] {
        const EvkObj *k = (const EvkObj *)evk;
        REQ(ok(k, TAG_EVK) && x && n > 0, "bad arguments");
        ColObj *col = new ColObj();
        col->ctx = c;
        col->n = n;
        try {
            const size_t nct = (n + c->S - 1) / c->S;
            std::vector<int64_t> m;
            for (size_t i = 0; i < nct; i++) {
                const size_t lo = i * c->S, cnt = std::min((size_t)c->S, n - lo);
                encode(*c, x + lo, cnt, c->scale, m);
                col->cts.push_back(encrypt_ints(*c, *k, m.data(), seed, (uint32_t)i, c->scale));
            }
        } catch (...) {
            for (CtObj *ct : col->cts) ct_free(ct);
            delete col;
            throw;
        }
        *out = (ppst_col *)col;
    });
}

int ppst_encrypt_ints(ppst_ctx *ctx, const ppst_evk *evk, const int64_t *m, uint64_t seed, uint32_t index,
                      double scale, ppst_ct **out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!out) return c->fail(PPST_E_ARG, "null output");
    *out = nullptr;
    return guard(c, [&] {
        const EvkObj *k = (const EvkObj *)evk;
        REQ(ok(k, TAG_EVK) && m && scale > 0, "bad arguments");
        *out = (ppst_ct *)encrypt_ints(*c, *k, m, seed, index, scale);
    });
}

int ppst_decrypt(ppst_ctx *ctx, const ppst_sk *sk, const ppst_res *res, double *out, size_t cap, size_t *n_out,
                 ppst_report *report)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        const SkObj *s = (const SkObj *)sk;
        const ResObj *r = (const ResObj *)res;
        REQ(ok(s, TAG_SK) && ok(r, TAG_RES) && (out || cap == 0), "bad arguments");
        std::vector<double> slots;
        size_t count;
        if (r->stat == PPST_ZSCORE) {
            count = r->n;
            size_t w = 0;
            for (size_t i = 0; i < r->cts.size() && w < std::min(cap, count); i++) {
                decrypt_to_slots(*c, *s, *r->cts[i], slots);
                for (int j = 0; j < c->S && w < std::min(cap, count); j++) out[w++] = slots[j];
            }
        } else {
            count = 1;
            decrypt_to_slots(*c, *s, *r->cts[0], slots, 1);  // a statistic sits in slot 0 (every slot)
            if (cap) out[0] = slots[0];
        }
        if (n_out) *n_out = count;
        if (report) {
            report->level_in = r->level_in;
            report->level_out = r->cts[0]->level;
            report->depth_used = r->level_in - r->cts[0]->level;
            report->scale = r->cts[0]->scale;
            report->n_cts = (uint32_t)r->cts.size();
        }
    });
}

int ppst_decrypt_ct(ppst_ctx *ctx, const ppst_sk *sk, const ppst_ct *ct, double *out, size_t cap)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        const SkObj *s = (const SkObj *)sk;
        const CtObj *a = (const CtObj *)ct;
        REQ(ok(s, TAG_SK) && ok(a, TAG_CT) && out && cap >= (size_t)c->S, "bad arguments");
        std::vector<double> slots;
        decrypt_to_slots(*c, *s, *a, slots);
        std::memcpy(out, slots.data(), (size_t)c->S * sizeof(double));
    });
}

static void run_checked(Ctx *c, const EvkObj *k, size_t count, const ppst_stat *stats, const ppst_col *const *xs,
                 const ppst_col *const *ys, const ppst_qopts *opts, ppst_res **outs)
{
    REQ(ok(k, TAG_EVK) && k->ctx == c && stats && xs && outs, "bad arguments");
    std::vector<QueryIn> qs;
    for (size_t i = 0; i < count; i++) {
        outs[i] = nullptr;
        QueryIn q;
        q.stat = stats[i];
        q.x = (const ColObj *)xs[i];
        q.y = ys ? (const ColObj *)ys[i] : nullptr;
        q.o = opts ? opts[i] : default_opts;
        validate_query(*c, q);
        qs.push_back(q);
    }
    std::vector<ResObj *> res;
    try {
        run_queries(*c, *k, qs, res);
    } catch (...) {
        for (ResObj *r : res) {
            for (CtObj *ct : r->cts) ct_free(ct);
            delete r;
        }
        throw;
    }
    for (size_t i = 0; i < count; i++) outs[i] = (ppst_res *)res[i];
}

int ppst_query(ppst_ctx *ctx, const ppst_evk *evk, ppst_stat stat, const ppst_col *x, const ppst_col *y,
               const ppst_qopts *opts, ppst_res **out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!out) return c->fail(PPST_E_ARG, "null output");
    *out = nullptr;
    return guard(c, [&] {
        const ppst_col *xs[1] = {x}, *ys[1] = {y};
        run_checked(c, (const EvkObj *)evk, 1, &stat, xs, ys, opts, out);
    });
}

int ppst_query_batch(ppst_ctx *ctx, const ppst_evk *evk, size_t count, const ppst_stat *stats,
                     const ppst_col *const *xs, const ppst_col *const *ys, const ppst_qopts *opts, ppst_res **outs)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] { run_checked(c, (const EvkObj *)evk, count, stats, xs, ys, opts, outs); });
}

int ppst_res_count(const ppst_res *res, uint32_t *n_cts)
{
    const ResObj *r = (const ResObj *)res;
    if (!ok(r, TAG_RES) || !n_cts) return PPST_E_ARG;
    *n_cts = (uint32_t)r->cts.size();
    return PPST_OK;
}

int ppst_res_ct(const ppst_res *res, uint32_t i, const ppst_ct **ct_out)
{
    const ResObj *r = (const ResObj *)res;
    if (!ok(r, TAG_RES) || !ct_out || i >= r->cts.size()) return PPST_E_ARG;
    *ct_out = (const ppst_ct *)r->cts[i];
    return PPST_OK;
}

int ppst_col_from_cts(ppst_ctx *ctx, const ppst_ct *const *cts, size_t n_cts, size_t n_rows, ppst_col **out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!out) return c->fail(PPST_E_ARG, "null output");
    *out = nullptr;
    return guard(c, [&] {
        REQ(cts && n_cts > 0 && n_rows > 0 && n_rows <= n_cts * (size_t)c->S && n_rows > (n_cts - 1) * (size_t)c->S,
            "row count does not match the ciphertext count");
        ColObj *col = new ColObj();
        col->ctx = c;
        col->n = n_rows;
        try {
            for (size_t i = 0; i < n_cts; i++) {
                const CtObj *a = (const CtObj *)cts[i];
                REQ(ok(a, TAG_CT) && a->ctx == c, "bad ciphertext");
                col->cts.push_back(ct_clone(*a));
            }
        } catch (...) {
            for (CtObj *ct : col->cts) ct_free(ct);
            delete col;
            throw;
        }
        *out = (ppst_col *)col;
    });
}

int ppst_col_info(const ppst_col *col, size_t *n_rows, uint32_t *n_cts)
{
    const ColObj *c = (const ColObj *)col;
    if (!ok(c, TAG_COL)) return PPST_E_ARG;
    if (n_rows) *n_rows = c->n;
    if (n_cts) *n_cts = (uint32_t)c->cts.size();
    return PPST_OK;
}

int ppst_col_ct(const ppst_col *col, uint32_t i, const ppst_ct **ct_out)
{
    const ColObj *c = (const ColObj *)col;
    if (!ok(c, TAG_COL) || !ct_out || i >= c->cts.size()) return PPST_E_ARG;
    *ct_out = (const ppst_ct *)c->cts[i];
    return PPST_OK;
}

int ppst_ct_import(ppst_ctx *ctx, const uint64_t *c0, const uint64_t *c1, uint32_t level, double scale,
                   ppst_ct **out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!out) return c->fail(PPST_E_ARG, "null output");
    *out = nullptr;
    return guard(c, [&] {
        REQ(c0 && c1 && (int)level <= c->L && scale > 0, "bad arguments");
        *out = (ppst_ct *)import_ct(*c, c0, c1, (int)level, scale);
    });
}

int ppst_ct_export(ppst_ctx *ctx, const ppst_ct *ct, uint64_t *c0, uint64_t *c1, uint32_t *level, double *scale)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    return guard(c, [&] {
        const CtObj *a = (const CtObj *)ct;
        REQ(ok(a, TAG_CT) && a->ctx == c, "bad ciphertext");
        if (level) *level = (uint32_t)a->level;
        if (scale) *scale = a->scale;
        if (c0 && c1) export_ct(*c, *a, c0, c1);
    });
}

int ppst_ct_level(const ppst_ct *ct, uint32_t *level, double *scale)
{
    const CtObj *a = (const CtObj *)ct;
    if (!ok(a, TAG_CT)) return PPST_E_ARG;
    if (level) *level = (uint32_t)a->level;
    if (scale) *scale = a->scale;
    return PPST_OK;
}

#define CT_OP(name, body)                                                          \
    Ctx *c = (Ctx *)ctx;                                                           \
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;                                        \
    if (!out) return c->fail(PPST_E_ARG, "null output");                           \
    *out = nullptr;                                                                \
    return guard(c, [&] {                                                          \
        const CtObj *A = (const CtObj *)a;                                         \
        REQ(ok(A, TAG_CT) && A->ctx == c, "bad ciphertext");                       \
        body                                                                       \
    });

int ppst_hmult(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, const ppst_ct *b, ppst_ct **out)
{
    CT_OP(hmult, {
        const CtObj *B = (const CtObj *)b;
        const EvkObj *k = (const EvkObj *)evk;
        REQ(ok(B, TAG_CT) && B->ctx == c && ok(k, TAG_EVK), "bad arguments");
        *out = (ppst_ct *)ev_hmult(*c, *k, *A, *B);
    })
}

int ppst_rotate(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, int32_t r, ppst_ct **out)
{
    CT_OP(rotate, {
        const EvkObj *k = (const EvkObj *)evk;
        REQ(ok(k, TAG_EVK), "bad key");
        *out = (ppst_ct *)ev_rotate(*c, *k, *A, r);
    })
}

int ppst_hmult_batch(ppst_ctx *ctx, const ppst_evk *evk, size_t n, const ppst_ct *const *a,
                     const ppst_ct *const *b, ppst_ct **out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!out || !a || !b) return c->fail(PPST_E_ARG, "null argument");
    for (size_t i = 0; i < n; i++) out[i] = nullptr;
    return guard(c, [&] {
        const EvkObj *k = (const EvkObj *)evk;
        REQ(ok(k, TAG_EVK), "bad key");
        REQ(n >= 1 && n <= 16, "hmult batch: 1 to 16 pairs");
        std::vector<const CtObj *> as(n), bs(n);
        for (size_t i = 0; i < n; i++) {
            as[i] = (const CtObj *)a[i];
            bs[i] = (const CtObj *)b[i];
            REQ(ok(as[i], TAG_CT) && as[i]->ctx == c && ok(bs[i], TAG_CT) && bs[i]->ctx == c, "bad ciphertext");
        }
        std::vector<CtObj *> r = ev_hmult_batch(*c, *k, as, bs);
        for (size_t i = 0; i < n; i++) out[i] = (ppst_ct *)r[i];
    });
}

int ppst_rotate_batch(ppst_ctx *ctx, const ppst_evk *evk, size_t n, const ppst_ct *const *a, int32_t r,
                      ppst_ct **out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!out || !a) return c->fail(PPST_E_ARG, "null argument");
    for (size_t i = 0; i < n; i++) out[i] = nullptr;
    return guard(c, [&] {
        const EvkObj *k = (const EvkObj *)evk;
        REQ(ok(k, TAG_EVK), "bad key");
        REQ(n >= 1 && n <= 16, "rotate batch: 1 to 16 ciphertexts");
        std::vector<const CtObj *> as(n);
        for (size_t i = 0; i < n; i++) {
            as[i] = (const CtObj *)a[i];
            REQ(ok(as[i], TAG_CT) && as[i]->ctx == c, "bad ciphertext");
        }
        std::vector<CtObj *> o = ev_rotate_batch(*c, *k, as, r);
        for (size_t i = 0; i < n; i++) out[i] = (ppst_ct *)o[i];
    });
}

int ppst_rotsum(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, ppst_ct **out)
{
    CT_OP(rotsum, {
        const EvkObj *k = (const EvkObj *)evk;
        REQ(ok(k, TAG_EVK), "bad key");
        *out = (ppst_ct *)ev_rotsum(*c, *k, *A);
    })
}

int ppst_inv_sqrt(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, double C, int32_t cheb_log2deg,
                  int32_t newton_steps, ppst_ct **out)
{
    CT_OP(inv_sqrt, {
        const EvkObj *k = (const EvkObj *)evk;
        REQ(ok(k, TAG_EVK) && k->ctx == c, "bad key");
        REQ(cheb_log2deg >= 2 && cheb_log2deg <= 10, "cheb_log2deg out of range [2, 10]");
        REQ(newton_steps >= 0 && newton_steps <= 10, "newton_steps out of range [0, 10]");
        REQ(C > 0 && std::isfinite(C), "C must be positive");
        *out = (ppst_ct *)ev_inv_sqrt(*c, *k, *A, C, cheb_log2deg, newton_steps);
    })
}

int ppst_rescale(ppst_ctx *ctx, const ppst_ct *a, ppst_ct **out)
{
    CT_OP(rescale, { *out = (ppst_ct *)ev_rescale(*c, *A); })
}

int ppst_add(ppst_ctx *ctx, const ppst_ct *a, const ppst_ct *b, ppst_ct **out)
{
    CT_OP(add, {
        const CtObj *B = (const CtObj *)b;
        REQ(ok(B, TAG_CT) && B->ctx == c, "bad ciphertext");
        *out = (ppst_ct *)ev_add(*c, *A, *B, false);
    })
}

int ppst_sub(ppst_ctx *ctx, const ppst_ct *a, const ppst_ct *b, ppst_ct **out)
{
    CT_OP(sub, {
        const CtObj *B = (const CtObj *)b;
        REQ(ok(B, TAG_CT) && B->ctx == c, "bad ciphertext");
        *out = (ppst_ct *)ev_add(*c, *A, *B, true);
    })
}

int ppst_add_const(ppst_ctx *ctx, const ppst_ct *a, double x, ppst_ct **out)
{
    CT_OP(add_const, { *out = (ppst_ct *)ev_add_const(*c, *A, x); })
}

int ppst_mul_const(ppst_ctx *ctx, const ppst_ct *a, double x, double target, ppst_ct **out)
{
    CT_OP(mul_const, { *out = (ppst_ct *)ev_mul_const(*c, *A, x, target); })
}

int ppst_mul_int(ppst_ctx *ctx, const ppst_ct *a, int64_t k, ppst_ct **out)
{
    CT_OP(mul_int, { *out = (ppst_ct *)ev_mul_int(*c, *A, k); })
}

int ppst_lin_comb(ppst_ctx *ctx, const ppst_ct *const *cts, const double *coeffs, size_t n, double target,
                  ppst_ct **out)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    if (!out) return c->fail(PPST_E_ARG, "null output");
    *out = nullptr;
    return guard(c, [&] {
        REQ(cts && coeffs && n >= 1 && n <= (size_t)LinArgs::MAXT, "bad arguments");
        std::vector<const CtObj *> v;
        std::vector<double> cs(coeffs, coeffs + n);
        for (size_t i = 0; i < n; i++) {
            const CtObj *A = (const CtObj *)cts[i];
            REQ(ok(A, TAG_CT) && A->ctx == c, "bad ciphertext");
            v.push_back(A);
        }
        *out = (ppst_ct *)ev_lin_comb(*c, v, cs, target);
    });
}

int ppst_drop(ppst_ctx *ctx, const ppst_ct *a, uint32_t level, ppst_ct **out)
{
    CT_OP(drop, { *out = (ppst_ct *)ev_drop(*c, *A, (int)level); })
}

int ppst_prof_start(ppst_ctx *ctx, const char *kernel_class)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    c->prof.on = true;
    c->prof.only = kernel_class ? kernel_class : "";
    return PPST_OK;
}

int ppst_prof_stop(ppst_ctx *ctx)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX)) return PPST_E_ARG;
    c->prof.on = false;
    return PPST_OK;
}

int ppst_prof_read(ppst_ctx *ctx, const char *kernel_class, uint64_t *launches, double *total_ms, uint64_t *units,
                   uint64_t *method_units)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX) || !kernel_class) return PPST_E_ARG;
    return guard(c, [&] {
        PPST_CUDA(cudaStreamSynchronize(c->stream));
        auto it = c->prof.rec.find(kernel_class);
        uint64_t n = 0, u = 0, mu = 0;
        double ms = 0;
        if (it != c->prof.rec.end()) {
            for (auto &pr : it->second) {
                float t = 0;
                PPST_CUDA(cudaEventElapsedTime(&t, pr.b, pr.e));
                ms += t;
                n++;
                u += pr.units;
                mu += pr.munits;
                c->prof.spare.push_back(pr.b);
                c->prof.spare.push_back(pr.e);
            }
            c->prof.rec.erase(it);
        }
        if (launches) *launches = n;
        if (total_ms) *total_ms = ms;
        if (units) *units = u;
        if (method_units) *method_units = mu;
    });
}

int ppst_launch_count(const ppst_ctx *ctx, uint64_t *launches)
{
    const Ctx *c = (const Ctx *)ctx;
    if (!ok(c, TAG_CTX) || !launches) return PPST_E_ARG;
    *launches = c->prof.launches;
    return PPST_OK;
}

int ppst_prof_classes(ppst_ctx *ctx, char *buf, size_t cap)
{
    Ctx *c = (Ctx *)ctx;
    if (!ok(c, TAG_CTX) || !buf || !cap) return PPST_E_ARG;
    std::string s;
    for (auto &kv : c->prof.rec) {
        if (!s.empty()) s += ",";
        s += kv.first;
    }
    std::strncpy(buf, s.c_str(), cap - 1);
    buf[cap - 1] = 0;
    return PPST_OK;
}

void ppst_free(void *handle)
{
    if (!handle) return;
    const uint32_t tag = *(const uint32_t *)handle;
    switch (tag) {
    case TAG_CTX: ctx_destroy((Ctx *)handle); break;
    case TAG_SK: {
        SkObj *s = (SkObj *)handle;
        std::fill(s->s.begin(), s->s.end(), 0);
        s->tag = TAG_DEAD;
        delete s;
        break;
    }
    case TAG_EVK: {
        EvkObj *k = (EvkObj *)handle;
        Ctx &c = *k->ctx;
        const size_t kb = (size_t)c.dnum * 2 * c.np * c.N * 8;
        c.pool.put(k->pk, c.ct_words() * 8);
        c.pool.put(k->relin.d, kb);
        for (auto &kv : k->rot) c.pool.put(kv.second.d, kb);
        k->tag = TAG_DEAD;
        delete k;
        break;
    }
    case TAG_CT: ct_free((CtObj *)handle); break;
    case TAG_COL: {
        ColObj *col = (ColObj *)handle;
        for (CtObj *ct : col->cts) ct_free(ct);
        col->tag = TAG_DEAD;
        delete col;
        break;
    }
    case TAG_RES: {
        ResObj *r = (ResObj *)handle;
        for (CtObj *ct : r->cts) ct_free(ct);
        r->tag = TAG_DEAD;
        delete r;
        break;
    }
    case TAG_SRV: server_destroy((Server *)handle); break;
    case TAG_PLAN: plan_destroy((Plan *)handle); break;
    default: break;
    }
}

}  // extern "C"
