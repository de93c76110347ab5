// stats.cu -- PP-STAT statistic programs over the GPU evaluator.
//
//  * CryptoInvSqrt(v, C) (Sec. 5, Alg. 2 with n = 2, Alg. 3, Eq. 1, Eq. 3):
//    u = v - 1 (Eq. 1); y0 = degree 2^k - 1 Chebyshev interpolant of
//    F(u, C) = 1 / (sqrt(C) sqrt(u + 1)) evaluated at u (Alg. 3 without
//    bootstrapping); then t Newton steps y <- 1.5 y - x' y^3, x' = v C / 2
//    (Alg. 2; the 1/n multiplier carries the constant C of Eq. 3).
//  * CryptoSqrt(v, C) (Eq. 4): the interpolant of sqrt(C) sqrt(u + 1) alone.
//  * Mean(x, B), Variance(x, B) with the 1/B constants folded into the
//    plaintext multipliers (Sec. 6.1, Eq. 2): Variance costs depth 2.
//  * ZNorm (Alg. 4), Kurt (Alg. 5), Skew (third-moment mirror of Alg. 5),
//    CV (Alg. 6 for a positive mean, no Sign), the sign-aware CV (Alg. 6 with
//    Sign(mu) = mu * CryptoInvSqrt(mu^2, B^2)), PCC (Sec. 6.5).
// Where the paper is silent: the Chebyshev sum is evaluated baby-step
// giant-step in the Chebyshev basis (T_2i = 2 T_i^2 - 1, T_2i+1 = 2 T_i T_i+1
// - T_1, giants T_2^m, recursive division by T_n); a leaf sum is one linear
// combination with integer weights round(c_i q_l) and a single rescale, steered
// to a common scale so that all Adds see equal scales; Newton's products are
// associated (x' y)(y y) (depth 2 per step); padding slots of multi-ciphertext
// columns are corrected with integer multiples of mu^p.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <exception>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>

#include "ctx.cuh"

namespace ppst {

namespace {

struct Holder {
    CtObj *ct;
    explicit Holder(CtObj *p) : ct(p) {}
    ~Holder()
    {
        if (ct) ct_free(ct);
    }
    CtObj *release()
    {
        CtObj *p = ct;
        ct = nullptr;
        return p;
    }
};
typedef std::shared_ptr<Holder> H;

// ---------------------------------------------------------------------------
// batch scheduler: the queries of a batch run their statistic programs on host
// threads; each evaluator op is a request. When every live query waits on a
// request, the scheduler thread (the caller's) executes them: HMults at one
// level and rotate-and-sums at one level as batched launches (keys read once
// per batch), the rest one by one. All GPU work is issued by that thread.
// ---------------------------------------------------------------------------
enum ReqKind { R_ADD, R_SUB, R_ADDC, R_MULI, R_MULC, R_LINC, R_HMULT, R_ROTSUM };

struct Req {
    ReqKind kind;
    const CtObj *a = nullptr, *b = nullptr;
    std::vector<const CtObj *> xs;
    std::vector<double> cs;
    double x = 0, target = 0;
    int64_t m = 0;
    CtObj *result = nullptr;
    std::exception_ptr err;
    bool done = false;
    bool last = true;  // last request of one worker's submission
};

// HMults grouped by level, at most 16 per launch sequence; results in input order
std::vector<CtObj *> hmult_grouped(Ctx &c, const EvkObj &k, const std::vector<const CtObj *> &a,
                                   const std::vector<const CtObj *> &b)
{
    std::vector<CtObj *> out(a.size(), nullptr);
    std::map<int, std::vector<size_t>> by;
    for (size_t i = 0; i < a.size(); i++) by[std::min(a[i]->level, b[i]->level)].push_back(i);
    try {
        for (auto &kv : by) {
            const std::vector<size_t> &ix = kv.second;
            for (size_t s = 0; s < ix.size(); s += 16) {
                std::vector<const CtObj *> as, bs;
                for (size_t j = s; j < std::min(s + 16, ix.size()); j++) {
                    as.push_back(a[ix[j]]);
                    bs.push_back(b[ix[j]]);
                }
                std::vector<CtObj *> r = ev_hmult_batch(c, k, as, bs);
                for (size_t j = 0; j < r.size(); j++) out[ix[s + j]] = r[j];
            }
        }
    } catch (...) {
        for (CtObj *x : out)
            if (x) ct_free(x);
        throw;
    }
    return out;
}

struct Sched {
    Ctx &c;
    const EvkObj &k;
    std::mutex mu;
    std::condition_variable cv_sched, cv_work;
    std::vector<Req *> pending;
    int active = 0, waiting = 0;  // live workers; workers blocked on a request
    bool stop = false;
    uint64_t rounds = 0;          // scheduling rounds executed

    CtObj *submit(Req &r)
    {
        std::unique_lock<std::mutex> lk(mu);
        pending.push_back(&r);
        waiting++;
        cv_sched.notify_one();
        cv_work.wait(lk, [&] { return r.done; });
        if (r.err) std::rethrow_exception(r.err);
        return r.result;
    }

    // independent requests of one worker, executed in one round (same-level
    // HMults share launches); the first error is rethrown after all finished
    void submit_many(std::vector<Req> &rs)
    {
        if (rs.empty()) return;
        std::unique_lock<std::mutex> lk(mu);
        for (Req &r : rs) {
            r.last = false;
            pending.push_back(&r);
        }
        rs.back().last = true;
        waiting++;
        cv_sched.notify_one();
        cv_work.wait(lk, [&] { return rs.back().done; });
        for (Req &r : rs)
            if (r.err) std::rethrow_exception(r.err);
    }

    void worker_started()
    {
        std::lock_guard<std::mutex> lk(mu);
        active++;
    }

    void worker_finished()
    {
        std::lock_guard<std::mutex> lk(mu);
        active--;
        cv_sched.notify_one();
    }

    void request_stop()
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
        cv_sched.notify_one();
    }

    // ---- values shared by the queries in flight: a column's rotate-and-sum,
    // its variance for a given B and that variance's inverse square root for
    // given approximation settings are computed by the first query that needs
    // them and reused by the others (the same ops on the same inputs: results
    // are bit-identical to a query run alone) ----
    struct Shared {
        bool ready = false;
        H val;
        std::exception_ptr err;
    };
    typedef std::tuple<const void *, int, double> SKey;
    std::map<SKey, std::shared_ptr<Shared>> shared;
    std::map<const void *, int> col_users;  // queries in flight per column
    std::condition_variable cv_shared;

    void col_acquire(const void *col)
    {
        if (!col) return;
        std::lock_guard<std::mutex> lk(mu);
        col_users[col]++;
    }

    // the last query on a column drops the column's shared values
    void col_release(const void *col)
    {
        if (!col) return;
        std::vector<H> drop;  // freed outside the lock
        {
            std::lock_guard<std::mutex> lk(mu);
            if (--col_users[col] > 0) return;
            col_users.erase(col);
            for (auto it = shared.begin(); it != shared.end();) {
                if (std::get<0>(it->first) == col) {
                    drop.push_back(it->second->val);
                    it = shared.erase(it);
                } else {
                    ++it;
                }
            }
        }
    }

    void exec_one(Req &r)
    {
        switch (r.kind) {
        case R_ADD: r.result = ev_add(c, *r.a, *r.b, false); break;
        case R_SUB: r.result = ev_add(c, *r.a, *r.b, true); break;
        case R_ADDC: r.result = ev_add_const(c, *r.a, r.x); break;
        case R_MULI: r.result = ev_mul_int(c, *r.a, r.m); break;
        case R_MULC: r.result = ev_mul_const(c, *r.a, r.x, r.target); break;
        case R_LINC: r.result = ev_lin_comb(c, r.xs, r.cs, r.target); break;
        case R_HMULT: r.result = ev_hmult(c, k, *r.a, *r.b); break;
        case R_ROTSUM: r.result = ev_rotsum(c, k, *r.a); break;
        }
    }

    void exec_hmults(std::vector<Req *> &rs)
    {
        std::vector<const CtObj *> as, bs;
        for (Req *r : rs) {
            as.push_back(r->a);
            bs.push_back(r->b);
        }
        std::vector<CtObj *> out = hmult_grouped(c, k, as, bs);
        for (size_t i = 0; i < rs.size(); i++) rs[i]->result = out[i];
    }

    // rotate-and-sums grouped by level: step s rotates every member by 2^s in one batch
    void exec_rotsums(std::vector<Req *> &rs)
    {
        std::map<int, std::vector<Req *>> by;
        for (Req *r : rs) by[r->a->level].push_back(r);
        for (auto &kv : by) {
            for (size_t s = 0; s < kv.second.size(); s += 16) {
                std::vector<Req *> g(kv.second.begin() + s, kv.second.begin() + std::min(s + 16, kv.second.size()));
                std::vector<CtObj *> acc;
                for (Req *r : g) acc.push_back(ct_clone(*r->a));
                try {
                    for (int st = 0; st < c.logN - 1; st++) {
                        std::vector<const CtObj *> in(acc.begin(), acc.end());
                        std::vector<CtObj *> rot = ev_rotate_batch(c, k, in, 1 << st);
                        for (size_t i = 0; i < g.size(); i++) {
                            CtObj *sum = nullptr;
                            try {
                                sum = ev_add(c, *acc[i], *rot[i], false);
                            } catch (...) {
                                for (CtObj *x : rot) ct_free(x);
                                throw;
                            }
                            ct_free(acc[i]);
                            acc[i] = sum;
                        }
                        for (CtObj *x : rot) ct_free(x);
                    }
                } catch (...) {
                    for (CtObj *x : acc) ct_free(x);
                    throw;
                }
                for (size_t i = 0; i < g.size(); i++) g[i]->result = acc[i];
            }
        }
    }

    void exec_pending(std::vector<Req *> &batch)
    {
        std::vector<Req *> hm, rsum;
        for (Req *r : batch) {
            if (r->kind == R_HMULT) hm.push_back(r);
            else if (r->kind == R_ROTSUM) rsum.push_back(r);
        }
        auto guarded = [&](std::vector<Req *> &group, auto fn) {
            try {
                fn(group);
            } catch (...) {  // a failed batch: run its members one by one to attribute errors
                for (Req *r : group) {
                    if (r->result) continue;
                    try {
                        exec_one(*r);
                    } catch (...) {
                        r->err = std::current_exception();
                    }
                }
            }
        };
        if (!hm.empty()) guarded(hm, [&](std::vector<Req *> &g) { exec_hmults(g); });
        if (!rsum.empty()) guarded(rsum, [&](std::vector<Req *> &g) { exec_rotsums(g); });
        for (Req *r : batch) {
            if (r->kind == R_HMULT || r->kind == R_ROTSUM) continue;
            try {
                exec_one(*r);
            } catch (...) {
                r->err = std::current_exception();
            }
        }
    }

    // Scheduler loop. A round runs when every live worker waits on a request:
    // workers that join meanwhile (continuous batching) are part of the next
    // round. forever = false: return once no worker is left; forever = true:
    // keep serving until request_stop() with no worker left.
    void run(bool forever)
    {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_sched.wait(lk, [&] {
                return (active > 0 && waiting == active && !pending.empty()) || (active == 0 && (!forever || stop));
            });
            if (active == 0) return;
            std::vector<Req *> batch;
            batch.swap(pending);
            lk.unlock();
            {
                std::lock_guard<std::recursive_mutex> g(c.exec_mu);
                exec_pending(batch);
            }
            lk.lock();
            rounds++;
            for (Req *r : batch) {
                r->done = true;
                waiting -= r->last ? 1 : 0;
            }
            cv_work.notify_all();
        }
    }
};

struct Ev {
    Ctx &c;
    const EvkObj &k;
    Sched *sched = nullptr;  // batched mode: ops go through the scheduler
    H w(CtObj *p) { return std::make_shared<Holder>(p); }
    int level(const H &a) const { return a->ct->level; }
    double scale(const H &a) const { return a->ct->scale; }
    uint64_t prime(int l) const { return c.primes[l]; }
    H req(Req &r) { return w(sched->submit(r)); }
    H add(const H &a, const H &b)
    {
        if (!sched) return w(ev_add(c, *a->ct, *b->ct, false));
        Req r{R_ADD};
        r.a = a->ct;
        r.b = b->ct;
        return req(r);
    }
    H sub(const H &a, const H &b)
    {
        if (!sched) return w(ev_add(c, *a->ct, *b->ct, true));
        Req r{R_SUB};
        r.a = a->ct;
        r.b = b->ct;
        return req(r);
    }
    H add_const(const H &a, double x)
    {
        if (!sched) return w(ev_add_const(c, *a->ct, x));
        Req r{R_ADDC};
        r.a = a->ct;
        r.x = x;
        return req(r);
    }
    H mul_int(const H &a, int64_t m)
    {
        if (!sched) return w(ev_mul_int(c, *a->ct, m));
        Req r{R_MULI};
        r.a = a->ct;
        r.m = m;
        return req(r);
    }
    H mul_const(const H &a, double x, double target = 0)
    {
        if (!sched) return w(ev_mul_const(c, *a->ct, x, target));
        Req r{R_MULC};
        r.a = a->ct;
        r.x = x;
        r.target = target;
        return req(r);
    }
    H hmult(const H &a, const H &b)
    {
        if (!sched) return w(ev_hmult(c, k, *a->ct, *b->ct));
        Req r{R_HMULT};
        r.a = a->ct;
        r.b = b->ct;
        return req(r);
    }
    H lin_comb(const std::vector<H> &xs, const std::vector<double> &cs, double target)
    {
        std::vector<const CtObj *> p;
        for (const H &x : xs) p.push_back(x->ct);
        if (!sched) return w(ev_lin_comb(c, p, cs, target));
        Req r{R_LINC};
        r.xs = p;
        r.cs = cs;
        r.target = target;
        return req(r);
    }
    // ---- independent ops over the ciphertexts of a column: one scheduling round ----
    std::vector<H> run_many(std::vector<Req> &rs)
    {
        sched->submit_many(rs);
        std::vector<H> out;
        for (Req &r : rs) out.push_back(w(r.result));
        return out;
    }
    std::vector<H> sub_v(const std::vector<H> &a, const H &b)
    {
        std::vector<H> out;
        if (!sched) {
            for (const H &x : a) out.push_back(sub(x, b));
            return out;
        }
        std::vector<Req> rs(a.size(), Req{R_SUB});
        for (size_t i = 0; i < a.size(); i++) {
            rs[i].a = a[i]->ct;
            rs[i].b = b->ct;
        }
        return run_many(rs);
    }
    std::vector<H> mul_const_v(const std::vector<H> &a, double x)
    {
        std::vector<H> out;
        if (!sched) {
            for (const H &y : a) out.push_back(mul_const(y, x));
            return out;
        }
        std::vector<Req> rs(a.size(), Req{R_MULC});
        for (size_t i = 0; i < a.size(); i++) {
            rs[i].a = a[i]->ct;
            rs[i].x = x;
        }
        return run_many(rs);
    }
    // elementwise products a[i] * b[i] (b of size 1: broadcast)
    std::vector<H> hmult_v(const std::vector<H> &a, const std::vector<H> &b)
    {
        auto rhs = [&](size_t i) { return b.size() == 1 ? b[0] : b[i]; };
        std::vector<H> out;
        if (a.size() == 1) {
            out.push_back(hmult(a[0], rhs(0)));
            return out;
        }
        if (!sched) {
            std::vector<const CtObj *> as, bs;
            for (size_t i = 0; i < a.size(); i++) {
                as.push_back(a[i]->ct);
                bs.push_back(rhs(i)->ct);
            }
            for (CtObj *p : hmult_grouped(c, k, as, bs)) out.push_back(w(p));
            return out;
        }
        std::vector<Req> rs(a.size(), Req{R_HMULT});
        for (size_t i = 0; i < a.size(); i++) {
            rs[i].a = a[i]->ct;
            rs[i].b = rhs(i)->ct;
        }
        return run_many(rs);
    }
    H sum(const std::vector<H> &x)
    {
        H acc = x[0];
        for (size_t i = 1; i < x.size(); i++) acc = add(acc, x[i]);
        return acc;
    }

    // a value shared with the other queries in flight (see Sched::Shared); a
    // query that finds it being computed waits without holding up the rounds
    template <class F>
    H shared_value(const void *col, int kind, double b, F &&compute)
    {
        if (!sched || !col) return compute();
        const Sched::SKey key{col, kind, b};
        std::shared_ptr<Sched::Shared> e;
        bool mine = false;
        {
            std::lock_guard<std::mutex> lk(sched->mu);
            std::shared_ptr<Sched::Shared> &slot = sched->shared[key];
            if (!slot) {
                slot = std::make_shared<Sched::Shared>();
                mine = true;
            }
            e = slot;
        }
        if (mine) {
            try {
                H v = compute();
                {
                    std::lock_guard<std::mutex> lk(sched->mu);
                    e->val = v;
                    e->ready = true;
                }
                sched->cv_shared.notify_all();
                return v;
            } catch (...) {
                {
                    std::lock_guard<std::mutex> lk(sched->mu);
                    e->err = std::current_exception();
                    e->ready = true;
                    sched->shared.erase(key);  // a later query computes it afresh
                }
                sched->cv_shared.notify_all();
                throw;
            }
        }
        {
            std::unique_lock<std::mutex> lk(sched->mu);
            if (!e->ready) {
                sched->waiting++;  // parked: the rounds go on without this worker
                sched->cv_sched.notify_one();
                sched->cv_shared.wait(lk, [&] { return e->ready; });
                sched->waiting--;
            }
        }
        if (e->err) std::rethrow_exception(e->err);
        return e->val;
    }

    // a level view: no GPU work, safe on any thread
    H drop(const H &a, int l) { return l == a->ct->level ? a : w(ev_drop(c, *a->ct, l)); }
    H rotsum(const H &a)
    {
        if (!sched) return w(ev_rotsum(c, k, *a->ct));
        Req r{R_ROTSUM};
        r.a = a->ct;
        return req(r);
    }
};

// ---- Chebyshev interpolation (Sec. 3.4, Eq. 1, 3, 4) ----
std::vector<double> cheb_coeffs(const std::function<double(double)> &F, int d)
{
    const int n = d + 1;
    std::vector<double> th(n), f(n), c(n);
    for (int j = 0; j < n; j++) th[j] = M_PI * (j + 0.5) / n;
    for (int j = 0; j < n; j++) f[j] = F(std::cos(th[j]));
    for (int k = 0; k < n; k++) {
        double s = 0.0;
        for (int j = 0; j < n; j++) s += f[j] * std::cos(k * th[j]);
        c[k] = 2.0 * s / n;
    }
    c[0] *= 0.5;
    return c;
}

std::function<double(double)> inv_sqrt_target(double C)
{
    return [C](double u) { return u > -1.0 ? 1.0 / (std::sqrt(C) * std::sqrt(u + 1.0)) : 0.0; };
}

std::function<double(double)> sqrt_target(double C)
{
    return [C](double u) { return u >= -1.0 ? std::sqrt(C) * std::sqrt(u + 1.0) : 0.0; };
}

// p = q T_n + r: q_0 = c_n, q_i = 2 c_{n+i}; r_0 = c_0, r_i = c_i - c_{2n-i}
void cheb_split(const std::vector<double> &c, std::vector<double> &q, std::vector<double> &r)
{
    const size_t n = c.size() / 2;
    q.assign(n, 0.0);
    r.assign(n, 0.0);
    q[0] = c[n];
    r[0] = c[0];
    for (size_t i = 1; i < n; i++) {
        q[i] = 2.0 * c[n + i];
        r[i] = c[i] - c[2 * n - i];
    }
}

struct Cheb {
    Ev &ev;
    std::map<int, H> T;
    int baby;

    int rec_level(int len)
    {
        if (len <= baby) {
            int lv = 1 << 30;
            for (int i = 1; i < len; i++) lv = std::min(lv, ev.level(T[i]));
            return lv - 1;
        }
        const int n = len / 2;
        const int lq = std::min(rec_level(n), ev.level(T[n])) - 1;
        return std::min(lq, rec_level(n));
    }

    H rec(const std::vector<double> &c, double target)
    {
        const int len = (int)c.size();
        if (len <= baby) {
            int lv = 1 << 30;
            for (int i = 1; i < len; i++) lv = std::min(lv, ev.level(T[i]));
            std::vector<H> terms;
            for (int i = 1; i < len; i++) terms.push_back(ev.drop(T[i], lv));
            H acc = ev.lin_comb(terms, std::vector<double>(c.begin() + 1, c.end()), target);
            return ev.add_const(acc, c[0]);
        }
        const int n = len / 2;
        std::vector<double> q, r;
        cheb_split(c, q, r);
        const int lvl = std::min(rec_level(n), ev.level(T[n]));
        const double tq = target * (double)ev.prime(lvl) / ev.scale(T[n]);
        H prod = ev.hmult(rec(q, tq), T[n]);
        H rest = rec(r, ev.scale(prod));
        return ev.add(prod, rest);
    }
};

H cheb_eval(Ev &ev, const H &u, const std::vector<double> &c)
{
    int k = 0;
    while ((1u << k) < c.size()) k++;
    if ((1u << k) != c.size() || k < 1) throw_err(PPST_E_ARG, "Chebyshev length must be a power of two");
    const int b = (k + 1) / 2;
    Cheb ch{ev, {}, 1 << b};
    ch.T[1] = u;
    for (int i = 2; i <= (1 << b); i++) {
        if (i % 2 == 0) {
            const H &h = ch.T[i / 2];
            ch.T[i] = ev.add_const(ev.mul_int(ev.hmult(h, h), 2), -1.0);
        } else {
            H p = ev.mul_int(ev.hmult(ch.T[(i - 1) / 2], ch.T[(i + 1) / 2]), 2);
            H t1 = ev.mul_const(ev.drop(ch.T[1], ev.level(p) + 1), 1.0, ev.scale(p));
            ch.T[i] = ev.sub(p, t1);
        }
    }
    for (int m = b + 1; m < k; m++) {
        const H &h = ch.T[1 << (m - 1)];
        ch.T[1 << m] = ev.add_const(ev.mul_int(ev.hmult(h, h), 2), -1.0);
    }
    return ch.rec(c, ev.c.scale);
}

H crypto_inv_sqrt(Ev &ev, const H &v, double C, int k, int t)
{
    const std::vector<double> c = cheb_coeffs(inv_sqrt_target(C), (1 << k) - 1);
    H y = cheb_eval(ev, ev.add_const(v, -1.0), c);
    H xh = ev.mul_const(v, C / 2.0);
    for (int it = 0; it < t; it++) {
        H y2 = ev.hmult(y, y);
        H xy = ev.hmult(xh, y);
        H b = ev.hmult(xy, y2);
        H a = ev.mul_const(ev.drop(y, ev.level(b) + 1), 1.5, ev.scale(b));
        y = ev.sub(a, b);
    }
    return y;
}

H crypto_sqrt(Ev &ev, const H &v, double C, int k)
{
    return cheb_eval(ev, ev.add_const(v, -1.0), cheb_coeffs(sqrt_target(C), (1 << k) - 1));
}

typedef std::vector<H> Col;

H col_sum(Ev &ev, const Col &x)
{
    H acc = x[0];
    for (size_t i = 1; i < x.size(); i++) acc = ev.add(acc, x[i]);
    return acc;
}

H variance(Ev &ev, const Col &x, size_t n, double B, const H &R)
{
    const double cst = 1.0 / (B * std::sqrt((double)n));
    const Col y = ev.mul_const_v(x, cst);
    H a = ev.rotsum(ev.sum(ev.hmult_v(y, y)));
    H m = ev.mul_const(R, 1.0 / (B * (double)n));
    return ev.sub(a, ev.hmult(m, m));
}

// rotsum of the column's entries: Mean's sum (Sec. 6.1), shared per column
H col_rsum(Ev &ev, const Col &x, const void *kx)
{
    return ev.shared_value(kx, 0, 0.0, [&] { return ev.rotsum(col_sum(ev, x)); });
}

// Variance(x, B) (Eq. 2), shared per column and B
H col_var(Ev &ev, const Col &x, size_t n, double B, const H &R, const void *kx)
{
    return ev.shared_value(kx, 1, B, [&] { return variance(ev, x, n, B, R); });
}

// CryptoInvSqrt(Variance(x, B), B^2) (Sec. 5, Eq. 3): 1 / sqrt(Var), shared per column,
// B and approximation settings (Z-score, skewness, kurtosis and PCC all start from it)
H col_inv_sd(Ev &ev, const Col &x, size_t n, double B, const H &R, const void *kx, int k, int t)
{
    return ev.shared_value(kx, 2 | (k << 8) | (t << 16), B,
                           [&] { return crypto_inv_sqrt(ev, col_var(ev, x, n, B, R, kx), B * B, k, t); });
}

// sum over the column's ciphertexts of (x - mu)^power, slot by slot (not yet reduced)
H centred_power_terms(Ev &ev, const Col &x, const H &mu, int power)
{
    const Col x1 = ev.sub_v(x, mu);
    const Col x2 = ev.hmult_v(x1, x1);
    return ev.sum(ev.hmult_v(x2, power == 4 ? x2 : x1));
}

// rotate-and-sum of a after dropping it to `level` (never above its own): a sum
// consumed only by a product many levels lower is reduced at that level, so its
// rotations switch keys over fewer limbs (Sec. 6.1 leaves the level open)
H rotsum_at(Ev &ev, const H &a, int level) { return ev.rotsum(ev.drop(a, std::min(level, ev.level(a)))); }

Col znorm(Ev &ev, const Col &x, size_t n, double B, int k, int t, const void *kx)
{
    H R = col_rsum(ev, x, kx);
    H mu = ev.mul_const(R, 1.0 / (double)n);
    H inv = col_inv_sd(ev, x, n, B, R, kx, k, t);
    return ev.hmult_v(ev.sub_v(x, mu), Col{inv});
}

H kurt(Ev &ev, const Col &x, size_t n, double B, int k, int t, const void *kx)
{
    H R = col_rsum(ev, x, kx);
    H mu = ev.mul_const(R, 1.0 / (double)n);
    H S4 = centred_power_terms(ev, x, mu, 4);
    H inv = col_inv_sd(ev, x, n, B, R, kx, k, t);
    H inv2 = ev.hmult(inv, inv);
    H inv4 = ev.hmult(inv2, inv2);
    H X = rotsum_at(ev, S4, ev.level(inv4) + 1);
    const int64_t pads = (int64_t)(x.size() * (size_t)ev.c.S) - (int64_t)n;
    if (pads) {
        H mu2 = ev.hmult(mu, mu);
        X = ev.sub(X, ev.mul_int(ev.hmult(mu2, mu2), pads));
    }
    H num = ev.mul_const(X, 1.0 / (double)n);
    return ev.hmult(num, inv4);
}

H skew(Ev &ev, const Col &x, size_t n, double B, int k, int t, const void *kx)
{
    H R = col_rsum(ev, x, kx);
    H mu = ev.mul_const(R, 1.0 / (double)n);
    H S3 = centred_power_terms(ev, x, mu, 3);
    H inv = col_inv_sd(ev, x, n, B, R, kx, k, t);
    H inv3 = ev.hmult(ev.hmult(inv, inv), inv);
    H X = rotsum_at(ev, S3, ev.level(inv3) + 1);
    const int64_t pads = (int64_t)(x.size() * (size_t)ev.c.S) - (int64_t)n;
    if (pads) {
        H mu2 = ev.hmult(mu, mu);
        X = ev.add(X, ev.mul_int(ev.hmult(mu2, mu), pads));
    }
    H num = ev.mul_const(X, 1.0 / (double)n);
    return ev.hmult(num, inv3);
}

H cv(Ev &ev, const Col &x, size_t n, double B, int k, int t, const void *kx)
{
    H R = col_rsum(ev, x, kx);
    H muB = ev.mul_const(R, 1.0 / (B * (double)n));
    H isq = crypto_inv_sqrt(ev, muB, B, k, t);
    H mu_inv = ev.hmult(isq, isq);
    H std_ = crypto_sqrt(ev, col_var(ev, x, n, B, R, kx), B * B, k);
    return ev.hmult(std_, mu_inv);
}

// Alg. 6 with Sign, for a mean of either sign: Sign(mu) = mu * CryptoInvSqrt(mu^2, B^2)
// (sign(x) = x / sqrt(x^2)), and the inverse of the sign-corrected mean,
// CryptoInvSqrt(mu sign(mu), B)^2 = 1 / |mu|, is that same inverse root; the lines
// keep Alg. 6's order: tmp = Std * mu_inv, CV = tmp * sign. One level more than cv.
H cv_signed(Ev &ev, const Col &x, size_t n, double B, int k, int t, const void *kx)
{
    H R = col_rsum(ev, x, kx);
    H mu = ev.mul_const(R, 1.0 / (double)n);
    H muB = ev.mul_const(R, 1.0 / (B * (double)n));
    H mu_inv = crypto_inv_sqrt(ev, ev.hmult(muB, muB), B * B, k, t);  // 1 / |mu|
    H sign = ev.hmult(mu, mu_inv);
    H std_ = crypto_sqrt(ev, col_var(ev, x, n, B, R, kx), B * B, k);
    return ev.hmult(ev.hmult(std_, mu_inv), sign);
}

H pcc(Ev &ev, const Col &x, const Col &y, size_t n, double Bx, double By, int k, int t, const void *kx,
      const void *ky)
{
    H Rx = col_rsum(ev, x, kx);
    H Ry = col_rsum(ev, y, ky);
    H mux = ev.mul_const(Rx, 1.0 / (double)n);
    H muy = ev.mul_const(Ry, 1.0 / (double)n);
    H P = ev.sum(ev.hmult_v(ev.sub_v(x, mux), ev.sub_v(y, muy)));
    H ix = col_inv_sd(ev, x, n, Bx, Rx, kx, k, t);
    H iy = col_inv_sd(ev, y, n, By, Ry, ky, k, t);
    H Cs = rotsum_at(ev, P, std::min(ev.level(ix), ev.level(iy)) + 1);
    const int64_t pads = (int64_t)(x.size() * (size_t)ev.c.S) - (int64_t)n;
    if (pads) Cs = ev.sub(Cs, ev.mul_int(ev.hmult(mux, muy), pads));
    H cov = ev.mul_const(Cs, 1.0 / (double)n);
    return ev.hmult(ev.hmult(cov, ix), iy);
}

// non-owning handles around a column's ciphertexts
Col view(const ColObj &col)
{
    Col out;
    for (CtObj *ct : col.cts) {
        auto h = std::shared_ptr<Holder>(new Holder(ct), [](Holder *p) {
            p->ct = nullptr;  // the column keeps ownership
            delete p;
        });
        out.push_back(h);
    }
    return out;
}

ResObj *run_one(Ev &ev, const QueryIn &q)
{
    const int kk = q.o.cheb_log2deg, tt = q.o.newton_steps;
    Col x = view(*q.x);
    const size_t n = q.x->n;
    Col res;
    switch (q.stat) {
    case PPST_ZSCORE: res = znorm(ev, x, n, q.o.B_x, kk, tt, q.x); break;
    case PPST_KURT: res.push_back(kurt(ev, x, n, q.o.B_x, kk, tt, q.x)); break;
    case PPST_SKEW: res.push_back(skew(ev, x, n, q.o.B_x, kk, tt, q.x)); break;
    case PPST_CV: res.push_back(cv(ev, x, n, q.o.B_x, kk, tt, q.x)); break;
    case PPST_CV_SIGNED: res.push_back(cv_signed(ev, x, n, q.o.B_x, kk, tt, q.x)); break;
    case PPST_PCC: res.push_back(pcc(ev, x, view(*q.y), n, q.o.B_x, q.o.B_y, kk, tt, q.x, q.y)); break;
    default: throw_err(PPST_E_ARG, "unknown statistic");
    }
    ResObj *r = new ResObj();
    r->ctx = &ev.c;
    r->stat = q.stat;
    r->n = n;
    r->level_in = q.x->cts[0]->level;
    for (H &h : res) r->cts.push_back(h->release());
    return r;
}

void free_res(ResObj *r)
{
    if (!r) return;
    for (CtObj *ct : r->cts) ct_free(ct);
    delete r;
}

}  // namespace

CtObj *ev_inv_sqrt(Ctx &c, const EvkObj &k, const CtObj &v, double C, int cheb_log2deg, int newton_steps)
{
    Ev ev{c, k};
    H in(new Holder(const_cast<CtObj *>(&v)), [](Holder *p) {
        p->ct = nullptr;  // the caller keeps the input
        delete p;
    });
    H r = crypto_inv_sqrt(ev, in, C, cheb_log2deg, newton_steps);
    if (r == in) return ct_clone(v);
    return r->release();
}

void run_queries(Ctx &c, const EvkObj &k, const std::vector<QueryIn> &qs, std::vector<ResObj *> &out)
{
    if (qs.size() <= 1) {
        Ev ev{c, k};
        for (const QueryIn &q : qs) out.push_back(run_one(ev, q));
        return;
    }
    Sched sched{c, k};
    std::vector<ResObj *> res(qs.size(), nullptr);
    std::vector<std::exception_ptr> errs(qs.size());
    std::vector<std::thread> th;
    for (size_t i = 0; i < qs.size(); i++) {
        sched.worker_started();
        sched.col_acquire(qs[i].x);
        sched.col_acquire(qs[i].y);
    }
    for (size_t i = 0; i < qs.size(); i++) {
        th.emplace_back([&, i] {
            try {
                Ev ev{c, k, &sched};
                res[i] = run_one(ev, qs[i]);
            } catch (...) {
                errs[i] = std::current_exception();
            }
            sched.col_release(qs[i].x);
            sched.col_release(qs[i].y);
            sched.worker_finished();
        });
    }
    sched.run(false);
    for (std::thread &t : th) t.join();
    for (size_t i = 0; i < qs.size(); i++) {
        if (errs[i]) {
            for (ResObj *r : res) free_res(r);
            std::rethrow_exception(errs[i]);
        }
    }
    for (ResObj *r : res) out.push_back(r);
}

// ---------------------------------------------------------------------------
// serving: continuous batching over the same scheduler
// ---------------------------------------------------------------------------
// A scheduler thread runs rounds forever; an admitted query gets a worker
// thread that joins the next round (so requests that arrive while others run
// are batched with them at op boundaries). Admission: at most max_batch
// queries at once, and the sum of their working-set estimates within the HBM
// budget. A query's estimate: (its ciphertexts + 40) full-size ciphertext
// buffers (the deepest statistic keeps about 40 temporaries alive) plus one
// item of key-switch workspace. Completion is marked when a CUDA event
// recorded after the query's last op has completed (stream order).
struct Server {
    uint32_t tag = TAG_SRV;
    Ctx *c;
    const EvkObj *k;
    size_t budget;
    uint32_t max_batch;
    Sched sched;
    struct Ticket {
        QueryIn q;
        size_t est = 0, res_bytes = 0;  // working-set estimate; result ciphertexts held until ppst_wait
        std::chrono::steady_clock::time_point t_submit, t_ready;
        ResObj *res = nullptr;
        std::exception_ptr err;
        cudaEvent_t ev = nullptr;
        bool ready = false, taken = false;
    };
    std::mutex mu;
    std::condition_variable cv_done, cv_compl, cv_idle;
    std::map<uint64_t, std::shared_ptr<Ticket>> tickets;
    std::deque<std::shared_ptr<Ticket>> queue, compl_q;
    size_t reserved = 0;  // working sets of the queries running
    size_t held = 0;      // results finished but not yet handed over by ppst_wait
    uint32_t running = 0;
    // a query that does not fit may be passed by later ones that do, until it has
    // waited this long; from then on nothing passes it
    std::chrono::milliseconds bypass_limit{500};
    uint64_t next_id = 1;
    bool stopping = false;
    std::thread sched_thread, compl_thread;

    Server(Ctx &cc, const EvkObj &kk, size_t b, uint32_t mb) : c(&cc), k(&kk), budget(b), max_batch(mb), sched{cc, kk}
    {
        sched_thread = std::thread([this] { sched.run(true); });
        compl_thread = std::thread([this] { completion_loop(); });
    }

    size_t estimate(const QueryIn &q) const
    {
        const size_t ct_bytes = c->ct_words() * 8;
        const size_t q1 = c->L + 1, e = c->ext_rows();
        const size_t ws_item = (4 * q1 + (size_t)c->dnum * e + 2 * e + 2) * c->N * 8;
        const size_t n = q.x->cts.size() + (q.y ? q.y->cts.size() : 0);
        return (n + 40) * ct_bytes + ws_item;
    }

    // bytes of a query's result ciphertexts (Z-score: one per input ciphertext)
    size_t result_bytes(const QueryIn &q) const
    {
        return (q.stat == PPST_ZSCORE ? q.x->cts.size() : 1) * c->ct_words() * 8;
    }

    // under mu: admit, in arrival order, every queued query that fits the budget
    // next to the running ones and the results not yet taken; a query that does
    // not fit is passed only until it has waited bypass_limit
    void try_admit()
    {
        const auto now = std::chrono::steady_clock::now();
        for (auto it = queue.begin(); it != queue.end() && running < max_batch;) {
            std::shared_ptr<Ticket> t = *it;
            if (reserved + held + t->est + t->res_bytes > budget) {
                if (now - t->t_submit >= bypass_limit) break;  // it is next; nothing passes it now
                ++it;
                continue;
            }
            it = queue.erase(it);
            reserved += t->est;
            running++;
            sched.worker_started();
            sched.col_acquire(t->q.x);
            sched.col_acquire(t->q.y);
            std::thread([this, t] { work(t); }).detach();
        }
    }

    void work(std::shared_ptr<Ticket> t)
    {
        try {
            Ev ev{*c, *k, &sched};
            t->res = run_one(ev, t->q);
        } catch (...) {
            t->err = std::current_exception();
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) cudaEventRecord(e, c->stream);
        t->ev = e;
        // leave the scheduler before `running` drops: the destructor tears the
        // scheduler down as soon as no worker runs
        sched.col_release(t->q.x);
        sched.col_release(t->q.y);
        sched.worker_finished();
        std::lock_guard<std::mutex> lk(mu);
        compl_q.push_back(t);
        reserved -= t->est;
        if (!t->err) held += t->res_bytes;  // until ppst_wait hands the result over
        else t->res_bytes = 0;
        running--;
        try_admit();
        cv_compl.notify_one();
        cv_idle.notify_all();
    }

    void completion_loop()
    {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_compl.wait(lk, [&] { return !compl_q.empty() || (stopping && running == 0 && queue.empty()); });
            if (compl_q.empty()) return;
            std::shared_ptr<Ticket> t = compl_q.front();
            compl_q.pop_front();
            lk.unlock();
            if (t->ev) {
                cudaEventSynchronize(t->ev);
                cudaEventDestroy(t->ev);
                t->ev = nullptr;
            }
            if (!t->err) {
                try {
                    check_device_error(*c);
                } catch (...) {
                    t->err = std::current_exception();
                }
            }
            lk.lock();
            t->t_ready = std::chrono::steady_clock::now();
            t->ready = true;
            cv_done.notify_all();
        }
    }

    uint64_t submit(const QueryIn &q)
    {
        auto t = std::make_shared<Ticket>();
        t->q = q;
        t->est = estimate(q);
        t->res_bytes = result_bytes(q);
        if (t->est + t->res_bytes > budget) throw_err(PPST_E_BUDGET, "the query's working set exceeds the HBM budget");
        std::lock_guard<std::mutex> lk(mu);
        if (stopping) throw_err(PPST_E_STATE, "server is shutting down");
        t->t_submit = std::chrono::steady_clock::now();
        const uint64_t id = next_id++;
        tickets[id] = t;
        queue.push_back(t);
        try_admit();
        return id;
    }

    int wait(uint64_t id, int timeout_ms, ResObj **out)
    {
        std::unique_lock<std::mutex> lk(mu);
        auto it = tickets.find(id);
        if (it == tickets.end()) throw_err(PPST_E_ARG, "unknown ticket");
        std::shared_ptr<Ticket> t = it->second;
        if (t->taken) throw_err(PPST_E_STATE, "result already taken");
        auto pred = [&] { return t->ready; };
        if (timeout_ms < 0) cv_done.wait(lk, pred);
        else if (!cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return PPST_E_TIMEOUT;
        t->taken = true;
        held -= t->res_bytes;  // the caller owns the result now
        t->res_bytes = 0;
        try_admit();
        if (t->err) std::rethrow_exception(t->err);
        *out = t->res;
        t->res = nullptr;
        return PPST_OK;
    }

    void info(ppst_server_stats &o)
    {
        std::lock_guard<std::mutex> lk(mu);
        o.budget = budget;
        o.reserved = reserved;
        o.held = held;
        o.running = running;
        o.queued = (uint32_t)queue.size();
    }

    double latency(uint64_t id)
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = tickets.find(id);
        if (it == tickets.end() || !it->second->ready) throw_err(PPST_E_STATE, "ticket not finished");
        return std::chrono::duration<double>(it->second->t_ready - it->second->t_submit).count();
    }

    ~Server()
    {
        {
            std::unique_lock<std::mutex> lk(mu);
            stopping = true;
            cv_idle.wait(lk, [&] { return running == 0 && queue.empty(); });
            cv_compl.notify_one();
        }
        sched.request_stop();
        sched_thread.join();
        compl_thread.join();
        for (auto &kv : tickets)
            if (kv.second->res) free_res(kv.second->res);
        tag = TAG_DEAD;
    }
};

void server_destroy(Server *s) { delete s; }

// ---------------------------------------------------------------------------
// prepared queries: one statistic program captured as a CUDA graph
// ---------------------------------------------------------------------------
// The program runs once for real with a private key-switch workspace (which
// sizes it and leaves every buffer the program uses in the pool's free lists),
// then once more under stream capture with allocation frozen, so that it takes
// exactly the same buffers. Afterwards the buffers the graph wrote are taken
// out of circulation and kept by the plan together with the workspace and the
// captured result; a replay is one graph launch followed by a copy of the
// result into fresh ciphertexts. The plan keeps its input columns' device
// buffers alive.
struct WsState {
    uint64_t *d2 = nullptr, *d2n = nullptr, *ext = nullptr, *acc = nullptr, *conv = nullptr, *top = nullptr;
    int items = 0;
    size_t bytes = 0;
};

static WsState ws_swap(Ctx &c, const WsState &in)
{
    WsState out{c.ws_d2, c.ws_d2n, c.ws_ext, c.ws_acc, c.ws_conv, c.ws_top, c.ws_items, c.ws_bytes};
    c.ws_d2 = in.d2;
    c.ws_d2n = in.d2n;
    c.ws_ext = in.ext;
    c.ws_acc = in.acc;
    c.ws_conv = in.conv;
    c.ws_top = in.top;
    c.ws_items = in.items;
    c.ws_bytes = in.bytes;
    return out;
}

static void ws_release(Ctx &c, const WsState &w)
{
    if (!w.d2) return;
    const size_t N = c.N, q = c.L + 1, e = c.ext_rows(), B = (size_t)w.items;
    c.pool.put(w.d2, B * q * N * 8);
    c.pool.put(w.d2n, B * q * N * 8);
    c.pool.put(w.ext, B * c.dnum * e * N * 8);
    c.pool.put(w.acc, B * 2 * e * N * 8);
    c.pool.put(w.conv, B * 2 * q * N * 8);
    c.pool.put(w.top, B * 2 * N * 8);
}

struct Plan {
    uint32_t tag = TAG_PLAN;
    Ctx *c = nullptr;
    std::vector<std::shared_ptr<uint64_t>> inputs;
    WsState ws;
    ResObj *res = nullptr;
    std::vector<std::pair<void *, size_t>> retained;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;  // kernels per replay

    ~Plan()
    {
        if (!c) return;
        cudaStreamSynchronize(c->stream);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        free_res(res);
        for (auto &b : retained) c->pool.put(b.first, b.second);
        ws_release(*c, ws);
        tag = TAG_DEAD;
    }
};

static CtObj *ct_copy(Ctx &c, const CtObj &a)
{
    CtObj *o = ct_new(c, a.level, a.scale);
    const size_t words = (size_t)(a.level + 1) * c.N, ps = (size_t)(c.L + 1) * c.N;
    k_copy(c, o->d, a.d, words);
    k_copy(c, o->d + ps, a.d + ps, words);
    return o;
}

Plan *plan_create(Ctx &c, const EvkObj &k, const QueryIn &q)
{
    std::unique_ptr<Plan> pl(new Plan());
    pl->c = &c;
    for (const CtObj *ct : q.x->cts) pl->inputs.push_back(ct->buf);
    if (q.y)
        for (const CtObj *ct : q.y->cts) pl->inputs.push_back(ct->buf);
    const bool prof_on = c.prof.on;
    const cudaStream_t s0 = c.stream;
    WsState user = ws_swap(c, WsState{});  // the program gets a workspace of its own
    auto restore = [&] {
        c.pool.recording = c.pool.frozen = false;
        c.pool.ledger.clear();
        c.stream = s0;
        c.prof.on = prof_on;
        pl->ws = ws_swap(c, user);
    };
    try {
        c.prof.on = false;
        {
            Ev ev{c, k};
            free_res(run_one(ev, q));
        }
        PPST_CUDA(cudaStreamSynchronize(s0));  // the warm-up's buffers are idle before the capture
        PPST_CUDA(cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking));
        c.stream = pl->cap;
        c.pool.ledger.clear();
        c.pool.recording = c.pool.frozen = true;
        const uint64_t l0 = c.prof.launches;  // captured launches do not run: not counted
        PPST_CUDA(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal));
        ResObj *r = nullptr;
        std::exception_ptr err;
        try {
            Ev ev{c, k};
            r = run_one(ev, q);
        } catch (...) {
            err = std::current_exception();
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(pl->cap, &g);
        c.prof.launches = l0;
        pl->graph = g;
        pl->res = r;
        if (err) std::rethrow_exception(err);
        if (ce != cudaSuccess || !g) throw_err(PPST_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        PPST_CUDA(cudaGraphInstantiate(&pl->exec, g, 0));
        size_t nodes = 0;
        PPST_CUDA(cudaGraphGetNodes(g, nullptr, &nodes));  // kernel nodes only: the program copies nothing
        pl->launches = nodes;
        // the intermediates the graph wrote stay with it (each buffer once)
        std::vector<std::pair<void *, size_t>> led = c.pool.ledger;
        std::sort(led.begin(), led.end());
        led.erase(std::unique(led.begin(), led.end()), led.end());
        for (auto &b : led)
            if (c.pool.withdraw(b.first, b.second)) pl->retained.push_back(b);
        restore();
    } catch (...) {
        cudaGetLastError();
        restore();
        throw;
    }
    return pl.release();
}

ResObj *plan_run(Plan &pl)
{
    Ctx &c = *pl.c;
    PPST_CUDA(cudaGraphLaunch(pl.exec, c.stream));
    c.prof.launches += pl.launches;
    std::unique_ptr<ResObj> out(new ResObj());
    out->ctx = &c;
    out->stat = pl.res->stat;
    out->n = pl.res->n;
    out->level_in = pl.res->level_in;
    try {
        for (const CtObj *ct : pl.res->cts) out->cts.push_back(ct_copy(c, *ct));
    } catch (...) {
        for (CtObj *ct : out->cts) ct_free(ct);
        throw;
    }
    return out.release();
}

void plan_destroy(Plan *p) { delete p; }

}  // namespace ppst

using namespace ppst;

extern "C" {

int ppst_server_create(ppst_ctx *ctx, const ppst_evk *evk, size_t hbm_budget, uint32_t max_batch, ppst_server **out)
{
    Ctx *c = (Ctx *)ctx;
    const EvkObj *k = (const EvkObj *)evk;
    if (!out) return PPST_E_ARG;
    *out = nullptr;
    if (!c || c->tag != TAG_CTX || !k || k->tag != TAG_EVK || k->ctx != c || max_batch < 1) return PPST_E_ARG;
    try {
        if (hbm_budget == 0) {  // what the device has free now (keys and columns are resident already)
            std::lock_guard<std::recursive_mutex> lk(c->exec_mu);
            size_t free_b = 0, total_b = 0;
            PPST_CUDA(cudaMemGetInfo(&free_b, &total_b));
            size_t in_use = 0, cached = 0;
            {
                std::lock_guard<std::recursive_mutex> pl(c->pool.mu);
                cached = c->pool.cached;
                in_use = c->pool.in_use;
            }
            (void)in_use;
            const size_t reserve = total_b / 20;  // 5 % of the device for everything else
            hbm_budget = free_b + cached > reserve ? free_b + cached - reserve : 0;
            if (hbm_budget == 0) return c->fail(PPST_E_BUDGET, "no device memory free for serving");
        }
        *out = (ppst_server *)new Server(*c, *k, hbm_budget, max_batch);
        return PPST_OK;
    } catch (const PpstError &e) {
        return c->fail(e.code, e.msg);
    } catch (...) {
        return PPST_E_OOM;
    }
}

int ppst_server_info(ppst_server *srv, ppst_server_stats *out)
{
    Server *s = (Server *)srv;
    if (!s || s->tag != TAG_SRV || !out) return PPST_E_ARG;
    s->info(*out);
    return PPST_OK;
}

int ppst_server_estimate(ppst_server *srv, ppst_stat stat, const ppst_col *x, const ppst_col *y, size_t *working,
                         size_t *result)
{
    Server *s = (Server *)srv;
    if (!s || s->tag != TAG_SRV) return PPST_E_ARG;
    try {
        QueryIn q;
        q.stat = stat;
        q.x = (const ColObj *)x;
        q.y = (const ColObj *)y;
        q.o = ppst_qopts{1.0, 1.0, 7, 3};
        validate_query(*s->c, q);
        if (working) *working = s->estimate(q);
        if (result) *result = s->result_bytes(q);
        return PPST_OK;
    } catch (const PpstError &e) {
        return s->c->fail(e.code, e.msg);
    } catch (...) {
        return PPST_E_ARG;
    }
}

int ppst_submit(ppst_server *srv, ppst_stat stat, const ppst_col *x, const ppst_col *y, const ppst_qopts *opts,
                uint64_t *ticket)
{
    Server *s = (Server *)srv;
    if (!s || s->tag != TAG_SRV || !ticket) return PPST_E_ARG;
    try {
        QueryIn q;
        q.stat = stat;
        q.x = (const ColObj *)x;
        q.y = (const ColObj *)y;
        q.o = opts ? *opts : ppst_qopts{1.0, 1.0, 7, 3};
        validate_query(*s->c, q);
        *ticket = s->submit(q);
        return PPST_OK;
    } catch (const PpstError &e) {
        return s->c->fail(e.code, e.msg);
    } catch (...) {
        return PPST_E_ARG;
    }
}

int ppst_wait(ppst_server *srv, uint64_t ticket, int32_t timeout_ms, ppst_res **out)
{
    Server *s = (Server *)srv;
    if (!s || s->tag != TAG_SRV || !out) return PPST_E_ARG;
    *out = nullptr;
    try {
        ResObj *r = nullptr;
        const int rc = s->wait(ticket, timeout_ms, &r);
        *out = (ppst_res *)r;
        return rc;
    } catch (const PpstError &e) {
        return s->c->fail(e.code, e.msg);
    } catch (...) {
        return PPST_E_ARG;
    }
}

int ppst_query_prepare(ppst_ctx *ctx, const ppst_evk *evk, ppst_stat stat, const ppst_col *x, const ppst_col *y,
                       const ppst_qopts *opts, ppst_plan **out)
{
    Ctx *c = (Ctx *)ctx;
    const EvkObj *k = (const EvkObj *)evk;
    if (!c || c->tag != TAG_CTX || !out) return PPST_E_ARG;
    *out = nullptr;
    if (!k || k->tag != TAG_EVK || k->ctx != c) return c->fail(PPST_E_ARG, "bad key");
    try {
        std::lock_guard<std::recursive_mutex> lk(c->exec_mu);
        QueryIn q;
        q.stat = stat;
        q.x = (const ColObj *)x;
        q.y = (const ColObj *)y;
        q.o = opts ? *opts : ppst_qopts{1.0, 1.0, 7, 3};
        validate_query(*c, q);
        *out = (ppst_plan *)plan_create(*c, *k, q);
        c->clear_err();
        return PPST_OK;
    } catch (const PpstError &e) {
        return c->fail(e.code, e.msg);
    } catch (const std::bad_alloc &) {
        return c->fail(PPST_E_OOM, "host allocation failed");
    } catch (...) {
        return c->fail(PPST_E_ARG, "unexpected error");
    }
}

int ppst_plan_run(ppst_plan *plan, ppst_res **out)
{
    Plan *p = (Plan *)plan;
    if (!p || p->tag != TAG_PLAN || !out) return PPST_E_ARG;
    *out = nullptr;
    Ctx *c = p->c;
    try {
        std::lock_guard<std::recursive_mutex> lk(c->exec_mu);
        *out = (ppst_res *)plan_run(*p);
        c->clear_err();
        return PPST_OK;
    } catch (const PpstError &e) {
        return c->fail(e.code, e.msg);
    } catch (...) {
        return c->fail(PPST_E_OOM, "result allocation failed");
    }
}

int ppst_ticket_latency(ppst_server *srv, uint64_t ticket, double *seconds)
{
    Server *s = (Server *)srv;
    if (!s || s->tag != TAG_SRV || !seconds) return PPST_E_ARG;
    try {
        *seconds = s->latency(ticket);
        return PPST_OK;
    } catch (const PpstError &e) {
        return s->c->fail(e.code, e.msg);
    }
}

}  // extern "C"
