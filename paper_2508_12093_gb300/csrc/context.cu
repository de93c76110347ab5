// context.cu -- parameter set, prime chain, device tables and memory pool.
#include <cmath>
#include <cstring>
#include <set>

#include "ctx.cuh"

namespace ppst {

[[noreturn]] void throw_err(int code, const std::string &m) { throw PpstError{code, m}; }

void cuda_check(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) throw_err(PPST_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw_err(PPST_E_CUDA, std::string("launch ") + what + ": " + cudaGetErrorString(e));
}

cudaEvent_t Prof::take()
{
    if (!spare.empty()) {
        cudaEvent_t e = spare.back();
        spare.pop_back();
        return e;
    }
    cudaEvent_t e;
    PPST_CUDA(cudaEventCreate(&e));
    return e;
}

ProfScope::ProfScope(Ctx &cc, const char *k, uint64_t u, uint64_t mu) : c(cc), cls(k), units(u), munits(mu)
{
    c.prof.launches++;
    if (c.prof.on && (c.prof.only.empty() || c.prof.only == cls)) {
        b = c.prof.take();
        PPST_CUDA(cudaEventRecord(b, c.stream));
    }
}

ProfScope::~ProfScope()
{
    if (!b) return;
    cudaEvent_t e = c.prof.take();
    cudaEventRecord(e, c.stream);
    c.prof.rec[cls].push_back(ProfRec{b, e, units, munits});
}

// ---------------------------------------------------------------------------
// host modular arithmetic (exact, 128-bit)
// ---------------------------------------------------------------------------
uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }

uint64_t h_powmod(uint64_t b, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    b %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = h_mulmod(r, b, q);
        b = h_mulmod(b, b, q);
    }
    return r;
}

uint64_t h_invmod(uint64_t a, uint64_t q) { return h_powmod(a % q, q - 2, q); }

uint64_t h_shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// Miller-Rabin with the first twelve primes as bases (deterministic below 3.3e24)
bool h_is_prime(uint64_t n)
{
    static const uint64_t B[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t b : B) {
        if (n == b) return true;
        if (n % b == 0) return false;
    }
    uint64_t d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        s++;
    }
    for (uint64_t b : B) {
        uint64_t x = h_powmod(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s && comp; r++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

// round half away from zero, exact: floor(|x|) plus one if the (exact) fraction >= 1/2
__int128 h_round_away(double x)
{
    if (!(std::fabs(x) < 0x1p126)) throw_err(PPST_E_ARG, "constant out of range");
    double a = std::fabs(x);
    double f = std::floor(a);
    __int128 m;
    if (f >= 0x1p63) {
        int e;
        double mant = std::frexp(f, &e);  // f = mant 2^e, mant in [0.5, 1)
        __int128 mi = (__int128)(int64_t)std::ldexp(mant, 53);
        m = mi << (e - 53);
    } else {
        m = (__int128)(uint64_t)f;
    }
    if (a - f >= 0.5) m += 1;
    return x < 0 ? -m : m;
}

// round half away from zero of the exact product k * m (m < 2^62)
__int128 h_round_mul(double k, uint64_t m)
{
    if (k == 0.0 || m == 0) return 0;
    if (!std::isfinite(k) || std::fabs(k) >= 0x1p60) throw_err(PPST_E_ARG, "constant out of range");
    int e;
    double mant = std::frexp(std::fabs(k), &e);      // |k| = mant 2^e
    uint64_t M = (uint64_t)std::ldexp(mant, 53);     // |k| = M 2^(e-53), exact
    int sh = e - 53;
    u128 prod = (u128)M * m;                          // < 2^115
    u128 r;
    if (sh >= 0) {
        r = prod << sh;  // |k| < 2^60 -> sh <= 7, product < 2^122
    } else {
        int s = -sh;
        if (s >= 127) {
            r = 0;
        } else {
            u128 q = prod >> s;
            u128 rem = prod - (q << s);
            u128 half = (u128)1 << (s - 1);
            r = q + (rem >= half ? 1 : 0);
        }
    }
    __int128 v = (__int128)r;
    return k < 0 ? -v : v;
}

uint64_t h_mod_i128(__int128 v, uint64_t q)
{
    if (v >= 0) return (uint64_t)((u128)v % q);
    uint64_t r = (uint64_t)((u128)(-v) % q);
    return r ? q - r : 0;
}

// ---------------------------------------------------------------------------
// memory pool
// ---------------------------------------------------------------------------
void *Pool::get(size_t bytes)
{
    std::lock_guard<std::recursive_mutex> lk(mu);
    auto &v = free_[bytes];
    if (!v.empty()) {
        void *p = v.back();
        v.pop_back();
        cached -= bytes;
        in_use += bytes;
        if (recording) ledger.emplace_back(p, bytes);
        return p;
    }
    if (frozen) throw_err(PPST_E_STATE, "device allocation while a graph is being captured");
    for (int attempt = 0; attempt < 2; attempt++) {
        void *p = nullptr;
        if (has_user) {
            p = user.alloc(user.user, bytes, (void *)stream);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) {
            in_use += bytes;
            return p;
        }
        trim();
    }
    throw_err(PPST_E_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
}

void Pool::put(void *p, size_t bytes)
{
    if (!p) return;
    std::lock_guard<std::recursive_mutex> lk(mu);
    free_[bytes].push_back(p);
    in_use -= bytes;
    cached += bytes;
}

bool Pool::withdraw(void *p, size_t bytes)
{
    std::lock_guard<std::recursive_mutex> lk(mu);
    auto it = free_.find(bytes);
    if (it == free_.end()) return false;
    for (size_t i = 0; i < it->second.size(); i++) {
        if (it->second[i] != p) continue;
        it->second.erase(it->second.begin() + i);
        cached -= bytes;
        in_use += bytes;
        return true;
    }
    return false;
}

void Pool::trim()
{
    std::lock_guard<std::recursive_mutex> lk(mu);
    cudaStreamSynchronize(stream);
    for (auto &kv : free_) {
        for (void *p : kv.second) {
            if (has_user) user.release(user.user, p, kv.first, (void *)stream);
            else cudaFree(p);
        }
        cached -= kv.first * kv.second.size();
        kv.second.clear();
    }
}

CtObj *ct_new(Ctx &c, int level, double scale)
{
    CtObj *ct = new CtObj();
    ct->ctx = &c;
    ct->level = level;
    ct->scale = scale;
    try {
        const size_t bytes = c.ct_words() * 8;
        uint64_t *p = (uint64_t *)c.pool.get(bytes);
        Ctx *cp = &c;
        ct->buf = std::shared_ptr<uint64_t>(p, [cp, bytes](uint64_t *q) { cp->pool.put(q, bytes); });
        ct->d = p;
    } catch (...) {
        delete ct;
        throw;
    }
    return ct;
}

void ct_free(CtObj *ct)
{
    if (!ct) return;
    ct->buf.reset();
    ct->tag = TAG_DEAD;
    delete ct;
}

CtObj *ct_view(const CtObj &a, int level)
{
    CtObj *o = new CtObj();
    o->ctx = a.ctx;
    o->buf = a.buf;
    o->d = a.d;
    o->level = level;
    o->scale = a.scale;
    return o;
}

CtObj *ct_clone(const CtObj &a) { return ct_view(a, a.level); }

LimbMap map_ct(const Ctx &c, uint64_t *d, int level)
{
    return LimbMap{d, (size_t)(c.L + 1) * c.N, level + 1, 2, level + 1, 0, 0};
}

LimbMap map_poly(const Ctx &c, uint64_t *d, int level)
{
    return LimbMap{d, (size_t)(c.L + 1) * c.N, level + 1, 1, level + 1, 0, 0};
}

void ensure_workspace(Ctx &c, int items)
{
    if (c.ws_items >= items && c.ws_d2) return;
    const size_t N = c.N, B = (size_t)std::max(items, c.ws_items);
    const size_t q = c.L + 1, e = c.ext_rows();
    if (c.ws_d2) {  // grow: the old buffers go back to the pool once the stream is past them
        c.pool.put(c.ws_d2, (size_t)c.ws_items * q * N * 8);
        c.pool.put(c.ws_d2n, (size_t)c.ws_items * q * N * 8);
        c.pool.put(c.ws_ext, (size_t)c.ws_items * c.dnum * e * N * 8);
        c.pool.put(c.ws_acc, (size_t)c.ws_items * 2 * e * N * 8);
        c.pool.put(c.ws_conv, (size_t)c.ws_items * 2 * q * N * 8);
        c.pool.put(c.ws_top, (size_t)c.ws_items * 2 * N * 8);
        c.ws_d2 = c.ws_d2n = c.ws_ext = c.ws_acc = c.ws_conv = c.ws_top = nullptr;
        c.ws_items = 0;
    }
    c.ws_d2 = (uint64_t *)c.pool.get(B * q * N * 8);
    c.ws_d2n = (uint64_t *)c.pool.get(B * q * N * 8);
    c.ws_ext = (uint64_t *)c.pool.get(B * c.dnum * e * N * 8);
    c.ws_acc = (uint64_t *)c.pool.get(B * 2 * e * N * 8);
    c.ws_conv = (uint64_t *)c.pool.get(B * 2 * q * N * 8);
    c.ws_top = (uint64_t *)c.pool.get(B * 2 * N * 8);
    c.ws_items = (int)B;
    c.ws_bytes = B * (2 * q + c.dnum * e + 2 * e + 2 * q + 2) * N * 8;
}

// ---------------------------------------------------------------------------
// prime chain (rule stated in ppst.h)
// ---------------------------------------------------------------------------
static uint64_t next_below(uint64_t &cur, uint64_t M)
{
    // cur: last candidate tried (= 1 mod M); move down to the next prime
    while (cur > M) {
        cur -= M;
        if (h_is_prime(cur)) return cur;
    }
    throw_err(PPST_E_ARG, "prime chain: ran out of candidates");
}

static uint64_t next_above(uint64_t &cur, uint64_t M)
{
    for (int guard = 0; guard < 100000000; guard++) {
        cur += M;
        if (h_is_prime(cur)) return cur;
    }
    throw_err(PPST_E_ARG, "prime chain: ran out of candidates");
}

static std::vector<uint64_t> make_chain(const ppst_params &p, std::vector<uint64_t> &pout)
{
    const uint64_t M = 2ull << p.log_n;
    std::set<uint64_t> used;
    // first candidate below 2^b: (2^b / M) M + 1 is above 2^b, so start there
    auto start = [&](uint32_t bits) { return ((1ull << bits) / M) * M + 1; };
    uint64_t cur = start(p.q0_bits);
    uint64_t q0 = next_below(cur, M);
    used.insert(q0);
    pout.clear();
    cur = start(p.p_bits);
    while (pout.size() < p.n_p) {
        uint64_t c = next_below(cur, M);
        if (!used.count(c)) {
            pout.push_back(c);
            used.insert(c);
        }
    }
    std::vector<uint64_t> q{q0};
    uint64_t up = start(p.q_bits) - M, down = start(p.q_bits);
    while (q.size() < p.n_q) {
        uint64_t c;
        do {
            c = (q.size() % 2 == 1) ? next_above(up, M) : next_below(down, M);
        } while (used.count(c));
        used.insert(c);
        q.push_back(c);
    }
    return q;
}

static uint64_t find_psi(uint64_t q, uint64_t N)
{
    for (uint64_t g = 2;; g++) {
        uint64_t psi = h_powmod(g, (q - 1) / (2 * N), q);
        if (h_powmod(psi, N, q) == q - 1) return psi;
    }
}

static uint32_t brv(uint32_t x, int bits)
{
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

template <class T>
static T *upload(Ctx &c, const std::vector<T> &v)
{
    T *d = (T *)c.pool.get(v.size() * sizeof(T) + 256);
    PPST_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c.stream));
    return d;
}

static uint64_t mont_form(uint64_t x, uint64_t q) { return (uint64_t)(((u128)x << 64) % q); }

Ctx *ctx_create(const ppst_params &pin, const ppst_allocator *alloc, cudaStream_t stream)
{
    ppst_params p = pin;
    if (p.sigma == 0) p.sigma = 3.2;
    if (p.gauss_bound == 0) p.gauss_bound = 19;
    if (p.log_n < 10 || p.log_n > 16 || p.n_q < 2 || p.n_q > 60 || p.n_p < 1 || p.n_p > 16 || p.dnum < 1 ||
        p.dnum > p.n_q || p.q0_bits > 61 || p.q_bits > 60 || p.p_bits > 61 || p.q0_bits < 20 || p.q_bits < 20 ||
        p.p_bits < 20 || !(p.log_scale > 0 && p.log_scale < 62) || p.gauss_bound > 64 ||
        p.n_q + p.n_p > (uint32_t)MAXL)
        throw_err(PPST_E_ARG, "parameters out of range");
    const uint32_t alpha = (p.n_q + p.dnum - 1) / p.dnum;
    if (alpha > 16) throw_err(PPST_E_ARG, "more than 16 primes per digit");

    Ctx *c = new Ctx();
    try {
        c->prm = p;
        c->logN = p.log_n;
        c->N = 1 << p.log_n;
        c->S = c->N / 2;
        c->L = p.n_q - 1;
        c->K = p.n_p;
        c->alpha = alpha;
        c->dnum = (p.n_q + alpha - 1) / alpha;
        c->scale = std::pow(2.0, p.log_scale);
        c->sigma = p.sigma;
        c->gbound = p.gauss_bound;
        c->stream = stream;
        c->pool.stream = stream;
        if (alloc && alloc->alloc) {
            c->pool.user = *alloc;
            c->pool.has_user = true;
        }
        std::vector<uint64_t> pp;
        std::vector<uint64_t> q = make_chain(p, pp);
        c->primes = q;
        c->primes.insert(c->primes.end(), pp.begin(), pp.end());
        c->np = (int)c->primes.size();
        const int N = c->N, np = c->np, L = c->L, K = c->K;

        // per-prime constants and transform tables
        c->hpc.resize(np);
        std::vector<Tw> twf((size_t)np * N), twi((size_t)np * N);
        std::vector<uint64_t> pw(N), ipw(N);
        for (int t = 0; t < np; t++) {
            const uint64_t qt = c->primes[t];
            const uint64_t psi = find_psi(qt, N), ipsi = h_invmod(psi, qt);
            c->psi.push_back(psi);
            PrimeC &pc = c->hpc[t];
            pc.q = qt;
            uint64_t inv = 1;  // Newton iteration for q^-1 mod 2^64
            for (int i = 0; i < 7; i++) inv *= 2 - qt * inv;
            pc.qinv = inv;
            pc.r2 = (uint64_t)(((u128)mont_form(1, qt) << 64) % qt);
            pc.ninv = h_invmod((uint64_t)N % qt, qt);
            pc.ninv_sh = h_shoup(pc.ninv, qt);
            pc.w64 = (uint64_t)((((u128)1) << 64) / qt);
            pw[0] = 1;
            ipw[0] = 1;
            for (int i = 1; i < N; i++) {
                pw[i] = h_mulmod(pw[i - 1], psi, qt);
                ipw[i] = h_mulmod(ipw[i - 1], ipsi, qt);
            }
            for (int k = 0; k < N; k++) {
                const uint32_t r = brv((uint32_t)k, c->logN);
                const size_t o = (size_t)t * N + k;
                twf[o] = Tw{pw[r], h_shoup(pw[r], qt)};
                twi[o] = Tw{ipw[r], h_shoup(ipw[r], qt)};
            }
        }
        {
            void *hp = nullptr;
            PPST_CUDA(cudaHostAlloc(&hp, 64, cudaHostAllocMapped));
            c->h_err = (volatile int *)hp;
            *c->h_err = 0;
            void *dp = nullptr;
            PPST_CUDA(cudaHostGetDevicePointer(&dp, hp, 0));
            c->d_err = (int *)dp;
        }
        c->d_pc = upload(*c, c->hpc);
        c->d_twf = upload(*c, twf);
        c->d_twi = upload(*c, twi);

        // discrete Gaussian CDT: T[k] = floor(2^64 P(|e| <= k)), IEEE double in this order
        {
            const double s = c->sigma;
            double tot = std::exp(-0.0 / (2.0 * s * s));
            for (uint32_t x = 1; x <= (uint32_t)c->gbound; x++)
                tot += 2.0 * std::exp(-(double)(x * x) / (2.0 * s * s));
            double cum = std::exp(-0.0 / (2.0 * s * s));
            c->cdt.resize(c->gbound);
            for (uint32_t k = 0; k < (uint32_t)c->gbound; k++) {
                if (k > 0) cum += 2.0 * std::exp(-(double)(k * k) / (2.0 * s * s));
                c->cdt[k] = (uint64_t)std::ldexp(cum / tot, 64);
            }
            c->d_cdt = upload(*c, c->cdt);
        }

        // key-switching tables
        std::vector<uint64_t> ks;
        c->modup_off.assign(L + 1, {});
        for (int l = 0; l <= L; l++) {
            const int E = l + 1 + K;
            for (int j = 0; j < c->ndigits(l); j++) {
                const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, l + 1), a = hi - lo;
                c->modup_off[l].push_back(ks.size());
                std::vector<uint64_t> hinv(a), hsh(a), hM((size_t)a * E);
                for (int i = 0; i < a; i++) {
                    const uint64_t qi = c->primes[lo + i];
                    uint64_t h = 1;
                    for (int k = 0; k < a; k++)
                        if (k != i) h = h_mulmod(h, c->primes[lo + k] % qi, qi);
                    hinv[i] = h_invmod(h, qi);
                    hsh[i] = h_shoup(hinv[i], qi);
                    for (int e = 0; e < E; e++) {
                        const uint64_t t = c->primes[e <= l ? e : L + 1 + (e - l - 1)];
                        uint64_t ht = 1 % t;
                        for (int k = 0; k < a; k++)
                            if (k != i) ht = h_mulmod(ht, c->primes[lo + k] % t, t);
                        hM[(size_t)i * E + e] = mont_form(ht, t);
                    }
                }
                ks.insert(ks.end(), hinv.begin(), hinv.end());
                ks.insert(ks.end(), hsh.begin(), hsh.end());
                ks.insert(ks.end(), hM.begin(), hM.end());
            }
        }
        c->moddown_off = ks.size();
        {
            std::vector<uint64_t> hinv(K), hsh(K), hM((size_t)K * (L + 1));
            for (int m = 0; m < K; m++) {
                const uint64_t pm = c->primes[L + 1 + m];
                uint64_t h = 1;
                for (int k = 0; k < K; k++)
                    if (k != m) h = h_mulmod(h, c->primes[L + 1 + k] % pm, pm);
                hinv[m] = h_invmod(h, pm);
                hsh[m] = h_shoup(hinv[m], pm);
                for (int i = 0; i <= L; i++) {
                    const uint64_t qi = c->primes[i];
                    uint64_t ht = 1 % qi;
                    for (int k = 0; k < K; k++)
                        if (k != m) ht = h_mulmod(ht, c->primes[L + 1 + k] % qi, qi);
                    hM[(size_t)m * (L + 1) + i] = mont_form(ht, qi);
                }
            }
            ks.insert(ks.end(), hinv.begin(), hinv.end());
            ks.insert(ks.end(), hsh.begin(), hsh.end());
            ks.insert(ks.end(), hM.begin(), hM.end());
        }
        c->d_ks = upload(*c, ks);
        // P^-1 mod q_i; P mod q_t (gadget); rescale constants
        std::memset(&c->pinv, 0, sizeof(ConstVec));
        ConstVec pm;
        std::memset(&pm, 0, sizeof(ConstVec));
        for (int t = 0; t < np; t++) {
            const uint64_t qt = c->primes[t];
            uint64_t P = 1;
            for (int k = 0; k < K; k++) P = h_mulmod(P, c->primes[L + 1 + k] % qt, qt);
            pm.c[t] = P;
            pm.sh[t] = h_shoup(P, qt);
            if (t <= L) {
                c->pinv.c[t] = h_invmod(P, qt);
                c->pinv.sh[t] = h_shoup(c->pinv.c[t], qt);
            }
        }
        c->pmod.push_back(pm);
        c->resc.assign(L + 1, ConstVec{});
        c->resc_qmodv.assign(L + 1, ConstVec{});
        for (int l = 1; l <= L; l++) {
            const uint64_t ql = c->primes[l];
            for (int i = 0; i < l; i++) {
                const uint64_t qi = c->primes[i];
                c->resc[l].c[i] = h_invmod(ql % qi, qi);
                c->resc[l].sh[i] = h_shoup(c->resc[l].c[i], qi);
                c->resc_qmodv[l].c[i] = ql % qi;
            }
        }
        // fused key switching tables
        {
            std::vector<Tw> mo;
            for (int l = 0; l <= L; l++) {
                c->modup_outmul_off.push_back(mo.size());
                for (int i = 0; i <= l; i++) {
                    const int lo = (i / c->alpha) * c->alpha, hi = std::min(lo + c->alpha, l + 1);
                    const uint64_t qi = c->primes[i];
                    uint64_t h = 1;
                    for (int k = lo; k < hi; k++)
                        if (k != i) h = h_mulmod(h, c->primes[k] % qi, qi);
                    const uint64_t v = h_mulmod(c->hpc[i].ninv, h_invmod(h, qi), qi);
                    mo.push_back(Tw{v, h_shoup(v, qi)});
                }
            }
            c->d_modup_outmul = upload(*c, mo);
            std::vector<Tw> md(2 * K);
            for (int b = 0; b < 2 * K; b++) {
                const int m = b % K;
                const uint64_t pm = c->primes[L + 1 + m];
                uint64_t h = 1;
                for (int k = 0; k < K; k++)
                    if (k != m) h = h_mulmod(h, c->primes[L + 1 + k] % pm, pm);
                const uint64_t v = h_mulmod(c->hpc[L + 1 + m].ninv, h_invmod(h, pm), pm);
                md[b] = Tw{v, h_shoup(v, pm)};
            }
            c->d_md_outmul = upload(*c, md);
            std::vector<Tw> mdt;
            for (int l = 0; l <= L; l++) {
                mdt.push_back(Tw{c->hpc[l].ninv, c->hpc[l].ninv_sh});
                for (int m = 0; m < K; m++) mdt.push_back(md[m]);
            }
            c->d_md_outmul_top = upload(*c, mdt);
            c->md_const.assign((size_t)(L + 1) * (L + 1), MdC{});
            for (int l = 0; l <= L; l++) {
                const uint64_t ql = c->primes[l];
                for (int i = 0; i <= l; i++) {
                    const uint64_t qi = c->primes[i];
                    MdC &m = c->md_const[(size_t)l * (L + 1) + i];
                    const uint64_t pinv = c->pinv.c[i];
                    const uint64_t qlinv = i < l ? h_invmod(ql % qi, qi) : 0;
                    const uint64_t pq = h_mulmod(pinv, qlinv, qi);
                    m.pinv = Tw{pinv, h_shoup(pinv, qi)};
                    m.qlinv = Tw{qlinv, h_shoup(qlinv, qi)};
                    m.pq = Tw{pq, h_shoup(pq, qi)};
                    m.qmod = ql % qi;
                }
            }
            c->d_md_const = upload(*c, c->md_const);
        }
        // commit the allocation-free HMult's static scratch on this device now,
        // while allocating is still possible (see noalloc.cu)
        noalloc_scratch_on_current_device();
        PPST_CUDA(cudaStreamSynchronize(stream));
    } catch (...) {
        ctx_destroy(c);
        throw;
    }
    return c;
}

void ctx_destroy(Ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    // return everything we own to the pool, then release the pool
    // (sizes are only needed by user allocators; tables were taken with +256 slack)
    c->pool.trim();
    // device tables and workspace are not in the free lists; release them directly
    std::vector<void *> own = {c->d_pc,          c->d_twf,      c->d_twi,   c->d_cdt,   c->d_ks,
                               c->d_modup_outmul, c->d_md_outmul, c->d_md_outmul_top, c->d_md_const, c->ws_d2, c->ws_d2n,
                               c->ws_ext,         c->ws_acc,     c->ws_conv, c->ws_top};
    for (void *p : own) {
        if (!p) continue;
        if (c->pool.has_user) c->pool.user.release(c->pool.user.user, p, 0, (void *)c->stream);
        else cudaFree(p);
    }
    if (c->h_err) cudaFreeHost((void *)c->h_err);
    c->tag = TAG_DEAD;
    delete c;
}

void check_device_error(Ctx &c)
{
    if (c.h_err && *c.h_err) {
        *c.h_err = 0;
        throw_err(PPST_E_CUDA, "a kernel's wait for its asynchronous copies timed out");
    }
}

}  // namespace ppst
