// keys.cu -- key generation, encryption, encoding, decryption, import/export.
//
// Client-side operations of the paper's system model (Sec. 4): the client
// generates the keys and encrypts with the public key; decryption happens on
// the client. Sampling: ChaCha20 streams keyed by SplitMix64(seed), nonce =
// (purpose, index, prime index); secret and ephemeral u ternary, errors from a
// discrete Gaussian (sigma 3.2, |e| <= 19) by a cumulative table.
#include <cmath>
#include <complex>
#include <thread>
#include <cstring>

#include "ctx.cuh"

namespace ppst {

namespace {

// RAII device scratch from the context pool
struct Scratch {
    Ctx &c;
    void *p;
    size_t bytes;
    Scratch(Ctx &cc, size_t b) : c(cc), p(cc.pool.get(b)), bytes(b) {}
    ~Scratch() { c.pool.put(p, bytes); }
    uint64_t *u64() const { return (uint64_t *)p; }
    int64_t *i64() const { return (int64_t *)p; }
};

LimbMap map_rows(uint64_t *d, int rows, int N, int first = 0)
{
    // rows consecutive limbs, row r <-> global prime first + r
    return LimbMap{d, (size_t)rows * N, rows, 1, rows, first, 0};
}

}  // namespace

uint64_t galois_elt(const Ctx &c, int r)
{
    const uint64_t M = 2ull * c.N;
    int rr = ((r % c.S) + c.S) % c.S;
    return h_powmod(5, (uint64_t)rr, M);
}

// switching key from s_new to s: digit j, row t of Q_L u P:
//   b_j[t] = -a_j[t] s + e_j + [t in digit j] (P mod q_t) s_new[t],  a_j uniform
static Swk gen_swk(Ctx &c, uint64_t seed, uint64_t key_id, const uint64_t *s_ntt, const uint64_t *snew_ntt)
{
    const int N = c.N, np = c.np;
    Swk k;
    k.d = (uint64_t *)c.pool.get((size_t)c.dnum * 2 * np * N * 8);
    Scratch e_i(c, (size_t)N * 8), e_r(c, (size_t)np * N * 8);
    for (int j = 0; j < c.dnum; j++) {
        uint64_t *b = k.d + (size_t)j * 2 * np * N, *a = b + (size_t)np * N;
        const uint32_t index = (uint32_t)(key_id * 64 + j);
        LimbMap ma = map_rows(a, np, N);
        k_sample_uniform(c, seed, P_SWK_A, index, ma);
        ntt_fwd(c, ma);
        k_sample_small(c, seed, P_SWK_E, index, true, e_i.i64());
        LimbMap me = map_rows(e_r.u64(), np, N);
        k_small_to_rns(c, e_i.i64(), me);
        ntt_fwd(c, me);
        const int lo = j * c.alpha, hi = std::min((j + 1) * c.alpha, c.L + 1);
        k_swk_combine(c, b, a, e_r.u64(), s_ntt, snew_ntt, lo, hi);
    }
    return k;
}

void keygen(Ctx &c, uint64_t seed, const std::vector<int> &rots, SkObj *&sk_out, EvkObj *&evk_out)
{
    const int N = c.N, np = c.np, L = c.L;
    SkObj *sk = new SkObj();
    EvkObj *evk = new EvkObj();
    sk->ctx = evk->ctx = &c;
    evk->seed = seed;
    try {
        Scratch s_i(c, (size_t)N * 8), s_r(c, (size_t)np * N * 8), tmp(c, (size_t)np * N * 8);
        k_sample_small(c, seed, P_SECRET, 0, false, s_i.i64());
        sk->s.resize(N);
        PPST_CUDA(cudaMemcpyAsync(sk->s.data(), s_i.p, (size_t)N * 8, cudaMemcpyDeviceToHost, c.stream));
        LimbMap ms = map_rows(s_r.u64(), np, N);
        k_small_to_rns(c, s_i.i64(), ms);
        ntt_fwd(c, ms);
        // public key over Q_L: (-a s + e, a)
        evk->pk = (uint64_t *)c.pool.get(c.ct_words() * 8);
        uint64_t *pk1 = evk->pk + (size_t)(L + 1) * N;
        LimbMap mq = map_rows(pk1, L + 1, N);
        k_sample_uniform(c, seed, P_PK_A, 0, mq);
        ntt_fwd(c, mq);
        k_sample_small(c, seed, P_PK_E, 0, true, tmp.i64());
        Scratch e_r(c, (size_t)(L + 1) * N * 8);
        LimbMap me = map_rows(e_r.u64(), L + 1, N);
        k_small_to_rns(c, tmp.i64(), me);
        ntt_fwd(c, me);
        k_pk_combine(c, evk->pk, pk1, e_r.u64(), s_r.u64());
        // relinearisation key: s^2 -> s
        k_pointwise_sq(c, s_r.u64(), tmp.u64(), map_rows(s_r.u64(), np, N));
        evk->relin = gen_swk(c, seed, 0, s_r.u64(), tmp.u64());
        // Galois keys: s(X^g) -> s
        for (int r : rots) {
            const int rr = ((r % c.S) + c.S) % c.S;
            if (rr == 0 || evk->rot.count(rr)) continue;
            const uint64_t g = galois_elt(c, rr);
            k_automorph(c, s_r.u64(), np - 1, g, tmp.u64(), (size_t)np * N, 1);
            evk->rot[rr] = gen_swk(c, seed, g, s_r.u64(), tmp.u64());
        }
        PPST_CUDA(cudaStreamSynchronize(c.stream));
    } catch (...) {
        if (evk->pk) c.pool.put(evk->pk, c.ct_words() * 8);
        if (evk->relin.d) c.pool.put(evk->relin.d, (size_t)c.dnum * 2 * np * N * 8);
        for (auto &kv : evk->rot) c.pool.put(kv.second.d, (size_t)c.dnum * 2 * np * N * 8);
        delete sk;
        delete evk;
        throw;
    }
    sk_out = sk;
    evk_out = evk;
}

// (u pk0 + e0 + m, u pk1 + e1) at the top level
CtObj *encrypt_ints(Ctx &c, const EvkObj &k, const int64_t *m, uint64_t seed, uint32_t index, double scale)
{
    const int N = c.N, L = c.L;
    CtObj *ct = ct_new(c, L, scale);
    try {
        Scratch mi(c, (size_t)N * 8), mr(c, (size_t)(L + 1) * N * 8), ur(c, (size_t)(L + 1) * N * 8),
            e0(c, (size_t)(L + 1) * N * 8), e1(c, (size_t)(L + 1) * N * 8), si(c, (size_t)N * 8);
        PPST_CUDA(cudaMemcpyAsync(mi.p, m, (size_t)N * 8, cudaMemcpyHostToDevice, c.stream));
        LimbMap mm = map_rows(mr.u64(), L + 1, N);
        k_small_to_rns(c, mi.i64(), mm);
        ntt_fwd(c, mm);
        k_sample_small(c, seed, P_ENC_U, index, false, si.i64());
        LimbMap mu = map_rows(ur.u64(), L + 1, N);
        k_small_to_rns(c, si.i64(), mu);
        ntt_fwd(c, mu);
        k_sample_small(c, seed, P_ENC_E0, index, true, si.i64());
        LimbMap m0 = map_rows(e0.u64(), L + 1, N);
        k_small_to_rns(c, si.i64(), m0);
        ntt_fwd(c, m0);
        k_sample_small(c, seed, P_ENC_E1, index, true, si.i64());
        LimbMap m1 = map_rows(e1.u64(), L + 1, N);
        k_small_to_rns(c, si.i64(), m1);
        ntt_fwd(c, m1);
        k_enc_combine(c, k.pk, ur.u64(), e0.u64(), e1.u64(), mr.u64(), *ct);
        // host buffer m must stay valid until the copy is done
        PPST_CUDA(cudaStreamSynchronize(c.stream));
    } catch (...) {
        ct_free(ct);
        throw;
    }
    return ct;
}

// ---------------------------------------------------------------------------
// canonical embedding: slot j <-> evaluation at zeta^(5^j), zeta = exp(i pi / N)
// ---------------------------------------------------------------------------
static void fft_inplace(std::vector<std::complex<double>> &a, int sign)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = sign * 2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len) {
            for (size_t k = 0; k < len / 2; k++) {
                const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

void encode(const Ctx &c, const double *z, size_t n, double scale, std::vector<int64_t> &m)
{
    const int N = c.N, S = c.S;
    const uint64_t M = 2ull * N;
    std::vector<std::complex<double>> w(N, 0.0);
    uint64_t e = 1;
    for (int j = 0; j < S; j++) {
        const double zj = (size_t)j < n ? z[j] : 0.0;
        w[(e - 1) / 2] = zj;
        w[(M - e - 1) / 2] = zj;
        e = e * 5 % M;
    }
    fft_inplace(w, -1);
    m.resize(N);
    for (int i = 0; i < N; i++) {
        const std::complex<double> zn(std::cos(-M_PI * i / N), std::sin(-M_PI * i / N));
        const double x = (zn * w[i]).real() / N * scale;
        if (!(std::fabs(x) < 0x1p62)) throw_err(PPST_E_ARG, "value too large for the scale");
        m[i] = (int64_t)h_round_away(x);
    }
}

// centred CRT of residues r[0..nl) (Garner mixed radix, exact) -> double
struct Crt {
    std::vector<uint64_t> q;
    std::vector<std::vector<uint64_t>> pref;  // pref[k][i] = prod_{m<k} q_m mod q_i
    std::vector<uint64_t> inv;                // inv[i] = (prod_{m<i} q_m)^-1 mod q_i
    std::vector<std::vector<uint64_t>> big;   // prod_{m<k} q_m as little-endian words
    std::vector<uint64_t> Q, halfQ;

    explicit Crt(const std::vector<uint64_t> &qs) : q(qs)
    {
        const int n = (int)q.size();
        pref.assign(n + 1, std::vector<uint64_t>(n, 0));
        for (int i = 0; i < n; i++) pref[0][i] = 1 % q[i];
        for (int k = 1; k <= n; k++)
            for (int i = 0; i < n; i++) pref[k][i] = h_mulmod(pref[k - 1][i], q[k - 1] % q[i], q[i]);
        inv.resize(n);
        for (int i = 0; i < n; i++) inv[i] = h_invmod(pref[i][i], q[i]);
        big.assign(n + 1, {});
        big[0] = {1};
        for (int k = 1; k <= n; k++) big[k] = mul_small(big[k - 1], q[k - 1]);
        Q = big[n];
        halfQ = Q;
        uint64_t carry = 0;
        for (int i = (int)halfQ.size() - 1; i >= 0; i--) {
            u128 cur = ((u128)carry << 64) | halfQ[i];
            halfQ[i] = (uint64_t)(cur >> 1);
            carry = (uint64_t)(cur & 1);
        }
    }
    static std::vector<uint64_t> mul_small(const std::vector<uint64_t> &a, uint64_t m)
    {
        std::vector<uint64_t> r(a.size() + 1, 0);
        u128 carry = 0;
        for (size_t i = 0; i < a.size(); i++) {
            u128 cur = (u128)a[i] * m + carry;
            r[i] = (uint64_t)cur;
            carry = cur >> 64;
        }
        r[a.size()] = (uint64_t)carry;
        while (r.size() > 1 && r.back() == 0) r.pop_back();
        return r;
    }
    static int cmp(const std::vector<uint64_t> &a, const std::vector<uint64_t> &b)
    {
        size_t n = std::max(a.size(), b.size());
        for (size_t i = n; i-- > 0;) {
            uint64_t x = i < a.size() ? a[i] : 0, y = i < b.size() ? b[i] : 0;
            if (x != y) return x < y ? -1 : 1;
        }
        return 0;
    }
    static double to_double(const std::vector<uint64_t> &a)
    {
        double r = 0;
        for (size_t i = a.size(); i-- > 0;) r = r * 0x1p64 + (double)a[i];
        return r;
    }
    // the centred value of the residues r[i stride] (Garner's mixed radix, then
    // the big integer x or x - Q), as a double; no allocation
    double centred(const uint64_t *r, size_t stride) const
    {
        const int n = (int)q.size();
        uint64_t v[MAXL];
        for (int i = 0; i < n; i++) {
            // x_{<i} mod q_i = sum_{k<i} v_k prod_{m<k} q_m
            uint64_t s = 0;
            for (int k = 0; k < i; k++) s = (s + h_mulmod(v[k], pref[k][i], q[i])) % q[i];
            uint64_t d = (r[(size_t)i * stride] % q[i] + q[i] - s) % q[i];
            v[i] = h_mulmod(d, inv[i], q[i]);
        }
        const size_t W = Q.size() + 1;
        uint64_t x[MAXL + 2] = {0};
        for (int k = 0; k < n; k++) {  // x += v_k * big[k]
            u128 carry = 0;
            const std::vector<uint64_t> &bk = big[k];
            for (size_t i = 0; i < W; i++) {
                u128 cur = (u128)x[i] + carry + (i < bk.size() ? (u128)bk[i] * v[k] : 0);
                x[i] = (uint64_t)cur;
                carry = cur >> 64;
            }
        }
        int c = 0;  // compare x with Q / 2
        for (size_t i = W; i-- > 0 && c == 0;) {
            const uint64_t hq = i < halfQ.size() ? halfQ[i] : 0;
            if (x[i] != hq) c = x[i] < hq ? -1 : 1;
        }
        double sign = 1.0;
        if (c > 0) {  // negative: Q - x
            sign = -1.0;
            uint64_t borrow = 0;
            for (size_t i = 0; i < W; i++) {
                const uint64_t qi = i < Q.size() ? Q[i] : 0;
                const u128 sub = (u128)x[i] + borrow;
                if ((u128)qi >= sub) {
                    x[i] = (uint64_t)((u128)qi - sub);
                    borrow = 0;
                } else {
                    x[i] = (uint64_t)((((u128)1) << 64) + qi - sub);
                    borrow = 1;
                }
            }
        }
        double r0 = 0;
        for (size_t i = W; i-- > 0;) r0 = r0 * 0x1p64 + (double)x[i];
        return sign * r0;
    }
};

// m_i / scale for every coefficient i, on up to 16 host threads
static void crt_scaled(const Crt &crt, const uint64_t *h, int N, double scale, std::vector<double> &m)
{
    m.resize(N);
    const int T = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    auto work = [&](int t) {
        for (int i = (int)((int64_t)N * t / T); i < (int)((int64_t)N * (t + 1) / T); i++)
            m[i] = crt.centred(h + i, (size_t)N) / scale;
    };
    std::vector<std::thread> th;
    for (int t = 1; t < T; t++) th.emplace_back(work, t);
    work(0);
    for (std::thread &x : th) x.join();
}

void decrypt_to_slots(Ctx &c, const SkObj &sk, const CtObj &ct, std::vector<double> &slots, int want)
{
    const int N = c.N, nl = ct.level + 1;
    Scratch si(c, (size_t)N * 8), sr(c, (size_t)nl * N * 8), mr(c, (size_t)nl * N * 8);
    PPST_CUDA(cudaMemcpyAsync(si.p, sk.s.data(), (size_t)N * 8, cudaMemcpyHostToDevice, c.stream));
    LimbMap ms = map_rows(sr.u64(), nl, N);
    k_small_to_rns(c, si.i64(), ms);
    ntt_fwd(c, ms);
    k_dec_combine(c, ct, sr.u64(), mr.u64());
    LimbMap mm = map_rows(mr.u64(), nl, N);
    ntt_inv(c, mm);
    std::vector<uint64_t> h((size_t)nl * N);
    PPST_CUDA(cudaMemcpyAsync(h.data(), mr.p, h.size() * 8, cudaMemcpyDeviceToHost, c.stream));
    PPST_CUDA(cudaStreamSynchronize(c.stream));
    check_device_error(c);
    Crt crt(std::vector<uint64_t>(c.primes.begin(), c.primes.begin() + nl));
    std::vector<double> m;
    crt_scaled(crt, h.data(), N, ct.scale, m);
    if (c.twist.size() != (size_t)N) {
        c.twist.resize(N);
        for (int i = 0; i < N; i++) c.twist[i] = std::complex<double>(std::cos(M_PI * i / N), std::sin(M_PI * i / N));
    }
    if (want == 1) {  // slot 0 alone: m(zeta) = sum_i m_i zeta^i, real part
        double s0 = 0;
        for (int i = 0; i < N; i++) s0 += m[i] * c.twist[i].real();
        slots.assign(c.S, 0.0);
        slots[0] = s0;
        return;
    }
    std::vector<std::complex<double>> v(N);
    for (int i = 0; i < N; i++) v[i] = m[i] * c.twist[i];
    fft_inplace(v, +1);
    slots.resize(c.S);
    const uint64_t M = 2ull * N;
    uint64_t e = 1;
    for (int j = 0; j < c.S; j++) {
        slots[j] = v[(e - 1) / 2].real();
        e = e * 5 % M;
    }
}

// ---------------------------------------------------------------------------
// import / export (coefficient domain on the host)
// ---------------------------------------------------------------------------
void export_ct(Ctx &c, const CtObj &ct, uint64_t *c0, uint64_t *c1)
{
    const int N = c.N, nl = ct.level + 1;
    const size_t ps = (size_t)(c.L + 1) * N;
    Scratch t(c, c.ct_words() * 8);
    k_copy(c, t.u64(), ct.d, (size_t)nl * N);
    k_copy(c, t.u64() + ps, ct.d + ps, (size_t)nl * N);
    ntt_inv(c, map_ct(c, t.u64(), ct.level));
    PPST_CUDA(cudaMemcpyAsync(c0, t.p, (size_t)nl * N * 8, cudaMemcpyDeviceToHost, c.stream));
    PPST_CUDA(cudaMemcpyAsync(c1, t.u64() + ps, (size_t)nl * N * 8, cudaMemcpyDeviceToHost, c.stream));
    PPST_CUDA(cudaStreamSynchronize(c.stream));
    check_device_error(c);
}

CtObj *import_ct(Ctx &c, const uint64_t *c0, const uint64_t *c1, int level, double scale)
{
    const int N = c.N, nl = level + 1;
    for (int i = 0; i < nl; i++)
        for (int k = 0; k < N; k++)
            if (c0[(size_t)i * N + k] >= c.primes[i] || c1[(size_t)i * N + k] >= c.primes[i])
                throw_err(PPST_E_ARG, "residue not reduced");
    CtObj *ct = ct_new(c, level, scale);
    const size_t ps = (size_t)(c.L + 1) * N;
    try {
        PPST_CUDA(cudaMemcpyAsync(ct->d, c0, (size_t)nl * N * 8, cudaMemcpyHostToDevice, c.stream));
        PPST_CUDA(cudaMemcpyAsync(ct->d + ps, c1, (size_t)nl * N * 8, cudaMemcpyHostToDevice, c.stream));
        ntt_fwd(c, map_ct(c, ct->d, level));
        PPST_CUDA(cudaStreamSynchronize(c.stream));
    } catch (...) {
        ct_free(ct);
        throw;
    }
    return ct;
}

void export_swk(Ctx &c, const Swk &k, int digit, uint64_t *b, uint64_t *a)
{
    const int N = c.N, np = c.np;
    Scratch t(c, (size_t)2 * np * N * 8);
    k_copy(c, t.u64(), k.d + (size_t)digit * 2 * np * N, (size_t)2 * np * N);
    LimbMap m{t.u64(), (size_t)np * N, np, 2, np, 0, 0};
    k_to_mont(c, t.u64(), m, false);
    ntt_inv(c, m);
    PPST_CUDA(cudaMemcpyAsync(b, t.p, (size_t)np * N * 8, cudaMemcpyDeviceToHost, c.stream));
    PPST_CUDA(cudaMemcpyAsync(a, t.u64() + (size_t)np * N, (size_t)np * N * 8, cudaMemcpyDeviceToHost, c.stream));
    PPST_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace ppst
