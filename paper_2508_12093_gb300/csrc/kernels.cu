// kernels.cu -- elementwise, key-switching, rescale, automorphism and sampling
// kernels. Layouts: a ciphertext buffer is [2][L+1][N] (c0 then c1, limb-major,
// limbs 0..level valid); an extended polynomial is [L+1+K][N] with rows
// q_0..q_level then p_0..p_{K-1}; a switching key is [dnum][2][L+1+K][N] with
// rows q_0..q_L, p_0..p_{K-1} (row index = global prime index).
#include "ntt.cuh"

namespace ppst {

constexpr int EW_THREADS = 256;

static inline dim3 ew_grid(const Ctx &c, int rows) { return dim3((c.N + EW_THREADS - 1) / EW_THREADS, rows); }

// ---------------------------------------------------------------------------
// ciphertext elementwise ops
// ---------------------------------------------------------------------------
enum EwOp { EW_ADD, EW_SUB, EW_NEG, EW_MULC, EW_ADDC0 };

template <int OP>
__global__ void __launch_bounds__(EW_THREADS) k_ct_ew(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b,
                                                      uint64_t *__restrict__ out, const PrimeC *__restrict__ pc,
                                                      ConstVec cv, int N, int nl, size_t pstride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int row = blockIdx.y, poly = row / nl, i = row - poly * nl;
    const size_t off = (size_t)poly * pstride + (size_t)i * N + c;
    const uint64_t q = pc[i].q;
    uint64_t x = a[off], r;
    if (OP == EW_ADD) r = add_mod(x, b[off], q);
    else if (OP == EW_SUB) r = sub_mod(x, b[off], q);
    else if (OP == EW_NEG) r = x ? q - x : 0;
    else if (OP == EW_MULC) r = csub(shoup(x, cv.c[i], cv.sh[i], q), q);
    else r = poly == 0 ? add_mod(x, cv.c[i], q) : x;
    out[off] = r;
}

void k_add(Ctx &c, const CtObj &a, const CtObj &b, CtObj &out, bool sub)
{
    const int nl = out.level + 1;
    ProfScope _ps(c, "elementwise", (uint64_t)6 * nl);  // limbs moved: 2 x 2nl read, 2nl written
    ConstVec cv{};
    if (sub)
        k_ct_ew<EW_SUB><<<ew_grid(c, 2 * nl), EW_THREADS, 0, c.stream>>>(a.d, b.d, out.d, c.d_pc, cv, c.N, nl,
                                                                         (size_t)(c.L + 1) * c.N);
    else
        k_ct_ew<EW_ADD><<<ew_grid(c, 2 * nl), EW_THREADS, 0, c.stream>>>(a.d, b.d, out.d, c.d_pc, cv, c.N, nl,
                                                                         (size_t)(c.L + 1) * c.N);
    check_launch("k_ct_ew add/sub");
}

void k_neg(Ctx &c, const CtObj &a, CtObj &out)
{
    const int nl = out.level + 1;
    ProfScope _ps(c, "elementwise", (uint64_t)4 * nl);
    ConstVec cv{};
    k_ct_ew<EW_NEG><<<ew_grid(c, 2 * nl), EW_THREADS, 0, c.stream>>>(a.d, nullptr, out.d, c.d_pc, cv, c.N, nl,
                                                                     (size_t)(c.L + 1) * c.N);
    check_launch("k_ct_ew neg");
}

void k_mul_scalar_ct(Ctx &c, const CtObj &a, const ConstVec &cv, CtObj &out)
{
    const int nl = out.level + 1;
    ProfScope _ps(c, "elementwise", (uint64_t)4 * nl);
    k_ct_ew<EW_MULC><<<ew_grid(c, 2 * nl), EW_THREADS, 0, c.stream>>>(a.d, nullptr, out.d, c.d_pc, cv, c.N, nl,
                                                                      (size_t)(c.L + 1) * c.N);
    check_launch("k_ct_ew mulc");
}

void k_add_scalar_c0(Ctx &c, const CtObj &a, const ConstVec &cv, CtObj &out)
{
    const int nl = out.level + 1;
    ProfScope _ps(c, "elementwise", (uint64_t)4 * nl);
    k_ct_ew<EW_ADDC0><<<ew_grid(c, 2 * nl), EW_THREADS, 0, c.stream>>>(a.d, nullptr, out.d, c.d_pc, cv, c.N, nl,
                                                                       (size_t)(c.L + 1) * c.N);
    check_launch("k_ct_ew addc0");
}

__global__ void k_copy_kernel(uint64_t *__restrict__ dst, const uint64_t *__restrict__ src, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < n; i += (size_t)gridDim.x * blockDim.x) dst[i] = src[i];
}

void k_copy(Ctx &c, uint64_t *dst, const uint64_t *src, size_t words)
{
    if (!words) return;
    ProfScope _ps(c, "copy", 2 * words / c.N);
    const size_t blocks = std::min<size_t>((words + 255) / 256, 4096);
    k_copy_kernel<<<(unsigned)blocks, 256, 0, c.stream>>>(dst, src, words);
    check_launch("k_copy");
}

// ---------------------------------------------------------------------------
// tensor product (evaluation domain): d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EW_THREADS) k_tensor_kernel(const uint64_t *__restrict__ a,
                                                              const uint64_t *__restrict__ b,
                                                              uint64_t *__restrict__ d0, uint64_t *__restrict__ d1,
                                                              uint64_t *__restrict__ d2, uint64_t *__restrict__ d2b,
                                                              const PrimeC *__restrict__ pc, int N, size_t pstride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const PrimeC p = pc[i];
    const size_t off = (size_t)i * N + c;
    const uint64_t x0 = a[off], x1 = a[pstride + off], y0 = b[off], y1 = b[pstride + off];
    d0[off] = mul_mod(x0, y0, p);
    const uint64_t v2 = mul_mod(x1, y1, p);
    d2[off] = v2;
    if (d2b) d2b[off] = v2;
    Acc128 acc{0, 0};
    mac(acc, x0, y1);
    mac(acc, x1, y0);
    d1[off] = mont_mul(mont_redc(acc.hi, acc.lo, p.q, p.qinv), p.r2, p.q, p.qinv);
}

void k_tensor2(Ctx &c, const CtObj &a, const CtObj &b, int level, uint64_t *d0, uint64_t *d1, uint64_t *d2,
               uint64_t *d2b)
{
    ProfScope _ps(c, "tensor", (uint64_t)(d2b ? 8 : 7) * (level + 1));
    k_tensor_kernel<<<ew_grid(c, level + 1), EW_THREADS, 0, c.stream>>>(a.d, b.d, d0, d1, d2, d2b, c.d_pc, c.N,
                                                                        (size_t)(c.L + 1) * c.N);
    check_launch("k_tensor");
}

void k_tensor(Ctx &c, const CtObj &a, const CtObj &b, int level, uint64_t *d0, uint64_t *d1, uint64_t *d2)
{
    k_tensor2(c, a, b, level, d0, d1, d2, nullptr);
}

// ---------------------------------------------------------------------------
// ModUp: fast base conversion of each digit (coefficient domain) to Q_l u P.
// ext[j][e][c]: e <= level -> q_e, e > level -> p_{e-level-1}.
// Digit j covers limbs [j alpha, min((j+1) alpha, level+1)); its own rows are
// copied, the others are sum_i [d_i (Q_j/q_i)^-1]_{q_i} (Q_j/q_i) mod t.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(EW_THREADS) k_modup_kernel(const uint64_t *__restrict__ d2,
                                                             uint64_t *__restrict__ ext,
                                                             const uint64_t *__restrict__ ks, DigitOffs offs,
                                                             const PrimeC *__restrict__ pc, int N, int level,
                                                             int alpha, int L, int K, size_t ext_stride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int j = blockIdx.y;
    const int lo = j * alpha, hi = min((j + 1) * alpha, level + 1), a = hi - lo;
    const int E = level + 1 + K;
    const uint64_t *tab = ks + offs.off[j];
    const uint64_t *hinv = tab, *hsh = tab + a, *hM = tab + 2 * a;
    uint64_t y[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        if (i < a) {
            const uint64_t q = pc[lo + i].q;
            y[i] = csub(shoup(d2[(size_t)(lo + i) * N + c], hinv[i], hsh[i], q), q);
        }
    }
    uint64_t *out = ext + (size_t)j * ext_stride + c;
    for (int e = 0; e < E; e++) {
        uint64_t v;
        if (e >= lo && e < hi) {
            v = d2[(size_t)e * N + c];
        } else {
            const int t = e <= level ? e : L + 1 + (e - level - 1);
            const PrimeC pt = pc[t];
            Acc128 acc{0, 0};
#pragma unroll
            for (int i = 0; i < 16; i++)
                if (i < a) mac(acc, y[i], hM[(size_t)i * E + e]);
            v = mont_redc(acc.hi, acc.lo, pt.q, pt.qinv);
        }
        out[(size_t)e * N] = v;
    }
}

void k_modup(Ctx &c, const uint64_t *d2coef, int level, uint64_t *ext)
{
    ProfScope _ps(c, "modup", (uint64_t)(level + 1) + (uint64_t)c.ndigits(level) * (level + 1 + c.K));
    const int nd = c.ndigits(level);
    DigitOffs offs;
    for (int j = 0; j < nd; j++) offs.off[j] = c.modup_off[level][j];
    k_modup_kernel<<<ew_grid(c, nd), EW_THREADS, 0, c.stream>>>(d2coef, ext, c.d_ks, offs, c.d_pc, c.N, level,
                                                                c.alpha, c.L, c.K, c.ext_rows() * c.N);
    check_launch("k_modup");
}

// inner product with the switching key: acc_k[e] = sum_j ext_j[e] * key_j,k[row(e)]
__global__ void __launch_bounds__(EW_THREADS) k_inner_kernel(const uint64_t *__restrict__ ext,
                                                             const uint64_t *__restrict__ key,
                                                             uint64_t *__restrict__ acc,
                                                             const PrimeC *__restrict__ pc, int N, int level, int L,
                                                             int K, int nd, size_t ext_stride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int e = blockIdx.y;
    const int row = e <= level ? e : L + 1 + (e - level - 1);
    const PrimeC p = pc[row];
    const size_t krow = (size_t)(L + 1 + K) * N;  // one key polynomial
    Acc128 a0{0, 0}, a1{0, 0};
    for (int j = 0; j < nd; j++) {
        const uint64_t x = ext[(size_t)j * ext_stride + (size_t)e * N + c];
        const uint64_t *kj = key + (size_t)j * 2 * krow + (size_t)row * N + c;
        mac(a0, x, kj[0]);
        mac(a1, x, kj[krow]);
    }
    acc[(size_t)e * N + c] = mont_redc(a0.hi, a0.lo, p.q, p.qinv);
    acc[ext_stride + (size_t)e * N + c] = mont_redc(a1.hi, a1.lo, p.q, p.qinv);
}

void k_inner_product(Ctx &c, const uint64_t *ext, const Swk &key, int level, uint64_t *acc)
{
    ProfScope _ps(c, "inner_product", (uint64_t)(level + 1 + c.K) * (3 * c.ndigits(level) + 2));
    const int E = level + 1 + c.K;
    k_inner_kernel<<<ew_grid(c, E), EW_THREADS, 0, c.stream>>>(ext, key.d, acc, c.d_pc, c.N, level, c.L, c.K,
                                                               c.ndigits(level), c.ext_rows() * c.N);
    check_launch("k_inner");
}

// ModDown step 1 (coefficient domain): conv_k[i] = sum_m [u_{p_m} (P/p_m)^-1]_{p_m} (P/p_m) mod q_i
__global__ void __launch_bounds__(EW_THREADS) k_moddown_conv_kernel(const uint64_t *__restrict__ acc,
                                                                    uint64_t *__restrict__ conv,
                                                                    const uint64_t *__restrict__ tab,
                                                                    const PrimeC *__restrict__ pc, int N, int level,
                                                                    int L, int K, size_t ext_stride,
                                                                    size_t conv_stride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int k = blockIdx.y;
    const uint64_t *u = acc + (size_t)k * ext_stride + (size_t)(level + 1) * N + c;
    const uint64_t *hinv = tab, *hsh = tab + K, *hM = tab + 2 * K;
    uint64_t y[16];
#pragma unroll
    for (int m = 0; m < 16; m++) {
        if (m < K) {
            const uint64_t pm = pc[L + 1 + m].q;
            y[m] = csub(shoup(u[(size_t)m * N], hinv[m], hsh[m], pm), pm);
        }
    }
    uint64_t *out = conv + (size_t)k * conv_stride + c;
    for (int i = 0; i <= level; i++) {
        const PrimeC p = pc[i];
        Acc128 a{0, 0};
#pragma unroll
        for (int m = 0; m < 16; m++)
            if (m < K) mac(a, y[m], hM[(size_t)m * (L + 1) + i]);
        out[(size_t)i * N] = mont_redc(a.hi, a.lo, p.q, p.qinv);
    }
}

// ModDown step 3 (evaluation domain): out_k[i] = add_k[i] + (acc_k[i] - conv_k[i]) P^-1
__global__ void __launch_bounds__(EW_THREADS) k_moddown_final_kernel(const uint64_t *__restrict__ acc,
                                                                     const uint64_t *__restrict__ conv,
                                                                     const uint64_t *add0, const uint64_t *add1,
                                                                     uint64_t *out0, uint64_t *out1,
                                                                     const PrimeC *__restrict__ pc, ConstVec pinv,
                                                                     int N, int nl, size_t ext_stride,
                                                                     size_t conv_stride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int row = blockIdx.y, k = row / nl, i = row - k * nl;
    const uint64_t q = pc[i].q;
    const size_t o = (size_t)i * N + c;
    uint64_t d = sub_mod(acc[(size_t)k * ext_stride + o], conv[(size_t)k * conv_stride + o], q);
    uint64_t v = csub(shoup(d, pinv.c[i], pinv.sh[i], q), q);
    const uint64_t *add = k == 0 ? add0 : add1;
    uint64_t *out = k == 0 ? out0 : out1;
    if (add) v = add_mod(v, add[o], q);
    out[o] = v;
}

void k_moddown(Ctx &c, uint64_t *acc, int level, const uint64_t *add0, const uint64_t *add1, uint64_t *out0,
               uint64_t *out1)
{
    const size_t es = c.ext_rows() * c.N, cs = (size_t)(c.L + 1) * c.N;
    // P rows of both accumulators to the coefficient domain
    LimbMap mp{acc + (size_t)(level + 1) * c.N, es, c.K, 2, 0, 0, c.L + 1};
    ntt_inv(c, mp);
    {
        ProfScope _ps(c, "moddown_conv", (uint64_t)2 * c.K + 2 * (level + 1));
        k_moddown_conv_kernel<<<ew_grid(c, 2), EW_THREADS, 0, c.stream>>>(acc, c.ws_conv, c.d_ks + c.moddown_off,
                                                                          c.d_pc, c.N, level, c.L, c.K, es, cs);
        check_launch("k_moddown_conv");
    }
    LimbMap mq{c.ws_conv, cs, level + 1, 2, level + 1, 0, 0};
    ntt_fwd(c, mq);
    ProfScope _ps(c, "moddown_final", (uint64_t)8 * (level + 1));
    k_moddown_final_kernel<<<ew_grid(c, 2 * (level + 1)), EW_THREADS, 0, c.stream>>>(
        acc, c.ws_conv, add0, add1, out0, out1, c.d_pc, c.pinv, c.N, level + 1, es, cs);
    check_launch("k_moddown_final");
}

// ---------------------------------------------------------------------------
// rescale: c_i <- (c_i - [c_l]_centred) q_l^-1 mod q_i
// ---------------------------------------------------------------------------
// top limb of both polynomials, times m (Shoup), into a scratch pair of rows
__global__ void __launch_bounds__(EW_THREADS) k_top_copy_kernel(const uint64_t *__restrict__ a,
                                                                uint64_t *__restrict__ top, uint64_t q, uint64_t m,
                                                                uint64_t msh, int N, size_t off0, size_t off1)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int k = blockIdx.y;
    const uint64_t v = a[(k ? off1 : off0) + c];
    top[(size_t)k * N + c] = csub(shoup(v, m, msh, q), q);
}

void k_rescale_mul(Ctx &c, const CtObj &a, const ConstVec *mul, CtObj &out)
{
    const int l = a.level;
    const size_t ps = (size_t)(c.L + 1) * c.N;
    const uint64_t ql = c.primes[l];
    // top limb of c0 and c1 (times m_l) -> scratch rows [0], [1] of ws_d2, to the coefficient domain
    uint64_t *top = c.ws_d2;
    {
        ProfScope _ps(c, "copy", 4);
        const uint64_t m = mul ? mul->c[l] : 1, msh = mul ? mul->sh[l] : h_shoup(1, ql);
        k_top_copy_kernel<<<ew_grid(c, 2), EW_THREADS, 0, c.stream>>>(a.d, top, ql, m, msh, c.N,
                                                                        (size_t)l * c.N, ps + (size_t)l * c.N);
        check_launch("k_top_copy");
    }
    LimbMap mt{top, (size_t)c.N, 1, 2, 1, l, 0};
    ntt_inv(c, mt);
    ConstVec mq;
    for (int i = 0; i < l; i++) {
        const uint64_t qi = c.primes[i];
        mq.c[i] = mul ? h_mulmod(mul->c[i], c.resc[l].c[i], qi) : c.resc[l].c[i];
        mq.sh[i] = h_shoup(mq.c[i], qi);
    }
    // the forward transform of [top]_centred mod q_i fused with its broadcast and the combine
    ks_rescale(c, a, top, c.ws_conv, mq, out);
}

void k_rescale(Ctx &c, const CtObj &a, CtObj &out) { k_rescale_mul(c, a, nullptr, out); }

// ---------------------------------------------------------------------------
// linear combination with integer weights: out = sum_k m_k ct_k (one level)
// ---------------------------------------------------------------------------
// Each thread owns two adjacent words of one limb row and reads them from every
// term with one 16-byte load; the loads of eight terms are issued before their
// products are accumulated, so a warp keeps eight independent requests in flight
// per term group instead of one (the kernel is bound by HBM, 8 (n + 1) bytes a word).
__global__ void __launch_bounds__(EW_THREADS) k_lincomb_kernel(LinArgs args, uint64_t *__restrict__ out,
                                                               const PrimeC *__restrict__ pc, int N, int nl,
                                                               size_t pstride)
{
    constexpr int G = 8;  // terms whose loads are in flight together
    __shared__ uint64_t r[LinArgs::MAXT], rs[LinArgs::MAXT];
    const int row = blockIdx.y, poly = row / nl, i = row - poly * nl;
    const uint64_t q = pc[i].q;
    if (threadIdx.x < args.n) {
        const __int128 v = args.m[threadIdx.x];
        const u128 av = v < 0 ? (u128)(-v) : (u128)v;
        uint64_t rr = (uint64_t)(av % q);
        if (v < 0 && rr) rr = q - rr;
        r[threadIdx.x] = rr;
        rs[threadIdx.x] = (uint64_t)(((u128)rr << 64) / q);
    }
    __syncthreads();
    const int c = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= N) return;
    const size_t o = (size_t)poly * pstride + (size_t)i * N + c;
    uint64_t a0 = 0, a1 = 0;
    for (int k0 = 0; k0 < args.n; k0 += G) {
        ulonglong2 v[G];
#pragma unroll
        for (int j = 0; j < G; j++)
            if (k0 + j < args.n) v[j] = __ldg(reinterpret_cast<const ulonglong2 *>(args.p[k0 + j] + o));
#pragma unroll
        for (int j = 0; j < G; j++)
            if (k0 + j < args.n) {
                const uint64_t w = r[k0 + j], ws = rs[k0 + j];
                a0 = add_mod(a0, csub(shoup(v[j].x, w, ws, q), q), q);
                a1 = add_mod(a1, csub(shoup(v[j].y, w, ws, q), q), q);
            }
    }
    *reinterpret_cast<ulonglong2 *>(out + o) = make_ulonglong2(a0, a1);
}

void k_lincomb(Ctx &c, const LinArgs &args, int level, CtObj &out)
{
    // every ciphertext buffer starts on a 256-byte boundary and its limb rows are
    // whole multiples of N words, so the 16-byte accesses are aligned
    for (int k = 0; k < args.n; k++)
        if ((uintptr_t)args.p[k] % 16) throw_err(PPST_E_ARG, "lin_comb: operand not 16-byte aligned");
    if ((uintptr_t)out.d % 16 || c.N % 2) throw_err(PPST_E_ARG, "lin_comb: output not 16-byte aligned");
    ProfScope _ps(c, "lincomb", (uint64_t)(args.n + 1) * 2 * (level + 1));
    const dim3 grid((c.N / 2 + EW_THREADS - 1) / EW_THREADS, 2 * (level + 1));
    k_lincomb_kernel<<<grid, EW_THREADS, 0, c.stream>>>(args, out.d, c.d_pc, c.N, level + 1, (size_t)(c.L + 1) * c.N);
    check_launch("k_lincomb");
}

// ---------------------------------------------------------------------------
// Galois automorphism X -> X^g in the evaluation domain: a permutation.
// Natural word n holds a(psi^(2 brv(n) + 1)); sigma_g(a) there equals a at
// psi^(g (2 brv(n) + 1)), i.e. natural word brv(((2 brv(n) + 1) g mod 2N - 1) / 2).
// Storage addresses map to natural words by eval_natural / eval_address.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EW_THREADS) k_automorph_kernel(const uint64_t *__restrict__ in,
                                                                 uint64_t *__restrict__ out, int logN, int nl,
                                                                 uint64_t g, size_t pstride)
{
    const int N = 1 << logN;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int row = blockIdx.y, poly = row / nl, i = row - poly * nl;
    const uint32_t n = eval_natural((uint32_t)k, logN);  // storage address -> natural position
    const uint32_t bk = __brev(n) >> (32 - logN);
    const uint64_t e = ((2ull * bk + 1) * g) & (2ull * N - 1);
    const uint32_t src = eval_address(__brev((uint32_t)((e - 1) >> 1)) >> (32 - logN), logN);
    const size_t base = (size_t)poly * pstride + (size_t)i * N;
    out[base + k] = in[base + src];
}

void k_automorph(Ctx &c, const uint64_t *in, int level, uint64_t galois, uint64_t *out, size_t poly_stride, int npoly)
{
    ProfScope _ps(c, "automorph", (uint64_t)2 * npoly * (level + 1));
    k_automorph_kernel<<<ew_grid(c, npoly * (level + 1)), EW_THREADS, 0, c.stream>>>(in, out, c.logN, level + 1,
                                                                                      galois, poly_stride);
    check_launch("k_automorph");
}

// ---------------------------------------------------------------------------
// sampling (ChaCha20 streams, counter-based: one block per 4 or 8 coefficients)
// ---------------------------------------------------------------------------
// uniform residues: coefficient c <- block c/4, words 2r (low), 2r+1 (high), reduced mod q
__global__ void k_uniform_kernel(ChaChaKey key, uint32_t purpose, uint32_t index, LimbMap m,
                                 const PrimeC *__restrict__ pc, int N)
{
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk * 4 >= N) return;
    const int b = blockIdx.y;
    const int p = m.prime(b);
    const uint64_t q = pc[p].q;
    uint32_t o[16];
    chacha20_block(key, (uint32_t)blk, purpose, index, (uint32_t)p, o);
    uint64_t *dst = m.ptr(b, N) + (size_t)blk * 4;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        uint64_t lo = (uint64_t)o[4 * r] | ((uint64_t)o[4 * r + 1] << 32);
        uint64_t hi = (uint64_t)o[4 * r + 2] | ((uint64_t)o[4 * r + 3] << 32);
        u128 v = ((u128)hi << 64) | lo;
        dst[r] = (uint64_t)(v % q);
    }
}

void k_sample_uniform(Ctx &c, uint64_t seed, uint32_t purpose, uint32_t index, const LimbMap &m)
{
    ChaChaKey key = chacha_key_from_seed(seed);
    dim3 grid((c.N / 4 + 127) / 128, m.count());
    k_uniform_kernel<<<grid, 128, 0, c.stream>>>(key, purpose, index, m, c.d_pc, c.N);
    check_launch("k_uniform");
}

// ternary: coefficient c <- word (c mod 8) of block c/8, (w mod 3) - 1
// gaussian: coefficient c <- block c/4, magnitude draw word 2r, sign bit word 2r+1
__global__ void k_small_kernel(ChaChaKey key, uint32_t purpose, uint32_t index, int gauss,
                               const uint64_t *__restrict__ cdt, int bound, int64_t *out, int N)
{
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    const int per = gauss ? 4 : 8;
    if (blk * per >= N) return;
    uint32_t o[16];
    chacha20_block(key, (uint32_t)blk, purpose, index, 0u, o);
    if (!gauss) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            uint64_t w = (uint64_t)o[2 * r] | ((uint64_t)o[2 * r + 1] << 32);
            out[(size_t)blk * 8 + r] = (int64_t)(w % 3) - 1;
        }
    } else {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            uint64_t draw = (uint64_t)o[4 * r] | ((uint64_t)o[4 * r + 1] << 32);
            uint32_t sgn = o[4 * r + 2] & 1u;
            int64_t mag = 0;
            for (int k = 0; k < bound; k++) mag += draw >= cdt[k] ? 1 : 0;
            out[(size_t)blk * 4 + r] = sgn ? -mag : mag;
        }
    }
}

void k_sample_small(Ctx &c, uint64_t seed, uint32_t purpose, uint32_t index, bool gauss, int64_t *out)
{
    ChaChaKey key = chacha_key_from_seed(seed);
    const int per = gauss ? 4 : 8;
    k_small_kernel<<<(c.N / per + 127) / 128, 128, 0, c.stream>>>(key, purpose, index, gauss ? 1 : 0, c.d_cdt,
                                                                   c.gbound, out, c.N);
    check_launch("k_small");
}

// signed 64-bit integers -> residues (coefficient domain)
__global__ void k_small_to_rns_kernel(const int64_t *__restrict__ v, LimbMap m, const PrimeC *__restrict__ pc, int N)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int b = blockIdx.y;
    const PrimeC p = pc[m.prime(b)];
    const int64_t x = v[c];
    const uint64_t ax = x < 0 ? (uint64_t)0 - (uint64_t)x : (uint64_t)x;
    uint64_t r = csub(shoup(ax, 1, p.w64, p.q), p.q);
    if (x < 0 && r) r = p.q - r;
    m.ptr(b, N)[c] = r;
}

void k_small_to_rns(Ctx &c, const int64_t *v, const LimbMap &m)
{
    k_small_to_rns_kernel<<<ew_grid(c, m.count()), EW_THREADS, 0, c.stream>>>(v, m, c.d_pc, c.N);
    check_launch("k_small_to_rns");
}

// ---------------------------------------------------------------------------
// key generation / encryption / decryption combines (evaluation domain)
// ---------------------------------------------------------------------------
// switching-key digit: b = -a s + e + [row in digit] (P mod q_row) s_new; b, a -> Montgomery form
__global__ void k_swk_kernel(uint64_t *b, uint64_t *a, const uint64_t *__restrict__ e, const uint64_t *__restrict__ s,
                             const uint64_t *__restrict__ snew, const PrimeC *__restrict__ pc, ConstVec pm, int N,
                             int lo, int hi)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int row = blockIdx.y;
    const PrimeC p = pc[row];
    const size_t o = (size_t)row * N + c;
    const uint64_t av = a[o];
    uint64_t v = sub_mod(e[o], mul_mod(av, s[o], p), p.q);
    if (row >= lo && row < hi) v = add_mod(v, csub(shoup(snew[o], pm.c[row], pm.sh[row], p.q), p.q), p.q);
    b[o] = mont_mul(v, p.r2, p.q, p.qinv);
    a[o] = mont_mul(av, p.r2, p.q, p.qinv);
}

void k_swk_combine(Ctx &c, uint64_t *b, const uint64_t *a, const uint64_t *e, const uint64_t *s, const uint64_t *snew,
                   int digit_lo, int digit_hi)
{
    k_swk_kernel<<<ew_grid(c, c.np), EW_THREADS, 0, c.stream>>>(b, const_cast<uint64_t *>(a), e, s, snew, c.d_pc,
                                                                 c.pmod[0], c.N, digit_lo, digit_hi);
    check_launch("k_swk");
}

__global__ void k_pk_kernel(uint64_t *b, const uint64_t *__restrict__ a, const uint64_t *__restrict__ e,
                            const uint64_t *__restrict__ s, const PrimeC *__restrict__ pc, int N)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int row = blockIdx.y;
    const PrimeC p = pc[row];
    const size_t o = (size_t)row * N + c;
    b[o] = sub_mod(e[o], mul_mod(a[o], s[o], p), p.q);
}

void k_pk_combine(Ctx &c, uint64_t *b, const uint64_t *a, const uint64_t *e, const uint64_t *s)
{
    k_pk_kernel<<<ew_grid(c, c.L + 1), EW_THREADS, 0, c.stream>>>(b, a, e, s, c.d_pc, c.N);
    check_launch("k_pk");
}

// c0 = u pk0 + e0 + m, c1 = u pk1 + e1
__global__ void k_enc_kernel(const uint64_t *__restrict__ pk, const uint64_t *__restrict__ u,
                             const uint64_t *__restrict__ e0, const uint64_t *__restrict__ e1,
                             const uint64_t *__restrict__ m, uint64_t *out, const PrimeC *__restrict__ pc, int N,
                             size_t pstride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const PrimeC p = pc[i];
    const size_t o = (size_t)i * N + c;
    const uint64_t uv = u[o];
    out[o] = add_mod(add_mod(mul_mod(uv, pk[o], p), e0[o], p.q), m[o], p.q);
    out[pstride + o] = add_mod(mul_mod(uv, pk[pstride + o], p), e1[o], p.q);
}

void k_enc_combine(Ctx &c, const uint64_t *pk, const uint64_t *u, const uint64_t *e0, const uint64_t *e1,
                   const uint64_t *m, CtObj &out)
{
    k_enc_kernel<<<ew_grid(c, c.L + 1), EW_THREADS, 0, c.stream>>>(pk, u, e0, e1, m, out.d, c.d_pc, c.N,
                                                                   (size_t)(c.L + 1) * c.N);
    check_launch("k_enc");
}

__global__ void k_dec_kernel(const uint64_t *__restrict__ ct, const uint64_t *__restrict__ s, uint64_t *m,
                             const PrimeC *__restrict__ pc, int N, size_t pstride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int i = blockIdx.y;
    const PrimeC p = pc[i];
    const size_t o = (size_t)i * N + c;
    m[o] = add_mod(ct[o], mul_mod(ct[pstride + o], s[o], p), p.q);
}

void k_dec_combine(Ctx &c, const CtObj &ct, const uint64_t *s, uint64_t *m)
{
    k_dec_kernel<<<ew_grid(c, ct.level + 1), EW_THREADS, 0, c.stream>>>(ct.d, s, m, c.d_pc, c.N,
                                                                        (size_t)(c.L + 1) * c.N);
    check_launch("k_dec");
}

// in place: to (x 2^64) or from (x 2^-64) the Montgomery form
__global__ void k_mont_kernel(LimbMap m, const PrimeC *__restrict__ pc, int N, int to)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int b = blockIdx.y;
    const PrimeC p = pc[m.prime(b)];
    uint64_t *d = m.ptr(b, N);
    d[c] = to ? mont_mul(d[c], p.r2, p.q, p.qinv) : mont_redc(0, d[c], p.q, p.qinv);
}

void k_to_mont(Ctx &c, uint64_t *d, const LimbMap &m, bool to)
{
    (void)d;
    k_mont_kernel<<<ew_grid(c, m.count()), EW_THREADS, 0, c.stream>>>(m, c.d_pc, c.N, to ? 1 : 0);
    check_launch("k_mont");
}

__global__ void k_sq_kernel(const uint64_t *__restrict__ a, uint64_t *out, LimbMap m, const PrimeC *__restrict__ pc,
                            int N)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int b = blockIdx.y;
    const PrimeC p = pc[m.prime(b)];
    const size_t o = (size_t)(m.ptr(b, N) - m.base) + c;
    out[o] = mul_mod(a[o], a[o], p);
}

void k_pointwise_sq(Ctx &c, const uint64_t *a, uint64_t *out, const LimbMap &m)
{
    k_sq_kernel<<<ew_grid(c, m.count()), EW_THREADS, 0, c.stream>>>(a, out, m, c.d_pc, c.N);
    check_launch("k_sq");
}

}  // namespace ppst
