// ks.cu -- fused hybrid key switching (the HMult and rotation hot path).
//
// Key switching of d (level l, dnum digits of alpha primes, K special primes)
// is computed as three fused stages, none of which writes an evaluation-domain
// digit to HBM:
//   1. inverse NTT of d whose final N^-1 carries (Q_j / q_i)^-1 of the limb's
//      digit: the first factor of ModUp's base conversion comes for free;
//   2. k_modup_cols: for every digit j and target limb e outside it, the load
//      of the COLS transform pass computes the base conversion
//      sum_i y_i (Q_j / q_i) mod t_e on the fly (the digit's alpha limbs stay in
//      L2), then runs the pass;
//   3. k_inner_chunks: one block per (target limb e, 16 chunks) loops over the
//      digits, finishes the transform in registers (the digit's own limbs are
//      taken from d in the evaluation domain instead) and accumulates both key
//      polynomials; the twiddles of prime e are reused by every digit.
// ModDown (and, in HMult, the rescale after it) is fused the same way. For
// limb i < l of the HMult output:
//   out_i = (d_i + acc_i P^-1 - NTT(conv_i P^-1 + [top]_centred mod q_i)) q_l^-1
// which equals ModDown followed by rescale limb for limb (the transform is
// linear mod q_i), so one forward transform replaces two. `top` is limb l of
// the ModDown output in the coefficient domain:
//   top = INTT(d_l + acc_l P^-1) - conv_l P^-1.
// All values are exact residues: results are bit-identical to the unfused
// sequence (tensor, ModUp, NTT, inner product, ModDown, rescale).
#include "ntt.cuh"

namespace ppst {

// ---------------------------------------------------------------------------
// 2. ModUp fused into the COLS pass
// ---------------------------------------------------------------------------
// sum_{i < A} src[i N + pos] f[i] mod q for the E words of this thread (A known at
// compile time: fully unrolled, all loads independent); A = 0: runtime count `a`
template <int A, int E, int T>
__device__ __forceinline__ void bconv_words(uint64_t (&x)[E], const uint64_t *__restrict__ src, const uint64_t *f,
                                            int a, int N, int C, int h, const PrimeC &pt)
{
    if (A > 0) {
        uint64_t fr[A > 0 ? A : 1];
#pragma unroll
        for (int i = 0; i < A; i++) fr[i] = f[i];
#pragma unroll
        for (int k = 0; k < E; k++) {
            const size_t pos = (size_t)(h + T * k) * C;
            Acc128 acc{0, 0};
#pragma unroll
            for (int i = 0; i < A; i++) mac(acc, src[(size_t)i * N + pos], fr[i]);
            x[k] = mont_redc(acc.hi, acc.lo, pt.q, pt.qinv);
        }
    } else {
#pragma unroll
        for (int k = 0; k < E; k++) {
            const size_t pos = (size_t)(h + T * k) * C;
            Acc128 acc{0, 0};
#pragma unroll 1
            for (int i = 0; i < a; i++) mac(acc, src[(size_t)i * N + pos], f[i]);
            x[k] = mont_redc(acc.hi, acc.lo, pt.q, pt.qinv);
        }
    }
}

// calls f(std::integral_constant<int, a>) for the digit sizes with a compiled fast path, else f(0)
template <class F>
void dispatch_a(int a, F &&f)
{
    switch (a) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    default: f(std::integral_constant<int, 0>{}); break;
    }
}

template <int S, int ALPHA>
__global__ void __launch_bounds__(PassShape<S>::THREADS, 2)
    k_modup_cols(const uint64_t *__restrict__ y, uint64_t *__restrict__ ext, const uint64_t *__restrict__ ks,
                 DigitOffs offs, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN, int level,
                 int alpha, int L, int K, size_t ext_stride)
{
    typedef PassShape<S> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN, C = N >> S;
    const int E_ext = level + 1 + K;
    const int j = blockIdx.y / E_ext, e = blockIdx.y - j * E_ext;
    const int lo = j * alpha, hi = min(lo + alpha, level + 1), a = hi - lo;
    if (e >= lo && e < hi) return;  // a digit's own limbs come from d itself (block-uniform)
    const int t = e <= level ? e : L + 1 + (e - level - 1);
    const PrimeC pt = pc[t];
    __shared__ uint64_t f[16];
    if (threadIdx.x < a) f[threadIdx.x] = ks[offs.off[j] + 2 * a + (size_t)threadIdx.x * E_ext + e];
    __syncthreads();
    int h, sub;
    pass_coords<S, true>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    uint64_t x[P::E];
    const uint64_t *yl = y + (size_t)lo * N + g;
    if (ALPHA > 0 && a == ALPHA) bconv_words<ALPHA, P::E, P::T>(x, yl, f, a, N, C, h, pt);
    else bconv_words<0, P::E, P::T>(x, yl, f, a, N, C, h, pt);  // a partial last digit
    cols_fwd_core<S>(x, sm, h, sub, tw + (size_t)t * N, pt.q);
    uint64_t *out = ext + (size_t)j * ext_stride + (size_t)e * N;
#pragma unroll
    for (int k = 0; k < P::E; k++) out[(size_t)(P::E * h + k) * C + g] = x[k];
}

// ---------------------------------------------------------------------------
// 3. CHUNKS pass fused with the key inner product
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(PassShape<S>::THREADS, 1)
    k_inner_chunks(const uint64_t *__restrict__ ext, const uint64_t *__restrict__ d2n, const uint64_t *__restrict__ key,
                   uint64_t *__restrict__ acc, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN,
                   int level, int alpha, int L, int K, int nd, size_t ext_stride)
{
    typedef PassShape<S> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN;
    const int e = blockIdx.y;
    const int row = e <= level ? e : L + 1 + (e - level - 1);
    const PrimeC p = pc[row];
    const Tw *T = tw + (size_t)row * N;
    int h, sub;
    pass_coords<S, false>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    const size_t krow = (size_t)(L + 1 + K) * N;
    const size_t fin = (size_t)g * P::M + P::E * h;  // this thread's E words in the store layout
    uint64_t a0[P::E], a1[P::E];
#pragma unroll
    for (int k = 0; k < P::E; k++) a0[k] = a1[k] = 0;
    for (int j = 0; j < nd; j++) {
        const int lo = j * alpha, hi = min(lo + alpha, level + 1);
        uint64_t x[P::E];
        if (e >= lo && e < hi) {  // block-uniform
            const uint64_t *src = d2n + (size_t)e * N + fin;
#pragma unroll
            for (int k = 0; k < P::E; k += 2) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(src + k);
                x[k] = v.x;
                x[k + 1] = v.y;
            }
        } else {
            const uint64_t *src = ext + (size_t)j * ext_stride + (size_t)e * N + (size_t)g * P::M;
#pragma unroll
            for (int k = 0; k < P::E; k++) x[k] = src[h + P::T * k];
            chunks_fwd_core<S>(x, sm, h, sub, g, N, T, p.q);
#pragma unroll
            for (int k = 0; k < P::E; k++) x[k] = reduce4q(x[k], p.q);
        }
        const uint64_t *k0 = key + (size_t)j * 2 * krow + (size_t)row * N + fin;
        const uint64_t *k1 = k0 + krow;
#pragma unroll
        for (int k = 0; k < P::E; k += 2) {
            const ulonglong2 u = *reinterpret_cast<const ulonglong2 *>(k0 + k);
            const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(k1 + k);
            a0[k] = add_mod(a0[k], mont_mul(x[k], u.x, p.q, p.qinv), p.q);
            a0[k + 1] = add_mod(a0[k + 1], mont_mul(x[k + 1], u.y, p.q, p.qinv), p.q);
            a1[k] = add_mod(a1[k], mont_mul(x[k], v.x, p.q, p.qinv), p.q);
            a1[k + 1] = add_mod(a1[k + 1], mont_mul(x[k + 1], v.y, p.q, p.qinv), p.q);
        }
    }
    uint64_t *o0 = acc + (size_t)e * N + fin, *o1 = o0 + ext_stride;
#pragma unroll
    for (int k = 0; k < P::E; k += 2) {
        *reinterpret_cast<ulonglong2 *>(o0 + k) = make_ulonglong2(a0[k], a0[k + 1]);
        *reinterpret_cast<ulonglong2 *>(o1 + k) = make_ulonglong2(a1[k], a1[k + 1]);
    }
}

// ---------------------------------------------------------------------------
// ModDown (+ rescale)
// ---------------------------------------------------------------------------
// u_k = d_k[l] + acc_k[l] P^-1 (evaluation domain), the top limb before its inverse transform
__global__ void k_md_top_kernel(const uint64_t *__restrict__ d, const uint64_t *__restrict__ acc,
                                uint64_t *__restrict__ top, const PrimeC *__restrict__ pc, Tw pinv, int N, int level,
                                size_t pstride, size_t ext_stride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int k = blockIdx.y;
    const uint64_t q = pc[level].q;
    const size_t o = (size_t)level * N + c;
    const uint64_t v = csub(shoup(acc[(size_t)k * ext_stride + o], pinv.w, pinv.s, q), q);
    top[(size_t)k * N + c] = add_mod(d[(size_t)k * pstride + o], v, q);
}

// top_k -= conv_l(y_k) P^-1 (coefficient domain), y_k = P rows of acc_k after ModDown's first factor
__global__ void k_md_topfix_kernel(const uint64_t *__restrict__ acc, uint64_t *__restrict__ top,
                                   const uint64_t *__restrict__ hMP, const PrimeC *__restrict__ pc, Tw pinv, int N,
                                   int level, int L, int K, size_t ext_stride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int k = blockIdx.y;
    const PrimeC p = pc[level];
    const uint64_t *ym = acc + (size_t)k * ext_stride + (size_t)(level + 1) * N + c;
    Acc128 a{0, 0};
    for (int m = 0; m < K; m++) mac(a, ym[(size_t)m * N], hMP[(size_t)m * (L + 1) + level]);
    const uint64_t conv = mont_redc(a.hi, a.lo, p.q, p.qinv);
    const uint64_t v = csub(shoup(conv, pinv.w, pinv.s, p.q), p.q);
    top[(size_t)k * N + c] = sub_mod(top[(size_t)k * N + c], v, p.q);
}

// COLS pass of z_i = conv_i(y) P^-1 (+ [top]_centred mod q_i when rescaling), limbs i < nl of both polys
template <int S, bool RESC, int KT>
__global__ void __launch_bounds__(PassShape<S>::THREADS, 2)
    k_md_cols(const uint64_t *__restrict__ acc, const uint64_t *__restrict__ top, uint64_t *__restrict__ z,
              const uint64_t *__restrict__ hMP, const MdC *__restrict__ mdc, const PrimeC *__restrict__ pc,
              const Tw *__restrict__ tw, int logN, int level, int nl, int L, int K, size_t ext_stride,
              size_t z_stride)
{
    typedef PassShape<S> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN, C = N >> S;
    const int k = blockIdx.y / nl, i = blockIdx.y - k * nl;
    const PrimeC p = pc[i];
    const MdC mc = mdc[i];
    __shared__ uint64_t f[16];
    if (threadIdx.x < K) f[threadIdx.x] = hMP[(size_t)threadIdx.x * (L + 1) + i];
    __syncthreads();
    const uint64_t ql = pc[level].q;
    int h, sub;
    pass_coords<S, true>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    const uint64_t *ym = acc + (size_t)k * ext_stride + (size_t)(level + 1) * N + g;
    const uint64_t *tk = top + (size_t)k * N + g;
    uint64_t x[P::E];
    bconv_words<KT, P::E, P::T>(x, ym, f, K, N, C, h, p);
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) {
        uint64_t v = csub(shoup(x[kk], mc.pinv.w, mc.pinv.s, p.q), p.q);
        if (RESC) {
            const uint64_t tv = tk[(size_t)(h + P::T * kk) * C];
            uint64_t r = csub(shoup(tv, 1, p.w64, p.q), p.q);
            if (tv > (ql >> 1)) r = sub_mod(r, mc.qmod, p.q);
            v = add_mod(v, r, p.q);
        }
        x[kk] = v;
    }
    cols_fwd_core<S>(x, sm, h, sub, tw + (size_t)i * N, p.q);
    uint64_t *out = z + (size_t)k * z_stride + (size_t)i * N;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) out[(size_t)(P::E * h + kk) * C + g] = x[kk];
}

// CHUNKS pass of z and the output combine:
//   RESC:  out_i = d_i q_l^-1 + acc_i (P^-1 q_l^-1) - Z_i q_l^-1
//   else:  out_i = add_i + acc_i P^-1 - Z_i             (add1 may be null: 0)
template <int S, bool RESC>
__global__ void __launch_bounds__(PassShape<S>::THREADS, 2)
    k_md_chunks(const uint64_t *__restrict__ z, const uint64_t *__restrict__ acc, const uint64_t *add0,
                const uint64_t *add1, uint64_t *out0, uint64_t *out1, const MdC *__restrict__ mdc,
                const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN, int nl, size_t ext_stride,
                size_t z_stride)
{
    typedef PassShape<S> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN;
    const int k = blockIdx.y / nl, i = blockIdx.y - k * nl;
    const PrimeC p = pc[i];
    const MdC mc = mdc[i];
    int h, sub;
    pass_coords<S, false>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    uint64_t x[P::E];
    const uint64_t *src = z + (size_t)k * z_stride + (size_t)i * N + (size_t)g * P::M;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) x[kk] = src[h + P::T * kk];
    chunks_fwd_core<S>(x, sm, h, sub, g, N, tw + (size_t)i * N, p.q);
    const size_t fin = (size_t)i * N + (size_t)g * P::M + P::E * h;
    const uint64_t *ad = k == 0 ? add0 : add1;
    uint64_t *od = k == 0 ? out0 : out1;
    const uint64_t *ak = acc + (size_t)k * ext_stride + fin;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) {
        const uint64_t Z = reduce4q(x[kk], p.q);
        const uint64_t av = ak[kk];
        uint64_t r;
        if (RESC) {
            const uint64_t dv = ad[fin + kk];
            r = csub(shoup(dv, mc.qlinv.w, mc.qlinv.s, p.q), p.q);
            r = add_mod(r, csub(shoup(av, mc.pq.w, mc.pq.s, p.q), p.q), p.q);
            r = sub_mod(r, csub(shoup(Z, mc.qlinv.w, mc.qlinv.s, p.q), p.q), p.q);
        } else {
            r = csub(shoup(av, mc.pinv.w, mc.pinv.s, p.q), p.q);
            if (ad) r = add_mod(r, ad[fin + kk], p.q);
            r = sub_mod(r, Z, p.q);
        }
        od[fin + kk] = r;
    }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static dim3 grid_s(const Ctx &c, int S, int rows) { return dim3((c.N >> S) / 16, rows); }

// stages 1-3: d (limbs 0..level) in the evaluation domain in ws_d2n and (as a
// copy to be transformed) in ws_d2; accumulators to ws_acc
static void ks_modup_inner(Ctx &c, int level, const Swk &key)
{
    const int nd = c.ndigits(level), E_ext = level + 1 + c.K;
    ntt_inv_mul(c, map_poly(c, c.ws_d2, level), c.d_modup_outmul + c.modup_outmul_off[level]);
    DigitOffs offs;
    for (int j = 0; j < nd; j++) offs.off[j] = c.modup_off[level][j];
    const size_t es = c.ext_rows() * c.N;
    {
        uint64_t targets = 0;
        for (int j = 0; j < nd; j++) targets += E_ext - (std::min((j + 1) * c.alpha, level + 1) - j * c.alpha);
        ProfScope _ps(c, "modup_cols", (uint64_t)(level + 1) + targets);  // limbs moved: d read once, targets written
        dispatch_s(ntt_s_rows(c.logN), [&](auto sv) {
            constexpr int S = decltype(sv)::value;
            dispatch_a(c.alpha, [&](auto av) {
                constexpr int A = decltype(av)::value;
                k_modup_cols<S, A><<<grid_s(c, S, nd * E_ext), PassShape<S>::THREADS, 0, c.stream>>>(
                    c.ws_d2, c.ws_ext, c.d_ks, offs, c.d_pc, c.d_twf, c.logN, level, c.alpha, c.L, c.K, es);
            });
        });
        check_launch("k_modup_cols");
    }
    // per target limb: one digit word and two key words per digit read, two accumulators written
    ProfScope _ps(c, "inner_chunks", (uint64_t)E_ext * (3 * nd + 2));
    dispatch_s(ntt_s_chunk(c.logN), [&](auto sv) {
        constexpr int S = decltype(sv)::value;
        k_inner_chunks<S><<<grid_s(c, S, E_ext), PassShape<S>::THREADS, 0, c.stream>>>(
            c.ws_ext, c.ws_d2n, key.d, c.ws_acc, c.d_pc, c.d_twf, c.logN, level, c.alpha, c.L, c.K, nd, es);
    });
    check_launch("k_inner_chunks");
}

// ModDown of ws_acc (+ rescale). RESC: out (level-1) = rescale(d + ModDown(acc)),
// d = the tensor product; else out0 = add0 + ModDown(acc_0), out1 = ModDown(acc_1).
template <bool RESC>
static void ks_moddown(Ctx &c, int level, const uint64_t *d, const uint64_t *add0, uint64_t *out0, uint64_t *out1)
{
    const size_t es = c.ext_rows() * c.N, ps = (size_t)(c.L + 1) * c.N;
    const int nl = RESC ? level : level + 1;
    const MdC *mdc = c.d_md_const + (size_t)level * (c.L + 1);
    const MdC &hm = c.md_const[(size_t)level * (c.L + 1) + level];
    uint64_t *top = c.ws_d2;  // [2][N], free once ModUp has run
    if (RESC) {
        ProfScope _ps(c, "moddown_top", 6);
        k_md_top_kernel<<<dim3(c.N / 256, 2), 256, 0, c.stream>>>(d, c.ws_acc, top, c.d_pc, hm.pinv, c.N, level, ps,
                                                                   es);
        check_launch("k_md_top");
    }
    // P rows of both accumulators to the coefficient domain, times (P / p_m)^-1
    LimbMap mp{c.ws_acc + (size_t)(level + 1) * c.N, es, c.K, 2, 0, 0, c.L + 1};
    ntt_inv_mul(c, mp, c.d_md_outmul);
    const uint64_t *hMP = c.d_ks + c.moddown_off + 2 * c.K;
    if (RESC) {
        LimbMap mt{top, (size_t)c.N, 1, 2, 1, level, 0};
        ntt_inv(c, mt);
        ProfScope _ps(c, "moddown_top", (uint64_t)2 * c.K + 4);
        k_md_topfix_kernel<<<dim3(c.N / 256, 2), 256, 0, c.stream>>>(c.ws_acc, top, hMP, c.d_pc, hm.pinv, c.N, level,
                                                                      c.L, c.K, es);
        check_launch("k_md_topfix");
    }
    {
        ProfScope _ps(c, "moddown_cols", (uint64_t)2 * c.K + (RESC ? 2 : 0) + 2 * nl);
        dispatch_s(ntt_s_rows(c.logN), [&](auto sv) {
            constexpr int S = decltype(sv)::value;
            dispatch_a(c.K, [&](auto kv) {
                constexpr int KT = decltype(kv)::value;
                k_md_cols<S, RESC, KT><<<grid_s(c, S, 2 * nl), PassShape<S>::THREADS, 0, c.stream>>>(
                    c.ws_acc, top, c.ws_conv, hMP, mdc, c.d_pc, c.d_twf, c.logN, level, nl, c.L, c.K, es, ps);
            });
        });
        check_launch("k_md_cols");
    }
    ProfScope _ps(c, "moddown_chunks", (uint64_t)(RESC ? 8 : 7) * nl);
    dispatch_s(ntt_s_chunk(c.logN), [&](auto sv) {
        constexpr int S = decltype(sv)::value;
        const uint64_t *a0 = RESC ? d : add0;
        const uint64_t *a1 = RESC ? d + ps : nullptr;
        k_md_chunks<S, RESC><<<grid_s(c, S, 2 * nl), PassShape<S>::THREADS, 0, c.stream>>>(
            c.ws_conv, c.ws_acc, a0, a1, out0, out1, mdc, c.d_pc, c.d_twf, c.logN, nl, es, ps);
    });
    check_launch("k_md_chunks");
}

// HMult: tensor -> key switch of d2 -> add -> rescale, fused as above
CtObj *ev_hmult(Ctx &c, const EvkObj &k, const CtObj &a, const CtObj &b)
{
    const int lv = std::min(a.level, b.level);
    if (lv < 1) throw_err(PPST_E_DEPTH, "hmult at level 0");
    if (!k.relin.d) throw_err(PPST_E_STATE, "no relinearisation key");
    ensure_workspace(c);
    CtObj *t = ct_new(c, lv, a.scale * b.scale);
    CtObj *o = nullptr;
    try {
        k_tensor2(c, a, b, lv, t->c0(), t->c1(), c.ws_d2n, c.ws_d2);
        ks_modup_inner(c, lv, k.relin);
        o = ct_new(c, lv - 1, (a.scale * b.scale) / (double)c.primes[lv]);
        ks_moddown<true>(c, lv, t->d, nullptr, o->c0(), o->c1());
    } catch (...) {
        ct_free(t);
        ct_free(o);
        throw;
    }
    ct_free(t);
    return o;
}

// Rot(r): automorphism of (c0, c1), key switch of the rotated c1
CtObj *ev_rotate(Ctx &c, const EvkObj &k, const CtObj &a, int r)
{
    const int rr = ((r % c.S) + c.S) % c.S;
    if (rr == 0) return ct_clone(a);
    auto it = k.rot.find(rr);
    if (it == k.rot.end()) throw_err(PPST_E_STATE, "no Galois key for rotation " + std::to_string(rr));
    ensure_workspace(c);
    const size_t ps = (size_t)(c.L + 1) * c.N;
    CtObj *o = ct_new(c, a.level, a.scale);
    try {
        // sigma(c0) -> o.c0; sigma(c1) -> ws_d2n, from which ws_d2 is copied
        k_automorph(c, a.d, a.level, galois_elt(c, rr), o->d, ps, 1);
        k_automorph(c, a.d + ps, a.level, galois_elt(c, rr), c.ws_d2n, ps, 1);
        k_copy(c, c.ws_d2, c.ws_d2n, (size_t)(a.level + 1) * c.N);
        ks_modup_inner(c, a.level, it->second);
        ks_moddown<false>(c, a.level, nullptr, o->c0(), o->c0(), o->c1());
    } catch (...) {
        ct_free(o);
        throw;
    }
    return o;
}

}  // namespace ppst
