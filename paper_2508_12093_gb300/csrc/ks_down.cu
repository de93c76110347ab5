// ks_down.cu -- ModDown fused with the rescale, and the rescale after Mul(P)
// (the second half of the key switch; the scheme is described in ks.cu).
#include "ks.cuh"

namespace ppst {

// ---------------------------------------------------------------------------
// ModDown (+ rescale)
// ---------------------------------------------------------------------------
// u_k = d_k[l] + acc_k[l] P^-1 (evaluation domain), the top limb before its inverse transform
__global__ void k_md_top_kernel(ItemPtrs ip, uint64_t *__restrict__ acc, const PrimeC *__restrict__ pc, Tw pinv,
                                int N, int level, size_t pstride, size_t ext_stride, Ws ws)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int it = blockIdx.y / 2, k = blockIdx.y - 2 * it;
    const uint64_t q = pc[level].q;
    const size_t o = (size_t)level * N + c;
    uint64_t *a = acc + it * ws.acc + (size_t)k * ext_stride + o;
    const uint64_t v = csub(shoup(*a, pinv.w, pinv.s, q), q);
    *a = add_mod(ip.in0[it][(size_t)k * pstride + o], v, q);  // in place: row l of acc_k is not needed otherwise
}

// top_k = INTT(u_k) - conv_l(y_k) P^-1 (coefficient domain): INTT(u_k) is row l of acc_k, y_k its P rows
// after ModDown's first factor
__global__ void k_md_topfix_kernel(const uint64_t *__restrict__ acc, uint64_t *__restrict__ top,
                                   const uint64_t *__restrict__ hMP, const PrimeC *__restrict__ pc, Tw pinv, int N,
                                   int level, int L, int K, size_t ext_stride, Ws ws)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int it = blockIdx.y / 2, k = blockIdx.y - 2 * it;
    const PrimeC p = pc[level];
    const uint64_t *ym = acc + it * ws.acc + (size_t)k * ext_stride + (size_t)(level + 1) * N + c;
    Acc128 a{0, 0};
    for (int m = 0; m < K; m++) mac(a, ym[(size_t)m * N], hMP[(size_t)m * (L + 1) + level]);
    const uint64_t conv = mont_redc(a.hi, a.lo, p.q, p.qinv);
    const uint64_t v = csub(shoup(conv, pinv.w, pinv.s, p.q), p.q);
    const uint64_t u = acc[it * ws.acc + (size_t)k * ext_stride + (size_t)level * N + c];
    top[it * ws.top + (size_t)k * N + c] = sub_mod(u, v, p.q);
}

// COLS pass of z_i = conv_i(y) P^-1 (+ [top]_centred mod q_i when rescaling), limbs i < nl of both polys
template <int S, bool RESC, int KT, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, 2)
    k_md_cols(const uint64_t *__restrict__ acc, const uint64_t *__restrict__ top, uint64_t *__restrict__ z,
              const uint64_t *__restrict__ hMP, const MdC *__restrict__ mdc, const PrimeC *__restrict__ pc,
              const Tw *__restrict__ tw, int logN, int level, int nl, int L, int K, size_t ext_stride,
              size_t z_stride, Ws ws)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN, C = N >> S;
    const int it = blockIdx.y / (2 * nl), rem = blockIdx.y - it * 2 * nl;
    const int k = rem / nl, i = rem - k * nl;
    const PrimeC p = pc[i];
    const MdC mc = mdc[i];
    __shared__ uint64_t f[16];
    if (threadIdx.x < K) f[threadIdx.x] = hMP[(size_t)threadIdx.x * (L + 1) + i];
    __syncthreads();
    const uint64_t ql = pc[level].q;
    int h, sub;
    pass_coords<S, true, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    const uint64_t *ym = acc + it * ws.acc + (size_t)k * ext_stride + (size_t)(level + 1) * N + g;
    const uint64_t *tk = top + it * ws.top + (size_t)k * N + g;
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
    cols_fwd_core<S, SUB>(x, sm, h, sub, tw + (size_t)i * N, p.q);
    uint64_t *out = z + it * ws.conv + (size_t)k * z_stride + (size_t)i * N;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) out[(size_t)(P::E * h + kk) * C + g] = x[kk];
}

// CHUNKS pass of z and the output combine:
//   RESC:  out_i = d_i q_l^-1 + acc_i (P^-1 q_l^-1) - Z_i q_l^-1     (d = in0[item])
//   else:  out_i = add_i + acc_i P^-1 - Z_i        (add = in0[item] for c0, 0 for c1)
// The block's acc and d tiles (contiguous SUB M words each) are fetched by bulk
// asynchronous copies issued at the start, so they arrive while z is transformed.
template <int S, int SUB>
struct MdSmem {
    typedef PassShape<S, SUB> P;
    static constexpr int TILE = P::SUB * P::M;
    static constexpr size_t A_OFF = 128;                           // acc tile
    static constexpr size_t D_OFF = A_OFF + (size_t)TILE * 8;      // d tile
    static constexpr size_t T_OFF = D_OFF + (size_t)TILE * 8;      // transpose buffer
    static constexpr size_t BYTES = T_OFF + (size_t)P::SMEM_WORDS * 8;
};

template <int S, bool RESC, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, 2)
    k_md_chunks(const uint64_t *__restrict__ z, const uint64_t *__restrict__ acc, ItemPtrs ip,
                const MdC *__restrict__ mdc, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN, int nl,
                size_t ext_stride, size_t z_stride, size_t pstride, Ws ws, int *err)
{
    typedef PassShape<S, SUB> P;
    typedef MdSmem<S, SUB> SM;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    const uint64_t *at = reinterpret_cast<const uint64_t *>(smem + SM::A_OFF);
    const uint64_t *dt = reinterpret_cast<const uint64_t *>(smem + SM::D_OFF);
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem + SM::T_OFF);
    constexpr uint32_t TB = SM::TILE * 8;
    const int N = 1 << logN;
    const int it = blockIdx.y / (2 * nl), rem = blockIdx.y - it * 2 * nl;
    const int k = rem / nl, i = rem - k * nl;
    const PrimeC p = pc[i];
    const MdC mc = mdc[i];
    const size_t t0 = (size_t)i * N + (size_t)blockIdx.x * SM::TILE;  // the block's tile in a polynomial
    const uint64_t *ad = (RESC || k == 0) ? ip.in0[it] + (size_t)k * pstride : nullptr;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_fence_init();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[0], ad ? 2 * TB : TB);
        bulk_g2s(smem + SM::A_OFF, acc + it * ws.acc + (size_t)k * ext_stride + t0, TB, &bar[0]);
        if (ad) bulk_g2s(smem + SM::D_OFF, ad + t0, TB, &bar[0]);
    }
    __syncthreads();
    int h, sub;
    pass_coords<S, false, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    const int w0 = sub * P::M + h;  // this thread's words of a tile: w0 + T kk (natural E h + kk)
    uint64_t x[P::E];
    const uint64_t *src = z + it * ws.conv + (size_t)k * z_stride + t0 + w0;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) x[kk] = src[P::T * kk];
    chunks_fwd_core<S>(x, sm, h, sub, g, N, tw + (size_t)i * N, p.q);
    if (__syncthreads_or(!mbar_wait(&bar[0], 0))) {  // the tiles did not arrive in time
        if (threadIdx.x == 0) {
            *(volatile int *)err = 1;
            mbar_wait(&bar[0], 0);
        }
        return;
    }
    uint64_t *od = ip.out[it] + (size_t)k * pstride + t0 + w0;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) {
        const uint64_t Z = reduce4q(x[kk], p.q);
        const uint64_t av = at[w0 + P::T * kk];
        uint64_t r;
        if (RESC) {
            const uint64_t dv = dt[w0 + P::T * kk];
            r = csub(shoup(dv, mc.qlinv.w, mc.qlinv.s, p.q), p.q);
            r = add_mod(r, csub(shoup(av, mc.pq.w, mc.pq.s, p.q), p.q), p.q);
            r = sub_mod(r, csub(shoup(Z, mc.qlinv.w, mc.qlinv.s, p.q), p.q), p.q);
        } else {
            r = csub(shoup(av, mc.pinv.w, mc.pinv.s, p.q), p.q);
            if (ad) r = add_mod(r, dt[w0 + P::T * kk], p.q);
            r = sub_mod(r, Z, p.q);
        }
        od[P::T * kk] = r;
    }
}

// the same pass with 8 words per thread (N = 2^15, 2^16): one warp per 256-point
// chunk, SUB chunks per block; z is read in natural order (words h + 32 k), the
// tiles of acc and d and the output in the evaluation domain's storage order
template <int SUB>
struct Md8Smem {
    static constexpr int TILE = SUB * 256;
    static constexpr size_t A_OFF = 128;                           // acc tile
    static constexpr size_t D_OFF = A_OFF + (size_t)TILE * 8;      // d tile
    static constexpr size_t X_OFF = D_OFF + (size_t)TILE * 8;      // exchange buffers
    static constexpr size_t BYTES = X_OFF + (size_t)TILE * 8;
};

template <bool RESC, int SUB>
__global__ void __launch_bounds__(32 * SUB, SUB == 8 ? 3 : 6)
    k_md_chunks8(const uint64_t *__restrict__ z, const uint64_t *__restrict__ acc, ItemPtrs ip,
                 const MdC *__restrict__ mdc, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN,
                 int nl, size_t ext_stride, size_t z_stride, size_t pstride, Ws ws, int *err)
{
    typedef Md8Smem<SUB> SM;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    const uint64_t *at = reinterpret_cast<const uint64_t *>(smem + SM::A_OFF);
    const uint64_t *dt = reinterpret_cast<const uint64_t *>(smem + SM::D_OFF);
    constexpr uint32_t TB = SM::TILE * 8;
    const int N = 1 << logN;
    const int it = blockIdx.y / (2 * nl), rem = blockIdx.y - it * 2 * nl;
    const int k = rem / nl, i = rem - k * nl;
    const PrimeC p = pc[i];
    const MdC mc = mdc[i];
    const size_t t0 = (size_t)i * N + (size_t)blockIdx.x * SM::TILE;  // the block's tile in a polynomial
    const uint64_t *ad = (RESC || k == 0) ? ip.in0[it] + (size_t)k * pstride : nullptr;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_fence_init();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[0], ad ? 2 * TB : TB);
        bulk_g2s(smem + SM::A_OFF, acc + it * ws.acc + (size_t)k * ext_stride + t0, TB, &bar[0]);
        if (ad) bulk_g2s(smem + SM::D_OFF, ad + t0, TB, &bar[0]);
    }
    __syncthreads();
    const int h = threadIdx.x & 31, sub = threadIdx.x >> 5;
    const int g = blockIdx.x * SUB + sub;
    uint64_t *ex = reinterpret_cast<uint64_t *>(smem + SM::X_OFF) + sub * 256;
    uint64_t x[8];
    const uint64_t *src = z + it * ws.conv + (size_t)k * z_stride + t0 + sub * 256 + h;
#pragma unroll
    for (int kk = 0; kk < 8; kk++) x[kk] = src[32 * kk];
    const Tw *T = tw + (size_t)i * N;
    chunks_fwd_core8<false>(x, ex, h, [&](int m, int j) { return ldtw(T + (size_t)m * ((N >> 8) + g) + j); },
                            p.q);
    if (__syncthreads_or(!mbar_wait(&bar[0], 0))) {  // the tiles did not arrive in time
        if (threadIdx.x == 0) {
            *(volatile int *)err = 1;
            mbar_wait(&bar[0], 0);
        }
        return;
    }
    uint64_t *od = ip.out[it] + (size_t)k * pstride + t0;
#pragma unroll
    for (int kk = 0; kk < 8; kk++) {
        const int a = sub * 256 + addr16(8 * h + kk);  // storage address of natural word 8 h + kk
        const uint64_t Z = reduce4q(x[kk], p.q);
        const uint64_t av = at[a];
        uint64_t r;
        if (RESC) {
            const uint64_t dv = dt[a];
            r = csub(shoup(dv, mc.qlinv.w, mc.qlinv.s, p.q), p.q);
            r = add_mod(r, csub(shoup(av, mc.pq.w, mc.pq.s, p.q), p.q), p.q);
            r = sub_mod(r, csub(shoup(Z, mc.qlinv.w, mc.qlinv.s, p.q), p.q), p.q);
        } else {
            r = csub(shoup(av, mc.pinv.w, mc.pinv.s, p.q), p.q);
            if (ad) r = add_mod(r, dt[a], p.q);
            r = sub_mod(r, Z, p.q);
        }
        od[a] = r;
    }
}

// ---------------------------------------------------------------------------
// rescale after Mul(P) (Sec. 3.1 levels): out_i = c_i m_i q_l^-1 - NTT([c_l]_centred mod q_i) q_l^-1
// ---------------------------------------------------------------------------
// COLS pass of [top]_centred mod q_i (top = limb l in the coefficient domain, L2-resident)
template <int S, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, 2)
    k_resc_cols(const uint64_t *__restrict__ top, uint64_t *__restrict__ z, const PrimeC *__restrict__ pc,
                ConstVec qmod, const Tw *__restrict__ tw, int logN, int level, size_t z_stride)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN, C = N >> S;
    const int k = blockIdx.y / level, i = blockIdx.y - k * level;
    const PrimeC p = pc[i];
    const uint64_t ql = pc[level].q;
    int h, sub;
    pass_coords<S, true, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    const uint64_t *tk = top + (size_t)k * N + g;
    uint64_t x[P::E];
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) {
        const uint64_t v = tk[(size_t)(h + P::T * kk) * C];
        uint64_t r = csub(shoup(v, 1, p.w64, p.q), p.q);  // v mod q_i
        if (v > (ql >> 1)) r = sub_mod(r, qmod.c[i], p.q);  // centred: v - q_l
        x[kk] = r;
    }
    cols_fwd_core<S, SUB>(x, sm, h, sub, tw + (size_t)i * N, p.q);
    uint64_t *out = z + (size_t)k * z_stride + (size_t)i * N;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) out[(size_t)(P::E * h + kk) * C + g] = x[kk];
}

// CHUNKS pass of z and the combine; the block's tile of c is fetched by a bulk
// asynchronous copy while z is transformed
template <int S, int SUB>
struct RescSmem {
    typedef PassShape<S, SUB> P;
    static constexpr int TILE = P::SUB * P::M;
    static constexpr size_t A_OFF = 128;
    static constexpr size_t T_OFF = A_OFF + (size_t)TILE * 8;
    static constexpr size_t BYTES = T_OFF + (size_t)P::SMEM_WORDS * 8;
};

template <int S, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, 2)
    k_resc_chunks(const uint64_t *__restrict__ z, const uint64_t *__restrict__ a, uint64_t *__restrict__ out,
                  const PrimeC *__restrict__ pc, ConstVec qlinv, ConstVec mq, const Tw *__restrict__ tw, int logN,
                  int level, size_t z_stride, size_t pstride, int *err)
{
    typedef PassShape<S, SUB> P;
    typedef RescSmem<S, SUB> SM;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    const uint64_t *at = reinterpret_cast<const uint64_t *>(smem + SM::A_OFF);
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem + SM::T_OFF);
    const int N = 1 << logN;
    const int k = blockIdx.y / level, i = blockIdx.y - k * level;
    const uint64_t q = pc[i].q;
    const size_t t0 = (size_t)i * N + (size_t)blockIdx.x * SM::TILE;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_fence_init();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[0], SM::TILE * 8);
        bulk_g2s(smem + SM::A_OFF, a + (size_t)k * pstride + t0, SM::TILE * 8, &bar[0]);
    }
    __syncthreads();
    int h, sub;
    pass_coords<S, false, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    const int w0 = sub * P::M + h;
    uint64_t x[P::E];
    const uint64_t *src = z + (size_t)k * z_stride + t0 + w0;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) x[kk] = src[P::T * kk];
    chunks_fwd_core<S>(x, sm, h, sub, g, N, tw + (size_t)i * N, q);
    if (__syncthreads_or(!mbar_wait(&bar[0], 0))) {  // the tile did not arrive in time
        if (threadIdx.x == 0) {
            *(volatile int *)err = 1;
            mbar_wait(&bar[0], 0);
        }
        return;
    }
    uint64_t *od = out + (size_t)k * pstride + t0 + w0;
#pragma unroll
    for (int kk = 0; kk < P::E; kk++) {
        const uint64_t Z = reduce4q(x[kk], q);
        const uint64_t xv = csub(shoup(at[w0 + P::T * kk], mq.c[i], mq.sh[i], q), q);
        const uint64_t yv = csub(shoup(Z, qlinv.c[i], qlinv.sh[i], q), q);
        od[P::T * kk] = sub_mod(xv, yv, q);
    }
}

// top: limb l of both polynomials in the coefficient domain ([2][N]); z: scratch [2][L+1][N]
void ks_rescale(Ctx &c, const CtObj &a, const uint64_t *top, uint64_t *z, const ConstVec &mq, CtObj &out)
{
    const int l = a.level;
    const size_t ps = (size_t)(c.L + 1) * c.N;
    {
        ProfScope _ps(c, "rescale_cols", (uint64_t)2 * l + 2);
        dispatch_pass(c, ntt_s_rows(c.logN), 2 * l, [&](auto sv, auto bv) {
            constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
            launch_on(c, k_resc_cols<S, SUB>, grid_s(c, S, SUB, 2 * l), PassShape<S, SUB>::THREADS, 0, top, z,
                c.d_pc, c.resc_qmodv[l], c.d_twf, c.logN, l, ps);
        });
        check_launch("k_resc_cols");
    }
    ProfScope _ps(c, "rescale_chunks", (uint64_t)6 * l);
    dispatch_pass(c, ntt_s_chunk(c.logN), 2 * l, [&](auto sv, auto bv) {
        constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
        const size_t smem = RescSmem<S, SUB>::BYTES;
        static std::atomic<bool> attr_set{false};
        if (!attr_set.load()) {
            PPST_CUDA(cudaFuncSetAttribute(k_resc_chunks<S, SUB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
            attr_set = true;
        }
        launch_on(c, k_resc_chunks<S, SUB>, grid_s(c, S, SUB, 2 * l), PassShape<S, SUB>::THREADS, smem, z, a.d,
            out.d, c.d_pc, c.resc[l], mq, c.d_twf, c.logN, l, ps, ps, c.d_err);
    });
    check_launch("k_resc_chunks");
}

// ModDown of ws_acc (+ rescale) for B items. RESC: out[b] (level-1) =
// rescale(in0[b] + ModDown(acc[b])), in0 = the tensor product; else out[b].c0 =
// in0[b] + ModDown(acc_0), out[b].c1 = ModDown(acc_1).
// first_pass_done: the inner product has already formed u (HMult) and run the first
// inverse pass on the rows ModDown transforms, so only their COLS pass is left.
template <bool RESC>
void ks_moddown(Ctx &c, int level, int B, const ItemPtrs &ip, bool first_pass_done)
{
    const Ws ws = ws_strides(c);
    const size_t es = c.ext_rows() * c.N, ps = (size_t)(c.L + 1) * c.N;
    const int nl = RESC ? level : level + 1;
    const MdC *mdc = c.d_md_const + (size_t)level * (c.L + 1);
    const MdC &hm = c.md_const[(size_t)level * (c.L + 1) + level];
    const dim3 eg(c.N / 256, 2 * B);
    if (RESC) {
        ProfScope _ps(c, "moddown_top", (uint64_t)6 * B);
        if (!first_pass_done) {
            launch_on(c, k_md_top_kernel, eg, 256, 0, ip, c.ws_acc, c.d_pc, hm.pinv, c.N, level, ps, es, ws);
            check_launch("k_md_top");
        }
        // rows l .. l + K of both accumulators of every item (the top limb u_k, then
        // the P rows) to the coefficient domain in one transform: row l times N^-1,
        // P row m times N^-1 (P / p_m)^-1
        LimbMap mp{c.ws_acc + (size_t)level * c.N, es, c.K + 1, 2 * B, 1, level, c.L + 1};
        if (first_pass_done) ntt_inv_cols_mul(c, mp, c.d_md_outmul_top + (size_t)level * (c.K + 1));
        else ntt_inv_mul(c, mp, c.d_md_outmul_top + (size_t)level * (c.K + 1));
    } else {
        // P rows of both accumulators of every item to the coefficient domain, times (P / p_m)^-1
        LimbMap mp{c.ws_acc + (size_t)(level + 1) * c.N, es, c.K, 2 * B, 0, 0, c.L + 1};
        if (first_pass_done) ntt_inv_cols_mul(c, mp, c.d_md_outmul);
        else ntt_inv_mul(c, mp, c.d_md_outmul);
    }
    const uint64_t *hMP = c.d_ks + c.moddown_off + 2 * c.K;
    if (RESC) {
        ProfScope _ps(c, "moddown_top", (uint64_t)B * (2 * c.K + 4));
        launch_on(c, k_md_topfix_kernel, eg, 256, 0, c.ws_acc, c.ws_top, hMP, c.d_pc, hm.pinv, c.N, level, c.L, c.K,
                                                      es, ws);
        check_launch("k_md_topfix");
    }
    {
        ProfScope _ps(c, "moddown_cols", (uint64_t)B * (2 * c.K + (RESC ? 2 : 0) + 2 * nl));
        dispatch_pass(c, ntt_s_rows(c.logN), B * 2 * nl, [&](auto sv, auto bv) {
            constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
            dispatch_a(c.K, [&](auto kv) {
                constexpr int KT = decltype(kv)::value;
                launch_on(c, k_md_cols<S, RESC, KT, SUB>, grid_s(c, S, SUB, B * 2 * nl), PassShape<S, SUB>::THREADS,
                    0, c.ws_acc, c.ws_top, c.ws_conv, hMP, mdc, c.d_pc, c.d_twf, c.logN, level, nl, c.L, c.K, es,
                    ps, ws);
            });
        });
        check_launch("k_md_cols");
    }
    ProfScope _ps(c, "moddown_chunks", (uint64_t)B * (RESC ? 8 : 7) * nl, (uint64_t)B * 2 * nl);  // writes out
    if (ntt_s_chunk(c.logN) == 8 && c.md_words == 8) {  // 8 words per thread, tiles of 8 or 4 chunks
        auto launch8 = [&](auto bv) {
            constexpr int SUB = decltype(bv)::value;
            const size_t smem = Md8Smem<SUB>::BYTES;
            static std::atomic<bool> attr_set{false};
            if (!attr_set.load()) {
                PPST_CUDA(cudaFuncSetAttribute(k_md_chunks8<RESC, SUB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
                attr_set = true;
            }
            launch_on(c, k_md_chunks8<RESC, SUB>, dim3(c.N / Md8Smem<SUB>::TILE, B * 2 * nl), 32 * SUB, smem,
                c.ws_conv, c.ws_acc, ip, mdc, c.d_pc, c.d_twf, c.logN, nl, es, ps, ps, ws, c.d_err);
        };
        if (pass_sub(c, 8, B * 2 * nl) >= 16) launch8(std::integral_constant<int, 8>{});
        else launch8(std::integral_constant<int, 4>{});
        check_launch("k_md_chunks8");
        return;
    }
    dispatch_pass(c, ntt_s_chunk(c.logN), B * 2 * nl, [&](auto sv, auto bv) {
        constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
        const size_t smem = MdSmem<S, SUB>::BYTES;
        static std::atomic<bool> attr_set{false};
        if (!attr_set.load()) {
            PPST_CUDA(cudaFuncSetAttribute(k_md_chunks<S, RESC, SUB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
            attr_set = true;
        }
        launch_on(c, k_md_chunks<S, RESC, SUB>, grid_s(c, S, SUB, B * 2 * nl), PassShape<S, SUB>::THREADS, smem,
            c.ws_conv, c.ws_acc, ip, mdc, c.d_pc, c.d_twf, c.logN, nl, es, ps, ps, ws, c.d_err);
    });
    check_launch("k_md_chunks");
}


template void ks_moddown<true>(Ctx &, int, int, const ItemPtrs &, bool);
template void ks_moddown<false>(Ctx &, int, int, const ItemPtrs &, bool);

}  // namespace ppst
