// ntt.cu -- limb-batched negacyclic NTT / inverse NTT for sm_103a.
//
// The transform evaluates a polynomial of Z_q[X]/(X^N + 1) at the odd powers
// of a primitive 2N-th root of unity psi: output word k holds
// a(psi^(2 brv(k) + 1)) (bit-reversed order). Forward: Cooley-Tukey with
// merged psi powers (twiddle of stage m, group i = psi^brv(m + i)); inverse:
// Gentleman-Sande with psi^-1 powers, then N^-1.
//
// Two passes over HBM per transform. N = R * C with R = 2^ceil(logN/2)
// "rows" and C = N / R "columns":
//   pass "cols"   the log2(R) stages whose butterfly distance is >= C: each
//                 column (elements c, c + C, c + 2C, ...) is independent; a
//                 block stages W whole columns (W * R = tile words) in shared
//                 memory, W consecutive words per row (coalesced);
//   pass "chunks" the remaining stages act inside contiguous chunks of C
//                 words; a block stages tile / C chunks.
// Every launch takes a LimbMap, so one launch transforms any set of limbs
// (both polynomials of a ciphertext, all digits of a ModUp, ...), each with
// its own prime.
#include "ctx.cuh"

namespace ppst {

constexpr int NTT_THREADS = 256;

// forward lazy butterfly: X, Y in [0, 4q) -> [0, 4q)
__device__ __forceinline__ void bfly_fwd(uint64_t &X, uint64_t &Y, uint64_t w, uint64_t wsh, uint64_t q, uint64_t q2)
{
    uint64_t x = X >= q2 ? X - q2 : X;
    uint64_t t = shoup(Y, w, wsh, q);
    X = x + t;
    Y = x - t + q2;
}

// inverse lazy butterfly: X, Y in [0, 2q) -> [0, 2q)
__device__ __forceinline__ void bfly_inv(uint64_t &X, uint64_t &Y, uint64_t w, uint64_t wsh, uint64_t q, uint64_t q2)
{
    uint64_t s = X + Y;
    uint64_t d = X - Y + q2;
    X = s >= q2 ? s - q2 : s;
    Y = shoup(d, w, wsh, q);
}

__device__ __forceinline__ uint64_t reduce4q(uint64_t x, uint64_t q)
{
    uint64_t q2 = 2 * q;
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

// pass over columns: stages m = 1 .. R/2 (forward) or R/2 .. 1 (inverse)
template <bool FWD>
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_cols(LimbMap map, const PrimeC *__restrict__ pc,
                                                          const uint64_t *__restrict__ tw,
                                                          const uint64_t *__restrict__ twsh, int logN, int logR,
                                                          int tile)
{
    extern __shared__ uint64_t sm[];
    const int N = 1 << logN, R = 1 << logR, C = N >> logR;
    const int W = tile >> logR;  // columns per block
    const int b = blockIdx.y;
    uint64_t *a = map.ptr(b, N);
    const int p = map.prime(b);
    const uint64_t q = pc[p].q, q2 = 2 * q;
    const uint64_t *T = tw + (size_t)p * N, *TS = twsh + (size_t)p * N;
    const int c0 = blockIdx.x * W;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int r = idx / W, w = idx - r * W;
        sm[idx] = a[(size_t)r * C + c0 + w];
    }
    __syncthreads();
    const int half = tile >> 1;
    if (FWD) {
        for (int m = 1, tr = R >> 1; m < R; m <<= 1, tr >>= 1) {
            for (int bf = threadIdx.x; bf < half; bf += blockDim.x) {
                int w = bf % W, k = bf / W;
                int i = k / tr, r = 2 * i * tr + (k - i * tr);
                uint64_t X = sm[r * W + w], Y = sm[(r + tr) * W + w];
                bfly_fwd(X, Y, T[m + i], TS[m + i], q, q2);
                sm[r * W + w] = X;
                sm[(r + tr) * W + w] = Y;
            }
            __syncthreads();
        }
    } else {
        for (int m = R >> 1, tr = 1; m >= 1; m >>= 1, tr <<= 1) {
            for (int bf = threadIdx.x; bf < half; bf += blockDim.x) {
                int w = bf % W, k = bf / W;
                int i = k / tr, r = 2 * i * tr + (k - i * tr);
                uint64_t X = sm[r * W + w], Y = sm[(r + tr) * W + w];
                bfly_inv(X, Y, T[m + i], TS[m + i], q, q2);
                sm[r * W + w] = X;
                sm[(r + tr) * W + w] = Y;
            }
            __syncthreads();
        }
    }
    const uint64_t ni = pc[p].ninv, nish = pc[p].ninv_sh;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int r = idx / W, w = idx - r * W;
        uint64_t v = sm[idx];
        if (!FWD) v = csub(shoup(v, ni, nish, q), q);  // last inverse pass: times N^-1, to [0, q)
        a[(size_t)r * C + c0 + w] = v;
    }
}

// pass over contiguous chunks of C words: stages m = R .. N/2 (forward, then
// reduce to [0, q)) or N/2 .. R (inverse)
template <bool FWD>
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_chunks(LimbMap map, const PrimeC *__restrict__ pc,
                                                            const uint64_t *__restrict__ tw,
                                                            const uint64_t *__restrict__ twsh, int logN, int logR,
                                                            int tile)
{
    extern __shared__ uint64_t sm[];
    const int N = 1 << logN, R = 1 << logR, C = N >> logR;
    const int b = blockIdx.y;
    uint64_t *a = map.ptr(b, N) + (size_t)blockIdx.x * tile;
    const int p = map.prime(b);
    const uint64_t q = pc[p].q, q2 = 2 * q;
    const uint64_t *T = tw + (size_t)p * N, *TS = twsh + (size_t)p * N;
    const int g0 = blockIdx.x * (tile / C);  // first chunk of this block
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) sm[idx] = a[idx];
    __syncthreads();
    const int half = tile >> 1, hc = C >> 1;
    if (FWD) {
        for (int m = R, t = C >> 1; m < N; m <<= 1, t >>= 1) {
            for (int bf = threadIdx.x; bf < half; bf += blockDim.x) {
                int g = bf / hc, k = bf - g * hc;
                int il = k / t, pos = g * C + 2 * il * t + (k - il * t);
                int i = (g0 + g) * (C / (2 * t)) + il;
                uint64_t X = sm[pos], Y = sm[pos + t];
                bfly_fwd(X, Y, T[m + i], TS[m + i], q, q2);
                sm[pos] = X;
                sm[pos + t] = Y;
            }
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) a[idx] = reduce4q(sm[idx], q);
    } else {
        for (int m = N >> 1, t = 1; m >= R; m >>= 1, t <<= 1) {
            for (int bf = threadIdx.x; bf < half; bf += blockDim.x) {
                int g = bf / hc, k = bf - g * hc;
                int il = k / t, pos = g * C + 2 * il * t + (k - il * t);
                int i = (g0 + g) * (C / (2 * t)) + il;
                uint64_t X = sm[pos], Y = sm[pos + t];
                bfly_inv(X, Y, T[m + i], TS[m + i], q, q2);
                sm[pos] = X;
                sm[pos + t] = Y;
            }
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) a[idx] = sm[idx];
    }
}

static inline int ntt_log_r(int logN) { return (logN + 1) / 2; }

void ntt_fwd(Ctx &c, const LimbMap &m)
{
    if (m.count() == 0) return;
    const int logN = c.logN, logR = ntt_log_r(logN);
    const int tile = c.N < 4096 ? c.N : 4096;
    const size_t smem = (size_t)tile * sizeof(uint64_t);
    dim3 grid(c.N / tile, m.count());
    k_ntt_cols<true><<<grid, NTT_THREADS, smem, c.stream>>>(m, c.d_pc, c.d_tw, c.d_tw_sh, logN, logR, tile);
    k_ntt_chunks<true><<<grid, NTT_THREADS, smem, c.stream>>>(m, c.d_pc, c.d_tw, c.d_tw_sh, logN, logR, tile);
}

void ntt_inv(Ctx &c, const LimbMap &m)
{
    if (m.count() == 0) return;
    const int logN = c.logN, logR = ntt_log_r(logN);
    const int tile = c.N < 4096 ? c.N : 4096;
    const size_t smem = (size_t)tile * sizeof(uint64_t);
    dim3 grid(c.N / tile, m.count());
    k_ntt_chunks<false><<<grid, NTT_THREADS, smem, c.stream>>>(m, c.d_pc, c.d_itw, c.d_itw_sh, logN, logR, tile);
    k_ntt_cols<false><<<grid, NTT_THREADS, smem, c.stream>>>(m, c.d_pc, c.d_itw, c.d_itw_sh, logN, logR, tile);
}

}  // namespace ppst
