// noalloc.cu -- HMult that allocates no device memory.
//
// Some callers cannot allocate device memory once they are running: a host
// that has given all free HBM to its own caching allocator, or a serving
// thread whose latency budget cannot absorb cudaMalloc's implicit device
// synchronisation. ppst_hmult_noalloc serves them: it is ppst_hmult with the
// result written into a ciphertext the caller already owns and with every
// temporary (tensor output, key-switching digits and accumulators, rescale
// buffers) carved from one static device array of NOALLOC_BYTES, which every
// GPU that loads this library holds until the process exits.
//
// Set-up: creating a context looks up its device's address of the array
// (cudaGetSymbolAddress, with the device current) and caches it. That lookup
// loads this file's module, which is when the driver commits the array's
// memory on the device, so the 32 MiB are taken while the caller can still
// allocate. The kernels a call launches are loaded on their first launch
// (CUDA's lazy loading), so a caller about to give the free memory away makes
// one call first. All calls share the array and it keeps the last call's
// contents; no word of it is read before the same call writes it, so nothing
// needs clearing. Calls whose GPU work overlaps (other threads, other
// streams, other contexts on the same device) race on the array. On an
// error the output ciphertext is left as it was: the result is built in the
// array and copied into the output only once every kernel has been issued.
#include <mutex>

#include "ctx.cuh"

namespace ppst {

constexpr size_t NOALLOC_BYTES = (size_t)32 << 20;  // 32 MiB
constexpr size_t NOALLOC_WORDS = NOALLOC_BYTES / 8;

static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS];

static std::mutex g_noalloc_mu;
static std::map<int, uint64_t *> g_noalloc_addr;  // device -> address of the array there

uint64_t *noalloc_scratch_on_current_device()
{
    int dev = 0;
    PPST_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) return it->second;
    uint64_t *p = nullptr;
    PPST_CUDA(cudaGetSymbolAddress((void **)&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
    return p;
}

// words of scratch: pre-rescale product [2][L+1][N], d2 [L+1][N],
// digits [dnum][L+1+K][N], accumulators [2][L+1+K][N], conversion [2][L+1][N],
// rescaled result [2][L+1][N]
static size_t noalloc_words(const Ctx &c)
{
    const size_t N = c.N, q = c.L + 1, e = c.ext_rows();
    return (2 * q + q + (size_t)c.dnum * e + 2 * e + 2 * q + 2 * q) * N;
}

void hmult_noalloc(Ctx &c, const EvkObj &k, const CtObj &a, const CtObj &b, CtObj &out)
{
    const int lv = std::min(a.level, b.level);
    if (lv < 1) throw_err(PPST_E_DEPTH, "hmult at level 0");
    if (!k.relin.d) throw_err(PPST_E_STATE, "no relinearisation key");
    const size_t need = noalloc_words(c);
    if (need > NOALLOC_WORDS)
        throw_err(PPST_E_ARG, "ppst_hmult_noalloc: these parameters need " + std::to_string(need * 8 >> 20) +
                                  " MiB of scratch; the static array holds " +
                                  std::to_string(NOALLOC_BYTES >> 20) + " MiB");
    uint64_t *s = noalloc_scratch_on_current_device();
    const size_t N = c.N, q = c.L + 1, e = c.ext_rows();
    CtObj tmp;  // pre-rescale product, inside the static array (not a pool buffer)
    tmp.ctx = &c;
    tmp.d = s;
    tmp.level = lv;
    tmp.scale = a.scale * b.scale;
    uint64_t *d2 = s + 2 * q * N, *ext = d2 + q * N, *acc = ext + (size_t)c.dnum * e * N, *conv = acc + 2 * e * N;
    // the key-switching kernels take their temporaries from the context's
    // workspace fields: point them into the static array for this call
    uint64_t *sv[4] = {c.ws_d2, c.ws_ext, c.ws_acc, c.ws_conv};
    c.ws_d2 = d2;
    c.ws_ext = ext;
    c.ws_acc = acc;
    c.ws_conv = conv;
    try {
        k_tensor(c, a, b, lv, tmp.c0(), tmp.c1(), d2);
        ntt_inv(c, map_poly(c, d2, lv));
        k_modup(c, d2, lv, ext);
        LimbMap me{ext, e * N, lv + 1 + c.K, c.ndigits(lv), lv + 1, 0, c.L + 1};
        ntt_fwd(c, me);
        k_inner_product(c, ext, k.relin, lv, acc);
        k_moddown(c, acc, lv, tmp.c0(), tmp.c1(), tmp.c0(), tmp.c1());
        CtObj res;  // the rescaled product, also inside the static array
        res.ctx = &c;
        res.d = conv + 2 * q * N;
        res.level = lv - 1;
        k_rescale(c, tmp, res);
        // only now does the caller's ciphertext change (a device-to-device copy, no allocation)
        PPST_CUDA(cudaMemcpyAsync(out.d, res.d, 2 * q * N * sizeof(uint64_t), cudaMemcpyDeviceToDevice, c.stream));
        out.level = lv - 1;
        out.scale = (a.scale * b.scale) / (double)c.primes[lv];
    } catch (...) {
        c.ws_d2 = sv[0];
        c.ws_ext = sv[1];
        c.ws_acc = sv[2];
        c.ws_conv = sv[3];
        throw;
    }
    c.ws_d2 = sv[0];
    c.ws_ext = sv[1];
    c.ws_acc = sv[2];
    c.ws_conv = sv[3];
}

}  // namespace ppst

using namespace ppst;

extern "C" int ppst_hmult_noalloc(ppst_ctx *ctx, const ppst_evk *evk, const ppst_ct *a, const ppst_ct *b,
                                  ppst_ct *out)
{
    Ctx *c = (Ctx *)ctx;
    if (!c || c->tag != TAG_CTX) return PPST_E_ARG;
    const EvkObj *k = (const EvkObj *)evk;
    const CtObj *A = (const CtObj *)a, *B = (const CtObj *)b;
    CtObj *O = (CtObj *)out;
    if (!k || k->tag != TAG_EVK || !A || A->tag != TAG_CT || !B || B->tag != TAG_CT || !O || O->tag != TAG_CT ||
        A->ctx != c || B->ctx != c || O->ctx != c)
        return c->fail(PPST_E_ARG, "bad handle");
    if (O == A || O == B || O->buf.use_count() != 1)
        return c->fail(PPST_E_ARG, "the output must own its buffer alone (not an input, not a level view)");
    try {
        std::lock_guard<std::recursive_mutex> lk(c->exec_mu);  // the workspace pointers are swapped meanwhile
        hmult_noalloc(*c, *k, *A, *B, *O);
        c->clear_err();
        return PPST_OK;
    } catch (const PpstError &e) {
        return c->fail(e.code, e.msg);
    } catch (...) {
        return c->fail(PPST_E_ARG, "unexpected error");
    }
}
