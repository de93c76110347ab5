// serve.cu -- continuous-batching request loop.
#include "serve.cuh"

namespace ppst {

struct Server {
    uint32_t tag = TAG_SRV;
};

void server_destroy(Server *s) { delete s; }

}  // namespace ppst

using namespace ppst;

extern "C" {

int ppst_server_create(ppst_ctx *, const ppst_evk *, size_t, uint32_t, ppst_server **out)
{
    if (out) *out = nullptr;
    return PPST_E_STATE;
}

int ppst_submit(ppst_server *, ppst_stat, const ppst_col *, const ppst_col *, const ppst_qopts *, uint64_t *)
{
    return PPST_E_STATE;
}

int ppst_wait(ppst_server *, uint64_t, int32_t, ppst_res **out)
{
    if (out) *out = nullptr;
    return PPST_E_STATE;
}

int ppst_ticket_latency(ppst_server *, uint64_t, double *) { return PPST_E_STATE; }

}  // extern "C"
