// serve.cuh -- continuous-batching request loop (declarations).
#pragma once
#include "ctx.cuh"

namespace ppst {
struct Server;
void server_destroy(Server *s);
}  // namespace ppst
