// Serving loop internals shared between gd_api.cu and gd_serve.cu.
#pragma once

#include <string>

#include "gd_internal.cuh"

namespace gd {

// the server's private execution context runs these (meshes of the user's
// context, same device)
gd_status serve_single(gd_ctx* ctx, const gd_query& q, gd_result* out);
gd_status serve_batch(gd_ctx* ctx, const gd_query* qs, long long m, int kind, gd_result* out);
// pipelined single queries (slot 0 or 1): launch, test for the stamp, collect
gd_status serve_single_launch(gd_ctx* ctx, const gd_query& q, int slot, unsigned long long* seq);
bool serve_single_ready(gd_ctx* ctx, int slot, unsigned long long seq);
gd_status serve_single_finish(gd_ctx* ctx, const gd_query& q, int slot, unsigned long long seq, gd_result* out);
// size ctx's work buffers for batches of up to m queries now, not at the
// first request
gd_status serve_prepare(gd_ctx* ctx, long long m);
int serve_device(gd_ctx* ctx);
int serve_sms(gd_ctx* ctx);
const gd_tunables& serve_tunables(gd_ctx* ctx);
bool serve_query_ok(gd_ctx* ctx, const gd_query& q, std::string* why);
long long serve_mesh_tris(const gd_mesh* m);

}  // namespace gd
