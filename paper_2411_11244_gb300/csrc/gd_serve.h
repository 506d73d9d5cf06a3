// Serving loop internals shared between gd_api.cu and gd_serve.cu.
#pragma once

#include <string>

#include "gd_internal.cuh"

namespace gd {

// work buffers and stream of one in-flight batch
struct SlotBuffers {
    cudaStream_t stream = nullptr;
    Item* front[2] = {nullptr, nullptr};
    Item* leafq = nullptr;
    Cand* cand = nullptr;
    double* cand_d = nullptr;
    double* cand_pts = nullptr;
    long long cap_front = 0, cap_leaf = 0, cap_cand = 0;
    QState* qs = nullptr;
    QIn* qin_dev = nullptr;
    QIn* qin_host = nullptr;
    gd_result* out_dev = nullptr;
    gd_result* out_host = nullptr;
    unsigned* mb_dev_ctr = nullptr;
    unsigned* ctr_host = nullptr;
    StatsDev* stats_dev = nullptr;
    float* rbox = nullptr;
    uint2* jobs = nullptr;
    long long cap_slots = 0;
    unsigned* slot_of = nullptr;
    long long cap_table = 0;
    long long cap_q = 0;
    int grid = 0;
};

gd_status serve_launch_batch(gd_ctx* ctx, SlotBuffers& sb, const gd_query* qs, long long m, int kind, int grid);
gd_status serve_single(gd_ctx* ctx, const gd_query& q, gd_result* out);
int serve_device(gd_ctx* ctx);
int serve_sms(gd_ctx* ctx);
const gd_tunables& serve_tunables(gd_ctx* ctx);
bool serve_query_ok(gd_ctx* ctx, const gd_query& q, std::string* why);
long long serve_mesh_tris(const gd_mesh* m);

}  // namespace gd
