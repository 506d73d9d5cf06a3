// gd_query_device_noalloc: the device-resident query without any allocation.
//
// Who needs it: callers that must not allocate device memory once they are
// running.  A control loop that queries distances every frame (motion
// planning, haptics) cannot afford a cudaMalloc that may stall for
// milliseconds or fail halfway through a frame, and a host whose device
// memory is reserved by another allocator (a framework's caching pool that
// holds nearly all of HBM) has nothing left for this library's own buffers.
// gd_query_device needs the context's work buffers, which the library sizes
// (and may grow) with cudaMalloc; this entry point instead carves every work
// buffer (front queues, leaf-pair queue, candidates, refit slots, counters,
// per-query state) out of one fixed array compiled into the library.
//
// The array is a file-scope static __device__ array of kScratchBytes bytes.
// Every GPU that loads the library holds it until the process exits.  In host
// code its name is only a host-side stand-in, so its device address is taken
// once per device with cudaGetSymbolAddress, with that device current, on the
// first call of this entry point on that device; make that first call before
// any stream capture starts.  All calls share the one array and it keeps the
// contents of the last call: the counters that must start at zero are cleared
// (cudaMemsetAsync, no allocation) at the start of every call, and two calls
// whose work overlaps on the GPU race on the array, so callers serialise them
// (one stream, or events).
#include <cstring>
#include <mutex>

#include "gd_internal.cuh"
#include "gd_launch.h"

namespace gd {

// fixed capacities carved out of the array (see the layout below)
constexpr unsigned long long kScratchBytes = 32ull << 20;
constexpr unsigned kNaFront = 1u << 18;     // front entries per buffer
constexpr unsigned kNaLeaf = 1u << 18;      // leaf pairs
constexpr unsigned kNaCand = 1u << 16;      // float64 candidates
constexpr unsigned kNaSlots = 1024;         // refit slots
constexpr unsigned kNaTableBits = 16;       // refit-root table: B with at most 24 tree levels

gd_ctx* mesh_ctx(const gd_mesh* m);
const MeshDev* mesh_desc(const gd_mesh* m);
int mesh_levels(const gd_mesh* m);
int serve_device(gd_ctx* ctx);
const gd_tunables& serve_tunables(gd_ctx* ctx);
int single_launch_fields(gd_ctx* c, const gd_mesh* B, int kind, KArgs& a);

namespace {

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Layout {
    unsigned long long ctr, stats, qs, slot_of, jobs, rbox, front0, front1, leafq, cand, cand_d, cand_pts, end;
};

constexpr unsigned long long up256(unsigned long long x) { return (x + 255ull) & ~255ull; }

constexpr Layout layout() {
    Layout L{};
    unsigned long long o = 0;
    L.ctr = o; o = up256(o + sizeof(unsigned) * kCtrWords);
    L.stats = o; o = up256(o + sizeof(StatsDev));
    L.qs = o; o = up256(o + sizeof(QState));
    L.slot_of = o; o = up256(o + sizeof(unsigned) * (1ull << kNaTableBits));
    L.jobs = o; o = up256(o + sizeof(uint2) * kNaSlots);
    L.rbox = o; o = up256(o + sizeof(float) * 6ull * kRefitBoxes * kNaSlots);
    L.front0 = o; o = up256(o + sizeof(Item) * (unsigned long long)kNaFront);
    L.front1 = o; o = up256(o + sizeof(Item) * (unsigned long long)kNaFront);
    L.leafq = o; o = up256(o + sizeof(Item) * (unsigned long long)kNaLeaf);
    L.cand = o; o = up256(o + sizeof(Cand) * (unsigned long long)kNaCand);
    L.cand_d = o; o = up256(o + sizeof(double) * (unsigned long long)kNaCand);
    L.cand_pts = o; o = up256(o + 6ull * sizeof(double) * kNaCand);
    L.end = o;
    return L;
}
static_assert(layout().end <= kScratchBytes, "the work buffers fit the static array");
static_assert(sizeof(unsigned) * kCtrWords <= 256, "counters fit their slot");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};

// device address of the array on the current device (taken once per device)
cudaError_t scratch_base(int device, unsigned char** out) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_base[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_base[device] = static_cast<unsigned char*>(p);
    }
    *out = g_base[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace gd

using namespace gd;

extern "C" GD_API gd_status gd_query_device_noalloc(const gd_mesh* A, const gd_mesh* B, gd_kind kind,
                                                    const double* d_xa, const double* d_xb, gd_result* d_out,
                                                    void* stream) {
    if (!A || !B || !d_xa || !d_xb || !d_out || (kind != GD_MIN && kind != GD_MAX)) return GD_ERR_INVALID_ARG;
    gd_ctx* ctx = mesh_ctx(A);
    const MeshDev* da = mesh_desc(A);
    const MeshDev* db = mesh_desc(B);
    if (!ctx || mesh_ctx(B) != ctx) return GD_ERR_INVALID_ARG;
    if (!da || !db) return GD_ERR_NOT_BUILT;
    // the meshes' descriptors live on their context's device, and the array
    // used is the current device's: they must be the same device (this call
    // changes no device state, so it is refused rather than switched)
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return GD_ERR_CUDA;
    if (device != serve_device(ctx)) return GD_ERR_INVALID_ARG;
    // the refit-root table of the array holds 2^16 entries: with refit on, B
    // may have at most 16 + 8 = 24 tree levels (fewer than 2^25 triangles);
    // with refit off the table is not used
    const bool refit = serve_tunables(ctx).refit_mode == 1;
    const int LB = mesh_levels(B);
    const int dR = LB > kRefitH ? LB - kRefitH : 0;
    if (refit && dR > (int)kNaTableBits) return GD_ERR_INVALID_ARG;
    constexpr Layout L = layout();
    unsigned char* base = nullptr;
    if (scratch_base(device, &base) != cudaSuccess) return GD_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // counters and barrier words must start at zero
    if (cudaMemsetAsync(base + L.ctr, 0, sizeof(unsigned) * kCtrWords, st) != cudaSuccess) return GD_ERR_CUDA;

    KArgs a{};
    a.nq = 1;
    a.qin = nullptr;
    a.mA = da;
    a.mB = db;
    a.xa_src = d_xa;
    a.xb_src = d_xb;
    a.qs = reinterpret_cast<QState*>(base + L.qs);
    a.front0 = reinterpret_cast<Item*>(base + L.front0);
    a.front1 = reinterpret_cast<Item*>(base + L.front1);
    a.cap_front = kNaFront;
    a.leafq = reinterpret_cast<Item*>(base + L.leafq);
    a.cap_leaf = kNaLeaf;
    a.cand = reinterpret_cast<Cand*>(base + L.cand);
    a.cand_d = reinterpret_cast<double*>(base + L.cand_d);
    a.cand_pts = reinterpret_cast<double*>(base + L.cand_pts);
    a.cap_cand = kNaCand;
    a.ctr = reinterpret_cast<unsigned*>(base + L.ctr);
    a.stats = reinterpret_cast<StatsDev*>(base + L.stats);
    a.out = d_out;
    a.rbox = reinterpret_cast<float*>(base + L.rbox);
    a.cap_slots = kNaSlots;
    a.slot_of = reinterpret_cast<unsigned*>(base + L.slot_of);
    a.n_slot_of = refit ? 1ull << dR : 0ull;
    a.jobs = reinterpret_cast<uint2*>(base + L.jobs);
    // tunables, grid, background probes and root push as gd_query_device
    // sets them, so both entry points run the same traversal
    const int grid = single_launch_fields(ctx, B, (int)kind, a);
    if (launch_query((int)kind, a, grid, st) != cudaSuccess) return GD_ERR_CUDA;
    return GD_OK;
}
