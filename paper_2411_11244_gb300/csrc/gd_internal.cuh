// Internal device-side declarations of the GB300 distance engine.
//
// Data layout in HBM (one mesh, T triangles, L = floor(log2 T), 2^L leaves):
//   box  : float[6 * 2^(L+1)], node i (heap order, root 1, children 2i, 2i+1)
//          at box[6i .. 6i+5] = (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z); entry 0
//          unused.  Implicit full binary tree with boxes only (Section 7.3).
//   tri  : float4[3 * T] in leaf (Morton) order, triangle j at tri[3j..3j+2] =
//          (v0x v0y v0z v1x) (v1y v1z v2x v2y) (v2z id 0 0), id = the caller's
//          original index stored as int bits.
//   leaf l owns sorted triangles [floor(l T / 2^L), floor((l+1) T / 2^L)):
//          one or two each, no per-leaf storage (the f12 rule of Section 7.3).
#pragma once
#include <cstddef>

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gdist.h"

namespace gd {

constexpr int kBlock = 256;          // threads per CTA of the persistent kernels
constexpr int kRefitH = 8;           // height of the B subtrees refit into A's frame
constexpr int kRefitBoxes = 2 << kRefitH;  // boxes per refit slot (heap 1 .. 2^(h+1)-1)
constexpr int kMaxLevels = 64;       // BVTT expansion levels per launch
constexpr unsigned kFull = 0xffffffffu;

struct MeshDev {
    const float* box;    // 6 floats per node
    const float4* tri;   // 3 float4 per triangle, leaf order
    long long T;         // triangles
    int L;               // leaves = 2^L
    float P;             // max |coordinate| over referenced vertices (exact)
};

// one BVTT front entry (Section 5): two node ids, the stored bound used to
// re-cull the entry against the running bound, and the query it belongs to
struct __align__(16) Item {
    uint32_t a, b;
    float bound;
    uint32_t q;
};

// a triangle pair kept for float64 refinement (sorted triangle ids)
struct __align__(16) Cand {
    uint32_t ta, tb;
    float bound;
    uint32_t q;
};

struct QIn {
    const MeshDev* A;
    const MeshDev* B;
    double xa[12], xb[12];
    unsigned slot_base;  // first entry of this query's refit-root table
    unsigned pad;
};

// per-query running state and derived constants
struct __align__(16) QState {
    unsigned U;                   // running bound, float bits (min: upper of
                                  // D_min, atomicMin; max: lower of D_max, atomicMax)
    unsigned status;              // kStat* bits
    unsigned long long best_d;    // float64 bits of the refined extreme
    unsigned long long best_key;  // (orig a << 32 | orig b) of the witness
    float R[9], t[3];             // B-local -> A-local, float32
    float Rl[9], tl[3];           // float32 remainders: R + Rl, t + tl carry ~48 bits
    float E_box, E_tri;           // absolute widening of box / triangle bounds
    float E_df;                   // error of the double-float map (absolute)
    const MeshDev* A;
    const MeshDev* B;
    double xa[12], xb[12];
    unsigned slot_base;           // refit-root table offset of this query
    int dR;                       // depth of B's refit roots (L_B - min(L_B, kRefitH)), -1: no refit
    unsigned cert;                // float64 intersection checks started (min kind)
    unsigned pushed[2];           // batch: entries pushed at the current level (by parity)
};

// kStatZero: a pair at float64 distance exactly 0 is a candidate, so D_min = 0
// and the query's traversal stops; kStatEvict: a query of a batch pushed more
// than its share of the queues in one level, so it stops and is run again
// alone.  (The status word shares an aligned 8-byte word with U, so one load
// gives both.)
constexpr unsigned kStatOverflow = 1u, kStatTimeout = 2u, kStatNoResult = 4u, kStatZero = 8u, kStatEvict = 16u;
constexpr unsigned kStatStop = kStatZero | kStatEvict;
constexpr unsigned kCertMax = 64;  // float64 intersection checks per query and launch
static_assert(offsetof(QState, status) == offsetof(QState, U) + 4 && offsetof(QState, U) % 8 == 0,
              "U and status must form one aligned 8-byte word");

// global counters, one uint32 array per context
enum : int {
    kCtrCnt = 0,      // [0..2] front entry counts, triple-buffered by level
    kCtrRem = 3,      // [3..5] max remaining depth of the entries of that front
    kCtrLeaf = 6,     // leaf-pair count
    kCtrCand = 7,     // candidate count
    kCtrPool0 = 8,    // batch: entries taken from the common pool in the current level
    kCtrOverflow = 9, // some push exceeded its capacity
    kCtrJobs = 10,    // refit jobs appended (slot j refits job j)
    kCtrJobsDone = 11,// refit jobs already run
    kCtrTailDone = 12,// CTAs done with their candidate in the one-per-CTA tail
    kCtrBadIndex = 13,// an index check failed (bit per site); the access was skipped
    kCtrRefined = 14, // candidates refined in float64 (their indices are listed)
    kCtrPool1 = 15,   //   ... by level parity (kCtrPool0: even pushes, kCtrPool1: odd)
    kCtrReset = 16,   // counters [0, kCtrReset) are cleared at kernel start
    kCtrAbort = 20,   // a wait gave up: every CTA leaves at its next barrier
    kCtrLastAbort = 21, // the abort flag of the last finished launch
    kCtrExit = 22,    // CTAs that left the kernel (the last one resets the barrier)
    kCtrSetupDone = 23, // query setup published (background probe CTAs wait for it)
    kCtrBarCount = 32,// grid-barrier arrivals of this launch (top bit: abort)
    kCtrWords = 64,
};

// CTA totals of a launch are added to copy (CTA index mod kAccWays) of each
// counter: one copy would queue the final atomics of 300 CTAs on one L2 word
// (measured: the last CTA then left 12-17 us after the rest); the host sums
// the copies
constexpr int kAccWays = 16;

struct StatsDev {
    unsigned levels;
    unsigned front[32];
    unsigned slots[32];
    unsigned long long acc_pairs[kAccWays];  // node pairs tested
    unsigned long long acc_bytes[kAccWays];  // algorithmic bytes
    unsigned acc_tri[kAccWays];              // float32 triangle pairs
    unsigned acc_ref[kAccWays];              // float64 refinements
    unsigned leaf_pairs, candidates;
    unsigned level_ns[32];  // device time of each level (CTA 0's view, barrier to barrier)
    unsigned phase_ns[12];  // setup, refit, probe, levels, leaf, refine, tail wait, select,
                            // finalize, total, -, -
    unsigned probes;        // greedy probes run
    float u_level[32];      // running bound of query 0 entering each level
    float u_probe;          // ... right after the probes
    unsigned refits;        // B subtrees refit into A's frame
    unsigned long long t_start;  // globaltimer at the launch's start (CTA 0)
};

// Result record of a single query in pinned host memory, written by the
// launch's last CTA (the host polls seq instead of copying and synchronising)
struct HostDone {
    gd_result out;
    unsigned last_abort;          // the launch's abort flag
    unsigned bad_index;           // sites of failed index checks
    unsigned long long seq;       // written last: the launch's sequence number
};

struct KArgs {
    int nq;
    const QIn* qin;             // batch: per-query meshes and transforms
    const MeshDev* mA;          // single query (qin == nullptr)
    const MeshDev* mB;
    const double* xa_src;       // single query: device transforms, or nullptr
    const double* xb_src;       //   to use xa_val / xb_val below
    double xa_val[12], xb_val[12];
    QState* qs;
    Item* front0;
    Item* front1;
    unsigned cap_front;
    Item* leafq;
    unsigned cap_leaf;
    Cand* cand;
    double* cand_d;
    double* cand_pts;           // float64 witness points of every candidate (6 each)
    unsigned cap_cand;
    unsigned* ctr;
    StatsDev* stats;
    gd_result* out;
    float* rbox;                // refit slots: kRefitBoxes boxes of 6 floats each
    unsigned cap_slots;
    unsigned* slot_of;          // refit-root table: slot of each claimed root
    unsigned long long n_slot_of;
    uint2* jobs;                // (query, root) of every refit slot
    int refit;                  // 0: map B's local boxes only; 1: lazy refit
    int conventional;           // 1: conventional bounds only (Eq. 9 for the min, the
                                // box gap for the max) instead of Eqs. 10-11
    int probes;                 // greedy probes per launch (at least one per query)
    long long work_target;
    int k_max;
    long long timeout_ns;
    unsigned q_budget;          // batch: entries one query may push per level (0: no limit)
    unsigned q_pool;            // batch: entries per level beyond their shares that the
                                // queries of the launch may take, first come first served
    int fuse_root;              // single query, no refit claim at the root: phase 0 pushes
                                // the root pair (phase 1 and its barrier are skipped)
    unsigned work_ctas;         // CTAs [0, work_ctas) run the traversal and meet at the
                                // grid barriers; the rest run background probes (0: all)
    HostDone* host_done;        // copy of the result (single query) for the host, the launch's
                                // abort and index-check words, and the sequence stamp (or nullptr)
    unsigned long long seq;     // ... stamped with this sequence number
    gd_result* host_out;        // with host_done: the nq results copied here (pinned host
                                // memory) before the stamp (or nullptr)
    unsigned long long* done_ns;// per query of the launch: globaltimer when its result record
                                // was final (or nullptr)
    float* ftree;               // single query, full refit (the paper's per-frame refit of
                                // B): 6 floats per node of B, heap order, B's boxes in A's
                                // frame, rebuilt at the start of the launch (or nullptr)
};

// ------------------------------------------------------------------ memory

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

constexpr unsigned kBarAbort = 0x80000000u;  // abort bit of the barrier word

// Raise the abort flag: every CTA waiting at (or reaching) a grid barrier
// returns false, and so does every later barrier of the launch.
__device__ __forceinline__ void raise_abort(const KArgs& A) {
    atomicExch(A.ctr + kCtrAbort, 1u);
    atomicOr(A.ctr + kCtrBarCount, kBarAbort);
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  One
// word counts arrivals over the whole launch: a CTA arriving as number c
// waits until the count reaches the next multiple of the grid size.  The
// arrival is a release and the wait an acquire at GPU scope, so every write
// made by any thread of a CTA before the barrier (ordered by __syncthreads)
// is visible to every thread after it; no other fence is needed.  The top
// bit of the same word is the abort flag, so the wait sees an abort with no
// extra load.  Every wait is bounded: after timeout_ns the CTA raises the
// abort and returns false.  post() runs on thread 0 after a successful wait,
// before the CTA's closing __syncthreads (it refreshes CTA-shared copies of
// global state).
template <class F>
__device__ __forceinline__ bool grid_sync(const KArgs& A, F&& post) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* count = A.ctr + kCtrBarCount;
        const unsigned G = A.work_ctas ? A.work_ctas : gridDim.x;
        const unsigned old = atom_add_release(count, 1u);
        int ok = (old & kBarAbort) == 0u;
        if (ok) {
            const unsigned target = ((old & ~kBarAbort) / G + 1u) * G;
            unsigned long long t0 = 0;
            for (unsigned spin = 0;; ++spin) {
                const unsigned v = ld_acquire(count);
                if (v & kBarAbort) { ok = 0; break; }
                if (v >= target) break;
                if ((spin & 63u) == 0u) {
                    const unsigned long long now = globaltimer();
                    if (t0 == 0) t0 = now;
                    else if ((long long)(now - t0) > A.timeout_ns) {
                        raise_abort(A);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (ok) post();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ bool grid_sync(const KArgs& A) {
    return grid_sync(A, [] {});
}

}  // namespace gd
