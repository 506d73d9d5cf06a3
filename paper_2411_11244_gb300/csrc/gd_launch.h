// Host-side entry points of the engine's kernels (shared by the C ABI file).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gd_internal.cuh"

namespace gd {

// ---- BVH build (gd_build.cu)
struct BuildBuffers {
    const float* verts;   // nv x 3, device
    const int32_t* tris;  // nt x 3, device
    long long nv, nt;
    int L;
    int morton_bits;
    float* box;           // 6 * 2^(L+1) floats, device
    float4* tri;          // 3 * nt float4, device
    unsigned* order;      // nt, device: original index of each sorted triangle (kept for refits)
    int32_t* stris;       // nt x 3, device: the sorted triangles' vertex indices (written by the
                          // build, read by refits; may be nullptr for a build that keeps none)
    unsigned* flags;      // device: [0] bad index, [1] non-finite vertex, [2..8] bounds scratch
    unsigned long long* keys[2];  // nt each, device
    unsigned* vals[2];            // nt each, device
    unsigned* hist;       // 256 * nblocks, device
};

size_t build_hist_words(long long nt);
// stable LSD radix sort of n (key, value) pairs on the low key_bits bits of
// the keys, 8 bits per pass, ping-ponging between keys[0|1] and vals[0|1]
// (hist: build_hist_words(n) words); returns the index of the buffers that
// hold the sorted pairs
int radix_sort_pairs(unsigned long long* const keys[2], unsigned* const vals[2], long long n, int key_bits,
                     unsigned* hist, cudaStream_t stream);
// checks indices and finiteness, and bounds the referenced vertices (flags)
cudaError_t build_validate(const BuildBuffers& b, cudaStream_t stream);
// the rest of the build; only after build_validate reported clean flags
cudaError_t build_tree(const BuildBuffers& b, cudaStream_t stream);
// refit of a built tree after its vertices moved (verts, tris, L, order, tri,
// box, flags): stored triangles and leaf boxes from the new vertices, then the
// unions up to the root.  flags[1] != 0 afterwards: a referenced coordinate is
// not finite; flags[8..13]: the root box (float bits); *P_out (device, may be
// null): max |coordinate| of the root box.
cudaError_t build_refit(const BuildBuffers& b, float* P_out, cudaStream_t stream);

// ---- naive comparator (gd_naive.cu)
// words of its device scratch (uint64 each)
enum : int {
    kNaiveU = 0,         // running bound: float bits of a squared distance (low 32 bits)
    kNaiveTests = 1,     // node boxes tested
    kNaiveLeaves = 2,    // triangle pairs evaluated
    kNaiveMaxTests = 3,  // most boxes tested by one thread
    kNaiveT0 = 4,        // globaltimer stamp of the first thread to start
    kNaiveTimeout = 5,   // some thread passed the deadline and stopped
    kNaiveBad = 6,       // a walk outgrew its stack (never, for at most 31 levels)
    kNaiveWords = 8,
};

struct NaiveArgs {
    const float4* triA;   // A's triangles in leaf order
    long long TA;
    const float* boxB;    // B's tree
    const float4* triB;
    long long TB;
    int LB;
    float R[9], t[3];     // A-local -> B-local, float32
    float E;              // widening of each mapped triangle's box
    unsigned long long* ws;
    long long timeout_ns;
};

cudaError_t launch_naive(int kind, const NaiveArgs& g, cudaStream_t stream);

// ---- point-to-mesh queries (gd_point.cu)
enum : int {
    kPointTests = 0,     // node boxes tested
    kPointExact = 1,     // float64 point-triangle distances
    kPointT0 = 2,        // globaltimer stamp of the first CTA to start
    kPointTimeout = 3,   // some point passed the deadline
    kPointWords = 4,
};

struct PointArgs {
    const float* box;     // the mesh's tree
    const float4* tri;
    long long T;
    int L;
    double x[12];         // mesh local -> world
    const double* pts;    // n x 3 world points, device
    long long n;
    gd_point_result* out; // n results, device
    const unsigned* order;// thread i answers point order[i] (nullptr: point i)
    unsigned long long* ws;
    long long timeout_ns;
};

// order the points along a Morton curve in the mesh's frame so that a warp's
// walks visit the same nodes: keys[0], vals[0] in, sorted pairs in buffers
// [returned index]; hist: build_hist_words(n) words
int sort_points(const PointArgs& g, unsigned long long* const keys[2], unsigned* const vals[2], unsigned* hist,
                cudaStream_t stream);
cudaError_t launch_point(const PointArgs& g, cudaStream_t stream);

// ---- query (gd_query.cu)
// co-resident CTAs per SM of the query kernel's single-query or batch launch
int query_max_blocks_per_sm(int kind, bool batch = false);
cudaError_t launch_query(int kind, const KArgs& args, int grid, cudaStream_t stream);
cudaError_t build_query_graph(int kind, const KArgs& args, int grid, cudaGraphExec_t* exec);

}  // namespace gd
