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
    unsigned* flags;      // device: [0] bad index, [1] non-finite vertex, [2..8] bounds scratch
    unsigned long long* keys[2];  // nt each, device
    unsigned* vals[2];            // nt each, device
    unsigned* hist;       // 256 * nblocks, device
};

size_t build_hist_words(long long nt);
// checks indices and finiteness, and bounds the referenced vertices (flags)
cudaError_t build_validate(const BuildBuffers& b, cudaStream_t stream);
// the rest of the build; only after build_validate reported clean flags
cudaError_t build_tree(const BuildBuffers& b, cudaStream_t stream);

// ---- query (gd_query.cu)
int query_max_blocks_per_sm(int kind);
cudaError_t launch_query(int kind, const KArgs& args, int grid, cudaStream_t stream);
cudaError_t build_query_graph(int kind, const KArgs& args, int grid, cudaGraphExec_t* exec);

}  // namespace gd
