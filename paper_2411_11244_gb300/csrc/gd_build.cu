// f12-BVH construction on the device (Section 7.3): Morton codes of the
// triangle centroids, a stable LSD radix sort (ties keep the original
// order), 2^L leaves of one or two consecutive sorted triangles, exact leaf
// boxes, and a level-by-level union up to the root.  Leaf boxes are exact
// bounds of their vertices, so every box is tight (Section 4: tight leaves
// make every node tight).  Refit for moved vertices (Section 8, deformable
// scenes): the same leaf and union kernels over the stored leaf order.
#include <cfloat>
#include <cstdint>

#include "gd_internal.cuh"
#include "gd_launch.h"

namespace gd {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                      // keys per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per CTA

// float -> uint32 whose unsigned order is the float order
__device__ __forceinline__ unsigned ordered(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// flags: [0] bad index, [1] non-finite vertex, [2..4] ordered min, [5..7] ordered max
__global__ void k_init_flags(unsigned* flags) {
    if (threadIdx.x < 8) flags[threadIdx.x] = (threadIdx.x >= 2 && threadIdx.x < 5) ? 0xffffffffu : 0u;
}

__global__ void k_validate(const float* verts, long long nv, const int32_t* tris, long long nt, unsigned* flags) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    bool bad_idx = false, bad_val = false;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        for (int k = 0; k < 3; ++k) {
            int32_t v = tris[3 * t + k];
            if (v < 0 || v >= nv) { bad_idx = true; continue; }
            for (int c = 0; c < 3; ++c) {
                float x = verts[3ll * v + c];
                if (!isfinite(x)) { bad_val = true; continue; }
                lo[c] = fminf(lo[c], x);
                hi[c] = fmaxf(hi[c], x);
            }
        }
    }
    if (__any_sync(kFull, bad_idx) && (threadIdx.x & 31) == 0) atomicOr(flags + 0, 1u);
    if (__any_sync(kFull, bad_val) && (threadIdx.x & 31) == 0) atomicOr(flags + 1, 1u);
    for (int c = 0; c < 3; ++c) {
        unsigned a = __reduce_min_sync(kFull, ordered(lo[c]));
        unsigned b = __reduce_max_sync(kFull, ordered(hi[c]));
        if ((threadIdx.x & 31) == 0) {
            atomicMin(flags + 2 + c, a);
            atomicMax(flags + 5 + c, b);
        }
    }
}

__device__ __forceinline__ unsigned long long spread3(unsigned v) {
    unsigned long long x = v & 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__global__ void k_morton(const float* verts, const int32_t* tris, long long nt, const unsigned* flags, int bits,
                         unsigned long long* keys, unsigned* vals) {
    // one scale for all three axes (cubic cells): per-axis scales would make
    // the cells of flat or thin meshes into slabs whose boxes are far from
    // the surface they bound
    float lo[3], ext[3], e = 0.f;
    for (int c = 0; c < 3; ++c) {
        lo[c] = unordered(flags[2 + c]);
        e = fmaxf(e, __fsub_rn(unordered(flags[5 + c]), lo[c]));
    }
    for (int c = 0; c < 3; ++c) ext[c] = e;
    const float cells = (float)(1u << bits);
    const unsigned top = (1u << bits) - 1u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        unsigned q[3];
        for (int c = 0; c < 3; ++c) {
            // explicit round-to-nearest steps (no contraction), so that the
            // codes can be reproduced bit for bit on the host
            float s = __fadd_rn(__fadd_rn(verts[3ll * tris[3 * t] + c], verts[3ll * tris[3 * t + 1] + c]),
                                verts[3ll * tris[3 * t + 2] + c]);
            float x = __fsub_rn(__fmul_rn(s, 1.0f / 3.0f), lo[c]);
            float f = ext[c] > 0.f ? __fmul_rn(__fdiv_rn(x, ext[c]), cells) : 0.f;
            unsigned qi = f <= 0.f ? 0u : (f >= (float)top ? top : (unsigned)f);
            q[c] = qi;
        }
        keys[t] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
        vals[t] = (unsigned)t;
    }
}

// ---- stable LSD radix sort of (64-bit key, 32-bit value), 8 bits per pass

__global__ void k_rs_hist(const unsigned long long* keys, long long n, int shift, unsigned* hist) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortItems; ++i) {
        long long j = base + (long long)i * kSortThreads + threadIdx.x;
        if (j < n) atomicAdd(&h[(unsigned)(keys[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m words in place, in three launches: every CTA of
// kScanCtas sums its contiguous chunk (k_scan_sums), one CTA scans those sums
// (k_scan_top), and every CTA scans its chunk tile by tile from its offset
// (k_scan_chunks).  Loads and stores are coalesced.
constexpr int kScanCtas = 256;
constexpr int kScanThreads = 256;
static_assert(kScanCtas == kScanThreads, "k_scan_top scans one sum per thread");

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* total) {
    __shared__ unsigned warp_sum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < kScanThreads / 32 ? warp_sum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_sum[lane] = w;
    }
    __syncthreads();
    const unsigned before = warp ? warp_sum[warp - 1] : 0u;
    *total = warp_sum[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_sums(const unsigned* a, long long m, unsigned* sums) {
    const long long chunk = (m + kScanCtas - 1) / kScanCtas;
    const long long b = blockIdx.x * chunk, e = b + chunk < m ? b + chunk : m;
    unsigned s = 0;
    for (long long i = b + threadIdx.x; i < e; i += kScanThreads) s += a[i];
    unsigned total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_top(unsigned* sums) {
    unsigned total;
    const unsigned v = sums[threadIdx.x];
    const unsigned x = block_excl_scan(v, &total);
    sums[threadIdx.x] = x;
}

__global__ void k_scan_chunks(unsigned* a, long long m, const unsigned* sums) {
    const long long chunk = (m + kScanCtas - 1) / kScanCtas;
    const long long b = blockIdx.x * chunk, e = b + chunk < m ? b + chunk : m;
    unsigned run = sums[blockIdx.x];
    for (long long t = b; t < e; t += kScanThreads) {
        const long long i = t + threadIdx.x;
        const unsigned v = i < e ? a[i] : 0u;
        unsigned total;
        const unsigned x = block_excl_scan(v, &total);
        if (i < e) a[i] = run + x;
        run += total;
    }
}

__global__ void k_rs_scatter(const unsigned long long* kin, const unsigned* vin, unsigned long long* kout,
                             unsigned* vout, long long n, int shift, const unsigned* hist) {
    __shared__ unsigned wcnt[kSortThreads / 32][256];
    __shared__ unsigned run[256];
    __shared__ unsigned off[256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    run[threadIdx.x] = 0;
    off[threadIdx.x] = hist[(long long)threadIdx.x * gridDim.x + blockIdx.x];
    long long base = (long long)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortItems; ++i) {
        for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        long long j = base + (long long)i * kSortThreads + threadIdx.x;
        bool ok = j < n;
        unsigned long long key = ok ? kin[j] : 0ull;
        unsigned val = ok ? vin[j] : 0u;
        unsigned d = ok ? (unsigned)(key >> shift) & 255u : 256u + (unsigned)lane;  // unique dummy digit
        unsigned peers = __match_any_sync(kFull, d);
        unsigned rank = __popc(peers & lanemask_lt());
        if (ok && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over warps, then advance the running count
        {
            unsigned acc = 0;
            for (int w = 0; w < kSortThreads / 32; ++w) {
                unsigned c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = acc;
                acc += c;
            }
            unsigned r0 = run[threadIdx.x];
            run[threadIdx.x] = r0 + acc;
            // stash the pre-advance running count in the slot of warp 0's prefix
            // (warp 0 prefix is always 0, so store r0 there and add below)
            wcnt[0][threadIdx.x] = r0;
            for (int w = 1; w < kSortThreads / 32; ++w) wcnt[w][threadIdx.x] += r0;
        }
        __syncthreads();
        if (ok) {
            unsigned pos = off[d] + wcnt[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

constexpr int kTreeLevels = 8;  // tree levels one CTA reduces (2^8 = 256 nodes in, one out)

// A node box (lo xyz, hi xyz, 24 bytes, 8-byte aligned) as three float2 stores.
__device__ __forceinline__ void store_box(float* o, const float lo[3], const float hi[3]) {
    float2* p = reinterpret_cast<float2*>(o);
    p[0] = make_float2(lo[0], lo[1]);
    p[1] = make_float2(lo[2], hi[0]);
    p[2] = make_float2(hi[1], hi[2]);
}

// Subtree union shared by the two tree kernels: on entry thread i holds node
// box (lo, hi) of the CTA's 2^levels consecutive nodes of depth d (heap ids
// from first = 2^d + CTA offset); each step makes node k of the level above
// the union of its children 2k, 2k+1 (Section 4: tight children make a tight
// parent) and stores it.  At the root (depth 0) the root box goes to
// root_out[0..5] and max |coordinate| to *P_out, when given.
__device__ __forceinline__ void reduce_subtree(float* box, long long first, int levels, float lo[3], float hi[3],
                                               float* root_out, float* P_out) {
    __shared__ float sb[6 << kTreeLevels];
    const int i = threadIdx.x;
    for (int s = 1; s <= levels; ++s) {
        sb[6 * i + 0] = lo[0]; sb[6 * i + 1] = lo[1]; sb[6 * i + 2] = lo[2];
        sb[6 * i + 3] = hi[0]; sb[6 * i + 4] = hi[1]; sb[6 * i + 5] = hi[2];
        __syncthreads();
        const int n = (int)blockDim.x >> s;
        if (i < n) {
            const float* l = sb + 12 * i;
            const float* r = l + 6;
            lo[0] = fminf(l[0], r[0]); lo[1] = fminf(l[1], r[1]); lo[2] = fminf(l[2], r[2]);
            hi[0] = fmaxf(l[3], r[3]); hi[1] = fmaxf(l[4], r[4]); hi[2] = fmaxf(l[5], r[5]);
        }
        __syncthreads();
        if (i < n) store_box(box + 6 * ((first >> s) + i), lo, hi);
    }
    if ((first >> levels) == 1 && i == 0) {
        if (root_out)
            for (int c = 0; c < 3; ++c) { root_out[c] = lo[c]; root_out[3 + c] = hi[c]; }
        if (P_out) {
            float P = 0.f;
            for (int c = 0; c < 3; ++c) P = fmaxf(P, fmaxf(fabsf(lo[c]), fabsf(hi[c])));
            *P_out = P;
        }
    }
}

// leaves: leaf l owns sorted triangles [floor(l T / 2^L), floor((l+1) T / 2^L)).
// One thread per leaf, 2^levels leaves per CTA: gather the leaf's triangles in
// sorted order (order[j] = original index of sorted triangle j), store them
// and the exact leaf box, then the CTA's subtree above its leaves.  The build
// (stris_in == nullptr) reads each triangle's vertex indices through order
// and stores them in leaf order (stris_out); the refit of a deformed mesh
// reads them from there, contiguously, so its vertex gathers wait on one
// load instead of two dependent ones.
// bad != nullptr: a non-finite coordinate sets *bad (the refit's check; the
// build validated the vertices before sorting).
__global__ void k_leaves(const float* verts, const int32_t* tris, long long nt, int L, const unsigned* order,
                         const int32_t* stris_in, int32_t* stris_out, float4* tri, float* box, int levels,
                         unsigned* bad, float* root_out, float* P_out) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // grid x block = 2^L exactly
    const long long s = (long long)(((unsigned long long)l * (unsigned long long)nt) >> L);
    const long long e = (long long)(((unsigned long long)(l + 1) * (unsigned long long)nt) >> L);
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    bool finite = true;
    for (long long j = s; j < e; ++j) {
        const unsigned id = order[j];
        int vi[3];
        if (stris_in) {
            vi[0] = stris_in[3 * j]; vi[1] = stris_in[3 * j + 1]; vi[2] = stris_in[3 * j + 2];
        } else {
            vi[0] = tris[3ll * id]; vi[1] = tris[3ll * id + 1]; vi[2] = tris[3ll * id + 2];
            if (stris_out) { stris_out[3 * j] = vi[0]; stris_out[3 * j + 1] = vi[1]; stris_out[3 * j + 2] = vi[2]; }
        }
        float v[9];
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) {
                const float x = verts[3ll * vi[k] + c];
                finite = finite && isfinite(x);
                v[3 * k + c] = x;
                lo[c] = fminf(lo[c], x);
                hi[c] = fmaxf(hi[c], x);
            }
        tri[3 * j] = make_float4(v[0], v[1], v[2], v[3]);
        tri[3 * j + 1] = make_float4(v[4], v[5], v[6], v[7]);
        tri[3 * j + 2] = make_float4(v[8], __int_as_float((int)id), 0.f, 0.f);
    }
    if (bad && __syncthreads_or(!finite) && threadIdx.x == 0) atomicOr(bad, 1u);
    store_box(box + 6 * ((1ll << L) + l), lo, hi);
    reduce_subtree(box, (1ll << L) + (long long)blockIdx.x * blockDim.x, levels, lo, hi, root_out, P_out);
}

// levels above depth d: each CTA loads 2^levels consecutive nodes of depth d
// and reduces them (grid x block = 2^d exactly)
__global__ void k_reduce_up(float* box, int d, int levels, float* root_out, float* P_out) {
    const long long first = (1ll << d) + (long long)blockIdx.x * blockDim.x;
    const float* b = box + 6 * (first + threadIdx.x);
    float lo[3] = {b[0], b[1], b[2]}, hi[3] = {b[3], b[4], b[5]};
    reduce_subtree(box, first, levels, lo, hi, root_out, P_out);
}

// all boxes from the sorted order: leaves plus the lowest levels, then one
// launch per further kTreeLevels levels (three launches for 2^22 leaves)
void tree_boxes(const float* verts, const int32_t* tris, long long nt, int L, const unsigned* order,
                const int32_t* stris_in, int32_t* stris_out, float4* tri, float* box, unsigned* bad, float* root_out,
                float* P_out, cudaStream_t st) {
    int lv = L < kTreeLevels ? L : kTreeLevels;
    k_leaves<<<(unsigned)(1ll << (L - lv)), 1u << lv, 0, st>>>(verts, tris, nt, L, order, stris_in, stris_out, tri, box,
                                                                 lv, bad, root_out, P_out);
    for (int d = L - lv; d > 0; d -= lv) {
        lv = d < kTreeLevels ? d : kTreeLevels;
        k_reduce_up<<<(unsigned)(1ll << (d - lv)), 1u << lv, 0, st>>>(box, d, lv, root_out, P_out);
    }
}

int grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

}  // namespace

// the histogram (256 digits x tiles) followed by the scan's per-CTA sums
size_t build_hist_words(long long nt) {
    long long nb = (nt + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    return (size_t)nb * 256 + kScanCtas;
}

cudaError_t build_validate(const BuildBuffers& b, cudaStream_t st) {
    k_init_flags<<<1, 32, 0, st>>>(b.flags);
    k_validate<<<grid_for(b.nt, 256), 256, 0, st>>>(b.verts, b.nv, b.tris, b.nt, b.flags);
    return cudaGetLastError();
}

int radix_sort_pairs(unsigned long long* const keys[2], unsigned* const vals[2], long long n, int key_bits,
                     unsigned* hist, cudaStream_t st) {
    const long long nb = (n + kSortTile - 1) / kSortTile;
    const int passes = (key_bits + 7) / 8;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        k_rs_hist<<<(unsigned)nb, kSortThreads, 0, st>>>(keys[cur], n, 8 * p, hist);
        unsigned* sums = hist + nb * 256;
        k_scan_sums<<<kScanCtas, kScanThreads, 0, st>>>(hist, nb * 256, sums);
        k_scan_top<<<1, kScanThreads, 0, st>>>(sums);
        k_scan_chunks<<<kScanCtas, kScanThreads, 0, st>>>(hist, nb * 256, sums);
        k_rs_scatter<<<(unsigned)nb, kSortThreads, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n,
                                                             8 * p, hist);
        cur ^= 1;
    }
    return cur;
}

cudaError_t build_tree(const BuildBuffers& b, cudaStream_t st) {
    k_morton<<<grid_for(b.nt, 256), 256, 0, st>>>(b.verts, b.tris, b.nt, b.flags, b.morton_bits, b.keys[0],
                                                  b.vals[0]);
    const int cur = radix_sort_pairs(b.keys, b.vals, b.nt, 3 * b.morton_bits, b.hist, st);
    cudaError_t e = cudaMemcpyAsync(b.order, b.vals[cur], sizeof(unsigned) * b.nt, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    tree_boxes(b.verts, b.tris, b.nt, b.L, b.order, nullptr, b.stris, b.tri, b.box, nullptr, nullptr, nullptr, st);
    return cudaGetLastError();
}

cudaError_t build_refit(const BuildBuffers& b, float* P_out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b.flags, 0, 16 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    tree_boxes(b.verts, b.tris, b.nt, b.L, b.order, b.stris, nullptr, b.tri, b.box, b.flags + 1,
               reinterpret_cast<float*>(b.flags + 8), P_out, st);
    return cudaGetLastError();
}

}  // namespace gd
