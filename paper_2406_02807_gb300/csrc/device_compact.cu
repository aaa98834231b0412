// De-duplicated ("compact") affordance sets.  Alg. 1 stores every point once per leaf
// cell that affords it, so a set is a copy of nearby cloud points and the total grows
// with the replication (Sec. VII names compressing or de-duplicating the sets as the
// way to larger clouds).  The compact form stores each point once:
//
//  * the cloud is put in Z-order (rank[id] = position along the curve) and cut into
//    chunks of 32 consecutive points, stored as 8 four-point blocks in three planes
//    (+inf in the unused slots of the last chunk), each with its FP32 box;
//  * every leaf keeps the ascending list of the chunks that hold at least one point of
//    its set P_i, and a record {lo, first list entry, hi, number of chunks} whose box
//    is still the box of P_i.
//
// The listed chunks hold a superset of P_i within the cloud, so a scan over them finds
// a point within r exactly when the scan of P_i does (a hit on any cloud point is a
// brute-force hit, and Lemma 1 puts every brute-force hit in P_i); the leaf box of P_i
// still rejects only spheres that miss P_i, hence miss the cloud.  Z-order keeps a
// chunk's points close together, so a set needs few chunks and a chunk box skips most
// of what it does not need.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/capt.h"
#include "capt_internal.h"
#include "device_common.cuh"
#include "kernels.h"
#include "morton.cuh"

namespace capt {
namespace {

constexpr uint32_t kChunkPoints = kChunkBlocks * 4;

// Morton key of every point (x most significant in each bit triple, over the cloud's
// bounding box), split in its low 32 and high 31 bits, with the point index as value.
__global__ void kc_keys(const float* __restrict__ cloud, uint32_t n, float lx, float ly, float lz, float hx, float hy,
                        float hz, uint32_t* __restrict__ klo, uint32_t* __restrict__ khi, uint32_t* __restrict__ idx) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* p = cloud + 3 * (size_t)i;
    const uint64_t k = (spread21(morton_q(p[0], lx, hx)) << 2) | (spread21(morton_q(p[1], ly, hy)) << 1) |
                       spread21(morton_q(p[2], lz, hz));
    klo[i] = (uint32_t)k;
    khi[i] = (uint32_t)(k >> 32);
    idx[i] = i;
}

__global__ void kc_gather(const uint32_t* __restrict__ src, const uint32_t* __restrict__ perm, uint32_t n,
                          uint32_t* __restrict__ dst) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = src[perm[j]];
}

__global__ void kc_rank(const uint32_t* __restrict__ order, uint32_t n, uint32_t* __restrict__ rank) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rank[order[i]] = i;
}

// Slot s of the Z-ordered cloud: block s / 4, element s % 4, in each of the three planes.
__global__ void kc_blocks(const float* __restrict__ cloud, const uint32_t* __restrict__ order, uint32_t n,
                          uint64_t slots, uint64_t plane, float* __restrict__ cb) {
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= slots) return;
    const uint64_t b = s >> 2, u = s & 3u;
    const uint32_t id = s < n ? order[s] : 0u;
    for (int d = 0; d < 3; d++) cb[((uint64_t)d * plane + b) * 4u + u] = s < n ? cloud[3 * (size_t)id + d] : INFINITY;
}

// One warp per leaf with a bitmap of the cloud's chunks in shared memory: the chunks
// of the set's points are marked, then counted (COUNT pass) or written in ascending
// order at the leaf's list offset together with its compact record (FILL pass).
template <bool FILL>
__global__ void kc_leaf_chunks(const LeafRec* __restrict__ leaves, const uint32_t* __restrict__ ids,
                               const uint32_t* __restrict__ rank, uint32_t N, uint32_t n_words,
                               uint32_t* __restrict__ counts, const unsigned long long* __restrict__ offsets,
                               uint32_t* __restrict__ clist, LeafRec* __restrict__ cleaves) {
    extern __shared__ uint32_t bm_all[];
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    uint32_t* bm = bm_all + (size_t)warp * n_words;
    for (uint32_t leaf = blockIdx.x * wpb + warp; leaf < N; leaf += gridDim.x * wpb) {
        const LeafRec r = leaves[leaf];
        for (uint32_t w = lane; w < n_words; w += 32) bm[w] = 0u;
        __syncwarp();
        const uint64_t s0 = 4ull * r.block;
        for (uint32_t j = lane; j < r.count; j += 32) {
            const uint32_t ch = rank[ids[s0 + j]] / kChunkPoints;
            atomicOr(&bm[ch >> 5], 1u << (ch & 31u));
        }
        __syncwarp();
        if (!FILL) {
            uint32_t c = 0;
            for (uint32_t w = lane; w < n_words; w += 32) c += __popc(bm[w]);
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane == 0) counts[leaf] = c;
        } else {
            const unsigned long long first = offsets[leaf];
            unsigned long long pos = first;
            for (uint32_t base = 0; base < n_words; base += 32) {
                const uint32_t w = base + lane;
                uint32_t bits = w < n_words ? bm[w] : 0u;
                const uint32_t pc = __popc(bits);
                const uint32_t incl = warp_incl_scan(pc);
                unsigned long long p = pos + incl - pc;
                while (bits) {
                    const uint32_t b = (uint32_t)__ffs(bits) - 1u;
                    clist[p++] = w * 32u + b;
                    bits &= bits - 1u;
                }
                pos += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) {
                LeafRec c = r;
                c.block = (uint32_t)first;
                c.count = (uint32_t)(offsets[leaf + 1] - first);
                cleaves[leaf] = c;
            }
        }
        __syncwarp();
    }
}

unsigned grid_for(uint64_t work, unsigned block) { return (unsigned)std::max<uint64_t>(1, (work + block - 1) / block); }

}  // namespace

void CompactSets::release() {
    for (void* p : {cleaves, clist, cblocks, ccbox})
        if (p) cudaFree(p);
    cleaves = clist = cblocks = ccbox = nullptr;
    n_chunks = list_len = 0;
    bytes = 0;
}

int device_compact(const DevArgs& t, size_t n, cudaStream_t st, CompactSets& out, std::string& err) {
    out.release();
    const uint32_t N = t.N;
    const uint64_t n_chunks = std::max<uint64_t>(1, (n + kChunkPoints - 1) / kChunkPoints);
    const uint64_t n_blocks = n_chunks * kChunkBlocks;
    const uint32_t n_words = (uint32_t)((n_chunks + 31) / 32);
    const size_t bm_bytes = (size_t)n_words * 4u;
    if (bm_bytes > 200u * 1024u) {
        err = "compact sets: too many chunks for the per-warp bitmap (at most 1.6M chunks of 32 points)";
        return CAPT_E_RANGE;
    }
    uint32_t *order = nullptr, *rank = nullptr, *counts = nullptr, *ka = nullptr, *kb = nullptr, *vb = nullptr,
             *khi = nullptr, *hist = nullptr;
    unsigned long long* offsets = nullptr;
    auto cleanup = [&]() {
        for (void* p : {(void*)order, (void*)rank, (void*)counts, (void*)offsets, (void*)ka, (void*)kb, (void*)vb,
                        (void*)khi, (void*)hist})
            if (p) cudaFree(p);
    };
    auto cuda_err = [&](cudaError_t e, const char* what) {
        cudaGetLastError();
        cleanup();
        out.release();
        err = std::string("compact sets, ") + what + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? CAPT_E_NOMEM : CAPT_E_CUDA;
    };
#define DC_TRY(call, what)                             \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_err(e_, what); \
    } while (0)
    const size_t sz_n = std::max<size_t>(1, n) * sizeof(uint32_t);
    DC_TRY(cudaMalloc((void**)&order, sz_n), "cudaMalloc order");
    DC_TRY(cudaMalloc((void**)&rank, sz_n), "cudaMalloc rank");
    DC_TRY(cudaMalloc((void**)&counts, (size_t)N * sizeof(uint32_t)), "cudaMalloc counts");
    DC_TRY(cudaMalloc((void**)&offsets, ((size_t)N + 1) * sizeof(unsigned long long)), "cudaMalloc offsets");
    DC_TRY(cudaMalloc(&out.cleaves, (size_t)N * sizeof(LeafRec)), "cudaMalloc leaf records");
    DC_TRY(cudaMalloc(&out.cblocks, n_blocks * 12 * sizeof(float)), "cudaMalloc blocks");
    DC_TRY(cudaMalloc(&out.ccbox, n_chunks * 8 * sizeof(float)), "cudaMalloc chunk boxes");
    if (n) {
        // the cloud's order along its Z-order curve: a stable sort by the keys' low 32
        // bits, then by their high 31 bits, so ties keep the point order
        const uint32_t un = (uint32_t)n;
        DC_TRY(cudaMalloc((void**)&ka, sz_n), "cudaMalloc keys");
        DC_TRY(cudaMalloc((void**)&kb, sz_n), "cudaMalloc keys");
        DC_TRY(cudaMalloc((void**)&vb, sz_n), "cudaMalloc values");
        DC_TRY(cudaMalloc((void**)&khi, sz_n), "cudaMalloc keys");
        DC_TRY(cudaMalloc((void**)&hist, 256 * sizeof(uint32_t) * ((n + 255) / 256)), "cudaMalloc histogram");
        kc_keys<<<grid_for(n, 256), 256, 0, st>>>(t.cloud, un, t.lo[0], t.lo[1], t.lo[2], t.hi[0], t.hi[1], t.hi[2],
                                                  ka, khi, order);
        DC_TRY(cudaGetLastError(), "key launch");
        int rc = launch_sort_pairs(ka, order, kb, vb, un, 4, hist, st, err);
        if (rc == CAPT_OK) {
            kc_gather<<<grid_for(n, 256), 256, 0, st>>>(khi, order, un, ka);
            rc = launch_sort_pairs(ka, order, kb, vb, un, 4, hist, st, err);
        }
        if (rc != CAPT_OK) {
            cleanup();
            out.release();
            return rc;
        }
        kc_rank<<<grid_for(n, 256), 256, 0, st>>>(order, un, rank);
    }
    kc_blocks<<<grid_for(n_chunks * kChunkPoints, 256), 256, 0, st>>>(t.cloud, order, (uint32_t)n,
                                                                        n_chunks * kChunkPoints, n_blocks,
                                                                        static_cast<float*>(out.cblocks));
    DC_TRY(cudaGetLastError(), "cloud blocks launch");
    if (launch_chunk_boxes(static_cast<const float*>(out.cblocks), n_blocks, static_cast<float*>(out.ccbox), st,
                           err) != CAPT_OK) {
        cleanup();
        out.release();
        return CAPT_E_CUDA;
    }
    // warps per block: as many bitmaps as fit in 48 KB (at least one)
    const unsigned wpb = (unsigned)std::max<size_t>(1, std::min<size_t>(8, (48u * 1024u) / bm_bytes));
    const size_t smem = wpb * bm_bytes;
    const unsigned grid = (unsigned)std::min<uint64_t>((N + wpb - 1) / wpb, (uint64_t)sm_count() * 16);
    DC_TRY(cudaFuncSetAttribute((const void*)kc_leaf_chunks<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem),
           "smem attribute");
    DC_TRY(cudaFuncSetAttribute((const void*)kc_leaf_chunks<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem),
           "smem attribute");
    kc_leaf_chunks<false><<<grid, wpb * 32, smem, st>>>(t.leaves, t.ids, rank, N, n_words, counts, nullptr, nullptr,
                                                       nullptr);
    DC_TRY(cudaGetLastError(), "chunk count launch");
    if (launch_scan64(counts, N, offsets, st, err) != CAPT_OK) {
        cleanup();
        out.release();
        return CAPT_E_CUDA;
    }
    unsigned long long total = 0;
    DC_TRY(cudaMemcpyAsync(&total, offsets + N, sizeof(total), cudaMemcpyDeviceToHost, st), "list length");
    DC_TRY(cudaStreamSynchronize(st), "list length");
    if (total >= (1ull << 32)) {
        cleanup();
        out.release();
        err = "compact sets: more than 2^32 list entries";
        return CAPT_E_RANGE;
    }
    DC_TRY(cudaMalloc(&out.clist, std::max<unsigned long long>(1, total) * sizeof(uint32_t)), "cudaMalloc list");
    kc_leaf_chunks<true><<<grid, wpb * 32, smem, st>>>(t.leaves, t.ids, rank, N, n_words, nullptr, offsets,
                                                      static_cast<uint32_t*>(out.clist),
                                                      static_cast<LeafRec*>(out.cleaves));
    DC_TRY(cudaGetLastError(), "chunk list launch");
    DC_TRY(cudaStreamSynchronize(st), "compact sets");
#undef DC_TRY
    cleanup();
    out.n_chunks = n_chunks;
    out.list_len = total;
    out.bytes = (size_t)N * sizeof(LeafRec) + n_blocks * 12 * sizeof(float) + n_chunks * 8 * sizeof(float) +
                std::max<unsigned long long>(1, total) * sizeof(uint32_t);
    return CAPT_OK;
}

}  // namespace capt
