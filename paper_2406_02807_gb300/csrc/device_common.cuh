// Device helpers shared by the CAPT kernels (sm_103a).
//
// Every floating-point expression on the query path uses the explicitly rounded
// intrinsics (__fadd_rn, __fsub_rn, __fmul_rn): nvcc never fuses them into an FMA, so
// a kernel computes exactly the FP32 predicate ((x0-p0)^2 + (x1-p1)^2) + (x2-p2)^2 <=
// fl(r*r) that defines a collision.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "capt_internal.h"

namespace capt {

// Device status bits (latched by kernels, read by capt_device_status).
constexpr int kStatusTimeout = 1;
constexpr int kStatusBounds = 2;

// Poll limits of the bounded mbarrier waits on bulk copies into shared memory.  A copy
// of a few KB lands within microseconds; a wait that gives up after kStagePolls latches
// kStatusTimeout and the kernel carries on from global memory.  Before that shared
// memory can be reused (by the warp's own direct loads, or by the next block on the SM
// once this one exits) the copy still in flight is waited for again, up to kDrainPolls
// (about 2^26 polls, tenths of a second): a copy outstanding after that means the memory
// system itself has failed, and the status word already says so.  A test build sets
// CAPT_STAGE_POLLS to 0, which makes every first wait give up at once while the copies
// still complete, to exercise this path.
#ifndef CAPT_STAGE_POLLS
#define CAPT_STAGE_POLLS (1u << 22)
#endif
#ifndef CAPT_DRAIN_POLLS
#define CAPT_DRAIN_POLLS (1u << 26)
#endif
constexpr uint32_t kStagePolls = CAPT_STAGE_POLLS;
constexpr uint32_t kDrainPolls = CAPT_DRAIN_POLLS;

// Bytes of the blocked split prefix staged into shared memory (a multiple of 16), and
// the offset of what follows it in dynamic shared memory (rounded up to 128).
__host__ __device__ __forceinline__ uint32_t stage_bytes(const DevArgs& t) { return t.stage_floats * 4u; }
__host__ __device__ __forceinline__ uint32_t stage_offset(const DevArgs& t) {
    return (stage_bytes(t) + 127u) & ~127u;
}

__device__ __forceinline__ float sq_dist(float x, float y, float z, float px, float py, float pz) {
    float dx = __fsub_rn(x, px);
    float dy = __fsub_rn(y, py);
    float dz = __fsub_rn(z, pz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Squared distance from (x, y, z) to the box [lo, hi] (clamped per axis, same order).
__device__ __forceinline__ float box_dist2(float x, float y, float z, const float4& a, const float4& b) {
    float gx = __fsub_rn(x, fminf(fmaxf(x, a.x), b.x));
    float gy = __fsub_rn(y, fminf(fmaxf(y, a.y), b.y));
    float gz = __fsub_rn(z, fminf(fmaxf(z, a.z), b.z));
    return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
}

// Three levels of the descent on one 8-float block (axes x, y, z in that order):
// i <- 2i + 1 + [x_d > T_i] three times.  `bits` collects the comparison results, which
// is the leaf's position once all L levels are done; `u` is the next block.
__device__ __forceinline__ void step3(float x, float y, float z, const float4& a, const float4& b, uint32_t& u,
                                      uint32_t& bits) {
    const uint32_t c0 = x > a.x ? 1u : 0u;
    const uint32_t c1 = y > (c0 ? a.z : a.y) ? 1u : 0u;
    const float t2 = c0 ? (c1 ? b.z : b.y) : (c1 ? b.x : a.w);
    const uint32_t c2 = z > t2 ? 1u : 0u;
    const uint32_t child = (c0 << 2) | (c1 << 1) | c2;
    u = 8u * u + 1u + child;
    bits = (bits << 3) | child;
}

// Fixed-length descent of Alg. 3 (exactly L = 3K + R comparisons, branch-free), over the
// blocked split array.  The first t.Ks block levels (and the tail, if t.tail_staged)
// come from the shared-memory copy `Ts` when it is non-null, the rest through the
// read-only cache.  Returns the leaf index i - (N - 1).
__device__ __forceinline__ uint32_t descend(float x, float y, float z, const DevArgs& t, const float* Ts) {
    uint32_t u = 0, bits = 0;
    int k = 0;
    if (Ts) {
        for (; k < t.Ks; k++) {
            const float4 a = *reinterpret_cast<const float4*>(Ts + 8u * u);
            const float4 b = *reinterpret_cast<const float4*>(Ts + 8u * u + 4u);
            step3(x, y, z, a, b, u, bits);
        }
    }
    for (; k < t.K; k++) {
        const float4* g = reinterpret_cast<const float4*>(t.T + 8ull * u);
        const float4 a = __ldg(g);
        const float4 b = __ldg(g + 1);
        step3(x, y, z, a, b, u, bits);
    }
    if (t.R) {
        const size_t o = (size_t)t.tail_off + 4ull * bits;
        const float4 q = (Ts && t.tail_staged) ? *reinterpret_cast<const float4*>(Ts + o)
                                               : __ldg(reinterpret_cast<const float4*>(t.T + o));
        const uint32_t c0 = x > q.x ? 1u : 0u;
        if (t.R == 2) {
            const uint32_t c1 = y > (c0 ? q.z : q.y) ? 1u : 0u;
            bits = (bits << 2) | (c0 << 1) | c1;
        } else {
            bits = (bits << 1) | c0;
        }
    }
    return bits;
}

// Stage the blocked prefix into `smem`; returns the pointer to use, or nullptr when
// there is nothing to stage or the copy did not complete (then T is read globally).
__device__ __forceinline__ const float* stage_splits(const DevArgs& t, void* smem, uint64_t* bar);

__device__ __forceinline__ void load_leaf(const LeafRec* leaves, uint32_t leaf, float4& a, float4& b) {
    const float4* p = reinterpret_cast<const float4*>(leaves + leaf);
    a = __ldg(p);
    b = __ldg(p + 1);
}

// ------------------------------------------------------------------------------------
// Staging of the top levels of T into shared memory with the bulk asynchronous copy
// engine (cp.async.bulk, completion counted on an mbarrier).  One elected thread
// issues the copies; every thread waits with a bounded spin.  When the wait gives up
// the block latches kStatusTimeout and reads T from global memory instead.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Returns true when the staged copy is complete and readable by the whole block.
// `bytes` must be a multiple of 16; src and dst 16-byte aligned.
__device__ __forceinline__ bool stage_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              int* status) {
    const uint32_t b = smem_u32(bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile(
            "{\n\t.reg .b64 st;\n\t"
            "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(b),
            "r"(bytes)
            : "memory");
        const uint32_t d = smem_u32(dst);
        const char* s = static_cast<const char*>(src);
        for (uint32_t off = 0; off < bytes; off += 16384u) {
            uint32_t sz = bytes - off < 16384u ? bytes - off : 16384u;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    d + off),
                "l"(s + off), "r"(sz), "r"(b)
                : "memory");
        }
    }
    // bounded wait: kStagePolls polls (far beyond the microseconds a 32 KB copy takes)
    bool done = false;
    for (uint32_t it = 0; it < kStagePolls; it++) {
        if (mbar_try_wait(b, 0)) { done = true; break; }
    }
    int all_done = __syncthreads_and(done ? 1 : 0);
    if (!all_done) {
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        // the block reads T from global memory from here on and never touches the
        // staged region; the copy still in flight is waited for (kDrainPolls) before
        // the block goes on, so it has landed before the block can exit and hand its
        // shared memory to the next one
        for (uint32_t it = 0; it < kDrainPolls; it++)
            if (mbar_try_wait(b, 0)) break;
        __syncthreads();
        return false;
    }
    return true;
}

__device__ __forceinline__ const float* stage_splits(const DevArgs& t, void* smem, uint64_t* bar) {
    const uint32_t bytes = stage_bytes(t);
    if (bytes == 0) return nullptr;
    return stage_to_smem(smem, t.T, bytes, bar, t.status) ? reinterpret_cast<const float*>(smem) : nullptr;
}

// L2 prefetch of [p, p + bytes) by the bulk copy engine (no registers or shared memory
// held while it is in flight); the range is trimmed inward to 16-byte boundaries, as
// the instruction requires, so it never reaches outside the buffer.
__device__ __forceinline__ void prefetch_l2(const void* p, uint64_t bytes) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15u) & ~uintptr_t(15);
    const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
    if (e > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

// Ask L2 for the line holding p (a hint: no data returned, no fault).
__device__ __forceinline__ void prefetch_l2_line(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p) : "memory");
}

// Distance-bound grid (dist_grid.cu): 0 when the grid proves that the sphere (x, r)
// misses every cloud point under the FP32 test, 1 when it proves that it hits one, 2
// when it cannot tell.
// Cell of the distance-bound grid that the kernels assign to x: floor(fl(fl(x - org) *
// inv_h)) per axis, clamped to the grid.  `inside`: x is inside the grid box, and then
// the cell (grown by h / 100) holds x.
__device__ __forceinline__ uint32_t grid_cell(const GridShape& g, float x, float y, float z, bool& inside) {
    const float ux = __fmul_rn(__fsub_rn(x, g.org[0]), g.inv_h);
    const float uy = __fmul_rn(__fsub_rn(y, g.org[1]), g.inv_h);
    const float uz = __fmul_rn(__fsub_rn(z, g.org[2]), g.inv_h);
    inside = ux >= 0.f && uy >= 0.f && uz >= 0.f && ux < (float)g.n[0] && uy < (float)g.n[1] && uz < (float)g.n[2];
    const uint32_t i = (uint32_t)fminf(fmaxf(ux, 0.f), (float)(g.n[0] - 1));
    const uint32_t j = (uint32_t)fminf(fmaxf(uy, 0.f), (float)(g.n[1] - 1));
    const uint32_t k = (uint32_t)fminf(fmaxf(uz, 0.f), (float)(g.n[2] - 1));
    return (k * (uint32_t)g.n[1] + j) * (uint32_t)g.n[0] + i;
}

__device__ __forceinline__ int grid_classify(const DevArgs& t, float x, float y, float z, float r) {
    const GridShape& g = t.g;
    bool inside;
    const uint32_t c = grid_cell(g, x, y, z, inside);
    const unsigned short q = __ldg(reinterpret_cast<const unsigned short*>(t.grid) + c);
    if (__fmul_rn((float)(q & 0xffu), g.unit) > r) return 0;
    if (inside && (q >> 8) < 255u && __fmul_rn((float)(q >> 8), g.unit) < r) return 1;
    return 2;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Order-preserving unsigned key of a float (-0 and +0 share one key, as they compare
// equal), and its inverse.
__host__ __device__ __forceinline__ uint32_t fkey_bits(uint32_t u) {
    if (u == 0x80000000u) u = 0u;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint32_t fkey(float f) { return fkey_bits(__float_as_uint(f)); }
__device__ __forceinline__ float fkey_float(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Inclusive warp prefix sum.
// Work scheduling of the persistent query kernels: with a counter (zeroed before the
// launch) a warp takes the next unclaimed tile whenever it needs one, so warps that
// draw cheap tiles take more of them; without one, warp w of the grid takes tiles
// w, w + warps, w + 2 warps, ...
struct TileSched {
    unsigned long long* ctr;
    uint64_t stride;
    __device__ __forceinline__ uint64_t first(uint64_t w) const { return ctr ? take() : w; }
    __device__ __forceinline__ uint64_t next(uint64_t cur) const { return ctr ? take() : cur + stride; }
    __device__ __forceinline__ uint64_t take() const {
        unsigned long long v = 0;
        if ((threadIdx.x & 31u) == 0) v = atomicAdd(ctr, 1ull);
        return __shfl_sync(0xffffffffu, v, 0);
    }
};

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (uint32_t)o) v += u;
    }
    return v;
}

}  // namespace capt
