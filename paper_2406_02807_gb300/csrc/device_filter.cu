// Space-filling-curve filter on the GPU (Alg. 2, Sec. IV-C).  The result is the host
// filter's bit for bit: the same kept points, in the same (last pass's curve) order.
//
// Per pass (one per axis permutation):
//  1. The survivors, taken in ascending point index, get their 63-bit Morton key (21
//     bits per axis over the input's bounding box, quantised in FP64 exactly as the
//     host does) and are sorted by it with a stable LSD radix sort: 8 digits of 8 bits,
//     4096 elements per block, stable inside a block because it ranks rounds of 256
//     elements in index order.
//  2. The greedy sweep of Alg. 2 keeps p_j iff its FP32 squared distance to the last
//     kept point exceeds fl(r^2).  That is a chain: with next(j) = the first k > j whose
//     distance to p_j exceeds the spacing, the kept positions are 0, next(0),
//     next(next(0)), ...  Every next(j) comes from an independent forward scan; the
//     chain is then marked by pointer doubling, ceil(log2 n) rounds in which every
//     marked position marks its 2^k-th successor (after round k every chain element of
//     rank below 2^(k+1) is marked).
//  3. The marked points survive into the next pass.
// The forward scans cost the lengths of the runs of points lying within the spacing of
// each other along the curve: a few points for sampled surfaces, but quadratic in the
// run length for many coincident points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "capt_internal.h"
#include "device_common.cuh"
#include "kernels.h"
#include "morton.cuh"

namespace capt {
namespace {

constexpr int kFT = 256;                  // threads per block
constexpr int kFE = 16;                   // elements per thread in the blocked kernels
constexpr uint32_t kFTile = kFT * kFE;    // 4096 elements per block
constexpr int kScanThreads = 1024;

// box: lo keys [0..2], hi keys [3..5], non-finite flag [6].
__global__ void kf_bbox(const float* __restrict__ pts, uint32_t n, uint32_t* __restrict__ box) {
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    uint32_t bad = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int d = 0; d < 3; d++) {
            const float v = pts[3 * (size_t)i + d];
            bad |= isfinite(v) ? 0u : 1u;
            const uint32_t k = fkey(v);
            lo[d] = min(lo[d], k);
            hi[d] = max(hi[d], k);
        }
    for (int o = 16; o > 0; o >>= 1)
        for (int d = 0; d < 3; d++) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    bad = __any_sync(0xffffffffu, bad != 0) ? 1u : 0u;
    if (lane_id() == 0) {
        for (int d = 0; d < 3; d++) {
            atomicMin(box + d, lo[d]);
            atomicMax(box + 3 + d, hi[d]);
        }
        if (bad) atomicOr(box + 6, 1u);
    }
}

// Spread quantised coordinates: q = min(2^21 - 1, floor((p - lo) / (hi - lo) * 2^21)) in
// FP64, q = 0 on an axis of zero extent.
__global__ void kf_spread(const float* __restrict__ pts, uint32_t n, const uint32_t* __restrict__ box,
                          uint64_t* __restrict__ sp) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < 3; a++)
        sp[3 * (size_t)i + a] = spread21(morton_q(pts[3 * (size_t)i + a], (double)fkey_float(box[a]),
                                                  (double)fkey_float(box[3 + a])));
}

// Block-wide exclusive prefix of one flag per thread (256 threads); returns the prefix
// and writes the block total to *total.  Uses ws[8].
__device__ __forceinline__ uint32_t block_prefix(bool f, uint32_t* ws, uint32_t* total) {
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) ws[warp] = __popc(b);
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kFT / 32; w++) {
        const uint32_t c = ws[w];
        before += (uint32_t)w < warp ? c : 0u;
        all += c;
    }
    __syncthreads();
    *total = all;
    return before + __popc(b & ((1u << lane) - 1u));
}

// Set flags per block of 4096 positions (positions < len, len = *d_len if given).
__global__ void __launch_bounds__(kFT) kf_flag_count(const uint8_t* __restrict__ flags, const uint32_t* d_len,
                                                      uint32_t len, uint32_t* __restrict__ counts) {
    __shared__ uint32_t ws[kFT / 32];
    if (d_len) len = *d_len;
    uint32_t c = 0;
    for (int r = 0; r < kFE; r++) {
        const uint32_t i = blockIdx.x * kFTile + (uint32_t)r * kFT + threadIdx.x;
        c += (i < len && flags[i]) ? 1u : 0u;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < kFT / 32; w++) s += ws[w];
        counts[blockIdx.x] = s;
    }
}

// Exclusive prefix of len values in place by one block; the sum goes to *total if given.
__global__ void __launch_bounds__(kScanThreads) kf_scan(uint32_t* __restrict__ v, uint32_t len,
                                                         uint32_t* __restrict__ total) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t base = 0; base < len; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < len ? v[i] : 0u;
        const uint32_t incl = warp_incl_scan(x);
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t y = lane < nw ? ws[lane] : 0u;
            y = warp_incl_scan(y);
            if (lane < nw) ws[lane] = y;
        }
        __syncthreads();
        const uint32_t before = carry + (warp ? ws[warp - 1] : 0u);
        if (i < len) v[i] = before + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// Stable compaction: out[k] = the k-th set position (or vals[position]) in order.
__global__ void __launch_bounds__(kFT) kf_flag_compact(const uint8_t* __restrict__ flags, const uint32_t* d_len,
                                                        uint32_t len, const uint32_t* __restrict__ offs,
                                                        const uint32_t* __restrict__ vals,
                                                        uint32_t* __restrict__ out) {
    __shared__ uint32_t ws[kFT / 32];
    if (d_len) len = *d_len;
    uint32_t base = offs[blockIdx.x];
    for (int r = 0; r < kFE; r++) {
        const uint32_t i = blockIdx.x * kFTile + (uint32_t)r * kFT + threadIdx.x;
        const bool f = i < len && flags[i];
        uint32_t tot;
        const uint32_t pre = block_prefix(f, ws, &tot);
        if (f) out[base + pre] = vals ? vals[i] : i;
        base += tot;
    }
}

// Morton keys of the survivors under one axis permutation (X[0] most significant in
// every bit triple), split into low and high words; val = point index.
__global__ void kf_keys(const uint32_t* __restrict__ asc, const uint32_t* __restrict__ d_m,
                        const uint64_t* __restrict__ sp, int x0, int x1, int x2, uint32_t* __restrict__ klo,
                        uint32_t* __restrict__ khi, uint32_t* __restrict__ val) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *d_m) return;
    const uint32_t i = asc[j];
    const uint64_t* s = sp + 3 * (size_t)i;
    const uint64_t key = (s[x0] << 2) | (s[x1] << 1) | s[x2];
    klo[j] = (uint32_t)key;
    khi[j] = (uint32_t)(key >> 32);
    val[j] = i;
}

// The radix-sort kernels take a tile of kFTile elements with kST threads, kSR rounds of
// kST consecutive elements each (a wide block: few rounds of dependent barriers).
constexpr int kST = 1024;
constexpr int kSR = (int)(kFTile / kST);

__global__ void __launch_bounds__(kST) kf_hist(const uint32_t* __restrict__ kw, const uint32_t* __restrict__ d_m,
                                               int shift, uint32_t* __restrict__ hist, uint32_t nblk) {
    __shared__ uint32_t h[256];
    if (threadIdx.x < 256) h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t m = *d_m;
    for (int r = 0; r < kSR; r++) {
        const uint32_t i = blockIdx.x * kFTile + (uint32_t)r * kST + threadIdx.x;
        if (i < m) atomicAdd(&h[(kw[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 256) hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];   // digit-major
}

// Stable scatter by the digit of ka at `shift`; kb and val travel with it.  Per round:
// each warp counts its digits (match_any), one thread per digit turns the per-warp
// counts into offsets (warps in order), and every element goes to base + warp offset +
// its rank among equal digits of its warp, so the order within a digit is the input
// order.
__global__ void __launch_bounds__(kST) kf_scatter(const uint32_t* __restrict__ ka, const uint32_t* __restrict__ kb,
                                                  const uint32_t* __restrict__ val, const uint32_t* __restrict__ d_m,
                                                  int shift, const uint32_t* __restrict__ off, uint32_t nblk,
                                                  uint32_t* __restrict__ ka_o, uint32_t* __restrict__ kb_o,
                                                  uint32_t* __restrict__ val_o) {
    constexpr int NW = kST / 32;
    __shared__ uint32_t base[256];
    __shared__ uint32_t cnt[NW][256];
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x < 256) base[threadIdx.x] = off[threadIdx.x * nblk + blockIdx.x];
    const uint32_t m = *d_m;
    for (int r = 0; r < kSR; r++) {
        for (uint32_t j = threadIdx.x; j < NW * 256; j += kST) (&cnt[0][0])[j] = 0;
        __syncthreads();
        const uint32_t i = blockIdx.x * kFTile + (uint32_t)r * kST + threadIdx.x;
        const bool valid = i < m;
        const uint32_t a = valid ? ka[i] : 0u;
        const uint32_t d = valid ? ((a >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) cnt[warp][d] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < 256) {
            // exclusive prefix over the warps for this digit; the round's total moves base
            uint32_t run = base[threadIdx.x];
            for (int w = 0; w < NW; w++) {
                const uint32_t c = cnt[w][threadIdx.x];
                cnt[w][threadIdx.x] = run;
                run += c;
            }
            base[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = cnt[warp][d] + rank;
            ka_o[pos] = a;
            kb_o[pos] = kb[i];
            val_o[pos] = val[i];
        }
        __syncthreads();
    }
}

// Coordinates of the sorted survivors, structure of arrays.
__global__ void kf_gather(const uint32_t* __restrict__ val, const uint32_t* __restrict__ d_m,
                          const float* __restrict__ pts, float* __restrict__ xs, float* __restrict__ ys,
                          float* __restrict__ zs) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *d_m) return;
    const float* p = pts + 3 * (size_t)val[j];
    xs[j] = p[0];
    ys[j] = p[1];
    zs[j] = p[2];
}

// next(j) = first k > j with fl(d^2(p_j, p_k)) > r2 (m if none); marks position 0.
__global__ void kf_next(const float* __restrict__ xs, const float* __restrict__ ys, const float* __restrict__ zs,
                        const uint32_t* __restrict__ d_m, float r2, uint32_t* __restrict__ next,
                        uint8_t* __restrict__ mark) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = *d_m;
    if (j >= m) return;
    const float ax = xs[j], ay = ys[j], az = zs[j];
    uint32_t k = j + 1;
    for (; k < m; k++) {
        const float dx = __fsub_rn(ax, xs[k]);
        const float dy = __fsub_rn(ay, ys[k]);
        const float dz = __fsub_rn(az, zs[k]);
        const float s = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        if (!(s <= r2)) break;   // s > r2 for finite input; a NaN (rejected input) also stops
    }
    next[j] = k;
    mark[j] = j == 0 ? 1 : 0;
}

// One round of pointer doubling: every marked position marks jin[j], and
// jout[j] = jin[jin[j]] (m where the chain ends).
__global__ void kf_double(const uint32_t* __restrict__ jin, uint32_t* __restrict__ jout,
                          const uint32_t* __restrict__ d_m, uint8_t* mark) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = *d_m;
    if (j >= m) return;
    const uint32_t k = jin[j];
    if (k < m) {
        if (mark[j]) mark[k] = 1;
        jout[j] = jin[k];
    } else {
        jout[j] = m;
    }
}

__global__ void kf_survive(const uint8_t* __restrict__ mark, const uint32_t* __restrict__ val,
                           const uint32_t* __restrict__ d_m, uint8_t* __restrict__ alive) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < *d_m) alive[val[j]] = mark[j];
}

// box[0..2] = lo keys, box[3..5] = hi keys (empty), box[6] = non-finite flag, box[7] =
// kept count (written at the end)
__global__ void kf_box_init(uint32_t* __restrict__ box) {
    if (threadIdx.x < 8) box[threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
}

__global__ void kf_fill_u8(uint8_t* __restrict__ p, uint32_t n, uint8_t v) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

unsigned blocks_of(uint64_t work, unsigned per) { return (unsigned)std::max<uint64_t>(1, (work + per - 1) / per); }


// Buffers of one filter plan, carved from one allocation.
struct FilterBufs {
    float* in = nullptr;          // copy of the input points [n][3]
    uint32_t* kept = nullptr;     // kept indices (n slots)
    uint32_t* box = nullptr;      // kf_box_init layout; box[6] non-finite, box[7] count
    uint32_t* d_m = nullptr;
    uint32_t* counts = nullptr;
    uint32_t* hist = nullptr;
    uint64_t* sp = nullptr;
    uint8_t* alive = nullptr;
    uint8_t* mark = nullptr;
    uint32_t* w[11] = {};
    uint32_t nblk = 0;
};

size_t carve(char* buf, size_t n, FilterBufs* b) {
    const uint32_t nblk = blocks_of(n, kFTile);
    size_t total = 0;
    auto take = [&](size_t bytes) { const size_t o = total; total += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_in = take(12 * n), o_kept = take(4 * n), o_box = take(8 * 4), o_m = take(4);
    const size_t o_counts = take(4 * (size_t)nblk), o_hist = take(4 * 256 * (size_t)nblk), o_sp = take(24 * n);
    const size_t o_alive = take(n), o_mark = take(n);
    size_t o_w[11];
    for (auto& o : o_w) o = take(4 * n);   // asc, klo/khi/val x 2, xs, ys, zs, next/jump
    if (buf && b) {
        auto U = [&](size_t o) { return reinterpret_cast<uint32_t*>(buf + o); };
        b->in = reinterpret_cast<float*>(buf + o_in);
        b->kept = U(o_kept);
        b->box = U(o_box);
        b->d_m = U(o_m);
        b->counts = U(o_counts);
        b->hist = U(o_hist);
        b->sp = reinterpret_cast<uint64_t*>(buf + o_sp);
        b->alive = reinterpret_cast<uint8_t*>(buf + o_alive);
        b->mark = reinterpret_cast<uint8_t*>(buf + o_mark);
        for (int k = 0; k < 11; k++) b->w[k] = U(o_w[k]);
        b->nblk = nblk;
    }
    return total;
}

// Every launch of one filter call on b (no host synchronisation, no host memory): the
// sequence depends on n and r only, so it is captured once into a CUDA graph.
void enqueue_filter(const FilterBufs& b, uint32_t n, float r, cudaStream_t st) {
    const uint32_t nblk = b.nblk;
    uint32_t* asc = b.w[0];
    uint32_t* ka[2] = {b.w[1], b.w[4]};
    uint32_t* kb[2] = {b.w[2], b.w[5]};
    uint32_t* vv[2] = {b.w[3], b.w[6]};
    float* xs = reinterpret_cast<float*>(b.w[7]);
    float* ys = reinterpret_cast<float*>(b.w[8]);
    float* zs = reinterpret_cast<float*>(b.w[9]);
    uint32_t* jmp[2] = {b.w[10], asc};   // asc is free once the keys are made
    const unsigned gn = blocks_of(n, kFT);
    kf_box_init<<<1, 32, 0, st>>>(b.box);
    kf_bbox<<<std::min(gn, 1024u), kFT, 0, st>>>(b.in, n, b.box);
    kf_spread<<<gn, kFT, 0, st>>>(b.in, n, b.box, b.sp);
    kf_fill_u8<<<gn, kFT, 0, st>>>(b.alive, n, 1);
    int doublings = 0;   // 2^doublings >= n: enough rounds of pointer doubling for any chain
    while ((1ull << doublings) < n) doublings++;
    const float r2 = r * r;   // fl(r^2), as the host filter
    for (int p = 0; p < 6; p++) {
        // survivors in ascending index order; m = their count
        kf_flag_count<<<nblk, kFT, 0, st>>>(b.alive, nullptr, n, b.counts);
        kf_scan<<<1, kScanThreads, 0, st>>>(b.counts, nblk, b.d_m);
        kf_flag_compact<<<nblk, kFT, 0, st>>>(b.alive, nullptr, n, b.counts, nullptr, asc);
        kf_keys<<<gn, kFT, 0, st>>>(asc, b.d_m, b.sp, kPerm[p][0], kPerm[p][1], kPerm[p][2], ka[0], kb[0], vv[0]);
        // stable sort by the low word, then by the high word (4 digits each)
        int cur = 0;
        for (int word = 0; word < 2; word++)
            for (int shift = 0; shift < 32; shift += 8) {
                const uint32_t* kw = word == 0 ? ka[cur] : kb[cur];
                const uint32_t* ko = word == 0 ? kb[cur] : ka[cur];
                uint32_t* kw_o = word == 0 ? ka[cur ^ 1] : kb[cur ^ 1];
                uint32_t* ko_o = word == 0 ? kb[cur ^ 1] : ka[cur ^ 1];
                kf_hist<<<nblk, kST, 0, st>>>(kw, b.d_m, shift, b.hist, nblk);
                kf_scan<<<1, kScanThreads, 0, st>>>(b.hist, 256 * nblk, nullptr);
                kf_scatter<<<nblk, kST, 0, st>>>(kw, ko, vv[cur], b.d_m, shift, b.hist, nblk, kw_o, ko_o, vv[cur ^ 1]);
                cur ^= 1;
            }
        const uint32_t* val = vv[cur];
        // greedy sweep as a chain, marked by pointer doubling
        kf_gather<<<gn, kFT, 0, st>>>(val, b.d_m, b.in, xs, ys, zs);
        kf_next<<<gn, kFT, 0, st>>>(xs, ys, zs, b.d_m, r2, jmp[0], b.mark);
        int j = 0;
        for (int k = 0; k < doublings; k++, j ^= 1) kf_double<<<gn, kFT, 0, st>>>(jmp[j], jmp[j ^ 1], b.d_m, b.mark);
        if (p < 5) {
            kf_survive<<<gn, kFT, 0, st>>>(b.mark, val, b.d_m, b.alive);
        } else {
            kf_flag_count<<<nblk, kFT, 0, st>>>(b.mark, b.d_m, n, b.counts);
            kf_scan<<<1, kScanThreads, 0, st>>>(b.counts, nblk, b.box + 7);
            kf_flag_compact<<<nblk, kFT, 0, st>>>(b.mark, b.d_m, n, b.counts, val, b.kept);
        }
    }
}

// A captured filter for one (device, n, r): its own buffers and graph.  A few are kept
// (least recently used out first), so that filtering frame after frame of one size costs
// one graph launch and two small copies.
struct FilterPlan {
    int dev = -1;
    size_t n = 0;
    uint32_t r_bits = 0;
    char* buf = nullptr;
    FilterBufs b;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (buf) cudaFree(buf);
        exec = nullptr;
        buf = nullptr;
    }
};

constexpr int kPlans = 4;
std::mutex g_plan_mu;
FilterPlan g_plans[kPlans];
uint64_t g_plan_clock = 0;

int make_plan(FilterPlan& pl, int dev, size_t n, float r, std::string& err) {
    pl.release();
    pl.dev = dev;
    pl.n = n;
    std::memcpy(&pl.r_bits, &r, 4);
    const size_t bytes = carve(nullptr, n, nullptr);
    if (cudaMalloc((void**)&pl.buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        pl.buf = nullptr;
        pl.n = 0;
        err = "device allocation failed in the filter";
        return CAPT_E_NOMEM;
    }
    carve(pl.buf, n, &pl.b);
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        enqueue_filter(pl.b, (uint32_t)n, r, cs);
        ce = cudaStreamEndCapture(cs, &g);
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&pl.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        pl.release();
        pl.n = 0;
        err = std::string("filter graph: ") + cudaGetErrorString(ce);
        return CAPT_E_CUDA;
    }
    return CAPT_OK;
}

}  // namespace

namespace {

__global__ void k_gather_points(const float* __restrict__ pts, const uint32_t* __restrict__ idx, uint32_t m,
                                float* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float* p = pts + 3 * (size_t)idx[i];
    out[3 * (size_t)i] = p[0];
    out[3 * (size_t)i + 1] = p[1];
    out[3 * (size_t)i + 2] = p[2];
}

}  // namespace

int launch_gather_points(const float* pts, const uint32_t* idx, size_t m, float* out, cudaStream_t st,
                         std::string& err) {
    if (m == 0) return CAPT_OK;
    k_gather_points<<<blocks_of(m, 256), 256, 0, st>>>(pts, idx, (uint32_t)m, out);
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("gather launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int device_sfc_filter(const float* d_points, size_t n, float r, uint32_t* d_kept, size_t* n_out, cudaStream_t st,
                      std::string& err) {
    if (!n_out || (n && (!d_points || !d_kept))) { err = "NULL argument"; return CAPT_E_ARG; }
    if (!(r >= 0.f)) { err = "min_spacing must be >= 0"; return CAPT_E_RANGE; }
    if (n >= (size_t(1) << 31)) { err = "the device filter takes fewer than 2^31 points"; return CAPT_E_ARG; }
    *n_out = 0;
    if (n == 0) return CAPT_OK;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) { err = std::string("cudaGetDevice: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    uint32_t r_bits;
    std::memcpy(&r_bits, &r, 4);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    FilterPlan* pl = nullptr;
    for (auto& p : g_plans)
        if (p.exec && p.dev == dev && p.n == n && p.r_bits == r_bits) pl = &p;
    if (!pl) {
        pl = &g_plans[0];
        for (auto& p : g_plans)
            if (!p.exec || p.used < pl->used) pl = &p;
        const int rc = make_plan(*pl, dev, n, r, err);
        if (rc) return rc;
    }
    pl->used = ++g_plan_clock;
    uint32_t res[2] = {0u, 0u};
    ce = cudaMemcpyAsync(pl->b.in, d_points, 12 * n, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(pl->exec, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_kept, pl->b.kept, 4 * n, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(res, pl->b.box + 6, sizeof(res), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        err = std::string("filter: ") + cudaGetErrorString(ce);
        return CAPT_E_CUDA;
    }
    if (res[0]) { err = "non-finite coordinate in points"; return CAPT_E_NONFINITE; }
    *n_out = res[1];
    return CAPT_OK;
}

}  // namespace capt
