// batch.cu -- many images of uneven size and K in one persistent launch.
//
// The paper quantizes one image at a time (Sections 2-3).  Here every image of a
// batch is taken from start to finish -- histogram, seeding, Weighted Sort-Means,
// pixel mapping -- by one group of thread blocks:
//   * images above a pixel threshold by a thread-block cluster of C CTAs, whose
//     group barrier is the hardware cluster barrier;
//   * the rest by single CTAs, whose group barrier is __syncthreads.
// Groups pull images from a device-side queue in the order the host planner gives
// (largest estimated work first within each class), so no group ever waits for
// another and the launch needs no grid-wide synchronisation.  Each group owns a
// slot of the workspace: a direct 2^24-entry counter table (zero between images),
// a presence bitmap with a one-bit-per-word summary, and the scratch of the
// seeding and Lloyd steps.  The arithmetic of every step is that of the
// single-image kernels (the same dist3, the same integer seeding, the same Lloyd
// body), so results agree with kq_histogram/kq_seed/kq_lloyd/kq_map up to the
// FP32 summation order of the SSE, whose block partition differs.
//
// A live launch (batch_live_kernel) runs the same groups on images that arrive
// while it runs: the host publishes items into a queue in page-locked host memory,
// groups claim them through counters in the workspace header and post a done mark
// per item; a group with nothing to take waits with a bounded idle limit.  The
// Wu moments, which the group's threads rewrite step by step, are read through L2
// (__ldcg), as most of the batched steps' cross-thread reads are: through L1 they
// were seen stale in a live launch, which runs many images on one SM.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "lloyd_body.cuh"
#include "seed_dev.cuh"

namespace kq {
namespace {

constexpr int kBT = kLloydBlock;  // threads per CTA
constexpr int kBW = kBT / 32;     // warps per CTA
constexpr int kMaxCluster = 16;
constexpr int kBatchChunks = 64;  // VAR / DEN chunks of an image's unique list
constexpr int kSummWords = kBitWords / 32;  // summary: one bit per bitmap word
constexpr size_t kHeaderBytes = 4096;       // queue counters at the start of the workspace
constexpr unsigned kBFull = 0xffffffffu;

static_assert(sizeof(kq_batch_item) == 136, "kq_batch_item layout (LP64)");
static_assert(sizeof(kq_batch_result) == 96 && offsetof(kq_batch_result, sse_num) == 48, "kq_batch_result layout");

struct SlotMisc {
    unsigned long long ndc;
    unsigned long long var_w, var_s1[3], var_s2[3];
    unsigned long long cellw[kDenCells];
    unsigned long long cs[5 * kMaxK];
    unsigned long long xch[2][kMaxCluster];       // group scan totals per CTA
    unsigned long long wtot[2][kMaxCluster * kBW];  // k-means++: per-warp totals
    unsigned long long cmax[2][kMaxCluster];      // minmax: per-CTA maxima
    uint32_t gcnt[3 * 256];
    int quota[2 * kDenCells];
    int32_t item;
    int32_t live_busy;        // live launches: a CTA of the cluster ran a single-CTA item
    long long live_dec;       // live launches: rank 0's decision for the cluster
    uint8_t lbg_pal[3 * kMaxK];
};

// Slot layout (bytes from the slot base).
constexpr size_t kSoCnt = 0;
constexpr size_t kSoBits = kSoCnt + sizeof(uint32_t) * (size_t)kKeySpace;
constexpr size_t kSoSumm = kSoBits + sizeof(uint32_t) * (size_t)kBitWords;
constexpr size_t kSoWl = kSoSumm + sizeof(uint32_t) * (size_t)kSummWords;
constexpr size_t kSoSums = kSoWl + sizeof(uint32_t) * (size_t)kBitWords;
constexpr size_t kSoSsep = kSoSums + sizeof(unsigned long long) * 3 * kMaxK * 4;
constexpr size_t kSoRows = kSoSsep + sizeof(float) * 2 * kMaxGrid;
constexpr size_t kSoChunk = kSoRows + sizeof(uint32_t) * kMaxK * kMaxK;
constexpr size_t kSoWu = kSoChunk + sizeof(uint32_t) * kBatchChunks * 3 * 256;
constexpr size_t kSoMisc = kSoWu + kWuBytes;
constexpr size_t kSlotBytes = (kSoMisc + sizeof(SlotMisc) + 4095) / 4096 * 4096;

// Dynamic shared memory: one region reused by the steps in turn.
constexpr size_t kDynFgy = sizeof(uint32_t) * (2 * kMapSlots + kMaxK);
constexpr size_t kDynSff = sizeof(uint32_t) * (2 * kMapSlots + 2 * kSffMax);
constexpr size_t kDynRows = sizeof(uint32_t) * (size_t)kMaxK * kRowStride + sizeof(float) * kChunkSlots;
constexpr size_t kDynBytes = kDynSff > kDynFgy ? (kDynSff > kDynRows ? kDynSff : kDynRows)
                                               : (kDynFgy > kDynRows ? kDynFgy : kDynRows);
static_assert(sizeof(WuShared) <= kDynBytes, "the Wu split state fits the dynamic shared memory");

struct BatchShared {
    unsigned long long scan[kBW];
    unsigned long long red[kBW];
    uint32_t cnt[3 * 256];
    unsigned long long cw[kDenCells];
    uint2 pal[kMaxK];
    uint32_t key;
    int32_t item;
};

struct BatchArgs {
    const kq_batch_item *items;
    const int32_t *order;
    int32_t n_items;
    int32_t n_big;
    int32_t C;
    uint32_t *queue;  // [0] next cluster item, [1] next single-CTA item
    char *slots;
};

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// A group of C CTAs working on one image.  Its barrier orders global memory
// among the group: the cluster barrier with release/acquire semantics, or
// __syncthreads for a group of one.
struct Group {
    int C;
    int rank;
    char *slot;
    __device__ __forceinline__ int nthreads() const { return C * kBT; }
    __device__ __forceinline__ int gtid() const { return rank * kBT + (int)threadIdx.x; }
    __device__ __forceinline__ bool operator()() const
    {
        if (C > 1) {
            asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        } else {
            __syncthreads();
        }
        return true;
    }
    __device__ __forceinline__ SlotMisc *misc() const { return reinterpret_cast<SlotMisc *>(slot + kSoMisc); }
    template <typename T>
    __device__ __forceinline__ T *at_slot(size_t off) const { return reinterpret_cast<T *>(slot + off); }
};

// Exclusive prefix of v over the group's threads in (rank, thread) order; the
// group total goes to *total.  `xb` selects the exchange buffer: two scans
// separated by no other group barrier must use different buffers.
__device__ unsigned long long group_excl_scan(const Group &g, unsigned long long v, unsigned long long *total, int xb,
                                              BatchShared &bs)
{
    unsigned long long btot;
    const unsigned long long ex = block_excl_scan_u64<kBT>(v, bs.scan, &btot);
    if (g.C == 1) {
        *total = btot;
        return ex;
    }
    SlotMisc *ms = g.misc();
    if (threadIdx.x == 0) ms->xch[xb][g.rank] = btot;
    g();
    unsigned long long before = 0ull, all = 0ull;
    for (int r = 0; r < g.C; ++r) {
        const unsigned long long t = __ldcg(&ms->xch[xb][r]);
        if (r < g.rank) before += t;
        all += t;
    }
    *total = all;
    return before + ex;
}

// ---------------------------------------------------------------- histogram
__device__ __forceinline__ uint32_t px_key(const uint8_t *rgb, int64_t p)
{
    const uint8_t *q = rgb + 3 * p;
    return ((uint32_t)q[0] << 16) | ((uint32_t)q[1] << 8) | (uint32_t)q[2];
}

template <int I>
__device__ __forceinline__ uint32_t pgroup_key(const uint32_t (&w)[12])
{
    constexpr int o = 3 * I, q = o >> 2, r = o & 3;
    const uint32_t lo = w[q];
    const uint32_t hi = (q + 1 < 12) ? w[q + 1] : 0u;
    return __byte_perm(lo, hi, (r + 2) | ((r + 1) << 4) | (r << 8)) & 0xFFFFFFu;
}

template <int I>
struct Keys16 {
    __device__ __forceinline__ static void get(const uint32_t (&w)[12], uint32_t (&k)[16])
    {
        k[I] = pgroup_key<I>(w);
        Keys16<I + 1>::get(w, k);
    }
};
template <>
struct Keys16<16> {
    __device__ __forceinline__ static void get(const uint32_t (&)[12], uint32_t (&)[16]) {}
};

// First pixel whose byte offset makes rgb + 3 p 16-byte aligned.
__device__ __forceinline__ int64_t aligned_head(const uint8_t *rgb, int64_t n)
{
    const uint64_t mis = reinterpret_cast<uintptr_t>(rgb) & 15u;
    int64_t head = (int64_t)(((16u - mis) * 11u) & 15u);  // 3 * 11 == 1 (mod 16)
    return head > n ? n : head;
}

__device__ __forceinline__ void touch(uint32_t *cnt, uint32_t *bits, uint32_t *summ, uint32_t key, uint32_t old)
{
    if (old == 0u) {
        const uint32_t ob = atomicOr(bits + (key >> 5), 1u << (key & 31u));
        if (ob == 0u) atomicOr(summ + (key >> 10), 1u << ((key >> 5) & 31u));
    }
}

// Unique colours of one image in ascending key order with their pixel counts
// (Section 2.2, items 1-2).  Returns N' (the true count, also when it exceeds the
// item's capacity, in which case nothing is written and the counters are cleared).
__device__ int64_t group_histogram(const Group &g, const kq_batch_item &it, BatchShared &bs)
{
    uint32_t *cnt = g.at_slot<uint32_t>(kSoCnt);
    uint32_t *bits = g.at_slot<uint32_t>(kSoBits);
    uint32_t *summ = g.at_slot<uint32_t>(kSoSumm);
    uint32_t *wl = g.at_slot<uint32_t>(kSoWl);
    const int GT = g.nthreads(), gt = g.gtid();
    const int64_t n = it.n_pixels;
    const uint8_t *rgb = it.rgb;
    // count
    const int64_t head = aligned_head(rgb, n);
    const int64_t ngroups = (n - head) / 16;
    const int64_t tail0 = head + ngroups * 16;
    for (int64_t p = gt; p < head; p += GT) {
        const uint32_t k = px_key(rgb, p);
        touch(cnt, bits, summ, k, atomicAdd(cnt + k, 1u));
    }
    for (int64_t p = tail0 + gt; p < n; p += GT) {
        const uint32_t k = px_key(rgb, p);
        touch(cnt, bits, summ, k, atomicAdd(cnt + k, 1u));
    }
    const uint4 *pg = reinterpret_cast<const uint4 *>(rgb + 3 * head);
    for (int64_t gi = gt; gi < ngroups; gi += GT) {
        const uint4 a = __ldcs(pg + 3 * gi), b = __ldcs(pg + 3 * gi + 1), c = __ldcs(pg + 3 * gi + 2);
        const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
        uint32_t key[16], old[16];
        Keys16<0>::get(w, key);
#pragma unroll
        for (int i = 0; i < 16; ++i) old[i] = atomicAdd(cnt + key[i], 1u);
#pragma unroll
        for (int i = 0; i < 16; ++i) touch(cnt, bits, summ, key[i], old[i]);
    }
    g();
    // non-empty bitmap words, in key order, from the summary
    const int SP = kSummWords / GT;  // GT divides 2^14
    const int w0 = gt * SP;
    unsigned long long nz = 0ull;
    for (int j = 0; j < SP; ++j) nz += __popc(__ldcg(summ + w0 + j));
    unsigned long long M;
    unsigned long long pos = group_excl_scan(g, nz, &M, 0, bs);
    for (int j = 0; j < SP; ++j) {
        uint32_t v = __ldcg(summ + w0 + j);
        if (!v) continue;
        summ[w0 + j] = 0u;
        while (v) {
            const int b = __ffs(v) - 1;
            v &= v - 1u;
            wl[pos++] = (uint32_t)((w0 + j) * 32 + b);
        }
    }
    g();
    // colours of those words, by output position
    int64_t lo, hi;
    slice_of((int64_t)M, gt, GT, &lo, &hi);
    unsigned long long c = 0ull;
    for (int64_t m = lo; m < hi; ++m) c += __popc(__ldcg(bits + __ldcg(wl + m)));
    unsigned long long nu;
    unsigned long long base = group_excl_scan(g, c, &nu, 1, bs);
    const bool over = nu > (unsigned long long)(it.capacity < 0 ? 0 : it.capacity);
    uint32_t *keys = it.keys, *weights = it.weights;
    for (int64_t m = lo; m < hi; ++m) {
        const uint32_t word = __ldcg(wl + m);
        uint32_t v = __ldcg(bits + word);
        bits[word] = 0u;
        while (v) {
            uint32_t k4[4], c4[4];
            int got = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                k4[q] = 0xFFFFFFFFu;
                if (v) {
                    k4[q] = (word << 5) | (uint32_t)(__ffs(v) - 1);
                    v &= v - 1u;
                    ++got;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) c4[q] = q < got ? __ldcg(cnt + k4[q]) : 0u;
            for (int q = 0; q < got; ++q) {
                if (over) {
                    cnt[k4[q]] = 0u;
                } else {
                    keys[base] = k4[q];
                    weights[base] = c4[q];
                }
                ++base;
            }
        }
    }
    g();
    return (int64_t)nu;
}

// ---------------------------------------------------------------- k-means++ / minmax
// Colour i belongs to 128-colour step i / 128, lane l of a warp holding colours
// 4l .. 4l + 3 of a step (16-byte loads).  The steps are cut into contiguous
// ranges, one per warp of the group in (rank, warp) order, so the order of
// (warp, step, lane, element) is the index order.  Per round each warp writes the
// running sum of P = w (first round) or w D^2 at the end of each of its steps and
// its total; the sample (the first colour whose running sum exceeds t) is then
// found through the warp totals, the step sums, one step's lane sums and one
// lane's four colours.
constexpr int kStep = 128;

struct FarScratch {
    uint32_t *d2;              // [2][cap4]
    unsigned long long *sp;    // [2][sstride]
    int64_t cap4, sstride;     // buffer strides
};

__host__ __device__ __forceinline__ int64_t far_cap4(int64_t cap) { return (cap + 3) / 4 * 4; }
__host__ __device__ __forceinline__ int64_t far_sstride(int64_t cap) { return (cap + kStep - 1) / kStep + 1; }

// Four consecutive 32-bit values from i (16-byte aligned), zero past n.
__device__ __forceinline__ uint4 ld4(const uint32_t *p, int64_t i, int64_t n)
{
    if (i + 3 < n) return __ldcg(reinterpret_cast<const uint4 *>(p + i));
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (i < n) v.x = __ldcg(p + i);
    if (i + 1 < n) v.y = __ldcg(p + i + 1);
    if (i + 2 < n) v.z = __ldcg(p + i + 2);
    return v;
}

__device__ __forceinline__ void st4(uint32_t *p, int64_t i, int64_t n, uint4 v)
{
    if (i + 3 < n) {
        *reinterpret_cast<uint4 *>(p + i) = v;
        return;
    }
    if (i < n) p[i] = v.x;
    if (i + 1 < n) p[i + 1] = v.y;
    if (i + 2 < n) p[i + 2] = v.z;
}

__device__ uint32_t far_locate(const kq_batch_item &it, const FarScratch &fs, int64_t n, int GW, int buf, int r,
                               const unsigned long long *wt)
{
    const int lane = threadIdx.x & 31;
    unsigned long long v[kMaxCluster * kBW / 32];
    unsigned long long total = 0ull;
#pragma unroll
    for (int j = 0; j < kMaxCluster * kBW / 32; ++j) {
        const int gw = 32 * j + lane;
        v[j] = gw < GW ? __ldcg(wt + gw) : 0ull;
        total += v[j];
    }
    for (int o = 16; o; o >>= 1) total += __shfl_xor_sync(kBFull, total, o);
    const unsigned long long t = below(rand64(it.seed, 2, (uint32_t)r), total);
    unsigned long long run = 0ull, resid = 0ull;
    int gstar = GW - 1;
#pragma unroll
    for (int j = 0; j < kMaxCluster * kBW / 32; ++j) {
        if (32 * j >= GW) break;
        unsigned long long x = v[j];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kBFull, x, o);
            if (lane >= o) x += y;
        }
        const unsigned bal = __ballot_sync(kBFull, run + x > t);
        if (bal) {
            const int l = __ffs(bal) - 1;
            gstar = 32 * j + l;
            resid = t - (run + __shfl_sync(kBFull, x, l) - __shfl_sync(kBFull, v[j], l));
            break;
        }
        run += __shfl_sync(kBFull, x, 31);
    }
    // the step of warp gstar holding the sample: blocks of 32 steps, then the step
    const unsigned long long *sp = fs.sp + (size_t)buf * fs.sstride;
    int64_t slo, shi;
    slice_of((n + kStep - 1) / kStep, gstar, GW, &slo, &shi);  // the partition group_far used
    int64_t sstar = shi - 1;
    unsigned long long before = 0ull;  // running sum of the warp before step sstar
    for (int64_t sb = slo; sb < shi; sb += 1024) {
        const int64_t e = sb + 32 * (int64_t)lane + 31;
        const bool in = sb + 32 * (int64_t)lane < shi;
        const unsigned long long ev = in ? __ldcg(sp + (e < shi ? e : shi - 1)) : ~0ull;
        const unsigned bal = __ballot_sync(kBFull, in && ev > resid);
        if (!bal) {
            before = __shfl_sync(kBFull, ev, 31);  // all 32 blocks lie below resid
            continue;
        }
        const int l = __ffs(bal) - 1;
        if (l > 0) before = __shfl_sync(kBFull, ev, l - 1);
        const int64_t b0 = sb + 32 * (int64_t)l;
        const bool in2 = b0 + lane < shi;
        const unsigned long long sv = in2 ? __ldcg(sp + b0 + lane) : ~0ull;
        const unsigned bal2 = __ballot_sync(kBFull, in2 && sv > resid);
        const int l2 = bal2 ? __ffs(bal2) - 1 : 0;
        const unsigned long long prev = __shfl_sync(kBFull, sv, l2 > 0 ? l2 - 1 : 0);
        if (l2 > 0) before = prev;
        sstar = b0 + l2;
        break;
    }
    const unsigned long long resid2 = resid - before;
    if (sstar < 0) sstar = 0;  // only for an all-zero total, which valid inputs never give
    // the lane, then the colour, within step sstar
    const int64_t i0 = sstar * kStep + 4 * lane;
    const uint4 w4 = ld4(it.weights, i0, n);
    unsigned long long p[4] = {w4.x, w4.y, w4.z, w4.w};
    if (r > 0) {
        const uint4 d4 = ld4(fs.d2 + (size_t)buf * fs.cap4, i0, n);
        p[0] *= d4.x;
        p[1] *= d4.y;
        p[2] *= d4.z;
        p[3] *= d4.w;
    }
    const unsigned long long ps = p[0] + p[1] + p[2] + p[3];
    unsigned long long x = ps;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kBFull, x, o);
        if (lane >= o) x += y;
    }
    const unsigned bal = __ballot_sync(kBFull, x > resid2);
    const int l = bal ? __ffs(bal) - 1 : 0;
    unsigned long long acc = __shfl_sync(kBFull, x - ps, l);  // running sum before lane l
    int64_t istar = sstar * kStep + 4 * l + 3;
    for (int j = 0; j < 4; ++j) {
        const unsigned long long pj = __shfl_sync(kBFull, p[j], l);
        if (acc + pj > resid2) {
            istar = sstar * kStep + 4 * l + j;
            break;
        }
        acc += pj;
    }
    return __ldcg(it.keys + (istar < n ? istar : n - 1));
}

// k-means++ (mode 0) or minmax (mode 1) with the rules of kq_seed; n > K.
__device__ void group_far(const Group &g, const kq_batch_item &it, int64_t n, int mode, BatchShared &bs)
{
    const int K = it.K;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int GW = g.C * kBW, gw = g.rank * kBW + warp;
    FarScratch fs;
    fs.cap4 = far_cap4(it.capacity);
    fs.sstride = far_sstride(it.capacity);
    fs.d2 = reinterpret_cast<uint32_t *>(it.scratch);
    fs.sp = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(it.scratch) +
                                                   align_up(sizeof(uint32_t) * 2 * (size_t)fs.cap4, 256));
    const int64_t steps = (n + kStep - 1) / kStep;
    int64_t slo, shi;
    slice_of(steps, gw, GW, &slo, &shi);
    SlotMisc *ms = g.misc();
    const uint32_t *__restrict__ keys = it.keys;
    const uint32_t *__restrict__ wts = it.weights;
    uint32_t ckey = 0u;
    constexpr int U = 4;  // steps in flight per warp
    for (int r = 0; r < K; ++r) {
        const int buf = r & 1;
        if (mode == 1 && r == 0) {
            ckey = __ldcg(keys + below(rand64(it.seed, 3, 0), (uint64_t)n));
        } else {
            uint32_t *__restrict__ d2w = fs.d2 + (size_t)buf * fs.cap4;
            const uint32_t *__restrict__ d2r = fs.d2 + (size_t)(buf ^ 1) * fs.cap4;
            unsigned long long *__restrict__ sp = fs.sp + (size_t)buf * fs.sstride;
            unsigned long long run = 0ull, best = 0ull;
            for (int64_t s0 = slo; s0 < shi; s0 += U) {
                uint4 k4[U], w4[U], d4[U];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int64_t i = (s0 + q) * kStep + 4 * lane;
                    const int64_t lim = s0 + q < shi ? n : 0;
                    k4[q] = ld4(keys, i, lim);
                    w4[q] = mode == 0 ? ld4(wts, i, lim) : make_uint4(0u, 0u, 0u, 0u);
                    d4[q] = r > 1 ? ld4(d2r, i, lim) : make_uint4(~0u, ~0u, ~0u, ~0u);
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    if (s0 + q >= shi) break;
                    const int64_t i = (s0 + q) * kStep + 4 * lane;
                    unsigned long long p = 0ull;
                    if (r == 0) {
                        p = (unsigned long long)w4[q].x + w4[q].y + w4[q].z + w4[q].w;
                    } else {
                        uint4 md;
                        md.x = min(d4[q].x, key_dist2(k4[q].x, ckey));
                        md.y = min(d4[q].y, key_dist2(k4[q].y, ckey));
                        md.z = min(d4[q].z, key_dist2(k4[q].z, ckey));
                        md.w = min(d4[q].w, key_dist2(k4[q].w, ckey));
                        st4(d2w, i, n, md);
                        if (mode == 0) {
                            p = (unsigned long long)w4[q].x * md.x + (unsigned long long)w4[q].y * md.y +
                                (unsigned long long)w4[q].z * md.z + (unsigned long long)w4[q].w * md.w;
                        } else {
                            const uint32_t mm[4] = {md.x, md.y, md.z, md.w};
                            const uint32_t kk[4] = {k4[q].x, k4[q].y, k4[q].z, k4[q].w};
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (i + j < n) {
                                    const unsigned long long pk = mmx_pack(mm[j], kk[j]);
                                    best = pk > best ? pk : best;
                                }
                            }
                        }
                    }
                    if (mode == 0) {
                        for (int o = 16; o; o >>= 1) p += __shfl_xor_sync(kBFull, p, o);
                        run += p;
                        if (lane == 0) sp[s0 + q] = run;
                    }
                }
            }
            if (mode == 0) {
                if (lane == 0) ms->wtot[buf][gw] = run;
            } else {
                for (int o = 16; o; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(kBFull, best, o);
                    best = other > best ? other : best;
                }
                if (lane == 0) bs.red[warp] = best;
                __syncthreads();
                if (tid == 0) {
                    unsigned long long b = 0ull;
                    for (int j = 0; j < kBW; ++j) b = bs.red[j] > b ? bs.red[j] : b;
                    ms->cmax[buf][g.rank] = b;
                }
            }
            g();
            if (warp == 0) {
                uint32_t k;
                if (mode == 0) {
                    k = far_locate(it, fs, n, GW, buf, r, ms->wtot[buf]);
                } else {
                    unsigned long long b = lane < g.C ? __ldcg(&ms->cmax[buf][lane]) : 0ull;
                    for (int o = 16; o; o >>= 1) {
                        const unsigned long long other = __shfl_xor_sync(kBFull, b, o);
                        b = other > b ? other : b;
                    }
                    k = 0xFFFFFFu - (uint32_t)(b & 0xFFFFFFull);
                }
                if (lane == 0) bs.key = k;
            }
            __syncthreads();
            ckey = bs.key;
        }
        if (g.rank == 0 && tid == 0) key_to_centre(it.centers + 3 * r, ckey);
    }
}

// ---------------------------------------------------------------- VAR / DEN / LBG
__device__ __forceinline__ void chunk_range(int64_t n, int c, int64_t *lo, int64_t *hi)
{
    const int64_t len = (n + kBatchChunks - 1) / kBatchChunks;
    *lo = (int64_t)c * len < n ? (int64_t)c * len : n;
    *hi = *lo + len < n ? *lo + len : n;
}

// mode 0: per-chunk counts of each value of each channel and the exact weighted
// moments; mode 1: per-chunk counts per density cell and the pixel weight per cell.
__device__ void group_chunk_counts(const Group &g, const kq_batch_item &it, int64_t n, int mode, BatchShared &bs)
{
    SlotMisc *ms = g.misc();
    uint32_t *chunk_cnt = g.at_slot<uint32_t>(kSoChunk);
    const int tid = threadIdx.x;
    if (g.rank == 0) {
        for (int j = tid; j < 3 * 256; j += kBT) ms->gcnt[j] = 0u;
        for (int j = tid; j < kDenCells; j += kBT) ms->cellw[j] = 0ull;
        if (tid < 7) (&ms->var_w)[tid] = 0ull;
    }
    g();
    const int width = mode == 0 ? 3 * 256 : kDenCells;
    unsigned long long mw = 0, m1[3] = {0, 0, 0}, m2[3] = {0, 0, 0};
    for (int c = g.rank; c < kBatchChunks; c += g.C) {
        for (int j = tid; j < width; j += kBT) bs.cnt[j] = 0u;
        for (int j = tid; j < kDenCells; j += kBT) bs.cw[j] = 0ull;
        __syncthreads();
        int64_t lo, hi;
        chunk_range(n, c, &lo, &hi);
        for (int64_t i = lo + tid; i < hi; i += kBT) {
            const uint32_t key = __ldcg(it.keys + i);
            const unsigned long long wi = __ldcg(it.weights + i);
            if (mode == 0) {
                const uint32_t x[3] = {key_r(key), key_g(key), key_b(key)};
                mw += wi;
                for (int ch = 0; ch < 3; ++ch) {
                    atomicAdd(&bs.cnt[ch * 256 + x[ch]], 1u);
                    m1[ch] += wi * x[ch];
                    m2[ch] += wi * x[ch] * x[ch];
                }
            } else {
                const int cell = den_cell(key);
                atomicAdd(&bs.cnt[cell], 1u);
                atomicAdd(&bs.cw[cell], wi);
            }
        }
        __syncthreads();
        for (int j = tid; j < width; j += kBT) {
            chunk_cnt[(size_t)c * width + j] = bs.cnt[j];
            if (bs.cnt[j]) atomicAdd(&ms->gcnt[j], bs.cnt[j]);
            if (mode == 1 && bs.cw[j]) atomicAdd(&ms->cellw[j], bs.cw[j]);
        }
        __syncthreads();
    }
    if (mode == 0) {
        unsigned long long t = block_sum_u64<kBT>(mw, bs.red);
        if (tid == 0 && t) atomicAdd(&ms->var_w, t);
        for (int ch = 0; ch < 3; ++ch) {
            t = block_sum_u64<kBT>(m1[ch], bs.red);
            if (tid == 0 && t) atomicAdd(&ms->var_s1[ch], t);
            t = block_sum_u64<kBT>(m2[ch], bs.red);
            if (tid == 0 && t) atomicAdd(&ms->var_s2[ch], t);
        }
    }
    g();
}

__device__ void group_var(const Group &g, const kq_batch_item &it, int64_t n, BatchShared &bs)
{
    group_chunk_counts(g, it, n, 0, bs);
    SlotMisc *ms = g.misc();
    unsigned long long s1[3], s2[3];
    for (int ch = 0; ch < 3; ++ch) {
        s1[ch] = __ldcg(&ms->var_s1[ch]);
        s2[ch] = __ldcg(&ms->var_s2[ch]);
    }
    const int ch = var_channel(__ldcg(&ms->var_w), s1, s2);
    for (int j = threadIdx.x; j < 3 * 256; j += kBT) bs.cnt[j] = __ldcg(&ms->gcnt[j]);
    __syncthreads();
    const uint32_t *chunk_cnt = g.at_slot<uint32_t>(kSoChunk);
    for (int gw = g.rank * kBW + (int)(threadIdx.x >> 5); gw < it.K; gw += g.C * kBW)
        var_pick_warp(it.keys, n, it.K, gw, ch, chunk_cnt, kBatchChunks, bs.cnt, it.centers);
    g();
}

__device__ void group_den(const Group &g, const kq_batch_item &it, int64_t n, BatchShared &bs, uint32_t *dyn)
{
    group_chunk_counts(g, it, n, 1, bs);
    SlotMisc *ms = g.misc();
    const int tid = threadIdx.x;
    for (int j = tid; j < kDenCells; j += kBT) {
        bs.cnt[j] = __ldcg(&ms->gcnt[j]);
        bs.cw[j] = __ldcg(&ms->cellw[j]);
    }
    __syncthreads();
    if (g.rank == 0 && tid == 0) den_quota(it.K, bs.cnt, bs.cw, ms->quota);
    g();
    const uint32_t *chunk_cnt = g.at_slot<uint32_t>(kSoChunk);
    uint32_t *pos1 = dyn, *val = dyn + 1024, *pick = dyn + 2048;
    FyMap m{pos1, val, 1023u};
    const int warp = tid >> 5;
    for (int cell = g.rank; cell < kDenCells; cell += g.C) {
        const int q = __ldcg(&ms->quota[cell]);
        if (q == 0) continue;
        const int off = __ldcg(&ms->quota[kDenCells + cell]);
        clear_map(pos1, 1024);
        __syncthreads();
        if (tid == 0) fisher_yates(bs.cnt[cell], (uint32_t)q, it.seed, 16u + (uint32_t)cell, m, pick);
        __syncthreads();
        for (int j = warp; j < q; j += kBW) {
            const int64_t idx = warp_locate(it.keys, n, chunk_cnt, kBatchChunks, kDenCells, cell, pick[j], 1, 0);
            if ((tid & 31) == 0) key_to_centre(it.centers + 3 * (off + j), __ldcg(it.keys + idx));
        }
        __syncthreads();
    }
    g();
}

__device__ void group_lloyd(Group &g, const kq_batch_item &it, int64_t n, int K, double eps, int max_iter,
                            uint8_t *palette, kq_lloyd_stats *stats, int32_t *status, LloydShared &sh,
                            uint32_t *row_cache)
{
    LloydArgs a;
    a.keys = it.keys;
    a.w = it.weights;
    a.n_unique = nullptr;
    a.K = K;
    a.eps = eps;
    a.max_iter = max_iter;
    a.flags = 0u;
    a.skip_if_n_le = 0;
    a.centers = it.centers;
    a.labels = it.labels;
    a.palette = palette;
    a.stats = stats;
    a.sse_hist = nullptr;
    a.ctl = nullptr;
    SlotMisc *ms = g.misc();
    a.ndc = &ms->ndc;
    a.status = status;
    a.sums = g.at_slot<unsigned long long>(kSoSums);
    a.sse_part = g.at_slot<float>(kSoSsep);
    a.rows = g.at_slot<uint32_t>(kSoRows);
    lloyd_body<RgbKeys>(a, sh, row_cache, n, g.rank, g.C, g);
    g();
}

// LBG: the centroid, then split rounds each refined by Lloyd (rules of kq_seed).
__device__ void group_lbg(Group &g, const kq_batch_item &it, int64_t n, BatchShared &bs, LloydShared &sh,
                          uint32_t *dyn, int32_t *status)
{
    SlotMisc *ms = g.misc();
    const int tid = threadIdx.x, GT = g.nthreads(), gt = g.gtid();
    if (g.rank == 0 && tid < 4) (&ms->var_w)[tid] = 0ull;
    g();
    unsigned long long mw = 0, m1[3] = {0, 0, 0};
    for (int64_t i = gt; i < n; i += GT) {
        const uint32_t key = __ldcg(it.keys + i);
        const unsigned long long wi = __ldcg(it.weights + i);
        mw += wi;
        m1[0] += wi * key_r(key);
        m1[1] += wi * key_g(key);
        m1[2] += wi * key_b(key);
    }
    unsigned long long t = block_sum_u64<kBT>(mw, bs.red);
    if (tid == 0 && t) atomicAdd(&ms->var_w, t);
    for (int ch = 0; ch < 3; ++ch) {
        t = block_sum_u64<kBT>(m1[ch], bs.red);
        if (tid == 0 && t) atomicAdd(&ms->var_s1[ch], t);
    }
    g();
    if (g.rank == 0 && tid == 0) {
        const double W = (double)__ldcg(&ms->var_w);
        for (int ch = 0; ch < 3; ++ch) it.centers[ch] = (double)__ldcg(&ms->var_s1[ch]) / W;
    }
    g();
    const int K = it.K;
    int m = 1;
    while (m < K) {
        const int split = (2 * m <= K) ? m : K - m;
        if (split < m) {
            if (g.rank == 0)
                for (int j = tid; j < 5 * kMaxK; j += kBT) ms->cs[j] = 0ull;
            g();
            for (int64_t i = gt; i < n; i += GT) {
                const uint32_t key = __ldcg(it.keys + i);
                const unsigned long long wi = __ldcg(it.weights + i);
                const unsigned long long r = key_r(key), gg = key_g(key), bb = key_b(key);
                unsigned long long *c = ms->cs + 5 * __ldcg(it.labels + i);
                atomicAdd(c + 0, wi * r);
                atomicAdd(c + 1, wi * gg);
                atomicAdd(c + 2, wi * bb);
                atomicAdd(c + 3, wi);
                atomicAdd(c + 4, wi * (r * r + gg * gg + bb * bb));
            }
            g();
        }
        if (g.rank == 0 && tid == 0) lbg_split(K, m, it.lbg_eps, ms->cs, it.centers);
        g();
        m += split;
        group_lloyd(g, it, n, m, it.lbg_conv_eps, it.lbg_max_iter, ms->lbg_pal, nullptr, status, sh, dyn);
    }
}

__device__ void group_seed(Group &g, const kq_batch_item &it, int64_t n, BatchShared &bs, LloydShared &sh,
                           uint32_t *dyn, int32_t *status)
{
    const int K = it.K, tid = threadIdx.x;
    if (it.scheme == KQ_INIT_USER) return;
    if (n <= K) {
        // the N' unique colours, padded with the last
        if (g.rank == 0)
            for (int k = tid; k < K; k += kBT) {
                if (n == 0) {
                    it.centers[3 * k] = it.centers[3 * k + 1] = it.centers[3 * k + 2] = 0.0;
                } else {
                    key_to_centre(it.centers + 3 * k, __ldcg(it.keys + (k < n ? k : n - 1)));
                }
            }
        g();
        return;
    }
    switch (it.scheme) {
    case KQ_INIT_FGY:
        if (g.rank == 0) {
            FyMap m{dyn, dyn + kMapSlots, kMapSlots - 1};
            uint32_t *pick = dyn + 2 * kMapSlots;
            clear_map(m.pos1, kMapSlots);
            __syncthreads();
            if (tid == 0) fisher_yates((uint32_t)n, (uint32_t)K, it.seed, 1, m, pick);
            __syncthreads();
            for (int k = tid; k < K; k += kBT) key_to_centre(it.centers + 3 * k, __ldcg(it.keys + pick[k]));
        }
        g();
        break;
    case KQ_INIT_SFF:
        if (g.rank == 0) {
            int s0 = (int)ceil(2.0 * K * log((double)K));
            if (s0 < K) s0 = K;
            sff_block(it.keys, n, K, it.seed, s0, it.centers, dyn);
        }
        g();
        break;
    case KQ_INIT_KPP:
        group_far(g, it, n, 0, bs);
        g();
        break;
    case KQ_INIT_MMX:
        group_far(g, it, n, 1, bs);
        g();
        break;
    case KQ_INIT_VAR:
        group_var(g, it, n, bs);
        break;
    case KQ_INIT_DEN:
        group_den(g, it, n, bs, dyn);
        break;
    case KQ_INIT_LBG:
        group_lbg(g, it, n, bs, sh, dyn, status);
        break;
    case KQ_INIT_WU: {
        // the split state in the step's dynamic shared memory (no other step's
        // data is live there during the seeding)
        WuShared &wsh = *reinterpret_cast<WuShared *>(dyn);
        unsigned long long *cell = g.at_slot<unsigned long long>(kSoWu);
        unsigned long long *cum = cell + 5 * (size_t)kWuCells;
        if (g.rank == 0)
            for (int j = tid; j < 5 * kWuCells; j += kBT) cell[j] = 0ull;
        g();
        wu_accumulate(it.keys, it.weights, n, cell, g.gtid(), g.nthreads());
        g();
        if (g.rank == 0) {
            wu_cumulate_block(cell, cum);
            wu_split_block(cum, K, it.centers, wsh);
        }
        g();
        break;
    }
    default:
        break;
    }
}

// ---------------------------------------------------------------- mapping
// Each unique colour's nearest palette entry (exact integers, lowest index on
// ties) goes into the counter table at its key; pixels then read it back; the
// touched entries are zeroed again at the end.
__device__ void group_map(const Group &g, const kq_batch_item &it, int64_t nu, BatchShared &bs)
{
    uint32_t *cnt = g.at_slot<uint32_t>(kSoCnt);
    const int GT = g.nthreads(), gt = g.gtid(), tid = threadIdx.x;
    const int K = it.K;
    for (int k = tid; k < K; k += kBT) {
        const uint32_t r = it.palette[3 * k], gg = it.palette[3 * k + 1], bb = it.palette[3 * k + 2];
        bs.pal[k] = make_uint2((r << 16) | (gg << 8) | bb, ((r * r + gg * gg + bb * bb) << 8) | (uint32_t)k);
    }
    __syncthreads();
    unsigned long long acc = 0ull;
    for (int64_t i = gt; i < nu; i += GT) {
        const uint32_t ka = __ldcg(it.keys + i);
        const uint32_t ba = __dp4a(ka, ka, 0u) << 8;
        uint32_t ma = 0xFFFFFFFFu;
#pragma unroll 8
        for (int k = 0; k < K; ++k) {
            const uint2 pk = bs.pal[k];
            ma = min(ma, ba + pk.y - (__dp4a(ka, pk.x, 0u) << 9));
        }
        cnt[ka] = ma & 0xFFu;
        acc += (unsigned long long)__ldcg(it.weights + i) * (ma >> 8);
    }
    const unsigned long long t = block_sum_u64<kBT>(acc, bs.red);
    if (tid == 0 && t && it.result) atomicAdd(reinterpret_cast<unsigned long long *>(&it.result->sse_num), t);
    g();
    const int64_t n = it.n_pixels;
    const uint8_t *rgb = it.rgb;
    uint8_t *idx = it.idx;
    const int64_t head = aligned_head(rgb, n);
    const int64_t ngroups = (n - head) / 16;
    const int64_t tail0 = head + ngroups * 16;
    for (int64_t p = gt; p < head; p += GT) idx[p] = (uint8_t)__ldcg(cnt + px_key(rgb, p));
    for (int64_t p = tail0 + gt; p < n; p += GT) idx[p] = (uint8_t)__ldcg(cnt + px_key(rgb, p));
    const uint4 *pg = reinterpret_cast<const uint4 *>(rgb + 3 * head);
    for (int64_t gi = gt; gi < ngroups; gi += GT) {
        const uint4 a = __ldcs(pg + 3 * gi), b = __ldcs(pg + 3 * gi + 1), c = __ldcs(pg + 3 * gi + 2);
        const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
        uint32_t key[16], v[16];
        Keys16<0>::get(w, key);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __ldcg(cnt + key[i]);
        uint8_t *dst = idx + head + 16 * gi;
#pragma unroll
        for (int i = 0; i < 16; ++i) dst[i] = (uint8_t)v[i];
    }
    g();
    for (int64_t i = gt; i < nu; i += GT) cnt[__ldcg(it.keys + i)] = 0u;
    g();
}

// ---------------------------------------------------------------- one image
__host__ __device__ __forceinline__ bool item_aligned(const kq_batch_item &it)
{
    return ((reinterpret_cast<uintptr_t>(it.keys) | reinterpret_cast<uintptr_t>(it.weights)) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(it.scratch) & 255u) == 0;
}

__device__ __forceinline__ bool item_ok(const kq_batch_item &it)
{
    return item_aligned(it) && it.n_pixels >= 0 && (it.rgb || it.n_pixels == 0) && (it.idx || it.n_pixels == 0) && it.K >= 1 &&
           it.K <= kMaxK && it.scheme >= KQ_INIT_FGY && it.scheme <= KQ_INIT_WU && it.max_iter >= 1 &&
           it.capacity >= 0 && it.keys && it.weights && it.labels && it.scratch && it.centers && it.palette &&
           it.result && (it.scheme != KQ_INIT_LBG || it.lbg_max_iter >= 1);
}

__device__ void run_item(Group &g, const kq_batch_item &it, BatchShared &bs, LloydShared &sh, uint32_t *dyn)
{
    const int tid = threadIdx.x;
    if (!item_ok(it)) {
        if (g.rank == 0 && tid == 0 && it.result) it.result->status = KQ_EINVAL;
        return;
    }
    kq_batch_result *res = it.result;
    if (g.rank == 0 && tid == 0) {
        res->t_ns[0] = (int64_t)globaltimer_ns();
        for (int j = 1; j < 5; ++j) res->t_ns[j] = 0;
        res->status = KQ_OK;
        res->n_unique = 0;
        res->sse_num = 0;
        res->lloyd.iters = 0;
        res->lloyd.converged = 0;
        res->lloyd.k_eff = 0;
        res->lloyd.status = KQ_OK;
        res->lloyd.ndc = 0;
        res->lloyd.sse = 0.0;
        res->lloyd.sse_prev = 0.0;
    }
    g();
    const int64_t nu = group_histogram(g, it, bs);
    if (nu > it.capacity) {
        if (g.rank == 0 && tid == 0) {
            res->n_unique = (int32_t)(nu < 0x7FFFFFFF ? nu : 0x7FFFFFFF);
            res->status = KQ_ECAPACITY;
        }
        g();
        return;
    }
    const bool lead = g.rank == 0 && tid == 0;
    if (lead) {
        res->n_unique = (int32_t)nu;
        res->t_ns[1] = (int64_t)globaltimer_ns();
    }
    group_seed(g, it, nu, bs, sh, dyn, &res->status);
    if (lead) res->t_ns[2] = (int64_t)globaltimer_ns();
    group_lloyd(g, it, nu, it.K, it.eps, it.max_iter, it.palette, &res->lloyd, &res->status, sh, dyn);
    if (lead) res->t_ns[3] = (int64_t)globaltimer_ns();
    group_map(g, it, nu, bs);
    if (lead) res->t_ns[4] = (int64_t)globaltimer_ns();
}

__global__ void __launch_bounds__(kBT, 1) batch_kernel(BatchArgs a)
{
    __shared__ LloydShared sh;
    __shared__ BatchShared bs;
    extern __shared__ __align__(16) uint32_t dyn[];
    const int tid = threadIdx.x;
    if (a.C > 1) {
        const int rank = (int)cluster_ctarank();
        Group g{a.C, rank, a.slots + (size_t)(blockIdx.x - rank) * kSlotBytes};
        SlotMisc *ms = g.misc();
        for (;;) {
            if (rank == 0 && tid == 0) ms->item = (int32_t)atomicAdd(&a.queue[0], 1u);
            g();
            const int j = __ldcg(&ms->item);
            g();
            if (j >= a.n_big) break;
            const int32_t id = __ldg(a.order + j);
            if (id < 0 || id >= a.n_items) continue;
            run_item(g, a.items[id], bs, sh, dyn);
        }
    }
    Group g{1, 0, a.slots + (size_t)blockIdx.x * kSlotBytes};
    const int n_small = a.n_items - a.n_big;
    for (;;) {
        if (tid == 0) bs.item = (int32_t)atomicAdd(&a.queue[1], 1u);
        __syncthreads();
        const int j = bs.item;
        __syncthreads();
        if (j >= n_small) break;
        const int32_t id = __ldg(a.order + a.n_big + j);
        if (id < 0 || id >= a.n_items) continue;
        run_item(g, a.items[id], bs, sh, dyn);
    }
}

// ---------------------------------------------------------------- live batches
// The queue lives in page-locked host memory: the host publishes items (release
// stores of the tails) while the kernel runs; groups claim them through counters
// in the workspace header and post each item's done mark with a release store.
constexpr size_t kLiveHeadOff = 64;  // the two claim counters in the workspace header
constexpr long long kLiveSingles = -1, kLiveExit = -2;

struct LiveArgs {
    const kq_live_queue *q;
    const kq_batch_item *items;  // [2][cap]
    uint32_t *done;              // [2][cap]
    uint32_t cap;
    uint32_t *head;              // [2] claims (device memory)
    int32_t C;
    uint64_t idle_ns;
    char *slots;
};

__device__ __forceinline__ uint32_t ld_acquire_sys_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Items published in class c and not yet claimed.
__device__ __forceinline__ bool live_pending(const LiveArgs &a, int c)
{
    const uint32_t t = ld_acquire_sys_u32(&a.q->tail[c]);
    return (int32_t)(t - *(volatile const uint32_t *)&a.head[c]) > 0;
}

// Claims the oldest unclaimed item of class c: its sequence number, or -1.
__device__ long long live_claim(const LiveArgs &a, int c)
{
    for (;;) {
        const uint32_t t = ld_acquire_sys_u32(&a.q->tail[c]);
        const uint32_t h = *(volatile const uint32_t *)&a.head[c];
        if ((int32_t)(t - h) <= 0) return -1;
        if (atomicCAS(&a.head[c], h, h + 1u) == h) return (long long)h;
    }
}

// Rank 0 of a cluster: a class-0 item to run, kLiveSingles while class-1 items
// wait, or kLiveExit once the queue is closed and drained or nothing came for the
// idle limit (measured from `last`, the group's last item).
__device__ long long live_decide(const LiveArgs &a, uint64_t last)
{
    for (;;) {
        const long long j = live_claim(a, 0);
        if (j >= 0) return j;
        if (live_pending(a, 1)) return kLiveSingles;
        if (ld_acquire_sys_u32(&a.q->closed) && !live_pending(a, 0) && !live_pending(a, 1)) return kLiveExit;
        if (globaltimer_ns() - last > a.idle_ns) return kLiveExit;
        __nanosleep(2000);
    }
}

// A class-1 item for a CTA on its own, or -1 (cluster launches: none waiting, or
// a class-0 item waits); single-CTA launches wait for one up to the idle limit
// and return kLiveExit after it, or once the queue is closed and drained.
__device__ long long live_next_single(const LiveArgs &a, uint64_t last)
{
    if (a.C > 1) return live_pending(a, 0) ? -1 : live_claim(a, 1);
    for (;;) {
        const long long k = live_claim(a, 1);
        if (k >= 0) return k;
        if (ld_acquire_sys_u32(&a.q->closed) && !live_pending(a, 1)) return kLiveExit;
        if (globaltimer_ns() - last > a.idle_ns) return kLiveExit;
        __nanosleep(2000);
    }
}

// The item of class c and sequence number seq, copied to shared memory (thread 0).
__device__ __forceinline__ void live_load(const LiveArgs &a, int c, uint32_t seq, kq_batch_item *dst)
{
    const unsigned long long *src =
        reinterpret_cast<const unsigned long long *>(a.items + (size_t)c * a.cap + seq % a.cap);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    for (int i = 0; i < (int)(sizeof(kq_batch_item) / 8); ++i) d[i] = __ldcv(src + i);
}

__device__ __forceinline__ void live_mark(const LiveArgs &a, int c, uint32_t seq)
{
    __threadfence_system();
    st_release_sys_u32(a.done + (size_t)c * a.cap + seq % a.cap, seq + 1u);
}

__global__ void __launch_bounds__(kBT, 1) batch_live_kernel(LiveArgs a)
{
    __shared__ LloydShared sh;
    __shared__ BatchShared bs;
    __shared__ kq_batch_item s_item;
    __shared__ long long s_dec;
    extern __shared__ __align__(16) uint32_t dyn[];
    const int tid = threadIdx.x, lane = tid & 31;
    const int rank = a.C > 1 ? (int)cluster_ctarank() : 0;
    Group gc{a.C, rank, a.slots + (size_t)(blockIdx.x - rank) * kSlotBytes};
    Group g1{1, 0, a.slots + (size_t)blockIdx.x * kSlotBytes};
    SlotMisc *ms = gc.misc();
    kq_batch_item *item = &s_item;
    uint64_t last = globaltimer_ns();
    // Lane 0 of warp 0 polls the queue; the rest of warp 0 waits for it in a
    // __shfl_sync, so that the warp reaches every block or cluster barrier
    // converged (an aligned barrier needs all of a warp's threads at once).
    for (;;) {
        if (a.C > 1) {
            if (rank == 0 && tid < 32) {
                long long d = 0;
                if (lane == 0) {
                    if (atomicExch(&ms->live_busy, 0)) last = globaltimer_ns();
                    d = live_decide(a, last);
                    ms->live_dec = d;
                }
                d = __shfl_sync(0xffffffffu, d, 0);
            }
            gc();
            const long long dec = __ldcg(&ms->live_dec);
            gc();
            if (dec == kLiveExit) return;
            if (dec >= 0) {
                __threadfence();
                if (tid == 0) live_load(a, 0, (uint32_t)dec, item);
                __syncwarp();
                __syncthreads();
                run_item(gc, *item, bs, sh, dyn);
                gc();
                if (rank == 0 && tid == 0) {
                    live_mark(a, 0, (uint32_t)dec);
                    last = globaltimer_ns();
                }
                __syncwarp();
                continue;
            }
        }
        // class-1 items, one CTA each
        bool ran = false;
        for (;;) {
            if (tid < 32) {
                long long d = 0;
                if (lane == 0) {
                    d = live_next_single(a, last);
                    s_dec = d;
                }
                d = __shfl_sync(0xffffffffu, d, 0);
            }
            __syncthreads();
            const long long k = s_dec;
            __syncthreads();
            if (k == kLiveExit) return;
            if (k < 0) break;
            __threadfence();
            if (tid == 0) live_load(a, 1, (uint32_t)k, item);
            __syncwarp();
            __syncthreads();
            run_item(g1, *item, bs, sh, dyn);
            __syncthreads();
            if (tid == 0) {
                live_mark(a, 1, (uint32_t)k);
                last = globaltimer_ns();
            }
            __syncwarp();
            ran = true;
        }
        if (a.C > 1 && ran && tid == 0) atomicExch(&ms->live_busy, 1);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- host side
struct BatchDev {
    bool done = false;
    int sms = 0;
    int per_sm = 0;
    int max_cluster = 1;
    int clusters[kMaxCluster + 1] = {};  // active clusters per size
};
BatchDev g_bdev[64];
std::mutex g_bmu;

int batch_attrs()
{
    if (cudaFuncSetAttribute((const void *)batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynBytes) !=
        cudaSuccess)
        return KQ_ECUDA;
    cudaFuncSetAttribute((const void *)batch_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    return KQ_OK;
}

const BatchDev *batch_dev()
{
    const DeviceInfo di = device_info();
    if (di.device < 0 || di.device >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_bmu);
    BatchDev &d = g_bdev[di.device];
    if (d.done) return &d;
    if (batch_attrs() != KQ_OK) return nullptr;
    d.sms = di.sms;
    d.per_sm = max_coresident((const void *)batch_kernel, kBT, kDynBytes);
    if (d.per_sm < 1) return nullptr;
    d.clusters[1] = d.sms * d.per_sm;
    d.max_cluster = 1;
    for (int c = 2; c <= kMaxCluster; c *= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kBT);
        cfg.dynamicSmemBytes = kDynBytes;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (const void *)batch_kernel, &cfg) == cudaSuccess && n >= 1) {
            d.clusters[c] = n;
            d.max_cluster = c;
        }
        cudaGetLastError();
    }
    d.done = true;
    return &d;
}

int grid_for(const BatchDev &d, int C) { return C > 1 ? d.clusters[C] * C : d.clusters[1]; }

bool host_item_ok(const kq_batch_item &it)
{
    return item_aligned(it) && it.n_pixels >= 0 && (it.rgb || it.n_pixels == 0) && (it.idx || it.n_pixels == 0) && it.K >= 1 &&
           it.K <= kMaxK && it.scheme >= KQ_INIT_FGY && it.scheme <= KQ_INIT_WU && it.max_iter >= 1 &&
           it.capacity >= 0 && it.keys && it.weights && it.labels && it.scratch && it.centers && it.palette &&
           it.result && it.eps == it.eps && (it.scheme != KQ_INIT_LBG || it.lbg_max_iter >= 1);
}

}  // namespace
}  // namespace kq

using namespace kq;

extern "C" KQ_API size_t kq_batch_scratch_bytes(int32_t capacity)
{
    if (capacity < 0) return 0;
    return align_up(sizeof(uint32_t) * 2 * (size_t)far_cap4(capacity), 256) +
           sizeof(unsigned long long) * 2 * (size_t)far_sstride(capacity) + 256;
}

extern "C" KQ_API size_t kq_batch_workspace_size(void)
{
    const BatchDev *d = batch_dev();
    if (!d) return 0;
    return kHeaderBytes + (size_t)d->clusters[1] * kSlotBytes;
}

extern "C" KQ_API int32_t kq_batch_max_cluster(void)
{
    const BatchDev *d = batch_dev();
    return d ? d->max_cluster : 0;
}

extern "C" KQ_API int kq_batch_plan(const kq_batch_item *h_items, int32_t n_items, const kq_batch_config *cfg,
                                    int32_t *h_order, int32_t *h_n_big)
{
    if (!h_items || n_items < 0 || !cfg || !h_order || !h_n_big) return KQ_EINVAL;
    if (cfg->cluster < 1 || cfg->cluster > kMaxCluster || (cfg->cluster & (cfg->cluster - 1))) return KQ_EINVAL;
    std::vector<int32_t> big, small;
    for (int32_t i = 0; i < n_items; ++i) {
        if (!host_item_ok(h_items[i])) return KQ_EINVAL;
        (cfg->cluster > 1 && h_items[i].n_pixels > cfg->split_pixels ? big : small).push_back(i);
    }
    // largest estimated work first: pixels (histogram, mapping) plus unique
    // colours times K (seeding and assignment), with N' ~ N / 3
    auto cost = [&](int32_t i) {
        const double n = (double)h_items[i].n_pixels;
        return n * (1.0 + h_items[i].K / 12.0);
    };
    auto by_cost = [&](int32_t x, int32_t y) {
        const double cx = cost(x), cy = cost(y);
        return cx != cy ? cx > cy : x < y;
    };
    std::sort(big.begin(), big.end(), by_cost);
    std::sort(small.begin(), small.end(), by_cost);
    int32_t o = 0;
    for (int32_t i : big) h_order[o++] = i;
    for (int32_t i : small) h_order[o++] = i;
    *h_n_big = (int32_t)big.size();
    return KQ_OK;
}

extern "C" KQ_API int kq_batch_run(const kq_batch_item *items, int32_t n_items, const int32_t *order, int32_t n_big,
                                   const kq_batch_config *cfg, void *ws, size_t ws_bytes, kq_stream_t stream)
{
    if (!cfg || !ws || n_items < 0 || n_big < 0 || n_big > n_items) return KQ_EINVAL;
    if (n_items > 0 && (!items || !order)) return KQ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return KQ_EINVAL;
    const int C = cfg->cluster;
    if (C < 1 || C > kMaxCluster || (C & (C - 1))) return KQ_EINVAL;
    if (C == 1 && n_big != 0) return KQ_EINVAL;
    const BatchDev *d = batch_dev();
    if (!d) return KQ_ECUDA;
    if (C > d->max_cluster || (C > 1 && d->clusters[C] < 1)) return KQ_EINVAL;
    const int grid = grid_for(*d, C);
    if (ws_bytes < kHeaderBytes + (size_t)grid * kSlotBytes) return KQ_ENOMEM;
    if (n_items == 0) return KQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BatchArgs a;
    a.items = items;
    a.order = order;
    a.n_items = n_items;
    a.n_big = n_big;
    a.C = C;
    a.queue = reinterpret_cast<uint32_t *>(ws);
    a.slots = static_cast<char *>(ws) + kHeaderBytes;
    if (cudaMemsetAsync(a.queue, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return KQ_ECUDA;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kBT);
    lc.dynamicSmemBytes = kDynBytes;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = C > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&lc, batch_kernel, a) == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

extern "C" KQ_API size_t kq_live_bytes(int32_t capacity)
{
    if (capacity < 1) return 0;
    return sizeof(kq_live_queue) + 2 * (size_t)capacity * (sizeof(kq_batch_item) + sizeof(uint32_t));
}

static kq_batch_item *live_items(kq_live_queue *q) { return reinterpret_cast<kq_batch_item *>(q + 1); }
static uint32_t *live_done(kq_live_queue *q)
{
    return reinterpret_cast<uint32_t *>(live_items(q) + 2 * (size_t)q->capacity);
}

extern "C" KQ_API int kq_live_init(kq_live_queue *q, int32_t capacity)
{
    if (!q || capacity < 1) return KQ_EINVAL;
    memset(q, 0, kq_live_bytes(capacity));
    q->capacity = (uint32_t)capacity;
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    return KQ_OK;
}

extern "C" KQ_API int kq_live_reset(void *ws, size_t ws_bytes, kq_stream_t stream)
{
    if (!ws || ws_bytes < kHeaderBytes || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return KQ_EINVAL;
    return cudaMemsetAsync(static_cast<char *>(ws) + kLiveHeadOff, 0, 2 * sizeof(uint32_t), (cudaStream_t)stream) ==
                   cudaSuccess
               ? KQ_OK
               : KQ_ECUDA;
}

extern "C" KQ_API int kq_live_publish(kq_live_queue *q, int32_t cls, const kq_batch_item *item, int64_t *h_seq)
{
    if (!q || !item || !h_seq || (cls != 0 && cls != 1) || q->capacity < 1) return KQ_EINVAL;
    if (__atomic_load_n(&q->closed, __ATOMIC_ACQUIRE) || !host_item_ok(*item)) return KQ_EINVAL;
    const uint32_t cap = q->capacity;
    const uint32_t t = __atomic_load_n(&q->tail[cls], __ATOMIC_RELAXED);
    uint32_t *done = live_done(q) + (size_t)cls * cap;
    const uint32_t slot = t % cap;
    // the slot's previous item (t - cap) must be done before it is overwritten
    if (t >= cap && __atomic_load_n(&done[slot], __ATOMIC_ACQUIRE) != t - cap + 1u) return KQ_ECAPACITY;
    live_items(q)[(size_t)cls * cap + slot] = *item;
    __atomic_store_n(&done[slot], 0u, __ATOMIC_RELAXED);
    __atomic_store_n(&q->tail[cls], t + 1u, __ATOMIC_RELEASE);
    *h_seq = (int64_t)t;
    return KQ_OK;
}

extern "C" KQ_API int kq_live_done(const kq_live_queue *q, int32_t cls, int64_t seq)
{
    if (!q || (cls != 0 && cls != 1) || seq < 0 || q->capacity < 1) return 0;
    const uint32_t cap = q->capacity;
    const uint32_t *done = live_done(const_cast<kq_live_queue *>(q)) + (size_t)cls * cap;
    return __atomic_load_n(&done[(uint32_t)seq % cap], __ATOMIC_ACQUIRE) == (uint32_t)seq + 1u ? 1 : 0;
}

extern "C" KQ_API int kq_live_close(kq_live_queue *q)
{
    if (!q) return KQ_EINVAL;
    __atomic_store_n(&q->closed, 1u, __ATOMIC_RELEASE);
    return KQ_OK;
}

extern "C" KQ_API int kq_live_run(kq_live_queue *q, const kq_batch_config *cfg, uint32_t idle_us, void *ws,
                                  size_t ws_bytes, kq_stream_t stream)
{
    if (!q || !cfg || !ws || idle_us < 1 || q->capacity < 1) return KQ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return KQ_EINVAL;
    const int C = cfg->cluster;
    if (C < 1 || C > kMaxCluster || (C & (C - 1))) return KQ_EINVAL;
    const BatchDev *d = batch_dev();
    if (!d) return KQ_ECUDA;
    if (C > d->max_cluster || (C > 1 && d->clusters[C] < 1)) return KQ_EINVAL;
    const int grid = grid_for(*d, C);
    if (ws_bytes < kHeaderBytes + (size_t)grid * kSlotBytes) return KQ_ENOMEM;
    // the queue must be page-locked host memory that the device can reach
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, q) != cudaSuccess || pa.type != cudaMemoryTypeHost || !pa.devicePointer) {
        cudaGetLastError();
        return KQ_EINVAL;
    }
    void *dq = pa.devicePointer;
    kq_live_queue *qd = static_cast<kq_live_queue *>(dq);
    LiveArgs a;
    a.q = qd;
    a.items = live_items(qd);
    a.cap = q->capacity;
    a.done = reinterpret_cast<uint32_t *>(live_items(qd) + 2 * (size_t)a.cap);
    a.head = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + kLiveHeadOff);
    a.C = C;
    a.idle_ns = (uint64_t)idle_us * 1000ull;
    a.slots = static_cast<char *>(ws) + kHeaderBytes;
    if (cudaFuncSetAttribute((const void *)batch_live_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kDynBytes) != cudaSuccess)
        return KQ_ECUDA;
    cudaFuncSetAttribute((const void *)batch_live_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kBT);
    lc.dynamicSmemBytes = kDynBytes;
    lc.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = C > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&lc, batch_live_kernel, a) == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

extern "C" KQ_API int kq_batch_tune(const kq_batch_item *h_items, const kq_batch_item *items, int32_t n_items,
                                    int32_t *order, kq_batch_config *h_best, int32_t *h_n_big, float *h_best_ms,
                                    void *ws, size_t ws_bytes, kq_stream_t stream)
{
    if (!h_items || !items || !order || !h_best || !h_n_big || n_items < 1) return KQ_EINVAL;
    const BatchDev *d = batch_dev();
    if (!d) return KQ_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<kq_batch_config> cands;
    cands.push_back(kq_batch_config{1, 0, 0});
    const int64_t splits[] = {1 << 18, 1 << 20, 1 << 22};
    for (int c = 2; c <= d->max_cluster; c *= 2)
        if (d->clusters[c] >= 1)
            for (int64_t sp : splits) cands.push_back(kq_batch_config{c, 0, sp});
    std::vector<int32_t> h_order((size_t)n_items);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return KQ_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KQ_ECUDA;
    }
    float best = -1.f;
    kq_batch_config best_cfg = cands[0];
    int st = KQ_OK;
    for (const kq_batch_config &c : cands) {
        int32_t nb = 0;
        st = kq_batch_plan(h_items, n_items, &c, h_order.data(), &nb);
        if (st != KQ_OK) break;
        if (cudaMemcpyAsync(order, h_order.data(), sizeof(int32_t) * n_items, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = KQ_ECUDA;
            break;
        }
        float ms_best = -1.f;
        for (int rep = 0; rep < 3 && st == KQ_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = kq_batch_run(items, n_items, order, nb, &c, ws, ws_bytes, stream);
            cudaEventRecord(e1, s);
            if (st != KQ_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = KQ_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (ms_best < 0.f || ms < ms_best)) ms_best = ms;  // first run warms up
        }
        if (st != KQ_OK) break;
        if (best < 0.f || ms_best < best) {
            best = ms_best;
            best_cfg = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KQ_OK) return st;
    *h_best = best_cfg;
    if (h_best_ms) *h_best_ms = best;
    int32_t nb = 0;
    st = kq_batch_plan(h_items, n_items, &best_cfg, h_order.data(), &nb);
    if (st != KQ_OK) return st;
    *h_n_big = nb;
    if (cudaMemcpyAsync(order, h_order.data(), sizeof(int32_t) * n_items, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return KQ_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? KQ_OK : KQ_ECUDA;
}
