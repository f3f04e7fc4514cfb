// seed.cu -- the generic initialization schemes of Section 2.3 on the GPU.
//
// Every scheme except LBG picks unique colours, so its arithmetic is integer and
// its result is exact.  Random draws follow the counter-based SplitMix64 streams
// documented in kq.h: stream 1 Forgy, 2 k-means++, 3 minmax, 4/5 subset farthest
// first, 16 + cell for the density scheme.
//
//   FGY  partial Fisher-Yates on one thread, the displaced entries in a shared
//        memory hash map.
//   KPP, MMX  one thread-block cluster (N' up to 16 x 11264) or one persistent
//        cooperative kernel over the grid: per round every block refreshes its
//        slice's nearest-centre distances (exact integers); KPP sums w D^2 per
//        block, every block finds from the block sums the block that holds the
//        sample, and that block finds the colour in its own slice and posts its
//        key; MMX takes a packed (D^2, lowest index) maximum with one atomic per
//        block.  One grid barrier per round.
//   SFF  one block: subset draw, sort, then minmax over the subset.
//   VAR  per-chunk value counts and exact weighted moments, then one warp per
//        group median locates the element of the requested rank.
//   DEN  per-chunk cell counts, the seat apportionment on one thread, then one
//        block per cell draws and locates its members.
//   LBG  centroid, then split rounds that call the Lloyd kernel.
//   WU   (Section 3.3's preclustering, the WSM-WU initializer) moments per 32^3
//        cell by atomics over the unique colours, cumulative moments line by line
//        over the grid, then one block makes the greedy splits.
#include <math.h>

#include "seed_dev.cuh"

namespace kq {
namespace {

constexpr int kFarBlock = 1024;
constexpr int kChunkBlock = 256;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- K >= N'
// The centres are the N' unique colours in key order, padded with the last.
__global__ void seed_all_unique(const uint32_t *keys, const int32_t *n_unique, int K, double *centers)
{
    const int64_t n = *n_unique;
    if (n > K) return;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (n == 0) {
            centers[3 * k] = centers[3 * k + 1] = centers[3 * k + 2] = 0.0;
        } else {
            key_to_centre(centers + 3 * k, keys[k < n ? k : n - 1]);
        }
    }
}

// Forgy: K distinct unique colours drawn uniformly (Algorithm 2, first line).
__global__ void seed_fgy(const uint32_t *keys, const int32_t *n_unique, int K, uint64_t seed, double *centers)
{
    extern __shared__ uint32_t smem[];
    const int64_t n = *n_unique;
    if (n <= K) return;
    FyMap m{smem, smem + kMapSlots, kMapSlots - 1};
    uint32_t *pick = smem + 2 * kMapSlots;
    clear_map(m.pos1, kMapSlots);
    __syncthreads();
    if (threadIdx.x == 0) fisher_yates((uint32_t)n, (uint32_t)K, seed, 1, m, pick);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) key_to_centre(centers + 3 * k, keys[pick[k]]);
}

// ---------------------------------------------------------------- SFF
// Minmax on a uniform random subset of size min(N', s0), s0 = max(K, ceil(2 K ln K)).
// The subset is taken in ascending index order; ties go to the lowest index.
constexpr int kSffBlock = 256;

__global__ void __launch_bounds__(kSffBlock) seed_sff(const uint32_t *keys, const int32_t *n_unique, int K,
                                                      uint64_t seed, int s0, double *centers)
{
    extern __shared__ uint32_t smem[];
    const int64_t n = *n_unique;
    if (n <= K) return;
    sff_block(keys, n, K, seed, s0, centers, smem);
}

// ---------------------------------------------------------------- KPP / MMX
struct FarArgs {
    const uint32_t *keys;
    const uint32_t *w;
    const int32_t *n_unique;
    int K;
    int mode;  // 0 = k-means++, 1 = minmax
    uint64_t seed;
    int64_t max_unique;
    double *centers;
    Ctl *ctl;
    uint32_t *d2;               // [2][max_unique]
    unsigned long long *part;   // [2][kMaxGrid] block sums
    unsigned long long *gpart;  // [2][gpart_cap] sums of 32-colour groups
    int64_t gpart_cap;
    unsigned long long *slot;   // [kMaxK]
    int64_t cluster_cap;        // N' served by seed_far_cluster (0 when it is not used)
};

constexpr int kFarWarps = kFarBlock / 32;
constexpr int kFarChunk = 2048;  // fewest colours per block
constexpr int kFarRes = 16384;  // colours a block keeps in shared memory (key, w, D^2)
constexpr size_t kFarSmem = 3 * sizeof(uint32_t) * (size_t)kFarRes;
constexpr int kFindRegs = 8;    // values per lane that warp_find keeps in registers
constexpr int kFarUnroll = 2;   // groups per warp step in the D^2 update

struct FarShared {
    unsigned long long wsum[kFarWarps];
    unsigned long long gp[kFarRes / 32];  // k-means++: sums of w D^2 of the slice's 32-colour groups
    uint32_t key;
};

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Round r's key as posted by the block that holds the sample (slot = key + 2^32),
// waited for with the limit of the grid barrier; 0xFFFFFFFF if the wait gave up.
__device__ __forceinline__ uint32_t far_await_key(const unsigned long long *slot, Ctl *ctl, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t spin = 0;; ++spin) {
        const unsigned long long v = ld_acquire_gpu_u64(slot);
        if (v) return (uint32_t)(v & 0xFFFFFFull);
        __nanosleep(64);
        if ((spin & 63u) == 63u) {
            if (ld_acquire_gpu(&ctl->abort)) return 0xFFFFFFFFu;
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > limit_ns) {
                fail(ctl, KQ_ETIMEOUT);
                atomicExch(&ctl->abort, 1u);
                return 0xFFFFFFFFu;
            }
        }
    }
}

// First index i < count whose running sum of vals[0..i] exceeds t, and t minus the
// sum before it (one warp; every lane returns the same).  Lane l sums the values
// [l m, l m + m), m = ceil(count / 32), with one round of loads; a warp scan of the
// lane sums finds the lane, which then walks its own values.  `draw`: t is
// below(u, total of all values) instead of u itself.
template <bool kShared = false>
__device__ __forceinline__ int warp_find(const unsigned long long *vals, int count, bool draw, uint64_t u,
                                         unsigned long long *resid)
{
    auto ld = [](const unsigned long long *q) { return kShared ? *q : __ldcg(q); };
    const int lane = threadIdx.x & 31;
    const int m = (count + 31) / 32;
    unsigned long long v[kFindRegs];
    unsigned long long ls = 0ull;
#pragma unroll
    for (int j = 0; j < kFindRegs; ++j) {
        const int i = lane * m + j;
        v[j] = (j < m && i < count) ? ld(vals + i) : 0ull;
        ls += v[j];
    }
    for (int j = kFindRegs; j < m; ++j) {
        const int i = lane * m + j;
        if (i < count) ls += ld(vals + i);
    }
    unsigned long long x = ls;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    const unsigned long long t = draw ? below(u, __shfl_sync(kFull, x, 31)) : u;
    const int L = __ffs(__ballot_sync(kFull, x > t)) - 1;  // exists: t < total
    unsigned long long run = x - ls;
    int idx = 0;
    if (lane == L) {
        bool found = false;
#pragma unroll
        for (int j = 0; j < kFindRegs; ++j) {
            if (!found && j < m) {
                if (run + v[j] > t) {
                    idx = lane * m + j;
                    found = true;
                } else {
                    run += v[j];
                }
            }
        }
        for (int j = kFindRegs; !found && j < m; ++j) {
            const unsigned long long vj = ld(vals + lane * m + j);
            if (run + vj > t) {
                idx = lane * m + j;
                found = true;
            } else {
                run += vj;
            }
        }
    }
    idx = __shfl_sync(kFull, idx, L);
    *resid = t - __shfl_sync(kFull, run, L);
    return idx;
}

// k-means++ sampling by inverse CDF (warp 0 of every block, all computing the same
// key).  With total = the sum of P over all colours (P = w in the first round, w D^2
// after) and t = below(u, total), the sample is the first colour, in key order,
// whose running sum of P exceeds t.  Three levels, one round of loads each: the
// block sums, the 32-colour group sums of that block, the colours of that group.
__device__ uint32_t far_locate(const FarArgs &a, int G, int64_t n, int64_t gstride, int buf, uint64_t u,
                               bool first_round)
{
    const int lane = threadIdx.x & 31;
    unsigned long long r1, r2;
    const int g = warp_find(a.part + (size_t)buf * kMaxGrid, G, true, u, &r1);
    int64_t lo, hi;
    slice_of(n, g, G, &lo, &hi);
    const int ng = (int)((hi - lo + 31) / 32);
    const int q = warp_find(a.gpart + (size_t)buf * a.gpart_cap + (size_t)g * gstride, ng, false, r1, &r2);
    const int64_t i = lo + 32 * (int64_t)q + lane;
    unsigned long long p = 0ull;
    uint32_t key = 0u;
    if (i < hi) {
        const unsigned long long wi = __ldcg(a.w + i);
        p = first_round ? wi : wi * (unsigned long long)__ldcg(a.d2 + (size_t)buf * a.max_unique + i);
        key = __ldcg(a.keys + i);
    }
    unsigned long long x = p;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    const int l3 = __ffs(__ballot_sync(kFull, x > r2)) - 1;
    return __shfl_sync(kFull, key, l3 < 0 ? 0 : l3);
}

// k-means++ sampling when every block keeps its slice in shared memory: every
// block finds, from the block sums, the block g whose range holds t = below(u,
// total); block g alone finds the group and the colour in its own shared memory
// and posts the key to round r's slot, which the other blocks wait for.
__device__ uint32_t far_locate_owner(const FarArgs &a, FarShared &sh, const uint32_t *s_key, const uint32_t *s_w,
                                     const uint32_t *s_d2, int G, int b, int cnt, int buf, int r, Ctl *ctl,
                                     uint64_t limit_ns)
{
    const int lane = threadIdx.x & 31;
    unsigned long long r1, r2;
    const int g = warp_find(a.part + (size_t)buf * kMaxGrid, G, true, rand64(a.seed, 2, (uint32_t)r), &r1);
    if (g != b) {
        uint32_t k = 0u;
        if (lane == 0) k = far_await_key(a.slot + r, ctl, limit_ns);
        return __shfl_sync(kFull, k, 0);
    }
    const int q = warp_find<true>(sh.gp, (cnt + 31) / 32, false, r1, &r2);
    const int j = 32 * q + lane;
    unsigned long long p = 0ull;
    uint32_t key = 0u;
    if (j < cnt) {
        key = s_key[j];
        p = r == 0 ? (unsigned long long)s_w[j] : (unsigned long long)s_w[j] * s_d2[j];
    }
    unsigned long long x = p;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    const int l3 = __ffs(__ballot_sync(kFull, x > r2)) - 1;
    key = __shfl_sync(kFull, key, l3 < 0 ? 0 : l3);
    if (lane == 0) st_release_gpu_u64(a.slot + r, (1ull << 32) | key);
    return key;
}

// KPP / minmax over the whole grid, for N' above what one cluster holds.  Block b
// owns a contiguous slice of the unique colours; while a slice fits kFarRes colours
// the block keeps its keys, weights and D^2 in shared memory for all K rounds, and
// k-means++ keeps the sums of w D^2 of its 32-colour groups there too: the block
// that holds a round's sample finds it locally (far_locate_owner).  Larger slices
// live in global memory, where every block locates the sample (far_locate).  Warps
// take the slice's groups in turn and sum P per group (k-means++) or fold the
// packed (D^2, key) maximum into the round's slot (minmax).  One grid barrier per
// round.
__global__ void __launch_bounds__(kFarBlock, 1) seed_far(FarArgs a)
{
    __shared__ FarShared sh;
    extern __shared__ uint32_t far_smem[];  // key[kFarRes], w[kFarRes], d2[kFarRes]
    uint32_t *s_key = far_smem, *s_w = far_smem + kFarRes, *s_d2 = far_smem + 2 * kFarRes;
    const int64_t n = *a.n_unique;
    if (n <= a.K || n <= a.cluster_cap) return;  // the cluster kernel serves N' <= cluster_cap
    const int K = a.K;
    const int64_t want = (n + kFarChunk - 1) / kFarChunk;
    const int G = (int)(want > gridDim.x ? gridDim.x : want);
    const int b = blockIdx.x;
    if (b >= G) return;
    Ctl *ctl = a.ctl;
    uint32_t bar_epoch = 0;
    const uint32_t bar_n = (uint32_t)G + *(volatile const uint32_t *)&ctl->missing;
    const uint64_t limit_ns = wait_limit_ns(ctl);
    if (n > a.max_unique) {
        if (b == 0 && threadIdx.x == 0) fail(ctl, KQ_ENOMEM);
        return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (n + G - 1) / G;
    const int64_t gstride = (per + 31) / 32;
    const bool res = per <= kFarRes;  // the same for every block
    int64_t lo, hi;
    slice_of(n, b, G, &lo, &hi);
    const int cnt = (int)(hi - lo);  // < 2^31: at most 2^24 colours in all
    const int ng = (cnt + 31) / 32;
    if (res) {
        for (int64_t j = tid; j < cnt; j += kFarBlock) {
            s_key[j] = a.keys[lo + j];
            s_w[j] = a.w[lo + j];
        }
    }
    if (b == 0)
        for (int k = tid; k < kMaxK; k += kFarBlock) a.slot[k] = 0ull;
    __syncthreads();
    uint32_t ckey = 0u;
    for (int r = 0; r < K; ++r) {
        const int buf = r & 1;
        if (r > 0 || a.mode == 0) {
            // D^2 of round r alternates between two global buffers: other blocks may
            // still read round r - 1's values while this block writes round r's.
            uint32_t *d2 = a.d2 + (size_t)buf * (size_t)a.max_unique + lo;
            const uint32_t *d2p = a.d2 + (size_t)(buf ^ 1) * (size_t)a.max_unique + lo;
            unsigned long long *gp = a.gpart + (size_t)buf * a.gpart_cap + (size_t)b * gstride;
            unsigned long long acc = 0ull;
            const uint32_t *kp = a.keys + lo, *wp = a.w + lo;
            // kFarUnroll groups per step (q0 + u kFarWarps): all loads first, then the
            // arithmetic, the stores and the group sums
            for (int q0 = warp; q0 < ng; q0 += kFarUnroll * kFarWarps) {
                uint32_t key[kFarUnroll], wj[kFarUnroll], dp[kFarUnroll];
                bool in[kFarUnroll];
#pragma unroll
                for (int u = 0; u < kFarUnroll; ++u) {
                    const int j = 32 * (q0 + u * kFarWarps) + lane;
                    in[u] = q0 + u * kFarWarps < ng && j < cnt;
                    key[u] = 0u;
                    wj[u] = 0u;
                    dp[u] = 0xFFFFFFFFu;
                    if (in[u]) {
                        key[u] = res ? s_key[j] : kp[j];
                        wj[u] = res ? s_w[j] : wp[j];
                        if (r >= 2) dp[u] = res ? s_d2[j] : __ldcg(d2p + j);
                    }
                }
                unsigned long long pv[kFarUnroll];
#pragma unroll
                for (int u = 0; u < kFarUnroll; ++u) {
                    const int q = q0 + u * kFarWarps;
                    const int j = 32 * q + lane;
                    pv[u] = 0ull;
                    if (r == 0) {
                        pv[u] = wj[u];  // k-means++ first centre: probability w / sum w
                    } else if (q < ng) {
                        const uint32_t md = min(dp[u], key_dist2(key[u], ckey));
                        if (in[u]) {
                            if (res) s_d2[j] = md;
                            else d2[j] = md;
                        }
                        if (in[u]) pv[u] = a.mode == 0 ? (unsigned long long)wj[u] * md : mmx_pack(md, key[u]);
                    }
                }
                if (a.mode == 0) {
                    // w D^2 < 2^32 * 3 * 255^2 < 2^50: the 25-bit halves of 32 such values
                    // sum exactly in 32 bits, one warp reduction each
#pragma unroll
                    for (int u = 0; u < kFarUnroll; ++u) {
                        const int q = q0 + u * kFarWarps;
                        const uint32_t slo = __reduce_add_sync(kFull, (uint32_t)(pv[u] & 0x1FFFFFFull));
                        const uint32_t shi = __reduce_add_sync(kFull, (uint32_t)(pv[u] >> 25));
                        const unsigned long long gs = ((unsigned long long)shi << 25) + slo;
                        if (q < ng) {
                            if (lane == 0) {
                                if (res) sh.gp[q] = gs;
                                else gp[q] = gs;
                            }
                            acc += gs;
                        }
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < kFarUnroll; ++u) acc = pv[u] > acc ? pv[u] : acc;
                }
            }
            if (a.mode == 0) {
                if (lane == 0) sh.wsum[warp] = acc;
                __syncthreads();
                if (tid == 0) {
                    unsigned long long s = 0ull;
                    for (int k = 0; k < kFarWarps; ++k) s += sh.wsum[k];
                    a.part[(size_t)buf * kMaxGrid + b] = s;
                }
            } else {
                for (int o = 16; o; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(kFull, acc, o);
                    acc = other > acc ? other : acc;
                }
                if (lane == 0) sh.wsum[warp] = acc;
                __syncthreads();
                if (tid == 0) {
                    unsigned long long mx = 0ull;
                    for (int k = 0; k < kFarWarps; ++k) mx = sh.wsum[k] > mx ? sh.wsum[k] : mx;
                    if (mx) atomicMax(a.slot + r, mx);
                }
            }
        }
        if (!grid_sync(ctl, bar_n, &bar_epoch, limit_ns)) return;
        if (a.mode == 0) {
            if (warp == 0) {
                const uint32_t k = res ? far_locate_owner(a, sh, s_key, s_w, s_d2, G, b, cnt, buf, r, ctl, limit_ns)
                                       : far_locate(a, G, n, gstride, buf, rand64(a.seed, 2, (uint32_t)r), r == 0);
                if (lane == 0) sh.key = k;
            }
        } else if (tid == 0) {
            sh.key = r == 0 ? __ldg(a.keys + below(rand64(a.seed, 3, 0), (uint64_t)n))
                            : 0xFFFFFFu - (uint32_t)(__ldcg(a.slot + r) & 0xFFFFFFull);
        }
        __syncthreads();
        ckey = sh.key;
        if (ckey == 0xFFFFFFFFu) return;  // a wait gave up (status KQ_ETIMEOUT)
        if (b == 0 && tid == 0) key_to_centre(a.centers + 3 * r, ckey);
    }
}

// ---------------------------------------------------------------- KPP / MMX in one cluster
// For N' up to C * kClPer colours (C = 16, else 8), one thread-block cluster runs
// every round.  Each CTA holds a contiguous slice of the unique colours, thread t
// a contiguous run of it: keys, weights, |x|^2 and D^2 stay in registers, and for
// k-means++ the running sum of w D^2 over the thread's colours goes to shared
// memory next to the keys.
//
// A round needs no whole-cluster barrier.  Its exchanges are pushes:
//  1. every warp sends its total of w D^2 (k-means++) or its packed (D^2, key)
//     maximum (minmax) to every CTA of the cluster with st.async, whose
//     complete_tx counts the bytes on the receiving CTA's "data" mbarrier;
//  2. minmax: once the data barrier has every warp's value, warp 0 takes the
//     maximum, which holds the next centre's key;
//     k-means++: warp 0 finds, from the CTA totals, the CTA g that holds the
//     sample (t = below(u, sum) falls in its range).  Only CTA g goes on to find
//     the warp, the thread and the colour -- all in its own shared memory -- and
//     sends the key to every CTA with st.async on their "key" mbarrier;
//  3. warp 0 passes the key to the other warps of its CTA (one __syncthreads).
// Only warp 0 waits on the mbarriers (waiting warps would take issue slots from
// the warps still working).  Each mbarrier exists twice and serves the rounds of
// one parity; warp 0 re-arms the barrier of round r (expect_tx for round r + 2)
// as soon as it has seen round r complete.  Pushes for round r + 2 cannot come
// earlier: they need every warp of this CTA to have pushed round r + 1, which
// each does after the __syncthreads that follows warp 0's waits of round r.  The
// same argument makes one copy of the running sums enough: CTA g reads them
// before it sends the key, and its warps rewrite them only after the key came.
// Every wait is bounded (kWaitNs, or the control block's wait_limit_us); when
// warp 0 gives up it records KQ_ETIMEOUT and the whole CTA leaves the rounds;
// all CTAs then meet at the final cluster barrier, so no CTA exits while another
// can still write to it.
constexpr int kClBlock = 512;
constexpr int kClWarps = kClBlock / 32;
constexpr int kClElems = 22;                 // colours per thread at most
constexpr int kClPer = kClBlock * kClElems;  // colours per CTA (11264)
// shared-memory slots per array: thread t uses t * (EPT | 1) + k, k < EPT <= kClElems
constexpr int kClSlots = kClBlock * (kClElems | 1);
constexpr int kClMaxCtas = 16;

struct ClusterArgs {
    const uint32_t *keys;
    const uint32_t *w;
    const int32_t *n_unique;
    int K;
    int mode;  // 0 = k-means++, 1 = minmax
    int ctas;  // cluster size: 8 or 16
    uint64_t seed;
    double *centers;
    Ctl *ctl;
};

struct ClusterShared {
    unsigned long long tpre[kClBlock];  // k-means++: warp-local inclusive prefix of the threads' sums
    // every CTA's warp totals (k-means++) or maxima (minmax), pushed by their warps;
    // rows padded to 17 entries
    unsigned long long wtot[2][kClMaxCtas][kClWarps + 1];
    unsigned long long bar_data[2];  // mbarriers: all C x 16 warp values of a round have arrived
    unsigned long long bar_key[2];   // mbarriers: the round's k-means++ sample has arrived
    uint32_t key[2];                 // the round's centre: pushed by CTA g (k-means++) or set by warp 0 (minmax)
    int dead;                        // warp 0 gave up waiting
};

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The shared::cluster address of the same variable in CTA `rank`.
__device__ __forceinline__ uint32_t dsmem_addr(const void *local, uint32_t rank)
{
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(local)), "r"(rank));
    return out;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// One arrival on the current phase, which also expects `bytes` of transactions.
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits (whole warp) until the phase of `bar` with the given parity has completed.
// Gives up after limit_ns: records KQ_ETIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, Ctl *ctl, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t spin = 0;; ++spin) {
        if (__all_sync(kFull, mbar_test(bar, parity))) return true;
        if ((spin & 15u) == 15u) {
            int give_up = 0;
            if ((threadIdx.x & 31) == 0) {
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > limit_ns) give_up = 1;
            }
            if (__shfl_sync(kFull, give_up, 0)) {
                if ((threadIdx.x & 31) == 0) fail(ctl, KQ_ETIMEOUT);
                return false;
            }
        }
    }
}

// st.async of one value into CTA-shared memory of a cluster peer; the receiving
// mbarrier's transaction count goes down by the value's size once it has landed.
__device__ __forceinline__ void push_u64(uint32_t addr, unsigned long long v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr), "l"(v),
                 "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void push_u32(uint32_t addr, uint32_t v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr), "r"(v),
                 "r"(bar)
                 : "memory");
}

// Inclusive scan over the first 2^S lanes (the other lanes add nothing useful).
template <int S>
__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long x, int lane)
{
#pragma unroll
    for (int o = 1; o < (1 << S); o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFull, x, o);
        x = y > x ? y : x;
    }
    return x;
}

// Which pushed warp values lane `lane` combines in cta_values (computed once per
// kernel: C is 8 or 16, so lanes_per_cta = 32 / C is 4 or 2).
struct CtaLanes {
    int row;   // CTA whose values this lane reads
    int col;   // first of its warps
    int per;   // warps per lane: 16 / lanes_per_cta
    int lpc;   // lanes per CTA
    int from;  // lane holding CTA (lane % C)'s result
};

__device__ __forceinline__ CtaLanes cta_lanes(int C, int lane)
{
    const int sh = C == 16 ? 1 : 2;
    CtaLanes L;
    L.lpc = 1 << sh;
    L.row = lane >> sh;
    L.per = kClWarps >> sh;
    L.col = (lane & (L.lpc - 1)) * L.per;
    L.from = (lane & (C - 1)) << sh;
    return L;
}

// Sum (k-means++) or maximum (minmax) per CTA of the C x 16 pushed warp values: the
// lanes of CTA c each combine `per` of its warps (a two-level tree), then the
// lanes_per_cta partial results are combined; the result for CTA c is returned in
// lane c (lanes >= C get copies).
template <bool KPP>
__device__ __forceinline__ unsigned long long cta_values(const ClusterShared &sh, int b, const CtaLanes &L)
{
    const unsigned long long *row = &sh.wtot[b][L.row][L.col];
    unsigned long long v[kClWarps / 2];
#pragma unroll
    for (int q = 0; q < kClWarps / 2; ++q) v[q] = q < L.per ? row[q] : 0ull;
#pragma unroll
    for (int w = kClWarps / 4; w; w >>= 1) {
#pragma unroll
        for (int q = 0; q < w; ++q) v[q] = KPP ? v[q] + v[q + w] : (v[q + w] > v[q] ? v[q + w] : v[q]);
    }
    unsigned long long s = v[0];
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        if (o < L.lpc) {
            const unsigned long long y = __shfl_down_sync(kFull, s, o);
            s = KPP ? s + y : (y > s ? y : s);
        }
    }
    return __shfl_sync(kFull, s, L.from);
}

// The K rounds of one CTA whose threads hold EPT or EPT - 1 colours each.  The CTA's
// `cnt` colours start at global index lo; thread t holds base + (t < rem) of them,
// from position t * base + min(t, rem), and keeps their keys (and running sums) in
// shared memory at t * kEps + k (an odd stride: a warp's accesses hit distinct banks).
template <int EPT, bool KPP>
__device__ __forceinline__ void cluster_rounds(const ClusterArgs &a, ClusterShared &sh, uint32_t *s_key,
                                               uint32_t *s_aux, unsigned long long *s_pre, int64_t lo, int cnt, int C,
                                               uint32_t rank, int64_t n)
{
    constexpr int kEps = EPT | 1;
    // up to 16 colours per thread |x|^2 and the weights stay in registers; above that
    // |x|^2 is recomputed and the weights are read from shared memory (no spills)
    constexpr bool kNormRegs = EPT <= 16;
    constexpr int kNr = kNormRegs ? EPT : 1;
    const int K = a.K, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int base = cnt / kClBlock, rem = cnt % kClBlock;
    const int mine = base + (tid < rem ? 1 : 0);  // EPT or EPT - 1
    const int64_t start = lo + (int64_t)tid * base + (tid < rem ? tid : rem);
    uint32_t key[EPT], aux[kNr], nrm[kNr], d2[EPT];  // aux: weight (k-means++) or 0xFFFFFF - key (minmax)
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        key[k] = 0u;
        if (kNormRegs) aux[k < kNr ? k : 0] = 0u;
        d2[k] = 0xFFFFFFFFu;
        if (k < mine) {
            key[k] = a.keys[start + k];
            const uint32_t ax = KPP ? a.w[start + k] : 0xFFFFFFu - key[k];
            if (kNormRegs) aux[k < kNr ? k : 0] = ax;
            else s_aux[tid * kEps + k] = ax;
            s_key[tid * kEps + k] = key[k];
        }
        if (kNormRegs) nrm[k < kNr ? k : 0] = key_norm2(key[k]);
    }
    // a round's warp values, plus one per arrival the test hook Ctl::missing asks for
    const uint32_t data_bytes =
        ((uint32_t)C * kClWarps + *(volatile const uint32_t *)&a.ctl->missing) * (uint32_t)sizeof(unsigned long long);
    const uint64_t limit_ns = wait_limit_ns(a.ctl);
    // addresses of the round-parity b copies: the b = 0 address plus b times the stride
    constexpr uint32_t kWtotStride = sizeof(sh.wtot[0]);
    const uint32_t bar_data0 = smem_u32(&sh.bar_data[0]), bar_key0 = smem_u32(&sh.bar_key[0]);
    if (tid == 0) {
        for (uint32_t b = 0; b < 2; ++b) {
            mbar_init(bar_data0 + 8u * b, 1);
            mbar_init(bar_key0 + 8u * b, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (uint32_t b = 0; b < 2; ++b) {
            mbar_arrive_expect(bar_data0 + 8u * b, data_bytes);
            mbar_arrive_expect(bar_key0 + 8u * b, (uint32_t)sizeof(uint32_t));
        }
        sh.dead = 0;
    }
    // Lane c < C sends to CTA c: this warp's slot and the barriers there.
    uint32_t to_wtot = 0u, to_data = 0u, to_key = 0u, to_kbar = 0u;
    if (lane < C) {
        to_wtot = dsmem_addr(&sh.wtot[0][rank][warp], (uint32_t)lane);
        to_data = dsmem_addr(&sh.bar_data[0], (uint32_t)lane);
        to_key = dsmem_addr(&sh.key[0], (uint32_t)lane);
        to_kbar = dsmem_addr(&sh.bar_key[0], (uint32_t)lane);
    }
    // every CTA's barriers exist and are armed before anyone pushes
    cluster_sync_all();

    const CtaLanes lanes = cta_lanes(C, lane);
    uint32_t ckey = 0u, cnorm = 0u;
    for (int r = 0; r < K; ++r) {
        const int b = r & 1;
        const uint32_t ph = (uint32_t)(r >> 1) & 1u;
        uint64_t u = 0;
        if (warp == 0) u = KPP ? rand64(a.seed, 2, (uint32_t)r) : rand64(a.seed, 3, 0);
        // ---- this thread's colours: D^2 to the newest centre; w D^2 running sums or the packed maximum
        unsigned long long acc = 0ull;
        if (r > 0) {
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
                if (k < EPT - 1 || k < mine) {
                    const uint32_t nk = kNormRegs ? nrm[k < kNr ? k : 0] : key_norm2(key[k]);
                    const uint32_t d = nk + cnorm - 2u * __dp4a(key[k], ckey, 0u);
                    const uint32_t md = min(d2[k], d);
                    d2[k] = md;
                    const uint32_t ax = kNormRegs ? aux[k < kNr ? k : 0] : s_aux[tid * kEps + k];
                    if (KPP) {
                        acc += (unsigned long long)ax * md;
                        s_pre[tid * kEps + k] = acc;
                    } else {
                        const unsigned long long pk = ((unsigned long long)md << 24) | ax;
                        acc = pk > acc ? pk : acc;
                    }
                }
            }
        } else if (KPP) {
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
                if (k < EPT - 1 || k < mine) {
                    acc += kNormRegs ? aux[k < kNr ? k : 0] : s_aux[tid * kEps + k];  // first centre: w / sum w
                    s_pre[tid * kEps + k] = acc;
                }
            }
        }
        // ---- the warp's total (with the threads' prefixes) or maximum, pushed to every CTA
        unsigned long long wv;
        if (KPP) {
            const unsigned long long x = warp_incl_scan_u64<5>(acc, lane);
            sh.tpre[tid] = x;
            wv = __shfl_sync(kFull, x, 31);
        } else {
            wv = warp_max_u64(acc);
        }
        __syncwarp();  // the lanes' shared-memory writes above precede the pushes below
        if (lane < C) push_u64(to_wtot + kWtotStride * (uint32_t)b, wv, to_data + 8u * (uint32_t)b);
        if (warp == 0) {
            bool alive = mbar_wait(bar_data0 + 8u * (uint32_t)b, ph, a.ctl, limit_ns);
            if (tid == 0 && alive) mbar_arrive_expect(bar_data0 + 8u * (uint32_t)b, data_bytes);  // re-arm for r + 2
            if (!KPP) {
                // minmax: the largest packed (D^2, key) of the cluster
                uint32_t next;
                if (r == 0) {
                    next = __ldg(a.keys + below(u, (uint64_t)n));
                } else {
                    const unsigned long long m = warp_max_u64(cta_values<false>(sh, b, lanes));
                    next = 0xFFFFFFu - (uint32_t)(m & 0xFFFFFFull);
                }
                if (lane == 0) sh.key[b] = next;
            } else if (alive) {
                // this CTA's own warp totals are scanned while the CTA totals are formed
                const unsigned long long wtv = lane < kClWarps ? sh.wtot[b][rank][lane] : 0ull;
                const unsigned long long xw = warp_incl_scan_u64<4>(wtv, lane);
                const unsigned long long ct = cta_values<true>(sh, b, lanes);
                const unsigned long long x = warp_incl_scan_u64<4>(lane < C ? ct : 0ull, lane);
                const unsigned long long t = below(u, __shfl_sync(kFull, x, C - 1));
                int g = __ffs(__ballot_sync(kFull, lane < C && x > t)) - 1;
                g = g < 0 ? 0 : g;  // t < the total whenever it is positive
                if (g == (int)rank) {
                    // the warp of this CTA, then its thread, then the thread's colour
                    const unsigned long long r1 = t - (__shfl_sync(kFull, x, g) - __shfl_sync(kFull, ct, g));
                    int ws = __ffs(__ballot_sync(kFull, lane < kClWarps && xw > r1)) - 1;
                    ws = ws < 0 ? 0 : ws;
                    const unsigned long long resid = r1 - (__shfl_sync(kFull, xw, ws) - __shfl_sync(kFull, wtv, ws));
                    const unsigned long long s2 = sh.tpre[ws * 32 + lane];
                    int l2 = __ffs(__ballot_sync(kFull, s2 > resid)) - 1;
                    l2 = l2 < 0 ? 0 : l2;
                    const unsigned long long prior = __shfl_sync(kFull, s2, l2 > 0 ? l2 - 1 : 0);
                    const unsigned long long r2 = resid - (l2 > 0 ? prior : 0ull);
                    const int ts = ws * 32 + l2;
                    const int tcnt = base + (ts < rem ? 1 : 0);
                    const unsigned long long pv = lane < tcnt ? s_pre[ts * kEps + lane] : ~0ull;
                    int l3 = __ffs(__ballot_sync(kFull, pv > r2)) - 1;
                    l3 = l3 < 0 ? 0 : l3;
                    const uint32_t kk = lane == l3 ? s_key[ts * kEps + lane] : 0u;
                    const uint32_t nk = __shfl_sync(kFull, kk, l3);
                    if (lane < C) push_u32(to_key + 4u * (uint32_t)b, nk, to_kbar + 8u * (uint32_t)b);
                }
                alive = mbar_wait(bar_key0 + 8u * (uint32_t)b, ph, a.ctl, limit_ns);
                if (tid == 0 && alive) mbar_arrive_expect(bar_key0 + 8u * (uint32_t)b, (uint32_t)sizeof(uint32_t));
            }
            if (!alive && lane == 0) sh.dead = 1;
        }
        __syncthreads();
        if (sh.dead) break;  // the same for the whole CTA
        ckey = sh.key[b];
        cnorm = key_norm2(ckey);
        if (rank == 0 && tid == 0) key_to_centre(a.centers + 3 * r, ckey);
    }
}

template <bool KPP>
__device__ __forceinline__ void cluster_dispatch(const ClusterArgs &a, ClusterShared &sh, uint32_t *s_key,
                                                 uint32_t *s_aux, unsigned long long *s_pre, int64_t lo, int cnt, int C,
                                                 uint32_t rank, int64_t n)
{
#define KQ_CL_CASE(E)                                                    \
    case E: cluster_rounds<E, KPP>(a, sh, s_key, s_aux, s_pre, lo, cnt, C, rank, n); \
        break;
    switch ((cnt + kClBlock - 1) / kClBlock) {
    case 0:
        KQ_CL_CASE(1)
        KQ_CL_CASE(2)
        KQ_CL_CASE(3)
        KQ_CL_CASE(4)
        KQ_CL_CASE(5)
        KQ_CL_CASE(6)
        KQ_CL_CASE(7)
        KQ_CL_CASE(8)
        KQ_CL_CASE(9)
        KQ_CL_CASE(10)
        KQ_CL_CASE(11)
        KQ_CL_CASE(12)
        KQ_CL_CASE(13)
        KQ_CL_CASE(14)
        KQ_CL_CASE(15)
        KQ_CL_CASE(16)
        KQ_CL_CASE(17)
        KQ_CL_CASE(18)
        KQ_CL_CASE(19)
        KQ_CL_CASE(20)
        KQ_CL_CASE(21)
    default: cluster_rounds<kClElems, KPP>(a, sh, s_key, s_aux, s_pre, lo, cnt, C, rank, n); break;
    }
#undef KQ_CL_CASE
}

__global__ void __launch_bounds__(kClBlock, 1) seed_far_cluster(ClusterArgs a)
{
    __shared__ ClusterShared sh;
    extern __shared__ unsigned long long cl_smem[];  // running sums, keys, weights (or 0xFFFFFF - key): kClSlots each
    unsigned long long *s_pre = cl_smem;
    uint32_t *s_key = reinterpret_cast<uint32_t *>(cl_smem + kClSlots);
    uint32_t *s_aux = s_key + kClSlots;
    const int64_t n = *a.n_unique;
    const int C = a.ctas;
    // this kernel serves K < N' <= C * kClPer; seed_far serves larger N'
    if (n <= a.K || n > (int64_t)C * kClPer) return;
    const uint32_t rank = cluster_rank();
    const int64_t cbase = n / C, crem = n % C;
    const int64_t lo = (int64_t)rank * cbase + ((int64_t)rank < crem ? (int64_t)rank : crem);
    const int cnt = (int)(cbase + ((int64_t)rank < crem ? 1 : 0));
    if (a.mode == 0) cluster_dispatch<true>(a, sh, s_key, s_aux, s_pre, lo, cnt, C, rank, n);
    else cluster_dispatch<false>(a, sh, s_key, s_aux, s_pre, lo, cnt, C, rank, n);
    // no CTA leaves while another may still push into its shared memory
    cluster_sync_all();
}

// ---------------------------------------------------------------- chunked counts (VAR, DEN)
__device__ __forceinline__ int64_t chunk_len(int64_t n) { return (n + kSeedChunks - 1) / kSeedChunks; }

// mode 0 (VAR): per chunk, counts of each value of each channel; exact moments.
// mode 1 (DEN): per chunk, counts per cell; pixel weight and colour count per cell.
__global__ void __launch_bounds__(kChunkBlock) seed_chunk_counts(const uint32_t *keys, const uint32_t *w,
                                                                 const int32_t *n_unique, int K, int mode,
                                                                 uint32_t *chunk_cnt, uint32_t *gcnt,
                                                                 unsigned long long *cell_w, Ctl *ctl)
{
    __shared__ uint32_t s_cnt[3 * 256];
    __shared__ unsigned long long s_w[kDenCells];
    __shared__ unsigned long long s_red[kChunkBlock / 32];
    const int64_t n = *n_unique;
    if (n <= K) return;
    const int c = blockIdx.x;
    const int64_t len = chunk_len(n);
    const int64_t lo = (int64_t)c * len < n ? (int64_t)c * len : n;
    const int64_t hi = lo + len < n ? lo + len : n;
    for (int i = threadIdx.x; i < 3 * 256; i += kChunkBlock) s_cnt[i] = 0u;
    for (int i = threadIdx.x; i < kDenCells; i += kChunkBlock) s_w[i] = 0ull;
    __syncthreads();
    unsigned long long mw = 0, m1[3] = {0, 0, 0}, m2[3] = {0, 0, 0};
    for (int64_t i = lo + threadIdx.x; i < hi; i += kChunkBlock) {
        const uint32_t key = keys[i];
        const unsigned long long wi = w[i];
        if (mode == 0) {
            const uint32_t x[3] = {key_r(key), key_g(key), key_b(key)};
            mw += wi;
            for (int ch = 0; ch < 3; ++ch) {
                atomicAdd(&s_cnt[ch * 256 + x[ch]], 1u);
                m1[ch] += wi * x[ch];
                m2[ch] += wi * x[ch] * x[ch];
            }
        } else {
            const int cell = den_cell(key);
            atomicAdd(&s_cnt[cell], 1u);
            atomicAdd(&s_w[cell], wi);
        }
    }
    __syncthreads();
    const int width = mode == 0 ? 3 * 256 : kDenCells;
    for (int i = threadIdx.x; i < width; i += kChunkBlock) {
        chunk_cnt[(size_t)c * width + i] = s_cnt[i];
        if (s_cnt[i]) atomicAdd(&gcnt[i], s_cnt[i]);
        if (mode == 1 && s_w[i]) atomicAdd(&cell_w[i], s_w[i]);
    }
    if (mode == 0) {
        unsigned long long t = block_sum_u64<kChunkBlock>(mw, s_red);
        if (threadIdx.x == 0 && t) atomicAdd(&ctl->var_w, t);
        for (int ch = 0; ch < 3; ++ch) {
            t = block_sum_u64<kChunkBlock>(m1[ch], s_red);
            if (threadIdx.x == 0 && t) atomicAdd(&ctl->var_s1[ch], t);
            t = block_sum_u64<kChunkBlock>(m2[ch], s_red);
            if (threadIdx.x == 0 && t) atomicAdd(&ctl->var_s2[ch], t);
        }
    }
}

// ---------------------------------------------------------------- VAR
__global__ void seed_var_pick(const uint32_t *keys, const int32_t *n_unique, int K, const uint32_t *chunk_cnt,
                              const uint32_t *gcnt, const Ctl *ctl, double *centers)
{
    const int64_t n = *n_unique;
    if (n <= K) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= K) return;
    const int ch = var_channel(ctl->var_w, ctl->var_s1, ctl->var_s2);
    var_pick_warp(keys, n, K, warp, ch, chunk_cnt, kSeedChunks, gcnt, centers);
}

// ---------------------------------------------------------------- DEN
// Seats in proportion to each cell's pixel count by largest remainder (ties to
// the lower cell); a cell whose share exceeds its colour count is fixed at that
// count and the remaining seats are shared again among the other cells.
__global__ void seed_den_quota(const int32_t *n_unique, int K, const uint32_t *celln_in,
                               const unsigned long long *cellw, int *quota_out)
{
    const int64_t n = *n_unique;
    if (n <= K || threadIdx.x != 0) return;
    den_quota(K, celln_in, cellw, quota_out);
}

// One block per cell: a uniform draw without replacement among the cell's
// colours (stream 16 + cell), then one warp per pick locates the colour.
__global__ void seed_den_pick(const uint32_t *keys, const int32_t *n_unique, int K, uint64_t seed,
                              const uint32_t *chunk_cnt, const uint32_t *celln, const int *quota, double *centers)
{
    __shared__ uint32_t s_pos1[1024], s_val[1024], s_pick[kMaxK];
    const int64_t n = *n_unique;
    if (n <= K) return;
    const int cell = blockIdx.x;
    const int q = quota[cell];
    if (q == 0) return;
    const int off = quota[kDenCells + cell];
    FyMap m{s_pos1, s_val, 1023u};
    clear_map(s_pos1, 1024);
    __syncthreads();
    if (threadIdx.x == 0) fisher_yates(celln[cell], (uint32_t)q, seed, 16u + (uint32_t)cell, m, s_pick);
    __syncthreads();
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < q; j += nw) {
        const int64_t idx = warp_locate(keys, n, chunk_cnt, kSeedChunks, kDenCells, cell, s_pick[j], 1, 0);
        if ((threadIdx.x & 31) == 0) key_to_centre(centers + 3 * (off + j), keys[idx]);
    }
}

// ---------------------------------------------------------------- LBG
__global__ void seed_lbg_start(const int32_t *n_unique, int K, const Ctl *ctl, double *centers)
{
    const int64_t n = *n_unique;
    if (n <= K || threadIdx.x != 0) return;
    const double W = (double)ctl->var_w;
    for (int ch = 0; ch < 3; ++ch) centers[ch] = (double)ctl->var_s1[ch] / W;
}

// Per-cluster S (3), W and Q = sum w |x|^2 of the current labels.
__global__ void seed_lbg_cluster_sums(const uint32_t *keys, const uint32_t *w, const int32_t *n_unique, int K,
                                      const uint8_t *labels, unsigned long long *cs)
{
    const int64_t n = *n_unique;
    if (n <= K) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = keys[i];
        const unsigned long long wi = w[i];
        const unsigned long long r = key_r(key), g = key_g(key), bb = key_b(key);
        unsigned long long *c = cs + 5 * labels[i];
        atomicAdd(c + 0, wi * r);
        atomicAdd(c + 1, wi * g);
        atomicAdd(c + 2, wi * bb);
        atomicAdd(c + 3, wi);
        atomicAdd(c + 4, wi * (r * r + g * g + bb * bb));
    }
}

// Split round: c_j - eps stays at j, c_j + eps goes to m + q (q-th chosen, in
// ascending j).  All clusters split when 2m <= K; otherwise the K - m clusters
// of largest SSE (ties to the lower index).
__global__ void seed_lbg_split(const int32_t *n_unique, int K, int m, double eps,
                               const unsigned long long *cs, double *centers)
{
    const int64_t n = *n_unique;
    if (n <= K || threadIdx.x != 0) return;
    lbg_split(K, m, eps, cs, centers);
}

// ---------------------------------------------------------------- WU
__global__ void seed_wu_acc(const uint32_t *keys, const uint32_t *w, const int32_t *n_unique, int K,
                            unsigned long long *cell)
{
    const int64_t n = *n_unique;
    if (n <= K) return;
    wu_accumulate(keys, w, n, cell, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Cumulative moments on the whole grid: step 0 copies the cells, steps 1-3 sum lines.
__global__ void seed_wu_cum(const int32_t *n_unique, int K, const unsigned long long *cell, unsigned long long *cum,
                            int step)
{
    const int64_t n = *n_unique;
    if (n <= K) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    if (step == 0) wu_cum_copy(cell, cum, t, nt);
    else wu_cum_lines(cum, step, t, nt);
}

__global__ void __launch_bounds__(1024) seed_wu_split(const int32_t *n_unique, int K, const unsigned long long *cum,
                                                      double *centers)
{
    __shared__ WuShared sh;
    const int64_t n = *n_unique;
    if (n <= K) return;
    wu_split_block(cum, K, centers, sh);
}

constexpr size_t kClSmem = (sizeof(unsigned long long) + 2 * sizeof(uint32_t)) * (size_t)kClSlots;  // sums, keys, aux

// Largest cluster (16, else 8) of seed_far_cluster this device can run, or 0.
int far_cluster_size()
{
    static int cached[64];
    static bool done[64];
    const int dev = device_info().device;
    if (done[dev]) return cached[dev];
    int best = 0;
    if (cudaFuncSetAttribute((const void *)seed_far_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kClSmem) == cudaSuccess &&
        cudaFuncSetAttribute((const void *)seed_far_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
        for (int c : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(kClBlock);
            cfg.dynamicSmemBytes = kClSmem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = c;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)seed_far_cluster, &cfg) == cudaSuccess &&
                clusters >= 1) {
                best = c;
                break;
            }
        }
    }
    cudaGetLastError();  // a refused size is not an error of this call
    cached[dev] = best;
    done[dev] = true;
    return best;
}

template <typename KFn>
int set_smem(KFn kernel, size_t bytes)
{
    return cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
                   cudaSuccess
               ? 0
               : -1;
}

}  // namespace

int launch_seed(const uint32_t *keys, const uint32_t *w, const int32_t *n_unique, int K, int scheme, uint64_t seed,
                const kq_seed_params &p, double *centers, void *ws, const Layout &L, cudaStream_t s)
{
    Ctl *ctl = at<Ctl>(ws, L.ctl);
    seed_all_unique<<<1, 256, 0, s>>>(keys, n_unique, K, centers);
    uint32_t *chunk_cnt = at<uint32_t>(ws, L.s_chunk);
    uint32_t *gcnt = at<uint32_t>(ws, L.s_gcnt);
    unsigned long long *cellw = reinterpret_cast<unsigned long long *>(gcnt + 3 * 256);
    switch (scheme) {
    case KQ_INIT_FGY: {
        const size_t smem = sizeof(uint32_t) * (2 * kMapSlots + kMaxK);
        if (set_smem(seed_fgy, smem)) return KQ_ECUDA;
        seed_fgy<<<1, 32, smem, s>>>(keys, n_unique, K, seed, centers);
        break;
    }
    case KQ_INIT_SFF: {
        const size_t smem = sizeof(uint32_t) * (2 * kMapSlots + 2 * kSffMax);
        if (set_smem(seed_sff, smem)) return KQ_ECUDA;
        int s0 = (int)ceil(2.0 * K * log((double)K));
        if (s0 < K) s0 = K;
        seed_sff<<<1, kSffBlock, smem, s>>>(keys, n_unique, K, seed, s0, centers);
        break;
    }
    case KQ_INIT_KPP:
    case KQ_INIT_MMX: {
        const DeviceInfo di = device_info();
        const int ctas = far_cluster_size();
        if (ctas > 0) {
            ClusterArgs ca;
            ca.keys = keys;
            ca.w = w;
            ca.n_unique = n_unique;
            ca.K = K;
            ca.mode = scheme == KQ_INIT_KPP ? 0 : 1;
            ca.ctas = ctas;
            ca.seed = seed;
            ca.centers = centers;
            ca.ctl = ctl;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(ctas);
            cfg.blockDim = dim3(kClBlock);
            cfg.dynamicSmemBytes = kClSmem;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = ctas;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaLaunchKernelEx(&cfg, seed_far_cluster, ca) != cudaSuccess) return KQ_ECUDA;
        }
        if (set_smem(seed_far, kFarSmem)) return KQ_ECUDA;
        const int per_sm = max_coresident((const void *)seed_far, kFarBlock, kFarSmem);
        if (per_sm < 1) return KQ_ECUDA;
        int grid = di.sms * per_sm;
        if (grid > kMaxGrid) grid = kMaxGrid;
        FarArgs a;
        a.keys = keys;
        a.w = w;
        a.n_unique = n_unique;
        a.K = K;
        a.mode = scheme == KQ_INIT_KPP ? 0 : 1;
        a.seed = seed;
        a.max_unique = L.max_unique;
        a.centers = centers;
        a.ctl = ctl;
        a.d2 = at<uint32_t>(ws, L.s_d2);
        a.part = at<unsigned long long>(ws, L.s_part);
        a.gpart = at<unsigned long long>(ws, L.s_gpart);
        a.gpart_cap = gpart_cap(L.max_unique);
        a.slot = at<unsigned long long>(ws, L.s_slot);
        a.cluster_cap = (int64_t)ctas * kClPer;
        if (cudaMemsetAsync(&ctl->bar_count, 0, sizeof(uint32_t), s) != cudaSuccess) return KQ_ECUDA;
        void *args[] = {&a};
        if (cudaLaunchCooperativeKernel((const void *)seed_far, dim3(grid), dim3(kFarBlock), args, kFarSmem, s) !=
            cudaSuccess)
            return KQ_ECUDA;
        break;
    }
    case KQ_INIT_VAR: {
        if (cudaMemsetAsync(gcnt, 0, sizeof(uint32_t) * 3 * 256, s) != cudaSuccess) return KQ_ECUDA;
        if (cudaMemsetAsync(&ctl->var_w, 0, sizeof(unsigned long long) * 7, s) != cudaSuccess) return KQ_ECUDA;
        seed_chunk_counts<<<kSeedChunks, kChunkBlock, 0, s>>>(keys, w, n_unique, K, 0, chunk_cnt, gcnt, cellw, ctl);
        seed_var_pick<<<(K * 32 + 255) / 256, 256, 0, s>>>(keys, n_unique, K, chunk_cnt, gcnt, ctl, centers);
        break;
    }
    case KQ_INIT_DEN: {
        int *quota = at<int>(ws, L.s_misc);
        if (cudaMemsetAsync(gcnt, 0, sizeof(uint32_t) * 3 * 256 + sizeof(unsigned long long) * kDenCells, s) !=
            cudaSuccess)
            return KQ_ECUDA;
        seed_chunk_counts<<<kSeedChunks, kChunkBlock, 0, s>>>(keys, w, n_unique, K, 1, chunk_cnt, gcnt, cellw, ctl);
        seed_den_quota<<<1, 32, 0, s>>>(n_unique, K, gcnt, cellw, quota);
        seed_den_pick<<<kDenCells, 256, 0, s>>>(keys, n_unique, K, seed, chunk_cnt, gcnt, quota, centers);
        break;
    }
    case KQ_INIT_WU: {
        unsigned long long *cell = at<unsigned long long>(ws, L.s_wu);
        unsigned long long *cum = cell + 5 * (size_t)kWuCells;
        if (cudaMemsetAsync(cell, 0, sizeof(unsigned long long) * 5 * (size_t)kWuCells, s) != cudaSuccess)
            return KQ_ECUDA;
        const DeviceInfo di = device_info();
        seed_wu_acc<<<di.sms * 4, 256, 0, s>>>(keys, w, n_unique, K, cell);
        seed_wu_cum<<<(5 * kWuCum + 255) / 256, 256, 0, s>>>(n_unique, K, cell, cum, 0);
        for (int step = 1; step <= 3; ++step)
            seed_wu_cum<<<(5 * 33 * 33 + 127) / 128, 128, 0, s>>>(n_unique, K, cell, cum, step);
        seed_wu_split<<<1, 1024, 0, s>>>(n_unique, K, cum, centers);
        break;
    }
    case KQ_INIT_LBG: {
        if (cudaMemsetAsync(gcnt, 0, sizeof(uint32_t) * 3 * 256, s) != cudaSuccess) return KQ_ECUDA;
        if (cudaMemsetAsync(&ctl->var_w, 0, sizeof(unsigned long long) * 7, s) != cudaSuccess) return KQ_ECUDA;
        seed_chunk_counts<<<kSeedChunks, kChunkBlock, 0, s>>>(keys, w, n_unique, K, 0, chunk_cnt, gcnt, cellw, ctl);
        seed_lbg_start<<<1, 32, 0, s>>>(n_unique, K, ctl, centers);
        unsigned long long *cs = at<unsigned long long>(ws, L.s_misc);
        uint8_t *labels = at<uint8_t>(ws, L.s_labels);
        uint8_t *pal = at<uint8_t>(ws, L.s_misc) + 32768;
        const DeviceInfo di = device_info();
        int m = 1;
        while (m < K) {
            const int split = (2 * m <= K) ? m : K - m;
            if (split < m) {
                if (cudaMemsetAsync(cs, 0, sizeof(unsigned long long) * 5 * kMaxK, s) != cudaSuccess) return KQ_ECUDA;
                seed_lbg_cluster_sums<<<di.sms * 4, 256, 0, s>>>(keys, w, n_unique, K, labels, cs);
            }
            seed_lbg_split<<<1, 32, 0, s>>>(n_unique, K, m, p.lbg_eps, cs, centers);
            m += split;
            int st = launch_lloyd(keys, w, n_unique, m, centers, p.conv_eps, p.max_iter, 0u, labels, pal, nullptr,
                                  nullptr, ws, L, s, K);
            if (st != KQ_OK) return st;
        }
        break;
    }
    default:
        return KQ_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

}  // namespace kq
