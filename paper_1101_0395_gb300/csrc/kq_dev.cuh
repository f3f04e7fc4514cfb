// kq_dev.cuh -- internal declarations shared by the CUDA translation units of libkq.
//
// Workspace layout, the device status word, the bounded grid barrier used by the
// cooperative (persistent) kernels, the counter-based random numbers and the one
// FP32 distance formula that every assignment path uses.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/kq.h"

namespace kq {

// ---------------------------------------------------------------- constants
constexpr int kMaxK = 256;                 // palette indices are uint8_t
constexpr int kKeyBits = 24;               // (R << 16) | (G << 8) | B
constexpr int64_t kKeySpace = int64_t(1) << kKeyBits;
constexpr int kBitWords = 1 << (kKeyBits - 5);   // presence bitmap, one bit per colour
constexpr int kHistChunkWords = 256;             // bitmap words per compaction block (8192 colours)
constexpr int kHistChunks = kBitWords / kHistChunkWords;  // 2048
constexpr int kMaxGrid = 4096;             // upper bound on persistent grid sizes
constexpr int kSeedChunks = 512;           // chunks of the unique list for VAR / DEN lookups
constexpr int kDenCells = 64;              // 4 levels per channel
constexpr int kMapCells = 32 * 32 * 32;    // kq_map's cells: 8^3 colours each
constexpr uint64_t kWaitNs = 4000000000ull;  // device-side wait limit (4 s)
constexpr int kWuCells = 32 * 32 * 32;     // Wu's grid: 5 bits per channel
constexpr int kWuCum = 33 * 33 * 33;       // cumulative moments with a zero border
constexpr size_t kWuBytes = sizeof(unsigned long long) * 5 * ((size_t)kWuCells + kWuCum);

// ---------------------------------------------------------------- control block
// Lives at the start of the workspace.  Fields touched by spinning blocks sit on
// their own 128-byte lines.
struct Ctl {
    int32_t status;            // first device-side error (kq_status), 0 = OK
    uint32_t abort;            // set when a wait timed out: every wait then gives up
    int64_t n_unique_true;     // N' before clamping to the caller's capacity
    unsigned long long ndc;    // distance calculations of the current kq_lloyd call
    uint32_t wait_limit_us;    // device-side wait limit of the following launches (0: kWaitNs)
    uint32_t missing;          // arrivals every wait expects beyond the launched blocks (test hook; 0)
    uint32_t pad0[24];
    uint32_t bar_count;        // grid barrier: arrivals since the launch (cleared before each launch)
    uint32_t pad1[31];
    uint32_t bar_gen;          // unused
    uint32_t pad2[31];
    // seeding scratch scalars
    unsigned long long var_w;  // sum of weights
    unsigned long long var_s1[3];
    unsigned long long var_s2[3];
    unsigned long long map_ndc;  // distance calculations of the last kq_map (candidates over all pixels)
    uint32_t pad3[16];
};
static_assert(sizeof(Ctl) <= 4096, "control block must fit its region");
static_assert(offsetof(Ctl, bar_count) == 128, "the barrier counter has its own 128-byte line");

// ---------------------------------------------------------------- workspace layout
struct Layout {
    size_t ctl, hist_cnt, hist_bits, hist_chunk, m_desc, m_list;
    size_t l_sums, l_sse, l_rows;
    size_t s_d2, s_part, s_slot, s_chunk, s_gcnt, s_misc, s_labels, s_centers, s_wu, s_gpart;
    size_t total;
    int64_t max_unique;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Entries per buffer of the seeding group sums: a sum per 32 colours of every block
// slice, for any grid of up to kMaxGrid blocks (sum over blocks of ceil(slice / 32)).
__host__ __device__ inline int64_t gpart_cap(int64_t max_unique) { return max_unique / 32 + 2 * (int64_t)kMaxGrid; }

// Fixed-size regions first, then the three that grow with the number of unique
// colours (8 + 1 + 0.5 bytes per colour), so that the layout of a workspace can be
// recovered from its size alone.
__host__ __device__ inline Layout layout_for(int64_t max_unique)
{
    Layout L{};
    int64_t mu = max_unique < kKeySpace ? max_unique : kKeySpace;
    if (mu < 1) mu = 1;
    L.max_unique = mu;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    L.ctl = take(4096);
    L.hist_cnt = take(sizeof(uint32_t) * (size_t)kKeySpace);
    L.hist_bits = take(sizeof(uint32_t) * (size_t)kBitWords);
    L.hist_chunk = take(sizeof(uint32_t) * 2 * (size_t)kHistChunks);  // totals, then bases
    L.m_desc = take(sizeof(unsigned long long) * (size_t)kMapCells);
    L.m_list = take((size_t)kMapCells * kMaxK);
    L.l_sums = take(sizeof(unsigned long long) * 3 * kMaxK * 4);
    L.l_sse = take(sizeof(double) * 2 * kMaxGrid);
    L.l_rows = take(sizeof(uint32_t) * kMaxK * kMaxK);
    L.s_part = take(sizeof(unsigned long long) * 2 * kMaxGrid);
    L.s_slot = take(sizeof(unsigned long long) * kMaxK);
    L.s_chunk = take(sizeof(uint32_t) * (size_t)kSeedChunks * 3 * 256);
    L.s_gcnt = take(sizeof(uint32_t) * 3 * 256 + sizeof(unsigned long long) * kDenCells * 2);
    L.s_misc = take(65536);
    L.s_centers = take(sizeof(double) * kMaxK * 3);
    L.s_wu = take(kWuBytes);
    L.s_d2 = take(2 * sizeof(uint32_t) * (size_t)mu);
    L.s_labels = take((size_t)mu);
    L.s_gpart = take(sizeof(unsigned long long) * 2 * (size_t)gpart_cap(mu));
    L.total = o;
    return L;
}

// Largest layout that fits in `bytes` (max_unique = 0 when even one colour does not fit).
inline Layout layout_from_bytes(size_t bytes)
{
    Layout base = layout_for(1);
    if (bytes < base.total) {
        Layout none{};
        none.max_unique = 0;
        return none;
    }
    int64_t mu = (int64_t)((bytes - base.s_d2) * 2 / 19);
    if (mu > kKeySpace) mu = kKeySpace;
    if (mu < 1) mu = 1;
    Layout L = layout_for(mu);
    while (L.total > bytes && mu > 1) {  // alignment padding: step down until it fits
        mu = mu > 256 ? mu - 256 : 1;
        L = layout_for(mu);
    }
    return L;
}

template <typename T>
__host__ __device__ inline T *at(void *ws, size_t off) { return reinterpret_cast<T *>(static_cast<char *>(ws) + off); }

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ void fail(Ctl *ctl, int code) { atomicCAS(&ctl->status, 0, code); }

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_add_gpu(uint32_t *p, uint32_t v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The wait limit of a launch (read once at its start).
__device__ __forceinline__ uint64_t wait_limit_ns(const Ctl *ctl)
{
    const uint32_t us = *(volatile const uint32_t *)&ctl->wait_limit_us;
    return us ? (uint64_t)us * 1000ull : kWaitNs;
}

// Barrier over `nblocks` blocks of a cooperative launch (normally all the blocks
// taking part; more only when the test hook Ctl::missing asks for arrivals that
// never come).  The arrival counter starts at 0 (the launcher clears it on the
// stream before the launch) and only grows: barrier m of the launch is passed once
// it reaches (m + 1) * nblocks, which the caller tracks in `*epoch`.  Thread 0 of
// each block arrives with one release reduction and polls with acquire loads.
// Every wait is bounded: after `limit_ns`, or when another block has given up, it
// records KQ_ETIMEOUT, raises `abort` and returns false; the caller then returns.
__device__ __forceinline__ bool grid_sync(Ctl *ctl, unsigned nblocks, uint32_t *epoch, uint64_t limit_ns)
{
    __shared__ int s_ok;
    *epoch += nblocks;
    const uint32_t target = *epoch;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        red_release_add_gpu(&ctl->bar_count, 1u);
        uint64_t t0 = 0;
        for (uint32_t spin = 0; ld_acquire_gpu(&ctl->bar_count) < target; ++spin) {
            if ((spin & 63u) == 63u) {
                if (ld_acquire_gpu(&ctl->abort)) { ok = 0; break; }
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > limit_ns) {
                    fail(ctl, KQ_ETIMEOUT);
                    atomicExch(&ctl->abort, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): draw `ctr` of stream `stream`
// is output number stream * 2^32 + ctr + 1 of the generator seeded with `seed`.
__host__ __device__ __forceinline__ uint64_t rand64(uint64_t seed, uint32_t stream, uint32_t ctr)
{
    uint64_t n = ((uint64_t)stream << 32) + (uint64_t)ctr + 1ull;
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Integer in [0, m): the high half of the 128-bit product.
__device__ __forceinline__ uint64_t below(uint64_t u, uint64_t m) { return __umul64hi(u, m); }

__device__ __forceinline__ uint32_t key_r(uint32_t k) { return k >> 16; }
__device__ __forceinline__ uint32_t key_g(uint32_t k) { return (k >> 8) & 255u; }
__device__ __forceinline__ uint32_t key_b(uint32_t k) { return k & 255u; }

// Squared distance in FP32: differences first, then squares summed by two fused
// multiply-adds, every operation rounded to nearest.  The pruned scan, the full
// search and the centre-to-centre table all call this one function, so equal
// inputs give bitwise-equal distances everywhere.
__device__ __forceinline__ float dist3(float x, float y, float z, float cx, float cy, float cz)
{
    float dx = __fsub_rn(x, cx), dy = __fsub_rn(y, cy), dz = __fsub_rn(z, cz);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Exact integer squared distance between two colours: with the key bytes as a
// vector, |a - b|^2 = |a|^2 + |b|^2 - 2 a.b, each dot product one byte-wise dp4a.
__device__ __forceinline__ uint32_t key_norm2(uint32_t a) { return __dp4a(a, a, 0u); }
__device__ __forceinline__ uint32_t key_dist2n(uint32_t a, uint32_t na, uint32_t b, uint32_t nb)
{
    return na + nb - 2u * __dp4a(a, b, 0u);
}
__device__ __forceinline__ uint32_t key_dist2(uint32_t a, uint32_t b)
{
    return key_dist2n(a, key_norm2(a), b, key_norm2(b));
}

// ---------------------------------------------------------------- block reductions
template <int BLOCK>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *scratch)
{
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < BLOCK / 32; ++i) t += scratch[i];
    return t;  // valid in thread 0
}

// Fixed-order FP64 block sum: a fixed shuffle tree per warp, then warp results
// in warp order.  The same inputs in the same threads give the same bits.
template <int BLOCK>
__device__ __forceinline__ double block_sum_f64(double v, double *scratch)
{
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < BLOCK / 32; ++i) t += scratch[i];
    return t;  // valid in thread 0
}

// Fixed-order FP32 block sum (same tree as block_sum_f64); valid in thread 0.
template <int BLOCK>
__device__ __forceinline__ float block_sum_f32(float v, float *scratch)
{
    for (int o = 16; o; o >>= 1) v = __fadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < BLOCK / 32; ++i) t = __fadd_rn(t, scratch[i]);
    return t;  // valid in thread 0
}

// Block-wide exclusive scan of 32-bit counts; returns this thread's exclusive
// prefix and writes the block total to *total (all threads).
template <int BLOCK>
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *scratch, uint32_t *total)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < BLOCK / 32 ? scratch[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < BLOCK / 32) scratch[lane] = s;
    }
    __syncthreads();
    uint32_t before = warp ? scratch[warp - 1] : 0u;
    *total = scratch[BLOCK / 32 - 1];
    return before + x - v;
}

template <int BLOCK>
__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long v, unsigned long long *scratch,
                                                                  unsigned long long *total)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long s = lane < BLOCK / 32 ? scratch[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < BLOCK / 32) scratch[lane] = s;
    }
    __syncthreads();
    unsigned long long before = warp ? scratch[warp - 1] : 0ull;
    *total = scratch[BLOCK / 32 - 1];
    return before + x - v;
}

// Contiguous slice [lo, hi) of n items for block b of g.
__device__ __forceinline__ void slice_of(int64_t n, int b, int g, int64_t *lo, int64_t *hi)
{
    int64_t per = (n + g - 1) / g;
    int64_t a = (int64_t)b * per;
    *lo = a < n ? a : n;
    int64_t e = a + per;
    *hi = e < n ? e : n;
}

}  // namespace kq

// ---------------------------------------------------------------- host-side launchers
namespace kq {
struct DeviceInfo {
    int device;
    int sms;
};
DeviceInfo device_info();
int max_coresident(const void *kernel, int block, size_t smem);

int launch_histogram(const uint8_t *rgb, int64_t n, uint32_t *keys, uint32_t *weights, int32_t cap, int32_t *n_unique,
                     void *ws, const Layout &L, cudaStream_t s);
int launch_lloyd(const uint32_t *keys, const uint32_t *w, const int32_t *n_unique, int K, double *centers, double eps,
                 int max_iter, uint32_t flags, uint8_t *labels, uint8_t *palette, kq_lloyd_stats *stats,
                 double *sse_hist, void *ws, const Layout &L, cudaStream_t s, int skip_if_n_le);
int launch_seed(const uint32_t *keys, const uint32_t *w, const int32_t *n_unique, int K, int scheme, uint64_t seed,
                const kq_seed_params &p, double *centers, void *ws, const Layout &L, cudaStream_t s);
int launch_histogram_strided(const uint8_t *rgb, int32_t h, int32_t w, int64_t pitch, int32_t stride, uint32_t *keys,
                             uint32_t *weights, int32_t cap, int32_t *n_unique, void *ws, const Layout &L,
                             cudaStream_t s);
int launch_pixel_keys(const uint8_t *rgb, int64_t n, uint32_t *keys, uint32_t *weights, int32_t *n_out,
                      cudaStream_t s);
int launch_map(const uint8_t *rgb, int64_t n, const uint8_t *palette, int K, uint8_t *idx, int64_t *sse_num,
               void *ws, const Layout &L, cudaStream_t s);
int launch_lloyd_points(const unsigned long long *pts, const uint32_t *w, const int32_t *n_unique, int K,
                        double *centers, double eps, int max_iter, uint32_t flags, uint8_t *labels,
                        kq_lloyd_stats *stats, double *sse_hist, void *ws, const Layout &L, cudaStream_t s);
int launch_lab_points(const uint32_t *keys, const int32_t *n_unique, unsigned long long *pts, cudaStream_t s);
int launch_seed_points(const unsigned long long *pts, const int32_t *n_unique, int K, uint64_t seed, double *centers,
                       cudaStream_t s);
int launch_lab_palette(const double *centers, int K, uint8_t *palette, cudaStream_t s);
int launch_map_labels(const uint8_t *rgb, int64_t n, const uint32_t *keys, const int32_t *n_unique,
                      const uint8_t *labels, uint8_t *idx, void *ws, const Layout &L, cudaStream_t s);
}  // namespace kq
