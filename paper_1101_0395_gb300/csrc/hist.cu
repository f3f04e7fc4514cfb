// hist.cu -- unique colours with integer weights (Section 2.2, items 1-2).
//
// The paper finds the unique colours with a chained hash table.  A 24-bit key
// is its own perfect hash, so on the GPU the "table" is a direct array of 2^24
// counters plus a 2^24-bit presence bitmap, both resident in the workspace and
// zero between calls:
//   1. hist_count   streams the packed pixels (three 16-byte loads per 16 pixels),
//                   adds one to cnt[key] and, on the first touch of a colour,
//                   sets its presence bit;
//   2. hist_chunks  counts set bits per 2048-word chunk of the bitmap;
//   3. hist_emit    turns the bitmap into ascending keys: each block offsets its
//                   chunk by the counts before it, scans its words, writes keys
//                   and counts, and zeroes the counters and bits it read.
// Pixels are read once; the tables are touched only at the colours present.
#include "kq_dev.cuh"

namespace kq {
namespace {

constexpr int kCountBlock = 256;
constexpr int kEmitBlock = 256;
static_assert(kHistChunkWords == kEmitBlock * 8, "eight bitmap words per emitting thread");

__device__ __forceinline__ void add_colour(uint32_t *cnt, uint32_t *bits, uint32_t key)
{
    uint32_t old = atomicAdd(cnt + key, 1u);
    if (old == 0u) atomicOr(bits + (key >> 5), 1u << (key & 31u));
}

__device__ __forceinline__ uint32_t key_at(const uint8_t *rgb, int64_t p)
{
    const uint8_t *q = rgb + 3 * p;
    return ((uint32_t)q[0] << 16) | ((uint32_t)q[1] << 8) | (uint32_t)q[2];
}

// Key of pixel i (0..15) of a 48-byte group held as twelve little-endian words.
template <int I>
__device__ __forceinline__ uint32_t group_key(const uint32_t (&w)[12])
{
    constexpr int o = 3 * I, q = o >> 2, r = o & 3;
    const uint32_t lo = w[q];
    const uint32_t hi = (q + 1 < 12) ? w[q + 1] : 0u;
    // result bytes (low to high): B, G, R, 0 -> (R << 16) | (G << 8) | B
    return __byte_perm(lo, hi, (r + 2) | ((r + 1) << 4) | (r << 8)) & 0xFFFFFFu;
}

template <int I>
struct Unroll16 {
    template <typename F>
    __device__ __forceinline__ static void run(const uint32_t (&w)[12], F &&f)
    {
        f(group_key<I>(w));
        Unroll16<I + 1>::run(w, f);
    }
};
template <>
struct Unroll16<16> {
    template <typename F>
    __device__ __forceinline__ static void run(const uint32_t (&)[12], F &&)
    {
    }
};

__global__ void __launch_bounds__(kCountBlock) hist_count(const uint8_t *__restrict__ rgb, int64_t n, int64_t head,
                                                          uint32_t *__restrict__ cnt, uint32_t *__restrict__ bits)
{
    const int64_t tid = (int64_t)blockIdx.x * kCountBlock + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kCountBlock;
    const int64_t ngroups = (n - head) / 16;
    const int64_t tail0 = head + ngroups * 16;
    // scalar head (pixels before the first 16-byte aligned group) and tail
    for (int64_t p = tid; p < head; p += nth) add_colour(cnt, bits, key_at(rgb, p));
    for (int64_t p = tail0 + tid; p < n; p += nth) add_colour(cnt, bits, key_at(rgb, p));
    const uint4 *g = reinterpret_cast<const uint4 *>(rgb + 3 * head);
    for (int64_t gi = tid; gi < ngroups; gi += nth) {
        const uint4 a = __ldcs(g + 3 * gi), b = __ldcs(g + 3 * gi + 1), c = __ldcs(g + 3 * gi + 2);
        const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
        Unroll16<0>::run(w, [&](uint32_t key) { add_colour(cnt, bits, key); });
    }
}

__global__ void __launch_bounds__(kEmitBlock) hist_chunks(const uint32_t *__restrict__ bits, uint32_t *__restrict__ chunk_tot)
{
    __shared__ unsigned long long s_red[kEmitBlock / 32];
    const uint4 *p = reinterpret_cast<const uint4 *>(bits + (size_t)blockIdx.x * kHistChunkWords) + 2 * threadIdx.x;
    const uint4 a = p[0], b = p[1];
    unsigned long long c = __popc(a.x) + __popc(a.y) + __popc(a.z) + __popc(a.w) + __popc(b.x) + __popc(b.y) +
                           __popc(b.z) + __popc(b.w);
    unsigned long long t = block_sum_u64<kEmitBlock>(c, s_red);
    if (threadIdx.x == 0) chunk_tot[blockIdx.x] = (uint32_t)t;
}

__global__ void __launch_bounds__(kEmitBlock) hist_emit(uint32_t *__restrict__ bits, uint32_t *__restrict__ cnt,
                                                        const uint32_t *__restrict__ chunk_tot,
                                                        uint32_t *__restrict__ keys, uint32_t *__restrict__ weights,
                                                        int32_t cap, int32_t *__restrict__ n_unique, Ctl *ctl)
{
    __shared__ uint32_t s_scan[kEmitBlock / 32];
    __shared__ uint32_t s_base;
    const int chunk = blockIdx.x;
    // offset of this chunk = colours in all chunks before it
    if (threadIdx.x < 32) {
        uint32_t s = 0;
        for (int c = threadIdx.x; c < chunk; c += 32) s += chunk_tot[c];
        for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) s_base = s;
    }
    const size_t w0 = (size_t)chunk * kHistChunkWords + (size_t)threadIdx.x * 8;
    uint4 *p = reinterpret_cast<uint4 *>(bits + w0);
    const uint4 a = p[0], b = p[1];
    const uint32_t wv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t pc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) pc += __popc(wv[k]);
    uint32_t tot;
    const uint32_t excl = block_excl_scan_u32<kEmitBlock>(pc, s_scan, &tot);
    __syncthreads();
    int64_t pos = (int64_t)s_base + excl;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        uint32_t m = wv[k];
        const uint32_t kbase = (uint32_t)(w0 + k) << 5;
        while (m) {
            const uint32_t bit = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t key = kbase | bit;
            const uint32_t c = cnt[key];
            cnt[key] = 0u;
            if (pos < cap) {
                keys[pos] = key;
                weights[pos] = c;
            }
            ++pos;
        }
    }
    if (pc) {
        p[0] = make_uint4(0, 0, 0, 0);
        p[1] = make_uint4(0, 0, 0, 0);
    }
    if (chunk == kHistChunks - 1 && threadIdx.x == kEmitBlock - 1) {
        // pos is now the total number of colours
        ctl->n_unique_true = pos;
        *n_unique = (int32_t)(pos < cap ? pos : cap);
        if (pos > cap) fail(ctl, KQ_ECAPACITY);
    }
}

}  // namespace

int launch_histogram(const uint8_t *rgb, int64_t n, uint32_t *keys, uint32_t *weights, int32_t cap, int32_t *n_unique,
                     void *ws, const Layout &L, cudaStream_t s)
{
    uint32_t *cnt = at<uint32_t>(ws, L.hist_cnt);
    uint32_t *bits = at<uint32_t>(ws, L.hist_bits);
    uint32_t *chunk_tot = at<uint32_t>(ws, L.hist_chunk);
    Ctl *ctl = at<Ctl>(ws, L.ctl);
    // first pixel p0 whose byte offset makes rgb + 3 * p0 16-byte aligned
    const uintptr_t mis = reinterpret_cast<uintptr_t>(rgb) & 15u;
    int64_t head = (int64_t)(((16u - mis) * 11u) & 15u);  // 3 * 11 == 1 (mod 16)
    if (head > n) head = n;
    const DeviceInfo di = device_info();
    int64_t groups = (n - head) / 16;
    int64_t want = (groups + kCountBlock - 1) / kCountBlock;
    int grid = (int)(want < (int64_t)di.sms * 8 ? want : (int64_t)di.sms * 8);
    if (grid < 1) grid = 1;
    if (n > 0) hist_count<<<grid, kCountBlock, 0, s>>>(rgb, n, head, cnt, bits);
    hist_chunks<<<kHistChunks, kEmitBlock, 0, s>>>(bits, chunk_tot);
    hist_emit<<<kHistChunks, kEmitBlock, 0, s>>>(bits, cnt, chunk_tot, keys, weights, cap, n_unique, ctl);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

}  // namespace kq
