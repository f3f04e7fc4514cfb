// hist.cu -- unique colours with integer weights (Section 2.2, items 1-2).
//
// The paper finds the unique colours with a chained hash table.  A 24-bit key
// is its own perfect hash, so on the GPU the "table" is a direct array of 2^24
// counters plus a 2^24-bit presence bitmap, both resident in the workspace and
// zero between calls:
//   1. hist_count   streams the packed pixels (three 16-byte loads per 16 pixels),
//                   adds one to cnt[key] and, on the first touch of a colour,
//                   sets its presence bit;
//   2. hist_chunks  counts set bits per 256-word chunk of the bitmap (8192 colours)
//                   and hist_bases turns the counts into each chunk's first output;
//   3. hist_emit    turns the bitmap into ascending keys: each block writes its
//                   chunk's keys and counts by output rank, zeroing the counters
//                   and bits it read.
// Pixels are read once; the tables are touched only at the colours present.
#include "kq_dev.cuh"

namespace kq {
namespace {

constexpr int kCountBlock = 256;
constexpr int kEmitBlock = 256;
static_assert(kHistChunkWords == kEmitBlock, "one bitmap word per emitting thread");
constexpr int kBaseBlock = 1024;
static_assert(kHistChunks == 2 * kBaseBlock, "two chunk totals per scanning thread");

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
        // all sixteen counter updates go out before any returned value is looked at,
        // so they overlap; then the first touches set their presence bits
        uint32_t key[16], old[16];
        int q = 0;
        Unroll16<0>::run(w, [&](uint32_t k) { key[q++] = k; });
#pragma unroll
        for (int i = 0; i < 16; ++i) old[i] = atomicAdd(cnt + key[i], 1u);
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (old[i] == 0u) atomicOr(bits + (key[i] >> 5), 1u << (key[i] & 31u));
    }
}

__global__ void __launch_bounds__(kEmitBlock) hist_chunks(const uint32_t *__restrict__ bits, uint32_t *__restrict__ chunk_tot)
{
    __shared__ unsigned long long s_red[kEmitBlock / 32];
    const unsigned long long c = __popc(bits[(size_t)blockIdx.x * kHistChunkWords + threadIdx.x]);
    const unsigned long long t = block_sum_u64<kEmitBlock>(c, s_red);
    if (threadIdx.x == 0) chunk_tot[blockIdx.x] = (uint32_t)t;
}

// Exclusive prefix of the chunk totals (each chunk's first output position), the
// number of colours, and the capacity check.
__global__ void __launch_bounds__(kBaseBlock) hist_bases(const uint32_t *__restrict__ chunk_tot,
                                                         uint32_t *__restrict__ chunk_base, int32_t cap,
                                                         int32_t *__restrict__ n_unique, Ctl *ctl)
{
    __shared__ uint32_t s_scan[kBaseBlock / 32];
    const uint32_t a = chunk_tot[2 * threadIdx.x], b = chunk_tot[2 * threadIdx.x + 1];
    uint32_t tot;
    const uint32_t ex = block_excl_scan_u32<kBaseBlock>(a + b, s_scan, &tot);
    chunk_base[2 * threadIdx.x] = ex;
    chunk_base[2 * threadIdx.x + 1] = ex + a;
    if (threadIdx.x == 0) {
        ctl->n_unique_true = tot;
        *n_unique = (int32_t)(tot < (uint32_t)cap ? tot : (uint32_t)cap);
        if (tot > (uint32_t)cap) fail(ctl, KQ_ECAPACITY);
    }
}

// Position of the k-th (0-based) set bit of v, by halving with population counts.
__device__ __forceinline__ uint32_t select_bit(uint32_t v, int k)
{
    uint32_t pos = 0;
    int c = __popc(v & 0xFFFFu);
    if (k >= c) { k -= c; v >>= 16; pos += 16; }
    c = __popc(v & 0xFFu);
    if (k >= c) { k -= c; v >>= 8; pos += 8; }
    c = __popc(v & 0xFu);
    if (k >= c) { k -= c; v >>= 4; pos += 4; }
    c = __popc(v & 0x3u);
    if (k >= c) { k -= c; v >>= 2; pos += 2; }
    if (k >= (int)(v & 1u)) pos += 1;
    return pos;
}

// Output by rank: a chunk's colours occupy positions [base, base + total) of the
// result; thread t writes positions base + t, base + t + 256, ...  The word holding
// the r-th set bit of the chunk is found by binary search over the per-word prefix
// counts, the bit itself by select_bit.  Threads get equal shares however unevenly
// the colours fall in the key space, four counter reads are in flight per thread,
// and the writes of keys and weights are coalesced.
__global__ void __launch_bounds__(kEmitBlock) hist_emit(uint32_t *__restrict__ bits, uint32_t *__restrict__ cnt,
                                                        const uint32_t *__restrict__ chunk_base,
                                                        uint32_t *__restrict__ keys, uint32_t *__restrict__ weights,
                                                        int32_t cap)
{
    __shared__ uint32_t s_pre[kHistChunkWords];  // exclusive prefix of set bits per word
    __shared__ uint32_t s_word[kHistChunkWords];
    __shared__ uint32_t s_scan[kEmitBlock / 32];
    const int chunk = blockIdx.x;
    const size_t wi = (size_t)chunk * kHistChunkWords + threadIdx.x;
    const uint32_t v = bits[wi];
    uint32_t tot;
    const uint32_t ex = block_excl_scan_u32<kEmitBlock>(__popc(v), s_scan, &tot);
    s_word[threadIdx.x] = v;
    s_pre[threadIdx.x] = ex;
    if (v) bits[wi] = 0u;
    __syncthreads();
    const int64_t base = chunk_base[chunk];
    constexpr int kBatch = 4;
    for (uint32_t r0 = threadIdx.x; r0 < tot; r0 += kEmitBlock * kBatch) {
        uint32_t key[kBatch], c[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const uint32_t r = r0 + (uint32_t)j * kEmitBlock;
            key[j] = 0xFFFFFFFFu;
            if (r < tot) {
                int lo = 0, hi = kHistChunkWords - 1;  // last word whose prefix is <= r
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_pre[mid] <= r) lo = mid;
                    else hi = mid - 1;
                }
                key[j] = ((uint32_t)(chunk * kHistChunkWords + lo) << 5) | select_bit(s_word[lo], (int)(r - s_pre[lo]));
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) c[j] = key[j] != 0xFFFFFFFFu ? cnt[key[j]] : 0u;
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            if (key[j] == 0xFFFFFFFFu) continue;
            cnt[key[j]] = 0u;
            const int64_t pos = base + r0 + (uint32_t)j * kEmitBlock;
            if (pos < cap) {
                keys[pos] = key[j];
                weights[pos] = c[j];
            }
        }
    }
}

// hist_count over the pixels (x, y) with x and y multiples of `stride` of an
// H x W image whose rows start `pitch` bytes apart (the 2:1 subsampling of
// Section 2.2 for stride 2).
__global__ void __launch_bounds__(kCountBlock) hist_count_strided(const uint8_t *__restrict__ rgb, int32_t h,
                                                                  int32_t w, int64_t pitch, int32_t stride,
                                                                  uint32_t *__restrict__ cnt,
                                                                  uint32_t *__restrict__ bits)
{
    const int64_t hs = (h + stride - 1) / stride, ws = (w + stride - 1) / stride;
    const int64_t total = hs * ws;
    const int64_t nth = (int64_t)gridDim.x * kCountBlock;
    for (int64_t q = (int64_t)blockIdx.x * kCountBlock + threadIdx.x; q < total; q += nth) {
        const int64_t y = (q / ws) * stride, x = (q % ws) * stride;
        const uint8_t *px = rgb + y * pitch + 3 * x;
        add_colour(cnt, bits, ((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | (uint32_t)px[2]);
    }
}

// Every pixel as its own point of weight 1 (the k-means baseline of Table 1).
__global__ void __launch_bounds__(256) pixel_keys(const uint8_t *__restrict__ rgb, int64_t n,
                                                  uint32_t *__restrict__ keys, uint32_t *__restrict__ w,
                                                  int32_t *__restrict__ n_out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        keys[p] = key_at(rgb, p);
        if (w) w[p] = 1u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && n_out) *n_out = (int32_t)n;
}

}  // namespace

int launch_pixel_keys(const uint8_t *rgb, int64_t n, uint32_t *keys, uint32_t *weights, int32_t *n_out,
                      cudaStream_t s)
{
    const DeviceInfo di = device_info();
    int64_t want = (n + 255) / 256;
    int grid = (int)(want < (int64_t)di.sms * 8 ? want : (int64_t)di.sms * 8);
    if (grid < 1) grid = 1;
    pixel_keys<<<grid, 256, 0, s>>>(rgb, n, keys, weights, n_out);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

int launch_histogram_strided(const uint8_t *rgb, int32_t h, int32_t w, int64_t pitch, int32_t stride, uint32_t *keys,
                             uint32_t *weights, int32_t cap, int32_t *n_unique, void *ws, const Layout &L,
                             cudaStream_t s)
{
    uint32_t *cnt = at<uint32_t>(ws, L.hist_cnt);
    uint32_t *bits = at<uint32_t>(ws, L.hist_bits);
    uint32_t *chunk_tot = at<uint32_t>(ws, L.hist_chunk);
    Ctl *ctl = at<Ctl>(ws, L.ctl);
    const DeviceInfo di = device_info();
    const int64_t total = (int64_t)((h + stride - 1) / stride) * ((w + stride - 1) / stride);
    int64_t want = (total + kCountBlock - 1) / kCountBlock;
    int grid = (int)(want < (int64_t)di.sms * 8 ? want : (int64_t)di.sms * 8);
    if (grid < 1) grid = 1;
    if (total > 0) hist_count_strided<<<grid, kCountBlock, 0, s>>>(rgb, h, w, pitch, stride, cnt, bits);
    uint32_t *chunk_base = chunk_tot + kHistChunks;
    hist_chunks<<<kHistChunks, kEmitBlock, 0, s>>>(bits, chunk_tot);
    hist_bases<<<1, kBaseBlock, 0, s>>>(chunk_tot, chunk_base, cap, n_unique, ctl);
    hist_emit<<<kHistChunks, kEmitBlock, 0, s>>>(bits, cnt, chunk_base, keys, weights, cap);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

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
    uint32_t *chunk_base = chunk_tot + kHistChunks;
    hist_chunks<<<kHistChunks, kEmitBlock, 0, s>>>(bits, chunk_tot);
    hist_bases<<<1, kBaseBlock, 0, s>>>(chunk_tot, chunk_base, cap, n_unique, ctl);
    hist_emit<<<kHistChunks, kEmitBlock, 0, s>>>(bits, cnt, chunk_base, keys, weights, cap);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

}  // namespace kq
