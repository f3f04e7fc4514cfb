// map.cu -- pixel mapping (Section 1; full palette search as in Section 2.1) and
// the squared-error sum behind the MSE of Section 3.1 (Eq. 2).
//
// Each unique colour is matched to the palette once (map_lut), writing its index
// into a 2^24-entry byte table and adding w * d to the error sum; the pixel stream
// (map_pixels) then reads 48 bytes per 16 pixels, looks each colour up in the
// table (16 MiB, resident in L2) and writes 16 indices with one 16-byte store.
// The table is laid out in 4 x 4 x 4 colour blocks (lut_slot), so that one 32-byte
// L2 sector holds a 2 x 4 x 4 neighbourhood of colours instead of 32 values of B:
// neighbouring pixels of an image touch far fewer sectors.  Distances between
// 8-bit colours are exact integers below 2^18.
#include "kq_dev.cuh"

namespace kq {
namespace {

constexpr int kLutBlock = 256;
constexpr int kPixBlock = 256;

// Table slot of colour (R << 16) | (G << 8) | B: the 4 x 4 x 4 block
// (R >> 2, G >> 2, B >> 2) times 64, plus (R & 3) * 16 + (G & 3) * 4 + (B & 3).
// A permutation of 0 .. 2^24 - 1.
__device__ __forceinline__ uint32_t lut_slot(uint32_t key)
{
    return (key & 0xFC0000u) | ((key & 0xFC00u) << 2) | ((key & 0xFCu) << 4) | ((key >> 12) & 0x30u) |
           ((key >> 6) & 0xCu) | (key & 3u);
}

// Nearest palette entry of each unique colour.  With colours as byte vectors,
// |x - p|^2 = |x|^2 + |p|^2 - 2 x.p is an exact integer below 2^18, the dot product
// one dp4a; the value (d << 8) | k then orders by distance and, on ties, by the
// lower index, so one 32-bit minimum per palette entry gives the exact argmin.
// Each thread takes two colours per pass over the palette.
__global__ void __launch_bounds__(kLutBlock) map_lut(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ w,
                                                     const int32_t *n_unique, const uint8_t *__restrict__ palette,
                                                     int K, uint8_t *__restrict__ lut,
                                                     unsigned long long *__restrict__ sse_num)
{
    __shared__ uint2 s_p[kMaxK];  // .x packed colour, .y = (|p|^2 << 8) | k
    __shared__ unsigned long long s_red[kLutBlock / 32];
    for (int k = threadIdx.x; k < K; k += kLutBlock) {
        const uint32_t r = palette[3 * k], g = palette[3 * k + 1], bb = palette[3 * k + 2];
        s_p[k] = make_uint2((r << 16) | (g << 8) | bb, ((r * r + g * g + bb * bb) << 8) | (uint32_t)k);
    }
    __syncthreads();
    const int64_t n = *n_unique;
    unsigned long long acc = 0ull;
    const int64_t stride = (int64_t)gridDim.x * kLutBlock * 2;
    for (int64_t i0 = ((int64_t)blockIdx.x * kLutBlock + threadIdx.x) * 2; i0 < n; i0 += stride) {
        const bool two = i0 + 1 < n;
        const uint32_t ka = keys[i0], kb = two ? keys[i0 + 1] : ka;
        const uint32_t ba = __dp4a(ka, ka, 0u) << 8, bbv = __dp4a(kb, kb, 0u) << 8;
        uint32_t ma = 0xFFFFFFFFu, mb = 0xFFFFFFFFu;
#pragma unroll 8
        for (int k = 0; k < K; ++k) {
            const uint2 pk = s_p[k];
            ma = min(ma, ba + pk.y - (__dp4a(ka, pk.x, 0u) << 9));
            mb = min(mb, bbv + pk.y - (__dp4a(kb, pk.x, 0u) << 9));
        }
        lut[lut_slot(ka)] = (uint8_t)(ma & 0xFFu);
        acc += (unsigned long long)w[i0] * (ma >> 8);
        if (two) {
            lut[lut_slot(kb)] = (uint8_t)(mb & 0xFFu);
            acc += (unsigned long long)w[i0 + 1] * (mb >> 8);
        }
    }
    if (sse_num) {
        const unsigned long long t = block_sum_u64<kLutBlock>(acc, s_red);
        if (threadIdx.x == 0 && t) atomicAdd(sse_num, t);
    }
}

__device__ __forceinline__ uint32_t pixel_key(const uint8_t *rgb, int64_t p)
{
    const uint8_t *q = rgb + 3 * p;
    return ((uint32_t)q[0] << 16) | ((uint32_t)q[1] << 8) | (uint32_t)q[2];
}

template <int I>
__device__ __forceinline__ uint32_t group_key(const uint32_t (&w)[12])
{
    constexpr int o = 3 * I, q = o >> 2, r = o & 3;
    const uint32_t lo = w[q];
    const uint32_t hi = (q + 1 < 12) ? w[q + 1] : 0u;
    return __byte_perm(lo, hi, (r + 2) | ((r + 1) << 4) | (r << 8)) & 0xFFFFFFu;
}

template <int I>
__device__ __forceinline__ uint32_t lut4(const uint8_t *lut, const uint32_t (&w)[12])
{
    return (uint32_t)lut[lut_slot(group_key<I>(w))] | ((uint32_t)lut[lut_slot(group_key<I + 1>(w))] << 8) |
           ((uint32_t)lut[lut_slot(group_key<I + 2>(w))] << 16) | ((uint32_t)lut[lut_slot(group_key<I + 3>(w))] << 24);
}

template <bool kVecOut>
__global__ void __launch_bounds__(kPixBlock) map_pixels(const uint8_t *__restrict__ rgb, int64_t n, int64_t head,
                                                        const uint8_t *__restrict__ lut, uint8_t *__restrict__ idx)
{
    const int64_t tid = (int64_t)blockIdx.x * kPixBlock + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kPixBlock;
    const int64_t ngroups = (n - head) / 16;
    const int64_t tail0 = head + ngroups * 16;
    for (int64_t p = tid; p < head; p += nth) idx[p] = lut[lut_slot(pixel_key(rgb, p))];
    for (int64_t p = tail0 + tid; p < n; p += nth) idx[p] = lut[lut_slot(pixel_key(rgb, p))];
    const uint4 *g = reinterpret_cast<const uint4 *>(rgb + 3 * head);
    for (int64_t gi = tid; gi < ngroups; gi += nth) {
        const uint4 a = __ldcs(g + 3 * gi), b = __ldcs(g + 3 * gi + 1), c = __ldcs(g + 3 * gi + 2);
        const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
        const uint4 o = make_uint4(lut4<0>(lut, w), lut4<4>(lut, w), lut4<8>(lut, w), lut4<12>(lut, w));
        uint8_t *dst = idx + head + 16 * gi;
        if (kVecOut) {
            __stcs(reinterpret_cast<uint4 *>(dst), o);
        } else {
            const uint32_t ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) dst[k] = (uint8_t)(ov[k >> 2] >> (8 * (k & 3)));
        }
    }
}

}  // namespace

int launch_map(const uint8_t *rgb, int64_t n, const uint32_t *keys, const uint32_t *w, const int32_t *n_unique,
               const uint8_t *palette, int K, uint8_t *idx, int64_t *sse_num, void *ws, const Layout &L,
               cudaStream_t s)
{
    uint8_t *lut = at<uint8_t>(ws, L.lut);
    const DeviceInfo di = device_info();
    if (sse_num && cudaMemsetAsync(sse_num, 0, sizeof(int64_t), s) != cudaSuccess) return KQ_ECUDA;
    map_lut<<<di.sms * 4, kLutBlock, 0, s>>>(keys, w, n_unique, palette, K, lut,
                                             reinterpret_cast<unsigned long long *>(sse_num));
    if (n > 0) {
        const uintptr_t mis = reinterpret_cast<uintptr_t>(rgb) & 15u;
        int64_t head = (int64_t)(((16u - mis) * 11u) & 15u);  // 3 * 11 == 1 (mod 16)
        if (head > n) head = n;
        const int64_t groups = (n - head) / 16;
        int64_t want = (groups + kPixBlock - 1) / kPixBlock;
        int grid = (int)(want < (int64_t)di.sms * 8 ? want : (int64_t)di.sms * 8);
        if (grid < 1) grid = 1;
        const bool vec = ((reinterpret_cast<uintptr_t>(idx) + (uintptr_t)head) & 15u) == 0;
        if (vec)
            map_pixels<true><<<grid, kPixBlock, 0, s>>>(rgb, n, head, lut, idx);
        else
            map_pixels<false><<<grid, kPixBlock, 0, s>>>(rgb, n, head, lut, idx);
    }
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

}  // namespace kq
