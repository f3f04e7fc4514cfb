// map.cu -- pixel mapping (Section 1; full palette search as in Section 2.1) and
// the squared-error sum behind the MSE of Section 3.1 (Eq. 2).
//
// Each unique colour is matched to the palette once (map_lut), writing its index
// into a 2^24-entry byte table at its key and adding w * d to the error sum; the
// pixel stream (map_pixels) then reads 48 bytes per 16 pixels, looks each key up
// in the table (16 MiB, resident in L2) and writes 16 indices with one 16-byte
// store.  Distances between 8-bit colours are integers below 2^18, so FP32
// arithmetic on them is exact and the argmin is the integer argmin.
#include "kq_dev.cuh"

namespace kq {
namespace {

constexpr int kLutBlock = 256;
constexpr int kPixBlock = 256;

__global__ void __launch_bounds__(kLutBlock) map_lut(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ w,
                                                     const int32_t *n_unique, const uint8_t *__restrict__ palette,
                                                     int K, uint8_t *__restrict__ lut,
                                                     unsigned long long *__restrict__ sse_num)
{
    __shared__ float4 s_p[kMaxK];
    __shared__ unsigned long long s_red[kLutBlock / 32];
    for (int k = threadIdx.x; k < K; k += kLutBlock)
        s_p[k] = make_float4((float)palette[3 * k], (float)palette[3 * k + 1], (float)palette[3 * k + 2], 0.f);
    __syncthreads();
    const int64_t n = *n_unique;
    unsigned long long acc = 0ull;
    for (int64_t i = (int64_t)blockIdx.x * kLutBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kLutBlock) {
        const uint32_t key = keys[i];
        const float x = (float)key_r(key), y = (float)key_g(key), z = (float)key_b(key);
        float best = __int_as_float(0x7f800000);
        int arg = 0;
        for (int k = 0; k < K; ++k) {
            const float4 p = s_p[k];
            const float d = dist3(x, y, z, p.x, p.y, p.z);
            if (d < best) {
                best = d;
                arg = k;
            }
        }
        lut[key] = (uint8_t)arg;
        acc += (unsigned long long)w[i] * (unsigned long long)best;
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
    return (uint32_t)lut[group_key<I>(w)] | ((uint32_t)lut[group_key<I + 1>(w)] << 8) |
           ((uint32_t)lut[group_key<I + 2>(w)] << 16) | ((uint32_t)lut[group_key<I + 3>(w)] << 24);
}

template <bool kVecOut>
__global__ void __launch_bounds__(kPixBlock) map_pixels(const uint8_t *__restrict__ rgb, int64_t n, int64_t head,
                                                        const uint8_t *__restrict__ lut, uint8_t *__restrict__ idx)
{
    const int64_t tid = (int64_t)blockIdx.x * kPixBlock + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kPixBlock;
    const int64_t ngroups = (n - head) / 16;
    const int64_t tail0 = head + ngroups * 16;
    for (int64_t p = tid; p < head; p += nth) idx[p] = lut[pixel_key(rgb, p)];
    for (int64_t p = tail0 + tid; p < n; p += nth) idx[p] = lut[pixel_key(rgb, p)];
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
