// lab.cu -- k-means in the CIE L*a*b* colour space (Section 2.1 names L*a*b* beside
// RGB as a space k-means runs in).
//
//   lab_points    each unique colour's 8-bit sRGB value (IEC 61966-2-1) made linear,
//                 taken to CIE XYZ by the sRGB matrix (D65) and to CIE 1976 L*a*b*
//                 relative to the D65 white, in FP64 with every operation separately
//                 rounded; then fixed point, 256 units per L*a*b* unit rounded to
//                 nearest (ties to even), each coordinate a signed 16-bit field of a
//                 64-bit word (every sRGB colour's L*a*b* lies within +-128).  The
//                 integer coordinates keep the weighted sums of Lloyd's update exact.
//   seed_points   Forgy seeds among the points (the draws of kq_seed's Forgy).
//   lab_palette   the inverse transform of K centres to an sRGB palette.
//   map_labels    each pixel's index is the label of its unique colour: the counter
//                 table of the histogram (zero between calls) holds label + 1 at the
//                 unique colours while the pixels are read, and is zeroed again.
// Lloyd itself is the same Weighted Sort-Means as for RGB (lloyd.cu, FixedPoints).
#include <math.h>

#include "seed_dev.cuh"

namespace kq {
namespace {

constexpr int kLabBlock = 256;
constexpr double kLabScale = 256.0;

// Linear value of each 8-bit sRGB level (IEC 61966-2-1 companding), computed on the
// host once and passed to the kernel by value.
struct SrgbLinear {
    double v[256];
};

const SrgbLinear &srgb_linear_table()
{
    static const SrgbLinear t = [] {
        SrgbLinear s;
        for (int i = 0; i < 256; ++i) {
            const double c = (double)i / 255.0;
            s.v[i] = c <= 0.04045 ? c / 12.92 : std::pow((c + 0.055) / 1.055, 2.4);
        }
        return s;
    }();
    return t;
}

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// (a x + b y) + c z, each product and sum rounded separately (no fused multiply-add).
__device__ __forceinline__ double dot3(double a, double x, double b, double y, double c, double z)
{
    return add(add(mul(a, x), mul(b, y)), mul(c, z));
}

__device__ __forceinline__ double lab_f(double t)
{
    const double d = 6.0 / 29.0;
    return t > mul(mul(d, d), d) ? cbrt(t) : add(t / mul(mul(3.0, d), d), 4.0 / 29.0);
}

__device__ __forceinline__ double lab_finv(double t)
{
    const double d = 6.0 / 29.0;
    return t > d ? mul(mul(t, t), t) : mul(mul(mul(3.0, d), d), sub(t, 4.0 / 29.0));
}

__device__ __forceinline__ unsigned long long pack_point(double L, double a, double b)
{
    const long long qL = __double2ll_rn(mul(L, kLabScale)), qa = __double2ll_rn(mul(a, kLabScale)),
                    qb = __double2ll_rn(mul(b, kLabScale));
    return (unsigned long long)(uint16_t)(int16_t)qL | ((unsigned long long)(uint16_t)(int16_t)qa << 16) |
           ((unsigned long long)(uint16_t)(int16_t)qb << 32);
}

__global__ void __launch_bounds__(kLabBlock) lab_points(const uint32_t *__restrict__ keys, const int32_t *n_unique,
                                                        SrgbLinear tab, unsigned long long *__restrict__ pts)
{
    __shared__ double s_lin[256];
    s_lin[threadIdx.x] = tab.v[threadIdx.x];
    __syncthreads();
    const int64_t n = *n_unique;
    const int64_t stride = (int64_t)gridDim.x * kLabBlock;
    for (int64_t i = (int64_t)blockIdx.x * kLabBlock + threadIdx.x; i < n; i += stride) {
        const uint32_t k = keys[i];
        const double r = s_lin[key_r(k)], g = s_lin[key_g(k)], b = s_lin[key_b(k)];
        const double X = dot3(0.4124564, r, 0.3575761, g, 0.1804375, b);
        const double Y = dot3(0.2126729, r, 0.7151522, g, 0.0721750, b);
        const double Z = dot3(0.0193339, r, 0.1191920, g, 0.9503041, b);
        const double fx = lab_f(X / 0.95047), fy = lab_f(Y / 1.0), fz = lab_f(Z / 1.08883);
        pts[i] = pack_point(sub(mul(116.0, fy), 16.0), mul(500.0, sub(fx, fy)), mul(200.0, sub(fy, fz)));
    }
}

__device__ __forceinline__ void point_to_centre(double *c, unsigned long long p)
{
    c[0] = (double)(int16_t)(p & 0xFFFFull);
    c[1] = (double)(int16_t)((p >> 16) & 0xFFFFull);
    c[2] = (double)(int16_t)((p >> 32) & 0xFFFFull);
}

// Forgy among the points: the partial Fisher-Yates draws of kq_seed's Forgy (stream
// 1); when K >= N' the points in order, padded with copies of the last.
__global__ void seed_points_fgy(const unsigned long long *pts, const int32_t *n_unique, int K, uint64_t seed,
                                double *centers)
{
    extern __shared__ uint32_t smem[];
    const int64_t n = *n_unique;
    if (n <= K) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            if (n == 0) centers[3 * k] = centers[3 * k + 1] = centers[3 * k + 2] = 0.0;
            else point_to_centre(centers + 3 * k, pts[k < n ? k : n - 1]);
        }
        return;
    }
    FyMap m{smem, smem + kMapSlots, kMapSlots - 1};
    uint32_t *pick = smem + 2 * kMapSlots;
    clear_map(m.pos1, kMapSlots);
    __syncthreads();
    if (threadIdx.x == 0) fisher_yates((uint32_t)n, (uint32_t)K, seed, 1, m, pick);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) point_to_centre(centers + 3 * k, pts[pick[k]]);
}

// sRGB of each centre (fixed-point L*a*b* units): inverse of lab_points, each
// channel clamped to [0, 1] and rounded half up to 0..255.
__global__ void lab_palette(const double *centers, int K, uint8_t *palette)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double L = centers[3 * k] / kLabScale, a = centers[3 * k + 1] / kLabScale, b = centers[3 * k + 2] / kLabScale;
    const double fy = add(L, 16.0) / 116.0;
    const double fx = add(fy, a / 500.0), fz = sub(fy, b / 200.0);
    const double X = mul(0.95047, lab_finv(fx)), Y = mul(1.0, lab_finv(fy)), Z = mul(1.08883, lab_finv(fz));
    double lin[3];
    lin[0] = sub(sub(mul(3.2404542, X), mul(1.5371385, Y)), mul(0.4985314, Z));
    lin[1] = add(add(mul(-0.9692660, X), mul(1.8760108, Y)), mul(0.0415560, Z));
    lin[2] = add(sub(mul(0.0556434, X), mul(0.2040259, Y)), mul(1.0572252, Z));
    for (int c = 0; c < 3; ++c) {
        double v = lin[c];
        v = v <= 0.0031308 ? mul(12.92, v) : sub(mul(1.055, pow(v, 1.0 / 2.4)), 0.055);
        v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
        palette[3 * k + c] = (uint8_t)floor(add(mul(v, 255.0), 0.5));
    }
}

// label + 1 at each unique colour of the counter table
__global__ void __launch_bounds__(kLabBlock) label_table(const uint32_t *__restrict__ keys, const int32_t *n_unique,
                                                         const uint8_t *__restrict__ labels, uint32_t *__restrict__ cnt)
{
    const int64_t n = *n_unique;
    const int64_t stride = (int64_t)gridDim.x * kLabBlock;
    for (int64_t i = (int64_t)blockIdx.x * kLabBlock + threadIdx.x; i < n; i += stride)
        cnt[keys[i]] = (uint32_t)labels[i] + 1u;
}

__global__ void __launch_bounds__(kLabBlock) label_pixels(const uint8_t *__restrict__ rgb, int64_t n,
                                                          const uint32_t *__restrict__ cnt, uint8_t *__restrict__ idx,
                                                          Ctl *ctl)
{
    const int64_t stride = (int64_t)gridDim.x * kLabBlock;
    uint32_t miss = 0u;
    for (int64_t p = (int64_t)blockIdx.x * kLabBlock + threadIdx.x; p < n; p += stride) {
        const uint8_t *q = rgb + 3 * p;
        const uint32_t v = cnt[((uint32_t)q[0] << 16) | ((uint32_t)q[1] << 8) | (uint32_t)q[2]];
        miss |= v == 0u;
        idx[p] = (uint8_t)(v ? v - 1u : 0u);
    }
    if (__syncthreads_or(miss != 0u) && threadIdx.x == 0) fail(ctl, KQ_EINVAL);
}

__global__ void __launch_bounds__(kLabBlock) label_clear(const uint32_t *__restrict__ keys, const int32_t *n_unique,
                                                         uint32_t *__restrict__ cnt)
{
    const int64_t n = *n_unique;
    const int64_t stride = (int64_t)gridDim.x * kLabBlock;
    for (int64_t i = (int64_t)blockIdx.x * kLabBlock + threadIdx.x; i < n; i += stride) cnt[keys[i]] = 0u;
}

}  // namespace

int launch_lab_points(const uint32_t *keys, const int32_t *n_unique, unsigned long long *pts, cudaStream_t s)
{
    lab_points<<<device_info().sms * 4, kLabBlock, 0, s>>>(keys, n_unique, srgb_linear_table(), pts);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

int launch_seed_points(const unsigned long long *pts, const int32_t *n_unique, int K, uint64_t seed, double *centers,
                       cudaStream_t s)
{
    const size_t smem = sizeof(uint32_t) * (2 * kMapSlots + kMaxK);
    if (cudaFuncSetAttribute((const void *)seed_points_fgy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return KQ_ECUDA;
    seed_points_fgy<<<1, 32, smem, s>>>(pts, n_unique, K, seed, centers);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

int launch_lab_palette(const double *centers, int K, uint8_t *palette, cudaStream_t s)
{
    lab_palette<<<1, kMaxK, 0, s>>>(centers, K, palette);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

int launch_map_labels(const uint8_t *rgb, int64_t n, const uint32_t *keys, const int32_t *n_unique,
                      const uint8_t *labels, uint8_t *idx, void *ws, const Layout &L, cudaStream_t s)
{
    uint32_t *cnt = at<uint32_t>(ws, L.hist_cnt);
    Ctl *ctl = at<Ctl>(ws, L.ctl);
    const DeviceInfo di = device_info();
    label_table<<<di.sms * 4, kLabBlock, 0, s>>>(keys, n_unique, labels, cnt);
    if (n > 0) {
        int64_t want = (n + kLabBlock - 1) / kLabBlock;
        const int grid = (int)(want < (int64_t)di.sms * 8 ? want : (int64_t)di.sms * 8);
        label_pixels<<<grid, kLabBlock, 0, s>>>(rgb, n, cnt, idx, ctl);
    }
    label_clear<<<di.sms * 4, kLabBlock, 0, s>>>(keys, n_unique, cnt);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

}  // namespace kq
