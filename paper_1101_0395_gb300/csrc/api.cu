// api.cu -- the extern "C" entry points declared in include/kq.h.
//
// Each entry point validates its arguments on the host (returning KQ_EINVAL and
// enqueueing nothing on error), recovers the workspace layout from the
// workspace size, and enqueues its kernels on the caller's stream.
#include <math.h>
#include <string.h>

#include <mutex>

#include "kq_dev.cuh"

namespace kq {

namespace {
constexpr int kMaxDevices = 64;
int g_sms[kMaxDevices];

struct OccEntry {
    const void *kernel;
    int device, block;
    size_t smem;
    int blocks;
};
OccEntry g_occ[64];
int g_occ_n = 0;
std::mutex g_occ_mu;
}  // namespace

DeviceInfo device_info()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) dev = 0;
    if (g_sms[dev] == 0) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = sms > 0 ? sms : 1;
    }
    return DeviceInfo{dev, g_sms[dev]};
}

int max_coresident(const void *kernel, int block, size_t smem)
{
    const int dev = device_info().device;
    std::lock_guard<std::mutex> lock(g_occ_mu);
    for (int i = 0; i < g_occ_n; ++i)
        if (g_occ[i].kernel == kernel && g_occ[i].device == dev && g_occ[i].block == block && g_occ[i].smem == smem)
            return g_occ[i].blocks;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, block, smem) != cudaSuccess) return 0;
    if (g_occ_n < 64) g_occ[g_occ_n++] = OccEntry{kernel, dev, block, smem, blocks};
    return blocks;
}

}  // namespace kq

using kq::Layout;

namespace {

__global__ void set_wait_fields(kq::Ctl *ctl, uint32_t limit_us, uint32_t missing)
{
    ctl->wait_limit_us = limit_us;
    ctl->missing = missing;
}

bool ws_ok(const void *ws, size_t ws_bytes, Layout *L)
{
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return false;
    *L = kq::layout_from_bytes(ws_bytes);
    return L->max_unique > 0;
}

}  // namespace

extern "C" {

size_t kq_workspace_size(int64_t max_pixels, int32_t max_K)
{
    if (max_pixels < 0 || max_K < 1 || max_K > kq::kMaxK) return 0;
    return kq::layout_for(max_pixels).total;
}

int kq_workspace_init(void *ws, size_t ws_bytes, kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    return cudaMemsetAsync(ws, 0, L.total, (cudaStream_t)stream) == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

int kq_histogram(const uint8_t *rgb, int64_t n_pixels, uint32_t *keys, uint32_t *weights, int32_t capacity,
                 int32_t *n_unique, void *ws, size_t ws_bytes, kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    if (n_pixels < 0 || capacity < 0 || !n_unique) return KQ_EINVAL;
    if (n_pixels > 0 && !rgb) return KQ_EINVAL;
    if (capacity > 0 && (!keys || !weights)) return KQ_EINVAL;
    if (n_pixels >= ((int64_t)1 << 32)) return KQ_EINVAL;  // counts are 32-bit
    return kq::launch_histogram(rgb, n_pixels, keys, weights, capacity, n_unique, ws, L, (cudaStream_t)stream);
}

int kq_histogram_strided(const uint8_t *rgb, int32_t height, int32_t width, int64_t pitch, int32_t stride,
                         uint32_t *keys, uint32_t *weights, int32_t capacity, int32_t *n_unique, void *ws,
                         size_t ws_bytes, kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    if (height < 0 || width < 0 || stride < 1 || capacity < 0 || !n_unique) return KQ_EINVAL;
    if (pitch < 3 * (int64_t)width) return KQ_EINVAL;
    if ((int64_t)height * width > 0 && !rgb) return KQ_EINVAL;
    if (capacity > 0 && (!keys || !weights)) return KQ_EINVAL;
    return kq::launch_histogram_strided(rgb, height, width, pitch, stride, keys, weights, capacity, n_unique, ws, L,
                                        (cudaStream_t)stream);
}

int kq_seed(const uint32_t *keys, const uint32_t *weights, const int32_t *n_unique, int32_t K, int32_t scheme,
            uint64_t seed, const kq_seed_params *params, double *centers, void *ws, size_t ws_bytes,
            kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    if (!keys || !weights || !n_unique || !centers) return KQ_EINVAL;
    if (K < 1 || K > kq::kMaxK) return KQ_EINVAL;
    if ((scheme < KQ_INIT_FGY || scheme > KQ_INIT_KPP) && scheme != KQ_INIT_WU) return KQ_EINVAL;
    kq_seed_params p{1.0, 1e-4, 100, 0};
    if (params) {
        p = *params;
        if (p.max_iter < 1 || p.reserved != 0 || !(p.conv_eps == p.conv_eps) || !(p.lbg_eps == p.lbg_eps))
            return KQ_EINVAL;
    }
    return kq::launch_seed(keys, weights, n_unique, K, scheme, seed, p, centers, ws, L, (cudaStream_t)stream);
}

int kq_lloyd(const uint32_t *keys, const uint32_t *weights, const int32_t *n_unique, int32_t K, double *centers,
             double eps, int32_t max_iter, uint32_t flags, uint8_t *labels, uint8_t *palette, kq_lloyd_stats *stats,
             double *sse_hist, void *ws, size_t ws_bytes, kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    if (!keys || !weights || !n_unique || !centers || !labels || !palette) return KQ_EINVAL;
    if (K < 1 || K > kq::kMaxK || max_iter < 1 || eps != eps) return KQ_EINVAL;
    if (flags & ~(KQ_LLOYD_LABELS_IN | KQ_LLOYD_DENSE)) return KQ_EINVAL;
    return kq::launch_lloyd(keys, weights, n_unique, K, centers, eps, max_iter, flags, labels, palette, stats,
                            sse_hist, ws, L, (cudaStream_t)stream, 0);
}

int kq_map(const uint8_t *rgb, int64_t n_pixels, const uint8_t *palette, int32_t K, uint8_t *idx, int64_t *sse_num,
           void *ws, size_t ws_bytes, kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    if (n_pixels < 0 || !palette) return KQ_EINVAL;
    if (n_pixels > 0 && (!rgb || !idx)) return KQ_EINVAL;
    if (K < 1 || K > kq::kMaxK) return KQ_EINVAL;
    return kq::launch_map(rgb, n_pixels, palette, K, idx, sse_num, ws, L, (cudaStream_t)stream);
}

int kq_lab_points(const uint32_t *keys, const int32_t *n_unique, uint64_t *points, kq_stream_t stream)
{
    if (!keys || !n_unique || !points) return KQ_EINVAL;
    return kq::launch_lab_points(keys, n_unique, reinterpret_cast<unsigned long long *>(points), (cudaStream_t)stream);
}

int kq_seed_points(const uint64_t *points, const int32_t *n_unique, int32_t K, int32_t scheme, uint64_t seed,
                   double *centers, kq_stream_t stream)
{
    if (!points || !n_unique || !centers) return KQ_EINVAL;
    if (K < 1 || K > kq::kMaxK || scheme != KQ_INIT_FGY) return KQ_EINVAL;
    return kq::launch_seed_points(reinterpret_cast<const unsigned long long *>(points), n_unique, K, seed, centers,
                                  (cudaStream_t)stream);
}

int kq_lloyd_points(const uint64_t *points, const uint32_t *weights, const int32_t *n_unique, int32_t K,
                    double *centers, double eps, int32_t max_iter, uint32_t flags, uint8_t *labels,
                    kq_lloyd_stats *stats, double *sse_hist, void *ws, size_t ws_bytes, kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    if (!points || !weights || !n_unique || !centers || !labels) return KQ_EINVAL;
    if (K < 1 || K > kq::kMaxK || max_iter < 1 || eps != eps) return KQ_EINVAL;
    if (flags & ~(KQ_LLOYD_LABELS_IN | KQ_LLOYD_DENSE)) return KQ_EINVAL;
    return kq::launch_lloyd_points(reinterpret_cast<const unsigned long long *>(points), weights, n_unique, K, centers,
                                   eps, max_iter, flags, labels, stats, sse_hist, ws, L, (cudaStream_t)stream);
}

int kq_lab_palette(const double *centers, int32_t K, uint8_t *palette, kq_stream_t stream)
{
    if (!centers || !palette || K < 1 || K > kq::kMaxK) return KQ_EINVAL;
    return kq::launch_lab_palette(centers, K, palette, (cudaStream_t)stream);
}

int kq_map_labels(const uint8_t *rgb, int64_t n_pixels, const uint32_t *keys, const int32_t *n_unique,
                  const uint8_t *labels, uint8_t *idx, void *ws, size_t ws_bytes, kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    if (n_pixels < 0 || !keys || !n_unique || !labels) return KQ_EINVAL;
    if (n_pixels > 0 && (!rgb || !idx)) return KQ_EINVAL;
    return kq::launch_map_labels(rgb, n_pixels, keys, n_unique, labels, idx, ws, L, (cudaStream_t)stream);
}

int kq_pixel_keys(const uint8_t *rgb, int64_t n_pixels, uint32_t *keys, uint32_t *weights, int32_t *n_out,
                  kq_stream_t stream)
{
    if (n_pixels < 0 || n_pixels > 0x7FFFFFFF) return KQ_EINVAL;
    if (n_pixels > 0 && (!rgb || !keys)) return KQ_EINVAL;
    if (n_pixels == 0 && !n_out) return KQ_OK;
    return kq::launch_pixel_keys(rgb, n_pixels, keys, weights, n_out, (cudaStream_t)stream);
}

int kq_set_wait_limit(void *ws, size_t ws_bytes, uint32_t wait_limit_us, uint32_t missing_arrivals,
                      kq_stream_t stream)
{
    Layout L;
    if (!ws_ok(ws, ws_bytes, &L)) return KQ_EINVAL;
    set_wait_fields<<<1, 1, 0, (cudaStream_t)stream>>>(kq::at<kq::Ctl>(ws, L.ctl), wait_limit_us, missing_arrivals);
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

int kq_status_read(const void *ws, int32_t *h_status, kq_stream_t stream)
{
    if (!ws || !h_status) return KQ_EINVAL;
    const kq::Ctl *ctl = reinterpret_cast<const kq::Ctl *>(ws);
    int32_t v = 0;
    if (cudaMemcpyAsync(&v, &ctl->status, sizeof(v), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
        return KQ_ECUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return KQ_ECUDA;
    *h_status = v;
    return KQ_OK;
}

int kq_map_ndc_read(const void *ws, int64_t *h_ndc, kq_stream_t stream)
{
    if (!ws || !h_ndc) return KQ_EINVAL;
    const kq::Ctl *ctl = reinterpret_cast<const kq::Ctl *>(ws);
    unsigned long long v = 0;
    if (cudaMemcpyAsync(&v, &ctl->map_ndc, sizeof(v), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
        return KQ_ECUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return KQ_ECUDA;
    *h_ndc = (int64_t)v;
    return KQ_OK;
}

int kq_status_clear(void *ws, kq_stream_t stream)
{
    if (!ws) return KQ_EINVAL;
    return cudaMemsetAsync(ws, 0, sizeof(kq::Ctl), (cudaStream_t)stream) == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

const char *kq_strerror(int status)
{
    switch (status) {
    case KQ_OK: return "ok";
    case KQ_EINVAL: return "invalid argument";
    case KQ_ECAPACITY: return "more unique colours than the capacity of keys/weights";
    case KQ_ECUDA: return "CUDA runtime error";
    case KQ_ETIMEOUT: return "device-side wait timed out";
    case KQ_ENOMEM: return "workspace too small for the request";
    default: return "unknown status";
    }
}

}  // extern "C"
