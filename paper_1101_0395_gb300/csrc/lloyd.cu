// lloyd.cu -- Weighted Sort-Means (Algorithm 2) as one persistent cooperative kernel.
//
// Every pass runs on the device with no host round trip:
//   A. assignment: the unique colours (in key order) are cut into chunks of 32, and
//      block b takes chunks b, b + G, b + 2G, ... (neighbouring lanes hold similar
//      colours; every block samples the whole key range, which evens out the work).
//      A point starts at its previous centre p and scans row p of the sorted
//      centre-distance table; the scan stops at the first centre t with
//      d(c_p, c_t) > 4 d(x, c_p) (1 + 2^-17) (Section 2.2, item 3: if
//      2 d(x, c_p) <= d(c_p, c_t) then c_t is no nearer).  The widened bound and a
//      row table rounded down make the stop conservative under FP32 rounding, so the
//      labels equal a full FP32 search with the lowest index winning ties.  Each
//      block accumulates exact integer sums (w R, w G, w B, w) per cluster in shared
//      memory, its distance count, and its FP32 SSE partial: a fixed-order tree (per
//      32-colour chunk, then over the block's chunks in slot order, where the pruned
//      pass balances its chunks over the warps), so the sum is deterministic; the
//      blocks' partials are added in block order, also in FP32.
//   -- grid barrier --
//   B. update, in every block: SSE_i (a fixed-order sum of the block partials)
//      and the stopping test of Section 3.3, evaluated identically; every
//      cluster's FP32 centre, the FP32 number nearest to the exact quotient S / W
//      of its integer sums (an empty cluster keeps its centre), so that no block
//      waits for another's; block b also divides the sums of the clusters it owns
//      (k = b, b + G, ...) in FP64, the centres returned when the loop stops.
//   C. with pruning, block b builds its rows of the squared centre-to-centre
//      distance table, each sorted ascending and packed as (distance bits with the
//      low 8 cleared) | index.
//   -- grid barrier (pruning only) --
// A pass therefore has two grid barriers with pruning, one without.
#include "lloyd_body.cuh"

namespace kq {
namespace {

// One grid barrier over the first G blocks of the cooperative launch.
struct GridSync {
    Ctl *ctl;
    uint32_t G;  // blocks the barrier waits for
    uint32_t epoch;
    uint64_t limit_ns;
    __device__ __forceinline__ bool operator()() { return grid_sync(ctl, G, &epoch, limit_ns); }
};

template <class P>
__global__ void __launch_bounds__(kLloydBlock, 1) lloyd_kernel(LloydArgs a)
{
    __shared__ LloydShared sh;
    extern __shared__ uint32_t row_cache[];  // [K][kRowStride]
    const int64_t n = *a.n_unique;
    if (a.skip_if_n_le > 0 && n <= a.skip_if_n_le) return;
    int64_t want = (n + (int64_t)kLloydBlock * kPtsPerThread - 1) / ((int64_t)kLloydBlock * kPtsPerThread);
    const int G = (int)(want < 1 ? 1 : (want > gridDim.x ? gridDim.x : want));
    if ((int)blockIdx.x >= G) return;
    GridSync sync{a.ctl, (uint32_t)G + *(volatile const uint32_t *)&a.ctl->missing, 0u, wait_limit_ns(a.ctl)};
    lloyd_body<P>(a, sh, row_cache, n, (int)blockIdx.x, G, sync);
}

// Dynamic shared memory: the row cache for the largest K (one size for every
// launch, so the occupancy query and the cooperative grid are the same for all K).
size_t lloyd_smem_bytes() { return sizeof(uint32_t) * (size_t)kMaxK * kRowStride + sizeof(float) * kChunkSlots; }

// One cooperative launch of the whole loop over points of kind P (the grid barrier's
// arrival counter cleared on the stream first).
template <class P>
int launch_lloyd_kernel(LloydArgs &a, cudaStream_t s)
{
    const void *fn = (const void *)lloyd_kernel<P>;
    const size_t smem = lloyd_smem_bytes();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return KQ_ECUDA;
    const int per_sm = max_coresident(fn, kLloydBlock, smem);
    if (per_sm < 1) return KQ_ECUDA;
    int grid = device_info().sms * per_sm;
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (cudaMemsetAsync(&a.ctl->bar_count, 0, sizeof(uint32_t), s) != cudaSuccess) return KQ_ECUDA;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kLloydBlock), args, smem, s) == cudaSuccess ? KQ_OK
                                                                                                          : KQ_ECUDA;
}

}  // namespace

int launch_lloyd(const uint32_t *keys, const uint32_t *w, const int32_t *n_unique, int K, double *centers, double eps,
                 int max_iter, uint32_t flags, uint8_t *labels, uint8_t *palette, kq_lloyd_stats *stats,
                 double *sse_hist, void *ws, const Layout &L, cudaStream_t s, int skip_if_n_le)
{
    LloydArgs a;
    a.keys = keys;
    a.w = w;
    a.n_unique = n_unique;
    a.K = K;
    a.eps = eps;
    a.max_iter = max_iter;
    a.flags = flags;
    a.skip_if_n_le = skip_if_n_le;
    a.centers = centers;
    a.labels = labels;
    a.palette = palette;
    a.stats = stats;
    a.sse_hist = sse_hist;
    a.ctl = at<Ctl>(ws, L.ctl);
    a.ndc = &a.ctl->ndc;
    a.status = &a.ctl->status;
    a.sums = at<unsigned long long>(ws, L.l_sums);
    a.sse_part = at<float>(ws, L.l_sse);
    a.rows = at<uint32_t>(ws, L.l_rows);
    return launch_lloyd_kernel<RgbKeys>(a, s);
}

int launch_lloyd_points(const unsigned long long *pts, const uint32_t *w, const int32_t *n_unique, int K,
                        double *centers, double eps, int max_iter, uint32_t flags, uint8_t *labels,
                        kq_lloyd_stats *stats, double *sse_hist, void *ws, const Layout &L, cudaStream_t s)
{
    LloydArgs a;
    a.keys = pts;
    a.w = w;
    a.n_unique = n_unique;
    a.K = K;
    a.eps = eps;
    a.max_iter = max_iter;
    a.flags = flags;
    a.skip_if_n_le = 0;
    a.centers = centers;
    a.labels = labels;
    a.palette = nullptr;
    a.stats = stats;
    a.sse_hist = sse_hist;
    a.ctl = at<Ctl>(ws, L.ctl);
    a.ndc = &a.ctl->ndc;
    a.status = &a.ctl->status;
    a.sums = at<unsigned long long>(ws, L.l_sums);
    a.sse_part = at<float>(ws, L.l_sse);
    a.rows = at<uint32_t>(ws, L.l_rows);
    return launch_lloyd_kernel<FixedPoints>(a, s);
}

// ---------------------------------------------------------------- allocation-free variant
// kq_lloyd_noalloc runs the same kernel as kq_lloyd, with its scratch (control
// block, cluster sums, SSE partials, centre-distance rows) in one file-scope
// device array instead of a caller-allocated workspace.
namespace {

constexpr size_t kNoAllocCtl = 0;
constexpr size_t kNoAllocSums = 4096;
constexpr size_t kNoAllocSse = kNoAllocSums + sizeof(unsigned long long) * 3 * kMaxK * 4;
constexpr size_t kNoAllocRows = kNoAllocSse + sizeof(double) * 2 * kMaxGrid;
constexpr size_t kNoAllocBytes = kNoAllocRows + sizeof(uint32_t) * kMaxK * kMaxK;  // 356,352 bytes
static_assert(sizeof(Ctl) <= kNoAllocSums, "control block fits its slot");

// Shared by every call on a device and kept for the life of the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array in the current context.  The host-side
// name g_noalloc_scratch is only a stand-in for the symbol; the address comes
// from cudaGetSymbolAddress with the caller's device current.  It is looked up on
// every call (a host-side query that allocates nothing), so a context that was
// destroyed and created again (cudaDeviceReset) never sees a stale address.
int noalloc_scratch(void **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KQ_ECUDA;
    *out = p;
    return KQ_OK;
}

}  // namespace
}  // namespace kq

extern "C" KQ_API int kq_lloyd_noalloc(const uint32_t *keys, const uint32_t *weights, const int32_t *n_unique,
                                       int32_t K, double *centers, double eps, int32_t max_iter, uint32_t flags,
                                       uint8_t *labels, uint8_t *palette, kq_lloyd_stats *stats, double *sse_hist,
                                       kq_stream_t stream)
{
    using namespace kq;
    if (!keys || !weights || !n_unique || !centers || !labels || !palette) return KQ_EINVAL;
    // the scratch array holds sums and distance rows for at most kMaxK (256) centres
    if (K < 1 || K > kMaxK || max_iter < 1 || eps != eps) return KQ_EINVAL;
    if (flags & ~(KQ_LLOYD_LABELS_IN | KQ_LLOYD_DENSE)) return KQ_EINVAL;
    void *base = nullptr;
    const int st = noalloc_scratch(&base);
    if (st != KQ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    char *b = static_cast<char *>(base);
    // status, abort flag and barrier counters must start at zero; the kernel
    // clears the sums and the distance count itself
    if (cudaMemsetAsync(b + kNoAllocCtl, 0, sizeof(Ctl), s) != cudaSuccess) return KQ_ECUDA;
    const DeviceInfo di = device_info();
    const size_t smem = lloyd_smem_bytes();
    if (cudaFuncSetAttribute((const void *)lloyd_kernel<RgbKeys>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return KQ_ECUDA;
    int per_sm = max_coresident((const void *)lloyd_kernel<RgbKeys>, kLloydBlock, smem);
    if (per_sm < 1) return KQ_ECUDA;
    int grid = di.sms * per_sm;
    if (grid > kMaxGrid) grid = kMaxGrid;
    LloydArgs a;
    a.keys = keys;
    a.w = weights;
    a.n_unique = n_unique;
    a.K = K;
    a.eps = eps;
    a.max_iter = max_iter;
    a.flags = flags;
    a.skip_if_n_le = 0;
    a.centers = centers;
    a.labels = labels;
    a.palette = palette;
    a.stats = stats;
    a.sse_hist = sse_hist;
    a.ctl = reinterpret_cast<Ctl *>(b + kNoAllocCtl);
    a.ndc = &a.ctl->ndc;
    a.status = &a.ctl->status;
    a.sums = reinterpret_cast<unsigned long long *>(b + kNoAllocSums);
    a.sse_part = reinterpret_cast<float *>(b + kNoAllocSse);
    a.rows = reinterpret_cast<uint32_t *>(b + kNoAllocRows);
    void *args[] = {&a};
    cudaError_t e =
        cudaLaunchCooperativeKernel((const void *)lloyd_kernel<RgbKeys>, dim3(grid), dim3(kLloydBlock), args, smem, s);
    return e == cudaSuccess ? KQ_OK : KQ_ECUDA;
}
