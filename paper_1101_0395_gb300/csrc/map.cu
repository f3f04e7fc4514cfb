// map.cu -- pixel mapping (Section 1; the palette search of k-means, Section 2.1) and
// the squared-error sum behind the MSE of Section 3.1 (Eq. 2).
//
// Every pixel gets the exact nearest palette entry (lowest index on ties) by a
// search restricted to the entries that can be nearest anywhere in its colour's
// cell (an 8 x 8 x 8 block of colours; 32^3 cells):
//   1. map_cells   for a cell B, U(B) = min over entries t of the largest squared
//                  distance from B to t bounds every colour's nearest distance, so
//                  an entry t with min distance d(B, t)^2 > U(B) is never nearest
//                  (nor tied) for a colour in B.  The other entries are B's
//                  candidates.  They are found per 32^3 super-cell S first (whose
//                  candidates include those of its 64 cells: U shrinks and the
//                  minimum distances grow on a sub-box), then per cell among S's.
//                  A cell with at most 7 candidates stores them in one 64-bit
//                  descriptor (unused slots repeat the first); a cell with more
//                  stores their count there and the list in its own 256-byte slot
//                  of the workspace;
//   2. map_pixels  reads 48 bytes per 16 pixels, takes the smallest packed
//                  (|x - p_k|^2 << 8) | k over its cell's candidates (the exact
//                  argmin, lowest index on ties), writes 16 indices with one
//                  16-byte store and adds the squared errors.
// The palette alone decides the cells, so a call needs no histogram and keeps no
// state between calls.  Squared distances between 8-bit colours are exact
// integers below 2^18.
#include "kq_dev.cuh"

namespace kq {
namespace {

constexpr int kCellBlock = 256;
constexpr int kPixBlock = 256;
constexpr int kCellSide = 8;                     // colours per cell edge
constexpr int kSuperSide = 32;                   // colours per super-cell edge
constexpr int kSubPerSuper = 64;                 // 4 x 4 x 4 cells per super-cell
constexpr int kSupers = 512;                     // 8 x 8 x 8 super-cells
constexpr int kInline = 7;                       // candidates a descriptor holds
constexpr unsigned long long kListed = 0xFFull << 56;  // descriptor: count in the low bits, list in the slot
constexpr unsigned kFullMask = 0xffffffffu;
static_assert(kCellBlock >= kMaxK, "one thread per palette entry in the super-cell pass");
static_assert(kCellBlock == 4 * kSubPerSuper, "four threads per cell in the cell pass");
static_assert(kMapCells == kSupers * kSubPerSuper, "cells tile the super-cells");

__device__ __forceinline__ uint32_t pal_key(const uint8_t *palette, int k)
{
    return ((uint32_t)palette[3 * k] << 16) | ((uint32_t)palette[3 * k + 1] << 8) | (uint32_t)palette[3 * k + 2];
}

// Squared distances from channel value v to the interval [lo, lo + side - 1]:
// the smallest (0 inside) and the largest.
__device__ __forceinline__ void span_d2(int v, int lo, int side, uint32_t &mn, uint32_t &mx)
{
    const int hi = lo + side - 1;
    const int a = v < lo ? lo - v : (v > hi ? v - hi : 0);
    const int b = max(v - lo, hi - v);
    mn = (uint32_t)(a * a);
    mx = (uint32_t)(b * b);
}

__device__ __forceinline__ void box_d2(uint32_t key, int r0, int g0, int b0, int side, uint32_t &mn, uint32_t &mx)
{
    uint32_t a, b, c, d, e, f;
    span_d2((int)(key >> 16), r0, side, a, b);
    span_d2((int)((key >> 8) & 255u), g0, side, c, d);
    span_d2((int)(key & 255u), b0, side, e, f);
    mn = a + c + e;
    mx = b + d + f;
}

// One block per super-cell.  Cell index: (R >> 3) * 1024 + (G >> 3) * 32 + (B >> 3).
__global__ void __launch_bounds__(kCellBlock) map_cells(const uint8_t *__restrict__ palette, int K,
                                                        unsigned long long *__restrict__ desc,
                                                        uint8_t *__restrict__ list, Ctl *ctl,
                                                        unsigned long long *sse_num)
{
    __shared__ uint32_t s_key[kMaxK];
    __shared__ uint8_t s_cand[kMaxK];
    __shared__ uint32_t s_red[kCellBlock / 32];
    __shared__ uint32_t s_cnt[kCellBlock / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = blockIdx.x;
    const int sr = (s >> 6) * kSuperSide, sg = ((s >> 3) & 7) * kSuperSide, sb = (s & 7) * kSuperSide;
    if (s == 0 && tid == 0) {
        if (sse_num) *sse_num = 0ull;
        ctl->map_ndc = 0ull;
    }
    // super-cell candidates: U(S) by a block minimum, then the entries with d_min <= U(S)
    uint32_t kt = 0u, mn = 0xFFFFFFFFu, mx = 0xFFFFFFFFu;
    if (tid < K) {
        kt = pal_key(palette, tid);
        s_key[tid] = kt;
        box_d2(kt, sr, sg, sb, kSuperSide, mn, mx);
    }
    uint32_t m = __reduce_min_sync(kFullMask, mx);
    if (lane == 0) s_red[warp] = m;
    __syncthreads();
    uint32_t u = s_red[0];
#pragma unroll
    for (int w = 1; w < kCellBlock / 32; ++w) u = min(u, s_red[w]);
    const bool cand = tid < K && mn <= u;
    const unsigned bal = __ballot_sync(kFullMask, cand);
    if (lane == 0) s_cnt[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kCellBlock / 32; ++w) {
        before += w < warp ? (int)s_cnt[w] : 0;
        total += (int)s_cnt[w];
    }
    if (cand) s_cand[before + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)tid;
    __syncthreads();
    // the 64 cells of S, four consecutive threads per cell, each taking every fourth
    // of S's candidates: U(B) by a minimum over the four, then B's candidates
    const int sub = tid >> 2, q = tid & 3;
    const int cr = sr + (sub >> 4) * kCellSide, cg = sg + ((sub >> 2) & 3) * kCellSide, cb = sb + (sub & 3) * kCellSide;
    uint32_t ub = 0xFFFFFFFFu;
    for (int j = q; j < total; j += 4) {
        uint32_t a, b;
        box_d2(s_key[s_cand[j]], cr, cg, cb, kCellSide, a, b);
        ub = min(ub, b);
    }
    ub = min(ub, __shfl_xor_sync(kFullMask, ub, 1));
    ub = min(ub, __shfl_xor_sync(kFullMask, ub, 2));
    unsigned long long d = 0ull;  // this thread's candidates, one byte each
    int n = 0;
    for (int j = q; j < total; j += 4) {
        const uint32_t t = s_cand[j];
        uint32_t a, b;
        box_d2(s_key[t], cr, cg, cb, kCellSide, a, b);
        if (a <= ub) {
            if (n < kInline) d |= (unsigned long long)t << (8 * n);
            ++n;
        }
    }
    // the four threads' candidates one after the other: shift by the ones before
    int pre = __shfl_up_sync(kFullMask, n, 1, 4);
    pre = q >= 1 ? pre : 0;
    const int two = __shfl_up_sync(kFullMask, n + pre, 2, 4);
    pre += q >= 2 ? two : 0;
    const int tot = __shfl_sync(kFullMask, pre + n, 3, 4);
    d = pre < kInline ? (d << (8 * pre)) & ((1ull << (8 * kInline)) - 1ull) : 0ull;
    d |= __shfl_xor_sync(kFullMask, d, 1);
    d |= __shfl_xor_sync(kFullMask, d, 2);
    const int cell = ((cr >> 3) << 10) | ((cg >> 3) << 5) | (cb >> 3);
    if (tot > kInline) {
        // the whole list in the cell's slot (each thread its own candidates, in order)
        uint8_t *dst = list + (size_t)cell * kMaxK + pre;
        int k = 0;
        for (int j = q; j < total; j += 4) {
            const uint32_t t = s_cand[j];
            uint32_t a, b;
            box_d2(s_key[t], cr, cg, cb, kCellSide, a, b);
            if (a <= ub) dst[k++] = (uint8_t)t;
        }
    }
    if (q == 0) {
        if (tot <= kInline) {
            // the unused slots repeat the first candidate, so that the pixel search can
            // evaluate a fixed number of slots without a branch
            const unsigned long long first = d & 0xFFull;
            for (int k = tot; k < kInline; ++k) d |= first << (8 * k);
            desc[cell] = d | ((unsigned long long)tot << 56);
        } else {
            desc[cell] = kListed | (unsigned)tot;
        }
    }
}

template <int I>
__device__ __forceinline__ uint32_t group_key(const uint32_t (&w)[12])
{
    constexpr int o = 3 * I, q = o >> 2, r = o & 3;
    const uint32_t lo = w[q];
    const uint32_t hi = (q + 1 < 12) ? w[q + 1] : 0u;
    return __byte_perm(lo, hi, (r + 2) | ((r + 1) << 4) | (r << 8)) & 0xFFFFFFu;
}

// Palette entry k as (packed colour, (|p_k|^2 << 8) | k): the packed value
// (|x|^2 << 8) + .y - (x.p << 9) is (|x - p|^2 << 8) | k.
struct PixCtx {
    const uint2 *pal;
    const unsigned long long *desc;
    const uint8_t *list;
};

__device__ __forceinline__ uint32_t map_cell(uint32_t x)
{
    return ((x >> 9) & 0x7C00u) | ((x >> 6) & 0x3E0u) | ((x >> 3) & 0x1Fu);
}

// (|x - p_k|^2 << 8) | k for palette entry k (xn = |x|^2 << 8).
__device__ __forceinline__ uint32_t packed_d(const PixCtx &c, uint32_t x, uint32_t xn, uint32_t k)
{
    const uint2 e = c.pal[k];
    return xn + e.y - (__dp4a(x, e.x, 0u) << 9);
}

// The rarely taken part of the search, out of line so that the 16 inlined copies
// of the common path stay small: inline slots FIX .. cnt - 1 (cnt <= 7), or, for a
// cell with more candidates (cnt field 0xFF), its list in the workspace.
__device__ __noinline__ uint32_t nearest_rest(const PixCtx &c, uint32_t x, uint32_t xn, unsigned long long d, int from,
                                             uint32_t &nd)
{
    uint32_t best = 0xFFFFFFFFu;
    const int cnt = (int)(d >> 56);
    if (cnt <= kInline) {
        for (int j = from; j < cnt; ++j) best = min(best, packed_d(c, x, xn, (uint32_t)(d >> (8 * j)) & 0xFFu));
        nd += (uint32_t)(cnt - from);
    } else {
        const int m = (int)(d & 0x1FFu);
        const uint8_t *l = c.list + (size_t)map_cell(x) * kMaxK;
        for (int j = 0; j < m; ++j) best = min(best, packed_d(c, x, xn, __ldg(l + j)));
        nd += (uint32_t)m;
    }
    return best;
}

// Nearest palette entry of colour x, packed as (d << 8) | k, from its cell's
// descriptor d; `nd` counts the distances computed.  The first FIX slots are
// evaluated without a branch (a cell has at least one candidate, and unused slots
// repeat the first); cells with more candidates finish in nearest_rest.  FIX grows
// with K, since larger palettes give cells more candidates.
template <int FIX>
__device__ __forceinline__ uint32_t nearest(const PixCtx &c, uint32_t x, unsigned long long d, uint32_t &nd)
{
    const uint32_t xn = __dp4a(x, x, 0u) << 8;
    const int cnt = (int)(d >> 56);
    if (cnt > kInline) return nearest_rest(c, x, xn, d, 0, nd);
    const uint32_t lo = (uint32_t)d;
    uint32_t best = packed_d(c, x, xn, lo & 0xFFu);
    if (FIX > 1) best = min(best, packed_d(c, x, xn, (lo >> 8) & 0xFFu));
    if (FIX > 2) best = min(best, packed_d(c, x, xn, (lo >> 16) & 0xFFu));
    nd += (uint32_t)(cnt < FIX ? cnt : FIX);
    if (cnt > FIX) best = min(best, nearest_rest(c, x, xn, d, FIX, nd));
    return best;
}

template <int FIX, int I, int E>
struct GroupRange {
    // descriptors of pixels I .. E - 1 of a group
    __device__ __forceinline__ static void load(const PixCtx &c, const uint32_t (&w)[12], unsigned long long (&d)[8])
    {
        d[I & 7] = __ldg(c.desc + map_cell(group_key<I>(w)));
        GroupRange<FIX, I + 1, E>::load(c, w, d);
    }
    // their searches (each key extracted again: cheaper than holding the keys)
    __device__ __forceinline__ static void search(const PixCtx &c, const uint32_t (&w)[12],
                                                  const unsigned long long (&d)[8], uint32_t (&o)[4],
                                                  unsigned long long &sse, uint32_t &nd)
    {
        const uint32_t v = nearest<FIX>(c, group_key<I>(w), d[I & 7], nd);
        sse += v >> 8;
        o[I >> 2] |= (v & 0xFFu) << (8 * (I & 3));
        GroupRange<FIX, I + 1, E>::search(c, w, d, o, sse, nd);
    }
};
template <int FIX, int E>
struct GroupRange<FIX, E, E> {
    __device__ __forceinline__ static void load(const PixCtx &, const uint32_t (&)[12], unsigned long long (&)[8]) {}
    __device__ __forceinline__ static void search(const PixCtx &, const uint32_t (&)[12],
                                                  const unsigned long long (&)[8], uint32_t (&)[4],
                                                  unsigned long long &, uint32_t &)
    {
    }
};

// The 16 pixels of a 48-byte group, eight at a time: the eight cell descriptors
// are loaded before the first of their searches, so their latencies overlap.
template <int FIX>
__device__ __forceinline__ uint4 map16(const PixCtx &c, const uint32_t (&w)[12], unsigned long long &sse,
                                       uint32_t &nd)
{
    unsigned long long d[8];
    uint32_t o[4] = {0u, 0u, 0u, 0u};
    GroupRange<FIX, 0, 8>::load(c, w, d);
    GroupRange<FIX, 0, 8>::search(c, w, d, o, sse, nd);
    GroupRange<FIX, 8, 16>::load(c, w, d);
    GroupRange<FIX, 8, 16>::search(c, w, d, o, sse, nd);
    return make_uint4(o[0], o[1], o[2], o[3]);
}

__device__ __forceinline__ uint32_t pixel_key(const uint8_t *rgb, int64_t p)
{
    const uint8_t *q = rgb + 3 * p;
    return ((uint32_t)q[0] << 16) | ((uint32_t)q[1] << 8) | (uint32_t)q[2];
}

template <bool kVecOut, int FIX>
__global__ void __launch_bounds__(kPixBlock, 3) map_pixels(const uint8_t *__restrict__ rgb, int64_t n, int64_t head,
                                                        const uint8_t *__restrict__ palette, int K,
                                                        const unsigned long long *__restrict__ desc,
                                                        const uint8_t *__restrict__ list, uint8_t *__restrict__ idx,
                                                        unsigned long long *sse_num, Ctl *ctl)
{
    __shared__ uint2 s_p[kMaxK];
    __shared__ unsigned long long s_red[kPixBlock / 32];
    for (int k = threadIdx.x; k < K; k += kPixBlock) {
        const uint32_t kk = pal_key(palette, k);
        s_p[k] = make_uint2(kk, (__dp4a(kk, kk, 0u) << 8) | (uint32_t)k);
    }
    __syncthreads();
    const PixCtx c{s_p, desc, list};
    const int64_t tid = (int64_t)blockIdx.x * kPixBlock + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kPixBlock;
    const int64_t ngroups = (n - head) / 16;
    const int64_t tail0 = head + ngroups * 16;
    unsigned long long sse = 0ull;
    uint32_t nd = 0u;
    for (int64_t p = tid; p < head; p += nth) {
        const uint32_t x = pixel_key(rgb, p);
        const uint32_t v = nearest<FIX>(c, x, __ldg(desc + map_cell(x)), nd);
        idx[p] = (uint8_t)(v & 0xFFu);
        sse += v >> 8;
    }
    for (int64_t p = tail0 + tid; p < n; p += nth) {
        const uint32_t x = pixel_key(rgb, p);
        const uint32_t v = nearest<FIX>(c, x, __ldg(desc + map_cell(x)), nd);
        idx[p] = (uint8_t)(v & 0xFFu);
        sse += v >> 8;
    }
    const uint4 *g = reinterpret_cast<const uint4 *>(rgb + 3 * head);
    unsigned long long ndc = 0ull;
    for (int64_t gi = tid; gi < ngroups; gi += nth) {
        const uint4 a = __ldcs(g + 3 * gi), b = __ldcs(g + 3 * gi + 1), cc = __ldcs(g + 3 * gi + 2);
        const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, cc.x, cc.y, cc.z, cc.w};
        const uint4 o = map16<FIX>(c, w, sse, nd);
        ndc += nd;
        nd = 0u;
        uint8_t *dst = idx + head + 16 * gi;
        if (kVecOut) {
            __stcs(reinterpret_cast<uint4 *>(dst), o);
        } else {
            const uint32_t ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) dst[k] = (uint8_t)(ov[k >> 2] >> (8 * (k & 3)));
        }
    }
    ndc += nd;
    const unsigned long long t = block_sum_u64<kPixBlock>(sse, s_red);
    const unsigned long long tn = block_sum_u64<kPixBlock>(ndc, s_red);
    if (threadIdx.x == 0) {
        if (sse_num && t) atomicAdd(sse_num, t);
        if (tn) atomicAdd(&ctl->map_ndc, tn);
    }
}

}  // namespace

int launch_map(const uint8_t *rgb, int64_t n, const uint8_t *palette, int K, uint8_t *idx, int64_t *sse_num,
               void *ws, const Layout &L, cudaStream_t s)
{
    unsigned long long *desc = at<unsigned long long>(ws, L.m_desc);
    uint8_t *list = at<uint8_t>(ws, L.m_list);
    Ctl *ctl = at<Ctl>(ws, L.ctl);
    unsigned long long *sse = reinterpret_cast<unsigned long long *>(sse_num);
    const DeviceInfo di = device_info();
    map_cells<<<kSupers, kCellBlock, 0, s>>>(palette, K, desc, list, ctl, sse);
    if (n > 0) {
        const uintptr_t mis = reinterpret_cast<uintptr_t>(rgb) & 15u;
        int64_t head = (int64_t)(((16u - mis) * 11u) & 15u);  // 3 * 11 == 1 (mod 16)
        if (head > n) head = n;
        const int64_t groups = (n - head) / 16;
        int64_t want = (groups + kPixBlock - 1) / kPixBlock;
        int grid = (int)(want < (int64_t)di.sms * 8 ? want : (int64_t)di.sms * 8);
        if (grid < 1) grid = 1;
        const bool vec = ((reinterpret_cast<uintptr_t>(idx) + (uintptr_t)head) & 15u) == 0;
        // branch-free slots per pixel: 1 for K <= 64, 2 for K <= 128, else 3
#define KQ_MAP_LAUNCH(V, F) map_pixels<V, F><<<grid, kPixBlock, 0, s>>>(rgb, n, head, palette, K, desc, list, idx, sse, ctl)
        if (vec) {
            if (K <= 64) KQ_MAP_LAUNCH(true, 1);
            else if (K <= 128) KQ_MAP_LAUNCH(true, 2);
            else KQ_MAP_LAUNCH(true, 3);
        } else {
            if (K <= 64) KQ_MAP_LAUNCH(false, 1);
            else if (K <= 128) KQ_MAP_LAUNCH(false, 2);
            else KQ_MAP_LAUNCH(false, 3);
        }
#undef KQ_MAP_LAUNCH
    }
    return cudaGetLastError() == cudaSuccess ? KQ_OK : KQ_ECUDA;
}

}  // namespace kq
