// lloyd_body.cuh -- the Weighted Sort-Means iteration (Algorithm 2) as a device
// function over a group of blocks, shared by the whole-grid kernel (lloyd.cu) and
// the batched kernel (batch.cu), which differ only in their barrier.
#pragma once

#include "kq_dev.cuh"

namespace kq {
namespace {

constexpr int kLloydBlock = 512;
constexpr int kPtsPerThread = 1;  // blocks used = ceil(N' / (block * this)), capped by the launch
// Row padding entry: distance bits of a huge finite float, so the scan always stops on it.
constexpr uint32_t kPadEntry = 0x7F7FFF00u;
// The first kRowCache entries of every row are copied to shared memory each pass
// (row stride kRowCache + 1 words, so lanes reading different rows hit different banks).
constexpr int kRowCache = 32;
constexpr int kRowStride = kRowCache + 1;
// A whole-grid launch whose blocks hold kChunkSlotsMin..kChunkSlots chunks balances
// the pruned pass over the block's warps (a shared chunk counter).
constexpr int kChunkSlots = 4096;
constexpr int kChunkSlotsMin = 64;
constexpr int kCoopLanes = 2;  // at most this many scanning lanes go to the warp-wide scan
constexpr int kDensePts = 2;   // points per lane in the full search
constexpr float kPruneSlack = 1.0f + 0x1p-17f;
constexpr unsigned kFull = 0xffffffffu;

// The points the iteration runs on.  RgbKeys: unique colours as 24-bit keys, the
// coordinates their bytes.  FixedPoints: fixed-point 3-D points (CIE L*a*b* x 256),
// three signed 16-bit coordinates packed in a 64-bit word.  Either way the
// coordinates are integers, so the weighted sums of a cluster are exact.
struct RgbKeys {
    using T = uint32_t;
    static constexpr bool kRgb = true;
    static constexpr unsigned long long kMaxAbs = 255;  // largest |coordinate|
    __device__ __forceinline__ static T load(const void *p, int64_t i) { return static_cast<const T *>(p)[i]; }
    __device__ __forceinline__ static int c0(T k) { return (int)key_r(k); }
    __device__ __forceinline__ static int c1(T k) { return (int)key_g(k); }
    __device__ __forceinline__ static int c2(T k) { return (int)key_b(k); }
};
struct FixedPoints {
    using T = unsigned long long;
    static constexpr bool kRgb = false;
    static constexpr unsigned long long kMaxAbs = 32768;
    __device__ __forceinline__ static T load(const void *p, int64_t i) { return static_cast<const T *>(p)[i]; }
    __device__ __forceinline__ static int c0(T k) { return (int)(int16_t)(k & 0xFFFFull); }
    __device__ __forceinline__ static int c1(T k) { return (int)(int16_t)((k >> 16) & 0xFFFFull); }
    __device__ __forceinline__ static int c2(T k) { return (int)(int16_t)((k >> 32) & 0xFFFFull); }
};

struct LloydArgs {
    const void *keys;          // RgbKeys: uint32_t keys; FixedPoints: packed 64-bit points
    const uint32_t *w;
    const int32_t *n_unique;
    int K;
    double eps;
    int max_iter;
    uint32_t flags;
    int skip_if_n_le;
    double *centers;
    uint8_t *labels;
    uint8_t *palette;          // RgbKeys only (K x 3 bytes); FixedPoints: unused
    kq_lloyd_stats *stats;
    double *sse_hist;
    Ctl *ctl;                  // grid barrier of the whole-grid launch (unused by groups)
    unsigned long long *ndc;   // distance count of the call
    const int32_t *status;     // device status word reported in the statistics
    unsigned long long *sums;  // [3][kMaxK][4]: pass i adds into buffer i % 3
    float *sse_part;           // [2][kMaxGrid] block SSE partials (FP32, fixed-order trees)
    uint32_t *rows;            // [K][Kp], Kp = K rounded up to a multiple of 4
};

struct LloydShared {
    float4 c[kMaxK];
    float cx[kMaxK], cy[kMaxK], cz[kMaxK];  // the same FP32 centres, one array per channel
    double c64[kMaxK * 3];
    unsigned long long sum[kMaxK * 4];
    uint32_t sum32[kMaxK * 4];  // used instead of sum when the block's sums fit 32 bits
    uint32_t row[2][kMaxK];     // rows being ranked (build_rows_rank)
    float red_f[kLloydBlock / 32];
    unsigned long long red_u[kLloydBlock / 32];
    double sse_i;
    int conv;
    int narrow;
    int next;  // next chunk slot of the balanced pruned schedule
};

// Ascending bitonic sort of the 32 * EPL values a warp holds, element e = lane * EPL
// + j in v[j] of that lane: pairs more than EPL apart are exchanged by shuffles,
// the others inside the lane.
template <int EPL>
__device__ __forceinline__ void warp_bitonic_sort(uint32_t (&v)[EPL], int lane)
{
    constexpr int P = 32 * EPL;
#pragma unroll
    for (int size = 2; size <= P; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= EPL) {
#pragma unroll
                for (int j = 0; j < EPL; ++j) {
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, v[j], stride / EPL);
                    const int e = lane * EPL + j;
                    const bool up = (e & size) == 0, low = (e & stride) == 0;
                    v[j] = (low == up) ? min(v[j], o) : max(v[j], o);
                }
            } else {
#pragma unroll
                for (int j = 0; j < EPL; ++j) {
                    if ((j & stride) == 0) {
                        const int e = lane * EPL + j;
                        const bool up = (e & size) == 0;
                        const uint32_t x = v[j], y = v[j + stride];
                        const bool sw = (x > y) == up;
                        v[j] = sw ? y : x;
                        v[j + stride] = sw ? x : y;
                    }
                }
            }
        }
    }
}

// Rows p = b + G m (m = 0, 1, ...) of the sorted centre-distance table, one row per
// warp at a time: entry (distance bits with the low 8 cleared) | index, sorted
// ascending by a warp-wide bitonic network (every entry is distinct).
template <int EPL>
__device__ __forceinline__ void build_rows_t(const LloydShared &sh, int K, int b, int G, uint32_t *rows)
{
    constexpr int kWarpsB = kLloydBlock / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Kp = (K + 3) & ~3;
    for (int m = warp; b + G * m < K; m += kWarpsB) {
        const int p = b + G * m;
        const float4 cp = sh.c[p];
        uint32_t v[EPL];
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
            const int t = lane * EPL + j;
            v[j] = 0xFFFFFFFFu;
            if (t < K) {
                const float4 ct = sh.c[t];
                const float d = dist3(cp.x, cp.y, cp.z, ct.x, ct.y, ct.z);
                v[j] = (__float_as_uint(d) & 0xFFFFFF00u) | (uint32_t)t;
            }
        }
        warp_bitonic_sort<EPL>(v, lane);
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
            const int e = lane * EPL + j;
            if (e < Kp) rows[(size_t)p * Kp + e] = e < K ? v[j] : kPadEntry;
        }
    }
}

// Rows p = b, b + G, b + 2G, ... of the sorted centre-distance table; the two
// halves of the block build two rows at once.  Entry rank = number of smaller
// packed entries (the index in the low byte makes every entry distinct).
__device__ __forceinline__ void build_rows_rank(LloydShared &sh, int K, int b, int G, uint32_t *rows)
{
    constexpr int kHalf = kLloydBlock / 2;  // >= kMaxK
    const int Kp = (K + 3) & ~3;
    const int hs = threadIdx.x / kHalf, ht = threadIdx.x % kHalf;
    for (int m = 0; b + G * m < K; m += 2) {
        const int p = b + G * (m + hs);
        const bool act = p < K;
        if (ht < Kp) {
            uint32_t v = 0xFFFFFFFFu;
            if (act && ht < K) {
                const float4 cp = sh.c[p], ct = sh.c[ht];
                const float d = dist3(cp.x, cp.y, cp.z, ct.x, ct.y, ct.z);
                v = (__float_as_uint(d) & 0xFFFFFF00u) | (uint32_t)ht;
            }
            sh.row[hs][ht] = v;
        }
        __syncthreads();
        if (act && ht < Kp) {
            if (ht < K) {
                const uint32_t v = sh.row[hs][ht];
                const uint4 *r4 = reinterpret_cast<const uint4 *>(sh.row[hs]);
                int r = 0;
#pragma unroll 8
                for (int u = 0; u < Kp / 4; ++u) {
                    const uint4 q = r4[u];
                    r += (q.x < v) + (q.y < v) + (q.z < v) + (q.w < v);
                }
                rows[(size_t)p * Kp + r] = v;
            } else {
                rows[(size_t)p * Kp + ht] = kPadEntry;
            }
        }
        __syncthreads();
    }
}

// Few rows per block (K <= 2G, the whole-grid launch): the rank count above, two rows
// at once over all threads, has the shortest latency.  Many rows per block (block
// groups of a batch): one row per warp, sorted by the bitonic network.
__device__ __forceinline__ void build_rows(LloydShared &sh, int K, int b, int G, uint32_t *rows)
{
    if (K <= 2 * G) build_rows_rank(sh, K, b, G, rows);
    else if (K <= 32) build_rows_t<1>(sh, K, b, G, rows);
    else if (K <= 64) build_rows_t<2>(sh, K, b, G, rows);
    else if (K <= 128) build_rows_t<4>(sh, K, b, G, rows);
    else build_rows_t<8>(sh, K, b, G, rows);
}

// The FP32 number nearest to the exact quotient num / W (ties to even), W > 0: a
// cluster's FP32 centre coordinate from its exact integer sums.  The FP32 first
// guess f = m 2^e (three roundings) is within two units in the last place; each
// step checks it exactly with the 128-bit residual D = s 2^(1-e) - 2 m W, i.e.
// 2 (s / W - f) in units of W 2^(e-1): f is the nearest when |D| < W (half a unit
// in the last place; a quarter below a power of two) and moves one unit toward
// s / W otherwise, a tie going to the even neighbour.  (For W < 2^28 the result is
// also (float)((double)num / (double)W): a quotient whose denominator is below
// 2^28 cannot fall within 2^-53 of a midpoint without being on it.)
__device__ __forceinline__ float div_rn_exact(long long num, unsigned long long W)
{
    if (num == 0) return 0.f;
    const bool neg = num < 0;
    const unsigned long long s = neg ? 0ull - (unsigned long long)num : (unsigned long long)num;
    uint32_t u = __float_as_uint(__fdiv_rn(__ull2float_rn(s), __ull2float_rn(W)));
    for (int step = 0; step < 4; ++step) {
        const unsigned long long m = (unsigned long long)((u & 0x7FFFFFu) | 0x800000u);
        const int sh = 1 - ((int)(u >> 23) - 150);  // 1 - e
        unsigned __int128 A = s, B = (unsigned __int128)(2ull * m) * W, T = W;
        if (sh >= 0) A <<= sh;
        else {
            B <<= -sh;
            T <<= -sh;
        }
        if (A >= B) {
            const unsigned __int128 D = A - B;
            if (D < T || (D == T && !(m & 1ull))) break;
            ++u;
        } else {
            // below a power of two the next FP32 number down is half as far
            const unsigned __int128 D = m == 0x800000ull ? (B - A) << 1 : B - A;
            if (D < T || (D == T && !(m & 1ull))) break;
            --u;
        }
    }
    return neg ? -__uint_as_float(u) : __uint_as_float(u);
}

__device__ __forceinline__ void set_centre(LloydShared &sh, int k, float4 c)
{
    sh.c[k] = c;
    sh.cx[k] = c.x;
    sh.cy[k] = c.y;
    sh.cz[k] = c.z;
}

// Channel ch of centre k (the float4 and the per-channel copies).
__device__ __forceinline__ void set_coord(LloydShared &sh, int k, int ch, float v)
{
    reinterpret_cast<float *>(&sh.c[k])[ch] = v;
    (ch == 0 ? sh.cx : ch == 1 ? sh.cy : sh.cz)[k] = v;
}

// Full search over all K centres with the lowest index winning ties.  Distances are
// taken eight at a time and folded with fminf; the running best moves only on a
// strictly smaller group minimum (so the earliest group holding the minimum wins),
// and the winning group is evaluated again to find its first centre at that
// distance.  The same dist3 values as a one-at-a-time scan, so the same argmin.
__device__ __forceinline__ void dense_argmin(const LloydShared &sh, int K, float x, float y, float z, float &best,
                                             int &arg)
{
    best = __int_as_float(0x7f800000);
    int bg = -1;
    int k0 = 0;
    for (; k0 + 8 <= K; k0 += 8) {
        float d[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) d[j] = dist3(x, y, z, sh.cx[k0 + j], sh.cy[k0 + j], sh.cz[k0 + j]);
        const float m = fminf(fminf(fminf(d[0], d[1]), fminf(d[2], d[3])), fminf(fminf(d[4], d[5]), fminf(d[6], d[7])));
        if (m < best) {
            best = m;
            bg = k0;
        }
    }
    arg = 0;
    if (bg >= 0) {
#pragma unroll
        for (int j = 7; j >= 0; --j)
            if (dist3(x, y, z, sh.cx[bg + j], sh.cy[bg + j], sh.cz[bg + j]) == best) arg = bg + j;
    }
    for (int k = k0; k < K; ++k) {
        const float d = dist3(x, y, z, sh.cx[k], sh.cy[k], sh.cz[k]);
        if (d < best) {
            best = d;
            arg = k;
        }
    }
}

// Two FP32 values in one 64-bit register pair, for the packed f32x2 instructions.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// dist3 of one point (x, y, z broadcast into both halves of X, Y, Z) to two centres
// (one per half of CX, CY, CZ) with the packed f32x2 subtract, multiply and fused
// multiply-add.  Each half takes the same operations in the same order with the
// same rounding as dist3, so each half equals dist3 bit for bit; one instruction
// does the work of two, which halves the issue slots of the distance arithmetic.
__device__ __forceinline__ unsigned long long dist3x2(unsigned long long X, unsigned long long Y,
                                                      unsigned long long Z, unsigned long long CX,
                                                      unsigned long long CY, unsigned long long CZ)
{
    unsigned long long dx, dy, dz, d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(X), "l"(CX));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(Y), "l"(CY));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(Z), "l"(CZ));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(d) : "l"(dx));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d) : "l"(dy), "l"(d));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d) : "l"(dz), "l"(d));
    return d;
}

// Minimum of three values: one three-input min instruction.
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// dense_argmin for NP points at once: each group of eight centres is loaded from
// shared memory once (16-byte loads of the per-channel arrays) and used for every
// point, which also gives the scheduler NP independent chains.  Per point the
// distances (dist3x2, equal to dist3), the order of the comparisons and so the
// results are those of dense_argmin: the minimum of a group is exact whatever the
// order it is taken in, and the first group holding the minimum is kept.
template <int NP>
__device__ __forceinline__ void dense_argmin_n(const LloydShared &sh, int K, const float (&x)[NP],
                                               const float (&y)[NP], const float (&z)[NP], float (&best)[NP],
                                               int (&arg)[NP])
{
    unsigned long long X[NP], Y[NP], Z[NP];
    int bg[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        best[q] = __int_as_float(0x7f800000);
        bg[q] = -1;
        X[q] = pack2(x[q], x[q]);
        Y[q] = pack2(y[q], y[q]);
        Z[q] = pack2(z[q], z[q]);
    }
    int k0 = 0;
    for (; k0 + 8 <= K; k0 += 8) {
        // centres k0 + 2h and k0 + 2h + 1 as one packed pair per channel
        const ulonglong2 xa = *reinterpret_cast<const ulonglong2 *>(&sh.cx[k0]);
        const ulonglong2 xb = *reinterpret_cast<const ulonglong2 *>(&sh.cx[k0 + 4]);
        const ulonglong2 ya = *reinterpret_cast<const ulonglong2 *>(&sh.cy[k0]);
        const ulonglong2 yb = *reinterpret_cast<const ulonglong2 *>(&sh.cy[k0 + 4]);
        const ulonglong2 za = *reinterpret_cast<const ulonglong2 *>(&sh.cz[k0]);
        const ulonglong2 zb = *reinterpret_cast<const ulonglong2 *>(&sh.cz[k0 + 4]);
        const unsigned long long cx[4] = {xa.x, xa.y, xb.x, xb.y};
        const unsigned long long cy[4] = {ya.x, ya.y, yb.x, yb.y};
        const unsigned long long cz[4] = {za.x, za.y, zb.x, zb.y};
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float d[8];
#pragma unroll
            for (int h = 0; h < 4; ++h) unpack2(dist3x2(X[q], Y[q], Z[q], cx[h], cy[h], cz[h]), d[2 * h], d[2 * h + 1]);
            const float m = fmin3(fmin3(d[0], d[1], d[2]), fmin3(d[3], d[4], d[5]), fminf(d[6], d[7]));
            if (m < best[q]) {
                best[q] = m;
                bg[q] = k0;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        arg[q] = 0;
        if (bg[q] >= 0) {
#pragma unroll
            for (int j = 7; j >= 0; --j)
                if (dist3(x[q], y[q], z[q], sh.cx[bg[q] + j], sh.cy[bg[q] + j], sh.cz[bg[q] + j]) == best[q])
                    arg[q] = bg[q] + j;
        }
    }
    for (int k = k0; k < K; ++k) {
        const float cxk = sh.cx[k], cyk = sh.cy[k], czk = sh.cz[k];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float e = dist3(x[q], y[q], z[q], cxk, cyk, czk);
            if (e < best[q]) {
                best[q] = e;
                arg[q] = k;
            }
        }
    }
}

// Adds (w x0, w x1, w x2, w) of each lane's point to its cluster's block sums
// (two's-complement arithmetic, so signed coordinates add exactly).  When all lanes
// of the warp chose the same cluster, one lane adds the warp total.  `narrow`: the
// block's whole slice has sum(w) * max|x| < 2^31, so 32-bit sums are exact and the
// native 32-bit shared-memory atomics can be used.
template <class P>
__device__ __forceinline__ void warp_accumulate(LloydShared &sh, bool narrow, bool active, int arg, uint32_t w,
                                                typename P::T key)
{
    const int a0 = __shfl_sync(kFull, arg, 0);
    const bool same = __all_sync(kFull, !active || arg == a0);
    if (narrow) {
        uint32_t W = active ? w : 0u;
        uint32_t r = W * (uint32_t)P::c0(key), g = W * (uint32_t)P::c1(key), bb = W * (uint32_t)P::c2(key);
        if (same) {
            for (int o = 16; o; o >>= 1) {
                r += __shfl_down_sync(kFull, r, o);
                g += __shfl_down_sync(kFull, g, o);
                bb += __shfl_down_sync(kFull, bb, o);
                W += __shfl_down_sync(kFull, W, o);
            }
            if ((threadIdx.x & 31) == 0 && W) {
                atomicAdd(&sh.sum32[a0 * 4 + 0], r);
                atomicAdd(&sh.sum32[a0 * 4 + 1], g);
                atomicAdd(&sh.sum32[a0 * 4 + 2], bb);
                atomicAdd(&sh.sum32[a0 * 4 + 3], W);
            }
        } else if (active) {
            atomicAdd(&sh.sum32[arg * 4 + 0], r);
            atomicAdd(&sh.sum32[arg * 4 + 1], g);
            atomicAdd(&sh.sum32[arg * 4 + 2], bb);
            atomicAdd(&sh.sum32[arg * 4 + 3], W);
        }
        return;
    }
    unsigned long long W = active ? (unsigned long long)w : 0ull;
    unsigned long long r = (unsigned long long)((long long)W * P::c0(key));
    unsigned long long g = (unsigned long long)((long long)W * P::c1(key));
    unsigned long long bb = (unsigned long long)((long long)W * P::c2(key));
    if (same) {
        for (int o = 16; o; o >>= 1) {
            r += __shfl_down_sync(kFull, r, o);
            g += __shfl_down_sync(kFull, g, o);
            bb += __shfl_down_sync(kFull, bb, o);
            W += __shfl_down_sync(kFull, W, o);
        }
        if ((threadIdx.x & 31) == 0 && W) {
            atomicAdd(&sh.sum[a0 * 4 + 0], r);
            atomicAdd(&sh.sum[a0 * 4 + 1], g);
            atomicAdd(&sh.sum[a0 * 4 + 2], bb);
            atomicAdd(&sh.sum[a0 * 4 + 3], W);
        }
    } else if (active) {
        atomicAdd(&sh.sum[arg * 4 + 0], r);
        atomicAdd(&sh.sum[arg * 4 + 1], g);
        atomicAdd(&sh.sum[arg * 4 + 2], bb);
        atomicAdd(&sh.sum[arg * 4 + 3], W);
    }
}

// The Lloyd iteration run by G blocks (ranks b = 0..G-1) over n unique colours.
// `sync` is a barrier across the G blocks that orders their global memory
// accesses; it returns false when the wait gave up, and the blocks then return.
// Sum of the 32 lanes' values in one fixed tree (the result in lane 0).
__device__ __forceinline__ float chunk_sse(float v)
{
    for (int o = 16; o; o >>= 1) v = __fadd_rn(v, __shfl_down_sync(kFull, v, o));
    return v;
}

// One step of the full search: chunks c, c + S, ..., c + (NP-1) S (all < the chunk
// count), one point of each per lane; labels, SSE and block sums.  The SSE goes to
// the lane's running sum in chunk order, or (csse non-null) per chunk to csse[slot],
// slot = (chunk - b) / G, the first chunk's slot being j0.
template <class P, int NP>
__device__ __forceinline__ void dense_step(const LloydArgs &a, LloydShared &sh, int K, int64_t n, int64_t c,
                                           int64_t S, int lane, bool narrow, float &sse32, unsigned long long &ndc,
                                           float *csse, int j0)
{
    typename P::T kk[NP];
    uint32_t ww[NP];
    float px[NP], py[NP], pz[NP], bd[NP];
    int ga[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int64_t iq = (c + q * S) * 32 + lane;
        kk[q] = 0u;
        ww[q] = 0u;
        if (iq < n) {
            kk[q] = P::load(a.keys, iq);
            ww[q] = a.w[iq];
        }
        px[q] = (float)P::c0(kk[q]);
        py[q] = (float)P::c1(kk[q]);
        pz[q] = (float)P::c2(kk[q]);
    }
    dense_argmin_n<NP>(sh, K, px, py, pz, bd, ga);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int64_t iq = (c + q * S) * 32 + lane;
        const bool act = iq < n;
        const float e = act ? __fmul_rn((float)ww[q], bd[q]) : 0.f;
        if (act) {
            a.labels[iq] = (uint8_t)ga[q];
            if (!csse) sse32 = __fadd_rn(sse32, e);
            ndc += (unsigned long long)K;
        }
        if (csse) {
            const float t = chunk_sse(e);
            if (lane == 0) csse[j0 + q * kLloydBlock / 32] = t;
        }
        warp_accumulate<P>(sh, narrow, act, ga[q], ww[q], kk[q]);
    }
}

// Statistics of a run that stopped because a barrier wait gave up (block 0).
__device__ __forceinline__ void lloyd_failed_stats(const LloydArgs &a, int64_t n, int it)
{
    if (threadIdx.x != 0 || !a.stats) return;
    const int32_t s = *(volatile const int32_t *)a.status;
    kq_lloyd_stats st;
    st.iters = it;
    st.converged = 0;
    st.k_eff = (int32_t)(n < a.K ? n : a.K);
    st.status = s ? s : KQ_ETIMEOUT;
    st.ndc = 0;
    st.sse = 0.0;
    st.sse_prev = 0.0;
    *a.stats = st;
}

template <class P, class Sync>
__device__ __forceinline__ void lloyd_body(const LloydArgs &a, LloydShared &sh, uint32_t *row_cache, int64_t n, int b,
                                           int G, Sync &sync)
{
    const int K = a.K;
    const int Kp = (K + 3) & ~3;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kLloydBlock / 32;
    const bool prune = !(a.flags & KQ_LLOYD_DENSE);
    const bool labels_in = (a.flags & KQ_LLOYD_LABELS_IN) != 0;
    const int64_t nch = (n + 31) / 32;  // 32-colour chunks; this block takes b, b + G, ...
    const int64_t nslot64 = nch > b ? (nch - 1 - b) / G + 1 : 0;  // this block's chunks
    const int nslot = (int)(nslot64 < kChunkSlots ? nslot64 : kChunkSlots);
    // the balanced schedule pays where a whole-grid launch gives a block many chunks
    // (few: one chunk's atomic and reduction cost more than the waiting they save;
    // the small groups of a batch measured slightly slower with it)
    float *csse = G >= 32 && nslot64 >= kChunkSlotsMin && nslot64 <= kChunkSlots
                      ? reinterpret_cast<float *>(row_cache + kMaxK * kRowStride)
                      : nullptr;

    for (int k = tid; k < K; k += kLloydBlock) {
        const double x = a.centers[3 * k], y = a.centers[3 * k + 1], z = a.centers[3 * k + 2];
        sh.c64[3 * k] = x;
        sh.c64[3 * k + 1] = y;
        sh.c64[3 * k + 2] = z;
        set_centre(sh, k, make_float4((float)x, (float)y, (float)z, 0.f));
    }
    {
        unsigned long long sw = 0ull;
        for (int64_t c = b + (int64_t)G * warp; c < nch; c += (int64_t)G * kWarps) {
            const int64_t i = c * 32 + lane;
            if (i < n) sw += a.w[i];
        }
        sw = block_sum_u64<kLloydBlock>(sw, sh.red_u);
        if (tid == 0) sh.narrow = sw * P::kMaxAbs < (1ull << 31) ? 1 : 0;
        __syncthreads();
    }
    const bool narrow = sh.narrow != 0;
    if (prune) build_rows(sh, K, b, G, a.rows);
    if (b == 0) {
        for (int j = tid; j < 3 * kMaxK * 4; j += kLloydBlock) a.sums[j] = 0ull;
        if (tid == 0) *a.ndc = 0ull;
    }
    if (!sync()) {
        if (b == 0) lloyd_failed_stats(a, n, 0);
        return;
    }

    double prev_sse = 0.0;
    int it = 0;
    for (;;) {
        // ---- A: assignment
        const int buf = it & 1;
        unsigned long long *gsum = a.sums + (size_t)(it % 3) * kMaxK * 4;
        for (int j = tid; j < K * 4; j += kLloydBlock) {
            sh.sum[j] = 0ull;
            sh.sum32[j] = 0u;
        }
        const bool use_prev = prune && (labels_in || it > 0);
        if (use_prev) {
            // the first kRowCache entries of every row, 16 bytes per load
            constexpr int kQ = kRowCache / 4;
            for (int j = tid; j < K * kQ; j += kLloydBlock) {
                const int pr = j / kQ, q4 = j % kQ;
                uint4 v = make_uint4(kPadEntry, kPadEntry, kPadEntry, kPadEntry);
                if (4 * q4 < Kp) v = __ldcg(reinterpret_cast<const uint4 *>(a.rows + (size_t)pr * Kp) + q4);
                uint32_t *dst = row_cache + pr * kRowStride + 4 * q4;
                dst[0] = v.x;
                dst[1] = v.y;
                dst[2] = v.z;
                dst[3] = v.w;
            }
        }
        if (tid == 0) sh.next = kWarps;
        __syncthreads();
        float sse32 = 0.f;
        unsigned long long ndc = 0ull;
        // Full search (first pass, or no pruning): chunks c, c + S, ..., c + (NP-1) S in
        // one step, NP points per lane; a warp's last chunks, when fewer than NP are
        // left, go one per step, so that no lane searches for a point it does not have.
        // The SSE is added as in the pruned loop: in chunk order per lane, or per chunk
        // into csse.
        const int64_t S = (int64_t)G * kWarps;
        int64_t c = b + (int64_t)G * warp;
        for (; !use_prev && c + (kDensePts - 1) * S < nch; c += kDensePts * S)
            dense_step<P, kDensePts>(a, sh, K, n, c, S, lane, narrow, sse32, ndc, csse, (int)((c - b) / G));
        for (; !use_prev && c < nch; c += S)
            dense_step<P, 1>(a, sh, K, n, c, S, lane, narrow, sse32, ndc, csse, (int)((c - b) / G));
        // The pruned loop does little arithmetic per colour, so the next chunk's key,
        // weight and previous label are loaded before the current chunk is scanned:
        // the memory latency overlaps the scan.
        typename P::T nkey = 0;
        uint32_t nw = 0u;
        int nlab = 0;
        int jc = warp;
        {
            const int64_t c0 = b + (int64_t)G * warp, i0 = c0 * 32 + lane;
            if (use_prev && c0 < nch && i0 < n) {
                nkey = P::load(a.keys, i0);
                nw = a.w[i0];
                nlab = a.labels[i0];
            }
        }
        // With csse (the balanced schedule, see kChunkSlots) the warps take the
        // block's chunks b + G j from a shared counter, so that a warp whose chunks
        // scan long rows does not hold up the block; the SSE is then kept per chunk.
        for (int64_t c = b + (int64_t)G * warp; use_prev && c < nch;) {
            const int64_t i = c * 32 + lane;
            const bool active = i < n;
            typename P::T key = nkey;
            uint32_t w = nw;
            const int lab = nlab;
            int arg = 0;
            float best = 0.f;
            int jn = jc + kWarps;
            if (csse) {
                if (lane == 0) jn = atomicAdd(&sh.next, 1);
                jn = __shfl_sync(kFull, jn, 0);
            }
            const int64_t cn = b + (int64_t)G * jn;
            {
                const int64_t i1 = cn * 32 + lane;
                if (cn < nch && i1 < n) {
                    nkey = P::load(a.keys, i1);
                    nw = a.w[i1];
                    nlab = a.labels[i1];
                }
            }
            if (use_prev) {
                // Sort-means scan from the previous centre p.  Each lane walks its own
                // point's row through the shared-memory copy of its first kRowCache
                // entries while more than kCoopLanes lanes of the warp are still scanning;
                // the points left then continue one at a time, the whole warp testing 32
                // further entries of that point's row per step (shared memory up to
                // kRowCache, then L2).  A few long scans thus cost a few warp steps instead
                // of holding every lane of the warp.
                int p = active ? lab : 0;
                if (p >= K) p = 0;
                const float x = (float)P::c0(key), y = (float)P::c1(key), z = (float)P::c2(key);
                const float4 cp = sh.c[p];
                const float prev = dist3(x, y, z, cp.x, cp.y, cp.z);
                const float thr = __fmul_rn(4.0f * prev, kPruneSlack);
                float bd = prev;
                uint32_t bt = (uint32_t)p;
                bool done = !active;
                const uint32_t *rc = row_cache + p * kRowStride;
                const int jl = Kp < kRowCache ? Kp : kRowCache;
                int jstop = jl;
                // Four row entries per step: their loads are independent, and since a
                // row ascends, an entry is within the bound exactly when every entry
                // before it is; only those entries' centres are loaded and their
                // distances evaluated (in row order, so the running minimum is the
                // one-at-a-time scan's).
                for (int j = 0; j < jl; j += 8) {
                    if (!done) {
                        uint32_t e[8];
                        float4 ct[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) e[q] = rc[j + q];
#pragma unroll
                        for (int q = 0; q < 8; ++q) ct[q] = sh.c[e[q] & 0xFFu];  // every index is < K
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const bool in = !(__uint_as_float(e[q] & 0xFFFFFF00u) > thr);
                            const uint32_t t = e[q] & 0xFFu;
                            if (in && t != (uint32_t)p) {
                                const float d = dist3(x, y, z, ct[q].x, ct[q].y, ct[q].z);
                                ++ndc;
                                if (d < bd || (d == bd && t < bt)) {
                                    bd = d;
                                    bt = t;
                                }
                            }
                        }
                        done = __uint_as_float(e[7] & 0xFFFFFF00u) > thr;
                    }
                    const unsigned left = __ballot_sync(kFull, !done);
                    if (__popc(left) <= kCoopLanes) {
                        jstop = j + 8;
                        break;
                    }
                }
                unsigned tail = __ballot_sync(kFull, !done && Kp > jstop);
                while (tail) {
                    const int q = __ffs(tail) - 1;
                    tail &= tail - 1;
                    const typename P::T kq = __shfl_sync(kFull, key, q);
                    const int pq = __shfl_sync(kFull, p, q);
                    const float thq = __shfl_sync(kFull, thr, q);
                    float qd = __shfl_sync(kFull, bd, q);
                    uint32_t qt = __shfl_sync(kFull, bt, q);
                    const float qx = (float)P::c0(kq), qy = (float)P::c1(kq), qz = (float)P::c2(kq);
                    const uint32_t *row = a.rows + (size_t)pq * Kp;
                    const uint32_t *rcq = row_cache + pq * kRowStride;
                    for (int j0 = jstop; j0 < Kp; j0 += 32) {
                        const int j = j0 + lane;
                        uint32_t e = kPadEntry;
                        if (j < Kp) e = j < kRowCache ? rcq[j] : __ldcg(row + j);
                        const bool brk = __uint_as_float(e & 0xFFFFFF00u) > thq;
                        const unsigned bal = __ballot_sync(kFull, brk);
                        const uint32_t t = e & 0xFFu;
                        if (!brk && t != (uint32_t)pq) {
                            const float4 ct = sh.c[t];
                            const float d = dist3(qx, qy, qz, ct.x, ct.y, ct.z);
                            ++ndc;
                            if (d < qd || (d == qd && t < qt)) {
                                qd = d;
                                qt = t;
                            }
                        }
                        if (bal) break;
                    }
                    const uint32_t md = __reduce_min_sync(kFull, __float_as_uint(qd));
                    const uint32_t mt = __reduce_min_sync(kFull, __float_as_uint(qd) == md ? qt : 0xFFFFFFFFu);
                    if (lane == q) {
                        bd = __uint_as_float(md);
                        bt = mt;
                    }
                }
                if (active) {
                    ++ndc;  // the distance to the previous centre
                    best = bd;
                    arg = (int)bt;
                }
            } else if (active) {
                dense_argmin(sh, K, (float)P::c0(key), (float)P::c1(key), (float)P::c2(key), best, arg);
                ndc += (unsigned long long)K;
            }
            const float e = active ? __fmul_rn((float)w, best) : 0.f;
            if (active) {
                a.labels[i] = (uint8_t)arg;
                // w < 2^32 and best are FP32; one rounding per product, FP64 above the block
                if (!csse) sse32 = __fadd_rn(sse32, e);
            }
            if (csse) {
                const float t = chunk_sse(e);
                if (lane == 0) csse[jc] = t;
            }
            warp_accumulate<P>(sh, narrow, active, arg, w, key);
            c = cn;
            jc = jn;
        }
        if (csse) {
            // the block's SSE: the chunks' sums in slot order, whoever computed them
            __syncthreads();
            sse32 = 0.f;
            for (int jj = tid; jj < nslot; jj += kLloydBlock) sse32 = __fadd_rn(sse32, csse[jj]);
        }
        // the block's SSE (a fixed shuffle tree per warp, then the warps in order)
        // and distance count, valid in thread 0
        float bsse = 0.f;
        unsigned long long bndc = 0ull;
        for (int o = 16; o; o >>= 1) {
            sse32 = __fadd_rn(sse32, __shfl_down_sync(kFull, sse32, o));
            ndc += __shfl_down_sync(kFull, ndc, o);
        }
        if (lane == 0) {
            sh.red_f[warp] = sse32;
            sh.red_u[warp] = ndc;
        }
        __syncthreads();
        if (tid == 0)
            for (int i = 0; i < kWarps; ++i) {
                bsse = __fadd_rn(bsse, sh.red_f[i]);
                bndc += sh.red_u[i];
            }
        for (int j = tid; j < K * 4; j += kLloydBlock) {
            // 32-bit sums: coordinate sums of signed points are sign-extended, weights never
            const unsigned long long v =
                narrow ? ((!P::kRgb && (j & 3) != 3) ? (unsigned long long)(long long)(int32_t)sh.sum32[j]
                                                     : (unsigned long long)sh.sum32[j])
                       : sh.sum[j];
            if (v) atomicAdd(gsum + j, v);
        }
        if (tid == 0) {
            a.sse_part[(size_t)buf * kMaxGrid + b] = bsse;
            atomicAdd(a.ndc, bndc);
        }
        if (!sync()) {
            if (b == 0) lloyd_failed_stats(a, n, it);
            return;
        }

        // ---- B: every block derives every cluster's FP32 centre itself from the exact
        // sums (the FP32 number nearest to S / W), so no block waits for another
        // before its rows or its next assignment.  Warp 0 evaluates SSE_i and the
        // stopping test; warps 1-3 divide the sums of the clusters the block owns
        // (k = b, b + G, ...) in FP64, the centres returned when the loop stops.
        ++it;
        if (warp == 0) {
            float s = 0.f;
            for (int g = lane; g < G; g += 32) s = __fadd_rn(s, __ldcg(a.sse_part + (size_t)buf * kMaxGrid + g));
            for (int o = 16; o; o >>= 1) s = __fadd_rn(s, __shfl_down_sync(kFull, s, o));
            if (lane == 0) {
                const double si = (double)s;
                bool conv = false;
                if (a.eps >= 0.0) {
                    if (si == 0.0) conv = true;
                    else if (it > 1 && (prev_sse - si) / si <= a.eps) conv = true;
                }
                sh.sse_i = si;
                sh.conv = conv ? 1 : 0;
            }
        } else if (warp <= 3) {
            const int ch = warp - 1;
            for (int k = b + G * lane; k < K; k += G * 32) {
                const unsigned long long W = __ldcg(gsum + 4 * k + 3);
                if (W) sh.c64[3 * k + ch] = (double)(long long)__ldcg(gsum + 4 * k + ch) / (double)W;
            }
        } else {
            // one (cluster, channel) per thread and step; an empty cluster keeps its
            // centre (its FP32 copy is left as it is)
            for (int j = tid - 128; j < 3 * K; j += kLloydBlock - 128) {
                const int k = j / 3, ch = j - 3 * k;
                const unsigned long long W = __ldcg(gsum + 4 * k + 3);
                if (W) set_coord(sh, k, ch, div_rn_exact((long long)__ldcg(gsum + 4 * k + ch), W));
            }
        }
        __syncthreads();
        const double sse_i = sh.sse_i;
        const bool conv = sh.conv != 0;
        const bool stop = conv || it >= a.max_iter;
        if (stop) {
            for (int k = b + G * tid; k < K; k += G * kLloydBlock) {
                const unsigned long long W = __ldcg(gsum + 4 * k + 3);
                const double x = sh.c64[3 * k], y = sh.c64[3 * k + 1], z = sh.c64[3 * k + 2];
                a.centers[3 * k] = x;
                a.centers[3 * k + 1] = y;
                a.centers[3 * k + 2] = z;
                for (int ch = 0; P::kRgb && ch < 3; ++ch) {
                    int v;
                    if (W) {
                        const unsigned long long S = __ldcg(gsum + 4 * k + ch);
                        v = (int)((2ull * S + W) / (2ull * W));
                    } else {
                        const double f = floor(sh.c64[3 * k + ch] + 0.5);
                        v = f < 0.0 ? 0 : (f > 255.0 ? 255 : (int)f);
                    }
                    a.palette[3 * k + ch] = (uint8_t)v;
                }
            }
        }
        {
            // Buffer (pass + 1) % 3 was last read in the previous pass and is next added
            // into two passes from now, after barriers every block must reach first;
            // the blocks clear it in slices, so that no block lags behind the others.
            unsigned long long *ahead = a.sums + (size_t)((it + 1) % 3) * kMaxK * 4;
            for (int j = b + G * tid; j < K * 4; j += G * kLloydBlock) ahead[j] = 0ull;
        }
        if (b == 0) {
            if (tid == 0 && a.sse_hist) a.sse_hist[it - 1] = sse_i;
            if (stop && tid == 0 && a.stats) {
                kq_lloyd_stats st;
                st.iters = it;
                st.converged = conv ? 1 : 0;
                st.k_eff = (int32_t)(n < K ? n : K);
                st.status = *(volatile const int32_t *)a.status;
                st.ndc = (int64_t)*(volatile unsigned long long *)a.ndc;
                st.sse = sse_i;
                st.sse_prev = it > 1 ? prev_sse : 0.0;
                *a.stats = st;
            }
        }
        if (stop) return;
        prev_sse = sse_i;

        // ---- C: this block's rows of the distance table (pruning only), from the
        // centres every block now holds
        if (prune) {
            build_rows(sh, K, b, G, a.rows);
            if (!sync()) {
                if (b == 0) lloyd_failed_stats(a, n, it);
                return;
            }
        }
    }
}


}  // namespace
}  // namespace kq
