// seed_dev.cuh -- pieces of the seeding schemes (Section 2.3) used both by the
// single-image kernels (seed.cu) and by the batched kernel (batch.cu).
#pragma once

#include "kq_dev.cuh"

namespace kq {
namespace {

constexpr int kMapSlots = 8192;  // Fisher-Yates displacement map (positions + values)
constexpr int kSffMax = 4096;    // ceil(2 * 256 * ln 256) = 2840 fits
constexpr unsigned kSeedFull = 0xffffffffu;

__device__ __forceinline__ void key_to_centre(double *c, uint32_t key)
{
    c[0] = (double)key_r(key);
    c[1] = (double)key_g(key);
    c[2] = (double)key_b(key);
}

// ---------------------------------------------------------------- Fisher-Yates
struct FyMap {
    uint32_t *pos1;  // position + 1, 0 = empty
    uint32_t *val;
    uint32_t mask;
};

__device__ __forceinline__ uint32_t fy_slot(uint32_t pos, uint32_t mask) { return (pos * 2654435761u) & mask; }

__device__ uint32_t fy_get(const FyMap &m, uint32_t pos)
{
    for (uint32_t h = fy_slot(pos, m.mask);; h = (h + 1) & m.mask) {
        if (m.pos1[h] == 0u) return pos;
        if (m.pos1[h] == pos + 1u) return m.val[h];
    }
}

__device__ void fy_set(const FyMap &m, uint32_t pos, uint32_t v)
{
    uint32_t h = fy_slot(pos, m.mask);
    while (m.pos1[h] != 0u && m.pos1[h] != pos + 1u) h = (h + 1) & m.mask;
    m.pos1[h] = pos + 1u;
    m.val[h] = v;
}

// The first `count` entries of a uniformly random permutation of 0..n-1
// (single thread; the map must hold 2 * count entries).
__device__ void fisher_yates(uint32_t n, uint32_t count, uint64_t seed, uint32_t stream, const FyMap &m, uint32_t *out)
{
    for (uint32_t j = 0; j < count; ++j) {
        const uint32_t r = j + (uint32_t)below(rand64(seed, stream, j), (uint64_t)(n - j));
        const uint32_t vj = fy_get(m, j), vr = fy_get(m, r);
        fy_set(m, j, vr);
        fy_set(m, r, vj);
        out[j] = vr;
    }
}

__device__ void clear_map(uint32_t *pos1, int slots)
{
    for (int i = threadIdx.x; i < slots; i += blockDim.x) pos1[i] = 0u;
}

// Minmax candidate: larger D^2 first, then the lower key (keys ascend with the
// index, so this is the lowest index among ties).
__device__ __forceinline__ unsigned long long mmx_pack(uint32_t d2, uint32_t key)
{
    return ((unsigned long long)d2 << 24) | (unsigned long long)(0xFFFFFFu - key);
}

__device__ __forceinline__ int den_cell(uint32_t key)
{
    return (int)(((key >> 22) & 3u) * 16u + ((key >> 14) & 3u) * 4u + ((key >> 6) & 3u));
}


// Exact per-cluster SSE about the mean is num / W with num = W Q - |S|^2.
__device__ __forceinline__ bool sse_greater(unsigned __int128 na, unsigned long long wa, unsigned __int128 nb,
                                            unsigned long long wb)
{
    if (wa == 0) return false;
    if (wb == 0) return true;
    return na * (unsigned __int128)wb > nb * (unsigned __int128)wa;
}

__device__ void den_quota(int K, const uint32_t *celln_in, const unsigned long long *cellw, int *quota_out)
{
    int64_t celln[kDenCells], q[kDenCells], rem[kDenCells];
    int fixed[kDenCells];
    for (int c = 0; c < kDenCells; ++c) {
        celln[c] = celln_in[c];
        fixed[c] = 0;
    }
    for (;;) {
        int64_t seats = K;
        unsigned long long wa = 0;
        for (int c = 0; c < kDenCells; ++c) {
            if (fixed[c]) seats -= celln[c];
            else if (celln[c] > 0) wa += cellw[c];
        }
        int64_t given = 0;
        for (int c = 0; c < kDenCells; ++c) {
            q[c] = 0;
            rem[c] = -1;
            if (fixed[c]) {
                q[c] = celln[c];
            } else if (celln[c] > 0 && wa > 0) {
                const unsigned long long num = (unsigned long long)seats * cellw[c];
                q[c] = (int64_t)(num / wa);
                rem[c] = (int64_t)(num % wa);
                given += q[c];
            }
        }
        for (int64_t left = seats - given; left > 0; --left) {
            int arg = -1;
            for (int c = 0; c < kDenCells; ++c)
                if (rem[c] >= 0 && (arg < 0 || rem[c] > rem[arg])) arg = c;
            q[arg] += 1;
            rem[arg] = -1;
        }
        int grew = 0;
        for (int c = 0; c < kDenCells; ++c) {
            if (!fixed[c] && q[c] > celln[c]) {
                fixed[c] = 1;
                grew = 1;
            }
        }
        if (!grew) break;
    }
    int off = 0;
    for (int c = 0; c < kDenCells; ++c) {
        quota_out[c] = (int)q[c];
        quota_out[kDenCells + c] = off;
        off += (int)q[c];
    }
}

__device__ void lbg_split(int K, int m, double eps, const unsigned long long *cs, double *centers)
{
    const int split = (2 * m <= K) ? m : K - m;
    bool chosen[kMaxK];
    for (int j = 0; j < m; ++j) chosen[j] = split == m;
    if (split < m) {
        for (int t = 0; t < split; ++t) {
            int arg = -1;
            unsigned __int128 na = 0;
            unsigned long long wa = 0;
            for (int k = 0; k < m; ++k) {
                if (chosen[k]) continue;
                const unsigned long long W = __ldcg(cs + 5 * k + 3);
                unsigned __int128 s2 = 0;
                for (int ch = 0; ch < 3; ++ch) s2 += (unsigned __int128)__ldcg(cs + 5 * k + ch) * __ldcg(cs + 5 * k + ch);
                const unsigned __int128 num = (unsigned __int128)W * __ldcg(cs + 5 * k + 4) - s2;
                if (arg < 0 || sse_greater(num, W, na, wa)) {
                    arg = k;
                    na = num;
                    wa = W;
                }
            }
            chosen[arg] = true;
        }
    }
    int q = 0;
    for (int j = 0; j < m; ++j) {
        if (!chosen[j]) continue;
        for (int ch = 0; ch < 3; ++ch) {
            const double base = centers[3 * j + ch];
            centers[3 * (m + q) + ch] = base + eps;
            centers[3 * j + ch] = base - eps;
        }
        ++q;
    }
}

// One block of any size (a multiple of 32, at most 1024 threads); `smem` holds
// 2 * kMapSlots + 2 * kSffMax words.  Requires n > K.
__device__ void sff_block(const uint32_t *keys, int64_t n, int K, uint64_t seed, int s0, double *centers,
                          uint32_t *smem)
{
    __shared__ unsigned long long s_red[32];
    __shared__ uint32_t s_cur;
    const int nt = blockDim.x;
    const uint32_t s = (uint32_t)(s0 < n ? s0 : n);
    FyMap m{smem, smem + kMapSlots, kMapSlots - 1};
    uint32_t *sub = smem + 2 * kMapSlots;   // kSffMax entries
    uint32_t *mind = sub + kSffMax;         // kSffMax entries
    clear_map(m.pos1, kMapSlots);
    __syncthreads();
    if (threadIdx.x == 0) fisher_yates((uint32_t)n, s, seed, 4, m, sub);
    __syncthreads();
    for (uint32_t i = s + threadIdx.x; i < kSffMax; i += nt) sub[i] = 0xFFFFFFFFu;
    __syncthreads();
    // bitonic sort of kSffMax entries, ascending
    for (int size = 2; size <= kSffMax; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < kSffMax; i += nt) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint32_t a = sub[i], b = sub[j];
                    if ((a > b) == up) {
                        sub[i] = b;
                        sub[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) s_cur = (uint32_t)below(rand64(seed, 5, 0), (uint64_t)s);
    __syncthreads();
    uint32_t cur = s_cur;
    if (threadIdx.x == 0) key_to_centre(centers, keys[sub[cur]]);
    for (int k = 1; k < K; ++k) {
        const uint32_t ck = keys[sub[cur]];
        unsigned long long best = 0ull;
        for (uint32_t i = threadIdx.x; i < s; i += nt) {
            const uint32_t d = key_dist2(keys[sub[i]], ck);
            const uint32_t md = (k == 1) ? d : min(mind[i], d);
            mind[i] = md;
            const unsigned long long packed = ((unsigned long long)md << 32) | (0xFFFFFFFFu - i);
            best = packed > best ? packed : best;
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long other = __shfl_down_sync(kSeedFull, best, o);
            best = other > best ? other : best;
        }
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = 0ull;
            for (int wv = 0; wv < nt / 32; ++wv) b = s_red[wv] > b ? s_red[wv] : b;
            s_cur = 0xFFFFFFFFu - (uint32_t)(b & 0xFFFFFFFFull);
            key_to_centre(centers + 3 * k, keys[sub[s_cur]]);
        }
        __syncthreads();
        cur = s_cur;
    }
}

// Warp-level: index of the element of rank `j` (0-based, in key order) among the
// unique colours whose class (channel value or cell) equals `cls`.
// The unique list is cut into `nchunks` (a multiple of 32) chunks of
// ceil(n / nchunks) colours; chunk_cnt[c * width + col] counts class `col` in chunk c.
__device__ int64_t warp_locate(const uint32_t *keys, int64_t n, const uint32_t *chunk_cnt, int nchunks, int width,
                               int col, uint32_t j, int mode, int ch)
{
    const int lane = threadIdx.x & 31;
    const int64_t len = (n + nchunks - 1) / nchunks;
    // chunk holding the element
    uint32_t run = 0;
    int cstar = nchunks - 1;
    for (int base = 0; base < nchunks; base += 32) {
        const uint32_t v = chunk_cnt[(size_t)(base + lane) * width + col];
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kSeedFull, x, o);
            if (lane >= o) x += y;
        }
        const unsigned bal = __ballot_sync(kSeedFull, run + x > j);
        if (bal) {
            const int l = __ffs(bal) - 1;
            cstar = base + l;
            run += __shfl_sync(kSeedFull, x, l) - __shfl_sync(kSeedFull, v, l);
            break;
        }
        run += __shfl_sync(kSeedFull, x, 31);
    }
    uint32_t r = j - run;
    const int64_t lo = (int64_t)cstar * len, hi = lo + len < n ? lo + len : n;
    for (int64_t base = lo; base < hi; base += 32) {
        const int64_t i = base + lane;
        bool match = false;
        if (i < hi) {
            const uint32_t key = keys[i];
            match = mode == 0 ? (int)((key >> (16 - 8 * ch)) & 255u) == col - ch * 256 : den_cell(key) == col;
        }
        const unsigned bal = __ballot_sync(kSeedFull, match);
        const uint32_t c = __popc(bal);
        if (r < c) {
            unsigned m = bal;
            for (uint32_t q = 0; q < r; ++q) m &= m - 1;
            return base + (__ffs(m) - 1);
        }
        r -= c;
    }
    return hi > 0 ? hi - 1 : 0;  // unreachable with consistent counts
}


// ---------------------------------------------------------------- VAR
// Channel of largest pixel-weighted variance, compared exactly as W S2 - S1^2
// (ties to the lower channel).
__device__ __forceinline__ int var_channel(unsigned long long w, const unsigned long long *s1,
                                           const unsigned long long *s2)
{
    const unsigned __int128 W = w;
    int ch = 0;
    unsigned __int128 best = 0;
    for (int c = 0; c < 3; ++c) {
        const unsigned __int128 a = s1[c], b = s2[c];
        const unsigned __int128 v = W * b - a * a;
        if (c == 0 || v > best) {
            best = v;
            ch = c;
        }
    }
    return ch;
}

// Warp-level: centre g is the middle element (rank floor((lo + hi - 1) / 2)) of
// group g = [g N' / K, (g + 1) N' / K) of the colours sorted by (channel value,
// key); gcnt[ch * 256 + v] counts the colours whose channel value is v.
__device__ void var_pick_warp(const uint32_t *keys, int64_t n, int K, int g, int ch, const uint32_t *chunk_cnt,
                              int nchunks, const uint32_t *gcnt, double *centers)
{
    const int lane = threadIdx.x & 31;
    const int64_t glo = (int64_t)g * n / K, ghi = (int64_t)(g + 1) * n / K;
    const uint32_t m = (uint32_t)((glo + ghi - 1) / 2);
    uint32_t run = 0;
    int v = 255;
    for (int base = 0; base < 256; base += 32) {
        const uint32_t cv = gcnt[ch * 256 + base + lane];
        uint32_t x = cv;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kSeedFull, x, o);
            if (lane >= o) x += y;
        }
        const unsigned bal = __ballot_sync(kSeedFull, run + x > m);
        if (bal) {
            const int l = __ffs(bal) - 1;
            v = base + l;
            run += __shfl_sync(kSeedFull, x, l) - __shfl_sync(kSeedFull, cv, l);
            break;
        }
        run += __shfl_sync(kSeedFull, x, 31);
    }
    const int64_t idx = warp_locate(keys, n, chunk_cnt, nchunks, 3 * 256, ch * 256 + v, m - run, 0, ch);
    if (lane == 0) key_to_centre(centers + 3 * g, keys[idx]);
}


// ---------------------------------------------------------------- WU (Section 3.3)
// Wu's greedy orthogonal bipartitioning.  Five moment arrays (W, S_R, S_G, S_B and
// Q = sum w |x|^2) over a 32^3 grid of cells, their 33^3 cumulative sums with a
// zero border (stored [grid point][moment]), and boxes [lo, hi) of cells whose
// moments are eight-corner differences of the cumulative sums (exact in 64-bit
// integers).  The FP64
// criterion and variance are evaluated with explicitly rounded operations in one
// fixed order: term = ((S_R^2 + S_G^2) + S_B^2) / W, criterion = term(a) +
// term(b), variance = Q - term; ties go to the lower box index, R before G before
// B, and the lower cut position.
struct WuMom {
    unsigned long long w, s[3], q;
};

struct WuBox {
    int8_t lo[3], hi[3];
};

__device__ __forceinline__ int wu_cell(uint32_t key)
{
    return (int)(((key >> 19) & 31u) * 1024u + ((key >> 11) & 31u) * 32u + ((key >> 3) & 31u));
}

__device__ __forceinline__ int wu_cidx(int r, int g, int b) { return (r * 33 + g) * 33 + b; }

// Moments of the cells [lo, hi) of a box from the cumulative moments cum[33^3][5]
// (the five moments of a grid point are adjacent).  Plain loads: the array is
// read-only while boxes are cut, and the corners that candidate cuts share stay
// in L1.
__device__ __forceinline__ WuMom wu_vol(const unsigned long long *cum, const int *lo, const int *hi)
{
    WuMom m;
    unsigned long long v[5];
    const unsigned long long *c000 = cum + 5 * (size_t)wu_cidx(lo[0], lo[1], lo[2]);
    const unsigned long long *c001 = cum + 5 * (size_t)wu_cidx(lo[0], lo[1], hi[2]);
    const unsigned long long *c010 = cum + 5 * (size_t)wu_cidx(lo[0], hi[1], lo[2]);
    const unsigned long long *c011 = cum + 5 * (size_t)wu_cidx(lo[0], hi[1], hi[2]);
    const unsigned long long *c100 = cum + 5 * (size_t)wu_cidx(hi[0], lo[1], lo[2]);
    const unsigned long long *c101 = cum + 5 * (size_t)wu_cidx(hi[0], lo[1], hi[2]);
    const unsigned long long *c110 = cum + 5 * (size_t)wu_cidx(hi[0], hi[1], lo[2]);
    const unsigned long long *c111 = cum + 5 * (size_t)wu_cidx(hi[0], hi[1], hi[2]);
#pragma unroll
    for (int j = 0; j < 5; ++j)
        v[j] = __ldcg(c111 + j) - __ldcg(c110 + j) - __ldcg(c101 + j) + __ldcg(c100 + j) - __ldcg(c011 + j) + __ldcg(c010 + j) + __ldcg(c001 + j) - __ldcg(c000 + j);
    m.w = v[0];
    m.s[0] = v[1];
    m.s[1] = v[2];
    m.s[2] = v[3];
    m.q = v[4];
    return m;
}

__device__ __forceinline__ double wu_term(const WuMom &m)
{
    const double sr = (double)m.s[0], sg = (double)m.s[1], sb = (double)m.s[2];
    return __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(sr, sr), __dmul_rn(sg, sg)), __dmul_rn(sb, sb)), (double)m.w);
}

__device__ __forceinline__ double wu_variance(const unsigned long long *cum, const WuBox &b)
{
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = b.lo[a];
        hi[a] = b.hi[a];
    }
    const int vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    if (vol <= 1) return 0.0;
    const WuMom m = wu_vol(cum, lo, hi);
    if (m.w == 0) return 0.0;
    return __dsub_rn((double)m.q, wu_term(m));
}

// Adds each colour's moments to its cell (cell[5][32^3], zero on entry); threads
// t of nt take colours t, t + nt, ...
__device__ void wu_accumulate(const uint32_t *keys, const uint32_t *w, int64_t n, unsigned long long *cell, int64_t t,
                              int64_t nt)
{
    for (int64_t i = t; i < n; i += nt) {
        const uint32_t key = keys[i];
        const unsigned long long wi = w[i];
        const unsigned long long r = key_r(key), g = key_g(key), b = key_b(key);
        const int c = wu_cell(key);
        atomicAdd(cell + c, wi);
        atomicAdd(cell + kWuCells + c, wi * r);
        atomicAdd(cell + 2 * kWuCells + c, wi * g);
        atomicAdd(cell + 3 * kWuCells + c, wi * b);
        atomicAdd(cell + 4 * kWuCells + c, wi * (r * r + g * g + b * b));
    }
}

// Cumulative sums cum[j][r][g][b] = sum of cell[j] over cells < (r, g, b) on every
// axis, with a zero border at index 0.  Step 0 copies the cells into the interior
// and zeroes the border; steps 1-3 take prefix sums along B, G and R, one line of
// 32 values per thread at a time (all 32 loaded before any is stored).  Threads t
// of nt; between steps every thread must see the previous step's stores.
__device__ __forceinline__ void wu_cum_copy(const unsigned long long *cell, unsigned long long *cum, int64_t t,
                                            int64_t nt)
{
    for (int64_t e = t; e < 5 * (int64_t)kWuCum; e += nt) {
        const int rgb = (int)(e / 5), j = (int)(e % 5);
        const int r = rgb / (33 * 33), g = (rgb / 33) % 33, b = rgb % 33;
        // the cells were filled by atomics (performed in L2): read them from L2
        cum[e] = (r && g && b) ? __ldcg(cell + (size_t)j * kWuCells + (r - 1) * 1024 + (g - 1) * 32 + (b - 1)) : 0ull;
    }
}

// step 1, 2, 3: lines along B, G, R
__device__ __forceinline__ void wu_cum_lines(unsigned long long *cum, int step, int64_t t, int64_t nt)
{
    const int st = step == 1 ? 1 : (step == 2 ? 33 : 33 * 33);
    for (int64_t l = t; l < 5 * 33 * 33; l += nt) {
        const int j = (int)(l / (33 * 33)), u = (int)(l % (33 * 33)), x = u / 33, y = u % 33;
        // the two coordinates other than the line's, each 0..32
        const int base = step == 1 ? (x * 33 + y) * 33 : (step == 2 ? x * 33 * 33 + y : x * 33 + y);
        unsigned long long *c = cum + 5 * (size_t)base + j;
        unsigned long long carry = 0ull;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned long long v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = __ldcg(c + 5 * (1 + 16 * h + i) * st);
            v[0] += carry;
#pragma unroll
            for (int i = 1; i < 16; ++i) v[i] += v[i - 1];
#pragma unroll
            for (int i = 0; i < 16; ++i) c[5 * (1 + 16 * h + i) * st] = v[i];
            carry = v[15];
        }
    }
}

// All four steps by one block (all its threads).  The moments written by other
// threads are read from L2 (__ldcg) throughout: through L1 the second and third
// steps were seen to read stale lines in a persistent kernel that runs many
// images on one SM.
__device__ void wu_cumulate_block(const unsigned long long *cell, unsigned long long *cum)
{
    wu_cum_copy(cell, cum, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int step = 1; step <= 3; ++step) {
        wu_cum_lines(cum, step, threadIdx.x, blockDim.x);
        __syncthreads();
    }
}

struct WuShared {
    WuBox box[kMaxK];
    WuMom mom[kMaxK];   // moments of each box
    WuMom half[96];     // each candidate cut's lower half
    double vv[kMaxK];
    double f[96], vh[96], vr[96];
    double wf[32];
    int wi[32];
    int nb, next, stop;
};

// Largest v with the lowest index among ties, over the lanes of a warp; returns
// (value, index) in every lane.  Lanes without a candidate pass index INT_MAX.
__device__ __forceinline__ void wu_warp_argmax(double &v, int &i)
{
    for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
}

// The greedy splits and the box means, by one block of 256 or more threads (a
// multiple of 32).  Every candidate cut (axis, position) is evaluated by its own
// thread, which also keeps the two halves' variances; the best cut and the next
// box to split are warp-level argmaxes (largest value, lowest index), so the
// choices are those of scanning candidates and boxes in order with a strict >.
// Requires n > K (the K >= N' case is handled by the caller).
__device__ void wu_split_block(const unsigned long long *cum, int K, double *centers, WuShared &sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        int lo[3] = {0, 0, 0}, hi[3] = {32, 32, 32};
        for (int a = 0; a < 3; ++a) {
            sh.box[0].lo[a] = 0;
            sh.box[0].hi[a] = 32;
        }
        sh.mom[0] = wu_vol(cum, lo, hi);
        sh.vv[0] = wu_variance(cum, sh.box[0]);
        sh.nb = 1;
        sh.next = 0;
        sh.stop = !(sh.vv[0] > 0.0) || K <= 1;
    }
    __syncthreads();
    while (!sh.stop) {
        const int nx = sh.next;
        if (tid < 96) {
            const int ax = tid / 32, p = sh.box[nx].lo[ax] + 1 + tid % 32;
            double f = -1.0, vh = 0.0, vr = 0.0;
            if (p < sh.box[nx].hi[ax]) {
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    lo[a] = sh.box[nx].lo[a];
                    hi[a] = sh.box[nx].hi[a];
                }
                const WuMom whole = sh.mom[nx];
                const int full = hi[ax];
                hi[ax] = p;
                const WuMom half = wu_vol(cum, lo, hi);
                sh.half[tid] = half;
                WuMom rest;
                rest.w = whole.w - half.w;
                for (int ch = 0; ch < 3; ++ch) rest.s[ch] = whole.s[ch] - half.s[ch];
                rest.q = whole.q - half.q;
                if (half.w != 0 && rest.w != 0) {
                    const double th = wu_term(half), tr = wu_term(rest);
                    f = __dadd_rn(th, tr);
                    // the halves' variances (0 for a single cell), as wu_variance gives them
                    const int other = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]) / (p - lo[ax]);
                    vh = other * (p - lo[ax]) > 1 ? __dsub_rn((double)half.q, th) : 0.0;
                    vr = other * (full - p) > 1 ? __dsub_rn((double)rest.q, tr) : 0.0;
                }
            }
            sh.f[tid] = f;
            sh.vh[tid] = vh;
            sh.vr[tid] = vr;
            double v = f;
            int i = f >= 0.0 ? tid : 0x7fffffff;
            wu_warp_argmax(v, i);
            if (lane == 0) {
                sh.wf[warp] = v;
                sh.wi[warp] = i;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double best = -1.0;
            int bt = -1;
            for (int q = 0; q < 3; ++q)
                if (sh.wi[q] != 0x7fffffff && sh.wf[q] > best) {
                    best = sh.wf[q];
                    bt = sh.wi[q];
                }
            if (bt < 0) {
                sh.vv[nx] = 0.0;
            } else {
                const int ax = bt / 32, p = sh.box[nx].lo[ax] + 1 + bt % 32;
                const int nb = sh.nb;
                sh.box[nb] = sh.box[nx];
                sh.box[nb].lo[ax] = (int8_t)p;
                sh.box[nx].hi[ax] = (int8_t)p;
                const WuMom h = sh.half[bt], whole = sh.mom[nx];
                WuMom rest;
                rest.w = whole.w - h.w;
                for (int ch = 0; ch < 3; ++ch) rest.s[ch] = whole.s[ch] - h.s[ch];
                rest.q = whole.q - h.q;
                sh.mom[nx] = h;
                sh.mom[nb] = rest;
                sh.vv[nx] = sh.vh[bt];
                sh.vv[nb] = sh.vr[bt];
                sh.nb = nb + 1;
            }
        }
        __syncthreads();
        // the next box: largest variance, lowest index
        const int nb = sh.nb;
        if (warp < (nb + 31) / 32) {
            const int k = tid;
            double v = k < nb ? sh.vv[k] : -1.0;
            int i = k < nb ? k : 0x7fffffff;
            wu_warp_argmax(v, i);
            if (lane == 0) {
                sh.wf[warp] = v;
                sh.wi[warp] = i;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double bv = sh.wf[0];
            int bi = sh.wi[0];
            for (int q = 1; q < (nb + 31) / 32; ++q)
                if (sh.wf[q] > bv) {
                    bv = sh.wf[q];
                    bi = sh.wi[q];
                }
            sh.next = bi;
            sh.stop = nb >= K || !(bv > 0.0);
        }
        __syncthreads();
    }
    const int nb = sh.nb;
    for (int k = tid; k < K; k += blockDim.x) {
        const WuMom m = sh.mom[k < nb ? k : nb - 1];
        for (int ch = 0; ch < 3; ++ch) centers[3 * k + ch] = __ddiv_rn((double)m.s[ch], (double)m.w);
    }
}

}  // namespace
}  // namespace kq
