// SC-Linear (Section 3.2, Algorithm 1): the subspace-collision method without
// an index.  For every query and subspace i the T points nearest to q in that
// subspace collide (ties by id); each point's SC-score counts its collisions
// (Definition 4); the C highest scores (ties by id) are re-ranked by exact
// squared distance and the k nearest returned.
//
// A batch of B queries runs as a pipeline of launches over a caller-provided
// workspace:
//   1. scl_dist_kernel    FP32 distance of every point to every query in every
//                         subspace (x_j - q_j, one fused multiply-add per
//                         dimension for the squared Euclidean distance, one
//                         addition of |x_j - q_j| for L1, in dimension order),
//                         stored [B][Ns][n];
//   2. scl_select_kernel  per (query, subspace), the exact T-th smallest key
//                         (distance bits, id): a radix select over the
//                         distance bits (11/11/10-bit digits, warp-aggregated
//                         shared-memory histograms), then, when the distance at
//                         the cut is shared by more points than still needed, a
//                         scan in id order finds the last colliding id;
//   3. scl_score_kernel   SC-scores (uint8) and each query's score histogram;
//   4. scl_cut_kernel     theta, the largest score with at least C points at or
//                         above it, and how many ties at theta are taken;
//   5. scl_tile_kernel    per 4096-id tile, the points above theta and at theta;
//      scl_scan_kernel    tile offsets (exclusive scans in id order);
//      scl_compact_kernel candidates: every point above theta and the
//                         lowest-id ties at theta;
//   6. scl_rerank_kernel  exact FP32 distances of the candidates, a radix
//                         select of the k-th smallest (distance, id) key, and
//                         the sorted top-k.
// Every decision that floating point takes (which points collide) is taken in
// FP32 in the order stated in 1, which is the order the CPU oracle's FP32 mode
// follows.
#include <cstring>

#include "suco_internal.cuh"

namespace suco {
namespace {

constexpr int SCL_TILE = 4096;     // ids per compaction tile
constexpr int SCL_QT = 32;         // queries per distance block

struct SclLayout {
    int64_t B = 0;                 // queries per batch
    size_t o_dist = 0, o_kappa = 0, o_score = 0, o_shist = 0, o_cut = 0, o_tcnt = 0, o_cands = 0, o_keys = 0;
    size_t bytes = 0;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

SclLayout scl_layout(const DeviceIndex* ix, int64_t B, int64_t C)
{
    SclLayout L;
    L.B = B;
    const int64_t n = ix->n, ntile = (n + SCL_TILE - 1) / SCL_TILE;
    size_t o = 0;
    L.o_dist = o;  // rows of ldn = n rounded up to 4 floats: 16-byte aligned
    o = align256(o + (size_t)B * ix->Ns * ((n + 3) & ~int64_t(3)) * 4);
    L.o_kappa = o;
    o = align256(o + (size_t)B * ix->Ns * 8);
    L.o_score = o;
    o = align256(o + (size_t)B * n);
    L.o_shist = o;
    o = align256(o + (size_t)B * 64 * 4);
    L.o_cut = o;
    o = align256(o + (size_t)B * 4 * 4);
    L.o_tcnt = o;
    o = align256(o + (size_t)B * ntile * 2 * 4);
    L.o_cands = o;
    o = align256(o + (size_t)B * C * 4);
    L.o_keys = o;
    o = align256(o + (size_t)B * C * 8);
    L.bytes = o;
    return L;
}

// Two FP32 lanes in one 64-bit register: element-wise subtract, fused
// multiply-add and add, each rounded to nearest even like the scalar
// operation; |x| of both lanes by clearing the sign bits.
__device__ __forceinline__ unsigned long long p2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long p2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long p2_add(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// 1. distances.  Block: 256 points x SCL_QT queries (grid.y picks the query
// group); per subspace the group's query slices are staged in shared memory
// dimension-major ([j][query], zero for missing queries), and every thread
// keeps one accumulator per query, two queries per 64-bit register: for each
// dimension in order it forms (x_j, x_j) once and updates the pairs with
// sub.f32x2 and fma.f32x2 (or the absolute value and add.f32x2 for L1).
// Each lane of a pair sees the scalar operations in the scalar order, so the
// distances are bit-identical to a one-query-at-a-time loop.
template <int MET>
__global__ void __launch_bounds__(256, 2) scl_dist_kernel(const float* __restrict__ X, int64_t ld, int64_t n, int32_t d,
                                                       int32_t Ns, int32_t sub_s, const float* __restrict__ Q, int64_t nq,
                                                       float* __restrict__ dist, int64_t ldn,
                                                       const int32_t* __restrict__ qperm)
{
    constexpr int NP = SCL_QT / 2;               // query pairs
    extern __shared__ __align__(16) float qs[];  // [maxlen][SCL_QT]
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t q0 = (int64_t)blockIdx.y * SCL_QT;
    const int nqg = (int)(nq - q0 < SCL_QT ? nq - q0 : SCL_QT);
    for (int i = 0; i < Ns; ++i) {
        const int off = i * sub_s, len = (i == Ns - 1) ? d - (Ns - 1) * sub_s : sub_s;
        __syncthreads();
        for (int t = threadIdx.x; t < SCL_QT * len; t += 256) {
            const int j = t / SCL_QT, qq = t - j * SCL_QT;
            qs[t] = qq < nqg ? query_col(Q + (q0 + qq) * d, qperm, off + j) : 0.f;
        }
        __syncthreads();
        if (p >= n) continue;
        unsigned long long acc[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) acc[m] = 0ull;  // (+0, +0)
        const float* xr = X + p * ld + off;
        const ulonglong2* q2 = reinterpret_cast<const ulonglong2*>(qs);
        for (int j = 0; j < len; ++j) {
            const unsigned u = __float_as_uint(__ldg(xr + j));
            const unsigned long long xx = (unsigned long long)u | ((unsigned long long)u << 32);
#pragma unroll
            for (int m = 0; m < NP; m += 2) {
                const ulonglong2 qv = q2[j * (NP / 2) + m / 2];  // queries 2m .. 2m+3 of dimension j
                const unsigned long long d0 = p2_sub(xx, qv.x), d1 = p2_sub(xx, qv.y);
                if constexpr (MET == SUCO_METRIC_L1) {
                    acc[m] = p2_add(acc[m], d0 & 0x7fffffff7fffffffull);
                    acc[m + 1] = p2_add(acc[m + 1], d1 & 0x7fffffff7fffffffull);
                } else {
                    acc[m] = p2_fma(d0, d0, acc[m]);
                    acc[m + 1] = p2_fma(d1, d1, acc[m + 1]);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const int qa = 2 * m, qb = 2 * m + 1;
            if (qa < nqg) dist[((q0 + qa) * Ns + i) * ldn + p] = __uint_as_float((unsigned)acc[m]);
            if (qb < nqg) dist[((q0 + qb) * Ns + i) * ldn + p] = __uint_as_float((unsigned)(acc[m] >> 32));
        }
    }
}

// Exclusive sum over the 1024 threads of a block (wtmp: 33 words); *tot gets
// the total.  Ends with a barrier, so wtmp can be reused at once.
__device__ __forceinline__ uint32_t block_scan_pairs_1024(uint32_t v, uint32_t* wtmp, uint32_t* tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtmp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = wtmp[lane];
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        wtmp[lane] = ti - t;
        if (lane == 31) wtmp[32] = ti;
    }
    __syncthreads();
    const uint32_t r = wtmp[w] + incl - v;
    *tot = wtmp[32];
    __syncthreads();
    return r;
}

// Adds 1 to hist[bin] for every lane with `valid`, one atomic per distinct
// bin in the warp (the lanes of a warp often share a bin).  Every lane of the
// warp calls it together.
__device__ __forceinline__ void hist_add(uint32_t* hist, uint32_t bin, bool valid)
{
    const uint32_t same = __match_any_sync(0xffffffffu, valid ? bin : 0xffffffffu);
    if (valid && (threadIdx.x & 31) == (uint32_t)(__ffs(same) - 1)) atomicAdd(&hist[bin], (uint32_t)__popc(same));
}

// In a block of NT threads: the bin of hist[0, nb) where the running count
// crosses need (exclusive < need <= inclusive); returns the bin, *below = the
// count before it, *inbin = its count.
template <int NT>
__device__ uint32_t block_find_bin(const uint32_t* hist, int nb, uint32_t need, uint32_t* below, uint32_t* inbin,
                                   uint32_t* wtmp /*[NT/32 + 4]*/)
{
    const int per = (nb + NT - 1) / NT;
    const int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int j = 0; j < per; ++j) s += b0 + j < nb ? hist[b0 + j] : 0u;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtmp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = lane < NT / 32 ? wtmp[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < NT / 32) wtmp[lane] = ti - t;
    }
    __syncthreads();
    uint32_t run = wtmp[w] + incl - s;
    __syncthreads();
    if (run < need && run + s >= need) {
        for (int j = 0; j < per; ++j) {
            const uint32_t v = b0 + j < nb ? hist[b0 + j] : 0u;
            if (run + v >= need) {
                wtmp[NT / 32] = (uint32_t)(b0 + j);
                wtmp[NT / 32 + 1] = run;
                wtmp[NT / 32 + 2] = v;
                break;
            }
            run += v;
        }
    }
    __syncthreads();
    const uint32_t bin = wtmp[NT / 32];
    *below = wtmp[NT / 32 + 1];
    *inbin = wtmp[NT / 32 + 2];
    __syncthreads();
    return bin;
}

// 2. exact T-th smallest key (distance bits, id) of one (query, subspace):
// grid = B * Ns blocks of 1024 threads.  Non-negative FP32 distances order as
// their bit patterns, so three radix passes over the bits (11, 11 and 10 bits
// from the top) find the T-th smallest distance d* and how many points at d*
// are still needed; when fewer than all of them are, a scan in id order finds
// the id of the last one taken.  kappa[(b*Ns+i)] = {d* bits, last id}: a point
// collides iff dist < d*, or dist == d* and id <= last id.
constexpr int SEL_NT = 1024;

__global__ void __launch_bounds__(SEL_NT) scl_select_kernel(const float* __restrict__ dist, int64_t n, int64_t ldn,
                                                            uint32_t T, uint32_t* __restrict__ kappa)
{
    __shared__ uint32_t hist[2048];
    __shared__ uint32_t wtmp[SEL_NT / 32 + 4];
    __shared__ uint32_t found;
    const uint32_t* v = reinterpret_cast<const uint32_t*>(dist) + (int64_t)blockIdx.x * ldn;  // 16-byte aligned
    uint32_t prefix = 0, need = T, inbin = 0;
    const int shifts[3] = {21, 10, 0}, widths[3] = {11, 11, 10};
    for (int pass = 0; pass < 3; ++pass) {
        const int sh = shifts[pass], nb = 1 << widths[pass], hi = sh + widths[pass];
        for (int t = threadIdx.x; t < 2048; t += SEL_NT) hist[t] = 0u;
        __syncthreads();
        const uint32_t want = hi >= 32 ? 0u : prefix >> hi;
        // four consecutive values per thread (one 16-byte load); block-uniform
        // trip count: hist_add takes whole warps
        for (int64_t p0 = 0; p0 < n; p0 += 4 * SEL_NT) {
            const int64_t p = p0 + 4 * threadIdx.x;
            uint4 x4 = make_uint4(0u, 0u, 0u, 0u);
            if (p < n) x4 = *reinterpret_cast<const uint4*>(v + p);  // p + 3 < ldn
            const uint32_t xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                hist_add(hist, (xs[e] >> sh) & (uint32_t)(nb - 1),
                         p + e < n && (hi >= 32 ? 0u : xs[e] >> hi) == want);
        }
        __syncthreads();
        uint32_t below;
        const uint32_t bin = block_find_bin<SEL_NT>(hist, nb, need, &below, &inbin, wtmp);
        prefix |= bin << sh;
        need -= below;
    }
    // prefix = d*; need in [1, inbin] points at d* collide, the lowest ids first:
    // a scan in id order, eight consecutive ids per thread per round
    uint32_t last = 0xffffffffu;
    if (need < inbin) {
        uint32_t run = 0;
        for (int64_t base = 0; base < n; base += 8 * SEL_NT) {  // block-uniform
            const int64_t p = base + 8 * threadIdx.x;
            uint32_t xs[8];
            uint4 a4 = make_uint4(0u, 0u, 0u, 0u), b4 = a4;
            if (p < n) a4 = *reinterpret_cast<const uint4*>(v + p);          // p + 3 < ldn
            if (p + 4 < n) b4 = *reinterpret_cast<const uint4*>(v + p + 4);  // p + 7 < ldn
            xs[0] = a4.x; xs[1] = a4.y; xs[2] = a4.z; xs[3] = a4.w;
            xs[4] = b4.x; xs[5] = b4.y; xs[6] = b4.z; xs[7] = b4.w;
            uint32_t c = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) c += (p + e < n && xs[e] == prefix) ? 1u : 0u;
            uint32_t tot;
            const uint32_t ex = block_scan_pairs_1024(c, wtmp, &tot);
            if (run + ex < need && run + ex + c >= need) {  // the need-th tie is among this thread's eight
                uint32_t r = run + ex;
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (p + e < n && xs[e] == prefix && ++r == need) found = (uint32_t)(p + e);
            }
            __syncthreads();
            if (run + tot >= need) {
                last = found;
                break;
            }
            run += tot;
        }
    }
    if (threadIdx.x == 0) {
        kappa[2 * blockIdx.x] = prefix;
        kappa[2 * blockIdx.x + 1] = last;
    }
}

// 3. SC-scores and each query's score histogram: grid (point blocks, B)
__global__ void __launch_bounds__(256) scl_score_kernel(const float* __restrict__ dist, int64_t n, int64_t ldn,
                                                        int32_t Ns,
                                                        const uint32_t* __restrict__ kappa, uint8_t* __restrict__ score,
                                                        uint32_t* __restrict__ shist)
{
    __shared__ uint32_t h[64];
    const int64_t b = blockIdx.y;
    if (threadIdx.x < 64) h[threadIdx.x] = 0u;
    __syncthreads();
    const uint32_t* v = reinterpret_cast<const uint32_t*>(dist) + b * Ns * ldn;
    for (int64_t p0 = (int64_t)blockIdx.x * 256; p0 < n; p0 += (int64_t)gridDim.x * 256) {
        const int64_t p = p0 + threadIdx.x;  // block-uniform trip count: hist_add takes whole warps
        uint32_t sc = 0;
        if (p < n) {
            for (int i = 0; i < Ns; ++i) {
                const uint32_t x = v[(int64_t)i * ldn + p];
                const uint32_t ds = kappa[2 * (b * Ns + i)], last = kappa[2 * (b * Ns + i) + 1];
                sc += (x < ds || (x == ds && (uint32_t)p <= last)) ? 1u : 0u;
            }
            score[b * n + p] = (uint8_t)sc;
        }
        hist_add(h, sc, p < n);
    }
    __syncthreads();
    if (threadIdx.x <= (unsigned)Ns && h[threadIdx.x]) atomicAdd(&shist[b * 64 + threadIdx.x], h[threadIdx.x]);
}

// 4. per query: theta = the largest score s with #{score >= s} >= C; the
// points above theta all stay, need_eq = C - #{score > theta} ties at theta
// stay (the lowest ids).  cut[b] = {theta, need_eq, #{score > theta}}.
__global__ void scl_cut_kernel(const uint32_t* __restrict__ shist, int32_t Ns, uint32_t C, uint32_t* __restrict__ cut)
{
    const int64_t b = blockIdx.x;
    if (threadIdx.x != 0) return;
    uint32_t above = 0;
    for (int s = Ns; s >= 0; --s) {
        const uint32_t c = shist[b * 64 + s];
        if (above + c >= C) {
            cut[4 * b] = (uint32_t)s;
            cut[4 * b + 1] = C - above;
            cut[4 * b + 2] = above;
            return;
        }
        above += c;
    }
    cut[4 * b] = 0;  // unreachable: every point has a score >= 0 and C <= n
    cut[4 * b + 1] = 0;
    cut[4 * b + 2] = above;
}

// Exclusive scan over a block of NT threads of (gt << 16 | eq) pairs (each
// count < 2^16); *tot gets the block's total.
template <int NT>
__device__ __forceinline__ uint32_t block_scan_pairs(uint32_t v, uint32_t* wtmp, uint32_t* tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtmp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = lane < NT / 32 ? wtmp[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        wtmp[lane] = ti - t;
        if (lane == 31) wtmp[32] = ti;
    }
    __syncthreads();
    const uint32_t r = wtmp[w] + incl - v;
    *tot = wtmp[32];
    __syncthreads();
    return r;
}

// 5a. per tile of SCL_TILE ids: points above theta and at theta
__global__ void __launch_bounds__(256) scl_tile_kernel(const uint8_t* __restrict__ score, int64_t n,
                                                       const uint32_t* __restrict__ cut, uint32_t* __restrict__ tcnt)
{
    __shared__ uint32_t wtmp[40];
    const int64_t b = blockIdx.y, ntile = gridDim.x;
    const uint32_t theta = cut[4 * b];
    uint32_t v = 0;
    for (int j = 0; j < SCL_TILE / 256; ++j) {
        const int64_t p = (int64_t)blockIdx.x * SCL_TILE + j * 256 + threadIdx.x;
        if (p < n) {
            const uint32_t sc = score[b * n + p];
            v += (sc > theta ? 1u << 16 : 0u) + (sc == theta ? 1u : 0u);
        }
    }
    uint32_t tot;
    block_scan_pairs<256>(v, wtmp, &tot);
    if (threadIdx.x == 0) {
        tcnt[2 * (b * ntile + blockIdx.x)] = tot >> 16;
        tcnt[2 * (b * ntile + blockIdx.x) + 1] = tot & 0xffffu;
    }
}

// 5b. tile offsets: exclusive scans over the tiles, in id order (grid = B)
__global__ void __launch_bounds__(1024) scl_scan_kernel(uint32_t* __restrict__ tcnt, int64_t ntile)
{
    __shared__ uint32_t wtmp[40];
    const int64_t b = blockIdx.x;
    uint32_t cg = 0, ce = 0;  // carries
    for (int64_t t0 = 0; t0 < ntile; t0 += 1024) {
        const int64_t t = t0 + threadIdx.x;
        const uint32_t g = t < ntile ? tcnt[2 * (b * ntile + t)] : 0u;
        const uint32_t e = t < ntile ? tcnt[2 * (b * ntile + t) + 1] : 0u;
        uint32_t tg, te;
        const uint32_t xg = block_scan_pairs<1024>(g, wtmp, &tg);  // counts below 2^32: one scan each
        const uint32_t xe = block_scan_pairs<1024>(e, wtmp, &te);
        if (t < ntile) {
            tcnt[2 * (b * ntile + t)] = cg + xg;
            tcnt[2 * (b * ntile + t) + 1] = ce + xe;
        }
        cg += tg;
        ce += te;
    }
}

// 5c. candidates: ids above theta at [0, #above), the lowest-id ties at
// theta at [#above, C); rounds of 256 consecutive ids keep the id order
__global__ void __launch_bounds__(256) scl_compact_kernel(const uint8_t* __restrict__ score, int64_t n,
                                                          const uint32_t* __restrict__ cut,
                                                          const uint32_t* __restrict__ toff, int64_t C,
                                                          int32_t* __restrict__ cands)
{
    __shared__ uint32_t wtmp[40];
    const int64_t b = blockIdx.y, ntile = gridDim.x;
    const uint32_t theta = cut[4 * b], need_eq = cut[4 * b + 1], above = cut[4 * b + 2];
    uint32_t gbase = toff[2 * (b * ntile + blockIdx.x)], ebase = toff[2 * (b * ntile + blockIdx.x) + 1];
    for (int j = 0; j < SCL_TILE / 256; ++j) {
        const int64_t p = (int64_t)blockIdx.x * SCL_TILE + j * 256 + threadIdx.x;
        const uint32_t sc = p < n ? score[b * n + p] : 0u;
        const bool gt = p < n && sc > theta, eq = p < n && sc == theta;
        uint32_t tot;
        const uint32_t x = block_scan_pairs<256>((gt ? 1u << 16 : 0u) | (eq ? 1u : 0u), wtmp, &tot);
        if (gt) {
            const uint32_t pos = gbase + (x >> 16);
            if (pos < above) cands[b * C + pos] = (int32_t)p;
        } else if (eq) {
            const uint32_t r = ebase + (x & 0xffffu);
            if (r < need_eq) cands[b * C + above + r] = (int32_t)p;
        }
        gbase += tot >> 16;
        ebase += tot & 0xffffu;
    }
}

// 6. exact re-rank of one query's C candidates (grid = B, 512 threads): FP32
// squared distances (8 lanes per row, 16-byte chunks, then a butterfly over
// the 8 lanes) into keys (distance bits << 32 | id), a radix select of the
// k-th smallest key over 8-bit digits, then the keys up to it sorted by rank.
constexpr int RR_NT = 512;

__global__ void __launch_bounds__(RR_NT) scl_rerank_kernel(const float* __restrict__ X, int64_t ld, const float* __restrict__ Q,
                                                           int32_t d, const int32_t* __restrict__ cands, int64_t C,
                                                           int32_t k, unsigned long long* __restrict__ keys,
                                                           int32_t* __restrict__ out_ids, float* __restrict__ out_dist,
                                                           const int32_t* __restrict__ qperm, int metric)
{
    __shared__ uint32_t hist[256];
    __shared__ uint32_t wtmp[RR_NT / 32 + 4];
    __shared__ unsigned long long best[256];
    __shared__ uint32_t nbest;
    extern __shared__ float4 qsm[];  // [ld / 4]
    const int64_t b = blockIdx.x;
    const int ld4 = (int)(ld / 4);
    for (int c = threadIdx.x; c < ld4; c += RR_NT) {
        float4 v;
        v.x = 4 * c + 0 < d ? query_col(Q + b * d, qperm, 4 * c + 0) : 0.f;
        v.y = 4 * c + 1 < d ? query_col(Q + b * d, qperm, 4 * c + 1) : 0.f;
        v.z = 4 * c + 2 < d ? query_col(Q + b * d, qperm, 4 * c + 2) : 0.f;
        v.w = 4 * c + 3 < d ? query_col(Q + b * d, qperm, 4 * c + 3) : 0.f;
        qsm[c] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane >> 3, gl = lane & 7;
    const float4* X4 = reinterpret_cast<const float4*>(X);
    unsigned long long* kb = keys + b * C;
    for (int64_t r0 = (int64_t)warp * 4; r0 < C; r0 += (RR_NT / 32) * 4) {
        const int64_t r = r0 + grp;
        const int32_t id = r < C ? cands[b * C + r] : 0;
        float acc = 0.f;
        if (r < C)
            for (int c = gl; c < ld4; c += 8) {
                const float4 x = __ldg(X4 + (int64_t)id * ld4 + c), q = qsm[c];
                const float df[4] = {__fsub_rn(x.x, q.x), __fsub_rn(x.y, q.y), __fsub_rn(x.z, q.z), __fsub_rn(x.w, q.w)};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    acc = metric == SUCO_METRIC_L1 ? __fadd_rn(acc, fabsf(df[e])) : __fmaf_rn(df[e], df[e], acc);
            }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if (r < C && gl == 0) kb[r] = ((unsigned long long)__float_as_uint(acc) << 32) | (uint32_t)id;
    }
    __syncthreads();
    // the k-th smallest key (keys are unique: ids are)
    const uint32_t want = (uint32_t)((int64_t)k < C ? (int64_t)k : C);
    unsigned long long prefix = 0ull;
    uint32_t need = want;
    for (int pass = 0; pass < 8 && want > 0; ++pass) {
        const int sh = 56 - 8 * pass;
        for (int t = threadIdx.x; t < 256; t += RR_NT) hist[t] = 0u;
        __syncthreads();
        for (int64_t j0 = 0; j0 < C; j0 += RR_NT) {
            const int64_t j = j0 + threadIdx.x;
            const unsigned long long x = j < C ? kb[j] : 0ull;
            const bool match = j < C && (sh == 56 || (x >> (sh + 8)) == (prefix >> (sh + 8)));
            hist_add(hist, (uint32_t)(x >> sh) & 255u, match);
        }
        __syncthreads();
        uint32_t below, inbin;
        const uint32_t bin = block_find_bin<RR_NT>(hist, 256, need, &below, &inbin, wtmp);
        prefix |= (unsigned long long)bin << sh;
        need -= below;
    }
    if (threadIdx.x == 0) nbest = 0u;
    __syncthreads();
    for (int64_t j0 = 0; j0 < C && want > 0; j0 += RR_NT) {
        const int64_t j = j0 + threadIdx.x;
        if (j < C && kb[j] <= prefix) best[atomicAdd(&nbest, 1u)] = kb[j];
    }
    __syncthreads();
    const uint32_t nb = nbest;  // == want
    for (uint32_t t = threadIdx.x; t < (uint32_t)k; t += RR_NT) {
        if (t < nb) {
            const unsigned long long v = best[t];
            uint32_t rank = 0;
            for (uint32_t j = 0; j < nb; ++j) rank += best[j] < v ? 1u : 0u;
            out_ids[b * k + rank] = (int32_t)(uint32_t)(v & 0xffffffffu);
            out_dist[b * k + rank] = __uint_as_float((uint32_t)(v >> 32));
        } else {
            out_ids[b * k + t] = -1;
            out_dist[b * k + t] = __int_as_float(0x7f800000);
        }
    }
}

}  // namespace

namespace {

int sc_linear_chunk(const DeviceIndex* ix, const float* Q, int64_t bq, uint32_t T, int64_t C, int32_t k,
                    const SclLayout& L, char* ws, int32_t* ids, float* dist_out, uint8_t* dbg_scores,
                    int32_t* dbg_cands, cudaStream_t st)
{
    const int64_t n = ix->n, ntile = (n + SCL_TILE - 1) / SCL_TILE, ldn = (n + 3) & ~int64_t(3);
    const int Ns = ix->Ns;
    float* dist = reinterpret_cast<float*>(ws + L.o_dist);
    uint32_t* kappa = reinterpret_cast<uint32_t*>(ws + L.o_kappa);
    uint8_t* score = reinterpret_cast<uint8_t*>(ws + L.o_score);
    uint32_t* shist = reinterpret_cast<uint32_t*>(ws + L.o_shist);
    uint32_t* cut = reinterpret_cast<uint32_t*>(ws + L.o_cut);
    uint32_t* tcnt = reinterpret_cast<uint32_t*>(ws + L.o_tcnt);
    int32_t* cands = reinterpret_cast<int32_t*>(ws + L.o_cands);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(ws + L.o_keys);
    const int maxlen = ix->d - (Ns - 1) * ix->sub_s;
    const size_t dsmem = (size_t)SCL_QT * maxlen * 4;
    const dim3 dgrid((unsigned)((n + 255) / 256), (unsigned)((bq + SCL_QT - 1) / SCL_QT));
    if (ix->metric == SUCO_METRIC_L1) {
        if (dsmem > 48 * 1024)
            SUCO_CUDA_TRY(cudaFuncSetAttribute(scl_dist_kernel<SUCO_METRIC_L1>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
        scl_dist_kernel<SUCO_METRIC_L1><<<dgrid, 256, dsmem, st>>>(ix->X, ix->ld, n, ix->d, Ns, ix->sub_s, Q, bq, dist,
                                                                  ldn, ix->dperm);
    } else {
        if (dsmem > 48 * 1024)
            SUCO_CUDA_TRY(cudaFuncSetAttribute(scl_dist_kernel<SUCO_METRIC_L2>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
        scl_dist_kernel<SUCO_METRIC_L2><<<dgrid, 256, dsmem, st>>>(ix->X, ix->ld, n, ix->d, Ns, ix->sub_s, Q, bq, dist,
                                                                  ldn, ix->dperm);
    }
    SUCO_LAUNCH_CHECK("scl_dist_kernel");
    scl_select_kernel<<<(unsigned)(bq * Ns), SEL_NT, 0, st>>>(dist, n, ldn, T, kappa);
    SUCO_LAUNCH_CHECK("scl_select_kernel");
    SUCO_CUDA_TRY(cudaMemsetAsync(shist, 0, (size_t)bq * 64 * 4, st));
    const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
    scl_score_kernel<<<dim3(gx, (unsigned)bq), 256, 0, st>>>(dist, n, ldn, Ns, kappa, score, shist);
    SUCO_LAUNCH_CHECK("scl_score_kernel");
    scl_cut_kernel<<<(unsigned)bq, 32, 0, st>>>(shist, Ns, (uint32_t)C, cut);
    SUCO_LAUNCH_CHECK("scl_cut_kernel");
    scl_tile_kernel<<<dim3((unsigned)ntile, (unsigned)bq), 256, 0, st>>>(score, n, cut, tcnt);
    SUCO_LAUNCH_CHECK("scl_tile_kernel");
    scl_scan_kernel<<<(unsigned)bq, 1024, 0, st>>>(tcnt, ntile);
    SUCO_LAUNCH_CHECK("scl_scan_kernel");
    scl_compact_kernel<<<dim3((unsigned)ntile, (unsigned)bq), 256, 0, st>>>(score, n, cut, tcnt, C, cands);
    SUCO_LAUNCH_CHECK("scl_compact_kernel");
    if ((size_t)ix->ld * 4 > 48 * 1024)
        SUCO_CUDA_TRY(cudaFuncSetAttribute(scl_rerank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(ix->ld * 4)));
    scl_rerank_kernel<<<(unsigned)bq, RR_NT, (size_t)ix->ld * 4, st>>>(ix->X, ix->ld, Q, ix->d, cands, C, k, keys,
                                                                       ids, dist_out, ix->dperm, ix->metric);
    SUCO_LAUNCH_CHECK("scl_rerank_kernel");
    if (dbg_scores)
        SUCO_CUDA_TRY(cudaMemcpyAsync(dbg_scores, score, (size_t)bq * n, cudaMemcpyDeviceToDevice, st));
    if (dbg_cands)
        SUCO_CUDA_TRY(cudaMemcpyAsync(dbg_cands, cands, (size_t)bq * C * 4, cudaMemcpyDeviceToDevice, st));
    return SUCO_OK;
}

int sc_linear_checks(const suco_index* index, int32_t k, double alpha, double beta)
{
    if (!index) return fail(SUCO_EINVAL, "index is NULL");
    if (k < 1 || k > 256) return fail(SUCO_EINVAL, "k=%d must be in [1, 256]", k);
    if (!(alpha > 0.0 && alpha <= 1.0)) return fail(SUCO_EINVAL, "alpha=%g must be in (0, 1]", alpha);
    if (!(beta > 0.0 && beta <= 1.0)) return fail(SUCO_EINVAL, "beta=%g must be in (0, 1]", beta);
    const DeviceIndex& ix = index->ix;
    if (ix.Ns > 63) return fail(SUCO_EUNSUPPORTED, "SC-Linear scores need Ns < 64");
    const int maxlen = ix.d - (ix.Ns - 1) * ix.sub_s;
    if ((size_t)ix.ld * 4 > 200 * 1024)
        return fail(SUCO_EUNSUPPORTED, "SC-Linear stages a query of %d dims in shared memory: too long", ix.d);
    if ((size_t)SCL_QT * maxlen * 4 > 200 * 1024)
        return fail(SUCO_EUNSUPPORTED, "SC-Linear stages %d query slices of %d dims in shared memory: too long", SCL_QT,
                    maxlen);
    return SUCO_OK;
}

}  // namespace
}  // namespace suco

using namespace suco;

extern "C" int suco_sc_linear_workspace_size(const suco_index* index, int64_t batch, int32_t k, double beta,
                                             size_t* bytes)
{
    clear_error();
    int rc = sc_linear_checks(index, k, 0.5, beta);
    if (rc) return rc;
    if (!bytes || batch < 1) return fail(SUCO_EINVAL, "bytes must not be NULL and batch must be >= 1");
    int64_t T = 0, C = 0;
    thresholds(index->ix.n, 0.5, beta, k, &T, &C);
    *bytes = scl_layout(&index->ix, batch, C).bytes;
    return SUCO_OK;
}

extern "C" int suco_sc_linear(const suco_index* index, const float* queries, int64_t nq, int32_t k, double alpha,
                              double beta, void* workspace, size_t workspace_bytes, int32_t* out_ids, float* out_dist,
                              uint8_t* dbg_scores, int32_t* dbg_cands, void* stream)
{
    clear_error();
    int rc = sc_linear_checks(index, k, alpha, beta);
    if (rc) return rc;
    if (nq < 0) return fail(SUCO_EINVAL, "nq=%lld is negative", (long long)nq);
    if (nq == 0) return SUCO_OK;
    if (!queries || !out_ids || !out_dist || !workspace)
        return fail(SUCO_EINVAL, "queries, workspace, out_ids and out_dist must not be NULL");
    const DeviceIndex* ix = &index->ix;
    int64_t T = 0, C = 0;
    thresholds(ix->n, alpha, beta, k, &T, &C);
    // the largest batch whose workspace fits (the layout grows with the batch)
    int64_t lo = 0, hi = std::min<int64_t>(nq, 65535);
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (scl_layout(ix, mid, C).bytes <= workspace_bytes) lo = mid; else hi = mid - 1;
    }
    if (lo < 1)
        return fail(SUCO_EINVAL, "workspace of %zu bytes is below the %zu bytes of one query", workspace_bytes,
                    scl_layout(ix, 1, C).bytes);
    const SclLayout L = scl_layout(ix, lo, C);
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < nq; c0 += lo) {
        const int64_t bq = std::min<int64_t>(lo, nq - c0);
        rc = sc_linear_chunk(ix, queries + c0 * ix->d, bq, (uint32_t)T, C, k, L, static_cast<char*>(workspace),
                             out_ids + c0 * k, out_dist + c0 * k, dbg_scores ? dbg_scores + c0 * ix->n : nullptr,
                             dbg_cands ? dbg_cands + c0 * C : nullptr, st);
        if (rc) return rc;
    }
    return SUCO_OK;
}
