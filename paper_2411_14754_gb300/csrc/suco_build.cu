// Index construction (Section 4.1, Algorithm 2) on the GPU:
//   K-means per half-subspace (Lloyd iterations) and the inverted multi-index
//   (IMI) of every subspace as a CSR of ids grouped by cell.
//
// K-means details the paper leaves open (Algorithm 2 only calls "Kmeans"):
// initial centroids are given point ids; assignments take the index's
// distance (squared Euclidean, or L1 for an L1 index) and updates the member
// means; an empty cluster keeps its centroid;
// argmin ties go to the lowest centroid index; the final assignment that
// defines the IMI is taken against the final centroids.  Centroid sums are
// accumulated in 64-bit fixed point so that the build is bitwise
// deterministic regardless of the order of the atomic additions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "suco_internal.cuh"

namespace suco {
namespace {

__global__ void init_centroids_kernel(const float* __restrict__ X, int64_t ld, int32_t d, int32_t Ns, int32_t sub_s,
                                      int32_t sqrtK, int32_t hmax, const int64_t* __restrict__ ids,
                                      float* __restrict__ cent)
{
    const int ih = blockIdx.y;
    int32_t off, len;
    half_dims(d, Ns, sub_s, ih >> 1, ih & 1, &off, &len);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < sqrtK * hmax; t += gridDim.x * blockDim.x) {
        const int a = t / hmax, j = t - a * hmax;
        float v = 0.f;
        if (j < len) v = X[ids[(int64_t)ih * sqrtK + a] * ld + off + j];
        cent[((int64_t)ih * sqrtK + a) * hmax + j] = v;
    }
}

// Largest |x| of each of the first H half-subspaces, as float bits
// (monotone for x >= 0).  Thread c of a block reads column c of the block's
// rows, so a warp reads consecutive columns of one row (coalesced).
__global__ void maxabs_kernel(const float* __restrict__ X, int64_t ld, int64_t n, int32_t d, int32_t Ns, int32_t sub_s,
                              int32_t H, unsigned* __restrict__ out)
{
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        const int i = min(c / sub_s, Ns - 1);
        const int slen = (i == Ns - 1) ? d - (Ns - 1) * sub_s : sub_s;
        const int ih = 2 * i + ((c - i * sub_s) >= slen / 2 ? 1 : 0);
        if (ih >= H) continue;
        float m = 0.f;
        for (int64_t p = blockIdx.x; p < n; p += gridDim.x) m = fmaxf(m, fabsf(X[p * ld + c]));
        atomicMax(out + ih, __float_as_uint(m));
    }
}

// One dimension's term of the index's distance, accumulated in FP32:
// squared Euclidean by one fused multiply-add, L1 by one addition.
__device__ __forceinline__ float dist_term(float acc, float df, int metric)
{
    return metric == SUCO_METRIC_L1 ? __fadd_rn(acc, fabsf(df)) : __fmaf_rn(df, df, acc);
}

template <int MET>
__device__ __forceinline__ float dist_term_m(float acc, float df)
{
    if constexpr (MET == SUCO_METRIC_L1)
        return __fadd_rn(acc, fabsf(df));
    else
        return __fmaf_rn(df, df, acc);
}

// Two FP32 lanes in one 64-bit register: element-wise subtract and fused
// multiply-add, each rounded to nearest even like __fsub_rn and __fmaf_rn.
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi)
{
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}

// Where the assignment kernel adds each point to its centroid's fixed-point
// sum (x * 2^S rounded to an int64, per half): shared-memory sums flushed at
// the end of the block, or the global ones directly when they do not fit.
// Integer addition is associative, so the sums do not depend on the order
// of the atomics and the build is bitwise deterministic.
struct AccumArgs {
    const float* scale = nullptr;          // [halves] 2^S
    unsigned long long* gsum = nullptr;    // [halves][sqrtK][hmax]
    unsigned* gcnt = nullptr;              // [halves][sqrtK]
    int use_smem = 0;
};

// Nearest centroid of every point in one half-subspace (grid.y = half), in
// the index's metric, and with ACC the point's addition to that centroid's
// sums for the next Lloyd update.  Each block stages the half's centroids
// and then, tile by tile, its points' half-slices in shared memory with
// coalesced loads (row stride len | 1, so the threads' reads fall in
// distinct banks); each thread then scans the centroids for its PP points,
// dims in order.
// LMAX > 0: halves of at most LMAX dims; the point slices sit in registers
// and the centroid rows are zero-padded to LMAX values; the padded dims add
// (0 - 0)^2 or |0 - 0| to the sum, which leaves it unchanged, so the result
// is the sum over the len dims.  With the squared distance and PP = 2 the
// two points' terms are computed as FP32 pairs (sub.f32x2, fma.f32x2) from
// centroid rows stored with every value twice; the pair operations round
// each lane as the scalar ones do.
// LMAX = 0: any length (one point per thread, the metric chosen at run time).
// Shared memory: sqrtK * (2 LMAX, LMAX or len) + blockDim.x * PP * (len | 1)
// floats, then with ACC and use_smem sqrtK * len 8-byte sums and sqrtK counts.
template <int LMAX, int PP, int MET, bool ACC>
__global__ void __launch_bounds__(256) kmeans_assign_kernel(const float* __restrict__ X, int64_t ld, int64_t n,
                                                            int32_t d, int32_t Ns, int32_t sub_s, int32_t sqrtK,
                                                            int32_t hmax, const float* __restrict__ cent,
                                                            int32_t* __restrict__ assign, int metric, AccumArgs acc_args)
{
    constexpr bool PAIR = LMAX > 0 && PP == 2 && MET == SUCO_METRIC_L2;
    extern __shared__ __align__(16) float s_cent[];  // sqrtK centroid rows, the tile, the sums
    const int ih = blockIdx.y;
    int32_t off, len;
    half_dims(d, Ns, sub_s, ih >> 1, ih & 1, &off, &len);
    const int cs = PAIR ? 2 * LMAX : LMAX > 0 ? LMAX : len;  // centroid row stride (floats)
    const float* cb = cent + (int64_t)ih * sqrtK * hmax;
    for (int t = threadIdx.x; t < sqrtK * cs; t += blockDim.x) {
        const int a = t / cs, j = (t - a * cs) >> (PAIR ? 1 : 0);
        s_cent[t] = j < len ? cb[a * hmax + j] : 0.f;
    }
    float* s_x = s_cent + sqrtK * cs;
    const int xs = len | 1;
    const int TP = blockDim.x, TT = TP * PP;  // threads, points per tile
    // sums: [len][SP] with SP = sqrtK | 1, so lanes adding to different
    // centroids of one dim fall in different banks
    const int SP = sqrtK | 1;
    unsigned long long* s_sum = nullptr;
    unsigned* s_cnt = nullptr;
    unsigned long long* gs = nullptr;
    unsigned* gc = nullptr;
    float sc = 0.f;
    if constexpr (ACC) {
        size_t o = ((size_t)sqrtK * cs + (size_t)TT * xs) * 4;
        o = (o + 15) & ~size_t(15);
        s_sum = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(s_cent) + o);
        s_cnt = reinterpret_cast<unsigned*>(s_sum + (size_t)len * SP);
        gs = acc_args.gsum + (int64_t)ih * sqrtK * hmax;
        gc = acc_args.gcnt + (int64_t)ih * sqrtK;
        sc = acc_args.scale[ih];
        if (acc_args.use_smem) {
            for (int t = threadIdx.x; t < len * SP; t += blockDim.x) s_sum[t] = 0ull;
            for (int t = threadIdx.x; t < sqrtK; t += blockDim.x) s_cnt[t] = 0u;
        }
    }
    for (int64_t p0 = (int64_t)blockIdx.x * TT; p0 < n; p0 += (int64_t)gridDim.x * TT) {  // block-uniform
        __syncthreads();
        for (int t = threadIdx.x; t < TT * len; t += TP) {
            const int pp = t / len, j = t - pp * len;
            const int64_t p = p0 + pp;
            s_x[pp * xs + j] = p < n ? X[p * ld + off + j] : 0.f;
        }
        __syncthreads();
        int best[PP];
        if constexpr (PAIR) {
            unsigned long long xr[LMAX];  // (point 0, point 1) per dim
            {
                const float* x0 = s_x + threadIdx.x * xs;
                const float* x1 = s_x + (threadIdx.x + TP) * xs;
#pragma unroll
                for (int j = 0; j < LMAX; ++j) xr[j] = j < len ? f2_pack(x0[j], x1[j]) : 0ull;
            }
            float bd0 = INFINITY, bd1 = INFINITY;
            best[0] = best[1] = 0;
            for (int a = 0; a < sqrtK; ++a) {
                const ulonglong2* c2 = reinterpret_cast<const ulonglong2*>(s_cent + a * cs);
                unsigned long long acc = 0ull;  // (+0, +0)
#pragma unroll
                for (int q = 0; q < LMAX / 2; ++q) {
                    const ulonglong2 v = c2[q];  // (c_2q, c_2q), (c_2q+1, c_2q+1)
                    const unsigned long long d0 = f2_sub(xr[2 * q], v.x);
                    acc = f2_fma(d0, d0, acc);
                    const unsigned long long d1 = f2_sub(xr[2 * q + 1], v.y);
                    acc = f2_fma(d1, d1, acc);
                }
                const float a0 = __uint_as_float((unsigned)acc), a1 = __uint_as_float((unsigned)(acc >> 32));
                if (a0 < bd0) {
                    bd0 = a0;
                    best[0] = a;
                }
                if (a1 < bd1) {
                    bd1 = a1;
                    best[1] = a;
                }
            }
        } else if constexpr (LMAX > 0) {
            float xr[PP][LMAX], bd[PP];
#pragma unroll
            for (int u = 0; u < PP; ++u) {
                const float* x = s_x + (threadIdx.x + u * TP) * xs;
#pragma unroll
                for (int j = 0; j < LMAX; ++j) xr[u][j] = j < len ? x[j] : 0.f;
                best[u] = 0;
                bd[u] = INFINITY;
            }
            for (int a = 0; a < sqrtK; ++a) {
                const float4* c4 = reinterpret_cast<const float4*>(s_cent + a * LMAX);
                float acc[PP];
#pragma unroll
                for (int u = 0; u < PP; ++u) acc[u] = 0.f;
#pragma unroll
                for (int q = 0; q < LMAX / 4; ++q) {
                    const float4 v = c4[q];
#pragma unroll
                    for (int u = 0; u < PP; ++u) {
                        acc[u] = dist_term_m<MET>(acc[u], __fsub_rn(xr[u][4 * q + 0], v.x));
                        acc[u] = dist_term_m<MET>(acc[u], __fsub_rn(xr[u][4 * q + 1], v.y));
                        acc[u] = dist_term_m<MET>(acc[u], __fsub_rn(xr[u][4 * q + 2], v.z));
                        acc[u] = dist_term_m<MET>(acc[u], __fsub_rn(xr[u][4 * q + 3], v.w));
                    }
                }
#pragma unroll
                for (int u = 0; u < PP; ++u)
                    if (acc[u] < bd[u]) {
                        bd[u] = acc[u];
                        best[u] = a;
                    }
            }
        } else {
            const float* x = s_x + threadIdx.x * xs;
            float bd = INFINITY;
            best[0] = 0;
            for (int a = 0; a < sqrtK; ++a) {
                const float* c = s_cent + a * len;
                float acc = 0.f;
                for (int j = 0; j < len; ++j) acc = dist_term(acc, __fsub_rn(x[j], c[j]), metric);
                if (acc < bd) {
                    bd = acc;
                    best[0] = a;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < PP; ++u) {
            const int pl = threadIdx.x + u * TP;
            const int64_t p = p0 + pl;
            if (p >= n) continue;
            const int a = best[u];
            assign[(int64_t)ih * n + p] = a;
            if constexpr (ACC) {
                const float* x = s_x + pl * xs;
                for (int j = 0; j < len; ++j) {
                    const unsigned long long v = (unsigned long long)__float2ll_rn(x[j] * sc);
                    if (acc_args.use_smem)
                        atomicAdd(&s_sum[j * SP + a], v);
                    else
                        atomicAdd(&gs[a * hmax + j], v);
                }
                if (acc_args.use_smem)
                    atomicAdd(&s_cnt[a], 1u);
                else
                    atomicAdd(&gc[a], 1u);
            }
        }
    }
    if constexpr (ACC) {
        if (acc_args.use_smem) {
            __syncthreads();
            for (int t = threadIdx.x; t < sqrtK * len; t += blockDim.x) {
                const int a = t / len, j = t - a * len;
                const unsigned long long v = s_sum[j * SP + a];
                if (v) atomicAdd(&gs[a * hmax + j], v);
            }
            for (int t = threadIdx.x; t < sqrtK; t += blockDim.x)
                if (s_cnt[t]) atomicAdd(&gc[t], s_cnt[t]);
        }
    }
}

// New centroid = member mean; an empty cluster keeps its centroid.
__global__ void kmeans_finalize_kernel(int32_t d, int32_t Ns, int32_t sub_s, int32_t sqrtK, int32_t hmax,
                                       const unsigned long long* __restrict__ gsum, const unsigned* __restrict__ gcnt,
                                       const float* __restrict__ inv_scale, float* __restrict__ cent)
{
    const int ih = blockIdx.y;
    int32_t off, len;
    half_dims(d, Ns, sub_s, ih >> 1, ih & 1, &off, &len);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < sqrtK * len; t += gridDim.x * blockDim.x) {
        const int a = t / len, j = t - a * len;
        const unsigned c = gcnt[(int64_t)ih * sqrtK + a];
        if (c == 0) continue;
        const long long s = (long long)gsum[((int64_t)ih * sqrtK + a) * hmax + j];
        cent[((int64_t)ih * sqrtK + a) * hmax + j] = __fdiv_rn(__ll2float_rn(s) * inv_scale[ih], (float)c);
    }
}

__global__ void cells_kernel(const int32_t* __restrict__ a1, const int32_t* __restrict__ a2, int64_t n,
                             int32_t sqrtK, uint32_t* __restrict__ cells, int32_t* __restrict__ iota)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        cells[p] = (uint32_t)a1[p] * (uint32_t)sqrtK + (uint32_t)a2[p];
        iota[p] = (int32_t)p;
    }
}

// Stable least-significant-digit radix sort of (cell, id) pairs by cell, 8
// bits per pass (one pass for K <= 256, two up to K = 65536): per tile of
// RS_TILE keys a digit histogram, an exclusive scan over (digit, tile) in
// digit-major order, then a scatter in which every tile places its keys in
// index order (sub-rounds of RS_NT keys; inside a sub-round a key's rank is
// the count of equal digits in the earlier warps plus its rank among the
// equal digits of its own warp).  Ids inside a cell therefore stay ascending.
constexpr int RS_NT = 256, RS_PER = 8, RS_TILE = RS_NT * RS_PER, RS_W = RS_NT / 32;

__global__ void __launch_bounds__(RS_NT) rs_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                         uint32_t* __restrict__ hist, int64_t ntiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int j = 0; j < RS_PER; ++j) {
        const int64_t i = base + j * RS_NT + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];  // [digit][tile]
}

// Exclusive scan of a[0, m) in place, in blocks of 1024: the block totals go
// to sums[blockIdx.x] (then scanned by scan_totals_kernel and added back).
__device__ __forceinline__ uint32_t block_scan_1024(uint32_t v, uint32_t* wsum, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = wsum[lane], u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        wsum[lane] = u - t;  // exclusive warp offsets
        if (lane == 31) wsum[32] = u;
    }
    __syncthreads();
    const uint32_t r = wsum[warp] + x - v;
    *total = wsum[32];
    __syncthreads();  // wsum is reused by the caller's next call
    return r;
}

__global__ void __launch_bounds__(1024) scan_blocks_kernel(uint32_t* __restrict__ a, int64_t m,
                                                            uint32_t* __restrict__ sums)
{
    __shared__ uint32_t wsum[33];
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    const uint32_t v = i < m ? a[i] : 0u;
    uint32_t tot;
    const uint32_t r = block_scan_1024(v, wsum, &tot);
    if (i < m) a[i] = r;
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_totals_kernel(uint32_t* __restrict__ sums, int64_t nb)
{
    __shared__ uint32_t wsum[33];
    uint32_t carry = 0;
    for (int64_t c = 0; c < nb; c += 1024) {  // block-uniform
        const int64_t i = c + threadIdx.x;
        const uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t tot;
        const uint32_t r = block_scan_1024(v, wsum, &tot);
        if (i < nb) sums[i] = carry + r;
        carry += tot;
    }
}

__global__ void add_totals_kernel(uint32_t* __restrict__ a, int64_t m, const uint32_t* __restrict__ sums)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += sums[i >> 10];
}

__global__ void __launch_bounds__(RS_NT) rs_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                                            const int32_t* __restrict__ vals_in, int64_t n, int shift,
                                                            const uint32_t* __restrict__ offs, int64_t ntiles,
                                                            uint32_t* __restrict__ keys_out,
                                                            int32_t* __restrict__ vals_out)
{
    __shared__ uint32_t pos[256];         // next output position of each digit for this tile
    __shared__ uint32_t wcnt[RS_W][256];  // keys per digit of each warp in the current sub-round
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    pos[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_PER; ++j) {
#pragma unroll
        for (int w = 0; w < RS_W; ++w) wcnt[w][threadIdx.x] = 0u;
        __syncthreads();
        const int64_t i = base + j * RS_NT + threadIdx.x;
        const bool valid = i < n;
        const uint32_t key = valid ? keys_in[i] : 0u;
        const uint32_t dg = valid ? (key >> shift) & 255u : 256u;  // 256: no key
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0u) wcnt[warp][dg] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t o = pos[dg] + rank;
            for (int w = 0; w < warp; ++w) o += wcnt[w][dg];
            keys_out[o] = key;
            vals_out[o] = vals_in[i];
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < RS_W; ++w) add += wcnt[w][threadIdx.x];
        pos[threadIdx.x] += add;
        // the next sub-round's zeroing is ordered after these reads by its barrier
        __syncthreads();
    }
}

// cell_off[x] = first position whose cell id is >= x, for x in [0, K].
__global__ void cell_off_kernel(const uint32_t* __restrict__ sorted_cells, int64_t n, int64_t K,
                                uint32_t* __restrict__ cell_off)
{
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x <= K; x += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (sorted_cells[mid] < (uint32_t)x) lo = mid + 1; else hi = mid;
        }
        cell_off[x] = (uint32_t)lo;
    }
}

// split[i][j][x] = position (inside perm[i]) of the first id >= j*n_ch in cell x.
__global__ void split_kernel(const uint32_t* __restrict__ cell_off, const int32_t* __restrict__ perm, int64_t n,
                             int32_t Ns, int64_t K, int64_t n_ch, int32_t nch, uint32_t* __restrict__ split)
{
    const int64_t total = (int64_t)Ns * (nch + 1) * K;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = t % K;
        const int64_t j = (t / K) % (nch + 1);
        const int64_t i = t / (K * (nch + 1));
        const uint32_t* co = cell_off + i * (K + 1);
        const int32_t* pm = perm + i * n;
        int64_t lo = co[x], hi = co[x + 1];
        const int64_t target = j * n_ch;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)pm[mid] < target) lo = mid + 1; else hi = mid;
        }
        split[t] = (uint32_t)lo;
    }
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes` and never
// lowers it: the K-means kernels are shared by the index build and the
// allocation-free entry point, which may run from different host threads.
template <class K>
cudaError_t raise_smem_limit(K* kern, size_t bytes)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess || (size_t)fa.maxDynamicSharedSizeBytes >= bytes) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Launch plan of the assignment kernel: the row bound LMAX (8, 16 or 32
// covering the longest half, else 0 for any length), points per thread, and
// threads per block (256, 128 or 64: the largest whose centroid table and
// point slices fit the opt-in shared memory) with its dynamic shared memory;
// for the accumulating launches, whether the sums fit in shared memory too
// and the bytes with them.
struct AssignPlan {
    int lmax = 0, pp = 1, tp = 0, use_smem = 0;
    size_t smem = 0, smem_acc = 0;
};

bool assign_plan(int k, int len, int metric, int optin, AssignPlan* pl)
{
    pl->lmax = len <= 8 ? 8 : len <= 16 ? 16 : len <= 32 ? 32 : 0;
    pl->pp = pl->lmax > 0 && pl->lmax <= 16 ? 2 : 1;
    const bool pair = pl->lmax > 0 && pl->pp == 2 && metric == SUCO_METRIC_L2;
    const int cs = pair ? 2 * pl->lmax : pl->lmax > 0 ? pl->lmax : len;
    for (int t = 256; t >= 64; t /= 2) {
        const size_t b = ((size_t)k * cs + (size_t)t * pl->pp * (len | 1)) * 4;
        if (b <= (size_t)optin) {
            pl->tp = t;
            pl->smem = b;
            const size_t acc = ((b + 15) & ~size_t(15)) + (size_t)len * (k | 1) * 8 + (size_t)k * 4;
            pl->use_smem = acc <= (size_t)optin ? 1 : 0;
            pl->smem_acc = pl->use_smem ? acc : b;
            return true;
        }
    }
    return false;
}

template <int LMAX, int PP, int MET, bool ACC>
cudaError_t launch_assign_t(const AssignPlan& pl, dim3 grid, cudaStream_t st, const float* X, int64_t ld, int64_t n,
                            int32_t d, int32_t Ns, int32_t sub_s, int32_t sqrtK, int32_t hmax, const float* cent,
                            int32_t* assign, int metric, const AccumArgs& aa)
{
    auto kern = kmeans_assign_kernel<LMAX, PP, MET, ACC>;
    const size_t smem = ACC ? pl.smem_acc : pl.smem;
    cudaError_t e = raise_smem_limit(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, pl.tp, smem, st>>>(X, ld, n, d, Ns, sub_s, sqrtK, hmax, cent, assign, metric, aa);
    return cudaSuccess;  // a launch error is read by the caller's launch check
}

// One assignment pass over every half (grid.y) with the planned kernel; with
// `aa` (non-null gsum) it also adds every point to its centroid's sums and
// count, which the caller zeroed.  The caller checks the launch.
cudaError_t launch_assign(const AssignPlan& pl, int blocks, int halves, cudaStream_t st, const float* X, int64_t ld,
                          int64_t n, int32_t d, int32_t Ns, int32_t sub_s, int32_t sqrtK, int32_t hmax,
                          const float* cent, int32_t* assign, int metric, const AccumArgs& aa)
{
    const dim3 g(blocks, halves);
    const bool l1 = metric == SUCO_METRIC_L1, acc = aa.gsum != nullptr;
    AccumArgs a2 = aa;
    a2.use_smem = pl.use_smem;
#define SUCO_ASSIGN_M(LM, PPV, M)                                                                                \
    return acc ? launch_assign_t<LM, PPV, M, true>(pl, g, st, X, ld, n, d, Ns, sub_s, sqrtK, hmax, cent, assign,  \
                                                   metric, a2)                                                  \
               : launch_assign_t<LM, PPV, M, false>(pl, g, st, X, ld, n, d, Ns, sub_s, sqrtK, hmax, cent, assign, \
                                                    metric, a2)
#define SUCO_ASSIGN(LM, PPV)                  \
    if (l1) SUCO_ASSIGN_M(LM, PPV, SUCO_METRIC_L1); \
    SUCO_ASSIGN_M(LM, PPV, SUCO_METRIC_L2)
    switch (pl.lmax) {
        case 8: SUCO_ASSIGN(8, 2);
        case 16: SUCO_ASSIGN(16, 2);
        case 32: SUCO_ASSIGN(32, 1);
        default: SUCO_ASSIGN_M(0, 1, SUCO_METRIC_L2);
    }
#undef SUCO_ASSIGN
#undef SUCO_ASSIGN_M
}

int grid_for(int64_t work, int threads, int cap = 65535)
{
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

int build_imi(DeviceIndex* ix, const int32_t* assign, cudaStream_t st)
{
    const int64_t n = ix->n, K = ix->K;
    int end_bit = 1;
    while ((int64_t(1) << end_bit) < K) ++end_bit;
    const int passes = (end_bit + 7) / 8;  // K <= 65536: one or two
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE, m = 256 * ntiles, nb = (m + 1023) / 1024;
    DevBuf cells, sorted, iota, k2, v2, hist, sums;
    if (cells.alloc(n * 4) || sorted.alloc(n * 4) || iota.alloc(n * 4) || hist.alloc((size_t)m * 4) ||
        sums.alloc((size_t)nb * 4) || (passes > 1 && (k2.alloc(n * 4) || v2.alloc(n * 4))))
        return SUCO_ENOMEM;
    for (int i = 0; i < ix->Ns; ++i) {
        cells_kernel<<<grid_for(n, 256), 256, 0, st>>>(assign + (int64_t)(2 * i) * n, assign + (int64_t)(2 * i + 1) * n,
                                                       n, ix->sqrtK, cells.as<uint32_t>(), iota.as<int32_t>());
        SUCO_LAUNCH_CHECK("cells_kernel");
        for (int pass = 0; pass < passes; ++pass) {
            // two passes: cells -> k2 -> sorted; one pass: cells -> sorted
            const uint32_t* kin = pass == 0 ? cells.as<uint32_t>() : k2.as<uint32_t>();
            const int32_t* vin = pass == 0 ? iota.as<int32_t>() : v2.as<int32_t>();
            const bool last = pass == passes - 1;
            uint32_t* kout = last ? sorted.as<uint32_t>() : k2.as<uint32_t>();
            int32_t* vout = last ? ix->perm + (int64_t)i * n : v2.as<int32_t>();
            const int shift = 8 * pass;
            rs_hist_kernel<<<(unsigned)ntiles, RS_NT, 0, st>>>(kin, n, shift, hist.as<uint32_t>(), ntiles);
            SUCO_LAUNCH_CHECK("rs_hist_kernel");
            scan_blocks_kernel<<<(unsigned)nb, 1024, 0, st>>>(hist.as<uint32_t>(), m, sums.as<uint32_t>());
            SUCO_LAUNCH_CHECK("scan_blocks_kernel");
            scan_totals_kernel<<<1, 1024, 0, st>>>(sums.as<uint32_t>(), nb);
            SUCO_LAUNCH_CHECK("scan_totals_kernel");
            add_totals_kernel<<<grid_for(m, 256), 256, 0, st>>>(hist.as<uint32_t>(), m, sums.as<uint32_t>());
            SUCO_LAUNCH_CHECK("add_totals_kernel");
            rs_scatter_kernel<<<(unsigned)ntiles, RS_NT, 0, st>>>(kin, vin, n, shift, hist.as<uint32_t>(), ntiles,
                                                                  kout, vout);
            SUCO_LAUNCH_CHECK("rs_scatter_kernel");
        }
        cell_off_kernel<<<grid_for(K + 1, 256), 256, 0, st>>>(sorted.as<uint32_t>(), n, K,
                                                              ix->cell_off + (int64_t)i * (K + 1));
        SUCO_LAUNCH_CHECK("cell_off_kernel");
    }
    split_kernel<<<grid_for((int64_t)ix->Ns * (ix->nch + 1) * K, 256), 256, 0, st>>>(
        ix->cell_off, ix->perm, n, ix->Ns, K, ix->n_ch, ix->nch, ix->split);
    SUCO_LAUNCH_CHECK("split_kernel");
    SUCO_CUDA_TRY(cudaStreamSynchronize(st));
    return SUCO_OK;
}

int kmeans_build(DeviceIndex* ix, const int64_t* init_ids_host, int32_t iters, cudaStream_t st)
{
    const int64_t n = ix->n;
    const int Ns = ix->Ns, sk = ix->sqrtK, hm = ix->hmax, H = 2 * Ns;
    DevBuf ids, assign, gsum, gcnt, maxabs, scale, inv_scale;
    if (ids.alloc((size_t)H * sk * 8) || assign.alloc((size_t)H * n * 4) || gsum.alloc((size_t)H * sk * hm * 8) ||
        gcnt.alloc((size_t)H * sk * 4) || maxabs.alloc((size_t)H * 4) || scale.alloc((size_t)H * 4) ||
        inv_scale.alloc((size_t)H * 4))
        return SUCO_ENOMEM;
    SUCO_CUDA_TRY(cudaMemcpyAsync(ids.p, init_ids_host, (size_t)H * sk * 8, cudaMemcpyHostToDevice, st));
    init_centroids_kernel<<<dim3(grid_for((int64_t)sk * hm, 256), H), 256, 0, st>>>(ix->X, ix->ld, ix->d, Ns, ix->sub_s,
                                                                                   sk, hm, ids.as<int64_t>(), ix->cent);
    SUCO_LAUNCH_CHECK("init_centroids_kernel");

    // fixed-point scale per half: max|x| * 2^S * n < 2^62
    SUCO_CUDA_TRY(cudaMemsetAsync(maxabs.p, 0, (size_t)H * 4, st));
    maxabs_kernel<<<grid_for(n, 1, 8 * 152), 256, 0, st>>>(ix->X, ix->ld, n, ix->d, Ns, ix->sub_s, H,
                                                            maxabs.as<unsigned>());
    SUCO_LAUNCH_CHECK("maxabs_kernel");
    std::vector<unsigned> mbits(H);
    SUCO_CUDA_TRY(cudaMemcpyAsync(mbits.data(), maxabs.p, (size_t)H * 4, cudaMemcpyDeviceToHost, st));
    SUCO_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<float> sc(H), isc(H);
    for (int h = 0; h < H; ++h) {
        float m;
        memcpy(&m, &mbits[h], 4);
        int S = 0;
        if (m > 0.f && std::isfinite(m)) {
            int e;
            std::frexp((double)m * (double)n, &e);  // m*n < 2^e
            S = 61 - e;
        }
        S = std::max(-120, std::min(120, S));
        sc[h] = std::ldexp(1.0f, S);
        isc[h] = std::ldexp(1.0f, -S);
    }
    SUCO_CUDA_TRY(cudaMemcpyAsync(scale.p, sc.data(), (size_t)H * 4, cudaMemcpyHostToDevice, st));
    SUCO_CUDA_TRY(cudaMemcpyAsync(inv_scale.p, isc.data(), (size_t)H * 4, cudaMemcpyHostToDevice, st));

    int max_len = 0;
    for (int ih = 0; ih < H; ++ih) {
        int32_t off, len;
        half_dims(ix->d, Ns, ix->sub_s, ih >> 1, ih & 1, &off, &len);
        max_len = std::max(max_len, (int)len);
    }
    int dev_smem_optin = 0;
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&dev_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device));
    AssignPlan ap;
    if (!assign_plan(sk, max_len, ix->metric, dev_smem_optin, &ap))
        return fail(SUCO_EUNSUPPORTED, "centroid table of %zu bytes exceeds shared memory", (size_t)sk * max_len * 4);
    int nsm = 0;
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ix->device));
    const int gx_assign = grid_for(n, ap.tp * ap.pp, 8 * nsm);
    AccumArgs aa;
    aa.scale = scale.as<float>();
    aa.gsum = gsum.as<unsigned long long>();
    aa.gcnt = gcnt.as<unsigned>();
    for (int it = 0; it < iters; ++it) {
        // assignment against the current centroids and the members' sums in one pass
        SUCO_CUDA_TRY(cudaMemsetAsync(gsum.p, 0, gsum.bytes, st));
        SUCO_CUDA_TRY(cudaMemsetAsync(gcnt.p, 0, gcnt.bytes, st));
        SUCO_CUDA_TRY(launch_assign(ap, gx_assign, H, st, ix->X, ix->ld, n, ix->d, Ns, ix->sub_s, sk, hm, ix->cent,
                                    assign.as<int32_t>(), ix->metric, aa));
        SUCO_LAUNCH_CHECK("kmeans_assign_kernel");
        kmeans_finalize_kernel<<<dim3(grid_for((int64_t)sk * max_len, 256), H), 256, 0, st>>>(
            ix->d, Ns, ix->sub_s, sk, hm, gsum.as<unsigned long long>(), gcnt.as<unsigned>(), inv_scale.as<float>(),
            ix->cent);
        SUCO_LAUNCH_CHECK("kmeans_finalize_kernel");
    }
    // the assignment that defines the IMI, against the final centroids
    SUCO_CUDA_TRY(launch_assign(ap, gx_assign, H, st, ix->X, ix->ld, n, ix->d, Ns, ix->sub_s, sk, hm, ix->cent,
                                assign.as<int32_t>(), ix->metric, AccumArgs()));
    SUCO_LAUNCH_CHECK("kmeans_assign_kernel");
    return build_imi(ix, assign.as<int32_t>(), st);
}

}  // namespace suco

// ---------------------------------------------------------------------------
// K-means on one column range without any allocation (suco_kmeans_noalloc).
//
// Some callers cannot allocate device memory while they run this step: a
// process whose device memory is already handed out to its own allocator, or a
// caller under a latency budget that rules out cudaMalloc and its implicit
// device synchronisation.  For them, the centroid sums, counts and the
// fixed-point scale live in one fixed array in device global memory, defined
// here at file scope.  Every GPU that loads this library keeps the array
// (NOALLOC_SCRATCH_BYTES) until the process exits.  Every call shares it, so
// calls whose GPU work overlaps in time race on it.
namespace suco {
namespace {

constexpr int NOALLOC_MAX_K = 256;    // centroids
constexpr int NOALLOC_MAX_DIM = 128;  // dimensions of the column range
constexpr size_t NOALLOC_SUM_BYTES = (size_t)NOALLOC_MAX_K * NOALLOC_MAX_DIM * 8;
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_SUM_BYTES + NOALLOC_MAX_K * 4 + 256;

static __device__ __align__(256) unsigned char g_kmeans_scratch[NOALLOC_SCRATCH_BYTES];

// host-side address of g_kmeans_scratch per device (the symbol's host name is
// only a stand-in: kernels must be given this address)
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};

int noalloc_scratch(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= 256) return fail(SUCO_ESTATE, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_kmeans_scratch);
        if (e != cudaSuccess)
            return fail(SUCO_ECUDA, "cudaGetSymbolAddress of the K-means scratch failed: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    return SUCO_OK;
}

}  // namespace
}  // namespace suco

extern "C" int suco_kmeans_noalloc(const float* data, int64_t n, int32_t d, int32_t dim_off, int32_t dim_len,
                                   int32_t k, int32_t iters, float* centroids, int32_t* assign, void* stream)
{
    using namespace suco;
    clear_error();
    if (!data || !centroids || !assign) return fail(SUCO_EINVAL, "data, centroids and assign must not be NULL");
    if (n < 1 || n > 0x7fffffffLL) return fail(SUCO_EINVAL, "n=%lld must be in [1, 2^31-1]", (long long)n);
    if (d < 1 || dim_off < 0 || dim_len < 1 || (int64_t)dim_off + dim_len > d)
        return fail(SUCO_EINVAL, "columns [%d, %d) are not inside d=%d", dim_off, dim_off + dim_len, d);
    if (k < 1 || k > n) return fail(SUCO_EINVAL, "k=%d must be in [1, n]", k);
    if (iters < 0 || iters > 10000) return fail(SUCO_EINVAL, "iters=%d must be in [0, 10000]", iters);
    if (k > NOALLOC_MAX_K || dim_len > NOALLOC_MAX_DIM)
        return fail(SUCO_EUNSUPPORTED,
                    "suco_kmeans_noalloc: k=%d, dim_len=%d exceed its fixed scratch (k <= %d, dim_len <= %d)", k,
                    dim_len, NOALLOC_MAX_K, NOALLOC_MAX_DIM);
    int dev = 0;
    SUCO_CUDA_TRY(cudaGetDevice(&dev));
    unsigned char* scratch = nullptr;
    int rc = noalloc_scratch(dev, &scratch);
    if (rc) return rc;
    unsigned long long* gsum = reinterpret_cast<unsigned long long*>(scratch);
    unsigned* gcnt = reinterpret_cast<unsigned*>(scratch + NOALLOC_SUM_BYTES);
    unsigned* maxabs = gcnt + NOALLOC_MAX_K;
    float* scale = reinterpret_cast<float*>(maxabs + 1);
    float* inv_scale = scale + 1;
    cudaStream_t st = (cudaStream_t)stream;
    // the column range as "half 0" of a one-subspace layout of width 2*dim_len
    const float* Xc = data + dim_off;
    const int32_t dd = 2 * dim_len, sub = 2 * dim_len;
    int nsm = 0, smem_optin = 0;
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

    // fixed-point scale: max|x| * 2^S * n < 2^62
    SUCO_CUDA_TRY(cudaMemsetAsync(maxabs, 0, 4, st));
    maxabs_kernel<<<grid_for(n, 1, 8 * 152), 256, 0, st>>>(Xc, d, n, dd, 1, sub, 1, maxabs);
    SUCO_LAUNCH_CHECK("maxabs_kernel");
    unsigned mbits = 0;
    SUCO_CUDA_TRY(cudaMemcpyAsync(&mbits, maxabs, 4, cudaMemcpyDeviceToHost, st));
    SUCO_CUDA_TRY(cudaStreamSynchronize(st));
    float m;
    memcpy(&m, &mbits, 4);
    int S = 0;
    if (m > 0.f && std::isfinite(m)) {
        int e;
        std::frexp((double)m * (double)n, &e);
        S = 61 - e;
    }
    S = std::max(-120, std::min(120, S));
    const float sc[2] = {std::ldexp(1.0f, S), std::ldexp(1.0f, -S)};
    SUCO_CUDA_TRY(cudaMemcpyAsync(scale, sc, 8, cudaMemcpyHostToDevice, st));

    AssignPlan ap;
    if (!assign_plan(k, dim_len, SUCO_METRIC_L2, smem_optin, &ap))
        return fail(SUCO_EUNSUPPORTED, "k=%d x dim_len=%d centroids exceed shared memory", k, dim_len);
    // launch_assign raises (never lowers) the assignment kernel's dynamic
    // shared-memory limit: the index build may run it from another thread
    const int gx_assign = grid_for(n, ap.tp * ap.pp, 8 * nsm);
    AccumArgs aa;
    aa.scale = scale;
    aa.gsum = gsum;
    aa.gcnt = gcnt;
    for (int it = 0; it < iters; ++it) {
        // sums and counts start from zero in every iteration (the array keeps the last call's contents)
        SUCO_CUDA_TRY(cudaMemsetAsync(gsum, 0, (size_t)k * dim_len * 8, st));
        SUCO_CUDA_TRY(cudaMemsetAsync(gcnt, 0, (size_t)k * 4, st));
        SUCO_CUDA_TRY(launch_assign(ap, gx_assign, 1, st, Xc, d, n, dd, 1, sub, k, dim_len, centroids, assign,
                                    SUCO_METRIC_L2, aa));
        SUCO_LAUNCH_CHECK("kmeans_assign_kernel");
        kmeans_finalize_kernel<<<dim3(grid_for((int64_t)k * dim_len, 256), 1), 256, 0, st>>>(
            dd, 1, sub, k, dim_len, gsum, gcnt, inv_scale, centroids);
        SUCO_LAUNCH_CHECK("kmeans_finalize_kernel");
    }
    // the assignment against the final centroids
    SUCO_CUDA_TRY(launch_assign(ap, gx_assign, 1, st, Xc, d, n, dd, 1, sub, k, dim_len, centroids, assign,
                                SUCO_METRIC_L2, AccumArgs()));
    SUCO_LAUNCH_CHECK("kmeans_assign_kernel");
    return SUCO_OK;
}
