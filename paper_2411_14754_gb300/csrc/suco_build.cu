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
#include <cub/device/device_radix_sort.cuh>

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

// Nearest centroid of every point in one half-subspace (grid.y = half), in
// the index's metric.  Each block stages the half's centroids and then, tile
// by tile, its points' half-slices in shared memory with coalesced loads
// (row stride len | 1, so the threads' reads fall in distinct banks); each
// thread then scans the centroids for its point, dims in order.
// Shared memory: sqrtK*len + blockDim.x*(len|1) floats.
__global__ void kmeans_assign_kernel(const float* __restrict__ X, int64_t ld, int64_t n, int32_t d, int32_t Ns,
                                     int32_t sub_s, int32_t sqrtK, int32_t hmax, const float* __restrict__ cent,
                                     int32_t* __restrict__ assign, int metric)
{
    extern __shared__ float s_cent[];  // sqrtK * len, then the tile
    const int ih = blockIdx.y;
    int32_t off, len;
    half_dims(d, Ns, sub_s, ih >> 1, ih & 1, &off, &len);
    const float* cb = cent + (int64_t)ih * sqrtK * hmax;
    for (int t = threadIdx.x; t < sqrtK * len; t += blockDim.x) {
        const int a = t / len, j = t - a * len;
        s_cent[t] = cb[a * hmax + j];
    }
    float* s_x = s_cent + sqrtK * len;
    const int xs = len | 1;
    const int TP = blockDim.x;
    for (int64_t p0 = (int64_t)blockIdx.x * TP; p0 < n; p0 += (int64_t)gridDim.x * TP) {  // block-uniform
        __syncthreads();
        for (int t = threadIdx.x; t < TP * len; t += TP) {
            const int pp = t / len, j = t - pp * len;
            const int64_t p = p0 + pp;
            s_x[pp * xs + j] = p < n ? X[p * ld + off + j] : 0.f;
        }
        __syncthreads();
        const int64_t p = p0 + threadIdx.x;
        if (p >= n) continue;
        const float* x = s_x + threadIdx.x * xs;
        int best = 0;
        float bd = INFINITY;
        if (len <= 32) {
            float xr[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) xr[j] = (j < len) ? x[j] : 0.f;
            for (int a = 0; a < sqrtK; ++a) {
                const float* c = s_cent + a * len;
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < len) acc = dist_term(acc, __fsub_rn(xr[j], c[j]), metric);
                if (acc < bd) {
                    bd = acc;
                    best = a;
                }
            }
        } else {
            for (int a = 0; a < sqrtK; ++a) {
                const float* c = s_cent + a * len;
                float acc = 0.f;
                for (int j = 0; j < len; ++j) acc = dist_term(acc, __fsub_rn(x[j], c[j]), metric);
                if (acc < bd) {
                    bd = acc;
                    best = a;
                }
            }
        }
        assign[(int64_t)ih * n + p] = best;
    }
}

// Per-centroid sums in 64-bit fixed point (x * 2^S rounded), staged in shared
// memory when they fit.  Integer addition is associative, so the result does
// not depend on the order of the atomics.
__global__ void kmeans_accum_kernel(const float* __restrict__ X, int64_t ld, int64_t n, int32_t d, int32_t Ns,
                                    int32_t sub_s, int32_t sqrtK, int32_t hmax, const int32_t* __restrict__ assign,
                                    const float* __restrict__ scale, unsigned long long* __restrict__ gsum,
                                    unsigned* __restrict__ gcnt, int use_smem)
{
    extern __shared__ unsigned long long s_sum[];  // sqrtK * len sums, then sqrtK counts
    const int ih = blockIdx.y;
    int32_t off, len;
    half_dims(d, Ns, sub_s, ih >> 1, ih & 1, &off, &len);
    unsigned* s_cnt = reinterpret_cast<unsigned*>(s_sum + sqrtK * len);
    const float sc = scale[ih];
    unsigned long long* gs = gsum + (int64_t)ih * sqrtK * hmax;
    unsigned* gc = gcnt + (int64_t)ih * sqrtK;
    if (use_smem) {
        for (int t = threadIdx.x; t < sqrtK * len; t += blockDim.x) s_sum[t] = 0ull;
        for (int t = threadIdx.x; t < sqrtK; t += blockDim.x) s_cnt[t] = 0u;
        __syncthreads();
    }
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int a = assign[(int64_t)ih * n + p];
        const float* x = X + p * ld + off;
        for (int j = 0; j < len; ++j) {
            const long long v = __float2ll_rn(__ldg(x + j) * sc);
            if (use_smem)
                atomicAdd(&s_sum[a * len + j], (unsigned long long)v);
            else
                atomicAdd(&gs[a * hmax + j], (unsigned long long)v);
        }
        if (use_smem)
            atomicAdd(&s_cnt[a], 1u);
        else
            atomicAdd(&gc[a], 1u);
    }
    if (use_smem) {
        __syncthreads();
        for (int t = threadIdx.x; t < sqrtK * len; t += blockDim.x)
            if (s_sum[t]) atomicAdd(&gs[(t / len) * hmax + (t % len)], s_sum[t]);
        for (int t = threadIdx.x; t < sqrtK; t += blockDim.x)
            if (s_cnt[t]) atomicAdd(&gc[t], s_cnt[t]);
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

// Points per block of the assignment kernel (256, 128 or 64: the largest
// whose centroid table and point slices fit the opt-in shared memory) and its
// dynamic shared memory; false if not even 64 fit.
bool assign_shape(int k, int len, int optin, int* tp, size_t* smem)
{
    for (int t = 256; t >= 64; t /= 2) {
        const size_t b = ((size_t)k * len + (size_t)t * (len | 1)) * 4;
        if (b <= (size_t)optin) {
            *tp = t;
            *smem = b;
            return true;
        }
    }
    return false;
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
    DevBuf cells, sorted, iota, tmp;
    if (cells.alloc(n * 4) || sorted.alloc(n * 4) || iota.alloc(n * 4)) return SUCO_ENOMEM;
    int end_bit = 1;
    while ((int64_t(1) << end_bit) < K) ++end_bit;
    size_t tmp_bytes = 0;
    SUCO_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, cells.as<uint32_t>(), sorted.as<uint32_t>(),
                                                  iota.as<int32_t>(), ix->perm, (int)n, 0, end_bit, st));
    if (tmp.alloc(tmp_bytes)) return SUCO_ENOMEM;
    for (int i = 0; i < ix->Ns; ++i) {
        cells_kernel<<<grid_for(n, 256), 256, 0, st>>>(assign + (int64_t)(2 * i) * n, assign + (int64_t)(2 * i + 1) * n,
                                                       n, ix->sqrtK, cells.as<uint32_t>(), iota.as<int32_t>());
        SUCO_LAUNCH_CHECK("cells_kernel");
        size_t tb = tmp_bytes;
        SUCO_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, tb, cells.as<uint32_t>(), sorted.as<uint32_t>(),
                                                      iota.as<int32_t>(), ix->perm + (int64_t)i * n, (int)n, 0,
                                                      end_bit, st));
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
    int atp = 0;
    size_t assign_smem = 0;
    const size_t accum_smem = (size_t)sk * max_len * 8 + (size_t)sk * 4;
    if (!assign_shape(sk, max_len, dev_smem_optin, &atp, &assign_smem))
        return fail(SUCO_EUNSUPPORTED, "centroid table of %zu bytes exceeds shared memory", (size_t)sk * max_len * 4);
    const int use_smem = accum_smem <= (size_t)dev_smem_optin ? 1 : 0;
    SUCO_CUDA_TRY(raise_smem_limit(kmeans_assign_kernel, assign_smem));
    if (use_smem) SUCO_CUDA_TRY(raise_smem_limit(kmeans_accum_kernel, accum_smem));
    int nsm = 0;
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ix->device));
    const dim3 g_assign(grid_for(n, atp, 8 * nsm), H);
    const dim3 g_accum(grid_for(n, 256, 2 * nsm), H);
    for (int it = 0; it < iters; ++it) {
        kmeans_assign_kernel<<<g_assign, atp, assign_smem, st>>>(ix->X, ix->ld, n, ix->d, Ns, ix->sub_s, sk, hm,
                                                                ix->cent, assign.as<int32_t>(), ix->metric);
        SUCO_LAUNCH_CHECK("kmeans_assign_kernel");
        SUCO_CUDA_TRY(cudaMemsetAsync(gsum.p, 0, gsum.bytes, st));
        SUCO_CUDA_TRY(cudaMemsetAsync(gcnt.p, 0, gcnt.bytes, st));
        kmeans_accum_kernel<<<g_accum, 256, use_smem ? accum_smem : 0, st>>>(
            ix->X, ix->ld, n, ix->d, Ns, ix->sub_s, sk, hm, assign.as<int32_t>(), scale.as<float>(),
            gsum.as<unsigned long long>(), gcnt.as<unsigned>(), use_smem);
        SUCO_LAUNCH_CHECK("kmeans_accum_kernel");
        kmeans_finalize_kernel<<<dim3(grid_for((int64_t)sk * max_len, 256), H), 256, 0, st>>>(
            ix->d, Ns, ix->sub_s, sk, hm, gsum.as<unsigned long long>(), gcnt.as<unsigned>(), inv_scale.as<float>(),
            ix->cent);
        SUCO_LAUNCH_CHECK("kmeans_finalize_kernel");
    }
    // the assignment that defines the IMI, against the final centroids
    kmeans_assign_kernel<<<g_assign, atp, assign_smem, st>>>(ix->X, ix->ld, n, ix->d, Ns, ix->sub_s, sk, hm, ix->cent,
                                                            assign.as<int32_t>(), ix->metric);
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

    int atp = 0;
    size_t assign_smem = 0;
    if (!assign_shape(k, dim_len, smem_optin, &atp, &assign_smem))
        return fail(SUCO_EUNSUPPORTED, "k=%d x dim_len=%d centroids exceed shared memory", k, dim_len);
    const size_t accum_smem = (size_t)k * dim_len * 8 + (size_t)k * 4;
    const int use_smem = accum_smem <= (size_t)smem_optin ? 1 : 0;
    // raise (never lower) the dynamic shared-memory limits of the shared kernels
    SUCO_CUDA_TRY(raise_smem_limit(kmeans_assign_kernel, assign_smem));
    if (use_smem) SUCO_CUDA_TRY(raise_smem_limit(kmeans_accum_kernel, accum_smem));
    const dim3 g_assign(grid_for(n, atp, 8 * nsm), 1);
    const dim3 g_accum(grid_for(n, 256, 2 * nsm), 1);
    for (int it = 0; it < iters; ++it) {
        kmeans_assign_kernel<<<g_assign, atp, assign_smem, st>>>(Xc, d, n, dd, 1, sub, k, dim_len, centroids, assign,
                                                                SUCO_METRIC_L2);
        SUCO_LAUNCH_CHECK("kmeans_assign_kernel");
        // sums and counts start from zero in every iteration (the array keeps the last call's contents)
        SUCO_CUDA_TRY(cudaMemsetAsync(gsum, 0, (size_t)k * dim_len * 8, st));
        SUCO_CUDA_TRY(cudaMemsetAsync(gcnt, 0, (size_t)k * 4, st));
        kmeans_accum_kernel<<<g_accum, 256, use_smem ? accum_smem : 0, st>>>(Xc, d, n, dd, 1, sub, k, dim_len, assign,
                                                                             scale, gsum, gcnt, use_smem);
        SUCO_LAUNCH_CHECK("kmeans_accum_kernel");
        kmeans_finalize_kernel<<<dim3(grid_for((int64_t)k * dim_len, 256), 1), 256, 0, st>>>(
            dd, 1, sub, k, dim_len, gsum, gcnt, inv_scale, centroids);
        SUCO_LAUNCH_CHECK("kmeans_finalize_kernel");
    }
    // the assignment against the final centroids
    kmeans_assign_kernel<<<g_assign, atp, assign_smem, st>>>(Xc, d, n, dd, 1, sub, k, dim_len, centroids, assign,
                                                            SUCO_METRIC_L2);
    SUCO_LAUNCH_CHECK("kmeans_assign_kernel");
    return SUCO_OK;
}
