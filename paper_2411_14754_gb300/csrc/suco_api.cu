// C ABI of libsuco: argument checks, index ownership, error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>
#include <unordered_set>
#include <vector>

#include "suco_internal.cuh"

namespace suco {

namespace {
thread_local char g_err[1024] = "";

uint64_t splitmix64(uint64_t* state)
{
    uint64_t z = (*state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
}  // namespace

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

namespace {
std::atomic<int32_t> g_fault_kind{SUCO_FAULT_NONE};
std::atomic<int32_t> g_fault_after{0};
}  // namespace

bool fault_fires(int32_t kind)
{
    if (g_fault_kind.load(std::memory_order_relaxed) != kind) return false;
    if (g_fault_after.fetch_sub(1) != 0) return false;
    g_fault_kind.store(SUCO_FAULT_NONE);
    return true;
}

int launch_status(const char* what)
{
    if (fault_fires(SUCO_FAULT_LAUNCH)) return fail(SUCO_ECUDA, "%s: injected launch failure", what);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SUCO_ECUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    return SUCO_OK;
}

int check_status(const DeviceIndex* ix)
{
    const uint32_t s = ix->status_host ? *ix->status_host : 0u;
    if (s)
        return fail(SUCO_ETIMEOUT, "a bounded device wait on this index gave up (status 0x%x): results since then "
                                   "are unreliable; suco_read_status reads and clears the word", s);
    return SUCO_OK;
}

int DevBuf::alloc(size_t b)
{
    bytes = b;
    if (b == 0) return SUCO_OK;
    if (fault_fires(SUCO_FAULT_ALLOC)) return fail(SUCO_ENOMEM, "cudaMalloc(%zu): injected allocation failure", b);
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(SUCO_ENOMEM, "cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
    }
    return SUCO_OK;
}

void thresholds(int64_t n, double alpha, double beta, int32_t k, int64_t* T, int64_t* C)
{
    // Algorithm 3 stops once alpha*n ids are retrieved; Algorithm 4 re-ranks beta*n ids.
    double t = std::ceil(alpha * (double)n - 1e-9);
    t = std::fmin(std::fmax(t, 1.0), (double)n);
    double c = std::ceil(beta * (double)n - 1e-9);
    c = std::fmax(c, (double)k);
    c = std::fmin(std::fmax(c, 1.0), (double)n);
    *T = (int64_t)t;
    *C = (int64_t)c;
}

namespace {

void free_index_memory(DeviceIndex* ix)
{
    cudaFree(ix->dperm);
    ix->dperm = nullptr;
    cudaFree(ix->X);
    cudaFree(ix->cent);
    cudaFree(ix->cell_off);
    cudaFree(ix->perm);
    cudaFree(ix->split);
    cudaFree(ix->work);
    cudaFree(ix->Xh);
    cudaFree(ix->rank_ws);
    cudaFree(ix->X8);
    cudaFree(ix->s8col);
    if (ix->status_host) cudaFreeHost((void*)ix->status_host);
    ix->status_host = nullptr;
    ix->status_dev = nullptr;
    ix->X8 = nullptr;
    ix->s8col = nullptr;
    ix->Xh = nullptr;
    ix->rank_ws = nullptr;
    ix->work = nullptr;
    ix->X = nullptr;
    ix->cent = nullptr;
    ix->cell_off = nullptr;
    ix->perm = nullptr;
    ix->split = nullptr;
}

int check_sizes(int64_t n, int32_t d, int32_t Ns, int32_t sqrtK)
{
    if (n < 1 || n > 0x7fffffffLL) return fail(SUCO_EINVAL, "n=%lld must be in [1, 2^31-1]", (long long)n);
    if (Ns < 1 || Ns > 32) return fail(SUCO_EINVAL, "Ns=%d must be in [1, 32]", Ns);
    if (d < 2 * Ns) return fail(SUCO_EINVAL, "d=%d must be at least 2*Ns=%d (each half needs a dimension)", d, 2 * Ns);
    if (sqrtK < 1 || sqrtK > 256) return fail(SUCO_EINVAL, "sqrtK=%d must be in [1, 256]", sqrtK);
    if ((int64_t)sqrtK > n) return fail(SUCO_EINVAL, "sqrtK=%d exceeds n=%lld", sqrtK, (long long)n);
    if ((uint64_t)Ns * (uint64_t)n >= (1ull << 32)) return fail(SUCO_EINVAL, "Ns*n must be below 2^32");
    return SUCO_OK;
}

// X[p][j] = data[p][perm[j]]: the dataset's columns in the sampling's order
__global__ void gather_columns_kernel(const float* __restrict__ data, int64_t n, int32_t d,
                                      const int32_t* __restrict__ perm, float* __restrict__ X, int64_t ld)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * ld; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / ld;
        const int j = (int)(t - p * ld);
        X[t] = j < d ? data[p * d + perm[j]] : 0.f;
    }
}

int check_perm(const int32_t* perm, int32_t d)
{
    std::vector<char> seen((size_t)d, 0);
    for (int32_t j = 0; j < d; ++j) {
        if (perm[j] < 0 || perm[j] >= d || seen[(size_t)perm[j]])
            return fail(SUCO_EINVAL, "dim_perm is not a permutation of [0, %d) (entry %d = %d)", d, j, perm[j]);
        seen[(size_t)perm[j]] = 1;
    }
    return SUCO_OK;
}

// Allocates the index arrays and copies the dataset (zero-padded to ld; with
// a dim_perm, its columns in the sampling's order).
int alloc_index(DeviceIndex* ix, const float* data, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK,
                const int32_t* dim_perm, int32_t metric, cudaStream_t st)
{
    ix->metric = metric;
    ix->n = n;
    ix->d = d;
    ix->Ns = Ns;
    ix->sqrtK = sqrtK;
    ix->sub_s = d / Ns;
    {
        const int32_t last = d - (Ns - 1) * ix->sub_s;
        ix->hmax = last - last / 2;
    }
    ix->K = (int64_t)sqrtK * sqrtK;
    ix->ld = (d + 3) & ~3;
    ix->nch = MIN_NCH;
    while ((n + ix->nch - 1) / ix->nch > MAX_CHUNK) ix->nch *= 2;
    ix->n_ch = (((n + ix->nch - 1) / ix->nch) + 31) & ~int64_t(31);
    SUCO_CUDA_TRY(cudaGetDevice(&ix->device));
    struct {
        void** p;
        size_t b;
    } a[] = {
        {(void**)&ix->X, (size_t)n * ix->ld * 4},
        {(void**)&ix->cent, (size_t)Ns * 2 * sqrtK * ix->hmax * 4},
        {(void**)&ix->cell_off, (size_t)Ns * (ix->K + 1) * 4},
        {(void**)&ix->perm, (size_t)Ns * n * 4 + 16},  // padded: the query scan reads whole 16-byte quads
        {(void**)&ix->split, (size_t)Ns * (ix->nch + 1) * ix->K * 4},
        {(void**)&ix->work, (size_t)WORK_SLOTS * WORK_STRIDE * 4},
    };
    ix->bytes = 0;
    for (auto& e : a) {
        cudaError_t err = fault_fires(SUCO_FAULT_ALLOC) ? cudaErrorMemoryAllocation : cudaMalloc(e.p, e.b);
        if (err != cudaSuccess) {
            cudaGetLastError();
            free_index_memory(ix);
            return fail(SUCO_ENOMEM, "cudaMalloc(%zu) for the index failed: %s", e.b, cudaGetErrorString(err));
        }
        ix->bytes += (int64_t)e.b;
    }
    {
        void* h = nullptr;
        cudaError_t err = fault_fires(SUCO_FAULT_ALLOC) ? cudaErrorMemoryAllocation
                                                        : cudaHostAlloc(&h, 4, cudaHostAllocMapped);
        if (err == cudaSuccess) {
            ix->status_host = static_cast<volatile uint32_t*>(h);
            *ix->status_host = 0u;
            err = cudaHostGetDevicePointer((void**)&ix->status_dev, h, 0);
        }
        if (err != cudaSuccess) {
            cudaGetLastError();
            free_index_memory(ix);
            return fail(SUCO_ENOMEM, "mapped host allocation of the status word failed: %s", cudaGetErrorString(err));
        }
    }
    SUCO_CUDA_TRY(cudaMemsetAsync(ix->cent, 0, a[1].b, st));
    SUCO_CUDA_TRY(cudaMemsetAsync(ix->work, 0, a[5].b, st));
    if (dim_perm) {
        cudaError_t err = fault_fires(SUCO_FAULT_ALLOC) ? cudaErrorMemoryAllocation
                                                        : cudaMalloc(&ix->dperm, (size_t)d * 4);
        if (err != cudaSuccess) {
            cudaGetLastError();
            ix->dperm = nullptr;
            free_index_memory(ix);
            return fail(SUCO_ENOMEM, "cudaMalloc of the dim permutation failed: %s", cudaGetErrorString(err));
        }
        ix->bytes += (int64_t)d * 4;
        SUCO_CUDA_TRY(cudaMemcpyAsync(ix->dperm, dim_perm, (size_t)d * 4, cudaMemcpyHostToDevice, st));
        gather_columns_kernel<<<(unsigned)std::min<int64_t>((n * ix->ld + 255) / 256, 152 * 64), 256, 0, st>>>(
            data, n, d, ix->dperm, ix->X, ix->ld);
        SUCO_LAUNCH_CHECK("gather_columns_kernel");
        SUCO_CUDA_TRY(cudaStreamSynchronize(st));  // the host copy of dim_perm is the caller's
        return SUCO_OK;
    }
    if (ix->ld != d) SUCO_CUDA_TRY(cudaMemsetAsync(ix->X, 0, a[0].b, st));
    SUCO_CUDA_TRY(cudaMemcpy2DAsync(ix->X, (size_t)ix->ld * 4, data, (size_t)d * 4, (size_t)d * 4, (size_t)n,
                                    cudaMemcpyDeviceToDevice, st));
    return SUCO_OK;
}

int check_query_params(const suco_index* index, const float* queries, int64_t nq, const suco_query_params* p,
                       const int32_t* ids, const float* dist)
{
    if (!index) return fail(SUCO_EINVAL, "index is NULL");
    if (!p) return fail(SUCO_EINVAL, "params is NULL");
    if (nq < 0) return fail(SUCO_EINVAL, "nq=%lld is negative", (long long)nq);
    if (p->k < 1 || p->k > 256) return fail(SUCO_EINVAL, "k=%d must be in [1, 256]", p->k);
    if (!(p->alpha > 0.0 && p->alpha <= 1.0)) return fail(SUCO_EINVAL, "alpha=%g must be in (0, 1]", p->alpha);
    if (!(p->beta > 0.0 && p->beta <= 1.0)) return fail(SUCO_EINVAL, "beta=%g must be in (0, 1]", p->beta);
    if (p->flags & ~SUCO_QUERY_ONE_CLUSTER_PER_QUERY) return fail(SUCO_EINVAL, "unknown flags 0x%x", p->flags);
    if (p->precision != SUCO_PRECISION_FP32 && p->precision != SUCO_PRECISION_BF16 &&
        p->precision != SUCO_PRECISION_FP8)
        return fail(SUCO_EINVAL, "precision=%d must be SUCO_PRECISION_FP32, _BF16 or _FP8", p->precision);
    if (p->precision == SUCO_PRECISION_BF16 && !index->ix.Xh)
        return fail(SUCO_ESTATE, "the index has no BF16 copy: call suco_add_reduced_copies first");
    if (p->precision == SUCO_PRECISION_FP8 && !index->ix.X8)
        return fail(SUCO_ESTATE, "the index has no FP8 copy: call suco_add_reduced_copies first");
    if (p->id_passes < 0) return fail(SUCO_EINVAL, "id_passes=%d must not be negative", p->id_passes);
    if (p->rank_precision != SUCO_RANK_FP32 && p->rank_precision != SUCO_RANK_BF16 &&
        p->rank_precision != SUCO_RANK_FP8)
        return fail(SUCO_EINVAL, "rank_precision=%d must be SUCO_RANK_FP32, _BF16 or _FP8", p->rank_precision);
    if (p->rank_precision != SUCO_RANK_FP32 && !index->ix.rank_ws)
        return fail(SUCO_ESTATE, "tensor-core ranking needs its tables workspace: call suco_add_reduced_copies with "
                                 "SUCO_COPY_RANK_BF16 first");
    if (p->rank_precision == SUCO_RANK_FP8 && !index->ix.s8col)
        return fail(SUCO_ESTATE, "FP8 ranking uses the scales of the FP8 copy: call suco_add_reduced_copies with "
                                 "SUCO_COPY_FP8 first");
    if (index->ix.metric == SUCO_METRIC_L1) {
        if (p->precision != SUCO_PRECISION_FP32 || p->rank_precision != SUCO_RANK_FP32)
            return fail(SUCO_EUNSUPPORTED, "an L1 index ranks and re-ranks in FP32 only (the tensor-core and coarse "
                                           "forms expand the squared Euclidean distance)");
        if (p->threads != 0 && p->threads != 512)
            return fail(SUCO_EUNSUPPORTED, "an L1 index runs CTAs of 512 threads (threads = 0 or 512)");
    }
    if (p->exact_rerank < 0 || p->exact_rerank > (1 << 24))
        return fail(SUCO_EINVAL, "exact_rerank=%d must be in [0, 2^24]", p->exact_rerank);
    if (nq > 0 && (!queries || !ids || !dist)) return fail(SUCO_EINVAL, "queries/out_ids/out_dist must not be NULL");
    return SUCO_OK;
}

}  // namespace
}  // namespace suco

using namespace suco;

extern "C" {

int suco_build_index(const float* data, int64_t n, int32_t d, const suco_build_params* params, void* stream,
                     suco_index** out)
{
    clear_error();
    if (!params || !out || !data) return fail(SUCO_EINVAL, "data, params and out must not be NULL");
    *out = nullptr;
    int rc = check_sizes(n, d, params->Ns, params->sqrtK);
    if (rc) return rc;
    if (params->kmeans_iters < 0 || params->kmeans_iters > 10000)
        return fail(SUCO_EINVAL, "kmeans_iters=%d must be in [0, 10000]", params->kmeans_iters);
    if (params->metric != SUCO_METRIC_L2 && params->metric != SUCO_METRIC_L1)
        return fail(SUCO_EINVAL, "metric=%d must be SUCO_METRIC_L2 or SUCO_METRIC_L1", params->metric);
    if (params->dim_perm && (rc = check_perm(params->dim_perm, d))) return rc;
    const int Ns = params->Ns, sk = params->sqrtK;
    std::vector<int64_t> init((size_t)2 * Ns * sk);
    if (params->init_ids) {
        for (size_t h = 0; h < (size_t)2 * Ns; ++h) {
            std::unordered_set<int64_t> seen;
            for (int a = 0; a < sk; ++a) {
                const int64_t v = params->init_ids[h * sk + a];
                if (v < 0 || v >= n) return fail(SUCO_EINVAL, "init_ids[%zu] = %lld out of range", h * sk + a, (long long)v);
                if (!seen.insert(v).second) return fail(SUCO_EINVAL, "init_ids repeat id %lld within a half", (long long)v);
                init[h * sk + a] = v;
            }
        }
    } else {
        // sqrtK distinct ids per half drawn with splitmix64 (Steele, Lea, Flood 2014)
        uint64_t state = params->seed;
        for (size_t h = 0; h < (size_t)2 * Ns; ++h) {
            std::unordered_set<int64_t> seen;
            int a = 0;
            while (a < sk) {
                const int64_t v = (int64_t)(splitmix64(&state) % (uint64_t)n);
                if (seen.insert(v).second) init[h * sk + a++] = v;
            }
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    suco_index* idx = fault_fires(SUCO_FAULT_ALLOC) ? nullptr : new (std::nothrow) suco_index();
    if (!idx) return fail(SUCO_ENOMEM, "host allocation failed");
    rc = alloc_index(&idx->ix, data, n, d, Ns, sk, params->dim_perm, params->metric, st);
    if (!rc) rc = kmeans_build(&idx->ix, init.data(), params->kmeans_iters, st);
    if (rc) {
        cudaStreamSynchronize(st);
        free_index_memory(&idx->ix);
        delete idx;
        return rc;
    }
    *out = idx;
    return SUCO_OK;
}

int suco_build_index_from_parts(const float* data, int64_t n, int32_t d, const suco_build_params* params,
                                const float* centroids, const int32_t* assign, void* stream, suco_index** out)
{
    clear_error();
    if (!data || !params || !centroids || !assign || !out) return fail(SUCO_EINVAL, "pointers must not be NULL");
    *out = nullptr;
    const int32_t Ns = params->Ns, sqrtK = params->sqrtK;
    int rc = check_sizes(n, d, Ns, sqrtK);
    if (rc) return rc;
    if (params->metric != SUCO_METRIC_L2 && params->metric != SUCO_METRIC_L1)
        return fail(SUCO_EINVAL, "metric=%d must be SUCO_METRIC_L2 or SUCO_METRIC_L1", params->metric);
    if (params->dim_perm && (rc = check_perm(params->dim_perm, d))) return rc;
    for (int64_t t = 0; t < (int64_t)2 * Ns * n; ++t)
        if (assign[t] < 0 || assign[t] >= sqrtK)
            return fail(SUCO_EINVAL, "assign[%lld] = %d out of [0, %d)", (long long)t, assign[t], sqrtK);
    cudaStream_t st = (cudaStream_t)stream;
    suco_index* idx = fault_fires(SUCO_FAULT_ALLOC) ? nullptr : new (std::nothrow) suco_index();
    if (!idx) return fail(SUCO_ENOMEM, "host allocation failed");
    DeviceIndex* ix = &idx->ix;
    rc = alloc_index(ix, data, n, d, Ns, sqrtK, params->dim_perm, params->metric, st);
    DevBuf dassign;
    std::vector<float> cent;
    if (!rc) {
        // copy the centroids with zeroed padding past each half's length
        cent.assign((size_t)Ns * 2 * sqrtK * ix->hmax, 0.f);
        for (int ih = 0; ih < 2 * Ns; ++ih) {
            int32_t off, len;
            half_dims(d, Ns, ix->sub_s, ih >> 1, ih & 1, &off, &len);
            for (int a = 0; a < sqrtK; ++a)
                memcpy(&cent[((size_t)ih * sqrtK + a) * ix->hmax], &centroids[((size_t)ih * sqrtK + a) * ix->hmax],
                       (size_t)len * 4);
        }
        rc = dassign.alloc((size_t)2 * Ns * n * 4);
    }
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(ix->cent, cent.data(), cent.size() * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dassign.p, assign, (size_t)2 * Ns * n * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) rc = fail(SUCO_ECUDA, "copy to the device failed: %s", cudaGetErrorString(e));
    }
    if (!rc) rc = build_imi(ix, dassign.as<int32_t>(), st);
    if (rc) {
        cudaStreamSynchronize(st);
        free_index_memory(ix);
        delete idx;
        return rc;
    }
    *out = idx;
    return SUCO_OK;
}

int suco_build_index_from_assignments(const float* data, int64_t n, int32_t d, int32_t Ns, int32_t sqrtK,
                                      const float* centroids, const int32_t* assign, void* stream, suco_index** out)
{
    suco_build_params p;
    memset(&p, 0, sizeof(p));
    p.Ns = Ns;
    p.sqrtK = sqrtK;
    return suco_build_index_from_parts(data, n, d, &p, centroids, assign, stream, out);
}

int suco_query_batch(const suco_index* index, const float* queries, int64_t nq, const suco_query_params* params,
                     int32_t* out_ids, float* out_dist, void* stream)
{
    clear_error();
    int rc = check_query_params(index, queries, nq, params, out_ids, out_dist);
    if (rc) return rc;
    if ((rc = check_status(&index->ix))) return rc;
    return launch_query(&index->ix, queries, nq, params, out_ids, out_dist, nullptr, (cudaStream_t)stream);
}

int suco_query_debug(const suco_index* index, const float* queries, int64_t nq, const suco_query_params* params,
                     int32_t* out_ids, float* out_dist, const suco_query_debug_out* debug, void* stream)
{
    clear_error();
    int rc = check_query_params(index, queries, nq, params, out_ids, out_dist);
    if (rc) return rc;
    if ((rc = check_status(&index->ix))) return rc;
    return launch_query(&index->ix, queries, nq, params, out_ids, out_dist, debug, (cudaStream_t)stream);
}

int suco_autotune(suco_index* index, const float* queries, int64_t nq, const suco_query_params* params, void* stream,
                  int32_t* cluster_size, int32_t* threads)
{
    clear_error();
    if (!index || !queries || !params || nq < 1) return fail(SUCO_EINVAL, "index, queries, params and nq >= 1 required");
    if (params->cluster_size || params->threads) return fail(SUCO_EINVAL, "autotune needs cluster_size = threads = 0");
    int rc = check_query_params(index, queries, nq, params, (const int32_t*)queries, queries);
    if (rc) return rc;
    DeviceIndex& ix = index->ix;
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf ids, dist;
    if (ids.alloc((size_t)nq * params->k * 4) || dist.alloc((size_t)nq * params->k * 4)) return SUCO_ENOMEM;
    cudaEvent_t e0, e1;
    SUCO_CUDA_TRY(cudaEventCreate(&e0));
    SUCO_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best_cl = 0, best_nt = 0;
    const int cls[] = {1, 2, 4, 8, 16}, nts[] = {256, 512, 1024};
    for (int cl : cls)
        for (int nt : nts) {
            suco_query_params q = *params;
            q.cluster_size = cl;
            q.threads = nt;
            if (launch_query(&ix, queries, nq, &q, ids.as<int32_t>(), dist.as<float>(), nullptr, st) != SUCO_OK) {
                cudaGetLastError();
                continue;  // this shape does not fit
            }
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < 3; ++rep)
                launch_query(&ix, queries, nq, &q, ids.as<int32_t>(), dist.as<float>(), nullptr, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return fail(SUCO_ECUDA, "autotune launch failed: %s", cudaGetErrorString(cudaGetLastError()));
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best_cl = cl;
                best_nt = nt;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!best_cl) return fail(SUCO_EUNSUPPORTED, "no launch shape fits this index and these parameters");
    int64_t T = 0, C = 0;
    thresholds(ix.n, params->alpha, params->beta, params->k, &T, &C);
    for (auto it = ix.tuned.begin(); it != ix.tuned.end();)
        it = (it->k == params->k && it->C == (uint32_t)C) ? ix.tuned.erase(it) : it + 1;
    ix.tuned.push_back({params->k, (uint32_t)C, best_cl, best_nt});
    if (cluster_size) *cluster_size = best_cl;
    if (threads) *threads = best_nt;
    return SUCO_OK;
}

int suco_index_get_info(const suco_index* index, suco_index_info* info)
{
    clear_error();
    if (!index || !info) return fail(SUCO_EINVAL, "index and info must not be NULL");
    const DeviceIndex& ix = index->ix;
    info->n = ix.n;
    info->d = ix.d;
    info->Ns = ix.Ns;
    info->sqrtK = ix.sqrtK;
    info->hmax = ix.hmax;
    info->K = ix.K;
    info->ld = ix.ld;
    info->device_bytes = ix.bytes;
    info->metric = ix.metric;
    info->sampled = ix.dperm != nullptr;
    return SUCO_OK;
}

int suco_export_index(const suco_index* index, float* centroids, uint32_t* cell_off, int32_t* perm)
{
    clear_error();
    if (!index) return fail(SUCO_EINVAL, "index is NULL");
    const DeviceIndex& ix = index->ix;
    if (centroids)
        SUCO_CUDA_TRY(cudaMemcpy(centroids, ix.cent, (size_t)ix.Ns * 2 * ix.sqrtK * ix.hmax * 4, cudaMemcpyDeviceToHost));
    if (cell_off)
        SUCO_CUDA_TRY(cudaMemcpy(cell_off, ix.cell_off, (size_t)ix.Ns * (ix.K + 1) * 4, cudaMemcpyDeviceToHost));
    if (perm) SUCO_CUDA_TRY(cudaMemcpy(perm, ix.perm, (size_t)ix.Ns * ix.n * 4, cudaMemcpyDeviceToHost));
    return SUCO_OK;
}

int suco_thresholds(int64_t n, double alpha, double beta, int32_t k, int64_t* T, int64_t* C)
{
    clear_error();
    if (!T || !C) return fail(SUCO_EINVAL, "T and C must not be NULL");
    if (n < 1) return fail(SUCO_EINVAL, "n must be positive");
    if (!(alpha > 0.0 && alpha <= 1.0) || !(beta > 0.0 && beta <= 1.0) || k < 1)
        return fail(SUCO_EINVAL, "alpha, beta must be in (0, 1] and k >= 1");
    thresholds(n, alpha, beta, k, T, C);
    return SUCO_OK;
}

int suco_read_status(suco_index* index, uint32_t* status)
{
    clear_error();
    if (!index || !status) return fail(SUCO_EINVAL, "index and status must not be NULL");
    SUCO_CUDA_TRY(cudaDeviceSynchronize());
    *status = *index->ix.status_host;
    *index->ix.status_host = 0u;
    return SUCO_OK;
}

int suco_inject_fault(int32_t kind, int32_t after)
{
    clear_error();
    if (kind != SUCO_FAULT_NONE && kind != SUCO_FAULT_ALLOC && kind != SUCO_FAULT_LAUNCH &&
        kind != SUCO_FAULT_WAIT_TIMEOUT)
        return fail(SUCO_EINVAL, "unknown fault kind %d", kind);
    if (after < 0) return fail(SUCO_EINVAL, "after=%d must not be negative", after);
    g_fault_kind.store(SUCO_FAULT_NONE);
    g_fault_after.store(after);
    g_fault_kind.store(kind);
    return SUCO_OK;
}

void suco_free(suco_index* index)
{
    if (!index) return;
    free_index_memory(&index->ix);
    delete index;
}

const char* suco_last_error(void) { return g_err; }

int suco_version(void) { return 100; }

}  // extern "C"
