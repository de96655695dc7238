// Internal definitions shared by the CUDA translation units of libsuco.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "suco.h"

namespace suco {

// The id range [0, n) is cut into nch equal chunks of n_ch ids (n_ch a
// multiple of 32; nch a power of two, at least MIN_NCH, with chunks of at most
// MAX_CHUNK ids).  For every (subspace, cell) the index stores where each
// chunk starts inside the cell's id list, so that a CTA that owns a chunk
// range reads only its own ids of a cell.
constexpr int WORK_SLOTS = 64;
constexpr int WORK_STRIDE = 8;  // 32 bytes per slot
constexpr int MIN_NCH = 64;
// queries per launch pair of the tensor-core ranking (tables workspace rows)
constexpr int64_t RANK_CHUNK = 4096;
constexpr int64_t MAX_CHUNK = 1 << 17;

struct DeviceIndex {
    int64_t n = 0;
    int32_t d = 0;
    int32_t Ns = 0;
    int32_t sqrtK = 0;
    int32_t hmax = 0;
    int32_t sub_s = 0;  // floor(d / Ns)
    int64_t K = 0;
    int64_t ld = 0;     // row stride of X in floats (d rounded up to 4)
    int64_t n_ch = 0;   // ids per chunk
    int32_t nch = 0;    // chunks
    float* X = nullptr;           // [n][ld]; columns d..ld-1 are zero
    uint16_t* Xh = nullptr;       // optional BF16 copy of X, [n][ldh] (ldh = d rounded up to 8), padding zero
    float* rank_ws = nullptr;     // optional [RANK_CHUNK][Ns][2][sqrtK] centroid-distance tables (tensor-core ranking)
    uint8_t* X8 = nullptr;        // optional FP8 E4M3 copy of X / scale, [n][ld8] (ld8 = d rounded up to 16)
    float* s8col = nullptr;       // [ld8] scale of every column (its subspace's), 0 past d
    int64_t ld8 = 0;
    int64_t ldh = 0;
    float* cent = nullptr;        // [Ns][2][sqrtK][hmax]; padding zero
    uint32_t* cell_off = nullptr; // [Ns][K+1] offsets into perm[i]
    int32_t* perm = nullptr;      // [Ns][n] ids grouped by cell, ascending inside a cell
    uint32_t* split = nullptr;    // [Ns][nch+1][K] absolute position in perm[i] where chunk j starts in cell x
    // work counters of persistent query launches: WORK_SLOTS pairs (next query,
    // finished clusters), WORK_STRIDE words apart, zero between launches; calls
    // take the slots in turn (work_next), so up to WORK_SLOTS calls on one index
    // may be in flight at once
    uint32_t* work = nullptr;
    uint32_t work_next = 0;
    // status word in mapped (pinned) host memory: a kernel whose bounded wait
    // gives up stores SUCO_STATUS_WAIT_TIMEOUT through status_dev; the host
    // reads status_host without synchronising
    volatile uint32_t* status_host = nullptr;
    uint32_t* status_dev = nullptr;
    int32_t metric = SUCO_METRIC_L2;
    // Definition 3's subspace sampling: X holds column dperm[j] of D at column
    // j, so every sampled subspace is contiguous; queries are read through it
    int32_t* dperm = nullptr;     // device [d], or null for contiguous subspaces
    int device = 0;
    int64_t bytes = 0;
    // launch shapes chosen by suco_autotune, per (k, candidate bound C)
    struct Tuned {
        int32_t k;
        uint32_t C;
        int32_t CL;
        int32_t NT;
    };
    std::vector<Tuned> tuned;
};

// Half-subspace geometry (Definition 3 contiguous case; Algorithm 2 halves).
__host__ __device__ inline void half_dims(int32_t d, int32_t Ns, int32_t sub_s, int32_t i, int32_t h,
                                          int32_t* off, int32_t* len)
{
    int32_t so = i * sub_s;
    int32_t sl = (i == Ns - 1) ? d - (Ns - 1) * sub_s : sub_s;
    int32_t first = sl / 2;
    *off = so + (h ? first : 0);
    *len = h ? sl - first : first;
}

// Error reporting: thread-local message, negative status.
int fail(int code, const char* fmt, ...);
void clear_error();

// Failure injection (suco_inject_fault): true when an armed fault of this
// kind fires now (it then disarms itself).
bool fault_fires(int32_t kind);
// After a kernel launch: an injected launch fault, or the launch's own error.
int launch_status(const char* what);
// A status word set by a kernel's bounded wait (or by an injected fault).
int check_status(const DeviceIndex* ix);

// Device memory with automatic release.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    int alloc(size_t b);
    template <class T> T* as() const { return static_cast<T*>(p); }
    void* release() { void* q = p; p = nullptr; return q; }
};

int build_imi(DeviceIndex* ix, const int32_t* assign_dev /*[Ns][2][n]*/, cudaStream_t st);
int kmeans_build(DeviceIndex* ix, const int64_t* init_ids_host, int32_t iters, cudaStream_t st);
// the query value a kernel stages at column j of a (possibly sampled) index
__device__ __forceinline__ float query_col(const float* q_row, const int32_t* dperm, int j)
{
    return q_row[dperm ? __ldg(dperm + j) : j];
}
int rank_tc_tables(const DeviceIndex* ix, const float* Q, int64_t nq, float* D, bool fp8, cudaStream_t st);
int launch_query(const DeviceIndex* ix, const float* Q, int64_t nq, const suco_query_params* p, int32_t* ids,
                 float* dist, const suco_query_debug_out* dbg, cudaStream_t st);

void thresholds(int64_t n, double alpha, double beta, int32_t k, int64_t* T, int64_t* C);

}  // namespace suco

struct suco_index {
    suco::DeviceIndex ix;
};

#define SUCO_LAUNCH_CHECK(what)                      \
    do {                                             \
        int rc_ = ::suco::launch_status(what);       \
        if (rc_) return rc_;                         \
    } while (0)

#define SUCO_CUDA_TRY(expr)                                                                          \
    do {                                                                                             \
        cudaError_t e_ = (expr);                                                                     \
        if (e_ != cudaSuccess) return ::suco::fail(SUCO_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)
