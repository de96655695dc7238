// The SuCo query path (Section 4.2: Algorithm 4, with Algorithm 3's cell walk)
// as one kernel in which a thread-block cluster of CL CTAs answers one query at
// a time; the grid holds as many clusters as fit on the GPU at once and each
// cluster loops over its share of the batch.
//
// Stages inside the kernel (one launch, no global scratch):
//   S0  the query row is staged in shared memory (copied in during the
//       previous query's S6 when the next query is already known).
//   S1  squared half-subspace centroid distances d1[a], d2[c] in FP32
//       (acc = fma(q_j - c_j, q_j - c_j, acc) over j ascending).
//   S2  stable ranks r1[a], r2[c] of those distances (ties by centroid index)
//       and their inverses idx1, idx2 (rank -> centroid).
//   S3  cell activation.  Algorithm 3 retrieves cells in ascending order of the
//       key (f32 bits of d1[a]+d2[c], r1[a], r2[c]) until alpha*n ids are
//       collected, so the retrieved cells are exactly those with key <= kappa*,
//       where kappa* is the smallest key whose cumulative cell size reaches T.
//       kappa* is found by a weighted histogram over linear value buckets of
//       the cell sums (one pass over the K cells), then among the few cells of
//       the bucket that crosses T (by counting smaller keys, or a weighted radix
//       select when the bucket is crowded).  Because the key grows along every
//       ranked row, the retrieved cells of a row form a prefix of that row in
//       r2 order: the retrieved set is a "staircase", published as row prefix
//       sums.  CTA r handles the subspaces i with i % CL == r (two at once, one
//       per half of the CTA, when it owns two).
//   S4  SC-score counting (Definition 4).  Each CTA owns a contiguous id range
//       and keeps the ids' SC-score counters in shared memory (4-bit counters
//       for up to 15 subspaces, one-bit planes past them).  It lists its part
//       of every retrieved cell's id list of every subspace (the index's chunk
//       splits), load-balances the flattened list over warps in 16-byte quads
//       of ids and adds 1 to each listed id's counter with one shared-memory
//       atomicAdd (an id occurs at most once per subspace, so a counter never
//       overflows); the counters are then turned into B = bits(Ns) bit planes.
//   S5  candidate selection.  Per-warp counts of scores >= s (bitwise
//       comparisons of the sliced counts) are summed over the cluster through
//       distributed shared memory; theta is the largest s with at least C
//       scores >= s; every id above theta and the lowest-id ties at theta
//       (C in total) are written, in id order, straight into the candidate
//       slots of the CTA that re-ranks them.
//   S6  exact re-rank: every CTA computes FP32 squared distances of its share
//       of the C candidates (8 lanes per row, several rows in flight per warp),
//       keeps a local top-k by (distance, id), and CTA 0 merges the CL sorted
//       lists by rank.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "suco_internal.cuh"

namespace suco {
namespace {

constexpr int MAXSEG = 512;   // retrieved-cell segments listed per scan round
constexpr int NB = 1024;      // linear value buckets of the cut search
constexpr int MCAP = 1024;    // cells of the crossing bucket resolved from a list
constexpr int SCAN_U = 3;     // 16-byte quads of ids in flight per lane in the scan
constexpr int NCLK = 20;      // per-stage clock stamps per (query, CTA) of the debug output

constexpr int S3_BYTES = 4 * NB + 12 * MCAP;  // S3 scratch at the start of the union region
constexpr int HIST_WORDS = 256 + 64;          // o_hist per S3 group: a 256-bin histogram, scan scratch
constexpr int SURV_CAP = 512; // keys kept for the final sort of a local top-k
// 16-byte chunks per lane per row in one S6 load round: 2 for rows of 64 to
// 127 chunks, 4 otherwise (measured at 32, 64 and 240 chunks)
constexpr int S6_CH_SHORT = 4, S6_CH_LONG = 2;

struct QArgs {
    const float* __restrict__ X;
    int64_t ld;
    int64_t n;
    int32_t d, Ns, sqrtK, K, hmax, sub_s;
    const float* __restrict__ cent;
    const uint32_t* __restrict__ cell_off;
    const int32_t* __restrict__ perm;
    const uint32_t* __restrict__ split;
    int64_t n_ch;
    int32_t cpc;  // chunks per CTA
    int32_t CL;
    const float* __restrict__ Q;
    int64_t nq;
    int32_t k, k_pad;
    uint32_t T, C, per_cta;  // scalar thresholds; C and per_cta are also the bounds of per-query values
    double alpha, beta;
    const int32_t* k_per;    // optional per-query k, alpha, beta
    const float* alpha_per;
    const float* beta_per;
    uint32_t* work;          // (next query, finished clusters) of this launch, zero at start; or null
    uint32_t span, G;  // ids per CTA, 32-id groups per CTA
    uint32_t nbits;    // B: bit planes of the sliced SC-score counts
    uint32_t nsets, nplanes, nstore;  // S4 counters: 4-bit nibble sets, one-bit planes, words per 32 ids
    const uint16_t* __restrict__ Xh;   // BF16 copy of X, [n][ldh] (precision 1)
    int64_t ldh;
    int64_t ldq;                       // staged query length (d rounded up to 16, zero padded)
    int32_t precision;                 // 0 exact FP32 re-rank; 1 BF16 coarse pass, then FP32 on R survivors
    uint32_t R;                        // survivors of the coarse pass
    uint8_t* dbg_surv;                 // [nq][n] 1 for the coarse pass's survivors (debug)
    uint32_t o_rsel;                   // [2][256] published radix histograms of the survivor cut
    uint32_t npass;                    // passes over the id range (S4 + S5 per pass)
    uint32_t o_run, run_stride;        // running candidate list of a multi-pass query: ids [2][stride], scores [2][stride]
    int32_t nch;                       // id chunks of the index (rows of split per subspace, minus one)
    const float* dtab_in;              // [nq][Ns][2][sqrtK] centroid distances computed before (BF16 ranking) or null
    const uint8_t* __restrict__ X8;    // FP8 E4M3 copy of X / column scale, [n][ld8] (precision 2)
    int64_t ld8;
    const float* __restrict__ s8col;   // [ld8] column scales of the FP8 copy
    const int32_t* __restrict__ qperm;   // Definition 3 sampling: staged query column j = q[qperm[j]] (or null)
    int32_t* out_ids;
    float* out_dist;
    int64_t* dbg_teff;
    uint8_t* dbg_act;
    float* dbg_dtab;
    uint8_t* dbg_scores;
    int32_t* dbg_cands;
    long long* dbg_clk;  // [nq][16][NCLK] per-stage clock64 stamps, row r = CTA r (debug)
    // shared-memory layout (byte offsets)
    uint32_t o_tab, tab_stride, o_q, o_hist, o_misc, o_cnt, o_seg, o_slots, o_keys, o_union;
    uint32_t sortP;       // power of two >= the CTA's candidate share (fallback sort)
    uint32_t stage_cent;  // 1: the subspace's centroids are staged in shared memory
    uint32_t o_cells;     // nonzero: the subspace's cell offsets are copied to o_union + o_cells for S3
    uint32_t tab_copy;    // leading bytes of a subspace table that the other CTAs copy (a multiple of 16)
    uint32_t o_qn;        // the next query's row, copied in while S6 runs
    uint32_t s3_stride;   // bytes of one S3 scratch group in the union region
    uint32_t pair_ok;     // 1: a CTA that owns two subspaces ranks them at once, one per half
    uint32_t o_bkt;       // nonzero: S3 keeps every cell's value bucket (u16) at o_union + group + o_bkt
};

// ---------------------------------------------------------------------------
// cluster / distributed-shared-memory primitives (inline PTX)

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// The .aligned barrier must be executed by every thread of a warp together:
// __syncwarp() reconverges the warp first (the compiler does not know that the
// inline barrier needs convergence).
__device__ __forceinline__ void cluster_sync()
{
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t map_rank(uint32_t local_addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
    return r;
}

__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ uint4 ld_cluster_v4(uint32_t addr)
{
    uint4 v;
    asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// 16-byte global load that bypasses L1 (candidate rows are read once)
// asynchronous 4-byte global -> shared copy (completes at cp_async_wait_all)
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ float4 ldg_stream(const float4* p)
{
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

// Per-stage clock stamp of the debug output: thread 0 of each CTA records its
// SM clock (after the stage's closing barrier) in slot `slot` of the
// (query, CTA) row; slot 0 holds the SM id, the last two the cycles S4 spent
// building segment lists and scanning them.
__device__ __forceinline__ void stamp(const QArgs& A, int64_t b, uint32_t r, int slot)
{
    if (A.dbg_clk && threadIdx.x == 0) {
        long long* row = A.dbg_clk + (b * 16 + r) * NCLK;
        if (slot == 1) {
            uint32_t sm;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
            row[0] = (long long)sm;
        }
        row[slot] = clock64();
    }
}

// ---------------------------------------------------------------------------

// One dimension's term of the index's distance in FP32: squared Euclidean by
// one fused multiply-add (MET 0), Manhattan by one addition (MET 1).
template <int MET>
__device__ __forceinline__ float dterm(float acc, float df)
{
    return MET == 1 ? __fadd_rn(acc, fabsf(df)) : __fmaf_rn(df, df, acc);
}

// Cell key of Algorithm 3's retrieval order: FP32 cell sum, then the ranks.
__device__ __forceinline__ unsigned long long cell_key(float a, float b, uint32_t r1, uint32_t r2)
{
    const float s = __fadd_rn(a, b);
    return ((unsigned long long)__float_as_uint(s) << 16) | (r1 << 8) | r2;
}

// One subspace's tables in shared memory (identical layout in every CTA).
struct Tab {
    unsigned long long* kappa;
    unsigned long long* teff;
    uint32_t* row_pre;  // [sqrtK+1] retrieved cells before each ranked row
    float* d1;
    float* d2;
    uint8_t* idx1;      // rank -> centroid
    uint8_t* idx2;
    uint8_t* r1;        // centroid -> rank
    uint8_t* r2;
};

__device__ __forceinline__ Tab tab_at(char* smem, const QArgs& A, int i)
{
    char* t = smem + A.o_tab + (size_t)i * A.tab_stride;
    const int sk = A.sqrtK;
    Tab T;
    // what the other CTAs read (the staircase and the rank -> centroid maps)
    // comes first, in the tab_copy bytes they copy; the owner's S1-S3 state after
    T.kappa = reinterpret_cast<unsigned long long*>(t);
    T.teff = reinterpret_cast<unsigned long long*>(t + 8);
    T.row_pre = reinterpret_cast<uint32_t*>(t + 16);
    T.idx1 = reinterpret_cast<uint8_t*>(t + 20 + 4 * sk);
    T.idx2 = T.idx1 + sk;
    T.d1 = reinterpret_cast<float*>(t + A.tab_copy);
    T.d2 = T.d1 + sk;
    T.r1 = reinterpret_cast<uint8_t*>(T.d2 + sk);
    T.r2 = T.r1 + sk;
    return T;
}

// Barrier over a group of NT threads (whole warps): id 0 with NT = the CTA's
// size is __syncthreads(); ids 1 and 2 are the two halves of the CTA.
template <int NT>
__device__ __forceinline__ void group_sync(int bar)
{
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(NT) : "memory");
}

// Exclusive prefix sum over a group of NT threads (tid within the group,
// barrier id bar); *total gets the group's sum.
template <int NT>
__device__ __forceinline__ uint32_t group_exclusive_scan(uint32_t v, uint32_t* wtmp, uint32_t* total, int tid, int bar)
{
    const int lane = tid & 31, w = tid >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtmp[w] = incl;
    group_sync<NT>(bar);
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
    group_sync<NT>(bar);
    const uint32_t res = wtmp[w] + incl - v;
    *total = wtmp[32];
    group_sync<NT>(bar);
    return res;
}

template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* wtmp, uint32_t* total)
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
    const uint32_t res = wtmp[w] + incl - v;
    *total = wtmp[32];
    __syncthreads();
    return res;
}

// The same over 64-bit values (two 32-bit sums carried in one scan).
template <int NT>
__device__ __forceinline__ unsigned long long block_exclusive_scan64(unsigned long long v, unsigned long long* wtmp,
                                                                     unsigned long long* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtmp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const unsigned long long t = lane < NT / 32 ? wtmp[lane] : 0ull;
        unsigned long long ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        wtmp[lane] = ti - t;
        if (lane == 31) wtmp[32] = ti;
    }
    __syncthreads();
    const unsigned long long res = wtmp[w] + incl - v;
    *total = wtmp[32];
    __syncthreads();
    return res;
}

template <int NT>
__device__ void block_bitonic_sort(unsigned long long* a, int P)
{
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += NT) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long x = a[lo], y = a[hi];
                if ((x > y) == asc) {
                    a[lo] = y;
                    a[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

// Slot of this lane among the lanes of its warp with pred set, after one
// atomicAdd of their number on *ctr (a warp's lanes would otherwise queue on
// the same shared word one by one).  Every lane of the warp calls it.
__device__ __forceinline__ uint32_t warp_alloc(uint32_t* ctr, bool pred)
{
    const int lane = threadIdx.x & 31;
    const uint32_t m = __ballot_sync(0xffffffffu, pred);
    const int leader = m ? __ffs(m) - 1 : 0;
    uint32_t base = 0u;
    if (m && lane == leader) base = atomicAdd(ctr, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + (uint32_t)__popc(m & ((1u << lane) - 1u));
}

// Number of keys smaller than v over CLT sorted lists of k keys each
// (all + o*k), by CLT binary searches taken in lock step: every step issues
// one unconditional (clamped) load per list, so a step costs one shared-memory
// round trip instead of CLT dependent ones.  P is a power of two with P > k.
// v's own list contributes v's position in it (keys are unique).
template <int CLT>
__device__ __forceinline__ uint32_t rank_in_lists(const unsigned long long* all, uint32_t k, uint32_t P,
                                                  unsigned long long v)
{
    uint32_t pos[CLT];
#pragma unroll
    for (int o = 0; o < CLT; ++o) pos[o] = 0u;
    for (uint32_t st = P >> 1; st; st >>= 1) {
        unsigned long long x[CLT];
#pragma unroll
        for (int o = 0; o < CLT; ++o) x[o] = all[(uint32_t)o * k + min(pos[o] + st, k) - 1u];
#pragma unroll
        for (int o = 0; o < CLT; ++o) pos[o] = (pos[o] + st <= k && x[o] < v) ? pos[o] + st : pos[o];
    }
    uint32_t rank = 0u;
#pragma unroll
    for (int o = 0; o < CLT; ++o) rank += pos[o];
    return rank;
}

__device__ __forceinline__ uint32_t next_pow2_dev(uint32_t x)
{
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Sorts in[0, n) ascending into out[0, n) by rank: the key at t goes to the
// number of keys below it plus the number of equal keys before t.  Every
// thread of a warp reads the same in[j] (a broadcast), the loads do not depend
// on one another, and there is no chain of exchange steps as in a sorting
// network; for the few keys it is used on (n <= 128) that is the shorter path.
template <int NT>
__device__ __forceinline__ void rank_sort(const unsigned long long* in, uint32_t n, unsigned long long* out)
{
    for (uint32_t t = threadIdx.x; t < n; t += NT) {
        const unsigned long long v = in[t];
        uint32_t rank = 0u;
        for (uint32_t j = 0; j < n; ++j) {
            const unsigned long long x = in[j];
            rank += (uint32_t)(x < v) | ((uint32_t)(x == v) & (uint32_t)(j < t));
        }
        out[rank] = v;
    }
}

// Value bucket of a cell sum: monotone non-decreasing in s (FP32 subtract,
// multiply and truncation are all monotone), so bucket order respects key order.
__device__ __forceinline__ int value_bucket(float s, float smin, float scale)
{
    if (!(s > smin)) return 0;
    const float t = fminf(__fmul_rn(__fsub_rn(s, smin), scale), (float)(NB - 1));
    return (int)t;
}

// S1-S3 for subspace i of query b (the CTA that owns i), by a group of NT
// threads: the whole CTA (tid = tid, barrier 0, scratch group 0), or
// one half of it when the CTA ranks two subspaces at once (tid within the
// half, named barrier 1 or 2, scratch group 0 or 1: its own S3 area of the
// union, its own o_hist histograms and o_misc slots).
template <int NT, int MET>
__device__ void rank_subspace(const QArgs& A, char* smem, int64_t b, int i, uint32_t T, int tid, int bar, int grp)
{
    const int sk = A.sqrtK;
    const int lane = tid & 31;
    const float* qs = reinterpret_cast<const float*>(smem + A.o_q);
    Tab tb = tab_at(smem, A, i);
    const int soff = i * A.sub_s;
    const int slen = (i == A.Ns - 1) ? A.d - (A.Ns - 1) * A.sub_s : A.sub_s;
    const int first = slen / 2;
    // the subspace's cell offsets (the index's cell sizes) are copied to shared
    // memory while S1 and S2 run; S3 reads each of them up to twice
    const uint32_t* co = A.cell_off + (int64_t)i * (A.K + 1);
    uint32_t* co_s = A.o_cells ? reinterpret_cast<uint32_t*>(smem + A.o_union + grp * A.s3_stride + A.o_cells) : nullptr;
    if (co_s)
        for (int t = tid; t <= A.K; t += NT) cp_async4(co_s + t, co + t);
    // S1: squared distances to the 2*sqrtK half-subspace centroids.  The
    // subspace's centroids are staged dimension-major ([h][j][a]) so that
    // consecutive threads read consecutive words.
    const float* cg = A.cent + (int64_t)i * 2 * sk * A.hmax;
    float* cst = reinterpret_cast<float*>(smem + A.o_union + grp * A.s3_stride + S3_BYTES);
    if (A.stage_cent) {
        for (int t = tid; t < 2 * sk * A.hmax; t += NT) {
            const int j = t % A.hmax, ha = t / A.hmax;
            const int h = ha >= sk, a = ha - h * sk;
            cst[(h * A.hmax + j) * sk + a] = __ldg(cg + t);
        }
        group_sync<NT>(bar);
    }
    for (int t = tid; t < 2 * sk; t += NT) {
        const int h = t >= sk;
        const int a = t - h * sk;
        if (A.dtab_in) {  // tables of the tensor-core ranking
            (h ? tb.d2 : tb.d1)[a] = A.dtab_in[((b * A.Ns + i) * 2 + h) * sk + a];
            continue;
        }
        const int off = soff + (h ? first : 0);
        const int len = h ? slen - first : first;
        float acc = 0.f;
        if (A.stage_cent) {
            const float* c = cst + h * A.hmax * sk + a;
            for (int j = 0; j < len; ++j) acc = dterm<MET>(acc, __fsub_rn(qs[off + j], c[j * sk]));
        } else {
            const float* c = cg + (int64_t)(h * sk + a) * A.hmax;
            for (int j = 0; j < len; ++j) acc = dterm<MET>(acc, __fsub_rn(qs[off + j], __ldg(c + j)));
        }
        (h ? tb.d2 : tb.d1)[a] = acc;
    }
    group_sync<NT>(bar);
    // S2: stable ranks and their inverses
    for (int t = tid; t < 2 * sk; t += NT) {
        const int h = t >= sk;
        const int a = t - h * sk;
        const float* dd = h ? tb.d2 : tb.d1;
        const float v = dd[a];
        int r = 0;
        for (int c = 0; c < sk; ++c) {
            const float w = dd[c];
            r += (w < v) || (w == v && c < a);
        }
        (h ? tb.r2 : tb.r1)[a] = (uint8_t)r;
        (h ? tb.idx2 : tb.idx1)[r] = (uint8_t)a;
    }
    group_sync<NT>(bar);

    // S3: the cut key kappa*
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + A.o_union + grp * A.s3_stride);  // [NB]
    unsigned long long* mkey = reinterpret_cast<unsigned long long*>(hist + NB);    // [MCAP]
    uint32_t* mw = reinterpret_cast<uint32_t*>(mkey + MCAP);                        // [MCAP]
    uint32_t* wtmp = reinterpret_cast<uint32_t*>(smem + A.o_hist) + grp * HIST_WORDS + 256;
    uint32_t* h256 = reinterpret_cast<uint32_t*>(smem + A.o_hist) + grp * HIST_WORDS;
    unsigned long long* bc = reinterpret_cast<unsigned long long*>(smem + A.o_misc + 64 * grp);  // [7] per group
    uint32_t* mcount = reinterpret_cast<uint32_t*>(smem + A.o_misc + 64 * grp) + 14;
    auto cell_size = [&](uint32_t x) -> uint32_t {
        return co_s ? co_s[x + 1] - co_s[x] : __ldg(co + x + 1) - __ldg(co + x);
    };
    const float smin = __fadd_rn(tb.d1[tb.idx1[0]], tb.d2[tb.idx2[0]]);
    const float smax = __fadd_rn(tb.d1[tb.idx1[sk - 1]], tb.d2[tb.idx2[sk - 1]]);
    const float range = __fsub_rn(smax, smin);
    const float scale = range > 0.f ? __fdiv_rn((float)NB, range) : 0.f;
    // 2-D mapping of threads onto cells: 2^lg threads per centroid row
    int lg = 0;
    while ((1 << lg) < sk) ++lg;
    const int c_of = tid & ((1 << lg) - 1);
    const int a_of = tid >> lg;
    const int a_step = NT >> lg;

    for (int t = tid; t < NB; t += NT) hist[t] = 0u;
    if (tid == 0) *mcount = 0u;
    if (co_s) cp_async_wait_all();
    group_sync<NT>(bar);
    // with a bucket store, cells in flat order x = a * sqrtK + c (thread tid
    // takes x = tid, tid + NT, ..., stepping (a, c) without a division) and
    // each cell's bucket kept for the member search; else the 2-D mapping
    uint16_t* bkt = A.o_bkt ? reinterpret_cast<uint16_t*>(smem + A.o_union + grp * A.s3_stride + A.o_bkt) : nullptr;
    const int K = sk * sk, step_a = NT / sk, step_c = NT - step_a * sk;
    if (bkt) {
        int a = tid / sk, c = tid - a * sk;
        for (int x = tid; x < K; x += NT) {
            const int bk = value_bucket(__fadd_rn(tb.d1[a], tb.d2[c]), smin, scale);
            bkt[x] = (uint16_t)bk;
            const uint32_t w = cell_size((uint32_t)x);
            if (w) atomicAdd(&hist[bk], w);
            a += step_a;
            c += step_c;
            if (c >= sk) {
                c -= sk;
                ++a;
            }
        }
    } else if (c_of < sk) {
        const float d2c = tb.d2[c_of];
        for (int a = a_of; a < sk; a += a_step) {
            const uint32_t x = (uint32_t)(a * sk + c_of);
            const uint32_t w = cell_size(x);
            if (w) atomicAdd(&hist[value_bucket(__fadd_rn(tb.d1[a], d2c), smin, scale)], w);
        }
    }
    group_sync<NT>(bar);
    // crossing bucket: exclusive prefix < T <= inclusive prefix
    {
        constexpr int BPT = NB / NT > 0 ? NB / NT : 1;
        uint32_t v[BPT], s = 0;
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
            const int e = tid * BPT + u;
            v[u] = e < NB ? hist[e] : 0u;
            s += v[u];
        }
        uint32_t tot;
        uint32_t run = group_exclusive_scan<NT>(s, wtmp, &tot, tid, bar);
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
            const int e = tid * BPT + u;
            if (e < NB && run < T && run + v[u] >= T) {
                bc[3] = (unsigned long long)e;
                bc[4] = run;
            }
            run += v[u];
        }
    }
    group_sync<NT>(bar);
    const int bstar = (int)bc[3];
    unsigned long long below = bc[4];
    // members of the crossing bucket (non-empty cells only)
    if (bkt) {
        int a = tid / sk, c = tid - a * sk;
        for (int x = tid; x < K; x += NT) {
            if (bkt[x] == (uint16_t)bstar) {
                const uint32_t w = cell_size((uint32_t)x);
                if (w) {
                    const float s = __fadd_rn(tb.d1[a], tb.d2[c]);
                    const uint32_t slot = atomicAdd(mcount, 1u);
                    if (slot < MCAP) {
                        mkey[slot] = ((unsigned long long)__float_as_uint(s) << 16) | ((uint32_t)tb.r1[a] << 8) |
                                     (uint32_t)tb.r2[c];
                        mw[slot] = w;
                    }
                }
            }
            a += step_a;
            c += step_c;
            if (c >= sk) {
                c -= sk;
                ++a;
            }
        }
    } else if (c_of < sk) {
        const float d2c = tb.d2[c_of];
        const uint32_t r2c = tb.r2[c_of];
        for (int a = a_of; a < sk; a += a_step) {
            const float s = __fadd_rn(tb.d1[a], d2c);
            if (value_bucket(s, smin, scale) != bstar) continue;
            const uint32_t x = (uint32_t)(a * sk + c_of);
            const uint32_t w = cell_size(x);
            if (!w) continue;
            const uint32_t slot = atomicAdd(mcount, 1u);
            if (slot < MCAP) {
                mkey[slot] = ((unsigned long long)__float_as_uint(s) << 16) | ((uint32_t)tb.r1[a] << 8) | r2c;
                mw[slot] = w;
            }
        }
    }
    group_sync<NT>(bar);
    const uint32_t nm = *mcount;
    const bool listed = nm <= MCAP;
    unsigned long long prefix = 0, mask = 0, last_w = 0;
    int pass0 = 0;
    if (nm <= 32) {
        // few members: lane m adds up the weights of the members with smaller
        // keys (broadcast loads, no dependent chain; keys are unique); the cut
        // cell is the member whose weight interval covers the remaining need
        if (tid < 32) {
            const bool act = lane < (int)nm;
            const unsigned long long key = act ? mkey[lane] : ~0ull;
            const uint32_t w = act ? mw[lane] : 0u;
            uint32_t excl = 0u;
            for (uint32_t j = 0; j < nm; ++j) excl += mkey[j] < key ? mw[j] : 0u;
            const uint32_t incl = excl + w;
            const uint32_t need = (uint32_t)(T - below);
            const uint32_t hit = __ballot_sync(0xffffffffu, act && excl < need && incl >= need);
            const int src = __ffs(hit) - 1;
            if (lane == src) {
                bc[0] = key;
                bc[1] = incl;
            }
        }
        group_sync<NT>(bar);  // nothing writes bc again before the staircase's barrier
        prefix = bc[0];
        last_w = 0;
        below += bc[1];
        pass0 = 6;
    } else if (listed) {
        // bytes shared by every member are already decided
        unsigned long long* kmm = bc + 5;  // [5] = min, [6] = max
        if (tid == 0) {
            kmm[0] = ~0ull;
            kmm[1] = 0ull;
        }
        group_sync<NT>(bar);
        unsigned long long lo = ~0ull, hi = 0ull;
        for (uint32_t m = tid; m < nm; m += NT) {
            lo = min(lo, mkey[m]);
            hi = max(hi, mkey[m]);
        }
        if (lo != ~0ull) atomicMin(&kmm[0], lo);
        if (hi) atomicMax(&kmm[1], hi);
        group_sync<NT>(bar);
        const unsigned long long diff = kmm[0] ^ kmm[1];
        while (pass0 < 6 && ((diff >> (40 - 8 * pass0)) & 255ull) == 0) {
            mask |= 255ull << (40 - 8 * pass0);
            ++pass0;
        }
        prefix = kmm[0] & mask;
        group_sync<NT>(bar);
    }
    // weighted radix select of the cut key over the bucket's members
    for (int pass = pass0; pass < 6; ++pass) {
        const int shift = 40 - 8 * pass;
        for (int t = tid; t < 256; t += NT) h256[t] = 0u;
        group_sync<NT>(bar);
        if (listed) {
            for (uint32_t m = tid; m < nm; m += NT) {
                const unsigned long long key = mkey[m];
                if ((key & mask) == prefix) atomicAdd(&h256[(key >> shift) & 255u], mw[m]);
            }
        } else if (c_of < sk) {
            const float d2c = tb.d2[c_of];
            const uint32_t r2c = tb.r2[c_of];
            for (int a = a_of; a < sk; a += a_step) {
                const float s = __fadd_rn(tb.d1[a], d2c);
                if (value_bucket(s, smin, scale) != bstar) continue;
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(s) << 16) | ((uint32_t)tb.r1[a] << 8) | r2c;
                if ((key & mask) != prefix) continue;
                const uint32_t x = (uint32_t)(a * sk + c_of);
                const uint32_t w = cell_size(x);
                if (w) atomicAdd(&h256[(key >> shift) & 255u], w);
            }
        }
        group_sync<NT>(bar);
        if (tid < 32) {
            uint32_t v[8];
            uint32_t s = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = h256[lane * 8 + j];
                s += v[j];
            }
            uint32_t incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - s;
            const uint32_t need = (uint32_t)(T - below);
            if (excl < need && incl >= need) {
                uint32_t cum = excl;
                int bin = lane * 8 + 7;
                uint32_t wbin = v[7];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (cum + v[j] >= need) {
                        bin = lane * 8 + j;
                        wbin = v[j];
                        break;
                    }
                    cum += v[j];
                }
                bc[0] = (unsigned long long)bin;
                bc[1] = cum;
                bc[2] = wbin;
            }
        }
        group_sync<NT>(bar);
        prefix |= bc[0] << shift;
        mask |= 255ull << shift;
        below += bc[1];
        last_w = bc[2];
        group_sync<NT>(bar);
    }
    // after the warp path `below` already counts the cut cell itself
    // the staircase: retrieved cells of ranked row rho are its first columns in
    // r2 order (the key grows along the row); store lengths, then prefix sums
    for (int rho = tid; rho < sk; rho += NT) {
        const int a = tb.idx1[rho];
        const float d1a = tb.d1[a];
        int lo = 0, hi = sk;  // number of columns with key <= kappa*
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const int c = tb.idx2[mid];
            if (cell_key(d1a, tb.d2[c], (uint32_t)rho, (uint32_t)mid) <= prefix) lo = mid + 1; else hi = mid;
        }
        tb.row_pre[rho + 1] = (uint32_t)lo;
    }
    group_sync<NT>(bar);
    if (tid < 32) {
        constexpr int RPL = 8;  // sqrtK <= 256 rows, 8 per lane
        uint32_t v[RPL], s = 0;
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
            const int rho = lane * RPL + u;
            v[u] = rho < sk ? tb.row_pre[rho + 1] : 0u;
            s += v[u];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncwarp();
        uint32_t run = incl - s;
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
            const int rho = lane * RPL + u;
            if (rho < sk) tb.row_pre[rho] = run;
            run += v[u];
        }
        if (lane == 31) tb.row_pre[sk] = run;
        if (lane == 0) {
            *tb.kappa = prefix;
            *tb.teff = below + last_w;
        }
    }
    group_sync<NT>(bar);
    if (A.dbg_teff && tid == 0) A.dbg_teff[b * A.Ns + i] = (int64_t)*tb.teff;
    if (A.dbg_dtab)
        for (int t = tid; t < 2 * sk; t += NT)
            A.dbg_dtab[(b * A.Ns + i) * 2 * sk + t] = t < sk ? tb.d1[t] : tb.d2[t - sk];
    if (A.dbg_act)
        for (int x = tid; x < A.K; x += NT) {
            const int a = x / sk, c = x - a * sk;
            A.dbg_act[(b * A.Ns + i) * A.K + x] = cell_key(tb.d1[a], tb.d2[c], tb.r1[a], tb.r2[c]) <= prefix;
        }
    group_sync<NT>(bar);
}

// S4 for entries [e0, e0+m) of the flattened retrieved-cell list (all
// subspaces, subspace-major): build the segments (this CTA's part of each
// cell's id list), then count their ids.  An id occurs at most once per
// subspace (every point lies in exactly one cell of each IMI), so subspace i
// adds 1 to the id's 4-bit counter of nibble set i / 15 (at most 15 increments
// each, no overflow), or sets the id's bit in a one-bit plane for the
// subspaces past the nibble sets: one shared-memory atomicAdd per id.
// Layout of a nibble set (4 words per 32-id group g): id 32g + t sits in word
// (t & 3) of the set, nibble t >> 2, i.e. bits [t & 28, (t & 28) + 4).
template <int NT>
__device__ void scan_segments(const QArgs& A, char* smem, uint32_t e0, uint32_t m, const uint32_t* sub_pre,
                              const uint32_t* sub_wb, uint32_t* cnt_words, uint32_t id0, int j0, int j1,
                              long long* cyc)
{
    // cyc (debug, thread 0 only): [0] += cycles listing segments, [1] += cycles
    // scanning them, accumulated in place so that no value lives across the scan
    if (cyc) cyc[0] -= clock64();
    // the non-empty segments in flat order, counted in 16-byte quads of the id
    // lists (perm): {quad index of the first quad minus the flat start, perm
    // position of the first id, perm position past the last id, counter word
    // base | nibble flag}, and their flat starts
    uint4* seg_info = reinterpret_cast<uint4*>(smem + A.o_seg);          // [MAXSEG]
    uint32_t* seg_pre = reinterpret_cast<uint32_t*>(seg_info + MAXSEG);  // [MAXSEG+1]
    const int sk = A.sqrtK;
    constexpr int EPT = (MAXSEG + NT - 1) / NT;
    uint32_t nqd[EPT], pP[EPT], pE[EPT], mode[EPT], s = 0, ne = 0;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
        const uint32_t e = threadIdx.x * EPT + u;
        nqd[u] = 0;
        pP[u] = 0;
        pE[u] = 0;
        mode[u] = 0;
        if (e < m) {
            const uint32_t g = e0 + e;
            int i = 0, ihi = A.Ns - 1;  // the last subspace whose list starts at or before g
            while (i < ihi) {
                const int mid = (i + ihi + 1) >> 1;
                if (sub_pre[mid] <= g) i = mid; else ihi = mid - 1;
            }
            Tab tb = tab_at(smem, A, i);
            const uint32_t rl = g - sub_pre[i];
            int lo = 0, hi = sk - 1;  // last ranked row with row_pre <= rl
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tb.row_pre[mid] <= rl) lo = mid; else hi = mid - 1;
            }
            const uint32_t sigma = rl - tb.row_pre[lo];
            const uint32_t cell = (uint32_t)tb.idx1[lo] * (uint32_t)sk + tb.idx2[sigma];
            const uint32_t* sp = A.split + (int64_t)i * (A.nch + 1) * A.K + cell;
            const uint32_t s0 = __ldg(sp + (int64_t)j0 * A.K);
            const uint32_t s1 = __ldg(sp + (int64_t)j1 * A.K);
            pP[u] = (uint32_t)i * (uint32_t)A.n + s0;
            pE[u] = (uint32_t)i * (uint32_t)A.n + s1;
            nqd[u] = s1 > s0 ? ((pE[u] + 3u) >> 2) - (pP[u] >> 2) : 0u;
            mode[u] = sub_wb[i];
        }
        s += nqd[u];
        ne += nqd[u] ? 1u : 0u;
    }
    // quads (high half) and segments (low half, at most MAXSEG) in one scan;
    // the radix histogram area of o_hist is free during S4
    unsigned long long tot2;
    const unsigned long long ex2 = block_exclusive_scan64<NT>(((unsigned long long)s << 32) | ne,
                                                              reinterpret_cast<unsigned long long*>(smem + A.o_hist), &tot2);
    const uint32_t F = (uint32_t)(tot2 >> 32), M = (uint32_t)tot2;
    uint32_t run = (uint32_t)(ex2 >> 32), slot = (uint32_t)ex2;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
        if (nqd[u]) {
            seg_pre[slot] = run;
            seg_info[slot] = make_uint4((pP[u] >> 2) - run, pP[u], pE[u], mode[u]);  // quad = .x + flat position
            ++slot;
        }
        run += nqd[u];
    }
    if (threadIdx.x == 0) seg_pre[M] = F;
    __syncthreads();
    if (cyc) {
        const long long t = clock64();
        cyc[0] += t;
        cyc[1] -= t;
    }
    // each warp takes a contiguous share [wb, we) of the F quads in windows of
    // 32 consecutive quads (one per lane); the warp holds the starts of the
    // next 32 segments in its lanes, so a lane finds the segment of its quad
    // with a ballot and a population count; it loads the quad's 4 ids with one
    // 16-byte load and keeps those inside the segment's perm range
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t share = (F + NW - 1) / NW;
    const uint32_t wb = min(F, (uint32_t)warp * share), we = min(F, wb + share);
    uint32_t lanemask_le;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(lanemask_le));
    const uint4* perm4 = reinterpret_cast<const uint4*>(A.perm);
    if (wb < we) {
        int lo = 0, hi = (int)M - 1;  // the segment holding wb
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_pre[mid] <= wb) lo = mid; else hi = mid - 1;
        }
        uint32_t sg0 = (uint32_t)lo;
        const uint32_t span = A.span, G = A.G;
        for (uint32_t w0 = wb; w0 < we;) {
            const uint32_t sj = sg0 + 1u + (uint32_t)lane;
            const uint32_t Bj = sj <= M ? seg_pre[sj] : 0xffffffffu;  // start of segment sg0+1+lane
            const uint32_t B31 = __shfl_sync(0xffffffffu, Bj, 31);
            const uint32_t wend = min(we, min(w0 + 32u * SCAN_U, B31));  // segments sg0 .. sg0+31 only
            uint4 q[SCAN_U];
            uint32_t vmask[SCAN_U], md[SCAN_U];  // ids of the quad inside the segment (bit j: element j)
#pragma unroll
            for (int u = 0; u < SCAN_U; ++u) {
                const uint32_t x = w0 + 32u * (uint32_t)u, pu = x + (uint32_t)lane;
                const uint32_t before = __popc(__ballot_sync(0xffffffffu, Bj <= x));
                const uint32_t o = Bj - x;  // segment starts strictly inside the window
                const uint32_t mk = __reduce_or_sync(0xffffffffu, o - 1u < 31u ? 1u << o : 0u);
                q[u] = make_uint4(0u, 0u, 0u, 0u);
                vmask[u] = 0u;
                md[u] = 0u;
                if (pu < wend) {
                    const uint4 inf = seg_info[sg0 + before + __popc(mk & lanemask_le)];
                    const uint32_t qi = inf.x + pu, p0 = qi << 2;
                    // the quad overlaps the segment's perm range [inf.y, inf.z)
                    const uint32_t lo = inf.y > p0 ? inf.y - p0 : 0u, hi = min(inf.z - p0, 4u);
                    vmask[u] = ((1u << hi) - 1u) & ~((1u << lo) - 1u);
                    md[u] = inf.w;
                    q[u] = __ldg(perm4 + qi);
                }
            }
#pragma unroll
            for (int u = 0; u < SCAN_U; ++u) {
                const uint32_t idq[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
                // the segment's counter layout, once per quad: a nibble set
                // puts id t of a group in word (t & 3), bits (t & 28)..+3; a
                // one-bit plane puts it at bit t of one word
                const bool nib = (md[u] >> 31) != 0u;
                const uint32_t wbase = md[u] & 0x7fffffffu;
                const uint32_t wstep = nib ? G : 0u, smask = nib ? 28u : 31u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t loc = idq[j] - id0;
                    if (((vmask[u] >> j) & 1u) && loc < span) {
                        const uint32_t t = loc & 31u;
                        atomicAdd(&cnt_words[wbase + (t & 3u) * wstep + (loc >> 5)], 1u << (t & smask));
                    }
                }
            }
            sg0 += __popc(__ballot_sync(0xffffffffu, Bj <= wend));
            w0 = wend;
        }
    }
    __syncthreads();
    if (cyc) cyc[1] += clock64();
}

// Turns the counters of every 32-id group of this CTA into B bit planes in
// place: plane j (word j*G + g) holds bit j of each id's SC-score.  A nibble
// set's four words are a 4 x 4 bit matrix per nibble position (word q, bit l)
// that is transposed with two rounds of masked swaps; the sets and the one-bit
// planes are then added with bit-sliced ripple adders.
template <int NT, int B>
__device__ void counters_to_planes(const QArgs& A, uint32_t* w, uint32_t ngroups)
{
    const uint32_t G = A.G;
    const int nsets = (int)A.nsets, nplanes = (int)A.nplanes;
    for (uint32_t g = threadIdx.x; g < ngroups; g += NT) {
        uint32_t acc[B];
#pragma unroll
        for (int j = 0; j < B; ++j) acc[j] = 0u;
        for (int st = 0; st < nsets; ++st) {
            uint32_t x0 = w[(4 * st + 0) * G + g], x1 = w[(4 * st + 1) * G + g];
            uint32_t x2 = w[(4 * st + 2) * G + g], x3 = w[(4 * st + 3) * G + g];
            uint32_t t = ((x0 >> 2) ^ x2) & 0x33333333u;
            x2 ^= t;
            x0 ^= t << 2;
            t = ((x1 >> 2) ^ x3) & 0x33333333u;
            x3 ^= t;
            x1 ^= t << 2;
            t = ((x0 >> 1) ^ x1) & 0x55555555u;
            x1 ^= t;
            x0 ^= t << 1;
            t = ((x2 >> 1) ^ x3) & 0x55555555u;
            x3 ^= t;
            x2 ^= t << 1;
            // now x_l holds bit l of the set's count of id 32g + t at bit t
            const uint32_t add[4] = {x0, x1, x2, x3};
            uint32_t c = 0u;
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const uint32_t y = j < 4 ? add[j] : 0u;
                const uint32_t s = acc[j] ^ y ^ c;
                c = (acc[j] & y) | (c & (acc[j] ^ y));
                acc[j] = s;
            }
        }
        for (int pl = 0; pl < nplanes; ++pl) {
            uint32_t c = w[(4 * nsets + pl) * G + g];
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const uint32_t s = acc[j] ^ c;
                c &= acc[j];
                acc[j] = s;
            }
        }
#pragma unroll
        for (int j = 0; j < B; ++j) w[(uint32_t)j * G + g] = acc[j];
    }
}

// The sliced SC-scores of 32-id group g: acc[j] holds bit j of each id's score.
template <int B>
__device__ __forceinline__ void load_scores(const uint32_t* planes, uint32_t G, uint32_t g, uint32_t acc[B])
{
#pragma unroll
    for (int j = 0; j < B; ++j) acc[j] = planes[(uint32_t)j * G + g];
}

// Bitwise "score >= s" over the 32 ids of a bit-sliced accumulator.
template <int B>
__device__ __forceinline__ uint32_t bitsliced_ge(const uint32_t acc[B], uint32_t s)
{
    uint32_t ge = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < B; ++j) ge = ((s >> j) & 1u) ? (acc[j] & ge) : (acc[j] | ge);
    if (s >> B) ge = 0u;
    return ge;
}

// S6 exact pass: FP32 squared distances of the rows listed in ids[0, count)
// into keys (distance bits << 32 | id; ~0 for an id outside [0, n)).  8 lanes
// per row, two groups of 4 rows per warp in flight; each lane keeps S6_CH
// float4 chunks of each of its two rows in registers per load round.
template <int NT, int S6_CH, int MET>
__device__ void rerank_fp32(const QArgs& A, const float4* q4, const uint32_t* ids, uint32_t count,
                            unsigned long long* keys)
{
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane >> 3, gl = lane & 7;
    const int ld4 = (int)(A.ld / 4);
    const float4* X4 = reinterpret_cast<const float4*>(A.X);
    for (uint32_t rb = (uint32_t)warp * 8u; rb < count; rb += (uint32_t)NW * 8u) {
        const uint32_t ra = rb + (uint32_t)grp, rc = ra + 4u;
        const uint32_t ida = ra < count ? ids[ra] : 0xffffffffu;
        const uint32_t idc = rc < count ? ids[rc] : 0xffffffffu;
        const bool va = ida < (uint32_t)A.n, vc = idc < (uint32_t)A.n;
        const float4* pa = X4 + (int64_t)(va ? ida : 0u) * ld4;
        const float4* pc = X4 + (int64_t)(vc ? idc : 0u) * ld4;
        float acc_a = 0.f, acc_c = 0.f;
        for (int c0 = gl; c0 < ld4; c0 += 8 * S6_CH) {
            float4 xa[S6_CH], xc[S6_CH];
#pragma unroll
            for (int u = 0; u < S6_CH; ++u) {
                const int c = c0 + 8 * u;
                xa[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                xc[u] = xa[u];
                if (c < ld4) {
                    if (va) xa[u] = ldg_stream(pa + c);
                    if (vc) xc[u] = ldg_stream(pc + c);
                }
            }
#pragma unroll
            for (int u = 0; u < S6_CH; ++u) {
                const int c = c0 + 8 * u;
                if (c < ld4) {
                    const float4 qv = q4[c];
                    acc_a = dterm<MET>(acc_a, __fsub_rn(xa[u].x, qv.x));
                    acc_a = dterm<MET>(acc_a, __fsub_rn(xa[u].y, qv.y));
                    acc_a = dterm<MET>(acc_a, __fsub_rn(xa[u].z, qv.z));
                    acc_a = dterm<MET>(acc_a, __fsub_rn(xa[u].w, qv.w));
                    acc_c = dterm<MET>(acc_c, __fsub_rn(xc[u].x, qv.x));
                    acc_c = dterm<MET>(acc_c, __fsub_rn(xc[u].y, qv.y));
                    acc_c = dterm<MET>(acc_c, __fsub_rn(xc[u].z, qv.z));
                    acc_c = dterm<MET>(acc_c, __fsub_rn(xc[u].w, qv.w));
                }
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            acc_a = __fadd_rn(acc_a, __shfl_xor_sync(0xffffffffu, acc_a, o));
            acc_c = __fadd_rn(acc_c, __shfl_xor_sync(0xffffffffu, acc_c, o));
        }
        if (gl == 0) {
            if (ra < count) keys[ra] = va ? ((unsigned long long)__float_as_uint(acc_a) << 32) | ida : ~0ull;
            if (rc < count) keys[rc] = vc ? ((unsigned long long)__float_as_uint(acc_c) << 32) | idc : ~0ull;
        }
    }
}

__device__ __forceinline__ uint4 ldg_stream_u4(const uint4* p)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// adds the squared differences of the 8 BF16 values in w (element 2i in the
// low half of word i) to q[0..8) into acc, in element order
__device__ __forceinline__ float bf16x8_sqdiff(uint4 w, const float4* q, float acc)
{
    const float4 q0 = q[0], q1 = q[1];
    const float x[8] = {__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xffff0000u),
                        __uint_as_float(w.y << 16), __uint_as_float(w.y & 0xffff0000u),
                        __uint_as_float(w.z << 16), __uint_as_float(w.z & 0xffff0000u),
                        __uint_as_float(w.w << 16), __uint_as_float(w.w & 0xffff0000u)};
    const float qq[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float df = __fsub_rn(x[j], qq[j]);
        acc = __fmaf_rn(df, df, acc);
    }
    return acc;
}

// S6 coarse pass: squared distances of the BF16 copies of the rows listed in
// ids[0, count), accumulated in FP32, into keys (same layout as rerank_fp32).
template <int NT, int S6_CH>
__device__ void rerank_bf16(const QArgs& A, const float4* q4, const uint32_t* ids, uint32_t count,
                            unsigned long long* keys)
{
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane >> 3, gl = lane & 7;
    const int ldc = (int)(A.ldh / 8);  // 16-byte chunks of 8 values per row
    const uint4* X16 = reinterpret_cast<const uint4*>(A.Xh);
    for (uint32_t rb = (uint32_t)warp * 8u; rb < count; rb += (uint32_t)NW * 8u) {
        const uint32_t ra = rb + (uint32_t)grp, rc = ra + 4u;
        const uint32_t ida = ra < count ? ids[ra] : 0xffffffffu;
        const uint32_t idc = rc < count ? ids[rc] : 0xffffffffu;
        const bool va = ida < (uint32_t)A.n, vc = idc < (uint32_t)A.n;
        const uint4* pa = X16 + (int64_t)(va ? ida : 0u) * ldc;
        const uint4* pc = X16 + (int64_t)(vc ? idc : 0u) * ldc;
        float acc_a = 0.f, acc_c = 0.f;
        for (int c0 = gl; c0 < ldc; c0 += 8 * S6_CH) {
            uint4 xa[S6_CH], xc[S6_CH];
#pragma unroll
            for (int u = 0; u < S6_CH; ++u) {
                const int c = c0 + 8 * u;
                xa[u] = make_uint4(0u, 0u, 0u, 0u);
                xc[u] = xa[u];
                if (c < ldc) {
                    if (va) xa[u] = ldg_stream_u4(pa + c);
                    if (vc) xc[u] = ldg_stream_u4(pc + c);
                }
            }
#pragma unroll
            for (int u = 0; u < S6_CH; ++u) {
                const int c = c0 + 8 * u;
                if (c < ldc) {
                    acc_a = bf16x8_sqdiff(xa[u], q4 + 2 * c, acc_a);
                    acc_c = bf16x8_sqdiff(xc[u], q4 + 2 * c, acc_c);
                }
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            acc_a = __fadd_rn(acc_a, __shfl_xor_sync(0xffffffffu, acc_a, o));
            acc_c = __fadd_rn(acc_c, __shfl_xor_sync(0xffffffffu, acc_c, o));
        }
        if (gl == 0) {
            if (ra < count) keys[ra] = va ? ((unsigned long long)__float_as_uint(acc_a) << 32) | ida : ~0ull;
            if (rc < count) keys[rc] = vc ? ((unsigned long long)__float_as_uint(acc_c) << 32) | idc : ~0ull;
        }
    }
}

// four E4M3 codes (byte j of w is element j) decoded exactly, times their scales
__device__ __forceinline__ float4 e4m3x4_scaled(uint32_t w, float4 s)
{
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
    return make_float4(__fmul_rn(a.x, s.x), __fmul_rn(a.y, s.y), __fmul_rn(b.x, s.z), __fmul_rn(b.y, s.w));
}

__device__ __forceinline__ float sqdiff4(float4 x, float4 q, float acc)
{
    float df = __fsub_rn(x.x, q.x);
    acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(x.y, q.y);
    acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(x.z, q.z);
    acc = __fmaf_rn(df, df, acc);
    df = __fsub_rn(x.w, q.w);
    return __fmaf_rn(df, df, acc);
}

// S6 coarse pass on the FP8 copy: 16 codes per 16-byte chunk, decoded as
// code * column scale in FP32, squared differences summed in FP32 in element
// order per lane, then over the 8 lanes of the row.
template <int NT>
__device__ void rerank_fp8(const QArgs& A, const float4* q4, const uint32_t* ids, uint32_t count,
                           unsigned long long* keys)
{
    constexpr int NW = NT / 32;
    constexpr int CH = 2;  // chunks per lane per row in one load round
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane >> 3, gl = lane & 7;
    const int ldc = (int)(A.ld8 / 16);
    const uint4* X16 = reinterpret_cast<const uint4*>(A.X8);
    const float4* s4 = reinterpret_cast<const float4*>(A.s8col);
    for (uint32_t rb = (uint32_t)warp * 8u; rb < count; rb += (uint32_t)NW * 8u) {
        const uint32_t ra = rb + (uint32_t)grp, rc = ra + 4u;
        const uint32_t ida = ra < count ? ids[ra] : 0xffffffffu;
        const uint32_t idc = rc < count ? ids[rc] : 0xffffffffu;
        const bool va = ida < (uint32_t)A.n, vc = idc < (uint32_t)A.n;
        const uint4* pa = X16 + (int64_t)(va ? ida : 0u) * ldc;
        const uint4* pc = X16 + (int64_t)(vc ? idc : 0u) * ldc;
        float acc_a = 0.f, acc_c = 0.f;
        for (int c0 = gl; c0 < ldc; c0 += 8 * CH) {
            uint4 xa[CH], xc[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int c = c0 + 8 * u;
                xa[u] = make_uint4(0u, 0u, 0u, 0u);
                xc[u] = xa[u];
                if (c < ldc) {
                    if (va) xa[u] = ldg_stream_u4(pa + c);
                    if (vc) xc[u] = ldg_stream_u4(pc + c);
                }
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int c = c0 + 8 * u;
                if (c < ldc) {
                    const uint32_t wa[4] = {xa[u].x, xa[u].y, xa[u].z, xa[u].w};
                    const uint32_t wc[4] = {xc[u].x, xc[u].y, xc[u].z, xc[u].w};
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float4 sc = __ldg(s4 + 4 * c + v);
                        const float4 qv = q4[4 * c + v];
                        acc_a = sqdiff4(e4m3x4_scaled(wa[v], sc), qv, acc_a);
                        acc_c = sqdiff4(e4m3x4_scaled(wc[v], sc), qv, acc_c);
                    }
                }
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            acc_a = __fadd_rn(acc_a, __shfl_xor_sync(0xffffffffu, acc_a, o));
            acc_c = __fadd_rn(acc_c, __shfl_xor_sync(0xffffffffu, acc_c, o));
        }
        if (gl == 0) {
            if (ra < count) keys[ra] = va ? ((unsigned long long)__float_as_uint(acc_a) << 32) | ida : ~0ull;
            if (rc < count) keys[rc] = vc ? ((unsigned long long)__float_as_uint(acc_c) << 32) | idc : ~0ull;
        }
    }
}

// The key of rank R (1-based) among the keys of every CTA of the cluster
// (keys are unique), by a radix select over 8-bit digits from the top: each
// pass every CTA histograms its keys that match the decided prefix, publishes
// the histogram, and after a cluster barrier every CTA sums the CL histograms
// and picks the digit where the running count reaches R.  It stops as soon as
// the whole crossing bin is needed, and returns the largest key of that bin,
// so that exactly R keys of the cluster are <= the result.  Histograms
// alternate between two published buffers: one is written while the previous
// pass's is still read by the other CTAs.  Every CTA takes the same passes.
template <int NT>
__device__ unsigned long long cluster_rank_cut(const QArgs& A, char* smem, const unsigned long long* keys,
                                               uint32_t count, uint32_t R)
{
    uint32_t* pub = reinterpret_cast<uint32_t*>(smem + A.o_rsel);   // [2][256]
    uint32_t* tot = reinterpret_cast<uint32_t*>(smem + A.o_hist);   // [256] local sums
    uint32_t* st = tot + 256;                                        // [0] digit, [1] below, [2] bin count
    const int lane = threadIdx.x & 31;
    const uint32_t CL = (uint32_t)A.CL;
    unsigned long long prefix = 0ull, mask = 0ull;
    uint32_t need = R;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        uint32_t* h = pub + (pass & 1) * 256;
        for (int t = threadIdx.x; t < 256; t += NT) h[t] = 0u;
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < count; t += NT) {
            const unsigned long long key = keys[t];
            if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
        }
        cluster_sync();
        for (int t = threadIdx.x; t < 256; t += NT) {
            const uint32_t a = smem_addr(h + t);
            uint32_t sum = 0u;
            for (uint32_t rr = 0; rr < CL; ++rr) sum += ld_cluster_u32(map_rank(a, rr));
            tot[t] = sum;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t v[8], s = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = tot[lane * 8 + j];
                s += v[j];
            }
            uint32_t incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - s;
            if (excl < need && incl >= need) {
                uint32_t cum = excl;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (cum + v[j] >= need) {
                        st[0] = (uint32_t)(lane * 8 + j);
                        st[1] = cum;
                        st[2] = v[j];
                        break;
                    }
                    cum += v[j];
                }
            }
        }
        __syncthreads();
        const uint32_t digit = st[0], below = st[1], inbin = st[2];
        __syncthreads();
        prefix |= (unsigned long long)digit << shift;
        mask |= 255ull << shift;
        need -= below;
        if (inbin == need) return prefix | (shift ? ((1ull << shift) - 1ull) : 0ull);
    }
    return prefix;
}

template <int NT, int NSMAX, int MET>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : (NT == 512 ? 2 : 1)) suco_query_kernel(const QArgs A)
{
    extern __shared__ __align__(16) char smem[];
    constexpr int B = NSMAX == 8 ? 4 : (NSMAX == 16 ? 5 : 6);
    constexpr int NW = NT / 32;
    constexpr int NC = NSMAX + 2;  // count slots: [0] = valid ids, [s] = #scores >= s
    const uint32_t r = cluster_rank();
    const int CL = A.CL;
    // persistent clusters: cluster c starts with query c of the G clusters in the
    // grid; with a work counter each cluster then takes the next unanswered query
    // (queries of uneven cost balance), without one it answers c + G, c + 2G, ...
    const uint32_t Gc = gridDim.x / (uint32_t)CL;
    uint32_t* next_q = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 120;  // this cluster's next query
    int64_t b = blockIdx.x / CL;
    // where subspace i counts its collisions (word base | nibble-set flag)
    uint32_t* sub_wb = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 128;  // [Ns]

    for (int i = threadIdx.x; i < A.Ns; i += NT) {
        const uint32_t ns15 = 15u * A.nsets;
        sub_wb[i] = (uint32_t)i < ns15 ? (4u * ((uint32_t)i / 15u) * A.G) | 0x80000000u
                                       : (4u * A.nsets + (uint32_t)i - ns15) * A.G;
    }
    bool q_next = false;  // the query row is already on its way to o_qn
    while (b < A.nq) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    stamp(A, b, r, 1);
    uint32_t grabbed = 0u;  // thread 0 of CTA 0: the query this cluster answers next
    if (A.work && r == 0 && threadIdx.x == 0) grabbed = Gc + atomicAdd(A.work, 1u);

    // ---- S0: this query's thresholds; stage the query; clear the published
    // counts and candidate slots
    uint32_t* qpar = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 110;  // T, C, k, per_cta
    if (threadIdx.x == 0) {
        uint32_t kq = (uint32_t)A.k, T = A.T, C = A.C;
        if (A.k_per) kq = (uint32_t)min(max(A.k_per[b], 1), A.k);
        if (A.alpha_per) {
            double a = (double)A.alpha_per[b];
            a = a > 0.0 ? fmin(a, 1.0) : 0.0;  // NaN and non-positive values give T = 1
            double t = ceil(a * (double)A.n - 1e-9);
            T = (uint32_t)fmin(fmax(t, 1.0), (double)A.n);
        }
        if (A.beta_per || A.k_per) {
            double be = A.beta;
            if (A.beta_per) {
                const double v = (double)A.beta_per[b];
                be = v > 0.0 ? fmin(v, A.beta) : A.beta;
            }
            double c = fmax(ceil(be * (double)A.n - 1e-9), (double)kq);
            c = fmin(fmax(c, 1.0), (double)A.n);
            C = min((uint32_t)c, A.C);
        }
        qpar[0] = T;
        qpar[1] = C;
        qpar[2] = kq;
        qpar[3] = (C + CL - 1) / CL;
    }
    {
        float* qs = reinterpret_cast<float*>(smem + A.o_q);
        if (q_next) {
            // copied in during the last query's S6 by this same thread (j
            // strides match), so its own completed copies need no barrier
            cp_async_wait_all();
            const float* qn = reinterpret_cast<const float*>(smem + A.o_qn);
            for (int j = threadIdx.x; j < A.ldq; j += NT) qs[j] = j < A.d ? qn[j] : 0.f;
            q_next = false;
        } else {
            const float* qg = A.Q + b * A.d;
            for (int j = threadIdx.x; j < A.ldq; j += NT) qs[j] = j < A.d ? query_col(qg, A.qperm, j) : 0.f;
        }
        uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + A.o_cnt);
        for (int t = threadIdx.x; t < 2 * NC; t += NT) cnt[t] = 0u;
    }
    __syncthreads();
    stamp(A, b, r, 2);

    const uint32_t qT = qpar[0], qC = qpar[1], qk = qpar[2], qper = qpar[3];
    // ---- S1-S3 for the subspaces this CTA owns
    if (A.pair_ok && (int)r + CL < A.Ns && (int)r + 2 * CL >= A.Ns) {
        // two subspaces: each half of the CTA ranks one (named barriers 1, 2)
        const int grp = threadIdx.x >= NT / 2;
        rank_subspace<NT / 2, MET>(A, smem, b, (int)r + grp * CL, qT, (int)threadIdx.x - grp * (NT / 2), 1 + grp,
                                   grp);
        __syncthreads();  // both halves are done with their scratch before the union is cleared
    } else {
        for (int i = (int)r; i < A.Ns; i += CL) rank_subspace<NT, MET>(A, smem, b, i, qT, (int)threadIdx.x, 0, 0);
    }
    stamp(A, b, r, 3);
    // clear the bit planes (the union region served as S3 scratch)
    {
        uint4* pw = reinterpret_cast<uint4*>(smem + A.o_union);
        const uint4 z = make_uint4(0, 0, 0, 0);
        const uint32_t n16 = (A.nstore * A.G + 3) / 4;  // the union region is a multiple of 16 bytes
        for (uint32_t w = threadIdx.x; w < n16; w += NT) pw[w] = z;
    }
    cluster_sync();  // #1: every subspace's cut and staircase are published
    stamp(A, b, r, 4);
    // every CTA has read the previous next_q before #1: publish the next query
    if (A.work && r == 0 && threadIdx.x == 0)
        for (int t = 0; t < CL; ++t) st_cluster_u32(map_rank(smem_addr(next_q), (uint32_t)t), grabbed);

    // ---- copy the parts of the other CTAs' tables that S4 reads (16-byte
    // loads: the table stride and the copied length are multiples of 16)
    {
        const uint32_t vecs = A.tab_copy / 16;
        for (uint32_t t = threadIdx.x; t < (uint32_t)A.Ns * vecs; t += NT) {
            const int i = t / vecs;
            const uint32_t owner = (uint32_t)(i % CL);
            if (owner == r) continue;
            uint4* dst = reinterpret_cast<uint4*>(smem + A.o_tab + (size_t)i * A.tab_stride) + (t - i * vecs);
            *dst = ld_cluster_v4(map_rank(smem_addr(dst), owner));
        }
    }
    __syncthreads();

    // ---- S4 + S5 over the id range in A.npass passes.  In pass p, CTA r owns
    // the ids of block p*CL + r (A.cpc chunks).  With one pass the cut of S5 is
    // final.  With several, the cluster keeps a running candidate list, the
    // first qC entries by (score desc, id asc) among the ids seen so far, in id
    // order and spread over the CTAs by position (qper each): every pass merges
    // its ids into it with the same cut.  An id of the final top-qC is in the
    // top-qC of the ids seen up to its own pass, so nothing it needs is lost.
    uint32_t* sub_pre = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 32;  // [Ns+1]
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int i = 0; i < A.Ns; ++i) {
            sub_pre[i] = acc;
            acc += tab_at(smem, A, i).row_pre[A.sqrtK];
        }
        sub_pre[A.Ns] = acc;
    }
    __syncthreads();  // sub_pre is read by every thread below
    stamp(A, b, r, 5);
    long long* seg_cyc = A.dbg_clk && threadIdx.x == 0 ? A.dbg_clk + (b * 16 + r) * NCLK + NCLK - 2 : nullptr;
    if (seg_cyc) seg_cyc[0] = seg_cyc[1] = 0;
    uint32_t* planes = reinterpret_cast<uint32_t*>(smem + A.o_union);  // counters, then [B][G] sliced scores
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + A.o_cnt);  // published: [NC] pass counts, [NC] list counts
    uint32_t* allc = cnt + 2 * NC;                                 // [CL][2][NC]
    uint32_t* wcnt = allc + 2 * CL * NC;                           // [NW][NC]
    uint32_t* sel = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 72;  // theta, keep, need_eq, RG, RE, rg_pre, re_pre
    uint32_t* slot_base = sel + 8;                                      // [CL] remote id-slot addresses
    uint32_t* wbase = reinterpret_cast<uint32_t*>(smem + A.o_hist);     // [NW][2] per-warp output bases
    const uint32_t L = sub_pre[A.Ns];
    const bool multi = A.npass > 1;
    uint32_t run_n = 0;  // entries of the running list (the same in every CTA)
    uint32_t* ids_out = reinterpret_cast<uint32_t*>(smem + A.o_slots);
    for (uint32_t pass = 0; pass < A.npass; ++pass) {
        const uint32_t blk = pass * (uint32_t)CL + r;
        const uint32_t id0 = blk * A.span;
        const int j0 = (int)(blk * (uint32_t)A.cpc), j1 = j0 + A.cpc;
        // list buffers: read [pass & 1], write [(pass + 1) & 1]; one pass writes the S6 slots
        const uint32_t* ids_in = multi ? reinterpret_cast<const uint32_t*>(smem + A.o_run) + (pass & 1) * A.run_stride
                                       : nullptr;
        const uint8_t* sc_in = multi ? reinterpret_cast<const uint8_t*>(smem + A.o_run + 8u * A.run_stride) +
                                           (pass & 1) * A.run_stride
                                     : nullptr;
        ids_out = multi ? reinterpret_cast<uint32_t*>(smem + A.o_run) + ((pass + 1) & 1) * A.run_stride
                        : reinterpret_cast<uint32_t*>(smem + A.o_slots);
        uint8_t* sc_out = multi ? reinterpret_cast<uint8_t*>(smem + A.o_run + 8u * A.run_stride) +
                                      ((pass + 1) & 1) * A.run_stride
                                : nullptr;
        if (pass > 0) {
            uint4* pw = reinterpret_cast<uint4*>(planes);
            const uint4 z = make_uint4(0, 0, 0, 0);
            for (uint32_t w = threadIdx.x; w < (A.nstore * A.G + 3) / 4; w += NT) pw[w] = z;
            for (int t = threadIdx.x; t < 2 * NC; t += NT) cnt[t] = 0u;
        }
        __syncthreads();
        for (uint32_t e0 = 0; e0 < L; e0 += MAXSEG)
            scan_segments<NT>(A, smem, e0, min((uint32_t)MAXSEG, L - e0), sub_pre, sub_wb, planes, id0, j0, j1,
                              seg_cyc);
        stamp(A, b, r, 6);

        const uint32_t valid = id0 >= A.n ? 0u : (uint32_t)min((int64_t)A.span, A.n - (int64_t)id0);
        if (!multi) {
            // the candidate slots share the (now dead) segment region; other CTAs
            // fill them after cluster barrier #2
            for (uint32_t t = threadIdx.x; t < A.per_cta; t += NT) ids_out[t] = 0xffffffffu;
        }
        counters_to_planes<NT, B>(A, planes, (valid + 31) / 32);
        __syncthreads();
        stamp(A, b, r, 7);
        if (A.dbg_scores)
            for (uint32_t j = threadIdx.x; j < valid; j += NT) {
                uint32_t sc = 0;
                for (int q = 0; q < B; ++q) sc |= ((planes[(uint32_t)q * A.G + (j >> 5)] >> (j & 31)) & 1u) << q;
                A.dbg_scores[b * A.n + id0 + j] = (uint8_t)sc;
            }

        // ---- S5: counts of scores >= s per warp range (this pass's ids) and
        // per score of the running list's entries; the cut; the hand-off
        const uint32_t ngroups = (valid + 31) / 32;
        const uint32_t gpw = (ngroups + NW - 1) / NW;
        const uint32_t gb = min(ngroups, (uint32_t)warp * gpw), ge = min(ngroups, gb + gpw);
        {
            uint32_t c[NSMAX];
#pragma unroll
            for (int s = 0; s < NSMAX; ++s) c[s] = 0u;
            for (uint32_t g = gb + lane; g < ge; g += 32) {
                uint32_t acc[B];
                load_scores<B>(planes, A.G, g, acc);
#pragma unroll
                for (int s = 0; s < NSMAX; ++s)
                    if (s < A.Ns) c[s] += __popc(bitsliced_ge<B>(acc, (uint32_t)(s + 1)));
            }
#pragma unroll
            for (int s = 0; s < NSMAX; ++s) {
                uint32_t v = c[s];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) {
                    wcnt[warp * NC + s + 1] = v;
                    if (v) atomicAdd(&cnt[s + 1], v);
                }
            }
            if (lane == 0) {
                const uint32_t lo = gb * 32, hi = min(valid, ge * 32);
                wcnt[warp * NC] = hi > lo ? hi - lo : 0u;
                wcnt[warp * NC + NSMAX + 1] = 0u;
            }
            if (threadIdx.x == 0) cnt[0] = valid;
        }
        const uint32_t mr = run_n > r * qper ? min(qper, run_n - r * qper) : 0u;  // my list entries
        if (multi) {
            uint32_t* rc = cnt + NC;  // [s] = my list entries with score exactly s, then made cumulative
            for (uint32_t t = threadIdx.x; t < mr; t += NT) atomicAdd(&rc[sc_in[t]], 1u);
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t acc = 0;
                for (int s = NC - 1; s >= 0; --s) {
                    acc += rc[s];
                    rc[s] = acc;
                }
            }
        }
        stamp(A, b, r, 8);
        cluster_sync();  // #2: every CTA's counts are published
        stamp(A, b, r, 9);
        for (int t = threadIdx.x; t < CL * 2 * NC; t += NT) {
            const int rr = t / (2 * NC), s = t - rr * 2 * NC;
            allc[t] = ld_cluster_u32(map_rank(smem_addr(cnt + s), (uint32_t)rr));
        }
        for (int t = threadIdx.x; t < CL; t += NT) slot_base[t] = map_rank(smem_addr(ids_out), (uint32_t)t);
        __syncthreads();
        if (warp == 0) {
            // the cut over the list entries and this pass's ids together, by
            // one warp: lane l sums the counts of score >= l+1 over the CTAs
            uint32_t total = 0, tot_s = 0;
            const int s1 = lane + 1;
            for (int rr = 0; rr < CL; ++rr) {
                const uint32_t* cp = allc + rr * 2 * NC;
                total += cp[0] + cp[NC];
                if (s1 <= A.Ns) tot_s += cp[s1] + cp[NC + s1];
            }
            const uint32_t keep = min(qC, total);
            // counts fall as s grows, so the lanes that reach keep are a prefix
            const int theta = __popc(__ballot_sync(0xffffffffu, s1 <= A.Ns && tot_s >= keep));
            // per-CTA splits at theta: lane rr < CL
            uint32_t rgt = 0, req = 0, pgt = 0, peq = 0;
            if (lane < CL) {
                const uint32_t* cp = allc + lane * 2 * NC;
                const uint32_t* cr = cp + NC;
                rgt = cr[theta + 1];
                req = cr[theta] - rgt;
                pgt = cp[theta + 1];
                peq = cp[theta] - pgt;
            }
            uint32_t x_rg = rgt, x_re = req, x_pg = pgt, x_pe = peq;  // inclusive scans over the CTAs
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t a1 = __shfl_up_sync(0xffffffffu, x_rg, o), a2 = __shfl_up_sync(0xffffffffu, x_re, o);
                const uint32_t a3 = __shfl_up_sync(0xffffffffu, x_pg, o), a4 = __shfl_up_sync(0xffffffffu, x_pe, o);
                if (lane >= o) {
                    x_rg += a1;
                    x_re += a2;
                    x_pg += a3;
                    x_pe += a4;
                }
            }
            const uint32_t RG = __shfl_sync(0xffffffffu, x_rg, 31), RE = __shfl_sync(0xffffffffu, x_re, 31);
            const uint32_t PG = __shfl_sync(0xffffffffu, x_pg, 31);
            // this CTA's exclusive prefixes (lane r holds the inclusive ones)
            const uint32_t rg_pre = __shfl_sync(0xffffffffu, x_rg - rgt, (int)r);
            const uint32_t re_pre = __shfl_sync(0xffffffffu, x_re - req, (int)r);
            const uint32_t pg_pre = __shfl_sync(0xffffffffu, x_pg - pgt, (int)r);
            const uint32_t pe_pre = __shfl_sync(0xffffffffu, x_pe - peq, (int)r);
            // per-warp bases of this pass's ids: entries of the output order before the warp's range
            uint32_t gt = 0, eq = 0;
            if (lane < NW) {
                gt = wcnt[lane * NC + theta + 1];
                eq = wcnt[lane * NC + theta] - gt;
            }
            uint32_t x_g = gt, x_e = eq;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t a1 = __shfl_up_sync(0xffffffffu, x_g, o), a2 = __shfl_up_sync(0xffffffffu, x_e, o);
                if (lane >= o) {
                    x_g += a1;
                    x_e += a2;
                }
            }
            if (lane < NW) {
                wbase[2 * lane] = RG + pg_pre + x_g - gt;
                wbase[2 * lane + 1] = RE + pe_pre + x_e - eq;
            }
            if (lane == 0) {
                sel[0] = (uint32_t)theta;
                sel[1] = keep;
                sel[2] = keep - (RG + PG);  // entries scoring exactly theta that are kept (the lowest ids)
                sel[3] = rg_pre;
                sel[4] = re_pre;
            }
        }
        __syncthreads();
        stamp(A, b, r, 10);
        const uint32_t theta = sel[0], keep = sel[1], need_eq = sel[2];
        if (multi) {
            // this CTA's list entries, in position order: kept ones move to
            // position G_before + E_before of the new list
            uint32_t gcar = sel[3], ecar = sel[4];
            uint32_t* wtmp = reinterpret_cast<uint32_t*>(smem + A.o_hist) + 256;
            for (uint32_t t0 = 0; t0 < mr; t0 += NT) {
                const uint32_t t = t0 + threadIdx.x;
                const uint32_t sc = t < mr ? sc_in[t] : 0u;
                const uint32_t isg = t < mr && sc > theta, ise = t < mr && sc == theta;
                uint32_t tot;
                const uint32_t ex = block_exclusive_scan<NT>((isg << 16) | ise, wtmp, &tot);
                const uint32_t gb4 = gcar + (ex >> 16), eb4 = ecar + (ex & 0xffffu);
                const uint32_t pos = gb4 + min(eb4, need_eq);
                // pos < keep <= qC when the counts agree; the bound keeps a
                // remote store inside the cluster's slots whatever they hold
                if ((isg || (ise && eb4 < need_eq)) && pos < qC) {
                    const uint32_t owner = pos / qper, sl = pos - owner * qper;
                    st_cluster_u32(slot_base[owner] + 4u * sl, ids_in[t]);
                    const uint32_t sa = map_rank(smem_addr(sc_out + sl), owner);
                    asm volatile("st.shared::cluster.u8 [%0], %1;" ::"r"(sa), "r"(sc) : "memory");
                }
                gcar += tot >> 16;
                ecar += tot & 0xffffu;
            }
        }
        {
            uint32_t pgb = wbase[2 * warp], peb = wbase[2 * warp + 1];
            for (uint32_t g0 = gb; g0 < ge; g0 += 32) {
                const bool want_eq = peb < need_eq;
                const uint32_t g = g0 + lane;
                uint32_t gm = 0, em = 0;
                uint32_t acc[B];
#pragma unroll
                for (int q = 0; q < B; ++q) acc[q] = 0u;
                if (g < ge) {
                    load_scores<B>(planes, A.G, g, acc);
                    gm = bitsliced_ge<B>(acc, theta + 1);
                    em = bitsliced_ge<B>(acc, theta) & ~gm;
                    const uint32_t base = g * 32;
                    if (base + 32 > valid) em &= valid > base ? (0xffffffffu >> (32 - (valid - base))) : 0u;
                }
                const uint32_t cg = __popc(gm), ce = __popc(em);
                const uint32_t any = __ballot_sync(0xffffffffu, (gm | (want_eq ? em : 0u)) != 0u);
                if (!any) {
                    if (want_eq) peb += __reduce_add_sync(0xffffffffu, ce);
                    continue;
                }
                uint32_t ig = cg, ie = ce;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t yg = __shfl_up_sync(0xffffffffu, ig, o);
                    const uint32_t ye = __shfl_up_sync(0xffffffffu, ie, o);
                    if (lane >= o) {
                        ig += yg;
                        ie += ye;
                    }
                }
                uint32_t pg = pgb + ig - cg, pe = peb + ie - ce;
                const uint32_t base_id = id0 + g * 32;
                // only the lowest-id ties at theta up to need_eq are taken:
                // keep just this lane's share of them (the first need_eq - pe
                // of its tie bits); the positions of the ids above theta count
                // the ties before them capped at need_eq, so they are unchanged
                {
                    const uint32_t room = pe < need_eq ? need_eq - pe : 0u;
                    if (room < ce) {
                        uint32_t drop = em;
                        for (uint32_t t = 0; t < room; ++t) drop &= drop - 1u;  // clear the lowest `room` set bits
                        em &= ~drop;
                    }
                }
                while (gm | em) {
                    const int j = __ffs(gm | em) - 1;
                    const uint32_t bit = 1u << j;
                    uint32_t pos = 0xffffffffu;
                    if (gm & bit) {
                        pos = pg + min(pe, need_eq);
                        ++pg;
                    } else {
                        if (pe < need_eq) pos = pg + pe;
                        ++pe;
                    }
                    gm &= ~bit;
                    em &= ~bit;
                    if (pos < qC) {  // (0xffffffff: not taken; the bound keeps the store in the slots)
                        const uint32_t owner = pos / qper, sl = pos - owner * qper;
                        st_cluster_u32(slot_base[owner] + 4u * sl, base_id + (uint32_t)j);
                        if (multi) {
                            uint32_t sc = 0;
#pragma unroll
                            for (int q = 0; q < B; ++q) sc |= ((acc[q] >> j) & 1u) << q;
                            const uint32_t sa = map_rank(smem_addr(sc_out + sl), owner);
                            asm volatile("st.shared::cluster.u8 [%0], %1;" ::"r"(sa), "r"(sc) : "memory");
                        }
                    }
                }
                pgb += __shfl_sync(0xffffffffu, ig, 31);
                peb += __shfl_sync(0xffffffffu, ie, 31);
            }
        }
        stamp(A, b, r, 11);
        cluster_sync();  // #3: the new list (or, after one pass, every candidate slot) is filled
        stamp(A, b, r, 12);
        run_n = keep;
    }

    if (A.dbg_cands) {
        const uint32_t mc = qC > r * qper ? min(qper, qC - r * qper) : 0u;
        for (uint32_t t = threadIdx.x; t < mc; t += NT) A.dbg_cands[b * A.C + r * qper + t] = (int32_t)ids_out[t];
    }

    // ---- S6: exact FP32 re-rank of this CTA's share of the candidates.  The
    // next query is known since cluster barrier #2: its row is copied into
    // o_qn meanwhile, for the next S0
    {
        const int64_t bn = A.work ? (int64_t)*reinterpret_cast<volatile uint32_t*>(next_q) : b + Gc;
        if (A.o_qn && bn < A.nq) {
            const float* qg = A.Q + bn * A.d;
            float* qn = reinterpret_cast<float*>(smem + A.o_qn);
            for (int j = threadIdx.x; j < A.d; j += NT) cp_async4(qn + j, qg + (A.qperm ? A.qperm[j] : j));
            q_next = true;
        }
    }
    const uint32_t* slots = ids_out;
    const uint32_t mine = qC > r * qper ? min(qper, qC - r * qper) : 0u;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem + A.o_keys);  // [sortP]
    const float4* q4 = reinterpret_cast<const float4*>(smem + A.o_q);
    uint32_t nk = mine;  // keys of this CTA that enter the local top-k
    if (MET != 0 || A.precision == 0 || qC <= A.R) {  // the coarse passes serve the squared distance only
        if (A.ld / 4 >= 64 && A.ld / 4 < 128)
            rerank_fp32<NT, S6_CH_LONG, MET>(A, q4, slots, mine, keys);
        else
            rerank_fp32<NT, S6_CH_SHORT, MET>(A, q4, slots, mine, keys);
        __syncthreads();
    } else if constexpr (MET == 0) {
        // coarse pass on the reduced-precision copy, then the R smallest
        // coarse keys of the whole cluster survive into the exact pass
        if (A.precision == 1)
            if (A.ldh / 8 >= 64 && A.ldh / 8 < 128)
                rerank_bf16<NT, S6_CH_LONG>(A, q4, slots, mine, keys);
            else
                rerank_bf16<NT, S6_CH_SHORT>(A, q4, slots, mine, keys);
        else
            rerank_fp8<NT>(A, q4, slots, mine, keys);
        __syncthreads();
        const unsigned long long cut = cluster_rank_cut<NT>(A, smem, keys, mine, A.R);
        uint32_t* ns = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 106;
        if (threadIdx.x == 0) *ns = 0u;
        __syncthreads();
        uint32_t* surv_ids = const_cast<uint32_t*>(slots);  // the candidate ids now live in the keys
        for (uint32_t t0 = 0; t0 < mine; t0 += NT) {  // CTA-uniform trip count: warp_alloc needs whole warps
            const uint32_t t = t0 + threadIdx.x;
            const unsigned long long key = t < mine ? keys[t] : ~0ull;
            const bool keep = t < mine && key <= cut;
            const uint32_t slot = warp_alloc(ns, keep);
            if (keep) {
                const uint32_t id = (uint32_t)(key & 0xffffffffu);
                surv_ids[slot] = id;
                if (A.dbg_surv) A.dbg_surv[b * A.n + id] = 1u;
            }
        }
        __syncthreads();
        nk = *ns;
        if (A.ld / 4 >= 64 && A.ld / 4 < 128)
            rerank_fp32<NT, S6_CH_LONG, 0>(A, q4, surv_ids, nk, keys);
        else
            rerank_fp32<NT, S6_CH_SHORT, 0>(A, q4, surv_ids, nk, keys);
        __syncthreads();
    }

    stamp(A, b, r, 13);
    // local top-k: a linear bucket histogram of the distances finds a bucket
    // that holds the k-th smallest; only keys up to it are sorted
    uint32_t* khist = reinterpret_cast<uint32_t*>(smem + A.o_union);               // [NB]
    unsigned long long* surv = reinterpret_cast<unsigned long long*>(khist + NB);   // [SURV_CAP]
    uint32_t* kv = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 100;             // min, max, bucket, count
    const uint32_t k = qk;           // this query's k (lists are stored at stride A.k)
    const uint32_t kst = (uint32_t)A.k;
    unsigned long long* best = keys;  // sorted top-k ends up here
    uint32_t nbest = 0;
    if (nk <= 2 * k || nk <= 64) {
        if (nk <= 128) {
            rank_sort<NT>(keys, nk, surv);
            best = surv;
            __syncthreads();
        } else {
            const uint32_t P = next_pow2_dev(nk);
            for (uint32_t t = nk + threadIdx.x; t < P; t += NT) keys[t] = ~0ull;
            __syncthreads();
            block_bitonic_sort<NT>(keys, (int)P);
        }
        nbest = min(k, nk);
    } else {
        if (threadIdx.x == 0) {
            kv[0] = 0xffffffffu;
            kv[1] = 0u;
            kv[3] = 0u;
        }
        for (int t = threadIdx.x; t < NB; t += NT) khist[t] = 0u;
        __syncthreads();
        uint32_t lo = 0xffffffffu, hi = 0u;
        for (uint32_t t = threadIdx.x; t < nk; t += NT) {
            const unsigned long long v = keys[t];
            if (v == ~0ull) continue;
            const uint32_t db = (uint32_t)(v >> 32);
            lo = min(lo, db);
            hi = max(hi, db);
        }
        lo = __reduce_min_sync(0xffffffffu, lo);  // one atomic per warp
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0 && lo != 0xffffffffu) atomicMin(&kv[0], lo);
        if (lane == 0 && hi) atomicMax(&kv[1], hi);
        __syncthreads();
        const float dmin = __uint_as_float(kv[0]);
        const float drange = __fsub_rn(__uint_as_float(kv[1]), dmin);
        const float dscale = drange > 0.f ? __fdiv_rn((float)NB, drange) : 0.f;
        for (uint32_t t = threadIdx.x; t < nk; t += NT) {
            const unsigned long long v = keys[t];
            if (v != ~0ull) atomicAdd(&khist[value_bucket(__uint_as_float((uint32_t)(v >> 32)), dmin, dscale)], 1u);
        }
        __syncthreads();
        {
            constexpr int BPT = NB / NT > 0 ? NB / NT : 1;
            uint32_t v[BPT], sum = 0;
#pragma unroll
            for (int u = 0; u < BPT; ++u) {
                const int e = threadIdx.x * BPT + u;
                v[u] = e < NB ? khist[e] : 0u;
                sum += v[u];
            }
            uint32_t tot;
            uint32_t run = block_exclusive_scan<NT>(sum, reinterpret_cast<uint32_t*>(smem + A.o_hist) + 256, &tot);
#pragma unroll
            for (int u = 0; u < BPT; ++u) {
                const int e = threadIdx.x * BPT + u;
                if (e < NB && ((run < k && run + v[u] >= k) || (tot < k && e == NB - 1))) {
                    kv[2] = (uint32_t)e;
                    kv[3] = run + v[u];
                }
                run += v[u];
            }
        }
        __syncthreads();
        const uint32_t kb = kv[2], ns = kv[3];
        if (ns <= SURV_CAP) {
            uint32_t* ctr = kv + 4;
            if (threadIdx.x == 0) *ctr = 0u;
            __syncthreads();
            for (uint32_t t0 = 0; t0 < nk; t0 += NT) {  // CTA-uniform trip count: warp_alloc needs whole warps
                const uint32_t t = t0 + threadIdx.x;
                const unsigned long long v = t < nk ? keys[t] : ~0ull;
                const bool keep =
                    v != ~0ull && (uint32_t)value_bucket(__uint_as_float((uint32_t)(v >> 32)), dmin, dscale) <= kb;
                const uint32_t slot = warp_alloc(ctr, keep);
                if (keep) surv[slot] = v;
            }
            __syncthreads();
            if (ns <= 128) {
                rank_sort<NT>(surv, ns, keys);  // the re-rank keys are no longer read
                __syncthreads();
                best = keys;
            } else {
                uint32_t P = 1;
                while (P < ns) P <<= 1;
                for (uint32_t t = ns + threadIdx.x; t < P; t += NT) surv[t] = ~0ull;
                __syncthreads();
                block_bitonic_sort<NT>(surv, (int)P);
                best = surv;
            }
            nbest = min(k, ns);
        } else {
            // a crowded bucket (many equal distances): sort the whole share
            const uint32_t P = next_pow2_dev(nk);
            for (uint32_t t = nk + threadIdx.x; t < P; t += NT) keys[t] = ~0ull;
            __syncthreads();
            block_bitonic_sort<NT>(keys, (int)P);
            nbest = min(k, nk);
        }
    }
    // hand the sorted local list (padded to k) to CTA 0
    {
        unsigned long long* recv = reinterpret_cast<unsigned long long*>(smem + A.o_seg);  // [CL][k] on CTA 0
        const uint32_t rb = map_rank(smem_addr(recv + (size_t)r * k), 0u);
        for (uint32_t t = threadIdx.x; t < k; t += NT) {
            const unsigned long long v = t < nbest ? best[t] : ~0ull;
            st_cluster_u32(rb + 8u * t, (uint32_t)v);
            st_cluster_u32(rb + 8u * t + 4u, (uint32_t)(v >> 32));
        }
    }
    stamp(A, b, r, 14);
    cluster_sync();  // #4: every local top-k is in CTA 0; the other CTAs are done
    stamp(A, b, r, 15);

    if (r == 0) {
        // merge by rank: a key's final position is the number of smaller keys
        // over all CL sorted lists (keys are unique because ids are)
        const unsigned long long* all = reinterpret_cast<const unsigned long long*>(smem + A.o_seg);
        const uint32_t tot = (uint32_t)CL * k;
        uint32_t* nreal = kv + 5;
        if (threadIdx.x == 0) *nreal = 0u;
        __syncthreads();
        uint32_t real = 0;
        uint32_t P = 2;  // a power of two above k
        while (P <= k) P <<= 1;
        for (uint32_t t = threadIdx.x; t < tot; t += NT) {
            const unsigned long long v = all[t];
            if (v == ~0ull) continue;
            ++real;
            uint32_t rank;
            switch (CL) {
                case 16: rank = rank_in_lists<16>(all, k, P, v); break;
                case 8: rank = rank_in_lists<8>(all, k, P, v); break;
                case 4: rank = rank_in_lists<4>(all, k, P, v); break;
                case 2: rank = rank_in_lists<2>(all, k, P, v); break;
                default: rank = rank_in_lists<1>(all, k, P, v); break;
            }
            if (rank < k) {
                A.out_ids[b * kst + rank] = (int32_t)(uint32_t)(v & 0xffffffffu);
                A.out_dist[b * kst + rank] = __uint_as_float((uint32_t)(v >> 32));
            }
        }
        real = __reduce_add_sync(0xffffffffu, real);  // one atomic per warp, not per key
        if (lane == 0 && real) atomicAdd(nreal, real);
        __syncthreads();
        // fewer than k real keys, or a per-query k below the row length: pad the tail
        for (uint32_t t = min(*nreal, k) + threadIdx.x; t < kst; t += NT) {
            A.out_ids[b * kst + t] = -1;
            A.out_dist[b * kst + t] = __int_as_float(0x7f800000);
        }
    }
    if (r == 0) {
        __syncthreads();
        stamp(A, b, r, 16);
    }
    // next query: the cluster barriers of its stages order every remote access
    // (next_q was written before #2 and is read after #4)
    if (A.work) {
        b = (int64_t)*reinterpret_cast<volatile uint32_t*>(next_q);
    } else {
        b += Gc;
    }
    }
    // the last cluster to finish returns the work counter to zero for the next launch
    if (A.work && r == 0 && threadIdx.x == 0) {
        if (atomicAdd(A.work + 1, 1u) == Gc - 1u) {
            atomicExch(A.work, 0u);
            atomicExch(A.work + 1, 0u);
        }
    }
}

uint32_t align16(uint64_t x) { return (uint32_t)((x + 15) & ~uint64_t(15)); }

uint32_t next_pow2(uint32_t x)
{
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

struct Layout {
    QArgs A;
    size_t smem = 0;
};

// One shared-memory layout.  pair: room for two S3 scratch groups (a CTA
// that owns two subspaces ranks them at once when they fit); qn: a buffer for
// the next query's row.
int layout_once(const DeviceIndex* ix, int CL, int npass, int nsmax, int NT, uint32_t C, int k, bool pair, bool qn,
                Layout* L)
{
    QArgs& A = L->A;
    memset(&A, 0, sizeof(A));
    A.CL = CL;
    A.npass = (uint32_t)npass;
    A.nch = ix->nch;
    A.cpc = ix->nch / (CL * npass);
    A.k = k;
    A.k_pad = (k + 1) & ~1;
    A.per_cta = (C + CL - 1) / CL;
    A.span = (uint32_t)(A.cpc * ix->n_ch);
    A.G = A.span / 32;
    const int sk = ix->sqrtK;
    const int NC = nsmax + 2;
    uint64_t o = 0;
    A.o_tab = (uint32_t)o;
    A.tab_copy = align16(20 + 6ull * sk);
    A.tab_stride = align16(A.tab_copy + 10ull * sk);
    // the radix histograms of the survivor cut (S6) reuse the subspace tables'
    // region: no CTA reads a table after S4, and the next query's tables are
    // written only after cluster barrier #4, when every remote read of the
    // histograms is done
    A.o_rsel = A.o_tab;
    o = align16(o + std::max<uint64_t>((uint64_t)ix->Ns * A.tab_stride, 4ull * 512));
    A.o_q = (uint32_t)o;
    A.ldq = (ix->d + 15) & ~15;
    o = align16(o + 4ull * A.ldq);
    if (qn) {
        A.o_qn = (uint32_t)o;
        o = align16(o + 4ull * A.ldq);
    }
    A.o_hist = (uint32_t)o;
    o = align16(o + 4ull * (pair ? 2 : 1) * HIST_WORDS);  // one per S3 group
    A.o_misc = (uint32_t)o;
    o = align16(o + 4ull * 160);

    A.o_cnt = (uint32_t)o;
    o = align16(o + 4ull * NC * (2 + 2 * CL + NT / 32));
    // S4's segment list; from S5 on, CTA 0's inbox of the CL local top-k lists
    // followed by this CTA's candidate slots
    A.o_seg = (uint32_t)o;
    A.o_slots = (uint32_t)(o + align16(8ull * CL * k));
    o = align16(o + std::max<uint64_t>(16ull * MAXSEG + 4ull * (MAXSEG + 1), align16(8ull * CL * k) + 4ull * A.per_cta));
    // a multi-pass query's running candidate list lives across the passes'
    // S4 (which reuses the segment region), so it has a region of its own
    A.run_stride = (A.per_cta + 15) & ~15u;
    A.o_run = (uint32_t)o;
    if (npass > 1) o = align16(o + 10ull * A.run_stride);
    // at least 128: the rank sort of up to 128 top-k survivors writes them here
    A.sortP = next_pow2(std::max<uint32_t>(A.per_cta, 128));
    A.o_union = (uint32_t)o;
    A.nbits = nsmax == 8 ? 4 : (nsmax == 16 ? 5 : 6);
    // S4 counters: nibble sets of up to 15 subspaces, then one-bit planes for
    // the last few (a second set only when 4 or more subspaces remain)
    {
        const int Ns = ix->Ns;
        A.nsets = (Ns <= 15 || Ns - 15 <= 3) ? 1u : 2u;
        A.nplanes = (uint32_t)std::max(0, Ns - 15 * (int)A.nsets);
        A.nstore = std::max(A.nbits, 4u * A.nsets + A.nplanes);
    }
    const uint64_t plane_bytes = 4ull * A.nstore * A.G;
    const uint64_t cent_bytes = 8ull * sk * ix->hmax;
    // staging the centroids dimension-major pays only for wide halves: with
    // halves of up to 16 dims each thread's direct row loads measured faster
    // (0.4-1.1 % per launch at the 8-dim halves of the 1M workloads)
    A.stage_cent = cent_bytes <= 65536 && ix->hmax > 16 ? 1u : 0u;
    const uint64_t s3_bytes = S3_BYTES + (A.stage_cent ? align16(cent_bytes) : 0);
    // S6 reuses the union: the distance histogram and survivors at its start,
    // the CTA's re-rank keys at its end
    const uint64_t keys_bytes = align16(8ull * A.sortP);
    const uint64_t s6_bytes = 4ull * NB + 8ull * SURV_CAP + keys_bytes;
    // S3's copy of the cell offsets, where the region has room for it anyway
    const uint64_t cells_bytes = 4ull * ((uint64_t)ix->K + 1);
    if (s3_bytes + cells_bytes <= std::max(plane_bytes, s6_bytes)) A.o_cells = (uint32_t)s3_bytes;
    const uint64_t ubytes = align16(std::max(plane_bytes, std::max(s3_bytes, s6_bytes)));
    // two S3 groups side by side fit in the union, and each half of the CTA
    // has a thread for every centroid column (the 2-D cell mapping of S3)
    A.s3_stride = align16(s3_bytes + (A.o_cells ? cells_bytes : 0));
    A.pair_ok = (pair && 2ull * A.s3_stride <= ubytes && (uint32_t)(NT / 2) >= next_pow2((uint32_t)sk)) ? 1u : 0u;
    // S3's per-cell bucket store, where the groups still fit the region with it
    {
        const uint64_t with = align16(A.s3_stride + 2ull * ix->K);
        if ((A.pair_ok ? 2ull : 1ull) * with <= ubytes) {
            A.o_bkt = (uint32_t)A.s3_stride;
            A.s3_stride = (uint32_t)with;
        }
    }
    A.o_keys = (uint32_t)(o + ubytes - keys_bytes);

    o = align16(o + ubytes);
    L->smem = o;
    return SUCO_OK;
}

// The layout of a launch shape: the paired S3 scratch and the next-row buffer
// are added only where they cost no CTAs per SM (228 KB of shared memory per
// SM, 1 KB reserved per CTA; 64 registers a thread allow 1024 / NT CTAs).
int make_layout(const DeviceIndex* ix, int CL, int npass, int nsmax, int NT, uint32_t C, int k, Layout* L)
{
    auto ctas = [&](const Layout& l) {
        return std::min<uint64_t>(233472ull / (l.smem + 1024ull), (uint64_t)(1024 / NT));
    };
    Layout best, t;
    layout_once(ix, CL, npass, nsmax, NT, C, k, false, false, &best);
    layout_once(ix, CL, npass, nsmax, NT, C, k, true, false, &t);
    if (t.A.pair_ok && ctas(t) >= ctas(best)) best = t;
    layout_once(ix, CL, npass, nsmax, NT, C, k, best.A.pair_ok != 0, true, &t);
    if (ctas(t) >= ctas(best)) best = t;
    *L = best;
    return SUCO_OK;
}

// Co-resident clusters for a launch shape, cached (the occupancy query is not
// repeated, so later calls can be captured into a CUDA graph).
struct OccKey {
    const void* fn;
    int CL;
    size_t smem;
};
std::mutex g_occ_mu;
std::vector<std::pair<OccKey, int>> g_occ;

template <int NT, int NSMAX, int MET>
int launch_t(const Layout& L, int64_t nq, bool persistent, uint32_t* work, cudaStream_t st)
{
    auto kern = suco_query_kernel<NT, NSMAX, MET>;
    SUCO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
    if (L.A.CL > 8) SUCO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)L.A.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int64_t G = nq;
    QArgs A = L.A;
    A.work = nullptr;
    if (persistent) {
        int nclusters = 0;
        {
            std::lock_guard<std::mutex> lock(g_occ_mu);
            for (auto& e : g_occ)
                if (e.first.fn == (const void*)kern && e.first.CL == L.A.CL && e.first.smem == L.smem)
                    nclusters = e.second;
        }
        if (nclusters == 0) {
            cfg.gridDim = dim3((unsigned)L.A.CL, 1, 1);
            if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
                cudaGetLastError();
                nclusters = 0;
            } else {
                std::lock_guard<std::mutex> lock(g_occ_mu);
                g_occ.push_back({OccKey{(const void*)kern, L.A.CL, L.smem}, nclusters});
            }
        }
        if (nclusters > 0) G = std::min<int64_t>(nq, nclusters);
        if (G < nq) A.work = work;
    }
    cfg.gridDim = dim3((unsigned)(G * L.A.CL), 1, 1);
    if (fault_fires(SUCO_FAULT_LAUNCH)) return fail(SUCO_ECUDA, "suco_query_kernel: injected launch failure");
    SUCO_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, A));
    return SUCO_OK;
}

// L1 indexes run 512-thread CTAs only (one more set of instantiations)
int dispatch(const Layout& L, int NT, int nsmax, int metric, int64_t nq, bool persistent, uint32_t* work,
             cudaStream_t st)
{
    if (metric == SUCO_METRIC_L1) {
        if (NT != 512) return fail(SUCO_EUNSUPPORTED, "an L1 index runs CTAs of 512 threads (this launch needs %d)", NT);
        if (nsmax == 8) return launch_t<512, 8, 1>(L, nq, persistent, work, st);
        if (nsmax == 16) return launch_t<512, 16, 1>(L, nq, persistent, work, st);
        return launch_t<512, 32, 1>(L, nq, persistent, work, st);
    }
    if (NT == 1024) {
        if (nsmax == 8) return launch_t<1024, 8, 0>(L, nq, persistent, work, st);
        if (nsmax == 16) return launch_t<1024, 16, 0>(L, nq, persistent, work, st);
        return launch_t<1024, 32, 0>(L, nq, persistent, work, st);
    }
    if (NT == 256) {
        if (nsmax == 8) return launch_t<256, 8, 0>(L, nq, persistent, work, st);
        if (nsmax == 16) return launch_t<256, 16, 0>(L, nq, persistent, work, st);
        return launch_t<256, 32, 0>(L, nq, persistent, work, st);
    }
    if (nsmax == 8) return launch_t<512, 8, 0>(L, nq, persistent, work, st);
    if (nsmax == 16) return launch_t<512, 16, 0>(L, nq, persistent, work, st);
    return launch_t<512, 32, 0>(L, nq, persistent, work, st);
}

}  // namespace

int launch_query(const DeviceIndex* ix, const float* Q, int64_t nq, const suco_query_params* p, int32_t* ids,
                 float* dist, const suco_query_debug_out* dbg, cudaStream_t st)
{
    if (nq == 0) return SUCO_OK;
    int64_t T = 0, C = 0;
    thresholds(ix->n, p->alpha, p->beta, p->k, &T, &C);
    const int nsmax = ix->Ns <= 8 ? 8 : (ix->Ns <= 16 ? 16 : 32);
    int NT = p->threads;
    if (NT != 0 && NT != 256 && NT != 512 && NT != 1024)
        return fail(SUCO_EINVAL, "threads must be 0, 256, 512 or 1024 (got %d)", NT);
    int CL = p->cluster_size;
    if (CL == 0 && NT == 0)
        for (const auto& t : ix->tuned)
            if (t.k == p->k && t.C == (uint32_t)C) {
                CL = t.CL;
                NT = t.NT;
            }
    if (CL != 0 && CL != 1 && CL != 2 && CL != 4 && CL != 8 && CL != 16)
        return fail(SUCO_EINVAL, "cluster_size must be 0, 1, 2, 4, 8 or 16 (got %d)", CL);
    int dev_smem = 0, sm_smem = 0, reserved = 0;
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device));
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ix->device));
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, ix->device));
    // two 512-thread CTAs per SM let the phases of two queries overlap
    const size_t two_per_sm = (size_t)sm_smem / 2 - (size_t)reserved;
    const int NP = p->id_passes;
    if (NP < 0 || (NP & (NP - 1)) != 0 || NP > ix->nch)
        return fail(SUCO_EINVAL, "id_passes=%d must be 0 or a power of two <= %d", NP, ix->nch);
    // the first shape that fits, in this order: two 512-thread CTAs per SM with
    // the fewest passes and the smallest cluster, then one 1024-thread CTA per SM
    Layout L;
    bool chosen = false;
    int npass = 1;
    for (int stage = 0; stage < 2 && !chosen; ++stage) {
        const int nt = stage == 0 ? 512 : (NT ? NT : 1024);
        if (stage == 0 && NT != 0 && NT != 512) continue;
        for (int np = NP ? NP : 1; np <= (NP ? NP : ix->nch) && !chosen; np *= 2) {
            for (int cl = CL ? CL : 1; cl <= (CL ? CL : 16) && !chosen; cl *= 2) {
                if (cl * np > ix->nch) continue;
                make_layout(ix, cl, np, nsmax, nt, (uint32_t)C, p->k, &L);
                const bool fits = stage == 0 ? (L.smem <= two_per_sm || (NT == 512 && L.smem <= (size_t)dev_smem))
                                             : L.smem <= (size_t)dev_smem;
                if (fits) {
                    CL = cl;
                    NT = nt;
                    npass = np;
                    chosen = true;
                }
            }
        }
    }
    if (!chosen)
        return fail(SUCO_EUNSUPPORTED,
                    "n=%lld with Ns=%d, C=%lld does not fit the shared memory of %s CTAs in up to %d passes",
                    (long long)ix->n, ix->Ns, (long long)C, p->cluster_size ? "the requested" : "up to 16",
                    NP ? NP : ix->nch);
    (void)npass;
    if (nq * CL > 0x7fffffffLL) return fail(SUCO_EINVAL, "too many queries in one call");
    QArgs& A = L.A;
    A.X = ix->X;
    A.ld = ix->ld;
    A.n = ix->n;
    A.d = ix->d;
    A.Ns = ix->Ns;
    A.sqrtK = ix->sqrtK;
    A.K = (int32_t)ix->K;
    A.hmax = ix->hmax;
    A.sub_s = ix->sub_s;
    A.cent = ix->cent;
    A.cell_off = ix->cell_off;
    A.perm = ix->perm;
    A.split = ix->split;
    A.n_ch = ix->n_ch;
    A.Q = Q;
    A.nq = nq;
    A.T = (uint32_t)T;
    A.C = (uint32_t)C;
    A.alpha = p->alpha;
    A.beta = p->beta;
    A.k_per = p->k_per_query;
    A.alpha_per = p->alpha_per_query;
    A.beta_per = p->beta_per_query;
    A.out_ids = ids;
    A.out_dist = dist;
    A.precision = p->precision;
    A.R = (uint32_t)(p->exact_rerank > 0 ? p->exact_rerank : 512);
    A.Xh = ix->Xh;
    A.ldh = ix->ldh;
    A.X8 = ix->X8;
    A.ld8 = ix->ld8;
    A.s8col = ix->s8col;
    A.qperm = ix->dperm;

    if (dbg) {
        A.dbg_teff = dbg->t_eff;
        A.dbg_act = dbg->activated;
        A.dbg_dtab = dbg->dtab;
        A.dbg_scores = dbg->scores;
        A.dbg_cands = dbg->cands;
        A.dbg_surv = dbg->survivors;
        A.dbg_clk = reinterpret_cast<long long*>(dbg->stage_clock);
    }
    const bool persistent = (p->flags & SUCO_QUERY_ONE_CLUSTER_PER_QUERY) == 0;
    if (p->rank_precision == SUCO_RANK_BF16 || p->rank_precision == SUCO_RANK_FP8) {
        // one tensor-core table launch and one query launch per RANK_CHUNK queries
        const QArgs base = A;
        for (int64_t c0 = 0; c0 < nq; c0 += RANK_CHUNK) {
            const int64_t cnt = std::min<int64_t>(RANK_CHUNK, nq - c0);
            int rc = rank_tc_tables(ix, Q + c0 * ix->d, cnt, ix->rank_ws, p->rank_precision == SUCO_RANK_FP8, st);
            if (!rc) rc = check_status(ix);  // a wait that gave up is reported before its tables are used
            if (rc) return rc;
            QArgs& C2 = L.A;
            C2 = base;
            C2.Q = base.Q + c0 * ix->d;
            C2.nq = cnt;
            C2.dtab_in = ix->rank_ws;
            C2.out_ids = base.out_ids + c0 * base.k;
            C2.out_dist = base.out_dist + c0 * base.k;
            if (base.k_per) C2.k_per = base.k_per + c0;
            if (base.alpha_per) C2.alpha_per = base.alpha_per + c0;
            if (base.beta_per) C2.beta_per = base.beta_per + c0;
            if (base.dbg_teff) C2.dbg_teff = base.dbg_teff + c0 * base.Ns;
            if (base.dbg_act) C2.dbg_act = base.dbg_act + c0 * base.Ns * (int64_t)base.K;
            if (base.dbg_dtab) C2.dbg_dtab = base.dbg_dtab + c0 * base.Ns * 2 * base.sqrtK;
            if (base.dbg_scores) C2.dbg_scores = base.dbg_scores + c0 * base.n;
            if (base.dbg_cands) C2.dbg_cands = base.dbg_cands + c0 * (int64_t)base.C;
            if (base.dbg_surv) C2.dbg_surv = base.dbg_surv + c0 * base.n;
            if (base.dbg_clk) C2.dbg_clk = base.dbg_clk + c0 * 16 * NCLK;
            uint32_t* work = ix->work + (size_t)WORK_STRIDE * (__atomic_fetch_add(&const_cast<DeviceIndex*>(ix)->work_next,
                                                                                1u, __ATOMIC_RELAXED) % WORK_SLOTS);
            rc = dispatch(L, NT, nsmax, ix->metric, cnt, persistent, work, st);
            if (rc) return rc;
        }
        return SUCO_OK;
    }
    // each call takes the next of the index's work counters in turn
    uint32_t* work = ix->work + (size_t)WORK_STRIDE *
                                    (__atomic_fetch_add(&const_cast<DeviceIndex*>(ix)->work_next, 1u,
                                                        __ATOMIC_RELAXED) % WORK_SLOTS);
    return dispatch(L, NT, nsmax, ix->metric, nq, persistent, work, st);
}

}  // namespace suco
