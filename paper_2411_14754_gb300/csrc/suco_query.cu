// The SuCo query path (Section 4.2: Algorithm 4, with Algorithm 3's cell walk)
// as one kernel in which a thread-block cluster of CL CTAs answers one query.
//
// Stages inside the kernel (all in one launch, no global scratch):
//   S0  the query row is staged in shared memory.
//   S1  squared half-subspace centroid distances d1[a], d2[c] in FP32
//       (acc = fma(q_j - c_j, q_j - c_j, acc) over j ascending).
//   S2  stable ranks r1[a], r2[c] of those distances (ties by centroid index).
//   S3  cell activation: Algorithm 3 retrieves cells in ascending order of the
//       key (f32 bits of d1[a]+d2[c], r1[a], r2[c]) until alpha*n ids are
//       collected.  Instead of walking the cells one by one, a weighted radix
//       select over the 48-bit keys (weights = cell sizes) finds the cut key
//       kappa* with W(key < kappa*) < T <= W(key <= kappa*); the retrieved
//       cells are exactly those with key <= kappa*.  CTA r handles the
//       subspaces i with i % CL == r and publishes its tables to the cluster.
//   S4  SC-score counting (Definition 4): each CTA owns a contiguous id range
//       and keeps one uint8 score per id in shared memory (four per 32-bit
//       word).  It scans, for every retrieved cell of every subspace, the part
//       of the cell's id list that falls in its range and adds 1 to the score
//       byte with a shared-memory atomic.
//   S5  candidate selection: counts of scores >= s are summed over the cluster
//       through distributed shared memory; theta is the largest s with at least
//       C scores >= s; every id above theta and the lowest-id ties at theta
//       (up to C in total) are written, in id order, straight into the
//       candidate slots of the CTA that will re-rank them.
//   S6  exact re-rank: every CTA computes FP32 squared distances of its share
//       of the C candidates (one warp per row, float4 loads), keeps a local
//       top-k by (distance, id), and CTA 0 merges the CL local lists.
#include <algorithm>
#include <cstring>

#include "suco_internal.cuh"

namespace suco {
namespace {

constexpr int MAXSEG = 4096;  // segment-list capacity per scan round
constexpr int RTILE = 2048;   // candidates per re-rank round

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
    uint32_t T, C, per_cta;
    int32_t* out_ids;
    float* out_dist;
    int64_t* dbg_teff;
    uint8_t* dbg_act;
    float* dbg_dtab;
    uint8_t* dbg_scores;
    int32_t* dbg_cands;
    // shared-memory layout (byte offsets)
    uint32_t o_tab, tab_stride, o_q, o_hist, o_misc, o_cnt, o_seg, o_slots, o_union;
    uint32_t score_words, sortP, mergeP;
};

// ---------------------------------------------------------------------------
// cluster / distributed-shared-memory primitives (inline PTX)

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
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

__device__ __forceinline__ unsigned long long ld_cluster_u64(uint32_t addr)
{
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------

// Cell key of Algorithm 3's retrieval order: FP32 cell sum, then the ranks.
__device__ __forceinline__ unsigned long long cell_key(float a, float b, uint32_t r1, uint32_t r2)
{
    const float s = __fadd_rn(a, b);
    return ((unsigned long long)__float_as_uint(s) << 16) | (r1 << 8) | r2;
}

struct Tab {  // one subspace's ranking tables inside shared memory
    unsigned long long* kappa;
    unsigned long long* teff;
    float* d1;
    float* d2;
    uint8_t* r1;
    uint8_t* r2;
};

__device__ __forceinline__ Tab tab_at(char* smem, const QArgs& A, int i)
{
    char* t = smem + A.o_tab + (size_t)i * A.tab_stride;
    Tab T;
    T.kappa = reinterpret_cast<unsigned long long*>(t);
    T.teff = reinterpret_cast<unsigned long long*>(t + 8);
    T.d1 = reinterpret_cast<float*>(t + 16);
    T.d2 = T.d1 + A.sqrtK;
    T.r1 = reinterpret_cast<uint8_t*>(T.d2 + A.sqrtK);
    T.r2 = T.r1 + A.sqrtK;
    return T;
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

// S1-S3 for subspace i of query b.
template <int NT>
__device__ void rank_subspace(const QArgs& A, char* smem, int64_t b, int i)
{
    const int sk = A.sqrtK;
    const float* qs = reinterpret_cast<const float*>(smem + A.o_q);
    Tab tb = tab_at(smem, A, i);
    int32_t soff, slen;
    soff = i * A.sub_s;
    slen = (i == A.Ns - 1) ? A.d - (A.Ns - 1) * A.sub_s : A.sub_s;
    const int first = slen / 2;
    // S1: squared distances to the 2*sqrtK half-subspace centroids
    for (int t = threadIdx.x; t < 2 * sk; t += NT) {
        const int h = t >= sk;
        const int a = t - h * sk;
        const int off = soff + (h ? first : 0);
        const int len = h ? slen - first : first;
        const float* c = A.cent + ((int64_t)(i * 2 + h) * sk + a) * A.hmax;
        float acc = 0.f;
        for (int j = 0; j < len; ++j) {
            const float df = __fsub_rn(qs[off + j], __ldg(c + j));
            acc = __fmaf_rn(df, df, acc);
        }
        (h ? tb.d2 : tb.d1)[a] = acc;
    }
    __syncthreads();
    // S2: stable ranks
    for (int t = threadIdx.x; t < 2 * sk; t += NT) {
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
    }
    __syncthreads();
    // S3: weighted radix select of the cut key over the K cells
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + A.o_hist);
    unsigned long long* bc = reinterpret_cast<unsigned long long*>(smem + A.o_misc);
    const uint32_t* co = A.cell_off + (int64_t)i * (A.K + 1);
    const int lane = threadIdx.x & 31;
    unsigned long long prefix = 0, mask = 0, below = 0, last_w = 0;
    for (int pass = 0; pass < 6; ++pass) {
        const int shift = 40 - 8 * pass;
        for (int t = threadIdx.x; t < 256; t += NT) hist[t] = 0u;
        __syncthreads();
        for (int x = threadIdx.x; x < A.K; x += NT) {
            const int a = x / sk, c = x - a * sk;
            const unsigned long long key = cell_key(tb.d1[a], tb.d2[c], tb.r1[a], tb.r2[c]);
            if ((key & mask) == prefix) {
                const uint32_t w = __ldg(co + x + 1) - __ldg(co + x);
                if (w) atomicAdd(&hist[(key >> shift) & 255u], w);
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t v[8];
            uint32_t s = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = hist[lane * 8 + j];
                s += v[j];
            }
            uint32_t incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - s;
            const uint32_t need = (uint32_t)(A.T - below);
            const bool mine = excl < need && incl >= need;
            if (mine) {
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
        __syncthreads();
        prefix |= bc[0] << shift;
        mask |= 255ull << shift;
        below += bc[1];
        last_w = bc[2];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *tb.kappa = prefix;
        *tb.teff = below + last_w;
    }
    if (A.dbg_teff && threadIdx.x == 0) A.dbg_teff[b * A.Ns + i] = (int64_t)(below + last_w);
    if (A.dbg_dtab)
        for (int t = threadIdx.x; t < 2 * sk; t += NT)
            A.dbg_dtab[(b * A.Ns + i) * 2 * sk + t] = t < sk ? tb.d1[t] : tb.d2[t - sk];
    if (A.dbg_act)
        for (int x = threadIdx.x; x < A.K; x += NT) {
            const int a = x / sk, c = x - a * sk;
            A.dbg_act[(b * A.Ns + i) * A.K + x] = cell_key(tb.d1[a], tb.d2[c], tb.r1[a], tb.r2[c]) <= prefix;
        }
    __syncthreads();
}

// S4 inner loop: add 1 to the score of every id in the listed segments.
template <int NT>
__device__ void score_segments(const QArgs& A, char* smem, uint32_t m, uint32_t id0, uint32_t span)
{
    uint32_t* scores = reinterpret_cast<uint32_t*>(smem + A.o_union);
    uint32_t* seg_start = reinterpret_cast<uint32_t*>(smem + A.o_seg);
    uint32_t* seg_pre = seg_start + MAXSEG;
    uint32_t* wtmp = reinterpret_cast<uint32_t*>(smem + A.o_hist) + 256;
    // exclusive prefix of the segment lengths (stored in seg_pre), EPT per thread
    constexpr int EPT = MAXSEG / NT;
    uint32_t l[EPT], s = 0;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
        const uint32_t e = threadIdx.x * EPT + u;
        l[u] = e < m ? seg_pre[e] : 0u;
        s += l[u];
    }
    uint32_t F;
    uint32_t run = block_exclusive_scan<NT>(s, wtmp, &F);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
        const uint32_t e = threadIdx.x * EPT + u;
        if (e < m) seg_pre[e] = run;
        run += l[u];
    }
    if (threadIdx.x == 0) seg_pre[m] = F;
    __syncthreads();
    constexpr int NW = NT / 32;
    constexpr int U = 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint32_t tb = (uint32_t)warp * 32 * U; tb < F; tb += NW * 32 * U) {
        const uint32_t p0 = tb + lane;
        int lo = 0, hi = (int)m - 1;
        const uint32_t pp = min(p0, F - 1);
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_pre[mid] <= pp) lo = mid; else hi = mid - 1;
        }
        int sg = lo;
        int32_t idv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t pu = p0 + 32 * u;
            idv[u] = -1;
            if (pu < F) {
                while (seg_pre[sg + 1] <= pu) ++sg;
                idv[u] = __ldg(A.perm + seg_start[sg] + (pu - seg_pre[sg]));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (idv[u] >= 0) {
                const uint32_t loc = (uint32_t)idv[u] - id0;
                if (loc < span) atomicAdd(&scores[loc >> 2], 1u << ((loc & 3u) * 8u));
            }
    }
    __syncthreads();
}

// S4: enumerate the retrieved cells of every subspace and scan their ids.
template <int NT>
__device__ void count_scores(const QArgs& A, char* smem, uint32_t r)
{
    uint32_t* seg_start = reinterpret_cast<uint32_t*>(smem + A.o_seg);
    uint32_t* seg_len = seg_start + MAXSEG;
    uint32_t* misc = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 8;
    const int sk = A.sqrtK;
    const uint32_t id0 = r * (uint32_t)A.cpc * (uint32_t)A.n_ch;
    const int j0 = r * A.cpc, j1 = (r + 1) * A.cpc;
    const int total = A.Ns * A.K;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) misc[0] = 0u;
    __syncthreads();
    for (int g0 = 0; g0 < total; g0 += NT) {
        const int g = g0 + threadIdx.x;
        bool act = false;
        uint32_t st = 0, len = 0;
        if (g < total) {
            const int i = g / A.K;
            const int x = g - i * A.K;
            Tab tb = tab_at(smem, A, i);
            const int a = x / sk, c = x - a * sk;
            if (cell_key(tb.d1[a], tb.d2[c], tb.r1[a], tb.r2[c]) <= *tb.kappa) {
                const uint32_t* sp = A.split + (int64_t)i * (NCH + 1) * A.K;
                const uint32_t s0 = __ldg(sp + (int64_t)j0 * A.K + x);
                const uint32_t s1 = __ldg(sp + (int64_t)j1 * A.K + x);
                len = s1 - s0;
                st = (uint32_t)i * (uint32_t)A.n + s0;
                act = len > 0;
            }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, act);
        uint32_t base = 0;
        if (lane == 0 && bal) base = atomicAdd(&misc[0], (uint32_t)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (act) {
            const uint32_t pos = base + __popc(bal & lanemask_lt());
            seg_start[pos] = st;
            seg_len[pos] = len;
        }
        __syncthreads();
        const uint32_t m = misc[0];
        const bool last = g0 + NT >= total;
        __syncthreads();
        if (m > (uint32_t)(MAXSEG - NT) || (last && m > 0)) {
            score_segments<NT>(A, smem, m, id0, (uint32_t)A.cpc * (uint32_t)A.n_ch);
            if (threadIdx.x == 0) misc[0] = 0u;
            __syncthreads();
        }
    }
}

template <int NT, int NSMAX>
__global__ void __launch_bounds__(NT, 1) suco_query_kernel(const QArgs A)
{
    extern __shared__ __align__(16) char smem[];
    const uint32_t r = cluster_rank();
    const int CL = A.CL;
    const int64_t b = blockIdx.x / CL;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;

    // ---- S0: stage the query, clear the score array and the published counts
    {
        float* qs = reinterpret_cast<float*>(smem + A.o_q);
        const float* qg = A.Q + b * A.d;
        for (int j = threadIdx.x; j < A.ld; j += NT) qs[j] = j < A.d ? qg[j] : 0.f;
        uint4* sw = reinterpret_cast<uint4*>(smem + A.o_union);
        const uint4 z = make_uint4(0, 0, 0, 0);
        for (uint32_t w = threadIdx.x; w < A.score_words / 4; w += NT) sw[w] = z;
        uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + A.o_cnt);
        for (int t = threadIdx.x; t < NSMAX + 2; t += NT) cnt[t] = 0u;
        uint32_t* sl = reinterpret_cast<uint32_t*>(smem + A.o_slots);
        for (uint32_t t = threadIdx.x; t < A.per_cta; t += NT) sl[t] = 0xffffffffu;
    }
    __syncthreads();

    // ---- S1-S3 for the subspaces this CTA owns
    for (int i = (int)r; i < A.Ns; i += CL) rank_subspace<NT>(A, smem, b, i);
    cluster_sync();  // #1: every subspace's cut key is published

    // ---- gather the other CTAs' tables
    {
        const uint32_t words = A.tab_stride / 4;
        for (uint32_t t = threadIdx.x; t < (uint32_t)A.Ns * words; t += NT) {
            const int i = t / words;
            const uint32_t owner = (uint32_t)(i % CL);
            if (owner == r) continue;
            uint32_t* dst = reinterpret_cast<uint32_t*>(smem + A.o_tab + (size_t)i * A.tab_stride) + (t - i * words);
            *dst = ld_cluster_u32(map_rank(smem_addr(dst), owner));
        }
    }
    __syncthreads();

    // ---- S4: SC-score counting over this CTA's id range
    count_scores<NT>(A, smem, r);
    const uint32_t id0 = r * (uint32_t)A.cpc * (uint32_t)A.n_ch;
    const uint32_t span = (uint32_t)A.cpc * (uint32_t)A.n_ch;
    const uint32_t valid = id0 >= A.n ? 0u : (uint32_t)min((int64_t)span, A.n - (int64_t)id0);
    const uint32_t* scores = reinterpret_cast<const uint32_t*>(smem + A.o_union);
    const uint32_t nwords = (valid + 3) / 4;
    if (A.dbg_scores)
        for (uint32_t j = threadIdx.x; j < valid; j += NT)
            A.dbg_scores[b * A.n + id0 + j] = (uint8_t)(scores[j >> 2] >> ((j & 3) * 8));

    // ---- S5: cluster-wide score histogram, cut, and candidate hand-off
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + A.o_cnt);  // [0] = valid ids, [s] = #scores >= s
    {
        uint32_t c[NSMAX];
#pragma unroll
        for (int s = 0; s < NSMAX; ++s) c[s] = 0u;
        for (uint32_t w = threadIdx.x; w < nwords; w += NT) {
            const uint32_t v = scores[w];
#pragma unroll
            for (int s = 0; s < NSMAX; ++s) c[s] += __popc(__vcmpgeu4(v, (uint32_t)(s + 1) * 0x01010101u)) >> 3;
        }
#pragma unroll
        for (int s = 0; s < NSMAX; ++s) {
            uint32_t v = c[s];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && v) atomicAdd(&cnt[s + 1], v);
        }
        if (threadIdx.x == 0) cnt[0] = valid;
    }
    cluster_sync();  // #2: every CTA's counts are published
    uint32_t* allc = cnt + (NSMAX + 2);                              // [CL][NSMAX+2]
    uint32_t* sel = reinterpret_cast<uint32_t*>(smem + A.o_misc) + 16;  // theta, n_gt, need_eq, gt_pre, eq_pre
    uint32_t* slot_base = sel + 8;                                    // [CL] remote slot addresses
    for (int t = threadIdx.x; t < CL * (NSMAX + 2); t += NT) {
        const int rr = t / (NSMAX + 2), s = t - rr * (NSMAX + 2);
        allc[t] = ld_cluster_u32(map_rank(smem_addr(cnt + s), (uint32_t)rr));
    }
    for (int t = threadIdx.x; t < CL; t += NT)
        slot_base[t] = map_rank(smem_addr(smem + A.o_slots), (uint32_t)t);
    __syncthreads();
    if (threadIdx.x == 0) {
        int theta = 0;
        for (int s = A.Ns; s >= 1; --s) {
            uint32_t tot = 0;
            for (int rr = 0; rr < CL; ++rr) tot += allc[rr * (NSMAX + 2) + s];
            if (tot >= A.C) {
                theta = s;
                break;
            }
        }
        uint32_t n_gt = 0, gt_pre = 0, eq_pre = 0;
        for (int rr = 0; rr < CL; ++rr) {
            const uint32_t* cr = allc + rr * (NSMAX + 2);
            const uint32_t gt = cr[theta + 1];
            const uint32_t eq = cr[theta] - gt;
            n_gt += gt;
            if (rr < (int)r) {
                gt_pre += gt;
                eq_pre += eq;
            }
        }
        sel[0] = (uint32_t)theta;
        sel[1] = n_gt;
        sel[2] = A.C - n_gt;
        sel[3] = gt_pre;
        sel[4] = eq_pre;
    }
    __syncthreads();
    {
        const uint32_t theta = sel[0], n_gt = sel[1], need_eq = sel[2];
        const uint32_t th4 = theta * 0x01010101u;
        const uint32_t wpw = (nwords + NW - 1) / NW;
        const uint32_t wb = min(nwords, (uint32_t)warp * wpw), we = min(nwords, wb + wpw);
        uint32_t* wtmp = reinterpret_cast<uint32_t*>(smem + A.o_hist);  // [0,NW) gt, [64,64+NW) eq
        // pass 1: per-warp counts
        uint32_t g = 0, e = 0;
        for (uint32_t w = wb + lane; w < we; w += 32) {
            const uint32_t v = scores[w];
            uint32_t em = __vcmpeq4(v, th4);
            if (4 * w + 4 > valid) em &= (1u << (8 * (valid - 4 * w))) - 1u;
            g += __popc(__vcmpgtu4(v, th4)) >> 3;
            e += __popc(em) >> 3;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g += __shfl_xor_sync(0xffffffffu, g, o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        if (lane == 0) {
            wtmp[warp] = g;
            wtmp[64 + warp] = e;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t sg = sel[3], se = sel[4];
            for (int w = 0; w < NW; ++w) {
                const uint32_t tg = wtmp[w], te = wtmp[64 + w];
                wtmp[w] = sg;
                wtmp[64 + w] = se;
                sg += tg;
                se += te;
            }
        }
        __syncthreads();
        // pass 2: hand each selected id to the CTA that re-ranks its position
        uint32_t gb = wtmp[warp], eb = wtmp[64 + warp];
        for (uint32_t w0 = wb; w0 < we; w0 += 32) {
            const uint32_t w = w0 + lane;
            uint32_t gm = 0, em = 0;
            if (w < we) {
                const uint32_t v = scores[w];
                gm = __vcmpgtu4(v, th4);
                em = __vcmpeq4(v, th4);
                if (4 * w + 4 > valid) em &= (1u << (8 * (valid - 4 * w))) - 1u;
            }
            const uint32_t cg = __popc(gm) >> 3, ce = __popc(em) >> 3;
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
            uint32_t pg = gb + ig - cg, pe = eb + ie - ce;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t id = id0 + 4 * w + j;
                uint32_t pos = 0xffffffffu;
                if ((gm >> (8 * j)) & 1u) {
                    pos = pg++;
                } else if ((em >> (8 * j)) & 1u) {
                    if (pe < need_eq) pos = n_gt + pe;
                    ++pe;
                }
                if (pos != 0xffffffffu) {
                    const uint32_t owner = pos / A.per_cta;
                    st_cluster_u32(slot_base[owner] + 4u * (pos - owner * A.per_cta), id);
                    if (A.dbg_cands) A.dbg_cands[b * A.C + pos] = (int32_t)id;
                }
            }
            gb += __shfl_sync(0xffffffffu, ig, 31);
            eb += __shfl_sync(0xffffffffu, ie, 31);
        }
    }
    cluster_sync();  // #3: every candidate slot is filled; scores are dead

    // ---- S6: exact FP32 re-rank of this CTA's share of the candidates
    unsigned long long* topk = reinterpret_cast<unsigned long long*>(smem + A.o_union);
    unsigned long long* sortbuf = topk + A.k_pad;
    const uint32_t* slots = reinterpret_cast<const uint32_t*>(smem + A.o_slots);
    const uint32_t mine = A.C > r * A.per_cta ? min(A.per_cta, A.C - r * A.per_cta) : 0u;
    const float4* q4 = reinterpret_cast<const float4*>(smem + A.o_q);
    const int ld4 = (int)(A.ld / 4);
    uint32_t kc = 0;
    for (uint32_t t0 = 0; t0 < mine; t0 += RTILE) {
        const uint32_t tc = min((uint32_t)RTILE, mine - t0);
        for (uint32_t t = threadIdx.x; t < (uint32_t)A.sortP; t += NT)
            if (t < kc) sortbuf[t] = topk[t]; else if (t >= kc + tc) sortbuf[t] = ~0ull;
        for (uint32_t j = (uint32_t)warp * 4; j < tc; j += NW * 4) {
            int32_t id[4];
            float acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t sv = j + u < tc ? slots[t0 + j + u] : 0xffffffffu;
                id[u] = sv < (uint32_t)A.n ? (int32_t)sv : -1;
                acc[u] = 0.f;
            }
            for (int c = lane; c < ld4; c += 32) {
                const float4 qv = q4[c];
                float4 xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (id[u] >= 0) xv[u] = __ldg(reinterpret_cast<const float4*>(A.X + (int64_t)id[u] * A.ld) + c);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (id[u] >= 0) {
                        float df = __fsub_rn(xv[u].x, qv.x);
                        acc[u] = __fmaf_rn(df, df, acc[u]);
                        df = __fsub_rn(xv[u].y, qv.y);
                        acc[u] = __fmaf_rn(df, df, acc[u]);
                        df = __fsub_rn(xv[u].z, qv.z);
                        acc[u] = __fmaf_rn(df, df, acc[u]);
                        df = __fsub_rn(xv[u].w, qv.w);
                        acc[u] = __fmaf_rn(df, df, acc[u]);
                    }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                float v = acc[u];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (lane == 0 && j + u < tc)
                    sortbuf[kc + j + u] =
                        id[u] >= 0 ? ((unsigned long long)__float_as_uint(v) << 32) | (uint32_t)id[u] : ~0ull;
            }
        }
        __syncthreads();
        block_bitonic_sort<NT>(sortbuf, (int)A.sortP);
        kc = min((uint32_t)A.k, kc + tc);
        for (uint32_t t = threadIdx.x; t < kc; t += NT) topk[t] = sortbuf[t];
        __syncthreads();
    }
    for (uint32_t t = kc + threadIdx.x; t < (uint32_t)A.k; t += NT) topk[t] = ~0ull;
    cluster_sync();  // #4: every local top-k is published

    if (r == 0) {
        const uint32_t tot = (uint32_t)CL * A.k;
        for (uint32_t t = threadIdx.x; t < (uint32_t)A.mergeP; t += NT) {
            unsigned long long v = ~0ull;
            if (t < tot) {
                const uint32_t rr = t / A.k, e = t - rr * A.k;
                v = rr == 0 ? topk[e] : ld_cluster_u64(map_rank(smem_addr(topk + e), rr));
            }
            sortbuf[t] = v;
        }
        __syncthreads();
        block_bitonic_sort<NT>(sortbuf, (int)A.mergeP);
        for (int t = threadIdx.x; t < A.k; t += NT) {
            const unsigned long long v = sortbuf[t];
            const bool pad = v == ~0ull;
            A.out_ids[b * A.k + t] = pad ? -1 : (int32_t)(uint32_t)(v & 0xffffffffu);
            A.out_dist[b * A.k + t] = pad ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(v >> 32));
        }
    }
    cluster_sync();  // #5: remote reads of the published top-k lists are done
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

int make_layout(const DeviceIndex* ix, int CL, int nsmax, uint32_t C, int k, Layout* L)
{
    QArgs& A = L->A;
    memset(&A, 0, sizeof(A));
    A.CL = CL;
    A.cpc = NCH / CL;
    A.k = k;
    A.k_pad = (k + 1) & ~1;
    A.per_cta = (C + CL - 1) / CL;
    const int sk = ix->sqrtK;
    uint64_t o = 0;
    A.o_tab = (uint32_t)o;
    A.tab_stride = align16(16 + 10ull * sk);
    o = align16(o + (uint64_t)ix->Ns * A.tab_stride);
    A.o_q = (uint32_t)o;
    o = align16(o + 4ull * ix->ld);
    A.o_hist = (uint32_t)o;
    o = align16(o + 4ull * (256 + 64));
    A.o_misc = (uint32_t)o;
    o = align16(o + 8ull * 16 + 4ull * (32 + 16));
    A.o_cnt = (uint32_t)o;
    o = align16(o + 4ull * (nsmax + 2) * (CL + 1));
    A.o_seg = (uint32_t)o;
    o = align16(o + 4ull * (2 * MAXSEG + 1));
    A.o_slots = (uint32_t)o;
    o = align16(o + 4ull * A.per_cta);
    A.o_union = (uint32_t)o;
    const uint64_t score_bytes = (uint64_t)A.cpc * ix->n_ch;
    A.score_words = (uint32_t)(score_bytes / 4);
    const uint32_t rt = std::min<uint32_t>(RTILE, std::max<uint32_t>(A.per_cta, 1));
    A.sortP = next_pow2((uint32_t)k + rt);
    A.mergeP = next_pow2((uint32_t)(CL * k));
    const uint64_t keys_bytes = 8ull * (A.k_pad + std::max(A.sortP, A.mergeP));
    o = align16(o + std::max(score_bytes, keys_bytes));
    L->smem = o;
    return SUCO_OK;
}

template <int NT, int NSMAX>
int launch_t(const Layout& L, int64_t nq, cudaStream_t st)
{
    auto kern = suco_query_kernel<NT, NSMAX>;
    SUCO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
    if (L.A.CL > 8) SUCO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(nq * L.A.CL), 1, 1);
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
    SUCO_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, L.A));
    return SUCO_OK;
}

}  // namespace

int launch_query(const DeviceIndex* ix, const float* Q, int64_t nq, const suco_query_params* p, int32_t* ids,
                 float* dist, const suco_query_debug_out* dbg, cudaStream_t st)
{
    if (nq == 0) return SUCO_OK;
    int64_t T = 0, C = 0;
    thresholds(ix->n, p->alpha, p->beta, p->k, &T, &C);
    const int nsmax = ix->Ns <= 8 ? 8 : (ix->Ns <= 16 ? 16 : 32);
    const int NT = p->threads ? p->threads : 1024;
    if (NT != 512 && NT != 1024) return fail(SUCO_EINVAL, "threads must be 0, 512 or 1024 (got %d)", p->threads);
    int dev_smem = 0;
    SUCO_CUDA_TRY(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device));
    Layout L;
    int CL = p->cluster_size;
    if (CL) {
        if (CL != 1 && CL != 2 && CL != 4 && CL != 8 && CL != 16)
            return fail(SUCO_EINVAL, "cluster_size must be 0, 1, 2, 4, 8 or 16 (got %d)", CL);
        make_layout(ix, CL, nsmax, (uint32_t)C, p->k, &L);
        if (L.smem > (size_t)dev_smem)
            return fail(SUCO_EUNSUPPORTED, "cluster_size %d needs %zu bytes of shared memory per CTA (max %d)", CL,
                        L.smem, dev_smem);
    } else {
        for (CL = 1; CL <= 16; CL *= 2) {
            make_layout(ix, CL, nsmax, (uint32_t)C, p->k, &L);
            if (L.smem <= (size_t)dev_smem) break;
        }
        if (CL > 16)
            return fail(SUCO_EUNSUPPORTED,
                        "n=%lld needs more than 16 CTAs of shared memory per query (SC-score array too large)",
                        (long long)ix->n);
    }
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
    A.out_ids = ids;
    A.out_dist = dist;
    if (dbg) {
        A.dbg_teff = dbg->t_eff;
        A.dbg_act = dbg->activated;
        A.dbg_dtab = dbg->dtab;
        A.dbg_scores = dbg->scores;
        A.dbg_cands = dbg->cands;
    }
    if (NT == 1024) {
        if (nsmax == 8) return launch_t<1024, 8>(L, nq, st);
        if (nsmax == 16) return launch_t<1024, 16>(L, nq, st);
        return launch_t<1024, 32>(L, nq, st);
    }
    if (nsmax == 8) return launch_t<512, 8>(L, nq, st);
    if (nsmax == 16) return launch_t<512, 16>(L, nq, st);
    return launch_t<512, 32>(L, nq, st);
}

}  // namespace suco
