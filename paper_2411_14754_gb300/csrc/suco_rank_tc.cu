// Half-subspace centroid distances of a batch of queries on the 5th-generation
// tensor cores (the reduced-precision ranking modes; the paper computes these
// distances directly, Section 4.2, Algorithm 4, in full precision).
//
// For every half-subspace h (length L <= hmax) the block of queries Q_h
// (128 x L) and the codebook C_h (sqrtK x L) are rounded to a narrow type and
//     D[b][h][c] = |q_bh|^2 - 2 <q_bh, c_hc> + |c_hc|^2
// with the inner products from tcgen05.mma (FP32 accumulation in tensor
// memory) and the squared norms of the rounded vectors summed in FP32.
//   BF16: kind::f16, both operands BF16 (round to nearest even).
//   FP8:  kind::f8f6f4, both operands E4M3 codes with one scale per subspace:
//         the centroids use the dataset's scale s_i (its largest |x| over the
//         subspace / 448, the scale of the index's FP8 copy) and each query its
//         own t_bi (largest |q| over the subspace / 448); codes are
//         e4m3(x / scale) (FP32 quotient, round to nearest even, saturating),
//         values code * scale.  The tensor cores sum code products; the
//         epilogue multiplies the sum by s_i * t_bi.
//
// One CTA of 128 threads handles 128 queries and one half-subspace: the
// threads stage both operands in shared memory in the canonical K-major
// layout without swizzle (core matrices of 8 rows x 16 bytes), one thread
// issues the MMAs into a 128-lane x NP-column FP32 accumulator, a commit
// arrives on an mbarrier, and each warp reads its 32 lanes back with
// tcgen05.ld (one query row per thread).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "suco_internal.cuh"

namespace suco {
namespace {

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (tcgen05): start address, leading and stride
// byte offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t instr_desc_bf16(uint32_t m, uint32_t n)
{
    return (1u << 4)            // D format F32
           | (1u << 7)          // A format BF16
           | (1u << 10)         // B format BF16
           | ((n >> 3) << 17)   // N / 8
           | ((m >> 4) << 24);  // M / 16
}

// instruction descriptor of kind::f8f6f4: FP32 accumulator, E4M3 A and B
// (format code 0), both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t instr_desc_e4m3(uint32_t m, uint32_t n)
{
    return (1u << 4)            // D format F32
           | ((n >> 3) << 17)   // N / 8
           | ((m >> 4) << 24);  // M / 16
}

// E4M3 code of x / scale (FP32 quotient, round to nearest even, saturating)
// and the value it stands for, code * scale in FP32
__device__ __forceinline__ uint32_t e4m3_code(float x, float scale, float* value)
{
    const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(__fdiv_rn(x, scale), __NV_SATFINITE, __NV_E4M3);
    const __half_raw h = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
    *value = __fmul_rn(__half2float(*reinterpret_cast<const __half*>(&h)), scale);
    return (uint32_t)c;
}

// one row of a K-major operand: 16 bytes per core-matrix column (8 BF16 or
// 16 E4M3 values), each a 16-byte store; returns the row's squared norm (FP32,
// element order) of the values the codes stand for
// src[k] of the row is base[idx ? idx[off + k] : off + k] (idx: a sampled
// index's column permutation, for query rows)
template <bool FP8>
__device__ __forceinline__ float stage_row(const float* __restrict__ base, const int32_t* __restrict__ idx, int off,
                                           int len, bool valid, float scale, int kcols, char* row_base)
{
    auto src = [&](int k) { return base[idx ? __ldg(idx + off + k) : off + k]; };
    float nrm = 0.f;
    for (int kc = 0; kc < kcols; ++kc) {
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (FP8) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int k = kc * 16 + e;
                float v = 0.f;
                const uint32_t code = (valid && k < len) ? e4m3_code(src(k), scale, &v) : 0u;
                nrm = __fmaf_rn(v, v, nrm);
                w[e >> 2] |= code << (8 * (e & 3));
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                const int k = kc * 8 + e;
                const float x0 = (valid && k < len) ? src(k) : 0.f;
                const float x1 = (valid && k + 1 < len) ? src(k + 1) : 0.f;
                const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
                const float r0 = __bfloat162float(h0), r1 = __bfloat162float(h1);
                nrm = __fmaf_rn(r0, r0, nrm);
                nrm = __fmaf_rn(r1, r1, nrm);
                w[e >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            }
        }
        *reinterpret_cast<uint4*>(row_base + kc * 128) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    return nrm;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// waits at most ~1 s for the phase; false if it gave up
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}

constexpr int TC_M = 128;

// dynamic shared memory: A [128 x KP] and B [NP x KP] elements (2 bytes for
// BF16, 1 for E4M3), |c|^2 [NP] f32, mbarrier (8 B), TMEM address (4 B).
// grid = (query tiles, 2*Ns halves).  col_scale: the dataset's FP8 column
// scales (FP8 only).
template <bool FP8>
__global__ void __launch_bounds__(128, 1)
    centroid_dist_tc_kernel(const float* __restrict__ Q, int64_t nq, int32_t d, int32_t Ns, int32_t sub_s,
                            int32_t sqrtK, int32_t hmax, const float* __restrict__ cent,
                            const float* __restrict__ col_scale, const int32_t* __restrict__ qperm, int32_t KP,
                            int32_t NP, int32_t ncols, float* __restrict__ D, uint32_t* status)
{
    extern __shared__ __align__(128) char smem[];
    constexpr int ESZ = FP8 ? 1 : 2;  // bytes per element
    char* As = smem;
    char* Bs = As + TC_M * KP * ESZ;
    float* cn = reinterpret_cast<float*>(Bs + NP * KP * ESZ);
    uint64_t* bar = reinterpret_cast<uint64_t*>(cn + NP);
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * TC_M;
    const int ih = (int)blockIdx.y;
    const int kcols = KP * ESZ / 16;  // core-matrix columns along K

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(taddr_s)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    int32_t off, len;
    half_dims(d, Ns, sub_s, ih >> 1, ih & 1, &off, &len);
    const int i = ih >> 1, soff = i * sub_s, slen = (i == Ns - 1) ? d - (Ns - 1) * sub_s : sub_s;
    // A: row m = query b0 + m; core-matrix column kc of a row is one 16-byte
    // store at ((m/8)*kcols + kc)*128 + (m%8)*16
    const int m = tid;
    const int64_t b = b0 + m;
    float t = 1.f;  // the query's scale over subspace i (FP8)
    if (FP8 && b < nq) {
        float mx = 0.f;
        for (int j = 0; j < slen; ++j) mx = fmaxf(mx, fabsf(query_col(Q + b * d, qperm, soff + j)));
        t = mx > 0.f ? __fdiv_rn(mx, 448.f) : 1.f;
    }
    const float qn = stage_row<FP8>(Q + (b < nq ? b : 0) * d, qperm, off, len, b < nq, t, kcols,
                                    As + ((m >> 3) * kcols) * 128 + (m & 7) * 16);
    // B: centroid c of this half, same layout with c in place of m
    const float s = FP8 ? col_scale[soff] : 1.f;
    for (int c = tid; c < NP; c += TC_M)
        cn[c] = stage_row<FP8>(cent + ((int64_t)ih * sqrtK + (c < sqrtK ? c : 0)) * hmax, nullptr, 0, len, c < sqrtK, s,
                               kcols, Bs + ((c >> 3) * kcols) * 128 + (c & 7) * 16);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr_s;
    // byte offsets between core matrices: along K (the descriptor's leading
    // byte offset) and along M or N (its stride byte offset)
    const uint32_t k_step = 128u, mn_step = (uint32_t)kcols * 128u;
    if (tid == 0) {
        // one MMA consumes 32 bytes along K (16 BF16 or 32 E4M3 values): two core-matrix columns
        const uint32_t idesc = FP8 ? instr_desc_e4m3(TC_M, (uint32_t)NP) : instr_desc_bf16(TC_M, (uint32_t)NP);
        for (int kk = 0; kk < kcols / 2; ++kk) {
            const uint64_t ad = smem_desc(sa(As) + (uint32_t)kk * 2u * k_step, k_step, mn_step);
            const uint64_t bd = smem_desc(sa(Bs) + (uint32_t)kk * 2u * k_step, k_step, mn_step);
            const uint32_t acc = kk > 0 ? 1u : 0u;
            if (FP8)
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            else
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(bar))
                     : "memory");
    }
    const bool ok = mbar_wait_bounded(sa(bar), 0u);
    if (!ok && status) {  // the word is in mapped host memory: a plain store, made visible to the host
        *reinterpret_cast<volatile uint32_t*>(status) = SUCO_STATUS_WAIT_TIMEOUT;
        __threadfence_system();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w reads lanes 32w..32w+31 (query rows), 16 columns at a time
    {
        const float m2st = -2.f * __fmul_rn(s, t);  // -2 * s_i * t_bi (FP8); -2 (BF16)
        for (int c0 = 0; c0 < NP; c0 += 16) {
            uint32_t r[16];
            const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(addr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (b < nq && ok)
                for (int j = 0; j < 16; ++j) {
                    const int c = c0 + j;
                    if (c < sqrtK) {
                        const float dot = __uint_as_float(r[j]);
                        D[(b * 2 * Ns + ih) * sqrtK + c] = __fadd_rn(__fmaf_rn(m2st, dot, qn), cn[c]);
                    }
                }
        }
    }
    // an MMA still in flight after a wait that gave up: one more bounded wait
    if (!ok) mbar_wait_bounded(sa(bar), 0u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

int rank_tc_tables(const DeviceIndex* ix, const float* Q, int64_t nq, float* D, bool fp8, cudaStream_t st)
{
    if (nq == 0) return SUCO_OK;
    const int esz = fp8 ? 1 : 2;
    const int kgran = 32 / esz;  // K elements per MMA
    const int KP = (ix->hmax + kgran - 1) / kgran * kgran;
    const int NP = (ix->sqrtK + 15) & ~15;
    int ncols = 32;
    while (ncols < NP) ncols *= 2;
    const size_t smem = (size_t)(TC_M + NP) * KP * esz + (size_t)NP * 4 + 16;
    // at least 100 KB of shared memory per CTA keeps at most two CTAs (and
    // 2 x ncols <= 512 TMEM columns) on an SM
    const size_t smem_req = std::max<size_t>(smem, 100 * 1024);
    if (fault_fires(SUCO_FAULT_WAIT_TIMEOUT)) {
        // as if the launch's bounded wait had given up: the status word is set
        // and the tables are not written
        *ix->status_host = SUCO_STATUS_WAIT_TIMEOUT;
        return SUCO_OK;
    }
    auto kern = fp8 ? centroid_dist_tc_kernel<true> : centroid_dist_tc_kernel<false>;
    SUCO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req));
    const int64_t tiles = (nq + TC_M - 1) / TC_M;
    kern<<<dim3((unsigned)tiles, (unsigned)(2 * ix->Ns)), TC_M, smem_req, st>>>(
        Q, nq, ix->d, ix->Ns, ix->sub_s, ix->sqrtK, ix->hmax, ix->cent, ix->s8col, ix->dperm, KP, NP, ncols, D,
        ix->status_dev);
    SUCO_LAUNCH_CHECK("centroid_dist_tc_kernel");
    return SUCO_OK;
}

}  // namespace suco
