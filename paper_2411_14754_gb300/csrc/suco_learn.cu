// Learned per-query collision and re-rank ratios (no counterpart in the paper;
// its conclusion names learning as future work).
//
// A small MLP reads per-query features taken from the same centroid distances
// that drive the cell ranking (Section 4.2, Algorithm 4's half-subspace
// distances, in the index's metric): for each subspace i the smallest distance to a
// first-half centroid, the smallest to a second-half centroid, and
// log(1 + size of the IMI cell formed by the two nearest centroids).  It
// predicts (log alpha, log beta); the query path then uses them per query.
//
// Network: x (F = 3*Ns) -> standardise -> z1 = xn W1 + b1 (H) -> h = GELU(z1)
// -> y = h W2 + b2 (2).  W1, W2 are BF16; every sum is FP32.  GELU is the erf
// form 0.5 z (1 + erf(z / sqrt 2)).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "suco_internal.cuh"

namespace suco {
namespace {

constexpr float kInvSqrt2 = 0.70710678118654752440f;
constexpr float kInvSqrt2Pi = 0.39894228040143267794f;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * kInvSqrt2)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    // d/dz [z * Phi(z)] = Phi(z) + z * phi(z)
    return 0.5f * (1.0f + erff(z * kInvSqrt2)) + z * kInvSqrt2Pi * expf(-0.5f * z * z);
}

__device__ __forceinline__ float bf(const uint16_t* p, size_t i)
{
    return __bfloat162float(__ushort_as_bfloat16(p[i]));
}

// Features of one query (block per query).  dist: [Ns][2][sqrtK] in shared memory.
__global__ void features_kernel(const float* __restrict__ cent, const uint32_t* __restrict__ cell_off, int32_t d,
                                int32_t Ns, int32_t sub_s, int32_t sqrtK, int32_t hmax, int64_t K,
                                const float* __restrict__ Q, int64_t nq, float* __restrict__ feats,
                                const int32_t* __restrict__ qperm, int metric)
{
    extern __shared__ float sh[];
    float* qs = sh;              // [d]
    float* dist = sh + d;        // [Ns][2][sqrtK]
    const int64_t b = blockIdx.x;
    for (int j = threadIdx.x; j < d; j += blockDim.x) qs[j] = query_col(Q + b * d, qperm, j);
    __syncthreads();
    const int npair = Ns * 2 * sqrtK;
    for (int t = threadIdx.x; t < npair; t += blockDim.x) {
        const int ih = t / sqrtK, a = t - ih * sqrtK;
        int32_t off, len;
        half_dims(d, Ns, sub_s, ih >> 1, ih & 1, &off, &len);
        const float* c = cent + ((int64_t)ih * sqrtK + a) * hmax;
        float acc = 0.f;
        for (int j = 0; j < len; ++j) {
            const float df = __fsub_rn(qs[off + j], __ldg(c + j));
            acc = metric == SUCO_METRIC_L1 ? __fadd_rn(acc, fabsf(df)) : __fmaf_rn(df, df, acc);
        }
        dist[t] = acc;
    }
    __syncthreads();
    // one warp per (subspace, half): minimum and its lowest index
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ int argm[64];
    for (int ih = warp; ih < 2 * Ns; ih += nw) {
        float best = INFINITY;
        int bi = 0x7fffffff;
        for (int a = lane; a < sqrtK; a += 32) {
            const float v = dist[ih * sqrtK + a];
            if (v < best || (v == best && a < bi)) {
                best = v;
                bi = a;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov < best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            feats[b * 3 * Ns + ih] = best;
            argm[ih] = bi;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
        const int64_t cell = (int64_t)argm[2 * i] * sqrtK + argm[2 * i + 1];
        const uint32_t* co = cell_off + (int64_t)i * (K + 1);
        feats[b * 3 * Ns + 2 * Ns + i] = log1pf((float)(co[cell + 1] - co[cell]));
    }
}

struct MlpDev {
    int32_t F, H;
    const uint16_t* w1;
    const float* b1;
    const uint16_t* w2;
    const float* b2;
    const float* mean;
    const float* stdv;
};

// Forward pass, one warp per sample; lane l owns hidden units l, l+32, ...
// (H <= 512).  Writes z1, h (nullable) and y.
__device__ __forceinline__ void mlp_warp_forward(const MlpDev& M, const float* x, float* z1_out, float* h_out,
                                                 float y[2], float* xn_sh)
{
    const int lane = threadIdx.x & 31;
    for (int f = lane; f < M.F; f += 32) xn_sh[f] = (x[f] - M.mean[f]) / M.stdv[f];
    __syncwarp();
    float y0 = 0.f, y1 = 0.f;
    for (int hh = lane; hh < M.H; hh += 32) {
        float z = M.b1[hh];
        for (int f = 0; f < M.F; ++f) z = __fmaf_rn(xn_sh[f], bf(M.w1, (size_t)f * M.H + hh), z);
        const float a = gelu(z);
        if (z1_out) z1_out[hh] = z;
        if (h_out) h_out[hh] = a;
        y0 = __fmaf_rn(a, bf(M.w2, (size_t)hh * 2), y0);
        y1 = __fmaf_rn(a, bf(M.w2, (size_t)hh * 2 + 1), y1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        y0 += __shfl_xor_sync(0xffffffffu, y0, o);
        y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    }
    y[0] = y0 + M.b2[0];
    y[1] = y1 + M.b2[1];
    __syncwarp();
}

__global__ void mlp_forward_kernel(MlpDev M, const float* __restrict__ X, int64_t B, float* __restrict__ z1,
                                   float* __restrict__ h, float* __restrict__ y)
{
    extern __shared__ float xn[];  // [warps][F]
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t s = (int64_t)blockIdx.x * nw + warp;
    if (s >= B) return;
    float out[2];
    mlp_warp_forward(M, X + s * M.F, z1 ? z1 + s * M.H : nullptr, h ? h + s * M.H : nullptr, out, xn + warp * M.F);
    if ((threadIdx.x & 31) == 0) {
        y[s * 2] = out[0];
        y[s * 2 + 1] = out[1];
    }
}

// dy = d(loss)/dy for loss = mean over samples and outputs of (y - t)^2;
// dz1 = (dy . W2^T) * GELU'(z1); loss sum into *loss.
__global__ void mlp_backward_z_kernel(MlpDev M, const float* __restrict__ y, const float* __restrict__ t, int64_t B,
                                      const float* __restrict__ z1, float* __restrict__ dy, float* __restrict__ dz1,
                                      float* __restrict__ loss)
{
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * nw + warp;
    if (s >= B) return;
    const float e0 = y[s * 2] - t[s * 2], e1 = y[s * 2 + 1] - t[s * 2 + 1];
    const float scale = 2.0f / (2.0f * (float)B);
    const float g0 = scale * e0, g1 = scale * e1;
    if (lane == 0) {
        dy[s * 2] = g0;
        dy[s * 2 + 1] = g1;
        atomicAdd(loss, (e0 * e0 + e1 * e1) / (2.0f * (float)B));
    }
    for (int hh = lane; hh < M.H; hh += 32) {
        const float dh = __fmaf_rn(g0, bf(M.w2, (size_t)hh * 2), g1 * bf(M.w2, (size_t)hh * 2 + 1));
        dz1[s * M.H + hh] = dh * gelu_grad(z1[s * M.H + hh]);
    }
}

// dW1[f][h] = sum_s xn[s][f] dz1[s][h]; row f = F is db1.  One thread per entry,
// samples summed in order (deterministic).
__global__ void mlp_backward_w1_kernel(MlpDev M, const float* __restrict__ X, int64_t B,
                                       const float* __restrict__ dz1, float* __restrict__ dw1,
                                       float* __restrict__ db1)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)(M.F + 1) * M.H) return;
    const int f = (int)(e / M.H), hh = (int)(e % M.H);
    float acc = 0.f;
    if (f < M.F) {
        const float mu = M.mean[f], sd = M.stdv[f];
        for (int64_t s = 0; s < B; ++s) acc = __fmaf_rn((X[s * M.F + f] - mu) / sd, dz1[s * M.H + hh], acc);
        dw1[(size_t)f * M.H + hh] = acc;
    } else {
        for (int64_t s = 0; s < B; ++s) acc += dz1[s * M.H + hh];
        db1[hh] = acc;
    }
}

// dW2[h][o] = sum_s h[s][h] dy[s][o]; db2[o] = sum_s dy[s][o].
__global__ void mlp_backward_w2_kernel(MlpDev M, const float* __restrict__ h, const float* __restrict__ dy, int64_t B,
                                       float* __restrict__ dw2, float* __restrict__ db2)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (M.H + 1) * 2) return;
    const int hh = e / 2, o = e % 2;
    float acc = 0.f;
    if (hh < M.H)
        for (int64_t s = 0; s < B; ++s) acc = __fmaf_rn(h[s * M.H + hh], dy[s * 2 + o], acc);
    else
        for (int64_t s = 0; s < B; ++s) acc += dy[s * 2 + o];
    if (hh < M.H) dw2[hh * 2 + o] = acc; else db2[o] = acc;
}

// AdamW (decoupled weight decay) on FP32 master values; optional BF16 copy.
__global__ void adamw_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps, float wd,
                             float bc1, float bc2, uint16_t* __restrict__ bf16_copy)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / bc1) / (sqrtf(vi / bc2) + eps);
    const float pi = p[i] - lr * (upd + wd * p[i]);
    p[i] = pi;
    if (bf16_copy) bf16_copy[i] = __bfloat16_as_ushort(__float2bfloat16_rn(pi));
}

// Features, then the MLP, then the per-query ratios (block per query; warp 0
// runs the network).  Out-of-range or non-finite outputs fall back to the
// fixed ratios.
__global__ void predict_kernel(MlpDev M, const float* __restrict__ cent, const uint32_t* __restrict__ cell_off,
                               int32_t d, int32_t Ns, int32_t sub_s, int32_t sqrtK, int32_t hmax, int64_t K,
                               const float* __restrict__ Q, int64_t nq, float off0, float off1, float la_lo,
                               float la_hi, float lb_lo, float lb_hi, float fb_alpha, float fb_beta,
                               float* __restrict__ alpha, float* __restrict__ beta, float* __restrict__ feats_scratch,
                               const int32_t* __restrict__ qperm, int metric)
{
    // the features of this query land in feats_scratch[b] first
    extern __shared__ float sh[];
    float* qs = sh;
    float* dist = sh + d;
    float* xn = dist + Ns * 2 * sqrtK;   // [F]
    float* fx = xn + 3 * Ns;             // [F]
    const int64_t b = blockIdx.x;
    for (int j = threadIdx.x; j < d; j += blockDim.x) qs[j] = query_col(Q + b * d, qperm, j);
    __syncthreads();
    const int npair = Ns * 2 * sqrtK;
    for (int t = threadIdx.x; t < npair; t += blockDim.x) {
        const int ih = t / sqrtK, a = t - ih * sqrtK;
        int32_t off, len;
        half_dims(d, Ns, sub_s, ih >> 1, ih & 1, &off, &len);
        const float* c = cent + ((int64_t)ih * sqrtK + a) * hmax;
        float acc = 0.f;
        for (int j = 0; j < len; ++j) {
            const float df = __fsub_rn(qs[off + j], __ldg(c + j));
            acc = metric == SUCO_METRIC_L1 ? __fadd_rn(acc, fabsf(df)) : __fmaf_rn(df, df, acc);
        }
        dist[t] = acc;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ int argm[64];
    for (int ih = warp; ih < 2 * Ns; ih += nw) {
        float best = INFINITY;
        int bi = 0x7fffffff;
        for (int a = lane; a < sqrtK; a += 32) {
            const float v = dist[ih * sqrtK + a];
            if (v < best || (v == best && a < bi)) {
                best = v;
                bi = a;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov < best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            fx[ih] = best;
            argm[ih] = bi;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
        const int64_t cell = (int64_t)argm[2 * i] * sqrtK + argm[2 * i + 1];
        const uint32_t* co = cell_off + (int64_t)i * (K + 1);
        fx[2 * Ns + i] = log1pf((float)(co[cell + 1] - co[cell]));
    }
    __syncthreads();
    if (feats_scratch)
        for (int f = threadIdx.x; f < 3 * Ns; f += blockDim.x) feats_scratch[b * 3 * Ns + f] = fx[f];
    if (warp == 0) {
        float y[2];
        mlp_warp_forward(M, fx, nullptr, nullptr, y, xn);
        if (lane == 0) {
            const float la = y[0] + off0, lb = y[1] + off1;
            const bool ok = isfinite(la) && isfinite(lb);
            alpha[b] = ok ? expf(fminf(fmaxf(la, la_lo), la_hi)) : fb_alpha;
            beta[b] = ok ? expf(fminf(fmaxf(lb, lb_lo), lb_hi)) : fb_beta;
        }
    }
}

int grid1(int64_t work, int threads)
{
    const int64_t g = (work + threads - 1) / threads;
    return (int)(g < 1 ? 1 : g);
}

int check_mlp(const suco_mlp* m, MlpDev* M)
{
    if (!m) return fail(SUCO_EINVAL, "model is NULL");
    if (m->in_dim < 1 || m->in_dim > 1024 || m->hidden < 1 || m->hidden > 4096 || m->out_dim != 2 ||
        m->reserved0 != 0)
        return fail(SUCO_EINVAL, "model sizes: 1 <= in_dim <= 1024, 1 <= hidden <= 4096, out_dim == 2");
    if (!m->w1 || !m->b1 || !m->w2 || !m->b2 || !m->feat_mean || !m->feat_std)
        return fail(SUCO_EINVAL, "model pointers must not be NULL");
    M->F = m->in_dim;
    M->H = m->hidden;
    M->w1 = m->w1;
    M->b1 = m->b1;
    M->w2 = m->w2;
    M->b2 = m->b2;
    M->mean = m->feat_mean;
    M->stdv = m->feat_std;
    return SUCO_OK;
}

}  // namespace
}  // namespace suco

using namespace suco;

extern "C" {

int suco_query_features(const suco_index* index, const float* queries, int64_t nq, float* feats, void* stream)
{
    clear_error();
    if (!index || (nq > 0 && (!queries || !feats))) return fail(SUCO_EINVAL, "index, queries, feats must not be NULL");
    if (nq == 0) return SUCO_OK;
    const DeviceIndex& ix = index->ix;
    if (ix.Ns > 32) return fail(SUCO_EUNSUPPORTED, "features need Ns <= 32");
    const size_t smem = 4ull * (ix.d + (size_t)ix.Ns * 2 * ix.sqrtK);
    if (smem > 200 * 1024) return fail(SUCO_EUNSUPPORTED, "feature tables of %zu bytes exceed shared memory", smem);
    SUCO_CUDA_TRY(cudaFuncSetAttribute(features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    features_kernel<<<(unsigned)nq, 128, smem, (cudaStream_t)stream>>>(ix.cent, ix.cell_off, ix.d, ix.Ns, ix.sub_s,
                                                                      ix.sqrtK, ix.hmax, ix.K, queries, nq, feats,
                                                                      ix.dperm, ix.metric);
    SUCO_LAUNCH_CHECK("features_kernel");
    return SUCO_OK;
}

int suco_mlp_predict(const suco_index* index, const suco_mlp* model, const float* queries, int64_t nq, float* alpha,
                     float* beta, void* stream)
{
    clear_error();
    if (!index || (nq > 0 && (!queries || !alpha || !beta)))
        return fail(SUCO_EINVAL, "index, queries, alpha, beta must not be NULL");
    MlpDev M;
    int rc = check_mlp(model, &M);
    if (rc) return rc;
    if (nq == 0) return SUCO_OK;
    const DeviceIndex& ix = index->ix;
    if (M.F != 3 * ix.Ns) return fail(SUCO_EINVAL, "model in_dim %d != 3*Ns = %d", M.F, 3 * ix.Ns);
    if (ix.Ns > 32) return fail(SUCO_EUNSUPPORTED, "features need Ns <= 32");
    const size_t smem = 4ull * (ix.d + (size_t)ix.Ns * 2 * ix.sqrtK + 6ull * ix.Ns);
    if (smem > 200 * 1024) return fail(SUCO_EUNSUPPORTED, "feature tables of %zu bytes exceed shared memory", smem);
    SUCO_CUDA_TRY(cudaFuncSetAttribute(predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    predict_kernel<<<(unsigned)nq, 128, smem, (cudaStream_t)stream>>>(
        M, ix.cent, ix.cell_off, ix.d, ix.Ns, ix.sub_s, ix.sqrtK, ix.hmax, ix.K, queries, nq, model->out_offset[0],
        model->out_offset[1], model->log_alpha_min, model->log_alpha_max, model->log_beta_min, model->log_beta_max,
        model->fallback_alpha, model->fallback_beta, alpha, beta, nullptr, ix.dperm, ix.metric);
    SUCO_LAUNCH_CHECK("predict_kernel");
    return SUCO_OK;
}

int suco_mlp_forward(const suco_mlp* model, const float* x, int64_t B, float* z1, float* h, float* y, void* stream)
{
    clear_error();
    MlpDev M;
    int rc = check_mlp(model, &M);
    if (rc) return rc;
    if (B < 0 || (B > 0 && (!x || !y))) return fail(SUCO_EINVAL, "x and y must not be NULL");
    if (B == 0) return SUCO_OK;
    const int warps = 8;
    const size_t smem = 4ull * warps * M.F;
    mlp_forward_kernel<<<(unsigned)((B + warps - 1) / warps), 32 * warps, smem, (cudaStream_t)stream>>>(M, x, B, z1, h,
                                                                                                        y);
    SUCO_LAUNCH_CHECK("mlp_forward_kernel");
    return SUCO_OK;
}

int suco_mlp_backward(const suco_mlp* model, const float* x, int64_t B, const float* z1, const float* h,
                      const float* y, const float* target, float* dz1, float* dy, float* dw1, float* db1, float* dw2,
                      float* db2, float* loss, void* stream)
{
    clear_error();
    MlpDev M;
    int rc = check_mlp(model, &M);
    if (rc) return rc;
    if (B < 1 || !x || !z1 || !h || !y || !target || !dz1 || !dy || !dw1 || !db1 || !dw2 || !db2 || !loss)
        return fail(SUCO_EINVAL, "backward needs B >= 1 and every buffer");
    cudaStream_t st = (cudaStream_t)stream;
    SUCO_CUDA_TRY(cudaMemsetAsync(loss, 0, 4, st));
    const int warps = 8;
    mlp_backward_z_kernel<<<(unsigned)((B + warps - 1) / warps), 32 * warps, 0, st>>>(M, y, target, B, z1, dy, dz1,
                                                                                       loss);
    SUCO_LAUNCH_CHECK("mlp_backward_z_kernel");
    mlp_backward_w1_kernel<<<grid1((int64_t)(M.F + 1) * M.H, 128), 128, 0, st>>>(M, x, B, dz1, dw1, db1);
    SUCO_LAUNCH_CHECK("mlp_backward_w1_kernel");
    mlp_backward_w2_kernel<<<grid1((M.H + 1) * 2, 128), 128, 0, st>>>(M, h, dy, B, dw2, db2);
    SUCO_LAUNCH_CHECK("mlp_backward_w2_kernel");
    return SUCO_OK;
}

int suco_adamw_step(float* param, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                    float beta2, float eps, float weight_decay, int32_t step, uint16_t* bf16_copy, void* stream)
{
    clear_error();
    if (!param || !grad || !m || !v || count < 0 || step < 1) return fail(SUCO_EINVAL, "bad AdamW arguments");
    if (count == 0) return SUCO_OK;
    const float bc1 = 1.0f - powf(beta1, (float)step), bc2 = 1.0f - powf(beta2, (float)step);
    adamw_kernel<<<grid1(count, 256), 256, 0, (cudaStream_t)stream>>>(param, grad, m, v, count, lr, beta1, beta2, eps,
                                                                      weight_decay, bc1, bc2, bf16_copy);
    SUCO_LAUNCH_CHECK("adamw_kernel");
    return SUCO_OK;
}

}  // extern "C"
