// Reduced-precision copies of the dataset for the coarse re-rank pass (no
// counterpart in the paper): the BF16 copy holds every value of D rounded to
// nearest even, rows padded with zeros to a multiple of 8 values (16 bytes).
// The same call reserves the workspace of the BF16 tensor-core ranking: the
// centroid-distance tables of up to RANK_CHUNK queries.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstring>
#include <vector>

#include "suco_internal.cuh"

namespace suco {
namespace {

// one thread per 8 output values (16 bytes) of a row
__global__ void to_bf16_kernel(const float* __restrict__ X, int64_t ld, int64_t n, int32_t d,
                               uint16_t* __restrict__ Xh, int64_t ldh)
{
    const int64_t chunks = ldh / 8;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * chunks;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / chunks;
        const int c = (int)(t - row * chunks);
        uint16_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = 8 * c + j;
            const float x = col < d ? X[row * ld + col] : 0.f;
            v[j] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
        }
        uint4 w;
        w.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
        w.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
        w.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
        w.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
        reinterpret_cast<uint4*>(Xh + row * ldh)[c] = w;
    }
}

// largest |x| of every subspace (grid.y = subspace), as FP32 bits
__global__ void subspace_maxabs_kernel(const float* __restrict__ X, int64_t ld, int64_t n, int32_t d, int32_t Ns,
                                       int32_t sub_s, unsigned* __restrict__ out)
{
    const int i = blockIdx.y;
    const int off = i * sub_s, len = (i == Ns - 1) ? d - (Ns - 1) * sub_s : sub_s;
    float m = 0.f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < len; ++j) m = fmaxf(m, fabsf(X[p * ld + off + j]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + i, __float_as_uint(m));
}

// one thread per 16 output bytes of a row: e4m3(x / scale of the column),
// round to nearest even with saturation to +-448
__global__ void to_fp8_kernel(const float* __restrict__ X, int64_t ld, int64_t n, int32_t d,
                              const float* __restrict__ col_scale, uint8_t* __restrict__ X8, int64_t ld8)
{
    const int64_t chunks = ld8 / 16;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * chunks;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / chunks;
        const int c = (int)(t - row * chunks);
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = 16 * c + j;
            uint32_t code = 0u;
            if (col < d) {
                const float q = __fdiv_rn(X[row * ld + col], col_scale[col]);
                code = (uint32_t)__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
            }
            w[j >> 2] |= code << (8 * (j & 3));
        }
        reinterpret_cast<uint4*>(X8 + row * ld8)[c] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

}  // namespace
}  // namespace suco

using namespace suco;

extern "C" int suco_add_reduced_copies(suco_index* index, int32_t mask, void* stream)
{
    clear_error();
    if (!index) return fail(SUCO_EINVAL, "index is NULL");
    if (mask & ~(SUCO_COPY_BF16 | SUCO_COPY_RANK_BF16 | SUCO_COPY_FP8))
        return fail(SUCO_EINVAL, "unknown copy bits 0x%x", mask);
    DeviceIndex* ix = &index->ix;
    cudaStream_t st = (cudaStream_t)stream;
    if ((mask & SUCO_COPY_BF16) && !ix->Xh) {
        const int64_t ldh = (ix->d + 7) & ~int64_t(7);
        DevBuf b;
        int rc = b.alloc((size_t)ix->n * ldh * 2);
        if (rc) return rc;
        const int64_t work = ix->n * (ldh / 8);
        const int grid = (int)std::min<int64_t>((work + 255) / 256, 152 * 16);
        to_bf16_kernel<<<grid, 256, 0, st>>>(ix->X, ix->ld, ix->n, ix->d, b.as<uint16_t>(), ldh);
        SUCO_LAUNCH_CHECK("to_bf16_kernel");
        SUCO_CUDA_TRY(cudaStreamSynchronize(st));
        ix->Xh = b.as<uint16_t>();
        ix->ldh = ldh;
        ix->bytes += (int64_t)b.bytes;
        b.release();
    }
    if ((mask & SUCO_COPY_FP8) && !ix->X8) {
        const int64_t ld8 = (ix->d + 15) & ~int64_t(15);
        DevBuf mx, cs, b;
        int rc = mx.alloc((size_t)ix->Ns * 4);
        if (!rc) rc = cs.alloc((size_t)ld8 * 4);
        if (!rc) rc = b.alloc((size_t)ix->n * ld8);
        if (rc) return rc;
        SUCO_CUDA_TRY(cudaMemsetAsync(mx.p, 0, (size_t)ix->Ns * 4, st));
        const int gx = (int)std::min<int64_t>((ix->n + 255) / 256, 1024);
        subspace_maxabs_kernel<<<dim3(gx, ix->Ns), 256, 0, st>>>(ix->X, ix->ld, ix->n, ix->d, ix->Ns, ix->sub_s,
                                                                 mx.as<unsigned>());
        SUCO_LAUNCH_CHECK("subspace_maxabs_kernel");
        std::vector<unsigned> mbits(ix->Ns);
        SUCO_CUDA_TRY(cudaMemcpyAsync(mbits.data(), mx.p, (size_t)ix->Ns * 4, cudaMemcpyDeviceToHost, st));
        SUCO_CUDA_TRY(cudaStreamSynchronize(st));
        // scale of subspace i: max|x| / 448 rounded to FP32 (1 for an all-zero subspace)
        std::vector<float> col((size_t)ld8, 0.f);
        for (int i = 0; i < ix->Ns; ++i) {
            float m;
            memcpy(&m, &mbits[i], 4);
            const volatile float q448 = 448.0f;
            const float sc = m > 0.f ? m / q448 : 1.0f;
            const int off = i * ix->sub_s, len = (i == ix->Ns - 1) ? ix->d - (ix->Ns - 1) * ix->sub_s : ix->sub_s;
            for (int j = 0; j < len; ++j) col[off + j] = sc;
        }
        SUCO_CUDA_TRY(cudaMemcpyAsync(cs.p, col.data(), (size_t)ld8 * 4, cudaMemcpyHostToDevice, st));
        const int64_t work = ix->n * (ld8 / 16);
        const int grid = (int)std::min<int64_t>((work + 255) / 256, 152 * 16);
        to_fp8_kernel<<<grid, 256, 0, st>>>(ix->X, ix->ld, ix->n, ix->d, cs.as<float>(), b.as<uint8_t>(), ld8);
        SUCO_LAUNCH_CHECK("to_fp8_kernel");
        SUCO_CUDA_TRY(cudaStreamSynchronize(st));
        ix->X8 = b.as<uint8_t>();
        ix->s8col = cs.as<float>();
        ix->ld8 = ld8;
        ix->bytes += (int64_t)(b.bytes + cs.bytes);
        b.release();
        cs.release();
    }
    if ((mask & SUCO_COPY_RANK_BF16) && !ix->rank_ws) {
        DevBuf b;
        int rc = b.alloc((size_t)RANK_CHUNK * ix->Ns * 2 * ix->sqrtK * 4);
        if (rc) return rc;
        ix->rank_ws = b.as<float>();
        ix->bytes += (int64_t)b.bytes;
        b.release();
    }
    return SUCO_OK;
}
