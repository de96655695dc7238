// Reduced-precision copies of the dataset for the coarse re-rank pass (no
// counterpart in the paper): the BF16 copy holds every value of D rounded to
// nearest even, rows padded with zeros to a multiple of 8 values (16 bytes).
// The same call reserves the workspace of the BF16 tensor-core ranking: the
// centroid-distance tables of up to RANK_CHUNK queries.
#include <cuda_bf16.h>

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

}  // namespace
}  // namespace suco

using namespace suco;

extern "C" int suco_add_reduced_copies(suco_index* index, int32_t mask, void* stream)
{
    clear_error();
    if (!index) return fail(SUCO_EINVAL, "index is NULL");
    if (mask & ~(SUCO_COPY_BF16 | SUCO_COPY_RANK_BF16)) return fail(SUCO_EINVAL, "unknown copy bits 0x%x", mask);
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
        SUCO_CUDA_TRY(cudaGetLastError());
        SUCO_CUDA_TRY(cudaStreamSynchronize(st));
        ix->Xh = b.as<uint16_t>();
        ix->ldh = ldh;
        ix->bytes += (int64_t)b.bytes;
        b.release();
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
