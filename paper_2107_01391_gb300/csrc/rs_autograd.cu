// rs_autograd.cu -- rs_scatter_rows: the backward of a row-wise sort.
//
// Sorting a row is a permutation, so its Jacobian is a permutation matrix:
// d sorted[j] / d x[perm[j]] = 1 and every other entry is 0.  The gradient of
// the input is therefore the upstream gradient scattered back through the
// permutation: grad_x[r, perm[r, j]] = grad_sorted[r, j].  (The paper has no
// gradient; this is the differentiable form of its output step.)

#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/rs.h"
#include "rs_sort_impl.cuh"

namespace rs {
namespace {

template <typename T>
__global__ void __launch_bounds__(BLOCK) scatter_rows_kernel(const T* __restrict__ src,
                                                             const int64_t* __restrict__ perm,
                                                             uint64_t rows, uint64_t cols,
                                                             T* __restrict__ dst,
                                                             uint32_t* status) {
    const uint64_t total = rows * cols;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * BLOCK) {
        const int64_t p = __ldcs(&perm[i]);
        const uint64_t r = i / cols;
        if (p < 0 || (uint64_t)p >= cols) {
            bad = true;  // not a permutation of the row: skip the element
            continue;
        }
        dst[r * cols + (uint64_t)p] = __ldcs(&src[i]);
    }
    if (bad) atomicOr(status, STATUS_RANGE);
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" rs_status rs_scatter_rows(rs_ctx* ctx, const void* src, const int64_t* perm,
                                     size_t rows, size_t cols, size_t elem_bytes, void* dst,
                                     rs_stream_t stream) {
    if (!ctx || (elem_bytes != 4 && elem_bytes != 8)) return RS_ERR_INVALID;
    const size_t n = rows * cols;
    if (cols && rows > RS_MAX_N / cols) return RS_ERR_INVALID;
    if (n == 0) return RS_OK;
    if (!src || !perm || !dst || (reinterpret_cast<uintptr_t>(src) % elem_bytes) ||
        (reinterpret_cast<uintptr_t>(dst) % elem_bytes) || (reinterpret_cast<uintptr_t>(perm) % 8))
        return RS_ERR_INVALID;
    if (src == dst) return RS_ERR_INVALID;  // a scatter cannot run in place
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return RS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = (int)std::max<size_t>(
        1, std::min<size_t>((n + BLOCK * 4 - 1) / (BLOCK * 4), (size_t)sm_count(ctx->device) * 8));
    {
        LaunchTimer lt(ctx, KC_SEG, st);
        if (elem_bytes == 4)
            scatter_rows_kernel<uint32_t><<<grid, BLOCK, 0, st>>>(
                static_cast<const uint32_t*>(src), perm, rows, cols, static_cast<uint32_t*>(dst),
                ctx->d_status);
        else
            scatter_rows_kernel<uint64_t><<<grid, BLOCK, 0, st>>>(
                static_cast<const uint64_t*>(src), perm, rows, cols, static_cast<uint64_t*>(dst),
                ctx->d_status);
    }
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}
