// rs_autograd.cu -- rs_scatter_rows: the backward of a row-wise sort.
//
// Sorting a row is a permutation, so its Jacobian is a permutation matrix:
// d sorted[j] / d x[perm[j]] = 1 and every other entry is 0.  The gradient of
// the input is therefore the upstream gradient scattered back through the
// permutation: grad_x[r, perm[r, j]] = grad_sorted[r, j].  (The paper has no
// gradient; this is the differentiable form of its output step.)

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "../../include/rs.h"
#include "rs_sort_impl.cuh"

namespace rs {
namespace {

// Rows that fit in shared memory: a CTA takes whole rows, reads the row's
// gradient and permutation once (coalesced), scatters into shared memory and
// writes the row back coalesced.  Entries outside 0..cols-1 are flagged and
// skipped; a row that is not a permutation leaves its output unspecified.
template <typename T>
__global__ void __launch_bounds__(BLOCK) scatter_rows_smem_kernel(const T* __restrict__ src,
                                                                  const int64_t* __restrict__ perm,
                                                                  uint64_t rows, uint32_t cols,
                                                                  T* __restrict__ dst,
                                                                  uint32_t* status) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    T* s_row = reinterpret_cast<T*>(smem_dyn);
    bool bad = false;
    for (uint64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const T* srow = src + r * cols;
        const int64_t* prow = perm + r * cols;
        for (uint32_t j = threadIdx.x; j < cols; j += BLOCK) {
            const int64_t p = __ldcs(&prow[j]);
            if (p < 0 || p >= (int64_t)cols) {
                bad = true;
                continue;
            }
            s_row[p] = __ldcs(&srow[j]);
        }
        __syncthreads();
        T* drow = dst + r * cols;
        for (uint32_t j = threadIdx.x; j < cols; j += BLOCK) __stcs(&drow[j], s_row[j]);
        __syncthreads();  // s_row is refilled by the next row
    }
    if (bad) atomicOr(status, STATUS_RANGE);
}

// Longer rows: a grid-stride walk over the elements; the row and column
// advance by constant steps, so no element needs a division.
template <typename T>
__global__ void __launch_bounds__(BLOCK) scatter_rows_kernel(const T* __restrict__ src,
                                                             const int64_t* __restrict__ perm,
                                                             uint64_t rows, uint64_t cols,
                                                             T* __restrict__ dst,
                                                             uint32_t* status) {
    const uint64_t total = rows * cols;
    const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
    const uint64_t dr = stride / cols, dc = stride % cols;
    uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
    uint64_t r = i / cols, c = i % cols;
    bool bad = false;
    for (; i < total; i += stride) {
        const int64_t p = __ldcs(&perm[i]);
        if (p < 0 || (uint64_t)p >= cols)
            bad = true;  // not a permutation of the row: skip the element
        else
            dst[r * cols + (uint64_t)p] = __ldcs(&src[i]);
        r += dr;
        c += dc;
        if (c >= cols) {
            c -= cols;
            r++;
        }
    }
    if (bad) atomicOr(status, STATUS_RANGE);
}

// Largest row kept in shared memory (bytes), with the opt-in above 48 KB.
constexpr size_t ROW_SMEM_MAX = 96 * 1024;

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
    const int sms = sm_count(ctx->device);
    const size_t row_bytes = cols * elem_bytes;
    if (row_bytes <= ROW_SMEM_MAX) {
        static std::atomic<bool> smem_set[64];  // zero-initialised: false
        if (ctx->device < 64 && !smem_set[ctx->device].load(std::memory_order_acquire)) {
            if (cudaFuncSetAttribute(scatter_rows_smem_kernel<uint32_t>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ROW_SMEM_MAX) != cudaSuccess ||
                cudaFuncSetAttribute(scatter_rows_smem_kernel<uint64_t>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ROW_SMEM_MAX) != cudaSuccess)
                return RS_ERR_CUDA;
            smem_set[ctx->device].store(true, std::memory_order_release);
        }
        // as many rows in flight as shared memory allows, at most 8 CTAs per SM
        const size_t per_sm = std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / row_bytes));
        const int grid = (int)std::max<size_t>(1, std::min<size_t>(rows, (size_t)sms * per_sm));
        LaunchTimer lt(ctx, KC_SEG, st);
        if (elem_bytes == 4)
            scatter_rows_smem_kernel<uint32_t><<<grid, BLOCK, row_bytes, st>>>(
                static_cast<const uint32_t*>(src), perm, rows, (uint32_t)cols,
                static_cast<uint32_t*>(dst), ctx->d_status);
        else
            scatter_rows_smem_kernel<uint64_t><<<grid, BLOCK, row_bytes, st>>>(
                static_cast<const uint64_t*>(src), perm, rows, (uint32_t)cols,
                static_cast<uint64_t*>(dst), ctx->d_status);
    } else {
        const int grid = (int)std::max<size_t>(
            1, std::min<size_t>((n + BLOCK * 4 - 1) / (BLOCK * 4), (size_t)sms * 8));
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
