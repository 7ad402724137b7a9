// rs_maps.cu -- rs_traverse_maps: the paper's count array, traverse maps and
// extraction cost on the device.
//
// For fixed-point decimals whose whole digit vector fits one count array S
// (one dimension per base-10 digit, Eq. 1 / Eq. 2, plus a leading radix-2 sign
// dimension when asked for), this computes what the hashing cycle builds
// (§3.1): S itself, H_Max (largest occupied last-axis coordinate per row) and
// H_Min ([touched flag, smallest occupied coordinate] per row) -- the two
// traverse maps of §3.1.3 -- and the extraction cost k of §5: the cells the
// extraction cycle (§3.2) visits when it walks every touched row from H_Min
// to H_Max.  The walk ends at the last occupied cell, which is H_Max of the
// last touched row, so k = sum over touched rows of (H_Max - H_Min + 1).
// The sort itself does not need the maps (they only skip empty cells); this
// entry point reports them.

#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/rs.h"
#include "rs_sort_impl.cuh"

namespace rs {
namespace {

constexpr uint32_t UNTOUCHED = 0xffffffffu;

__device__ __forceinline__ bool decimal_cell(int64_t v, uint64_t p10, uint32_t signed_dim,
                                             uint64_t* cell) {
    const uint64_t mag = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
    if (mag >= p10 || (v < 0 && !signed_dim)) return false;
    if (!signed_dim) {
        *cell = mag;
    } else {
        // sign dimension first (negative = 0), magnitude digits complemented
        // (9 - d) for negative keys: digits of (10^D - 1 - |v|)
        *cell = v < 0 ? (p10 - 1 - mag) : p10 + mag;
    }
    return true;
}

__global__ void __launch_bounds__(BLOCK) maps_hash_kernel(const int64_t* keys, uint64_t n,
                                                          uint64_t p10, uint32_t signed_dim,
                                                          uint32_t* S, uint32_t* hmax,
                                                          uint32_t* hmin_col, uint32_t* status) {
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * BLOCK) {
        uint64_t cell;
        if (!decimal_cell(keys[i], p10, signed_dim, &cell)) {
            bad = true;
            continue;
        }
        const uint64_t row = cell / 10;
        const uint32_t col = (uint32_t)(cell % 10);
        if (S) atomicAdd(&S[cell], 1u);
        atomicMax(&hmax[row], col);
        atomicMin(&hmin_col[row], col);
    }
    if (bad) atomicOr(status, STATUS_RANGE);
}

// H_Min in the paper's layout: [touched flag, smallest coordinate] per row.
__global__ void __launch_bounds__(BLOCK) maps_finish_kernel(uint64_t rows, const uint32_t* hmin_col,
                                                            uint32_t* hmin_out) {
    for (uint64_t r = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; r < rows;
         r += (uint64_t)gridDim.x * BLOCK) {
        const uint32_t lo = hmin_col[r];
        const bool touched = lo != UNTOUCHED;
        hmin_out[2 * r] = touched ? 1u : 0u;
        hmin_out[2 * r + 1] = touched ? lo : 0u;
    }
}

__global__ void __launch_bounds__(BLOCK) maps_cost_kernel(uint64_t rows, const uint32_t* hmin_out,
                                                          const uint32_t* hmax,
                                                          unsigned long long* k_out) {
    __shared__ unsigned long long s_k;
    if (threadIdx.x == 0) s_k = 0;
    __syncthreads();
    unsigned long long k = 0;
    for (uint64_t r = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; r < rows;
         r += (uint64_t)gridDim.x * BLOCK)
        if (hmin_out[2 * r]) k += hmax[r] - hmin_out[2 * r + 1] + 1;
    atomicAdd(&s_k, k);
    __syncthreads();
    if (threadIdx.x == 0 && s_k) atomicAdd(k_out, s_k);
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" rs_status rs_traverse_maps(rs_ctx* ctx, const int64_t* keys, size_t n, int int_digits,
                                      int frac_digits, int signed_dim, uint32_t* S_out,
                                      uint32_t* hmax_out, uint32_t* hmin_out, uint64_t* k_out,
                                      void* temp, size_t* temp_bytes, rs_stream_t stream) {
    if (!ctx || !temp_bytes) return RS_ERR_INVALID;
    const int D = int_digits + frac_digits;
    if (int_digits < 0 || frac_digits < 0 || D < 1 || D > 18 || n > RS_MAX_N) return RS_ERR_INVALID;
    uint64_t p10 = 1;
    for (int i = 0; i < D; i++) p10 *= 10;
    const uint64_t cells = (signed_dim ? 2 : 1) * p10;
    if (cells > RS_MAX_MAP_CELLS) return RS_ERR_UNSUPPORTED;
    const uint64_t rows = cells / 10;
    const size_t need = align_up(sizeof(uint32_t) * rows);
    if (!temp) {
        *temp_bytes = need;
        return RS_OK;
    }
    if (*temp_bytes < need || (reinterpret_cast<uintptr_t>(temp) % 256)) return RS_ERR_TEMP_TOO_SMALL;
    if (!hmax_out || !hmin_out || !k_out || (n > 0 && !keys)) return RS_ERR_INVALID;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return RS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* hmin_col = static_cast<uint32_t*>(temp);
    if ((S_out && cudaMemsetAsync(S_out, 0, sizeof(uint32_t) * cells, st) != cudaSuccess) ||
        cudaMemsetAsync(hmax_out, 0, sizeof(uint32_t) * rows, st) != cudaSuccess ||
        cudaMemsetAsync(hmin_col, 0xff, sizeof(uint32_t) * rows, st) != cudaSuccess ||
        cudaMemsetAsync(k_out, 0, sizeof(uint64_t), st) != cudaSuccess)
        return RS_ERR_CUDA;
    const int sms = sm_count(ctx->device);
    const int grid_n = (int)std::max<size_t>(1, std::min<size_t>((n + BLOCK - 1) / BLOCK, (size_t)sms * 8));
    const int grid_r = (int)std::max<uint64_t>(1, std::min<uint64_t>((rows + BLOCK - 1) / BLOCK, (uint64_t)sms * 8));
    {
        LaunchTimer lt(ctx, KC_HIST, st);
        if (n) maps_hash_kernel<<<grid_n, BLOCK, 0, st>>>(keys, n, p10, signed_dim ? 1u : 0u,
                                                          S_out, hmax_out, hmin_col, ctx->d_status);
    }
    {
        LaunchTimer lt(ctx, KC_HIST, st);
        maps_finish_kernel<<<grid_r, BLOCK, 0, st>>>(rows, hmin_col, hmin_out);
    }
    {
        LaunchTimer lt(ctx, KC_HIST, st);
        maps_cost_kernel<<<grid_r, BLOCK, 0, st>>>(
            rows, hmin_out, hmax_out, reinterpret_cast<unsigned long long*>(k_out));
    }
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}
