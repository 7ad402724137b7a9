// rs_api.cu -- the extern "C" boundary declared in include/rs.h.
//
// Host work only: argument checks, workspace sizing, and dispatch to the
// typed launch sequences (rs_sort_impl.cuh, instantiated in inst_*.cu).
// Every step of the sort itself runs in the CUDA kernels.

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "../../include/rs.h"
#include "rs_ctx.hpp"
#include "rs_kernels.cuh"

namespace rs {
template <class C, typename V>
rs_status run_sort(rs_ctx*, const void*, void*, const void*, void*, size_t, CodecParams, uint32_t,
                   void*, size_t*, cudaStream_t, const uint32_t* skip = nullptr);
}  // namespace rs

using namespace rs;

namespace {

constexpr uint64_t kPow10[19] = {1ull,
                                 10ull,
                                 100ull,
                                 1000ull,
                                 10000ull,
                                 100000ull,
                                 1000000ull,
                                 10000000ull,
                                 100000000ull,
                                 1000000000ull,
                                 10000000000ull,
                                 100000000000ull,
                                 1000000000000ull,
                                 10000000000000ull,
                                 100000000000000ull,
                                 1000000000000000ull,
                                 10000000000000000ull,
                                 100000000000000000ull,
                                 1000000000000000000ull};

uint32_t bits_for(uint64_t max_value) {
    uint32_t b = 1;
    while (b < 64 && (max_value >> b) != 0) b++;
    return b;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Common argument checks; returns RS_OK when the call may proceed.
rs_status check_common(rs_ctx* ctx, const void* in, const void* out, size_t n, size_t elem,
                       size_t* temp_bytes) {
    if (!ctx || !temp_bytes) return RS_ERR_INVALID;
    if (n > RS_MAX_N) return RS_ERR_INVALID;
    if (n > 0 && (!in || !out)) return RS_ERR_INVALID;
    if (n > 0 && (!aligned(in, elem) || !aligned(out, elem))) return RS_ERR_INVALID;
    return RS_OK;
}

rs_status remember(rs_ctx* ctx, rs_status s) {
    if (s != RS_OK && s != RS_ERR_TEMP_TOO_SMALL && s != RS_ERR_INVALID && ctx)
        ctx->host_error = s;
    return s;
}

rs_status sort_decimal(rs_ctx* ctx, const int64_t* in, int64_t* out, const void* vin, void* vout,
                       size_t val_bytes, size_t n, int int_digits, int frac_digits, void* temp,
                       size_t* temp_bytes, cudaStream_t st) {
    if (int_digits < 0 || frac_digits < 0 || int_digits + frac_digits < 1 ||
        int_digits + frac_digits > 18)
        return RS_ERR_INVALID;
    const int D = int_digits + frac_digits;
    CodecParams prm{kPow10[D] - 1};
    const uint64_t max_cell = 2 * prm.bias;  // cell of +(10^D - 1)
    const uint32_t bits = bits_for(max_cell);
    if (max_cell <= 0xffffffffull) {
        using C = CodecDec<uint32_t>;
        if (val_bytes == 0) return run_sort<C, NoVal>(ctx, in, out, nullptr, nullptr, n, prm, bits, temp, temp_bytes, st);
        if (val_bytes == 4) return run_sort<C, uint32_t>(ctx, in, out, vin, vout, n, prm, bits, temp, temp_bytes, st);
        return run_sort<C, uint64_t>(ctx, in, out, vin, vout, n, prm, bits, temp, temp_bytes, st);
    }
    using C = CodecDec<uint64_t>;
    if (val_bytes == 0) return run_sort<C, NoVal>(ctx, in, out, nullptr, nullptr, n, prm, bits, temp, temp_bytes, st);
    if (val_bytes == 4) return run_sort<C, uint32_t>(ctx, in, out, vin, vout, n, prm, bits, temp, temp_bytes, st);
    return run_sort<C, uint64_t>(ctx, in, out, vin, vout, n, prm, bits, temp, temp_bytes, st);
}

}  // namespace

extern "C" {

const char* rs_version(void) { return "rsort 0.1 (sm_103a)"; }

rs_status rs_ctx_create(rs_ctx** ctx, int device) {
    if (!ctx) return RS_ERR_INVALID;
    *ctx = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
        return RS_ERR_INVALID;
    rs_ctx* c = new rs_ctx();
    c->device = device;
    DeviceGuard dg(device);
    if (!dg.ok || cudaMalloc(&c->d_area, 256) != cudaSuccess) {
        delete c;
        return RS_ERR_CUDA;
    }
    if (cudaMemset(c->d_area, 0, 256) != cudaSuccess) {
        cudaFree(c->d_area);
        delete c;
        return RS_ERR_CUDA;
    }
    c->d_status = static_cast<uint32_t*>(c->d_area);
    c->d_info = static_cast<unsigned char*>(c->d_area) + 64;
    *ctx = c;
    return RS_OK;
}

rs_status rs_ctx_destroy(rs_ctx* ctx) {
    if (!ctx) return RS_ERR_INVALID;
    {
        DeviceGuard dg(ctx->device);
        for (auto& v : ctx->timed)
            for (auto& tl : v) {
                cudaEventDestroy(tl.begin);
                cudaEventDestroy(tl.end);
            }
        for (auto e : ctx->event_pool) cudaEventDestroy(e);
        if (ctx->d_area) cudaFree(ctx->d_area);
    }
    delete ctx;
    return RS_OK;
}

rs_status rs_ctx_status(rs_ctx* ctx, int synchronize) {
    if (!ctx) return RS_ERR_INVALID;
    rs_status known = ctx->host_error;
    ctx->host_error = RS_OK;
    if (!synchronize) return known;
    DeviceGuard dg(ctx->device);
    if (!dg.ok || cudaDeviceSynchronize() != cudaSuccess) return RS_ERR_CUDA;
    uint32_t word = 0;
    if (cudaMemcpy(&word, ctx->d_status, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess)
        return RS_ERR_CUDA;
    if (word && cudaMemset(ctx->d_status, 0, sizeof(word)) != cudaSuccess) return RS_ERR_CUDA;
    if (known != RS_OK) return known;
    if (word & STATUS_TIMEOUT) return RS_ERR_TIMEOUT;
    if (word & STATUS_RANGE) return RS_ERR_RANGE;
    return RS_OK;
}

rs_status rs_ctx_last_plan(rs_ctx* ctx, rs_plan_info* info) {
    if (!ctx || !info) return RS_ERR_INVALID;
    DeviceGuard dg(ctx->device);
    DevInfo di{};
    if (!dg.ok || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&di, ctx->d_info, sizeof(di), cudaMemcpyDeviceToHost) != cudaSuccess)
        return RS_ERR_CUDA;
    info->mode = di.mode;
    info->passes_run = di.passes_run;
    info->passes_total = ctx->last_passes_total;
    info->tiles = ctx->last_tiles;
    return RS_OK;
}

rs_status rs_ctx_set_pass_tile_limit(rs_ctx* ctx, uint64_t narrow_max_n) {
    if (!ctx) return RS_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->narrow_max_n = narrow_max_n;
    return RS_OK;
}

rs_status rs_ctx_pass_tile_limit(rs_ctx* ctx, uint64_t* narrow_max_n) {
    if (!ctx || !narrow_max_n) return RS_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    *narrow_max_n = ctx->narrow_max_n;
    return RS_OK;
}

rs_status rs_ctx_set_timing(rs_ctx* ctx, int enable) {
    if (!ctx) return RS_ERR_INVALID;
    ctx->timing = enable != 0;
    return RS_OK;
}

rs_status rs_ctx_reset_timing(rs_ctx* ctx) {
    if (!ctx) return RS_ERR_INVALID;
    DeviceGuard dg(ctx->device);
    for (auto& v : ctx->timed) {
        for (auto& tl : v) {
            ctx->event_pool.push_back(tl.begin);
            ctx->event_pool.push_back(tl.end);
        }
        v.clear();
    }
    return RS_OK;
}

rs_status rs_ctx_kernel_time(rs_ctx* ctx, const char* kernel_class, double* total_ms,
                             uint64_t* launches) {
    if (!ctx || !total_ms || !launches) return RS_ERR_INVALID;
    const int k = kernel_class_of(kernel_class);
    if (k < 0) return RS_ERR_INVALID;
    DeviceGuard dg(ctx->device);
    double sum = 0.0;
    for (auto& tl : ctx->timed[k]) {
        if (cudaEventSynchronize(tl.end) != cudaSuccess) return RS_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, tl.begin, tl.end) != cudaSuccess) return RS_ERR_CUDA;
        sum += ms;
    }
    *total_ms = sum;
    *launches = ctx->timed[k].size();
    return RS_OK;
}

uint64_t rs_ctx_launch_count(const rs_ctx* ctx) { return ctx ? ctx->launches : 0; }

rs_status rs_debug_wait_timeout(rs_ctx* ctx, void* temp, size_t temp_bytes, uint64_t timeout_ns,
                                rs_stream_t stream) {
    if (!ctx || !temp || temp_bytes < RADIX * sizeof(uint32_t) || timeout_ns == 0 ||
        timeout_ns > LOOKBACK_TIMEOUT_NS || (reinterpret_cast<uintptr_t>(temp) % 4))
        return RS_ERR_INVALID;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return RS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(temp, 0, RADIX * sizeof(uint32_t), st) != cudaSuccess) return RS_ERR_CUDA;
    wait_timeout_kernel<<<1, BLOCK, 0, st>>>(static_cast<const uint32_t*>(temp), ctx->d_status,
                                              timeout_ns);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

rs_status rs_sort_u32(rs_ctx* ctx, const uint32_t* keys_in, uint32_t* keys_out, size_t n,
                      void* temp, size_t* temp_bytes, rs_stream_t stream) {
    rs_status s = check_common(ctx, keys_in, keys_out, n, 4, temp_bytes);
    if (s != RS_OK) return s;
    return remember(ctx, run_sort<CodecU32, NoVal>(ctx, keys_in, keys_out, nullptr, nullptr, n,
                                                   CodecParams{0}, 32, temp, temp_bytes,
                                                   (cudaStream_t)stream));
}

rs_status rs_sort_u64(rs_ctx* ctx, const uint64_t* keys_in, uint64_t* keys_out, size_t n,
                      void* temp, size_t* temp_bytes, rs_stream_t stream) {
    rs_status s = check_common(ctx, keys_in, keys_out, n, 8, temp_bytes);
    if (s != RS_OK) return s;
    return remember(ctx, run_sort<CodecU64, NoVal>(ctx, keys_in, keys_out, nullptr, nullptr, n,
                                                   CodecParams{0}, 64, temp, temp_bytes,
                                                   (cudaStream_t)stream));
}

rs_status rs_sort_fixed_decimal(rs_ctx* ctx, const int64_t* keys_in, int64_t* keys_out,
                                size_t n, int int_digits, int frac_digits, void* temp,
                                size_t* temp_bytes, rs_stream_t stream) {
    rs_status s = check_common(ctx, keys_in, keys_out, n, 8, temp_bytes);
    if (s != RS_OK) return s;
    return remember(ctx, sort_decimal(ctx, keys_in, keys_out, nullptr, nullptr, 0, n, int_digits,
                                      frac_digits, temp, temp_bytes, (cudaStream_t)stream));
}

rs_status rs_sort_pairs(rs_ctx* ctx, rs_key_type kt, const void* keys_in, void* keys_out,
                        const void* vals_in, void* vals_out, size_t val_bytes, size_t n,
                        const rs_key_params* params, void* temp, size_t* temp_bytes,
                        rs_stream_t stream) {
    if (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) return RS_ERR_INVALID;
    const size_t kbytes = (kt == RS_KEY_U32 || kt == RS_KEY_F32) ? 4 : 8;
    if (kt != RS_KEY_U32 && kt != RS_KEY_U64 && kt != RS_KEY_I64_DEC && kt != RS_KEY_F32 &&
        kt != RS_KEY_F64)
        return RS_ERR_UNSUPPORTED;
    rs_status s = check_common(ctx, keys_in, keys_out, n, kbytes, temp_bytes);
    if (s != RS_OK) return s;
    if (val_bytes == 0) {
        // keys only: no value arrays
        if (vals_in || vals_out) return RS_ERR_INVALID;
    } else {
        if (n > 0 && (!vals_in || !vals_out || !aligned(vals_in, val_bytes) ||
                      !aligned(vals_out, val_bytes)))
            return RS_ERR_INVALID;
        if ((keys_in == keys_out) != (vals_in == vals_out)) return RS_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (val_bytes == 0) {
        switch (kt) {
        case RS_KEY_U32:
            return remember(ctx, run_sort<CodecU32, NoVal>(ctx, keys_in, keys_out, nullptr, nullptr, n, CodecParams{0}, 32, temp, temp_bytes, st));
        case RS_KEY_U64:
            return remember(ctx, run_sort<CodecU64, NoVal>(ctx, keys_in, keys_out, nullptr, nullptr, n, CodecParams{0}, 64, temp, temp_bytes, st));
        case RS_KEY_F32:
            return remember(ctx, run_sort<CodecF32, NoVal>(ctx, keys_in, keys_out, nullptr, nullptr, n, CodecParams{0}, 32, temp, temp_bytes, st));
        case RS_KEY_F64:
            return remember(ctx, run_sort<CodecF64, NoVal>(ctx, keys_in, keys_out, nullptr, nullptr, n, CodecParams{0}, 64, temp, temp_bytes, st));
        default:
            if (!params) return RS_ERR_INVALID;
            return remember(ctx, sort_decimal(ctx, static_cast<const int64_t*>(keys_in),
                                              static_cast<int64_t*>(keys_out), nullptr, nullptr, 0,
                                              n, params->int_digits, params->frac_digits, temp,
                                              temp_bytes, st));
        }
    }
    switch (kt) {
    case RS_KEY_U32:
        if (val_bytes == 4)
            return remember(ctx, run_sort<CodecU32, uint32_t>(ctx, keys_in, keys_out, vals_in, vals_out, n, CodecParams{0}, 32, temp, temp_bytes, st));
        return remember(ctx, run_sort<CodecU32, uint64_t>(ctx, keys_in, keys_out, vals_in, vals_out, n, CodecParams{0}, 32, temp, temp_bytes, st));
    case RS_KEY_U64:
        if (val_bytes == 4)
            return remember(ctx, run_sort<CodecU64, uint32_t>(ctx, keys_in, keys_out, vals_in, vals_out, n, CodecParams{0}, 64, temp, temp_bytes, st));
        return remember(ctx, run_sort<CodecU64, uint64_t>(ctx, keys_in, keys_out, vals_in, vals_out, n, CodecParams{0}, 64, temp, temp_bytes, st));
    case RS_KEY_F32:
        if (val_bytes == 4)
            return remember(ctx, run_sort<CodecF32, uint32_t>(ctx, keys_in, keys_out, vals_in, vals_out, n, CodecParams{0}, 32, temp, temp_bytes, st));
        return remember(ctx, run_sort<CodecF32, uint64_t>(ctx, keys_in, keys_out, vals_in, vals_out, n, CodecParams{0}, 32, temp, temp_bytes, st));
    case RS_KEY_F64:
        if (val_bytes == 4)
            return remember(ctx, run_sort<CodecF64, uint32_t>(ctx, keys_in, keys_out, vals_in, vals_out, n, CodecParams{0}, 64, temp, temp_bytes, st));
        return remember(ctx, run_sort<CodecF64, uint64_t>(ctx, keys_in, keys_out, vals_in, vals_out, n, CodecParams{0}, 64, temp, temp_bytes, st));
    default:
        if (!params) return RS_ERR_INVALID;
        return remember(ctx, sort_decimal(ctx, static_cast<const int64_t*>(keys_in),
                                          static_cast<int64_t*>(keys_out), vals_in, vals_out,
                                          val_bytes, n, params->int_digits, params->frac_digits,
                                          temp, temp_bytes, st));
    }
}

}  // extern "C"
