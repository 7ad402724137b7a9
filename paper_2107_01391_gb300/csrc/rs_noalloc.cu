// rs_noalloc.cu -- rs_sort_u32_noalloc: the uint32 keys-only sort with its
// workspace in a fixed device array compiled into the library.
//
// Some callers cannot allocate device memory when they sort: cudaFree waits
// for the whole device and cudaMalloc can stall, which a latency-bound loop
// cannot afford, and code that runs inside another framework's memory budget
// (a plugin or a server that owns every device byte through its own pool) has
// no allocator it may call and no way to hand a workspace through.  For them
// this entry point takes only the keys, the output and a stream: the
// workspace of the ordinary rs_sort_u32 launch sequence (counts, plan,
// look-back rows, ping-pong buffer) lives in g_scratch below, sized for
// RS_NOALLOC_MAX_N keys.  Every GPU that loads the library holds that array
// until the process exits.
//
// g_scratch is one array per device shared by every call: a call clears the
// parts that must start at zero before it uses them, and two calls whose work
// overlaps on the GPU (different streams, or different host threads without
// ordering) race on it.  In host code the name g_scratch is only a host-side
// stand-in, so the host passes the kernels the device address obtained from
// cudaGetSymbolAddress, fetched once per device by the first call on that
// device (with the device current).  That first call should therefore be made
// before any stream capture begins.

#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rs.h"
#include "rs_sort_impl.cuh"

namespace {

using namespace rs;

// [0, 256): status word (when the caller passes none) and plan info;
// [256, ...): the workspace layout of one rs_sort_u32 call.
constexpr size_t kHeader = 256;

static __device__ __align__(256) unsigned char g_scratch[RS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

using Cu32 = CodecU32;
constexpr int kIPT = ipt_for<Cu32, NoVal>();
constexpr int kPB = pass_block<Cu32, NoVal>();
constexpr size_t kLaneHist = LANE_HIST_WORDS * sizeof(uint32_t);

// Per-device set-up, done once by the first call on a device (with that
// device current): the device address of g_scratch, and the opt-in of this
// file's copies of the counting and pass kernels to more than 48 KB of
// shared memory (static + dynamic).
rs_status setup_device(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr)
            return RS_ERR_CUDA;
        using Smem = PassSmem<uint32_t, NoVal, kIPT, kPB>;
        if (cudaFuncSetAttribute(count_kernel<Cu32, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kLaneHist) != cudaSuccess ||
            cudaFuncSetAttribute(pass_kernel<Cu32, NoVal, kIPT, kPB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem::kBytes) != cudaSuccess)
            return RS_ERR_CUDA;
        g_scratch_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[device];
    return RS_OK;
}

}  // namespace

extern "C" rs_status rs_sort_u32_noalloc(const uint32_t* keys_in, uint32_t* keys_out, size_t n,
                                         uint32_t* status, rs_stream_t stream) {
    if (n > RS_NOALLOC_MAX_N) return RS_ERR_TEMP_TOO_SMALL;  // beyond the built-in workspace
    if (n > 0 && (!keys_in || !keys_out)) return RS_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(keys_in) | reinterpret_cast<uintptr_t>(keys_out)) % 4)
        return RS_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(status) % 4) return RS_ERR_INVALID;
    if (n == 0) return RS_OK;

    using C = Cu32;
    constexpr int IPT = kIPT;
    constexpr int PB = kPB;
    constexpr int TILE = PB * IPT;
    constexpr uint32_t passes = 4;
    const Layout L = make_layout(n, passes, TILE, sizeof(uint32_t), 0);
    if (kHeader + L.total > RS_NOALLOC_SCRATCH_BYTES) return RS_ERR_TEMP_TOO_SMALL;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
        return RS_ERR_CUDA;
    unsigned char* base = nullptr;
    rs_status s = setup_device(device, &base);
    if (s != RS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;

    uint32_t* status_word = status ? status : reinterpret_cast<uint32_t*>(base);
    DevInfo* info = reinterpret_cast<DevInfo*>(base + 64);
    unsigned char* T = base + kHeader;
    DevPlan* plan = reinterpret_cast<DevPlan*>(T + L.plan);
    uint32_t* bin_offsets = reinterpret_cast<uint32_t*>(T + L.bin_offsets);
    uint32_t* fill_offsets = reinterpret_cast<uint32_t*>(T + L.fill_offsets);
    uint32_t* lb[2] = {reinterpret_cast<uint32_t*>(T + L.lookback0),
                       reinterpret_cast<uint32_t*>(T + L.lookback1)};

    // the previous call's plan, counts and look-back rows must not leak in
    if (cudaMemsetAsync(T, 0, L.memset_bytes, st) != cudaSuccess) return RS_ERR_CUDA;

    CountArgs a{};
    a.keys_in = keys_in;
    a.n = n;
    a.passes = passes;
    a.fill_allowed = 1;
    a.in_is_out = keys_in == keys_out;
    a.prm = CodecParams{0};
    a.plan = plan;
    a.hist = reinterpret_cast<uint32_t*>(T + L.hist);
    a.bin_offsets = bin_offsets;
    a.fill_hist = reinterpret_cast<uint32_t*>(T + L.fill_hist);
    a.fill_offsets = fill_offsets;
    a.status = status_word;
    a.info = info;
    count_kernel<C, true><<<count_grid(n, sm_count(device)), BLOCK, kLaneHist, st>>>(a);

    FillArgs f{};
    f.keys_out = keys_out;
    f.n = n;
    f.prm = CodecParams{0};
    f.plan = plan;
    f.fill_offsets = fill_offsets;
    const size_t per_cta = (size_t)BLOCK * FILL_IPT;
    fill_kernel<C><<<(unsigned)((n + per_cta - 1) / per_cta), BLOCK, 0, st>>>(f);

    using Smem = PassSmem<uint32_t, NoVal, IPT, PB>;
    for (uint32_t p = 0; p < passes; p++) {
        PassArgs pa{};
        pa.keys_in = keys_in;
        pa.keys_tmp = T + L.keys_tmp;
        pa.keys_out = keys_out;
        pa.n = n;
        pa.pass = p;
        pa.shift = p * RADIX_BITS;
        pa.prm = CodecParams{0};
        pa.plan = plan;
        pa.bin_offsets = bin_offsets + p * RADIX;
        pa.lookback = lb[p & 1];
        pa.lookback_next = lb[(p + 1) & 1];
        pa.tile_counter = &plan->tile_counter[p];
        pa.status = status_word;
        pa.prefetch_ahead = prefetch_ahead_for(PassShape<C, NoVal>::kCTAs * sm_count(device));
        pass_kernel<C, NoVal, IPT, PB><<<(unsigned)L.tiles, PB, Smem::kBytes, st>>>(pa);
    }
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}
