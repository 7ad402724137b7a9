// Launch sequences for 64-bit unsigned keys (keys only, 4- and 8-byte payloads).
#include "rs_sort_impl.cuh"

namespace rs {
RS_DECLARE_SORT(CodecU64, NoVal)
RS_DECLARE_SORT(CodecU64, uint32_t)
RS_DECLARE_SORT(CodecU64, uint64_t)
}  // namespace rs
