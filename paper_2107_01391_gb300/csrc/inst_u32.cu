// Launch sequences for 32-bit unsigned keys (keys only, 4- and 8-byte payloads).
#include "rs_sort_impl.cuh"

namespace rs {
RS_DECLARE_SORT(CodecU32, NoVal)
RS_DECLARE_SORT(CodecU32, uint32_t)
RS_DECLARE_SORT(CodecU32, uint64_t)
}  // namespace rs
