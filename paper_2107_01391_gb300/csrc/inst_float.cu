// Launch sequences for IEEE-754 keys (keys only, 4- and 8-byte payloads): float and
// double keys are mapped to order-preserving unsigned cells (-0.0 ties +0.0,
// NaN last) and sorted like unsigned keys of the same width.
#include "rs_sort_impl.cuh"

namespace rs {
RS_DECLARE_SORT(CodecF32, NoVal)
RS_DECLARE_SORT(CodecF32, uint32_t)
RS_DECLARE_SORT(CodecF32, uint64_t)
RS_DECLARE_SORT(CodecF64, NoVal)
RS_DECLARE_SORT(CodecF64, uint32_t)
RS_DECLARE_SORT(CodecF64, uint64_t)
}  // namespace rs
