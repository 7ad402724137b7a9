// Launch sequences for fixed-point decimal keys: 32-bit cells (up to 9 digits)
// and 64-bit cells (up to 18 digits), keys only and with payloads.
#include "rs_sort_impl.cuh"

namespace rs {
RS_DECLARE_SORT(CodecDec<uint32_t>, NoVal)
RS_DECLARE_SORT(CodecDec<uint32_t>, uint32_t)
RS_DECLARE_SORT(CodecDec<uint32_t>, uint64_t)
RS_DECLARE_SORT(CodecDec<uint64_t>, NoVal)
RS_DECLARE_SORT(CodecDec<uint64_t>, uint32_t)
RS_DECLARE_SORT(CodecDec<uint64_t>, uint64_t)
}  // namespace rs
