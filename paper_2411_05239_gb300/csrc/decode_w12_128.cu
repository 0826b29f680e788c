// Decoder kernels with 12-bit pair tables and 128-thread CTAs (one translation
// unit per table width and CTA size, so that the kernels compile in parallel).
#include "decode_kernels.cuh"

namespace zipnn {

const void* decode_kernel_w12_128(int dtype, bool gen) { return kernel_handle<12, 128>(dtype, gen); }

}  // namespace zipnn
