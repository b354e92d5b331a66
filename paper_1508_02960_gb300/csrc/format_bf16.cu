// format_bf16.cu -- kernels of the BF16 population storage format.
#include "lbm_format_impl.cuh"

namespace lbm {
const FormatOps ops_bf16 = detail::make_ops<ST_BF16>();
}  // namespace lbm
