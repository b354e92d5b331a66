// format_f16.cu -- kernels of the F16 population storage format.
#include "lbm_format_impl.cuh"

namespace lbm {
const FormatOps ops_f16 = detail::make_ops<ST_F16>();
}  // namespace lbm
