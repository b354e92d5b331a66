// format_f64.cu -- kernels of the F64 population storage format.
#include "lbm_format_impl.cuh"

namespace lbm {
const FormatOps ops_f64 = detail::make_ops<ST_F64>();
}  // namespace lbm
