// format_f32.cu -- kernels of the F32 population storage format.
#include "lbm_format_impl.cuh"

namespace lbm {
const FormatOps ops_f32 = detail::make_ops<ST_F32>();
}  // namespace lbm
