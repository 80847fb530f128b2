// Query kernel instantiations for counter widths 10, 12 and 16.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_WIDTH(10)
THR_DEFINE_WIDTH(12)
THR_DEFINE_WIDTH(16)
}  // namespace thr
