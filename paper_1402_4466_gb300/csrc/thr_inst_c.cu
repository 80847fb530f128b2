// Query kernel instantiations for counter widths 10, 12, 16 and 20.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_WIDTH(10)
THR_DEFINE_WIDTH(12)
THR_DEFINE_WIDTH(16)
THR_DEFINE_WIDTH(20)
}  // namespace thr
