// Query kernel instantiations for counter widths 5..8.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_WIDTH(5)
THR_DEFINE_WIDTH(6)
THR_DEFINE_WIDTH(7)
THR_DEFINE_WIDTH(8)
}  // namespace thr
