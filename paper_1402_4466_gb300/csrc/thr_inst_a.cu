// Query kernel instantiations for counter widths 1..4.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_WIDTH(1)
THR_DEFINE_WIDTH(2)
THR_DEFINE_WIDTH(3)
THR_DEFINE_WIDTH(4)
}  // namespace thr
