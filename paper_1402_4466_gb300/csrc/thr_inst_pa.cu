// Query kernel instantiations with the position-major decode of mixed
// inputs, counter widths 1..4.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_WIDTH_POS(1)
THR_DEFINE_WIDTH_POS(2)
THR_DEFINE_WIDTH_POS(3)
THR_DEFINE_WIDTH_POS(4)
}  // namespace thr
