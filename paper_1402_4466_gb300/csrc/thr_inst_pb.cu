// Query kernel instantiations with the position-major decode of mixed
// inputs, counter widths 5..8.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_WIDTH_POS(5)
THR_DEFINE_WIDTH_POS(6)
THR_DEFINE_WIDTH_POS(7)
THR_DEFINE_WIDTH_POS(8)
}  // namespace thr
