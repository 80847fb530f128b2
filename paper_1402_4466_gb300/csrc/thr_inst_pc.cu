// Query kernel instantiations with the position-major decode of mixed
// inputs, counter widths 10, 12 and 16.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_WIDTH_POS(10)
THR_DEFINE_WIDTH_POS(12)
THR_DEFINE_WIDTH_POS(16)
}  // namespace thr
