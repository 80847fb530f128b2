// Query kernel instantiations with the position-major decode of mixed
// inputs, counter widths 10, 12, 16 and 20.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_WIDTH_POS(10)
THR_DEFINE_WIDTH_POS(12)
THR_DEFINE_WIDTH_POS(16)
THR_DEFINE_WIDTH_POS(20)
}  // namespace thr
