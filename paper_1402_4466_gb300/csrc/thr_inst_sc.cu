// Staged query kernel instantiations for counter widths 10, 12, 16 and 20.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_STAGED(10)
THR_DEFINE_STAGED(12)
THR_DEFINE_STAGED(16)
THR_DEFINE_STAGED(20)
}  // namespace thr
