// Staged query kernel instantiations for counter widths 5..8.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_STAGED(5)
THR_DEFINE_STAGED(6)
THR_DEFINE_STAGED(7)
THR_DEFINE_STAGED(8)
}  // namespace thr
