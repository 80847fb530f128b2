// Staged query kernel instantiations for counter widths 1..4.
#include "thr_inst_macro.cuh"

namespace thr {
THR_DEFINE_STAGED(1)
THR_DEFINE_STAGED(2)
THR_DEFINE_STAGED(3)
THR_DEFINE_STAGED(4)
}  // namespace thr
