// Opt-threshold profiling kernels for counter widths 7, 8, 10, 12 and 16.
#include "thr_opt.cuh"

namespace thr {
THR_DEFINE_OPT(7)
THR_DEFINE_OPT(8)
THR_DEFINE_OPT(10)
THR_DEFINE_OPT(12)
THR_DEFINE_OPT(16)
}  // namespace thr
