// Opt-threshold profiling kernels for counter widths 1..6, and the table of
// every instantiated width.
#include "thr_opt.cuh"

namespace thr {
THR_DEFINE_OPT(1)
THR_DEFINE_OPT(2)
THR_DEFINE_OPT(3)
THR_DEFINE_OPT(4)
THR_DEFINE_OPT(5)
THR_DEFINE_OPT(6)
THR_DECLARE_OPT(7)
THR_DECLARE_OPT(8)
THR_DECLARE_OPT(10)
THR_DECLARE_OPT(12)
THR_DECLARE_OPT(16)

const OptEntry* opt_kernel_table(int* count) {
#define THR_OPT_ENTRY(S) {S, launch_opt_##S, occupancy_opt_##S}
    static const OptEntry table[] = {THR_OPT_ENTRY(1),  THR_OPT_ENTRY(2),  THR_OPT_ENTRY(3),
                                     THR_OPT_ENTRY(4),  THR_OPT_ENTRY(5),  THR_OPT_ENTRY(6),
                                     THR_OPT_ENTRY(7),  THR_OPT_ENTRY(8),  THR_OPT_ENTRY(10),
                                     THR_OPT_ENTRY(12), THR_OPT_ENTRY(16)};
#undef THR_OPT_ENTRY
    *count = int(sizeof(table) / sizeof(table[0]));
    return table;
}
}  // namespace thr
