// Hot kernels compiled for state dimension n = 5.
#include "kernels_hot.cuh"

namespace lq2d {
const KernelTable* kernel_table_n5() { return hot::make_table<5>(); }
}  // namespace lq2d
