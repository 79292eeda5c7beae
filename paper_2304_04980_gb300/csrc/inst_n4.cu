// Hot kernels compiled for state dimension n = 4.
#include "kernels_hot.cuh"

namespace lq2d {
const KernelTable* kernel_table_n4() { return hot::make_table<4>(); }
}  // namespace lq2d
