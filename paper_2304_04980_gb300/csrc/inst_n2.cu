// Hot kernels compiled for state dimension n = 2.
#include "kernels_hot.cuh"

namespace lq2d {
const KernelTable* kernel_table_n2() { return hot::make_table<2>(); }
}  // namespace lq2d
