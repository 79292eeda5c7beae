// Hot kernels compiled for state dimension n = 3.
#include "kernels_hot.cuh"

namespace lq2d {
const KernelTable* kernel_table_n3() { return hot::make_table<3>(); }
}  // namespace lq2d
