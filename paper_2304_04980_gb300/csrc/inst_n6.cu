// Hot kernels compiled for state dimension n = 6.
#include "kernels_hot.cuh"

namespace lq2d {
const KernelTable* kernel_table_n6() { return hot::make_table<6>(); }
}  // namespace lq2d
