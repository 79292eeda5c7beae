// Hot kernels compiled for state dimension n = 7.
#include "kernels_hot.cuh"

namespace lq2d {
const KernelTable* kernel_table_n7() { return hot::make_table<7>(); }
}  // namespace lq2d
