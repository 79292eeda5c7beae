// Hot kernels compiled for state dimension n = 1.
#include "kernels_hot.cuh"

namespace lq2d {
const KernelTable* kernel_table_n1() { return hot::make_table<1>(); }
}  // namespace lq2d
