// Hot kernels compiled for state dimension n = 8.
#include "kernels_hot.cuh"

namespace lq2d {
const KernelTable* kernel_table_n8() { return hot::make_table<8>(); }
}  // namespace lq2d
