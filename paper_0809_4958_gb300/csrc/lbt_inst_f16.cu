// Kernels of the step for one population storage format.
#include "lbt_kernels.cuh"

namespace lbt {
template struct Launch<kF16>;
}  // namespace lbt
