// Kernel instances for the D3Q19 lattice with __half population storage.
#include "olb_kernels.cuh"

namespace olb {
const KernelTable* table_d3q19_f16() { return Launch<D3Q19, __half>::table(); }
}  // namespace olb
