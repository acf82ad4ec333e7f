// Kernel instances for the D3Q19 lattice with float population storage.
#include "olb_kernels.cuh"

namespace olb {
const KernelTable* table_d3q19_f32() { return Launch<D3Q19, float>::table(); }
}  // namespace olb
