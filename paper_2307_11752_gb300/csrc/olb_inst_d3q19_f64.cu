// Kernel instances for the D3Q19 lattice with double population storage.
#include "olb_kernels.cuh"

namespace olb {
const KernelTable* table_d3q19_f64() { return Launch<D3Q19, double>::table(); }
}  // namespace olb
