// Kernel instances for the D3Q19 lattice with __nv_bfloat16 population storage.
#include "olb_kernels.cuh"

namespace olb {
const KernelTable* table_d3q19_bf16() { return Launch<D3Q19, __nv_bfloat16>::table(); }
}  // namespace olb
