// Kernel instances for the D2Q9 lattice with __nv_bfloat16 population storage.
#include "olb_kernels.cuh"

namespace olb {
const KernelTable* table_d2q9_bf16() { return Launch<D2Q9, __nv_bfloat16>::table(); }
}  // namespace olb
