// Kernel instances for the D2Q9 lattice with __half population storage.
#include "olb_kernels.cuh"

namespace olb {
const KernelTable* table_d2q9_f16() { return Launch<D2Q9, __half>::table(); }
}  // namespace olb
