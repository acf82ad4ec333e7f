// Kernel instances for the D2Q9 lattice with float population storage.
#include "olb_kernels.cuh"

namespace olb {
const KernelTable* table_d2q9_f32() { return Launch<D2Q9, float>::table(); }
}  // namespace olb
