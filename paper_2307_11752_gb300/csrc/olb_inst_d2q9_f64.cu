// Kernel instances for the D2Q9 lattice with double population storage.
#include "olb_kernels.cuh"

namespace olb {
const KernelTable* table_d2q9_f64() { return Launch<D2Q9, double>::table(); }
}  // namespace olb
