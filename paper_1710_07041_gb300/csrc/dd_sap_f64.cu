// Schwarz kernel instances for double storage (see dd_sap.cu).
#include "dd_sap_kernels.cuh"

namespace dd {
int sap_run_f64(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp,
                const AuxPtrs *ax, cudaStream_t st) {
  return sap_variants<double>(L, nl, p, rp, ax, st);
}
}  // namespace dd
