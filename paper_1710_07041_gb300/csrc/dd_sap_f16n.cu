// Schwarz kernel instances for DD_F16N storage: FP16 operator tiles,
// spinors in 16-bit fixed point with a per-site scale (see dd_sap.cu).
#include "dd_sap_kernels.cuh"

namespace dd {
int sap_run_f16n(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp,
                 const AuxPtrs *ax, cudaStream_t st) {
  return sap_variants<hn16>(L, nl, p, rp, ax, st);
}
}  // namespace dd
