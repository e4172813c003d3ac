// Schwarz kernel instances for __nv_bfloat16 storage (see dd_sap.cu).
#include "dd_sap_kernels.cuh"

namespace dd {
int sap_run_bf16(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp,
                const AuxPtrs *ax, cudaStream_t st) {
  return sap_variants<__nv_bfloat16>(L, nl, p, rp, ax, st);
}
}  // namespace dd
