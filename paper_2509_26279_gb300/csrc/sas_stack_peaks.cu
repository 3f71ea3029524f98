// The stack kernel's instantiations with peak selection (two thresholds, or
// the tile-local peaks alone; see sas_stack_kernel.cuh), reached through the
// dispatch in sas_stack.cu.
#include "sas_stack_kernel.cuh"

namespace sas {

cudaError_t launch_stack_peaks(const StackArgs& a, int grid, cudaStream_t s) {
#define SAS_LAUNCH(KX, KY, CB) \
  if (a.tc.kx == KX && a.tc.ky == KY && a.tc.cb == CB) return launch_t<KX, KY, CB, true>(a, grid, s);
  SAS_STACK_CONFIGS(SAS_LAUNCH)
#undef SAS_LAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t launch_stack_multi_peaks(int kx, int ky, int cb, const StackArgs* fargs,
                                     const unsigned long long* unit_base, int n_fields,
                                     unsigned long long* counter, size_t smem, int grid, cudaStream_t s) {
  StackArgs proto{};
#define SAS_LAUNCH_M(KX, KY, CB)                                                                  \
  if (kx == KX && ky == KY && cb == CB)                                                           \
    return launch_multi_t<KX, KY, CB, true>(proto, fargs, unit_base, n_fields, counter, smem, grid, s);
  SAS_STACK_CONFIGS(SAS_LAUNCH_M)
#undef SAS_LAUNCH_M
  return cudaErrorInvalidValue;
}

cudaError_t stack_set_smem_attr_peaks(int kx, int ky, int cb, size_t smem) {
#define SAS_ATTR(KX, KY, CB) if (kx == KX && ky == KY && cb == CB) return attr_t<KX, KY, CB, true>(smem);
  SAS_STACK_CONFIGS(SAS_ATTR)
#undef SAS_ATTR
  return cudaErrorInvalidValue;
}

}  // namespace sas
