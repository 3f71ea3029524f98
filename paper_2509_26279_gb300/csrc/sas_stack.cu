// The stack kernel's instantiations without peak selection (one threshold),
// the dispatch to them and to those with it (sas_stack_peaks.cu), and the
// tiling helpers.  The kernel itself is in sas_stack_kernel.cuh; the two sets
// of instantiations are compiled apart so that each keeps its own register
// allocation (the peak tests' code would otherwise weigh on the hot loop of
// the plain search) and the two compile in parallel.
#include "sas_stack_kernel.cuh"

namespace sas {

bool stack_config_supported(int kx, int ky, int cb) {
#define SAS_CHECK(KX, KY, CB) if (kx == KX && ky == KY && cb == CB) return true;
  SAS_STACK_CONFIGS(SAS_CHECK)
#undef SAS_CHECK
  return false;
}

size_t stack_smem_bytes(const TileCfg& tc) { return layout(tc).total; }

size_t stack_counter_bytes(const TileCfg& tc) { return layout(tc).staged - layout(tc).cells; }

int stack_threads() { return kNT; }

cudaError_t launch_stack(const StackArgs& a, int grid, cudaStream_t s) {
  if (a.select != kSelectAll) return launch_stack_peaks(a, grid, s);
#define SAS_LAUNCH(KX, KY, CB) \
  if (a.tc.kx == KX && a.tc.ky == KY && a.tc.cb == CB) return launch_t<KX, KY, CB, false>(a, grid, s);
  SAS_STACK_CONFIGS(SAS_LAUNCH)
#undef SAS_LAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t launch_stack_multi(int kx, int ky, int cb, bool peaks, const StackArgs* fargs,
                               const unsigned long long* unit_base, int n_fields,
                               unsigned long long* counter, size_t smem, int grid, cudaStream_t s) {
  if (peaks) return launch_stack_multi_peaks(kx, ky, cb, fargs, unit_base, n_fields, counter, smem, grid, s);
  StackArgs proto{};
#define SAS_LAUNCH_M(KX, KY, CB)                                                                   \
  if (kx == KX && ky == KY && cb == CB)                                                            \
    return launch_multi_t<KX, KY, CB, false>(proto, fargs, unit_base, n_fields, counter, smem, grid, s);
  SAS_STACK_CONFIGS(SAS_LAUNCH_M)
#undef SAS_LAUNCH_M
  return cudaErrorInvalidValue;
}

cudaError_t stack_set_smem_attr(int kx, int ky, int cb, size_t smem) {
  cudaError_t e = cudaErrorInvalidValue;
#define SAS_ATTR(KX, KY, CB) if (kx == KX && ky == KY && cb == CB) e = attr_t<KX, KY, CB, false>(smem);
  SAS_STACK_CONFIGS(SAS_ATTR)
#undef SAS_ATTR
  if (e != cudaSuccess) return e;
  return stack_set_smem_attr_peaks(kx, ky, cb, smem);
}

}  // namespace sas
