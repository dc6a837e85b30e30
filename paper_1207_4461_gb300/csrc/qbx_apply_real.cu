// qbx_apply_real.cu -- instances of the fused apply for real k (the fitted
// real-argument H0/H1 path), every operator subset, 1/4/8 rhs per pass.
#include "qbx_apply_impl.cuh"

namespace qbx {

cudaError_t launch_apply_fused_real(const ApplyArgs& a, cudaStream_t st) {
  return launch_apply_ops<double>(a, st);
}

size_t apply_smem_bytes_real(int ops, int p, int nr) { return apply_smem_t<double>(ops, p, nr); }

}  // namespace qbx
