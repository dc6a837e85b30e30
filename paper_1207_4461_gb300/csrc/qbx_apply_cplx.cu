// qbx_apply_cplx.cu -- instances of the fused apply for complex k (Im k > 0),
// every operator subset, 1/4/8 rhs per pass.
#include "qbx_apply_impl.cuh"

namespace qbx {

cudaError_t launch_apply_fused_cplx(const ApplyArgs& a, cudaStream_t st) {
  return launch_apply_ops<cplx>(a, st);
}

size_t apply_smem_bytes_cplx(int ops, int p, int nr) { return apply_smem_t<cplx>(ops, p, nr); }

}  // namespace qbx
