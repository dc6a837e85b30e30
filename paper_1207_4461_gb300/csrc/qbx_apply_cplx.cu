// qbx_apply_cplx.cu -- instances of the fused apply and of the group kernel
// for complex k (Im k > 0).
#include "qbx_group_impl.cuh"

namespace qbx {

cudaError_t launch_apply_fused_cplx(const ApplyArgs& a, cudaStream_t st) {
  return launch_apply_ops<cplx>(a, st);
}
size_t apply_smem_bytes_cplx(int ops, int p, int nr) { return apply_smem_t<cplx>(ops, p, nr); }
int apply_occupancy_cplx(int ops, int p, int nr, bool one_w) {
  return apply_occupancy_t<cplx>(ops, p, nr, one_w);
}

cudaError_t launch_group_cplx(const GroupArgs& a, int rg, int grid, cudaStream_t st) {
  return launch_group_any<cplx>(a, rg, grid, st);
}
size_t group_smem_cplx(int ops, int p, int rg) { return group_smem_any<cplx>(ops, p, rg); }
int group_occupancy_cplx(int ops, int p, int rg) { return group_occupancy_any<cplx>(ops, p, rg); }
const void* group_ptr_cplx(int ops, int rg) { return group_ptr_any<cplx>(ops, rg); }

}  // namespace qbx

#include "qbx_adjoint_impl.cuh"
namespace qbx {
cudaError_t launch_adjoint_cplx(const AdjArgs& a, cudaStream_t st) { return launch_adjoint_any<cplx>(a, st); }
}  // namespace qbx
