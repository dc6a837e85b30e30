// qbx_apply_real.cu -- instances of the fused apply and of the group kernel
// for real k (the fitted real-argument H0/H1 path).
#include "qbx_group_impl.cuh"

namespace qbx {

cudaError_t launch_apply_fused_real(const ApplyArgs& a, cudaStream_t st) {
  return launch_apply_ops<double>(a, st);
}
size_t apply_smem_bytes_real(int ops, int p, int nr) { return apply_smem_t<double>(ops, p, nr); }
int apply_occupancy_real(int ops, int p, int nr, bool one_w) {
  return apply_occupancy_t<double>(ops, p, nr, one_w);
}

cudaError_t launch_group_real(const GroupArgs& a, int rg, int grid, cudaStream_t st) {
  return launch_group_any<double>(a, rg, grid, st);
}
size_t group_smem_real(int ops, int p, int rg) { return group_smem_any<double>(ops, p, rg); }
int group_occupancy_real(int ops, int p, int rg) { return group_occupancy_any<double>(ops, p, rg); }
const void* group_ptr_real(int ops, int rg) { return group_ptr_any<double>(ops, rg); }

}  // namespace qbx

#include "qbx_adjoint_impl.cuh"
namespace qbx {
cudaError_t launch_adjoint_real(const AdjArgs& a, cudaStream_t st) { return launch_adjoint_any<double>(a, st); }
}  // namespace qbx
