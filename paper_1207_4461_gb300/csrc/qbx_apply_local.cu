// qbx_apply_local.cu -- instances of the near-only variant of the fused
// apply and of the group kernel (sources beyond eta r by the smooth rule at
// the target), real and complex k, kept apart from the global instances.
#include "qbx_group_impl.cuh"

namespace qbx {

cudaError_t launch_apply_fused_local_real(const ApplyArgs& a, cudaStream_t st) {
  return launch_apply_ops<double, true>(a, st);
}
cudaError_t launch_apply_fused_local_cplx(const ApplyArgs& a, cudaStream_t st) {
  return launch_apply_ops<cplx, true>(a, st);
}
int apply_occupancy_local(int ops, bool ck, int p, int nr, bool one_w) {
  return ck ? apply_occupancy_t<cplx, true>(ops, p, nr, one_w) : apply_occupancy_t<double, true>(ops, p, nr, one_w);
}

cudaError_t launch_group_local(const GroupArgs& a, bool ck, int rg, int grid, cudaStream_t st) {
  return ck ? launch_group_any<cplx, true>(a, rg, grid, st) : launch_group_any<double, true>(a, rg, grid, st);
}
int group_occupancy_local(int ops, bool ck, int p, int rg) {
  return ck ? group_occupancy_any<cplx, true>(ops, p, rg) : group_occupancy_any<double, true>(ops, p, rg);
}
const void* group_ptr_local(int ops, bool ck, int rg) {
  return ck ? group_ptr_any<cplx, true>(ops, rg) : group_ptr_any<double, true>(ops, rg);
}

}  // namespace qbx
