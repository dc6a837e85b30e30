// qbx_static.cu -- qbx_apply_static: the on-surface apply (same kernels as
// qbx_apply) for callers that cannot allocate device memory.  Its scratch --
// the oversampled density and the split partial sums -- lives in a file-scope
// __device__ array of fixed size instead of a plan's workspace; the
// per-panel interpolation matrix, the complex-k amplitude table of the last
// k and a status word live in three more fixed arrays.
//
// Why: qbx_apply needs a plan, and qbx_plan_create calls cudaMalloc.  Some
// callers must not: code whose device memory is owned by a pooling allocator
// (a raw cudaMalloc goes behind the pool's back and can fail once the pool
// holds the memory), and latency-critical loops where cudaMalloc's implicit
// device synchronisation is not acceptable.  This entry point calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// Every GPU that loads the library holds these arrays until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <algorithm>
#include <mutex>
#include <vector>
#include "../../include/qbx.h"
#include "qbx_internal.h"

// The scratch, the interpolation matrix, the amplitude table of the last
// complex k and a status word, one copy per device.  Every call shares them
// and they keep the last call's contents.
constexpr int kStaticHkDoubles = 4096;   // >= hk_table_doubles() (checked at set-up)
static __device__ __align__(256) unsigned char g_static_scratch[QBX_STATIC_SCRATCH_BYTES];
static __device__ __align__(256) double g_static_interp[QBX_MAX_Q * QBX_MAX_Q];
static __device__ __align__(256) double g_static_hktab[kStaticHkDoubles];
static __device__ int g_static_status;

namespace {

constexpr int kMaxDevices = 64;

struct DeviceState {
  bool ready = false;
  void* scratch = nullptr;   // device address of g_static_scratch on this device
  double* interp = nullptr;  // device address of g_static_interp
  double* hktab = nullptr;   // device address of g_static_hktab
  int* status = nullptr;     // device address of g_static_status
  int num_sms = 0;
  int q_tgt = 0, q_src = 0;  // grid pair whose matrix is in g_static_interp
  double tab_kre = 0.0, tab_kim = 0.0;   // k whose ray table is in g_static_hktab (kim = 0: none)
};

std::mutex g_mu;
DeviceState g_state[kMaxDevices];

int cuda_err(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "qbx_apply_static: %s: %s", what, cudaGetErrorString(e));
  return qbx::host_fail(QBX_ECUDA, buf);
}

int invalid(const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "qbx_apply_static: %s", what);
  return qbx::host_fail(QBX_EINVAL, buf);
}

// Once per device, with that device current: the device addresses of the
// arrays.  In host code the arrays' names stand for host-side shadows, not
// device addresses, so a kernel must be given these addresses instead.  Then,
// whenever the grid pair changes, upload that pair's interpolation matrix in
// the order of `st`: the stream is drained first (earlier calls on it may
// still read the old matrix), and again after the copy (the host vector
// must outlive it).  For Im k > 0, (re)make the amplitude table of k's ray
// on `st` when k changes.
int prepare(int dev, int q_tgt, int q_src, qbx_c64 k, cudaStream_t st, DeviceState** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& s = g_state[dev];
  if (!s.ready) {
    if (qbx::hk_table_doubles() > kStaticHkDoubles) return invalid("amplitude table larger than its fixed array");
    cudaError_t e = cudaGetSymbolAddress(&s.scratch, g_static_scratch);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(scratch)");
    e = cudaGetSymbolAddress((void**)&s.interp, g_static_interp);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(interp)");
    e = cudaGetSymbolAddress((void**)&s.hktab, g_static_hktab);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(hktab)");
    e = cudaGetSymbolAddress((void**)&s.status, g_static_status);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(status)");
    e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_err(e, "cudaDeviceGetAttribute");
    e = cudaMemsetAsync(s.status, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_err(e, "clearing the status word");
    s.ready = true;
  }
  if (s.q_tgt != q_tgt || s.q_src != q_src) {
    std::vector<double> M;
    qbx::host_interp_matrix(q_tgt, q_src, M);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e, "draining the stream before the matrix upload");
    s.q_tgt = s.q_src = 0;   // unknown contents until the copy has completed
    e = cudaMemcpyAsync(s.interp, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e, "upload of the interpolation matrix");
    s.q_tgt = q_tgt;
    s.q_src = q_src;
  }
  if (k.im != 0.0 && (s.tab_kre != k.re || s.tab_kim != k.im)) {
    s.tab_kim = 0.0;
    cudaError_t e = qbx::launch_hk_table(k.re, k.im, s.hktab, st);
    if (e != cudaSuccess) return cuda_err(e, "complex-k amplitude table");
    s.tab_kre = k.re;
    s.tab_kim = k.im;
  }
  *out = &s;
  return QBX_OK;
}

}  // namespace

extern "C" int qbx_apply_static(const qbx_geom* g, int op, int side, int limit, qbx_c64 k, int p,
                                const qbx_c64* dens_tgt, int nrhs, qbx_c64* out_on, void* stream) {
  using namespace qbx;
  // ---- arguments (host checks; nothing is launched on error) ----
  if (!g) return invalid("geometry is NULL");
  if (g->M < 1 || g->q_tgt < 1 || g->q_tgt > QBX_MAX_Q || g->q_src < 1 || g->q_src > QBX_MAX_Q)
    return invalid("geometry: bad M, q_tgt or q_src");
  if (g->n_tgt != g->M * g->q_tgt || g->n_src != g->M * g->q_src)
    return invalid("geometry: n_tgt/n_src inconsistent with M*q");
  if (!g->src_x || !g->src_y || !g->src_nx || !g->src_ny || !g->src_w || !g->tgt_x || !g->tgt_y ||
      !g->tgt_nx || !g->tgt_ny || !g->ctr_x || !g->ctr_y)
    return invalid("geometry: NULL array");
  if (op != QBX_OP_S && op != QBX_OP_D && op != QBX_OP_GRAD_S) return invalid("bad op");
  if (limit != QBX_LIMIT_ONE_SIDED && limit != QBX_LIMIT_PV) return invalid("bad limit");
  if (side != QBX_SIDE_INT && side != QBX_SIDE_EXT && side != QBX_SIDE_TWO) return invalid("bad side");
  if (!isfinite(k.re) || !isfinite(k.im) || k.im < 0.0 || (k.im == 0.0 && !(k.re > 0.0)))
    return invalid("k must be finite with Im k >= 0 (real k > 0)");
  if (p < 0 || p > QBX_MAX_P) return invalid("p outside [0, QBX_MAX_P]");
  if (nrhs < 1) return invalid("nrhs < 1");
  if (!dens_tgt || !out_on) return invalid("NULL density or output");

  // ---- sizes against the fixed scratch ----
  const int c0 = side == QBX_SIDE_EXT ? g->n_tgt : 0;
  const int nc = side == QBX_SIDE_TWO ? 2 * g->n_tgt : g->n_tgt;
  const int ncomp = op == QBX_OP_GRAD_S ? 2 : 1;
  const size_t wd_bytes = host_align256((size_t)g->n_src * nrhs * 16);
  const size_t per_split = (size_t)nc * ncomp * nrhs * 16;
  if (wd_bytes + per_split > QBX_STATIC_SCRATCH_BYTES) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "qbx_apply_static: the call needs at least %zu bytes of scratch, more than the fixed "
             "%zu (n_src = %d, centres = %d, nrhs = %d); use qbx_apply with a plan",
             wd_bytes + per_split, (size_t)QBX_STATIC_SCRATCH_BYTES, g->n_src, nc, nrhs);
    return host_fail(QBX_ENOMEM, buf);
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return invalid("device index beyond the supported range");
  cudaStream_t st = (cudaStream_t)stream;
  DeviceState* s = nullptr;
  if (int rc = prepare(dev, g->q_tgt, g->q_src, k, st, &s)) return rc;

  // split choice as qbx_apply's (resident CTAs of the kernel instance that runs)
  const bool ck = k.im != 0.0;
  const bool one_w = nrhs == 1;
  const int chunk = apply_chunk(1 << op);
  const int occ = ck ? apply_occupancy_cplx(1 << op, p, std::min(chunk, nrhs), one_w)
                     : apply_occupancy_real(1 << op, p, std::min(chunk, nrhs), one_w);
  const int units = (nc + kApplyThreads - 1) / kApplyThreads;
  const int ns = host_choose_split_waves(s->num_sms, occ, units, g->n_src, per_split,
                                         QBX_STATIC_SCRATCH_BYTES - wd_bytes, 1);
  if (ns < 1) return invalid("no source split fits the fixed scratch");
  if (apply_smem_bytes(1 << op, ck, p, chunk) > 220 * 1024) return invalid("p too large");
  char* base = static_cast<char*>(s->scratch);
  void* wd = base;
  void* part = base + wd_bytes;

  // the same launch sequence as qbx_apply's on-surface part
  e = launch_upsample(g->M, g->q_tgt, g->q_src, nrhs, s->interp, g->src_w, dens_tgt, wd, st);
  if (e != cudaSuccess) return cuda_err(e, "upsample kernel");
  ApplyArgs a{};
  a.ops = 1 << op;
  a.wd[0] = a.wd[1] = a.wd[2] = wd;
  a.p = p;
  a.kre = k.re;
  a.kim = k.im;
  a.n_ctr = nc;
  a.cx = g->ctr_x + c0;
  a.cy = g->ctr_y + c0;
  a.n_tgt = g->n_tgt;
  a.tx = g->tgt_x;
  a.ty = g->tgt_y;
  a.src = SrcView{g->src_x, g->src_y, g->src_nx, g->src_ny, g->n_src};
  a.nrhs = nrhs;
  a.nsplit = ns;
  a.src_per_split = host_split_len(g->n_src, ns);
  a.part = part;
  a.near_q_tgt = g->q_tgt;   // near-field items first, as qbx_apply
  a.near_q_src = g->q_src;
  a.one_w = one_w ? 1 : 0;
  a.hk_tab = ck ? s->hktab : nullptr;
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    a.rhs0 = r0;
    a.nr = std::min(chunk, nrhs - r0);
    e = launch_apply_fused(a, st);
    if (e != cudaSuccess) return cuda_err(e, "apply kernel");
  }
  e = launch_apply_finish(op, side, limit, g->n_tgt, ns, nc, nrhs, 0, ncomp, part, dens_tgt, g->tgt_nx,
                          g->tgt_ny, out_on, s->status, st);
  if (e != cudaSuccess) return cuda_err(e, "apply finish");
  return QBX_OK;
}

extern "C" int qbx_apply_static_status(void* stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return invalid("device index beyond the supported range");
  int* status = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_state[dev].ready) return QBX_OK;   // no call has run on this device
    status = g_state[dev].status;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(e, "reading the status word");
  if (h) return qbx::host_fail(QBX_ENONFINITE, "qbx_apply_static: a kernel produced a non-finite value");
  return QBX_OK;
}
