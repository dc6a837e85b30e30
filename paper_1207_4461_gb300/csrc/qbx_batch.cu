// qbx_batch.cu -- many curves (each with its own panels, wavenumber and
// densities) applied in one persistent launch of the group kernel, run as a
// CUDA graph: [zero the item counter] -> [oversample every curve's
// densities] -> [group kernel over the longest-first item list] -> [scale,
// jump terms / two-sided average into every curve's outputs].
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>
#include "../../include/qbx.h"
#include "qbx_device.cuh"
#include "qbx_internal.h"

using namespace qbx;

struct qbx_batch {
  int device = 0, n_inst = 0, p = 0, ops = 0, side = 0, limit = 0, nrhs = 0, ncomp = 0, rg = 8;
  bool ck = false;
  int n_items = 0, grid = 0, max_src = 0, max_tgt = 0, num_sms = 0;
  int chunk = 0;                    // sources per work item (multiple of 32)
  double eta2 = 0.0;                // near-only QBX when > 0 (qbx_batch_set_eta)
  double* d_hk = nullptr;           // amplitude tables of the complex-k curves' rays
  size_t part_cap = 0;              // bytes allocated for the partial sums
  std::vector<qbx::GroupInst> h_inst;
  GroupInst* d_inst = nullptr;
  GroupItem* d_items = nullptr;
  int* d_counter = nullptr;
  int* d_status = nullptr;
  void* d_wd = nullptr;
  void* d_part = nullptr;
  const double* d_interp = nullptr;  // the plan's
  int q_tgt = 0, q_src = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int bfail(int code, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_batch: %s", what);
  return host_fail(code, buf);
}

int bcuda(cudaError_t e, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_batch: %s: %s", what, cudaGetErrorString(e));
  return host_fail(QBX_ECUDA, buf);
}

// a1 for every curve: blockIdx.y = curve, wd[s][r] = w_s sum_i P[j][i] dens[m q_tgt + i][r]
__global__ void k_batch_upsample(const GroupInst* inst, int q_tgt, int q_src, int nrhs, const double* P) {
  const GroupInst& in = inst[blockIdx.y];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= in.n_src * nrhs) return;
  const int s = idx / nrhs, r = idx - s * nrhs;
  const int m = s / q_src, j = s - m * q_src;
  const double* row = P + (size_t)j * q_tgt;
  const cplx* d = reinterpret_cast<const cplx*>(in.dens) + (size_t)m * q_tgt * nrhs + r;
  double re = 0.0, im = 0.0;
  for (int i = 0; i < q_tgt; ++i) {
    const double c = row[i];
    const cplx v = d[(size_t)i * nrhs];
    re = fma(c, v.re, re);
    im = fma(c, v.im, im);
  }
  const double w = in.sw[s];
  reinterpret_cast<cplx*>(const_cast<void*>(in.wd))[idx] = cplx{w * re, w * im};
}

// a7 for every curve: blockIdx.y = curve; component q of the partial rows
// belongs to operator op_of[q] (S, D, grad S x, grad S y in that order).
__global__ void k_batch_finish(const GroupInst* inst, int ops, int ncomp, int limit, int nrhs, int* status) {
  const GroupInst& in = inst[blockIdx.y];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= in.n_tgt * ncomp * nrhs) return;
  const int t = idx / (ncomp * nrhs);
  const int rem = idx - t * ncomp * nrhs;
  const int q = rem / nrhs, r = rem - q * nrhs;
  // operator and component within it
  int op = 0, comp = 0, qq = q;
  for (int o = 0; o < 3; ++o) {
    if (!(ops >> o & 1)) continue;
    const int n = (o == QBX_OP_GRAD_S) ? 2 : 1;
    if (qq < n) {
      op = o;
      comp = qq;
      break;
    }
    qq -= n;
  }
  const cplx* part = reinterpret_cast<const cplx*>(in.part);
  const int nsides = in.side == QBX_SIDE_TWO ? 2 : 1;
  cplx res{0.0, 0.0};
  for (int sd = 0; sd < nsides; ++sd) {
    const int c = t + sd * in.n_tgt;
    cplx u{0.0, 0.0};
    for (int k = 0; k < in.nsplit; ++k) u = u + part[(((size_t)k * in.n_ctr + c) * ncomp + q) * nrhs + r];
    u = mul_i(0.25 * u);
    if (in.side != QBX_SIDE_TWO && limit == QBX_LIMIT_PV) {
      const double sg = in.side == QBX_SIDE_EXT ? 1.0 : -1.0;
      const cplx dv = reinterpret_cast<const cplx*>(in.dens)[(size_t)t * nrhs + r];
      if (op == QBX_OP_D) u = u - (0.5 * sg) * dv;
      else if (op == QBX_OP_GRAD_S) u = u + (0.5 * sg * (comp == 0 ? in.tnx[t] : in.tny[t])) * dv;
    }
    res = res + u;
  }
  if (nsides == 2) res = 0.5 * res;
  const int nc_op = op == QBX_OP_GRAD_S ? 2 : 1;
  cplx* out = reinterpret_cast<cplx*>(in.out[op]);
  out[((size_t)t * nc_op + comp) * nrhs + r] = res;
  if (!(isfinite(res.re) && isfinite(res.im))) atomicOr(status, 1);
}

void destroy(qbx_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_inst);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  cudaFree(b->d_status);
  cudaFree(b->d_wd);
  cudaFree(b->d_part);
  cudaFree(b->d_hk);
  delete b;
}


// Work items of a configuration: 32 centres of one curve x a range of at
// most `chunk` of its sources (equal ranges per curve), longest first.
std::vector<GroupItem> make_items(const std::vector<GroupInst>& inst, int chunk, std::vector<int>& nsplit) {
  std::vector<GroupItem> items;
  nsplit.assign(inst.size(), 1);
  for (size_t i = 0; i < inst.size(); ++i) {
    int ns = std::max(1, (inst[i].n_src + chunk - 1) / chunk);
    const int len = (inst[i].n_src + ns - 1) / ns;
    ns = (inst[i].n_src + len - 1) / len;   // every range non-empty
    nsplit[i] = ns;
    for (int c = 0; c < inst[i].n_ctr; c += kGrpCentres)
      for (int k = 0; k < ns; ++k)
        items.push_back(GroupItem{(int)i, c, k, k * len, std::min(inst[i].n_src, (k + 1) * len)});
  }
  std::stable_sort(items.begin(), items.end(), [&](const GroupItem& x, const GroupItem& y) {
    const long cx = (long)std::min(kGrpCentres, inst[x.inst].n_ctr - x.ctr0) * (x.src1 - x.src0);
    const long cy = (long)std::min(kGrpCentres, inst[y.inst].n_ctr - y.ctr0) * (y.src1 - y.src0);
    return cx > cy;
  });
  return items;
}

size_t part_bytes(const std::vector<GroupInst>& inst, const std::vector<int>& nsplit, int ncomp, int nrhs) {
  size_t t = 0;
  for (size_t i = 0; i < inst.size(); ++i)
    t += host_align256((size_t)nsplit[i] * inst[i].n_ctr * ncomp * nrhs * 16);
  return t;
}

// Predicted makespan (in pair units) of the persistent grid taking the items
// in list order: each of `slots` CTAs takes the next item when it finishes
// (the atomic counter), an item costs its pairs plus a fixed set-up share.
double lpt_makespan(const std::vector<GroupInst>& inst, const std::vector<GroupItem>& items, int slots) {
  std::vector<double> heap(std::max(1, slots), 0.0);   // min-heap of finish times
  auto cmp = [](double x, double y) { return x > y; };
  for (const GroupItem& it : items) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    const double pairs = (double)std::min(kGrpCentres, inst[it.inst].n_ctr - it.ctr0) * (it.src1 - it.src0);
    heap.back() += pairs + 32.0 * kGrpTile;   // + one tile's worth of set-up per item
    std::push_heap(heap.begin(), heap.end(), cmp);
  }
  return *std::max_element(heap.begin(), heap.end());
}

// The source chunk the model prefers: the smallest predicted makespan over
// chunks 2^j * 32 (and all sources), ties to the larger chunk (fewer
// partial sums), within the partial-sum memory budget.
int model_chunk(const qbx_batch* b, int slots, size_t budget) {
  std::vector<int> cand{(b->max_src + kGrpTile - 1) / kGrpTile * kGrpTile};
  for (int c = 1 << 20; c >= 512; c /= 2)
    if (c < b->max_src) cand.push_back(c);
  int best = cand[0];
  double bt = 1e300;
  std::vector<int> ns;
  for (int c : cand) {
    std::vector<GroupItem> items = make_items(b->h_inst, c, ns);
    if (part_bytes(b->h_inst, ns, b->ncomp, b->nrhs) > budget) break;
    const double t = lpt_makespan(b->h_inst, items, slots);
    if (t < bt * 0.995) {
      bt = t;
      best = c;
    }
  }
  return best;
}

// (Re)build the batch for (rg, chunk): items, partial-sum layout, device
// tables, and the graph [counter := 0] -> [oversample] -> [group] -> [finish].
int configure(qbx_batch* b, int rg, int chunk) {
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bcuda(e, "device");
  std::vector<int> ns;
  std::vector<GroupItem> items = make_items(b->h_inst, chunk, ns);
  const size_t pb = part_bytes(b->h_inst, ns, b->ncomp, b->nrhs);
  if (pb > b->part_cap) {
    cudaFree(b->d_part);
    b->d_part = nullptr;
    b->part_cap = 0;
    e = cudaMalloc(&b->d_part, pb);
    if (e != cudaSuccess) return bcuda(e, "partial-sum allocation");
    b->part_cap = pb;
  }
  if (items.size() > (size_t)b->n_items) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    e = cudaMalloc(&b->d_items, sizeof(GroupItem) * items.size());
    if (e != cudaSuccess) return bcuda(e, "item-list allocation");
  }
  size_t off = 0;
  for (int i = 0; i < b->n_inst; ++i) {
    b->h_inst[i].nsplit = ns[i];
    b->h_inst[i].part = static_cast<char*>(b->d_part) + off;
    off += host_align256((size_t)ns[i] * b->h_inst[i].n_ctr * b->ncomp * b->nrhs * 16);
  }
  e = cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(GroupInst) * b->n_inst, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_items, items.data(), sizeof(GroupItem) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(e, "upload");
  b->n_items = (int)items.size();
  b->rg = rg;
  b->chunk = chunk;
  const bool local = b->eta2 > 0.0;
  const int occ = local ? group_occupancy_local(b->ops, b->ck, b->p, rg)
                        : (b->ck ? group_occupancy_cplx(b->ops, b->p, rg) : group_occupancy_real(b->ops, b->p, rg));
  const size_t gsmem = b->ck ? group_smem_cplx(b->ops, b->p, rg) : group_smem_real(b->ops, b->p, rg);
  if (occ < 1 || gsmem > 220 * 1024) return bfail(QBX_EINVAL, "p too large for the group kernel");
  b->grid = std::min(b->n_items, b->num_sms * occ);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  GroupArgs ga{};
  ga.ops = b->ops;
  ga.p = b->p;
  ga.nrhs = b->nrhs;
  ga.inst = b->d_inst;
  ga.n_items = b->n_items;
  ga.items = b->d_items;
  ga.counter = b->d_counter;
  ga.eta2 = b->eta2;
  const void* gk = local ? group_ptr_local(b->ops, b->ck, rg)
                         : (b->ck ? group_ptr_cplx(b->ops, rg) : group_ptr_real(b->ops, rg));
  if (!gk) return bfail(QBX_EINVAL, "no group kernel for this operator set");
  e = cudaFuncSetAttribute(gk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem);
  if (e == cudaSuccess) e = cudaGraphCreate(&b->graph, 0);
  cudaGraphNode_t n_memset, n_up, n_group, n_fin;
  if (e == cudaSuccess) {
    cudaMemsetParams mp{};
    mp.dst = b->d_counter;
    mp.value = 0;
    mp.elementSize = sizeof(int);
    mp.width = 1;
    mp.height = 1;
    e = cudaGraphAddMemsetNode(&n_memset, b->graph, nullptr, 0, &mp);
  }
  int q_tgt = b->q_tgt, q_src = b->q_src, nr = b->nrhs, ncomp = b->ncomp, lim = b->limit, opsv = b->ops;
  const GroupInst* di = b->d_inst;
  const double* P = b->d_interp;
  int* st = b->d_status;
  if (e == cudaSuccess) {
    void* args[] = {(void*)&di, &q_tgt, &q_src, &nr, (void*)&P};
    cudaKernelNodeParams kp{};
    kp.func = (void*)k_batch_upsample;
    kp.gridDim = dim3((b->max_src * nr + 255) / 256, b->n_inst);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&n_up, b->graph, &n_memset, 1, &kp);
  }
  if (e == cudaSuccess) {
    void* args[] = {&ga};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(gk);
    kp.gridDim = dim3(b->grid);
    kp.blockDim = dim3(kGrpCentres * kGrpWarps);
    kp.sharedMemBytes = (unsigned)gsmem;
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&n_group, b->graph, &n_up, 1, &kp);
  }
  if (e == cudaSuccess) {
    void* args[] = {(void*)&di, &opsv, &ncomp, &lim, &nr, &st};
    cudaKernelNodeParams kp{};
    kp.func = (void*)k_batch_finish;
    kp.gridDim = dim3((b->max_tgt * ncomp * nr + 255) / 256, b->n_inst);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&n_fin, b->graph, &n_group, 1, &kp);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return bcuda(e, "graph construction");
  return QBX_OK;
}

// Tuned configurations, cached per (device, p, operators, side, nrhs, real or
// complex k, global or near-only, and the power-of-two buckets of the largest
// curve, the total pairs and the curve count): a batch created later with the
// same key starts from the measured choice instead of the model's.
typedef std::tuple<int, int, int, int, int, int, int, int, int, int> TuneKey;
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;

int log2i(double v) { return v < 1.0 ? 0 : (int)std::floor(std::log2(v)); }

TuneKey tune_key(const qbx_batch* b) {
  double pairs = 0.0;
  for (const GroupInst& in : b->h_inst) pairs += (double)in.n_ctr * in.n_src;
  return TuneKey{b->device, b->p, b->ops, b->side, b->nrhs, b->ck ? 1 : 0, b->eta2 > 0.0 ? 1 : 0,
                 log2i(b->max_src), log2i(pairs), log2i(b->n_inst)};
}

// partial-sum budget: a quarter of the free device memory
size_t part_budget(int device) {
  size_t fr = 0, tot = 0;
  cudaSetDevice(device);
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return (size_t)1 << 30;
  return fr / 4;
}

}  // namespace

extern "C" {

int qbx_batch_create(qbx_batch** batch, qbx_plan* plan, int n_inst, const qbx_geom* geoms, const qbx_c64* k,
                     int p, int ops, int side, int limit, int nrhs, const qbx_c64* const* dens,
                     qbx_c64* const* out) {
  if (!batch) return bfail(QBX_EINVAL, "batch out-pointer is NULL");
  *batch = nullptr;
  if (!plan) return bfail(QBX_EINVAL, "plan is NULL");
  if (n_inst < 1 || !geoms || !k || !dens || !out) return bfail(QBX_EINVAL, "empty batch or NULL table");
  if (ops != QBX_OPS_S && ops != QBX_OPS_D && ops != (QBX_OPS_S | QBX_OPS_D) &&
      ops != (QBX_OPS_S | QBX_OPS_D | QBX_OPS_GRAD_S))
    return bfail(QBX_EINVAL, "operator set must be S, D, S+D or S+D+grad S");
  if (side != QBX_SIDE_INT && side != QBX_SIDE_EXT && side != QBX_SIDE_TWO) return bfail(QBX_EINVAL, "bad side");
  if (limit != QBX_LIMIT_ONE_SIDED && limit != QBX_LIMIT_PV) return bfail(QBX_EINVAL, "bad limit");
  if (p < 0 || p > QBX_MAX_P) return bfail(QBX_EINVAL, "p outside [0, QBX_MAX_P]");
  if (nrhs < 1) return bfail(QBX_EINVAL, "nrhs < 1");
  qbx_batch* b = new qbx_batch();
  b->n_inst = n_inst;
  b->p = p;
  b->ops = ops;
  b->side = side;
  b->limit = limit;
  b->nrhs = nrhs;
  b->ncomp = (ops & 1) + ((ops >> 1) & 1) + 2 * ((ops >> 2) & 1);
  b->rg = nrhs > 8 ? 8 : 2;
  // the plan's device, grid pair and interpolation matrix
  int num_sms = 0;
  host_plan_info(plan, &b->device, &b->q_tgt, &b->q_src, &b->d_interp);
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    destroy(b);
    return bcuda(e, "device");
  }
  // ---- instances ----
  std::vector<GroupInst> inst(n_inst);
  size_t wd_total = 0;
  std::vector<size_t> wd_off(n_inst);
  for (int i = 0; i < n_inst; ++i) {
    const qbx_geom& g = geoms[i];
    if (g.q_tgt != b->q_tgt || g.q_src != b->q_src || g.M < 1 || g.n_tgt != g.M * g.q_tgt ||
        g.n_src != g.M * g.q_src || !g.src_x || !g.ctr_x || !g.tgt_x || !g.src_w) {
      destroy(b);
      return bfail(QBX_EINVAL, "geometry of an instance inconsistent with the plan");
    }
    if (!isfinite(k[i].re) || !isfinite(k[i].im) || k[i].im < 0.0 || (k[i].im == 0.0 && !(k[i].re > 0.0))) {
      destroy(b);
      return bfail(QBX_EINVAL, "k of an instance must be finite with Im k >= 0 (real k > 0)");
    }
    if (!dens[i]) {
      destroy(b);
      return bfail(QBX_EINVAL, "NULL density");
    }
    for (int o = 0; o < 3; ++o)
      if ((ops >> o & 1) && !out[3 * i + o]) {
        destroy(b);
        return bfail(QBX_EINVAL, "NULL output of a requested operator");
      }
    if (k[i].im != 0.0) b->ck = true;
    GroupInst& in = inst[i];
    in.kre = k[i].re;
    in.kim = k[i].im;
    in.n_src = g.n_src;
    in.n_tgt = g.n_tgt;
    in.M = g.M;
    in.side = side;
    in.n_ctr = side == QBX_SIDE_TWO ? 2 * g.n_tgt : g.n_tgt;
    const int c0 = side == QBX_SIDE_EXT ? g.n_tgt : 0;
    in.nsplit = 1;
    in.sx = g.src_x;
    in.sy = g.src_y;
    in.snx = g.src_nx;
    in.sny = g.src_ny;
    in.sw = g.src_w;
    in.cx = g.ctr_x + c0;
    in.cy = g.ctr_y + c0;
    in.tx = g.tgt_x;
    in.ty = g.tgt_y;
    in.tnx = g.tgt_nx;
    in.tny = g.tgt_ny;
    in.dens = dens[i];
    for (int o = 0; o < 3; ++o) in.out[o] = out[3 * i + o];
    wd_off[i] = wd_total;
    wd_total += host_align256((size_t)g.n_src * nrhs * 16);
    b->max_src = std::max(b->max_src, g.n_src);
    b->max_tgt = std::max(b->max_tgt, g.n_tgt);
  }
  b->num_sms = num_sms;
  b->h_inst = inst;
  // ---- device memory: instance table, densities, counter, status ----
  int n_ck = 0;
  for (int i = 0; i < n_inst; ++i) n_ck += inst[i].kim != 0.0 ? 1 : 0;
  e = cudaMalloc(&b->d_wd, wd_total);
  if (e == cudaSuccess && n_ck > 0) e = cudaMalloc(&b->d_hk, (size_t)n_ck * hk_table_doubles() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, sizeof(GroupInst) * n_inst);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    destroy(b);
    return bcuda(e, "allocation");
  }
  for (int i = 0; i < n_inst; ++i) b->h_inst[i].wd = static_cast<char*>(b->d_wd) + wd_off[i];
  // complex k: each curve's amplitude table (the k of a curve is fixed for the batch's life)
  for (int i = 0, j = 0; i < n_inst; ++i) {
    GroupInst& in = b->h_inst[i];
    in.hk_tab = nullptr;
    if (in.kim == 0.0) continue;
    double* t = b->d_hk + (size_t)(j++) * hk_table_doubles();
    e = launch_hk_table(in.kre, in.kim, t, 0);
    if (e != cudaSuccess) {
      destroy(b);
      return bcuda(e, "complex-k amplitude tables");
    }
    in.hk_tab = t;
  }
  e = cudaStreamSynchronize(0);   // made before any apply, on whatever stream it runs
  if (e != cudaSuccess) {
    destroy(b);
    return bcuda(e, "complex-k amplitude tables");
  }
  // ---- items: the source chunk the makespan model prefers ----
  const int occ = b->ck ? group_occupancy_cplx(ops, p, b->rg) : group_occupancy_real(ops, p, b->rg);
  if (occ < 1) {
    destroy(b);
    return bfail(QBX_EINVAL, "p too large for the group kernel");
  }
  int rg = b->rg, chunk = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(b));
    if (it != g_tune_cache.end()) {
      rg = it->second.first;
      chunk = it->second.second;
    }
  }
  if (chunk > 0) {   // a cached choice, if its partial sums fit
    std::vector<int> ns;
    make_items(b->h_inst, chunk, ns);
    if (part_bytes(b->h_inst, ns, b->ncomp, b->nrhs) > part_budget(b->device)) chunk = 0;
  }
  if (chunk == 0) {
    rg = b->rg;
    chunk = model_chunk(b, num_sms * occ, part_budget(b->device));
  }
  if (int rc = configure(b, rg, chunk)) {
    destroy(b);
    return rc;
  }
  *batch = b;
  return QBX_OK;
}

int qbx_batch_tune(qbx_batch* b, void* stream, int* rg_out, int* chunk_out) {
  if (!b) return bfail(QBX_EINVAL, "batch is NULL");
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bcuda(e, "device");
  cudaStream_t st = (cudaStream_t)stream;
  // candidates: the model's chunk and its neighbours, for the rhs groupings
  // that apply (8 rhs per warp needs more than 8 rhs to pay off)
  const size_t budget = part_budget(b->device) + b->part_cap;
  const int c0 = b->chunk;
  std::vector<int> chunks{c0};
  if (c0 / 2 >= 512) chunks.push_back(c0 / 2);
  if (c0 < b->max_src) chunks.push_back(std::min(2 * c0, (b->max_src + kGrpTile - 1) / kGrpTile * kGrpTile));
  std::vector<int> rgs{b->nrhs > 8 ? 8 : 2};
  if (b->nrhs > 2 && b->nrhs % 32 != 0) rgs.push_back(rgs[0] == 8 ? 2 : 8);
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return bcuda(e, "event");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bcuda(e, "event");
  }
  float best_ms = 1e30f;
  int best_rg = b->rg, best_chunk = c0;
  int rc = QBX_OK;
  for (int rg : rgs) {
    for (int c : chunks) {
      std::vector<int> ns;
      make_items(b->h_inst, c, ns);
      if (part_bytes(b->h_inst, ns, b->ncomp, b->nrhs) > budget) continue;
      if ((rc = configure(b, rg, c))) break;
      // one untimed launch, then one timed
      e = cudaGraphLaunch(b->exec, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        rc = bcuda(e, "tuning launch");
        break;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best_rg = rg;
        best_chunk = c;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = configure(b, best_rg, best_chunk))) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(b)] = std::make_pair(best_rg, best_chunk);
  }
  if (rg_out) *rg_out = best_rg;
  if (chunk_out) *chunk_out = best_chunk;
  return QBX_OK;
}

int qbx_batch_set_eta(qbx_batch* b, double eta) {
  if (!b) return bfail(QBX_EINVAL, "NULL batch");
  if (!(eta >= 0.0) || !isfinite(eta)) return bfail(QBX_EINVAL, "eta must be finite and >= 0");
  b->eta2 = eta * eta;
  return configure(b, b->rg, b->chunk);
}

int qbx_batch_info(const qbx_batch* b, int* rg, int* chunk, int* n_items, int* grid) {
  if (!b) return bfail(QBX_EINVAL, "batch is NULL");
  if (rg) *rg = b->rg;
  if (chunk) *chunk = b->chunk;
  if (n_items) *n_items = b->n_items;
  if (grid) *grid = b->grid;
  return QBX_OK;
}

int qbx_batch_apply(qbx_batch* b, void* stream) {
  if (!b) return bfail(QBX_EINVAL, "batch is NULL");
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return bcuda(e, "graph launch");
  return QBX_OK;
}

int qbx_batch_status(qbx_batch* b, void* stream) {
  if (!b) return bfail(QBX_EINVAL, "batch is NULL");
  int h = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bcuda(e, "status");
  if (h) return bfail(QBX_ENONFINITE, "a kernel produced a non-finite value");
  return QBX_OK;
}

int qbx_batch_destroy(qbx_batch* b) {
  destroy(b);
  return QBX_OK;
}

}  // extern "C"
