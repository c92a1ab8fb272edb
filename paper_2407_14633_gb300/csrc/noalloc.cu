// A no-allocation entry point: one NEGF evaluation of a single mode-space chain (1 x 1
// blocks) whose scratch -- work items, per-item partial ring sums, the forward-sweep
// staging, the lead data and the reduction descriptor -- lives in one fixed file-scope
// device array instead of memory the library allocates.
//
// Who needs it: callers that cannot call cudaMalloc from where they run, such as code
// inside a CUDA graph being built, allocator-free embedding hosts, or tools that hand the
// library only pre-registered buffers.  They still pass every input and output as device
// memory they own; this entry point allocates nothing and calls no allocating routine.
//
// The array (NOALLOC_SCRATCH_BYTES) is reserved on every GPU that loads the library,
// until process exit.  Its device address is looked up with the device current on every
// call made outside stream capture (a lookup is cheap and picks up a new address after a
// device reset reloaded the module); a call made while its stream is being captured uses the
// address of the device's last uncaptured call.  So make a first call on each device, and
// again after any cudaDeviceReset, before capturing one.  All calls
// share the array and it keeps the previous call's contents, so the set-up kernel clears
// what must start at zero (the work counter and the T(E) partials), and calls that overlap
// on the GPU (different streams, or different host threads on one device) race on it.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "../../include/negf.h"

namespace negf {

constexpr size_t NOALLOC_SCRATCH_BYTES = 32u << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {nullptr};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NoallocLayout {
  size_t view, rdesc, lead, gb, counter, items, order, tpart, partial, stage, end;
};

NoallocLayout layout(int n_items, int n_rings, int n_real, int warps) {
  NoallocLayout o;
  size_t p = 0;
  o.view = p;    p = align256(p + sizeof(DeviceView));
  o.rdesc = p;   p = align256(p + sizeof(ReduceDev));
  o.lead = p;    p = align256(p + 6 * sizeof(double));
  o.gb = p;      p = align256(p + 8 * sizeof(double));
  o.counter = p; p = align256(p + 4 * sizeof(int));
  o.items = p;   p = align256(p + (size_t)n_items * sizeof(WorkItem));
  o.order = p;   p = align256(p + (size_t)n_items * sizeof(int));
  o.tpart = p;   p = align256(p + (size_t)(n_real > 0 ? n_real : 1) * sizeof(double));
  o.partial = p; p = align256(p + (size_t)n_items * n_rings * sizeof(double));
  o.stage = p;   p = align256(p + (size_t)warps * n_rings * 4 * 32 * sizeof(double));
  o.end = p;
  return o;
}

// Fills the launch metadata inside the scratch and clears what must start at zero.
__global__ void noalloc_setup_kernel(unsigned char* base, NoallocLayout lo, DeviceView v, ReduceDev rd,
                                     double a1S, double a2S, double atS, double a1D, double a2D,
                                     double atD, double g_b, int items_real, int items_cont) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  const int n_items = items_real + items_cont;
  WorkItem* items = reinterpret_cast<WorkItem*>(base + lo.items);
  int* order = reinterpret_cast<int*>(base + lo.order);
  for (int i = tid; i < n_items; i += stride) {
    WorkItem W;
    W.dev = 0;
    W.chain = 0;
    W.kind = i < items_real ? 0 : 1;
    W.e0 = (i < items_real ? i : i - items_real) * LANES;
    const int ne = W.kind == 0 ? v.n_real : v.n_cont;
    W.ne = min(LANES, ne - W.e0);
    W.pad = 0;
    W.part = (long long)i * v.n_rings;
    W.tout = W.e0;
    items[i] = W;
    order[i] = i;
  }
  double* tpart = reinterpret_cast<double*>(base + lo.tpart);
  for (int k = tid; k < v.n_real; k += stride) tpart[k] = 0.0;
  if (tid == 0) {
    *reinterpret_cast<DeviceView*>(base + lo.view) = v;
    *reinterpret_cast<ReduceDev*>(base + lo.rdesc) = rd;
    double* ld = reinterpret_cast<double*>(base + lo.lead);
    ld[0] = a1S; ld[1] = a2S; ld[2] = atS; ld[3] = a1D; ld[4] = a2D; ld[5] = atD;
    double* gb = reinterpret_cast<double*>(base + lo.gb);
    for (int c = 0; c < 8; ++c) gb[c] = c == 0 ? g_b : 0.0;
    int* counter = reinterpret_cast<int*>(base + lo.counter);
    for (int c = 0; c < 4; ++c) counter[c] = 0;
  }
}

// Device address of the scratch for the current device: looked up again unless `s` is being
// captured (then the address of the last uncaptured call on this device; none is an error).
int scratch_address(cudaStream_t s, unsigned char** out) {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return NEGF_ECUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return NEGF_ECUDA;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (cs != cudaStreamCaptureStatusNone) {
    if (!g_noalloc_ptr[d]) return NEGF_EINVAL;   // no uncaptured call on this device yet
  } else {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return NEGF_ECUDA;
    }
    g_noalloc_ptr[d] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[d];
  return NEGF_OK;
}

}  // namespace
}  // namespace negf

using namespace negf;

extern "C" int negf_chain1_compute_noalloc(void* stream, int n_rings, const double* Hdiag, const double* U,
                                           const double* hsq, double g_b, const double* lead_S,
                                           const double* lead_D, int n_real, const double* E,
                                           const double* w, const double* fS, const double* fD, double eta,
                                           int n_cont, const double* z, const double* c, double* n,
                                           double* T, double* I) {
  if (n_rings < 1 || !Hdiag || !U || (n_rings > 1 && !hsq) || !(g_b > 0.0) || !lead_S || !lead_D || !n)
    return NEGF_EINVAL;
  if (n_real < 0 || n_cont < 0 || n_real + n_cont == 0) return NEGF_EINVAL;
  if (n_real > 0 && (!E || !w || !fS || !fD || !(eta > 0.0))) return NEGF_EINVAL;
  if (n_cont > 0 && (!z || !c)) return NEGF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  int rc = scratch_address(s, &base);
  if (rc) return rc;
  const int items_real = (n_real + LANES - 1) / LANES, items_cont = (n_cont + LANES - 1) / LANES;
  const int n_items = items_real + items_cont;
  // as many resident warps as items, occupancy and the fixed scratch allow
  const int threads = 256, wpb = threads / 32;
  const size_t smem = (size_t)wpb * 32 * 33 * sizeof(double);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = sweep_chain_occupancy(0, threads, smem);
  int blocks = std::min(sms * per_sm, (n_items + wpb - 1) / wpb);
  const NoallocLayout empty = layout(n_items, n_rings, n_real, 0);
  const size_t per_block = (size_t)wpb * n_rings * 4 * 32 * sizeof(double);
  if (empty.end + per_block > NOALLOC_SCRATCH_BYTES) return NEGF_ENOMEM;   // does not fit 32 MiB
  blocks = std::max(1, std::min<int>(blocks, (int)((NOALLOC_SCRATCH_BYTES - empty.end) / per_block)));
  const NoallocLayout lo = layout(n_items, n_rings, n_real, blocks * wpb);
  if (lo.end > NOALLOC_SCRATCH_BYTES) return NEGF_ENOMEM;

  DeviceView v;
  memset(&v, 0, sizeof(v));
  v.n_rings = n_rings;
  v.L = n_rings;
  v.b = 1;
  v.rpb = 1;
  v.n_chains = 1;
  v.U = U;
  v.n_real = n_real;
  v.E = E;
  v.w = w;
  v.fS = fS;
  v.fD = fD;
  v.eta = eta;
  v.n_cont = n_cont;
  v.z = reinterpret_cast<const cd*>(z);
  v.c = reinterpret_cast<const cd*>(c);
  ChainView& cv = v.ch[0];
  cv.Hdiag = reinterpret_cast<const cd*>(Hdiag);
  cv.hd_step = 1;
  cv.cp_step = 1;
  cv.hsq = n_rings > 1 ? hsq : U;   // never read when there is one ring
  cv.g_b = g_b;
  const double* ld = reinterpret_cast<const double*>(base + lo.lead);
  for (int side = 0; side < 2; ++side) {
    LeadView& L = cv.lead[side];
    L.m = 1;
    L.U = side ? lead_D[3] : lead_S[3];
    L.a1 = ld + 3 * side;
    L.a2 = ld + 3 * side + 1;
    L.at = ld + 3 * side + 2;
  }
  ReduceDev rd;
  memset(&rd, 0, sizeof(rd));
  rd.n_rings = n_rings;
  rd.n_real = n_real;
  rd.n_chains = 1;
  rd.it0 = 0;
  rd.it1 = n_items;
  rd.items = reinterpret_cast<const WorkItem*>(base + lo.items);
  rd.partial = reinterpret_cast<const double*>(base + lo.partial);
  rd.Tpart = reinterpret_cast<const double*>(base + lo.tpart);
  rd.g_b = reinterpret_cast<const double*>(base + lo.gb);
  rd.w = w;
  rd.fS = fS;
  rd.fD = fD;
  rd.n = n;
  rd.T = T;
  rd.I = I;
  noalloc_setup_kernel<<<std::max(1, std::min(64, (n_items + 255) / 256)), 256, 0, s>>>(
      base, lo, v, rd, lead_S[0], lead_S[1], lead_S[2], lead_D[0], lead_D[1], lead_D[2], g_b, items_real,
      items_cont);
  if (cudaGetLastError() != cudaSuccess) return NEGF_ECUDA;
  SweepArgs a;
  a.devs = reinterpret_cast<const DeviceView*>(base + lo.view);
  a.items = reinterpret_cast<const WorkItem*>(base + lo.items);
  a.order = reinterpret_cast<const int*>(base + lo.order);
  a.n_items = n_items;
  a.counter = reinterpret_cast<int*>(base + lo.counter);
  a.partial = reinterpret_cast<double*>(base + lo.partial);
  a.Tpart = reinterpret_cast<double*>(base + lo.tpart);
  a.resid = nullptr;
  a.growth = nullptr;
  a.stage = base + lo.stage;
  a.stage_stride = (long long)n_rings * 4 * 32 * sizeof(double);
  a.status = reinterpret_cast<int*>(base + lo.counter) + 3;
  a.lane_stats = nullptr;
  if (launch_sweep_b1_f64(a, blocks, threads, s)) return NEGF_ECUDA;
  if (launch_reduce(reinterpret_cast<const ReduceDev*>(base + lo.rdesc), 1, s)) return NEGF_ECUDA;
  return NEGF_OK;
}
