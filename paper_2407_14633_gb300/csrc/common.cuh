// Shared declarations of the NEGF CUDA library: complex arithmetic, the device views the
// kernels read, work items of the batched sweep, and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace negf {

// ---------------------------------------------------------------- complex arithmetic
template <typename T>
struct cx {
  T re, im;
};
using cd = cx<double>;
using cf = cx<float>;

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
// Every product that feeds a sum is an explicit fused multiply-add, so the compiler has no
// contraction left to choose and each template instantiation (CTA width, element type)
// evaluates it in the same bits.
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re));
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> scale(cx<T> a, T s) { return mk(a.re * s, a.im * s); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> conjg(cx<T> a) { return mk(a.re, -a.im); }
template <typename T>
__host__ __device__ __forceinline__ T abs2(cx<T> a) { return fma(a.re, a.re, a.im * a.im); }
// acc + a * b with fused multiply-adds (4 FMA)
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmac(cx<T> acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmac_cj(cx<T> acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
// acc - a * b (the negation folds into the multiply-adds)
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmsub(cx<T> acc, cx<T> a, cx<T> b) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
// 1 / a = conj(a) / |a|^2
template <typename T>
__host__ __device__ __forceinline__ cx<T> crecip(cx<T> a) {
  T s = T(1) / fma(a.re, a.re, a.im * a.im);
  return mk(a.re * s, -a.im * s);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> cvt(cd a);
template <>
__host__ __device__ __forceinline__ cd cvt<double>(cd a) { return a; }
template <>
__host__ __device__ __forceinline__ cf cvt<float>(cd a) { return mk((float)a.re, (float)a.im); }

// ---------------------------------------------------------------- limits
constexpr int MAX_BLOCK = 64;     // widest ring block
constexpr int MAX_LEAD = 64;      // widest lead ring
constexpr int LANES = 32;         // energies per warp item of the thread-per-lane sweep

// ---------------------------------------------------------------- device-side views
// One lead of one chain: the closed-form surface Green's function of every angular mode j
// needs a1_j = |lambda_j(T1)|^2, a2_j = |lambda_j(T2)|^2 and at_j = |lambda_j(tau)|^2.
struct LeadView {
  int m;            // sites of the lead ring
  double U;         // lead potential energy
  const double* a1; // m
  const double* a2; // m
  const double* at; // m
  const int* sites; // m site indices inside the boundary layer
  const double* tw; // 2m: cos, sin of 2 pi k / m (k = 0..m-1), interleaved
  // general (non-circulant) lead: Sigma and a factor L of Gamma = L L^dagger at every energy
  // of the view (real-axis energies first, then contour nodes), m x m each, from the
  // decimation kernel of the launch plan
  int gen;
  const cd* gsig;
  const cd* gfac;
};

// Decimation job of one general lead over every energy of one device view (lead_general.cu).
struct GenLeadJob {
  const cd* mats;   // H0, H1, T1, T2, tau: 5 m x m blocks (lead rings s0, s1; H_{s1,s0}, H_{s2,s1}, H_{s0,device})
  int m;
  double U;         // lead potential energy (added on both rings)
  int n_real, n_cont;
  const double* E;  // real-axis energies (E + i eta)
  double eta;
  const cd* z;      // contour nodes
  cd* sig;          // out: (n_real + n_cont) x m x m
  cd* fac;          // out: (n_real + n_cont) x m x m
  int max_iter;
  double tol;
};
constexpr int MAX_GEN_LEAD = 20;   // widest general lead ring (its two-ring layers are 2m wide)
int launch_lead_general(const GenLeadJob* jobs, int n_jobs, int max_energies, int m_max, int* status,
                        cudaStream_t s);

// One chain of one device.
struct ChainView {
  const cd* Hdiag;  // L*b*b, without potential
  const cd* Hup;    // (L-1)*b*b
  // padded sparse forms of H_{l,l+1}: row r: rs_cnt[l*b+r] entries (col rs_idx, val rs_val)
  // and column c: cs_cnt (row cs_idx, val cs_val); kmax entries per row/column
  const int* rs_cnt;
  const int* rs_idx;
  const cd* rs_val;
  const int* cs_cnt;
  const int* cs_idx;
  const cd* cs_val;
  int kmax;
  // elements between consecutive layers of Hdiag (b*b) and of the sparse forms' count arrays
  // (b; kmax times that for idx and val); 0 when every layer holds the same block, so that
  // the block sweeps read one L1-resident copy (the arrays still hold every layer)
  int hd_step, cp_step;
  const cf* Hdiag_f;  // complex64 copies of Hdiag, cs_val, rs_val (complex64 sweeps)
  const cf* cs_val_f;
  const cf* rs_val_f;
  const double* hsq; // block 1: |H_{l,l+1}|^2 per layer (L-1)
  const float* hsq_f; // its FP32 copy
  // block 1: Re H_ll + U_l per layer for this launch (FP64 and FP32), formed once per launch
  // by prep_kernel; null where the sweep forms it itself.  diag_real: Im H_ll = 0 everywhere.
  const double* hu;
  const float* hu_f;
  int diag_real;
  double g_b;
  int sym;           // real H blocks and real lead rows: every G_ll is complex symmetric
  LeadView lead[2];
};

struct DeviceView {
  int n_rings, L, b, rpb, n_chains;
  const double* U;        // n_rings potential energy per ring
  // real-axis grid
  int n_real;
  const double* E;
  const double* w;
  const double* fS;
  const double* fD;
  double eta;
  // contour grid
  int n_cont;
  const cd* z;
  const cd* c;
  ChainView ch[8];        // up to 8 chains (modes)
};

// A work item of the sweep: one warp handles up to LANES energies (thread-per-lane kernels)
// or one energy (warp-per-lane kernels) of one (device, chain, kind).
struct WorkItem {
  int dev;        // index into the DeviceView array of the launch
  int chain;
  int kind;       // 0 real axis, 1 contour
  int e0;         // first energy index of the kind
  int ne;         // number of energies
  int pad;
  long long part; // offset of this item's per-ring partial sums (n_rings doubles)
  long long tout; // offset of its T(E) outputs (real items) in the T-partial buffer
};

struct SweepArgs {
  const DeviceView* devs;
  const WorkItem* items;
  const int* order;       // schedule order of items (longest first)
  int n_items;
  int* counter;           // persistent-scheduling counter (zeroed before launch)
  double* partial;        // per-item per-ring partial sums
  double* Tpart;          // per-chain T(E)
  double* resid;          // per-lane sum-rule residual (may be null)
  double* growth;         // per-lane max |gL entry| over the forward sweep (may be null)
  unsigned char* stage;   // staging of the forward sweep, per resident warp
  long long stage_stride; // bytes per resident warp
  int* status;            // device error flag (0 ok)
  unsigned long long* lane_stats;  // per-form lane counts (profiling; may be null)
  // thread-per-lane sweeps: each real-axis lane's weighted contribution at ring cap_ring, one
  // slot per T slot (the integrand of the semi-adaptive grid); null when not wanted
  double* ring_cap = nullptr;
  int cap_ring = -1;
  // mixed precision, register-tiled complex64 sweep of wide blocks: a real-axis lane whose
  // residual exceeds flag_threshold, whose growth exceeds growth_threshold or whose energy is
  // flagged in edge (per T slot) is re-swept in FP64 by the same CTA (FP64 shared-memory layout
  // for fuse_bmax x fuse_mmax blocks), which sets flags[T slot] = 1
  int fuse = 0;
  int fuse_bmax = 0, fuse_mmax = 0;
  double flag_threshold = 0.0, growth_threshold = 0.0;
  const unsigned char* edge = nullptr;
  int* flags = nullptr;
};

// ---------------------------------------------------------------- launchers
// thread-per-lane sweep of 1x1 blocks (every chain of every item has b == 1)
int launch_sweep_b1_f64(const SweepArgs& a, int grid, int block, cudaStream_t s);
int launch_sweep_b1_f32(const SweepArgs& a, int grid, int block, cudaStream_t s);
// thread-per-lane sweep of 2x2 blocks
int launch_sweep_b2_f64(const SweepArgs& a, int grid, int block, cudaStream_t s);
int launch_sweep_b2_f32(const SweepArgs& a, int grid, int block, cudaStream_t s);
// warp-per-lane sweep of b x b blocks (b <= MAX_BLOCK) with smem matrices
int launch_sweep_blk_f64(const SweepArgs& a, int b_max, int m_max, int grid, int warps,
                         cudaStream_t s);
// shared memory of one CTA for element size esize (16: FP64, 8: FP32) and CTA width warps
__host__ __device__ size_t sweep_blk_smem_bytes_t(int b, int m, int esize, int warps);
__host__ __device__ bool sweep_blk_compact(int b, int m, int esize, int warps);
int launch_sweep_blk_t(bool fp32, const SweepArgs& a, int b_max, int m_max, int grid, int warps, cudaStream_t s);
// resident CTAs per SM of the block sweep (sets the dynamic shared memory limit first)
int sweep_blk_occupancy_t(bool fp32, int warps, int b, int m);
// resident CTAs per SM of a sweep kernel (sets the dynamic shared memory limit first)
int sweep_chain_occupancy(int cls, int threads, size_t smem);
int sweep_chain_occupancy_t(bool fp32, int cls, int threads, size_t smem);

struct ReduceDev {
  int n_rings, n_real, n_chains;
  int it0, it1;           // item range of the device
  const WorkItem* items;
  const double* partial;
  const double* Tpart;    // n_chains x n_real (base of the device)
  const double* g_b;      // per chain (device array)
  const double* w;
  const double* fS;
  const double* fD;
  double* n;              // outputs (device)
  double* n_real_part;
  double* n_cont;
  double* T;
  double* I;
};
int launch_reduce(const ReduceDev* devs, int n_devs, cudaStream_t s);

// Zero-bias conductance of one device (Eq. zeroBiasG): G = g_s (e^2/h) sum_k w_k T_k (-df/dE)(E_k - mu).
struct CondDev {
  int n_real;
  const double* E;
  const double* w;
  const double* T;   // transmission per energy, summed over chains with g_b
  double mu, kT;
  double* G;         // output (device)
};
int launch_conductance(const CondDev* devs, int n_devs, cudaStream_t s);

// Per-launch layer diagonals of the 1 x 1 chains: hu[l] = Re H_ll + U_l, hu_f its FP32 copy.
struct PrepDesc {
  int L;
  const cd* Hdiag;
  const double* U;
  double* hu;
  float* hu_f;
};
int launch_prep(const PrepDesc* descs, int n, int max_L, cudaStream_t s);

// per-layer potential added to diagonal blocks is applied inside the sweep kernels.

// self-consistency kernels
struct ScDev {
  int N, M;
  double zeta, tol, kappa, r, U_G, U_S, U_D;
  double* n_in;      // N
  double* n_in_old;  // N
  double* f_old;     // N
  double* V;         // M x N
  double* W;         // M x N (column j of W stored as row j)
  double* n0;        // N
  double* U;         // N (Poisson output -> sweep input)
  const double* n_out; // N (sweep output)
  double* hist;      // M
  int* m;            // Broyden counter
  int* state;        // 0 running, 1 converged, 2 limit reached
  double* cp;        // N scratch (Thomas)
};
int launch_broyden(const ScDev* devs, int n, cudaStream_t s);
int launch_poisson(const ScDev* devs, int n, cudaStream_t s);
int launch_gather_states(const ScDev* devs, int n, int* out, cudaStream_t s);

// host quadrature helper: the upper semicircle contour over [E_B, E_end]
void contour_arc(double E_B, double E_end, int n, double* z, double* zw);

}  // namespace negf
