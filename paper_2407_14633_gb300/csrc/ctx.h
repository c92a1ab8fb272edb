// Host-side state of the NEGF library: context, device arena, devices.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/negf.h"
#include "common.cuh"
#include "sweep_seg.cuh"

namespace negf {

// A device allocation owned by a context; freed with it.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Arena {
  size_t used = 0, budget = 0, peak = 0;
  long long allocs = 0;
  int fail_after = 0;  // host-side fault injection: the n-th allocation fails
  std::string err;
  bool alloc(DBuf& b, size_t bytes);
  void release(DBuf& b);
};

struct HostLead {
  int m = 0;
  double U = 0.0;
  std::vector<double> a1, a2;   // per-mode |lambda_j(T1)|^2, |lambda_j(T2)|^2 (band edges)
  std::vector<double> T1, T2, tau;  // first rows, 2m each
  std::vector<int> sites;
  bool set = false;
  // general lead (negf_set_lead_general): full m x m blocks H0, H1, T1, T2, tau (interleaved
  // complex, 2 m^2 doubles each), decimation limits
  bool gen = false;
  std::vector<double> gmats;   // H0 | H1 | T1 | T2 | tau
  int max_iter = 400;
  double tol = 1e-14;
};

struct ChainData {
  std::vector<double> Hdiag, Hup;  // interleaved complex
  double g_b = 1.0;
  bool h_set = false;
  bool h_sym = false;   // every H_ll real symmetric and every H_{l,l+1} real
  HostLead lead[2];
  // device copies
  DBuf dHdiag, dHup, dcs_cnt, dcs_idx, dcs_val, drs_cnt, drs_idx, drs_val, dhsq;
  DBuf dHdiag_f, dcs_val_f, drs_val_f, dhsq_f;   // FP32 copies for the complex64 sweeps
  bool diag_real = false;                        // Im H_ll = 0 everywhere
  int hd_step = 0, cp_step = 0;                  // layer steps of Hdiag and the sparse forms (0: uniform)
  DBuf da1[2], da2[2], dat[2], dsites[2], dtw[2];
  DBuf dgen[2];   // general leads: the five m x m blocks on the device
  int kmax = 0;
};

// Device scratch of one launch plan.  The context owns one for ad-hoc evaluations; a
// self-consistent session owns its own, so its captured graph never sees a buffer that a
// later call reallocated.
struct PlanBufs {
  DBuf views, items, order, counter, partial, tpart, stage, reduce, status, resid, order2, growth;
  DBuf prep, hu;   // layer diagonals of the 1 x 1 chains (descriptors, values)
  DBuf gen, genjobs, genstat;   // general leads: per-energy Sigma and Gamma factors, jobs, status
  DBuf segitems, recitem, segrec;   // chains split along the channel: items, record owners, records
  DBuf flags, edge;   // mixed path: per T slot, re-swept in FP64 in the complex64 kernel; band-edge marks
};

struct ScSession;

struct Dev {
  int n_rings = 0, block = 1, rpb = 1, n_chains = 1, L = 0;
  std::vector<ChainData> ch;
  std::vector<double> U;
  bool u_set = false;
  // grid (host copies) and spec
  int n_real = 0, n_cont = 0;
  double eta = 0.0;
  std::vector<double> hE;        // host copy of the real-axis nodes
  bool grid_set = false;
  bool spec_set = false;
  negf_grid_spec spec{};
  // device buffers
  DBuf dU, dE, dw, dfS, dfD, dz, dc, dgb;
  DBuf dn, dnr, dnc, dT, dI;
  ScSession* sc = nullptr;   // active self-consistent session (sc.cu)
  // semi-adaptive real-axis grid (adaptive.cu): settings, current clipped limits, segment sizes
  bool adaptive = false;
  negf_adaptive ad{};
  double l1 = 0.0, l2 = 0.0;
  int seg[3] = {0, 0, 0};
};

struct Ctx {
  int ordinal = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  negf_opts opts{};
  int sms = 0;
  Arena arena;
  std::map<int, std::unique_ptr<Dev>> devs;
  int next_dev = 1;
  std::string last_error;
  uint64_t launches = 0;
  // scratch of ad-hoc batched sweeps, grown on demand
  PlanBufs scratch;
  // kernel timing (negf_profile): event pairs around sweep launches outside graph capture
  bool profile = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  double prof_ms = 0.0;
  uint64_t prof_count = 0;
  DBuf lane_stats;   // 4 counters of negf_sweep_lanes
  DBuf cond;         // descriptors and outputs of negf_conductance
  DBuf refine;       // unit weights and the located peak of the semi-adaptive grid
  // launch shapes (CTA width, resident CTAs per SM) chosen by the autotuner of the
  // wide-block sweep, keyed by (element type, b, m, items); the latest per (type, b, m)
  std::map<std::tuple<int, int, int, int>, std::pair<int, int>> blk_tuned;
  std::map<std::tuple<int, int, int>, std::pair<int, int>> blk_last;
  // CTA width (warps) of the thread-per-lane sweeps chosen by the autotuner, keyed by (kernel
  // class, element type, item-count bucket); the latest per (class, element type)
  std::map<std::tuple<int, int, int>, int> chain_tuned;
  std::map<std::tuple<int, int>, int> chain_last;
  // set while the serving loop plans a step: its batch changes every few steps, and a trial of
  // every width at each new item-count bucket cost more than it saved (the default is kept)
  bool chain_tuning_off = false;
  // serving state (serve.cu)
  struct Serve* serve = nullptr;
  std::mutex serve_mu;
};

struct Serve;
void serve_free(Ctx* c);
int set_err(Ctx* c, int code, const std::string& msg);
int set_grid_internal(Ctx* c, Dev* d, const negf_grid* g);
void gl_rule(int n, std::vector<double>& x, std::vector<double>& w);
double fermi_host(double x, double kT);
// semi-adaptive grid (adaptive.cu): peak of the refinement ring's integrand with the device's
// current potential and grid, then the grid rebuilt around it
int refine_grid_internal(Ctx* c, Dev* d, double* E_s);
bool ensure(Ctx* c, DBuf& b, size_t bytes);
int upload(Ctx* c, DBuf& b, const void* src, size_t bytes);

// Compute one NEGF evaluation of a list of devices with optional view overrides.
struct ViewOverride {
  const double* U = nullptr;       // device pointer replacing the potential
  bool zero_lead_U = false;        // leads at zero potential
  // replacement grid (device pointers); n_real < 0 keeps the device grid
  int n_real = -1;
  const double *E = nullptr, *w = nullptr, *fS = nullptr, *fD = nullptr;
  double eta = 0.0;
  int n_cont = -1;
  const cd *z = nullptr, *c = nullptr;
  bool one_energy_per_item = false;
};
// Items are launched in groups: kernel class (1x1, 2x2, wide blocks by CTA width 1/2/4
// warps) x element type (FP64, FP32), ten groups.  The CTA width of a wide-block item follows
// from its own block size, so a device's arithmetic never depends on its batch.  MIXED runs
// real-axis lanes in FP32 and contour lanes in FP64, then re-runs flagged real-axis items in
// FP64 into the same partial slots.
constexpr int NGROUPS = 10;
struct Plan {
  PlanBufs* bufs = nullptr;
  std::vector<Dev*> devs;
  std::vector<DeviceView> views;
  std::vector<WorkItem> items;
  std::vector<int> it0;
  std::vector<long long> tbase;
  int prec = NEGF_PREC_FP64;
  int n_items = 0;
  int grid[NGROUPS] = {0}, ooff[NGROUPS] = {0}, ncls[NGROUPS] = {0};
  int gb[NGROUPS] = {0}, gm[NGROUPS] = {0}, gw[NGROUPS] = {0};   // bmax, mmax, warps of wide-block groups
  int gcap[NGROUPS] = {0};                                          // tuned resident CTAs per SM (0: rule)
  int fuse[NGROUPS] = {0};   // mixed path: the complex64 kernel of group g re-sweeps flagged lanes in FP64
  long long stride[NGROUPS] = {0};
  long long tpos = 0;
  std::vector<unsigned char> edge_flag;   // per real energy of each device (tbase order, chain 0)
  std::vector<int> flags;                 // per T slot after the MIXED recompute
  std::vector<double> resid;              // per T slot
  std::vector<double> growth;             // per T slot
  int recomputed = 0;
  bool want_diag = false;
  int n_prep = 0, prep_L = 0;             // prep_kernel descriptors and longest chain
  double* ring_cap = nullptr;             // per-energy contributions at ring cap_ring (1 x 1, 2 x 2)
  int cap_ring = -1;
  // FP64 1 x 1 items swept split along the channel (sweep_seg.cu), run in waves whose staging
  // fits the stage buffer
  struct SegWave {
    int i0, ni;          // range of SegItems
    long long r0, nr;    // range of records
  };
  std::vector<SegItem> seg;
  std::vector<SegWave> seg_waves;
};
int build_plan(Ctx* c, const std::vector<Dev*>& devs, const std::vector<ViewOverride>* ov, int chain_only,
               Plan& P, PlanBufs* bufs = nullptr);
void free_plan_bufs(Ctx* c, PlanBufs& b);
void sc_session_free(Ctx* c, Dev* d);
int launch_plan(Ctx* c, Plan& P);
int copy_out(Ctx* c, const Plan& P, const negf_out* outs);
int check_ready(Ctx* c, Dev* d);
Dev* find_device(Ctx* c, int dev);
int compute_batch(Ctx* c, const std::vector<Dev*>& devs, const std::vector<ViewOverride>* ov,
                  std::vector<double*>* n_out, bool sync_copy, const negf_out* outs);
DeviceView make_view(Ctx* c, Dev* d, const ViewOverride* o);

}  // namespace negf

struct negf_ctx : public negf::Ctx {};

namespace negf {
// every Ctx is created as a negf_ctx (negf_create); internal code calling the public API
inline negf_ctx* pub(Ctx* c) { return static_cast<negf_ctx*>(c); }
}  // namespace negf
