// One NEGF evaluation of a batch of devices (Eq. Rho, Eq. deviceCharacteristics).
//
// Planning: every (device, chain, kind, energy chunk) becomes a work item -- 32 energies
// for the thread-per-lane kernels (b <= 2), one energy for the warp-per-lane kernel
// (b > 2).  Items of a device are contiguous, so its second-stage reduction sums them in a
// fixed order; the persistent kernels pull items through an atomic counter in a
// longest-first schedule order, which balances uneven devices without touching results.
// Staging of the forward sweep is per resident warp, so its size is bounded by the grid,
// not by the batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "blk32.cuh"
#include "ctx.h"

namespace negf {

namespace {

int kernel_class(const Dev* d) { return d->block == 1 ? 0 : (d->block == 2 ? 1 : 2); }

// CTA width (warps, one item each) of the thread-per-lane (1 x 1, 2 x 2) sweeps when the
// autotuner has not picked one: small CTAs spread a batch evenly over the SMs (2048 items in
// 8-warp CTAs left 104 SMs with two CTAs and 48 with one; the eight-device mode-space case ran
// 10% faster at two warps).  Groups of at least one item per SM are tuned over 1, 2, 4, 8 warps.
constexpr int CHAIN_WARPS_DEFAULT = 2;
// shared memory of a thread-per-lane CTA: one 32 x 33 transpose buffer per warp, of the sweep's
// element type
size_t chain_smem(int warps, bool f32) { return (size_t)warps * 32 * 33 * (f32 ? sizeof(float) : sizeof(double)); }
// tuning key of a thread-per-lane group: item counts are bucketed by powers of two, so a serving
// loop whose batch changes step by step tunes once per bucket
int chain_bucket(int n) {
  int b = 0;
  while ((1 << (b + 1)) <= n) ++b;
  return b;
}

}  // namespace

// Waves of the sweep split along the channel: consecutive items whose staging fits cap (an
// item alone may exceed it and then forms a wave of its own).  Sets each item's first record
// and staging offset within its wave, fills `waves`, and returns the largest staging of a
// wave; *max_recs receives the most records any wave holds (the record buffer's size).
long long seg_partition(std::vector<SegItem>& seg, const std::vector<long long>& stage, long long cap,
                        std::vector<Plan::SegWave>& waves, long long* max_recs) {
  waves.clear();
  long long st = 0, rec = 0, r0 = 0, worst = 0, most = 0;
  int i0 = 0;
  for (int j = 0; j < (int)seg.size(); ++j) {
    if (j > i0 && st + stage[j] > cap) {
      waves.push_back({i0, j - i0, r0, rec});
      most = std::max(most, rec);
      r0 += rec;
      i0 = j;
      st = 0;
      rec = 0;
    }
    seg[j].rec0 = rec;
    seg[j].stage = st;
    st += stage[j];
    rec += seg[j].n_seg;
    worst = std::max(worst, st);
  }
  if (!seg.empty()) {
    waves.push_back({i0, (int)seg.size() - i0, r0, rec});
    most = std::max(most, rec);
  }
  if (max_recs) *max_recs = most;
  return worst;
}


DeviceView make_view(Ctx* c, Dev* d, const ViewOverride* o) {
  DeviceView v;
  memset(&v, 0, sizeof(v));
  v.n_rings = d->n_rings;
  v.L = d->L;
  v.b = d->block;
  v.rpb = d->rpb;
  v.n_chains = d->n_chains;
  v.U = (o && o->U) ? o->U : (const double*)d->dU.p;
  v.n_real = d->n_real;
  v.E = (const double*)d->dE.p;
  v.w = (const double*)d->dw.p;
  v.fS = (const double*)d->dfS.p;
  v.fD = (const double*)d->dfD.p;
  v.eta = d->eta;
  v.n_cont = d->n_cont;
  v.z = (const cd*)d->dz.p;
  v.c = (const cd*)d->dc.p;
  if (o && o->n_real >= 0) {
    v.n_real = o->n_real;
    v.E = o->E;
    v.w = o->w;
    v.fS = o->fS;
    v.fD = o->fD;
    v.eta = o->eta;
  }
  if (o && o->n_cont >= 0) {
    v.n_cont = o->n_cont;
    v.z = o->z;
    v.c = o->c;
  }
  for (int ci = 0; ci < d->n_chains; ++ci) {
    ChainData& ch = d->ch[ci];
    ChainView& cv = v.ch[ci];
    cv.Hdiag = (const cd*)ch.dHdiag.p;
    cv.Hup = (const cd*)ch.dHup.p;
    cv.cs_cnt = (const int*)ch.dcs_cnt.p;
    cv.cs_idx = (const int*)ch.dcs_idx.p;
    cv.cs_val = (const cd*)ch.dcs_val.p;
    cv.rs_cnt = (const int*)ch.drs_cnt.p;
    cv.rs_idx = (const int*)ch.drs_idx.p;
    cv.rs_val = (const cd*)ch.drs_val.p;
    cv.kmax = ch.kmax;
    cv.hd_step = ch.hd_step;
    cv.cp_step = ch.cp_step;
    cv.Hdiag_f = (const cf*)ch.dHdiag_f.p;
    cv.cs_val_f = (const cf*)ch.dcs_val_f.p;
    cv.rs_val_f = (const cf*)ch.drs_val_f.p;
    cv.hsq = (const double*)ch.dhsq.p;
    cv.hsq_f = (const float*)ch.dhsq_f.p;
    cv.diag_real = ch.diag_real ? 1 : 0;
    cv.hu = nullptr;   // set by build_plan for 1 x 1 chains
    cv.hu_f = nullptr;
    cv.g_b = ch.g_b;
    // complex symmetric Green's functions: real symmetric H blocks, real couplings and leads
    // whose circulant couplings have real first rows (their Sigma is then symmetric)
    bool lead_real = true;
    for (int s2 = 0; s2 < 2; ++s2)
      for (const std::vector<double>* f : {&ch.lead[s2].T1, &ch.lead[s2].T2, &ch.lead[s2].tau})
        for (size_t i = 1; i < f->size(); i += 2) lead_real = lead_real && (*f)[i] == 0.0;
    // (general leads take the general update: their Sigma comes from decimation)
    cv.sym = (ch.h_sym && lead_real && !ch.lead[0].gen && !ch.lead[1].gen && !c->opts.general_update) ? 1 : 0;
    for (int s = 0; s < 2; ++s) {
      LeadView& lv = cv.lead[s];
      lv.m = ch.lead[s].m;
      lv.U = (o && o->zero_lead_U) ? 0.0 : ch.lead[s].U;
      lv.a1 = (const double*)ch.da1[s].p;
      lv.a2 = (const double*)ch.da2[s].p;
      lv.at = (const double*)ch.dat[s].p;
      lv.sites = (const int*)ch.dsites[s].p;
      lv.tw = (const double*)ch.dtw[s].p;
      lv.gen = ch.lead[s].gen ? 1 : 0;   // per-energy blocks are attached by build_plan
      lv.gsig = nullptr;
      lv.gfac = nullptr;
    }
  }
  return v;
}

int check_ready(Ctx* c, Dev* d) {
  for (auto& ch : d->ch) {
    if (!ch.h_set) return set_err(c, NEGF_EINVAL, "hamiltonian not set");
    if (!ch.lead[0].set || !ch.lead[1].set) return set_err(c, NEGF_EINVAL, "leads not set");
  }
  if (!d->u_set) return set_err(c, NEGF_EINVAL, "potential not set");
  if (!d->grid_set) return set_err(c, NEGF_EINVAL, "energy grid not set");
  return NEGF_OK;
}

// Plan of one batched evaluation: host-side work items and schedule, uploaded to the
// context scratch.  launch_plan then issues only stream-ordered device work (counter
// reset, sweeps, second stage), so it can be captured in a CUDA graph and replayed.
void free_plan_bufs(Ctx* c, PlanBufs& b) {
  for (DBuf* x : {&b.views, &b.items, &b.order, &b.counter, &b.partial, &b.tpart, &b.stage, &b.reduce, &b.status,
                  &b.resid, &b.order2, &b.growth, &b.prep, &b.hu, &b.gen, &b.genjobs, &b.genstat,
                  &b.segitems, &b.recitem, &b.segrec, &b.flags, &b.edge})
    c->arena.release(*x);
}

// CTA width of the wide-block kernel: enough threads for the b x b products
static int blk_warps_for(int b) { return b <= 20 ? 1 : (b <= 28 ? 2 : 4); }

static bool item_f32(int kind, int prec) {
  return prec == NEGF_PREC_FP32 || (prec == NEGF_PREC_MIXED && kind == 0);
}
// group of an item: 0 (1x1), 1 (2x2), 2/3/4 (wide blocks, 1/2/4 warps), + 5 for FP32
static int group_of(int cls, int b, bool f32) {
  int g = cls < 2 ? cls : 2 + (blk_warps_for(b) == 1 ? 0 : (blk_warps_for(b) == 2 ? 1 : 2));
  return g + (f32 ? 5 : 0);
}
static int group_class(int g) { return std::min(g % 5, 2); }
static bool group_f32(int g) { return g >= 5; }

static SweepArgs group_args(const Plan& P, int g, const int* order, int n, double* resid, double* growth) {
  const PlanBufs& B = *P.bufs;
  SweepArgs a;
  a.devs = (const DeviceView*)B.views.p;
  a.items = (const WorkItem*)B.items.p;
  a.order = order;
  a.n_items = n;
  a.counter = (int*)B.counter.p + g;
  a.partial = (double*)B.partial.p;
  a.Tpart = (double*)B.tpart.p;
  a.resid = resid;
  a.growth = growth;
  a.stage = (unsigned char*)B.stage.p;
  a.stage_stride = P.stride[g % 5];
  a.status = (int*)B.status.p;
  a.lane_stats = nullptr;
  a.ring_cap = P.ring_cap;
  a.cap_ring = P.cap_ring;
  return a;
}

// Resident CTAs per SM of the wide-block sweep for n items on sms SMs when at most occ fit:
// the largest cap whose last wave is empty or at least half full.  A thin last wave leaves
// most SMs with one or two lanes, too few to keep the FP64 pipe busy.
static int cap_rule(long long n, int sms, int occ) {
  const double L = (double)n / sms;
  for (int cap = occ; cap > (occ + 1) / 2; --cap) {
    const double q = L - std::floor(L / cap) * cap;
    if (q < 1e-9 || q >= 0.5 * cap) return cap;
  }
  return occ;
}

// Wide-block sweep kernels: complex64 blocks that a tile class holds run the register-tiled
// kernel (sweep_block32.cu) at that class's width (at least the requested one); the rest run
// the shared-memory kernel of sweep_block.cu.
static int blk32_of(bool f32, int b, int m, int w) { return f32 ? blk32_class(b, m, w) : 0; }
static int blk_eff_width(bool f32, int b, int m, int w) {
  const int k = blk32_of(f32, b, m, w);
  return k ? k : w;
}
static size_t blk_smem(bool f32, int b, int m, int w) {
  const int k = blk32_of(f32, b, m, w);
  return k ? blk32_smem_bytes(k) : sweep_blk_smem_bytes_t(b, m, f32 ? 8 : 16, w);
}
static int blk_occupancy(bool f32, int w, int b, int m, bool fuse = false) {
  const int k = blk32_of(f32, b, m, w);
  return k ? blk32_occupancy(k, fuse ? 1 : 0) : sweep_blk_occupancy_t(f32, w, b, m);
}
static int blk_launch(bool f32, const SweepArgs& a, int b, int m, int grid, int w, cudaStream_t s) {
  const int k = blk32_of(f32, b, m, w);
  return k ? launch_blk32(a, grid, k, s) : launch_sweep_blk_t(f32, a, b, m, grid, w, s);
}
// staging bytes per layer of one wide-block lane: FP64 gL_l and R_l (the FP64 sweep and the
// mixed path's recompute), or the tiles of the complex64 kernel at width w
static long long blk_layer_bytes(bool f32, int b, int m, int w) {
  const int k = blk32_of(f32, b, m, w);
  return k ? blk32_stage_layer_bytes(k) : (long long)(b * b + b * m) * 16;
}

static int blk_occ(Ctx* c, bool f32, int w, int b, int m, bool fuse = false) {
  if (blk_smem(f32, b, m, w) > 227 * 1024) return 0;
  int occ = blk_occupancy(f32, w, b, m, fuse);
  if (c->opts.blk_ctas_per_sm > 0) occ = std::min(occ, c->opts.blk_ctas_per_sm);
  return occ;
}

// CTA width for a group of n lanes: the widest whose resident CTAs still hold every lane at
// once, so that a few lanes are spread over the warps of otherwise idle SMs (the arithmetic
// does not depend on the width); 0 when no width holds them all in one wave.
static int partial_wave_width(Ctx* c, bool f32, int b, int m, int n) {
  for (int w : {4, 2, 1}) {
    const int occ = blk_occ(c, f32, w, b, m);
    if (occ > 0 && (long long)n <= (long long)c->sms * occ) return w;
  }
  return 0;
}

// Autotuner of the wide-block sweep's launch shape: CTA width (1, 2, 4 warps) and resident
// CTAs per SM.  Every output element and every reduction of that kernel has an evaluation
// order that depends on neither, so the choice changes speed only.  The candidates are, per
// width, the occupancy limit and the cap of cap_rule; each runs the whole group (so that the
// last wave is measured too) after one single-item launch per width has loaded the kernel.
// The fastest is cached per (element type, b, m, items); trial outputs are overwritten by the
// real launch.
static int tune_width(Ctx* c, Plan& P, int g) {
  const PlanBufs& B = *P.bufs;
  const bool f32 = group_f32(g);
  const int n = P.ncls[g];
  const long long stride = P.stride[g % 5];
  const long long max_grid = stride > 0 ? (long long)(B.stage.bytes / stride) : 0;
  struct Cand {
    int w, cap, grid;
  };
  std::vector<Cand> cand;
  for (int w : {1, 2, 4}) {
    if (blk_eff_width(f32, P.gb[g], P.gm[g], w) != w) continue;   // the same kernel as a wider width
    const int occ = blk_occ(c, f32, w, P.gb[g], P.gm[g]);
    if (occ < 1) continue;
    for (int cap : {occ, cap_rule(n, c->sms, occ)}) {
      const int grid = (int)std::min<long long>(std::min<long long>((long long)c->sms * cap, n), max_grid);
      bool dup = grid < 1;
      for (const Cand& x : cand) dup = dup || (x.w == w && x.grid == grid);
      if (!dup) cand.push_back({w, cap, grid});
    }
  }
  if (cand.empty()) return NEGF_OK;
  cudaStream_t s = c->stream;
  const int* order = (const int*)B.order.p + P.ooff[g];
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "event creation failed");
  int rc = NEGF_OK;
  for (int w : {1, 2, 4}) {   // load each kernel once
    bool has = false;
    for (const Cand& x : cand) has = has || x.w == w;
    if (!has) continue;
    const SweepArgs a = group_args(P, g, order, 1, nullptr, nullptr);
    if (cudaMemsetAsync(a.counter, 0, sizeof(int), s) != cudaSuccess ||
        blk_launch(f32, a, P.gb[g], P.gm[g], 1, w, s)) {
      rc = set_err(c, NEGF_ECUDA, "tuning launch failed");
      break;
    }
    ++c->launches;
  }
  float best = 0.0f;
  int bi = -1;
  for (size_t i = 0; i < cand.size() && !rc; ++i) {
    const SweepArgs a = group_args(P, g, order, n, nullptr, nullptr);
    if (cudaMemsetAsync(a.counter, 0, sizeof(int), s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess ||
        blk_launch(f32, a, P.gb[g], P.gm[g], cand[i].grid, cand[i].w, s) ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = set_err(c, NEGF_ECUDA, "tuning launch failed");
      break;
    }
    ++c->launches;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (bi < 0 || ms < best) {
      best = ms;
      bi = (int)i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const Cand& x = cand[bi];
  c->blk_tuned[std::make_tuple((int)f32, P.gb[g], P.gm[g], n)] = std::make_pair(x.w, x.cap);
  c->blk_last[std::make_tuple((int)f32, P.gb[g], P.gm[g])] = std::make_pair(x.w, x.cap);
  P.gw[g] = x.w;
  P.gcap[g] = x.cap;
  P.grid[g] = std::max(1, x.grid);
  return NEGF_OK;
}

// CTA width of a thread-per-lane group (g of class 0 or 1): every width of 1, 2, 4, 8 warps
// runs the whole group twice under events (at the most resident CTAs the staging holds, one
// item per warp; the faster run counts), and the fastest width is cached per (class, element
// type, item-count bucket) if it beats the default width by more than 3%: smaller differences
// between widths are within the run-to-run spread of these sweeps.  The trials write the same
// outputs as the real launch.
static int tune_chain_width(Ctx* c, Plan& P, int g) {
  const PlanBufs& B = *P.bufs;
  const int cls = group_class(g);
  const bool f32 = group_f32(g);
  const int n = P.ncls[g];
  const long long max_warps = P.stride[g] > 0 ? (long long)(B.stage.bytes / P.stride[g]) : 0;
  struct Cand {
    int w, grid;
  };
  std::vector<Cand> cand;
  for (int w : {1, 2, 4, 8}) {
    const int occ = sweep_chain_occupancy_t(f32, cls, 32 * w, chain_smem(w, f32));
    const long long grid = std::min<long long>(std::min<long long>((long long)c->sms * occ, (n + w - 1) / w),
                                               max_warps / w);
    if (grid >= 1) cand.push_back({w, (int)grid});
  }
  if (cand.empty()) return NEGF_OK;
  cudaStream_t s = c->stream;
  const int* order = (const int*)B.order.p + P.ooff[g];
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "event creation failed");
  int rc = NEGF_OK;
  {   // load the kernel once
    const SweepArgs a = group_args(P, g, order, 1, nullptr, nullptr);
    if (cudaMemsetAsync(a.counter, 0, sizeof(int), s) != cudaSuccess ||
        (cls == 0 ? (f32 ? launch_sweep_b1_f32(a, 1, 32, s) : launch_sweep_b1_f64(a, 1, 32, s))
                  : (f32 ? launch_sweep_b2_f32(a, 1, 32, s) : launch_sweep_b2_f64(a, 1, 32, s))))
      rc = set_err(c, NEGF_ECUDA, "tuning launch failed");
    ++c->launches;
  }
  std::vector<float> tbest(cand.size(), -1.0f);
  for (size_t t = 0; t < 2 * cand.size() && !rc; ++t) {
    const size_t i = t % cand.size();
    const SweepArgs a = group_args(P, g, order, n, nullptr, nullptr);
    const int blk = 32 * cand[i].w;
    if (cudaMemsetAsync(a.counter, 0, sizeof(int), s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess ||
        (cls == 0 ? (f32 ? launch_sweep_b1_f32(a, cand[i].grid, blk, s) : launch_sweep_b1_f64(a, cand[i].grid, blk, s))
                  : (f32 ? launch_sweep_b2_f32(a, cand[i].grid, blk, s) : launch_sweep_b2_f64(a, cand[i].grid, blk, s))) ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = set_err(c, NEGF_ECUDA, "tuning launch failed");
      break;
    }
    ++c->launches;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (tbest[i] < 0.0f || ms < tbest[i]) tbest[i] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  int bi = 0, di = -1;
  for (size_t i = 0; i < cand.size(); ++i) {
    if (tbest[i] < tbest[bi]) bi = (int)i;
    if (cand[i].w == CHAIN_WARPS_DEFAULT) di = (int)i;
  }
  if (di >= 0 && bi != di && !(tbest[bi] < 0.97f * tbest[di])) bi = di;
  c->chain_tuned[std::make_tuple(cls, (int)f32, chain_bucket(n))] = cand[bi].w;
  c->chain_last[std::make_tuple(cls, (int)f32)] = cand[bi].w;
  P.gw[g] = cand[bi].w;
  P.grid[g] = cand[bi].grid;
  return NEGF_OK;
}

int build_plan(Ctx* c, const std::vector<Dev*>& devs, const std::vector<ViewOverride>* ov, int chain_only,
               Plan& P, PlanBufs* bufs) {
  cudaSetDevice(c->ordinal);
  const int nd = (int)devs.size();
  P = Plan();
  P.bufs = bufs ? bufs : &c->scratch;
  PlanBufs& B = *P.bufs;
  P.prec = c->opts.precision;
  P.devs = devs;
  P.views.resize(nd);
  std::vector<WorkItem>& items = P.items;
  P.it0.assign(nd + 1, 0);
  long long part = 0, tpos = 0;
  std::vector<long long>& tbase = P.tbase;
  tbase.assign(nd, 0);
  int Lmax[5] = {0, 0, 0, 0, 0};
  for (int g = 0; g < NGROUPS; ++g) {
    P.gb[g] = 1;
    P.gm[g] = 1;
    P.gw[g] = 1;
  }
  for (int di = 0; di < nd; ++di) {
    Dev* d = devs[di];
    const ViewOverride* o = ov ? &(*ov)[di] : nullptr;
    P.views[di] = make_view(c, d, o);
    const DeviceView& v = P.views[di];
    const int cls = kernel_class(d);
    const int g0 = group_of(cls, d->block, false);
    Lmax[g0] = std::max(Lmax[g0], d->L);
    if (cls == 2) {
      int mm = 1;
      for (auto& ch : d->ch) mm = std::max(mm, std::max(ch.lead[0].m, ch.lead[1].m));
      for (int f = 0; f < 2; ++f) {
        P.gb[g0 + 5 * f] = std::max(P.gb[g0 + 5 * f], d->block);
        P.gm[g0 + 5 * f] = std::max(P.gm[g0 + 5 * f], mm);
        P.gw[g0 + 5 * f] = blk_warps_for(d->block);
      }
    }
    const int chunk = (cls == 2 || (o && o->one_energy_per_item)) ? 1 : LANES;
    P.it0[di] = (int)items.size();
    tbase[di] = tpos;
    for (int ch = 0; ch < d->n_chains; ++ch) {
      if (chain_only >= 0 && ch != chain_only) continue;
      for (int kind = 0; kind < 2; ++kind) {
        const int ne = kind == 0 ? v.n_real : v.n_cont;
        for (int e0 = 0; e0 < ne; e0 += chunk) {
          WorkItem W;
          W.dev = di;
          W.chain = ch;
          W.kind = kind;
          W.e0 = e0;
          W.ne = std::min(chunk, ne - e0);
          W.pad = group_of(cls, d->block, item_f32(kind, c->opts.precision));
          W.part = part;
          W.tout = tpos + (long long)ch * v.n_real + e0;
          part += d->n_rings;
          items.push_back(W);
        }
      }
    }
    tpos += (long long)d->n_chains * std::max(v.n_real, 1);
  }
  P.it0[nd] = (int)items.size();
  const int n_items = (int)items.size();
  if (n_items == 0) return set_err(c, NEGF_EINVAL, "nothing to compute");
  P.n_items = n_items;
  P.tpos = tpos;

  // FP64 1 x 1 items of long channels with few energies are swept split along the channel
  // (sweep_seg.cu).  The rule looks at the device alone, never at the rest of the batch.
  std::vector<char> is_seg(n_items, 0);
  if (c->opts.long_chain_split >= 0) {
    for (int di = 0; di < nd; ++di) {
      if (devs[di]->block != 1) continue;
      int n64 = 0;
      for (int i = P.it0[di]; i < P.it0[di + 1]; ++i) n64 += items[i].pad == 0;
      const bool split = c->opts.long_chain_split == 1 || (P.views[di].L >= SEG_MIN_L && n64 <= SEG_MAX_ITEMS);
      if (!split) continue;
      for (int i = P.it0[di]; i < P.it0[di + 1]; ++i)
        if (items[i].pad == 0) {
          is_seg[i] = 1;
          SegItem S;
          S.item = i;
          S.n_seg = (P.views[di].L + SEG_LEN - 1) / SEG_LEN;
          S.rec0 = 0;
          S.stage = 0;
          P.seg.push_back(S);
        }
    }
    // the per-warp staging of the 1 x 1 groups is sized by the items they still run
    if (!P.seg.empty()) {
      Lmax[0] = 0;
      for (int i = 0; i < n_items; ++i)
        if (!is_seg[i] && (items[i].pad == 0 || items[i].pad == 5)) Lmax[0] = std::max(Lmax[0], P.views[items[i].dev].L);
    }
  }

  // band-edge flags of the mixed path: |E - U_lead - e| < window for an edge e of a lead
  // mode, e in {+-|sqrt(a1) - sqrt(a2)|, +-(sqrt(a1) + sqrt(a2))}
  if (P.prec == NEGF_PREC_MIXED) {
    P.edge_flag.assign(tpos, 0);
    const double win = c->opts.edge_window;
    for (int di = 0; di < nd; ++di) {
      Dev* d = devs[di];
      const DeviceView& v = P.views[di];
      if (!(ov && (*ov)[di].n_real >= 0)) {
        for (int ch = 0; ch < d->n_chains; ++ch) {
          for (int k = 0; k < v.n_real && k < (int)d->hE.size(); ++k) {
            bool near = false;
            for (int side = 0; side < 2 && !near; ++side) {
              const HostLead& Ld = d->ch[ch].lead[side];
              const double Ul = (ov && (*ov)[di].zero_lead_U) ? 0.0 : Ld.U;
              for (size_t j = 0; j < Ld.a1.size() && !near; ++j) {
                const double p = std::sqrt(Ld.a1[j]), q = std::sqrt(Ld.a2[j]);
                const double e[4] = {std::fabs(p - q), -std::fabs(p - q), p + q, -(p + q)};
                for (int t = 0; t < 4; ++t)
                  if (std::fabs(d->hE[k] - Ul - e[t]) < win) near = true;
              }
            }
            P.edge_flag[tbase[di] + (long long)ch * v.n_real + k] = near;
          }
        }
      }
    }
  }

  // schedule order per group: longest first
  std::vector<int> order[NGROUPS];
  for (int i = 0; i < n_items; ++i)
    if (!is_seg[i]) order[items[i].pad].push_back(i);
  for (int g = 0; g < NGROUPS; ++g) {
    auto cost = [&](int i) {
      const Dev* d = devs[items[i].dev];
      return (double)d->L * (items[i].kind == 0 ? 2.0 : 1.0) * (double)d->block * d->block * d->block;
    };
    std::stable_sort(order[g].begin(), order[g].end(), [&](int a, int b) { return cost(a) > cost(b); });
  }
  std::vector<int> order_all;
  for (int g = 0; g < NGROUPS; ++g) {
    P.ooff[g] = (int)order_all.size();
    P.ncls[g] = (int)order[g].size();
    order_all.insert(order_all.end(), order[g].begin(), order[g].end());
  }

  // CTA width of the wide-block groups: forced, cached from an earlier tuning, or the size
  // policy (tuned at the end of this call when the group fills the GPU)
  bool tune_g[NGROUPS] = {false};
  cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->stream, &capst);
  for (int g = 0; g < NGROUPS; ++g) {
    if (group_class(g) != 2 || !P.ncls[g]) continue;
    if (c->opts.blk_warps > 0) {
      P.gw[g] = c->opts.blk_warps;
    } else if (c->opts.blk_warps == 0) {
      auto it = c->blk_tuned.find(std::make_tuple((int)group_f32(g), P.gb[g], P.gm[g], P.ncls[g]));
      if (it != c->blk_tuned.end()) {
        P.gw[g] = it->second.first;
        P.gcap[g] = it->second.second;
      } else if (P.ncls[g] >= c->sms && capst == cudaStreamCaptureStatusNone) {
        tune_g[g] = true;
      } else if (P.ncls[g] < c->sms) {
        const int w = partial_wave_width(c, group_f32(g), P.gb[g], P.gm[g], P.ncls[g]);
        if (w) P.gw[g] = w;
      }
    }
  }

  // CTA width of the thread-per-lane groups: cached from an earlier tuning, tuned at the end of
  // this call (a group of at least one item per SM, autotuning on, not under capture), or the
  // default
  bool tune_chain[NGROUPS] = {false};
  for (int g = 0; g < NGROUPS; ++g) {
    if (group_class(g) == 2 || !P.ncls[g]) continue;
    P.gw[g] = c->opts.chain_warps > 0 ? c->opts.chain_warps : CHAIN_WARPS_DEFAULT;
    if (c->opts.chain_warps > 0 || c->opts.blk_warps != 0) continue;
    auto it = c->chain_tuned.find(std::make_tuple(group_class(g), (int)group_f32(g), chain_bucket(P.ncls[g])));
    if (it != c->chain_tuned.end())
      P.gw[g] = it->second;
    else if (P.ncls[g] >= c->sms && capst == cudaStreamCaptureStatusNone && !c->chain_tuning_off)
      tune_chain[g] = true;
  }

  // mixed path: the complex64 kernel of a wide-block group re-sweeps flagged lanes in FP64 in
  // the same CTA when the FP64 compact layout fits its shared memory and the group has enough
  // lanes per resident CTA for those re-sweeps to overlap with complex64 lanes of other CTAs:
  // a single-warp FP64 re-sweep takes several complex64 lane times, so a lane flagged near the
  // end of a short group would trail the launch (measured: with 3.4 lanes per CTA the fused
  // kernel took 1.25x the two passes).  The launch shape then follows the size policy.
  constexpr int FUSE_LANES_PER_CTA = 16;
  if (P.prec == NEGF_PREC_MIXED && c->opts.mixed_two_pass <= 0)
    for (int g = 5; g < NGROUPS; ++g) {
      if (group_class(g) != 2 || !P.ncls[g]) continue;
      const int w = blk_eff_width(true, P.gb[g], P.gm[g], P.gw[g]);
      if (!blk32_of(true, P.gb[g], P.gm[g], P.gw[g]) || !blk32_can_fuse(P.gb[g], P.gm[g], w)) continue;
      const long long slots = (long long)c->sms * blk_occ(c, true, w, P.gb[g], P.gm[g], true);
      if (c->opts.mixed_two_pass == 0 && P.ncls[g] < FUSE_LANES_PER_CTA * slots) continue;
      P.fuse[g] = 1;
      P.gw[g] = w;
      tune_g[g] = false;
    }

  // launch geometry and staging per group (staging sized for FP64 elements)
  long long stage_bytes = 0;
  for (int g = 0; g < NGROUPS; ++g) {
    const int cls = group_class(g);
    const int L = Lmax[g % 5];
    if (cls == 0) P.stride[g] = (long long)L * 5 * 32 * 8;
    else if (cls == 1) P.stride[g] = (long long)L * 12 * 32 * 8;
    else {
      // one stride serves the FP64 group g % 5 and its FP32 group g % 5 + 5 (whose items the
      // mixed path recomputes in FP64): the larger of their per-layer needs, at every width
      // the FP32 group may run (all trial widths when it is tuned)
      const int g5 = g % 5, gf = g5 + 5;
      long long per = blk_layer_bytes(false, P.gb[g5], P.gm[g5], 1);
      if (P.ncls[gf])
        for (int w : {1, 2, 4})
          if (tune_g[gf] || w == P.gw[gf]) per = std::max(per, blk_layer_bytes(true, P.gb[gf], P.gm[gf], w));
      P.stride[g] = (long long)L * per;
    }
    P.grid[g] = 0;
    if (!P.ncls[g]) continue;
    const bool f32 = group_f32(g);
    int per_sm, wpb;
    if (cls < 2) {
      per_sm = sweep_chain_occupancy_t(f32, cls, 32 * P.gw[g], chain_smem(P.gw[g], f32));
      wpb = P.gw[g];
      if (tune_chain[g])   // staging for the most resident warps of any trial width
        for (int w : {1, 2, 4, 8}) {
          const int occ = sweep_chain_occupancy_t(f32, cls, 32 * w, chain_smem(w, f32));
          const long long warps = std::min<long long>((long long)c->sms * occ * w, ((P.ncls[g] + w - 1) / w) * (long long)w);
          stage_bytes = std::max(stage_bytes, P.stride[g] * warps);
        }
    } else {
      const size_t sm = blk_smem(f32, P.gb[g], P.gm[g], P.gw[g]);
      if (sm > 227 * 1024) return set_err(c, NEGF_EINVAL, "ring block too wide for shared memory");
      const int occ = blk_occ(c, f32, P.gw[g], P.gb[g], P.gm[g], P.fuse[g] != 0);
      per_sm = P.gcap[g] > 0 ? std::min(occ, P.gcap[g]) : cap_rule(P.ncls[g], c->sms, occ);
      wpb = 1;   // one lane (item) per CTA
      if (tune_g[g]) {   // staging for the widest trial grid
        int occ_max = occ;
        for (int w : {1, 2, 4}) occ_max = std::max(occ_max, blk_occ(c, f32, w, P.gb[g], P.gm[g]));
        const int tgrid = std::max(1, std::min(c->sms * occ_max, P.ncls[g]));
        stage_bytes = std::max(stage_bytes, P.stride[g] * tgrid);
      }
    }
    const int need = cls < 2 ? (P.ncls[g] + wpb - 1) / wpb : P.ncls[g];
    P.grid[g] = std::max(1, std::min(c->sms * per_sm, need));
    stage_bytes = std::max(stage_bytes, P.stride[g] * P.grid[g] * wpb);
  }
  // the MIXED recompute runs flagged FP32 items of group g + 5 through FP64 group g,
  // with the FP32 group's grid and the FP64 group's staging stride and shared memory
  if (P.prec == NEGF_PREC_MIXED)
    for (int g = 0; g < 5; ++g) {
      if (!P.ncls[g + 5]) continue;
      const int cls = group_class(g);
      const int wpb = cls < 2 ? P.gw[g + 5] : 1;
      stage_bytes = std::max(stage_bytes, P.stride[g] * (long long)P.grid[g + 5] * wpb);
      if (cls == 2) {
        const size_t sm = sweep_blk_smem_bytes_t(P.gb[g], P.gm[g], 16, P.gw[g]);
        if (sm > 227 * 1024) return set_err(c, NEGF_EINVAL, "ring block too wide for shared memory");
        sweep_blk_occupancy_t(false, P.gw[g], P.gb[g], P.gm[g]);
      } else {
        sweep_chain_occupancy_t(false, cls, 32 * P.gw[g + 5], chain_smem(P.gw[g + 5], false));
      }
    }

  // split items in waves (seg_partition); the record buffer holds the largest wave's records
  std::vector<long long> seg_stage(P.seg.size());
  for (size_t j = 0; j < P.seg.size(); ++j) {
    const WorkItem& W = items[P.seg[j].item];
    seg_stage[j] = (long long)seg_stage_bytes(P.views[W.dev].L, W.kind);
  }
  long long seg_recs = 0;
  auto seg_waves = [&](long long cap) -> long long {
    return seg_partition(P.seg, seg_stage, cap, P.seg_waves, &seg_recs);
  };
  constexpr long long SEG_WAVE_BYTES = 4LL << 30;
  stage_bytes = std::max(stage_bytes, seg_waves(SEG_WAVE_BYTES));
  long long seg_rec_total = 0;
  for (const SegItem& S : P.seg) seg_rec_total += S.n_seg;
  auto segrec_size = [](long long recs) { return (size_t)std::max<long long>(recs * SEG_FIELDS * 32 * 8, 16); };
  size_t segrec_bytes = segrec_size(seg_recs);
  const size_t segitem_bytes = std::max<size_t>(sizeof(SegItem) * P.seg.size(), 16);
  const size_t recitem_bytes = (size_t)std::max<long long>(seg_rec_total * 4, 16);

  // layer diagonals of the 1 x 1 chains, formed once per launch by prep_kernel
  long long hu_elems = 0;
  int n_prep = 0, prep_L = 0;
  for (int di = 0; di < nd; ++di)
    if (devs[di]->block == 1) {
      hu_elems += (long long)devs[di]->n_chains * P.views[di].L;
      n_prep += devs[di]->n_chains;
      prep_L = std::max(prep_L, P.views[di].L);
    }
  const size_t hu_bytes = (size_t)std::max<long long>(hu_elems * 12, 16);
  const size_t prep_bytes = std::max<size_t>(sizeof(PrepDesc) * n_prep, 16);

  // Under an HBM budget the staging of the forward sweep (per resident warp / CTA) is what
  // adapts: resident CTAs are capped so that it fits beside everything else.
  if (c->arena.budget) {
    // a buffer that has to grow is released before its replacement is allocated
    auto extra = [](const DBuf& b, size_t need) -> long long {
      return need > b.bytes ? (long long)(need - b.bytes) : 0;
    };
    long long other = extra(B.views, sizeof(DeviceView) * nd) + extra(B.items, sizeof(WorkItem) * n_items) +
                      extra(B.order, sizeof(int) * n_items) + extra(B.partial, sizeof(double) * std::max<long long>(part, 1)) +
                      extra(B.tpart, sizeof(double) * std::max<long long>(tpos, 1)) + extra(B.reduce, sizeof(ReduceDev) * nd) +
                      extra(B.counter, sizeof(int) * 16) + extra(B.status, sizeof(int)) + extra(B.hu, hu_bytes) +
                      extra(B.prep, prep_bytes) + extra(B.segitems, segitem_bytes) + extra(B.recitem, recitem_bytes) +
                      extra(B.segrec, segrec_size(seg_rec_total));
    if (P.prec != NEGF_PREC_FP64)
      other += extra(B.resid, sizeof(double) * tpos) + extra(B.growth, sizeof(double) * tpos) + extra(B.order2, sizeof(int) * n_items);
    for (int di = 0; di < nd; ++di) {
      Dev* d = devs[di];
      const size_t nr8 = (size_t)d->n_rings * 8;
      other += extra(d->dT, sizeof(double) * std::max(P.views[di].n_real, 1)) + extra(d->dn, nr8) +
               extra(d->dnr, nr8) + extra(d->dnc, nr8) + extra(d->dI, 8) + extra(d->dgb, 64);
    }
    const long long cap = (long long)c->arena.budget - (long long)c->arena.used + (long long)B.stage.bytes - other;
    if (stage_bytes > cap) {
      stage_bytes = 0;
      for (int g = 0; g < NGROUPS; ++g) {
        if (!P.ncls[g]) continue;
        const int wpb = group_class(g) < 2 ? P.gw[g] : 1;
        // an FP32 group's grid also runs its FP64 recompute, with the FP64 stride
        const long long per = std::max(P.stride[g], P.stride[g % 5]) * wpb;
        const long long fit = per > 0 ? cap / per : 1;
        if (fit < 1) return set_err(c, NEGF_ENOMEM, "budget too small for one resident block of the sweep");
        P.grid[g] = (int)std::min<long long>(P.grid[g], fit);
        stage_bytes = std::max(stage_bytes, per * P.grid[g]);
      }
      if (!P.seg.empty()) {
        const long long sw = seg_waves(cap);
        if (sw > cap) return set_err(c, NEGF_ENOMEM, "budget too small for the staging of one split chain");
        stage_bytes = std::max(stage_bytes, sw);
        segrec_bytes = segrec_size(seg_recs);   // the records of the final partition's largest wave
      }
    }
  }
  if (!ensure(c, B.views, sizeof(DeviceView) * nd) || !ensure(c, B.items, sizeof(WorkItem) * n_items) ||
      !ensure(c, B.order, sizeof(int) * n_items) || !ensure(c, B.counter, sizeof(int) * 16) ||
      !ensure(c, B.partial, sizeof(double) * std::max<long long>(part, 1)) ||
      !ensure(c, B.tpart, sizeof(double) * std::max<long long>(tpos, 1)) ||
      !ensure(c, B.stage, (size_t)std::max<long long>(stage_bytes, 16)) ||
      !ensure(c, B.reduce, sizeof(ReduceDev) * nd) || !ensure(c, B.status, sizeof(int)) ||
      !ensure(c, B.hu, hu_bytes) || !ensure(c, B.prep, prep_bytes) ||
      (!P.seg.empty() && (!ensure(c, B.segitems, segitem_bytes) || !ensure(c, B.recitem, recitem_bytes) ||
                          !ensure(c, B.segrec, segrec_bytes))) ||
      (P.prec != NEGF_PREC_FP64 && (!ensure(c, B.resid, sizeof(double) * std::max<long long>(tpos, 1)) ||
                                    !ensure(c, B.growth, sizeof(double) * std::max<long long>(tpos, 1)) ||
                                    !ensure(c, B.order2, sizeof(int) * n_items))))
    return NEGF_ENOMEM;
  bool any_fuse = false;
  for (int g = 0; g < NGROUPS; ++g) any_fuse = any_fuse || P.fuse[g];
  if (any_fuse && (!ensure(c, B.flags, sizeof(int) * std::max<long long>(tpos, 1)) ||
                   !ensure(c, B.edge, (size_t)std::max<long long>(tpos, 16))))
    return NEGF_ENOMEM;
  std::vector<ReduceDev> rd(nd);
  for (int di = 0; di < nd; ++di) {
    Dev* d = devs[di];
    const DeviceView& v = P.views[di];
    const size_t nr = (size_t)std::max(v.n_real, 1);
    if (!ensure(c, d->dn, d->n_rings * 8) || !ensure(c, d->dnr, d->n_rings * 8) ||
        !ensure(c, d->dnc, d->n_rings * 8) || !ensure(c, d->dT, nr * 8) || !ensure(c, d->dI, 8) ||
        !ensure(c, d->dgb, 8 * 8))
      return NEGF_ENOMEM;
    double gb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int ci = 0; ci < d->n_chains; ++ci) gb[ci] = (chain_only < 0 || ci == chain_only) ? d->ch[ci].g_b : 0.0;
    if (cudaMemcpy(d->dgb.p, gb, sizeof(gb), cudaMemcpyHostToDevice) != cudaSuccess)
      return set_err(c, NEGF_ECUDA, "copy failed");
    ReduceDev& R = rd[di];
    R.n_rings = d->n_rings;
    R.n_real = v.n_real;
    R.n_chains = d->n_chains;
    R.it0 = P.it0[di];
    R.it1 = P.it0[di + 1];
    R.items = (const WorkItem*)B.items.p;
    R.partial = (const double*)B.partial.p;
    R.Tpart = (const double*)B.tpart.p + tbase[di];
    R.g_b = (const double*)d->dgb.p;
    R.w = v.w;
    R.fS = v.fS;
    R.fD = v.fD;
    R.n = (double*)d->dn.p;
    R.n_real_part = (double*)d->dnr.p;
    R.n_cont = (double*)d->dnc.p;
    R.T = (double*)d->dT.p;
    R.I = (double*)d->dI.p;
  }
  std::vector<PrepDesc> prep;
  {
    double* hud = (double*)B.hu.p;
    float* huf = (float*)(hud + hu_elems);
    long long off = 0;
    for (int di = 0; di < nd; ++di) {
      if (devs[di]->block != 1) continue;
      DeviceView& v = P.views[di];
      for (int ch = 0; ch < v.n_chains; ++ch) {
        PrepDesc q;
        q.L = v.L;
        q.Hdiag = v.ch[ch].Hdiag;
        q.U = v.U;
        q.hu = hud + off;
        q.hu_f = huf + off;
        v.ch[ch].hu = q.hu;
        v.ch[ch].hu_f = q.hu_f;
        prep.push_back(q);
        off += v.L;
      }
    }
  }
  P.n_prep = n_prep;
  P.prep_L = prep_L;
  // general leads: Sigma and the factor of Gamma at every energy of each view, by decimation
  // (lead_general.cu), computed once per plan: the plan's energies and lead potentials are fixed
  std::vector<GenLeadJob> jobs;
  {
    long long gen_elems = 0;
    for (int di = 0; di < nd; ++di)
      for (int ch = 0; ch < devs[di]->n_chains; ++ch)
        for (int sd = 0; sd < 2; ++sd)
          if (devs[di]->ch[ch].lead[sd].gen) {
            const int m = devs[di]->ch[ch].lead[sd].m;
            gen_elems += 2LL * (P.views[di].n_real + P.views[di].n_cont) * m * m;
          }
    if (gen_elems > 0) {
      if (!ensure(c, B.gen, sizeof(cd) * gen_elems) || !ensure(c, B.genstat, sizeof(int))) return NEGF_ENOMEM;
      cd* base = (cd*)B.gen.p;
      long long off = 0;
      for (int di = 0; di < nd; ++di) {
        DeviceView& v = P.views[di];
        for (int ch = 0; ch < devs[di]->n_chains; ++ch)
          for (int sd = 0; sd < 2; ++sd) {
            const HostLead& HL = devs[di]->ch[ch].lead[sd];
            if (!HL.gen) continue;
            const long long ne = (long long)(v.n_real + v.n_cont) * HL.m * HL.m;
            GenLeadJob j;
            j.mats = (const cd*)devs[di]->ch[ch].dgen[sd].p;
            j.m = HL.m;
            j.U = v.ch[ch].lead[sd].U;   // zero under the neutral-charge override
            j.n_real = v.n_real;
            j.n_cont = v.n_cont;
            j.E = v.E;
            j.eta = v.eta;
            j.z = v.z;
            j.sig = base + off;
            j.fac = base + off + ne;
            j.max_iter = HL.max_iter;
            j.tol = HL.tol;
            v.ch[ch].lead[sd].gsig = j.sig;
            v.ch[ch].lead[sd].gfac = j.fac;
            jobs.push_back(j);
            off += 2 * ne;
          }
      }
      if (!ensure(c, B.genjobs, sizeof(GenLeadJob) * jobs.size())) return NEGF_ENOMEM;
    }
  }
  // synchronous uploads: the host vectors die with this call
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      (n_prep && cudaMemcpy(B.prep.p, prep.data(), sizeof(PrepDesc) * n_prep, cudaMemcpyHostToDevice)) ||
      cudaMemcpy(B.views.p, P.views.data(), sizeof(DeviceView) * nd, cudaMemcpyHostToDevice) ||
      cudaMemcpy(B.items.p, items.data(), sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice) ||
      (!order_all.empty() &&   // split items have no place in the schedule of the sweep groups
       cudaMemcpy(B.order.p, order_all.data(), sizeof(int) * order_all.size(), cudaMemcpyHostToDevice)) ||
      cudaMemcpy(B.reduce.p, rd.data(), sizeof(ReduceDev) * nd, cudaMemcpyHostToDevice) ||
      (any_fuse && (cudaMemset(B.edge.p, 0, (size_t)std::max<long long>(tpos, 16)) ||
                    (!P.edge_flag.empty() &&
                     cudaMemcpy(B.edge.p, P.edge_flag.data(), P.edge_flag.size(), cudaMemcpyHostToDevice)))))
    return set_err(c, NEGF_ECUDA, "upload of the launch plan failed");
  if (!P.seg.empty()) {
    // owner of every record, relative to its wave's first item
    std::vector<int> owner;
    owner.reserve((size_t)seg_rec_total);
    for (const Plan::SegWave& wv : P.seg_waves)
      for (int j = 0; j < wv.ni; ++j)
        owner.insert(owner.end(), (size_t)P.seg[wv.i0 + j].n_seg, j);
    if ((long long)owner.size() != seg_rec_total ||
        cudaMemcpy(B.segitems.p, P.seg.data(), sizeof(SegItem) * P.seg.size(), cudaMemcpyHostToDevice) ||
        cudaMemcpy(B.recitem.p, owner.data(), sizeof(int) * owner.size(), cudaMemcpyHostToDevice))
      return set_err(c, NEGF_ECUDA, "upload of the split-chain plan failed");
  }
  if (!jobs.empty()) {
    int max_e = 1, m_max = 1;
    for (const GenLeadJob& j : jobs) {
      max_e = std::max(max_e, j.n_real + j.n_cont);
      m_max = std::max(m_max, j.m);
    }
    int nonconv = 0;
    if (cudaMemcpy(B.genjobs.p, jobs.data(), sizeof(GenLeadJob) * jobs.size(), cudaMemcpyHostToDevice) ||
        cudaMemsetAsync(B.genstat.p, 0, sizeof(int), c->stream) ||
        launch_lead_general((const GenLeadJob*)B.genjobs.p, (int)jobs.size(), max_e, m_max, (int*)B.genstat.p,
                            c->stream) ||
        cudaMemcpyAsync(&nonconv, B.genstat.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) ||
        cudaStreamSynchronize(c->stream))
      return set_err(c, NEGF_ECUDA, "lead decimation failed");
    ++c->launches;
    if (nonconv) return set_err(c, NEGF_ENOTCONVERGED, "lead decimation did not converge at some energies");
  }
  for (int g = 0; g < NGROUPS; ++g)
    if (tune_g[g]) {
      int rc = tune_width(c, P, g);
      if (rc) return rc;
    }
  for (int g = 0; g < NGROUPS; ++g)
    if (tune_chain[g]) {
      int rc = tune_chain_width(c, P, g);
      if (rc) return rc;
    }
  return NEGF_OK;
}

static int launch_group(Ctx* c, const Plan& P, int g, const int* order, int n, int grid, double* resid,
                        double* growth, int warps = 0) {
  const int cls = group_class(g);
  const bool f32 = group_f32(g);
  SweepArgs a = group_args(P, g, order, n, resid, growth);
  if (c->profile && c->lane_stats.p) a.lane_stats = (unsigned long long*)c->lane_stats.p;
  if (P.fuse[g] && warps <= 0) {   // (a recompute launch passes its own width: never fused)
    const PlanBufs& B = *P.bufs;
    a.fuse = 1;
    a.fuse_bmax = P.gb[g];
    a.fuse_mmax = P.gm[g];
    a.flag_threshold = c->opts.flag_threshold;
    a.growth_threshold = c->opts.growth_threshold > 0.0 ? c->opts.growth_threshold : HUGE_VAL;
    a.edge = (const unsigned char*)B.edge.p;
    a.flags = (int*)B.flags.p;
  }
  cudaStream_t s = c->stream;
  int rc;
  if (cls == 0)
    rc = f32 ? launch_sweep_b1_f32(a, grid, 32 * (warps > 0 ? warps : P.gw[g]), s)
             : launch_sweep_b1_f64(a, grid, 32 * (warps > 0 ? warps : P.gw[g]), s);
  else if (cls == 1)
    rc = f32 ? launch_sweep_b2_f32(a, grid, 32 * (warps > 0 ? warps : P.gw[g]), s)
             : launch_sweep_b2_f64(a, grid, 32 * (warps > 0 ? warps : P.gw[g]), s);
  else
    rc = blk_launch(f32, a, P.gb[g], P.gm[g], grid, warps > 0 ? warps : P.gw[g], s);
  if (rc) return set_err(c, NEGF_ECUDA, "sweep launch failed");
  ++c->launches;
  return NEGF_OK;
}

// MIXED: the FP64 group g < 5 whose lanes (the contour lanes) join the recompute launch of
// the flagged real-axis lanes instead of a launch of their own: its complex64 partner group
// has lanes and re-sweeps them in a second pass.  Alone, a few dozen contour lanes are a thin
// partial wave that holds the GPU for a whole FP64 lane time.
static bool mixed_deferred(const Plan& P, int g) {
  return P.prec == NEGF_PREC_MIXED && g < 5 && P.ncls[g] && P.ncls[g + 5] && !P.fuse[g + 5];
}

// MIXED: read the FP32 residuals, flag real-axis lanes (sum-rule residual above the
// threshold, or a lead band edge within the window) and re-run the items holding them in
// FP64 into the same partial and T slots, followed in the same launch by the deferred FP64
// groups' lanes.
static int mixed_recompute(Ctx* c, Plan& P) {
  const PlanBufs& B = *P.bufs;
  cudaStream_t s = c->stream;
  P.resid.assign(P.tpos, 0.0);
  P.growth.assign(P.tpos, 0.0);
  if (cudaMemcpyAsync(P.resid.data(), B.resid.p, sizeof(double) * P.tpos, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(P.growth.data(), B.growth.p, sizeof(double) * P.tpos, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "mixed-precision sweep failed");
  const double thr = c->opts.flag_threshold;
  const double gthr = c->opts.growth_threshold > 0.0 ? c->opts.growth_threshold : HUGE_VAL;   // 0: off
  P.flags.assign(P.tpos, 0);
  bool any_fuse = false;
  for (int g = 0; g < NGROUPS; ++g) any_fuse = any_fuse || (P.fuse[g] && P.ncls[g]);
  std::vector<int> fused_flags;
  if (any_fuse) {   // lanes the complex64 kernel re-swept in FP64 itself
    fused_flags.assign(P.tpos, 0);
    if (cudaMemcpy(fused_flags.data(), B.flags.p, sizeof(int) * P.tpos, cudaMemcpyDeviceToHost) != cudaSuccess)
      return set_err(c, NEGF_ECUDA, "mixed-precision flags read failed");
  }
  std::vector<int> redo[5], late[5];
  for (int i = 0; i < P.n_items; ++i) {
    const WorkItem& W = P.items[i];
    if (W.pad < 5) {
      if (mixed_deferred(P, W.pad)) late[W.pad].push_back(i);
      continue;
    }
    if (W.kind != 0) continue;
    if (P.fuse[W.pad]) {
      for (int e = 0; e < W.ne; ++e) P.flags[W.tout + e] = fused_flags[W.tout + e];
      continue;
    }
    bool any = false;
    for (int e = 0; e < W.ne; ++e) {
      const long long t = W.tout + e;
      if (!(P.resid[t] <= thr) || !(P.growth[t] <= gthr) || (!P.edge_flag.empty() && P.edge_flag[t])) any = true;
    }
    if (any) {
      redo[W.pad - 5].push_back(i);
      for (int e = 0; e < W.ne; ++e) P.flags[W.tout + e] = 1;
    }
  }
  std::vector<int> all;
  int off[5];
  P.recomputed = 0;
  for (int g = 0; g < 5; ++g) {
    P.recomputed += (int)redo[g].size();
    // the real-axis lanes (the longer sweeps) first, then the deferred contour lanes
    redo[g].insert(redo[g].end(), late[g].begin(), late[g].end());
    off[g] = (int)all.size();
    all.insert(all.end(), redo[g].begin(), redo[g].end());
  }
  if (all.empty()) return NEGF_OK;
  if (cudaMemcpy(B.order2.p, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemsetAsync(B.counter.p, 0, sizeof(int) * 16, s) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "recompute upload failed");
  for (int g = 0; g < 5; ++g) {
    if (redo[g].empty()) continue;
    const int cls = group_class(g);
    const int n = (int)redo[g].size();
    // a thread-per-lane recompute runs at the FP32 group's CTA width and grid, which its
    // staging was sized for
    const int cw = cls < 2 ? P.gw[g + 5] : 1;
    const int grid = std::max(1, std::min(P.grid[g + 5], cls < 2 ? (n + cw - 1) / cw : n));
    // the flagged energies are usually a fraction of a wave: spread them over wider CTAs
    // when that still holds them all at once (else the FP64 group's own width)
    const int w = cls < 2 ? cw
                          : ((c->opts.blk_warps == 0) ? partial_wave_width(c, false, P.gb[g], P.gm[g], n) : 0);
    int rc = launch_group(c, P, g, (const int*)B.order2.p + off[g], n, grid, nullptr, nullptr, w);
    if (rc) return rc;
  }
  return NEGF_OK;
}

int launch_plan(Ctx* c, Plan& P) {
  cudaStream_t s = c->stream;
  const PlanBufs& B = *P.bufs;
  if (cudaMemsetAsync(B.counter.p, 0, sizeof(int) * 16, s) != cudaSuccess ||
      cudaMemsetAsync(B.tpart.p, 0, sizeof(double) * std::max<long long>(P.tpos, 1), s) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "counter reset failed");
  for (int g = 0; g < NGROUPS; ++g)
    if (P.fuse[g] && P.ncls[g]) {
      if (cudaMemsetAsync(B.flags.p, 0, sizeof(int) * std::max<long long>(P.tpos, 1), s) != cudaSuccess)
        return set_err(c, NEGF_ECUDA, "flag reset failed");
      break;
    }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool timed = c->profile && cap == cudaStreamCaptureStatusNone;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timed) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  if (P.n_prep) {
    if (launch_prep((const PrepDesc*)B.prep.p, P.n_prep, P.prep_L, s)) return set_err(c, NEGF_ECUDA, "prep launch failed");
    ++c->launches;
  }
  for (int g = 0; g < NGROUPS; ++g) {
    if (!P.ncls[g] || mixed_deferred(P, g)) continue;
    double* resid = group_f32(g) ? (double*)B.resid.p : nullptr;
    double* growth = group_f32(g) ? (double*)B.growth.p : nullptr;
    int rc = launch_group(c, P, g, (const int*)B.order.p + P.ooff[g], P.ncls[g], P.grid[g], resid, growth);
    if (rc) return rc;
  }
  for (const Plan::SegWave& wv : P.seg_waves) {
    SegArgs a;
    a.devs = (const DeviceView*)B.views.p;
    a.items = (const WorkItem*)B.items.p;
    a.segs = (const SegItem*)B.segitems.p + wv.i0;
    a.rec_item = (const int*)B.recitem.p + wv.r0;
    a.n_rec = wv.nr;
    a.n_segitems = wv.ni;
    a.rec = (double*)B.segrec.p;
    a.stage = (unsigned char*)B.stage.p;
    a.partial = (double*)B.partial.p;
    a.Tpart = (double*)B.tpart.p;
    a.ring_cap = P.ring_cap;
    a.cap_ring = P.cap_ring;
    if (launch_seg(a, s)) return set_err(c, NEGF_ECUDA, "split-chain sweep launch failed");
    c->launches += 5;
  }
  if (P.prec == NEGF_PREC_MIXED) {
    if (cap != cudaStreamCaptureStatusNone) return set_err(c, NEGF_EINVAL, "mixed precision cannot be captured");
    int rc = mixed_recompute(c, P);
    if (rc) return rc;
  } else if (P.prec == NEGF_PREC_FP32 && cap == cudaStreamCaptureStatusNone && P.want_diag) {
    P.resid.assign(P.tpos, 0.0);
    P.growth.assign(P.tpos, 0.0);
    if (cudaMemcpyAsync(P.resid.data(), B.resid.p, sizeof(double) * P.tpos, cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(P.growth.data(), B.growth.p, sizeof(double) * P.tpos, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
      return set_err(c, NEGF_ECUDA, "diagnostics read failed");
  }
  if (timed) {
    cudaEventRecord(e1, s);
    c->prof_events.emplace_back(e0, e1);
  }
  if (launch_reduce((const ReduceDev*)B.reduce.p, (int)P.devs.size(), s))
    return set_err(c, NEGF_ECUDA, "reduce launch failed");
  ++c->launches;
  return NEGF_OK;
}

int copy_out(Ctx* c, const Plan& P, const negf_out* outs) {
  cudaStream_t s = c->stream;
  for (size_t di = 0; di < P.devs.size(); ++di) {
    Dev* d = P.devs[di];
    const negf_out& o = outs[di];
    const cudaMemcpyKind k = o.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const int nr = P.views[di].n_real;
    if (o.n && cudaMemcpyAsync(o.n, d->dn.p, d->n_rings * 8, k, s)) return set_err(c, NEGF_ECUDA, "copy out failed");
    if (o.n_real_part && cudaMemcpyAsync(o.n_real_part, d->dnr.p, d->n_rings * 8, k, s)) return set_err(c, NEGF_ECUDA, "copy out failed");
    if (o.n_cont && cudaMemcpyAsync(o.n_cont, d->dnc.p, d->n_rings * 8, k, s)) return set_err(c, NEGF_ECUDA, "copy out failed");
    if (o.T && nr > 0 && cudaMemcpyAsync(o.T, d->dT.p, (size_t)nr * 8, k, s)) return set_err(c, NEGF_ECUDA, "copy out failed");
    if (o.I && cudaMemcpyAsync(o.I, d->dI.p, 8, k, s)) return set_err(c, NEGF_ECUDA, "copy out failed");
    // per-energy flags / residuals / growth over the chains (host summaries of the precision path)
    if ((o.flags || o.resid || o.growth) && nr > 0) {
      std::vector<int> fl(nr, 0);
      std::vector<double> rs(nr, 0.0), gr(nr, 0.0);
      for (int ch = 0; ch < d->n_chains; ++ch)
        for (int e = 0; e < nr; ++e) {
          const long long t = P.tbase[di] + (long long)ch * nr + e;
          if (!P.flags.empty()) fl[e] |= P.flags[t];
          if (!P.resid.empty()) rs[e] = std::max(rs[e], P.resid[t]);
          if (!P.growth.empty()) gr[e] = std::max(gr[e], P.growth[t]);
        }
      if (o.growth && cudaMemcpyAsync(o.growth, gr.data(), (size_t)nr * 8, o.on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s))
        return set_err(c, NEGF_ECUDA, "copy out failed");
      if (o.flags && cudaMemcpyAsync(o.flags, fl.data(), (size_t)nr * 4, o.on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s))
        return set_err(c, NEGF_ECUDA, "copy out failed");
      if (o.resid && cudaMemcpyAsync(o.resid, rs.data(), (size_t)nr * 8, o.on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s))
        return set_err(c, NEGF_ECUDA, "copy out failed");
      if (cudaStreamSynchronize(s) != cudaSuccess) return set_err(c, NEGF_ECUDA, "copy out failed");
    }
  }
  return NEGF_OK;
}

static int run_batch(Ctx* c, const std::vector<Dev*>& devs, const std::vector<ViewOverride>* ov,
                     const negf_out* outs, std::vector<WorkItem>* items_out,
                     std::vector<int>* dev_item0, int chain_only) {
  Plan P;
  int rc = build_plan(c, devs, ov, chain_only, P);
  if (rc) return rc;
  if (outs)
    for (size_t i = 0; i < devs.size(); ++i)
      if (outs[i].resid || outs[i].growth) P.want_diag = true;
  if ((rc = launch_plan(c, P))) return rc;
  if (outs && (rc = copy_out(c, P, outs))) return rc;
  if (items_out) *items_out = P.items;
  if (dev_item0) *dev_item0 = P.it0;
  return NEGF_OK;
}

int compute_batch(Ctx* c, const std::vector<Dev*>& devs, const std::vector<ViewOverride>* ov,
                  std::vector<double*>* n_out, bool sync_copy, const negf_out* outs) {
  (void)n_out;
  int rc = run_batch(c, devs, ov, outs, nullptr, nullptr, -1);
  if (rc) return rc;
  if (sync_copy && cudaStreamSynchronize(c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "kernel execution failed");
  return NEGF_OK;
}

}  // namespace negf

using namespace negf;

static Dev* find_dev(Ctx* c, int dev) {
  auto it = c->devs.find(dev);
  return it == c->devs.end() ? nullptr : it->second.get();
}
Dev* negf::find_device(Ctx* c, int dev) { return find_dev(c, dev); }

extern "C" {

int negf_compute(negf_ctx* c, const int* devs, int n_devs, negf_out* outs) {
  if (!c) return NEGF_EINVAL;
  if (!devs || !outs || n_devs < 1) return set_err(c, NEGF_EINVAL, "bad compute arguments");
  std::vector<Dev*> list;
  for (int i = 0; i < n_devs; ++i) {
    Dev* d = find_dev(c, devs[i]);
    if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
    if (d->sc) return set_err(c, NEGF_EBUSY, "device is in a self-consistent session");
    for (int j = 0; j < i; ++j)
      if (devs[j] == devs[i]) return set_err(c, NEGF_EINVAL, "device listed twice");
    int rc = check_ready(c, d);
    if (rc) return rc;
    if (!outs[i].n) return set_err(c, NEGF_EINVAL, "output n is required");
    list.push_back(d);
  }
  const bool on_dev = outs[0].on_device != 0;
  int rc = compute_batch(c, list, nullptr, nullptr, !on_dev, outs);
  return rc;
}

int negf_sample_lanes(negf_ctx* c, int dev, int k_real, const int* idx_real, double* AS, double* AD,
                      int k_cont, const int* idx_cont, double* G) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  int rc = check_ready(c, d);
  if (rc) return rc;
  if (k_real < 0 || k_cont < 0 || (k_real && (!idx_real || !AS || !AD)) || (k_cont && (!idx_cont || !G)))
    return set_err(c, NEGF_EINVAL, "bad sample arguments");
  for (int i = 0; i < k_real; ++i)
    if (idx_real[i] < 0 || idx_real[i] >= d->n_real) return set_err(c, NEGF_EINVAL, "sample index out of range");
  for (int i = 0; i < k_cont; ++i)
    if (idx_cont[i] < 0 || idx_cont[i] >= d->n_cont) return set_err(c, NEGF_EINVAL, "sample index out of range");
  cudaSetDevice(c->ordinal);
  // host copies of the grid nodes
  std::vector<double> Eh(std::max(d->n_real, 1)), zh(2 * std::max(d->n_cont, 1));
  cudaMemcpy(Eh.data(), d->dE.p, Eh.size() * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(zh.data(), d->dz.p, zh.size() * 8, cudaMemcpyDeviceToHost);
  const int NR = d->n_rings;
  if (AS) std::fill(AS, AS + (size_t)k_real * NR, 0.0);
  if (AD) std::fill(AD, AD + (size_t)k_real * NR, 0.0);
  if (G) std::fill(G, G + (size_t)2 * k_cont * NR, 0.0);
  DBuf bE, bw, bfa, bfb, bz, bc;
  auto cleanup = [&]() {
    for (DBuf* b : {&bE, &bw, &bfa, &bfb, &bz, &bc}) c->arena.release(*b);
  };
  for (int ch = 0; ch < d->n_chains; ++ch) {
    const double g = 2.0 * d->ch[ch].g_b;
    // passes: 0 -> Tr A_S, 1 -> Tr A_D (real), 2 -> Im Tr G, 3 -> Re Tr G (contour)
    for (int pass = 0; pass < 4; ++pass) {
      const bool realp = pass < 2;
      const int kk = realp ? k_real : k_cont;
      if (kk == 0) continue;
      std::vector<double> E(kk), w(kk, 2.0 * M_PI / g), fa(kk, pass == 0 ? 1.0 : 0.0), fb(kk, pass == 1 ? 1.0 : 0.0);
      std::vector<double> z(2 * kk), cc(2 * kk);
      for (int i = 0; i < kk; ++i) {
        if (realp) {
          E[i] = Eh[idx_real[i]];
        } else {
          z[2 * i] = zh[2 * idx_cont[i]];
          z[2 * i + 1] = zh[2 * idx_cont[i] + 1];
          cc[2 * i] = pass == 2 ? M_PI / g : 0.0;
          cc[2 * i + 1] = pass == 3 ? M_PI / g : 0.0;
        }
      }
      ViewOverride o;
      o.one_energy_per_item = true;
      if (realp) {
        if ((rc = upload(c, bE, E.data(), kk * 8)) || (rc = upload(c, bw, w.data(), kk * 8)) ||
            (rc = upload(c, bfa, fa.data(), kk * 8)) || (rc = upload(c, bfb, fb.data(), kk * 8))) {
          cleanup();
          return rc;
        }
        o.n_real = kk;
        o.E = (const double*)bE.p;
        o.w = (const double*)bw.p;
        o.fS = (const double*)bfa.p;
        o.fD = (const double*)bfb.p;
        o.eta = d->eta;
        o.n_cont = 0;
      } else {
        if ((rc = upload(c, bz, z.data(), kk * 16)) || (rc = upload(c, bc, cc.data(), kk * 16))) {
          cleanup();
          return rc;
        }
        o.n_real = 0;
        o.eta = d->eta;
        o.n_cont = kk;
        o.z = (const cd*)bz.p;
        o.c = (const cd*)bc.p;
      }
      std::vector<Dev*> one{d};
      std::vector<ViewOverride> ov{o};
      std::vector<WorkItem> items;
      std::vector<int> i0;
      if ((rc = run_batch(c, one, &ov, nullptr, &items, &i0, ch))) {
        cleanup();
        return rc;
      }
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cleanup();
        return set_err(c, NEGF_ECUDA, "sample sweep failed");
      }
      std::vector<double> part((size_t)items.size() * NR);
      cudaMemcpy(part.data(), c->scratch.partial.p, part.size() * 8, cudaMemcpyDeviceToHost);
      for (size_t it = 0; it < items.size(); ++it) {
        const WorkItem& W = items[it];
        for (int r = 0; r < NR; ++r) {
          const double v = part[it * NR + r];
          if (pass == 0) AS[(size_t)W.e0 * NR + r] += v;
          if (pass == 1) AD[(size_t)W.e0 * NR + r] += v;
          if (pass == 2) G[2 * ((size_t)W.e0 * NR + r) + 1] += v;
          if (pass == 3) G[2 * ((size_t)W.e0 * NR + r)] += v;
        }
      }
    }
  }
  cleanup();
  return NEGF_OK;
}

int negf_neutral_charge(negf_ctx* c, int dev, int n_cont, double E_B, double* n0) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  if (n_cont < 1 || !n0 || !(E_B < 0.0)) return set_err(c, NEGF_EINVAL, "bad neutral-charge arguments");
  for (auto& ch : d->ch)
    if (!ch.h_set || !ch.lead[0].set || !ch.lead[1].set) return set_err(c, NEGF_EINVAL, "device not built");
  cudaSetDevice(c->ordinal);
  // contour over [E_B, 0] with occupation 1: c_k = W_k z'_k
  std::vector<double> z(2 * n_cont), cz(2 * n_cont);
  contour_arc(E_B, 0.0, n_cont, z.data(), cz.data());
  int rc;
  DBuf bz, bc, bU;
  std::vector<double> zeroU(d->n_rings, 0.0);
  if ((rc = upload(c, bz, z.data(), z.size() * 8)) || (rc = upload(c, bc, cz.data(), cz.size() * 8)) ||
      (rc = upload(c, bU, zeroU.data(), zeroU.size() * 8))) {
    for (DBuf* b : {&bz, &bc, &bU}) c->arena.release(*b);
    return rc;
  }
  ViewOverride o;
  o.U = (const double*)bU.p;
  o.zero_lead_U = true;
  o.n_real = 0;
  o.n_cont = n_cont;
  o.z = (const cd*)bz.p;
  o.c = (const cd*)bc.p;
  std::vector<Dev*> one{d};
  std::vector<ViewOverride> ov{o};
  negf_out out;
  memset(&out, 0, sizeof(out));
  std::vector<double> tmp(d->n_rings);
  out.n = tmp.data();
  out.n_cont = n0;
  rc = run_batch(c, one, &ov, &out, nullptr, nullptr, -1);
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = set_err(c, NEGF_ECUDA, "neutral sweep failed");
  for (DBuf* b : {&bz, &bc, &bU}) c->arena.release(*b);
  return rc;
}

int negf_conductance(negf_ctx* c, const int* devs, int n_devs, double mu, double kT, double* G, double* T) {
  if (!c) return NEGF_EINVAL;
  if (!devs || !G || n_devs < 1 || !std::isfinite(mu) || !(kT > 0.0) || !std::isfinite(kT))
    return set_err(c, NEGF_EINVAL, "bad conductance arguments");
  std::vector<Dev*> list;
  for (int i = 0; i < n_devs; ++i) {
    Dev* d = find_dev(c, devs[i]);
    if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
    if (d->sc) return set_err(c, NEGF_EBUSY, "device is in a self-consistent session");
    for (int j = 0; j < i; ++j)
      if (devs[j] == devs[i]) return set_err(c, NEGF_EINVAL, "device listed twice");
    int rc = check_ready(c, d);
    if (rc) return rc;
    if (d->n_real < 1) return set_err(c, NEGF_EINVAL, "the conductance needs real-axis energies");
    list.push_back(d);
  }
  cudaSetDevice(c->ordinal);
  // T(E) needs the real-axis lanes only
  std::vector<ViewOverride> ov(n_devs);
  for (auto& o : ov) o.n_cont = 0;
  int rc = run_batch(c, list, &ov, nullptr, nullptr, nullptr, -1);
  if (rc) return rc;
  const size_t desc = (size_t)n_devs * sizeof(CondDev);
  if (!ensure(c, c->cond, desc + (size_t)n_devs * sizeof(double))) return NEGF_ENOMEM;
  double* gdev = reinterpret_cast<double*>(static_cast<unsigned char*>(c->cond.p) + desc);
  std::vector<CondDev> cds(n_devs);
  for (int i = 0; i < n_devs; ++i) {
    Dev* d = list[i];
    cds[i].n_real = d->n_real;
    cds[i].E = (const double*)d->dE.p;
    cds[i].w = (const double*)d->dw.p;
    cds[i].T = (const double*)d->dT.p;
    cds[i].mu = mu;
    cds[i].kT = kT;
    cds[i].G = gdev + i;
  }
  if (cudaMemcpyAsync(c->cond.p, cds.data(), desc, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "upload failed");
  if (launch_conductance((const CondDev*)c->cond.p, n_devs, c->stream))
    return set_err(c, NEGF_ECUDA, "conductance launch failed");
  ++c->launches;
  if (cudaMemcpyAsync(G, gdev, (size_t)n_devs * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "copy out failed");
  if (T) {
    size_t off = 0;
    for (Dev* d : list) {
      if (cudaMemcpyAsync(T + off, d->dT.p, (size_t)d->n_real * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return set_err(c, NEGF_ECUDA, "copy out failed");
      off += d->n_real;
    }
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return set_err(c, NEGF_ECUDA, "conductance failed");
  return NEGF_OK;
}

}  // extern "C"

namespace negf {
__global__ void fp64_fma_probe(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace negf

extern "C" {

int negf_profile(negf_ctx* c, int enable) {
  if (!c) return NEGF_EINVAL;
  c->profile = enable != 0;
  if (c->profile) {
    cudaSetDevice(c->ordinal);
    if (!ensure(c, c->lane_stats, 4 * sizeof(unsigned long long))) return NEGF_ENOMEM;
    if (cudaMemsetAsync(c->lane_stats.p, 0, 4 * sizeof(unsigned long long), c->stream) != cudaSuccess)
      return set_err(c, NEGF_ECUDA, "counter reset failed");
  }
  return NEGF_OK;
}

int negf_sweep_lanes(negf_ctx* c, uint64_t lanes[4]) {
  if (!c || !lanes) return NEGF_EINVAL;
  for (int i = 0; i < 4; ++i) lanes[i] = 0;
  if (!c->lane_stats.p) return NEGF_OK;
  cudaSetDevice(c->ordinal);
  unsigned long long h[4];
  if (cudaMemcpyAsync(h, c->lane_stats.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->lane_stats.p, 0, sizeof(h), c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "counter read failed");
  for (int i = 0; i < 4; ++i) lanes[i] = h[i];
  return NEGF_OK;
}

int negf_kernel_time(negf_ctx* c, double* sweep_ms, uint64_t* sweeps) {
  if (!c || !sweep_ms || !sweeps) return NEGF_EINVAL;
  cudaSetDevice(c->ordinal);
  for (auto& pr : c->prof_events) {
    float ms = 0.0f;
    if (cudaEventSynchronize(pr.second) != cudaSuccess || cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess)
      return set_err(c, NEGF_ECUDA, "event timing failed");
    c->prof_ms += ms;
    ++c->prof_count;
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  c->prof_events.clear();
  *sweep_ms = c->prof_ms;
  *sweeps = c->prof_count;
  c->prof_ms = 0.0;
  c->prof_count = 0;
  return NEGF_OK;
}

int negf_plan_seg_waves(int n, const long long* stage, const int* n_seg, long long cap, int* wave_of,
                        long long* max_stage, long long* max_records) {
  if (n < 0 || (n > 0 && (!stage || !n_seg || !wave_of)) || cap < 0) return NEGF_EINVAL;
  std::vector<SegItem> seg((size_t)n);
  std::vector<long long> st((size_t)n);
  for (int i = 0; i < n; ++i) {
    if (stage[i] < 0 || n_seg[i] < 1) return NEGF_EINVAL;
    seg[i].item = i;
    seg[i].n_seg = n_seg[i];
    st[i] = stage[i];
  }
  std::vector<Plan::SegWave> waves;
  long long recs = 0;
  const long long worst = seg_partition(seg, st, cap, waves, &recs);
  for (int w = 0; w < (int)waves.size(); ++w)
    for (int j = 0; j < waves[w].ni; ++j) wave_of[waves[w].i0 + j] = w;
  if (max_stage) *max_stage = worst;
  if (max_records) *max_records = recs;
  return NEGF_OK;
}

int negf_chain_width(negf_ctx* c, int fp32, int block, int* warps) {
  if (!c || !warps || (block != 1 && block != 2)) return NEGF_EINVAL;
  auto it = c->chain_last.find(std::make_tuple(block == 1 ? 0 : 1, fp32 ? 1 : 0));
  if (it == c->chain_last.end()) return NEGF_EINVAL;
  *warps = it->second;
  return NEGF_OK;
}

int negf_blk_width(negf_ctx* c, int fp32, int b, int m, int* warps, int* ctas_per_sm) {
  if (!c || !warps) return NEGF_EINVAL;
  auto it = c->blk_last.find(std::make_tuple(fp32 != 0 ? 1 : 0, b, m));
  if (it == c->blk_last.end()) return NEGF_EINVAL;
  *warps = it->second.first;
  if (ctas_per_sm) *ctas_per_sm = it->second.second;
  return NEGF_OK;
}

int negf_fp64_peak(negf_ctx* c, double* tflops) {
  if (!c || !tflops) return NEGF_EINVAL;
  cudaSetDevice(c->ordinal);
  const int blocks = c->sms * 8, threads = 256, iters = 4000;
  DBuf out;
  if (!ensure(c, out, (size_t)blocks * threads * 8)) return NEGF_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, c->stream);
    fp64_fma_probe<<<blocks, threads, 0, c->stream>>>((double*)out.p, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, c->stream);
    ++c->launches;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      c->arena.release(out);
      return set_err(c, NEGF_ECUDA, "probe failed");
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->arena.release(out);
  *tflops = 2.0 * 8.0 * (double)blocks * threads * iters / (best * 1e-3) / 1e12;
  return NEGF_OK;
}

}  // extern "C"
