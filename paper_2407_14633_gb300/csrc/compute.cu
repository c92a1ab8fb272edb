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

#include "ctx.h"

namespace negf {

namespace {

int kernel_class(const Dev* d) { return d->block == 1 ? 0 : (d->block == 2 ? 1 : 2); }

struct Tune {
  int block_threads = 256;  // thread-per-lane kernels
  int blk_warps = 1;        // warps per CTA of the warp-per-lane kernel
};


}  // namespace


DeviceView make_view(Ctx* c, Dev* d, const ViewOverride* o) {
  (void)c;
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
    cv.kmax = ch.kmax;
    cv.hsq = (const double*)ch.dhsq.p;
    cv.g_b = ch.g_b;
    for (int s = 0; s < 2; ++s) {
      LeadView& lv = cv.lead[s];
      lv.m = ch.lead[s].m;
      lv.U = (o && o->zero_lead_U) ? 0.0 : ch.lead[s].U;
      lv.a1 = (const double*)ch.da1[s].p;
      lv.a2 = (const double*)ch.da2[s].p;
      lv.at = (const double*)ch.dat[s].p;
      lv.sites = (const int*)ch.dsites[s].p;
      lv.tw = (const double*)ch.dtw[s].p;
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
  for (DBuf* x : {&b.views, &b.items, &b.order, &b.counter, &b.partial, &b.tpart, &b.stage, &b.reduce, &b.status})
    c->arena.release(*x);
}

int build_plan(Ctx* c, const std::vector<Dev*>& devs, const std::vector<ViewOverride>* ov, int chain_only,
               Plan& P, PlanBufs* bufs) {
  cudaSetDevice(c->ordinal);
  const int nd = (int)devs.size();
  P = Plan();
  P.bufs = bufs ? bufs : &c->scratch;
  PlanBufs& B = *P.bufs;
  P.devs = devs;
  P.views.resize(nd);
  std::vector<WorkItem>& items = P.items;
  P.it0.assign(nd + 1, 0);
  long long part = 0, tpos = 0;
  std::vector<long long> tbase(nd);
  int Lmax[3] = {0, 0, 0}, bmax = 1, mmax = 1;
  for (int di = 0; di < nd; ++di) {
    Dev* d = devs[di];
    const ViewOverride* o = ov ? &(*ov)[di] : nullptr;
    P.views[di] = make_view(c, d, o);
    const DeviceView& v = P.views[di];
    const int cls = kernel_class(d);
    Lmax[cls] = std::max(Lmax[cls], d->L);
    if (cls == 2) {
      bmax = std::max(bmax, d->block);
      for (auto& ch : d->ch) mmax = std::max(mmax, std::max(ch.lead[0].m, ch.lead[1].m));
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
          W.pad = cls;
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
  P.bmax = bmax;
  P.mmax = mmax;

  // schedule order per kernel class: longest first
  std::vector<int> order[3];
  for (int i = 0; i < n_items; ++i) order[items[i].pad].push_back(i);
  for (int cls = 0; cls < 3; ++cls) {
    auto cost = [&](int i) {
      const Dev* d = devs[items[i].dev];
      return (double)d->L * (items[i].kind == 0 ? 2.0 : 1.0) * (double)d->block * d->block * d->block;
    };
    std::stable_sort(order[cls].begin(), order[cls].end(), [&](int a, int b) { return cost(a) > cost(b); });
  }
  std::vector<int> order_all;
  for (int cls = 0; cls < 3; ++cls) {
    P.ooff[cls] = (int)order_all.size();
    P.ncls[cls] = (int)order[cls].size();
    order_all.insert(order_all.end(), order[cls].begin(), order[cls].end());
  }

  // launch geometry and staging
  const Tune tune;
  P.block_threads = tune.block_threads;
  P.blk_warps = tune.blk_warps;
  size_t smem[3];
  smem[0] = smem[1] = (size_t)(tune.block_threads / 32) * 32 * 33 * sizeof(double);
  smem[2] = sweep_blk_smem_bytes(bmax, mmax, tune.blk_warps);
  P.stride[0] = (long long)Lmax[0] * 4 * 32 * 8;
  P.stride[1] = (long long)Lmax[1] * 12 * 32 * 8;
  P.stride[2] = (long long)Lmax[2] * (bmax * bmax + bmax * mmax) * 16;
  for (int cls = 0; cls < 3; ++cls) P.grid[cls] = 0;
  if (P.ncls[0]) P.grid[0] = c->sms * sweep_chain_occupancy(0, tune.block_threads, smem[0]);
  if (P.ncls[1]) P.grid[1] = c->sms * sweep_chain_occupancy(1, tune.block_threads, smem[1]);
  if (P.ncls[2]) {
    if (smem[2] > 227 * 1024) return set_err(c, NEGF_EINVAL, "ring block too wide for shared memory");
    P.grid[2] = c->sms * sweep_blk_occupancy(tune.blk_warps, smem[2]);
  }
  long long stage_bytes = 0;
  for (int cls = 0; cls < 3; ++cls) {
    if (!P.ncls[cls]) continue;
    const int wpb = cls == 2 ? tune.blk_warps : tune.block_threads / 32;
    const int need_blocks = (P.ncls[cls] + wpb - 1) / wpb;
    P.grid[cls] = std::max(1, std::min(P.grid[cls], need_blocks));
    stage_bytes = std::max(stage_bytes, P.stride[cls] * P.grid[cls] * wpb);
  }

  if (!ensure(c, B.views, sizeof(DeviceView) * nd) || !ensure(c, B.items, sizeof(WorkItem) * n_items) ||
      !ensure(c, B.order, sizeof(int) * n_items) || !ensure(c, B.counter, sizeof(int) * 4) ||
      !ensure(c, B.partial, sizeof(double) * std::max<long long>(part, 1)) ||
      !ensure(c, B.tpart, sizeof(double) * std::max<long long>(tpos, 1)) ||
      !ensure(c, B.stage, (size_t)std::max<long long>(stage_bytes, 16)) ||
      !ensure(c, B.reduce, sizeof(ReduceDev) * nd) || !ensure(c, B.status, sizeof(int)))
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
  // synchronous uploads: the host vectors die with this call
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(B.views.p, P.views.data(), sizeof(DeviceView) * nd, cudaMemcpyHostToDevice) ||
      cudaMemcpy(B.items.p, items.data(), sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice) ||
      cudaMemcpy(B.order.p, order_all.data(), sizeof(int) * n_items, cudaMemcpyHostToDevice) ||
      cudaMemcpy(B.reduce.p, rd.data(), sizeof(ReduceDev) * nd, cudaMemcpyHostToDevice))
    return set_err(c, NEGF_ECUDA, "upload of the launch plan failed");
  return NEGF_OK;
}

int launch_plan(Ctx* c, const Plan& P) {
  cudaStream_t s = c->stream;
  const PlanBufs& B = *P.bufs;
  if (cudaMemsetAsync(B.counter.p, 0, sizeof(int) * 4, s) != cudaSuccess ||
      cudaMemsetAsync(B.tpart.p, 0, sizeof(double) * std::max<long long>(P.tpos, 1), s) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "counter reset failed");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool timed = c->profile && cap == cudaStreamCaptureStatusNone;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timed) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  for (int cls = 0; cls < 3; ++cls) {
    if (!P.ncls[cls]) continue;
    SweepArgs a;
    a.devs = (const DeviceView*)B.views.p;
    a.items = (const WorkItem*)B.items.p;
    a.order = (const int*)B.order.p + P.ooff[cls];
    a.n_items = P.ncls[cls];
    a.counter = (int*)B.counter.p + cls;
    a.partial = (double*)B.partial.p;
    a.Tpart = (double*)B.tpart.p;
    a.resid = nullptr;
    a.stage = (unsigned char*)B.stage.p;
    a.stage_stride = P.stride[cls];
    a.status = (int*)B.status.p;
    int rc;
    if (cls == 0)
      rc = launch_sweep_b1_f64(a, P.grid[0], P.block_threads, s);
    else if (cls == 1)
      rc = launch_sweep_b2_f64(a, P.grid[1], P.block_threads, s);
    else
      rc = launch_sweep_blk_f64(a, P.bmax, P.mmax, P.grid[2], P.blk_warps, s);
    if (rc) return set_err(c, NEGF_ECUDA, "sweep launch failed");
    ++c->launches;
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
    if (o.flags && nr > 0) {
      if (o.on_device) {
        if (cudaMemsetAsync(o.flags, 0, (size_t)nr * 4, s)) return set_err(c, NEGF_ECUDA, "copy out failed");
      } else {
        memset(o.flags, 0, (size_t)nr * 4);
      }
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
