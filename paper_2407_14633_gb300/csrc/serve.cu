// Serving: continuous batching of self-consistent solves (bias points of an I-V sweep).
//
// Requests queue on the host.  A scheduler step (negf_serve_step, also driven by
// negf_wait) retires finished or cancelled requests, admits queued ones in arrival order
// while their estimated device memory fits the budget, then advances every active request
// by one self-consistent iteration: one Poisson launch (a CTA per request), one batched
// NEGF sweep over all active devices (one work-item list, longest lanes first), one
// second-stage reduction and one Broyden launch (a CTA per request).  While the set of
// active requests is unchanged the step is replayed from a captured CUDA graph.  Requests that enter
// while others run join the next step, so their work overlaps on the GPU.  Each request's
// arithmetic -- its lanes, its partial sums, its reductions -- is the same alone and in any
// mix, so its result is bitwise the same.
#include <chrono>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <deque>

#include "ctx.h"

namespace negf {

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { Q_QUEUED = 0, Q_ACTIVE = 1, Q_DONE = 2, Q_FAILED = 3, Q_CANCELLED = 4 };

struct Req {
  uint64_t ticket = 0;
  int state = Q_QUEUED;
  int status = NEGF_OK;
  // request parameters
  int N = 0, n_tube = 17, n_real = 0, n_cont = 0;
  std::vector<int> modes;
  double t = -2.7, kT = 0.025, eta = 1e-6, E_B = -10.0;
  negf_bias bias{};
  negf_poisson pois{};
  negf_broyden br{};
  std::vector<double> U0;
  // device side while active
  int dev = 0;
  size_t bytes = 0;
  DBuf nin, nold, fold, V, W, n0, hist, m, state_d, cp;
  ScDev sd{};
  int iterations = 0;
  // results
  std::vector<double> n, U, T, history;
  double I = 0.0;
  int converged = 0;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
};

}  // namespace

struct Serve {
  uint64_t next_ticket = 1;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::map<uint64_t, Req*> all;
  size_t active_bytes = 0;
  PlanBufs bufs;
  Plan plan;
  bool plan_valid = false;
  DBuf sc_desc;
  DBuf states_d;                 // gathered state flags of the active solves
  int* states_h = nullptr;       // pinned host copy
  int states_cap = 0;
  // one scheduler step captured as a CUDA graph, replayed while the membership is unchanged
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_kernels = 0;
  void drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
  ~Serve() {
    drop_graph();
    if (states_h) cudaFreeHost(states_h);
    for (auto& kv : all) delete kv.second;
  }
};

void serve_free(Ctx* c) {
  Serve* s = c->serve;
  if (!s) return;
  for (Req* r : s->active) {
    for (DBuf* b : {&r->nin, &r->nold, &r->fold, &r->V, &r->W, &r->n0, &r->hist, &r->m, &r->state_d, &r->cp})
      c->arena.release(*b);
  }
  s->drop_graph();
  free_plan_bufs(c, s->bufs);
  c->arena.release(s->sc_desc);
  c->arena.release(s->states_d);
  delete s;
  c->serve = nullptr;
}

namespace {

Serve* serve_of(Ctx* c) {
  if (!c->serve) c->serve = new Serve();
  return c->serve;
}

// device memory of one request while active (its own buffers; the shared staging is the
// batch's and is bounded by the resident warps)
size_t request_bytes(const Req& r) {
  const size_t N = r.N, C = r.modes.size(), nr = r.n_real, nc = r.n_cont, M = r.br.M;
  const size_t items = C * ((nr + LANES - 1) / LANES + (nc + LANES - 1) / LANES);
  size_t b = 0;
  b += C * (N * 16 * 2 + N * 8 + N * 64);     // blocks, |h|^2, sparse form
  b += N * 8 * 4 + nr * 8 * 5 + nc * 32;      // U, outputs, grid
  b += items * N * 8 + C * nr * 8;            // partial sums, T partials
  b += C * N * 12 + C * 64;                   // per-launch layer diagonals and their descriptors
  b += 2 * M * N * 8 + 6 * N * 8 + M * 8;     // Broyden state
  return b;
}

void release_request(Ctx* c, Req* r) {
  for (DBuf* b : {&r->nin, &r->nold, &r->fold, &r->V, &r->W, &r->n0, &r->hist, &r->m, &r->state_d, &r->cp})
    c->arena.release(*b);
  if (r->dev) {
    negf_device_destroy(pub(c), r->dev);
    r->dev = 0;
  }
}

int activate(Ctx* c, Req* r) {
  int rc;
  const int N = r->N;
  const int nm = (int)r->modes.size();
  if ((rc = negf_device_create(pub(c), N, 1, 1, nm, &r->dev))) return rc;
  const double U_S = 0.0, U_D = -r->bias.V_DS;
  if ((rc = negf_build_cnt_modespace(pub(c), r->dev, r->n_tube, r->t, r->modes.data(), U_S, U_D))) return rc;
  negf_grid_spec gs;
  memset(&gs, 0, sizeof(gs));
  gs.mu_S = 0.0;
  gs.mu_D = -r->bias.V_DS;
  gs.kT = r->kT;
  gs.eta = r->eta;
  gs.E_B = r->E_B;
  gs.E_min = gs.E_max = gs.f1 = gs.f2 = NAN;
  gs.n_real = r->n_real;
  gs.n_cont = r->n_cont;
  gs.rule = NEGF_RULE_GAUSS;
  if ((rc = negf_set_grid_spec(pub(c), r->dev, &gs))) return rc;
  if (r->U0.empty()) {
    r->U0.resize(N);
    for (int i = 0; i < N; ++i) r->U0[i] = N > 1 ? U_D * i / (N - 1) : 0.0;
  }
  std::vector<double> n0(N), nin(N);
  if ((rc = negf_neutral_charge(pub(c), r->dev, r->n_cont, r->E_B, n0.data()))) return rc;
  const double rr = (r->pois.lam_nm / r->pois.dx_nm) * (r->pois.lam_nm / r->pois.dx_nm);
  const double U_G = r->pois.phi_gate - r->bias.V_GS;
  for (int i = 0; i < N; ++i) {
    const double left = i > 0 ? r->U0[i - 1] : U_S;
    const double right = i < N - 1 ? r->U0[i + 1] : U_D;
    nin[i] = n0[i] + ((1.0 + 2.0 * rr) * r->U0[i] - rr * (left + right) - U_G) / r->pois.kappa;
  }
  if ((rc = negf_set_potential(pub(c), r->dev, r->U0.data()))) return rc;
  const int M = r->br.M;
  if ((rc = upload(c, r->nin, nin.data(), N * 8)) || (rc = upload(c, r->n0, n0.data(), N * 8))) return rc;
  if (!ensure(c, r->nold, N * 8) || !ensure(c, r->fold, N * 8) || !ensure(c, r->V, (size_t)M * N * 8) ||
      !ensure(c, r->W, (size_t)M * N * 8) || !ensure(c, r->hist, M * 8) || !ensure(c, r->m, 4) ||
      !ensure(c, r->state_d, 4) || !ensure(c, r->cp, N * 8))
    return NEGF_ENOMEM;
  cudaMemset(r->nold.p, 0, N * 8);
  cudaMemset(r->fold.p, 0, N * 8);
  cudaMemset(r->V.p, 0, (size_t)M * N * 8);
  cudaMemset(r->W.p, 0, (size_t)M * N * 8);
  cudaMemset(r->hist.p, 0, M * 8);
  cudaMemset(r->m.p, 0, 4);
  cudaMemset(r->state_d.p, 0, 4);
  Dev* d = find_device(c, r->dev);
  // the sweep's outputs must exist before the descriptors point at them
  if (!ensure(c, d->dn, (size_t)N * 8)) return NEGF_ENOMEM;
  ScDev& s = r->sd;
  s.N = N;
  s.M = M;
  s.zeta = r->br.zeta;
  s.tol = r->br.tol;
  s.kappa = r->pois.kappa;
  s.r = rr;
  s.U_G = U_G;
  s.U_S = U_S;
  s.U_D = U_D;
  s.n_in = (double*)r->nin.p;
  s.n_in_old = (double*)r->nold.p;
  s.f_old = (double*)r->fold.p;
  s.V = (double*)r->V.p;
  s.W = (double*)r->W.p;
  s.n0 = (double*)r->n0.p;
  s.U = (double*)d->dU.p;
  s.n_out = (const double*)d->dn.p;
  s.hist = (double*)r->hist.p;
  s.m = (int*)r->m.p;
  s.state = (int*)r->state_d.p;
  s.cp = (double*)r->cp.p;
  return NEGF_OK;
}

void finish(Ctx* c, Req* r, int st) {
  Dev* d = find_device(c, r->dev);
  const int N = r->N;
  r->n.resize(N);
  r->U.resize(N);
  r->T.resize(r->n_real);
  r->history.resize(std::min(r->iterations, r->br.M));
  cudaMemcpy(r->n.data(), d->dn.p, N * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(r->U.data(), d->dU.p, N * 8, cudaMemcpyDeviceToHost);
  if (r->n_real) cudaMemcpy(r->T.data(), d->dT.p, (size_t)r->n_real * 8, cudaMemcpyDeviceToHost);
  if (!r->history.empty()) cudaMemcpy(r->history.data(), r->hist.p, r->history.size() * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(&r->I, d->dI.p, 8, cudaMemcpyDeviceToHost);
  r->converged = (st == 1);
  r->status = r->converged ? NEGF_OK : NEGF_ENOTCONVERGED;
  r->state = Q_DONE;
  r->t_done = now_s();
}

int step_locked(Ctx* c, Serve* s, int* n_active) {
  cudaSetDevice(c->ordinal);
  bool changed = false;
  // retire cancelled
  for (size_t i = 0; i < s->active.size();) {
    Req* r = s->active[i];
    if (r->state == Q_CANCELLED) {
      release_request(c, r);
      s->active_bytes -= r->bytes;
      s->active.erase(s->active.begin() + i);
      changed = true;
    } else {
      ++i;
    }
  }
  // admit in arrival order while the budget allows
  const size_t budget = c->opts.hbm_budget_bytes;
  bool released = false;
  while (!s->queue.empty()) {
    Req* r = s->queue.front();
    if (r->state == Q_CANCELLED) {
      s->queue.pop_front();
      continue;
    }
    const size_t need = request_bytes(*r);
    // room for eight warps of forward-sweep staging (8 x L layers x 1280 B; at least one
    // resident CTA of the thread-per-lane sweep)
    size_t Lmax = r->N;
    for (Req* q : s->active) Lmax = std::max<size_t>(Lmax, q->N);
    const size_t stage_min = Lmax * 8 * 5 * 32 * 8;
    const size_t margin = 1 << 20;   // plan descriptors, counters, allocation rounding
    if (budget && !s->active.empty() && s->active_bytes + need + stage_min + margin > budget) break;
    if (budget && !released) {
      // the batch plan is rebuilt after admission anyway; its staging is released first so
      // the set-up of the new request (its neutral charge) has room for its own sweep
      cudaStreamSynchronize(c->stream);
      s->drop_graph();
      free_plan_bufs(c, s->bufs);
      s->plan_valid = false;
      released = true;
    }
    s->queue.pop_front();
    r->bytes = need;
    int rc = activate(c, r);
    if (rc) {
      release_request(c, r);
      r->state = Q_FAILED;
      r->status = rc;
      r->t_done = now_s();
      continue;
    }
    r->state = Q_ACTIVE;
    r->t_start = now_s();
    s->active.push_back(r);
    s->active_bytes += need;
    changed = true;
  }
  // under a budget, the ad-hoc scratch used while admitting (neutral charges) is released
  // so the batch's own staging fits
  if (changed && budget) {
    cudaStreamSynchronize(c->stream);
    free_plan_bufs(c, c->scratch);
  }
  *n_active = (int)s->active.size();
  if (s->active.empty()) return NEGF_OK;
  // plan over all active devices (rebuilt when membership changes)
  const int na = (int)s->active.size();
  if (changed || !s->plan_valid) {
    s->drop_graph();
    std::vector<Dev*> devs;
    for (Req* r : s->active) devs.push_back(find_device(c, r->dev));
    c->chain_tuning_off = true;
    int rc = build_plan(c, devs, nullptr, -1, s->plan, &s->bufs);
    c->chain_tuning_off = false;
    if (rc) return rc;
    std::vector<ScDev> sds;
    for (Req* r : s->active) sds.push_back(r->sd);
    if (!ensure(c, s->sc_desc, sizeof(ScDev) * na) || !ensure(c, s->states_d, sizeof(int) * na)) return NEGF_ENOMEM;
    if (cudaMemcpy(s->sc_desc.p, sds.data(), sizeof(ScDev) * na, cudaMemcpyHostToDevice) != cudaSuccess)
      return set_err(c, NEGF_ECUDA, "upload failed");
    if (na > s->states_cap) {
      if (s->states_h) cudaFreeHost(s->states_h);
      s->states_h = nullptr;
      s->states_cap = 0;
      if (cudaMallocHost(&s->states_h, sizeof(int) * na) != cudaSuccess) return set_err(c, NEGF_ENOMEM, "pinned buffer");
      s->states_cap = na;
    }
    s->plan_valid = true;
  }
  const ScDev* dsc = (const ScDev*)s->sc_desc.p;
  int* states = (int*)s->states_d.p;
  // Poisson -> batched sweep -> reduce -> Broyden -> gathered state flags.  The mixed
  // precision path decides its recompute on the host, so it is launched directly; otherwise
  // the step is captured once per membership and replayed.
  auto enqueue = [&]() -> int {
    if (launch_poisson(dsc, na, c->stream)) return set_err(c, NEGF_ECUDA, "poisson launch failed");
    int rc = launch_plan(c, s->plan);
    if (rc) return rc;
    if (launch_broyden(dsc, na, c->stream) || launch_gather_states(dsc, na, states, c->stream))
      return set_err(c, NEGF_ECUDA, "broyden launch failed");
    c->launches += 3;
    return NEGF_OK;
  };
  const bool graphable = s->plan.prec != NEGF_PREC_MIXED && !c->profile;
  if (graphable && !s->graph) {
    const uint64_t l0 = c->launches;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int rc = enqueue();
      const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ec == cudaSuccess && g && cudaGraphInstantiate(&s->graph, g, 0) != cudaSuccess) s->graph = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    s->graph_kernels = c->launches - l0;
    c->launches = l0;
  }
  if (s->graph) {
    if (cudaGraphLaunch(s->graph, c->stream) != cudaSuccess) return set_err(c, NEGF_ECUDA, "graph launch failed");
    c->launches += s->graph_kernels;
  } else {
    const int rc = enqueue();
    if (rc) return rc;
  }
  if (cudaMemcpyAsync(s->states_h, states, sizeof(int) * na, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "serving step failed");
  std::vector<int> st(s->states_h, s->states_h + na);
  std::vector<Req*> keep;
  for (int i = 0; i < na; ++i) {
    Req* r = s->active[i];
    ++r->iterations;
    const bool limit = r->iterations >= r->br.M;
    if (r->state == Q_CANCELLED) {
      keep.push_back(r);   // retired at the next step
    } else if (st[i] != 0 || limit) {
      finish(c, r, st[i]);
      release_request(c, r);
      s->active_bytes -= r->bytes;
      s->plan_valid = false;
    } else {
      keep.push_back(r);
    }
  }
  s->active = keep;
  *n_active = (int)s->active.size();
  return NEGF_OK;
}

int fill_result(Req* r, negf_sc_result* res) {
  if (!res) return r->status;
  if (res->n && !r->n.empty()) memcpy(res->n, r->n.data(), r->n.size() * 8);
  if (res->U && !r->U.empty()) memcpy(res->U, r->U.data(), r->U.size() * 8);
  if (res->T && !r->T.empty()) memcpy(res->T, r->T.data(), r->T.size() * 8);
  if (res->history && !r->history.empty()) memcpy(res->history, r->history.data(), r->history.size() * 8);
  res->I = r->I;
  res->converged = r->converged;
  res->iterations = r->iterations;
  return r->status;
}

}  // namespace
}  // namespace negf

using namespace negf;

extern "C" {

int negf_submit(negf_ctx* c, const negf_request* q, uint64_t* ticket) {
  if (!c) return NEGF_EINVAL;
  if (!q || !ticket || q->n_rings < 2 || q->n_modes < 1 || q->n_modes > 8 || !q->modes || q->n_tube < 1 ||
      q->n_real < 1 || q->n_cont < 1 || !(q->kT > 0.0) || !(q->eta > 0.0) || !(q->broyden.zeta > 0.0) ||
      q->broyden.M < 1 || q->broyden.M > 256 || !(q->broyden.tol > 0.0) || !(q->pois.kappa > 0.0) ||
      !(q->pois.dx_nm > 0.0))
    return set_err(c, NEGF_EINVAL, "bad request");
  std::lock_guard<std::mutex> g(c->serve_mu);
  Serve* s = serve_of(c);
  Req* r = new Req();
  r->ticket = s->next_ticket++;
  r->N = q->n_rings;
  r->n_tube = q->n_tube;
  r->modes.assign(q->modes, q->modes + q->n_modes);
  r->t = q->t;
  r->kT = q->kT;
  r->eta = q->eta;
  r->E_B = q->E_B;
  r->n_real = q->n_real;
  r->n_cont = q->n_cont;
  r->bias = q->bias;
  r->pois = q->pois;
  r->br = q->broyden;
  if (q->U0) r->U0.assign(q->U0, q->U0 + q->n_rings);
  r->t_submit = now_s();
  s->queue.push_back(r);
  s->all[r->ticket] = r;
  *ticket = r->ticket;
  return NEGF_OK;
}

int negf_serve_step(negf_ctx* c, int* active) {
  if (!c) return NEGF_EINVAL;
  std::lock_guard<std::mutex> g(c->serve_mu);
  int na = 0;
  const int rc = step_locked(c, serve_of(c), &na);
  if (active) *active = na;
  return rc;
}

int negf_poll(negf_ctx* c, uint64_t ticket, negf_sc_result* res) {
  if (!c) return NEGF_EINVAL;
  std::lock_guard<std::mutex> g(c->serve_mu);
  Serve* s = serve_of(c);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return set_err(c, NEGF_ENOTFOUND, "unknown ticket");
  Req* r = it->second;
  if (r->state == Q_QUEUED || r->state == Q_ACTIVE) return NEGF_EBUSY;
  if (r->state == Q_CANCELLED) return set_err(c, NEGF_ENOTFOUND, "request was cancelled");
  return fill_result(r, res);
}

int negf_wait(negf_ctx* c, uint64_t ticket, int timeout_ms, negf_sc_result* res) {
  if (!c) return NEGF_EINVAL;
  const double t_end = now_s() + timeout_ms * 1e-3;
  for (;;) {
    int rc = negf_poll(c, ticket, res);
    if (rc != NEGF_EBUSY) return rc;
    if (now_s() >= t_end) return set_err(c, NEGF_ETIMEDOUT, "request not finished within the timeout");
    int na = 0;
    if ((rc = negf_serve_step(c, &na))) return rc;
  }
}

int negf_cancel(negf_ctx* c, uint64_t ticket) {
  if (!c) return NEGF_EINVAL;
  std::lock_guard<std::mutex> g(c->serve_mu);
  Serve* s = serve_of(c);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return set_err(c, NEGF_ENOTFOUND, "unknown ticket");
  Req* r = it->second;
  if (r->state == Q_QUEUED || r->state == Q_ACTIVE) r->state = Q_CANCELLED;
  return NEGF_OK;
}

int negf_request_times(negf_ctx* c, uint64_t ticket, double* t_submit, double* t_start, double* t_done) {
  if (!c) return NEGF_EINVAL;
  std::lock_guard<std::mutex> g(c->serve_mu);
  Serve* s = serve_of(c);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return set_err(c, NEGF_ENOTFOUND, "unknown ticket");
  if (t_submit) *t_submit = it->second->t_submit;
  if (t_start) *t_start = it->second->t_start;
  if (t_done) *t_done = it->second->t_done;
  return NEGF_OK;
}

}  // extern "C"
