// Self-consistent NEGF-Poisson loop of one device (Sec. 2.3, Alg. 3) kept on the GPU.
//
// A session owns the Broyden state (n_in, n_in_old, f_old, V, W, m; Alg. 3 stores V^T and
// W per rank), its own launch-plan scratch, and one iteration -- Poisson (Thomas) ->
// batched NEGF sweep -> second-stage quadrature -> Broyden step -- captured once as a CUDA
// graph and replayed.  The potential the Poisson kernel writes is the buffer the sweep
// reads, and the charge the second stage writes is the buffer the Broyden kernel reads:
// inside the loop no data leaves the device; the host reads one status word when asked.
#include <cmath>
#include <cstring>

#include "ctx.h"

namespace negf {

struct ScSession {
  int N = 0, M = 0;
  DBuf nin, nold, fold, V, W, n0, hist, m, state, cp, sc;
  PlanBufs bufs;
  Plan plan;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* h_state = nullptr;
  int iterations = 0;
  int last_state = 0;
  int refines = 0;
  uint64_t kernels_per_iter = 0;
};

void sc_session_free(Ctx* c, Dev* d) {
  ScSession* s = d->sc;
  if (!s) return;
  cudaStreamSynchronize(c->stream);
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  if (s->h_state) cudaFreeHost(s->h_state);
  for (DBuf* b : {&s->nin, &s->nold, &s->fold, &s->V, &s->W, &s->n0, &s->hist, &s->m, &s->state, &s->cp, &s->sc})
    c->arena.release(*b);
  free_plan_bufs(c, s->bufs);
  delete s;
  d->sc = nullptr;
}

// Capture one iteration -- Poisson, the plan's sweeps and second stage, Broyden -- as a CUDA
// graph (left uncaptured if the stream cannot be captured; the iteration then launches directly).
static void capture_iteration(Ctx* c, ScSession* s) {
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->exec = nullptr;
  s->graph = nullptr;
  // Poisson, the sweep groups, the layer-diagonal prep of 1 x 1 chains, second stage, Broyden
  s->kernels_per_iter = 3 + (s->plan.n_prep > 0 ? 1 : 0);
  for (int g = 0; g < NGROUPS; ++g) s->kernels_per_iter += (s->plan.ncls[g] > 0);
  s->kernels_per_iter += 5 * s->plan.seg_waves.size();
  const ScDev* dsc = (const ScDev*)s->sc.p;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const uint64_t l0 = c->launches;
    const bool ok = launch_poisson(dsc, 1, c->stream) == 0 && launch_plan(c, s->plan) == NEGF_OK &&
                    launch_broyden(dsc, 1, c->stream) == 0;
    c->launches = l0;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(c->stream, &g) == cudaSuccess && ok && cudaGraphInstantiate(&s->exec, g, 0) == cudaSuccess)
      s->graph = g;
    else if (g)
      cudaGraphDestroy(g);
    cudaGetLastError();
  }
}

// An iteration that refines a semi-adaptive grid (Sec. 3.3): Poisson, then the peak of the
// refinement ring's integrand with the new potential on the grid in use, the grid rebuilt
// around it, a new plan and graph, then the NEGF evaluation and Broyden step on the new grid.
// A session that has already stopped (converged or out of history) is left as it is.
static int refine_iteration(Ctx* c, Dev* d, ScSession* s) {
  const ScDev* dsc = (const ScDev*)s->sc.p;
  if (cudaMemcpyAsync(s->h_state, s->state.p, 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "self-consistent iteration failed");
  if (*s->h_state != 0) return NEGF_OK;
  if (launch_poisson(dsc, 1, c->stream)) return set_err(c, NEGF_ECUDA, "poisson launch failed");
  ++c->launches;
  int rc = refine_grid_internal(c, d, nullptr);
  if (rc) return rc;
  ++s->refines;
  std::vector<Dev*> one{d};
  if ((rc = build_plan(c, one, nullptr, -1, s->plan, &s->bufs))) return rc;
  capture_iteration(c, s);
  if ((rc = launch_plan(c, s->plan))) return rc;
  if (launch_broyden(dsc, 1, c->stream)) return set_err(c, NEGF_ECUDA, "broyden launch failed");
  ++c->launches;
  return NEGF_OK;
}

static int run_iteration(Ctx* c, ScSession* s) {
  const ScDev* dsc = (const ScDev*)s->sc.p;
  if (s->exec) {
    if (cudaGraphLaunch(s->exec, c->stream) != cudaSuccess) return set_err(c, NEGF_ECUDA, "graph launch failed");
    c->launches += s->kernels_per_iter;
    return NEGF_OK;
  }
  if (launch_poisson(dsc, 1, c->stream)) return set_err(c, NEGF_ECUDA, "poisson launch failed");
  int rc = launch_plan(c, s->plan);
  if (rc) return rc;
  if (launch_broyden(dsc, 1, c->stream)) return set_err(c, NEGF_ECUDA, "broyden launch failed");
  c->launches += 2;
  return NEGF_OK;
}

}  // namespace negf

using namespace negf;

extern "C" {

int negf_sc_begin(negf_ctx* c, int dev, const negf_bias* bias, const negf_poisson* pois,
                  const negf_broyden* br, const double* U0) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  if (d->sc) return set_err(c, NEGF_EBUSY, "a session is already active on this device");
  if (!bias || !pois || !br || !U0) return set_err(c, NEGF_EINVAL, "null argument");
  if (!(br->zeta > 0.0) || br->M < 1 || br->M > 256 || !(br->tol > 0.0))
    return set_err(c, NEGF_EINVAL, "bad Broyden settings (zeta > 0, 1 <= M <= 256, tol > 0)");
  if (!(pois->kappa > 0.0) || !(pois->dx_nm > 0.0) || !(pois->lam_nm >= 0.0))
    return set_err(c, NEGF_EINVAL, "bad Poisson settings");
  if (!d->spec_set) return set_err(c, NEGF_EINVAL, "the device grid must be set with negf_set_grid_spec");
  for (auto& ch : d->ch)
    if (!ch.h_set || !ch.lead[0].set || !ch.lead[1].set) return set_err(c, NEGF_EINVAL, "device not built");
  for (int i = 0; i < d->n_rings; ++i)
    if (!std::isfinite(U0[i])) return set_err(c, NEGF_EINVAL, "non-finite U0");
  cudaSetDevice(c->ordinal);
  const int N = d->n_rings, M = br->M;
  const double U_S = 0.0, U_D = -bias->V_DS;
  const double U_G = pois->phi_gate - bias->V_GS;
  const double r = (pois->lam_nm / pois->dx_nm) * (pois->lam_nm / pois->dx_nm);
  int rc = negf_set_lead_potentials(c, dev, U_S, U_D);
  if (rc) return rc;
  std::vector<double> n0(N), nin(N);
  if ((rc = negf_neutral_charge(c, dev, d->spec.n_cont, d->spec.E_B, n0.data()))) return rc;
  // the charge whose Poisson solution is U0, so the loop starts from U0
  for (int i = 0; i < N; ++i) {
    const double left = i > 0 ? U0[i - 1] : U_S;
    const double right = i < N - 1 ? U0[i + 1] : U_D;
    nin[i] = n0[i] + ((1.0 + 2.0 * r) * U0[i] - r * (left + right) - U_G) / pois->kappa;
  }
  if ((rc = negf_set_potential(c, dev, U0))) return rc;

  ScSession* s = new ScSession();
  d->sc = s;
  s->N = N;
  s->M = M;
  auto fail = [&](int code) {
    sc_session_free(c, d);
    return code;
  };
  if ((rc = upload(c, s->nin, nin.data(), N * 8)) || (rc = upload(c, s->n0, n0.data(), N * 8))) return fail(rc);
  if (!ensure(c, s->nold, N * 8) || !ensure(c, s->fold, N * 8) || !ensure(c, s->V, (size_t)M * N * 8) ||
      !ensure(c, s->W, (size_t)M * N * 8) || !ensure(c, s->hist, M * 8) || !ensure(c, s->m, 4) ||
      !ensure(c, s->state, 4) || !ensure(c, s->cp, N * 8) || !ensure(c, s->sc, sizeof(ScDev)))
    return fail(NEGF_ENOMEM);
  cudaMemset(s->nold.p, 0, N * 8);
  cudaMemset(s->fold.p, 0, N * 8);
  cudaMemset(s->V.p, 0, (size_t)M * N * 8);
  cudaMemset(s->W.p, 0, (size_t)M * N * 8);
  cudaMemset(s->hist.p, 0, M * 8);
  cudaMemset(s->m.p, 0, 4);
  cudaMemset(s->state.p, 0, 4);
  std::vector<Dev*> one{d};
  if ((rc = build_plan(c, one, nullptr, -1, s->plan, &s->bufs))) return fail(rc);
  ScDev sd;
  sd.N = N;
  sd.M = M;
  sd.zeta = br->zeta;
  sd.tol = br->tol;
  sd.kappa = pois->kappa;
  sd.r = r;
  sd.U_G = U_G;
  sd.U_S = U_S;
  sd.U_D = U_D;
  sd.n_in = (double*)s->nin.p;
  sd.n_in_old = (double*)s->nold.p;
  sd.f_old = (double*)s->fold.p;
  sd.V = (double*)s->V.p;
  sd.W = (double*)s->W.p;
  sd.n0 = (double*)s->n0.p;
  sd.U = (double*)d->dU.p;
  sd.n_out = (const double*)d->dn.p;
  sd.hist = (double*)s->hist.p;
  sd.m = (int*)s->m.p;
  sd.state = (int*)s->state.p;
  sd.cp = (double*)s->cp.p;
  if (cudaMemcpy(s->sc.p, &sd, sizeof(sd), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(set_err(c, NEGF_ECUDA, "upload failed"));
  if (cudaMallocHost(&s->h_state, sizeof(int)) != cudaSuccess) return fail(set_err(c, NEGF_ENOMEM, "pinned alloc failed"));
  // capture one iteration (a semi-adaptive grid is refined at the first iteration, which
  // captures its own graph)
  if (!d->adaptive) capture_iteration(c, s);
  return NEGF_OK;
}

int negf_sc_step(negf_ctx* c, int dev, int k, int* state) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  ScSession* s = d->sc;
  if (!s) return set_err(c, NEGF_EINVAL, "no self-consistent session on this device");
  if (k < 1) return set_err(c, NEGF_EINVAL, "k must be >= 1");
  cudaSetDevice(c->ordinal);
  for (int i = 0; i < k; ++i) {
    if (s->last_state != 0) break;
    const int it = s->iterations;
    const bool refine = d->adaptive && (it == 0 || (d->ad.period > 0 && it % d->ad.period == 0));
    int rc = refine ? refine_iteration(c, d, s) : run_iteration(c, s);
    if (rc) return rc;
    if (state) {
      if (cudaMemcpyAsync(s->h_state, s->state.p, 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        return set_err(c, NEGF_ECUDA, "self-consistent iteration failed");
      ++s->iterations;
      s->last_state = *s->h_state;
    } else {
      ++s->iterations;
    }
  }
  if (state) *state = s->last_state;
  return NEGF_OK;
}

int negf_sc_end(negf_ctx* c, int dev, negf_sc_result* res) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  ScSession* s = d->sc;
  if (!s) return set_err(c, NEGF_EINVAL, "no self-consistent session on this device");
  cudaSetDevice(c->ordinal);
  int rc = NEGF_OK;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = set_err(c, NEGF_ECUDA, "kernel execution failed");
  int st = 0;
  cudaMemcpy(&st, s->state.p, 4, cudaMemcpyDeviceToHost);
  if (!rc && res) {
    const int N = s->N, nr = s->plan.views[0].n_real;
    const int iters = s->iterations;
    if (res->n) cudaMemcpy(res->n, d->dn.p, N * 8, cudaMemcpyDeviceToHost);
    if (res->U) cudaMemcpy(res->U, d->dU.p, N * 8, cudaMemcpyDeviceToHost);
    if (res->T && nr > 0) cudaMemcpy(res->T, d->dT.p, (size_t)nr * 8, cudaMemcpyDeviceToHost);
    if (res->history) cudaMemcpy(res->history, s->hist.p, (size_t)std::min(iters, s->M) * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(&res->I, d->dI.p, 8, cudaMemcpyDeviceToHost);
    res->converged = (st == 1);
    res->iterations = iters;
  }
  cudaMemcpy(d->U.data(), d->dU.p, (size_t)s->N * 8, cudaMemcpyDeviceToHost);
  sc_session_free(c, d);
  if (!rc && res && !res->converged)
    rc = set_err(c, NEGF_ENOTCONVERGED, "Broyden history exhausted before eps_max < tol");
  return rc;
}

int negf_sc_get_state(negf_ctx* c, int dev, double* n_in, double* n_in_old, double* f_old, double* V,
                      double* W, int* m) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  ScSession* s = d->sc;
  if (!s) return set_err(c, NEGF_EINVAL, "no self-consistent session on this device");
  cudaSetDevice(c->ordinal);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return set_err(c, NEGF_ECUDA, "kernel execution failed");
  const size_t N = s->N, M = s->M;
  if (n_in) cudaMemcpy(n_in, s->nin.p, N * 8, cudaMemcpyDeviceToHost);
  if (n_in_old) cudaMemcpy(n_in_old, s->nold.p, N * 8, cudaMemcpyDeviceToHost);
  if (f_old) cudaMemcpy(f_old, s->fold.p, N * 8, cudaMemcpyDeviceToHost);
  if (V) cudaMemcpy(V, s->V.p, M * N * 8, cudaMemcpyDeviceToHost);
  if (W) cudaMemcpy(W, s->W.p, M * N * 8, cudaMemcpyDeviceToHost);
  if (m) cudaMemcpy(m, s->m.p, 4, cudaMemcpyDeviceToHost);
  return NEGF_OK;
}

int negf_sc_set_state(negf_ctx* c, int dev, const double* n_in, const double* n_in_old, const double* f_old,
                      const double* V, const double* W, int m) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  ScSession* s = d->sc;
  if (!s) return set_err(c, NEGF_EINVAL, "no self-consistent session on this device");
  if (!n_in || m < 0 || m >= s->M || (m > 0 && (!n_in_old || !f_old || !V || !W)))
    return set_err(c, NEGF_EINVAL, "bad state");
  cudaSetDevice(c->ordinal);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return set_err(c, NEGF_ECUDA, "kernel execution failed");
  const size_t N = s->N, M = s->M;
  cudaMemcpy(s->nin.p, n_in, N * 8, cudaMemcpyHostToDevice);
  if (m > 0) {
    cudaMemcpy(s->nold.p, n_in_old, N * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(s->fold.p, f_old, N * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(s->V.p, V, M * N * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(s->W.p, W, M * N * 8, cudaMemcpyHostToDevice);
  }
  cudaMemcpy(s->m.p, &m, 4, cudaMemcpyHostToDevice);
  const int zero = 0;
  cudaMemcpy(s->state.p, &zero, 4, cudaMemcpyHostToDevice);
  s->last_state = 0;
  return NEGF_OK;
}

int negf_sc_solve(negf_ctx* c, int dev, const negf_bias* bias, const negf_poisson* pois,
                  const negf_broyden* br, const double* U0, negf_sc_result* res) {
  if (!c) return NEGF_EINVAL;
  if (!res) return set_err(c, NEGF_EINVAL, "null result");
  int rc = negf_sc_begin(c, dev, bias, pois, br, U0);
  if (rc) return rc;
  int state = 0;
  for (int it = 0; it < br->M && state == 0; ++it) {
    if ((rc = negf_sc_step(c, dev, 1, &state))) {
      negf_sc_end(c, dev, nullptr);
      return rc;
    }
  }
  return negf_sc_end(c, dev, res);
}

}  // extern "C"
