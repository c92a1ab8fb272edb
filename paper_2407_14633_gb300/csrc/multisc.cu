// Self-consistent loop of several channels with one Broyden vector (Sec. 2.3: the charge
// vectors of all channel materials are concatenated before the Broyden step and split after
// it).  The channels are tubes of equal length sharing contacts and gate; their 1D Poisson
// stand-ins are coupled through a C x C matrix K in the source term,
//   U_c,i - U_G - r (U_c,i+1 - 2 U_c,i + U_c,i-1) = sum_c' K[c][c'] (n_c',i - n0_c',i),
// a builder-defined stand-in for the paper's 3D electrostatics.  One iteration -- coupled
// Poisson (one CTA per channel), the sweeps of every channel in one batched plan, a gather of
// the channel charges into the concatenated vector, the Broyden step over the whole vector --
// is captured once as a CUDA graph and replayed; the host reads one status word per iteration.
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace negf {

namespace {

struct ChanDesc {
  double* U;          // the channel device's potential (Poisson output, sweep input)
  const double* n;    // the channel device's electron count (second-stage output)
};

// One CTA per channel; thread 0 runs the Thomas recurrence (N sequential steps, negligible
// next to the sweep).  K is C x C row-major; S->n_in / n0 / cp are concatenated (C x N).
__global__ void poisson_multi_kernel(const ScDev* S, const ChanDesc* ch, const double* K, int C, int N) {
  const int c = blockIdx.x;
  if (threadIdx.x != 0 || *S->state != 0) return;
  const double r = S->r, dg = 1.0 + 2.0 * r;
  double* cp = S->cp + (long long)c * N;
  double* U = ch[c].U;
  double cprev = 0.0, dprev = 0.0;
  for (int i = 0; i < N; ++i) {
    double q = 0.0;
    for (int d = 0; d < C; ++d) q += K[c * C + d] * (S->n_in[(long long)d * N + i] - S->n0[(long long)d * N + i]);
    double rhs = S->U_G + q;
    if (i == 0) rhs += r * S->U_S;
    if (i == N - 1) rhs += r * S->U_D;
    const double den = dg + r * cprev;
    const double cpi = (i < N - 1) ? -r / den : 0.0;
    const double dpi = (rhs + r * dprev) / den;
    cp[i] = cpi;
    U[i] = dpi;
    cprev = cpi;
    dprev = dpi;
  }
  for (int i = N - 2; i >= 0; --i) U[i] = U[i] - cp[i] * U[i + 1];
}

__global__ void gather_multi_kernel(const ChanDesc* ch, double* nout, int N) {
  const int c = blockIdx.x;
  for (int i = threadIdx.x; i < N; i += blockDim.x) nout[(long long)c * N + i] = ch[c].n[i];
}

// LU with partial pivoting of the C x C matrix K, then per ring q = K^{-1} L (host set-up).
bool solve_rings(std::vector<double> K, int C, int N, const std::vector<double>& L, std::vector<double>& q) {
  std::vector<int> piv(C);
  for (int k = 0; k < C; ++k) {
    int p = k;
    for (int i = k + 1; i < C; ++i)
      if (std::fabs(K[i * C + k]) > std::fabs(K[p * C + k])) p = i;
    if (!(std::fabs(K[p * C + k]) > 0.0)) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < C; ++j) std::swap(K[k * C + j], K[p * C + j]);
    for (int i = k + 1; i < C; ++i) {
      const double f = K[i * C + k] / K[k * C + k];
      K[i * C + k] = f;
      for (int j = k + 1; j < C; ++j) K[i * C + j] -= f * K[k * C + j];
    }
  }
  q.assign((size_t)C * N, 0.0);
  std::vector<double> x(C);
  for (int i = 0; i < N; ++i) {
    for (int c = 0; c < C; ++c) x[c] = L[(size_t)c * N + i];
    for (int k = 0; k < C; ++k)
      if (piv[k] != k) std::swap(x[k], x[piv[k]]);
    for (int a = 1; a < C; ++a)
      for (int b = 0; b < a; ++b) x[a] -= K[a * C + b] * x[b];
    for (int a = C - 1; a >= 0; --a) {
      for (int b = a + 1; b < C; ++b) x[a] -= K[a * C + b] * x[b];
      x[a] /= K[a * C + a];
    }
    for (int c = 0; c < C; ++c) q[(size_t)c * N + i] = x[c];
  }
  return true;
}

}  // namespace

}  // namespace negf

using namespace negf;

extern "C" {

int negf_sc_solve_multi(negf_ctx* c, const int* devs, int C, const negf_bias* bias, const negf_poisson* pois,
                        const double* Kh, const negf_broyden* br, const double* U0, negf_sc_result* res) {
  if (!c) return NEGF_EINVAL;
  if (!devs || C < 1 || C > 64 || !bias || !pois || !Kh || !br || !U0 || !res)
    return set_err(c, NEGF_EINVAL, "bad multi-channel arguments");
  if (!(br->zeta > 0.0) || br->M < 1 || br->M > 256 || !(br->tol > 0.0))
    return set_err(c, NEGF_EINVAL, "bad Broyden settings (zeta > 0, 1 <= M <= 256, tol > 0)");
  if (!(pois->dx_nm > 0.0) || !(pois->lam_nm >= 0.0)) return set_err(c, NEGF_EINVAL, "bad Poisson settings");
  for (int i = 0; i < C * C; ++i)
    if (!std::isfinite(Kh[i])) return set_err(c, NEGF_EINVAL, "non-finite coupling matrix");
  std::vector<Dev*> list;
  for (int i = 0; i < C; ++i) {
    Dev* d = find_device(c, devs[i]);
    if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
    if (d->sc) return set_err(c, NEGF_EBUSY, "device is in a self-consistent session");
    for (int j = 0; j < i; ++j)
      if (devs[j] == devs[i]) return set_err(c, NEGF_EINVAL, "device listed twice");
    if (!d->spec_set) return set_err(c, NEGF_EINVAL, "every device grid must be set from a grid spec");
    for (auto& ch : d->ch)
      if (!ch.h_set || !ch.lead[0].set || !ch.lead[1].set) return set_err(c, NEGF_EINVAL, "device not built");
    if (!list.empty() && d->n_rings != list[0]->n_rings)
      return set_err(c, NEGF_EINVAL, "coupled channels need equal ring counts");
    list.push_back(d);
  }
  const int N = list[0]->n_rings, M = br->M;
  const long long NT = (long long)C * N;
  for (long long i = 0; i < NT; ++i)
    if (!std::isfinite(U0[i])) return set_err(c, NEGF_EINVAL, "non-finite U0");
  cudaSetDevice(c->ordinal);
  const double U_S = 0.0, U_D = -bias->V_DS, U_G = pois->phi_gate - bias->V_GS;
  const double r = (pois->lam_nm / pois->dx_nm) * (pois->lam_nm / pois->dx_nm);
  // neutral charges, the starting charges whose coupled Poisson solution is U0, potentials
  std::vector<double> n0(NT), L(NT), nin;
  int rc;
  for (int ci = 0; ci < C; ++ci) {
    Dev* d = list[ci];
    if ((rc = negf_set_lead_potentials(c, devs[ci], U_S, U_D))) return rc;
    if ((rc = negf_neutral_charge(c, devs[ci], d->spec.n_cont, d->spec.E_B, n0.data() + (size_t)ci * N))) return rc;
    const double* u = U0 + (size_t)ci * N;
    for (int i = 0; i < N; ++i) {
      const double left = i > 0 ? u[i - 1] : U_S, right = i < N - 1 ? u[i + 1] : U_D;
      L[(size_t)ci * N + i] = (1.0 + 2.0 * r) * u[i] - r * (left + right) - U_G;
    }
    if ((rc = negf_set_potential(c, devs[ci], u))) return rc;
  }
  std::vector<double> K(Kh, Kh + C * C), q;
  if (!solve_rings(K, C, N, L, q)) return set_err(c, NEGF_EINVAL, "singular coupling matrix");
  nin.resize(NT);
  for (long long i = 0; i < NT; ++i) nin[i] = n0[i] + q[i];

  DBuf bnin, bnold, bfold, bV, bW, bn0, bhist, bm, bstate, bcp, bsc, bnout, bK, bch;
  PlanBufs bufs;
  Plan plan;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* h_state = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (h_state) cudaFreeHost(h_state);
    for (DBuf* b : {&bnin, &bnold, &bfold, &bV, &bW, &bn0, &bhist, &bm, &bstate, &bcp, &bsc, &bnout, &bK, &bch})
      c->arena.release(*b);
    free_plan_bufs(c, bufs);
  };
  if ((rc = upload(c, bnin, nin.data(), NT * 8)) || (rc = upload(c, bn0, n0.data(), NT * 8)) ||
      (rc = upload(c, bK, K.data(), (size_t)C * C * 8))) {
    cleanup();
    return rc;
  }
  if (!ensure(c, bnold, NT * 8) || !ensure(c, bfold, NT * 8) || !ensure(c, bV, (size_t)M * NT * 8) ||
      !ensure(c, bW, (size_t)M * NT * 8) || !ensure(c, bhist, M * 8) || !ensure(c, bm, 4) || !ensure(c, bstate, 4) ||
      !ensure(c, bcp, NT * 8) || !ensure(c, bsc, sizeof(ScDev)) || !ensure(c, bnout, NT * 8) ||
      !ensure(c, bch, C * sizeof(ChanDesc))) {
    cleanup();
    return NEGF_ENOMEM;
  }
  cudaMemsetAsync(bnold.p, 0, NT * 8, c->stream);
  cudaMemsetAsync(bfold.p, 0, NT * 8, c->stream);
  cudaMemsetAsync(bV.p, 0, (size_t)M * NT * 8, c->stream);
  cudaMemsetAsync(bW.p, 0, (size_t)M * NT * 8, c->stream);
  cudaMemsetAsync(bhist.p, 0, M * 8, c->stream);
  cudaMemsetAsync(bm.p, 0, 4, c->stream);
  cudaMemsetAsync(bstate.p, 0, 4, c->stream);
  if ((rc = build_plan(c, list, nullptr, -1, plan, &bufs))) {
    cleanup();
    return rc;
  }
  // channel potentials and charges, taken once the plan has sized every output buffer
  std::vector<ChanDesc> chd(C);
  for (int ci = 0; ci < C; ++ci) chd[ci] = ChanDesc{(double*)list[ci]->dU.p, (const double*)list[ci]->dn.p};
  if (cudaMemcpyAsync(bch.p, chd.data(), C * sizeof(ChanDesc), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    cleanup();
    return set_err(c, NEGF_ECUDA, "upload failed");
  }
  ScDev sd;
  memset(&sd, 0, sizeof(sd));
  sd.N = (int)NT;
  sd.M = M;
  sd.zeta = br->zeta;
  sd.tol = br->tol;
  sd.kappa = 0.0;
  sd.r = r;
  sd.U_G = U_G;
  sd.U_S = U_S;
  sd.U_D = U_D;
  sd.n_in = (double*)bnin.p;
  sd.n_in_old = (double*)bnold.p;
  sd.f_old = (double*)bfold.p;
  sd.V = (double*)bV.p;
  sd.W = (double*)bW.p;
  sd.n0 = (double*)bn0.p;
  sd.U = nullptr;
  sd.n_out = (const double*)bnout.p;
  sd.hist = (double*)bhist.p;
  sd.m = (int*)bm.p;
  sd.state = (int*)bstate.p;
  sd.cp = (double*)bcp.p;
  if (cudaMemcpyAsync(bsc.p, &sd, sizeof(sd), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cleanup();
    return set_err(c, NEGF_ECUDA, "upload failed");
  }
  if (cudaMallocHost(&h_state, sizeof(int)) != cudaSuccess) {
    h_state = nullptr;
    cleanup();
    return set_err(c, NEGF_ENOMEM, "pinned alloc failed");
  }
  const ScDev* dsc = (const ScDev*)bsc.p;
  const ChanDesc* dch = (const ChanDesc*)bch.p;
  auto iteration = [&]() -> int {
    poisson_multi_kernel<<<C, 32, 0, c->stream>>>(dsc, dch, (const double*)bK.p, C, N);
    if (cudaGetLastError() != cudaSuccess) return set_err(c, NEGF_ECUDA, "poisson launch failed");
    int e = launch_plan(c, plan);
    if (e) return e;
    gather_multi_kernel<<<C, 256, 0, c->stream>>>(dch, (double*)bnout.p, N);
    if (cudaGetLastError() != cudaSuccess) return set_err(c, NEGF_ECUDA, "gather launch failed");
    if (launch_broyden(dsc, 1, c->stream)) return set_err(c, NEGF_ECUDA, "broyden launch failed");
    return NEGF_OK;
  };
  // launches per captured iteration: Poisson, prep of 1 x 1 chains, sweep groups, second stage,
  // gather, Broyden (an uncaptured iteration counts the plan's own launches in launch_plan)
  uint64_t per_iter = 4 + (plan.n_prep > 0 ? 1 : 0);
  for (int g = 0; g < NGROUPS; ++g) per_iter += (plan.ncls[g] > 0);
  per_iter += 5 * plan.seg_waves.size();
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const uint64_t l0 = c->launches;
    const bool ok = iteration() == NEGF_OK;
    c->launches = l0;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(c->stream, &g) == cudaSuccess && ok && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess)
      graph = g;
    else if (g)
      cudaGraphDestroy(g);
    cudaGetLastError();
  }
  int iters = 0, st = 0;
  for (int it = 0; it < M && st == 0; ++it) {
    if (exec) {
      if (cudaGraphLaunch(exec, c->stream) != cudaSuccess) rc = set_err(c, NEGF_ECUDA, "graph launch failed");
      c->launches += per_iter;
    } else {
      rc = iteration();
      c->launches += 3;
    }
    if (rc) break;
    if (cudaMemcpyAsync(h_state, bstate.p, 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      rc = set_err(c, NEGF_ECUDA, "self-consistent iteration failed");
      break;
    }
    ++iters;
    st = *h_state;
  }
  if (!rc) {
    std::vector<double> hist(std::min(iters, M));
    if (!hist.empty()) cudaMemcpy(hist.data(), bhist.p, hist.size() * 8, cudaMemcpyDeviceToHost);
    for (int ci = 0; ci < C; ++ci) {
      Dev* d = list[ci];
      negf_sc_result& R = res[ci];
      const int nr = plan.views[ci].n_real;
      if (R.n) cudaMemcpy(R.n, d->dn.p, (size_t)N * 8, cudaMemcpyDeviceToHost);
      if (R.U) cudaMemcpy(R.U, d->dU.p, (size_t)N * 8, cudaMemcpyDeviceToHost);
      if (R.T && nr > 0) cudaMemcpy(R.T, d->dT.p, (size_t)nr * 8, cudaMemcpyDeviceToHost);
      if (R.history && !hist.empty()) memcpy(R.history, hist.data(), hist.size() * 8);
      cudaMemcpy(&R.I, d->dI.p, 8, cudaMemcpyDeviceToHost);
      R.converged = (st == 1);
      R.iterations = iters;
      cudaMemcpy(d->U.data(), d->dU.p, (size_t)N * 8, cudaMemcpyDeviceToHost);
    }
    if (cudaGetLastError() != cudaSuccess) rc = set_err(c, NEGF_ECUDA, "copy out failed");
  }
  cleanup();
  if (!rc && st != 1) rc = set_err(c, NEGF_ENOTCONVERGED, "Broyden history exhausted before eps_max < tol");
  return rc;
}

}  // extern "C"
