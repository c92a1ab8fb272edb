// Semi-adaptive real-axis grid (Sec. 3.3).  The path [E_min, E_max] is split at E_l1 <= E_l2
// into three sub-intervals with their own Gauss-Legendre rules, at a point density per kT
// chosen per sub-interval; the limits follow the peak E_s of one ring's charge integrand
// (the van Hove singularity at a subband edge, which sharpens as the channel grows):
// E_l1 = E_s - a kT, E_l2 = E_s + b kT.  The grid itself is host set-up data (FP64); the
// integrand is evaluated by the ordinary sweep kernels with one lane per energy and unit
// weights, and its peak is located on the GPU by a fixed-shape argmax.
#include <cmath>
#include <vector>

#include "ctx.h"

namespace negf {

namespace {

// Limits, clipped limits and per-segment Gauss-Legendre sizes of a semi-adaptive grid.
struct AdaptiveShape {
  double Emin = 0.0, Emax = 0.0, l1 = 0.0, l2 = 0.0;
  int n[3] = {0, 0, 0};
  int total() const { return n[0] + n[1] + n[2]; }
};

int adaptive_shape(const negf_grid_spec* s, double E_l1, double E_l2, const double dens[3], AdaptiveShape& A) {
  if (!s || !(s->kT > 0.0) || !std::isfinite(E_l1) || !std::isfinite(E_l2)) return NEGF_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (!(dens[i] > 0.0) || !std::isfinite(dens[i])) return NEGF_EINVAL;
  const double mu_min = std::min(s->mu_S, s->mu_D), mu_max = std::max(s->mu_S, s->mu_D);
  const double f1 = std::isnan(s->f1) ? 14.0 : s->f1, f2 = std::isnan(s->f2) ? 14.0 : s->f2;
  A.Emin = std::isnan(s->E_min) ? mu_min - f1 * s->kT : s->E_min;
  A.Emax = std::isnan(s->E_max) ? mu_max + f2 * s->kT : s->E_max;
  if (!(A.Emax > A.Emin)) return NEGF_EINVAL;
  A.l1 = std::min(std::max(E_l1, A.Emin), A.Emax);
  A.l2 = std::min(std::max(E_l2, A.l1), A.Emax);
  const double lo[3] = {A.Emin, A.l1, A.l2}, hi[3] = {A.l1, A.l2, A.Emax};
  for (int i = 0; i < 3; ++i) {
    if (!(hi[i] > lo[i])) {
      A.n[i] = 0;
      continue;
    }
    // points per kT; the slack of a millionth of a point keeps a width that is a whole number
    // of kT up to rounding from gaining a point
    const double want = std::ceil(dens[i] * ((hi[i] - lo[i]) / s->kT) - 1e-6);
    if (!(want < 1e8)) return NEGF_EINVAL;
    A.n[i] = std::max(1, (int)want);
  }
  return A.total() > 0 ? NEGF_OK : NEGF_EINVAL;
}

// Nodes, weights and occupations of the three segments, in ascending energy.
void adaptive_fill(const negf_grid_spec* s, const AdaptiveShape& A, double* E, double* w, double* fS, double* fD) {
  const double lo[3] = {A.Emin, A.l1, A.l2}, hi[3] = {A.l1, A.l2, A.Emax};
  int k0 = 0;
  for (int i = 0; i < 3; ++i) {
    if (!A.n[i]) continue;
    std::vector<double> x, wg;
    gl_rule(A.n[i], x, wg);
    const double h = 0.5 * (hi[i] - lo[i]), m = 0.5 * (hi[i] + lo[i]);
    for (int k = 0; k < A.n[i]; ++k) {
      E[k0 + k] = m + h * x[k];
      w[k0 + k] = h * wg[k];
    }
    k0 += A.n[i];
  }
  for (int k = 0; k < A.total(); ++k) {
    fS[k] = fermi_host(E[k] - s->mu_S, s->kT);
    fD[k] = fermi_host(E[k] - s->mu_D, s->kT);
  }
}

// Rebuild the device grid around limits (l1, l2) with the device's stored settings.
int set_adaptive(Ctx* c, Dev* d, const negf_grid_spec& spec, const negf_adaptive& ad, double l1, double l2) {
  AdaptiveShape A;
  if (adaptive_shape(&spec, l1, l2, ad.density, A)) return set_err(c, NEGF_EINVAL, "bad semi-adaptive grid");
  const int nr = A.total(), nc = spec.n_cont;
  std::vector<double> E(nr), w(nr), fS(nr), fD(nr), z(2 * std::max(nc, 1)), cz(2 * std::max(nc, 1));
  adaptive_fill(&spec, A, E.data(), w.data(), fS.data(), fD.data());
  if (nc > 0) {
    negf_grid_spec cs = spec;
    cs.n_real = 0;
    if (negf_make_grid(&cs, nullptr, nullptr, nullptr, nullptr, z.data(), cz.data()))
      return set_err(c, NEGF_EINVAL, "bad contour of the semi-adaptive grid");
  }
  negf_grid g{nr, E.data(), w.data(), fS.data(), fD.data(), spec.eta, nc, z.data(), cz.data()};
  int rc = set_grid_internal(c, d, &g);
  if (rc) return rc;
  d->spec = spec;
  d->spec.n_real = nr;
  d->spec_set = true;
  d->adaptive = true;
  d->ad = ad;
  d->l1 = A.l1;
  d->l2 = A.l2;
  for (int i = 0; i < 3; ++i) d->seg[i] = A.n[i];
  return NEGF_OK;
}

// Integrand of one ring per energy, I_k = sum over chains in chain order, from either the
// per-lane values the thread-per-lane sweeps captured at that ring (cap, slot chain * n_real + k)
// or, for wider blocks, the per-item partial ring sums of a one-energy-per-item run (item =
// chain * n_real + k); both with unit weights.  The peak is the largest I_k, the lowest k on
// ties: strided scan, then a fixed-shape tree.
__global__ void __launch_bounds__(256) integrand_peak_kernel(const double* partial, const double* cap,
                                                             int n_chains, int n_real, int N, int ring,
                                                             const double* E, double* out, double* best) {
  __shared__ double sv[256];
  __shared__ int sk[256];
  const int t = threadIdx.x;
  double bv = -INFINITY;
  int bk = 0x7fffffff;
  for (int k = t; k < n_real; k += blockDim.x) {
    double v = 0.0;
    for (int ch = 0; ch < n_chains; ++ch)
      v += cap ? cap[(long long)ch * n_real + k] : partial[((long long)ch * n_real + k) * N + ring];
    if (out) out[k] = v;
    if (v > bv) {
      bv = v;
      bk = k;
    }
  }
  sv[t] = bv;
  sk[t] = bk;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s && (sv[t + s] > sv[t] || (sv[t + s] == sv[t] && sk[t + s] < sk[t]))) {
      sv[t] = sv[t + s];
      sk[t] = sk[t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    const int k = sk[0] < n_real ? sk[0] : 0;
    best[0] = E[k];
    best[1] = (double)k;
  }
}

// One sweep of every real-axis energy of d (unit weights, the device's occupations and
// potential), then the integrand of `ring` (out, device, may be null) and its peak into the
// context's refine buffer: best[0] = E_s, best[1] = index, the unit weights (written whenever the
// buffer grows, never overwritten), then the captured values.  Chains of 1 x 1 and 2 x 2 blocks
// keep 32 energies per item and capture each lane's value at the ring; wider blocks run one
// energy per item (their usual item) and read the per-item ring sums.
int integrand_run(Ctx* c, Dev* d, int ring, double* out) {
  const int nr = d->n_real;
  const bool capture = d->block <= 2;
  const size_t bytes = (size_t)(nr + 2 + (size_t)d->n_chains * nr) * sizeof(double);
  if (c->refine.bytes < bytes) {
    std::vector<double> ones(nr + 2 + (size_t)d->n_chains * nr, 1.0);
    int rc = upload(c, c->refine, ones.data(), bytes);
    if (rc) return rc;
  }
  double* best = (double*)c->refine.p;
  const double* ones = best + 2;
  double* cap = best + 2 + nr;
  ViewOverride o;
  o.n_real = nr;
  o.E = (const double*)d->dE.p;
  o.w = ones;
  o.fS = (const double*)d->dfS.p;
  o.fD = (const double*)d->dfD.p;
  o.eta = d->eta;
  o.n_cont = 0;
  o.one_energy_per_item = !capture;
  std::vector<Dev*> one{d};
  std::vector<ViewOverride> ov{o};
  Plan P;
  int rc = build_plan(c, one, &ov, -1, P);
  if (rc) return rc;
  if (capture) {
    P.ring_cap = cap;   // T slots of a one-device plan: chain * n_real + k
    P.cap_ring = ring;
  }
  if ((rc = launch_plan(c, P))) return rc;
  integrand_peak_kernel<<<1, 256, 0, c->stream>>>((const double*)c->scratch.partial.p, capture ? cap : nullptr,
                                                  d->n_chains, nr, d->n_rings, ring, (const double*)d->dE.p, out,
                                                  best);
  if (cudaGetLastError() != cudaSuccess) return set_err(c, NEGF_ECUDA, "integrand launch failed");
  ++c->launches;
  return NEGF_OK;
}

bool adaptive_args_ok(const negf_adaptive* ad) {
  return ad && std::isfinite(ad->a) && std::isfinite(ad->b) && ad->a >= 0.0 && ad->b >= 0.0 && ad->period >= 0;
}

}  // namespace

int refine_grid_internal(Ctx* c, Dev* d, double* E_s) {
  if (!d->adaptive) return set_err(c, NEGF_EINVAL, "the device grid is not semi-adaptive");
  const int ring = d->ad.ring < 0 ? d->n_rings / 2 : d->ad.ring;
  int rc = integrand_run(c, d, ring, nullptr);
  if (rc) return rc;
  double best[2];
  if (cudaMemcpyAsync(best, c->refine.p, sizeof(best), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "integrand sweep failed");
  if (E_s) *E_s = best[0];
  const double kT = d->spec.kT;
  return set_adaptive(c, d, d->spec, d->ad, best[0] - d->ad.a * kT, best[0] + d->ad.b * kT);
}

}  // namespace negf

using namespace negf;

extern "C" {

int negf_make_grid_adaptive(const negf_grid_spec* s, const negf_adaptive* ad, int* n_real, double* E, double* w,
                            double* fS, double* fD, double* z, double* cz) {
  if (!s || !n_real || !adaptive_args_ok(ad)) return NEGF_EINVAL;
  AdaptiveShape A;
  if (adaptive_shape(s, ad->E_l1, ad->E_l2, ad->density, A)) return NEGF_EINVAL;
  *n_real = A.total();
  if (!E) return NEGF_OK;
  if (!w || !fS || !fD) return NEGF_EINVAL;
  adaptive_fill(s, A, E, w, fS, fD);
  if (s->n_cont > 0) {
    negf_grid_spec cs = *s;
    cs.n_real = 0;
    return negf_make_grid(&cs, nullptr, nullptr, nullptr, nullptr, z, cz);
  }
  return NEGF_OK;
}

int negf_set_grid_adaptive(negf_ctx* c, int dev, const negf_grid_spec* s, const negf_adaptive* ad) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  if (d->sc) return set_err(c, NEGF_EBUSY, "device is in a self-consistent session");
  if (!s || !adaptive_args_ok(ad) || (ad->ring < -1 || ad->ring >= d->n_rings))
    return set_err(c, NEGF_EINVAL, "bad semi-adaptive grid arguments");
  cudaSetDevice(c->ordinal);
  return set_adaptive(c, d, *s, *ad, ad->E_l1, ad->E_l2);
}

int negf_ring_integrand(negf_ctx* c, int dev, int ring, double* I) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  if (d->sc) return set_err(c, NEGF_EBUSY, "device is in a self-consistent session");
  int rc = check_ready(c, d);
  if (rc) return rc;
  if (!I || ring < 0 || ring >= d->n_rings || d->n_real < 1) return set_err(c, NEGF_EINVAL, "bad integrand arguments");
  cudaSetDevice(c->ordinal);
  DBuf out;
  if (!ensure(c, out, (size_t)d->n_real * 8)) return NEGF_ENOMEM;
  rc = integrand_run(c, d, ring, (double*)out.p);
  if (!rc && (cudaMemcpyAsync(I, out.p, (size_t)d->n_real * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
              cudaStreamSynchronize(c->stream) != cudaSuccess))
    rc = set_err(c, NEGF_ECUDA, "integrand sweep failed");
  c->arena.release(out);
  return rc;
}

int negf_refine_grid(negf_ctx* c, int dev, double* E_s) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  if (d->sc) return set_err(c, NEGF_EBUSY, "device is in a self-consistent session");
  int rc = check_ready(c, d);
  if (rc) return rc;
  cudaSetDevice(c->ordinal);
  return refine_grid_internal(c, d, E_s);
}

int negf_grid_info(negf_ctx* c, int dev, int* n_real, int* n_cont, double* E_l1, double* E_l2) {
  if (!c) return NEGF_EINVAL;
  Dev* d = find_device(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  if (n_real) *n_real = d->n_real;
  if (n_cont) *n_cont = d->n_cont;
  if (E_l1) *E_l1 = d->adaptive ? d->l1 : NAN;
  if (E_l2) *E_l2 = d->adaptive ? d->l2 : NAN;
  return NEGF_OK;
}

}  // extern "C"
