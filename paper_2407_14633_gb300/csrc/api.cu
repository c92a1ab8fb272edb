// C ABI of libnegf: contexts, device arena, devices, nanotube builders, leads, grids.
// The NEGF evaluation itself is in compute.cu, the self-consistent loop in sc.cu and the
// serving scheduler in serve.cu.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <thread>

#include "ctx.h"

using namespace negf;

namespace negf {

int set_err(Ctx* c, int code, const std::string& msg) {
  if (c) c->last_error = msg;
  return code;
}

bool Arena::alloc(DBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return true;
  release(b);
  if (bytes == 0) bytes = 16;
  ++allocs;
  if (fail_after > 0 && allocs == fail_after) {
    err = "injected allocation failure";
    return false;
  }
  if (budget && used + bytes > budget) {
    err = "device memory budget exceeded";
    return false;
  }
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    err = "cudaMalloc failed";
    return false;
  }
  b.bytes = bytes;
  used += bytes;
  if (used > peak) peak = used;
  return true;
}

void Arena::release(DBuf& b) {
  if (b.p) {
    cudaFree(b.p);
    used -= b.bytes;
  }
  b.p = nullptr;
  b.bytes = 0;
}

bool ensure(Ctx* c, DBuf& b, size_t bytes) {
  if (!c->arena.alloc(b, bytes)) {
    c->last_error = c->arena.err;
    return false;
  }
  return true;
}

int upload(Ctx* c, DBuf& b, const void* src, size_t bytes) {
  if (!ensure(c, b, bytes)) return NEGF_ENOMEM;
  if (bytes && cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "host to device copy failed");
  // keep host buffers valid only for the duration of the call
  if (cudaStreamSynchronize(c->stream) != cudaSuccess)
    return set_err(c, NEGF_ECUDA, "stream synchronize failed");
  return NEGF_OK;
}

}  // namespace negf

namespace {

Dev* get_dev(Ctx* c, int dev) {
  auto it = c->devs.find(dev);
  return it == c->devs.end() ? nullptr : it->second.get();
}

// setters refuse devices that a self-consistent session is using
#define NEGF_NOT_IN_SESSION(c, d) \
  if ((d)->sc) return set_err((c), NEGF_EBUSY, "device is in a self-consistent session")

void free_dev(Ctx* c, Dev* d) {
  for (auto& ch : d->ch) {
    for (DBuf* b : {&ch.dHdiag, &ch.dHup, &ch.dcs_cnt, &ch.dcs_idx, &ch.dcs_val, &ch.drs_cnt, &ch.drs_idx,
                    &ch.drs_val, &ch.dhsq, &ch.dHdiag_f, &ch.dcs_val_f, &ch.drs_val_f, &ch.dhsq_f})
      c->arena.release(*b);
    for (int s = 0; s < 2; ++s)
      for (DBuf* b : {&ch.da1[s], &ch.da2[s], &ch.dat[s], &ch.dsites[s], &ch.dtw[s], &ch.dgen[s]})
        c->arena.release(*b);
  }
  for (DBuf* b : {&d->dU, &d->dE, &d->dw, &d->dfS, &d->dfD, &d->dz, &d->dc, &d->dgb, &d->dn,
                  &d->dnr, &d->dnc, &d->dT, &d->dI})
    c->arena.release(*b);
}

// |lambda_j|^2 of a circulant matrix given by its first row (m complex)
void circulant_moduli(const std::vector<double>& row, int m, std::vector<double>& out) {
  out.assign(m, 0.0);
  for (int j = 0; j < m; ++j) {
    std::complex<double> acc(0.0, 0.0);
    for (int d = 0; d < m; ++d) {
      const double ang = 2.0 * M_PI * (double)((long long)j * d % m) / m;
      acc += std::complex<double>(row[2 * d], row[2 * d + 1]) *
             std::complex<double>(std::cos(ang), std::sin(ang));
    }
    out[j] = std::norm(acc);
  }
}

int upload_lead(Ctx* c, ChainData& ch, int side) {
  HostLead& L = ch.lead[side];
  std::vector<double> a1, a2, at, tw(2 * L.m);
  circulant_moduli(L.T1, L.m, a1);
  circulant_moduli(L.T2, L.m, a2);
  circulant_moduli(L.tau, L.m, at);
  L.a1 = a1;
  L.a2 = a2;
  for (int k = 0; k < L.m; ++k) {
    const double ang = 2.0 * M_PI * k / L.m;
    tw[2 * k] = std::cos(ang);
    tw[2 * k + 1] = std::sin(ang);
  }
  int rc;
  if ((rc = upload(c, ch.da1[side], a1.data(), a1.size() * 8))) return rc;
  if ((rc = upload(c, ch.da2[side], a2.data(), a2.size() * 8))) return rc;
  if ((rc = upload(c, ch.dat[side], at.data(), at.size() * 8))) return rc;
  if ((rc = upload(c, ch.dtw[side], tw.data(), tw.size() * 8))) return rc;
  if ((rc = upload(c, ch.dsites[side], L.sites.data(), L.sites.size() * 4))) return rc;
  return NEGF_OK;
}

// device copies of a chain's Hamiltonian: dense blocks, column-sparse couplings, |h|^2
// complex64 copy of an interleaved complex128 array
static int upload_f32(Ctx* c, DBuf& b, const std::vector<double>& v) {
  std::vector<float> f(std::max<size_t>(v.size(), 2));
  for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
  return upload(c, b, f.data(), f.size() * 4);
}

int upload_chain(Ctx* c, Dev* d, ChainData& ch) {
  const int b = d->block, L = d->L;
  int rc;
  ch.h_sym = true;
  for (int l = 0; l < L && ch.h_sym; ++l)
    for (int r = 0; r < b && ch.h_sym; ++r)
      for (int q = 0; q < b; ++q) {
        const double* v = &ch.Hdiag[2 * ((size_t)l * b * b + (size_t)r * b + q)];
        const double* w = &ch.Hdiag[2 * ((size_t)l * b * b + (size_t)q * b + r)];
        if (v[1] != 0.0 || v[0] != w[0]) {
          ch.h_sym = false;
          break;
        }
      }
  for (size_t i = 1; i < ch.Hup.size() && ch.h_sym; i += 2)
    if (ch.Hup[i] != 0.0) ch.h_sym = false;
  // uniform layers (a tube of one ring type): the block sweeps read layer 0's blocks only
  const size_t bb2 = 2 * (size_t)b * b;
  bool hd_uniform = true, cp_uniform = true;
  for (int l = 1; l < L && hd_uniform; ++l)
    hd_uniform = std::equal(ch.Hdiag.begin() + l * bb2, ch.Hdiag.begin() + (l + 1) * bb2, ch.Hdiag.begin());
  for (int l = 1; l < L - 1 && cp_uniform; ++l)
    cp_uniform = std::equal(ch.Hup.begin() + l * bb2, ch.Hup.begin() + (l + 1) * bb2, ch.Hup.begin());
  ch.hd_step = hd_uniform ? 0 : b * b;
  ch.cp_step = cp_uniform ? 0 : b;
  if ((rc = upload(c, ch.dHdiag, ch.Hdiag.data(), ch.Hdiag.size() * 8))) return rc;
  if ((rc = upload_f32(c, ch.dHdiag_f, ch.Hdiag))) return rc;
  if ((rc = upload(c, ch.dHup, ch.Hup.data(), std::max<size_t>(ch.Hup.size(), 2) * 8))) return rc;
  int kmax = 1;
  for (int l = 0; l < L - 1; ++l)
    for (int col = 0; col < b; ++col) {
      int n = 0;
      for (int r = 0; r < b; ++r) {
        const double* v = &ch.Hup[2 * ((size_t)l * b * b + (size_t)r * b + col)];
        if (v[0] != 0.0 || v[1] != 0.0) ++n;
      }
      kmax = std::max(kmax, n);
    }
  const int nl = std::max(L - 1, 1);
  std::vector<int> cnt((size_t)nl * b, 0), idx((size_t)nl * b * kmax, 0);
  std::vector<double> val((size_t)nl * b * kmax * 2, 0.0);
  for (int l = 0; l < L - 1; ++l)
    for (int col = 0; col < b; ++col) {
      int n = 0;
      for (int r = 0; r < b; ++r) {
        const double* v = &ch.Hup[2 * ((size_t)l * b * b + (size_t)r * b + col)];
        if (v[0] != 0.0 || v[1] != 0.0) {
          const size_t e = ((size_t)l * b + col) * kmax + n;
          idx[e] = r;
          val[2 * e] = v[0];
          val[2 * e + 1] = v[1];
          ++n;
        }
      }
      cnt[(size_t)l * b + col] = n;
    }
  ch.kmax = kmax;
  if ((rc = upload(c, ch.dcs_cnt, cnt.data(), cnt.size() * 4))) return rc;
  if ((rc = upload(c, ch.dcs_idx, idx.data(), idx.size() * 4))) return rc;
  if ((rc = upload(c, ch.dcs_val, val.data(), val.size() * 8))) return rc;
  if ((rc = upload_f32(c, ch.dcs_val_f, val))) return rc;
  // row-sparse form (row r: entries (column, value)), padded to the same kmax
  int rkmax = 1;
  for (int l = 0; l < L - 1; ++l)
    for (int r = 0; r < b; ++r) {
      int n = 0;
      for (int col = 0; col < b; ++col) {
        const double* v = &ch.Hup[2 * ((size_t)l * b * b + (size_t)r * b + col)];
        if (v[0] != 0.0 || v[1] != 0.0) ++n;
      }
      rkmax = std::max(rkmax, n);
    }
  const int km = std::max(kmax, rkmax);
  if (km != kmax) {
    // re-pad the column form to the common width
    std::vector<int> idx2((size_t)nl * b * km, 0);
    std::vector<double> val2((size_t)nl * b * km * 2, 0.0);
    for (size_t q = 0; q < (size_t)nl * b; ++q)
      for (int e = 0; e < kmax; ++e) {
        idx2[q * km + e] = idx[q * kmax + e];
        val2[2 * (q * km + e)] = val[2 * (q * kmax + e)];
        val2[2 * (q * km + e) + 1] = val[2 * (q * kmax + e) + 1];
      }
    if ((rc = upload(c, ch.dcs_idx, idx2.data(), idx2.size() * 4))) return rc;
    if ((rc = upload(c, ch.dcs_val, val2.data(), val2.size() * 8))) return rc;
    if ((rc = upload_f32(c, ch.dcs_val_f, val2))) return rc;
    ch.kmax = km;
  }
  std::vector<int> rcnt((size_t)nl * b, 0), ridx((size_t)nl * b * km, 0);
  std::vector<double> rval((size_t)nl * b * km * 2, 0.0);
  for (int l = 0; l < L - 1; ++l)
    for (int r = 0; r < b; ++r) {
      int n = 0;
      for (int col = 0; col < b; ++col) {
        const double* v = &ch.Hup[2 * ((size_t)l * b * b + (size_t)r * b + col)];
        if (v[0] != 0.0 || v[1] != 0.0) {
          const size_t e = ((size_t)l * b + r) * km + n;
          ridx[e] = col;
          rval[2 * e] = v[0];
          rval[2 * e + 1] = v[1];
          ++n;
        }
      }
      rcnt[(size_t)l * b + r] = n;
    }
  if ((rc = upload(c, ch.drs_cnt, rcnt.data(), rcnt.size() * 4))) return rc;
  if ((rc = upload(c, ch.drs_idx, ridx.data(), ridx.size() * 4))) return rc;
  if ((rc = upload(c, ch.drs_val, rval.data(), rval.size() * 8))) return rc;
  if ((rc = upload_f32(c, ch.drs_val_f, rval))) return rc;
  std::vector<double> hsq(nl, 0.0);
  if (b == 1)
    for (int l = 0; l < L - 1; ++l) hsq[l] = ch.Hup[2 * l] * ch.Hup[2 * l] + ch.Hup[2 * l + 1] * ch.Hup[2 * l + 1];
  ch.diag_real = true;
  for (size_t i = 1; i < ch.Hdiag.size(); i += 2) ch.diag_real = ch.diag_real && ch.Hdiag[i] == 0.0;
  std::vector<float> hsq_f(hsq.begin(), hsq.end());
  if ((rc = upload(c, ch.dhsq_f, hsq_f.data(), hsq_f.size() * 4))) return rc;
  return upload(c, ch.dhsq, hsq.data(), hsq.size() * 8);
}

// ---- nanotube bonds (Sec. 3.1 nearest-neighbour ring coupling)
int pmod(long long k, int m) { return (int)(((k % m) + m) % m); }

double mode_bond(long long k, double t, double bj) { return pmod(k, 2) == 0 ? t : bj; }

// first row of the circulant bond H_{k,k+1} of the real-space (n,0) tube:
// t I (k even), t (I + S) (k = 1 mod 4), t (I + S^T) (k = 3 mod 4), S[r][r-1] = 1
std::vector<double> real_bond_row(long long k, double t, int n) {
  std::vector<double> row(2 * n, 0.0);
  row[0] = t;
  if (pmod(k, 2) == 1) {
    if (pmod(k, 4) == 1)
      row[2 * (n - 1)] += t;   // S: entry at (r, r-1) -> d = -1
    else
      row[2 * 1] += t;         // S^T: entry at (r, r+1) -> d = +1
  }
  return row;
}
// first row of the Hermitian conjugate of a circulant matrix given by its first row
std::vector<double> dagger_row(const std::vector<double>& row, int n) {
  std::vector<double> out(2 * n);
  for (int d = 0; d < n; ++d) {
    const int s = pmod(-d, n);
    out[2 * d] = row[2 * s];
    out[2 * d + 1] = -row[2 * s + 1];
  }
  return out;
}

// ---- quadrature on the host (grids are set-up data, uploaded once per bias point)
// Gauss-Legendre by Newton iteration on P_n with the three-term recurrence.  The rule is
// symmetric (x_{n-1-k} = -x_k), so only the upper half of the nodes is iterated; large
// rules spread the nodes over host threads (each node is independent).
void gl_node(int n, int i, double& x_out, double& w_out) {
  double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = z;
    for (int j = 1; j < n; ++j) {
      const double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
      p0 = p1;
      p1 = p2;
    }
    const double dp = n * (z * p1 - p0) / (z * z - 1.0);
    const double dz = p1 / dp;
    z -= dz;
    if (std::fabs(dz) < 1e-16) break;
  }
  double p0 = 1.0, p1 = z;
  for (int j = 1; j < n; ++j) {
    const double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
    p0 = p1;
    p1 = p2;
  }
  const double dp = n * (z * p1 - p0) / (z * z - 1.0);
  x_out = z;
  w_out = 2.0 / ((1.0 - z * z) * dp * dp);
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const int half = (n + 1) / 2;   // nodes i = 0..half-1 are the non-negative ones
  auto work = [&](int i0, int i1) {
    for (int i = i0; i < i1; ++i) {
      double z, wz;
      gl_node(n, i, z, wz);
      x[n - 1 - i] = z;
      w[n - 1 - i] = wz;
      x[i] = -z;
      w[i] = wz;
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (n < 512 || nt < 2) {
    work(0, half);
  } else {
    nt = std::min<unsigned>(nt, 32);
    std::vector<std::thread> th;
    const int chunk = (half + (int)nt - 1) / (int)nt;
    for (unsigned t = 0; t < nt; ++t) {
      const int i0 = (int)t * chunk, i1 = std::min(half, i0 + chunk);
      if (i0 < i1) th.emplace_back(work, i0, i1);
    }
    for (auto& t : th) t.join();
  }
  if (n % 2) x[n / 2] = 0.0;   // the middle node of an odd rule is exactly 0
}

}  // namespace

namespace negf {
// nodes z_k and weights W_k z'(theta_k) of the upper semicircle over [E_B, E_end]:
// theta_k = (pi/2)(1 + x_k), W_k = (pi/2) w_k, z = c + R e^{i theta}, z' = i R e^{i theta}
void contour_arc(double E_B, double E_end, int n, double* z, double* zw) {
  std::vector<double> x, wg;
  gauss_legendre(n, x, wg);
  const double cc = 0.5 * (E_B + E_end), R = 0.5 * (E_end - E_B);
  for (int k = 0; k < n; ++k) {
    const double th = 0.5 * M_PI * (1.0 + x[k]);
    const double W = 0.5 * M_PI * wg[k];
    const std::complex<double> e(std::cos(th), std::sin(th));
    const std::complex<double> zk = cc + R * e;
    const std::complex<double> dz = std::complex<double>(0.0, R) * e;
    z[2 * k] = zk.real();
    z[2 * k + 1] = zk.imag();
    zw[2 * k] = (W * dz).real();
    zw[2 * k + 1] = (W * dz).imag();
  }
}
}  // namespace negf

namespace {
double fermi_real(double x, double kT) {
  const double y = x / kT;
  if (y > 0.0) {
    const double e = std::exp(-y);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + std::exp(y));
}

}  // namespace

namespace negf {
void gl_rule(int n, std::vector<double>& x, std::vector<double>& w) { gauss_legendre(n, x, w); }
double fermi_host(double x, double kT) { return fermi_real(x, kT); }

// negf_set_grid without the session check (the semi-adaptive grid is rebuilt inside a
// self-consistent session)
int set_grid_internal(Ctx* c, Dev* d, const negf_grid* g) {
  if (!g || g->n_real < 0 || g->n_cont < 0 || g->n_real + g->n_cont == 0 || !(g->eta >= 0.0))
    return set_err(c, NEGF_EINVAL, "bad grid");
  if (g->n_real > 0 && (!g->E || !g->w || !g->fS || !g->fD)) return set_err(c, NEGF_EINVAL, "null real-axis grid array");
  if (g->n_cont > 0 && (!g->z || !g->c)) return set_err(c, NEGF_EINVAL, "null contour array");
  for (int k = 0; k < g->n_cont; ++k)
    if (!(g->z[2 * k + 1] > 0.0)) return set_err(c, NEGF_EINVAL, "contour node not in the upper half plane");
  if (g->n_real > 0 && !(g->eta > 0.0)) return set_err(c, NEGF_EINVAL, "real-axis energies need eta > 0");
  cudaSetDevice(c->ordinal);
  int rc;
  const size_t nr = std::max(g->n_real, 1), nc = std::max(g->n_cont, 1);
  std::vector<double> zero(2 * std::max(nr, nc), 0.0);
  if ((rc = upload(c, d->dE, g->n_real ? g->E : zero.data(), nr * 8))) return rc;
  if ((rc = upload(c, d->dw, g->n_real ? g->w : zero.data(), nr * 8))) return rc;
  if ((rc = upload(c, d->dfS, g->n_real ? g->fS : zero.data(), nr * 8))) return rc;
  if ((rc = upload(c, d->dfD, g->n_real ? g->fD : zero.data(), nr * 8))) return rc;
  if ((rc = upload(c, d->dz, g->n_cont ? g->z : zero.data(), nc * 16))) return rc;
  if ((rc = upload(c, d->dc, g->n_cont ? g->c : zero.data(), nc * 16))) return rc;
  d->n_real = g->n_real;
  d->n_cont = g->n_cont;
  d->eta = g->eta;
  d->hE.assign(g->E, g->E + g->n_real);
  d->grid_set = true;
  d->spec_set = false;
  d->adaptive = false;
  return NEGF_OK;
}
}  // namespace negf

// =====================================================================================
extern "C" {

const char* negf_strerror(int s) {
  switch (s) {
    case NEGF_OK: return "ok";
    case NEGF_EINVAL: return "invalid argument";
    case NEGF_ENOMEM: return "out of device memory or over budget";
    case NEGF_ECUDA: return "CUDA error";
    case NEGF_ETIMEDOUT: return "timed out";
    case NEGF_ENOTCONVERGED: return "self-consistent loop did not converge";
    case NEGF_EBUSY: return "busy";
    case NEGF_ENOTFOUND: return "not found";
  }
  return "unknown status";
}

const char* negf_last_error(const negf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int negf_create(negf_ctx** out, const negf_opts* opts) {
  if (!out) return NEGF_EINVAL;
  *out = nullptr;
  negf_ctx* c = new (std::nothrow) negf_ctx();
  if (!c) return NEGF_ENOMEM;
  if (opts) c->opts = *opts;
  const int bw = c->opts.blk_warps, cw = c->opts.chain_warps;
  if (c->opts.precision < 0 || c->opts.precision > 2 || !(bw == -1 || bw == 0 || bw == 1 || bw == 2 || bw == 4) ||
      c->opts.blk_ctas_per_sm < 0 || !(cw == 0 || cw == 1 || cw == 2 || cw == 4 || cw == 8) ||
      c->opts.long_chain_split < -1 || c->opts.long_chain_split > 1 || c->opts.mixed_two_pass < -1 ||
      c->opts.mixed_two_pass > 1) {
    delete c;
    return NEGF_EINVAL;
  }
  if (c->opts.flag_threshold <= 0.0) c->opts.flag_threshold = 1e-3;
  if (c->opts.edge_window <= 0.0) c->opts.edge_window = 0.002;
  c->ordinal = c->opts.device_ordinal;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    delete c;
    return NEGF_ECUDA;
  }
  if (c->ordinal < 0 || c->ordinal >= ndev || cudaSetDevice(c->ordinal) != cudaSuccess) {
    delete c;
    return NEGF_EINVAL;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->ordinal);
  if (c->opts.stream) {
    c->stream = (cudaStream_t)c->opts.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return NEGF_ECUDA;
    }
    c->own_stream = true;
  }
  c->arena.budget = c->opts.hbm_budget_bytes;
  c->arena.fail_after = c->opts.fault_alloc_after;
  *out = c;
  return NEGF_OK;
}

int negf_destroy(negf_ctx* c) {
  if (!c) return NEGF_EINVAL;
  cudaSetDevice(c->ordinal);
  cudaStreamSynchronize(c->stream);
  serve_free(c);
  for (auto& kv : c->devs) {
    sc_session_free(c, kv.second.get());
    free_dev(c, kv.second.get());
  }
  c->devs.clear();
  for (auto& pr : c->prof_events) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  free_plan_bufs(c, c->scratch);
  c->arena.release(c->lane_stats);
  c->arena.release(c->cond);
  c->arena.release(c->refine);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return NEGF_OK;
}

int negf_launch_count(const negf_ctx* c, uint64_t* n) {
  if (!c || !n) return NEGF_EINVAL;
  *n = c->launches;
  return NEGF_OK;
}

int negf_device_create(negf_ctx* c, int n_rings, int block, int rpb, int n_chains, int* dev) {
  if (!c || !dev) return NEGF_EINVAL;
  if (n_rings < 1 || block < 1 || block > MAX_BLOCK || (rpb != 1 && rpb != 2) || block % rpb ||
      n_rings % rpb || n_chains < 1 || n_chains > 8)
    return set_err(c, NEGF_EINVAL, "device shape out of range");
  std::unique_ptr<Dev> d(new Dev());
  d->n_rings = n_rings;
  d->block = block;
  d->rpb = rpb;
  d->n_chains = n_chains;
  d->L = n_rings / rpb;
  d->ch.resize(n_chains);
  d->U.assign(n_rings, 0.0);
  const int id = c->next_dev++;
  c->devs[id] = std::move(d);
  *dev = id;
  return NEGF_OK;
}

int negf_device_destroy(negf_ctx* c, int dev) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  cudaStreamSynchronize(c->stream);
  sc_session_free(c, d);
  free_dev(c, d);
  c->devs.erase(dev);
  return NEGF_OK;
}

int negf_set_hamiltonian(negf_ctx* c, int dev, int chain, const double* Hdiag, const double* Hup,
                         double g_b) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  if (chain < 0 || chain >= d->n_chains || !Hdiag || (!Hup && d->L > 1) || !(g_b > 0.0))
    return set_err(c, NEGF_EINVAL, "bad hamiltonian arguments");
  ChainData& ch = d->ch[chain];
  const size_t bb = (size_t)d->block * d->block;
  ch.Hdiag.assign(Hdiag, Hdiag + 2 * bb * d->L);
  if (d->L > 1)
    ch.Hup.assign(Hup, Hup + 2 * bb * (d->L - 1));
  else
    ch.Hup.assign(2, 0.0);
  for (double v : ch.Hdiag)
    if (!std::isfinite(v)) return set_err(c, NEGF_EINVAL, "non-finite hamiltonian entry");
  for (double v : ch.Hup)
    if (!std::isfinite(v)) return set_err(c, NEGF_EINVAL, "non-finite hamiltonian entry");
  ch.g_b = g_b;
  cudaSetDevice(c->ordinal);
  int rc = upload_chain(c, d, ch);
  if (rc) return rc;
  ch.h_set = true;
  return NEGF_OK;
}

int negf_set_lead(negf_ctx* c, int dev, int chain, int side, const negf_lead* lead) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  if (!lead || chain < 0 || chain >= d->n_chains || (side != 0 && side != 1) || lead->m < 1 ||
      lead->m > MAX_LEAD || lead->m > d->block || !lead->T1 || !lead->T2 || !lead->tau || !lead->sites)
    return set_err(c, NEGF_EINVAL, "bad lead arguments");
  if (d->block <= 2 && lead->m != 1)
    return set_err(c, NEGF_EINVAL, "blocks of width 1 or 2 take single-site leads");
  for (int s = 0; s < lead->m; ++s) {
    if (lead->sites[s] < 0 || lead->sites[s] >= d->block)
      return set_err(c, NEGF_EINVAL, "lead site outside the boundary layer");
    for (int t = 0; t < s; ++t)
      if (lead->sites[t] == lead->sites[s]) return set_err(c, NEGF_EINVAL, "lead site listed twice");
  }
  HostLead& L = d->ch[chain].lead[side];
  L.gen = false;
  L.m = lead->m;
  L.U = lead->U_lead;
  L.T1.assign(lead->T1, lead->T1 + 2 * L.m);
  L.T2.assign(lead->T2, lead->T2 + 2 * L.m);
  L.tau.assign(lead->tau, lead->tau + 2 * L.m);
  L.sites.assign(lead->sites, lead->sites + L.m);
  cudaSetDevice(c->ordinal);
  int rc = upload_lead(c, d->ch[chain], side);
  if (rc) return rc;
  L.set = true;
  return NEGF_OK;
}

int negf_set_lead_general(negf_ctx* c, int dev, int chain, int side, const negf_lead_general* g) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  if (!g || chain < 0 || chain >= d->n_chains || (side != 0 && side != 1) || g->m < 1 || g->m > MAX_GEN_LEAD ||
      g->m > d->block || !g->T1 || !g->T2 || !g->tau || !g->sites || !std::isfinite(g->U_lead) ||
      g->max_iter < 0 || !(g->tol >= 0.0))
    return set_err(c, NEGF_EINVAL, "bad general lead arguments");
  if (d->block <= 2)
    return set_err(c, NEGF_EINVAL, "general leads need ring blocks wider than 2 (single-site leads have a closed form)");
  const int m = g->m;
  for (int s = 0; s < m; ++s) {
    if (g->sites[s] < 0 || g->sites[s] >= d->block) return set_err(c, NEGF_EINVAL, "lead site outside the boundary layer");
    for (int t = 0; t < s; ++t)
      if (g->sites[t] == g->sites[s]) return set_err(c, NEGF_EINVAL, "lead site listed twice");
  }
  const size_t mm2 = (size_t)2 * m * m;
  std::vector<double> mats(5 * mm2, 0.0);
  const double* src[5] = {g->H0, g->H1, g->T1, g->T2, g->tau};
  for (int k = 0; k < 5; ++k)
    if (src[k]) std::copy(src[k], src[k] + mm2, mats.begin() + k * mm2);
  for (double v : mats)
    if (!std::isfinite(v)) return set_err(c, NEGF_EINVAL, "non-finite general lead entry");
  // the on-site blocks must be Hermitian
  for (int k = 0; k < 2; ++k)
    for (int r = 0; r < m; ++r)
      for (int q = 0; q < m; ++q) {
        const double* a = mats.data() + k * mm2 + 2 * (r * m + q);
        const double* b = mats.data() + k * mm2 + 2 * (q * m + r);
        if (std::fabs(a[0] - b[0]) > 1e-12 * (1.0 + std::fabs(a[0])) || std::fabs(a[1] + b[1]) > 1e-12 * (1.0 + std::fabs(a[1])))
          return set_err(c, NEGF_EINVAL, "on-site block of a general lead is not Hermitian");
      }
  cudaSetDevice(c->ordinal);
  ChainData& ch = d->ch[chain];
  int rc = upload(c, ch.dgen[side], mats.data(), mats.size() * 8);
  if (rc) return rc;
  std::vector<int> sites(g->sites, g->sites + m);
  if ((rc = upload(c, ch.dsites[side], sites.data(), sites.size() * sizeof(int)))) return rc;
  HostLead& L = ch.lead[side];
  L.m = m;
  L.U = g->U_lead;
  L.gen = true;
  L.gmats = mats;
  L.max_iter = g->max_iter ? g->max_iter : 400;
  L.tol = g->tol > 0.0 ? g->tol : 1e-14;
  L.sites = sites;
  // no closed-form band edges (the mixed path's edge windows skip this lead) and no first rows
  L.a1.clear();
  L.a2.clear();
  L.T1.assign(2 * m, 0.0);
  L.T2.assign(2 * m, 0.0);
  L.tau.assign(2 * m, 0.0);
  L.set = true;
  return NEGF_OK;
}

int negf_set_lead_potentials(negf_ctx* c, int dev, double U_S, double U_D) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  for (auto& ch : d->ch) {
    ch.lead[0].U = U_S;
    ch.lead[1].U = U_D;
  }
  return NEGF_OK;
}

int negf_build_cnt_modespace(negf_ctx* c, int dev, int n_tube, double t, const int* modes,
                             double U_S, double U_D) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  if (!modes || n_tube < 1) return set_err(c, NEGF_EINVAL, "bad builder arguments");
  const bool cells = (d->block == 2 && d->rpb == 2);
  if (!(d->block == 1 && d->rpb == 1) && !cells)
    return set_err(c, NEGF_EINVAL, "mode space needs block 1, or block 2 with 2 rings per block");
  const int N = d->n_rings, L = d->L, b = d->block;
  for (int ci = 0; ci < d->n_chains; ++ci) {
    const double bj = 2.0 * t * std::cos(M_PI * modes[ci] / n_tube);
    std::vector<double> Hd((size_t)2 * b * b * L, 0.0), Hu((size_t)2 * b * b * std::max(L - 1, 1), 0.0);
    if (!cells) {
      for (int l = 0; l < L - 1; ++l) Hu[2 * l] = mode_bond(l, t, bj);
    } else {
      for (int l = 0; l < L; ++l) {
        const double h = mode_bond(2LL * l, t, bj);
        Hd[2 * (4 * l + 1)] = h;   // (0,1)
        Hd[2 * (4 * l + 2)] = h;   // (1,0)
      }
      for (int l = 0; l < L - 1; ++l) Hu[2 * (4 * l + 2)] = mode_bond(2LL * l + 1, t, bj);  // (1,0)
    }
    int rc = negf_set_hamiltonian(c, dev, ci, Hd.data(), Hu.data(), 2.0);
    if (rc) return rc;
    const double zero = 0.0;
    (void)zero;
    double T1[2], T2[2], tau[2];
    int site = 0;
    negf_lead ld{1, U_S, T1, T2, tau, &site};
    T1[0] = mode_bond(-2, t, bj); T1[1] = 0.0;
    T2[0] = mode_bond(-3, t, bj); T2[1] = 0.0;
    tau[0] = mode_bond(-1, t, bj); tau[1] = 0.0;
    if ((rc = negf_set_lead(c, dev, ci, NEGF_SOURCE, &ld))) return rc;
    int siteD = cells ? 1 : 0;
    T1[0] = mode_bond(N, t, bj);
    T2[0] = mode_bond((long long)N + 1, t, bj);
    tau[0] = mode_bond((long long)N - 1, t, bj);
    negf_lead ldD{1, U_D, T1, T2, tau, &siteD};
    if ((rc = negf_set_lead(c, dev, ci, NEGF_DRAIN, &ldD))) return rc;
  }
  return NEGF_OK;
}

int negf_build_cnt_realspace(negf_ctx* c, int dev, int n_tube, double t, double U_S, double U_D) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  if (d->block != n_tube || d->rpb != 1 || d->n_chains != 1)
    return set_err(c, NEGF_EINVAL, "real space needs block = n_tube, 1 ring per block, 1 chain");
  const int n = n_tube, N = d->n_rings, L = d->L;
  std::vector<double> Hd((size_t)2 * n * n * L, 0.0), Hu((size_t)2 * n * n * std::max(L - 1, 1), 0.0);
  for (int l = 0; l < L - 1; ++l) {
    const std::vector<double> row = real_bond_row(l, t, n);
    for (int r = 0; r < n; ++r)
      for (int s = 0; s < n; ++s) {
        const int dd = pmod(s - r, n);
        Hu[2 * ((size_t)l * n * n + (size_t)r * n + s)] = row[2 * dd];
        Hu[2 * ((size_t)l * n * n + (size_t)r * n + s) + 1] = row[2 * dd + 1];
      }
  }
  int rc = negf_set_hamiltonian(c, dev, 0, Hd.data(), Hu.data(), 1.0);
  if (rc) return rc;
  std::vector<int> sites(n);
  for (int s = 0; s < n; ++s) sites[s] = s;
  std::vector<double> T1 = real_bond_row(-2, t, n), T2 = real_bond_row(-3, t, n), tau = real_bond_row(-1, t, n);
  negf_lead lS{n, U_S, T1.data(), T2.data(), tau.data(), sites.data()};
  if ((rc = negf_set_lead(c, dev, 0, NEGF_SOURCE, &lS))) return rc;
  std::vector<double> T1d = dagger_row(real_bond_row(N, t, n), n);
  std::vector<double> T2d = dagger_row(real_bond_row((long long)N + 1, t, n), n);
  std::vector<double> taud = dagger_row(real_bond_row((long long)N - 1, t, n), n);
  negf_lead lD{n, U_D, T1d.data(), T2d.data(), taud.data(), sites.data()};
  return negf_set_lead(c, dev, 0, NEGF_DRAIN, &lD);
}

int negf_set_potential(negf_ctx* c, int dev, const double* U) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  if (!U) return set_err(c, NEGF_EINVAL, "null potential");
  for (int i = 0; i < d->n_rings; ++i)
    if (!std::isfinite(U[i])) return set_err(c, NEGF_EINVAL, "non-finite potential");
  d->U.assign(U, U + d->n_rings);
  cudaSetDevice(c->ordinal);
  int rc = upload(c, d->dU, U, (size_t)d->n_rings * 8);
  if (rc) return rc;
  d->u_set = true;
  return NEGF_OK;
}

int negf_set_grid(negf_ctx* c, int dev, const negf_grid* g) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  return set_grid_internal(c, d, g);
}

int negf_make_grid(const negf_grid_spec* s, double* E, double* w, double* fS, double* fD, double* z,
                   double* cz) {
  if (!s || s->n_real < 0 || s->n_cont < 0 || !(s->kT > 0.0)) return NEGF_EINVAL;
  if (s->n_real > 0 && (!E || !w || !fS || !fD)) return NEGF_EINVAL;
  if (s->n_cont > 0 && (!z || !cz)) return NEGF_EINVAL;
  const double mu_min = std::min(s->mu_S, s->mu_D), mu_max = std::max(s->mu_S, s->mu_D);
  const double f1 = std::isnan(s->f1) ? 14.0 : s->f1, f2 = std::isnan(s->f2) ? 14.0 : s->f2;
  const double Emin = std::isnan(s->E_min) ? mu_min - f1 * s->kT : s->E_min;
  const double Emax = std::isnan(s->E_max) ? mu_max + f2 * s->kT : s->E_max;
  if (!(Emax > Emin)) return NEGF_EINVAL;
  if (s->n_real > 0) {
    if (s->rule == NEGF_RULE_GAUSS) {
      std::vector<double> x, wg;
      gauss_legendre(s->n_real, x, wg);
      const double h = 0.5 * (Emax - Emin), m = 0.5 * (Emax + Emin);
      for (int k = 0; k < s->n_real; ++k) {
        E[k] = m + h * x[k];
        w[k] = h * wg[k];
      }
    } else if (s->rule == NEGF_RULE_MIDPOINT) {
      const double h = (Emax - Emin) / s->n_real;
      for (int k = 0; k < s->n_real; ++k) {
        E[k] = Emin + (k + 0.5) * h;
        w[k] = h;
      }
    } else {
      return NEGF_EINVAL;
    }
    for (int k = 0; k < s->n_real; ++k) {
      fS[k] = fermi_real(E[k] - s->mu_S, s->kT);
      fD[k] = fermi_real(E[k] - s->mu_D, s->kT);
    }
  }
  if (s->n_cont > 0) {
    if (!(Emin > s->E_B)) return NEGF_EINVAL;
    contour_arc(s->E_B, Emin, s->n_cont, z, cz);
    for (int k = 0; k < s->n_cont; ++k) {
      const std::complex<double> zk(z[2 * k], z[2 * k + 1]);
      const std::complex<double> f = 1.0 / (1.0 + std::exp((zk - mu_min) / s->kT));
      const std::complex<double> ck = std::complex<double>(cz[2 * k], cz[2 * k + 1]) * f;
      cz[2 * k] = ck.real();
      cz[2 * k + 1] = ck.imag();
    }
  }
  return NEGF_OK;
}

int negf_set_grid_spec(negf_ctx* c, int dev, const negf_grid_spec* s) {
  if (!c) return NEGF_EINVAL;
  Dev* d = get_dev(c, dev);
  if (!d) return set_err(c, NEGF_ENOTFOUND, "unknown device");
  NEGF_NOT_IN_SESSION(c, d);
  if (!s) return set_err(c, NEGF_EINVAL, "null grid spec");
  std::vector<double> E(s->n_real), w(s->n_real), fS(s->n_real), fD(s->n_real), z(2 * s->n_cont), cz(2 * s->n_cont);
  int rc = negf_make_grid(s, E.data(), w.data(), fS.data(), fD.data(), z.data(), cz.data());
  if (rc) return set_err(c, rc, "bad grid spec");
  negf_grid g{s->n_real, E.data(), w.data(), fS.data(), fD.data(), s->eta, s->n_cont, z.data(), cz.data()};
  if ((rc = negf_set_grid(c, dev, &g))) return rc;
  d->spec = *s;
  d->spec_set = true;
  return NEGF_OK;
}

double negf_poisson_kappa(double eps_r, double d_nm, double t_ox_nm, double dx_nm) {
  const double eps0 = 8.8541878128e-12, e = 1.602176634e-19;
  const double Cg = 2.0 * M_PI * eps0 * eps_r / std::log((2.0 * t_ox_nm + d_nm) / d_nm);
  return e / (Cg * dx_nm * 1e-9);
}

}  // extern "C"
