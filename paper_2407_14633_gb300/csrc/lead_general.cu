// Self-energies of general (non-circulant) leads by decimation (Eq. GR, Sec. 2.2.2: the
// paper computes the surface Green's function by Lopez Sancho-Rubio decimation where no closed
// form applies).  The lead is a chain of rings s0, s1, s2, ... with couplings H_{s1,s0} = T1,
// H_{s2,s1} = T2 alternating, on-site blocks U + H0 (even rings) and U + H1 (odd rings),
// written as a uniform chain of two-ring principal layers:
//   h = [[H0, T1^dag], [T1, H1]],  a = H_{k,k+1} = [[0, 0], [T2^dag, 0]],  c = a^dagger.
// Eliminating every odd layer renormalises (g = (eps - U - h)^{-1}):
//   h_s <- h_s + a g c,  h <- h + a g c + c g a,  a <- a g a,  c <- c g c
// until the couplings vanish; g_s = (eps - U - h_s)^{-1}, g_{s0} its upper-left m x m block,
// Sigma = tau^dagger g_{s0} tau, Gamma = i (Sigma - Sigma^dagger), and the sweep takes a
// factor L of Gamma = L L^dagger from a Cholesky factorisation with diagonal pivoting (columns
// past the numerical rank are zero).
// One CTA per (lead, energy); the 2m x 2m matrices live in shared memory.  The loop is
// bounded: a decimation that has not converged after max_iter steps counts in *status.
#include <cmath>

#include "common.cuh"

namespace negf {

namespace {

// threads per CTA (one CTA per SM: its 2m x 2m matrices fill most of the shared memory).  The
// decimation is bound by the sequential pivot steps of its inverses; 512 threads were no faster.
constexpr int GT = 256;

__device__ __forceinline__ cd cconj(cd a) { return mk(a.re, -a.im); }

// In-place Gauss-Jordan inverse of the n x n matrix A (ld n) with partial pivoting; col and
// perm are n-long scratch.  Row swaps are undone on the columns at the end.
__device__ void gj_inverse(cd* A, int n, cd* col, int* perm, double* rv, int* ri) {
  const int t = threadIdx.x;
  for (int k = 0; k < n; ++k) {
    if (t < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + t; i < n; i += 32) {
        const double v = abs2(A[i * n + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (t == 0) {
        rv[0] = best;
        ri[0] = bi;
        perm[k] = bi;
      }
    }
    __syncthreads();
    const int p = ri[0];
    if (p != k)
      for (int j = t; j < n; j += GT) {
        const cd x = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = x;
      }
    __syncthreads();
    const cd piv = A[k * n + k];
    const double s = 1.0 / abs2(piv);
    const cd ip = mk(piv.re * s, -piv.im * s);
    for (int i = t; i < n; i += GT) col[i] = A[i * n + k];
    __syncthreads();
    for (int j = t; j < n; j += GT) A[k * n + j] = (j == k) ? ip : A[k * n + j] * ip;
    __syncthreads();
    for (int o = t; o < n * n; o += GT) {
      const int i = o / n, j = o - i * n;
      if (i == k) continue;
      const cd rk = A[k * n + j];
      const cd base = (j == k) ? mk(0.0, 0.0) : A[o];
      A[o] = base - col[i] * rk;
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = t; i < n; i += GT) {
        const cd x = A[i * n + k];
        A[i * n + k] = A[i * n + p];
        A[i * n + p] = x;
      }
    __syncthreads();
  }
}

// sum_k X[i][k] Y[k][j] over n
__device__ __forceinline__ cd rowcol(const cd* X, const cd* Y, int i, int j, int n) {
  cd v = mk(0.0, 0.0);
  for (int k = 0; k < n; ++k) v = cmac(v, X[i * n + k], Y[k * n + j]);
  return v;
}

__global__ void __launch_bounds__(GT, 1) lead_general_kernel(const GenLeadJob* jobs, int* status) {
  const GenLeadJob& J = jobs[blockIdx.y];
  const int e = blockIdx.x;
  if (e >= J.n_real + J.n_cont) return;
  const int m = J.m, n = 2 * m, nn = n * n, t = threadIdx.x;
  extern __shared__ __align__(16) unsigned char sm_gen[];
  cd* hs = reinterpret_cast<cd*>(sm_gen);
  cd* h = hs + nn;
  cd* a = h + nn;
  cd* c = a + nn;
  cd* W1 = c + nn;
  cd* W2 = W1 + nn;
  cd* W3 = W2 + nn;
  cd* col = W3 + nn;
  int* perm = reinterpret_cast<int*>(col + n);
  double* rv = reinterpret_cast<double*>(perm + n + (n & 1));
  int* ri = reinterpret_cast<int*>(rv + GT);
  __shared__ int s_done;

  const cd* H0 = J.mats;
  const cd* H1 = H0 + m * m;
  const cd* T1 = H1 + m * m;
  const cd* T2 = T1 + m * m;
  const cd* tau = T2 + m * m;
  const cd eps = e < J.n_real ? mk(J.E[e] - J.U, J.eta) : mk(J.z[e - J.n_real].re - J.U, J.z[e - J.n_real].im);

  // h = [[H0, T1^dag], [T1, H1]], a = [[0, 0], [T2^dag, 0]], c = a^dagger = [[0, T2], [0, 0]]
  double sc = 1.0;
  for (int o = t; o < nn; o += GT) {
    const int i = o / n, j = o - i * n;
    const int bi = i / m, bj = j / m, r = i - bi * m, q = j - bj * m;
    cd hv, av, cv;
    if (bi == 0 && bj == 0) hv = H0[r * m + q];
    else if (bi == 1 && bj == 1) hv = H1[r * m + q];
    else if (bi == 1 && bj == 0) hv = T1[r * m + q];
    else hv = cconj(T1[q * m + r]);
    av = (bi == 1 && bj == 0) ? cconj(T2[q * m + r]) : mk(0.0, 0.0);
    cv = (bi == 0 && bj == 1) ? T2[r * m + q] : mk(0.0, 0.0);
    hs[o] = hv;
    h[o] = hv;
    a[o] = av;
    c[o] = cv;
    // the convergence scale is max |entry| of the layer blocks with U on the diagonal
    const cd hu = (i == j) ? mk(hv.re + J.U, hv.im) : hv;
    sc = fmax(sc, fmax(sqrt(abs2(hu)), sqrt(abs2(av))));
  }
  for (int off = 16; off > 0; off >>= 1) sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, off));
  if ((t & 31) == 0) rv[t >> 5] = sc;
  __syncthreads();
  if (t == 0) {
    double s2 = rv[0];
    for (int w = 1; w < GT / 32; ++w) s2 = fmax(s2, rv[w]);
    rv[GT - 1] = s2;
  }
  __syncthreads();
  const double thr = J.tol * rv[GT - 1];
  __syncthreads();

  int it = 0;
  for (; it < J.max_iter; ++it) {
    for (int o = t; o < nn; o += GT) {
      const int i = o / n, j = o - i * n;
      W1[o] = mk((i == j ? eps.re : 0.0) - h[o].re, (i == j ? eps.im : 0.0) - h[o].im);
    }
    __syncthreads();
    gj_inverse(W1, n, col, perm, rv, ri);                     // g
    for (int o = t; o < nn; o += GT) {
      const int i = o / n, j = o - i * n;
      W2[o] = rowcol(a, W1, i, j, n);                          // a g
      W3[o] = rowcol(c, W1, i, j, n);                          // c g
    }
    __syncthreads();
    for (int o = t; o < nn; o += GT) {
      const int i = o / n, j = o - i * n;
      const cd agc = rowcol(W2, c, i, j, n);
      const cd cga = rowcol(W3, a, i, j, n);
      hs[o] = hs[o] + agc;
      h[o] = h[o] + agc + cga;
    }
    // a <- (a g) a, c <- (c g) c: through registers, since a and c are operands
    cd na[(4 * MAX_GEN_LEAD * MAX_GEN_LEAD + GT - 1) / GT], nc[(4 * MAX_GEN_LEAD * MAX_GEN_LEAD + GT - 1) / GT];
    double amax = 0.0;
#pragma unroll
    for (int p = 0; p < (4 * MAX_GEN_LEAD * MAX_GEN_LEAD + GT - 1) / GT; ++p) {
      const int o = t + p * GT;
      if (o < nn) {
        const int i = o / n, j = o - i * n;
        na[p] = rowcol(W2, a, i, j, n);
        nc[p] = rowcol(W3, c, i, j, n);
        amax = fmax(amax, fmax(abs2(na[p]), abs2(nc[p])));
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < (4 * MAX_GEN_LEAD * MAX_GEN_LEAD + GT - 1) / GT; ++p) {
      const int o = t + p * GT;
      if (o < nn) {
        a[o] = na[p];
        c[o] = nc[p];
      }
    }
    for (int off = 16; off > 0; off >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    if ((t & 31) == 0) rv[t >> 5] = amax;
    __syncthreads();
    if (t == 0) {
      double s2 = rv[0];
      for (int w = 1; w < GT / 32; ++w) s2 = fmax(s2, rv[w]);
      s_done = sqrt(s2) < thr;
    }
    __syncthreads();
    if (s_done) break;
  }
  if (t == 0 && it == J.max_iter) atomicAdd(status, 1);

  // g_s = (eps - h_s)^{-1}; Sigma = tau^dagger g_{s0} tau with g_{s0} the upper-left m x m block
  for (int o = t; o < nn; o += GT) {
    const int i = o / n, j = o - i * n;
    W1[o] = mk((i == j ? eps.re : 0.0) - hs[o].re, (i == j ? eps.im : 0.0) - hs[o].im);
  }
  __syncthreads();
  gj_inverse(W1, n, col, perm, rv, ri);
  for (int o = t; o < m * m; o += GT) {   // W2 = g_{s0} tau (m x m, ld m)
    const int i = o / m, j = o - i * m;
    cd v = mk(0.0, 0.0);
    for (int k = 0; k < m; ++k) v = cmac(v, W1[i * n + k], tau[k * m + j]);
    W2[o] = v;
  }
  __syncthreads();
  cd* sig = J.sig + (long long)e * m * m;
  for (int o = t; o < m * m; o += GT) {   // W3 = Sigma = tau^dagger W2
    const int i = o / m, j = o - i * m;
    cd v = mk(0.0, 0.0);
    for (int k = 0; k < m; ++k) v = cmac(v, cconj(tau[k * m + i]), W2[k * m + j]);
    W3[o] = v;
    sig[o] = v;
  }
  __syncthreads();
  // Gamma = i (Sigma - Sigma^dagger) into W2; pivoted Cholesky into W1 (one thread: m <= 20)
  for (int o = t; o < m * m; o += GT) {
    const int i = o / m, j = o - i * m;
    const cd d = W3[i * m + j] - cconj(W3[j * m + i]);
    W2[o] = mk(-d.im, d.re);
  }
  __syncthreads();
  if (t == 0) {
    double* dg = rv;          // remaining diagonal
    int* piv = perm;          // column k of L belongs to pivot row piv[k]
    for (int i = 0; i < m; ++i) {
      dg[i] = W2[i * m + i].re;
      for (int j = 0; j < m; ++j) W1[i * m + j] = mk(0.0, 0.0);
    }
    bool used[2 * MAX_GEN_LEAD];
    for (int i = 0; i < m; ++i) used[i] = false;
    for (int k = 0; k < m; ++k) {
      int p = -1;
      double best = 0.0;
      for (int i = 0; i < m; ++i)
        if (!used[i] && dg[i] > best) {
          best = dg[i];
          p = i;
        }
      if (p < 0) break;   // the rest of Gamma is zero to rounding
      used[p] = true;
      piv[k] = p;
      const double lkk = sqrt(best);
      W1[p * m + k] = mk(lkk, 0.0);
      for (int i = 0; i < m; ++i) {
        if (used[i]) continue;
        cd v = W2[i * m + p];
        for (int j = 0; j < k; ++j) v = v - W1[i * m + j] * cconj(W1[p * m + j]);
        v = scale(v, 1.0 / lkk);
        W1[i * m + k] = v;
        dg[i] -= abs2(v);
      }
    }
  }
  __syncthreads();
  cd* fac = J.fac + (long long)e * m * m;
  for (int o = t; o < m * m; o += GT) fac[o] = W1[o];
}

}  // namespace

size_t lead_general_smem(int m_max) {
  const int n = 2 * m_max;
  return (size_t)7 * n * n * sizeof(cd) + (size_t)n * sizeof(cd) + (size_t)(n + 2) * sizeof(int) +
         (size_t)GT * sizeof(double) + 16;
}

int launch_lead_general(const GenLeadJob* jobs, int n_jobs, int max_energies, int m_max, int* status, cudaStream_t s) {
  if (n_jobs <= 0 || max_energies <= 0) return 0;
  if (m_max > MAX_GEN_LEAD) return -1;
  const size_t smem = lead_general_smem(m_max);
  if (cudaFuncSetAttribute(lead_general_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  const dim3 grid((unsigned)max_energies, (unsigned)n_jobs);
  lead_general_kernel<<<grid, GT, smem, s>>>(jobs, status);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace negf
