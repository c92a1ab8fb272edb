// Device-resident self-consistency step (Sec. 2.3, Alg. 3) and the 1D Poisson stand-in.
//
// Broyden's modified second method on the electron counts n (reading: the loop runs while
// eps_max > tol and m < M; the mixing fraction of the W update is zeta; f_old is kept;
// a zero ||Delta f||^2 gives a zero V column):
//   f = n_in - n_out, eps_max = max |f| / (n_in + n_out), Delta f = f - f_old,
//   d = ||Delta f||^2; if m > 0: s = sum_{j<m} W_j (V_j . Delta f), V_m = Delta f / d,
//   W_m = -zeta Delta f + (n_in - n_in_old) - s, s = sum_{j<=m} W_j (V_j . f);
//   n_in_old = n_in; n_in = n_in_old - zeta f - s; f_old = f; m = m + 1.
// One CTA per device; every reduction (max, dot products, the M-vector k) is a
// fixed-shape shared-memory tree, so a device gives the same bits alone or in a batch.
// The step stops (state 1) when eps_max < tol before updating, or marks state 2 when the
// history is full.
//
// Poisson: U_i - U_G - r (U_{i+1} - 2 U_i + U_{i-1}) = kappa (n_i - n0_i), r = (lam/dx)^2,
// Dirichlet U_{-1} = U_S, U_N = U_D, solved by the Thomas algorithm (one thread per
// device: a sequential O(N) recurrence, negligible next to the sweep).
#include "common.cuh"

namespace negf {

namespace {
constexpr int TB = 512;

__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = TB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}
__device__ double block_max(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = TB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}
}  // namespace

__global__ void __launch_bounds__(TB) broyden_kernel(const ScDev* devs) {
  const ScDev& S = devs[blockIdx.x];
  __shared__ double sh[TB];
  __shared__ double kv[256];
  if (*S.state != 0) return;
  const int N = S.N, M = S.M;
  const int m = *S.m;
  // f, eps_max, d
  double emax = 0.0, dsum = 0.0;
  for (int i = threadIdx.x; i < N; i += TB) {
    const double f = S.n_in[i] - S.n_out[i];
    emax = fmax(emax, fabs(f) / (S.n_in[i] + S.n_out[i]));
    const double df = f - S.f_old[i];
    dsum += df * df;
  }
  emax = block_max(emax, sh);
  const double d = block_sum(dsum, sh);
  if (threadIdx.x == 0) S.hist[m < M ? m : M - 1] = emax;
  if (emax < S.tol) {
    if (threadIdx.x == 0) *S.state = 1;
    return;
  }
  if (m >= M) {
    if (threadIdx.x == 0) *S.state = 2;
    return;
  }
  if (m > 0) {
    // k_j = V_j . Delta f, j < m-1 (columns 0..m-2 hold the paper's 1..m-1)
    for (int j = 0; j < m - 1; ++j) {
      double p = 0.0;
      for (int i = threadIdx.x; i < N; i += TB) p += S.V[(long long)j * N + i] * ((S.n_in[i] - S.n_out[i]) - S.f_old[i]);
      const double kj = block_sum(p, sh);
      if (threadIdx.x == 0) kv[j] = kj;
    }
    __syncthreads();
    const double inv_d = d > 0.0 ? 1.0 / d : 0.0;
    for (int i = threadIdx.x; i < N; i += TB) {
      double s = 0.0;
      for (int j = 0; j < m - 1; ++j) s += S.W[(long long)j * N + i] * kv[j];
      const double f = S.n_in[i] - S.n_out[i];
      const double df = f - S.f_old[i];
      S.V[(long long)(m - 1) * N + i] = df * inv_d;
      S.W[(long long)(m - 1) * N + i] = -S.zeta * df + (S.n_in[i] - S.n_in_old[i]) - s;
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      double p = 0.0;
      for (int i = threadIdx.x; i < N; i += TB) p += S.V[(long long)j * N + i] * (S.n_in[i] - S.n_out[i]);
      const double kj = block_sum(p, sh);
      if (threadIdx.x == 0) kv[j] = kj;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += TB) {
    double s = 0.0;
    if (m > 0)
      for (int j = 0; j < m; ++j) s += S.W[(long long)j * N + i] * kv[j];
    const double f = S.n_in[i] - S.n_out[i];
    const double nin = S.n_in[i];
    S.n_in_old[i] = nin;
    S.n_in[i] = nin - S.zeta * f - s;
    S.f_old[i] = f;
  }
  __syncthreads();
  if (threadIdx.x == 0) *S.m = m + 1;
}

__global__ void poisson_kernel(const ScDev* devs) {
  const ScDev& S = devs[blockIdx.x];
  if (threadIdx.x != 0) return;
  if (*S.state != 0) return;
  const int N = S.N;
  const double r = S.r, dg = 1.0 + 2.0 * r;
  // forward elimination with sub = sup = -r: cp_i = -r / den_i, dp_i stored in U
  double cprev = 0.0, dprev = 0.0;
  for (int i = 0; i < N; ++i) {
    double rhs = S.U_G + S.kappa * (S.n_in[i] - S.n0[i]);
    if (i == 0) rhs += r * S.U_S;
    if (i == N - 1) rhs += r * S.U_D;
    const double den = dg + r * cprev;    // diag - sub * cp_{i-1} with sub = -r
    const double cpi = (i < N - 1) ? -r / den : 0.0;
    const double dpi = (rhs + r * dprev) / den;
    S.cp[i] = cpi;
    S.U[i] = dpi;
    cprev = cpi;
    dprev = dpi;
  }
  for (int i = N - 2; i >= 0; --i) S.U[i] = S.U[i] - S.cp[i] * S.U[i + 1];
}

int launch_broyden(const ScDev* devs, int n, cudaStream_t s) {
  broyden_kernel<<<n, TB, 0, s>>>(devs);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
int launch_poisson(const ScDev* devs, int n, cudaStream_t s) {
  poisson_kernel<<<n, 32, 0, s>>>(devs);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// state flag of every solve in one array (one host read per serving step)
__global__ void gather_states_kernel(const ScDev* devs, int n, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = *devs[i].state;
}
int launch_gather_states(const ScDev* devs, int n, int* out, cudaStream_t s) {
  if (n <= 0) return 0;
  gather_states_kernel<<<(n + 255) / 256, 256, 0, s>>>(devs, n, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace negf
