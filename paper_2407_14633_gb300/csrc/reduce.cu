// Second stage of the energy quadrature (Eq. Rho, Eq. deviceCharacteristics): per device,
// sum the per-item partial ring sums in item order (deterministic, independent of the
// schedule and of the rest of the batch), sum T(E) over chains with their band
// degeneracy, and reduce the Landauer current I = g_s (e^2/h) sum_k w_k T_k (fS_k - fD_k)
// with a fixed-shape tree in shared memory; the zero-bias conductance (Eq. zeroBiasG) the
// same way.  Also the per-launch layer diagonals of the 1 x 1
// chains (prep_kernel), which the sweep would otherwise form in every lane.
#include <algorithm>

#include "common.cuh"

namespace negf {

// e^2/h in A/V from the exact SI 2019 elementary charge and Planck constant
__constant__ double kE2H = 1.602176634e-19 * 1.602176634e-19 / 6.62607015e-34;

// Grid: one column of CTAs per device (blockIdx.x), its rings spread over blockIdx.y.  Each
// ring's sum runs over the device's items in order in one thread, whichever thread that is;
// the first CTA of a column also reduces T(E) and the current.
__global__ void __launch_bounds__(256) reduce_kernel(const ReduceDev* devs) {
  const ReduceDev& R = devs[blockIdx.x];
  __shared__ double sh[256];
  // ring sums: real-axis items and contour items separately
  for (int r = blockIdx.y * blockDim.x + threadIdx.x; r < R.n_rings; r += gridDim.y * blockDim.x) {
    double sr = 0.0, sc = 0.0;
    for (int it = R.it0; it < R.it1; ++it) {
      const WorkItem& W = R.items[it];
      const double v = R.partial[W.part + r];
      if (W.kind == 0)
        sr += v;
      else
        sc += v;
    }
    R.n[r] = sr + sc;
    if (R.n_real_part) R.n_real_part[r] = sr;
    if (R.n_cont) R.n_cont[r] = sc;
  }
  if (blockIdx.y != 0) return;
  // T(E) and the current
  double acc = 0.0;
  for (int k = threadIdx.x; k < R.n_real; k += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < R.n_chains; ++c) t += R.g_b[c] * R.Tpart[(long long)c * R.n_real + k];
    if (R.T) R.T[k] = t;
    acc += R.w[k] * t * (R.fS[k] - R.fD[k]);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && R.I) *R.I = 2.0 * kE2H * sh[0];
}

// 128 CTAs per device along its rings (a CTA past a short device's rings exits at once)
int launch_reduce(const ReduceDev* devs, int n_devs, cudaStream_t s) {
  reduce_kernel<<<dim3(n_devs, 128), 256, 0, s>>>(devs);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Zero-bias conductance (Eq. zeroBiasG) from the transmission of the real-axis lanes:
// G = g_s (e^2/h) sum_k w_k T_k (-df/dE)(E_k - mu), with -df/dE = e / (kT (1 + e)^2),
// e = exp(-|E - mu| / kT) (no overflow in the tails).  One CTA per device, strided partial
// sums then a fixed-shape shared-memory tree: the same bits alone or in a batch.
__global__ void __launch_bounds__(256) conductance_kernel(const CondDev* devs) {
  const CondDev& D = devs[blockIdx.x];
  __shared__ double sh[256];
  double acc = 0.0;
  for (int k = threadIdx.x; k < D.n_real; k += blockDim.x) {
    const double e = exp(-fabs(D.E[k] - D.mu) / D.kT);
    const double mdf = e / (D.kT * (1.0 + e) * (1.0 + e));
    acc += D.w[k] * D.T[k] * mdf;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *D.G = 2.0 * kE2H * sh[0];
}

int launch_conductance(const CondDev* devs, int n_devs, cudaStream_t s) {
  if (n_devs <= 0) return 0;
  conductance_kernel<<<n_devs, 256, 0, s>>>(devs);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void prep_kernel(const PrepDesc* descs, int n) {
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const PrepDesc q = descs[i];
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < q.L; l += gridDim.x * blockDim.x) {
      const double v = q.Hdiag[l].re + q.U[l];
      q.hu[l] = v;
      q.hu_f[l] = (float)v;
    }
  }
}

int launch_prep(const PrepDesc* descs, int n, int max_L, cudaStream_t s) {
  if (n <= 0) return 0;
  const dim3 grid((unsigned)std::min((max_L + 255) / 256, 64), (unsigned)std::min(n, 65535));
  prep_kernel<<<grid, 256, 0, s>>>(descs, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace negf
