// Persistent kernel and host launchers of the block sweep for wide ring blocks (real space).
// The method and the per-lane device code are in sweep_block_item.cuh.
#include "sweep_block_item.cuh"

namespace negf {

__host__ __device__ bool sweep_blk_compact(int b, int m, int esize, int warps) {
  const int cap = 2 * MAXP * 32 * warps;
  return esize == 16 && b * b <= cap && b * m <= cap;
}
__host__ __device__ size_t sweep_blk_smem_bytes_t(int b, int m, int esize, int warps) {
  const bool cmp = sweep_blk_compact(b, m, esize, warps);
  const int nm = esize == 8 ? 6 : (cmp ? 3 : 4), nv = cmp ? 1 : 3;
  size_t per = (size_t)(nm * b * b + nv * b * m + b) * esize;
  per = (per + 15) & ~(size_t)15;
  per += (size_t)2 * m * 16 + (size_t)2 * m * 8 + (size_t)(b + 1) * 4 + 8 * 8 + 8 * 4 + 8 * 4;
  return (per + 15) & ~(size_t)15;
}

template <typename T, int NW, bool TWO, bool CMP>
__global__ void __launch_bounds__(32 * NW, NW == 1 ? 9 : (NW == 2 ? 6 : 3)) sweep_blk_kernel(SweepArgs a, int bmax, int mmax) {
  extern __shared__ __align__(16) unsigned char sm_blk[];
  const int tid = threadIdx.x;
  __shared__ int s_item;
  unsigned char* stage = a.stage + (long long)blockIdx.x * a.stage_stride;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= a.n_items) break;
    const WorkItem W = a.items[a.order[it]];
    blk_item<T, NW, TWO, CMP>(a, W, sm_blk, stage, bmax, mmax);
  }
}

template <typename T, int NW, bool CMP>
static int blk_occupancy(size_t smem) {
  constexpr bool TWO = sizeof(T) == 4;
  cudaFuncSetAttribute(sweep_blk_kernel<T, NW, TWO, CMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep_blk_kernel<T, NW, TWO, CMP>, 32 * NW, smem) !=
          cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    per = 1;
  }
  return per;
}

int sweep_blk_occupancy_t(bool fp32, int warps, int b, int m) {
  const size_t smem = sweep_blk_smem_bytes_t(b, m, fp32 ? 8 : 16, warps);
  if (fp32) {
    if (warps == 1) return blk_occupancy<float, 1, false>(smem);
    if (warps == 2) return blk_occupancy<float, 2, false>(smem);
    return blk_occupancy<float, 4, false>(smem);
  }
  const bool cmp = sweep_blk_compact(b, m, 16, warps);
  if (warps == 1) return cmp ? blk_occupancy<double, 1, true>(smem) : blk_occupancy<double, 1, false>(smem);
  if (warps == 2) return cmp ? blk_occupancy<double, 2, true>(smem) : blk_occupancy<double, 2, false>(smem);
  return cmp ? blk_occupancy<double, 4, true>(smem) : blk_occupancy<double, 4, false>(smem);
}

int launch_sweep_blk_t(bool fp32, const SweepArgs& a, int b_max, int m_max, int grid, int warps, cudaStream_t s) {
  // the dynamic shared memory limit was raised by the occupancy query when planning
  const size_t smem = sweep_blk_smem_bytes_t(b_max, m_max, fp32 ? 8 : 16, warps);
  if (fp32) {
    if (warps == 1)
      sweep_blk_kernel<float, 1, true, false><<<grid, 32, smem, s>>>(a, b_max, m_max);
    else if (warps == 2)
      sweep_blk_kernel<float, 2, true, false><<<grid, 64, smem, s>>>(a, b_max, m_max);
    else
      sweep_blk_kernel<float, 4, true, false><<<grid, 128, smem, s>>>(a, b_max, m_max);
  } else if (sweep_blk_compact(b_max, m_max, 16, warps)) {
    if (warps == 1)
      sweep_blk_kernel<double, 1, false, true><<<grid, 32, smem, s>>>(a, b_max, m_max);
    else if (warps == 2)
      sweep_blk_kernel<double, 2, false, true><<<grid, 64, smem, s>>>(a, b_max, m_max);
    else
      sweep_blk_kernel<double, 4, false, true><<<grid, 128, smem, s>>>(a, b_max, m_max);
  } else {
    if (warps == 1)
      sweep_blk_kernel<double, 1, false, false><<<grid, 32, smem, s>>>(a, b_max, m_max);
    else if (warps == 2)
      sweep_blk_kernel<double, 2, false, false><<<grid, 64, smem, s>>>(a, b_max, m_max);
    else
      sweep_blk_kernel<double, 4, false, false><<<grid, 128, smem, s>>>(a, b_max, m_max);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sweep_blk_f64(const SweepArgs& a, int b_max, int m_max, int grid, int warps, cudaStream_t s) {
  return launch_sweep_blk_t(false, a, b_max, m_max, grid, warps, s);
}

}  // namespace negf
