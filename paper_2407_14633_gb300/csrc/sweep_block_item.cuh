// Device code of the block sweep for wide ring blocks: the helpers and the per-lane body
// blk_item, shared by the persistent kernel of sweep_block.cu and by the complex64 kernel of
// sweep_block32.cu (which re-sweeps a lane that the mixed-precision path flags in FP64 without
// leaving its CTA).
//
// Recursive Green's function sweep for wide ring blocks (real space): one CTA of NW warps
// owns one (device, chain, energy) lane and keeps its b x b complex blocks in shared
// memory; every product spreads its outputs over the CTA's threads.
//
// The algorithm is the left-connected recursion (Alg. 2 reading) with the lead columns
// propagated as factors of the broadening matrices, Gamma_l = L_l L_l^dagger with
// L_l = F diag(sqrt(gamma_j)) from a circulant lead (F the ring Fourier basis), or the
// pivoted Cholesky factor that the launch plan computes per energy for a general lead:
//   forward   X = H_{l,l-1} gL_{l-1},  gL_l = (alpha_l - X H_{l-1,l})^{-1},
//             R_l = X R_{l-1} (R_0 = L_S)                 [R_l = G_{l,l}^{-1} G_{l,0} L_S]
//   backward  Z = gL_l H_{l,l+1},  G_ll = gL_l + Z G_{l+1,l+1} (H_{l+1,l} gL_l),
//             K_l = Z K_{l+1} (K_{L-1} = G_{L-1,L-1} L_D)  [K_l = G_{l,L-1} L_D]
//   A_S,ll = (G_ll R_l)(G_ll R_l)^dagger,  A_D,ll = K_l K_l^dagger,
//   T = || L_S^dagger K_0 ||_F^2 = Tr[Gamma_S G_{0,L-1} Gamma_D G_{0,L-1}^dagger].
// Products with the coupling blocks use their column-sparse form (kmax entries per
// column; kmax = b for dense couplings).  gL_l and R_l are staged per resident CTA in
// global memory.
//
// Element type T: double (the FP64 path; on GB300 the FP64 pipe is the bound) or float
// (the complex64 sweep of the mixed-precision path; lead self-energies are still formed
// in FP64 and the quadrature weights applied in FP64).  For real-axis lanes the kernel
// can also record the lane's residual of the sum rule
//   -2 Im G_aa = A_S,aa + A_D,aa + 2 eta (G G^dagger)_aa,
// max(0, max_a (A_S,aa + A_D,aa + 2 Im G_aa)) / max_a |2 Im G_aa|.  The eta term is not
// available to the sweep and is never negative, so only the excess of A_S + A_D over
// -2 Im G is a rounding error; the mixed path recomputes energies whose excess, relative
// to the largest spectral weight of the lane, passes a threshold.
#pragma once
#include "common.cuh"
#include "lead.cuh"

namespace negf {

namespace {

template <int NW>
__device__ __forceinline__ void csync() {
  if (NW == 1)
    __syncwarp();
  else
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ cx<T> cz() {
  return mk(T(0), T(0));
}
template <typename T>
__device__ __forceinline__ cx<T> tc(cd v) {
  return mk((T)v.re, (T)v.im);
}

// Outputs o0 and o1 = o0 + NT of C = [Add +] A (R x K, lda) * B (K x N, ldb), one
// accumulator each in k order (on GB300 a dependent FP64 multiply-add issues as soon as the
// narrow FP64 pipe is free again, so two chains per thread are enough).  Every output is
// evaluated in the same order whichever thread computes it.
template <typename T, int NT>
__device__ __forceinline__ void dot2(cx<T>& v0, cx<T>& v1, int o0, int tot, const cx<T>* A, int lda,
                                     const cx<T>* B, int ldb, int K, int N, const cx<T>* Add, int ldadd) {
  const int o1 = o0 + NT;
  const bool two = o1 < tot;
  const int r0 = o0 / N, c0 = o0 - r0 * N;
  const int r1 = two ? o1 / N : r0, c1 = two ? o1 - r1 * N : c0;
  const cx<T>* a0 = A + r0 * lda;
  const cx<T>* a1 = A + r1 * lda;
  const cx<T>* b0 = B + c0;
  const cx<T>* b1 = B + c1;
  cx<T> s0 = cz<T>(), s1 = cz<T>();
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    s0 = cmac(s0, a0[k], b0[k * ldb]);
    s1 = cmac(s1, a1[k], b1[k * ldb]);
  }
  v0 = s0;
  v1 = s1;
  if (Add) {
    v0 = v0 + Add[r0 * ldadd + c0];
    v1 = v1 + Add[r1 * ldadd + c1];
  }
}

// One output o of the same product, same order.
template <typename T>
__device__ __forceinline__ cx<T> dot1(int o, const cx<T>* A, int lda, const cx<T>* B, int ldb, int K, int N,
                                      const cx<T>* Add, int ldadd) {
  const int r = o / N, c = o - r * N;
  const cx<T>* a = A + r * lda;
  const cx<T>* bc = B + c;
  cx<T> v = cz<T>();
#pragma unroll 4
  for (int k = 0; k < K; ++k) v = cmac(v, a[k], bc[k * ldb]);
  if (Add) v = v + Add[r * ldadd + c];
  return v;
}

// One output o computed by a whole warp: lane j takes the terms k = j and j + 32 (K <= 64),
// then a fixed butterfly sums the lanes; every lane returns the result.
template <typename T>
__device__ __forceinline__ cx<T> dot_split(int o, const cx<T>* A, int lda, const cx<T>* B, int ldb, int K, int N,
                                           const cx<T>* Add, int ldadd, int lane) {
  const int r = o / N, c = o - r * N;
  cx<T> p = cz<T>();
  if (lane < K) p = cmac(p, A[r * lda + lane], B[lane * ldb + c]);
  if (lane + 32 < K) p = cmac(p, A[r * lda + lane + 32], B[(lane + 32) * ldb + c]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    p.re += __shfl_xor_sync(0xffffffffu, p.re, off);
    p.im += __shfl_xor_sync(0xffffffffu, p.im, off);
  }
  if (Add) p = p + Add[r * ldadd + c];
  return p;
}

// Output split of a product with tot = R N outputs.  When tot mod 32 <= SPLIT_LEFT, the first
// tot - tot mod 32 outputs go one per thread (pairs o, o + NT share a pass, a last unpaired
// pass takes one output) and the few left over are summed across warp 0 (dot_split), so no
// pass is half empty: 17 x 17 = 289 = 9 x 32 + 1 costs 9 thread-outputs and one split
// output instead of 10 thread-outputs.  Otherwise every output goes one per thread in pairs.
// Which rule an output follows depends on tot only, never on the CTA width.
constexpr int SPLIT_LEFT = 4;
__device__ __forceinline__ bool split_mode(int tot) { return (tot & 31) <= SPLIT_LEFT; }

// C (R x N, ldc) = [Add +] A (R x K, lda) * B (K x N, ldb)
template <typename T, int NT>
__device__ __forceinline__ void bgemm(cx<T>* C, int ldc, const cx<T>* A, int lda, const cx<T>* B, int ldb,
                                      int R, int K, int N, const cx<T>* Add, int ldadd, int tid) {
  const int tot = R * N;
  if (split_mode(tot)) {
    const int main = tot & ~31;   // warp-uniform branches below
    for (int o0 = tid; o0 < main; o0 += 2 * NT) {
      const int o1 = o0 + NT;
      if (o1 < main) {
        cx<T> v0, v1;
        dot2<T, NT>(v0, v1, o0, tot, A, lda, B, ldb, K, N, Add, ldadd);
        C[(o0 / N) * ldc + o0 % N] = v0;
        C[(o1 / N) * ldc + o1 % N] = v1;
      } else {
        C[(o0 / N) * ldc + o0 % N] = dot1(o0, A, lda, B, ldb, K, N, Add, ldadd);
      }
    }
    if (tid < 32)
      for (int o = main; o < tot; ++o) {
        const cx<T> v = dot_split(o, A, lda, B, ldb, K, N, Add, ldadd, tid);
        if (tid == 0) C[(o / N) * ldc + o % N] = v;
      }
    return;
  }
  for (int o0 = tid; o0 < tot; o0 += 2 * NT) {
    cx<T> v0, v1;
    dot2<T, NT>(v0, v1, o0, tot, A, lda, B, ldb, K, N, Add, ldadd);
    C[(o0 / N) * ldc + o0 % N] = v0;
    const int o1 = o0 + NT;
    if (o1 < tot) C[(o1 / N) * ldc + o1 % N] = v1;
  }
}

// The same product held in registers (at most 2 * MAXP outputs per thread, plus one split
// output on lanes 0 .. SPLIT_LEFT - 1 of warp 0), so that it can overwrite one of its
// operands: bgemm_r, a CTA barrier, then store_r.
constexpr int MAXP = 5;
template <typename T>
struct RegTile {
  cx<T> v[2 * MAXP];
  cx<T> lv;
};
template <typename T, int NT>
__device__ __forceinline__ void bgemm_r(RegTile<T>& t, const cx<T>* A, int lda, const cx<T>* B, int ldb, int R, int K,
                                        int N, const cx<T>* Add, int ldadd, int tid) {
  const int tot = R * N;
  if (split_mode(tot)) {
    const int main = tot & ~31;
#pragma unroll
    for (int p = 0; p < MAXP; ++p) {
      const int o0 = tid + p * 2 * NT;
      if (o0 < main) {
        if (o0 + NT < main)
          dot2<T, NT>(t.v[2 * p], t.v[2 * p + 1], o0, tot, A, lda, B, ldb, K, N, Add, ldadd);
        else
          t.v[2 * p] = dot1(o0, A, lda, B, ldb, K, N, Add, ldadd);
      }
    }
    if (tid < 32)
      for (int q = 0; q < tot - main; ++q) {
        const cx<T> v = dot_split(main + q, A, lda, B, ldb, K, N, Add, ldadd, tid);
        if (tid == q) t.lv = v;
      }
    return;
  }
#pragma unroll
  for (int p = 0; p < MAXP; ++p) {
    const int o0 = tid + p * 2 * NT;
    if (o0 < tot) dot2<T, NT>(t.v[2 * p], t.v[2 * p + 1], o0, tot, A, lda, B, ldb, K, N, Add, ldadd);
  }
}
template <typename T, int NT>
__device__ __forceinline__ void store_r(cx<T>* C, int ldc, const RegTile<T>& t, int R, int N, int tid) {
  const int tot = R * N;
  const bool split = split_mode(tot);
  const int main = split ? (tot & ~31) : tot;
#pragma unroll
  for (int p = 0; p < MAXP; ++p) {
    const int o0 = tid + p * 2 * NT, o1 = o0 + NT;
    if (o0 < main) C[(o0 / N) * ldc + o0 % N] = t.v[2 * p];
    if (o1 < main) C[(o1 / N) * ldc + o1 % N] = t.v[2 * p + 1];
  }
  if (split && tid < tot - main) C[((main + tid) / N) * ldc + (main + tid) % N] = t.lv;
}

// Upper triangle of a symmetric b x b result, row by row: index t -> (r, c), r <= c.  Row r
// starts at r b - r (r - 1) / 2; counting from the end, u = T - 1 - t falls in the block of
// k = b - 1 - r rows, found from the triangular root of u (exact in FP32 for b <= 64).
__device__ __forceinline__ void tri_rc(int t, int b, int& r, int& c) {
  const int u = b * (b + 1) / 2 - 1 - t;
  int k = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  if ((k + 1) * (k + 2) / 2 <= u) ++k;
  if (k * (k + 1) / 2 > u) --k;
  r = b - 1 - k;
  c = b - 1 - (u - k * (k + 1) / 2);
}

// Upper triangle of Add + W Z^T (all b x b; W Z^T is symmetric when it equals Z G Z^T with G
// symmetric), one output per thread and pass, into registers.
template <typename T, int NT>
__device__ __forceinline__ void bgemm_symt_r(RegTile<T>& t, const cx<T>* W, const cx<T>* Z, const cx<T>* Add, int b,
                                             int tid) {
  const int tot = b * (b + 1) / 2;
#pragma unroll
  for (int p = 0; p < MAXP + 1; ++p) {   // b (b + 1) / 2 <= (MAXP + 1) NT when b^2 <= 2 MAXP NT
    const int o = tid + p * NT;
    if (o < tot) {
      int r, c;
      tri_rc(o, b, r, c);
      const cx<T>* w = W + r * b;
      const cx<T>* z = Z + c * b;
      cx<T> v = cz<T>();
#pragma unroll 4
      for (int k = 0; k < b; ++k) v = cmac(v, w[k], z[k]);
      t.v[p] = v + Add[r * b + c];
    }
  }
}
// Gate of the symmetric G_ll update: largest |gL_l diagonal entry| (1/eV) of a lane.  Away from
// bound states of the half chain it stays near 1 / |t|, a few 1/eV at band edges; near one it
// grows like 1 / distance, and the update's rounding error grows like u |gL|^2 / |G|, so at
// 100 it stays near 1e-12 relative.  (The zigzag end of every half chain of a nanotube carries
// edge states at the local potential, so lanes crossing one somewhere are common.)
constexpr double SYM_GL_MAX = 100.0;

// A := (A + A^T) / 2 in place, one (r, c) pair per thread.  For a chain with complex
// symmetric Green's functions the computed inverse gL_l is symmetric only up to rounding
// times its condition number; averaging keeps it the inverse of a nearby symmetric matrix,
// which the symmetric G_ll update needs.
template <typename T, int NT>
__device__ __forceinline__ void symmetrize(cx<T>* A, int b, int tid) {
  const int tot = b * (b + 1) / 2;
  for (int o = tid; o < tot; o += NT) {
    int r, c;
    tri_rc(o, b, r, c);
    if (r == c) continue;
    const cx<T> v = scale(A[r * b + c] + A[c * b + r], T(0.5));
    A[r * b + c] = v;
    A[c * b + r] = v;
  }
}

// The same, written straight to C (C must not alias W, Z or Add).
template <typename T, int NT>
__device__ __forceinline__ void bgemm_symt(cx<T>* C, const cx<T>* W, const cx<T>* Z, const cx<T>* Add, int b,
                                           int tid) {
  const int tot = b * (b + 1) / 2;
  for (int o = tid; o < tot; o += NT) {
    int r, c;
    tri_rc(o, b, r, c);
    const cx<T>* w = W + r * b;
    const cx<T>* z = Z + c * b;
    cx<T> v = cz<T>();
#pragma unroll 4
    for (int k = 0; k < b; ++k) v = cmac(v, w[k], z[k]);
    v = v + Add[r * b + c];
    C[r * b + c] = v;
    C[c * b + r] = v;
  }
}
template <typename T, int NT>
__device__ __forceinline__ void store_sym(cx<T>* C, const RegTile<T>& t, int b, int tid) {
  const int tot = b * (b + 1) / 2;
#pragma unroll
  for (int p = 0; p < MAXP + 1; ++p) {   // b (b + 1) / 2 <= (MAXP + 1) NT when b^2 <= 2 MAXP NT
    const int o = tid + p * NT;
    if (o < tot) {
      int r, c;
      tri_rc(o, b, r, c);
      C[r * b + c] = t.v[p];
      C[c * b + r] = t.v[p];
    }
  }
}

// Hamiltonian data in the sweep's element type (complex64 copies for the complex64 sweep, so
// that no conversion from FP64 sits in its inner loops)
template <typename T>
__device__ __forceinline__ const cx<T>* hdiag_t(const ChainView& C);
template <>
__device__ __forceinline__ const cd* hdiag_t<double>(const ChainView& C) { return C.Hdiag; }
template <>
__device__ __forceinline__ const cf* hdiag_t<float>(const ChainView& C) { return C.Hdiag_f; }
template <typename T>
__device__ __forceinline__ const cx<T>* csval_t(const ChainView& C);
template <>
__device__ __forceinline__ const cd* csval_t<double>(const ChainView& C) { return C.cs_val; }
template <>
__device__ __forceinline__ const cf* csval_t<float>(const ChainView& C) { return C.cs_val_f; }
template <typename T>
__device__ __forceinline__ const cx<T>* rsval_t(const ChainView& C);
template <>
__device__ __forceinline__ const cd* rsval_t<double>(const ChainView& C) { return C.rs_val; }
template <>
__device__ __forceinline__ const cf* rsval_t<float>(const ChainView& C) { return C.rs_val_f; }

// C (b x N) = H_{l+1,l} M where H_{l+1,l} = Hup_l^dagger: row r uses column r of Hup_l
template <typename T, int NT>
__device__ __forceinline__ void hdn_times(cx<T>* C, const cx<T>* M, int ldm, int N, int b, const int* cnt,
                                          const int* idx, const cx<T>* val, int kmax, int tid) {
  const int tot = b * N;
  for (int o = tid; o < tot; o += NT) {
    const int r = o / N, c = o - r * N;
    cx<T> acc = cz<T>();
    const int n = cnt[r];
    for (int e = 0; e < n; ++e) acc = cmac_cj(acc, val[r * kmax + e], M[idx[r * kmax + e] * ldm + c]);
    C[r * N + c] = acc;
  }
}

// C (R x b) = M (R x b) Hup_l: column c uses column c of Hup_l
template <typename T, int NT>
__device__ __forceinline__ void times_hup(cx<T>* C, const cx<T>* M, int R, int b, const int* cnt, const int* idx,
                                          const cx<T>* val, int kmax, int tid) {
  const int tot = R * b;
  for (int o = tid; o < tot; o += NT) {
    const int r = o / b, c = o - r * b;
    cx<T> acc = cz<T>();
    const int n = cnt[c];
    for (int e = 0; e < n; ++e) acc = cmac(acc, M[r * b + idx[c * kmax + e]], val[c * kmax + e]);
    C[r * b + c] = acc;
  }
}

// In-place Gauss-Jordan inverse of the b x b block A with partial pivoting (row swaps
// recorded in perm, undone on the columns at the end).  Pivot step k: save column k
// (f_i = A[i][k]); scale row k by 1/A[k][k] with A[k][k] := 1/A[k][k]; zero column k
// elsewhere; then one uniform update A[i][j] -= f_i A[k][j] for every i != k and every j
// (for j = k it yields -f_i / A[k][k]): four fused multiply-adds per element.
template <typename T, int NW>
__device__ void binv(cx<T>* A, int b, cx<T>* col, int* perm, float* rbest, int* ridx, int tid) {
  constexpr int NT = 32 * NW;
  const int lane = tid & 31, wid = tid >> 5;
  for (int k = 0; k < b; ++k) {
    float best = -1.0f;
    int bi = k;
    for (int i = k + tid; i < b; i += NT) {
      const cx<T> v = A[i * b + k];
      const float m = fmaf((float)v.re, (float)v.re, (float)v.im * (float)v.im);
      if (m > best) {
        best = m;
        bi = i;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (NW > 1) {
      if (lane == 0) {
        rbest[wid] = best;
        ridx[wid] = bi;
      }
      __syncthreads();
      best = rbest[0];
      bi = ridx[0];
      for (int w = 1; w < NW; ++w)
        if (rbest[w] > best || (rbest[w] == best && ridx[w] < bi)) {
          best = rbest[w];
          bi = ridx[w];
        }
    }
    if (tid == 0) perm[k] = bi;
    if (bi != k) {
      csync<NW>();
      for (int j = tid; j < b; j += NT) {
        const cx<T> t = A[k * b + j];
        A[k * b + j] = A[bi * b + j];
        A[bi * b + j] = t;
      }
    }
    csync<NW>();
    const cx<T> ip = crecip(A[k * b + k]);
    for (int i = tid; i < b; i += NT) col[i] = A[i * b + k];
    csync<NW>();
    for (int j = tid; j < b; j += NT) A[k * b + j] = (j == k) ? ip : A[k * b + j] * ip;
    for (int i = tid; i < b; i += NT)
      if (i != k) A[i * b + k] = cz<T>();
    csync<NW>();
    // three independent elements per thread and pass: loads, then updates, then stores
    const int tot = (b - 1) * b;
    for (int o0 = tid; o0 < tot; o0 += 3 * NT) {
      int q[3];
      cx<T> x[3], f[3], r[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int o = o0 + u * NT;
        const int oo = o < tot ? o : o0;
        int i = oo / b;
        const int j = oo - i * b;
        i += (i >= k);
        q[u] = o < tot ? i * b + j : -1;
        x[u] = A[i * b + j];
        f[u] = col[i];
        r[u] = A[k * b + j];
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) x[u] = cmsub(x[u], f[u], r[u]);
#pragma unroll
      for (int u = 0; u < 3; ++u)
        if (q[u] >= 0) A[q[u]] = x[u];
    }
    csync<NW>();
  }
  for (int k = b - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      for (int i = tid; i < b; i += NT) {
        const cx<T> t = A[i * b + k];
        A[i * b + k] = A[i * b + p];
        A[i * b + p] = t;
      }
    }
    csync<NW>();
  }
}

// warp butterfly sum (every lane receives the total)
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// CTA max (exact in any order)
template <int NW>
__device__ __forceinline__ double cta_max(double v, double* red, int tid) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if (NW == 1) return v;
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = red[0];
  for (int w = 1; w < NW; ++w) s = fmax(s, red[w]);
  __syncthreads();
  return s;
}

}  // namespace

// row-sparse products for the two-sided variant:
// C (b x N) = H_{l,l+1} M: row r uses row r of Hup_l
template <typename T, int NT>
__device__ __forceinline__ void hup_times(cx<T>* C, const cx<T>* M, int ldm, int N, int b, const int* cnt,
                                          const int* idx, const cx<T>* val, int kmax, int tid) {
  const int tot = b * N;
  for (int o = tid; o < tot; o += NT) {
    const int r = o / N, c = o - r * N;
    cx<T> acc = cz<T>();
    const int n = cnt[r];
    for (int e = 0; e < n; ++e) acc = cmac(acc, val[r * kmax + e], M[idx[r * kmax + e] * ldm + c]);
    C[r * N + c] = acc;
  }
}
// C (R x b) = M H_{l+1,l} = M Hup_l^dagger: column c uses row c of Hup_l, conjugated
template <typename T, int NT>
__device__ __forceinline__ void times_hdn(cx<T>* C, const cx<T>* M, int R, int b, const int* cnt, const int* idx,
                                          const cx<T>* val, int kmax, int tid) {
  const int tot = R * b;
  for (int o = tid; o < tot; o += NT) {
    const int r = o / b, c = o - r * b;
    cx<T> acc = cz<T>();
    const int n = cnt[c];
    for (int e = 0; e < n; ++e) acc = cmac_cj(acc, val[c * kmax + e], M[r * b + idx[c * kmax + e]]);
    C[r * b + c] = acc;
  }
}

// Layout of one CTA's shared memory: NM b x b and NV b x m element buffers plus b pivot
// elements, then FP64 lead rows (2 m complex + 2 m real), b pivot ints and reductions.
//   FP32, two-sided backward:              NM = 6, NV = 3
//   FP64, Dyson backward:                  NM = 4, NV = 3
//   FP64, Dyson, products in registers:    NM = 3, NV = 1 (compact; when every b x b and
//                                          b x m product fits 2 MAXP outputs per thread;
//                                          R_l of the backward sweep shares the gL_l buffer)
// alpha_l - Sub (Sub may be null): eps I - H_ll - U_ring - Sigma_S (l = 0) - Sigma_D (l = L-1),
// assembled in FP64 and rounded to T.  A circulant lead's Sigma comes from its first row
// (sigS / sigD); a general lead's from the plan's per-energy blocks (energy index eidx).
template <typename T, int NW>
__device__ __forceinline__ void alpha_minus(cx<T>* out, const cx<T>* Sub, int l, int L, int b, int rpb, int spr,
                                            cd eps, const DeviceView& D, const ChainView& C, const cd* sigS,
                                            const cd* sigD, int eidx, int tid) {
  constexpr int NT = 32 * NW;
  const cx<T>* hd = hdiag_t<T>(C) + (long long)l * C.hd_step;
  const int nn = b * b;
  for (int o = tid; o < nn; o += NT) out[o] = Sub ? mk(-hd[o].re - Sub[o].re, -hd[o].im - Sub[o].im) : mk(-hd[o].re, -hd[o].im);
  csync<NW>();
  // eps - U on the diagonal, formed in FP64 and rounded once
  for (int r = tid; r < b; r += NT)
    out[r * b + r] = out[r * b + r] + mk((T)(eps.re - D.U[l * rpb + r / spr]), (T)eps.im);
  csync<NW>();
  for (int side = 0; side < 2; ++side) {
    if ((side == 0 && l != 0) || (side == 1 && l != L - 1)) continue;
    const LeadView& Lv = C.lead[side];
    const cd* row = side ? sigD : sigS;
    const int m = Lv.m;
    const cd* gsig = Lv.gen ? Lv.gsig + (long long)eidx * m * m : nullptr;
    for (int o = tid; o < m * m; o += NT) {
      const int s = o / m, t = o - s * m;
      const int q = Lv.sites[s] * b + Lv.sites[t];
      out[q] = out[q] - tc<T>(gsig ? gsig[o] : row[((s - t) % m + m) % m]);
    }
    csync<NW>();
  }
}

// One lane (work item) of the block sweep: everything the persistent kernel does per item.
// Every thread of the CTA calls it; sm_blk is the CTA's dynamic shared memory (layout of
// sweep_blk_smem_bytes_t), stage its staging.
template <typename T, int NW, bool TWO, bool CMP>
__device__ __forceinline__ void blk_item(const SweepArgs a, const WorkItem& W, unsigned char* sm_blk,
                                         unsigned char* stage, int bmax, int mmax) {
  constexpr int NT = 32 * NW;
  constexpr int NM = TWO ? 6 : (CMP ? 3 : 4);
  constexpr int NV = CMP ? 1 : 3;
  const int tid = threadIdx.x;
  const int bb = bmax * bmax, bm = bmax * mmax;
  cx<T>* M0 = reinterpret_cast<cx<T>*>(sm_blk);
  cx<T>* M1 = M0 + bb;
  cx<T>* M2 = M1 + bb;
  cx<T>* M3 = M2 + bb;   // not in the compact layout
  cx<T>* M4 = M3 + bb;   // two-sided only
  cx<T>* M5 = M4 + bb;   // two-sided only
  cx<T>* V0 = M0 + NM * bb;
  cx<T>* V1 = V0 + bm;   // not in the compact layout
  cx<T>* V2 = V1 + bm;   // not in the compact layout
  cx<T>* col = V0 + NV * bm;
  size_t off = (size_t)(NM * bb + NV * bm + bmax) * sizeof(cx<T>);
  off = (off + 15) & ~(size_t)15;
  cd* sigS = reinterpret_cast<cd*>(sm_blk + off);
  cd* sigD = sigS + mmax;
  double* sqS = reinterpret_cast<double*>(sigD + mmax);
  double* sqD = sqS + mmax;
  double* redd = sqD + mmax;
  float* redf = reinterpret_cast<float*>(redd + 8);
  int* redi = reinterpret_cast<int*>(redf + 8);
  int* perm = redi + 8;

  const DeviceView& D = a.devs[W.dev];
  const ChainView& C = D.ch[W.chain];
  const int L = D.L, b = D.b, rpb = D.rpb;
  const int spr = b / rpb;
  const int k = W.e0;
  const double g = 2.0 * C.g_b;
  const bool real = (W.kind == 0);
  const LeadView& LS = C.lead[0];
  const LeadView& LD = C.lead[1];
  const int mS = LS.m, mD = LD.m;
  double* part = a.partial + W.part;
  const int kmax = C.kmax;
  const int nn = b * b;

  cd eps;
  double wS = 0.0, wD = 0.0;
  cd kap = mk(0.0, 0.0);
  const int eidx = real ? k : D.n_real + k;   // energy index of the view (general leads)
  if (real) {
    eps = mk(D.E[k], D.eta);
    wS = g * D.w[k] * D.fS[k] * (0.5 / 3.14159265358979323846);
    wD = g * D.w[k] * D.fD[k] * (0.5 / 3.14159265358979323846);
  } else {
    eps = D.z[k];
    kap = scale(D.c[k], g / 3.14159265358979323846);
  }

  // ---- lead self-energies in FP64: per-mode roots sigma_j, then the circulant first
  //      row Sigma[s][t] = (1/m) sum_j sigma_j w^{j (s - t)}, kept as row[d], d = (s - t) mod m
  //      (a thread holds at most two modes: m <= MAX_LEAD <= 2 * NT)
  for (int side = 0; side < 2; ++side) {
    const LeadView& Lv = C.lead[side];
    if (Lv.gen) continue;   // general lead: Sigma and its Gamma factor come from the plan
    cd* row = side ? sigD : sigS;
    double* sq = side ? sqD : sqS;
    const int m = Lv.m;
    for (int j = tid; j < m; j += NT) {
      const cd sj = mode_sigma(Lv, j, eps);
      row[j] = sj;
      sq[j] = sqrt(fmax(-2.0 * sj.im, 0.0) / m);
    }
    csync<NW>();
    cd keep[2] = {mk(0.0, 0.0), mk(0.0, 0.0)};
    for (int d = tid, q = 0; d < m && q < 2; d += NT, ++q) {
      cd acc = mk(0.0, 0.0);
      for (int j = 0; j < m; ++j) {
        const int e = (j * d) % m;
        acc = cmac(acc, row[j], mk(Lv.tw[2 * e], Lv.tw[2 * e + 1]));
      }
      keep[q] = scale(acc, 1.0 / m);
    }
    csync<NW>();
    for (int d = tid, q = 0; d < m && q < 2; d += NT, ++q) row[d] = keep[q];
    csync<NW>();
  }

  // ---- forward sweep: P = gL_{l-1} (M0), A (M1), X (M2); R (V0), Rn (V1).  The compact
  //      layout updates R in place through registers (Rn aliases R).
  RegTile<T> rt;
  cx<T>* P = M0;
  cx<T>* A = M1;
  cx<T>* X = M2;
  cx<T>* R = V0;
  cx<T>* Rn = CMP ? V0 : V1;
  const long long lstride = (long long)(bb + (real ? bm : 0)) * sizeof(cx<T>);
  float gmax = 0.0f;   // largest |gL_l entry|^2 of this thread (growth diagnostic)
  float gdg = 0.0f;
  for (int l = 0; l < L; ++l) {
    if (l > 0) {
      const int* ccnt = C.cs_cnt + (long long)(l - 1) * C.cp_step;
      const int* cidx = C.cs_idx + (long long)(l - 1) * C.cp_step * kmax;
      const cx<T>* cval = csval_t<T>(C) + (long long)(l - 1) * C.cp_step * kmax;
      hdn_times<T, NT>(X, P, b, b, b, ccnt, cidx, cval, kmax, tid);            // X = H_{l,l-1} gL_{l-1}
      csync<NW>();
      times_hup<T, NT>(A, X, b, b, ccnt, cidx, cval, kmax, tid);               // y_l = X H_{l-1,l}
      if (real) {                                                                // R_l = X R_{l-1}
        if constexpr (CMP)
          bgemm_r<T, NT>(rt, X, b, R, mS, b, b, mS, nullptr, 0, tid);
        else
          bgemm<T, NT>(Rn, mS, X, b, R, mS, b, b, mS, nullptr, 0, tid);
      }
      csync<NW>();
      if constexpr (CMP) {
        if (real) store_r<T, NT>(Rn, mS, rt, b, mS, tid);   // read before the next barrier (binv)
      }
      alpha_minus<T, NW>(A, A, l, L, b, rpb, spr, eps, D, C, sigS, sigD, eidx, tid);  // alpha_l - y_l
    } else {
      if (real) {
        // R_0 = L_S: rows at the lead sites, L_S[site_s][j] = w^{j s} sqrt(gamma_j / m)
        // (circulant lead) or the plan's factor of Gamma_S (general lead)
        for (int o = tid; o < b * mS; o += NT) Rn[o] = cz<T>();
        csync<NW>();
        const cd* fS = LS.gen ? LS.gfac + (long long)eidx * mS * mS : nullptr;
        for (int o = tid; o < mS * mS; o += NT) {
          const int s = o / mS, j = o - s * mS;
          const int e = (j * s) % mS;
          Rn[LS.sites[s] * mS + j] = tc<T>(fS ? fS[o] : scale(mk(LS.tw[2 * e], LS.tw[2 * e + 1]), sqS[j]));
        }
      }
      alpha_minus<T, NW>(A, nullptr, 0, L, b, rpb, spr, eps, D, C, sigS, sigD, eidx, tid);
    }
    binv<T, NW>(A, b, col, perm, redf, redi, tid);
    if (!TWO && C.sym)   // largest |gL_l diagonal|^2 seen by this thread (symmetric-update gate)
      for (int r = tid; r < b; r += NT)
        gdg = fmaxf(gdg, fmaf((float)A[r * b + r].re, (float)A[r * b + r].re,
                              (float)A[r * b + r].im * (float)A[r * b + r].im));
    // stage gL_l (and R_l)
    cx<T>* sg = reinterpret_cast<cx<T>*>(stage + (long long)l * lstride);
    for (int o = tid; o < nn; o += NT) {
      sg[o] = A[o];
      if (a.growth) gmax = fmaxf(gmax, fmaf((float)A[o].re, (float)A[o].re, (float)A[o].im * (float)A[o].im));
    }
    if (real)
      for (int o = tid; o < b * mS; o += NT) sg[bb + o] = Rn[o];
    csync<NW>();
    cx<T>* t = P;
    P = A;
    A = t;
    if constexpr (!CMP) {
      t = R;
      R = Rn;
      Rn = t;
    }
  }

  // The symmetric form of the G_ll update is used for a lane only while every gL_l stays
  // moderate.  Near a bound state of the half chain [0, l] (a pole of gL_l broadened by eta
  // only) the Dyson update cancels terms of size |gL|^2 / |G|, and the mirrored form then
  // turns the rounding asymmetry of gL_l into errors of order one; those lanes take the
  // general update.
  const bool lsym = !TWO && C.sym && cta_max<NW>((double)gdg, redd, tid) <= SYM_GL_MAX * SYM_GL_MAX;
  if (a.lane_stats && tid == 0) atomicAdd(a.lane_stats + (real ? 0 : 2) + (lsym ? 0 : 1), 1ull);

  // ---- backward sweep
  //  Dyson variant:     G (P: gL_{L-1} = G_{L-1,L-1}), Gl, Z, Wm
  //  two-sided variant: G, Gr = gR_{l+1}, Wk, W1, GlB = gL_l, GpB = gL_{l-1}
  //  both:              K, Kn (drain column factor), Rl (R_l)
  //  compact Dyson:     G, Gl (gL_l, then R_l), Z; K (in place); Wm and the new G in
  //                     registers
  cx<T>* G = P;
  cx<T>* Gl = A;       // Dyson: gL_l;  two-sided: work matrix Wk
  cx<T>* Z = X;        // Dyson: Z;     two-sided: W1
  cx<T>* Wm = M3;      // Dyson: Wm;    two-sided: Gr
  cx<T>* GlB = M4;     // two-sided only
  cx<T>* GpB = M5;     // two-sided only
  if (lsym) {
    symmetrize<T, NT>(G, b, tid);
    csync<NW>();
  }
  // compact: K takes V0, R_l lives in the Gl buffer (loaded after each G_ll update)
  cx<T>* K = CMP ? V0 : ((R == V0) ? V1 : V0);
  cx<T>* Kn = CMP ? K : V2;
  cx<T>* Rl = CMP ? Gl : R;
  if (CMP && real) {
    for (int o = tid; o < b * mS; o += NT) Rl[o] = R[o];   // R_{L-1} out of V0
    csync<NW>();
  }
  if (real) {
    // K_{L-1} = G_{L-1,L-1} L_D: K[r][j] = sum_s G[r][site_s] w^{j s} sqrt(gamma_j/m)
    // (circulant lead) or sum_s G[r][site_s] L_D[s][j] (general lead)
    const cd* fD = LD.gen ? LD.gfac + (long long)eidx * mD * mD : nullptr;
    for (int o = tid; o < b * mD; o += NT) {
      const int r = o / mD, j = o - r * mD;
      cx<T> acc = cz<T>();
      if (fD) {
        for (int s = 0; s < mD; ++s) acc = cmac(acc, G[r * b + LD.sites[s]], tc<T>(fD[s * mD + j]));
        K[o] = acc;
      } else {
        for (int s = 0; s < mD; ++s) {
          const int e = (j * s) % mD;
          acc = cmac(acc, G[r * b + LD.sites[s]], tc<T>(mk(LD.tw[2 * e], LD.tw[2 * e + 1])));
        }
        K[o] = scale(acc, (T)sqD[j]);
      }
    }
    csync<NW>();
  }
  if (TWO && L > 1) {
    // gR_{L-1} = alpha_{L-1}^{-1} (into Wm), gL_{L-2} into GlB
    alpha_minus<T, NW>(Wm, nullptr, L - 1, L, b, rpb, spr, eps, D, C, sigS, sigD, eidx, tid);
    binv<T, NW>(Wm, b, col, perm, redf, redi, tid);
    const cx<T>* sg = reinterpret_cast<const cx<T>*>(stage + (long long)(L - 2) * lstride);
    for (int o = tid; o < nn; o += NT) GlB[o] = sg[o];
    csync<NW>();
  }
  T rnum = T(0), rden = T(0);   // sum-rule residual: max(0, A_S + A_D + 2 Im G) / max |2 Im G|
  for (int l = L - 1; l >= 0; --l) {
    if (l < L - 1) {
      const cx<T>* sg = reinterpret_cast<const cx<T>*>(stage + (long long)l * lstride);
      const int* ccnt = C.cs_cnt + (long long)l * C.cp_step;
      const int* cidx = C.cs_idx + (long long)l * C.cp_step * kmax;
      const cx<T>* cval = csval_t<T>(C) + (long long)l * C.cp_step * kmax;
      if (!TWO) {
        for (int o = tid; o < nn; o += NT) Gl[o] = sg[o];
        if (real && !CMP)
          for (int o = tid; o < b * mS; o += NT) Rl[o] = sg[bb + o];
        csync<NW>();
        if (lsym) {   // the symmetric update needs gL_l symmetric to the last bit
          symmetrize<T, NT>(Gl, b, tid);
          csync<NW>();
        }
        times_hup<T, NT>(Z, Gl, b, b, ccnt, cidx, cval, kmax, tid);                // Z = gL_l H_{l,l+1}
        csync<NW>();
        if constexpr (CMP) {
          bgemm_r<T, NT>(rt, Z, b, G, b, b, b, b, nullptr, 0, tid);                 // Wm = Z G_{l+1}
          csync<NW>();
          store_r<T, NT>(G, b, rt, b, b, tid);                                      // G := Wm
          if (real) {
            bgemm_r<T, NT>(rt, Z, b, K, mD, b, b, mD, nullptr, 0, tid);             // K_l = Z K_{l+1}
            csync<NW>();
            store_r<T, NT>(K, mD, rt, b, mD, tid);
          }
          csync<NW>();
          if (lsym) {
            // G_ll = gL_l + Z G_{l+1} Z^T is symmetric: upper triangle, mirrored
            bgemm_symt_r<T, NT>(rt, G, Z, Gl, b, tid);
            csync<NW>();
            store_sym<T, NT>(G, rt, b, tid);
          } else {
            hdn_times<T, NT>(Z, Gl, b, b, b, ccnt, cidx, cval, kmax, tid);         // Z = H_{l+1,l} gL_l
            csync<NW>();
            bgemm_r<T, NT>(rt, G, b, Z, b, b, b, b, Gl, b, tid);                    // gL_l + Wm Z
            csync<NW>();
            store_r<T, NT>(G, b, rt, b, b, tid);
          }
          if (real)
            for (int o = tid; o < b * mS; o += NT) Rl[o] = sg[bb + o];             // R_l into Gl
          csync<NW>();
        } else {
          if (real) bgemm<T, NT>(Kn, mD, Z, b, K, mD, b, b, mD, nullptr, 0, tid);  // K_l = Z K_{l+1}
          bgemm<T, NT>(Wm, b, Z, b, G, b, b, b, b, nullptr, 0, tid);               // Wm = Z G_{l+1}
          csync<NW>();
          if (lsym) {
            bgemm_symt<T, NT>(G, Wm, Z, Gl, b, tid);                                // gL_l + Wm Z^T
          } else {
            hdn_times<T, NT>(Z, Gl, b, b, b, ccnt, cidx, cval, kmax, tid);         // Z = H_{l+1,l} gL_l
            csync<NW>();
            bgemm<T, NT>(G, b, Wm, b, Z, b, b, b, b, Gl, b, tid);                   // G = gL_l + Wm Z
          }
          csync<NW>();
        }
      } else {
        // G_ll = (alpha_l - x_l - y_l)^{-1} with x_l = H_{l,l+1} gR_{l+1} H_{l+1,l} and
        // y_l = H_{l,l-1} gL_{l-1} H_{l-1,l}: no cancellation between large terms
        cx<T>* Wk = Gl;
        cx<T>* W1 = Z;
        cx<T>* Gr = Wm;
        const int* rcnt = C.rs_cnt + (long long)l * C.cp_step;
        const int* ridx = C.rs_idx + (long long)l * C.cp_step * kmax;
        const cx<T>* rval = rsval_t<T>(C) + (long long)l * C.cp_step * kmax;
        if (real)
          for (int o = tid; o < b * mS; o += NT) Rl[o] = sg[bb + o];
        if (l > 0) {
          const cx<T>* sp = reinterpret_cast<const cx<T>*>(stage + (long long)(l - 1) * lstride);
          for (int o = tid; o < nn; o += NT) GpB[o] = sp[o];
        }
        hup_times<T, NT>(W1, Gr, b, b, b, rcnt, ridx, rval, kmax, tid);             // H_{l,l+1} gR_{l+1}
        if (real) times_hup<T, NT>(Z == W1 ? Wk : Wk, GlB, b, b, ccnt, cidx, cval, kmax, tid);  // gL_l H_{l,l+1}
        csync<NW>();
        if (real) bgemm<T, NT>(Kn, mD, Wk, b, K, mD, b, b, mD, nullptr, 0, tid);   // K_l = gL_l H K_{l+1}
        times_hdn<T, NT>(G, W1, b, b, rcnt, ridx, rval, kmax, tid);                  // x_l (into G)
        csync<NW>();
        alpha_minus<T, NW>(Gr, G, l, L, b, rpb, spr, eps, D, C, sigS, sigD, eidx, tid);  // alpha_l - x_l
        if (l > 0) {
          const int* pcnt = C.cs_cnt + (long long)(l - 1) * C.cp_step;
          const int* pidx = C.cs_idx + (long long)(l - 1) * C.cp_step * kmax;
          const cx<T>* pval = csval_t<T>(C) + (long long)(l - 1) * C.cp_step * kmax;
          hdn_times<T, NT>(W1, GpB, b, b, b, pcnt, pidx, pval, kmax, tid);          // H_{l,l-1} gL_{l-1}
          csync<NW>();
          times_hup<T, NT>(Wk, W1, b, b, pcnt, pidx, pval, kmax, tid);              // y_l
          csync<NW>();
          for (int o = tid; o < nn; o += NT) G[o] = Gr[o] - Wk[o];
        } else {
          for (int o = tid; o < nn; o += NT) G[o] = Gr[o];
        }
        csync<NW>();
        binv<T, NW>(G, b, col, perm, redf, redi, tid);                              // G_ll
        if (l > 0) binv<T, NW>(Gr, b, col, perm, redf, redi, tid);                  // gR_l
        cx<T>* t = GlB;
        GlB = GpB;
        GpB = t;
      }
      if (real && !CMP) {
        cx<T>* t = K;
        K = Kn;
        Kn = t;
      }
    }
    // per-site contributions of layer l, summed per ring.  The row sums and ring sums run
    // on warp 0 with a fixed lane mapping, so the result does not depend on the CTA width.
    double vr[2] = {0.0, 0.0};
    cx<T>* Pm = (TWO || CMP) ? Z : Wm;   // free b x m buffer for G_ll R_l (m <= b)
    if (real) {
      bgemm<T, NT>(Pm, mS, G, b, Rl, mS, b, b, mS, nullptr, 0, tid);               // G_ll R_l
      csync<NW>();
      if (tid < 32)
        for (int r = tid; r < b; r += 32) {
          T as = T(0), ad = T(0);
          for (int j = 0; j < mS; ++j) as = fma(Pm[r * mS + j].im, Pm[r * mS + j].im, fma(Pm[r * mS + j].re, Pm[r * mS + j].re, as));
          for (int j = 0; j < mD; ++j) ad = fma(K[r * mD + j].im, K[r * mD + j].im, fma(K[r * mD + j].re, K[r * mD + j].re, ad));
          vr[r / spr] = fma(wS, (double)as, fma(wD, (double)ad, vr[r / spr]));
          if (a.resid) {
            rnum = fmax(rnum, fma(T(2), G[r * b + r].im, as + ad));
            rden = fmax(rden, fabs(T(2) * G[r * b + r].im));
          }
        }
    } else if (tid < 32) {
      for (int r = tid; r < b; r += 32) {
        const cx<T> gd = G[r * b + r];
        vr[r / spr] = fma(kap.re, (double)gd.im, fma(kap.im, (double)gd.re, vr[r / spr]));
      }
    }
    if (tid < 32)
      for (int q = 0; q < rpb; ++q) {
        const double s = wsum(vr[q]);
        if (tid == 0) part[l * rpb + q] = s;
      }
    csync<NW>();
  }
  if (real) {
    // T = || L_S^dag K_0 ||_F^2, (L_S^dag K_0)[i][j] = sum_s conj(L_S[site_s][i]) K_0[site_s][j]
    // (warp 0, fixed lane mapping)
    double tv = 0.0;
    const cd* fS = LS.gen ? LS.gfac + (long long)eidx * mS * mS : nullptr;
    if (tid < 32)
      for (int o = tid; o < mS * mD; o += 32) {
        const int i = o / mD, j = o - i * mD;
        cx<T> acc = cz<T>();
        if (fS) {
          for (int s = 0; s < mS; ++s) acc = cmac_cj(acc, tc<T>(fS[s * mS + i]), K[LS.sites[s] * mD + j]);
          tv += (double)abs2(acc);
        } else {
          for (int s = 0; s < mS; ++s) {
            const int e = (i * s) % mS;
            acc = cmac_cj(acc, tc<T>(mk(LS.tw[2 * e], LS.tw[2 * e + 1])), K[LS.sites[s] * mD + j]);
          }
          tv = fma((double)abs2(acc), sqS[i] * sqS[i], tv);
        }
      }
    const double Tval = tid < 32 ? wsum(tv) : 0.0;
    if (tid == 0) a.Tpart[W.tout] = Tval;
    if (a.resid) {
      const double rn = cta_max<NW>((double)rnum, redd, tid);
      const double rd = cta_max<NW>((double)rden, redd, tid);
      if (tid == 0) a.resid[W.tout] = rn / fmax(rd, 1e-300);
    }
    if (a.growth) {
      const double gm = cta_max<NW>((double)gmax, redd, tid);
      if (tid == 0) a.growth[W.tout] = sqrt(gm);
    }
  }
  csync<NW>();
}

}  // namespace negf
