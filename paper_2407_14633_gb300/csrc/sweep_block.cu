// Warp-per-lane recursive Green's function sweep for wide ring blocks (real space).
//
// One warp owns one (device, chain, energy) lane and keeps its b x b complex blocks in
// shared memory; every product spreads its outputs over the 32 threads.  The algorithm
// is the left-connected recursion (Alg. 2 reading) with the lead columns propagated as
// factors of the broadening matrices:  Gamma_l = L_l L_l^dagger with
// L_l = F diag(sqrt(gamma_j)) from the circulant lead (F the ring Fourier basis), so that
//   forward   X = H_{l,l-1} gL_{l-1},  gL_l = (alpha_l - X H_{l-1,l})^{-1},
//             R_l = X R_{l-1} (R_0 = L_S)                 [R_l = G_{l,l}^{-1} G_{l,0} L_S]
//   backward  Z = gL_l H_{l,l+1},  G_ll = gL_l + Z G_{l+1,l+1} (H_{l+1,l} gL_l),
//             K_l = Z K_{l+1} (K_{L-1} = G_{L-1,L-1} L_D)  [K_l = G_{l,L-1} L_D]
//   A_S,ll = (G_ll R_l)(G_ll R_l)^dagger,  A_D,ll = K_l K_l^dagger,
//   T = || L_S^dagger K_0 ||_F^2 = Tr[Gamma_S G_{0,L-1} Gamma_D G_{0,L-1}^dagger].
// Products with the coupling blocks use their padded sparse form (kmax entries per row or
// column; kmax = b for dense couplings).  gL_l and R_l are staged per resident warp in
// global memory.  FP64 throughout; the FP64 pipe is the bound on GB300.
#include "common.cuh"
#include "lead.cuh"

namespace negf {

namespace {

__device__ __forceinline__ cd czero() { return mk(0.0, 0.0); }

// C (R x N, ldc) = [Add +] A (R x K, lda) * B (K x N, ldb); outputs spread over the warp
__device__ __forceinline__ void wgemm(cd* C, int ldc, const cd* A, int lda, const cd* B, int ldb,
                                      int R, int K, int N, const cd* Add, int ldadd, int lane) {
  const int tot = R * N;
  for (int o = lane; o < tot; o += 32) {
    const int r = o / N, c = o - r * N;
    cd acc = Add ? Add[r * ldadd + c] : czero();
    const cd* a = A + r * lda;
    const cd* b = B + c;
#pragma unroll 4
    for (int k = 0; k < K; ++k) acc = cmac(acc, a[k], b[k * ldb]);
    C[r * ldc + c] = acc;
  }
}

// C (b x N) = H_{l+1,l} * M  where H_{l+1,l} = Hup_l^dagger: row r uses column r of Hup_l
__device__ __forceinline__ void hdn_times(cd* C, const cd* M, int ldm, int N, int b,
                                          const int* cs_cnt, const int* cs_idx,
                                          const cd* cs_val, int kmax, int lane) {
  const int tot = b * N;
  for (int o = lane; o < tot; o += 32) {
    const int r = o / N, c = o - r * N;
    cd acc = czero();
    const int n = cs_cnt[r];
    for (int e = 0; e < n; ++e) {
      const int k = cs_idx[r * kmax + e];
      acc = cmac_cj(acc, cs_val[r * kmax + e], M[k * ldm + c]);
    }
    C[r * N + c] = acc;
  }
}

// C (R x b) = M (R x b) * Hup_l : column c uses column c of Hup_l
__device__ __forceinline__ void times_hup(cd* C, const cd* M, int R, int b, const int* cs_cnt,
                                          const int* cs_idx, const cd* cs_val, int kmax,
                                          int lane) {
  const int tot = R * b;
  for (int o = lane; o < tot; o += 32) {
    const int r = o / b, c = o - r * b;
    cd acc = czero();
    const int n = cs_cnt[c];
    for (int e = 0; e < n; ++e) {
      const int k = cs_idx[c * kmax + e];
      acc = cmac(acc, M[r * b + k], cs_val[c * kmax + e]);
    }
    C[r * b + c] = acc;
  }
}

// in-place Gauss-Jordan inverse of the b x b block A with partial pivoting (row swaps
// recorded in perm, undone on the columns at the end); col: b scratch entries
__device__ void winv(cd* A, int b, cd* col, int* perm, int lane) {
  for (int k = 0; k < b; ++k) {
    // pivot search on column k, rows k..b-1
    double best = -1.0;
    int bi = k;
    for (int i = k + lane; i < b; i += 32) {
      const double m = abs2(A[i * b + k]);
      if (m > best) {
        best = m;
        bi = i;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) perm[k] = bi;
    if (bi != k) {
      for (int j = lane; j < b; j += 32) {
        const cd t = A[k * b + j];
        A[k * b + j] = A[bi * b + j];
        A[bi * b + j] = t;
      }
    }
    __syncwarp();
    const cd ip = crecip(A[k * b + k]);
    for (int i = lane; i < b; i += 32) col[i] = A[i * b + k];
    __syncwarp();
    for (int j = lane; j < b; j += 32) A[k * b + j] = (j == k) ? ip : A[k * b + j] * ip;
    __syncwarp();
    const int tot = (b - 1) * b;
    for (int o = lane; o < tot; o += 32) {
      int i = o / b;
      const int j = o - i * b;
      i += (i >= k);
      const cd f = col[i];
      if (j == k) {
        A[i * b + k] = czero() - f * ip;
      } else {
        A[i * b + j] = A[i * b + j] - f * A[k * b + j];
      }
    }
    __syncwarp();
  }
  __syncwarp();
  for (int k = b - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      for (int i = lane; i < b; i += 32) {
        const cd t = A[i * b + k];
        A[i * b + k] = A[i * b + p];
        A[i * b + p] = t;
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace

__host__ __device__ size_t sweep_blk_smem_bytes(int b, int m, int warps) {
  // per warp: 4 b^2 + 3 b m complex, 2 m sigma/gamma rows, b scratch column, b ints
  size_t per = (size_t)(4 * b * b + 3 * b * m + 4 * m + b) * sizeof(cd) + (size_t)b * sizeof(int);
  per = (per + 15) & ~(size_t)15;
  return per * warps;
}

__global__ void __launch_bounds__(256) sweep_blk_kernel(SweepArgs a, int bmax, int mmax) {
  extern __shared__ __align__(16) unsigned char sm_blk[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const size_t per = sweep_blk_smem_bytes(bmax, mmax, 1);
  cd* base = reinterpret_cast<cd*>(sm_blk + per * wib);
  const int bb = bmax * bmax, bm = bmax * mmax;
  cd* M0 = base;             // b x b
  cd* M1 = M0 + bb;          // b x b
  cd* M2 = M1 + bb;          // b x b
  cd* M3 = M2 + bb;          // b x b
  cd* V0 = M3 + bb;          // b x m
  cd* V1 = V0 + bm;          // b x m
  cd* V2 = V1 + bm;          // b x m
  cd* sigS = V2 + bm;        // m: circulant first row of Sigma_S / per-mode sqrt(gamma) in .re
  cd* sigD = sigS + mmax;
  cd* sqS = sigD + mmax;     // m: sqrt(gamma_j / m) of the source (re)
  cd* sqD = sqS + mmax;
  cd* col = sqD + mmax;      // b
  int* perm = reinterpret_cast<int*>(col + bmax);
  unsigned char* stage = a.stage + (long long)gw * a.stage_stride;

  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(a.counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= a.n_items) break;
    const WorkItem W = a.items[a.order[it]];
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
    cd kap = czero();
    if (real) {
      eps = mk(D.E[k], D.eta);
      wS = g * D.w[k] * D.fS[k] * (0.5 / 3.14159265358979323846);
      wD = g * D.w[k] * D.fD[k] * (0.5 / 3.14159265358979323846);
    } else {
      eps = D.z[k];
      kap = scale(D.c[k], g / 3.14159265358979323846);
    }

    // ---- lead self-energies: per-mode roots (FP64), circulant first rows
    //      Sigma[s][t] = (1/m) sum_j sigma_j w^{j (s - t)}, stored as row[d], d = (s - t) mod m
    for (int side = 0; side < 2; ++side) {
      const LeadView& Lv = C.lead[side];
      cd* row = side ? sigD : sigS;
      cd* sq = side ? sqD : sqS;
      const int m = Lv.m;
      // per-mode sigma_j into `col` scratch (m <= MAX_LEAD, col has b >= m entries)
      for (int j = lane; j < m; j += 32) {
        const cd sj = mode_sigma(Lv, j, eps);
        col[j] = sj;
        sq[j] = mk(sqrt(fmax(-2.0 * sj.im, 0.0) / m), 0.0);
      }
      __syncwarp();
      for (int d = lane; d < m; d += 32) {
        cd acc = czero();
        for (int j = 0; j < m; ++j) {
          const int e = (j * d) % m;
          acc = cmac(acc, col[j], mk(Lv.tw[2 * e], Lv.tw[2 * e + 1]));
        }
        row[d] = scale(acc, 1.0 / m);
      }
      __syncwarp();
    }

    // ---- forward sweep: P = gL_{l-1} (M0), A (M1), X (M2); R (V0), Rn (V1)
    cd* P = M0;
    cd* A = M1;
    cd* X = M2;
    cd* R = V0;
    cd* Rn = V1;
    const long long lstride = (long long)(bb + (real ? bm : 0)) * sizeof(cd);
    for (int l = 0; l < L; ++l) {
      const cd* hd = C.Hdiag + (long long)l * b * b;
      if (l > 0) {
        const int* ccnt = C.cs_cnt + (long long)(l - 1) * b;
        const int* cidx = C.cs_idx + (long long)(l - 1) * b * kmax;
        const cd* cval = C.cs_val + (long long)(l - 1) * b * kmax;
        // X = H_{l,l-1} gL_{l-1}
        hdn_times(X, P, b, b, b, ccnt, cidx, cval, kmax, lane);
        __syncwarp();
        // A = X H_{l-1,l}  (subtracted below)
        times_hup(A, X, b, b, ccnt, cidx, cval, kmax, lane);
        if (real) {
          __syncwarp();
          wgemm(Rn, mS, X, b, R, mS, b, b, mS, nullptr, 0, lane);
        }
      } else {
        for (int o = lane; o < nn; o += 32) A[o] = czero();
        if (real) {
          // R_0 = L_S: rows at the lead sites, L_S[site_s][j] = w^{j s} sqrt(gamma_j / m)
          for (int o = lane; o < b * mS; o += 32) Rn[o] = czero();
          __syncwarp();
          for (int o = lane; o < mS * mS; o += 32) {
            const int s = o / mS, j = o - s * mS;
            const int e = (j * s) % mS;
            Rn[LS.sites[s] * mS + j] = scale(mk(LS.tw[2 * e], LS.tw[2 * e + 1]), sqS[j].re);
          }
        }
      }
      __syncwarp();
      // A = eps I - H_ll - U - X H_{l-1,l} - Sigma
      for (int o = lane; o < nn; o += 32) {
        const int r = o / b, c = o - r * b;
        cd v = czero() - hd[o] - A[o];
        if (r == c) {
          const int ring = l * rpb + r / spr;
          v = v + mk(eps.re - D.U[ring], eps.im);
        }
        A[o] = v;
      }
      __syncwarp();
      if (l == 0) {
        for (int o = lane; o < mS * mS; o += 32) {
          const int s = o / mS, t = o - s * mS;
          const int d = ((s - t) % mS + mS) % mS;
          const int rs = LS.sites[s], rt = LS.sites[t];
          A[rs * b + rt] = A[rs * b + rt] - sigS[d];
        }
        __syncwarp();
      }
      if (l == L - 1) {
        for (int o = lane; o < mD * mD; o += 32) {
          const int s = o / mD, t = o - s * mD;
          const int d = ((s - t) % mD + mD) % mD;
          const int rs = LD.sites[s], rt = LD.sites[t];
          A[rs * b + rt] = A[rs * b + rt] - sigD[d];
        }
        __syncwarp();
      }
      winv(A, b, col, perm, lane);
      // stage gL_l (and R_l)
      cd* sg = reinterpret_cast<cd*>(stage + (long long)l * lstride);
      for (int o = lane; o < nn; o += 32) sg[o] = A[o];
      if (real)
        for (int o = lane; o < b * mS; o += 32) sg[bb + o] = Rn[o];
      __syncwarp();
      cd* t = P;
      P = A;
      A = t;
      t = R;
      R = Rn;
      Rn = t;
    }

    // ---- backward sweep.  G (P: gL_{L-1} = G_{L-1,L-1}), Gl, Z, Wm; K, Kn, Rl
    cd* G = P;
    cd* Gl = A;
    cd* Z = X;
    cd* Wm = M3;   // the forward used M0..M2 only
    cd* K = (R == V0) ? V1 : V0;   // R holds R_{L-1}; use the other two for K
    cd* Kn = V2;
    cd* Rl = R;
    if (real) {
      // K_{L-1} = G_{L-1,L-1} L_D: K[r][j] = sum_s G[r][site_s] w^{j s} sqrt(gamma_j/m)
      for (int o = lane; o < b * mD; o += 32) {
        const int r = o / mD, j = o - r * mD;
        cd acc = czero();
        for (int s = 0; s < mD; ++s) {
          const int e = (j * s) % mD;
          acc = cmac(acc, G[r * b + LD.sites[s]], mk(LD.tw[2 * e], LD.tw[2 * e + 1]));
        }
        K[o] = scale(acc, sqD[j].re);
      }
      __syncwarp();
    }
    double Tval = 0.0;
    for (int l = L - 1; l >= 0; --l) {
      if (l < L - 1) {
        const cd* sg = reinterpret_cast<const cd*>(stage + (long long)l * lstride);
        for (int o = lane; o < nn; o += 32) Gl[o] = sg[o];
        if (real)
          for (int o = lane; o < b * mS; o += 32) Rl[o] = sg[bb + o];
        __syncwarp();
        const int* ccnt = C.cs_cnt + (long long)l * b;
        const int* cidx = C.cs_idx + (long long)l * b * kmax;
        const cd* cval = C.cs_val + (long long)l * b * kmax;
        // Z = gL_l H_{l,l+1}
        times_hup(Z, Gl, b, b, ccnt, cidx, cval, kmax, lane);
        __syncwarp();
        if (real) wgemm(Kn, mD, Z, b, K, mD, b, b, mD, nullptr, 0, lane);
        // Wm = Z G_{l+1}
        wgemm(Wm, b, Z, b, G, b, b, b, b, nullptr, 0, lane);
        __syncwarp();
        // Z = H_{l+1,l} gL_l
        hdn_times(Z, Gl, b, b, b, ccnt, cidx, cval, kmax, lane);
        __syncwarp();
        // G = gL_l + Wm Z
        wgemm(G, b, Wm, b, Z, b, b, b, b, Gl, b, lane);
        __syncwarp();
        if (real) {
          cd* t = K;
          K = Kn;
          Kn = t;
        }
      }
      // per-site contributions of layer l, summed per ring
      double vr[2] = {0.0, 0.0};
      if (real) {
        // Pm = G_ll R_l into Wm, then row norms
        wgemm(Wm, mS, G, b, Rl, mS, b, b, mS, nullptr, 0, lane);
        __syncwarp();
        for (int r = lane; r < b; r += 32) {
          double as = 0.0, ad = 0.0;
          for (int j = 0; j < mS; ++j) as += abs2(Wm[r * mS + j]);
          for (int j = 0; j < mD; ++j) ad += abs2(K[r * mD + j]);
          vr[r / spr] += wS * as + wD * ad;
        }
      } else {
        for (int r = lane; r < b; r += 32) {
          const cd gd = G[r * b + r];
          vr[r / spr] += kap.re * gd.im + kap.im * gd.re;
        }
      }
      for (int q = 0; q < rpb; ++q) {
        const double s = warp_sum(vr[q]);
        if (lane == 0) part[l * rpb + q] = s;
      }
      __syncwarp();
    }
    if (real) {
      // T = || L_S^dag K_0 ||_F^2, (L_S^dag K_0)[i][j] = sum_s conj(L_S[site_s][i]) K_0[site_s][j]
      double tv = 0.0;
      for (int o = lane; o < mS * mD; o += 32) {
        const int i = o / mD, j = o - i * mD;
        cd acc = czero();
        for (int s = 0; s < mS; ++s) {
          const int e = (i * s) % mS;
          acc = cmac_cj(acc, mk(LS.tw[2 * e], LS.tw[2 * e + 1]), K[LS.sites[s] * mD + j]);
        }
        tv += abs2(acc) * sqS[i].re * sqS[i].re;
      }
      Tval = warp_sum(tv);
      if (lane == 0) a.Tpart[W.tout] = Tval;
    }
    __syncwarp();
  }
}

int launch_sweep_blk_f64(const SweepArgs& a, int b_max, int m_max, int grid, int warps,
                         cudaStream_t s) {
  // the dynamic shared memory limit was raised by sweep_blk_occupancy when planning
  const size_t smem = sweep_blk_smem_bytes(b_max, m_max, warps);
  sweep_blk_kernel<<<grid, warps * 32, smem, s>>>(a, b_max, m_max);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace negf

namespace negf {
int sweep_blk_occupancy(int warps, size_t smem) {
  cudaFuncSetAttribute(sweep_blk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep_blk_kernel, warps * 32, smem) != cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    per = 1;
  }
  return per;
}
}  // namespace negf
