// Thread-per-lane recursive Green's function sweeps for narrow blocks (b = 1, 2).
//
// One warp takes a work item of up to 32 energies of one (device, chain, kind); each
// thread runs the whole forward and backward sweep of its energy (the paper's Alg. 2
// recursion done per energy, Sec. 2.2.4 "future work": store the per-energy recursion
// vectors instead of recomputing them).  The forward quantities are staged per resident
// warp in global memory, interleaved [layer][field][lane] so every warp access is one
// coalesced 256-byte line.  Per-ring contributions of the 32 energies are reduced through
// a 32 x 33 shared-memory transpose (one add per ring and lane, fixed order) into the
// item's partial sums; the second stage (reduce.cu) sums items in item order, so results
// do not depend on how items are scheduled or batched.
//
// b = 1 (mode space): with scalar blocks the lead columns need only moduli,
//   q_l = |G_{l,0}|^2 / |G_{l,l}|^2 = |h_{l-1}|^2 |gL_{l-1}|^2 q_{l-1},  q_0 = 1,
//   c_l = |G_{l,L-1}|^2 = |gL_l|^2 |h_l|^2 c_{l+1},  c_{L-1} = |G_{L-1,L-1}|^2,
//   G_{l,l} = gL_l + gL_l^2 |h_l|^2 G_{l+1,l+1},
//   A_S,ll = Gamma_S q_l |G_ll|^2, A_D,ll = Gamma_D c_l, T = Gamma_S Gamma_D c_0.
#include <algorithm>

#include "common.cuh"
#include "lead.cuh"

namespace negf {

namespace {

__device__ __forceinline__ int next_item(int* counter, int lane) {
  int it = 0;
  if (lane == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}

// flush ring slots [base, base + count) of the 32 x 33 transpose buffer into `dst`; the
// buffer holds the sweep's element type (the complex64 sweep accumulates its per-lane ring
// contributions in FP32: the FP64 pipe of this part is 1/62 of the FP32 one)
template <typename T>
__device__ __forceinline__ void flush_rings(T* red, int lane, int count, double* dst) {
  __syncwarp();
  if (lane < count) {
    T s = T(0);
#pragma unroll 8
    for (int j = 0; j < 32; ++j) s += red[lane * 33 + j];
    dst[lane] = (double)s;
  }
  __syncwarp();
}

// 1 / x: IEEE division in FP64; in FP32 the hardware's approximate reciprocal (PTX
// rcp.approx.f32, at most one ulp from the correctly rounded value)
template <typename T>
__device__ __forceinline__ T recip(T x);
template <>
__device__ __forceinline__ double recip<double>(double x) {
  return 1.0 / x;
}
template <>
__device__ __forceinline__ float recip<float>(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// eps - U on the diagonal of a 2 x 2 layer: in FP64; in the complex64 sweep from the operands
// rounded to FP32 (within an ulp of the larger of |eps| and |U|; the 1 x 1 sweep reads it
// formed in FP64 and rounded once by prep_kernel)
template <typename T>
__device__ __forceinline__ T eps_minus(double e, double u);
template <>
__device__ __forceinline__ double eps_minus<double>(double e, double u) {
  return e - u;
}
template <>
__device__ __forceinline__ float eps_minus<float>(double e, double u) {
  return (float)e - (float)u;
}

template <typename T>
__device__ __forceinline__ cx<T> ld_c(const unsigned char* p) {
  return *reinterpret_cast<const cx<T>*>(p);
}

}  // namespace

// ------------------------------------------------------------------ b = 1
// the FP64 or FP32 copy of a per-layer array
template <typename T>
__device__ __forceinline__ const T* pick(const double* d, const float* f);
template <>
__device__ __forceinline__ const double* pick<double>(const double* d, const float* f) {
  (void)f;
  return d;
}
template <>
__device__ __forceinline__ const float* pick<float>(const double* d, const float* f) {
  (void)d;
  return f;
}

template <typename T>
__global__ void __launch_bounds__(256) sweep_b1_kernel(SweepArgs a) {
  extern __shared__ double sm_b1[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  T* red = reinterpret_cast<T*>(sm_b1) + wib * (32 * 33);
  T* st = reinterpret_cast<T*>(a.stage + (long long)gw * a.stage_stride);

  for (;;) {
    const int it = next_item(a.counter, lane);
    if (it >= a.n_items) break;
    const WorkItem W = a.items[a.order[it]];
    const DeviceView& D = a.devs[W.dev];
    const ChainView& C = D.ch[W.chain];
    const int L = D.L;
    const bool act = lane < W.ne;
    const int k = W.e0 + (act ? lane : 0);
    const double g = 2.0 * C.g_b;
    double* part = a.partial + W.part;

    cd eps;
    double wS = 0.0, wD = 0.0;     // real axis: g w f / (2 pi)
    cd kap = mk(0.0, 0.0);         // contour: (g / pi) c_k
    if (W.kind == 0) {
      eps = mk(D.E[k], D.eta);
      if (act) {
        wS = g * D.w[k] * D.fS[k] * (0.5 / 3.14159265358979323846);
        wD = g * D.w[k] * D.fD[k] * (0.5 / 3.14159265358979323846);
      }
    } else {
      eps = D.z[k];
      if (act) kap = scale(D.c[k], g / 3.14159265358979323846);
    }
    // contact self-energies in FP64
    const cd sS = mode_sigma(C.lead[0], 0, eps);
    const cd sD = mode_sigma(C.lead[1], 0, eps);
    const double gamS = -2.0 * sS.im, gamD = -2.0 * sD.im;

    const cx<T> e = mk((T)eps.re, (T)eps.im);
    const cx<T> SS = mk((T)sS.re, (T)sS.im), SD = mk((T)sD.re, (T)sD.im);
    const double* U = D.U;
    const cd* Hd = C.Hdiag;
    const T* hsq = pick<T>(C.hsq, C.hsq_f);
    const T* hu = pick<T>(C.hu, C.hu_f);   // Re H_ll + U_l of this launch (may be null)

    // ---------------- forward sweep
    cx<T> gl = mk(T(0), T(0));
    T rl = T(0);              // |gL_l|^2
    T ql = (T)(wS * gamS);    // (g w fS / 2pi) Gamma_S |Q_l|^2
    const bool want_r = a.resid != nullptr && W.kind == 0;
    T qu = T(1);              // |Q_l|^2 (residual only)
    T rmaxg = T(0);           // largest |gL_l|^2 (growth diagnostic)
    const int nf = (W.kind == 0) ? (want_r ? 5 : 4) : 2;
    for (int l = 0; l < L; ++l) {
      cx<T> x;
      if (hu) {
        x.re = e.re - hu[l];
        x.im = C.diag_real ? e.im : (T)(eps.im - Hd[l].im);
      } else {
        const cd h = Hd[l];
        x = mk((T)(eps.re - h.re - U[l]), (T)(eps.im - h.im));
      }
      if (l == 0) x = x - SS;
      if (l == L - 1) x = x - SD;
      T p = T(0);               // |h_{l-1,l}|^2 |gL_{l-1}|^2
      if (l > 0) {
        const T hs = hsq[l - 1];
        x.re = fma(-hs, gl.re, x.re);
        x.im = fma(-hs, gl.im, x.im);
        p = hs * rl;
        if (W.kind == 0) ql = p * ql;
        if (want_r) qu = p * qu;
      }
      const T r = recip<T>(fma(x.re, x.re, x.im * x.im));
      gl = mk(x.re * r, -x.im * r);
      rl = r;
      if (a.growth) rmaxg = r > rmaxg ? r : rmaxg;
      T* s = st + (long long)l * nf * 32;
      s[lane] = gl.re;
      s[32 + lane] = gl.im;
      if (W.kind == 0) {
        s[64 + lane] = p;       // used by the backward step at layer l - 1
        s[96 + lane] = ql;
        if (want_r) s[128 + lane] = qu;
      }
    }

    // ---------------- backward sweep
    cx<T> G = gl;             // G_{L-1,L-1}
    T c = abs2(G);            // |G_{l,L-1}|^2
    // sum-rule residual of the lane: max(0, max_l (A_S + A_D + 2 Im G)_ll) / max_l |2 Im G_ll|
    // (in the element type, as the per-layer contributions)
    T rnum = T(0), rden = T(0);
    const T wDg = (T)(wD * gamD);
    T pn = T(0);              // |h_{l,l+1}|^2 |gL_l|^2, read one layer ahead
    for (int l = L - 1; l >= 0; --l) {
      const T* s = st + (long long)l * nf * 32;
      if (l < L - 1) {
        const cx<T> gll = mk(s[lane], s[32 + lane]);
        const T hs = hsq[l];
        cx<T> t = scale(gll * G, hs);        // |h|^2 gL G_{l+1}
        G = cmac(gll, gll, t);               // gL + gL (|h|^2 gL G_{l+1})
        if (W.kind == 0) c = pn * c;         // |G_{l,L-1}|^2
      }
      if (W.kind == 0) pn = s[64 + lane];
      T v;
      if (W.kind == 0) {
        const T q = s[96 + lane];
        v = fma(wDg, c, q * abs2(G));
        if (want_r) {
          // A_S + A_D + 2 Im G <= 0 up to rounding (equality up to 2 eta |G|^2 terms)
          const T as = (T)gamS * s[128 + lane] * abs2(G);
          const T gim = G.im;
          rnum = fmax(rnum, as + (T)gamD * c + T(2) * gim);
          rden = fmax(rden, fabs(T(2) * gim));
        }
      } else {
        v = (T)kap.re * G.im + (T)kap.im * G.re;
      }
      if (a.ring_cap && l == a.cap_ring && W.kind == 0 && act) a.ring_cap[W.tout + lane] = (double)v;
      red[(l & 31) * 33 + lane] = v;
      if ((l & 31) == 0) {
        const int cnt = min(32, L - l);
        flush_rings(red, lane, cnt, part + l);
      }
    }
    if (W.kind == 0 && act) {
      a.Tpart[W.tout + lane] = gamS * gamD * (double)c;
      if (want_r) a.resid[W.tout + lane] = (double)rnum / fmax((double)rden, 1e-300);
      if (a.growth) a.growth[W.tout + lane] = sqrt((double)rmaxg);
    }
  }
}

// ------------------------------------------------------------------ b = 2
// 2 x 2 layers with the leads on one site each (unit cells of two mode-space rings).
template <typename T>
struct m2 {
  cx<T> a[2][2];
};

template <typename T>
__device__ __forceinline__ m2<T> mul2(const m2<T>& A, const m2<T>& B) {
  m2<T> C;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) C.a[i][j] = cmac(A.a[i][0] * B.a[0][j], A.a[i][1], B.a[1][j]);
  return C;
}
template <typename T>
__device__ __forceinline__ m2<T> inv2(const m2<T>& A) {
  cx<T> det = A.a[0][0] * A.a[1][1] - A.a[0][1] * A.a[1][0];
  const T s = recip<T>(fma(det.re, det.re, det.im * det.im));
  const cx<T> id = mk(det.re * s, -det.im * s);
  m2<T> B;
  B.a[0][0] = A.a[1][1] * id;
  B.a[1][1] = A.a[0][0] * id;
  B.a[0][1] = mk(T(0), T(0)) - A.a[0][1] * id;
  B.a[1][0] = mk(T(0), T(0)) - A.a[1][0] * id;
  return B;
}
template <typename T>
__device__ __forceinline__ m2<T> load2(const cd* p, bool dagger) {
  m2<T> M;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      cd v = dagger ? conjg(p[j * 2 + i]) : p[i * 2 + j];
      M.a[i][j] = mk((T)v.re, (T)v.im);
    }
  return M;
}

template <typename T>
__global__ void __launch_bounds__(256) sweep_b2_kernel(SweepArgs a) {
  extern __shared__ double sm_b2[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  T* red = reinterpret_cast<T*>(sm_b2) + wib * (32 * 33);
  T* st = reinterpret_cast<T*>(a.stage + (long long)gw * a.stage_stride);
  constexpr int NF = 12;  // gL (8 reals) + R (4 reals)

  for (;;) {
    const int it = next_item(a.counter, lane);
    if (it >= a.n_items) break;
    const WorkItem W = a.items[a.order[it]];
    const DeviceView& D = a.devs[W.dev];
    const ChainView& C = D.ch[W.chain];
    const int L = D.L;
    const bool act = lane < W.ne;
    const int k = W.e0 + (act ? lane : 0);
    const double g = 2.0 * C.g_b;
    double* part = a.partial + W.part;

    cd eps;
    double wS = 0.0, wD = 0.0;
    cd kap = mk(0.0, 0.0);
    if (W.kind == 0) {
      eps = mk(D.E[k], D.eta);
      if (act) {
        wS = g * D.w[k] * D.fS[k] * (0.5 / 3.14159265358979323846);
        wD = g * D.w[k] * D.fD[k] * (0.5 / 3.14159265358979323846);
      }
    } else {
      eps = D.z[k];
      if (act) kap = scale(D.c[k], g / 3.14159265358979323846);
    }
    const cd sS = mode_sigma(C.lead[0], 0, eps);
    const cd sD = mode_sigma(C.lead[1], 0, eps);
    const int siteS = C.lead[0].sites[0], siteD = C.lead[1].sites[0];
    const int rpb = D.rpb;
    const double gamS = -2.0 * sS.im, gamD = -2.0 * sD.im;
    const T lS = (T)sqrt(fmax(gamS, 0.0)), lD = (T)sqrt(fmax(gamD, 0.0));
    const double* U = D.U;

    // forward: gL_l and R_l = Q_l L_S (a 2-vector, L_S = sqrt(Gamma_S) e_siteS)
    m2<T> gl;
    cx<T> R[2];
    T gmax2 = T(0);   // largest |gL_l entry|^2 (growth diagnostic)
    for (int l = 0; l < L; ++l) {
      m2<T> A = load2<T>(C.Hdiag + (long long)l * 4, false);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) A.a[i][j] = mk(T(0), T(0)) - A.a[i][j];
      // ring of site a: 2l + a for unit cells (rpb = 2), l for a two-site ring (rpb = 1)
      const int ring0 = l * rpb, ring1 = l * rpb + (rpb - 1);
      A.a[0][0] = A.a[0][0] + mk(eps_minus<T>(eps.re, U[ring0]), (T)eps.im);
      A.a[1][1] = A.a[1][1] + mk(eps_minus<T>(eps.re, U[ring1]), (T)eps.im);
      if (l == 0) A.a[siteS][siteS] = A.a[siteS][siteS] - mk((T)sS.re, (T)sS.im);
      if (l == L - 1) A.a[siteD][siteD] = A.a[siteD][siteD] - mk((T)sD.re, (T)sD.im);
      cx<T> Rn[2];
      if (l > 0) {
        const cd* hu = C.Hup + (long long)(l - 1) * 4;
        m2<T> X = mul2(load2<T>(hu, true), gl);      // H_{l,l-1} gL_{l-1}
        m2<T> Y = mul2(X, load2<T>(hu, false));      // ... H_{l-1,l}
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) A.a[i][j] = A.a[i][j] - Y.a[i][j];
        if (W.kind == 0) {
#pragma unroll
          for (int i = 0; i < 2; ++i) Rn[i] = cmac(X.a[i][0] * R[0], X.a[i][1], R[1]);
        }
      } else {
        Rn[0] = mk(T(0), T(0));
        Rn[1] = mk(T(0), T(0));
        Rn[siteS] = mk(lS, T(0));
      }
      gl = inv2(A);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) gmax2 = abs2(gl.a[i][j]) > gmax2 ? abs2(gl.a[i][j]) : gmax2;
      R[0] = Rn[0];
      R[1] = Rn[1];
      T* s = st + (long long)l * NF * 32;
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          s[((i * 2 + j) * 2) * 32 + lane] = gl.a[i][j].re;
          s[((i * 2 + j) * 2 + 1) * 32 + lane] = gl.a[i][j].im;
        }
      if (W.kind == 0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          s[(8 + 2 * i) * 32 + lane] = R[i].re;
          s[(9 + 2 * i) * 32 + lane] = R[i].im;
        }
      }
    }

    // backward: G_ll, K_l = G_{l,L-1} L_D, P_l = G_ll R_l
    const bool want_r = a.resid != nullptr && W.kind == 0;
    T rnum = T(0), rden = T(0);   // sum-rule residual, as in the 1 x 1 sweep
    m2<T> G = gl;
    cx<T> K[2];
    K[0] = scale(G.a[0][siteD], lD);
    K[1] = scale(G.a[1][siteD], lD);
    for (int l = L - 1; l >= 0; --l) {
      const T* s = st + (long long)l * NF * 32;
      if (l < L - 1) {
        m2<T> gll;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j)
            gll.a[i][j] = mk(s[((i * 2 + j) * 2) * 32 + lane], s[((i * 2 + j) * 2 + 1) * 32 + lane]);
        const cd* hu = C.Hup + (long long)l * 4;
        m2<T> Z = mul2(gll, load2<T>(hu, false));     // gL_l H_{l,l+1}
        m2<T> Wm = mul2(Z, G);
        m2<T> Y = mul2(load2<T>(hu, true), gll);      // H_{l+1,l} gL_l
        m2<T> WY = mul2(Wm, Y);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) G.a[i][j] = gll.a[i][j] + WY.a[i][j];
        if (W.kind == 0) {
          cx<T> Kn[2];
#pragma unroll
          for (int i = 0; i < 2; ++i) Kn[i] = cmac(Z.a[i][0] * K[0], Z.a[i][1], K[1]);
          K[0] = Kn[0];
          K[1] = Kn[1];
        }
      }
      T v0, v1;   // in the element type, as the 1 x 1 sweep
      if (W.kind == 0) {
        cx<T> Rl[2];
        Rl[0] = mk(s[8 * 32 + lane], s[9 * 32 + lane]);
        Rl[1] = mk(s[10 * 32 + lane], s[11 * 32 + lane]);
        cx<T> P0 = cmac(G.a[0][0] * Rl[0], G.a[0][1], Rl[1]);
        cx<T> P1 = cmac(G.a[1][0] * Rl[0], G.a[1][1], Rl[1]);
        v0 = (T)wS * abs2(P0) + (T)wD * abs2(K[0]);
        v1 = (T)wS * abs2(P1) + (T)wD * abs2(K[1]);
        if (want_r) {
          const T g0 = G.a[0][0].im, g1 = G.a[1][1].im;
          rnum = fmax(rnum, abs2(P0) + abs2(K[0]) + T(2) * g0);
          rnum = fmax(rnum, abs2(P1) + abs2(K[1]) + T(2) * g1);
          rden = fmax(rden, fmax(fabs(T(2) * g0), fabs(T(2) * g1)));
        }
      } else {
        v0 = (T)kap.re * G.a[0][0].im + (T)kap.im * G.a[0][0].re;
        v1 = (T)kap.re * G.a[1][1].im + (T)kap.im * G.a[1][1].re;
      }
      // rings of the layer -> transpose slots ring & 31
      const int r0 = l * rpb;
      if (a.ring_cap && W.kind == 0 && act && a.cap_ring >= r0 && a.cap_ring < r0 + rpb)
        a.ring_cap[W.tout + lane] = (double)(rpb == 2 ? (a.cap_ring == r0 ? v0 : v1) : v0 + v1);
      if (rpb == 2) {
        red[(r0 & 31) * 33 + lane] = v0;
        red[((r0 + 1) & 31) * 33 + lane] = v1;
      } else {
        red[(r0 & 31) * 33 + lane] = v0 + v1;
      }
      if ((r0 & 31) == 0) {
        const int cnt = min(32, D.n_rings - r0);
        flush_rings(red, lane, cnt, part + r0);
      }
    }
    if (W.kind == 0 && act) {
      // T = Tr[Gamma_S G_{0,L-1} Gamma_D G_{0,L-1}^dag] = Gamma_S |K_0[siteS]|^2
      a.Tpart[W.tout + lane] = gamS * (double)abs2(K[siteS]);
      if (want_r) a.resid[W.tout + lane] = (double)rnum / fmax((double)rden, 1e-300);
      if (a.growth) a.growth[W.tout + lane] = sqrt((double)gmax2);
    }
  }
}

static int launch_common(void (*kern)(SweepArgs), const SweepArgs& a, int grid, int block, size_t esize,
                         cudaStream_t s) {
  // the dynamic shared memory limit was raised by sweep_chain_occupancy when planning; one
  // 32 x 33 transpose buffer of the element type per warp
  const size_t smem = (size_t)(block / 32) * 32 * 33 * esize;
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sweep_b1_f64(const SweepArgs& a, int grid, int block, cudaStream_t s) {
  return launch_common(sweep_b1_kernel<double>, a, grid, block, sizeof(double), s);
}
int launch_sweep_b1_f32(const SweepArgs& a, int grid, int block, cudaStream_t s) {
  return launch_common(sweep_b1_kernel<float>, a, grid, block, sizeof(float), s);
}
int launch_sweep_b2_f64(const SweepArgs& a, int grid, int block, cudaStream_t s) {
  return launch_common(sweep_b2_kernel<double>, a, grid, block, sizeof(double), s);
}
int launch_sweep_b2_f32(const SweepArgs& a, int grid, int block, cudaStream_t s) {
  return launch_common(sweep_b2_kernel<float>, a, grid, block, sizeof(float), s);
}

}  // namespace negf

namespace negf {
int sweep_chain_occupancy(int cls, int threads, size_t smem) {
  return sweep_chain_occupancy_t(false, cls, threads, smem);
}
int sweep_chain_occupancy_t(bool fp32, int cls, int threads, size_t smem) {
  void (*k)(SweepArgs) = fp32 ? (cls == 0 ? sweep_b1_kernel<float> : sweep_b2_kernel<float>)
                              : (cls == 0 ? sweep_b1_kernel<double> : sweep_b2_kernel<double>);
  // the limit covers the widest CTA (8 warps), so a launch of any tuned width fits under it
  const size_t widest = (size_t)8 * 32 * 33 * sizeof(double);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max(smem, widest));
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem) != cudaSuccess || per < 1) {
    cudaGetLastError();
    per = 1;
  }
  return per;
}
}  // namespace negf
