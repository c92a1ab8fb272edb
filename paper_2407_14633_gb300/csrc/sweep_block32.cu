// Complex64 sweep of wide ring blocks (the bulk of the mixed-precision path), register-tiled.
//
// Same method as the two-sided complex64 variant of sweep_block.cu (left-connected forward
// sweep, G_ll = (alpha_l - x_l - y_l)^{-1} and gR_l = (alpha_l - x_l)^{-1} backward, lead
// columns propagated as factors of Gamma; Alg. 1 / Alg. 2 as read), organised for the FP32
// pipe rather than the FP64 one:
//   - every b x b (and b x m) product gives each thread a 3 x 4 tile of outputs held in
//     registers, so one k step loads 3 + 4 operands from shared memory for 12 complex
//     multiply-adds (48 FFMA);
//   - the block inverses are Gauss-Jordan eliminations with implicit partial pivoting: no
//     row swaps; each pivot step publishes the pivot row and the column multipliers, every
//     thread updates its own 3 x 4 tile, and one permuted copy at the end puts the inverse in
//     place.  The pivot search packs |v|^2 and the row index into one 32-bit key for a single
//     warp max-reduction.  The two inverses of a backward step run interleaved, sharing their
//     barriers;
//   - y_l, gL_l and R_l are staged to global memory in tile order (each thread writes and
//     later reads its own six 16-byte chunks); the backward sweep reads y_l back rather than
//     forming it again, which saves a matrix buffer (10 one-warp CTAs per SM) and two sparse
//     products per layer;
//   - a tube whose layers all hold the same blocks reads layer 0's H_ll and couplings for
//     every layer (an L1-resident copy);
//   - the per-layer ring sums run in FP32 (a warp-wide FP64 operation costs the FP64 pipe of
//     this part about as much as 60 FP32 ones); FP64 remains for the lead roots, eps - U and
//     T(E), once per lane or layer.
// Tile classes (CTA width): 1 warp for b <= 18 (6 x 5 tiles), 2 warps for b <= 27 (9 x 7), 4
// warps for b <= 36 (12 x 9), at 10, 4 and 3 resident CTAs per SM; wider blocks keep the
// shared-memory kernel.  Matrices are kept
// with exact zero padding outside b x b, so padded rows and columns never feed a result.
// Every output element, and every row, ring and T(E) sum, is evaluated in an order that does
// not depend on the tile class, so all CTA widths give the same bits.
#include "blk32.cuh"
#include "lead.cuh"
#include "sweep_block_item.cuh"

namespace negf {

namespace {

template <int NW>
struct T32 {
  static constexpr int TR = 3, TC = 4;
  static constexpr int NCT = NW == 1 ? 5 : (NW == 2 ? 7 : 9);    // column tiles
  static constexpr int NRT = NW == 1 ? 6 : (NW == 2 ? 9 : 12);   // row tiles
  static constexpr int PR = TR * NRT, PC = TC * NCT;            // padded rows / columns
  // row stride (elements): 6 LD (mod 32 words) spaces the first rows of a warp's tile rows
  // over distinct banks (LD = 22, 38: 4 words apart; LD = 42: 4 words apart in reverse); it
  // also holds the column swizzle pcol (2 spare elements per 16 columns)
  static constexpr int LD = NW == 1 ? 22 : (NW == 2 ? 38 : 42);
  static constexpr int BMAX = PR < PC ? PR : PC;                 // 18, 27, 36
  static constexpr int NT = 32 * NW;
  static constexpr int NTA = NRT * NCT;                          // threads that own a tile
  static constexpr int MAT = PR * LD;                            // elements per matrix buffer
  static constexpr int NBUF = 6;
};

constexpr int B32_RED = 8;

template <int NW>
__device__ __forceinline__ void bar() {
  if (NW == 1)
    __syncwarp();
  else
    __syncthreads();
}

// Physical column of logical column c in a shared-memory matrix: two spare elements after
// every 16 columns, so that the 5th to 8th column tiles of a row (32 bytes each) fall on other
// banks than the 1st to 4th in a 128-bit access.
__device__ __forceinline__ int pcol(int c) { return c + ((c >> 4) << 1); }

// 1 / a through the approximate hardware reciprocal of |a|^2 (PTX rcp.approx.f32: at most
// one ulp from 1 / |a|^2), for the pivots
__device__ __forceinline__ cf crecip32(cf a) {
  float s;
  asm("rcp.approx.f32 %0, %1;" : "=f"(s) : "f"(fmaf(a.re, a.re, a.im * a.im)));
  return mk(a.re * s, -a.im * s);
}

struct Tile {
  cf v[3][4];
};

__device__ __forceinline__ void tzero(Tile& t) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) t.v[i][j] = mk(0.0f, 0.0f);
}

// C tile = A (rows r0.., smem, stride LD) * B (cols c0.., smem, stride LD), k < K, one
// accumulator per output in k order
template <int LD>
__device__ __forceinline__ void tgemm(Tile& t, const cf* A, const cf* B, int K, int r0, int c0) {
  tzero(t);
  const cf* a0 = A + r0 * LD;
  const cf* bb = B + pcol(c0);
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    const int kp = pcol(k);
    const cf x0 = a0[kp], x1 = a0[LD + kp], x2 = a0[2 * LD + kp];
    const float4 p = *reinterpret_cast<const float4*>(bb + k * LD);
    const float4 q = *reinterpret_cast<const float4*>(bb + k * LD + 2);
    const cf y[4] = {mk(p.x, p.y), mk(p.z, p.w), mk(q.x, q.y), mk(q.z, q.w)};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      t.v[0][j] = cmac(t.v[0][j], x0, y[j]);
      t.v[1][j] = cmac(t.v[1][j], x1, y[j]);
      t.v[2][j] = cmac(t.v[2][j], x2, y[j]);
    }
  }
}

template <int LD>
__device__ __forceinline__ void tstore(cf* C, const Tile& t, int r0, int c0) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float4* d = reinterpret_cast<float4*>(C + (r0 + i) * LD + pcol(c0));
    d[0] = make_float4(t.v[i][0].re, t.v[i][0].im, t.v[i][1].re, t.v[i][1].im);
    d[1] = make_float4(t.v[i][2].re, t.v[i][2].im, t.v[i][3].re, t.v[i][3].im);
  }
}

// tile <-> global staging: chunk q (q = 0..5, two elements) of thread t at 16-byte slot
// q NTA + t, so that each chunk of a warp is one contiguous, coalesced access
template <int NTA>
__device__ __forceinline__ void gstore(float4* g, int t, const Tile& x) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    g[(2 * i) * NTA + t] = make_float4(x.v[i][0].re, x.v[i][0].im, x.v[i][1].re, x.v[i][1].im);
    g[(2 * i + 1) * NTA + t] = make_float4(x.v[i][2].re, x.v[i][2].im, x.v[i][3].re, x.v[i][3].im);
  }
}
template <int NTA>
__device__ __forceinline__ void gload(Tile& x, const float4* g, int t) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float4 p = g[(2 * i) * NTA + t], q = g[(2 * i + 1) * NTA + t];
    x.v[i][0] = mk(p.x, p.y);
    x.v[i][1] = mk(p.z, p.w);
    x.v[i][2] = mk(q.x, q.y);
    x.v[i][3] = mk(q.z, q.w);
  }
}

// L2 prefetch of a staged tile (bytes from g) ahead of its gload: one line per thread
template <int NT>
__device__ __forceinline__ void gprefetch(const float4* g, long long bytes, int tid) {
  const char* p = reinterpret_cast<const char*>(g);
  const int nl = (int)((bytes + 127) / 128) + 1;   // lines a range of this length can touch
  for (int o = tid; o < nl; o += NT) {
    const long long off = (long long)o * 128 < bytes - 16 ? (long long)o * 128 : bytes - 16;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
  }
}

// out[r][c] += sum_e s(val[r][e]) M[idx[r][e]][c]  (rows r < b; s = conj when CJ).  Every
// row holds kmax slots (unused ones index 0 with value 0); the count only predicates the
// multiply-adds.  Up to KS slots per row (the (n,0) tubes have 2) run unrolled, every slot
// load of the three rows issued before the first operand load; wider couplings loop.
constexpr int KS = 2;
template <int LD, bool CJ>
__device__ __forceinline__ void trow(Tile& t, const int* cnt, const int* idx, const cf* val, int kmax, const cf* M,
                                     int b, int r0, int c0) {
  if (kmax <= KS) {
    int n[3], q[3][KS];
    cf v[3][KS];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int r = r0 + i;
      const int rr = r < b ? r : 0;
      n[i] = r < b ? cnt[rr] : 0;
#pragma unroll
      for (int e = 0; e < KS; ++e) {
        const bool in = e < kmax;
        v[i][e] = in ? val[rr * kmax + e] : mk(0.0f, 0.0f);
        q[i][e] = in ? idx[rr * kmax + e] : 0;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int e = 0; e < KS; ++e)
        if (e < n[i]) {
          const cf* m = M + q[i][e] * LD + pcol(c0);
          const float4 p = *reinterpret_cast<const float4*>(m);
          const float4 u = *reinterpret_cast<const float4*>(m + 2);
          const cf y[4] = {mk(p.x, p.y), mk(p.z, p.w), mk(u.x, u.y), mk(u.z, u.w)};
#pragma unroll
          for (int j = 0; j < 4; ++j)
            t.v[i][j] = CJ ? cmac_cj(t.v[i][j], v[i][e], y[j]) : cmac(t.v[i][j], v[i][e], y[j]);
        }
    return;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int r = r0 + i;
    const int rr = r < b ? r : 0;
    const int n = r < b ? cnt[rr] : 0;
    for (int e = 0; e < kmax; ++e) {
      const cf v = val[rr * kmax + e];
      const int q = idx[rr * kmax + e];
      if (e < n) {
        const cf* m = M + q * LD + pcol(c0);
        const float4 p = *reinterpret_cast<const float4*>(m);
        const float4 u = *reinterpret_cast<const float4*>(m + 2);
        const cf y[4] = {mk(p.x, p.y), mk(p.z, p.w), mk(u.x, u.y), mk(u.z, u.w)};
#pragma unroll
        for (int j = 0; j < 4; ++j) t.v[i][j] = CJ ? cmac_cj(t.v[i][j], v, y[j]) : cmac(t.v[i][j], v, y[j]);
      }
    }
  }
}

// out[r][c] += sum_e M[r][idx[c][e]] s(val[c][e])  (columns c < b; s = conj when CJ), slots as
// in trow
template <int LD, bool CJ>
__device__ __forceinline__ void tcol(Tile& t, const cf* M, const int* cnt, const int* idx, const cf* val, int kmax,
                                     int b, int r0, int c0) {
  if (kmax <= KS) {
    int n[4], q[4][KS];
    cf v[4][KS];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + j;
      const int cc = c < b ? c : 0;
      n[j] = c < b ? cnt[cc] : 0;
#pragma unroll
      for (int e = 0; e < KS; ++e) {
        const bool in = e < kmax;
        v[j][e] = in ? val[cc * kmax + e] : mk(0.0f, 0.0f);
        q[j][e] = pcol(in ? idx[cc * kmax + e] : 0);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < KS; ++e)
        if (e < n[j]) {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const cf x = M[(r0 + i) * LD + q[j][e]];
            t.v[i][j] = CJ ? cmac_cj(t.v[i][j], v[j][e], x) : cmac(t.v[i][j], x, v[j][e]);
          }
        }
    return;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + j;
    const int cc = c < b ? c : 0;
    const int n = c < b ? cnt[cc] : 0;
    for (int e = 0; e < kmax; ++e) {
      const cf v = val[cc * kmax + e];
      const int q = pcol(idx[cc * kmax + e]);
      if (e < n) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const cf x = M[(r0 + i) * LD + q];
          t.v[i][j] = CJ ? cmac_cj(t.v[i][j], v, x) : cmac(t.v[i][j], x, v);
        }
      }
    }
  }
}

// Per-item pointers and sizes, copied once into shared memory so that the layer loops read
// them there instead of chasing the device and chain views in global memory after every
// staging store.
struct ItemPtrs {
  const cf* hd;        // H_ll (complex64), layer-major
  const double* U;     // ring potentials
  const cd* gS;        // general leads: this energy's Sigma blocks (null for circulant leads)
  const cd* gD;
  const int* cs_cnt;
  const int* cs_idx;
  const cf* cs_val;
  const int* rs_cnt;
  const int* rs_idx;
  const cf* rs_val;
  int kmax, mS, mD;
  int hd_step, cp_step;   // layer steps of hd and of the sparse forms (0: every layer the same)
  int pad;
  float wS, wD;           // the lane's weights of A_S and A_D in the ring sums (real axis)
  cf kap;                 // and of G (contour)
};

// In place: t := alpha_l - t on r, c < b (0 elsewhere), alpha_l = eps I - H_ll - U_ring -
// Sigma_S (l = 0) - Sigma_D (l = L - 1); eps - U formed in FP64 and rounded once; a circulant
// lead's Sigma from its first row (FP64, shared memory), a general lead's from the plan's
// per-energy blocks.
__device__ __forceinline__ void talpha(Tile& t, int l, int L, int b, int rpb, int spr, cd eps, const ItemPtrs& P,
                                       const cd* sigS, const cd* sigD, const int* sinvS, const int* sinvD, int r0,
                                       int c0) {
  const cf* hd = P.hd + (long long)l * P.hd_step;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int r = r0 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + j;
      if (r >= b || c >= b) {
        t.v[i][j] = mk(0.0f, 0.0f);
        continue;
      }
      const cf h = hd[r * b + c];
      cf a = mk(-h.re - t.v[i][j].re, -h.im - t.v[i][j].im);
      if (r == c) a = a + mk((float)(eps.re - P.U[l * rpb + (rpb == 2 && r >= spr ? 1 : 0)]), (float)eps.im);
      if (l == 0) {
        const int s = sinvS[r], u = sinvS[c];
        if (s >= 0 && u >= 0) {
          const int m = P.mS;
          const cd v = P.gS ? P.gS[s * m + u] : sigS[((s - u) % m + m) % m];
          a = a - mk((float)v.re, (float)v.im);
        }
      }
      if (l == L - 1) {
        const int s = sinvD[r], u = sinvD[c];
        if (s >= 0 && u >= 0) {
          const int m = P.mD;
          const cd v = P.gD ? P.gD[s * m + u] : sigD[((s - u) % m + m) % m];
          a = a - mk((float)v.re, (float)v.im);
        }
      }
      t.v[i][j] = a;
    }
  }
}

// Scratch of the inverses: per matrix and step parity the pivot column and the pivot row,
// and the pivot order.  (Each row's deferred scale, 1 / its pivot, goes to a matrix buffer that
// is free while the inverse runs.)
template <int NW>
struct InvBuf {
  cf colb[2][2][T32<NW>::PR];
  cf rowb[2][2][T32<NW>::LD];
  unsigned char piv[2][64];
  unsigned char qinv[2][64];
};

// One Gauss-Jordan step on a register tile (column k is column jj of tile column kt), with
// the pivot row's scaling deferred: every row other than p takes A[i][j] - (A[i][k] / A[p][k])
// A[p][j] (column k: -A[i][k] / A[p][k], from a cleared column and a unit pivot-row entry);
// row p keeps its values and gets 1 in column k, i.e. it holds A[p][k] times its scaled row,
// which every later step treats linearly; the inverse's final store multiplies it by
// 1 / A[p][k].
template <int LD>
__device__ __forceinline__ void gj_update(Tile& t, const cf* colb, const cf* rowb, cf ip, int p, int jj, bool own,
                                          int r0, int c0) {
  cf f[3], rs[4];
#pragma unroll
  for (int i = 0; i < 3; ++i) f[i] = (r0 + i == p) ? mk(0.0f, 0.0f) : colb[r0 + i] * ip;
  const float4 u = *reinterpret_cast<const float4*>(rowb + pcol(c0));
  const float4 w = *reinterpret_cast<const float4*>(rowb + pcol(c0) + 2);
  rs[0] = mk(u.x, u.y);
  rs[1] = mk(u.z, u.w);
  rs[2] = mk(w.x, w.y);
  rs[3] = mk(w.z, w.w);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (own && j == jj) {
      rs[j] = mk(1.0f, 0.0f);
#pragma unroll
      for (int i = 0; i < 3; ++i) t.v[i][j] = mk(r0 + i == p ? 1.0f : 0.0f, 0.0f);
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) t.v[i][j] = cmsub(t.v[i][j], f[i], rs[j]);
}

// Pivot of column k (values in colb, rows < b): the unused row of largest |v| (magnitudes
// within 2^-17 of each other go to the lowest row), found by every warp from the same values.
template <int BMAX>
__device__ __forceinline__ int gj_pivot(const cf* colb, int b, unsigned long long& used, int lane, cf& vp) {
  unsigned key = 0u;
  if (lane < b && !((used >> lane) & 1ull)) {
    const cf v = colb[lane];
    key = (__float_as_uint(fmaf(v.re, v.re, v.im * v.im)) & ~63u) | (unsigned)(63 - lane);
  }
  if (BMAX > 32 && lane + 32 < b && !((used >> (lane + 32)) & 1ull)) {
    const cf v = colb[lane + 32];
    key = max(key, (__float_as_uint(fmaf(v.re, v.re, v.im * v.im)) & ~63u) | (unsigned)(31 - lane));
  }
  key = __reduce_max_sync(0xffffffffu, key);
  const int p = 63 - (int)(key & 63u);
  used |= 1ull << p;
  vp = colb[p];
  return p;
}

// Gauss-Jordan inverses of NM (1 or 2) b x b matrices held as register tiles (t0, t1; exact
// zeros outside b x b), implicit partial pivoting.  Step k: the owners of column k publish it;
// every warp finds the pivot p (the unused row of largest |A[p][k]|); the owners of row p
// publish it; every thread then updates its tile (gj_update: row p stays, scaled by A[p][k]
// until the end, with 1 in column k; every other row takes A[i][j] - A[i][k] A[p][j] / A[p][k],
// column k -A[i][k] / A[p][k]).  After b steps physical (i, j) holds inv[q(i)][piv(j)] times
// the pivot of row i, q the step of row i; D0, D1 receive the inverses, rows rescaled, in
// place of their rows and columns (zeros outside b x b).  Pivot
// columns and rows alternate between two buffers, so a step's writes never meet a slower
// warp's reads of the step before.  vs (2 BMAX elements) is scratch for the rows' scales; it
// must not be read by any thread between the call and the next full store into it.  The caller
// synchronises before reading D0, D1.
template <int NW, int NM>
__device__ __forceinline__ void tinv(Tile& t0, Tile& t1, cf* D0, cf* D1, int b, InvBuf<NW>& W, cf* vs, int tid,
                                     bool act, int tc, int r0, int c0) {
  using C = T32<NW>;
  constexpr int LD = C::LD;
  const int lane = tid & 31;
  unsigned long long used0 = 0ull, used1 = 0ull;
  for (int kt = 0; 4 * kt < b; ++kt) {
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int k = 4 * kt + jj;
      if (k < b) {
        const int h = k & 1;
        const bool own = act && tc == kt;
        if (own) {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            W.colb[0][h][r0 + i] = t0.v[i][jj];
            if (NM > 1) W.colb[1][h][r0 + i] = t1.v[i][jj];
          }
        }
        bar<NW>();
        cf v0, v1 = mk(0.0f, 0.0f);
        const int p0 = gj_pivot<C::BMAX>(W.colb[0][h], b, used0, lane, v0);
        const int p1 = NM > 1 ? gj_pivot<C::BMAX>(W.colb[1][h], b, used1, lane, v1) : 0;
        const cf ip0 = crecip32(v0);
        const cf ip1 = NM > 1 ? crecip32(v1) : mk(0.0f, 0.0f);
        if (act) {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            if (r0 + i == p0) {
              float4* d = reinterpret_cast<float4*>(&W.rowb[0][h][pcol(c0)]);
              d[0] = make_float4(t0.v[i][0].re, t0.v[i][0].im, t0.v[i][1].re, t0.v[i][1].im);
              d[1] = make_float4(t0.v[i][2].re, t0.v[i][2].im, t0.v[i][3].re, t0.v[i][3].im);
            }
            if (NM > 1 && r0 + i == p1) {
              float4* d = reinterpret_cast<float4*>(&W.rowb[1][h][pcol(c0)]);
              d[0] = make_float4(t1.v[i][0].re, t1.v[i][0].im, t1.v[i][1].re, t1.v[i][1].im);
              d[1] = make_float4(t1.v[i][2].re, t1.v[i][2].im, t1.v[i][3].re, t1.v[i][3].im);
            }
          }
        }
        if (tid == 0) {
          W.piv[0][k] = (unsigned char)p0;
          W.qinv[0][p0] = (unsigned char)k;
          vs[p0] = ip0;
          if (NM > 1) {
            W.piv[1][k] = (unsigned char)p1;
            W.qinv[1][p1] = (unsigned char)k;
            vs[T32<NW>::BMAX + p1] = ip1;
          }
        }
        bar<NW>();
        if (act) {
          gj_update<LD>(t0, W.colb[0][h], W.rowb[0][h], ip0, p0, jj, own, r0, c0);
          if (NM > 1) gj_update<LD>(t1, W.colb[1][h], W.rowb[1][h], ip1, p1, jj, own, r0, c0);
        }
      }
    }
  }
  bar<NW>();   // the pivot order and scales of the last step
  // permuted stores: physical (r, c) -> inverse (q(r), piv(c)), row r times its deferred
  // scale; padding stays zero
  if (act) {
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const Tile& t = m == 0 ? t0 : t1;
      cf* D = m == 0 ? D0 : D1;
      int qr[3], pc[4];
      cf sc[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        qr[i] = r0 + i < b ? (int)W.qinv[m][r0 + i] : r0 + i;
        sc[i] = r0 + i < b ? vs[m * T32<NW>::BMAX + r0 + i] : mk(0.0f, 0.0f);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) pc[j] = pcol(c0 + j < b ? (int)W.piv[m][c0 + j] : c0 + j);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          D[qr[i] * LD + pc[j]] = (r0 + i < b && c0 + j < b) ? t.v[i][j] * sc[i] : mk(0.0f, 0.0f);
    }
  }
}

__device__ __forceinline__ float wsumf(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ double wsumd(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <int NW>
__device__ __forceinline__ double cta_maxd(double v, double* red, int tid) {
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

template <int NW>
struct Smem32 {
  cf mat[T32<NW>::NBUF][T32<NW>::MAT];
  InvBuf<NW> inv;
  double sqS[T32<NW>::BMAX], sqD[T32<NW>::BMAX];
  int sinvS[T32<NW>::BMAX], sinvD[T32<NW>::BMAX];
  double red[B32_RED];
  ItemPtrs ip;
};

}  // namespace

// FUSE: re-sweep flagged real-axis lanes in FP64 in the same CTA (mixed precision; the FP64
// compact layout of the block sweep in this CTA's shared memory)
template <int NW, bool FUSE>
__global__ void __launch_bounds__(32 * NW, NW == 1 ? 10 : (NW == 2 ? 4 : 3)) sweep_blk32_kernel(SweepArgs a) {
  using Cf = T32<NW>;
  constexpr int LD = Cf::LD, NT = Cf::NT, NTA = Cf::NTA, MAT = Cf::MAT;
  extern __shared__ __align__(16) unsigned char sm_b32[];
  Smem32<NW>& S = *reinterpret_cast<Smem32<NW>*>(sm_b32);
  __shared__ int s_item;
  const int tid = threadIdx.x;
  const bool act = tid < NTA;
  const int tr = act ? tid / Cf::NCT : 0, tc = act ? tid % Cf::NCT : 0;
  const int r0 = 3 * tr, c0 = 4 * tc;
  unsigned char* stage = a.stage + (long long)blockIdx.x * a.stage_stride;
  constexpr long long TILEB = (long long)NTA * 12 * sizeof(cf);   // one staged matrix

  // zero every buffer once: padding outside b x b stays zero from here on
  for (int o = tid; o < (int)(sizeof(Smem32<NW>) / 4); o += NT) reinterpret_cast<float*>(&S)[o] = 0.0f;
  __syncthreads();

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
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
    const LeadView& LDv = C.lead[1];
    const int mS = LS.m, mD = LDv.m;
    double* part = a.partial + W.part;
    const int kmax = C.kmax;
    const long long lstride = (real ? 3 : 1) * TILEB;
    // staging of layer l: the y_l tile chunks, then (real-axis lanes) the gL_l and R_l tile
    // chunks.  The backward sweep reads y_l back instead of forming it again from gL_{l-1};
    // only the real-axis lanes need gL_l there (for K_l).
    auto yl_of = [&](int l) { return reinterpret_cast<float4*>(stage + (long long)l * lstride); };
    auto gl_of = [&](int l) { return reinterpret_cast<float4*>(stage + (long long)l * lstride) + 6 * NTA; };
    auto rl_of = [&](int l) { return reinterpret_cast<float4*>(stage + (long long)l * lstride) + 12 * NTA; };

    cd eps;
    double wS = 0.0, wD = 0.0;
    cd kap = mk(0.0, 0.0);
    const int eidx = real ? k : D.n_real + k;
    if (real) {
      eps = mk(D.E[k], D.eta);
      wS = g * D.w[k] * D.fS[k] * (0.5 / 3.14159265358979323846);
      wD = g * D.w[k] * D.fD[k] * (0.5 / 3.14159265358979323846);
    } else {
      eps = D.z[k];
      kap = scale(D.c[k], g / 3.14159265358979323846);
    }

    if (tid == 0) {
      ItemPtrs q;
      q.hd = C.Hdiag_f;
      q.U = D.U;
      q.gS = LS.gen ? LS.gsig + (long long)eidx * mS * mS : nullptr;
      q.gD = LDv.gen ? LDv.gsig + (long long)eidx * mD * mD : nullptr;
      q.cs_cnt = C.cs_cnt;
      q.cs_idx = C.cs_idx;
      q.cs_val = C.cs_val_f;
      q.rs_cnt = C.rs_cnt;
      q.rs_idx = C.rs_idx;
      q.rs_val = C.rs_val_f;
      q.kmax = kmax;
      q.mS = mS;
      q.mD = mD;
      q.hd_step = C.hd_step;
      q.cp_step = C.cp_step;
      q.pad = 0;
      q.wS = (float)wS;
      q.wD = (float)wD;
      q.kap = mk((float)kap.re, (float)kap.im);
      S.ip = q;
    }
    // ---- lead self-energies in FP64 (per-mode roots, circulant first rows), site maps
    for (int r = tid; r < b; r += NT) {
      S.sinvS[r] = -1;
      S.sinvD[r] = -1;
    }
    __syncthreads();
    // the circulant leads' Sigma rows (FP64) sit in the staging slot of y_0, which the sweep
    // never stages (y_0 = 0): they are read at the first and last layer only
    cd* const sigS = reinterpret_cast<cd*>(yl_of(0));
    cd* const sigD = sigS + T32<NW>::BMAX;
    for (int s = tid; s < mS; s += NT) S.sinvS[LS.sites[s]] = s;
    for (int s = tid; s < mD; s += NT) S.sinvD[LDv.sites[s]] = s;
    for (int side = 0; side < 2; ++side) {
      const LeadView& Lv = C.lead[side];
      if (Lv.gen) continue;
      cd* row = side ? sigD : sigS;
      double* sq = side ? S.sqD : S.sqS;
      const int m = Lv.m;
      for (int j = tid; j < m; j += NT) {
        const cd sj = mode_sigma(Lv, j, eps);
        row[j] = sj;
        sq[j] = sqrt(fmax(-2.0 * sj.im, 0.0) / m);
      }
      __syncthreads();
      // a thread holds at most two of the m <= b <= 36 < 2 NT entries
      cd keep0 = mk(0.0, 0.0), keep1 = mk(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int d = tid + q * NT;
        if (d >= m) continue;
        cd acc = mk(0.0, 0.0);
        for (int j = 0; j < m; ++j) {
          const int e = (j * d) % m;
          acc = cmac(acc, row[j], mk(Lv.tw[2 * e], Lv.tw[2 * e + 1]));
        }
        if (q == 0)
          keep0 = scale(acc, 1.0 / m);
        else
          keep1 = scale(acc, 1.0 / m);
      }
      __syncthreads();
      if (tid < m) row[tid] = keep0;
      if (tid + NT < m) row[tid + NT] = keep1;
    }
    __syncthreads();

    // buffers: P/G, T1, GL, GR, K, R
    cf* const bG = S.mat[0];
    cf* const bT = S.mat[1];
    cf* const bGL = S.mat[2];
    cf* const bGR = S.mat[3];
    cf* const bK = S.mat[4];
    cf* const bR = S.mat[5];
    float gmax = 0.0f;   // largest |gL_l entry|^2 seen by this thread (growth diagnostic)

    // ---- forward sweep: gL_l into bG (logical), staged with y_l and R_l
    Tile ta, tr_;
    if (real) {
      // R_0 = L_S: rows at the lead sites, zeros elsewhere
      for (int o = tid; o < MAT; o += NT) bR[o] = mk(0.0f, 0.0f);
      __syncthreads();
      const cd* fS = LS.gen ? LS.gfac + (long long)eidx * mS * mS : nullptr;
      for (int o = tid; o < mS * mS; o += NT) {
        const int s = o / mS, j = o - s * mS;
        const int e = (j * s) % mS;
        const cd v = fS ? fS[o] : scale(mk(LS.tw[2 * e], LS.tw[2 * e + 1]), S.sqS[j]);
        bR[LS.sites[s] * LD + pcol(j)] = mk((float)v.re, (float)v.im);
      }
      __syncthreads();
    }
    for (int l = 0; l < L; ++l) {
      if (l > 0) {
        const long long cp = (long long)(l - 1) * S.ip.cp_step;
        const int* ccnt = S.ip.cs_cnt + cp;
        const int* cidx = S.ip.cs_idx + cp * kmax;
        const cf* cval = S.ip.cs_val + cp * kmax;
        if (act) {   // X = H_{l,l-1} gL_{l-1} = Hup_{l-1}^dagger gL_{l-1}
          tzero(ta);
          trow<LD, true>(ta, ccnt, cidx, cval, kmax, bG, b, r0, c0);
          tstore<LD>(bT, ta, r0, c0);
        }
        bar<NW>();
        if (act) {
          tzero(ta);
          tcol<LD, false>(ta, bT, ccnt, cidx, cval, kmax, b, r0, c0);   // y_l = X H_{l-1,l}
          gstore<NTA>(yl_of(l), tid, ta);
          talpha(ta, l, L, b, rpb, spr, eps, S.ip, sigS, sigD, S.sinvS, S.sinvD, r0, c0);
          if (real) tgemm<LD>(tr_, bT, bR, b, r0, c0);                   // R_l = X R_{l-1}
        }
        if (real) {
          bar<NW>();
          if (act) {
            tstore<LD>(bR, tr_, r0, c0);
            gstore<NTA>(rl_of(l), tid, tr_);
          }
        }
      } else {
        if (act) {
          tzero(ta);
          talpha(ta, 0, L, b, rpb, spr, eps, S.ip, sigS, sigD, S.sinvS, S.sinvD, r0, c0);
          if (real) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) tr_.v[i][j] = bR[(r0 + i) * LD + pcol(c0 + j)];
            gstore<NTA>(rl_of(0), tid, tr_);
          }
        }
      }
      tinv<NW, 1>(ta, ta, bG, nullptr, b, S.inv, bT, tid, act, tc, r0, c0);   // gL_l = (alpha_l - y_l)^{-1}
      bar<NW>();
      if (act) {   // stage gL_l (logical tile, real-axis lanes) and track its largest entry
        Tile tg;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            tg.v[i][j] = bG[(r0 + i) * LD + pcol(c0 + j)];
            if (a.growth) gmax = fmaxf(gmax, fmaf(tg.v[i][j].re, tg.v[i][j].re, tg.v[i][j].im * tg.v[i][j].im));
          }
        if (real && l < L - 1) gstore<NTA>(gl_of(l), tid, tg);
      }
    }
    if (a.lane_stats && tid == 0) atomicAdd(a.lane_stats + (real ? 1 : 3), 1ull);

    // ---- backward sweep.  bG = gL_{L-1} = G_{L-1,L-1}; K_{L-1} = G L_D; gR_{L-1} =
    //      alpha_{L-1}^{-1}; bGL = gL_{L-2}
    if (real) {
      for (int o = tid; o < MAT; o += NT) bK[o] = mk(0.0f, 0.0f);
      __syncthreads();
      const cd* fD = LDv.gen ? LDv.gfac + (long long)eidx * mD * mD : nullptr;
      for (int o = tid; o < b * mD; o += NT) {
        const int r = o / mD, j = o - r * mD;
        cf acc = mk(0.0f, 0.0f);
        if (fD) {
          for (int s = 0; s < mD; ++s) {
            const cd v = fD[s * mD + j];
            acc = cmac(acc, bG[r * LD + pcol(LDv.sites[s])], mk((float)v.re, (float)v.im));
          }
          bK[r * LD + pcol(j)] = acc;
        } else {
          for (int s = 0; s < mD; ++s) {
            const int e = (j * s) % mD;
            acc = cmac(acc, bG[r * LD + pcol(LDv.sites[s])], mk((float)LDv.tw[2 * e], (float)LDv.tw[2 * e + 1]));
          }
          bK[r * LD + pcol(j)] = scale(acc, (float)S.sqD[j]);
        }
      }
    }
    if (L > 1) {
      if (act) {
        tzero(ta);
        talpha(ta, L - 1, L, b, rpb, spr, eps, S.ip, sigS, sigD, S.sinvS, S.sinvD, r0, c0);
        if (real) {
          Tile tg;
          gload<NTA>(tg, gl_of(L - 2), tid);
          tstore<LD>(bGL, tg, r0, c0);
        }
      }
      tinv<NW, 1>(ta, ta, bGR, nullptr, b, S.inv, bT, tid, act, tc, r0, c0);  // gR_{L-1} = alpha_{L-1}^{-1}
    }
    __syncthreads();

    float rnum = 0.0f, rden = 0.0f;   // sum-rule residual: max(0, A_S + A_D + 2 Im G) / max |2 Im G|
    for (int l = L - 1; l >= 0; --l) {
      // the next layer's staged tiles (y_{l-1}, gL_{l-2}, R_{l-1}) on their way to L2
      if (l >= 2) gprefetch<NT>(yl_of(l - 1), TILEB, tid);
      if (real && l >= 2) gprefetch<NT>(gl_of(l - 2), TILEB, tid);
      if (real && l >= 1) gprefetch<NT>(rl_of(l - 1), TILEB, tid);
      if (l < L - 1) {
        // entering: bG and bT free, bGR = gR_{l+1}, bK = K_{l+1}, bGL = gL_l
        const long long cp = (long long)l * S.ip.cp_step;
        const int* rcnt = S.ip.rs_cnt + cp;
        const int* ridx = S.ip.rs_idx + cp * kmax;
        const cf* rval = S.ip.rs_val + cp * kmax;
        const int* ccnt = S.ip.cs_cnt + cp;
        const int* cidx = S.ip.cs_idx + cp * kmax;
        const cf* cval = S.ip.cs_val + cp * kmax;
        if (act) {
          if (real) {    // R_l
            Tile tg;
            gload<NTA>(tg, rl_of(l), tid);
            tstore<LD>(bR, tg, r0, c0);
          }
          tzero(ta);
          trow<LD, false>(ta, rcnt, ridx, rval, kmax, bGR, b, r0, c0);         // W1 = H_{l,l+1} gR_{l+1}
          tstore<LD>(bT, ta, r0, c0);
          if (real) {
            tzero(ta);
            tcol<LD, false>(ta, bGL, ccnt, cidx, cval, kmax, b, r0, c0);       // Wk = gL_l H_{l,l+1}
            tstore<LD>(bG, ta, r0, c0);
          }
        }
        bar<NW>();
        Tile tk, tm1;
        if (act) {
          if (real) {
            tgemm<LD>(tk, bG, bK, b, r0, c0);                                  // K_l = Wk K_{l+1}
            if (l > 0) {   // gL_{l-1}, the next layer's gL (bGL was last read by Wk)
              Tile tg;
              gload<NTA>(tg, gl_of(l - 1), tid);
              tstore<LD>(bGL, tg, r0, c0);
            }
          }
          tzero(tm1);
          tcol<LD, true>(tm1, bT, rcnt, ridx, rval, kmax, b, r0, c0);          // x_l = W1 H_{l+1,l}
          talpha(tm1, l, L, b, rpb, spr, eps, S.ip, sigS, sigD, S.sinvS, S.sinvD, r0, c0);
        }
        bar<NW>();
        if (act && real) tstore<LD>(bK, tk, r0, c0);
        if (l > 0) {
          if (act) {   // y_l as the forward sweep formed it
            gload<NTA>(ta, yl_of(l), tid);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) ta.v[i][j] = tm1.v[i][j] - ta.v[i][j];   // alpha_l - x_l - y_l
          }
          // G_ll = (alpha_l - x_l - y_l)^{-1} into bG (free since K_l was formed), gR_l =
          // (alpha_l - x_l)^{-1} into bGR (gR_{l+1} was last read by W1)
          tinv<NW, 2>(ta, tm1, bG, bGR, b, S.inv, bT, tid, act, tc, r0, c0);
        } else {
          tinv<NW, 1>(tm1, tm1, bG, nullptr, b, S.inv, bT, tid, act, tc, r0, c0);   // G_00 = (alpha_0 - x_0)^{-1}
        }
        bar<NW>();
      }
      // per-site contributions of layer l, summed per ring: rows on warp 0 with a fixed lane
      // mapping and fixed-order row sums, so the result does not depend on the CTA width
      // (in FP32: an FP64 operation costs the FP64 pipe about as much as 60 FP32 ones)
      float vr0 = 0.0f, vr1 = 0.0f;   // the layer's first and second ring (rpb <= 2)
      if (real) {
        if (act) {
          Tile tp;
          tgemm<LD>(tp, bG, bR, b, r0, c0);                                    // G_ll R_l
          tstore<LD>(bT, tp, r0, c0);
        }
        bar<NW>();
        if (tid < 32)
          for (int r = tid; r < b; r += 32) {
            // even and odd columns in two chains each, added at the end
            float as0 = 0.0f, as1 = 0.0f, ad0 = 0.0f, ad1 = 0.0f;
            const cf* tr = bT + r * LD;
            const cf* kr = bK + r * LD;
            for (int j = 0; j < mS; j += 2) {
              const cf x = tr[pcol(j)];
              as0 = fmaf(x.im, x.im, fmaf(x.re, x.re, as0));
              if (j + 1 < mS) {
                const cf y = tr[pcol(j + 1)];
                as1 = fmaf(y.im, y.im, fmaf(y.re, y.re, as1));
              }
            }
            for (int j = 0; j < mD; j += 2) {
              const cf x = kr[pcol(j)];
              ad0 = fmaf(x.im, x.im, fmaf(x.re, x.re, ad0));
              if (j + 1 < mD) {
                const cf y = kr[pcol(j + 1)];
                ad1 = fmaf(y.im, y.im, fmaf(y.re, y.re, ad1));
              }
            }
            const float as = as0 + as1, ad = ad0 + ad1;
            if (r < spr)
              vr0 = fmaf(S.ip.wS, as, fmaf(S.ip.wD, ad, vr0));
            else
              vr1 = fmaf(S.ip.wS, as, fmaf(S.ip.wD, ad, vr1));
            if (a.resid) {
              rnum = fmaxf(rnum, fmaf(2.0f, bG[r * LD + pcol(r)].im, as + ad));
              rden = fmaxf(rden, fabsf(2.0f * bG[r * LD + pcol(r)].im));
            }
          }
      } else if (tid < 32) {
        for (int r = tid; r < b; r += 32) {
          const cf gd = bG[r * LD + pcol(r)];
          if (r < spr)
            vr0 = fmaf(S.ip.kap.re, gd.im, fmaf(S.ip.kap.im, gd.re, vr0));
          else
            vr1 = fmaf(S.ip.kap.re, gd.im, fmaf(S.ip.kap.im, gd.re, vr1));
        }
      }
      if (tid < 32)
        for (int q = 0; q < rpb; ++q) {
          const float s = wsumf(q == 0 ? vr0 : vr1);
          if (tid == 0) part[l * rpb + q] = (double)s;
        }
      bar<NW>();
    }
    if (real) {
      // T = || L_S^dag K_0 ||_F^2 (warp 0, fixed lane mapping)
      double tv = 0.0;
      const cd* fS = LS.gen ? LS.gfac + (long long)eidx * mS * mS : nullptr;
      if (tid < 32)
        for (int o = tid; o < mS * mD; o += 32) {
          const int i = o / mD, j = o - i * mD;
          cf acc = mk(0.0f, 0.0f);
          if (fS) {
            for (int s = 0; s < mS; ++s) {
              const cd v = fS[s * mS + i];
              acc = cmac_cj(acc, mk((float)v.re, (float)v.im), bK[LS.sites[s] * LD + pcol(j)]);
            }
            tv += (double)abs2(acc);
          } else {
            for (int s = 0; s < mS; ++s) {
              const int e = (i * s) % mS;
              acc = cmac_cj(acc, mk((float)LS.tw[2 * e], (float)LS.tw[2 * e + 1]), bK[LS.sites[s] * LD + pcol(j)]);
            }
            tv = fma((double)abs2(acc), S.sqS[i] * S.sqS[i], tv);
          }
        }
      const double Tval = tid < 32 ? wsumd(tv) : 0.0;
      if (tid == 0) a.Tpart[W.tout] = Tval;
      double rs = 0.0, gr = 0.0;
      if (a.resid || FUSE) {
        const double rn = cta_maxd<NW>((double)rnum, S.red, tid);
        const double rd = cta_maxd<NW>((double)rden, S.red, tid);
        rs = rn / fmax(rd, 1e-300);
        if (tid == 0 && a.resid) a.resid[W.tout] = rs;
      }
      if (a.growth || FUSE) {
        gr = sqrt(cta_maxd<NW>((double)gmax, S.red, tid));
        if (tid == 0 && a.growth) a.growth[W.tout] = gr;
      }
      if (FUSE) {
        // the flag of the mixed path, the same on every thread (maxima are exact)
        const bool redo = !(rs <= a.flag_threshold) || !(gr <= a.growth_threshold) || (a.edge && a.edge[W.tout]);
        if (redo) {
          __syncthreads();
          if (tid == 0) a.flags[W.tout] = 1;
          SweepArgs a64 = a;
          a64.resid = nullptr;
          a64.growth = nullptr;
          a64.lane_stats = nullptr;
          blk_item<double, NW, false, true>(a64, W, sm_b32, stage, a.fuse_bmax, a.fuse_mmax);
          __syncthreads();
          // the FP64 layout overwrote this CTA's matrices: restore the zero padding
          for (int o = tid; o < (int)(sizeof(Smem32<NW>) / 4); o += NT) reinterpret_cast<float*>(&S)[o] = 0.0f;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host side

int blk32_class(int b, int m, int warps) {
  if (b < 1 || m > b || b > T32<4>::BMAX) return 0;
  const int need = b <= T32<1>::BMAX ? 1 : (b <= T32<2>::BMAX ? 2 : 4);
  const int w = warps <= 1 ? 1 : (warps <= 2 ? 2 : 4);
  return need > w ? need : w;
}

size_t blk32_smem_bytes(int nw) {
  return nw == 1 ? sizeof(Smem32<1>) : (nw == 2 ? sizeof(Smem32<2>) : sizeof(Smem32<4>));
}

long long blk32_stage_layer_bytes(int nw) {
  const int nta = nw == 1 ? T32<1>::NTA : (nw == 2 ? T32<2>::NTA : T32<4>::NTA);
  return 3LL * nta * 12 * (long long)sizeof(cf);   // y_l, gL_l, R_l
}

bool blk32_can_fuse(int b, int m, int nw) {
  return blk32_class(b, m, nw) == nw && sweep_blk_compact(b, m, 16, nw) &&
         sweep_blk_smem_bytes_t(b, m, 16, nw) <= blk32_smem_bytes(nw);
}

template <int NW, bool FUSE>
static int occ32() {
  const size_t smem = sizeof(Smem32<NW>);
  cudaFuncSetAttribute(sweep_blk32_kernel<NW, FUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep_blk32_kernel<NW, FUSE>, 32 * NW, smem) !=
          cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    per = 1;
  }
  return per;
}

int blk32_occupancy(int nw, int fuse) {
  if (fuse) return nw == 1 ? occ32<1, true>() : (nw == 2 ? occ32<2, true>() : occ32<4, true>());
  return nw == 1 ? occ32<1, false>() : (nw == 2 ? occ32<2, false>() : occ32<4, false>());
}

int launch_blk32(const SweepArgs& a, int grid, int nw, cudaStream_t s) {
  // the dynamic shared memory limit was raised by the occupancy query when planning
  if (a.fuse) {
    if (nw == 1)
      sweep_blk32_kernel<1, true><<<grid, 32, sizeof(Smem32<1>), s>>>(a);
    else if (nw == 2)
      sweep_blk32_kernel<2, true><<<grid, 64, sizeof(Smem32<2>), s>>>(a);
    else
      sweep_blk32_kernel<4, true><<<grid, 128, sizeof(Smem32<4>), s>>>(a);
  } else if (nw == 1) {
    sweep_blk32_kernel<1, false><<<grid, 32, sizeof(Smem32<1>), s>>>(a);
  } else if (nw == 2) {
    sweep_blk32_kernel<2, false><<<grid, 64, sizeof(Smem32<2>), s>>>(a);
  } else {
    sweep_blk32_kernel<4, false><<<grid, 128, sizeof(Smem32<4>), s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace negf
