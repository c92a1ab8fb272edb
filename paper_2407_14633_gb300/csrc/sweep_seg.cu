// Sweeps of 1 x 1 chains split along the channel, for chains with many more layers than
// energies (the mode-space shapes of the paper's Table 2: half a million rings, 90 contour
// nodes).  The thread-per-lane sweep runs every layer of a lane in one thread, so a handful of
// lanes leaves the GPU idle.  Here a lane's L layers are cut into segments of SEG_LEN; one
// warp handles one segment of 32 energies, and the dependence between segments is carried by
// maps composed per segment and chained by a short scan.
//
// Forward (left-connected) recursion, Alg. 2 read as the textbook RGF:
//   gL_l = 1 / (x_l - h_{l-1}^2 gL_{l-1}),  x_l = eps - H_ll - U_l (- Sigma_S at l = 0, - Sigma_D at L - 1)
// is the Moebius map of [[0, 1], [-h_{l-1}^2, x_l]].  A segment's product matrix maps the gL
// entering it to the gL leaving it.
// Backward update (Alg. 1 by the left-connected blocks):
//   G_l = gL_l + h_l^2 gL_l^2 G_{l+1}   (G_{L-1} = gL_{L-1})
// is affine in G_{l+1}; a segment composes to G_{l0} = A + B G_{l1}.  The drain column
// |G_{l,L-1}|^2 = h_l^2 |gL_l|^2 |G_{l+1,L-1}|^2 and the source weight
// |G_{l,0}|^2 / |G_ll|^2 = prod_{j<=l} h_{j-1}^2 |gL_{j-1}|^2 are products.
//
// Five launches per wave of items: (1) segment maps, (2) scan of the forward maps, (3) the
// forward recursion re-run from the scanned entry value (staging gL and the source weight,
// composing the backward maps), (4) scan of the backward maps and products, (5) the backward
// recursion with the per-ring quadrature reduction of the thread-per-lane sweep.  The scans
// are two-level: maps composed per chunk of segments, chained, then walked per chunk.  Segments
// are fixed per device (SEG_LEN layers), so every result is the same in any batch.
#include "sweep_seg.cuh"
#include "lead.cuh"

namespace negf {

namespace {

// record fields (each 32 doubles, one per lane)
enum {
  F_MAP = 0,      // 8: forward map a, b, c, d
  F_GEND = 8,     // 2: gL at the segment's last layer
  F_A = 10,       // 2: backward map G_{l0} = A + B G_{l1}
  F_B = 12,       // 2
  F_QP = 14,      // product of the source-weight factors over the segment
  F_CP = 15,      // product of the drain-column factors over the segment
  F_Q0 = 16,      // segment 0: g w f_S Gamma_S / (2 pi) of the lane
  F_GIN = 17,     // 2: G_{l1} entering the backward re-run
  F_CIN = 19,     // |G_{l1,L-1}|^2 (1 past the last layer)
  F_QIN = 20,     // source weight entering the segment
};

__device__ __forceinline__ double* rec_ptr(const SegArgs& a, long long r) {
  return a.rec + r * (long long)SEG_FIELDS * 32;
}

// Lane set-up shared by the per-segment kernels: energy, weights and contact self-energies.
struct Lane {
  cd eps, sS, sD, kap;
  double wS, wD;
  bool act;
};

__device__ __forceinline__ Lane lane_setup(const DeviceView& D, const ChainView& C, const WorkItem& W, int lane,
                                           bool sigS, bool sigD) {
  Lane o;
  o.act = lane < W.ne;
  const int k = W.e0 + (o.act ? lane : 0);
  const double g = 2.0 * C.g_b;
  o.wS = o.wD = 0.0;
  o.kap = mk(0.0, 0.0);
  if (W.kind == 0) {
    o.eps = mk(D.E[k], D.eta);
    if (o.act) {
      o.wS = g * D.w[k] * D.fS[k] * (0.5 / 3.14159265358979323846);
      o.wD = g * D.w[k] * D.fD[k] * (0.5 / 3.14159265358979323846);
    }
  } else {
    o.eps = D.z[k];
    if (o.act) o.kap = scale(D.c[k], g / 3.14159265358979323846);
  }
  o.sS = sigS ? mode_sigma(C.lead[0], 0, o.eps) : mk(0.0, 0.0);
  o.sD = sigD ? mode_sigma(C.lead[1], 0, o.eps) : mk(0.0, 0.0);
  return o;
}

// x_l = eps - H_ll - U_l, less the contact self-energies at the ends
__device__ __forceinline__ cd layer_x(const DeviceView& D, const ChainView& C, const Lane& q, int l, int L) {
  cd x;
  if (C.hu) {
    x.re = q.eps.re - C.hu[l];
    x.im = C.diag_real ? q.eps.im : q.eps.im - C.Hdiag[l].im;
  } else {
    const cd h = C.Hdiag[l];
    x = mk(q.eps.re - h.re - D.U[l], q.eps.im - h.im);
  }
  if (l == 0) x = x - q.sS;
  if (l == L - 1) x = x - q.sD;
  return x;
}

struct Where {
  const WorkItem* W;
  const DeviceView* D;
  const ChainView* C;
  SegItem S;
  int s, l0, l1, L;
};

__device__ __forceinline__ bool locate(const SegArgs& a, long long r, Where& w) {
  if (r >= a.n_rec) return false;
  w.S = a.segs[a.rec_item[r]];
  w.s = (int)(r - w.S.rec0);
  w.W = &a.items[w.S.item];
  w.D = &a.devs[w.W->dev];
  w.C = &w.D->ch[w.W->chain];
  w.L = w.D->L;
  w.l0 = w.s * SEG_LEN;
  w.l1 = min(w.L, w.l0 + SEG_LEN);
  return true;
}

// scale the four entries of a projective map by a power of two (exact) so that the largest
// is in [1, 2)
__device__ __forceinline__ void renorm(cd& a, cd& b, cd& c, cd& d) {
  const double m = fmax(fmax(fmax(fabs(a.re), fabs(a.im)), fmax(fabs(b.re), fabs(b.im))),
                        fmax(fmax(fabs(c.re), fabs(c.im)), fmax(fabs(d.re), fabs(d.im))));
  if (!(m > 0.0) || !isfinite(m)) return;
  const int e = -ilogb(m);
  a = mk(scalbn(a.re, e), scalbn(a.im, e));
  b = mk(scalbn(b.re, e), scalbn(b.im, e));
  c = mk(scalbn(c.re, e), scalbn(c.im, e));
  d = mk(scalbn(d.re, e), scalbn(d.im, e));
}

// (1) product of the segment's forward maps
__global__ void __launch_bounds__(128) seg_map_kernel(SegArgs a) {
  const int lane = threadIdx.x & 31;
  Where w;
  if (!locate(a, (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), w)) return;
  const DeviceView& D = *w.D;
  const ChainView& C = *w.C;
  const Lane q = lane_setup(D, C, *w.W, lane, w.l0 == 0, w.l1 == w.L);
  cd ma = mk(1.0, 0.0), mb = mk(0.0, 0.0), mc = mk(0.0, 0.0), md = mk(1.0, 0.0);
  for (int l = w.l0; l < w.l1; ++l) {
    const cd x = layer_x(D, C, q, l, w.L);
    const double hs = l > 0 ? C.hsq[l - 1] : 0.0;
    // [[0, 1], [-hs, x]] [[a, b], [c, d]]
    const cd na = mc, nb = md;
    cd nc = x * mc, nd = x * md;
    nc.re = fma(-hs, ma.re, nc.re);
    nc.im = fma(-hs, ma.im, nc.im);
    nd.re = fma(-hs, mb.re, nd.re);
    nd.im = fma(-hs, mb.im, nd.im);
    ma = na;
    mb = nb;
    mc = nc;
    md = nd;
    if (((l - w.l0) & 7) == 7) renorm(ma, mb, mc, md);
  }
  renorm(ma, mb, mc, md);
  double* rp = rec_ptr(a, (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
  rp[(F_MAP + 0) * 32 + lane] = ma.re;
  rp[(F_MAP + 1) * 32 + lane] = ma.im;
  rp[(F_MAP + 2) * 32 + lane] = mb.re;
  rp[(F_MAP + 3) * 32 + lane] = mb.im;
  rp[(F_MAP + 4) * 32 + lane] = mc.re;
  rp[(F_MAP + 5) * 32 + lane] = mc.im;
  rp[(F_MAP + 6) * 32 + lane] = md.re;
  rp[(F_MAP + 7) * 32 + lane] = md.im;
}

// Scans over an item's segments, one CTA of SCAN_WARPS warps per item (lane = energy): each
// warp composes the maps of one chunk of consecutive segments, warp 0 chains the chunks, then
// each warp walks its own segments from its chunk's entry value.
constexpr int SCAN_WARPS = 16;

__device__ __forceinline__ void chunk_range(int n, int w, int& s0, int& s1) {
  const int per = (n + SCAN_WARPS - 1) / SCAN_WARPS;
  s0 = min(n, w * per);
  s1 = min(n, s0 + per);
}

// (2) gL leaving each segment: g <- (a g + b) / (c g + d) over the segments in order
__global__ void __launch_bounds__(32 * SCAN_WARPS) seg_fscan_kernel(SegArgs a) {
  __shared__ double chm[SCAN_WARPS][8][32];   // chunk maps
  __shared__ double ent[SCAN_WARPS][2][32];   // gL entering each chunk
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const SegItem S = a.segs[blockIdx.x];
  int s0, s1;
  chunk_range(S.n_seg, w, s0, s1);
  // chunk product M = M_{s1-1} ... M_{s0}
  cd A = mk(1.0, 0.0), B = mk(0.0, 0.0), C = mk(0.0, 0.0), D = mk(1.0, 0.0);
  for (int s = s0; s < s1; ++s) {
    const double* rp = rec_ptr(a, S.rec0 + s);
    const cd ma = mk(rp[(F_MAP + 0) * 32 + lane], rp[(F_MAP + 1) * 32 + lane]);
    const cd mb = mk(rp[(F_MAP + 2) * 32 + lane], rp[(F_MAP + 3) * 32 + lane]);
    const cd mc = mk(rp[(F_MAP + 4) * 32 + lane], rp[(F_MAP + 5) * 32 + lane]);
    const cd md = mk(rp[(F_MAP + 6) * 32 + lane], rp[(F_MAP + 7) * 32 + lane]);
    const cd nA = cmac(ma * A, mb, C), nB = cmac(ma * B, mb, D);
    const cd nC = cmac(mc * A, md, C), nD = cmac(mc * B, md, D);
    A = nA;
    B = nB;
    C = nC;
    D = nD;
    renorm(A, B, C, D);
  }
  chm[w][0][lane] = A.re;
  chm[w][1][lane] = A.im;
  chm[w][2][lane] = B.re;
  chm[w][3][lane] = B.im;
  chm[w][4][lane] = C.re;
  chm[w][5][lane] = C.im;
  chm[w][6][lane] = D.re;
  chm[w][7][lane] = D.im;
  __syncthreads();
  if (w == 0) {
    cd g = mk(0.0, 0.0);
    for (int k = 0; k < SCAN_WARPS; ++k) {
      ent[k][0][lane] = g.re;
      ent[k][1][lane] = g.im;
      g = cdiv(cmac(mk(chm[k][2][lane], chm[k][3][lane]), mk(chm[k][0][lane], chm[k][1][lane]), g),
               cmac(mk(chm[k][6][lane], chm[k][7][lane]), mk(chm[k][4][lane], chm[k][5][lane]), g));
    }
  }
  __syncthreads();
  cd g = mk(ent[w][0][lane], ent[w][1][lane]);
  for (int s = s0; s < s1; ++s) {
    double* rp = rec_ptr(a, S.rec0 + s);
    g = cdiv(cmac(mk(rp[(F_MAP + 2) * 32 + lane], rp[(F_MAP + 3) * 32 + lane]),
                  mk(rp[(F_MAP + 0) * 32 + lane], rp[(F_MAP + 1) * 32 + lane]), g),
             cmac(mk(rp[(F_MAP + 6) * 32 + lane], rp[(F_MAP + 7) * 32 + lane]),
                  mk(rp[(F_MAP + 4) * 32 + lane], rp[(F_MAP + 5) * 32 + lane]), g));
    rp[(F_GEND + 0) * 32 + lane] = g.re;
    rp[(F_GEND + 1) * 32 + lane] = g.im;
  }
}

// (3) forward re-run from the scanned entry value: stage gL_l (and the source weight relative
// to the segment's entry), compose the backward map and the segment's products
__global__ void __launch_bounds__(128) seg_rerun_kernel(SegArgs a) {
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  Where w;
  if (!locate(a, r, w)) return;
  const DeviceView& D = *w.D;
  const ChainView& C = *w.C;
  const WorkItem& W = *w.W;
  const bool real = W.kind == 0;
  const Lane q = lane_setup(D, C, W, lane, w.l0 == 0, w.l1 == w.L);
  const int nf = real ? 3 : 2;
  double* st = reinterpret_cast<double*>(a.stage + w.S.stage);
  double* rp = rec_ptr(a, r);
  cd gp = mk(0.0, 0.0);
  if (w.s > 0) {
    const double* pp = rec_ptr(a, r - 1);
    gp = mk(pp[(F_GEND + 0) * 32 + lane], pp[(F_GEND + 1) * 32 + lane]);
  }
  double rl = abs2(gp);     // |gL_{l-1}|^2
  double qrel = 1.0;        // prod over the segment of h_{j-1}^2 |gL_{j-1}|^2
  double cp = 1.0;          // prod over the segment of the drain-column factors
  cd A = mk(0.0, 0.0), B = mk(1.0, 0.0);
  for (int l = w.l0; l < w.l1; ++l) {
    cd x = layer_x(D, C, q, l, w.L);
    if (l > 0) {
      const double hs = C.hsq[l - 1];
      x.re = fma(-hs, gp.re, x.re);
      x.im = fma(-hs, gp.im, x.im);
      if (real) qrel = (hs * rl) * qrel;
    }
    const double rr = 1.0 / fma(x.re, x.re, x.im * x.im);
    const cd g = mk(x.re * rr, -x.im * rr);
    rl = rr;
    double* sp = st + (long long)l * nf * 32;
    sp[lane] = g.re;
    sp[32 + lane] = g.im;
    if (real) sp[64 + lane] = qrel;
    // G_l = g + b_l G_{l+1}: A <- A + B g, B <- B b_l
    A = cmac(A, B, g);
    const double a2 = abs2(g);
    if (l < w.L - 1) {
      const double hn = C.hsq[l];
      B = B * scale(g * g, hn);
      cp = (hn * a2) * cp;
    } else {
      B = mk(0.0, 0.0);
      cp = a2 * cp;
    }
    gp = g;
  }
  rp[(F_A + 0) * 32 + lane] = A.re;
  rp[(F_A + 1) * 32 + lane] = A.im;
  rp[(F_B + 0) * 32 + lane] = B.re;
  rp[(F_B + 1) * 32 + lane] = B.im;
  rp[F_QP * 32 + lane] = qrel;
  rp[F_CP * 32 + lane] = cp;
  if (w.s == 0) rp[F_Q0 * 32 + lane] = real ? q.wS * (-2.0 * q.sS.im) : 0.0;
}

// (4) entry values of the backward re-run: G and the drain column from the right, the source
// weight from the left (chunks as in the forward scan)
__global__ void __launch_bounds__(32 * SCAN_WARPS) seg_bscan_kernel(SegArgs a) {
  __shared__ double chm[SCAN_WARPS][6][32];   // chunk maps: A, B, CP, QP
  __shared__ double ent[SCAN_WARPS][4][32];   // G and c at each chunk's right end, q at its left end
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const SegItem S = a.segs[blockIdx.x];
  int s0, s1;
  chunk_range(S.n_seg, w, s0, s1);
  // chunk composition: G_{left} = A + B G_{right}; products of the drain and source factors
  cd A = mk(0.0, 0.0), B = mk(1.0, 0.0);
  double cp = 1.0, qp = 1.0;
  for (int s = s0; s < s1; ++s) {
    const double* rp = rec_ptr(a, S.rec0 + s);
    A = cmac(A, B, mk(rp[(F_A + 0) * 32 + lane], rp[(F_A + 1) * 32 + lane]));
    B = B * mk(rp[(F_B + 0) * 32 + lane], rp[(F_B + 1) * 32 + lane]);
    cp = cp * rp[F_CP * 32 + lane];
    qp = rp[F_QP * 32 + lane] * qp;
  }
  chm[w][0][lane] = A.re;
  chm[w][1][lane] = A.im;
  chm[w][2][lane] = B.re;
  chm[w][3][lane] = B.im;
  chm[w][4][lane] = cp;
  chm[w][5][lane] = qp;
  __syncthreads();
  if (w == 0) {
    cd G = mk(0.0, 0.0);
    double c = 1.0;
    for (int k = SCAN_WARPS - 1; k >= 0; --k) {
      ent[k][0][lane] = G.re;
      ent[k][1][lane] = G.im;
      ent[k][2][lane] = c;
      G = cmac(mk(chm[k][0][lane], chm[k][1][lane]), mk(chm[k][2][lane], chm[k][3][lane]), G);
      c = chm[k][4][lane] * c;
    }
    double q = rec_ptr(a, S.rec0)[F_Q0 * 32 + lane];
    for (int k = 0; k < SCAN_WARPS; ++k) {
      ent[k][3][lane] = q;
      q = chm[k][5][lane] * q;
    }
  }
  __syncthreads();
  cd G = mk(ent[w][0][lane], ent[w][1][lane]);
  double c = ent[w][2][lane];
  for (int s = s1 - 1; s >= s0; --s) {
    double* rp = rec_ptr(a, S.rec0 + s);
    rp[(F_GIN + 0) * 32 + lane] = G.re;
    rp[(F_GIN + 1) * 32 + lane] = G.im;
    rp[F_CIN * 32 + lane] = c;
    G = cmac(mk(rp[(F_A + 0) * 32 + lane], rp[(F_A + 1) * 32 + lane]),
             mk(rp[(F_B + 0) * 32 + lane], rp[(F_B + 1) * 32 + lane]), G);
    c = rp[F_CP * 32 + lane] * c;
  }
  double q = ent[w][3][lane];
  for (int s = s0; s < s1; ++s) {
    double* rp = rec_ptr(a, S.rec0 + s);
    rp[F_QIN * 32 + lane] = q;
    q = rp[F_QP * 32 + lane] * q;
  }
}

// flush ring slots [base, base + count) of the 32 x 33 transpose buffer into `dst`
__device__ __forceinline__ void flush_seg(double* red, int lane, int count, double* dst) {
  __syncwarp();
  if (lane < count) {
    double s = 0.0;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) s += red[lane * 33 + j];
    dst[lane] = s;
  }
  __syncwarp();
}

// (5) backward re-run and the fused quadrature: per ring, the 32 energies of the warp summed
// in lane order into the item's partial slot, as in the thread-per-lane sweep
__global__ void __launch_bounds__(128) seg_back_kernel(SegArgs a) {
  extern __shared__ double sm_seg[];
  const int lane = threadIdx.x & 31;
  double* red = sm_seg + (threadIdx.x >> 5) * (32 * 33);
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  Where w;
  if (!locate(a, r, w)) return;
  const DeviceView& D = *w.D;
  const ChainView& C = *w.C;
  const WorkItem& W = *w.W;
  const bool real = W.kind == 0;
  const Lane q = lane_setup(D, C, W, lane, real, real);
  const double gamS = -2.0 * q.sS.im, gamD = -2.0 * q.sD.im;
  const double wDg = q.wD * gamD;
  const int nf = real ? 3 : 2;
  const double* st = reinterpret_cast<const double*>(a.stage + w.S.stage);
  const double* rp = rec_ptr(a, r);
  cd G = mk(rp[(F_GIN + 0) * 32 + lane], rp[(F_GIN + 1) * 32 + lane]);
  double c = rp[F_CIN * 32 + lane];
  const double q0 = rp[F_QIN * 32 + lane];
  double* part = a.partial + W.part;
  for (int l = w.l1 - 1; l >= w.l0; --l) {
    const double* sp = st + (long long)l * nf * 32;
    const cd gll = mk(sp[lane], sp[32 + lane]);
    if (l < w.L - 1) {
      const double hs = C.hsq[l];
      const cd t = scale(gll * G, hs);     // |h|^2 gL G_{l+1}
      G = cmac(gll, gll, t);                // gL + gL (|h|^2 gL G_{l+1})
      c = (hs * abs2(gll)) * c;             // |G_{l,L-1}|^2
    } else {
      G = gll;
      c = abs2(gll) * c;
    }
    double v;
    if (real) {
      const double ql = q0 * sp[64 + lane];
      v = fma(wDg, c, ql * abs2(G));
    } else {
      v = q.kap.re * G.im + q.kap.im * G.re;
    }
    if (a.ring_cap && l == a.cap_ring && real && q.act) a.ring_cap[W.tout + lane] = v;
    red[(l & 31) * 33 + lane] = v;
    if ((l & 31) == 0) flush_seg(red, lane, min(32, w.L - l), part + l);
  }
  if (w.l0 == 0 && real && q.act) a.Tpart[W.tout + lane] = gamS * gamD * c;
}

}  // namespace

size_t seg_stage_bytes(int L, int kind) { return (size_t)L * (kind == 0 ? 3 : 2) * 32 * sizeof(double); }

int launch_seg(const SegArgs& a, cudaStream_t s) {
  if (a.n_rec <= 0 || a.n_segitems <= 0) return 0;
  // one warp per CTA: the records spread over the SMs within one CTA of each other
  constexpr int WPB = 1;
  const long long grid = (a.n_rec + WPB - 1) / WPB;
  if (grid > 0x7fffffffLL) return -1;
  const size_t smem = (size_t)WPB * 32 * 33 * sizeof(double);
  seg_map_kernel<<<(unsigned)grid, 32 * WPB, 0, s>>>(a);
  seg_fscan_kernel<<<a.n_segitems, 32 * SCAN_WARPS, 0, s>>>(a);
  seg_rerun_kernel<<<(unsigned)grid, 32 * WPB, 0, s>>>(a);
  seg_bscan_kernel<<<a.n_segitems, 32 * SCAN_WARPS, 0, s>>>(a);
  seg_back_kernel<<<(unsigned)grid, 32 * WPB, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace negf
