/*
 * negf.h -- C ABI of the GB300-native energy-parallel NEGF / recursive Green's function
 * library (libnegf.so), after ELEQTRONeX, arXiv 2407.14633.
 *
 * What it computes.  For a block-tridiagonal tight-binding channel (Sec. 2.2.1: the
 * Hamiltonian is block tridiagonal with the electrostatic potential energy on its
 * diagonal) attached to two semi-infinite leads, and for every energy of an equilibrium
 * complex contour and of the real-axis bias window (Eq. Rho), the library forms the
 * contact self-energies (Eq. GR), the diagonal blocks of G^R and of the lead spectral
 * functions A_l = G Gamma_l G^dagger (Alg. 1 / Alg. 2), the transmission
 * T(E) = Tr[Gamma_S G Gamma_D G^dagger] (Eq. deviceCharacteristics) and reduces them by
 * Fermi-weighted quadrature to per-ring electron counts and the current.  A Broyden
 * mixed self-consistent loop (Alg. 3) with a 1D Poisson stand-in closes the loop with
 * electrostatics.  Everything after the host set-up calls runs in CUDA kernels on one
 * GPU (sm_103a).
 *
 * Conventions (all calls):
 *   - Every call returns an int status: NEGF_OK (0) or a negative NEGF_E* code.  On error
 *     nothing the caller owns is modified except where stated, and the context's last
 *     error message (negf_last_error) describes the failure.
 *   - Complex numbers are interleaved pairs double[2] = {re, im} (C99 double _Complex
 *     layout).  Matrices are row-major; a stack of blocks is contiguous block after block.
 *   - Host arrays passed in are copied before the call returns; the caller keeps
 *     ownership and may free or reuse them.  No call keeps a caller pointer.
 *   - Output arrays are caller-owned host memory unless a call says "device".
 *   - Units: energies and potential energies in eV, voltages in V, lengths in nm,
 *     kT in eV, current in A.  Electron counts are dimensionless (the paper's rho is
 *     minus the electron density, Eq. Rho; this API reports electron counts n).
 *   - One context per host thread, or external locking.
 */
#ifndef NEGF_H
#define NEGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------- */
#define NEGF_OK 0
#define NEGF_EINVAL (-1)        /* bad argument, size or state                       */
#define NEGF_ENOMEM (-2)        /* device or host allocation failed / over budget    */
#define NEGF_ECUDA (-3)         /* a CUDA runtime call failed                        */
#define NEGF_ETIMEDOUT (-4)     /* a bounded wait ran out                            */
#define NEGF_ENOTCONVERGED (-5) /* the self-consistent loop hit its iteration limit  */
#define NEGF_EBUSY (-6)         /* the request is still running                      */
#define NEGF_ENOTFOUND (-7)     /* unknown handle or ticket                          */

/* ---- precision policy ------------------------------------------------------------ */
#define NEGF_PREC_FP64 0   /* complex128 sweep, FP64 everywhere                          */
#define NEGF_PREC_MIXED 1  /* complex64 sweep; flagged energies recomputed in FP64       */
#define NEGF_PREC_FP32 2   /* complex64 sweep only (FP64 lead roots and accumulation)    */

/* ---- lead sides --------------------------------------------------------------------- */
#define NEGF_SOURCE 0
#define NEGF_DRAIN 1

/* ---- grid rules ------------------------------------------------------------------------ */
#define NEGF_RULE_GAUSS 0      /* Gauss-Legendre on [E_min, E_max]                    */
#define NEGF_RULE_MIDPOINT 1   /* midpoint rule on [E_min, E_max]                     */

typedef struct negf_ctx negf_ctx;

/* Context options.  stream: a cudaStream_t to run on (e.g. torch.cuda.Stream.cuda_stream),
 * or NULL for a library-owned stream.  hbm_budget_bytes: cap on the library's device
 * memory (0 = no cap); allocations beyond it fail with NEGF_ENOMEM.  precision: one of
 * NEGF_PREC_*.  flag_threshold: mixed precision, the per-energy sum-rule residual (see
 * negf_out.resid) above which an energy is recomputed in FP64 (0 = default 1e-3).
 * edge_window: mixed precision, energies closer than this (eV) to a lead subband edge are
 * recomputed in FP64 (0 = default 0.002).  fault_alloc_after:
 * host-side fault injection for tests, the n-th arena allocation fails (0 = off).
 * growth_threshold: mixed precision, energies whose complex64 sweep saw a gL entry larger
 * than this (1/eV) are recomputed in FP64 (0 = criterion off, the default).  blk_warps: CTA width (warps)
 * of the sweep of ring blocks wider than 2: 0 = autotuned (each width is timed once per
 * context, with the resident CTAs per SM, on the first batch of a given element type,
 * block size, lead width and item count that has at least one item per SM, then cached;
 * smaller batches use the size policy), -1 = the size policy (1 warp up to b = 20, 2 up to
 * 28, else 4), 1 / 2 / 4 = that width.  Results are bitwise the same for every width.  blk_ctas_per_sm: cap on the resident CTAs per SM of
 * that sweep (0 = as many as fit); the grid is the cap times the SMs.  general_update: 1 =
 * never use the complex-symmetric form of the G_ll update, even for chains whose blocks and
 * lead rows are real (0 = use it there).  chain_warps: CTA width (warps, one 32-energy item each) of
 * the thread-per-lane sweeps of 1 x 1 and 2 x 2 blocks: 0 = autotuned when blk_warps is 0 (every
 * width of 1, 2, 4, 8 warps timed once on the first group of at least one item per SM, per kernel
 * class, element type and power-of-two bucket of the item count, then cached; else 2), 1 / 2 /
 * 4 / 8 = that width.  Results are bitwise the same for every width.  long_chain_split: FP64
 * sweeps of 1 x 1 chains split along the channel into segments of 512 layers, one warp per
 * segment of 32 energies, joined by scans of the per-segment maps of the forward and backward
 * recursions: 0 = for devices with at least 16384 layers and at most 128 such 32-energy items
 * of their own (long channels, few energies), 1 = for every 1 x 1 chain, -1 = never.  The choice
 * is made per device, so a device's results do not depend on its batch; they differ from the
 * unsplit sweep by rounding only.  mixed_two_pass: mixed precision, 1 = recompute flagged
 * energies of ring blocks in a second FP64 pass after the complex64 sweep; 0 = re-sweep a
 * flagged energy in FP64 inside the complex64 kernel, right after its own complex64 sweep,
 * for blocks whose FP64 layout fits that kernel's shared memory and groups of at least 16
 * lanes per resident CTA (the others take the second pass); -1 = re-sweep inside the kernel
 * wherever the layout fits.  All give bitwise the same results. */
typedef struct {
  int device_ordinal;
  void* stream;
  size_t hbm_budget_bytes;
  int precision;
  double flag_threshold;
  double edge_window;
  int fault_alloc_after;
  double growth_threshold;
  int blk_warps;
  int blk_ctas_per_sm;
  int general_update;
  int chain_warps;
  int long_chain_split;
  int mixed_two_pass;
} negf_opts;

/* Create / destroy a context on one GPU.  opts may be NULL (defaults: device 0, own
 * stream, no budget, FP64).  negf_destroy frees every device buffer the context owns. */
int negf_create(negf_ctx** out, const negf_opts* opts);
int negf_destroy(negf_ctx* ctx);

/* Static description of a status code, and the context's last error message. */
const char* negf_strerror(int status);
const char* negf_last_error(const negf_ctx* ctx);

/* ---- devices (Sec. 2.2.1 block-tridiagonal H, Sec. 2.2.2 multi-mode arrays) -------- */

/* A device is a channel of n_rings rings made of n_chains independent block-tridiagonal
 * chains sharing one potential (several mode-space subbands are independent chains,
 * Sec. 2.2.2).  Each chain has L = n_rings / rings_per_block layers of width `block`;
 * site a of layer l belongs to ring l * rings_per_block + a / (block / rings_per_block).
 * Supported: block in 1..64, rings_per_block in {1, 2} dividing block and n_rings.
 * Returns the device handle in *dev. */
int negf_device_create(negf_ctx* ctx, int n_rings, int block, int rings_per_block,
                       int n_chains, int* dev);
int negf_device_destroy(negf_ctx* ctx, int dev);

/* Hamiltonian of one chain without the electrostatic potential (Sec. 2.2.1):
 * Hdiag: L blocks H_{l,l} (L*block*block complex), Hup: L-1 blocks H_{l,l+1}
 * ((L-1)*block*block complex); the lower blocks are Hup^dagger (H Hermitian).
 * g_b: band degeneracy of the chain (the spin degeneracy g_s = 2 is fixed). */
int negf_set_hamiltonian(negf_ctx* ctx, int dev, int chain, const double* Hdiag,
                         const double* Hup, double g_b);

/* Semi-infinite lead of one chain (Eq. GR, Sec. 2.2.2).  The lead is a sequence of rings
 * s0, s1, ... moving away from the device with m sites each, on-site potential energy
 * U_lead, couplings H_{s1,s0} = T1, H_{s2,s1} = T2, H_{s3,s2} = T1, ... and device
 * coupling tau = H_{s0, boundary ring}.  T1, T2, tau must be circulant m x m matrices and
 * are given by their first rows (m complex each); their surface Green's function is then
 * the closed-form root of each angular mode (the analytic nanotube lead the paper uses).
 * sites: the m site indices (0..block-1) of the boundary ring inside the first (source)
 * or last (drain) layer.  side: NEGF_SOURCE or NEGF_DRAIN. */
typedef struct {
  int m;
  double U_lead;
  const double* T1;
  const double* T2;
  const double* tau;
  const int* sites;
} negf_lead;
int negf_set_lead(negf_ctx* ctx, int dev, int chain, int side, const negf_lead* lead);

/* A general (non-circulant) lead of one chain, for ring blocks wider than 2 (Eq. GR, Sec. 2.2.2:
 * where no closed form applies the surface Green's function comes from Lopez Sancho-Rubio
 * decimation).  The lead is a sequence of rings s0, s1, s2, ... moving away from the device,
 * with m sites each (1 <= m <= 20), on-site blocks U_lead I + H0 on s0, s2, ... and
 * U_lead I + H1 on s1, s3, ... (Hermitian; NULL = zero), couplings H_{s1,s0} = T1,
 * H_{s2,s1} = T2, H_{s3,s2} = T1, ..., and device coupling tau = H_{s0, boundary ring}.  All
 * blocks are full m x m complex matrices (row-major, interleaved), copied.  sites: the m
 * distinct site indices of the boundary ring inside the first (source) or last (drain) layer.
 * Every launch plan decimates the lead at each of its energies (two-ring principal layers,
 * until the renormalised couplings fall below tol times the largest block entry, at most
 * max_iter steps; 0 = defaults 1e-14 and 400), forms Sigma = tau^dagger g_{s0} tau and
 * Gamma = i (Sigma - Sigma^dagger) and a pivoted Cholesky factor of Gamma for the sweep.
 * Evaluations return NEGF_ENOTCONVERGED if a decimation hits max_iter.  negf_set_lead and
 * the builders replace a general lead; negf_set_lead_potentials sets its U_lead. */
typedef struct {
  int m;
  double U_lead;
  const double* H0;
  const double* H1;
  const double* T1;
  const double* T2;
  const double* tau;
  const int* sites;
  int max_iter;
  double tol;
} negf_lead_general;
int negf_set_lead_general(negf_ctx* ctx, int dev, int chain, int side, const negf_lead_general* lead);

/* Lead potential energies only (U_S, U_D), keeping the couplings. */
int negf_set_lead_potentials(negf_ctx* ctx, int dev, double U_S, double U_D);

/* Convenience builders for (n,0) zigzag nanotubes with nearest-neighbour coupling t
 * (Sec. 3.1), leads continuing the tube, lead potentials U_S / U_D.
 * Mode space: chain c is subband modes[c] (bond k = t for even k, 2 t cos(pi j / n) for
 * odd k, g_b = 2); a device created with block = 2, rings_per_block = 2 groups rings
 * (2l, 2l+1) into 2 x 2 unit-cell blocks.  Real space: n x n ring blocks,
 * bonds t I and t (I + S) / t (I + S^T) alternating, g_b = 1 (block = n, one chain). */
int negf_build_cnt_modespace(negf_ctx* ctx, int dev, int n_tube, double t, const int* modes,
                             double U_S, double U_D);
int negf_build_cnt_realspace(negf_ctx* ctx, int dev, int n_tube, double t, double U_S,
                             double U_D);

/* Electrostatic potential energy per ring (n_rings doubles), added to every site of the
 * ring (Sec. 2.2.1: the diagonal of H is -e phi per ring). */
int negf_set_potential(negf_ctx* ctx, int dev, const double* U);

/* ---- energy grids (Eq. Rho) ----------------------------------------------------------- */

/* An energy grid of one bias point.  Real axis: n_real nodes E, weights w, occupations
 * fS = f(E - mu_S), fD = f(E - mu_D), broadening eta (energies E + i eta).  Contour:
 * n_cont nodes z (complex, Im z > 0) and complex weights c such that
 *   integral_{E_B}^{E_min} G(E) f(E - mu_min) dE = - sum_k c_k G(z_k).
 * The electron count of ring r is
 *   n_r = (g_s g_b/pi) Im sum_k c_k Tr_r G(z_k)
 *       + (g_s g_b/2pi) sum_k w_k [fS_k Tr_r A_S(E_k) + fD_k Tr_r A_D(E_k)]. */
typedef struct {
  int n_real;
  const double* E;
  const double* w;
  const double* fS;
  const double* fD;
  double eta;
  int n_cont;
  const double* z;
  const double* c;
} negf_grid;
int negf_set_grid(negf_ctx* ctx, int dev, const negf_grid* grid);

/* Default grid of a bias point (Eq. Rho, Sec. 3.3).  Real axis on [E_min, E_max] with
 * E_min = mu_min - f1 kT and E_max = mu_max + f2 kT unless given (pass NaN for the
 * default), by `rule`.  Contour: Gauss-Legendre in theta on the upper semicircle over
 * [E_B, E_min], c_k = W_k z'(theta_k) f(z_k - mu_min).  E_B must lie below every band. */
typedef struct {
  double mu_S, mu_D, kT, eta;
  double E_B, E_min, E_max, f1, f2;
  int n_real, n_cont, rule;
} negf_grid_spec;

/* Host helper: fill caller arrays E, w, fS, fD (n_real each) and z, c (2*n_cont each). */
int negf_make_grid(const negf_grid_spec* spec, double* E, double* w, double* fS, double* fD,
                   double* z, double* c);
/* Build the default grid and set it on a device. */
int negf_set_grid_spec(negf_ctx* ctx, int dev, const negf_grid_spec* spec);

/* ---- semi-adaptive real-axis grid (Sec. 3.3) ---------------------------------------------- */

/* The real-axis path [E_min, E_max] split at E_l1 <= E_l2 into three sub-intervals, each with
 * its own Gauss-Legendre rule of ceil(density * width / kT - 1e-6) points (at least one; none
 * for an empty sub-interval).  The limits are clipped into [E_min, E_max].  Refinement locates
 * the peak E_s of the charge integrand of one ring (the van Hove singularity that sharpens
 * with channel length) and moves the limits to E_l1 = E_s - a kT, E_l2 = E_s + b kT (the paper
 * uses a = 3, b = 1).  In a self-consistent session (negf_sc_begin on a device whose grid was
 * set with negf_set_grid_adaptive) the limits are refined at the first iteration and at every
 * iteration that is a multiple of `period` (the paper uses 50; 0 = the first only), with that
 * iteration's potential, before its NEGF evaluation.  ring: the ring whose integrand is used
 * (-1 = the centre ring n_rings / 2). */
typedef struct {
  double E_l1, E_l2;
  double density[3];
  double a, b;
  int period;
  int ring;
} negf_adaptive;

/* Host helper: the grid of spec with the semi-adaptive real axis (spec->n_real and spec->rule
 * are ignored; the contour, E_min, E_max and occupations follow spec as in negf_make_grid).
 * *n_real receives the number of real-axis nodes; E, w, fS, fD may be NULL to count only,
 * else they need *n_real doubles each (call once with NULL to size them).  z, c as in
 * negf_make_grid (NULL when spec->n_cont = 0 or when counting). */
int negf_make_grid_adaptive(const negf_grid_spec* spec, const negf_adaptive* ad, int* n_real, double* E,
                            double* w, double* fS, double* fD, double* z, double* c);
/* Set the semi-adaptive grid on a device (it then also serves negf_sc_begin like
 * negf_set_grid_spec).  Any later negf_set_grid / negf_set_grid_spec replaces it. */
int negf_set_grid_adaptive(negf_ctx* ctx, int dev, const negf_grid_spec* spec, const negf_adaptive* ad);
/* Charge integrand of one ring at every real-axis node of the device's grid, with the device's
 * current potential (host output, n_real doubles):
 *   I_r(E_k) = sum_chains (g_s g_b / 2 pi) [fS_k Tr_r A_S(E_k) + fD_k Tr_r A_D(E_k)],
 * so that sum_k w_k I_r(E_k) is the real-axis part of n_r.  One lane per energy. */
int negf_ring_integrand(negf_ctx* ctx, int dev, int ring, double* I);
/* Refine a semi-adaptive grid once: E_s = the node of largest integrand (the first on ties)
 * of the refinement ring, then the grid rebuilt with E_l1 = E_s - a kT, E_l2 = E_s + b kT.
 * E_s may be NULL.  NEGF_EINVAL if the device grid is not semi-adaptive. */
int negf_refine_grid(negf_ctx* ctx, int dev, double* E_s);
/* Current grid sizes, and the current (clipped) limits of a semi-adaptive grid (NaN for other
 * grids).  Any pointer may be NULL.  Valid during a self-consistent session. */
int negf_grid_info(negf_ctx* ctx, int dev, int* n_real, int* n_cont, double* E_l1, double* E_l2);

/* ---- one NEGF evaluation ----------------------------------------------------------------- */

/* Outputs of one device.  n (n_rings, required): electron count per ring.  T (n_real,
 * optional): sum over chains of g_b T_chain(E).  I (1, optional): Landauer current
 * I = g_s (e^2/h) sum_k w_k T(E_k) (fS_k - fD_k).  n_cont / n_real_part (n_rings,
 * optional): the two parts of n.  flags (n_real, optional, int): per-energy precision
 * flags of the mixed path (1 = recomputed in FP64).  resid (n_real, optional): per-energy
 * sum-rule residual of the complex64 sweep,
 * max(0, max_a (A_S,aa + A_D,aa + 2 Im G_aa)) / max_a |2 Im G_aa| over the sites a of the
 * chain, largest over chains (exact arithmetic gives A_S + A_D = -2 Im G - 2 eta G G^dagger
 * <= -2 Im G on the diagonal, so a positive excess is rounding error).  growth (n_real, optional): per-energy
 * largest entry modulus of the left-connected gL_l seen by the complex64 sweep (large
 * near resonances of the half-open chain, where the backward sweep must cancel it).  Any
 * pointer may be NULL except n.  If on_device != 0 every pointer is device memory on the
 * context's GPU and the results are left there (no host copy). */
typedef struct {
  double* n;
  double* T;
  double* I;
  double* n_cont;
  double* n_real_part;
  int* flags;
  double* resid;
  double* growth;
  int on_device;
} negf_out;

/* Evaluate n_devs devices in one persistent launch (every (device, chain, energy) lane
 * of the batch, scheduled by the autotuned plan).  outs[i] receives device devs[i].
 * Results of a device are bitwise the same alone and inside any batch. */
int negf_compute(negf_ctx* ctx, const int* devs, int n_devs, negf_out* outs);

/* Per-energy ring traces for sampled checks of one device: for the real-axis energies
 * listed in idx_real (count k_real) Tr_r A_S and Tr_r A_D (k_real x n_rings each, summed
 * over chains, without degeneracy factors), and for contour nodes idx_cont (count k_cont)
 * Tr_r G (k_cont x n_rings complex).  Same kernels as negf_compute. */
int negf_sample_lanes(negf_ctx* ctx, int dev, int k_real, const int* idx_real, double* AS,
                      double* AD, int k_cont, const int* idx_cont, double* G);

/* Neutral reference electron count n0 per ring (Sec. 2.2.1, rho_0 with E_l = E_u = 0):
 * contour over [E_B, 0] with occupation 1 and zero potential in the device and leads. */
int negf_neutral_charge(negf_ctx* ctx, int dev, int n_cont, double E_B, double* n0);

/* Zero-bias conductance (Eq. zeroBiasG, Sec. 2.2.1) of n_devs devices in their current state:
 *   G = G_0 integral T(E) (-df/dE) dE  ~=  g_s (e^2/h) sum_k w_k T(E_k) (-df/dE)(E_k - mu),
 * with G_0 = g_s e^2/h (siemens), f the Fermi function at temperature kT (eV), and T(E) the
 * transmission (summed over chains with g_b) at the real-axis nodes E_k and weights w_k of
 * each device's grid.  Only the real-axis lanes are swept (T needs no contour); the sum runs
 * on the GPU in a fixed order, so a device gives the same bits alone or in a batch.  The grid
 * should cover mu -+ ~14 kT (e.g. negf_set_grid_spec with mu_S = mu_D = mu).  G: n_devs
 * doubles (host).  T: NULL, or host room for every device's n_real transmissions,
 * concatenated in the order of devs.  The device's other outputs are overwritten.  Errors:
 * NEGF_EINVAL (kT <= 0, non-finite mu, a device without real-axis energies or listed twice),
 * NEGF_ENOTFOUND, NEGF_EBUSY (a device in a self-consistent session). */
int negf_conductance(negf_ctx* ctx, const int* devs, int n_devs, double mu, double kT, double* G,
                     double* T);

/* ---- self-consistent loop (Alg. 3) with the 1D Poisson stand-in ------------------------ */

/* Poisson stand-in, one node per ring:
 *   U_i - U_G - (lam/dx)^2 (U_{i+1} - 2 U_i + U_{i-1}) = kappa (n_i - n0_i),
 * Dirichlet U_{-1} = U_S, U_N = U_D, U_G = phi_gate - V_GS.  kappa (eV per electron) of a
 * coaxial gate: negf_poisson_kappa. */
typedef struct {
  double kappa, dx_nm, lam_nm, phi_gate;
} negf_poisson;
double negf_poisson_kappa(double eps_r, double d_nm, double t_ox_nm, double dx_nm);

/* Bias point: lead potentials U_S = 0, U_D = -V_DS; mu_S = 0, mu_D = -V_DS. */
typedef struct {
  double V_DS, V_GS;
} negf_bias;

/* Broyden's modified second method: fraction zeta, history M (also the iteration limit),
 * tolerance on eps_max = max_i |n_in - n_out| / (n_in + n_out). */
typedef struct {
  double zeta;
  int M;
  double tol;
} negf_broyden;

/* Result of a solve.  n, U (n_rings), T (n_real), history (M) are caller arrays (NULL to
 * skip); converged, iterations, I are written. */
typedef struct {
  double* n;
  double* U;
  double* T;
  double* history;
  double I;
  int converged;
  int iterations;
} negf_sc_result;

/* Self-consistent solve of one device at one bias point, starting from potential U0
 * (n_rings): n_in = the charge whose Poisson solution is U0; then repeat
 * U = Poisson(n_in) -> n_out = NEGF(U) -> Broyden until eps_max < tol or M evaluations.
 * The grid of the device must already match the bias (negf_set_grid_spec).  The loop runs
 * on the device (one captured CUDA graph per iteration); the host reads one flag per
 * iteration.  Returns NEGF_ENOTCONVERGED (with the result filled) if the limit is hit. */
int negf_sc_solve(negf_ctx* ctx, int dev, const negf_bias* bias, const negf_poisson* pois,
                  const negf_broyden* br, const double* U0, negf_sc_result* res);

/* Stateful form of the same loop, for callers that interleave work or checkpoint.
 * negf_sc_begin: as negf_sc_solve up to the first iteration (bias, n0, starting charge,
 * Broyden state, captured graph); the device then refuses set-up calls (NEGF_EBUSY) until
 * negf_sc_end.  negf_sc_step: run k iterations; with state != NULL the host waits after
 * each one and stops early once it is nonzero (1 converged, 2 history exhausted); with
 * state == NULL the k iterations are only enqueued (iterations after convergence leave the
 * result unchanged).  negf_sc_end: wait, fill res (may be NULL), free the session; returns
 * NEGF_ENOTCONVERGED if res is given and the loop did not converge.
 * negf_sc_get_state / negf_sc_set_state: the Broyden state (n_in, n_in_old, f_old:
 * n_rings each; V, W: M x n_rings each, row j = column j of Alg. 3's V^T / W; m) for
 * checkpoint and warm start (Sec. 3.3 starts each V_gs from the previous solution). */
int negf_sc_begin(negf_ctx* ctx, int dev, const negf_bias* bias, const negf_poisson* pois,
                  const negf_broyden* br, const double* U0);
int negf_sc_step(negf_ctx* ctx, int dev, int k, int* state);
int negf_sc_end(negf_ctx* ctx, int dev, negf_sc_result* res);
int negf_sc_get_state(negf_ctx* ctx, int dev, double* n_in, double* n_in_old, double* f_old,
                      double* V, double* W, int* m);
int negf_sc_set_state(negf_ctx* ctx, int dev, const double* n_in, const double* n_in_old,
                      const double* f_old, const double* V, const double* W, int m);

/* Self-consistent solve of C channels with one Broyden vector (Sec. 2.3: the charge vectors
 * of several channel materials are concatenated, n = (n^1, ..., n^C), so eps_max and every
 * dot product of Alg. 3 run over all channels).  The channels are the devices devs[0..C-1]
 * (1 <= C <= 64), tubes of equal n_rings sharing contacts and gate, each with its grid set
 * from a grid spec (negf_set_grid_spec; a semi-adaptive grid is used as it stands, without
 * refinement).  Their Poisson stand-ins are coupled through the C x C row-major matrix K (eV
 * per electron per ring), which replaces pois->kappa:
 *   U_c,i - U_G - (lam/dx)^2 (U_c,i+1 - 2 U_c,i + U_c,i-1) = sum_c' K[c][c'] (n_c',i - n0_c',i)
 * (K[c][c] a tube's own gate-screened coupling, e.g. negf_poisson_kappa; K[c][c'] the
 * capacitive cross-coupling of two tubes at the same ring position: a stand-in for the
 * paper's 3D electrostatics, which couples the tubes through the shared field).  U0: C x
 * n_rings starting potentials (the loop starts from the charges whose coupled Poisson
 * solution is U0; K must be invertible).  All channels' sweeps run in one batched launch per
 * iteration, captured as one CUDA graph.  res: C results (n, U, T per channel; history,
 * iterations and converged are shared).  Returns NEGF_ENOTCONVERGED (results filled) if M
 * evaluations pass without eps_max < tol; NEGF_EINVAL for unequal ring counts, a device
 * listed twice, a singular or non-finite K. */
int negf_sc_solve_multi(negf_ctx* ctx, const int* devs, int n_channels, const negf_bias* bias,
                        const negf_poisson* pois, const double* K, const negf_broyden* br,
                        const double* U0, negf_sc_result* res);

/* ---- serving: continuous batching of self-consistent solves ----------------------------- */

/* A request: a mode-space (n_tube,0) nanotube of n_rings rings with n_modes subbands
 * (1 x 1 blocks, g_b = 2 each), bias point, grid sizes (Gauss-Legendre real axis on the
 * bias window, contour from E_B), Poisson and Broyden settings.  U0 (n_rings) may be NULL:
 * the loop then starts from the linear drop between the contacts. */
typedef struct {
  int n_rings, n_tube, n_modes;
  const int* modes;
  double t, kT, eta, E_B;
  int n_real, n_cont;
  negf_bias bias;
  negf_poisson pois;
  negf_broyden broyden;
  const double* U0;
} negf_request;

/* Queue a request (its arrays are copied); returns a ticket.  Requests are admitted into
 * device slots in arrival order while their estimated device memory fits the context's
 * hbm_budget_bytes (one request is always admitted); each scheduler step advances every
 * admitted request by one self-consistent iteration, all of them in one batched sweep
 * launch, and retires the finished ones.  A request's result is bitwise the same alone and
 * in any mix. */
int negf_submit(negf_ctx* ctx, const negf_request* req, uint64_t* ticket);
/* Run one scheduler step; *active receives the number of requests on the GPU. */
int negf_serve_step(negf_ctx* ctx, int* active);
/* NEGF_EBUSY while the request is queued or running; then fills res (n, U: n_rings; T:
 * n_real; history: iterations) and returns its status (NEGF_OK or NEGF_ENOTCONVERGED). */
int negf_poll(negf_ctx* ctx, uint64_t ticket, negf_sc_result* res);
/* Drive the scheduler until the request finished or timeout_ms passed (NEGF_ETIMEDOUT). */
int negf_wait(negf_ctx* ctx, uint64_t ticket, int timeout_ms, negf_sc_result* res);
/* Cancel a queued or running request; its slot is freed at the next step. */
int negf_cancel(negf_ctx* ctx, uint64_t ticket);
/* Host wall-clock times (s, steady clock) of submission, admission and completion. */
int negf_request_times(negf_ctx* ctx, uint64_t ticket, double* t_submit, double* t_start,
                       double* t_done);

/* ---- evaluation without allocation ------------------------------------------------------ */

/* One NEGF evaluation of a single mode-space chain (1 x 1 blocks) that allocates nothing.
 * The paper has no counterpart: it exists for callers that cannot allocate device memory
 * where they run (code building a CUDA graph, allocator-free embedding hosts, tools that
 * only hand over pre-registered buffers).  The caller owns every input and output; the
 * library's scratch (work items, per-item ring sums, forward-sweep staging) lives in one
 * fixed 32 MiB device array that every GPU loading the library reserves until exit.  Each
 * call made outside stream capture looks up that array's address with the device current;
 * a call on a stream under capture reuses the address of the device's last uncaptured call
 * (NEGF_EINVAL if there was none).  So make one call on each device before capturing, and
 * again after a cudaDeviceReset, which may move the array.  All calls share the array and
 * it keeps the last call's contents (what must start at zero is cleared on every call):
 * calls that overlap on the GPU race on it.  No cudaMalloc, cudaFree or other allocating
 * routine is called.
 *
 * stream: cudaStream_t to run on.  Device inputs: Hdiag (n_rings complex, H_{l,l} without
 * potential), U (n_rings), hsq (n_rings - 1, |H_{l,l+1}|^2), grid E, w, fS, fD (n_real) and
 * z, c (n_cont complex) as in negf_grid.  Host inputs: lead_S / lead_D = {a1, a2, at, U_lead}
 * with a1 = |H_{s1,s0}|^2, a2 = |H_{s2,s1}|^2, at = |tau|^2 of the scalar lead (its closed
 * form, as in negf_set_lead with m = 1).  Device outputs: n (n_rings, required), T (n_real)
 * and I (1) may be NULL.  Results equal negf_compute's for the same chain.  Returns
 * NEGF_ENOMEM when ceil(n_real/32) + ceil(n_cont/32) items with n_rings partial sums each,
 * plus the staging of one 8-warp block (n_rings x 8 KiB), do not fit in the 32 MiB array;
 * the call is asynchronous on `stream` otherwise. */
int negf_chain1_compute_noalloc(void* stream, int n_rings, const double* Hdiag, const double* U,
                                const double* hsq, double g_b, const double* lead_S,
                                const double* lead_D, int n_real, const double* E,
                                const double* w, const double* fS, const double* fD, double eta,
                                int n_cont, const double* z, const double* c, double* n,
                                double* T, double* I);

/* ---- diagnostics ---------------------------------------------------------------------- */

/* Number of kernel launches the context issued since creation (for accounting). */
int negf_launch_count(const negf_ctx* ctx, uint64_t* launches);

/* Kernel timing: with profiling on, every batched sweep issued outside graph capture is
 * bracketed by CUDA events on the context's stream; negf_kernel_time waits for them and
 * returns (and resets) the summed sweep time in ms and the number of timed sweeps. */
int negf_profile(negf_ctx* ctx, int enable);
int negf_kernel_time(negf_ctx* ctx, double* sweep_ms, uint64_t* sweeps);
/* With profiling on, the sweep of ring blocks wider than 2 also counts its lanes by update
 * form: lanes[0] real-axis lanes with the complex-symmetric G_ll update, lanes[1] real-axis
 * lanes with the general one, lanes[2] / lanes[3] the same for contour lanes.  Returns the
 * counts accumulated since the last call (or since profiling was switched on) and resets
 * them. */
int negf_sweep_lanes(negf_ctx* ctx, uint64_t lanes[4]);

/* The launch shape the autotuner last chose for ring blocks of width b with leads of m
 * sites in FP64 (fp32 = 0) or FP32 (fp32 = 1): CTA width in warps and resident CTAs per SM
 * (ctas_per_sm may be NULL); NEGF_EINVAL if that shape was not tuned. */
int negf_blk_width(negf_ctx* ctx, int fp32, int b, int m, int* warps, int* ctas_per_sm);
/* The CTA width (warps) the autotuner last chose for the thread-per-lane sweep of blocks of
 * width `block` (1 or 2) in FP64 (fp32 = 0) or FP32 (fp32 = 1); NEGF_EINVAL if none was tuned. */
int negf_chain_width(negf_ctx* ctx, int fp32, int block, int* warps);

/* Wave planner of the sweep split along the channel (host only; needs no device or context).
 * Split items are taken in order; consecutive items share a wave while their staging fits
 * `cap` bytes (an item alone may exceed it and then forms a wave of its own).  Item i has
 * stage[i] bytes of staging and n_seg[i] >= 1 segment records.  wave_of[i] receives the wave
 * of item i, *max_stage the largest staging of a wave and *max_records the most records a
 * wave holds: negf_compute sizes its record buffer by that figure for the partition it
 * finally uses (under an HBM budget, a partition at the budget's cap).  NEGF_EINVAL for a
 * negative size or cap, or a missing array. */
int negf_plan_seg_waves(int n, const long long* stage, const int* n_seg, long long cap, int* wave_of,
                        long long* max_stage, long long* max_records);

/* Measured FP64 FMA throughput of this GPU (TFLOP/s): a register-resident FMA loop over
 * every SM, best of three, for the FP64 roofline of the sweep kernels. */
int negf_fp64_peak(negf_ctx* ctx, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* NEGF_H */
