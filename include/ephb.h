/*
 * ephb.h -- C ABI of the GB300 e-ph scattering + coupled-BTE library.
 *
 * The library computes, on one CUDA GPU, the hot path of the coupled electron-phonon
 * Boltzmann transport method of arXiv 2109.08547:
 *   - Wannier-to-Bloch interpolation of H, D and the e-ph vertex g (section
 *     "Electrons, phonons, and interactions", Eqs. H_mn(k), D_ss'(q), g^smn_kq);
 *   - transition rates X^+/X^- over irreducible k x full q inside the transport window
 *     (Eq. X^e-ph) and the phonon-side rates Y (Eq. Y^ph-e);
 *   - the RTA, self and drag terms and the unified single-iterator coupled solution with
 *     the Kelvin-Onsager correction (section "Coupled and decoupled BTEs" and
 *     "Transport coefficients");
 *   - the transport coefficient tensors (Eqs. sigma/sigmaS, alpha_el/kappa0_el,
 *     alpha_ph/kappa_ph).
 *
 * Conventions for every call:
 *   - All pointers in argument structs are HOST pointers; the library copies what it
 *     needs during the call and keeps no reference to caller memory.
 *   - All device memory is owned by the context and released by ephb_destroy.
 *   - Every kernel runs on the context's stream (the stream given to ephb_create, or a
 *     stream the context creates when NULL is given).  Calls return after the work they
 *     enqueue has completed, unless stated otherwise.
 *   - No call aborts or throws; failures return a status and set a message readable with
 *     ephb_last_error.  Calls made in the wrong order return EPHB_ESTATE.
 *   - There is no CPU fallback: every numerical step runs in the library's CUDA kernels.
 *
 * Units: energies eV, lengths Angstrom, temperatures K, rates 1/s, velocities m/s,
 * coefficient tensors SI (sigma S/m, S V/K, kappa W/(m K), alpha A/m), row-major 3x3.
 */
#ifndef EPHB_H
#define EPHB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ephb_ctx ephb_ctx;

typedef enum {
  EPHB_OK = 0,
  EPHB_EINVAL = 1,     /* bad argument (sizes, pointers, unsupported option)           */
  EPHB_ENOMEM = 2,     /* device or host allocation failed                             */
  EPHB_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed                  */
  EPHB_ESTATE = 4,     /* call made before the calls it depends on                     */
  EPHB_ENOCONV = 5,    /* iteration limit reached; outputs hold the last iterate       */
  EPHB_ETIMEOUT = 6,   /* a bounded device-side wait gave up                           */
  EPHB_EINTERNAL = 7
} ephb_status;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t (or NULL
 * for a context-owned stream).  On success *out receives the context. */
ephb_status ephb_create(ephb_ctx **out, int device, void *cuda_stream);

/* Release every device buffer of the context.  NULL is accepted. */
void ephb_destroy(ephb_ctx *ctx);

/* Message of the last failed call on ctx (valid until the next call on ctx). */
const char *ephb_last_error(const ephb_ctx *ctx);

/* ----------------------------------------------------------------------------------
 * Wannier model (section "Electrons, phonons, and interactions").
 *   H(k)   = sum_r exp(i 2pi k.Re[r]) H_R[r]                     (Eq. H_mn(k))
 *   D(q)   = sum_r exp(i 2pi q.Rd[r]) D_R[r]                     (Eq. D_ss'(q), short range)
 *   g^s_mn(k,q) = sqrt(omega_ref/hbar w_sq) sum_{m'n'alpha} c*_{n'n}(k') c_{m'm}(k)
 *          [sum_{re,rp} exp(i 2pi (k.Rge[re] + q.Rgp[rp])) g_R[re][rp][m'][n'][alpha]]
 *          u_{alpha s}(q) / sqrt(mass[alpha/3]/mean mass)          (Eq. g^smn_kq)
 * with c the eigenvector columns of H (the paper's U_k = c^dagger) and u those of D.
 * The 1/N_e, 1/N_ph and Wigner-Seitz weights are taken as already folded into the arrays.
 * Complex arrays are interleaved (re, im) doubles, row-major in the order shown.
 * --------------------------------------------------------------------------------*/
typedef struct {
  double lattice[3][3];        /* rows a1, a2, a3 (Angstrom)                               */
  int nat;                     /* atoms per cell; branches = 3*nat (<= 12)                 */
  const double *mass_amu;      /* [nat]                                                    */
  const double *tau_cart;      /* [nat][3] Angstrom (informational)                        */
  int nb;                      /* Wannier bands (<= 8)                                     */
  int nRe;                     /* Hamiltonian R vectors                                    */
  const int32_t *Re;           /* [nRe][3] integer crystal coordinates                     */
  const double *H_R;           /* [nRe][nb][nb] complex, eV                                */
  int nRd;
  const int32_t *Rd;           /* [nRd][3]                                                 */
  const double *D_R;           /* [nRd][3nat][3nat] complex, eV^2 (mass scaled)            */
  int nRge, nRgp;
  const int32_t *Rge;          /* [nRge][3]                                                */
  const int32_t *Rgp;          /* [nRgp][3]                                                */
  const double *g_R;           /* [nRge][nRgp][nb][nb][3nat] complex, eV                   */
  double omega_ref_eV;         /* hbar*omega at which g_R is quoted                        */
  int nsym;                    /* point operations (1..48); 1 = identity only              */
  const int32_t *sym_rot;      /* [nsym][3][3] integer, acting on reciprocal crystal k     */
  const double *sym_cart;      /* [nsym][3][3] the same operations on Cartesian vectors    */
  double spin_deg;             /* d_s                                                      */
  double bg_rate_coeff;        /* phonon background rate W_bg = coeff (w/w_bg)^2 (T/T_bg)  */
  double bg_omega_ref_eV;
  double bg_T_ref;
} ephb_model;

/* Validate and copy the model to the device.  Resets meshes, rates and solutions.
 * EPHB_EINVAL for an out-of-range size, a non-group operation list, non-positive masses or
 * scalars, or a lattice-vector component (Re, Rd, Rge, Rgp) outside +-65535. */
ephb_status ephb_set_wannier_model(ephb_ctx *ctx, const ephb_model *model);

/* ----------------------------------------------------------------------------------
 * Meshes, bands, phonons, irreducible wedge and transport window
 * (Eqs. H_mn(k), v_mk, D_ss'(q), v_sq; section "Workflow and structure": symmetry,
 * window-restricted IBZ).  Gamma-centred meshes; the k mesh must be an integer multiple
 * of the q mesh per dimension, and cubic (n x n x n) when nsym > 1.  An electron state
 * is active when window_lo <= eps <= window_hi.  Modes with hbar w <= omega_min are
 * excluded from every rate and sum.  Velocities and |g|^2 are averaged over degenerate
 * subspaces (|d eps| < degen_tol).
 * --------------------------------------------------------------------------------*/
typedef struct {
  int kmesh[3];
  int qmesh[3];
  double window_lo_eV, window_hi_eV;
  double degen_tol_eV;         /* default 1e-6 */
  double omega_min_eV;         /* default 1e-4 */
} ephb_mesh_opts;

typedef struct {
  int64_t nk, nq;              /* full mesh sizes                                          */
  int64_t n_active_states;     /* active (k,m) on the full k mesh                          */
  int64_t n_ibz;               /* irreducible points of the k mesh                         */
  int64_t n_ibz_window;        /* irreducible points with an active band                   */
  int64_t n_pairs;             /* (irreducible-window k, q) with an active band at k+q     */
  double ms;                   /* device time of the call (CUDA events)                    */
} ephb_mesh_info;

ephb_status ephb_build_meshes_ibz(ephb_ctx *ctx, const ephb_mesh_opts *opts, ephb_mesh_info *out);

/* ----------------------------------------------------------------------------------
 * Transition rates (Eq. X^e-ph, with Y^ph-e = X^+ N_q/N_k for the phonon side):
 *   X^+ = 2pi/(hbar N_q) |g|^2 f_mk (1-f_nk') n_sq     delta(eps_nk' - eps_mk - hbar w_sq)
 *   X^- = 2pi/(hbar N_q) |g|^2 f_mk (1-f_nk') (1+n_sq) delta(eps_nk' - eps_mk + hbar w_sq)
 * for every irreducible-window k, active m, q with k' = [k+q], active n and branch s.
 * delta is a Gaussian of standard deviation sigma, exactly zero beyond cutoff*sigma; an
 * entry is stored when either argument is within the cut.
 *
 * Instances.  inst[0..ninst-1] (1 <= ninst <= EPHB_MAX_INSTANCES) are (T, mu, window)
 * right-hand sides on the same meshes.  An instance's window [window_lo_eV, window_hi_eV] is
 * clipped to the mesh window; window_lo_eV >= window_hi_eV means the mesh window.  A state is
 * active for an instance when it is active on the meshes and its energy lies in the instance
 * window.  With one instance on the mesh window the rates are computed directly.  Otherwise
 * |g|^2 and delta (which do not depend on T or mu) are interpolated once, over the mesh window,
 * as V+- = 2pi/(hbar N_q)|g|^2 delta(...), and every instance keeps the entries whose two
 * states lie in its window, with X+- = V+- f (1-f') {n, 1+n} from its own T and mu (the
 * vertex reuse across temperatures and chemical potentials of section "Workflow and
 * structure").  Degenerate averages of |g|^2 are then taken over the bands active on the
 * meshes.  Every later call acts on all instances (solve) or names one (coefficients,
 * ephb_select_instance for the array views).
 * --------------------------------------------------------------------------------*/
typedef struct {
  double T_K, mu_eV;
  double window_lo_eV, window_hi_eV;   /* instance window; lo >= hi: the mesh window           */
} ephb_thermo;
#define EPHB_MAX_INSTANCES 64
/* Energy-conserving delta of Eq. X^e-ph.  kind EPHB_DELTA_GAUSS: Gaussian of standard deviation
 * sigma_eV, zero beyond cutoff_sigmas standard deviations (readings [A10], [A11]).  kind
 * EPHB_DELTA_TETRA: the analytic (linear) tetrahedron method of "Workflow and structure": the
 * energy balance eps_n(k + q) - eps_m(k) -/+ hbar w_s(q) is interpolated linearly in the six
 * tetrahedra of every cube of the q mesh and (1/N_q) delta becomes the weight of the mesh point
 * q in that zone integral (reading [A22]); sigma_eV and cutoff_sigmas are ignored.  A zeroed
 * struct's kind is the Gaussian. */
#define EPHB_DELTA_GAUSS 0
#define EPHB_DELTA_TETRA 1
typedef struct {
  double sigma_eV, cutoff_sigmas;
  int kind;
} ephb_delta;
/* Precision of the R_ph contraction of the vertex (the largest part of the work):
 *   EPHB_FP64         FP64 on the CUDA cores.
 *   EPHB_FP64_SLICED  tensor cores (tcgen05, BF16 in, FP32 accumulate) on exact fixed-point
 *                     slices: operands rounded to 2^-55 of their scale and split into 7 slices
 *                     of 8 bits, the 28 slice products of the leading diagonals, the four
 *                     largest diagonals each kept in an accumulator where the FP32 sums are
 *                     exact; FP64-grade results.  Needs 2 nRgp <= 256 (EPHB_EINVAL otherwise).
 *   EPHB_SPLIT_BF16   4 slices, the leading diagonal exact, the rest in one FP32 accumulator,
 *                     and the band/branch rotations of the epilogue in FP32 (mixed precision,
 *                     ~1e-7 relative).  Needs 2 nRgp <= 1024.
 *   EPHB_SPLIT_TF32   not available (EPHB_EINVAL).
 * In both tensor-core modes the stage-A contraction (R_e sum) runs on the tensor cores in the
 * FP64-grade 7-slice form when 2 nRe <= 256 (else in FP64).  |g|^2 averages, occupations and
 * delta stay FP64 in every mode, and so do the rotations except in EPHB_SPLIT_BF16. */
typedef enum { EPHB_FP64 = 0, EPHB_SPLIT_TF32 = 1, EPHB_SPLIT_BF16 = 2, EPHB_FP64_SLICED = 3 } ephb_precision;

typedef struct {
  int64_t n_tuples;            /* (k m, q, n, s) tuples interpolated and delta-weighted    */
  int64_t n_entries;           /* stored electron-side entries (rows: k, m)                */
  int64_t n_ph_entries;        /* stored phonon-side entries (rows: q, s)                  */
  int64_t n_pairs;
  double ms;                   /* device time of the call (CUDA events)                    */
  double ms_stage_a;           /* device time of the R_e contraction kernels               */
  double ms_stage_b;           /* device time of the R_ph contraction + rate kernels       */
  double stage_a_flops;        /* algorithmic flops of the R_e contraction                 */
  double stage_b_flops;        /* algorithmic flops of the R_ph contraction + rotations    */
  double ms_epilogue;          /* tensor-core modes: device time of the rotation/rate kernel */
  double tensor_flops;         /* tensor-core modes: flops issued as tcgen05.mma by the
                                  stage-B contraction (the work ms_gemm times)              */
  double rot_flops;            /* algorithmic flops of the band and branch rotations       */
  double ms_gemm;              /* tensor-core modes: device time of the tcgen05 GEMM kernel  */
  int tc_cols;                 /* tensor-core modes: column-chunk width used               */
  int autotuned;               /* 1 if this call chose the tile shape by timing candidates */
  int tc_kblock;               /* tensor-core modes: K per shared-memory stage             */
  int tc_stages;               /* tensor-core modes: shared-memory stages (K16 x 2: 2 CTAs/SM;
                                  K16 x 5: the persistent warp-specialised form)          */
  double tensor_flops_a;       /* flops issued as tcgen05.mma by stage A (tensor cores)    */
} ephb_rates_info;

ephb_status ephb_compute_transition_rates(ephb_ctx *ctx, const ephb_thermo *inst, int ninst,
                                          const ephb_delta *delta, ephb_precision precision,
                                          ephb_rates_info *out);

/* ----------------------------------------------------------------------------------
 * Coupled BTE (section "Coupled and decoupled BTEs"; Kelvin-Onsager correction from
 * "Transport coefficients").  Iteration 0 is the RTA.  Each later (phonon) iteration
 * sets F = F0 + dF^D[I], G = dG^D[J]; iterates the electron equations
 * I = I0 + dI^S[I] + dI^D[F], J = J0 + dJ^S[J] + dJ^D[G] until the electron tensors
 * change by less than inner_tol; then (ko_correction) replaces I by I_diff + lambda I_drag
 * with lambda the least-squares solution of sigmaS_drag[lambda I_drag] = alpha_ph/T.
 * Convergence: max relative Frobenius change of the coefficient tensors < tol.
 * The phonon background W_bg stands in for ph-ph and ph-isotope scattering, whose self
 * terms are therefore absent.
 * --------------------------------------------------------------------------------*/
typedef enum { EPHB_RTA = 0, EPHB_PARTIAL = 1, EPHB_DRAGLESS = 2, EPHB_DRAGGED = 3 } ephb_level;
/* Arithmetic of the electron loop.
 *   EPHB_SOLVE_FP64   plain FP64 Jacobi sweeps (the paper's iteration).
 *   EPHB_SOLVE_MIXED  iterative refinement: every FP64 sweep x' = b + A x supplies the
 *                     residual r = x' - x and the convergence test of the electron loop; then
 *                     12 FP32 sweeps of d <- r + A d (FP32 run weights) and x <- x + d before the
 *                     next FP64 sweep.  At the dragged level the electron loop of an outer
 *                     iteration stops at 1e-2 of the previous outer residual (1e-2 in the
 *                     first), never before inner_tol, and the solve ends only after an outer
 *                     iteration whose electron loop reached inner_tol.  Same fixed point and
 *                     outer test; fewer sweeps.  At the dragged level the phonon scatter and
 *                     the drag term of an outer iteration begun with the outer residual at or
 *                     above 1e-5 run in FP32 (FP32 copies of X, Y, I, J, F, G; FP64 partial
 *                     sums across segments); later ones in float-float arithmetic (pairs of
 *                     FP32 numbers, ~2^-47 relative, on the FP32 pipe), and the solve ends
 *                     only after an outer iteration with both in float-float.  The phonon
 *                     update, KO step and coefficients stay FP64. */
typedef enum { EPHB_SOLVE_FP64 = 0, EPHB_SOLVE_MIXED = 1 } ephb_solve_precision;

typedef struct {
  int level;                   /* ephb_level                                               */
  double tol;                  /* outer tolerance (e.g. 1e-10)                             */
  double inner_tol;            /* electron loop tolerance (<= 0: 0.1*tol)                  */
  int max_outer, max_inner;
  int ko_correction;           /* 1: apply the Kelvin-Onsager step (dragged levels)        */
  int warm_start;              /* 1: start from ephb_set_warm_start's responses where set   */
  int precision;               /* ephb_solve_precision                                     */
  int accel_depth;             /* 0: the plain outer iteration (the paper's).  1..EPHB_MAX_ACCEL_DEPTH:
                                  Anderson acceleration of the outer iteration (dragged level
                                  only) with that history depth m over the iterate x = (F, G):
                                  the last m+1 phonon updates g_j and residuals f_j = g_j - x_j
                                  are kept, and from the third outer iteration on the electrons
                                  are solved against sum_j alpha_j g_j with alpha minimising
                                  |sum_j alpha_j f_j| (F and G parts weighted by the first
                                  residual's) subject to sum_j alpha_j = 1; a singular or
                                  ill-bounded system falls back to the newest g alone.  Same
                                  fixed point and convergence test as the plain iteration.
                                  Outside 0..EPHB_MAX_ACCEL_DEPTH: EPHB_EINVAL.              */
  int device_loop;             /* 0: the host drives the loops (a residual read back after
                                  every FP64 sweep and every outer iteration).  1: the whole
                                  solve of every instance is ONE CUDA graph launch: the outer
                                  iteration and the electron loop are conditional WHILE nodes
                                  and the choices (phonon-side arithmetic, converged or
                                  correct) SWITCH nodes, whose conditions one-thread kernels
                                  set from the residuals on the device; each instance is an
                                  independent branch, so all instances' sweeps are in flight
                                  together.  Same kernels in the same order per instance:
                                  bit-identical answers and counts.  Needs accel_depth 0 and
                                  a level other than EPHB_RTA (otherwise EPHB_EINVAL).  The
                                  graph is kept and launched again while the instances'
                                  buffers, sizes and options are unchanged.  The per-kernel
                                  times of ephb_solve_info are not measured in this mode (0);
                                  ms is the device time of the launch.  A loop that runs past
                                  600 s on the device stops and the call returns
                                  EPHB_ETIMEOUT.  When the instances derive their lists at
                                  solve time (memory bound), each instance is one launch.   */
} ephb_solve_opts;
#define EPHB_MAX_ACCEL_DEPTH 8

typedef struct {
  int outer_iters;
  int inner_iters_total;
  int converged;
  int n_zero_rate_states;      /* active states without partners (I = J = 0)              */
  double residual;             /* last outer residual                                      */
  double lambda;               /* last Kelvin-Onsager scalar (1 if not applied)            */
  int64_t n_sweeps;            /* electron sweeps performed                                */
  double ms;                   /* device time of the call                                  */
  double ms_e_sweep;           /* summed device time of the electron sweep kernels         */
  double ms_ph_sweep;          /* summed device time of the phonon drag sweep kernels      */
  double e_sweep_bytes;        /* algorithmic HBM bytes of one electron sweep              */
  double ms_drag;              /* summed device time of the electron drag-term kernels     */
  int64_t n_runs;              /* partner runs: entries of a row merged over branches      */
  double ms_self_kernel;       /* summed device time of the self-term gather kernel alone  */
  double e_sweep_flops;        /* algorithmic FP64 flops of one self-term sweep            */
  int64_t n_sweeps32;          /* FP32 correction sweeps (EPHB_SOLVE_MIXED)                */
  double ms_corr;              /* device time of the FP32 corrections                      */
  int outer_iters32;           /* outer iterations whose phonon scatter and drag term ran in
                                  FP32 (EPHB_SOLVE_MIXED, dragged level: those begun with the
                                  outer residual at or above 1e-5; never the last one)      */
  int graph_launches;          /* device_loop: graph launches of the call (0: host-driven)   */
  int graph_reused;            /* device_loop: 1 if the graph of the previous call was reused */
} ephb_solve_info;

/* Solves every instance.  `out` (optional) sums the counts and device times over the
 * instances and keeps the largest residual and outer-iteration count; converged is 1 only if
 * every instance converged, else the call returns EPHB_ENOCONV after solving all of them. */
ephb_status ephb_solve_coupled_bte(ephb_ctx *ctx, const ephb_solve_opts *opts, ephb_solve_info *out);

/* ---- Electron-charged-impurity (e-chimp) scattering -----------------------------------
 * "Electrons, phonons, and interactions", Eqs. |g^e-chimp_q|^2, q_TF^2 and X^e-chimp: the
 * dopants' screened Coulomb potential in the first Born approximation,
 *   |g_q|^2 = (1/V) sum_i n_i [Z_i e / (eps0 eps (q^2 + q_TF^2))]^2,
 *   q_TF^2  = d_s e^2 / (k_B T N_k V eps0 eps) sum_{mk} f (1 - f)   (every band, full k mesh),
 *   X^e-chimp_{mk -> nk'} = 2 pi/(hbar N_k) |g_q|^2 (1 - k.k'/(k k')) f (1 - f) delta(eps' - eps),
 * q = [k' - k], V the cell volume.  It enters the electron RTA rate W^RTA only (Matthiessen's
 * rule, Eq. W^RTA_mk): its transport factor stands for the elastic in-scattering, so the self
 * term keeps the e-ph rates alone.  Readings: k, k' and q are the Cartesian vectors of the
 * centred crystal coordinates (each in [-1/2, 1/2); for a cubic lattice q is then measured from
 * the nearest zone centre); a zero-length k or k' has transport factor 1; the final states are
 * the window's, as for the e-ph rates; delta is the rates call's Gaussian (its sigma_eV and
 * cutoff_sigmas, also with the tetrahedron kind).  The rates are made at each instance's next
 * solve, one warp per state over every k' of the mesh.  Errors: EPHB_EINVAL for n_species
 * outside 0..EPHB_MAX_DOPANTS, a negative concentration or eps_r <= 0; a solve returns
 * EPHB_EINVAL if the rates call had no positive sigma_eV and cutoff_sigmas. */
#define EPHB_MAX_DOPANTS 4
typedef struct {
  int n_species;                   /* 0: no charged impurities (the default)                */
  double n_cm3[EPHB_MAX_DOPANTS];  /* dopant concentrations n_i, cm^-3                       */
  double Z[EPHB_MAX_DOPANTS];      /* their ionizations Z_i                                  */
  double eps_r;                    /* zero-frequency dielectric constant of the host         */
} ephb_impurities;
/* Sets (NULL or n_species = 0: clears) the charged impurities; every instance's RTA terms are
 * made again at its next solve. */
ephb_status ephb_set_impurities(ephb_ctx *ctx, const ephb_impurities *imp);

/* ---- Phonon-isotope (Tamura) scattering ----------------------------------------------
 * "Electrons, phonons, and interactions", Eq. W^ph-x: on-site mass defects in the first Born
 * approximation.  Its part of the phonon RTA rate (Eq. W^RTA_sq, Matthiessen's rule; the paper's
 * phonon self term sums the ph-ph rates alone) is
 *   W^iso_sq = pi (hbar w_sq)^2 / (2 hbar N_q) sum_tau g_tau sum_{s'q'} |xi*_{tau,sq} . xi_{tau,s'q'}|^2
 *              delta(hbar w_s'q' - hbar w_sq),
 * xi the eigenvectors of the mass-scaled dynamical matrix, g_tau the mass-variance parameter of
 * atom tau.  Readings: the rate carries 1/N_q (the printed formula omits it; a mesh sum needs
 * it, as Eq. X^e-ph has it); modes at or below omega_min take no part; delta is the rates call's
 * Gaussian; the rate is averaged over the degenerate group of sq.  Computed at each instance's
 * next solve, one block per q representative over every q' of the mesh, the other q taking
 * their representative's rates.  g: nat values (nat = the model's atoms, at most 4; NULL or
 * nat = 0 clears).  Errors: EPHB_EINVAL for nat outside 0..4 or a negative g; a solve returns
 * EPHB_EINVAL if nat differs from the model's or the rates call had no positive Gaussian. */
ephb_status ephb_set_isotopes(ephb_ctx *ctx, const double *g, int nat);
/* The last solve of one instance. */
ephb_status ephb_instance_solve_info(ephb_ctx *ctx, int inst, ephb_solve_info *out);

/* ----------------------------------------------------------------------------------
 * Learned warm start (an extension: the paper starts the iteration from the RTA).
 * A network proposes, per electron state, coordinates a = (a_I, a_J) of the responses along
 * the RTA direction J0 = v/W; the next solve of the instance (opts.warm_start = 1) then starts
 * from I = I0 + a_I k_B J0, J = J0 (1 + a_J) instead of I0, J0 (a = 0 is the RTA start), with
 * the phonons from the RTA as before.  The iteration
 * and its convergence test are unchanged, so the answer is the same to the tolerance; if the
 * warm-started solve does not converge, the instance is solved again from the RTA start.
 * States: the n_states = ephb_num_states() electron states (irreducible-window k x band) of
 * the meshes; inactive states get zero inputs and are ignored.
 *   features: EPHB_NFEAT floats per state: (eps-mu)/kT clipped to +-40 and divided by 10,
 *             log10(W_RTA) - 13,
 *             |v|/max|v|, T/300 K, mu/0.1 eV, eps/0.3 eV (device, FP32, [n_states][6]).
 *   targets:  after a solve, a_I = (I.J0)/(J0.J0)/k_B - (eps-mu)/(k_B T) and
 *             a_J = (J.J0)/(J0.J0) - 1 per state (0 where J0 = 0 or |v| < 1e-6 max|v|).
 * All pointers are device pointers owned by the caller.
 * --------------------------------------------------------------------------------*/
#define EPHB_NFEAT 6
int64_t ephb_num_states(const ephb_ctx *ctx);
ephb_status ephb_state_features(ephb_ctx *ctx, int inst, float *feat_dev, int64_t n_states);
ephb_status ephb_state_targets(ephb_ctx *ctx, int inst, float *targ_dev, int64_t n_states);
/* scale_dev = NULL clears the instance's warm start. */
ephb_status ephb_set_warm_start(ephb_ctx *ctx, int inst, const float *scale_dev, int64_t n_states);

/* The network: n_in inputs, depth hidden tanh layers of the given width, n_out linear outputs;
 * FP32 master parameters (layer by layer: W [fan_out][fan_in] row-major, then b), Glorot
 * uniform weights from a counter-based generator (splitmix64 of seed and index), zero biases.
 * Products take BF16-rounded operands with FP32 accumulation (ephb_mlp_set_bf16(net, 0): FP32
 * operands).  Loss 1/(2n) sum |y - t|^2.  Training: full-batch Adam (0.9, 0.999, 1e-8). */
typedef struct ephb_mlp ephb_mlp;
ephb_status ephb_mlp_create(ephb_mlp **out, int device, void *cuda_stream, int n_in, int width, int depth, int n_out,
                            uint64_t seed);
void ephb_mlp_destroy(ephb_mlp *net);
const char *ephb_mlp_last_error(const ephb_mlp *net);
int64_t ephb_mlp_num_params(const ephb_mlp *net);
ephb_status ephb_mlp_set_bf16(ephb_mlp *net, int on);
ephb_status ephb_mlp_get_params(ephb_mlp *net, float *host, int64_t n);
ephb_status ephb_mlp_set_params(ephb_mlp *net, const float *host, int64_t n);   /* also resets Adam */
/* y_dev [n][n_out] = net(x_dev [n][n_in]) */
ephb_status ephb_mlp_forward(ephb_mlp *net, const float *x_dev, int64_t n, float *y_dev);
/* loss (host, optional) and its gradient (device [num_params], optional) on (x, t) */
ephb_status ephb_mlp_loss_grad(ephb_mlp *net, const float *x_dev, const float *t_dev, int64_t n, float *loss_host,
                               float *grad_dev);
/* one Adam step of learning rate lr on the full batch (x, t); loss before the step */
ephb_status ephb_mlp_train_step(ephb_mlp *net, const float *x_dev, const float *t_dev, int64_t n, float lr,
                                float *loss_host);

/* ----------------------------------------------------------------------------------
 * Transport coefficients of the current responses (Eqs. sigma/sigmaS,
 * alpha_el/kappa0_el, alpha_ph/kappa_ph with 1/N_k and 1/N_q on the zone sums):
 *   sigma, sigmaS = d_s e/(V N_k k_B T) sum_{mk} f(1-f) v (x) {J, -I}
 *   alpha_el, kappa0_el = -d_s/(V N_k k_B T) sum (eps-mu) f(1-f) v (x) {J, -I}
 *   alpha_ph, kappa_ph = 1/(V N_q k_B T) sum_{sq} hbar w n(1+n) v (x) {-G, F}
 *   S = sigma^-1 sigmaS, kappa_el = kappa0_el - alpha_el S.
 * `out` is caller-owned host memory.  inst selects the instance (0 <= inst < ninst).
 * --------------------------------------------------------------------------------*/
typedef struct {
  double sigma[9], sigmaS[9], S[9], alpha_el[9], kappa0_el[9], kappa_el[9], alpha_ph[9], kappa_ph[9];
} ephb_coeffs;

ephb_status ephb_transport_coefficients(ephb_ctx *ctx, int inst, ephb_coeffs *out);

/* ----------------------------------------------------------------------------------
 * Inspection: borrowed views of the context's device arrays (valid until the next call
 * that rebuilds them) and a copy into caller host memory.  Shapes are reported in
 * shape[0..3] (unused dimensions 1); dtype codes: 0 f64, 1 c128, 2 i32, 3 i64, 4 u32.
 * --------------------------------------------------------------------------------*/
typedef enum {
  EPHB_ARR_EPS = 0,            /* [nk][nb] f64                                             */
  EPHB_ARR_VEL = 1,            /* [nk][nb][3] f64                                          */
  EPHB_ARR_OMEGA = 2,          /* [nq][nbr] f64                                            */
  EPHB_ARR_VPH = 3,            /* [nq][nbr][3] f64                                         */
  EPHB_ARR_IBZ_REP = 4,        /* [nk] i32 full index of the representative                */
  EPHB_ARR_IBZ_OP = 5,         /* [nk] i32 first operation S with S<k> = k                 */
  EPHB_ARR_IBZW_LIST = 6,      /* [n_ibz_window] i32 full index of each irreducible point  */
  EPHB_ARR_ROW_PTR = 7,        /* [n_ibz_window*nb + 1] i64 electron rows (k,m)            */
  EPHB_ARR_ENTRY_KPNS = 8,     /* [n_entries] u32: k' | n<<21 | s<<25                      */
  EPHB_ARR_ENTRY_X = 9,        /* [n_entries][2] f64: X^+, X^-                             */
  EPHB_ARR_PAIR_Q = 10,        /* [n_pairs] i32 q of each pair                             */
  EPHB_ARR_W_E = 11,           /* [n_ibz_window*nb] f64 electron W^RTA (0 when inactive)   */
  EPHB_ARR_W_PH = 12,          /* [nq][nbr] f64 phonon W^RTA                               */
  EPHB_ARR_I = 13,             /* [n_ibz_window*nb][3] f64                                 */
  EPHB_ARR_J = 14,
  EPHB_ARR_F = 15,             /* [nq][nbr][3] f64                                         */
  EPHB_ARR_G = 16,
  EPHB_ARR_PAIR_PTR = 17,      /* [n_ibz_window + 1] i64                                   */
  EPHB_ARR_ACTIVE = 18,        /* [nk] u32 bit mask of active bands                        */
  EPHB_ARR_STATE_EPS = 19,     /* [n_ibz_window*nb] f64 band energy of each state          */
  EPHB_ARR_STATE_VEL = 20,     /* [n_ibz_window*nb][3] f64 velocity of each state          */
  EPHB_ARR_STATE_WEIGHT = 21,  /* [n_ibz_window*nb] f64 1/|stabiliser| (0 when inactive)   */
  EPHB_ARR_COUNT = 22
} ephb_array;

/* Tuning.  EPHB_TUNE_TC_COLS: tile shape of the tensor-core R_ph contraction (the tile is
 * 128 (k,q) pairs x width columns, K streamed in stages of kblock).  0 (default): the first
 * tensor-core rates call of a context times the candidate shapes on its first chunk (FP64-grade:
 * widths 48/64/96 with two K stages of 32 and one CTA per SM, width 48 with two stages of 16
 * and two CTAs per SM, width 96 with four stages of 16; mixed: 64/128/256, 128 with two CTAs
 * per SM, 256 with four stages) and keeps the fastest for the
 * context; setting 0 again re-tunes.  Otherwise the given width (a multiple of 16, at most
 * 96 / 256) is used with stages of 32.  The results do not depend on the shape. */
#define EPHB_TUNE_TC_COLS 0
/* EPHB_TUNE_WITHHOLD_MMA (value 1): the stage-B contraction issues no tensor-core MMA, so the
 * barriers its CTAs wait on never complete; every wait gives up after its 2 s bound, the CTAs
 * record the timeout, free their tensor memory and return, and the rates call returns
 * EPHB_ETIMEOUT with the context still usable.  It exists to check that failure path; value 0
 * restores normal operation. */
#define EPHB_TUNE_WITHHOLD_MMA 1
/* EPHB_TUNE_DEFER_INSTANCES, value 1: with several instances, compute_transition_rates keeps the
 * union lists only and every instance derives its own lists when the solve reaches it, releasing
 * them (and its sweep arrays) after its solve; the responses, RTA rates and coefficient inputs
 * stay.  This is what the library does by itself when the instances' lists would exceed half of
 * the free device memory; the key forces it (the results are the same).  Value 0: automatic. */
#define EPHB_TUNE_DEFER_INSTANCES 2
/* EPHB_TUNE_STAGE_A_TMEM_A, value 1: the tensor-core stage A (R_e contraction) copies its A
 * slices into tensor memory once per K step (tcgen05.cp) and the products read them there
 * instead of from shared memory; before overwriting an A buffer it waits for the products that
 * read it.  Value 0 (default): every product reads its A slice from shared memory, which
 * measured faster.  The results are bit-identical. */
#define EPHB_TUNE_STAGE_A_TMEM_A 3
ephb_status ephb_set_tuning(ephb_ctx *ctx, int key, int value);

/* Make instance inst the one whose arrays the views and copies below return (and the one
 * whose solution a later solve leaves in place).  EPHB_EINVAL if inst is out of range. */
ephb_status ephb_select_instance(ephb_ctx *ctx, int inst);
/* Number of instances of the last compute_transition_rates call (1 before any). */
int ephb_num_instances(const ephb_ctx *ctx);
ephb_status ephb_get_device_array(ephb_ctx *ctx, int which, void **dptr, int64_t shape[4], int *dtype);
ephb_status ephb_copy_array_to_host(ephb_ctx *ctx, int which, void *host_dst, int64_t nbytes);

/* Number of CUDA kernels the library has launched in this process (all contexts). */
int64_t ephb_kernel_launches(void);

/* Accuracy check of the library's float-float exponential, the e^(-x^2/2 sigma^2) of the
 * Gaussian delta weights (Eq. X^e-ph, reading [A10]) in the FP64-grade rate epilogue:
 * out_dev[i] = e^(y_dev[i]) for -60 <= y <= 0, the input taken as a float-float pair (nearest
 * FP32 and nearest FP32 of the remainder) and the result returned as hi + lo in FP64.  Device
 * pointers of n doubles; the work is enqueued on cuda_stream (NULL: the legacy default
 * stream).  EPHB_EINVAL for n < 0 or a NULL pointer with n > 0, EPHB_ECUDA for a launch
 * failure. */
ephb_status ephb_selftest_exp_ff(const double *y_dev, double *out_dev, int64_t n, void *cuda_stream);

/* ----------------------------------------------------------------------------------
 * Transport coefficients without any memory allocation.
 *
 * The paper has no counterpart: this is a service for callers that may not allocate GPU
 * memory when they need the coefficients -- hosts whose every allocation must come from
 * their own pool, embedders that may only use buffers they were handed.  It computes the
 * same tensors as ephb_transport_coefficients
 * from response arrays the caller already holds on the device, and calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * Inputs (all device pointers, row-major, FP64): per electron state its energy (eV),
 * velocity (m/s, [n][3]), weight 1/|stabiliser of its k| (0 for an inactive state) and
 * responses I, J ([n][3]); per phonon mode hbar*omega (eV), velocity ([n][3]) and F, G
 * ([n][3]).  The symmetry operations are copied from the struct at call time.
 * Output: out_dev, 72 doubles on the device in the order of ephb_coeffs (sigma, sigmaS,
 * S, alpha_el, kappa0_el, kappa_el, alpha_ph, kappa_ph).
 *
 * Scratch: one file-scope __device__ array of 442 KB that every GPU loading the library
 * holds until the process exits; it bounds n_states and n_modes to EPHB_NOALLOC_MAX_ITEMS
 * each (larger inputs return EPHB_EINVAL).  Every call overwrites the scratch it reads,
 * so nothing needs clearing, but all calls on a device share it: calls whose work
 * overlaps on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller.
 * The first call on a device looks up the scratch's device address for that device (with
 * that device current) and keeps it; make that first call before starting any stream
 * capture.  A device reset (cudaDeviceReset) invalidates the kept address: after one, this
 * entry point must not be called again in the same process.
 * The work is enqueued on cuda_stream (NULL: the legacy default stream) and the call
 * returns without waiting; out_dev is valid once the stream reaches that point.
 * Errors: EPHB_EINVAL for NULL or out-of-range arguments, EPHB_ECUDA for a launch
 * failure.
 * --------------------------------------------------------------------------------*/
#define EPHB_NOALLOC_MAX_ITEMS 4194304

typedef struct {
  int64_t n_states;
  const double *eps, *vel, *weight, *I, *J;
  int64_t n_modes;
  const double *omega, *vph, *F, *G;
  double T_K, mu_eV, spin_deg;
  double volume_A3;            /* unit-cell volume                                          */
  int64_t nk, nq;              /* full k and q mesh sizes (the 1/N_k, 1/N_q of the sums)    */
  double omega_min_eV;         /* modes at or below it are left out                         */
  int nsym;                    /* 1..48 operations ...                                      */
  double sym_cart[48][9];      /* ... on Cartesian vectors, for the electron-side zone sum  */
} ephb_coeff_inputs;

ephb_status ephb_transport_coefficients_noalloc(const ephb_coeff_inputs *in, double *out_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* EPHB_H */
