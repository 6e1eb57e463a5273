// Internal declarations shared by the translation units of the CUDA library.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ephb {

// Device copy of the Wannier model (pointers are device pointers).
struct ModelDev {
  int nat = 0, nb = 0, nbr = 0, nRe = 0, nRd = 0, nRge = 0, nRgp = 0, nsym = 0;
  double lattice[9] = {0};
  double omega_ref = 0, spin_deg = 2, bg_coeff = 0, bg_w = 1, bg_T = 300;
  double mass[4] = {0};
  double mass_mean = 1;
  const int *Re = nullptr, *Rd = nullptr, *Rge = nullptr, *Rgp = nullptr;
  const double2 *H_R = nullptr, *D_R = nullptr, *g_R = nullptr;
  const int *sym_rot = nullptr;       // [nsym][9]
  const double *sym_cart = nullptr;   // [nsym][9]
  const int *sym_inv = nullptr;       // [nsym]
  // sum over the operations of S_ae S_bf, at [(a*3+b)*9 + e*3+f]: the symmetrised tensor
  // sum_S S M S^T is then sum_ef sym_pair[ab][ef] M_ef
  const double *sym_pair = nullptr;   // [81]
  // atom maps of the operations: S tau_a = tau_{perm[s][a]} + shift[s][a] (crystal coordinates)
  const int *atom_perm = nullptr;     // [nsym][nat]
  const int *atom_shift = nullptr;    // [nsym][nat][3]
};

// Views of the mesh-level arrays.
struct MeshDev {
  Mesh km, qm;
  int ratio[3];
  int64_t nk, nq;
  const double2 *ktab, *qtab;         // per-dimension phase tables
  const double *eps;                  // [nk][nb]
  const double2 *cvec;                // [nk][nb][nb]  c[k][row][col]
  const double *vel;                  // [nk][nb][3]
  const uint8_t *egrp;                // [nk][nb][2] degenerate group [lo, hi)
  const uint32_t *amask;              // [nk] bands inside the window (the states of the BTE)
  const uint32_t *rmask;              // [nk] amask plus every band degenerate with an active one:
                                      //      the bands whose |g|^2 enters the degenerate averages
  const double *w;                    // [nq][nbr]
  const double2 *u;                   // [nq][nbr][nbr]
  const double *vph;                  // [nq][nbr][3]
  const uint8_t *pgrp;                // [nq][nbr][2]
  const int *qrep, *qop;              // [nq] representative of the q star and S with S <q> = q
  const int *qrep_of;                 // [nq] index of a representative in the representative list
  const int *qlist;                   // [n_qrep] the representatives
  const int *qstab;                   // [nq] order of the stabiliser of q's representative
  int64_t n_qrep;
  const int *rep, *op, *stab;         // [nk]
  const int *ibzw_of;                 // [nk] index in the irreducible-window list or -1
  const int *ibzw_list;               // [n_ibzw]
  int64_t n_ibzw;
  const int64_t *pair_ptr;            // [n_ibzw+1]
  const int *pair_q;                  // [n_pairs]
  const int *pair_i;                  // [n_pairs]
  const int64_t *qpair_ptr;           // [nq+1]
  const int *pq_rank;                 // [n_pairs] rank of pair among the pairs of its q
  int64_t n_pairs;
  double omega_min, degen_tol;
};

// ---- scan.cu
// out[i] = sum_{j<i} in[j]; returns the total through *total_dev (device int64).
template <typename T>
cudaError_t exclusive_scan(const T *in, int64_t *out, int64_t n, int64_t *total_dev, int64_t *scratch,
                           int64_t scratch_elems, cudaStream_t st);
int64_t scan_scratch_elems(int64_t n);

// ---- bloch.cu
cudaError_t launch_phase_tables(double2 *tab, Mesh m, cudaStream_t st);
// Bands / phonons of the points of a list: the Fourier sums of H (D) and its gradient by
// k_fourier_interp into scratch (4 nb^2 x min(n, interp_chunk()) complex), then the
// eigen-decompositions.
int64_t interp_chunk();
cudaError_t launch_electron_bands(const ModelDev &M, Mesh km, const int *list, int64_t n, const double2 *ktab,
                                  double degen_tol, double lo, double hi, double *eps, double2 *cvec, double *vel,
                                  uint8_t *egrp, uint32_t *amask, uint32_t *rmask, double2 *scratch,
                                  cudaStream_t st);
cudaError_t launch_bands_from_rep(const ModelDev &M, Mesh km, const int *rep, const int *op, double *eps, double *vel,
                                  uint8_t *egrp, uint32_t *amask, uint32_t *rmask, int *flag, cudaStream_t st);
cudaError_t launch_ibzw_flag(int64_t nk, const int *rep, const uint32_t *amask, int *flag, cudaStream_t st);
cudaError_t launch_compact(int64_t n, const int *flag, const int64_t *pos, int *list, cudaStream_t st);
cudaError_t launch_phonon_modes(const ModelDev &M, Mesh qm, const int *list, int64_t n, const double2 *qtab,
                                double degen_tol, double omega_min, double *w, double2 *u, double *vph, uint8_t *pgrp,
                                double2 *scratch, cudaStream_t st);
cudaError_t launch_ibz(const ModelDev &M, Mesh km, int *rep, int *op, int *stab, int *flag, cudaStream_t st);
cudaError_t launch_phonons_from_rep(const ModelDev &M, Mesh qm, const double2 *qtab, const int *qrep, const int *qop,
                                    double *w, double2 *u, double *vph, uint8_t *pgrp, cudaStream_t st);
cudaError_t launch_rep_index(int64_t n, const int *list, int64_t nlist, int *of, cudaStream_t st);
cudaError_t launch_ibzw_fill(int64_t nk, const int *flag, const int64_t *pos, int *ibzw_list, int *ibzw_of,
                             cudaStream_t st);
// pair lists: chunk counts cnt[n_ibzw][pair_chunks(nq)], their exclusive scan off (n_ibzw x
// nch + 1 entries), the pair pointers from it, then the k-major, q-ascending fill
int pair_chunks(int64_t nq);
cudaError_t launch_pair_count(const MeshDev &D, int *cnt, cudaStream_t st);
cudaError_t launch_pair_ptr(int64_t n_ibzw, int nch, const int64_t *off, int64_t *pair_ptr, cudaStream_t st);
cudaError_t launch_pair_fill(const MeshDev &D, const int64_t *off, int *pair_q, int *pair_i, cudaStream_t st);
cudaError_t launch_qpair_count(const MeshDev &D, int *qcount, cudaStream_t st);
cudaError_t launch_qpair_fill(const MeshDev &D, int *pq_rank, cudaStream_t st);
cudaError_t launch_count_bits(const uint32_t *amask, int64_t n, int64_t *out, cudaStream_t st);
cudaError_t launch_count_reps(const int *rep, int64_t n, int64_t *out, cudaStream_t st);

// ---- vertex.cu
struct RateParams {
  double T, mu, sigma, cut, inv_Nq_pref;   // inv_Nq_pref = 2 pi / (hbar N_q)
  double inv_sigma, gnorm;                 // 1 / sigma, 1 / (sigma sqrt(2 pi))
  float2 inv_sigma_ff, gnorm_ff;           // the same as float-float pairs
  double y_scale;                          // N_q / N_k
  int vertex_only;                         // 1: store V+- = 2pi/(hbar N_q)|g|^2 delta (no occupations)
  int rot_fp32;                            // 1: band/branch rotations in FP32 (mixed mode)
  int tetra = 0;                           // 1: linear tetrahedron delta weights instead of the Gaussian
  const float *eps32 = nullptr, *w32 = nullptr;   // FP32 copies of eps [nk][nb] and w [nq][nbr]
};
cudaError_t launch_rate_count(const ModelDev &M, const MeshDev &D, RateParams rp, int *cntE, int *cntPh,
                              unsigned long long *n_tuples, cudaStream_t st);
cudaError_t launch_row_ptrs(const MeshDev &D, int nb, int nbr, const int64_t *escan, const int64_t *phscan,
                            int64_t e_total, int64_t ph_total, int64_t *row_ptr, int64_t *ph_row_ptr,
                            cudaStream_t st);
cudaError_t launch_stage_a(const ModelDev &M, const MeshDev &D, int64_t i0, int64_t nkc, double2 *T, double2 *A,
                           cudaStream_t st);
cudaError_t launch_stage_b_rates(const ModelDev &M, const MeshDev &D, RateParams rp, int64_t i0, int64_t nkc,
                                 const double2 *A, const int64_t *escan, const int64_t *phscan, uint32_t *e_kpns,
                                 double2 *e_X, int *ph_st, uint32_t *ph_kpn, double *ph_Y, cudaStream_t st);
size_t stage_a_T_elems(const ModelDev &M);
size_t stage_a_A_elems(const ModelDev &M);
// Tables of the rate epilogue: fk [nk][nb] Fermi, nbq [nq][nbr] Bose, wr [nq][nbr] w_ref/w,
// ut [nq][nbr][nbr] mass-scaled phonon eigenvectors.
cudaError_t launch_epi_tables(const ModelDev &M, const MeshDev &D, double T, double mu, double *fk, double *nbq,
                              double *wr, double2 *ut, cudaStream_t st);
// float-float copies of c(k) and of the mass-scaled u(q) for the FP64-grade epilogue
cudaError_t launch_ff_tables(const ModelDev &M, const MeshDev &D, const double2 *ut, float4 *cff, float4 *uff,
                             cudaStream_t st);
// Rates of pairs [pbeg, pend) from a contraction already in Cbuf[pair - pair_base][Nmax]
// (tensor-core path: float-float pairs), one thread per pair.
cudaError_t launch_vertex_epilogue(const ModelDev &M, const MeshDev &D, RateParams rp, int64_t pbeg, int64_t pend,
                                   int64_t pair_base, const double *Cbuf, int Nmax, const double *fk,
                                   const double *nbq, const double *wr, const double2 *ut, const float4 *cff,
                                   const float4 *uff, const int64_t *escan,
                                   const int64_t *phscan, uint32_t *e_kpns, double2 *e_X, int *ph_st,
                                   uint32_t *ph_kpn, double *ph_Y, cudaStream_t st);

// ---- vertex_tc.cu (tcgen05 R_ph contraction with exact BF16 fixed-point slices)
int tc_kp(const ModelDev &M);     // padded K = 2 nRgp rounded up to the K block
int tc_nmax(const ModelDev &M);   // column stride of B' = 2 nb^2 nbr rounded up to 16
cudaError_t launch_phase_slices(const ModelDev &M, const MeshDev &D, int ns, __nv_bfloat16 *phis,
                                __nv_bfloat16 *angle_tab, cudaStream_t st);
cudaError_t launch_vertex_tc(const ModelDev &M, const MeshDev &D, int ns, int64_t i0, int64_t nkc, int64_t pair_base,
                             const double2 *A, const __nv_bfloat16 *phis, __nv_bfloat16 *bs, double *bscale,
                             int *nitem, int64_t *item_ptr, int64_t *scratch, int64_t scratch_elems,
                             int64_t *total_dev, double *Cbuf, int *err, cudaStream_t st, cudaEvent_t gemm0,
                             cudaEvent_t gemm1, int ncm, int kc, int stages, int withhold, int64_t *ws_desc,
                             int64_t ws_cap);
// ws_desc: scratch of 4 int64 per work item (descriptors of the persistent form), ws_cap items
// Stage A on tensor cores: T[kc][col] = sum_Re e^{ik.Re} g[Re][col] for the k of a chunk, as
// the same exact-slice GEMM with the model's g slices (made once by launch_g_slices, BF16,
// pre-tiled by 128 columns and K blocks of 16, + column scales) as the rows and the k phase
// slices as the columns.  ns: 7 or 8.  T is written as float-float pairs (two FP32 numbers per real value,
// in the place of one double), read by launch_stage_a2 with t_ff set.
int tc_kp_a(const ModelDev &M);
int tc_ncols_a(const ModelDev &M);
// elements of the pre-tiled g slices and of the phase-slice operand of a group of <= chunk k
size_t tc_gs_elems_a(const ModelDev &M, int ns);
size_t stage_a_phik_elems(const ModelDev &M, int ns, int64_t chunk);
cudaError_t launch_g_slices(const ModelDev &M, int ns, __nv_bfloat16 *gs, double *gscale, cudaStream_t st);
// a_tmem: the A slices are copied into tensor memory once per K step (tcgen05.cp) and the
// products read them there; otherwise every product reads its A slice from shared memory.
// The two forms give bit-identical results.
cudaError_t launch_stage_a_tc(const ModelDev &M, const MeshDev &D, int ns, int64_t i0, int64_t nkc,
                              __nv_bfloat16 *phik, const __nv_bfloat16 *gs, const double *gscale, double2 *T, int *err,
                              bool a_tmem, cudaStream_t st, double *flops_acc);
// The band rotation of stage A: A[kc][rp][(m,n',a)] = sum_m' c_{m'm}(k) T[kc][rp][m'][n'][a]
// (T in FP64, or as float-float pairs when t_ff).
cudaError_t launch_stage_a2(const ModelDev &M, const MeshDev &D, int64_t i0, int64_t nkc, const double2 *T, double2 *A,
                            bool t_ff, cudaStream_t st);
// Tile shape of the contraction: column-chunk width and K per shared-memory stage (16: two CTAs
// per SM).  The result does not depend on it: every column is summed in the same order.
struct TcShape {
  int width, kc, stages;
};
cudaError_t launch_selftest_exp_ff(const double *y, double *out, int64_t n, cudaStream_t st);
int tc_nc_max(int ns);
// slices of the exact fixed-point form for a contraction length kp: FP64-grade 7 (kp <= 256)
// or 8 (base-128 digits, kp <= 816), split-BF16 3 (kp <= 1024); 0 where none applies
int tc_slices_for(int kp, bool fp64_grade);
bool tc_nc_valid(int ns, int ncm, int kc, int stages);
std::vector<TcShape> tc_shape_candidates(int ns);

// ---- bte.cu
struct BteDev {
  int nb, nbr, nsym;
  int64_t nst, nq;
  double T, mu, spin_deg, Pe, Pph;
  const int64_t *row_ptr;
  const uint32_t *e_kpns;
  const double2 *e_X;
  const int64_t *ph_row_ptr;
  const int *ph_st;
  const uint32_t *ph_kpn;
  const double *ph_Y;
  const uint32_t *kcrd;    // packed k coordinates (10 bits each)
  const double *st_eps;    // [nst]
  const double *st_vel;    // [nst][3]
  const double *st_ff;     // [nst] f(1-f)
  const double *st_wt;     // [nst] 1/|stab| (0 for inactive)
};
// kinfo[k] = (state base of the representative <k> = ibzw index * nb (or -1), op taking <k> to k)
// States active for the BTE: active on the meshes and lo <= eps <= hi (the instance window).
cudaError_t launch_state_setup(const ModelDev &M, const MeshDev &D, double T, double mu, double lo, double hi,
                               double *st_eps, double *st_vel, double *st_ff, double *st_wt, uint32_t *kcrd,
                               int2 *kinfo, cudaStream_t st);
// Rate lists of one (T, mu, window) instance from the T-independent vertex lists (V+-, V+ Y-scaled):
// count the kept entries of every electron row (k, m) and phonon row (q, s), then write them
// (order kept) with X+- = V+- f(1-f') {n, 1+n} and Y = V f(1-f') n.  fk, nbq: occupation tables.
struct InstWindow { double lo, hi; };
cudaError_t launch_inst_count(const ModelDev &M, const MeshDev &D, InstWindow w, const int64_t *u_row_ptr,
                              const uint32_t *u_kpns, const int64_t *u_ph_row_ptr, const int *u_ph_st,
                              const uint32_t *u_ph_kpn, int *cnt_e, int *cnt_ph, cudaStream_t st);
cudaError_t launch_inst_fill(const ModelDev &M, const MeshDev &D, InstWindow w, const double *fk, const double *nbq,
                             const int64_t *u_row_ptr, const uint32_t *u_kpns, const double2 *u_X,
                             const int64_t *u_ph_row_ptr, const int *u_ph_st, const uint32_t *u_ph_kpn,
                             const double *u_ph_V, const int64_t *row_ptr, const int64_t *ph_row_ptr,
                             uint32_t *e_kpns, double2 *e_X, int *ph_st, uint32_t *ph_kpn, double *ph_Y,
                             cudaStream_t st);
// W_add (optional, per state): rates of other channels added to W^RTA (Matthiessen's rule)
cudaError_t launch_rta_electron(const BteDev &B, double *W_e, double *inv_ffW, double *I0, double *J0,
                                unsigned long long *n_zero, cudaStream_t st, const double *W_add = nullptr);
// Electron-charged-impurity scattering: the e-chimp part of W^RTA of every state.
struct ChimpParams {
  int nspec;
  double n_m3[4], Z[4];             // dopant concentrations (1/m^3) and ionizations
  double eps_r, V;                  // dielectric constant, cell volume (m^3)
  double rec[3][3];                 // reciprocal lattice vectors (rows, 1/m)
  double sigma, cut_sigmas, gnorm;  // Gaussian delta: width, cut, 1/(sigma sqrt(2 pi))
  double pref;                      // 2 pi / (hbar N_k)
  double win_lo, win_hi;            // window of the final states
};
int chimp_partials();
// q_TF^2 = ff_scale * sum over the n_eps energies eps_all of f(1 - f) (into q_tf2, device), then
// W[state] (part: chimp_partials() doubles of scratch)
cudaError_t launch_chimp_rates(const MeshDev &D, const BteDev &B, const ChimpParams &P, const double *eps_all,
                               int64_t n_eps, double ff_scale, double *part, double *q_tf2, double *W,
                               cudaStream_t st);
cudaError_t launch_ph_rowsum(const BteDev &B, double *Bt, cudaStream_t st);
cudaError_t launch_rta_phonon(const ModelDev &M, const MeshDev &D, const BteDev &B, const double *Bt, double *W_ph,
                              double *inv_nnW, double *F0, cudaStream_t st, const double *W_add = nullptr);
// Phonon-isotope (Tamura) scattering: its part of W^RTA_sq on the q representatives (Wrep
// [n_qrep][nbr]), then on every q (W [nq][nbr]).
struct IsoParams {
  double g[4];                      // mass-variance parameter of each atom
  double sigma, cut_sigmas, gnorm;  // Gaussian delta: width, cut, 1/(sigma sqrt(2 pi))
  double pref;                      // pi / (2 hbar N_q)
};
cudaError_t launch_iso_rates(const ModelDev &M, const MeshDev &D, const IsoParams &P, double *Wrep, double *W,
                             cudaStream_t st);
// Segments of a row-structured stream (at most sweep_segment_len() items, within one row).
struct SweepSegs {
  int64_t nseg = 0;
  const int *seg_row = nullptr;       // [nseg] row of the segment
  const int64_t *seg_begin = nullptr; // [nseg] first item
  const int64_t *seg_ptr = nullptr;   // [nrow+1] first segment of each row
  const int64_t *row_ptr = nullptr;   // [nrow+1] items of each row
};
int sweep_segment_len();
cudaError_t launch_build_segments(int64_t nrow, const int64_t *row_ptr, int *nseg_row, int64_t *seg_ptr,
                                  int64_t *scratch, int64_t scratch_elems, int64_t &nseg_host, cudaStream_t st);
cudaError_t launch_fill_segments(int64_t nrow, const int64_t *row_ptr, const int64_t *seg_ptr, int *seg_row,
                                 int64_t *seg_begin, cudaStream_t st);
// Partner runs: the entries of a row sharing (k', n), merged over branches.
cudaError_t launch_build_runs(const BteDev &B, int64_t n_entries, const int2 *kinfo, int *flag, int64_t *runidx,
                              int64_t *scratch, int64_t scratch_elems, int64_t *run_ptr, uint32_t *run_col,
                              double *run_w, int64_t &nruns, int64_t *total_dev, cudaStream_t st);
cudaError_t launch_fill_runs(const BteDev &B, int64_t n_entries, int64_t nruns, const int2 *kinfo, const int *flag,
                             const int64_t *runidx, int64_t *run_ptr, uint32_t *run_col, double *run_w,
                             cudaStream_t st);
// Coefficient assembly fused into the finalisation (its last block does what
// launch_coeff_final does, with the same arguments); counter: a zeroed device word.
struct CoeffFuse {
  const double *ppart = nullptr;
  double *res = nullptr, *prev = nullptr;
  int *ctl = nullptr;
  int max_sweeps = 0;
  double tol = 0.0;
  unsigned *counter = nullptr;
};
// One electron sweep (self term over the runs) and the per-row finalisation
// I = I0 + (self + Dterm)/(f(1-f)W), which also writes the electron coefficient partials.
// ctl == nullptr: reads (Ia, Ja), writes (Ib, Jb).  Otherwise the loop is driven on the device:
// nothing runs once ctl[0] is set, and sweep number ctl[1] reads (Ia, Ja) when even and
// (Ib, Jb) when odd and writes the other pair (ctl[1] is advanced by launch_coeff_final).
cudaError_t launch_self_sweep(const ModelDev &M, const BteDev &B, const SweepSegs &S, const uint32_t *run_col,
                              const double *run_w, const double *I0, const double *J0, const double *inv_ffW,
                              double *Ia, double *Ja, double *Ib, double *Jb, const double *Dterm, double *part,
                              double *epart, const int *ctl, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                              cudaEvent_t ev1 = nullptr,    // events around the self-term kernel
                              double2 *IJa = nullptr, double2 *IJb = nullptr, const CoeffFuse *fuse = nullptr);
// Packed copy of the responses for the gathers: IJ[st] = (I0 I1 | I2 J0 | J1 J2) as 3 double2.
// With IJa/IJb given the sweep gathers from them (by the same parity as Ia/Ib) and the
// finalisation writes both layouts.
cudaError_t launch_pack_ij(int64_t nst, const double *I, const double *J, double2 *IJ, cudaStream_t st);
// Drag term of every row for the current F, G: Dterm[st][6].
cudaError_t launch_drag_term(const MeshDev &D, const BteDev &B, const SweepSegs &S, const double *F, const double *G,
                             double *part, double *Dterm, cudaStream_t st);
// Phonon drag scatter over the phonon rows (q, s) cut into segments S (built over ph_row_ptr
// like the electron segments): per-segment partials into part[nseg][6], then Btv[row][6].
cudaError_t launch_ph_sweep(const ModelDev &M, const BteDev &B, const SweepSegs &S, const int2 *kinfo,
                            const double *I, const double *J, double *part, double *Btv, cudaStream_t st);
cudaError_t launch_ph_update(const ModelDev &M, const MeshDev &D, const double *Btv, const double *F0,
                             const double *inv_nnW, double *F, double *G, double *Afold, cudaStream_t st);
// Coefficient tensors: fixed-count partial sums (electron: 36 per block, phonon: 18 per
// block) and a single-block finalisation into `res`.
//   res layout: [0] sigma [9] sigmaS [18] alpha_el [27] kappa0_el [36] alpha_ph [45] kappa_ph
//               [54] S [63] kappa_el [72] residual_e [73] residual_all [74] lambda [75] ko_valid
constexpr int kResLen = 80;
int coeff_partials();
cudaError_t launch_e_partial(const BteDev &B, const double *I, const double *J, double *epart, cudaStream_t st);
cudaError_t launch_ph_partial(const MeshDev &D, const BteDev &B, const double *F, const double *G, const double *W_ph,
                              const double *inv_nnW, double *ppart, cudaStream_t st);
// Mixed-precision electron loop: FP32 copies, the correction start r = x' - x (d = r), one FP32
// correction sweep d_out = r + (1/(f(1-f)W)) sum_runs w d[partner], and x += d.
cudaError_t launch_to_f32(int64_t n, const double *a, float *b, cudaStream_t st);
cudaError_t launch_corr_init(int64_t nst, const double *I1, const double *I0x, const double *J1, const double *J0x,
                             float *rI, float *rJ, float *dI, float *dJ, cudaStream_t st);
cudaError_t launch_corr_sweep(const ModelDev &M, int64_t nst, const SweepSegs &S, const uint32_t *run_col,
                              const float *run_w32, const double *inv_ffW, const float *rI, const float *rJ,
                              const float *dI, const float *dJ, float *part, float *dI_out, float *dJ_out,
                              cudaStream_t st);
cudaError_t launch_corr_apply(int64_t nst, const float *dI, const float *dJ, double *I, double *J, cudaStream_t st);
// FP32 forms of the phonon-side terms for the mixed iteration's early outer iterations:
// drag term from X32 (float2 per entry) and FG32 ([mode][F | G] floats), phonon scatter from
// Y32 (float per phonon entry) and IJ32 ([state][I | J] floats); pack6: out[i] = (A[i], B[i]).
cudaError_t launch_drag_term32(const MeshDev &D, const BteDev &B, const SweepSegs &S, const float2 *X32,
                               const float *FG32, double *part, double *Dterm, cudaStream_t st);
cudaError_t launch_ph_sweep32(const ModelDev &M, const BteDev &B, const SweepSegs &S, const int2 *kinfo,
                              const float *Y32, const float *IJ32, double *part, double *Btv, cudaStream_t st);
cudaError_t launch_pack6_f32(int64_t n, const double *A, const double *Bv, float *out, cudaStream_t st);
// Float-float forms of the same two terms for the later outer iterations of the mixed
// iteration: Xff (X+ hi, lo, X- hi, lo per entry), Yff, IJff ([state][6] pairs), FGff
// ([mode][6] pairs); partial sums converted to FP64 per lane and reduced in FP64.
cudaError_t launch_drag_termff(const MeshDev &D, const BteDev &B, const SweepSegs &S, const float4 *Xff,
                               const float2 *FGff, double *part, double *Dterm, cudaStream_t st);
cudaError_t launch_ph_sweepff(const ModelDev &M, const BteDev &B, const SweepSegs &S, const int2 *kinfo,
                              const float2 *Yff, const float2 *IJff, double *part, double *Btv, cudaStream_t st);
cudaError_t launch_copy_ff(int64_t n, const double *a, float2 *out, cudaStream_t st);
cudaError_t launch_pack6_ff(int64_t n, const double *A, const double *Bv, float2 *out, cudaStream_t st);
cudaError_t launch_copy_f32(int64_t n, const double *a, float *b, cudaStream_t st);
// Anderson acceleration of the outer iteration over x = (F, G) (2 * half doubles): the
// residual f = g - x, the dot products of a new residual with up to kAndMaxSlots ring vectors
// (F and G halves apart: dots[2j], dots[2j+1]; part holds and_part_len() doubles), and the
// mixed iterate x = sum_j alpha_j g_j (ring vectors `stride` doubles apart).
constexpr int kAndMaxSlots = 9;
struct AndCoef { double a[kAndMaxSlots]; };
cudaError_t launch_and_resid(int64_t half, const double *g, const double *F, const double *G, double *f,
                             cudaStream_t st);
cudaError_t launch_and_dots(int64_t half, const double *fnew, const double *ring, int64_t stride, int nslot,
                            double *part, double *dots, cudaStream_t st);
size_t and_part_len();
cudaError_t launch_and_mix(int64_t half, const double *ring, int64_t stride, int nslot, const AndCoef &al, double *F,
                           double *G, cudaStream_t st);
// Warm start: network inputs per state (kNFeat floats), training targets (2 floats: the
// converged I, J along the RTA direction J0 = v/W), and starting responses from them.
constexpr int kNFeat = 6;
cudaError_t launch_state_features(const BteDev &B, const double *W_e, unsigned *vmax_bits, float *feat,
                                  cudaStream_t st);
cudaError_t launch_state_targets(const BteDev &B, const double *I, const double *J, const double *J0,
                                 unsigned *vmax_bits, float *t, cudaStream_t st);
cudaError_t launch_apply_warm(int64_t nst, const double *I0, const double *J0, const float *a, double *I, double *J,
                              cudaStream_t st);
cudaError_t launch_coeff_final(const ModelDev &M, const BteDev &B, const double *epart, const double *ppart,
                               double *res, double *prev, cudaStream_t st, int *ctl = nullptr, int max_sweeps = 0,
                               double tol = 0.0);
cudaError_t launch_ko(const ModelDev &M, const MeshDev &D, const BteDev &B, double *I, const double *J,
                      double *kpart, double *res, cudaStream_t st);

// Mixed-precision iteration constants shared by the host-driven and graph-driven loops.
constexpr int kCorrSweeps = 12;       // FP32 correction sweeps per FP64 sweep
constexpr double kPh32Until = 1e-5;   // outer residual below which the phonon-side terms are FP64-grade

// ---- solve_graph.cu: the coupled iteration of several instances as ONE CUDA graph launch.
// The loops of "Coupled and decoupled BTEs" (the outer phonon/electron iteration, the inner
// electron loop) run on the device: conditional graph nodes (WHILE for the loops, SWITCH for
// the choice of the phonon-side arithmetic and for "converged / correct") whose conditions are
// set by one-thread control kernels reading the residuals.  Every instance is an independent
// branch of the graph, so the instances' kernels overlap on the GPU.  Kernels and their order
// within an instance are those of the host-driven loop, so the results are bit-identical.
struct GraphCtl {                       // per instance, device memory, read back after the launch
  int outer, outer32, outer_seen, ph_mode;   // ph_mode: 0 FP32, 1 float-float, 2 FP64 phonon-side terms
  int inner_it, inner_ok, converged, timed_out;
  long long sweeps, sweeps32, inner_total;
  long long n_outer_body, n_inner_body, n_ph_body[3], n_in_body[2];   // body executions
  double residual, tol_k, last_tol_k, lambda;
  unsigned long long t0;                // %globaltimer at the start of the instance
};
struct GraphOpts {
  int level, precision, ko, max_outer, max_inner, ph32_allowed;
  double tol, inner_tol, time_limit_s;
};
// Everything the capture of one instance reads (device pointers, counts, views).
struct GraphInst {
  BteDev B;
  SweepSegs Sr, Se, Sp;                 // segments of the partner runs, the entry stream, the phonon entries
  int64_t nst, nph, n_entries, n_ph_entries, nruns;
  const int2 *kinfo;
  const uint32_t *run_col;
  const double *run_w, *I0, *J0, *inv_ffW, *W_ph, *inv_nnW, *F0, *ph_Y;
  const double2 *e_X;
  double *I, *J, *I2, *J2, *F, *G, *Btv, *Afold, *Dterm, *seg_part, *ph_part, *epart, *ppart, *kpart, *res, *prev_in,
      *prev_out;
  float *run_w32, *rI, *rJ, *dI, *dJ, *dI2, *dJ2, *part32;     // mixed electron loop
  float2 *X32;                                                 // mixed, FP32 phonon-side terms
  float *Y32, *IJ32, *FG32;
  float4 *Xff;                                                 // mixed, float-float phonon-side terms
  float2 *Yff, *IJff, *FGff;
  int *sctl;                                                   // FP64 electron loop (fused finalisation)
  unsigned *fuse_ctr;
  double2 *IJ, *IJ2;
  const float *warm;                                           // warm-start factors, or nullptr (RTA start)
  GraphCtl *ctl;
};
// Kernels captured per body, for the launch count of an execution.
struct GraphKernels {
  long long prologue = 0, outer_fixed = 0, ph[3] = {0, 0, 0}, inner_fixed = 0, in[2] = {0, 0};
};
// Builds and instantiates the graph of all instances (levels partial, dragless, dragged;
// accel_depth 0).  cs: a stream used only for capture.  The kernel count of every body is
// returned per instance; the library's launch counter is left unchanged by the capture.
cudaError_t build_solve_graph(const ModelDev &M, const MeshDev &D, const std::vector<GraphInst> &insts,
                              const GraphOpts &o, cudaStream_t cs, cudaGraph_t *graph, cudaGraphExec_t *exec,
                              std::vector<GraphKernels> &kernels);
long long launch_count();

}  // namespace ephb
