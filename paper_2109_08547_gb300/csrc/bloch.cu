// Wannier-to-Bloch interpolation of H(k) and D(q), their diagonalisation, Hellmann-Feynman
// velocities (Eqs. H_mn(k), v_mk, D_ss'(q), v_sq of arXiv 2109.08547), the transport
// window, the irreducible wedge of the k mesh and the (k, q) pair lists.
#include "internal.h"
#include "jacobi.cuh"
#include "jacobi_warp.cuh"

namespace ephb {

namespace {

__global__ void k_phase_tables(double2 *tab, Mesh m) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int total = m.n[0] + m.n[1] + m.n[2];
  if (t >= total) return;
  int d = t < m.n[0] ? 0 : (t < m.n[0] + m.n[1] ? 1 : 2);
  int j = t - (d == 0 ? 0 : (d == 1 ? m.n[0] : m.n[0] + m.n[1]));
  double s, c;
  sincospi(2.0 * double(j) / double(m.n[d]), &s, &c);
  tab[t] = cmk(c, s);
}

// ---- Fourier interpolation, one warp per point ------------------------------------------
// O(k) = sum_R e^{i k.R} O_R and grad_k O(k) = sum_R i R e^{i k.R} O_R (Eqs. H_mn(k) and
// D_ss'(q) and the Hellmann-Feynman velocities), for the points of a list.  The lanes share the
// matrix elements (lane l takes elements l, l + 32, ...); lane l computes the phase and the
// Cartesian R of the l-th vector of each block of 32, which the loop over R broadcasts by
// shuffles.  Every element sums over R in the order of the R list, exactly as a thread that did
// the whole matrix alone.  Output, transposed for the one-thread-per-point decomposition that
// reads it: out[(v ne + e) ldn + t], v = 0 for O and 1..3 for the components of its gradient.
constexpr int kInterpWarps = 4;

template <int EPL>
__global__ void __launch_bounds__(32 * kInterpWarps) k_fourier_interp(ModelDev M, Mesh m, const double2 *__restrict__ tab,
                                                                   const int *__restrict__ list, int64_t n, int64_t ldn,
                                                                   const int *__restrict__ Rv, int nR,
                                                                   const double2 *__restrict__ OR, int ne,
                                                                   double2 *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t t = blockIdx.x * int64_t(kInterpWarps) + (threadIdx.x >> 5);
  if (t >= n) return;   // whole warps leave together
  int i0, i1, i2;
  m.unflat(list[t], i0, i1, i2);
  double2 acc[EPL], grad[EPL][3];
  for (int k = 0; k < EPL; ++k) {
    acc[k] = cmk(0, 0);
    grad[k][0] = grad[k][1] = grad[k][2] = cmk(0, 0);
  }
  for (int r0 = 0; r0 < nR; r0 += 32) {
    double2 myph = cmk(0, 0);
    double myR[3] = {0, 0, 0};
    if (r0 + lane < nR) {
      const int *R = Rv + 3 * (r0 + lane);
      myph = mesh_phase(tab, m, i0, i1, i2, R[0], R[1], R[2]);
      for (int a = 0; a < 3; ++a) myR[a] = R[0] * M.lattice[a] + R[1] * M.lattice[3 + a] + R[2] * M.lattice[6 + a];
    }
    const int nr = nR - r0 < 32 ? nR - r0 : 32;
    for (int rr = 0; rr < nr; ++rr) {
      const double2 ph = cmk(__shfl_sync(0xffffffffu, myph.x, rr), __shfl_sync(0xffffffffu, myph.y, rr));
      double Rc[3];
      for (int a = 0; a < 3; ++a) Rc[a] = __shfl_sync(0xffffffffu, myR[a], rr);
      const double2 *h = OR + size_t(r0 + rr) * ne;
      for (int k = 0; k < EPL; ++k) {
        const int e = lane + 32 * k;
        if (e < ne) {
          const double2 tt = cmul(ph, h[e]);
          acc[k] = cadd(acc[k], tt);
          for (int a = 0; a < 3; ++a) {   // i R_a t
            grad[k][a].x -= Rc[a] * tt.y;
            grad[k][a].y += Rc[a] * tt.x;
          }
        }
      }
    }
  }
  for (int k = 0; k < EPL; ++k) {
    const int e = lane + 32 * k;
    if (e < ne) {
      out[size_t(e) * ldn + t] = acc[k];
      for (int a = 0; a < 3; ++a) out[size_t((1 + a) * ne + e) * ldn + t] = grad[k][a];
    }
  }
}

// One thread per listed k point (launches of many points: every FP64 instruction serves 32
// matrices): eigen-decomposition of H(k) (read from the interpolation),
// velocities <m| grad H |m> averaged over degenerate groups, the window masks.
template <int NB>
__global__ void __launch_bounds__(64) k_electron_bands(ModelDev M, Mesh km, const int *__restrict__ list, int64_t n,
                                                       const double2 *__restrict__ HdH, int64_t ldn,
                                                       double degen_tol, double lo, double hi, double *eps,
                                                       double2 *cvec, double *vel, uint8_t *egrp,
                                                       uint32_t *amask, uint32_t *rmask) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const int k = list[t];
  const int nb = M.nb, ne = nb * nb;
  double2 H[NB * NB], V[NB * NB];
  double e[NB];
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) H[i * NB + j] = HdH[size_t(i * nb + j) * ldn + t];
  herm_jacobi<NB>(H, V, e, nb);
  // v_m = <m| grad H |m>: for each component and row i, w_m = sum_j dH_ij V_jm, then
  // v_m += Re(conj(V_im) w_m); every gradient element is read once
  double vd[NB][3];
  for (int m = 0; m < nb; ++m) vd[m][0] = vd[m][1] = vd[m][2] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < nb; ++i) {
      double2 w[NB];
      for (int m = 0; m < nb; ++m) w[m] = cmk(0, 0);
      for (int j = 0; j < nb; ++j) {
        const double2 d = HdH[size_t((1 + a) * ne + i * nb + j) * ldn + t];
        for (int m = 0; m < nb; ++m) cfma(w[m], d, V[j * NB + m]);
      }
      for (int m = 0; m < nb; ++m) vd[m][a] += V[i * NB + m].x * w[m].x + V[i * NB + m].y * w[m].y;
    }
  uint8_t grp[2 * NB];
  degenerate_groups(e, nb, degen_tol, grp);
  const double conv = kAngstrom / kHbarEVs;
  uint32_t mask = 0;
  for (int m = 0; m < nb; ++m) {
    int g0 = grp[2 * m], g1 = grp[2 * m + 1];
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int j = g0; j < g1; ++j) s += vd[j][a];
      vel[(size_t(k) * nb + m) * 3 + a] = s / double(g1 - g0) * conv;
    }
    eps[size_t(k) * nb + m] = e[m];
    egrp[(size_t(k) * nb + m) * 2] = grp[2 * m];
    egrp[(size_t(k) * nb + m) * 2 + 1] = grp[2 * m + 1];
    if (e[m] >= lo && e[m] <= hi) mask |= 1u << m;
    for (int i = 0; i < nb; ++i) cvec[(size_t(k) * nb + i) * nb + m] = V[i * NB + m];
  }
  amask[k] = mask;
  // the degenerate subspaces of the active bands, whole ([A9]: a subspace cut by a window edge
  // still averages |g|^2 over all its bands)
  uint32_t rot = 0;
  for (int m = 0; m < nb; ++m)
    if ((mask >> m) & 1u)
      for (int a = grp[2 * m]; a < grp[2 * m + 1]; ++a) rot |= 1u << a;
  rmask[k] = rot;
}

// One thread per listed q point (launches of many points): eigen-decomposition of D(q) (read from the interpolation),
// hbar w = sqrt(max(lambda, 0)), velocities.
template <int NB>
__global__ void __launch_bounds__(64) k_phonon_modes(ModelDev M, Mesh qm, const int *__restrict__ list, int64_t n,
                                                     const double2 *__restrict__ DdD, int64_t ldn,
                                                     double degen_tol, double omega_min, double *w, double2 *u,
                                                     double *vph, uint8_t *pgrp) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const int q = list[t];
  const int nb = M.nbr, ne = nb * nb;
  double2 D[NB * NB], V[NB * NB];
  double e[NB];
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) D[i * NB + j] = DdD[size_t(i * nb + j) * ldn + t];
  herm_jacobi<NB>(D, V, e, nb);
  double om[NB];
  for (int s = 0; s < nb; ++s) om[s] = sqrt(fmax(e[s], 0.0));
  double vd[NB][3];
  for (int s = 0; s < nb; ++s) vd[s][0] = vd[s][1] = vd[s][2] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < nb; ++i) {
      double2 ws[NB];
      for (int s = 0; s < nb; ++s) ws[s] = cmk(0, 0);
      for (int j = 0; j < nb; ++j) {
        const double2 d = DdD[size_t((1 + a) * ne + i * nb + j) * ldn + t];
        for (int s = 0; s < nb; ++s) cfma(ws[s], d, V[j * NB + s]);
      }
      for (int s = 0; s < nb; ++s) vd[s][a] += V[i * NB + s].x * ws[s].x + V[i * NB + s].y * ws[s].y;
    }
  uint8_t grp[2 * NB];
  degenerate_groups(om, nb, degen_tol, grp);
  const double conv = kAngstrom / kHbarEVs;
  for (int s = 0; s < nb; ++s) {
    int g0 = grp[2 * s], g1 = grp[2 * s + 1];
    for (int a = 0; a < 3; ++a) {
      double v = 0.0;
      if (om[s] > omega_min) {
        double acc = 0.0;
        for (int j = g0; j < g1; ++j) acc += vd[j][a];
        v = acc / double(g1 - g0) / (2.0 * om[s]) * conv;
      }
      vph[(size_t(q) * nb + s) * 3 + a] = v;
    }
    w[size_t(q) * nb + s] = om[s];
    pgrp[(size_t(q) * nb + s) * 2] = grp[2 * s];
    pgrp[(size_t(q) * nb + s) * 2 + 1] = grp[2 * s + 1];
    for (int i = 0; i < nb; ++i) u[(size_t(q) * nb + i) * nb + s] = V[i * NB + s];
  }
}

constexpr int kDecompWarps = 4;   // points (one warp each) per block of the warp form
// Launches of fewer points take the warp form: one thread per matrix leaves most SMs idle and
// each busy one waiting on a single thread's dependency chain (the time of a launch is that
// chain, ~0.8 ms, whatever its size), while the warp form keeps ~16 of 32 lanes of each FP64
// instruction busy and so costs about twice the FP64 work (~0.13 us per point on the FP64 pipe).
constexpr int64_t kWarpDecompMax = 4096;

// One warp per listed k point (launches of few points): eigen-decomposition of H(k) (read from the interpolation) by
// the warp-cooperative Jacobi, velocities <m| grad H |m> averaged over degenerate groups, the
// window masks.
template <int NB>
__global__ void __launch_bounds__(32 * kDecompWarps) k_electron_bands_warp(ModelDev M, Mesh km, const int *__restrict__ list,
                                                                      int64_t n, const double2 *__restrict__ HdH,
                                                                      int64_t ldn, double degen_tol, double lo,
                                                                      double hi, double *eps, double2 *cvec,
                                                                      double *vel, uint8_t *egrp, uint32_t *amask,
                                                                      uint32_t *rmask) {
  __shared__ JacobiWarpSmem<NB> sm[kDecompWarps];
  __shared__ double vds[kDecompWarps][NB * 3];
  __shared__ uint8_t grps[kDecompWarps][2 * NB];
  const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = int64_t(blockIdx.x) * kDecompWarps + wq;
  if (t >= n) return;   // the whole warp
  JacobiWarpSmem<NB> &S = sm[wq];
  const int k = list[t];
  const int nb = M.nb, ne = nb * nb;
  for (int x = lane; x < ne; x += 32) S.A[(x / nb) * NB + x % nb] = HdH[size_t(x) * ldn + t];
  __syncwarp();
  herm_jacobi_warp<NB>(S, nb);
  // v_m = <m| grad H |m>: for component a and row i, w = sum_j dH_ij V_jm, v += Re(conj(V_im) w)
  for (int x = lane; x < nb * 3; x += 32) {
    const int m = x / 3, a = x % 3, col = S.perm[m];
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) {
      double2 w = cmk(0.0, 0.0);
      for (int j = 0; j < nb; ++j) cfma(w, HdH[size_t((1 + a) * ne + i * nb + j) * ldn + t], S.V[j * NB + col]);
      const double2 vi = S.V[i * NB + col];
      acc += vi.x * w.x + vi.y * w.y;
    }
    vds[wq][x] = acc;
  }
  if (lane == 0) degenerate_groups(S.e, nb, degen_tol, grps[wq]);
  __syncwarp();
  const uint8_t *grp = grps[wq];
  const double conv = kAngstrom / kHbarEVs;
  for (int x = lane; x < nb * 3; x += 32) {
    const int m = x / 3, a = x % 3, g0 = grp[2 * m], g1 = grp[2 * m + 1];
    double s = 0.0;
    for (int j = g0; j < g1; ++j) s += vds[wq][j * 3 + a];
    vel[(size_t(k) * nb + m) * 3 + a] = s / double(g1 - g0) * conv;
  }
  for (int m = lane; m < nb; m += 32) {
    eps[size_t(k) * nb + m] = S.e[m];
    egrp[(size_t(k) * nb + m) * 2] = grp[2 * m];
    egrp[(size_t(k) * nb + m) * 2 + 1] = grp[2 * m + 1];
  }
  for (int x = lane; x < ne; x += 32) {
    const int i = x / nb, m = x % nb;
    cvec[(size_t(k) * nb + i) * nb + m] = S.V[i * NB + S.perm[m]];
  }
  if (lane == 0) {
    uint32_t mask = 0;
    for (int m = 0; m < nb; ++m)
      if (S.e[m] >= lo && S.e[m] <= hi) mask |= 1u << m;
    amask[k] = mask;
    // the degenerate subspaces of the active bands, whole ([A9]: a subspace cut by a window
    // edge still averages |g|^2 over all its bands)
    uint32_t rot = 0;
    for (int m = 0; m < nb; ++m)
      if ((mask >> m) & 1u)
        for (int a = grp[2 * m]; a < grp[2 * m + 1]; ++a) rot |= 1u << a;
    rmask[k] = rot;
  }
}

// One warp per listed q point: eigen-decomposition of D(q) (read from the interpolation),
// hbar w = sqrt(max(lambda, 0)), velocities.
template <int NB>
__global__ void __launch_bounds__(32 * kDecompWarps) k_phonon_modes_warp(ModelDev M, Mesh qm, const int *__restrict__ list,
                                                                    int64_t n, const double2 *__restrict__ DdD,
                                                                    int64_t ldn, double degen_tol, double omega_min,
                                                                    double *w, double2 *u, double *vph,
                                                                    uint8_t *pgrp) {
  __shared__ JacobiWarpSmem<NB> sm[kDecompWarps];
  __shared__ double vds[kDecompWarps][NB * 3];
  __shared__ double oms[kDecompWarps][NB];
  __shared__ uint8_t grps[kDecompWarps][2 * NB];
  const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = int64_t(blockIdx.x) * kDecompWarps + wq;
  if (t >= n) return;   // the whole warp
  JacobiWarpSmem<NB> &S = sm[wq];
  const int q = list[t];
  const int nb = M.nbr, ne = nb * nb;
  for (int x = lane; x < ne; x += 32) S.A[(x / nb) * NB + x % nb] = DdD[size_t(x) * ldn + t];
  __syncwarp();
  herm_jacobi_warp<NB>(S, nb);
  for (int s = lane; s < nb; s += 32) oms[wq][s] = sqrt(fmax(S.e[s], 0.0));
  for (int x = lane; x < nb * 3; x += 32) {
    const int s = x / 3, a = x % 3, col = S.perm[s];
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) {
      double2 ws = cmk(0.0, 0.0);
      for (int j = 0; j < nb; ++j) cfma(ws, DdD[size_t((1 + a) * ne + i * nb + j) * ldn + t], S.V[j * NB + col]);
      const double2 vi = S.V[i * NB + col];
      acc += vi.x * ws.x + vi.y * ws.y;
    }
    vds[wq][x] = acc;
  }
  __syncwarp();
  if (lane == 0) degenerate_groups(oms[wq], nb, degen_tol, grps[wq]);
  __syncwarp();
  const uint8_t *grp = grps[wq];
  const double conv = kAngstrom / kHbarEVs;
  for (int x = lane; x < nb * 3; x += 32) {
    const int s = x / 3, a = x % 3, g0 = grp[2 * s], g1 = grp[2 * s + 1];
    const double om = oms[wq][s];
    double v = 0.0;
    if (om > omega_min) {
      double acc = 0.0;
      for (int j = g0; j < g1; ++j) acc += vds[wq][j * 3 + a];
      v = acc / double(g1 - g0) / (2.0 * om) * conv;
    }
    vph[(size_t(q) * nb + s) * 3 + a] = v;
  }
  for (int s = lane; s < nb; s += 32) {
    w[size_t(q) * nb + s] = oms[wq][s];
    pgrp[(size_t(q) * nb + s) * 2] = grp[2 * s];
    pgrp[(size_t(q) * nb + s) * 2 + 1] = grp[2 * s + 1];
  }
  for (int x = lane; x < ne; x += 32) {
    const int i = x / nb, s = x % nb;
    u[(size_t(q) * nb + i) * nb + s] = S.V[i * NB + S.perm[s]];
  }
}

// Phonons of every q that is not the representative of its star, from the representative's
// (Eq. D_ss'(q) is covariant): with q = S <q> and the atom map S tau_a = tau_{p(a)} + L_a,
// D(S q)_{p(a) p(b)} = e^{i q.(L_b - L_a)} S D(<q>)_{ab} S^T, so
//   u_{p(a) x, s}(q) = e^{-i q.L_a} sum_y S_xy u_{a y, s}(<q>)
// is an eigenvector set of D(q) (a gauge of the degenerate subspaces, which every |g|^2 average
// leaves invariant); hbar w and the degenerate groups are the representative's and
// v_s(q) = S v_s(<q>).
__global__ void k_phonons_from_rep(ModelDev M, Mesh qm, const double2 *__restrict__ qtab, const int *qrep,
                                   const int *qop, double *w, double2 *u, double *vph, uint8_t *pgrp) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= qm.size()) return;
  const int r = qrep[q];
  if (r == int(q)) return;
  const int nbr = M.nbr, nat = M.nat, o = qop[q];
  const double *S = M.sym_cart + 9 * o;
  int b0, b1, b2;
  qm.unflat(int(q), b0, b1, b2);
  for (int s = 0; s < nbr; ++s) {
    w[q * nbr + s] = w[size_t(r) * nbr + s];
    pgrp[(q * nbr + s) * 2] = pgrp[(size_t(r) * nbr + s) * 2];
    pgrp[(q * nbr + s) * 2 + 1] = pgrp[(size_t(r) * nbr + s) * 2 + 1];
    const double *v = vph + (size_t(r) * nbr + s) * 3;
    for (int x = 0; x < 3; ++x)
      vph[(q * nbr + s) * 3 + x] = S[3 * x] * v[0] + S[3 * x + 1] * v[1] + S[3 * x + 2] * v[2];
  }
  for (int a = 0; a < nat; ++a) {
    const int pa = M.atom_perm[o * nat + a];
    const int *L = M.atom_shift + (o * nat + a) * 3;
    const double2 ph = mesh_phase(qtab, qm, b0, b1, b2, L[0], L[1], L[2]);   // e^{i q.L_a}
    const double2 phc = make_double2(ph.x, -ph.y);
    for (int s = 0; s < nbr; ++s)
      for (int x = 0; x < 3; ++x) {
        double2 acc = cmk(0, 0);
        for (int y = 0; y < 3; ++y) {
          const double2 v = u[(size_t(r) * nbr + 3 * a + y) * nbr + s];
          acc.x += S[3 * x + y] * v.x;
          acc.y += S[3 * x + y] * v.y;
        }
        u[(q * nbr + 3 * pa + x) * nbr + s] = cmul(phc, acc);
      }
  }
}

// of[list[j]] = j
__global__ void k_rep_index(int64_t nlist, const int *list, int *of) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j < nlist) of[list[j]] = int(j);
}

// Irreducible wedge: representative = smallest image index, first op S with S<k> = k,
// stabiliser size.  flag = 1 for the representatives.
// Representative <k> of each mesh point (the smallest flat index of its star), the first
// operation S with S <k> = k and the order of the stabiliser of <k>, in one pass over the
// group.  With img_s = S_s k and <k> = min_s img_s, the set H = {s : img_s = <k>} is a coset
// of the stabiliser of <k> (so |H| = |stab(<k>)|), and S_s <k> = k exactly when s^-1 is in H:
// the operation sought is the first s whose inverse lies in H.
__global__ void k_ibz(ModelDev M, Mesh km, int *rep, int *op, int *stab, int *flag) {
  __shared__ int rot[kMaxSym * 9];
  __shared__ int inv[kMaxSym];
  for (int t = threadIdx.x; t < M.nsym * 9; t += blockDim.x) rot[t] = M.sym_rot[t];
  for (int t = threadIdx.x; t < M.nsym; t += blockDim.x) inv[t] = M.sym_inv[t];
  __syncthreads();
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= km.size()) return;
  int i[3];
  km.unflat(k, i[0], i[1], i[2]);
  int best = k;
  uint64_t hit = 0;   // operations s with img_s == best
  for (int s = 0; s < M.nsym; ++s) {
    const int *S = rot + 9 * s;
    int j0 = pmod(S[0] * i[0] + S[1] * i[1] + S[2] * i[2], km.n[0]);
    int j1 = pmod(S[3] * i[0] + S[4] * i[1] + S[5] * i[2], km.n[1]);
    int j2 = pmod(S[6] * i[0] + S[7] * i[1] + S[8] * i[2], km.n[2]);
    int img = km.flat(j0, j1, j2);
    if (img < best) {
      best = img;
      hit = 0;
    }
    if (img == best) hit |= 1ull << s;
  }
  int first = -1;
  for (int s = 0; s < M.nsym && first < 0; ++s)
    if ((hit >> inv[s]) & 1ull) first = s;
  rep[k] = best;
  op[k] = first;
  stab[k] = __popcll(hit);
  flag[k] = best == k ? 1 : 0;
}

// Every point that is not a representative: when its representative has no band in the window
// (band energies are symmetric, eps(S<k>) = eps(<k>), so neither has this point) it takes the
// representative's energies and degenerate groups and the rotated velocities v(S<k>) = S v(<k>),
// with no active band; otherwise flag = 1 asks for its own eigen-decomposition (the rates need
// its eigenvectors).  Representatives: flag = 0.
__global__ void k_bands_from_rep(ModelDev M, Mesh km, const int *rep, const int *op, double *eps, double *vel,
                                 uint8_t *egrp, uint32_t *amask, uint32_t *rmask, int *flag) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= km.size()) return;
  const int r = rep[k];
  if (r == int(k)) {
    flag[k] = 0;
    return;
  }
  if (amask[r] != 0u) {
    flag[k] = 1;
    return;
  }
  flag[k] = 0;
  const int nb = M.nb;
  const double *S = M.sym_cart + 9 * op[k];
  for (int m = 0; m < nb; ++m) {
    eps[k * nb + m] = eps[size_t(r) * nb + m];
    egrp[(k * nb + m) * 2] = egrp[(size_t(r) * nb + m) * 2];
    egrp[(k * nb + m) * 2 + 1] = egrp[(size_t(r) * nb + m) * 2 + 1];
    const double *v = vel + (size_t(r) * nb + m) * 3;
    for (int a = 0; a < 3; ++a) vel[(k * nb + m) * 3 + a] = S[3 * a] * v[0] + S[3 * a + 1] * v[1] + S[3 * a + 2] * v[2];
  }
  amask[k] = 0u;
  rmask[k] = 0u;
}

// flag = 1 for representatives with an active band
__global__ void k_ibzw_flag(int64_t nk, const int *rep, const uint32_t *amask, int *flag) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k < nk) flag[k] = (rep[k] == int(k) && amask[k] != 0u) ? 1 : 0;
}

// list[pos[k]] = k for the flagged points
__global__ void k_compact(int64_t n, const int *flag, const int64_t *pos, int *list) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k < n && flag[k]) list[pos[k]] = int(k);
}

__global__ void k_ibzw_fill(int64_t nk, const int *flag, const int64_t *pos, int *list, int *of) {
  int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= nk) return;
  if (flag[k]) {
    list[pos[k]] = int(k);
    of[k] = int(pos[k]);
  } else {
    of[k] = -1;
  }
}

__device__ inline int kplusq(const MeshDev &D, int k, int q) {
  int a0, a1, a2, b0, b1, b2;
  D.km.unflat(k, a0, a1, a2);
  D.qm.unflat(q, b0, b1, b2);
  return D.km.flat(pmod(a0 + D.ratio[0] * b0, D.km.n[0]), pmod(a1 + D.ratio[1] * b1, D.km.n[1]),
                   pmod(a2 + D.ratio[2] * b2, D.km.n[2]));
}

// block per irreducible-window k: number of q with an active band at k+q
// Pairs (k, q) of the irreducible window points with an active band at k + q, k-major and in
// increasing q within each k.  The q range of each k is cut into chunks of kPairChunk: block
// (c, i) counts (then writes) the pairs of chunk c of point i, so that a scan over the counts in
// (i, c) order gives every block its output offset and the pair pointers of each i.
constexpr int kPairChunk = 4096;

__global__ void k_pair_count(MeshDev D, int nch, int *cnt) {
  __shared__ int red[32];
  const int c = blockIdx.x, i = blockIdx.y;
  const int k = D.ibzw_list[i];
  const int q1 = int(D.nq - int64_t(c) * kPairChunk < kPairChunk ? D.nq : int64_t(c + 1) * kPairChunk);
  int n = 0;
  for (int q = c * kPairChunk + threadIdx.x; q < q1; q += blockDim.x) n += D.amask[kplusq(D, k, q)] != 0u;
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) cnt[int64_t(i) * nch + c] = v;
  }
}

// ordered compaction helper: exclusive rank of `flag` within the block (blockDim = 256)
__device__ inline int block_rank(int flag, int *warp_tot, int &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned b = __ballot_sync(0xffffffffu, flag);
  int r = __popc(b & ((1u << lane) - 1u));
  if (lane == 0) warp_tot[wid] = __popc(b);
  __syncthreads();
  int off = 0;
  total = 0;
  for (int w = 0; w < nw; ++w) {
    if (w < wid) off += warp_tot[w];
    total += warp_tot[w];
  }
  __syncthreads();
  return off + r;
}

// off: exclusive scan of the chunk counts in (i, c) order
__global__ void k_pair_fill(MeshDev D, int nch, const int64_t *__restrict__ off, int *pair_q, int *pair_i) {
  __shared__ int wt[32];
  const int c = blockIdx.x, i = blockIdx.y;
  const int k = D.ibzw_list[i];
  const int q0 = c * kPairChunk;
  const int q1 = int(D.nq - int64_t(c) * kPairChunk < kPairChunk ? D.nq : int64_t(c + 1) * kPairChunk);
  int64_t base = off[int64_t(i) * nch + c];
  for (int qb = q0; qb < q1; qb += blockDim.x) {
    const int q = qb + threadIdx.x;
    const int f = q < q1 ? (D.amask[kplusq(D, k, q)] != 0u) : 0;
    int total;
    const int r = block_rank(f, wt, total);
    if (f) {
      pair_q[base + r] = q;
      pair_i[base + r] = i;
    }
    base += total;
  }
}

// pair pointers of each irreducible window point from the chunk offsets
__global__ void k_pair_ptr(int64_t n_ibzw, int nch, const int64_t *__restrict__ off, int64_t *pair_ptr) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i <= n_ibzw) pair_ptr[i] = off[i * nch];
}

// one warp per q: how many irreducible-window k pair with it
__global__ void k_qpair_count(MeshDev D, int *qcount) {
  const int64_t q = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= D.nq) return;
  int n = 0;
  for (int i = lane; i < D.n_ibzw; i += 32) n += D.amask[kplusq(D, D.ibzw_list[i], int(q))] != 0u;
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if (lane == 0) qcount[q] = n;
}

// one warp per q: rank of each pair (i, q) among the pairs of q, in increasing i
__global__ void k_qpair_fill(MeshDev D, int *pq_rank) {
  const int64_t q64 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q64 >= D.nq) return;
  const int q = int(q64);
  int base = 0;
  for (int i0 = 0; i0 < D.n_ibzw; i0 += 32) {
    const int i = i0 + lane;
    const int f = i < D.n_ibzw ? (D.amask[kplusq(D, D.ibzw_list[i], q)] != 0u) : 0;
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if (f) {
      // pair index of (i, q): binary search in the q-sorted list of i
      int64_t lo = D.pair_ptr[i], hi = D.pair_ptr[i + 1];
      while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (D.pair_q[mid] <= q) lo = mid; else hi = mid;
      }
      pq_rank[lo] = base + __popc(b & ((1u << lane) - 1u));
    }
    base += __popc(b);
  }
}

__global__ void k_count_bits(const uint32_t *m, int64_t n, unsigned long long *out) {
  unsigned long long c = 0;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x)
    c += __popc(m[t]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

__global__ void k_count_reps(const int *rep, int64_t n, unsigned long long *out) {
  unsigned long long c = 0;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x)
    c += rep[t] == int(t);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

}  // namespace

cudaError_t launch_phase_tables(double2 *tab, Mesh m, cudaStream_t st) {
  int total = m.n[0] + m.n[1] + m.n[2];
  EPHB_LAUNCH(k_phase_tables, (total + 127) / 128, 128, 0, st, tab, m);
  return cudaGetLastError();
}

// the interpolation of a list, in chunks of at most interp_chunk() points (scratch: 4 ne x chunk)
int64_t interp_chunk() { return 65536; }

static cudaError_t fourier_interp(const ModelDev &M, Mesh m, const double2 *tab, const int *list, int64_t n,
                                  int64_t ldn, const int *Rv, int nR, const double2 *OR, int ne, double2 *out,
                                  cudaStream_t st) {
  const unsigned grid = unsigned((n + kInterpWarps - 1) / kInterpWarps);
  if (ne <= 32)
    EPHB_LAUNCH(k_fourier_interp<1>, grid, 32 * kInterpWarps, 0, st, M, m, tab, list, n, ldn, Rv, nR, OR, ne, out);
  else if (ne <= 64)
    EPHB_LAUNCH(k_fourier_interp<2>, grid, 32 * kInterpWarps, 0, st, M, m, tab, list, n, ldn, Rv, nR, OR, ne, out);
  else
    EPHB_LAUNCH(k_fourier_interp<5>, grid, 32 * kInterpWarps, 0, st, M, m, tab, list, n, ldn, Rv, nR, OR, ne, out);
  return cudaGetLastError();
}

cudaError_t launch_electron_bands(const ModelDev &M, Mesh km, const int *list, int64_t n, const double2 *ktab,
                                  double degen_tol, double lo, double hi, double *eps, double2 *cvec, double *vel,
                                  uint8_t *egrp, uint32_t *amask, uint32_t *rmask, double2 *scratch,
                                  cudaStream_t st) {
  const int ne = M.nb * M.nb;
  for (int64_t c0 = 0; c0 < n; c0 += interp_chunk()) {
    const int64_t nc = n - c0 < interp_chunk() ? n - c0 : interp_chunk();
    cudaError_t e = fourier_interp(M, km, ktab, list + c0, nc, nc, M.Re, M.nRe, M.H_R, ne, scratch, st);
    if (e != cudaSuccess) return e;
    if (nc >= kWarpDecompMax) {   // one thread per point, two warps per block
      const int grid = int((nc + 63) / 64), bs = 64;
      if (M.nb <= 1)
        EPHB_LAUNCH(k_electron_bands<1>, grid, bs, 0, st, M, km, list + c0, nc, scratch, nc, degen_tol, lo, hi, eps,
                    cvec, vel, egrp, amask, rmask);
      else if (M.nb <= 4)
        EPHB_LAUNCH(k_electron_bands<4>, grid, bs, 0, st, M, km, list + c0, nc, scratch, nc, degen_tol, lo, hi, eps,
                    cvec, vel, egrp, amask, rmask);
      else
        EPHB_LAUNCH(k_electron_bands<8>, grid, bs, 0, st, M, km, list + c0, nc, scratch, nc, degen_tol, lo, hi, eps,
                    cvec, vel, egrp, amask, rmask);
    } else {   // one warp per point, four points per block
      const int grid = int((nc + kDecompWarps - 1) / kDecompWarps), bs = 32 * kDecompWarps;
      if (M.nb <= 1)
        EPHB_LAUNCH(k_electron_bands_warp<1>, grid, bs, 0, st, M, km, list + c0, nc, scratch, nc, degen_tol, lo, hi,
                    eps, cvec, vel, egrp, amask, rmask);
      else if (M.nb <= 4)
        EPHB_LAUNCH(k_electron_bands_warp<4>, grid, bs, 0, st, M, km, list + c0, nc, scratch, nc, degen_tol, lo, hi,
                    eps, cvec, vel, egrp, amask, rmask);
      else
        EPHB_LAUNCH(k_electron_bands_warp<8>, grid, bs, 0, st, M, km, list + c0, nc, scratch, nc, degen_tol, lo, hi,
                    eps, cvec, vel, egrp, amask, rmask);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_bands_from_rep(const ModelDev &M, Mesh km, const int *rep, const int *op, double *eps, double *vel,
                                  uint8_t *egrp, uint32_t *amask, uint32_t *rmask, int *flag, cudaStream_t st) {
  const int64_t n = km.size();
  EPHB_LAUNCH(k_bands_from_rep, int((n + 255) / 256), 256, 0, st, M, km, rep, op, eps, vel, egrp, amask, rmask, flag);
  return cudaGetLastError();
}

cudaError_t launch_ibzw_flag(int64_t nk, const int *rep, const uint32_t *amask, int *flag, cudaStream_t st) {
  EPHB_LAUNCH(k_ibzw_flag, int((nk + 255) / 256), 256, 0, st, nk, rep, amask, flag);
  return cudaGetLastError();
}

cudaError_t launch_compact(int64_t n, const int *flag, const int64_t *pos, int *list, cudaStream_t st) {
  EPHB_LAUNCH(k_compact, int((n + 255) / 256), 256, 0, st, n, flag, pos, list);
  return cudaGetLastError();
}

cudaError_t launch_phonon_modes(const ModelDev &M, Mesh qm, const int *list, int64_t n, const double2 *qtab,
                                double degen_tol, double omega_min, double *w, double2 *u, double *vph, uint8_t *pgrp,
                                double2 *scratch, cudaStream_t st) {
  const int ne = M.nbr * M.nbr;
  for (int64_t c0 = 0; c0 < n; c0 += interp_chunk()) {
    const int64_t nc = n - c0 < interp_chunk() ? n - c0 : interp_chunk();
    cudaError_t e = fourier_interp(M, qm, qtab, list + c0, nc, nc, M.Rd, M.nRd, M.D_R, ne, scratch, st);
    if (e != cudaSuccess) return e;
    if (nc >= kWarpDecompMax) {   // one thread per point
      const int grid = int((nc + 63) / 64), bs = 64;
      if (M.nbr <= 3)
        EPHB_LAUNCH(k_phonon_modes<3>, grid, bs, 0, st, M, qm, list + c0, nc, scratch, nc, degen_tol, omega_min, w, u,
                    vph, pgrp);
      else if (M.nbr <= 6)
        EPHB_LAUNCH(k_phonon_modes<6>, grid, bs, 0, st, M, qm, list + c0, nc, scratch, nc, degen_tol, omega_min, w, u,
                    vph, pgrp);
      else
        EPHB_LAUNCH(k_phonon_modes<12>, grid, bs, 0, st, M, qm, list + c0, nc, scratch, nc, degen_tol, omega_min, w, u,
                    vph, pgrp);
    } else {   // one warp per point
      const int grid = int((nc + kDecompWarps - 1) / kDecompWarps), bs = 32 * kDecompWarps;
      if (M.nbr <= 3)
        EPHB_LAUNCH(k_phonon_modes_warp<3>, grid, bs, 0, st, M, qm, list + c0, nc, scratch, nc, degen_tol, omega_min,
                    w, u, vph, pgrp);
      else if (M.nbr <= 6)
        EPHB_LAUNCH(k_phonon_modes_warp<6>, grid, bs, 0, st, M, qm, list + c0, nc, scratch, nc, degen_tol, omega_min,
                    w, u, vph, pgrp);
      else
        EPHB_LAUNCH(k_phonon_modes_warp<12>, grid, bs, 0, st, M, qm, list + c0, nc, scratch, nc, degen_tol, omega_min,
                    w, u, vph, pgrp);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_phonons_from_rep(const ModelDev &M, Mesh qm, const double2 *qtab, const int *qrep, const int *qop,
                                    double *w, double2 *u, double *vph, uint8_t *pgrp, cudaStream_t st) {
  const int64_t n = qm.size();
  EPHB_LAUNCH(k_phonons_from_rep, int((n + 127) / 128), 128, 0, st, M, qm, qtab, qrep, qop, w, u, vph, pgrp);
  return cudaGetLastError();
}

cudaError_t launch_rep_index(int64_t n, const int *list, int64_t nlist, int *of, cudaStream_t st) {
  (void)n;
  if (nlist <= 0) return cudaSuccess;
  EPHB_LAUNCH(k_rep_index, int((nlist + 255) / 256), 256, 0, st, nlist, list, of);
  return cudaGetLastError();
}

cudaError_t launch_ibz(const ModelDev &M, Mesh km, int *rep, int *op, int *stab, int *flag, cudaStream_t st) {
  int64_t n = km.size();
  EPHB_LAUNCH(k_ibz, int((n + 127) / 128), 128, 0, st, M, km, rep, op, stab, flag);
  return cudaGetLastError();
}

cudaError_t launch_ibzw_fill(int64_t nk, const int *flag, const int64_t *pos, int *list, int *of, cudaStream_t st) {
  EPHB_LAUNCH(k_ibzw_fill, int((nk + 255) / 256), 256, 0, st, nk, flag, pos, list, of);
  return cudaGetLastError();
}

int pair_chunks(int64_t nq) { return int((nq + kPairChunk - 1) / kPairChunk); }

cudaError_t launch_pair_count(const MeshDev &D, int *cnt, cudaStream_t st) {
  if (D.n_ibzw == 0) return cudaSuccess;
  EPHB_LAUNCH(k_pair_count, dim3(unsigned(pair_chunks(D.nq)), unsigned(D.n_ibzw)), 256, 0, st, D, pair_chunks(D.nq),
              cnt);
  return cudaGetLastError();
}

cudaError_t launch_pair_ptr(int64_t n_ibzw, int nch, const int64_t *off, int64_t *pair_ptr, cudaStream_t st) {
  EPHB_LAUNCH(k_pair_ptr, unsigned((n_ibzw + 1 + 255) / 256), 256, 0, st, n_ibzw, nch, off, pair_ptr);
  return cudaGetLastError();
}

cudaError_t launch_pair_fill(const MeshDev &D, const int64_t *off, int *pair_q, int *pair_i, cudaStream_t st) {
  if (D.n_ibzw == 0) return cudaSuccess;
  EPHB_LAUNCH(k_pair_fill, dim3(unsigned(pair_chunks(D.nq)), unsigned(D.n_ibzw)), 256, 0, st, D, pair_chunks(D.nq),
              off, pair_q, pair_i);
  return cudaGetLastError();
}

cudaError_t launch_qpair_count(const MeshDev &D, int *qcount, cudaStream_t st) {
  EPHB_LAUNCH(k_qpair_count, unsigned((D.nq * 32 + 255) / 256), 256, 0, st, D, qcount);
  return cudaGetLastError();
}

cudaError_t launch_qpair_fill(const MeshDev &D, int *pq_rank, cudaStream_t st) {
  EPHB_LAUNCH(k_qpair_fill, unsigned((D.nq * 32 + 255) / 256), 256, 0, st, D, pq_rank);
  return cudaGetLastError();
}

cudaError_t launch_count_bits(const uint32_t *amask, int64_t n, int64_t *out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  EPHB_LAUNCH(k_count_bits, 152, 256, 0, st, amask, n, reinterpret_cast<unsigned long long *>(out));
  return cudaGetLastError();
}

cudaError_t launch_count_reps(const int *rep, int64_t n, int64_t *out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  EPHB_LAUNCH(k_count_reps, 152, 256, 0, st, rep, n, reinterpret_cast<unsigned long long *>(out));
  return cudaGetLastError();
}

}  // namespace ephb
