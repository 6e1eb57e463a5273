// e-ph vertex interpolation (Eq. g^smn_kq of arXiv 2109.08547) fused with the transition
// rates (Eq. X^e-ph; Y^ph-e as the same + process on the phonon side).
//
// The double Fourier sum over (R_e, R_ph) is evaluated in two contractions:
//   stage A, per irreducible-window k:  A[rp][m,n',a] = sum_m' c_{m'm}(k) sum_re e^{ik.Re} gW[re][rp][m'][n'][a]
//   stage B, per (k, q) pair:           B[m,n',a]    = sum_rp e^{iq.Rp} A[rp][m,n',a]
// followed, in the same kernel, by the final-band and branch rotations, |g|^2, the
// degenerate-subspace average, occupations, the Gaussian delta and the compacted writes
// into the electron rows (k,m) and the phonon rows (q,s).
#include "internal.h"

namespace ephb {

namespace {

__device__ inline int kplusq_d(const MeshDev &D, int k, int q) {
  int a0, a1, a2, b0, b1, b2;
  D.km.unflat(k, a0, a1, a2);
  D.qm.unflat(q, b0, b1, b2);
  return D.km.flat(pmod(a0 + D.ratio[0] * b0, D.km.n[0]), pmod(a1 + D.ratio[1] * b1, D.km.n[1]),
                   pmod(a2 + D.ratio[2] * b2, D.km.n[2]));
}

__device__ inline int nth_bit(uint32_t m, int n) {
  for (int b = 0; b < 32; ++b)
    if ((m >> b) & 1u) {
      if (n == 0) return b;
      --n;
    }
  return -1;
}

__device__ inline double fermi_d(double e, double mu, double kT) { return 1.0 / (exp((e - mu) / kT) + 1.0); }
__device__ inline double bose_d(double w, double kT) { return w > 0.0 ? 1.0 / expm1(w / kT) : 0.0; }
// (1/(sigma sqrt(2 pi))) exp(-x^2 / (2 sigma^2)) inside the cutoff, from the reciprocals
// held in the parameters (no FP64 division on the per-tuple path)
__device__ inline double gauss_d(double x, const RateParams &rp) {
  if (fabs(x) > rp.cut) return 0.0;
  const double r = x * rp.inv_sigma;
  return exp(-0.5 * r * r) * rp.gnorm;
}
// the same for x already known to lie inside the cutoff
__device__ inline double gauss_in(double x, const RateParams &rp) {
  const double r = x * rp.inv_sigma;
  return exp(-0.5 * r * r) * rp.gnorm;
}

// 1/n! for n = 0..13 and ln 2 as float-float pairs (hi = nearest FP32, lo = nearest FP32 of
// the remainder; computed from the exact rationals and a 60-digit ln 2)
__constant__ float2 kInvFact[14] = {
    {0x1p+0f, 0.f}, {0x1p+0f, 0.f}, {0x1p-1f, 0.f}, {0x1.555556p-3f, -0x1.555556p-28f},
    {0x1.555556p-5f, -0x1.555556p-30f}, {0x1.111112p-7f, -0x1.ddddde0p-32f}, {0x1.6c16c2p-10f, -0x1.27d27ep-35f},
    {0x1.a01a02p-13f, -0x1.7f97fap-39f}, {0x1.a01a02p-16f, -0x1.7f97fap-42f}, {0x1.71de3ap-19f, 0x1.55b1ccp-45f},
    {0x1.27e4fcp-22f, -0x1.10ec14p-47f}, {0x1.ae6456p-26f, 0x1.fd5138p-52f}, {0x1.1eed8ep-29f, 0x1.ff1b12p-54f},
    {0x1.612462p-33f, -0x1.8af25ep-58f}};

// e^y in float-float for -60 <= y <= 0: y = k ln2 + r with |r| <= ln2/2 (plus rounding),
// e^r from its Taylor series to r^13/13! (the remainder is below 1e-17 of the sum) by
// float-float Horner steps, then the exact scaling by 2^k.  The reduction subtracts k ln2 in
// three parts (Cody and Waite's splitting of the constant): C1 and C2 carry 17 significant bits,
// so k C1 and k C2 are exact FP32 products for |k| <= 127, and C3 the rest of ln 2 (the three
// sum to ln 2 within 3e-19); r then carries ~2^-49 absolute error instead of 2^-48 of |y|.
// ~2^-46 relative overall, FP32 pipe only.
__device__ inline float2 exp_ff(float2 y) {
  const float C1 = 0x1.62e4p-1f, C2 = 0x1.7f7ep-20f, C3 = -0x1.c610cap-37f;
  const int k = __float2int_rn(__fmul_rn(y.x, 0x1.715476p+0f));   // y / ln2, nearest integer
  const float kf = float(k);
  // y.x - k C1 is exact (Sterbenz: the two are within a factor 2 for k != 0); then y.y and
  // -k C2 join by error-free TwoSums, and the error terms with -k C3 in one FP32 sum
  const float a = __fsub_rn(y.x, __fmul_rn(kf, C1));
  float s1, e1, s2, e2;
  ff_two_sum(a, y.y, s1, e1);
  ff_two_sum(s1, __fmul_rn(-kf, C2), s2, e2);
  const float e = __fmaf_rn(-kf, C3, __fadd_rn(e1, e2));
  float2 r;
  ff_two_sum(s2, e, r.x, r.y);
  float2 p = kInvFact[13];
  for (int n = 12; n >= 0; --n) p = ff_add(ff_mul(p, r), kInvFact[n]);
  const float s = __int_as_float((k + 127) << 23);   // 2^k, k >= -87 here
  return make_float2(__fmul_rn(p.x, s), __fmul_rn(p.y, s));
}

// e^y of n values through exp_ff (the input converted to float-float as the epilogue does,
// the result summed back to FP64): the library's own exponential, exposed for its accuracy test
__global__ void k_selftest_exp_ff(const double *y, double *out, int64_t n) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const float2 e = exp_ff(ff_from_double(y[i]));
  out[i] = double(e.x) + double(e.y);
}

// gauss_in with the exponential in float-float: the FP64 pipe sees only the conversions of x
// in and of the result out; arguments past 60 in the exponent (values below e^-60 of the
// peak) take the FP64 form
__device__ inline double gauss_ff(double x, const RateParams &rp) {
  const float2 r = ff_mul(ff_from_double(x), rp.inv_sigma_ff);
  const float2 r2 = ff_mul(r, r);
  const float2 y = make_float2(-0.5f * r2.x, -0.5f * r2.y);
  if (!(y.x >= -60.f)) return gauss_in(x, rp);
  const float2 g = ff_mul(exp_ff(y), rp.gnorm_ff);
  return double(g.x) + double(g.y);
}

// Delta-cutoff flags of a tuple (bit 0: |e' - e - w| <= cut, bit 1: |e' - e + w| <= cut), the
// decisions of the FP64 expressions below.  An FP32 estimate from FP32 copies of the three
// energies settles every case farther from the cutoff than its error bound: the FP32 inputs
// and two FP32 operations are within 2^-22 of S = |e'| + |e| + |w| of the FP64 values, the FP64
// expressions within 2^-52 S, and cut's FP32 copy within 2^-24 cut; the margin 2^-20 (S + cut)
// covers them with room.  The rest take the FP64 expressions.  The count pass and the rate
// epilogue use this one function, so their decisions agree.
__device__ inline int cut_flags(double ekpn, double ekm, double wqs, float fkpn, float fkm, float fwqs, double cut) {
  const float cutf = float(cut);
  const float de = __fsub_rn(fkpn, fkm);
  const float ap = fabsf(__fsub_rn(de, fwqs)), am = fabsf(__fadd_rn(de, fwqs));
  const float tol = __fmul_rn(__fadd_rn(__fadd_rn(__fadd_rn(fabsf(fkpn), fabsf(fkm)), fabsf(fwqs)), cutf), 0x1p-20f);
  const float lo = __fsub_rn(cutf, tol), hi = __fadd_rn(cutf, tol);
  if ((ap < lo || ap > hi) && (am < lo || am > hi)) return (ap < lo ? 1 : 0) | (am < lo ? 2 : 0);
  const double dxp = ekpn - ekm - wqs;
  const double dxm = ekpn - ekm + wqs;
  return (fabs(dxp) <= cut ? 1 : 0) | (fabs(dxm) <= cut ? 2 : 0);
}

// ------------------------------------------------------------------------ tetrahedron delta
// The analytic (linear) tetrahedron method of "Workflow and structure" for the energy-conserving
// delta (reading [A22]): for the process <k>m -> k'n with k' = <k> + r q, the function
// Delta+-(q') = eps_n(<k> + r q') - eps_m(<k>) -/+ hbar w_s(q') is interpolated linearly in the six
// tetrahedra of every cube of the q mesh, and (1/N_q) delta(Delta) at mesh point q becomes the
// weight of q in that integral: the sum over the 24 tetrahedra containing q of q's corner weight
// W_c = (1/V) int_T delta(Delta) lambda_c, divided by 6 N_q.  Modes at or below omega_min enter
// Delta with w = 0.  The six tetrahedra of a cube lie around one body diagonal; that subdivision
// is not invariant under the cubic group, so the weights are averaged over the four diagonals
// (the diagonal 0-7 and its images: corners c -> c ^ a, a = 1, 2, 4).  No width and no cutoff:
// an entry exists where a weight is positive.
__constant__ unsigned char kCubeTets[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                              {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

// weight W_c of corner c of one tetrahedron with corner values e at the level 0: the level set is
// a triangle or a quadrilateral on the edges (i, j) of the energy-sorted corners with
// e_i < 0 < e_j; int lambda_c dA / |grad e| over it in the coordinates (lambda_2, lambda_3,
// lambda_4) of the sorted corners, where the simplex has volume 1/6
__device__ inline double tetra_corner_weight(const double e[4], int c) {
  int o[4] = {0, 1, 2, 3};
  for (int i = 1; i < 4; ++i) {   // stable sort of the corners by value
    const int x = o[i];
    int j = i - 1;
    while (j >= 0 && e[o[j]] > e[x]) {
      o[j + 1] = o[j];
      --j;
    }
    o[j + 1] = x;
  }
  const double es[4] = {e[o[0]], e[o[1]], e[o[2]], e[o[3]]};
  if (!(es[0] < 0.0 && 0.0 < es[3])) return 0.0;
  int pc = 0;
  for (int i = 0; i < 4; ++i)
    if (o[i] == c) pc = i;
  int ei[4], ej[4], np;
  if (0.0 < es[1]) {
    np = 3; ei[0] = 0; ej[0] = 1; ei[1] = 0; ej[1] = 2; ei[2] = 0; ej[2] = 3;
  } else if (0.0 < es[2]) {
    np = 4; ei[0] = 0; ej[0] = 2; ei[1] = 0; ej[1] = 3; ei[2] = 1; ej[2] = 3; ei[3] = 1; ej[3] = 2;
  } else {
    np = 3; ei[0] = 0; ej[0] = 3; ei[1] = 1; ej[1] = 3; ei[2] = 2; ej[2] = 3;
  }
  double x[4][3], lc[4];
  for (int p = 0; p < np; ++p) {
    const double t = (0.0 - es[ei[p]]) / (es[ej[p]] - es[ei[p]]);
    double lam[4] = {0.0, 0.0, 0.0, 0.0};
    lam[ei[p]] = 1.0 - t;
    lam[ej[p]] = t;
    x[p][0] = lam[1];
    x[p][1] = lam[2];
    x[p][2] = lam[3];
    lc[p] = lam[pc];
  }
  auto tri = [&](int a, int b, int d) {
    const double u0 = x[b][0] - x[a][0], u1 = x[b][1] - x[a][1], u2 = x[b][2] - x[a][2];
    const double v0 = x[d][0] - x[a][0], v1 = x[d][1] - x[a][1], v2 = x[d][2] - x[a][2];
    const double c0 = u1 * v2 - u2 * v1, c1 = u2 * v0 - u0 * v2, c2 = u0 * v1 - u1 * v0;
    return 0.5 * sqrt(c0 * c0 + c1 * c1 + c2 * c2) * (lc[a] + lc[b] + lc[d]) / 3.0;
  };
  double acc = tri(0, 1, 2);
  if (np == 4) acc += tri(0, 2, 3);
  const double g0 = es[1] - es[0], g1 = es[2] - es[0], g2 = es[3] - es[0];
  return acc / (sqrt(g0 * g0 + g1 * g1 + g2 * g2) / 6.0);
}

// N_q times the tetrahedron weights of mesh point q for both processes: wp for
// Delta+ = eps_n(k + r q') - eps_m(k) - w_s(q') and wm for Delta- (+ w_s)
__device__ inline void tetra_pair_weights(const MeshDev &D, int nb, int nbr, int k, int m, int n, int s, int q,
                                          double &wp, double &wm) {
  int a0, a1, a2, b0, b1, b2;
  D.km.unflat(k, a0, a1, a2);
  D.qm.unflat(q, b0, b1, b2);
  const double em = D.eps[size_t(k) * nb + m];
  double accp = 0.0, accm = 0.0;
  for (int cb = 0; cb < 8; ++cb) {
    const int o0 = b0 - (cb & 1), o1 = b1 - ((cb >> 1) & 1), o2 = b2 - ((cb >> 2) & 1);
    for (int dt = 0; dt < 24; ++dt) {
      const int t = dt % 6, flip = dt < 6 ? 0 : (1 << (dt / 6 - 1));   // diagonal images c ^ 1, 2, 4
      int c = -1;
      for (int i = 0; i < 4; ++i)
        if ((kCubeTets[t][i] ^ flip) == cb) c = i;
      if (c < 0) continue;
      double ep[4], en[4];
      for (int i = 0; i < 4; ++i) {
        const int cr = kCubeTets[t][i] ^ flip;
        const int q0 = pmod(o0 + (cr & 1), D.qm.n[0]), q1 = pmod(o1 + ((cr >> 1) & 1), D.qm.n[1]),
                  q2 = pmod(o2 + ((cr >> 2) & 1), D.qm.n[2]);
        const int qq = D.qm.flat(q0, q1, q2);
        const int kk = D.km.flat(pmod(a0 + D.ratio[0] * q0, D.km.n[0]), pmod(a1 + D.ratio[1] * q1, D.km.n[1]),
                                 pmod(a2 + D.ratio[2] * q2, D.km.n[2]));
        const double wv = D.w[size_t(qq) * nbr + s];
        const double w = wv > D.omega_min ? wv : 0.0;
        const double d = D.eps[size_t(kk) * nb + n] - em;
        ep[i] = d - w;
        en[i] = d + w;
      }
      accp += tetra_corner_weight(ep, c);
      accm += tetra_corner_weight(en, c);
    }
  }
  wp = accp / 24.0;   // 1/6 per tetrahedron, 1/4 per subdivision
  wm = accm / 24.0;
}

// ------------------------------------------------------------------------ count pass
__global__ void k_rate_count(ModelDev M, MeshDev D, RateParams rp, int *cntE, int *cntPh,
                             unsigned long long *n_tuples) {
  int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  unsigned long long nt = 0, fl = 0, ns = 0, rf = 0;
  if (p < D.n_pairs) {
    const int nb = M.nb, nbr = M.nbr;
    int i = D.pair_i[p], q = D.pair_q[p];
    int k = D.ibzw_list[i];
    int kp = kplusq_d(D, k, q);
    uint32_t am = D.amask[k], an = D.amask[kp];
    int64_t p0 = D.pair_ptr[i];
    int64_t npl = D.pair_ptr[i + 1] - p0, pl = p - p0;
    // algorithmic flops of stage B for this pair: R_ph sum, branch rotation, band rotation (over
    // the rotation bands: the active ones and their degenerate partners)
    const unsigned long long na = __popc(D.rmask[k]), nap = __popc(D.rmask[kp]);
    fl = 8ull * (na * nb * nbr * (unsigned long long)M.nRgp + na * nb * nbr * nbr + na * nap * nb * nbr);
    if (pl == 0) ns = na;
    rf = 8ull * (na * nb * nbr * nbr + na * nap * nb * nbr);   // rotations only
    const double *ek = D.eps + size_t(k) * nb, *ekp = D.eps + size_t(kp) * nb, *wq = D.w + size_t(q) * nbr;
    const float *fk = rp.eps32 + size_t(k) * nb, *fkp = rp.eps32 + size_t(kp) * nb, *fw = rp.w32 + size_t(q) * nbr;
    int64_t qb = D.qpair_ptr[q];
    int64_t npq = D.qpair_ptr[q + 1] - qb;
    int cph[kMaxBranches];
    for (int s = 0; s < nbr; ++s) cph[s] = 0;
    for (int m = 0; m < nb; ++m) {
      int c = 0;
      if ((am >> m) & 1u)
        for (int n = 0; n < nb; ++n) {
          if (!((an >> n) & 1u)) continue;
          for (int s = 0; s < nbr; ++s) {
            if (!(wq[s] > D.omega_min)) continue;
            ++nt;
            int f;
            if (rp.tetra) {
              double wpt, wmt;
              tetra_pair_weights(D, nb, nbr, k, m, n, s, q, wpt, wmt);
              f = (wpt > 0.0 ? 1 : 0) | (wmt > 0.0 ? 2 : 0);
            } else {
              f = cut_flags(ekp[n], ek[m], wq[s], fkp[n], fk[m], fw[s], rp.cut);
            }
            c += f != 0;
            cph[s] += f & 1;
          }
        }
      cntE[p0 * nb + m * npl + pl] = c;
    }
    for (int s = 0; s < nbr; ++s) cntPh[qb * nbr + s * npq + D.pq_rank[p]] = cph[s];
  }
  for (int o = 16; o > 0; o >>= 1) {
    nt += __shfl_down_sync(0xffffffffu, nt, o);
    fl += __shfl_down_sync(0xffffffffu, fl, o);
    rf += __shfl_down_sync(0xffffffffu, rf, o);
    ns += __shfl_down_sync(0xffffffffu, ns, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (nt) atomicAdd(n_tuples, nt);
    if (fl) atomicAdd(n_tuples + 2, fl);
    if (rf) atomicAdd(n_tuples + 4, rf);
    if (ns) atomicAdd(n_tuples + 3, ns);
  }
}

// electron row starts (k,m) and phonon row starts (q,s) from the scanned count layouts
__global__ void k_row_ptrs(MeshDev D, int nb, int nbr, const int64_t *escan, const int64_t *phscan,
                           int64_t e_total, int64_t ph_total, int64_t *row_ptr, int64_t *ph_row_ptr) {
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int64_t ne = D.n_ibzw * nb, nph = D.nq * nbr;
  if (t < ne) {
    int64_t i = t / nb, m = t % nb;
    int64_t p0 = D.pair_ptr[i], npl = D.pair_ptr[i + 1] - p0;
    int64_t idx = p0 * nb + m * npl;
    row_ptr[t] = idx < D.n_pairs * nb ? escan[idx] : e_total;
  }
  if (t == ne) row_ptr[ne] = e_total;
  if (t < nph) {
    int64_t q = t / nbr, s = t % nbr;
    int64_t qb = D.qpair_ptr[q], npq = D.qpair_ptr[q + 1] - qb;
    int64_t idx = qb * nbr + s * npq;
    ph_row_ptr[t] = idx < D.n_pairs * nbr ? phscan[idx] : ph_total;
  }
  if (t == nph) ph_row_ptr[nph] = ph_total;
}

// ------------------------------------------------------------------------ stage A
constexpr int kAKT = 8;   // k points per block

// T[kc][col] = sum_re e^{i k.Re} gW[re][col], col = (rp, m', n', a)
__global__ void __launch_bounds__(256) k_stage_a1(ModelDev M, MeshDev D, int64_t i0, int64_t nkc, double2 *T) {
  extern __shared__ double2 sph[];   // [kAKT][nRge]
  const int64_t ncol = int64_t(M.nRgp) * M.nb * M.nb * M.nbr;
  const int64_t kc0 = int64_t(blockIdx.y) * kAKT;
  for (int t = threadIdx.x; t < kAKT * M.nRge; t += blockDim.x) {
    int kk = t / M.nRge, re = t % M.nRge;
    double2 ph = cmk(0, 0);
    if (kc0 + kk < nkc) {
      int k = D.ibzw_list[i0 + kc0 + kk];
      int a0, a1, a2;
      D.km.unflat(k, a0, a1, a2);
      ph = mesh_phase(D.ktab, D.km, a0, a1, a2, M.Rge[3 * re], M.Rge[3 * re + 1], M.Rge[3 * re + 2]);
    }
    sph[t] = ph;
  }
  __syncthreads();
  int64_t col = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (col >= ncol) return;
  double2 acc[kAKT];
  for (int kk = 0; kk < kAKT; ++kk) acc[kk] = cmk(0, 0);
  for (int re = 0; re < M.nRge; ++re) {
    double2 g = M.g_R[re * ncol + col];
    for (int kk = 0; kk < kAKT; ++kk) cfma(acc[kk], sph[kk * M.nRge + re], g);
  }
  for (int kk = 0; kk < kAKT; ++kk)
    if (kc0 + kk < nkc) T[(kc0 + kk) * ncol + col] = acc[kk];
}

// A[kc][rp][j], j = ml*(nb*nbr) + n'*nbr + a over the rotation bands m of k (the active bands
// and their degenerate partners):
//   A = sum_m' c_{m'm}(k) T[kc][rp][m'][n'][a]
// FF: T holds float-float pairs (hi, lo) per real value, each read as the FP64 value hi + lo.
template <bool FF>
__global__ void k_stage_a2(ModelDev M, MeshDev D, int64_t i0, int64_t nkc, const double2 *T, double2 *A) {
  const int nb = M.nb, nbr = M.nbr;
  const int64_t jmax = int64_t(nb) * nb * nbr;
  const int64_t per_k = int64_t(M.nRgp) * jmax;
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nkc * per_k) return;
  int64_t kc = t / per_k, r = t % per_k;
  int rp = int(r / jmax), j = int(r % jmax);
  int ml = j / (nb * nbr), na = j % (nb * nbr);
  int k = D.ibzw_list[i0 + kc];
  uint32_t rm = D.rmask[k];
  // the tensor-core path's B' slicing reads only the rows of rotating bands (it writes zero
  // slices for the others), so there the rest is not written at all
  if (FF && ml >= __popc(rm)) return;
  double2 acc = cmk(0, 0);
  if (ml < __popc(rm)) {
    int m = nth_bit(rm, ml);
    const int64_t t0 = kc * per_k + int64_t(rp) * jmax;
    const double2 *ck = D.cvec + size_t(k) * nb * nb;
    for (int mp = 0; mp < nb; ++mp) {
      const int64_t idx = t0 + mp * nb * nbr + na;
      double2 tv;
      if (FF) {
        const float4 f = reinterpret_cast<const float4 *>(T)[idx];
        tv = cmk(double(f.x) + double(f.y), double(f.z) + double(f.w));
      } else {
        tv = T[idx];
      }
      cfma(acc, ck[mp * nb + m], tv);
    }
  }
  A[t] = acc;
}

// ------------------------------------------------------------------------ stage B + rates
constexpr int kBT = 256;       // threads
constexpr int kNR = 12;        // complex accumulators per thread
constexpr int kRC = 16;        // R_ph chunk
constexpr int kTPMax = 64;     // pairs per tile

struct StageBSmem {
  int jmax, tpmax, rc;
  size_t off_B, off_ph, off_A, off_w, per_warp, total;
};

__host__ __device__ inline StageBSmem stage_b_layout(int nb, int nbr) {
  StageBSmem L;
  L.jmax = nb * nb * nbr;
  L.tpmax = kTPMax;
  L.rc = L.jmax > 192 ? 8 : kRC;
  L.off_B = 0;
  L.off_ph = L.off_B + size_t(kBT) * kNR * sizeof(double2);
  L.off_A = L.off_ph + size_t(L.tpmax) * L.rc * sizeof(double2);
  L.off_w = L.off_A + size_t(L.rc) * L.jmax * sizeof(double2);
  L.per_warp = size_t(L.jmax) * sizeof(double2) + 3 * size_t(nb) * nb * nbr * sizeof(double);
  L.per_warp = (L.per_warp + 15) & ~size_t(15);   // every warp's double2 scratch stays 16-byte aligned
  L.total = L.off_w + (kBT / 32) * L.per_warp;
  return L;
}

// Rotations, |g|^2, degenerate average, occupations, delta and the compacted writes of one
// (k, q) pair, executed by one warp.  Bp holds B[ml][n'][alpha] = sum_Rp e^{iq.Rp} A (complex).
__device__ void pair_epilogue(const ModelDev &M, const MeshDev &D, const RateParams &rp, int64_t i, int k,
                              uint32_t am, uint32_t rm, int nrot, int Jk, int64_t p0, int64_t npl, int64_t pg,
                              const double2 *Bp, double2 *Zs, double *g2s, double *Xps, double *Xms,
                              const double *mscale, double inv_stab, const double *ek, double kT,
                              const int64_t *__restrict__ escan, const int64_t *__restrict__ phscan,
                              uint32_t *e_kpns, double2 *e_X, int *ph_st, uint32_t *ph_kpn, double *ph_Y) {
  const int nb = M.nb, nbr = M.nbr;
  const int lane = threadIdx.x & 31;
  const int q = D.pair_q[pg];
  const int kp = kplusq_d(D, k, q);
  // emission: active bands am (k), an (k'); rotations: rm, rn (with the degenerate partners)
  const uint32_t an = D.amask[kp], rn = D.rmask[kp];
  const int nact = __popc(am), nactp = __popc(an), nrotp = __popc(rn);
  const double2 *uq = D.u + size_t(q) * nbr * nbr;
  const double *wq = D.w + size_t(q) * nbr;
  const double2 *ckp = D.cvec + size_t(kp) * nb * nb;
  const double *ekp = D.eps + size_t(kp) * nb;
    // Z[ml][n'][s] = sum_a B[ml][n'][a] u_{a s}(q) / sqrt(m_a / m_bar)
  for (int t = lane; t < Jk; t += 32) {
    int ml = t / (nb * nbr), np_ = (t / nbr) % nb, s = t % nbr;
    double2 z = cmk(0, 0);
    for (int a = 0; a < nbr; ++a)
      cfma(z, Bp[(ml * nb + np_) * nbr + a], cscale(uq[a * nbr + s], mscale[a]));
    Zs[t] = z;
  }
  __syncwarp();
  // g[ml][nl][s] = sqrt(w_ref / w_s) sum_n' conj(c_{n'n}(k')) Z[ml][n'][s], rotation bands
  const int nrtup = nrot * nrotp * nbr;
  for (int t = lane; t < nrtup; t += 32) {
    int ml = t / (nrotp * nbr), nl = (t / nbr) % nrotp, s = t % nbr;
    int n = nth_bit(rn, nl);
    double v = 0.0;
    if (wq[s] > D.omega_min) {
      double2 g = cmk(0, 0);
      for (int np_ = 0; np_ < nb; ++np_) cfma_conj(g, ckp[np_ * nb + n], Zs[(ml * nb + np_) * nbr + s]);
      v = cabs2(g) * (M.omega_ref / wq[s]);
    }
    g2s[t] = v;
  }
  __syncwarp();
  // degenerate averages, occupations, delta; pass flags go to the (now free) Z scratch
  int *flg = reinterpret_cast<int *>(Zs);
  const uint8_t *gk = D.egrp + size_t(k) * nb * 2, *gkp = D.egrp + size_t(kp) * nb * 2;
  const uint8_t *gq = D.pgrp + size_t(q) * nbr * 2;
  const int ntup = nact * nactp * nbr;
  for (int t = lane; t < ntup; t += 32) {
    int ml = t / (nactp * nbr), nl = (t / nbr) % nactp, s = t % nbr;
    int m = nth_bit(am, ml), n = nth_bit(an, nl);
    double xp = 0.0, xm = 0.0;
    if (wq[s] > D.omega_min) {
      // average over the whole degenerate subspaces (every member is a rotation band)
      double sum = 0.0;
      int cnt = 0;
      for (int a = gk[2 * m]; a < gk[2 * m + 1]; ++a) {
        int al = __popc(rm & ((1u << a) - 1u));
        for (int b = gkp[2 * n]; b < gkp[2 * n + 1]; ++b) {
          int bl = __popc(rn & ((1u << b) - 1u));
          for (int c = gq[2 * s]; c < gq[2 * s + 1]; ++c) {
            sum += g2s[(al * nrotp + bl) * nbr + c];
            ++cnt;
          }
        }
      }
      double g2 = cnt == 1 ? sum : sum / double(cnt);
      double dxp = ekp[n] - ek[m] - wq[s];
      double dxm = ekp[n] - ek[m] + wq[s];
      double dp, dm;   // N_q times the (1/N_q) delta weights
      if (rp.tetra) {
        tetra_pair_weights(D, nb, nbr, k, m, n, s, q, dp, dm);
      } else {
        dp = gauss_d(dxp, rp);
        dm = gauss_d(dxm, rp);
      }
      if (rp.vertex_only) {   // T-independent vertex weights V+-: occupation factors left out
        const double v = rp.inv_Nq_pref * g2;
        xp = v * dp;
        xm = v * dm;
      } else {
        double fm = fermi_d(ek[m], rp.mu, kT), fn = fermi_d(ekp[n], rp.mu, kT), nq = bose_d(wq[s], kT);
        double occ = rp.inv_Nq_pref * g2 * fm * (1.0 - fn);
        xp = occ * nq * dp;
        xm = occ * (1.0 + nq) * dm;
      }
      Xps[t] = xp;
      Xms[t] = xm;
      flg[t] = rp.tetra ? ((dp > 0.0 ? 1 : 0) | (dm > 0.0 ? 2 : 0))
                        : ((fabs(dxp) <= rp.cut ? 1 : 0) | (fabs(dxm) <= rp.cut ? 2 : 0));
    } else {
      Xps[t] = 0.0;
      Xms[t] = 0.0;
      flg[t] = 0;
    }
  }
  __syncwarp();
  // electron rows (k, m): entries ordered (n, s)
  const int64_t pl = pg - p0;
  for (int ml = 0; ml < nact; ++ml) {
    const int m = nth_bit(am, ml);
    int64_t base = escan[p0 * nb + m * npl + pl];
    const int nit = nactp * nbr;
    for (int c0 = 0; c0 < nit; c0 += 32) {
      int t = c0 + lane;
      int flag = 0, idx = 0;
      if (t < nit) {
        idx = ml * nit + t;
        flag = flg[idx] != 0;
      }
      unsigned b = __ballot_sync(0xffffffffu, flag);
      if (flag) {
        int64_t pos = base + __popc(b & ((1u << lane) - 1u));
        int nl = t / nbr, s = t % nbr;
        e_kpns[pos] = pack_kpns(kp, nth_bit(an, nl), s);
        e_X[pos] = cmk(Xps[idx], Xms[idx]);
      }
      base += __popc(b);
    }
  }
  // phonon rows (q, s): entries ordered (m, n), absorption (+) processes only
  const int64_t qb = D.qpair_ptr[q];
  const int64_t npq = D.qpair_ptr[q + 1] - qb;
  const int rk = D.pq_rank[pg];
  for (int s = 0; s < nbr; ++s) {
    if (!(wq[s] > D.omega_min)) continue;
    int64_t base = phscan[qb * nbr + s * npq + rk];
    const int nit = nact * nactp;
    for (int c0 = 0; c0 < nit; c0 += 32) {
      int t = c0 + lane;
      int flag = 0, idx = 0;
      if (t < nit) {
        idx = t * nbr + s;
        flag = (flg[idx] & 1) != 0;
      }
      unsigned b = __ballot_sync(0xffffffffu, flag);
      if (flag) {
        int64_t pos = base + __popc(b & ((1u << lane) - 1u));
        int ml = t / nactp, nl = t % nactp;
        ph_st[pos] = int(i) * nb + nth_bit(am, ml);
        ph_kpn[pos] = pack_kpns(kp, nth_bit(an, nl), 0);
        ph_Y[pos] = Xps[idx] * rp.y_scale * inv_stab;
      }
      base += __popc(b);
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kBT) k_stage_b_rates(ModelDev M, MeshDev D, RateParams rp, int64_t i0,
                                                       const double2 *__restrict__ A,
                                                       const int64_t *__restrict__ escan,
                                                       const int64_t *__restrict__ phscan, uint32_t *e_kpns,
                                                       double2 *e_X, int *ph_st, uint32_t *ph_kpn, double *ph_Y) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nb = M.nb, nbr = M.nbr;
  const StageBSmem L = stage_b_layout(nb, nbr);
  double2 *Bsh = reinterpret_cast<double2 *>(smem + L.off_B);
  double2 *phs = reinterpret_cast<double2 *>(smem + L.off_ph);
  double2 *Ash = reinterpret_cast<double2 *>(smem + L.off_A);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char *wscr = smem + L.off_w + wid * L.per_warp;
  double2 *Zs = reinterpret_cast<double2 *>(wscr);
  double *g2s = reinterpret_cast<double *>(wscr + size_t(L.jmax) * sizeof(double2));
  double *Xps = g2s + nb * nb * nbr;
  double *Xms = Xps + nb * nb * nbr;

  const int64_t i = i0 + blockIdx.x;
  const int k = D.ibzw_list[i];
  const uint32_t am = D.amask[k], rm = D.rmask[k];
  const int nrot = __popc(rm);
  const int Jk = nrot * nb * nbr;
  const int64_t p0 = D.pair_ptr[i];
  const int64_t npl = D.pair_ptr[i + 1] - p0;
  const double2 *Ak = A + size_t(blockIdx.x) * M.nRgp * L.jmax;
  int TP = (kBT * kNR) / Jk;
  TP = TP > L.tpmax ? L.tpmax : TP;
  const double kT = kKbEVK * rp.T;
  const double *ek = D.eps + size_t(k) * nb;
  const double inv_stab = 1.0 / double(D.stab[k]);
  double mscale[kMaxBranches];
  for (int a = 0; a < nbr; ++a) mscale[a] = 1.0 / sqrt(M.mass[a / 3] / M.mass_mean);

  for (int64_t t0 = 0; t0 < npl; t0 += TP) {
    const int npt = int((npl - t0) < TP ? (npl - t0) : TP);
    double2 acc[kNR];
#pragma unroll
    for (int r = 0; r < kNR; ++r) acc[r] = cmk(0, 0);
    for (int r0 = 0; r0 < M.nRgp; r0 += L.rc) {
      const int rc = (M.nRgp - r0) < L.rc ? (M.nRgp - r0) : L.rc;
      __syncthreads();
      for (int t = threadIdx.x; t < rc * Jk; t += kBT) {
        int rr = t / Jk, j = t % Jk;
        Ash[rr * L.jmax + j] = Ak[size_t(r0 + rr) * L.jmax + j];
      }
      for (int t = threadIdx.x; t < npt * L.rc; t += kBT) {
        int p = t / L.rc, rr = t % L.rc;
        double2 ph = cmk(0, 0);
        if (rr < rc) {
          int q = D.pair_q[p0 + t0 + p];
          int b0, b1, b2;
          D.qm.unflat(q, b0, b1, b2);
          const int *R = M.Rgp + 3 * (r0 + rr);
          ph = mesh_phase(D.qtab, D.qm, b0, b1, b2, R[0], R[1], R[2]);
        }
        phs[t] = ph;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kNR; ++r) {
        int o = threadIdx.x + kBT * r;
        if (o < npt * Jk) {
          int p = o / Jk, j = o - p * Jk;
          const double2 *php = phs + p * L.rc;
          for (int rr = 0; rr < rc; ++rr) cfma(acc[r], php[rr], Ash[rr * L.jmax + j]);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kNR; ++r) {
      int o = threadIdx.x + kBT * r;
      if (o < npt * Jk) Bsh[o] = acc[r];
    }
    __syncthreads();

    // ---- epilogue: one warp per pair
    for (int p = wid; p < npt; p += kBT / 32)
      pair_epilogue(M, D, rp, i, k, am, rm, nrot, Jk, p0, npl, p0 + t0 + p, Bsh + p * Jk, Zs, g2s, Xps, Xms, mscale,
                    inv_stab, ek, kT, escan, phscan, e_kpns, e_X, ph_st, ph_kpn, ph_Y);
  }
}

// Per-rate-build tables of the rate epilogue: Fermi occupation of every (k, band); Bose
// occupation, w_ref/w prefactor (0 for excluded modes) and mass-scaled eigenvectors
// u_{a s}(q) / sqrt(m_a / m_bar) of every (q, branch).
__global__ void k_epi_tables(ModelDev M, MeshDev D, double T, double mu, double *fk, double *nbq, double *wr,
                             double2 *ut) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int nb = M.nb, nbr = M.nbr;
  const double kT = kKbEVK * T;
  // occupations are read only at the end points of pairs, whose bands rotate (rmask != 0);
  // the rest are set to 0 without the exponential
  if (t < D.nk * nb) fk[t] = D.rmask[t / nb] ? fermi_d(D.eps[t], mu, kT) : 0.0;
  if (t < D.nq * nbr) {
    const double w = D.w[t];
    nbq[t] = bose_d(w, kT);
    wr[t] = w > D.omega_min ? M.omega_ref / w : 0.0;
  }
  if (t < D.nq * nbr * nbr) {
    const int a = int((t / nbr) % nbr);
    ut[t] = cscale(D.u[t], 1.0 / sqrt(M.mass[a / 3] / M.mass_mean));
  }
}

// Float-float copies of the final-band eigenvectors c(k) ([k][n'][n]) and of the mass-scaled
// phonon eigenvectors ([q][a][s]) for the FP64-grade epilogue: (re hi, re lo, im hi, im lo).
// c(k) is read only for k' = k + q of a pair, which has an active band: points without one
// (rmask 0) are not written.
__global__ void k_ff_tables(int64_t nc, int nb2, const uint32_t *__restrict__ rmask, const double2 *cvec, int64_t nu,
                            const double2 *ut, float4 *cff, float4 *uff) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < nc && rmask[t / nb2]) {
    const float2 r = ff_from_double(cvec[t].x), i = ff_from_double(cvec[t].y);
    cff[t] = make_float4(r.x, r.y, i.x, i.y);
  }
  if (t < nu) {
    const float2 r = ff_from_double(ut[t].x), i = ff_from_double(ut[t].y);
    uff[t] = make_float4(r.x, r.y, i.x, i.y);
  }
}

// Rates from a contraction held in Cbuf: C'[pair][j'] with j' = ml*(2 nb nbr) + part*(nb nbr)
// + n'*nbr + a (part 0: real, 1: imaginary).  One thread per (k, q) pair, so every lane works
// even when a pair has only a handful of (m, n, s) tuples.  The final-band index is contracted
// before the branch index, W[m n a] = sum_n' conj(c_{n'n}(k')) B[m n' a], then
// g[m n s] = sqrt(w_ref/w_s) sum_a W[m n a] u_{a s}(q)/sqrt(m_a/m_bar): the same product as
// the fused kernel, with nact' instead of nb final-band rows in the branch rotation.
// ROT32: the band and branch rotations in FP32 (mixed mode, whose contraction is ~1e-7 accurate
// anyway); |g|^2 is then carried on in FP64 like the rest of the epilogue.
template <int NBM, int NBRM, bool ROT32>
__global__ void __launch_bounds__(128) k_rate_epilogue(ModelDev M, MeshDev D, RateParams rp, int64_t pbeg,
                                                       int64_t pend, int64_t pair_base, const double *__restrict__ Cbuf,
                                                       int Nmax, const double *__restrict__ fk,
                                                       const double *__restrict__ nbq, const double *__restrict__ wr,
                                                       const double2 *__restrict__ ut,
                                                       const float4 *__restrict__ cff, const float4 *__restrict__ uff,
                                                       const int64_t *__restrict__ escan,
                                                       const int64_t *__restrict__ phscan, uint32_t *e_kpns,
                                                       double2 *e_X, int *ph_st, uint32_t *ph_kpn, double *ph_Y) {
  const int64_t pg = pbeg + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (pg >= pend) return;
  const int nb = M.nb, nbr = M.nbr, nbnbr = nb * nbr;
  const int i = D.pair_i[pg], q = D.pair_q[pg];
  const int k = D.ibzw_list[i];
  const int kp = kplusq_d(D, k, q);
  // emission: active bands am (k), an (k'); rotations: rm, rn (with the degenerate partners)
  const uint32_t am = D.amask[k], an = D.amask[kp], rm = D.rmask[k], rn = D.rmask[kp];
  const int nact = __popc(am), nactp = __popc(an), nrot = __popc(rm), nrotp = __popc(rn);
  const int64_t p0 = D.pair_ptr[i];
  const int64_t npl = D.pair_ptr[i + 1] - p0;
  const float2 *crow = reinterpret_cast<const float2 *>(Cbuf) + (pg - pair_base) * Nmax;
  const double2 *ckp = D.cvec + size_t(kp) * nb * nb;
  const double2 *uq = ut + size_t(q) * nbr * nbr;
  const double *wrq = wr + size_t(q) * nbr;
  // |g|^2 per (m, n, s) as a float-float pair; the FP64 conversion and the w_ref/w factor are
  // applied only where a tuple inside the delta cutoff needs the value
  float2 g2[NBM * NBM * NBRM];
  if (ROT32) {
    for (int ml = 0; ml < nrot; ++ml)
      for (int nl = 0; nl < nrotp; ++nl) {
        const int n = nth_bit(rn, nl);
        float Wr[NBRM], Wi[NBRM];
        for (int a = 0; a < nbr; ++a) Wr[a] = Wi[a] = 0.f;
        for (int np_ = 0; np_ < nb; ++np_) {
          const double2 c = ckp[np_ * nb + n];
          const float cr = float(c.x), ci = float(c.y);
          const float2 *re = crow + ml * 2 * nbnbr + np_ * nbr;
          for (int a = 0; a < nbr; ++a) {   // W += conj(c) B
            const float br = re[a].x + re[a].y, bi = re[nbnbr + a].x + re[nbnbr + a].y;
            Wr[a] = fmaf(cr, br, fmaf(ci, bi, Wr[a]));
            Wi[a] = fmaf(cr, bi, fmaf(-ci, br, Wi[a]));
          }
        }
        for (int s = 0; s < nbr; ++s) {
          float gr = 0.f, gi = 0.f;
          for (int a = 0; a < nbr; ++a) {   // g += W u
            const double2 u = uq[a * nbr + s];
            const float ur = float(u.x), ui = float(u.y);
            gr = fmaf(Wr[a], ur, fmaf(-Wi[a], ui, gr));
            gi = fmaf(Wr[a], ui, fmaf(Wi[a], ur, gi));
          }
          g2[(ml * nrotp + nl) * nbr + s] = make_float2(gr * gr + gi * gi, 0.f);
        }
      }
  } else {
    // FP64-grade rotations in float-float arithmetic (~2^-47 of the summed magnitudes) on the
    // FP32 pipe: C' arrives as float-float pairs, c(k') and u(q) from float-float tables;
    // |g|^2 goes to FP64 once per (m, n, s)
    const float4 *cf = cff + size_t(kp) * nb * nb;
    const float4 *uf = uff + size_t(q) * nbr * nbr;
    for (int ml = 0; ml < nrot; ++ml)
      for (int nl = 0; nl < nrotp; ++nl) {
        const int n = nth_bit(rn, nl);
        FFAcc Wr[NBRM], Wi[NBRM];
        for (int np_ = 0; np_ < nb; ++np_) {
          const float4 c4 = cf[np_ * nb + n];
          const float2 cr = make_float2(c4.x, c4.y), ci = make_float2(c4.z, c4.w);
          const float2 *re = crow + ml * 2 * nbnbr + np_ * nbr;
          for (int a = 0; a < nbr; ++a) {   // W += conj(c) B
            const float2 br = re[a], bi = re[nbnbr + a];
            ff_acc_mul(Wr[a], cr, br);
            ff_acc_mul(Wr[a], ci, bi);
            ff_acc_mul(Wi[a], cr, bi);
            ff_acc_mul(Wi[a], ff_neg(ci), br);
          }
        }
        float2 wr2[NBRM], wi2[NBRM];
        for (int a = 0; a < nbr; ++a) {
          wr2[a] = ff_norm(Wr[a]);
          wi2[a] = ff_norm(Wi[a]);
        }
        for (int s = 0; s < nbr; ++s) {
          FFAcc gr, gi;
          for (int a = 0; a < nbr; ++a) {   // g += W u
            const float4 u4 = uf[a * nbr + s];
            const float2 ur = make_float2(u4.x, u4.y), ui = make_float2(u4.z, u4.w);
            ff_acc_mul(gr, wr2[a], ur);
            ff_acc_mul(gr, ff_neg(wi2[a]), ui);
            ff_acc_mul(gi, wr2[a], ui);
            ff_acc_mul(gi, wi2[a], ur);
          }
          const float2 Gr = ff_norm(gr), Gi = ff_norm(gi);
          FFAcc m2;
          ff_acc_mul(m2, Gr, Gr);
          ff_acc_mul(m2, Gi, Gi);
          g2[(ml * nrotp + nl) * nbr + s] = ff_norm(m2);
        }
      }
  }
  // degenerate averages, occupations (tables), delta
  const double *ek = D.eps + size_t(k) * nb, *ekp = D.eps + size_t(kp) * nb, *wq = D.w + size_t(q) * nbr;
  const uint8_t *gk = D.egrp + size_t(k) * nb * 2, *gkp = D.egrp + size_t(kp) * nb * 2;
  const uint8_t *gq = D.pgrp + size_t(q) * nbr * 2;
  double Xp[NBM * NBM * NBRM], Xm[NBM * NBM * NBRM];
  uint8_t flg[NBM * NBM * NBRM];
  const int ntup = nact * nactp * nbr;
  const float *fk32 = rp.eps32 + size_t(k) * nb, *fkp32 = rp.eps32 + size_t(kp) * nb, *fw32 = rp.w32 + size_t(q) * nbr;
  for (int t = 0; t < ntup; ++t) {
    const int ml = t / (nactp * nbr), nl = (t / nbr) % nactp, s = t % nbr;
    const int m = nth_bit(am, ml), n = nth_bit(an, nl);
    Xp[t] = 0.0;
    Xm[t] = 0.0;
    flg[t] = 0;
    if (!(wq[s] > D.omega_min)) continue;
    // the cutoff test first: tuples with neither delta inside it need no average or occupation
    double tp = 0.0, tm = 0.0;
    int f;
    if (rp.tetra) {
      tetra_pair_weights(D, nb, nbr, k, m, n, s, q, tp, tm);
      f = (tp > 0.0 ? 1 : 0) | (tm > 0.0 ? 2 : 0);
    } else {
      f = cut_flags(ekp[n], ek[m], wq[s], fkp32[n], fk32[m], fw32[s], rp.cut);
    }
    if (!f) continue;
    const bool inp = f & 1, inm = f & 2;
    flg[t] = uint8_t(f);
    const double dxp = ekp[n] - ek[m] - wq[s];
    const double dxm = ekp[n] - ek[m] + wq[s];
    // average over the whole degenerate subspaces (every member is a rotation band)
    double sum = 0.0;
    int cnt = 0;
    for (int a = gk[2 * m]; a < gk[2 * m + 1]; ++a) {
      const int al = __popc(rm & ((1u << a) - 1u));
      for (int b = gkp[2 * n]; b < gkp[2 * n + 1]; ++b) {
        const int bl = __popc(rn & ((1u << b) - 1u));
        for (int c = gq[2 * s]; c < gq[2 * s + 1]; ++c) {
          const float2 v = g2[(al * nrotp + bl) * nbr + c];
          sum += (double(v.x) + double(v.y)) * wrq[c];
          ++cnt;
        }
      }
    }
    const double gp = rp.tetra ? tp : (inp ? gauss_ff(dxp, rp) : 0.0);
    const double gm = rp.tetra ? tm : (inm ? gauss_ff(dxm, rp) : 0.0);
    if (rp.vertex_only) {   // T-independent vertex weights V+-: occupation factors left out
      const double v = rp.inv_Nq_pref * (cnt == 1 ? sum : sum / double(cnt));
      Xp[t] = v * gp;
      Xm[t] = v * gm;
    } else {
      const double nqs = nbq[size_t(q) * nbr + s];
      const double occ =
          rp.inv_Nq_pref * (cnt == 1 ? sum : sum / double(cnt)) * fk[size_t(k) * nb + m] * (1.0 - fk[size_t(kp) * nb + n]);
      Xp[t] = occ * nqs * gp;
      Xm[t] = occ * (1.0 + nqs) * gm;
    }
  }
  // electron rows (k, m): entries ordered (n, s)
  const int64_t pl = pg - p0;
  for (int ml = 0; ml < nact; ++ml) {
    const int m = nth_bit(am, ml);
    int64_t pos = escan[p0 * nb + m * npl + pl];
    for (int u = 0; u < nactp * nbr; ++u) {
      const int t = ml * nactp * nbr + u;
      if (!flg[t]) continue;
      e_kpns[pos] = pack_kpns(kp, nth_bit(an, u / nbr), u % nbr);
      e_X[pos] = cmk(Xp[t], Xm[t]);
      ++pos;
    }
  }
  // phonon rows (q, s): entries ordered (m, n), absorption (+) processes only
  const int64_t qb = D.qpair_ptr[q];
  const int64_t npq = D.qpair_ptr[q + 1] - qb;
  const int rk = D.pq_rank[pg];
  const double ysc = rp.y_scale / double(D.stab[k]);
  for (int s = 0; s < nbr; ++s) {
    if (!(wq[s] > D.omega_min)) continue;
    int64_t pos = phscan[qb * nbr + s * npq + rk];
    for (int u = 0; u < nact * nactp; ++u) {
      const int t = u * nbr + s;
      if (!(flg[t] & 1)) continue;
      ph_st[pos] = i * nb + nth_bit(am, u / nactp);
      ph_kpn[pos] = pack_kpns(kp, nth_bit(an, u % nactp), 0);
      ph_Y[pos] = Xp[t] * ysc;
      ++pos;
    }
  }
}

}  // namespace

cudaError_t launch_epi_tables(const ModelDev &M, const MeshDev &D, double T, double mu, double *fk, double *nbq,
                              double *wr, double2 *ut, cudaStream_t st) {
  int64_t n = D.nk * M.nb;
  if (D.nq * M.nbr * M.nbr > n) n = D.nq * M.nbr * M.nbr;
  EPHB_LAUNCH(k_epi_tables, unsigned((n + 255) / 256), 256, 0, st, M, D, T, mu, fk, nbq, wr, ut);
  return cudaGetLastError();
}

cudaError_t launch_ff_tables(const ModelDev &M, const MeshDev &D, const double2 *ut, float4 *cff, float4 *uff,
                             cudaStream_t st) {
  const int64_t nc = D.nk * M.nb * M.nb, nu = D.nq * M.nbr * M.nbr;
  const int64_t n = nc > nu ? nc : nu;
  if (n == 0) return cudaSuccess;
  EPHB_LAUNCH(k_ff_tables, unsigned((n + 255) / 256), 256, 0, st, nc, M.nb * M.nb, D.rmask, D.cvec, nu, ut, cff,
              uff);
  return cudaGetLastError();
}

cudaError_t launch_vertex_epilogue(const ModelDev &M, const MeshDev &D, RateParams rp, int64_t pbeg, int64_t pend,
                                   int64_t pair_base, const double *Cbuf, int Nmax, const double *fk,
                                   const double *nbq, const double *wr, const double2 *ut, const float4 *cff,
                                   const float4 *uff, const int64_t *escan,
                                   const int64_t *phscan, uint32_t *e_kpns, double2 *e_X, int *ph_st,
                                   uint32_t *ph_kpn, double *ph_Y, cudaStream_t st) {
  if (pend <= pbeg) return cudaSuccess;
  const unsigned grid = unsigned((pend - pbeg + 127) / 128);
  auto go = [&](auto kern) {
    EPHB_LAUNCH(kern, grid, 128, 0, st, M, D, rp, pbeg, pend, pair_base, Cbuf, Nmax, fk, nbq, wr, ut, cff, uff, escan,
                phscan, e_kpns, e_X, ph_st, ph_kpn, ph_Y);
  };
  if (M.nb <= 1 && M.nbr <= 3)
    rp.rot_fp32 ? go(k_rate_epilogue<1, 3, true>) : go(k_rate_epilogue<1, 3, false>);
  else if (M.nb <= 4 && M.nbr <= 6)
    rp.rot_fp32 ? go(k_rate_epilogue<4, 6, true>) : go(k_rate_epilogue<4, 6, false>);
  else if (M.nbr <= 6)
    rp.rot_fp32 ? go(k_rate_epilogue<kMaxBands, 6, true>) : go(k_rate_epilogue<kMaxBands, 6, false>);
  else
    rp.rot_fp32 ? go(k_rate_epilogue<kMaxBands, kMaxBranches, true>)
                : go(k_rate_epilogue<kMaxBands, kMaxBranches, false>);
  return cudaGetLastError();
}

cudaError_t launch_selftest_exp_ff(const double *y, double *out, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  EPHB_LAUNCH(k_selftest_exp_ff, unsigned((n + 255) / 256), 256, 0, st, y, out, n);
  return cudaGetLastError();
}

size_t stage_a_T_elems(const ModelDev &M) { return size_t(M.nRgp) * M.nb * M.nb * M.nbr; }
size_t stage_a_A_elems(const ModelDev &M) { return size_t(M.nRgp) * M.nb * M.nb * M.nbr; }

cudaError_t launch_rate_count(const ModelDev &M, const MeshDev &D, RateParams rp, int *cntE, int *cntPh,
                              unsigned long long *n_tuples, cudaStream_t st) {
  // counters: [0] tuples, [2] stage-B flops, [3] active states in irreducible rows
  cudaError_t e = cudaMemsetAsync(n_tuples, 0, 5 * sizeof(unsigned long long), st);
  if (e != cudaSuccess || D.n_pairs == 0) return e;
  EPHB_LAUNCH(k_rate_count, unsigned((D.n_pairs + 127) / 128), 128, 0, st, M, D, rp, cntE, cntPh, n_tuples);
  return cudaGetLastError();
}

cudaError_t launch_row_ptrs(const MeshDev &D, int nb, int nbr, const int64_t *escan, const int64_t *phscan,
                            int64_t e_total, int64_t ph_total, int64_t *row_ptr, int64_t *ph_row_ptr,
                            cudaStream_t st) {
  int64_t n = (D.n_ibzw * nb > D.nq * nbr ? D.n_ibzw * nb : D.nq * nbr) + 1;
  EPHB_LAUNCH(k_row_ptrs, unsigned((n + 255) / 256), 256, 0, st, D, nb, nbr, escan, phscan, e_total, ph_total, row_ptr,
                                                        ph_row_ptr);
  return cudaGetLastError();
}

cudaError_t launch_stage_a(const ModelDev &M, const MeshDev &D, int64_t i0, int64_t nkc, double2 *T, double2 *A,
                           cudaStream_t st) {
  const int64_t ncol = int64_t(M.nRgp) * M.nb * M.nb * M.nbr;
  size_t smem = size_t(kAKT) * M.nRge * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_stage_a1, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  dim3 g1(unsigned((ncol + 255) / 256), unsigned((nkc + kAKT - 1) / kAKT));
  EPHB_LAUNCH(k_stage_a1, g1, 256, smem, st, M, D, i0, nkc, T);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t n2 = nkc * ncol;
  EPHB_LAUNCH(k_stage_a2<false>, unsigned((n2 + 255) / 256), 256, 0, st, M, D, i0, nkc, T, A);
  return cudaGetLastError();
}

cudaError_t launch_stage_a2(const ModelDev &M, const MeshDev &D, int64_t i0, int64_t nkc, const double2 *T, double2 *A,
                            bool t_ff, cudaStream_t st) {
  const int64_t n2 = nkc * int64_t(M.nRgp) * M.nb * M.nb * M.nbr;
  if (n2 == 0) return cudaSuccess;
  if (t_ff)
    EPHB_LAUNCH(k_stage_a2<true>, unsigned((n2 + 255) / 256), 256, 0, st, M, D, i0, nkc, T, A);
  else
    EPHB_LAUNCH(k_stage_a2<false>, unsigned((n2 + 255) / 256), 256, 0, st, M, D, i0, nkc, T, A);
  return cudaGetLastError();
}

cudaError_t launch_stage_b_rates(const ModelDev &M, const MeshDev &D, RateParams rp, int64_t i0, int64_t nkc,
                                 const double2 *A, const int64_t *escan, const int64_t *phscan, uint32_t *e_kpns,
                                 double2 *e_X, int *ph_st, uint32_t *ph_kpn, double *ph_Y, cudaStream_t st) {
  StageBSmem L = stage_b_layout(M.nb, M.nbr);
  cudaError_t e = cudaFuncSetAttribute(k_stage_b_rates, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.total));
  if (e != cudaSuccess) return e;
  EPHB_LAUNCH(k_stage_b_rates, unsigned(nkc), kBT, L.total, st, M, D, rp, i0, A, escan, phscan, e_kpns, e_X, ph_st, ph_kpn,
                                                       ph_Y);
  return cudaGetLastError();
}

}  // namespace ephb
