// Coupled electron-phonon BTE sweeps (section "Coupled and decoupled BTEs" of arXiv
// 2109.08547): RTA rates and terms, the electron gather sweep (self + drag terms), the
// phonon drag scatter over the (q,s) rows with the symmetry fold, the transport-coefficient
// reductions and the Kelvin-Onsager correction.  Every reduction runs in a fixed order,
// so repeated runs give bit-identical results.
#include "internal.h"

namespace ephb {

namespace {

__device__ inline double fermi_b(double e, double mu, double kT) { return 1.0 / (exp((e - mu) / kT) + 1.0); }
__device__ inline double bose_b(double w, double kT) { return w > 0.0 ? 1.0 / expm1(w / kT) : 0.0; }

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline void rot3(const double *C, const double *x, double *y) {
  y[0] = C[0] * x[0] + C[1] * x[1] + C[2] * x[2];
  y[1] = C[3] * x[0] + C[4] * x[1] + C[5] * x[2];
  y[2] = C[6] * x[0] + C[7] * x[1] + C[8] * x[2];
}

// image of q (flat) under operation s (integer rotation on reciprocal crystal coords)
__device__ inline int q_image(const Mesh &qm, const int *rot, int q) {
  int b0, b1, b2;
  qm.unflat(q, b0, b1, b2);
  return qm.flat(pmod(rot[0] * b0 + rot[1] * b1 + rot[2] * b2, qm.n[0]),
                 pmod(rot[3] * b0 + rot[4] * b1 + rot[5] * b2, qm.n[1]),
                 pmod(rot[6] * b0 + rot[7] * b1 + rot[8] * b2, qm.n[2]));
}

__global__ void k_state_setup(ModelDev M, MeshDev D, double T, double mu, double lo, double hi, double *st_eps,
                              double *st_vel, double *st_ff, double *st_wt, uint32_t *kcrd, int2 *kinfo) {
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int nb = M.nb;
  if (t < D.n_ibzw * nb) {
    int64_t i = t / nb;
    int m = int(t % nb);
    int k = D.ibzw_list[i];
    double e = D.eps[size_t(k) * nb + m];
    bool act = ((D.amask[k] >> m) & 1u) && e >= lo && e <= hi;
    double f = fermi_b(e, mu, kKbEVK * T);
    st_eps[t] = e;
    for (int a = 0; a < 3; ++a) st_vel[t * 3 + a] = D.vel[(size_t(k) * nb + m) * 3 + a];
    st_ff[t] = act ? f * (1.0 - f) : 0.0;
    st_wt[t] = act ? 1.0 / double(D.stab[k]) : 0.0;
  }
  if (t < D.nk) {
    int a0, a1, a2;
    D.km.unflat(int(t), a0, a1, a2);
    kcrd[t] = uint32_t(a0) | (uint32_t(a1) << 10) | (uint32_t(a2) << 20);
    int r = D.rep[t];
    int iw = D.ibzw_of[r];
    kinfo[t] = make_int2(iw >= 0 ? iw * nb : -1, D.op[t]);
  }
}

// W_e = sum_row (X+ + X-) / (f(1-f)) (+ W_add, other channels by Matthiessen's rule);
// I0 = (eps-mu)/T v/W; J0 = v/W   (Eqs. W^RTA_mk, I0/J0)
__global__ void k_rta_electron(BteDev B, double *W_e, double *inv_ffW, double *I0, double *J0,
                               unsigned long long *n_zero, const double *__restrict__ W_add) {
  int64_t st = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (st >= B.nst) return;
  double s = 0.0;
  for (int64_t e = B.row_ptr[st] + lane; e < B.row_ptr[st + 1]; e += 32) {
    double2 x = B.e_X[e];
    s += x.x + x.y;
  }
  s = warp_sum(s);
  if (lane == 0) {
    double ff = B.st_ff[st];
    double W = 0.0, inv = 0.0;
    const double add = ff > 0.0 && W_add ? W_add[st] : 0.0;
    if (ff > 0.0 && (s > 0.0 || add > 0.0)) {
      W = s / ff + add;
      inv = 1.0 / (ff * W);
    } else if (ff > 0.0) {
      atomicAdd(n_zero, 1ull);
    }
    W_e[st] = W;
    inv_ffW[st] = inv;
    double c = W > 0.0 ? (B.st_eps[st] - B.mu) / B.T : 0.0;
    for (int a = 0; a < 3; ++a) {
      double v = W > 0.0 ? B.st_vel[st * 3 + a] / W : 0.0;
      I0[st * 3 + a] = c * v;
      J0[st * 3 + a] = v;
    }
  }
}

// Bt(q,s) = sum over the phonon row of Y/|stab|
__global__ void k_ph_rowsum(BteDev B, double *Bt) {
  int64_t row = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= B.nq * B.nbr) return;
  double s = 0.0;
  for (int64_t e = B.ph_row_ptr[row] + lane; e < B.ph_row_ptr[row + 1]; e += 32) s += B.ph_Y[e];
  s = warp_sum(s);
  if (lane == 0) Bt[row] = s;
}

// W_ph = d_s sum_S Bt(S^-1 q) / (n(1+n)) + W_bg; F0 = (hbar w/T) v / W   (Eqs. W^RTA_sq, F0/G0)
__global__ void k_rta_phonon(ModelDev M, MeshDev D, BteDev B, const double *Bt, double *W_ph, double *inv_nnW,
                             double *F0, const double *__restrict__ W_add) {
  __shared__ int rot[kMaxSym * 9];
  __shared__ int inv[kMaxSym];
  for (int t = threadIdx.x; t < M.nsym * 9; t += blockDim.x) rot[t] = M.sym_rot[t];
  for (int t = threadIdx.x; t < M.nsym; t += blockDim.x) inv[t] = M.sym_inv[t];
  __syncthreads();
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int nbr = M.nbr;
  if (t >= D.nq * nbr) return;
  int q = int(t / nbr), s = int(t % nbr);
  double w = D.w[t];
  double kT = kKbEVK * B.T;
  double W = 0.0, invw = 0.0;
  if (w > D.omega_min) {
    double sum = 0.0;
    for (int o = 0; o < M.nsym; ++o) sum += Bt[size_t(q_image(D.qm, rot + 9 * inv[o], q)) * nbr + s];
    double n = bose_b(w, kT);
    double nn1 = n * (1.0 + n);
    double wr = w / M.bg_w;
    W = M.spin_deg * sum / nn1 + M.bg_coeff * wr * wr * (B.T / M.bg_T) + (W_add ? W_add[t] : 0.0);
    invw = 1.0 / (nn1 * W);
  }
  W_ph[t] = W;
  inv_nnW[t] = invw;
  for (int a = 0; a < 3; ++a) F0[t * 3 + a] = W > 0.0 ? (w / B.T) * D.vph[t * 3 + a] / W : 0.0;
}

// ---------------------------------------------------------------- electron sweeps
// Entry streams (the rate entries of the electron rows, or the partner runs below) are
// cut into segments of at most kSeg items that never cross a row.  One warp reduces one
// segment into 6 partial sums; a finalisation kernel adds a row's segment partials in
// segment order, so results do not depend on scheduling.
//
// Self term (Eq. dI^S): sum_{n k' s} (X+ + X-) S_k' I_<k'>n.  The entries of one row that
// share the partner state (k', n) differ only in the branch s, so their weights are merged
// once per rate build into "runs" {partner state, rotation, w = sum_s (X+ + X-)}; every
// inner sweep then streams runs (12 B) instead of entries (20 B) and does a third of the
// FP64 work.
// Drag term (Eq. dI^D): sum (-F_qs X+ + F_-qs X-).  It depends on F, G only, which are
// fixed during the electron iteration, so it is evaluated once per phonon iteration.
constexpr int kSeg = 1024;
constexpr int kUnroll = 4;
constexpr uint32_t kRunColMask = (1u << 26) - 1u;
constexpr uint32_t kRunNone = kRunColMask;      // partner without a representative row

__global__ void k_seg_count(int64_t nrow, const int64_t *row_ptr, int *nseg) {
  int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (r >= nrow) return;
  int64_t len = row_ptr[r + 1] - row_ptr[r];
  nseg[r] = int((len + kSeg - 1) / kSeg);
}

__global__ void k_seg_fill(int64_t nrow, const int64_t *row_ptr, const int64_t *seg_ptr, int *seg_row,
                           int64_t *seg_begin) {
  int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (r >= nrow) return;
  int64_t g = seg_ptr[r];
  for (int64_t b = row_ptr[r]; b < row_ptr[r + 1]; b += kSeg, ++g) {
    seg_row[g] = int(r);
    seg_begin[g] = b;
  }
}

// run starts: an entry whose (k', n) differs from the previous entry's, or a row's first entry
__global__ void k_run_flags(int64_t n, const uint32_t *kpns, int *flag) {
  int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= n) return;
  const uint32_t key = kpns[e] & ((1u << (kKpBits + 4)) - 1u);   // k' and n, without s
  flag[e] = (e == 0 || (kpns[e - 1] & ((1u << (kKpBits + 4)) - 1u)) != key) ? 1 : 0;
}

__global__ void k_run_rowstarts(int64_t nrow, const int64_t *row_ptr, int *flag) {
  int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (r >= nrow) return;
  if (row_ptr[r + 1] > row_ptr[r]) flag[row_ptr[r]] = 1;
}

__global__ void k_run_fill(int64_t n, const uint32_t *kpns, const double2 *X, const int *flag,
                           const int64_t *runidx, const int2 *kinfo, uint32_t *run_col, double *run_w) {
  int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= n || !flag[e]) return;
  double w = 0.0;
  for (int64_t f = e; f < n && (f == e || !flag[f]); ++f) w += X[f].x + X[f].y;
  const int2 inf = kinfo[unpack_kp(kpns[e])];
  const uint32_t col = inf.x >= 0 ? uint32_t(inf.x + unpack_n(kpns[e])) : kRunNone;
  run_col[runidx[e]] = col | (uint32_t(inf.y) << 26);
  run_w[runidx[e]] = w;
}

__global__ void k_run_ptr(int64_t nrow, const int64_t *row_ptr, const int64_t *runidx, int64_t n_entries,
                          int64_t nruns, int64_t *run_ptr) {
  int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (r > nrow) return;
  const int64_t e = row_ptr[r];
  run_ptr[r] = e < n_entries ? runidx[e] : nruns;
}

// self term over the runs of one segment
template <bool SYM>
__global__ void __launch_bounds__(256) k_self_sweep_seg(ModelDev M, SweepSegs S, const uint32_t *__restrict__ run_col,
                                                        const double *__restrict__ run_w,
                                                        const double *__restrict__ I, const double *__restrict__ J,
                                                        const double *__restrict__ I2, const double *__restrict__ J2,
                                                        const double2 *__restrict__ IJ,
                                                        const double2 *__restrict__ IJ2,
                                                        const int *__restrict__ ctl, double *__restrict__ part) {
  // device-driven loop: skip once stopped; odd sweeps read the second buffer pair
  if (ctl) {
    if (ctl[0]) return;
    if (ctl[1] & 1) {
      I = I2;
      J = J2;
      IJ = IJ2;
    }
  }
  __shared__ double C[kMaxSym * 9];
  if (SYM) {
    for (int t = threadIdx.x; t < M.nsym * 9; t += blockDim.x) C[t] = M.sym_cart[t];
    __syncthreads();
  }
  const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= S.nseg) return;
  const int row = S.seg_row[g];
  const int64_t b = S.seg_begin[g];
  const int64_t rend = S.row_ptr[row + 1];
  const int64_t e_end = b + kSeg < rend ? b + kSeg : rend;
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t e0 = b + lane; e0 < e_end; e0 += 32 * kUnroll) {
    uint32_t pc[kUnroll];
    double w[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t e = e0 + 32 * u;
      pc[u] = e < e_end ? __ldcs(run_col + e) : kRunNone;
      w[u] = e < e_end ? __ldcs(run_w + e) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t col = pc[u] & kRunColMask;
      if (col == kRunNone) continue;
      double vi[3], vj[3];
      if (IJ) {   // packed (I, J) of the partner: three 16-byte loads
        const double2 *p = IJ + int64_t(col) * 3;
        const double2 a = p[0], b = p[1], c = p[2];
        vi[0] = a.x; vi[1] = a.y; vi[2] = b.x;
        vj[0] = b.y; vj[1] = c.x; vj[2] = c.y;
      } else {
        vi[0] = I[int64_t(col) * 3]; vi[1] = I[int64_t(col) * 3 + 1]; vi[2] = I[int64_t(col) * 3 + 2];
        vj[0] = J[int64_t(col) * 3]; vj[1] = J[int64_t(col) * 3 + 1]; vj[2] = J[int64_t(col) * 3 + 2];
      }
      if (SYM) {
        double r[3];
        const double *Cs = C + 9 * (pc[u] >> 26);
        rot3(Cs, vi, r);
        vi[0] = r[0]; vi[1] = r[1]; vi[2] = r[2];
        rot3(Cs, vj, r);
        vj[0] = r[0]; vj[1] = r[1]; vj[2] = r[2];
      }
      for (int c = 0; c < 3; ++c) {
        a[c] += w[u] * vi[c];
        a[3 + c] += w[u] * vj[c];
      }
    }
  }
  for (int c = 0; c < 6; ++c) a[c] = warp_sum(a[c]);
  if (lane == 0)
    for (int c = 0; c < 6; ++c) part[g * 6 + c] = a[c];
}

// drag term over the rate entries of one segment
__global__ void __launch_bounds__(256) k_drag_sweep_seg(MeshDev D, BteDev B, SweepSegs S,
                                                        const double *__restrict__ F, const double *__restrict__ G,
                                                        double *__restrict__ part) {
  const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= S.nseg) return;
  const int st = S.seg_row[g];
  const int64_t b = S.seg_begin[g];
  const int64_t rend = S.row_ptr[st + 1];
  const int64_t e_end = b + kSeg < rend ? b + kSeg : rend;
  const int nbr = B.nbr;
  const uint32_t kc = B.kcrd[D.ibzw_list[st / B.nb]];
  const int k0 = kc & 1023u, k1 = (kc >> 10) & 1023u, k2 = kc >> 20;
  const bool unit_ratio = D.ratio[0] == 1 && D.ratio[1] == 1 && D.ratio[2] == 1;
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t e = b + lane; e < e_end; e += 32) {
    const uint32_t pk = __ldcs(B.e_kpns + e);
    const double2 X = __ldcs(B.e_X + e);
    const int kp = unpack_kp(pk), s = unpack_s(pk);
    const uint32_t pc = B.kcrd[kp];
    // q = (k' - k) / ratio per dimension (k' - k is a multiple of the ratio); -q on the q mesh
    int d0 = int(pc & 1023u) - k0, d1 = int((pc >> 10) & 1023u) - k1, d2 = int(pc >> 20) - k2;
    d0 += d0 < 0 ? D.km.n[0] : 0;
    d1 += d1 < 0 ? D.km.n[1] : 0;
    d2 += d2 < 0 ? D.km.n[2] : 0;
    if (!unit_ratio) {
      d0 /= D.ratio[0];
      d1 /= D.ratio[1];
      d2 /= D.ratio[2];
    }
    const int64_t q = D.qm.flat(d0, d1, d2);
    const int64_t mq = D.qm.flat(d0 ? D.qm.n[0] - d0 : 0, d1 ? D.qm.n[1] - d1 : 0, d2 ? D.qm.n[2] - d2 : 0);
    const double *Fq = F + (q * nbr + s) * 3, *Fm = F + (mq * nbr + s) * 3;
    const double *Gq = G + (q * nbr + s) * 3, *Gm = G + (mq * nbr + s) * 3;
    for (int c = 0; c < 3; ++c) {
      a[c] += -Fq[c] * X.x + Fm[c] * X.y;
      a[3 + c] += -Gq[c] * X.x + Gm[c] * X.y;
    }
  }
  for (int c = 0; c < 6; ++c) a[c] = warp_sum(a[c]);
  if (lane == 0)
    for (int c = 0; c < 6; ++c) part[g * 6 + c] = a[c];
}

// Float-float form of the drag term (mixed iteration once the outer residual is small): the
// same sums from float-float copies of the rates (Xff: X+ hi, lo, X- hi, lo) and of F, G
// (FGff: [mode][F0 F1 F2 G0 G1 G2] pairs), ~2^-47 of the summed magnitudes, on the FP32 pipe.
__global__ void __launch_bounds__(256) k_drag_sweep_segff(MeshDev D, BteDev B, SweepSegs S,
                                                          const float4 *__restrict__ Xff,
                                                          const float2 *__restrict__ FGff, double *__restrict__ part) {
  const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= S.nseg) return;
  const int st = S.seg_row[g];
  const int64_t b = S.seg_begin[g];
  const int64_t rend = S.row_ptr[st + 1];
  const int64_t e_end = b + kSeg < rend ? b + kSeg : rend;
  const int nbr = B.nbr;
  const uint32_t kc = B.kcrd[D.ibzw_list[st / B.nb]];
  const int k0 = kc & 1023u, k1 = (kc >> 10) & 1023u, k2 = kc >> 20;
  const bool unit_ratio = D.ratio[0] == 1 && D.ratio[1] == 1 && D.ratio[2] == 1;
  FFAcc a[6];
  for (int64_t e = b + lane; e < e_end; e += 32) {
    const uint32_t pk = __ldcs(B.e_kpns + e);
    const float4 X = __ldcs(Xff + e);
    const int kp = unpack_kp(pk), s = unpack_s(pk);
    const uint32_t pc = B.kcrd[kp];
    int d0 = int(pc & 1023u) - k0, d1 = int((pc >> 10) & 1023u) - k1, d2 = int(pc >> 20) - k2;
    d0 += d0 < 0 ? D.km.n[0] : 0;
    d1 += d1 < 0 ? D.km.n[1] : 0;
    d2 += d2 < 0 ? D.km.n[2] : 0;
    if (!unit_ratio) {
      d0 /= D.ratio[0];
      d1 /= D.ratio[1];
      d2 /= D.ratio[2];
    }
    const int64_t q = D.qm.flat(d0, d1, d2);
    const int64_t mq = D.qm.flat(d0 ? D.qm.n[0] - d0 : 0, d1 ? D.qm.n[1] - d1 : 0, d2 ? D.qm.n[2] - d2 : 0);
    const float2 *pq = FGff + (q * nbr + s) * 6, *pm = FGff + (mq * nbr + s) * 6;
    const float2 xp = make_float2(X.x, X.y), xm = make_float2(X.z, X.w);
    for (int c = 0; c < 6; ++c) {
      ff_acc_mul(a[c], ff_neg(pq[c]), xp);
      ff_acc_mul(a[c], pm[c], xm);
    }
  }
  for (int c = 0; c < 6; ++c) {
    const double v = warp_sum(ff_to_double(a[c]));
    if (lane == 0) part[g * 6 + c] = v;
  }
}

// FP32 form of the drag term (mixed iteration while the outer residual is large): the same
// sums from FP32 copies of the rates (X32) and of F, G (FG32: [mode][F0 F1 F2 G0 G1 G2]).
__global__ void __launch_bounds__(256) k_drag_sweep_seg32(MeshDev D, BteDev B, SweepSegs S,
                                                          const float2 *__restrict__ X32,
                                                          const float *__restrict__ FG32, double *__restrict__ part) {
  const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= S.nseg) return;
  const int st = S.seg_row[g];
  const int64_t b = S.seg_begin[g];
  const int64_t rend = S.row_ptr[st + 1];
  const int64_t e_end = b + kSeg < rend ? b + kSeg : rend;
  const int nbr = B.nbr;
  const uint32_t kc = B.kcrd[D.ibzw_list[st / B.nb]];
  const int k0 = kc & 1023u, k1 = (kc >> 10) & 1023u, k2 = kc >> 20;
  const bool unit_ratio = D.ratio[0] == 1 && D.ratio[1] == 1 && D.ratio[2] == 1;
  float a[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t e = b + lane; e < e_end; e += 32) {
    const uint32_t pk = __ldcs(B.e_kpns + e);
    const float2 X = __ldcs(X32 + e);
    const int kp = unpack_kp(pk), s = unpack_s(pk);
    const uint32_t pc = B.kcrd[kp];
    int d0 = int(pc & 1023u) - k0, d1 = int((pc >> 10) & 1023u) - k1, d2 = int(pc >> 20) - k2;
    d0 += d0 < 0 ? D.km.n[0] : 0;
    d1 += d1 < 0 ? D.km.n[1] : 0;
    d2 += d2 < 0 ? D.km.n[2] : 0;
    if (!unit_ratio) {
      d0 /= D.ratio[0];
      d1 /= D.ratio[1];
      d2 /= D.ratio[2];
    }
    const int64_t q = D.qm.flat(d0, d1, d2);
    const int64_t mq = D.qm.flat(d0 ? D.qm.n[0] - d0 : 0, d1 ? D.qm.n[1] - d1 : 0, d2 ? D.qm.n[2] - d2 : 0);
    const float *pq = FG32 + (q * nbr + s) * 6, *pm = FG32 + (mq * nbr + s) * 6;
    for (int c = 0; c < 6; ++c) a[c] = fmaf(pm[c], X.y, fmaf(-pq[c], X.x, a[c]));
  }
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_down_sync(0xffffffffu, a[c], o);
  if (lane == 0)
    for (int c = 0; c < 6; ++c) part[g * 6 + c] = double(a[c]);
}

// Dterm[st] = sum of the row's drag segment partials (in segment order)
__global__ void k_drag_finalize(int64_t nst, SweepSegs S, const double *part, double *Dterm) {
  int64_t st = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (st >= nst) return;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t g = S.seg_ptr[st]; g < S.seg_ptr[st + 1]; ++g)
    for (int c = 0; c < 6; ++c) s[c] += part[g * 6 + c];
  for (int c = 0; c < 6; ++c) Dterm[st * 6 + c] = s[c];
}

// The phonon drag scatter Btv(q,s) = sum Y/|stab| (S_k' I_<k'>n - I_km), fields I and J, over
// the entries of each phonon row.  Rows are cut into segments of at most kSeg entries, one warp
// per segment (lanes strided over its entries, a fixed-order warp sum into part[seg][6]); the
// rows of a fine q mesh are very uneven (those near q = 0 and at the inter-valley q gather
// every irreducible window k, most hold none), which one thread per row turned into a few long
// serial chains of gathers.  k_ph_seg_finalize adds each row's segments in order.
// Float-float form (mixed iteration once the outer residual is small), from float-float
// copies of Y and of the responses (IJff: [state][I0 I1 I2 J0 J1 J2]).
template <bool SYM>
__global__ void __launch_bounds__(256) k_ph_sweepff(ModelDev M, BteDev B, SweepSegs S, const int2 *__restrict__ kinfo,
                                                    const float2 *__restrict__ Yff,
                                                    const float2 *__restrict__ IJff, double *part) {
  __shared__ float2 C[kMaxSym * 9];
  if (SYM) {
    for (int t = threadIdx.x; t < M.nsym * 9; t += blockDim.x) C[t] = ff_from_double(M.sym_cart[t]);
    __syncthreads();
  }
  const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= S.nseg) return;
  const int64_t b = S.seg_begin[g], rend = S.row_ptr[S.seg_row[g] + 1];
  const int64_t e_end = b + kSeg < rend ? b + kSeg : rend;
  FFAcc a[6];
  for (int64_t e = b + lane; e < e_end; e += 32) {
    const int st = B.ph_st[e];
    const uint32_t pk = B.ph_kpn[e];
    const float2 y = Yff[e];
    const int2 inf = kinfo[unpack_kp(pk)];
    const float2 *own = IJff + int64_t(st) * 6;
    float2 r[6];
    for (int c = 0; c < 6; ++c) r[c] = make_float2(0.f, 0.f);
    if (inf.x >= 0) {   // inf.x < 0: see the electron sweep
      const float2 *src = IJff + (int64_t(inf.x) + unpack_n(pk)) * 6;
      if (SYM) {
        const float2 *Cs = C + 9 * (inf.y > 0 ? inf.y : 0);
        for (int f = 0; f < 2; ++f)
          for (int x = 0; x < 3; ++x) {
            FFAcc t;
            for (int z = 0; z < 3; ++z) ff_acc_mul(t, Cs[3 * x + z], src[3 * f + z]);
            r[3 * f + x] = ff_norm(t);
          }
      } else {
        for (int c = 0; c < 6; ++c) r[c] = src[c];
      }
    }
    for (int c = 0; c < 6; ++c) ff_acc_mul(a[c], y, ff_sub(r[c], own[c]));
  }
  for (int c = 0; c < 6; ++c) {
    const double v = warp_sum(ff_to_double(a[c]));
    if (lane == 0) part[g * 6 + c] = v;
  }
}

// Btv[row] = the sum of the row's segment partials, in order (zero for rows without entries)
__global__ void k_ph_seg_finalize(int64_t nrow, SweepSegs S, const double *__restrict__ part, double *Btv) {
  const int64_t row = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (row >= nrow) return;
  double sum[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t g = S.seg_ptr[row]; g < S.seg_ptr[row + 1]; ++g)
    for (int c = 0; c < 6; ++c) sum[c] += part[g * 6 + c];
  for (int c = 0; c < 6; ++c) Btv[row * 6 + c] = sum[c];
}

// float-float copies: out[i] = ff(a[i]) (n values); pack: out[i][0..2] = ff(A[i][..]),
// out[i][3..5] = ff(B[i][..])
__global__ void k_copy_ff(int64_t n, const double *a, float2 *out) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = ff_from_double(a[i]);
}

__global__ void k_pack6_ff(int64_t n, const double *A, const double *Bv, float2 *out) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  for (int c = 0; c < 3; ++c) {
    out[i * 6 + c] = ff_from_double(A[i * 3 + c]);
    out[i * 6 + 3 + c] = ff_from_double(Bv[i * 3 + c]);
  }
}

// FP32 form of the phonon drag scatter (mixed iteration while the outer residual is large),
// from FP32 copies of Y and of the responses (IJ32: [state][I0 I1 I2 J0 J1 J2]).
// FP32 form of the phonon drag scatter (early outer iterations of the mixed iteration), the
// segments as in k_ph_sweepff; lane sums in FP32, the warp sum in FP32, partials stored FP64.
template <bool SYM>
__global__ void __launch_bounds__(256) k_ph_sweep32(ModelDev M, BteDev B, SweepSegs S, const int2 *__restrict__ kinfo,
                                                    const float *__restrict__ Y32, const float *__restrict__ IJ32,
                                                    double *part) {
  __shared__ float C[kMaxSym * 9];
  if (SYM) {
    for (int t = threadIdx.x; t < M.nsym * 9; t += blockDim.x) C[t] = float(M.sym_cart[t]);
    __syncthreads();
  }
  const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= S.nseg) return;
  const int64_t b = S.seg_begin[g], rend = S.row_ptr[S.seg_row[g] + 1];
  const int64_t e_end = b + kSeg < rend ? b + kSeg : rend;
  float a[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t e = b + lane; e < e_end; e += 32) {
    const int st = B.ph_st[e];
    const uint32_t pk = B.ph_kpn[e];
    const float y = Y32[e];
    const int2 inf = kinfo[unpack_kp(pk)];
    const float *own = IJ32 + int64_t(st) * 6;
    float r[6] = {0, 0, 0, 0, 0, 0};
    if (inf.x >= 0) {   // inf.x < 0: see the electron sweep
      const float *src = IJ32 + (int64_t(inf.x) + unpack_n(pk)) * 6;
      if (SYM) {
        const float *Cs = C + 9 * (inf.y > 0 ? inf.y : 0);
        for (int f = 0; f < 2; ++f)
          for (int x = 0; x < 3; ++x)
            r[3 * f + x] = Cs[3 * x] * src[3 * f] + Cs[3 * x + 1] * src[3 * f + 1] + Cs[3 * x + 2] * src[3 * f + 2];
      } else {
        for (int c = 0; c < 6; ++c) r[c] = src[c];
      }
    }
    for (int c = 0; c < 6; ++c) a[c] = fmaf(y, r[c] - own[c], a[c]);
  }
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_down_sync(0xffffffffu, a[c], o);
  if (lane == 0)
    for (int c = 0; c < 6; ++c) part[g * 6 + c] = double(a[c]);
}

// FP32 copies: out[i][0..2] = A[i][0..2], out[i][3..5] = B[i][0..2]; and plain element copies
__global__ void k_pack6_f32(int64_t n, const double *A, const double *Bv, float *out) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  for (int c = 0; c < 3; ++c) {
    out[i * 6 + c] = float(A[i * 3 + c]);
    out[i * 6 + 3 + c] = float(Bv[i * 3 + c]);
  }
}

__global__ void k_copy_f32(int64_t n, const double *a, float *b) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) b[i] = float(a[i]);
}

// FP64 form of the phonon drag scatter, the segments as in k_ph_sweepff.
template <bool SYM>
__global__ void __launch_bounds__(256) k_ph_sweep(ModelDev M, BteDev B, SweepSegs S, const int2 *__restrict__ kinfo,
                                                  const double *__restrict__ I, const double *__restrict__ J,
                                                  double *part) {
  __shared__ double C[kMaxSym * 9];
  if (SYM) {
    for (int t = threadIdx.x; t < M.nsym * 9; t += blockDim.x) C[t] = M.sym_cart[t];
    __syncthreads();
  }
  const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= S.nseg) return;
  const int64_t b = S.seg_begin[g], rend = S.row_ptr[S.seg_row[g] + 1];
  const int64_t e_end = b + kSeg < rend ? b + kSeg : rend;
  double aI[3] = {0, 0, 0}, aJ[3] = {0, 0, 0};
  for (int64_t e = b + lane; e < e_end; e += 32) {
    int st = B.ph_st[e];
    uint32_t pk = B.ph_kpn[e];
    double y = B.ph_Y[e];
    int kp = unpack_kp(pk), n = unpack_n(pk);
    int2 inf = kinfo[kp];
    double r[3] = {0.0, 0.0, 0.0};
    const int64_t st2 = inf.x + n;
    // inf.x < 0: see the electron sweep.  Without symmetry every k is its own representative.
    if (SYM) {
      const double *Cs = C + 9 * (inf.y > 0 ? inf.y : 0);
      if (inf.x >= 0) rot3(Cs, I + st2 * 3, r);
    } else if (inf.x >= 0) {
      for (int a = 0; a < 3; ++a) r[a] = I[st2 * 3 + a];
    }
    for (int a = 0; a < 3; ++a) aI[a] += y * (r[a] - I[int64_t(st) * 3 + a]);
    if (SYM) {
      const double *Cs = C + 9 * (inf.y > 0 ? inf.y : 0);
      if (inf.x >= 0) rot3(Cs, J + st2 * 3, r);
    } else if (inf.x >= 0) {
      for (int a = 0; a < 3; ++a) r[a] = J[st2 * 3 + a];
    }
    for (int a = 0; a < 3; ++a) aJ[a] += y * (r[a] - J[int64_t(st) * 3 + a]);
  }
  for (int a = 0; a < 3; ++a) {
    aI[a] = warp_sum(aI[a]);
    aJ[a] = warp_sum(aJ[a]);
  }
  if (lane == 0)
    for (int a = 0; a < 3; ++a) {
      part[g * 6 + a] = aI[a];
      part[g * 6 + 3 + a] = aJ[a];
    }
}

// The full-zone k sum of the phonon drag term from the irreducible rows (reading [A13]):
// A(q) = sum_S C_S Btv(S^-1 q).  It is covariant, A(S q) = C_S A(q) (rearranging the group sum),
// so the 48-term sum runs on the representatives of the q wedge only and every other q takes
// its representative's A rotated by the operation that maps the representative onto it.
// Eight lanes per (representative, branch): lane l sums the operations l, l + 8, ...; the eight
// partial sums are added by shuffles (a fixed order: the result is reproducible).
__global__ void k_ph_fold_rep(ModelDev M, MeshDev D, const double *Btv, double *Afold) {
  __shared__ int rot[kMaxSym * 9];
  __shared__ int inv[kMaxSym];
  __shared__ double C[kMaxSym * 9];
  for (int t = threadIdx.x; t < M.nsym * 9; t += blockDim.x) {
    rot[t] = M.sym_rot[t];
    C[t] = M.sym_cart[t];
  }
  for (int t = threadIdx.x; t < M.nsym; t += blockDim.x) inv[t] = M.sym_inv[t];
  __syncthreads();
  const int64_t t = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 3;
  const int l = threadIdx.x & 7;
  const int nbr = M.nbr;
  const bool live = t < D.n_qrep * nbr;
  double a[6] = {0, 0, 0, 0, 0, 0};
  if (live) {
    const int j = int(t / nbr), s = int(t % nbr);
    const int q = D.qlist[j];
    for (int o = l; o < M.nsym; o += 8) {
      const int64_t src = int64_t(q_image(D.qm, rot + 9 * inv[o], q)) * nbr + s;
      double r[3];
      rot3(C + 9 * o, Btv + src * 6, r);
      for (int x = 0; x < 3; ++x) a[x] += r[x];
      rot3(C + 9 * o, Btv + src * 6 + 3, r);
      for (int x = 0; x < 3; ++x) a[3 + x] += r[x];
    }
  }
  for (int off = 4; off > 0; off >>= 1)
    for (int c = 0; c < 6; ++c) a[c] += __shfl_xor_sync(0xffffffffu, a[c], off);
  if (live && l == 0)
    for (int c = 0; c < 6; ++c) Afold[t * 6 + c] = a[c];
}

// F = F0 + d_s/(n(1+n)W) A_I(q); G = d_s/(n(1+n)W) A_J(q)   (Eq. dF^D), A(q) = C_S A(<q>)
__global__ void k_ph_update(ModelDev M, MeshDev D, const double *Afold, const double *F0, const double *inv_nnW,
                            double *F, double *G) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int nbr = M.nbr;
  if (t >= D.nq * nbr) return;
  const int q = int(t / nbr), s = int(t % nbr);
  const double *A = Afold + (int64_t(D.qrep_of[D.qrep[q]]) * nbr + s) * 6;
  const double *Cs = M.sym_cart + 9 * D.qop[q];
  double aI[3], aJ[3];
  rot3(Cs, A, aI);
  rot3(Cs, A + 3, aJ);
  const double c = M.spin_deg * inv_nnW[t];
  for (int x = 0; x < 3; ++x) {
    F[t * 3 + x] = F0[t * 3 + x] + c * aI[x];
    G[t * 3 + x] = c * aJ[x];
  }
}

// ---------------------------------------------------------------- coefficient reductions
constexpr int kNPart = 48;      // fixed number of partial-sum blocks (few: the assembly adds them)
// Threads of the partial-sum kernels (three warps: the coefficient assembly fused into the
// last block needs at least 72).  An FP64 warp instruction holds the SM's FP64 pipe ~16 cycles
// whatever its active lanes, so these kernels keep few warps per SM and few FP64 instructions
// per warp.
constexpr int kCT = 96;
constexpr int kNE = 36;         // electron sums: sigma, sigmaS, alpha_el, kappa0_el (3x3 each)
constexpr int kNP = 18;         // phonon sums: alpha_ph, kappa_ph

// Block sums of nacc (<= kNE) per-thread values into out[0..nacc).  Within a warp the values go
// through shared memory and lane l adds value l (and l + 32) over the 32 lanes: 2 FP64
// instructions per lane-column instead of 5 shuffle-adds per value; then the warps' sums are
// added in a fixed order (reproducible).
__device__ inline void block_reduce_store(double *acc, int nacc, double *out) {
  __shared__ double tr[kCT / 32][32][kNE + 1];   // +1: column reads without bank conflicts
  __shared__ double wsum[kCT / 32][kNE];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < nacc; ++j) tr[wid][lane][j] = acc[j];
  __syncwarp();
  for (int v = lane; v < nacc; v += 32) {
    double sum = 0.0;
    for (int r = 0; r < 32; ++r) sum += tr[wid][r][v];
    wsum[wid][v] = sum;
  }
  __syncthreads();
  if (threadIdx.x < nacc) {
    double sum = 0.0;
    for (int w = 0; w < kCT / 32; ++w) sum += wsum[w][threadIdx.x];
    out[threadIdx.x] = sum;
  }
}

// f(1-f)/|stab| weighted v (x) {J, -I} and (eps-mu) v (x) {J, -I} of one state
__device__ inline void e_tensor_acc(const BteDev &B, int64_t st, const double *Is, const double *Js, double *acc) {
  const double wff = B.st_wt[st] * B.st_ff[st];
  if (wff == 0.0) return;
  const double d = B.st_eps[st] - B.mu;
  const double *v = B.st_vel + st * 3;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double vj = wff * v[a] * Js[b];
      double vi = -wff * v[a] * Is[b];
      acc[a * 3 + b] += vj;
      acc[9 + a * 3 + b] += vi;
      acc[18 + a * 3 + b] += d * vj;
      acc[27 + a * 3 + b] += d * vi;
    }
}

// Final assembly, spread over threads (single-thread FP64 chains are slow on this GPU).
// res: [0] sigma [9] sigmaS [18] alpha_el [27] kappa0_el [36] alpha_ph [45] kappa_ph [54] S [63] kappa_el
//      [72] residual_e [73] residual_all
__device__ void coeff_final_body(const ModelDev &M, const BteDev &B, const double *epart, const double *ppart,
                                 int npart, double *res, double *prev, int *ctl, int max_sweeps, double tol) {
  // device-driven loop (ctl != nullptr): ctl[0] stop flag, ctl[1] sweeps done, ctl[2] converged
  if (ctl && ctl[0]) return;
  __shared__ double Ms[kNE + kNP];
  __shared__ double R[72];
  __shared__ double inv[10];
  __shared__ double rc[6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < kNE + kNP; j += nw) {
    double s = 0.0;
    for (int b = lane; b < npart; b += 32)
      s += j < kNE ? __ldcg(epart + size_t(b) * kNE + j) : __ldcg(ppart + size_t(b) * kNP + (j - kNE));
    s = warp_sum(s);
    if (lane == 0) Ms[j] = s;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < 36) {   // symmetrised electron tensors: sum_S S M S^T = sum_ef sym_pair[ab][ef] M_ef
    const int c = t / 9, ab = t % 9;
    const double *Mc = Ms + 9 * c;
    double s = 0.0;
    for (int ef = 0; ef < 9; ++ef) s += M.sym_pair[ab * 9 + ef] * Mc[ef];
    R[t] = (c < 2 ? 1.0 : -1.0) * B.Pe * s;
  } else if (t < 54) {   // phonon tensors: the group sum of the wedge sums
    const int c = (t - 36) / 9, ab = (t - 36) % 9;
    const double *Mc = Ms + 36 + 9 * c;
    double s = 0.0;
    for (int ef = 0; ef < 9; ++ef) s += M.sym_pair[ab * 9 + ef] * Mc[ef];
    R[t] = B.Pph * s;
  }
  __syncthreads();
  if (t < 9) {    // adjugate of sigma
    const double *s = R;
    const int i0 = t / 3, j0 = t % 3;
    // inv[j0][i0] = cofactor(i0, j0)
    const int r1 = (i0 + 1) % 3, r2 = (i0 + 2) % 3, c1 = (j0 + 1) % 3, c2 = (j0 + 2) % 3;
    inv[j0 * 3 + i0] = s[r1 * 3 + c1] * s[r2 * 3 + c2] - s[r1 * 3 + c2] * s[r2 * 3 + c1];
  }
  __syncthreads();
  if (t == 0) inv[9] = R[0] * inv[0] + R[1] * inv[3] + R[2] * inv[6];
  __syncthreads();
  if (t < 9) {    // S = sigma^-1 sigmaS
    const int a = t / 3, b = t % 3;
    double v = 0.0;
    for (int c = 0; c < 3; ++c) v += inv[a * 3 + c] * R[9 + c * 3 + b];
    R[54 + t] = inv[9] != 0.0 ? v / inv[9] : 0.0;
  }
  __syncthreads();
  if (t < 9) {    // kappa_el = kappa0_el - alpha_el S
    const int a = t / 3, b = t % 3;
    double v = 0.0;
    for (int c = 0; c < 3; ++c) v += R[18 + a * 3 + c] * R[54 + c * 3 + b];
    R[63 + t] = R[27 + t] - v;
  }
  if (t >= 32 && t < 38) {   // relative change of each of the six tensors
    const int c = t - 32;
    double n = 0.0, d = 0.0;
    for (int j = 0; j < 9; ++j) {
      const double x = R[9 * c + j], y = prev[9 * c + j];
      n += x * x;
      d += (x - y) * (x - y);
    }
    rc[c] = n == 0.0 ? 0.0 : sqrt(d) / sqrt(n);
  }
  __syncthreads();
  if (t < 72) res[t] = R[t];
  if (t < 54) prev[t] = R[t];
  if (t == 0) {
    double re = 0.0, ra = 0.0;
    for (int c = 0; c < 6; ++c) {
      if (c < 4) re = fmax(re, rc[c]);
      ra = fmax(ra, rc[c]);
    }
    res[72] = re;
    res[73] = ra;
    if (ctl) {
      const int n = ctl[1] + 1;
      ctl[1] = n;
      const bool conv = re < tol;
      if (conv) ctl[2] = 1;
      if (conv || n >= max_sweeps) ctl[0] = 1;
    }
  }
}

// I = I0 + (self partials + drag term) / (f(1-f) W), same for J; plus the electron
// coefficient partial sums of the new responses.
__global__ void __launch_bounds__(kCT) k_e_finalize(BteDev B, SweepSegs S, const double *__restrict__ part,
                                                    const double *__restrict__ Dterm, const double *__restrict__ I0,
                                                    const double *__restrict__ J0, const double *__restrict__ inv_ffW,
                                                    double *I_out, double *J_out, double *I_alt, double *J_alt,
                                                    double2 *IJ_out, double2 *IJ_alt,
                                                    const int *__restrict__ ctl, double *epart, ModelDev M,
                                                    CoeffFuse F) {
  if (ctl) {
    if (ctl[0]) return;
    if (ctl[1] & 1) {
      I_out = I_alt;
      J_out = J_alt;
      IJ_out = IJ_alt;
    }
  }
  double acc[kNE];
  for (int j = 0; j < kNE; ++j) acc[j] = 0.0;
  const int64_t stride = int64_t(gridDim.x) * kCT;
  for (int64_t st = blockIdx.x * int64_t(kCT) + threadIdx.x; st < B.nst; st += stride) {
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t g = S.seg_ptr[st]; g < S.seg_ptr[st + 1]; ++g)
      for (int c = 0; c < 6; ++c) s[c] += part[g * 6 + c];
    if (Dterm)
      for (int c = 0; c < 6; ++c) s[c] += Dterm[st * 6 + c];
    const double c0 = inv_ffW[st];
    double In[3], Jn[3];
    for (int c = 0; c < 3; ++c) {
      In[c] = I0[st * 3 + c] + s[c] * c0;
      Jn[c] = J0[st * 3 + c] + s[3 + c] * c0;
      I_out[st * 3 + c] = In[c];
      J_out[st * 3 + c] = Jn[c];
    }
    if (IJ_out) {
      double2 *p = IJ_out + st * 3;
      p[0] = make_double2(In[0], In[1]);
      p[1] = make_double2(In[2], Jn[0]);
      p[2] = make_double2(Jn[1], Jn[2]);
    }
    e_tensor_acc(B, st, In, Jn, acc);
  }
  block_reduce_store(acc, kNE, epart + size_t(blockIdx.x) * kNE);
  if (!F.counter) return;
  // the last block to finish assembles the coefficients (and advances the sweep loop), so a
  // sweep costs two launches instead of three
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(F.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  coeff_final_body(M, B, epart, F.ppart, gridDim.x, F.res, F.prev, F.ctl, F.max_sweeps, F.tol);
  if (threadIdx.x == 0) *F.counter = 0u;
}

__global__ void __launch_bounds__(kCT) k_e_partial(BteDev B, const double *I, const double *J, double *epart) {
  double acc[kNE];
  for (int j = 0; j < kNE; ++j) acc[j] = 0.0;
  const int64_t stride = int64_t(gridDim.x) * kCT;
  for (int64_t st = blockIdx.x * int64_t(kCT) + threadIdx.x; st < B.nst; st += stride)
    e_tensor_acc(B, st, I + st * 3, J + st * 3, acc);
  block_reduce_store(acc, kNE, epart + size_t(blockIdx.x) * kNE);
}

// Phonon coefficient sums over the representatives of the q wedge, each weighted by
// 1/|stabiliser|: the responses, velocities and weights are covariant (F(S q) = C_S F(q)), so
// the sum over a star is (1/|stab|) sum_S C_S M(<q>) C_S^T, and the assembly applies the group
// sum.  w n(1+n) comes from the solve's RTA tables (n(1+n) = 1 / (inv_nnW W)) instead of the
// Bose factor's exponential.
__global__ void __launch_bounds__(kCT) k_ph_partial(MeshDev D, BteDev B, const double *F, const double *G,
                                                    const double *__restrict__ W_ph,
                                                    const double *__restrict__ inv_nnW, double *ppart) {
  double acc[kNP];
  for (int j = 0; j < kNP; ++j) acc[j] = 0.0;
  const int64_t stride = int64_t(gridDim.x) * kCT;
  for (int64_t r = blockIdx.x * int64_t(kCT) + threadIdx.x; r < D.n_qrep * B.nbr; r += stride) {
    const int q = D.qlist[r / B.nbr];
    const int64_t t = int64_t(q) * B.nbr + r % B.nbr;
    const double w = D.w[t], W = W_ph[t];
    if (!(w > D.omega_min) || !(W > 0.0)) continue;
    const double wt = w / (inv_nnW[t] * W * double(D.qstab[q]));
    const double *v = D.vph + t * 3;
    for (int a = 0; a < 3; ++a) {
      const double u = wt * v[a];
      for (int b = 0; b < 3; ++b) {
        acc[a * 3 + b] -= u * G[t * 3 + b];
        acc[9 + a * 3 + b] += u * F[t * 3 + b];
      }
    }
  }
  block_reduce_store(acc, kNP, ppart + size_t(blockIdx.x) * kNP);
}

__global__ void __launch_bounds__(512) k_coeff_final(ModelDev M, BteDev B, const double *epart,
                                                     const double *ppart, int npart, double *res, double *prev,
                                                     int *ctl, int max_sweeps, double tol) {
  coeff_final_body(M, B, epart, ppart, npart, res, prev, ctl, max_sweeps, tol);
}

// Kelvin-Onsager step: B = sigmaS[I_drag], A = alpha_ph / T, lambda = <A,B>/<B,B>
__global__ void __launch_bounds__(kCT) k_ko_partial(BteDev B, const double *I, const double *J, double *kpart) {
  double acc[9];
  for (int j = 0; j < 9; ++j) acc[j] = 0.0;
  const int64_t stride = int64_t(gridDim.x) * kCT;
  for (int64_t st = blockIdx.x * int64_t(kCT) + threadIdx.x; st < B.nst; st += stride) {
    double wff = B.st_wt[st] * B.st_ff[st];
    if (wff == 0.0) continue;
    double d = (B.st_eps[st] - B.mu) / B.T;
    const double *v = B.st_vel + st * 3;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) acc[a * 3 + b] += -wff * v[a] * (I[st * 3 + b] - d * J[st * 3 + b]);
  }
  block_reduce_store(acc, 9, kpart + size_t(blockIdx.x) * 9);
}

__global__ void k_ko_final(ModelDev M, BteDev B, const double *kpart, int npart, double *res) {
  __shared__ double Ms[9];
  __shared__ double Bt[9];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < 9; j += nw) {
    double s = 0.0;
    for (int b = lane; b < npart; b += 32) s += kpart[size_t(b) * 9 + j];
    s = warp_sum(s);
    if (lane == 0) Ms[j] = s;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < 9) {
    double s = 0.0;
    for (int ef = 0; ef < 9; ++ef) s += M.sym_pair[t * 9 + ef] * Ms[ef];
    Bt[t] = B.Pe * s;
  }
  __syncthreads();
  if (t != 0) return;
  double bb = 0.0, ab = 0.0;
  for (int j = 0; j < 9; ++j) {
    double a = res[36 + j] / B.T;
    bb += Bt[j] * Bt[j];
    ab += a * Bt[j];
  }
  if (sqrt(bb) > 1e-30) {
    res[74] = ab / bb;
    res[75] = 1.0;
  } else {
    res[75] = 0.0;
  }
}

__global__ void k_ko_apply(BteDev B, double *I, const double *J, const double *res) {
  if (res[75] == 0.0) return;
  double lam = res[74];
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= B.nst * 3) return;
  int64_t st = t / 3;
  double d = (B.st_eps[st] - B.mu) / B.T;
  double idiff = d * J[t];
  I[t] = idiff + lam * (I[t] - idiff);
}

}  // namespace

int coeff_partials() { return kNPart; }
int sweep_segment_len() { return kSeg; }

cudaError_t launch_state_setup(const ModelDev &M, const MeshDev &D, double T, double mu, double lo, double hi,
                               double *st_eps, double *st_vel, double *st_ff, double *st_wt, uint32_t *kcrd,
                               int2 *kinfo, cudaStream_t st) {
  int64_t n = D.n_ibzw * M.nb > D.nk ? D.n_ibzw * M.nb : D.nk;
  EPHB_LAUNCH(k_state_setup, unsigned((n + 255) / 256), 256, 0, st, M, D, T, mu, lo, hi, st_eps, st_vel, st_ff, st_wt,
              kcrd, kinfo);
  return cudaGetLastError();
}

cudaError_t launch_rta_electron(const BteDev &B, double *W_e, double *inv_ffW, double *I0, double *J0,
                                unsigned long long *n_zero, cudaStream_t st, const double *W_add) {
  cudaError_t e = cudaMemsetAsync(n_zero, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess || B.nst == 0) return e;
  EPHB_LAUNCH(k_rta_electron, unsigned((B.nst * 32 + 255) / 256), 256, 0, st, B, W_e, inv_ffW, I0, J0, n_zero,
              W_add);
  return cudaGetLastError();
}

namespace {

// ---- electron-charged-impurity scattering (e-chimp): Eqs. |g^e-chimp_q|^2, q_TF^2, X^e-chimp

constexpr int kChimpSumBlocks = 152;
constexpr double kEps0 = 8.8541878128e-12;   // F / m

// partial sums of f(1 - f) over every band of every k point (fixed grid: reproducible)
__global__ void __launch_bounds__(256) k_ff_sum(int64_t n, const double *__restrict__ eps, double mu, double kT,
                                                double *part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double f = fermi_b(eps[i], mu, kT);
    s += f * (1.0 - f);
  }
  s = warp_sum(s);
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += w[i];
    part[blockIdx.x] = t;
  }
}

// q_TF^2 = ff_scale * sum f(1 - f) (1/m^2)
__global__ void k_tf_final(const double *part, int nparts, double ff_scale, double *q_tf2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < nparts; ++i) t += part[i];
  *q_tf2 = ff_scale * t;
}

__device__ inline double centred_frac(int i, int n) {
  const double f = double(i) / double(n);
  return f - floor(f + 0.5);
}

// One warp per state (irreducible window k, band): W^chimp = 2 pi/(hbar N_k) sum over the
// window states (k', n) of the full mesh of |g_q|^2 (1 - k.k'/(k k')) delta(eps' - eps), with
// q = [k' - k] and k, k', q Cartesian vectors of the centred crystal coordinates (a zero-length
// k or k' has transport factor 1, the cosine is clipped to [-1, 1]); |g_q|^2 = (1/V) sum_i n_i
// [Z_i e / (eps0 eps (q^2 + q_TF^2))]^2 (numerically eV^2); Gaussian delta with the e-ph cut.
__global__ void __launch_bounds__(256) k_chimp_rates(MeshDev D, BteDev B, ChimpParams P, const double *q_tf2_dev,
                                                     double *W) {
  const int64_t st = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (st >= B.nst) return;
  if (!(B.st_ff[st] > 0.0)) {
    if (lane == 0) W[st] = 0.0;
    return;
  }
  const int nb = B.nb;
  const int k = D.ibzw_list[st / nb];
  const double e0 = B.st_eps[st];
  const double q_tf2 = *q_tf2_dev;
  int a0, a1, a2;
  D.km.unflat(k, a0, a1, a2);
  const double fk[3] = {centred_frac(a0, D.km.n[0]), centred_frac(a1, D.km.n[1]), centred_frac(a2, D.km.n[2])};
  double kv[3];
  for (int x = 0; x < 3; ++x) kv[x] = fk[0] * P.rec[0][x] + fk[1] * P.rec[1][x] + fk[2] * P.rec[2][x];
  const double kn = sqrt(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
  const double cut = P.cut_sigmas * P.sigma, inv2s2 = 0.5 / (P.sigma * P.sigma);
  double acc = 0.0;
  for (int64_t kp = lane; kp < D.nk; kp += 32) {
    const uint32_t mask = D.amask[kp];
    if (!mask) continue;
    int b0, b1, b2;
    D.km.unflat(int(kp), b0, b1, b2);
    double g2 = -1.0, tf = 0.0;   // computed at the first band inside the cut
    for (int n = 0; n < nb; ++n) {
      if (!((mask >> n) & 1u)) continue;
      const double e1 = D.eps[size_t(kp) * nb + n];
      if (e1 < P.win_lo || e1 > P.win_hi) continue;
      const double x = e1 - e0;
      if (fabs(x) > cut) continue;
      if (g2 < 0.0) {
        const double fp[3] = {centred_frac(b0, D.km.n[0]), centred_frac(b1, D.km.n[1]), centred_frac(b2, D.km.n[2])};
        double fq[3], qv[3], pv[3];
        for (int y = 0; y < 3; ++y) {
          const double d = fp[y] - fk[y];
          fq[y] = d - floor(d + 0.5);
        }
        for (int y = 0; y < 3; ++y) {
          qv[y] = fq[0] * P.rec[0][y] + fq[1] * P.rec[1][y] + fq[2] * P.rec[2][y];
          pv[y] = fp[0] * P.rec[0][y] + fp[1] * P.rec[1][y] + fp[2] * P.rec[2][y];
        }
        const double q2 = qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2];
        g2 = 0.0;
        for (int i = 0; i < P.nspec; ++i) {
          const double u = P.Z[i] * kECharge / (kEps0 * P.eps_r * (q2 + q_tf2));
          g2 += P.n_m3[i] * u * u;
        }
        g2 /= P.V;
        const double pn = sqrt(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
        const double den = kn * pn;
        double c = den > 0.0 ? (kv[0] * pv[0] + kv[1] * pv[1] + kv[2] * pv[2]) / den : 0.0;
        c = fmin(fmax(c, -1.0), 1.0);
        tf = 1.0 - c;
      }
      acc += g2 * tf * exp(-x * x * inv2s2) * P.gnorm;
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) W[st] = P.pref * acc;
}

}  // namespace

cudaError_t launch_chimp_rates(const MeshDev &D, const BteDev &B, const ChimpParams &P, const double *eps_all,
                               int64_t n_eps, double ff_scale, double *part, double *q_tf2, double *W,
                               cudaStream_t st) {
  EPHB_LAUNCH(k_ff_sum, kChimpSumBlocks, 256, 0, st, n_eps, eps_all, B.mu, kKbEVK * B.T, part);
  EPHB_LAUNCH(k_tf_final, 1, 32, 0, st, part, kChimpSumBlocks, ff_scale, q_tf2);
  if (B.nst > 0) EPHB_LAUNCH(k_chimp_rates, unsigned((B.nst * 32 + 255) / 256), 256, 0, st, D, B, P, q_tf2, W);
  return cudaGetLastError();
}

int chimp_partials() { return kChimpSumBlocks; }

cudaError_t launch_ph_rowsum(const BteDev &B, double *Bt, cudaStream_t st) {
  EPHB_LAUNCH(k_ph_rowsum, unsigned((B.nq * B.nbr * 32 + 255) / 256), 256, 0, st, B, Bt);
  return cudaGetLastError();
}

cudaError_t launch_rta_phonon(const ModelDev &M, const MeshDev &D, const BteDev &B, const double *Bt, double *W_ph,
                              double *inv_nnW, double *F0, cudaStream_t st, const double *W_add) {
  EPHB_LAUNCH(k_rta_phonon, unsigned((D.nq * M.nbr + 255) / 256), 256, 0, st, M, D, B, Bt, W_ph, inv_nnW, F0,
              W_add);
  return cudaGetLastError();
}

namespace {

// ---- phonon-isotope scattering (Tamura): Eq. W^ph-x, its part of W^RTA_sq

constexpr int kIsoThreads = 256;

// One block per representative q of the q wedge, all its branches s: threads strided over q'
// sum g_tau |xi*_{tau,sq} . xi_{tau,s'q'}|^2 delta(E' - E) over the branches s' above omega_min
// (the Gaussian of the rates call), then the warps' and the block's sums in a fixed order;
// W = pi E^2 / (2 hbar N_q) x sum, averaged over the degenerate group of s, zero for modes at or
// below omega_min.  Wrep[rep][s].
__global__ void __launch_bounds__(kIsoThreads) k_iso_rates(ModelDev M, MeshDev D, IsoParams P, double *Wrep) {
  const int nbr = M.nbr;
  const int r = blockIdx.x;
  const int q = D.qlist[r];
  __shared__ double2 xi[kMaxBranches * kMaxBranches];
  __shared__ double wq[kMaxBranches];
  __shared__ double part[kIsoThreads / 32][kMaxBranches];
  __shared__ double raw[kMaxBranches];
  for (int t = threadIdx.x; t < nbr * nbr; t += blockDim.x) xi[t] = D.u[size_t(q) * nbr * nbr + t];
  for (int t = threadIdx.x; t < nbr; t += blockDim.x) wq[t] = D.w[size_t(q) * nbr + t];
  __syncthreads();
  double acc[kMaxBranches];
  for (int s = 0; s < kMaxBranches; ++s) acc[s] = 0.0;
  const double cut = P.cut_sigmas * P.sigma, inv2s2 = 0.5 / (P.sigma * P.sigma);
  for (int64_t qp = threadIdx.x; qp < D.nq; qp += blockDim.x) {
    const double2 *up = D.u + size_t(qp) * nbr * nbr;
    for (int sp = 0; sp < nbr; ++sp) {
      const double wp = D.w[size_t(qp) * nbr + sp];
      if (!(wp > D.omega_min)) continue;
      for (int s = 0; s < nbr; ++s) {
        const double x = wp - wq[s];
        if (fabs(x) > cut) continue;
        double ov = 0.0;
        for (int a = 0; a < M.nat; ++a) {
          double2 d = cmk(0.0, 0.0);
          for (int c = 0; c < 3; ++c) cfma_conj(d, xi[(3 * a + c) * nbr + s], up[(3 * a + c) * nbr + sp]);
          ov += P.g[a] * (d.x * d.x + d.y * d.y);
        }
        acc[s] += ov * exp(-x * x * inv2s2) * P.gnorm;
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int s = 0; s < nbr; ++s) {
    const double v = warp_sum(acc[s]);
    if (lane == 0) part[wid][s] = v;
  }
  __syncthreads();
  if (threadIdx.x < nbr) {
    const int s = threadIdx.x;
    double t = 0.0;
    for (int w = 0; w < kIsoThreads / 32; ++w) t += part[w][s];
    raw[s] = wq[s] > D.omega_min ? P.pref * wq[s] * wq[s] * t : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < nbr) {
    const int s = threadIdx.x;
    const int g0 = D.pgrp[(size_t(q) * nbr + s) * 2], g1 = D.pgrp[(size_t(q) * nbr + s) * 2 + 1];
    double t = 0.0;
    for (int j = g0; j < g1; ++j) t += raw[j];
    Wrep[size_t(r) * nbr + s] = t / double(g1 - g0);
  }
}

// every q takes its representative's rates (W^ph-x is invariant under the point group)
__global__ void k_iso_spread(MeshDev D, int nbr, const double *Wrep, double *W) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= D.nq * nbr) return;
  const int q = int(t / nbr), s = int(t % nbr);
  W[t] = Wrep[size_t(D.qrep_of[D.qrep[q]]) * nbr + s];
}

}  // namespace

cudaError_t launch_iso_rates(const ModelDev &M, const MeshDev &D, const IsoParams &P, double *Wrep, double *W,
                             cudaStream_t st) {
  if (D.n_qrep > 0) EPHB_LAUNCH(k_iso_rates, unsigned(D.n_qrep), kIsoThreads, 0, st, M, D, P, Wrep);
  if (D.nq * M.nbr > 0) EPHB_LAUNCH(k_iso_spread, unsigned((D.nq * M.nbr + 255) / 256), 256, 0, st, D, M.nbr, Wrep, W);
  return cudaGetLastError();
}


cudaError_t launch_build_segments(int64_t nrow, const int64_t *row_ptr, int *nseg_row, int64_t *seg_ptr,
                                  int64_t *scratch, int64_t scratch_elems, int64_t &nseg_host, cudaStream_t st) {
  if (nrow == 0) {
    nseg_host = 0;
    return cudaMemsetAsync(seg_ptr, 0, sizeof(int64_t), st);
  }
  EPHB_LAUNCH(k_seg_count, unsigned((nrow + 255) / 256), 256, 0, st, nrow, row_ptr, nseg_row);
  cudaError_t e = exclusive_scan<int>(nseg_row, seg_ptr, nrow, seg_ptr + nrow, scratch, scratch_elems, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(&nseg_host, seg_ptr + nrow, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t launch_fill_segments(int64_t nrow, const int64_t *row_ptr, const int64_t *seg_ptr, int *seg_row,
                                 int64_t *seg_begin, cudaStream_t st) {
  if (nrow == 0) return cudaSuccess;
  EPHB_LAUNCH(k_seg_fill, unsigned((nrow + 255) / 256), 256, 0, st, nrow, row_ptr, seg_ptr, seg_row, seg_begin);
  return cudaGetLastError();
}

cudaError_t launch_build_runs(const BteDev &B, int64_t n_entries, const int2 *kinfo, int *flag, int64_t *runidx,
                              int64_t *scratch, int64_t scratch_elems, int64_t *run_ptr, uint32_t *run_col,
                              double *run_w, int64_t &nruns, int64_t *total_dev, cudaStream_t st) {
  nruns = 0;
  if (n_entries > 0) {
    const unsigned ge = unsigned((n_entries + 255) / 256);
    EPHB_LAUNCH(k_run_flags, ge, 256, 0, st, n_entries, B.e_kpns, flag);
    EPHB_LAUNCH(k_run_rowstarts, unsigned((B.nst + 255) / 256), 256, 0, st, B.nst, B.row_ptr, flag);
    cudaError_t e = exclusive_scan<int>(flag, runidx, n_entries, total_dev, scratch, scratch_elems, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(&nruns, total_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_fill_runs(const BteDev &B, int64_t n_entries, int64_t nruns, const int2 *kinfo, const int *flag,
                             const int64_t *runidx, int64_t *run_ptr, uint32_t *run_col, double *run_w,
                             cudaStream_t st) {
  if (n_entries > 0)
    EPHB_LAUNCH(k_run_fill, unsigned((n_entries + 255) / 256), 256, 0, st, n_entries, B.e_kpns, B.e_X, flag, runidx,
                kinfo, run_col, run_w);
  EPHB_LAUNCH(k_run_ptr, unsigned((B.nst + 1 + 255) / 256), 256, 0, st, B.nst, B.row_ptr, runidx, n_entries, nruns,
              run_ptr);
  return cudaGetLastError();
}

cudaError_t launch_self_sweep(const ModelDev &M, const BteDev &B, const SweepSegs &S, const uint32_t *run_col,
                              const double *run_w, const double *I0, const double *J0, const double *inv_ffW,
                              double *Ia, double *Ja, double *Ib, double *Jb, const double *Dterm, double *part,
                              double *epart, const int *ctl, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1,
                              double2 *IJa, double2 *IJb, const CoeffFuse *fuse) {
  if (ev0) {
    cudaError_t e = cudaEventRecord(ev0, st);
    if (e != cudaSuccess) return e;
  }
  if (S.nseg > 0) {
    const unsigned grid = unsigned((S.nseg * 32 + 255) / 256);
    if (M.nsym > 1)
      EPHB_LAUNCH(k_self_sweep_seg<true>, grid, 256, 0, st, M, S, run_col, run_w, Ia, Ja, Ib, Jb, IJa, IJb, ctl,
                  part);
    else
      EPHB_LAUNCH(k_self_sweep_seg<false>, grid, 256, 0, st, M, S, run_col, run_w, Ia, Ja, Ib, Jb, IJa, IJb, ctl,
                  part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (ev1) {
    cudaError_t e = cudaEventRecord(ev1, st);
    if (e != cudaSuccess) return e;
  }
  EPHB_LAUNCH(k_e_finalize, kNPart, kCT, 0, st, B, S, part, Dterm, I0, J0, inv_ffW, Ib, Jb, Ia, Ja, IJb, IJa, ctl,
              epart, M, fuse ? *fuse : CoeffFuse{});
  return cudaGetLastError();
}

namespace {

// ---- mixed-precision electron loop: FP32 correction sweeps between FP64 residual sweeps
// d <- r + (1/(f(1-f)W)) sum_runs w d[partner] in FP32 over the same runs and segments.

__global__ void __launch_bounds__(256) k_corr_sweep_seg(ModelDev M, SweepSegs S, const uint32_t *__restrict__ run_col,
                                                        const float *__restrict__ run_w32,
                                                        const float *__restrict__ dI, const float *__restrict__ dJ,
                                                        float *__restrict__ part) {
  __shared__ float C[kMaxSym * 9];
  const bool sym = M.nsym > 1;
  if (sym) {
    for (int t = threadIdx.x; t < M.nsym * 9; t += blockDim.x) C[t] = float(M.sym_cart[t]);
    __syncthreads();
  }
  const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= S.nseg) return;
  const int row = S.seg_row[g];
  const int64_t b = S.seg_begin[g];
  const int64_t rend = S.row_ptr[row + 1];
  const int64_t e_end = b + kSeg < rend ? b + kSeg : rend;
  float a[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t e0 = b + lane; e0 < e_end; e0 += 32 * kUnroll) {
    // the run words and weights of kUnroll runs first, then their gathers (more loads in flight)
    uint32_t pcs[kUnroll];
    float ws[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t e = e0 + 32 * u;
      pcs[u] = e < e_end ? __ldcs(run_col + e) : kRunNone;
      ws[u] = e < e_end ? __ldcs(run_w32 + e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t pc = pcs[u];
      const uint32_t col = pc & kRunColMask;
      if (col == kRunNone) continue;
      const float w = ws[u];
      float vi[3] = {dI[int64_t(col) * 3], dI[int64_t(col) * 3 + 1], dI[int64_t(col) * 3 + 2]};
      float vj[3] = {dJ[int64_t(col) * 3], dJ[int64_t(col) * 3 + 1], dJ[int64_t(col) * 3 + 2]};
      if (sym) {
        const float *Cs = C + 9 * (pc >> 26);
        float r[3];
        for (int x = 0; x < 3; ++x) r[x] = Cs[3 * x] * vi[0] + Cs[3 * x + 1] * vi[1] + Cs[3 * x + 2] * vi[2];
        for (int x = 0; x < 3; ++x) vi[x] = r[x];
        for (int x = 0; x < 3; ++x) r[x] = Cs[3 * x] * vj[0] + Cs[3 * x + 1] * vj[1] + Cs[3 * x + 2] * vj[2];
        for (int x = 0; x < 3; ++x) vj[x] = r[x];
      }
      for (int c = 0; c < 3; ++c) {
        a[c] = fmaf(w, vi[c], a[c]);
        a[3 + c] = fmaf(w, vj[c], a[3 + c]);
      }
    }
  }
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_down_sync(0xffffffffu, a[c], o);
  if (lane == 0)
    for (int c = 0; c < 6; ++c) part[g * 6 + c] = a[c];
}

__global__ void k_corr_finalize(int64_t nst, SweepSegs S, const float *__restrict__ part,
                                const float *__restrict__ rI, const float *__restrict__ rJ,
                                const double *__restrict__ inv_ffW, float *dI, float *dJ) {
  const int64_t st = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (st >= nst) return;
  float sum[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t g = S.seg_ptr[st]; g < S.seg_ptr[st + 1]; ++g)
    for (int c = 0; c < 6; ++c) sum[c] += part[g * 6 + c];
  const float c0 = float(inv_ffW[st]);
  for (int c = 0; c < 3; ++c) {
    dI[st * 3 + c] = rI[st * 3 + c] + c0 * sum[c];
    dJ[st * 3 + c] = rJ[st * 3 + c] + c0 * sum[3 + c];
  }
}

// r = x' - x (FP32), d = r
__global__ void k_corr_init(int64_t n3, const double *I1, const double *I0x, const double *J1, const double *J0x,
                            float *rI, float *rJ, float *dI, float *dJ) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n3) return;
  const float a = float(I1[t] - I0x[t]), b = float(J1[t] - J0x[t]);
  rI[t] = a;
  dI[t] = a;
  rJ[t] = b;
  dJ[t] = b;
}

// x <- x + d (FP64)
__global__ void k_corr_apply(int64_t n3, const float *dI, const float *dJ, double *I, double *J) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n3) return;
  I[t] += double(dI[t]);
  J[t] += double(dJ[t]);
}

__global__ void k_to_f32(int64_t n, const double *a, float *b) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < n) b[t] = float(a[t]);
}

}  // namespace

namespace {
__global__ void k_pack_ij(int64_t nst, const double *I, const double *J, double2 *IJ) {
  const int64_t st = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (st >= nst) return;
  double2 *p = IJ + st * 3;
  p[0] = make_double2(I[st * 3], I[st * 3 + 1]);
  p[1] = make_double2(I[st * 3 + 2], J[st * 3]);
  p[2] = make_double2(J[st * 3 + 1], J[st * 3 + 2]);
}
}  // namespace

cudaError_t launch_pack_ij(int64_t nst, const double *I, const double *J, double2 *IJ, cudaStream_t st) {
  if (nst == 0) return cudaSuccess;
  EPHB_LAUNCH(k_pack_ij, unsigned((nst + 255) / 256), 256, 0, st, nst, I, J, IJ);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(int64_t n, const double *a, float *b, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  EPHB_LAUNCH(k_to_f32, unsigned((n + 255) / 256), 256, 0, st, n, a, b);
  return cudaGetLastError();
}

cudaError_t launch_corr_init(int64_t nst, const double *I1, const double *I0x, const double *J1, const double *J0x,
                             float *rI, float *rJ, float *dI, float *dJ, cudaStream_t st) {
  const int64_t n3 = nst * 3;
  if (n3 == 0) return cudaSuccess;
  EPHB_LAUNCH(k_corr_init, unsigned((n3 + 255) / 256), 256, 0, st, n3, I1, I0x, J1, J0x, rI, rJ, dI, dJ);
  return cudaGetLastError();
}

cudaError_t launch_corr_sweep(const ModelDev &M, int64_t nst, const SweepSegs &S, const uint32_t *run_col,
                              const float *run_w32, const double *inv_ffW, const float *rI, const float *rJ,
                              const float *dI, const float *dJ, float *part, float *dI_out, float *dJ_out,
                              cudaStream_t st) {
  if (S.nseg > 0)
    EPHB_LAUNCH(k_corr_sweep_seg, unsigned((S.nseg * 32 + 255) / 256), 256, 0, st, M, S, run_col, run_w32, dI, dJ,
                part);
  if (nst > 0)
    EPHB_LAUNCH(k_corr_finalize, unsigned((nst + 255) / 256), 256, 0, st, nst, S, part, rI, rJ, inv_ffW, dI_out,
                dJ_out);
  return cudaGetLastError();
}

cudaError_t launch_corr_apply(int64_t nst, const float *dI, const float *dJ, double *I, double *J, cudaStream_t st) {
  const int64_t n3 = nst * 3;
  if (n3 == 0) return cudaSuccess;
  EPHB_LAUNCH(k_corr_apply, unsigned((n3 + 255) / 256), 256, 0, st, n3, dI, dJ, I, J);
  return cudaGetLastError();
}

// ---- Anderson acceleration of the outer iteration.  The iterate is x = (F, G) (F: nph*3
// doubles, then G: nph*3); g = the phonon update from the electrons solved against x; f = g - x.

__global__ void k_and_resid(int64_t half, const double *g, const double *F, const double *G, double *f) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= 2 * half) return;
  f[i] = g[i] - (i < half ? F[i] : G[i - half]);
}

// dot products of f_new with the nslot ring vectors, F half and G half apart, per block
// (fixed grid and per-thread assignment: the sums do not depend on timing)
constexpr int kAndBlocks = 296, kAndThreads = 256;
__global__ void __launch_bounds__(kAndThreads) k_and_dots(int64_t half, const double *fnew, const double *ring,
                                                          int64_t stride, int nslot, double *part) {
  __shared__ double red[kAndThreads / 32][2 * kAndMaxSlots];
  double a[2 * kAndMaxSlots];
  for (int j = 0; j < 2 * kAndMaxSlots; ++j) a[j] = 0.0;
  const int64_t n = 2 * half;
  for (int64_t i = blockIdx.x * int64_t(kAndThreads) + threadIdx.x; i < n; i += int64_t(kAndBlocks) * kAndThreads) {
    const double x = fnew[i];
    const int h = i < half ? 0 : 1;
    for (int j = 0; j < kAndMaxSlots; ++j)
      if (j < nslot) a[2 * j + h] += x * ring[j * stride + i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = 0; j < 2 * kAndMaxSlots; ++j) {
    double v = a[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * kAndMaxSlots) {
    double v = 0.0;
    for (int k = 0; k < kAndThreads / 32; ++k) v += red[k][threadIdx.x];
    part[blockIdx.x * 2 * kAndMaxSlots + threadIdx.x] = v;
  }
}

__global__ void k_and_dots_final(const double *part, double *dots) {
  const int j = threadIdx.x;
  if (j >= 2 * kAndMaxSlots) return;
  double v = 0.0;
  for (int b = 0; b < kAndBlocks; ++b) v += part[b * 2 * kAndMaxSlots + j];
  dots[j] = v;
}

// x = sum_j alpha_j g_j over the ring slots, written to F and G
__global__ void k_and_mix(int64_t half, const double *ring, int64_t stride, int nslot, AndCoef al, double *F,
                          double *G) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= 2 * half) return;
  double x = 0.0;
  for (int j = 0; j < nslot; ++j) x += al.a[j] * ring[j * stride + i];
  if (i < half) F[i] = x; else G[i - half] = x;
}

cudaError_t launch_and_resid(int64_t half, const double *g, const double *F, const double *G, double *f,
                             cudaStream_t st) {
  if (half == 0) return cudaSuccess;
  EPHB_LAUNCH(k_and_resid, unsigned((2 * half + 255) / 256), 256, 0, st, half, g, F, G, f);
  return cudaGetLastError();
}

cudaError_t launch_and_dots(int64_t half, const double *fnew, const double *ring, int64_t stride, int nslot,
                            double *part, double *dots, cudaStream_t st) {
  if (nslot < 1 || nslot > kAndMaxSlots) return cudaErrorInvalidValue;
  EPHB_LAUNCH(k_and_dots, kAndBlocks, kAndThreads, 0, st, half, fnew, ring, stride, nslot, part);
  EPHB_LAUNCH(k_and_dots_final, 1, 32, 0, st, part, dots);
  return cudaGetLastError();
}

size_t and_part_len() { return size_t(kAndBlocks) * 2 * kAndMaxSlots; }

cudaError_t launch_and_mix(int64_t half, const double *ring, int64_t stride, int nslot, const AndCoef &al, double *F,
                           double *G, cudaStream_t st) {
  if (half == 0) return cudaSuccess;
  if (nslot < 1 || nslot > kAndMaxSlots) return cudaErrorInvalidValue;
  EPHB_LAUNCH(k_and_mix, unsigned((2 * half + 255) / 256), 256, 0, st, half, ring, stride, nslot, al, F, G);
  return cudaGetLastError();
}

cudaError_t launch_drag_termff(const MeshDev &D, const BteDev &B, const SweepSegs &S, const float4 *Xff,
                               const float2 *FGff, double *part, double *Dterm, cudaStream_t st) {
  if (B.nst == 0) return cudaSuccess;
  if (S.nseg > 0)
    EPHB_LAUNCH(k_drag_sweep_segff, unsigned((S.nseg * 32 + 255) / 256), 256, 0, st, D, B, S, Xff, FGff, part);
  EPHB_LAUNCH(k_drag_finalize, unsigned((B.nst + 255) / 256), 256, 0, st, B.nst, S, part, Dterm);
  return cudaGetLastError();
}

cudaError_t launch_ph_sweepff(const ModelDev &M, const BteDev &B, const SweepSegs &S, const int2 *kinfo,
                              const float2 *Yff, const float2 *IJff, double *part, double *Btv, cudaStream_t st) {
  const int64_t nrow = B.nq * B.nbr;
  if (S.nseg > 0) {
    const unsigned g = unsigned((S.nseg * 32 + 255) / 256);
    if (M.nsym > 1)
      EPHB_LAUNCH(k_ph_sweepff<true>, g, 256, 0, st, M, B, S, kinfo, Yff, IJff, part);
    else
      EPHB_LAUNCH(k_ph_sweepff<false>, g, 256, 0, st, M, B, S, kinfo, Yff, IJff, part);
  }
  if (nrow > 0) EPHB_LAUNCH(k_ph_seg_finalize, unsigned((nrow + 255) / 256), 256, 0, st, nrow, S, part, Btv);
  return cudaGetLastError();
}

cudaError_t launch_copy_ff(int64_t n, const double *a, float2 *out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  EPHB_LAUNCH(k_copy_ff, unsigned((n + 255) / 256), 256, 0, st, n, a, out);
  return cudaGetLastError();
}

cudaError_t launch_pack6_ff(int64_t n, const double *A, const double *Bv, float2 *out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  EPHB_LAUNCH(k_pack6_ff, unsigned((n + 255) / 256), 256, 0, st, n, A, Bv, out);
  return cudaGetLastError();
}

cudaError_t launch_drag_term32(const MeshDev &D, const BteDev &B, const SweepSegs &S, const float2 *X32,
                               const float *FG32, double *part, double *Dterm, cudaStream_t st) {
  if (B.nst == 0) return cudaSuccess;
  if (S.nseg > 0)
    EPHB_LAUNCH(k_drag_sweep_seg32, unsigned((S.nseg * 32 + 255) / 256), 256, 0, st, D, B, S, X32, FG32, part);
  EPHB_LAUNCH(k_drag_finalize, unsigned((B.nst + 255) / 256), 256, 0, st, B.nst, S, part, Dterm);
  return cudaGetLastError();
}

cudaError_t launch_ph_sweep32(const ModelDev &M, const BteDev &B, const SweepSegs &S, const int2 *kinfo,
                              const float *Y32, const float *IJ32, double *part, double *Btv, cudaStream_t st) {
  const int64_t nrow = B.nq * B.nbr;
  if (S.nseg > 0) {
    const unsigned g = unsigned((S.nseg * 32 + 255) / 256);
    if (M.nsym > 1)
      EPHB_LAUNCH(k_ph_sweep32<true>, g, 256, 0, st, M, B, S, kinfo, Y32, IJ32, part);
    else
      EPHB_LAUNCH(k_ph_sweep32<false>, g, 256, 0, st, M, B, S, kinfo, Y32, IJ32, part);
  }
  if (nrow > 0) EPHB_LAUNCH(k_ph_seg_finalize, unsigned((nrow + 255) / 256), 256, 0, st, nrow, S, part, Btv);
  return cudaGetLastError();
}

cudaError_t launch_pack6_f32(int64_t n, const double *A, const double *Bv, float *out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  EPHB_LAUNCH(k_pack6_f32, unsigned((n + 255) / 256), 256, 0, st, n, A, Bv, out);
  return cudaGetLastError();
}

cudaError_t launch_copy_f32(int64_t n, const double *a, float *b, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  EPHB_LAUNCH(k_copy_f32, unsigned((n + 255) / 256), 256, 0, st, n, a, b);
  return cudaGetLastError();
}

cudaError_t launch_drag_term(const MeshDev &D, const BteDev &B, const SweepSegs &S, const double *F, const double *G,
                             double *part, double *Dterm, cudaStream_t st) {
  if (B.nst == 0) return cudaSuccess;
  if (S.nseg > 0) EPHB_LAUNCH(k_drag_sweep_seg, unsigned((S.nseg * 32 + 255) / 256), 256, 0, st, D, B, S, F, G, part);
  EPHB_LAUNCH(k_drag_finalize, unsigned((B.nst + 255) / 256), 256, 0, st, B.nst, S, part, Dterm);
  return cudaGetLastError();
}

cudaError_t launch_ph_sweep(const ModelDev &M, const BteDev &B, const SweepSegs &S, const int2 *kinfo,
                            const double *I, const double *J, double *part, double *Btv, cudaStream_t st) {
  const int64_t nrow = B.nq * B.nbr;
  if (S.nseg > 0) {
    const unsigned g = unsigned((S.nseg * 32 + 255) / 256);
    if (M.nsym > 1)
      EPHB_LAUNCH(k_ph_sweep<true>, g, 256, 0, st, M, B, S, kinfo, I, J, part);
    else
      EPHB_LAUNCH(k_ph_sweep<false>, g, 256, 0, st, M, B, S, kinfo, I, J, part);
  }
  if (nrow > 0) EPHB_LAUNCH(k_ph_seg_finalize, unsigned((nrow + 255) / 256), 256, 0, st, nrow, S, part, Btv);
  return cudaGetLastError();
}

cudaError_t launch_ph_update(const ModelDev &M, const MeshDev &D, const double *Btv, const double *F0,
                             const double *inv_nnW, double *F, double *G, double *Afold, cudaStream_t st) {
  EPHB_LAUNCH(k_ph_fold_rep, unsigned((D.n_qrep * M.nbr * 8 + 255) / 256), 256, 0, st, M, D, Btv, Afold);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  EPHB_LAUNCH(k_ph_update, unsigned((D.nq * M.nbr + 255) / 256), 256, 0, st, M, D, Afold, F0, inv_nnW, F, G);
  return cudaGetLastError();
}

cudaError_t launch_e_partial(const BteDev &B, const double *I, const double *J, double *epart, cudaStream_t st) {
  EPHB_LAUNCH(k_e_partial, kNPart, kCT, 0, st, B, I, J, epart);
  return cudaGetLastError();
}

cudaError_t launch_ph_partial(const MeshDev &D, const BteDev &B, const double *F, const double *G, const double *W_ph,
                              const double *inv_nnW, double *ppart, cudaStream_t st) {
  EPHB_LAUNCH(k_ph_partial, kNPart, kCT, 0, st, D, B, F, G, W_ph, inv_nnW, ppart);
  return cudaGetLastError();
}

cudaError_t launch_coeff_final(const ModelDev &M, const BteDev &B, const double *epart, const double *ppart,
                               double *res, double *prev, cudaStream_t st, int *ctl, int max_sweeps, double tol) {
  EPHB_LAUNCH(k_coeff_final, 1, 512, 0, st, M, B, epart, ppart, kNPart, res, prev, ctl, max_sweeps, tol);
  return cudaGetLastError();
}

namespace {

// largest electron speed over the active states (non-negative floats order as their bits)
__global__ void k_speed_max(BteDev B, unsigned *vmax_bits) {
  const int64_t st = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (st >= B.nst || !(B.st_wt[st] > 0.0)) return;
  const double *v = B.st_vel + st * 3;
  const float sp = float(sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
  atomicMax(vmax_bits, __float_as_uint(sp));
}

// inputs of the warm-start network per state: (eps-mu)/kT (clipped to +-40) / 10, log10(W)-13,
// |v|/max|v|, T/300 K, mu/0.1 eV, eps/0.3 eV; zeros for inactive states
__global__ void k_state_features(BteDev B, const double *__restrict__ W_e, const unsigned *vmax_bits, float *feat) {
  const int64_t st = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (st >= B.nst) return;
  float *f = feat + st * kNFeat;
  if (!(B.st_wt[st] > 0.0)) {
    for (int c = 0; c < kNFeat; ++c) f[c] = 0.f;
    return;
  }
  const double e = B.st_eps[st], kT = kKbEVK * B.T, W = W_e[st];
  const double *v = B.st_vel + st * 3;
  const float vmax = __uint_as_float(*vmax_bits);
  const double sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  f[0] = float(fmin(fmax((e - B.mu) / kT, -40.0), 40.0) / 10.0);
  f[1] = W > 0.0 ? float(log10(W) - 13.0) : 0.f;
  f[2] = vmax > 0.f ? float(sp / double(vmax)) : 0.f;
  f[3] = float(B.T / 300.0);
  f[4] = float(B.mu / 0.1);
  f[5] = float(e / 0.3);
}

// training targets along the RTA direction J0 = v/W: a_I = (I.J0)/(J0.J0)/k_B - (eps-mu)/(k_B T),
// a_J = (J.J0)/(J0.J0) - 1; zero for inactive states, J0 = 0, or speeds below 1e-6 of the largest
__global__ void k_state_targets(BteDev B, const double *I, const double *J, const double *J0,
                                const unsigned *vmax_bits, float *t) {
  const int64_t st = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (st >= B.nst) return;
  const double *v = B.st_vel + st * 3, *b = J0 + st * 3;
  const double sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double d = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const bool ok = B.st_wt[st] > 0.0 && d > 0.0 && sp > 1e-6 * double(__uint_as_float(*vmax_bits));
  if (!ok) {
    t[st * 2] = 0.f;
    t[st * 2 + 1] = 0.f;
    return;
  }
  const double *x = I + st * 3, *y = J + st * 3;
  const double pi = x[0] * b[0] + x[1] * b[1] + x[2] * b[2];
  const double pj = y[0] * b[0] + y[1] * b[1] + y[2] * b[2];
  t[st * 2] = float(pi / d / kKbEVK - (B.st_eps[st] - B.mu) / (kKbEVK * B.T));
  t[st * 2 + 1] = float(pj / d - 1.0);
}

// starting responses I = I0 + a_I k_B J0, J = J0 (1 + a_J)
__global__ void k_apply_warm(int64_t nst, const double *I0, const double *J0, const float *a, double *I, double *J) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nst * 3) return;
  const int64_t st = t / 3;
  I[t] = I0[t] + double(a[st * 2]) * kKbEVK * J0[t];
  J[t] = J0[t] * (1.0 + double(a[st * 2 + 1]));
}

}  // namespace

cudaError_t launch_state_features(const BteDev &B, const double *W_e, unsigned *vmax_bits, float *feat,
                                  cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned), st);
  if (e != cudaSuccess || B.nst == 0) return e;
  const unsigned g = unsigned((B.nst + 255) / 256);
  EPHB_LAUNCH(k_speed_max, g, 256, 0, st, B, vmax_bits);
  EPHB_LAUNCH(k_state_features, g, 256, 0, st, B, W_e, vmax_bits, feat);
  return cudaGetLastError();
}

cudaError_t launch_state_targets(const BteDev &B, const double *I, const double *J, const double *J0,
                                 unsigned *vmax_bits, float *t, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned), st);
  if (e != cudaSuccess || B.nst == 0) return e;
  const unsigned g = unsigned((B.nst + 255) / 256);
  EPHB_LAUNCH(k_speed_max, g, 256, 0, st, B, vmax_bits);
  EPHB_LAUNCH(k_state_targets, g, 256, 0, st, B, I, J, J0, vmax_bits, t);
  return cudaGetLastError();
}

cudaError_t launch_apply_warm(int64_t nst, const double *I0, const double *J0, const float *a, double *I, double *J,
                              cudaStream_t st) {
  if (nst == 0) return cudaSuccess;
  EPHB_LAUNCH(k_apply_warm, unsigned((nst * 3 + 255) / 256), 256, 0, st, nst, I0, J0, a, I, J);
  return cudaGetLastError();
}

cudaError_t launch_ko(const ModelDev &M, const MeshDev &D, const BteDev &B, double *I, const double *J,
                      double *kpart, double *res, cudaStream_t st) {
  (void)D;
  EPHB_LAUNCH(k_ko_partial, kNPart, kCT, 0, st, B, I, J, kpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  EPHB_LAUNCH(k_ko_final, 1, 288, 0, st, M, B, kpart, kNPart, res);
  e = cudaGetLastError();
  if (e != cudaSuccess || B.nst == 0) return e;
  EPHB_LAUNCH(k_ko_apply, unsigned((B.nst * 3 + 255) / 256), 256, 0, st, B, I, J, res);
  return cudaGetLastError();
}

}  // namespace ephb
