// Rate lists of one (T, mu, window) instance derived from the T-independent vertex lists.
//
// Many (T, mu) instances share the expensive part of Eq. X^e-ph: the interpolated |g|^2 and
// the delta weight depend on the energies only.  The vertex pass stores, over the union of the
// instance windows,
//   V+- = 2pi/(hbar N_q) |g|^2 delta(eps_nk' - eps_mk -/+ hbar w_sq)    (electron rows)
//   V   = V+ N_q / (N_k |stab_k|)                                     (phonon rows)
// and each instance keeps the entries whose two electron states lie in its window, with
//   X+ = V+ f_mk (1 - f_nk') n_sq,   X- = V- f_mk (1 - f_nk') (1 + n_sq),   Y = V f (1 - f') n,
// in the order of the vertex lists, so every row stays ordered as a single-instance row is.
#include "internal.h"

namespace ephb {

namespace {

__device__ inline bool in_window(double e, InstWindow w) { return e >= w.lo && e <= w.hi; }

// q with k' = [k + q] (the k mesh is ratio x the q mesh per dimension)
__device__ inline int q_of(const MeshDev &D, int k, int kp) {
  int a0, a1, a2, b0, b1, b2;
  D.km.unflat(k, a0, a1, a2);
  D.km.unflat(kp, b0, b1, b2);
  return D.qm.flat(pmod(b0 - a0, D.km.n[0]) / D.ratio[0], pmod(b1 - a1, D.km.n[1]) / D.ratio[1],
                   pmod(b2 - a2, D.km.n[2]) / D.ratio[2]);
}

__device__ inline double state_energy(const MeshDev &D, int nb, int st) {
  return D.eps[size_t(D.ibzw_list[st / nb]) * nb + st % nb];
}

// one warp per row: electron rows (k, m) first, then phonon rows (q, s)
__global__ void k_inst_count(ModelDev M, MeshDev D, InstWindow w, const int64_t *__restrict__ u_row_ptr,
                             const uint32_t *__restrict__ u_kpns, const int64_t *__restrict__ u_ph_row_ptr,
                             const int *__restrict__ u_ph_st, const uint32_t *__restrict__ u_ph_kpn, int *cnt_e,
                             int *cnt_ph) {
  const int64_t row = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nb = M.nb;
  const int64_t nst = D.n_ibzw * nb, nph = D.nq * M.nbr;
  if (row >= nst + nph) return;
  int c = 0;
  if (row < nst) {
    if (in_window(state_energy(D, nb, int(row)), w))
      for (int64_t e = u_row_ptr[row] + lane; e < u_row_ptr[row + 1]; e += 32) {
        const uint32_t v = u_kpns[e];
        c += in_window(D.eps[size_t(unpack_kp(v)) * nb + unpack_n(v)], w);
      }
  } else {
    const int64_t r = row - nst;
    for (int64_t e = u_ph_row_ptr[r] + lane; e < u_ph_row_ptr[r + 1]; e += 32) {
      const uint32_t v = u_ph_kpn[e];
      c += in_window(state_energy(D, nb, u_ph_st[e]), w) && in_window(D.eps[size_t(unpack_kp(v)) * nb + unpack_n(v)], w);
    }
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) {
    if (row < nst) cnt_e[row] = c;
    else cnt_ph[row - nst] = c;
  }
}

__global__ void k_inst_fill(ModelDev M, MeshDev D, InstWindow w, const double *__restrict__ fk,
                            const double *__restrict__ nbq, const int64_t *__restrict__ u_row_ptr,
                            const uint32_t *__restrict__ u_kpns, const double2 *__restrict__ u_X,
                            const int64_t *__restrict__ u_ph_row_ptr, const int *__restrict__ u_ph_st,
                            const uint32_t *__restrict__ u_ph_kpn, const double *__restrict__ u_ph_V,
                            const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ ph_row_ptr,
                            uint32_t *e_kpns, double2 *e_X, int *ph_st, uint32_t *ph_kpn, double *ph_Y) {
  const int64_t row = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nb = M.nb, nbr = M.nbr;
  const int64_t nst = D.n_ibzw * nb, nph = D.nq * nbr;
  if (row >= nst + nph) return;
  const unsigned below = (1u << lane) - 1u;
  if (row < nst) {
    const int k = D.ibzw_list[row / nb], m = int(row % nb);
    if (!in_window(D.eps[size_t(k) * nb + m], w)) return;
    const double fm = fk[size_t(k) * nb + m];
    int64_t pos = row_ptr[row];
    const int64_t e1 = u_row_ptr[row + 1];
    for (int64_t b = u_row_ptr[row]; b < e1; b += 32) {
      const int64_t e = b + lane;
      uint32_t v = 0;
      bool keep = false;
      if (e < e1) {
        v = u_kpns[e];
        keep = in_window(D.eps[size_t(unpack_kp(v)) * nb + unpack_n(v)], w);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int kp = unpack_kp(v), n = unpack_n(v), s = unpack_s(v);
        const double occ = fm * (1.0 - fk[size_t(kp) * nb + n]);
        const double nq = nbq[size_t(q_of(D, k, kp)) * nbr + s];
        const double2 V = u_X[e];
        const int64_t o = pos + __popc(bal & below);
        e_kpns[o] = v;
        e_X[o] = make_double2(V.x * occ * nq, V.y * occ * (1.0 + nq));
      }
      pos += __popc(bal);
    }
  } else {
    const int64_t r = row - nst;
    const double nq = nbq[r];   // row r = q * nbr + s
    int64_t pos = ph_row_ptr[r];
    const int64_t e1 = u_ph_row_ptr[r + 1];
    for (int64_t b = u_ph_row_ptr[r]; b < e1; b += 32) {
      const int64_t e = b + lane;
      uint32_t v = 0;
      int st = 0;
      bool keep = false;
      if (e < e1) {
        v = u_ph_kpn[e];
        st = u_ph_st[e];
        keep = in_window(state_energy(D, nb, st), w) && in_window(D.eps[size_t(unpack_kp(v)) * nb + unpack_n(v)], w);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int k = D.ibzw_list[st / nb], m = st % nb;
        const double occ = fk[size_t(k) * nb + m] * (1.0 - fk[size_t(unpack_kp(v)) * nb + unpack_n(v)]);
        const int64_t o = pos + __popc(bal & below);
        ph_st[o] = st;
        ph_kpn[o] = v;
        ph_Y[o] = u_ph_V[e] * occ * nq;
      }
      pos += __popc(bal);
    }
  }
}

}  // namespace

cudaError_t launch_inst_count(const ModelDev &M, const MeshDev &D, InstWindow w, const int64_t *u_row_ptr,
                              const uint32_t *u_kpns, const int64_t *u_ph_row_ptr, const int *u_ph_st,
                              const uint32_t *u_ph_kpn, int *cnt_e, int *cnt_ph, cudaStream_t st) {
  const int64_t rows = D.n_ibzw * M.nb + D.nq * M.nbr;
  if (rows == 0) return cudaSuccess;
  EPHB_LAUNCH(k_inst_count, unsigned((rows * 32 + 255) / 256), 256, 0, st, M, D, w, u_row_ptr, u_kpns, u_ph_row_ptr,
              u_ph_st, u_ph_kpn, cnt_e, cnt_ph);
  return cudaGetLastError();
}

cudaError_t launch_inst_fill(const ModelDev &M, const MeshDev &D, InstWindow w, const double *fk, const double *nbq,
                             const int64_t *u_row_ptr, const uint32_t *u_kpns, const double2 *u_X,
                             const int64_t *u_ph_row_ptr, const int *u_ph_st, const uint32_t *u_ph_kpn,
                             const double *u_ph_V, const int64_t *row_ptr, const int64_t *ph_row_ptr,
                             uint32_t *e_kpns, double2 *e_X, int *ph_st, uint32_t *ph_kpn, double *ph_Y,
                             cudaStream_t st) {
  const int64_t rows = D.n_ibzw * M.nb + D.nq * M.nbr;
  if (rows == 0) return cudaSuccess;
  EPHB_LAUNCH(k_inst_fill, unsigned((rows * 32 + 255) / 256), 256, 0, st, M, D, w, fk, nbq, u_row_ptr, u_kpns, u_X,
              u_ph_row_ptr, u_ph_st, u_ph_kpn, u_ph_V, row_ptr, ph_row_ptr, e_kpns, e_X, ph_st, ph_kpn, ph_Y);
  return cudaGetLastError();
}

}  // namespace ephb
