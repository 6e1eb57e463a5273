// Complex-Hermitian eigen-decomposition by the cyclic Jacobi method with one WARP per matrix
// (n <= NMAX <= 12, FP64), for H(k) and D(q).
//
// The one-thread-per-matrix form spends its time in the dependency chain of one thread (a
// few warps per SM, each instruction waiting on the previous one).  Here a warp shares the
// work of every rotation round: in the parallel ("round-robin") ordering the index pairs of
// a round are disjoint, so their rotations commute and are applied together.  Round r of a
// sweep pairs position i with position m-1-i (m = n rounded up to even), the positions of
// indices 1..m-1 shifted by r (the circle method), so a sweep of m-1 rounds visits every
// pair once.  Each rotation is the serial form's: J = D R D^dagger with the phase D making
// a_pq real and the real rotation R (t = tan of its angle, the smaller root of
// t^2 + 2 t theta = 1, theta = (a_qq - a_pp) / (2 |a_pq|)); the 2 x 2 block of a pair takes
// its closed form diag(a_pp - t |a_pq|, a_qq + t |a_pq|), the other elements
// A' = J^dagger A J with A' kept Hermitian (the upper triangle computed, the lower mirrored).
#pragma once
#include "common.cuh"

namespace ephb {

template <int NMAX>
struct JacobiWarpSmem {
  double2 A[NMAX * NMAX];
  double2 V[NMAX * NMAX];
  double2 sph[NMAX / 2 + 1];   // s e^{i phi} of each pair of the round
  double c[NMAX / 2 + 1];
  double dp[NMAX / 2 + 1], dq[NMAX / 2 + 1];   // new diagonal values of the pair
  double e[NMAX];
  int pp[NMAX / 2 + 1], pq[NMAX / 2 + 1];
  int pair_of[NMAX];           // pair of each index in this round, -1 if it sits out
  int perm[NMAX];              // ascending order of the eigenvalues
  double red[32];
};

__device__ inline double jw_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Row coefficient conj(J_{a x}) and column coefficient J_{b x} of index x in pair k: the two
// indices a (b) of x's pair with their coefficients; an index outside every pair has J = 1.
__device__ inline void jw_coef(int x, int k, const int *pp, const int *pq, const double *c, const double2 *sph,
                               bool row, int *idx, double2 *cf) {
  if (k < 0) {
    idx[0] = x;
    cf[0] = cmk(1.0, 0.0);
    idx[1] = -1;
    cf[1] = cmk(0.0, 0.0);
    return;
  }
  const int p = pp[k], q = pq[k];
  const double2 s = sph[k];
  idx[0] = p;
  idx[1] = q;
  // J_pp = c, J_qp = -conj(s), J_pq = s, J_qq = c
  if (x == p) {
    cf[0] = cmk(c[k], 0.0);
    cf[1] = row ? cmk(-s.x, -s.y) : cmk(-s.x, s.y);   // conj(J_qp) = -s ; J_qp = -conj(s)
  } else {
    cf[0] = row ? cconj(s) : s;                        // conj(J_pq) = conj(s) ; J_pq = s
    cf[1] = cmk(c[k], 0.0);
  }
}

// The warp's matrix is in S.A (leading n x n block, Hermitian; destroyed).  On return S.e[i]
// holds the eigenvalues ascending, S.perm[i] the column of S.V holding the eigenvector of
// S.e[i] (S.V is not permuted).  All 32 lanes of the warp call it.
template <int NMAX>
__device__ void herm_jacobi_warp(JacobiWarpSmem<NMAX> &S, int n) {
  const int lane = threadIdx.x & 31;
  const int nn = n * n, nup = n * (n + 1) / 2;
  for (int t = lane; t < nn; t += 32) S.V[(t / n) * NMAX + t % n] = cmk(t / n == t % n ? 1.0 : 0.0, 0.0);
  double loc = 0.0;
  for (int t = lane; t < nn; t += 32) loc += cabs2(S.A[(t / n) * NMAX + t % n]);
  const double norm2 = jw_warp_sum(loc);
  const int m = n + (n & 1), npair = m / 2;
  __syncwarp();
  for (int sweep = 0; sweep < 60; ++sweep) {
    loc = 0.0;
    for (int t = lane; t < nn; t += 32) {
      const int r = t / n, s = t % n;
      if (r < s) loc += cabs2(S.A[r * NMAX + s]);
    }
    const double off = jw_warp_sum(loc);
    if (off <= 1e-36 * norm2) break;
    for (int round = 0; round < m - 1; ++round) {
      if (lane < npair) {
        const int i = lane;
        const int a = i == 0 ? 0 : 1 + (i - 1 + round) % (m - 1);
        const int j = m - 1 - i;
        const int b = 1 + (j - 1 + round) % (m - 1);
        const int p = a < b ? a : b, q = a < b ? b : a;
        S.pp[i] = p;
        S.pq[i] = q;
        if (q < n) {
          const double2 apq = S.A[p * NMAX + q];
          const double b2 = cabs2(apq);
          const double app = S.A[p * NMAX + p].x, aqq = S.A[q * NMAX + q].x;
          if (b2 > 0.0) {
            const double ib = rsqrt(b2), bb = b2 * ib;
            const double2 ph = cscale(apq, ib);
            const double theta = (aqq - app) * 0.5 * ib;
            const double t = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double cc = rsqrt(t * t + 1.0), ss = t * cc;
            S.c[i] = cc;
            S.sph[i] = cscale(ph, ss);
            S.dp[i] = app - t * bb;
            S.dq[i] = aqq + t * bb;
          } else {
            S.c[i] = 1.0;
            S.sph[i] = cmk(0.0, 0.0);
            S.dp[i] = app;
            S.dq[i] = aqq;
          }
          S.pair_of[p] = i;
          S.pair_of[q] = i;
        } else {
          S.pair_of[p] = -1;   // p sits out this round (odd n)
        }
      }
      __syncwarp();
      // A' = J^dagger A J on the upper triangle, then mirrored
      constexpr int kMaxPerLane = (NMAX * (NMAX + 1) / 2 + 31) / 32;
      double2 nv[kMaxPerLane];
      int k = 0;
      for (int t = lane; t < nup; t += 32, ++k) {
        int r = 0, rem = t;
        while (rem >= n - r) {
          rem -= n - r;
          ++r;
        }
        const int s = r + rem;
        const int kr = S.pair_of[r], ks = S.pair_of[s];
        double2 v;
        if (kr >= 0 && kr == ks) {
          v = r != s ? cmk(0.0, 0.0) : cmk(r == S.pp[kr] ? S.dp[kr] : S.dq[kr], 0.0);
        } else {
          int ia[2], ib[2];
          double2 ca[2], cb[2];
          jw_coef(r, kr, S.pp, S.pq, S.c, S.sph, true, ia, ca);
          jw_coef(s, ks, S.pp, S.pq, S.c, S.sph, false, ib, cb);
          v = cmk(0.0, 0.0);
          for (int x = 0; x < 2; ++x) {
            if (ia[x] < 0) continue;
            double2 row = cmk(0.0, 0.0);
            for (int y = 0; y < 2; ++y)
              if (ib[y] >= 0) cfma(row, S.A[ia[x] * NMAX + ib[y]], cb[y]);
            cfma(v, ca[x], row);
          }
          if (r == s) v.y = 0.0;
        }
        nv[k] = v;
      }
      // V' = V J
      constexpr int kMaxVPerLane = (NMAX * NMAX + 31) / 32;
      double2 vv[kMaxVPerLane];
      k = 0;
      for (int t = lane; t < nn; t += 32, ++k) {
        const int r = t / n, s = t % n;
        int ib[2];
        double2 cb[2];
        jw_coef(s, S.pair_of[s], S.pp, S.pq, S.c, S.sph, false, ib, cb);
        double2 v = cmk(0.0, 0.0);
        for (int y = 0; y < 2; ++y)
          if (ib[y] >= 0) cfma(v, S.V[r * NMAX + ib[y]], cb[y]);
        vv[k] = v;
      }
      __syncwarp();
      k = 0;
      for (int t = lane; t < nup; t += 32, ++k) {
        int r = 0, rem = t;
        while (rem >= n - r) {
          rem -= n - r;
          ++r;
        }
        const int s = r + rem;
        S.A[r * NMAX + s] = nv[k];
        if (r != s) S.A[s * NMAX + r] = cconj(nv[k]);
      }
      k = 0;
      for (int t = lane; t < nn; t += 32, ++k) S.V[(t / n) * NMAX + t % n] = vv[k];
      __syncwarp();
    }
  }
  if (lane == 0) {
    for (int i = 0; i < n; ++i) {
      S.e[i] = S.A[i * NMAX + i].x;
      S.perm[i] = i;
    }
    for (int i = 0; i < n - 1; ++i) {   // ascending (selection sort of the order)
      int mi = i;
      for (int j = i + 1; j < n; ++j)
        if (S.e[j] < S.e[mi]) mi = j;
      if (mi != i) {
        const double te = S.e[i];
        S.e[i] = S.e[mi];
        S.e[mi] = te;
        const int tp = S.perm[i];
        S.perm[i] = S.perm[mi];
        S.perm[mi] = tp;
      }
    }
  }
  __syncwarp();
}

}  // namespace ephb
