// Small dense complex-Hermitian eigen-decomposition by the cyclic Jacobi method, one
// matrix per thread.  Used for H(k) (<= 8 bands) and D(q) (<= 12 branches) in FP64.
// Each rotation J = D R D^dagger combines a diagonal phase D = diag(1, e^{-i phi}) that
// makes a_pq real with the classic real Jacobi rotation R of the (p,q) plane (t = tan of its
// angle from theta = (a_qq - a_pp) / (2 |a_pq|), the smaller root of t^2 + 2 t theta = 1).
// Only the off-block entries are rotated; the Hermitian mirror is copied and the 2 x 2 block
// takes its closed form, which halves the FP64 work of a rotation.
#pragma once
#include "common.cuh"

namespace ephb {

// A: NMAX x NMAX row-major, Hermitian in its leading n x n block (destroyed).
// On return e[0..n) ascending and V columns the matching orthonormal eigenvectors.
template <int NMAX>
__device__ inline void herm_jacobi(double2 *A, double2 *V, double *e, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * NMAX + j] = cmk(i == j ? 1.0 : 0.0, 0.0);
  double norm2 = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) norm2 += cabs2(A[i * NMAX + j]);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += cabs2(A[p * NMAX + q]);
    if (off <= 1e-36 * norm2) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double2 apq = A[p * NMAX + q];
        const double b2 = cabs2(apq);
        if (b2 == 0.0) continue;
        const double ib = rsqrt(b2), b = b2 * ib;   // 1 / |a_pq| and |a_pq|
        const double2 ph = cscale(apq, ib);          // e^{i phi}
        const double app = A[p * NMAX + p].x, aqq = A[q * NMAX + q].x;
        const double theta = (aqq - app) * 0.5 * ib;
        const double t = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = rsqrt(t * t + 1.0), s = t * c;
        const double2 sph = cscale(ph, s);          // s e^{i phi}
        const double2 sphc = cconj(sph);            // s e^{-i phi}
        // A <- J^dagger A J.  Columns p, q of every other row r; rows p, q are their conjugates
        // (A stays Hermitian), and the (p, q) block becomes diag(a_pp - t |a_pq|, a_qq + t |a_pq|).
        for (int r = 0; r < n; ++r) {
          if (r == p || r == q) continue;
          const double2 tp = A[r * NMAX + p], tq = A[r * NMAX + q];
          const double2 np = csub(cscale(tp, c), cmul(sphc, tq));
          const double2 nq = cadd(cmul(sph, tp), cscale(tq, c));
          A[r * NMAX + p] = np;
          A[r * NMAX + q] = nq;
          A[p * NMAX + r] = cconj(np);
          A[q * NMAX + r] = cconj(nq);
        }
        A[p * NMAX + p] = cmk(app - t * b, 0.0);
        A[q * NMAX + q] = cmk(aqq + t * b, 0.0);
        A[p * NMAX + q] = cmk(0.0, 0.0);
        A[q * NMAX + p] = cmk(0.0, 0.0);
        // V <- V J
        for (int r = 0; r < n; ++r) {
          const double2 tp = V[r * NMAX + p], tq = V[r * NMAX + q];
          V[r * NMAX + p] = csub(cscale(tp, c), cmul(sphc, tq));
          V[r * NMAX + q] = cadd(cmul(sph, tp), cscale(tq, c));
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) e[i] = A[i * NMAX + i].x;
  // ascending order (selection sort, columns follow)
  for (int i = 0; i < n - 1; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (e[j] < e[m]) m = j;
    if (m != i) {
      double te = e[i];
      e[i] = e[m];
      e[m] = te;
      for (int r = 0; r < n; ++r) {
        double2 tv = V[r * NMAX + i];
        V[r * NMAX + i] = V[r * NMAX + m];
        V[r * NMAX + m] = tv;
      }
    }
  }
}

// Degenerate groups of ascending values: chains of neighbours closer than tol.
// grp[2*i] = first index of i's group, grp[2*i+1] = one past its last index.
__host__ __device__ inline void degenerate_groups(const double *e, int n, double tol, uint8_t *grp) {
  int start = 0;
  for (int i = 1; i <= n; ++i) {
    if (i == n || e[i] - e[i - 1] >= tol) {
      for (int j = start; j < i; ++j) {
        grp[2 * j] = uint8_t(start);
        grp[2 * j + 1] = uint8_t(i);
      }
      start = i;
    }
  }
}

}  // namespace ephb
