// Shared device helpers of the CUDA path: complex arithmetic on double2, physical
// constants, mesh index arithmetic and the plain-old-data views the kernels receive.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ephb {

// Process-wide count of kernels launched by the library (defined in api.cu).
void note_launches(int n);

}  // namespace ephb

// Every kernel launch of the library goes through this macro so that launches are counted.
#define EPHB_LAUNCH(kernel, grid, block, smem, stream, ...) \
  (::ephb::note_launches(1), kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__))

namespace ephb {

// Physical constants (CODATA 2018 / SI 2019), eV, K, s, C.
constexpr double kHbarEVs = 6.582119569e-16;
constexpr double kKbEVK = 8.617333262e-5;
constexpr double kECharge = 1.602176634e-19;
constexpr double kAngstrom = 1.0e-10;
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxBands = 8;       // electron Wannier bands
constexpr int kMaxBranches = 12;   // phonon branches (4 atoms)
constexpr int kMaxSym = 48;

// entry packing of the electron-side rate list: k' (21 bits) | n (4 bits) | s (6 bits)
constexpr int kKpBits = 21;
constexpr uint32_t kKpMask = (1u << kKpBits) - 1u;
__host__ __device__ inline uint32_t pack_kpns(int kp, int n, int s) {
  return uint32_t(kp) | (uint32_t(n) << kKpBits) | (uint32_t(s) << (kKpBits + 4));
}
__host__ __device__ inline int unpack_kp(uint32_t v) { return int(v & kKpMask); }
__host__ __device__ inline int unpack_n(uint32_t v) { return int((v >> kKpBits) & 15u); }
__host__ __device__ inline int unpack_s(uint32_t v) { return int(v >> (kKpBits + 4)); }

// complex helpers ------------------------------------------------------------------------
__host__ __device__ inline double2 cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cconj(double2 a) { return cmk(a.x, -a.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return cmk(a.x * s, a.y * s); }
// acc += a * b
__host__ __device__ inline void cfma(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__host__ __device__ inline void cfma_conj(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Float-float arithmetic: a value carried as hi + lo in two FP32 numbers (~48 significant
// bits).  TwoSum (Knuth) gives the exact rounding error of a sum in 6 operations; the FMA
// gives the exact error of a product.  The compensated accumulator below adds products the
// way the compensated dot product of Ogita, Rump and Oishi does: the leading parts through
// TwoSum, every error term into a second FP32 sum.  Used where the FP64 rate (1/64 of FP32
// on this part) would bound a kernel and 2^-47 relative accuracy suffices.  The explicit
// _rn intrinsics keep the compiler from contracting the sums into FMAs.
__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
struct FFAcc {
  float s = 0.f, e = 0.f;
};
// a += x * y for float-float x = (x.x + x.y), y = (y.x + y.y); the lo * lo term (2^-48 of the
// product) is left out
__device__ __forceinline__ void ff_acc_mul(FFAcc &a, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float err = __fmaf_rn(x.x, y.x, -p);
  err = __fmaf_rn(x.x, y.y, err);
  err = __fmaf_rn(x.y, y.x, err);
  float s, t;
  ff_two_sum(a.s, p, s, t);
  a.s = s;
  a.e = __fadd_rn(a.e, __fadd_rn(t, err));
}
__device__ __forceinline__ float2 ff_norm(const FFAcc &a) {
  float h, l;
  ff_two_sum(a.s, a.e, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ float2 ff_neg(float2 x) { return make_float2(-x.x, -x.y); }
// float-float product: the leading product exactly (FMA), the cross terms in FP32
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float h, l;
  ff_two_sum(p, e, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  float s, t;
  ff_two_sum(a.x, b.x, s, t);
  t = __fadd_rn(t, __fadd_rn(a.y, b.y));
  float h, l;
  ff_two_sum(s, t, h, l);
  return make_float2(h, l);
}
// a - b in float-float
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) {
  float s, t;
  ff_two_sum(a.x, -b.x, s, t);
  t = __fadd_rn(t, __fsub_rn(a.y, b.y));
  float h, l;
  ff_two_sum(s, t, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ double ff_to_double(const FFAcc &a) {
  const float2 n = ff_norm(a);
  return double(n.x) + double(n.y);
}
// float-float of a double (hi = nearest float, lo = nearest float of the remainder)
__device__ __forceinline__ float2 ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - double(h)));
}

// mesh helpers -----------------------------------------------------------------------------
struct Mesh {
  int n[3];
  __host__ __device__ int64_t size() const { return int64_t(n[0]) * n[1] * n[2]; }
  __host__ __device__ int flat(int i0, int i1, int i2) const { return (i0 * n[1] + i1) * n[2] + i2; }
  __host__ __device__ void unflat(int k, int &i0, int &i1, int &i2) const {
    i2 = k % n[2];
    int t = k / n[2];
    i1 = t % n[1];
    i0 = t / n[1];
  }
};

// a mod n in [0, n), 32-bit: every argument is a small mesh-index expression (mesh sizes
// below 1024, lattice-vector components below 2^16, checked when the model is set)
__host__ __device__ inline int pmod(int a, int n) {
  const int r = a % n;
  return r < 0 ? r + n : r;
}

// exp(i 2 pi sum_d i_d R_d / n_d) from per-dimension tables tab[off_d + j] = exp(i 2 pi j / n_d)
__device__ inline double2 mesh_phase(const double2 *__restrict__ tab, const Mesh &m, int i0, int i1, int i2,
                                     int r0, int r1, int r2) {
  double2 p0 = tab[pmod(i0 * r0, m.n[0])];
  double2 p1 = tab[m.n[0] + pmod(i1 * r1, m.n[1])];
  double2 p2 = tab[m.n[0] + m.n[1] + pmod(i2 * r2, m.n[2])];
  return cmul(cmul(p0, p1), p2);
}

}  // namespace ephb
