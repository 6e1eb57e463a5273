// Tensor-core (tcgen05) form of the R_ph contraction of the vertex (Eq. g^smn_kq):
//   B[p][m n' a] = sum_Rp e^{i q_p.Rp} A_k[Rp][m n' a]
// written as a real GEMM C'[p][j'] = sum_r Phi'[p][r] B'[r][j'] with
//   Phi'[p][r] = (cos, sin)(2 pi q_p.Rp_r) for r < R and R <= r < 2R,
//   B'(Re columns) = (Re A; -Im A),  B'(Im columns) = (Im A; Re A).
//
// Exact fixed-point slicing.  Every operand x in [-1, 1] (the phases as they are, each B'
// column divided by a power of two sigma_j >= its largest entry) is rounded to a multiple of
// 2^(-7-8(ns-1)) and split as
//   x = sum_i s_i,  s_i = n_i 2^(-7-8(i-1)),  |n_i| <= 128,
// so each slice is an exact BF16 number.  A product of two slices is an integer multiple of
// 2^(-14-8(i+l-2)) below 2^(-8(i+l-2)) in size, and a K = 256 sum of such products (or the
// two products of the second diagonal, or the four of the fourth as long as K <= 256) fits
// the 24-bit FP32 significand: the tensor core computes those diagonals exactly.  FP64-grade
// mode: 7 slices (inputs to 2^-55 of the column scale, which the Fourier sums need because
// they cancel: a result 1e-3 of its column scale keeps ~1e-13 relative accuracy), the 28
// products with i + l <= 8, accumulators (i+l = 2), (3), (4), (5) -- each summed exactly --
// and (i+l >= 6), which rounds at 2^-24 of a sum below 2^-30 of the column scale.  (With
// the fourth diagonal in the tail, its rounding, ~2^-42 of the column scale, reached 1.2e-10
// relative on the smallest rates; with the third there too, 1e-8.)  Mixed mode: 4 slices, the
// 10 products with i + l <= 5, accumulators (i+l = 2) (exact) and (i+l >= 3).
// Wide-K FP64-grade mode (contraction lengths 256 < K <= 816, e.g. 7^3 R grids): 8 slices of
// balanced base-128 digits (|n_i| <= 64, s_i = n_i 2^(-6-7(i-1)), the same 2^-55 input
// resolution), the 36 products with i + l <= 9, accumulators (i+l = 2) .. (6) -- a diagonal of
// d - 1 products of magnitude <= 2^12 units stays below 2^24 units for (d - 1) K <= 4096,
// i.e. K <= 819 for the fifth -- and (i+l >= 7).
//
// The GEMM runs on 5th-generation tensor cores: operands in shared memory in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix), accumulators in
// tensor memory, one thread issuing tcgen05.mma, completion through tcgen05.commit on an
// mbarrier, results read back with tcgen05.ld.  All waits are bounded; on expiry the CTA
// records an error code, still waits (bounded) for its MMAs, frees its tensor memory and
// returns.
#include <cuda_bf16.h>

#include <vector>

#include "internal.h"

namespace ephb {

namespace {

constexpr int kTcM = 128;        // pairs per tile (tensor-memory lanes)
constexpr int kTcKc = 32;        // K per shared-memory stage (2 MMA K-steps of 16)
constexpr int kTcThreads = 128;  // 4 warps: one per tensor-memory lane quadrant
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s bound on any wait

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Digit width of the slicing: 8 bits (base 256) for 3 and 7 slices, 7 bits (base 128) for the
// 8-slice wide-K form.  Slice i (0-based) of a value is n_i 2^-(B-1+B i), |n_i| <= 2^(B-1).
__host__ __device__ constexpr int digit_bits(int ns) { return ns == 8 ? 7 : 8; }
__host__ __device__ constexpr int slice_top(int ns) { return (digit_bits(ns) - 1) + digit_bits(ns) * (ns - 1); }

// the ns slices of the integer N = rint(x 2^slice_top): balanced base-2^B digits cut from the
// bottom (each in [-2^(B-1), 2^(B-1) - 1], the top one within [-2^(B-1), 2^(B-1)]); digit i
// becomes the BF16 number n_i 2^(-(B-1)-B i), which is exact
__device__ inline void int_slices(long long N, int ns, __nv_bfloat16 *out, size_t stride) {
  const int B = digit_bits(ns);
  const long long half = 1ll << (B - 1), mask = (1ll << B) - 1;
  for (int i = ns - 1; i >= 1; --i) {
    const long long d = ((N + half) & mask) - half;   // balanced digit, N - d divisible by 2^B
    N = (N - d) >> B;
    out[i * stride] = __float2bfloat16_rn(ldexpf(float(d), -(B - 1) - B * i));
  }
  out[0] = __float2bfloat16_rn(ldexpf(float(N), -(B - 1)));
}

// ns slices of 8 fixed-point integers into ns 16-byte vectors (8 BF16 each)
__device__ inline void int_slices8(const long long *N, int ns, uint4 *out) {
  __nv_bfloat16 v[8][8];
  for (int e = 0; e < 8; ++e) int_slices(N[e], ns, &v[e][0], 1);
  for (int sl = 0; sl < ns; ++sl) {
    __nv_bfloat16 w[8];
    for (int e = 0; e < 8; ++e) w[e] = v[e][sl];
    out[sl] = *reinterpret_cast<const uint4 *>(w);
  }
}

// Split x in [-1,1] into ns exact BF16 fixed-point slices: x is rounded once to the 64-bit
// integer N = rint(x 2^slice_top(ns)) (2^55 in every FP64-grade form); the rest is integer.
__device__ inline void fixed_slices(double x, int ns, __nv_bfloat16 *out, size_t stride) {
  int_slices(__double2ll_rn(ldexp(x, slice_top(ns))), ns, out, stride);
}

// rint(x 2^p) (ties to even) from the bits of x, by integer operations only; the same value
// as the FP64 scaling and conversion for every |x 2^p| < 2^62 (p <= 9 above the exponent of
// x's leading bit keeps the shift in range).  Zero and subnormal x give 0.
__device__ inline long long fixed_round(double x, int p) {
  const unsigned long long b = __double_as_longlong(x);
  const int e = int((b >> 52) & 0x7ff);
  if (e == 0) return 0;
  const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
  const int sh = e - 1075 + p;   // x 2^p = m 2^sh
  unsigned long long n;
  if (sh >= 0) {
    n = m << sh;
  } else if (sh < -53) {
    n = 0;                       // below 1/2
  } else {
    const int r = -sh;
    const unsigned long long q = m >> r, rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
    n = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  }
  return (b >> 63) ? -(long long)n : (long long)n;
}

// Phase slices of every q of the phonon mesh: PhiS[q][slice][Kp] (BF16)
__global__ void k_phase_slices(ModelDev M, MeshDev D, int ns, int Kp, __nv_bfloat16 *phis) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int R = M.nRgp;
  if (t >= D.nq * int64_t(Kp)) return;
  const int q = int(t / Kp), r = int(t % Kp);
  double x = 0.0;
  if (r < 2 * R) {
    const int rr = r < R ? r : r - R;
    int b0, b1, b2;
    D.qm.unflat(q, b0, b1, b2);
    const int *Rv = M.Rgp + 3 * rr;
    const double2 ph = mesh_phase(D.qtab, D.qm, b0, b1, b2, Rv[0], Rv[1], Rv[2]);
    x = r < R ? ph.x : ph.y;
  }
  fixed_slices(x, ns, phis + (size_t(q) * ns) * Kp + r, size_t(Kp));
}

// On an n x n x n mesh every phase 2 pi q.R is 2 pi j / n with j = (q.R) mod n: the slices of
// cos and sin of the n angles once (table [j][cos, sin][slice]), then every phase slice is a
// lookup.  The angles' cosines and sines are FP64 library values of 2 pi j / n.
// tab[2 j + part][8]: the ns slices of cos (part 0) or sin (part 1) of 2 pi j / n, padded to 8
// BF16 (16 bytes) per entry so that one vector load fetches them
__global__ void k_phase_angle_table(int n, int ns, __nv_bfloat16 *tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * n) return;
  const int j = t >> 1, part = t & 1;
  double sv, cv;
  sincospi(2.0 * double(j) / double(n), &sv, &cv);
  for (int sl = ns; sl < 8; ++sl) tab[size_t(t) * 8 + sl] = __float2bfloat16_rn(0.f);
  fixed_slices(part == 0 ? cv : sv, ns, tab + size_t(t) * 8, 1);
}

__global__ void k_phase_slices_cubic(ModelDev M, MeshDev D, int ns, int Kp, const __nv_bfloat16 *__restrict__ tab,
                                     __nv_bfloat16 *phis) {
  // one thread per (q, 8 consecutive r): 16-byte stores of each slice
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int R = M.nRgp, n = D.qm.n[0], n8 = Kp / 8;
  if (t >= D.nq * int64_t(n8)) return;
  const int q = int(t / n8), r0 = int(t % n8) * 8;
  int b0, b1, b2;
  D.qm.unflat(q, b0, b1, b2);
  // the 8 slices of each of the 8 elements with one 16-byte load, then transposed to 8
  // elements of each slice
  __nv_bfloat16 in[8][8], v[8][8];
  for (int e = 0; e < 8; ++e) {
    const int r = r0 + e;
    uint4 x = make_uint4(0u, 0u, 0u, 0u);
    if (r < 2 * R) {
      const int rr = r < R ? r : r - R;
      const int *Rv = M.Rgp + 3 * rr;
      const int j = pmod(b0 * Rv[0] + b1 * Rv[1] + b2 * Rv[2], n);
      x = *reinterpret_cast<const uint4 *>(tab + (size_t(j) * 2 + (r < R ? 0 : 1)) * 8);
    }
    *reinterpret_cast<uint4 *>(in[e]) = x;
  }
  for (int sl = 0; sl < 8; ++sl)
    for (int e = 0; e < 8; ++e) v[sl][e] = in[e][sl];
  __nv_bfloat16 *dst = phis + (size_t(q) * ns) * Kp + r0;
  for (int sl = 0; sl < ns; ++sl) *reinterpret_cast<uint4 *>(dst + sl * size_t(Kp)) = *reinterpret_cast<const uint4 *>(v[sl]);
}

// B' slices of the k points of a chunk: BS[kc][slice][Nmax][Kp] (BF16) and column scales.
// Column j' = ml*(2 nb nbr) + part*(nb nbr) + n'*nbr + a.  One block per (k, ml, column group):
// the stage-A rows of that initial band for the group's (n', a) range (R x h complex values,
// both parts) are read once, coalesced, into shared memory; each column gets the power of two
// sigma >= its largest magnitude; the slices are written with consecutive threads on
// consecutive r.  Integer arithmetic only (the scale, the rounding to 2^-55 of sigma and the
// digits): no FP64 operation.  Blocks y = nb (group 0) write the zero padding columns past
// 2 nb nb nbr.
__global__ void __launch_bounds__(256) k_b_slices(ModelDev M, MeshDev D, int64_t i0, const double2 *A, int ns,
                                                  int Kp, int Nmax, int ngrp, __nv_bfloat16 *bs, double *bscale) {
  extern __shared__ double2 tileA[];            // [R][h]
  __shared__ int sh_ex[2 * kMaxBands * kMaxBranches];   // exponent of sigma per local column (-2000: zero column)
  const int64_t kc = blockIdx.x;
  const int ml = blockIdx.y, grp = blockIdx.z;
  const int nb = M.nb, nbr = M.nbr, R = M.nRgp;
  const int nbnbr = nb * nbr, jmax = nb * nb * nbr;
  const int h = (nbnbr + ngrp - 1) / ngrp;                     // (n', a) values per group
  const int r0 = grp * h;
  const int hg = nbnbr - r0 < h ? nbnbr - r0 : h;              // this group's share
  const size_t sstride = size_t(Nmax) * Kp;
  __nv_bfloat16 *dstk = bs + size_t(kc) * ns * Nmax * Kp;
  if (ml >= nb) {   // zero padding columns, scale 1 (group 0 only)
    if (grp != 0) return;
    const int c0 = 2 * nb * nbnbr, ncol = Nmax - c0;
    for (int t = threadIdx.x; t < ncol * Kp; t += blockDim.x) {
      const int c = t / Kp, r = t - c * Kp;
      for (int sl = 0; sl < ns; ++sl) dstk[sl * sstride + size_t(c0 + c) * Kp + r] = __float2bfloat16_rn(0.f);
    }
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) bscale[kc * Nmax + c0 + c] = 1.0;
    return;
  }
  if (hg <= 0) return;
  const int k = D.ibzw_list[i0 + kc];
  const bool live = ml < __popc(D.rmask[k]);
  const int ncol = 2 * hg;
  // local column lc: part = lc / hg, (n', a) index rest = r0 + lc % hg; global column c0 + gcol(lc)
  const int c0 = ml * 2 * nbnbr;
  auto gcol = [&](int lc) { return lc < hg ? r0 + lc : nbnbr + r0 + (lc - hg); };
  if (!live) {   // zero slices, scale 1
    for (int t = threadIdx.x; t < ncol * Kp; t += blockDim.x) {
      const int lc = t / Kp, r = t - lc * Kp;
      for (int sl = 0; sl < ns; ++sl)
        dstk[sl * sstride + size_t(c0 + gcol(lc)) * Kp + r] = __float2bfloat16_rn(0.f);
    }
    for (int lc = threadIdx.x; lc < ncol; lc += blockDim.x) bscale[kc * Nmax + c0 + gcol(lc)] = 1.0;
    return;
  }
  const double2 *Ak = A + size_t(kc) * R * jmax + size_t(ml) * nbnbr + r0;
  for (int t = threadIdx.x; t < R * hg; t += blockDim.x) {
    const int r = t / hg, j = t - r * hg;
    tileA[t] = Ak[size_t(r) * jmax + j];
  }
  __syncthreads();
  // local column lc; row r < R: (Re, Im)[part] of A[r]; r >= R: (-Im, Re)[part]
  auto value_bits = [&](int lc, int r) -> unsigned long long {
    const int part = lc >= hg, rest = lc - part * hg;
    const double2 a = tileA[(r < R ? r : r - R) * hg + rest];
    const double v = r < R ? (part == 0 ? a.x : a.y) : (part == 0 ? -a.y : a.x);
    return (unsigned long long)__double_as_longlong(v);
  };
  for (int lc = threadIdx.x; lc < ncol; lc += blockDim.x) {
    unsigned long long mx = 0;   // largest |v| as bits (the order of non-negative doubles)
    for (int r = 0; r < 2 * R; ++r) {
      const unsigned long long ab = value_bits(lc, r) & 0x7fffffffffffffffull;
      mx = ab > mx ? ab : mx;
    }
    const int e = int(mx >> 52);
    // sigma = 2^ex with ex = e - 1022 (2^ex >= mx, as frexp gives); a zero (or subnormal) column: 1
    const int ex = e == 0 ? 0 : e - 1022;
    sh_ex[lc] = e == 0 ? -2000 : ex;
    bscale[kc * Nmax + c0 + gcol(lc)] = __longlong_as_double((long long)(ex + 1023) << 52);
  }
  __syncthreads();
  // one thread per (column, 8 consecutive r): 16-byte stores of each slice
  const int top = slice_top(ns), n8 = Kp / 8;
  for (int t = threadIdx.x; t < ncol * n8; t += blockDim.x) {
    const int lc = t / n8, r0 = (t - lc * n8) * 8;
    long long N[8];
    for (int e = 0; e < 8; ++e) {
      const int r = r0 + e;
      N[e] = r < 2 * R && sh_ex[lc] != -2000 ? fixed_round(__longlong_as_double(value_bits(lc, r)), top - sh_ex[lc])
                                             : 0;
    }
    uint4 o[8];
    int_slices8(N, ns, o);
    __nv_bfloat16 *dst = dstk + size_t(c0 + gcol(lc)) * Kp + r0;
    for (int sl = 0; sl < ns; ++sl) *reinterpret_cast<uint4 *>(dst + sl * sstride) = o[sl];
  }
}

// column groups of k_b_slices: the fewest whose shared-memory tile stays within 96 KB
static int b_slices_groups(const ModelDev &M) {
  const int nbnbr = M.nb * M.nbr;
  for (int g = 1; g < nbnbr; ++g) {
    const int h = (nbnbr + g - 1) / g;
    if (size_t(M.nRgp) * h * sizeof(double2) <= 96 * 1024) return g;
  }
  return nbnbr;
}
static size_t b_slices_smem(const ModelDev &M) {
  const int g = b_slices_groups(M), nbnbr = M.nb * M.nbr;
  return size_t(M.nRgp) * ((nbnbr + g - 1) / g) * sizeof(double2);
}

// ---- stage-A operands, pre-tiled ---------------------------------------------------------
// Both operands of the stage-A contraction are stored in HBM in the order the pipeline
// consumes them: for each (tile of rows, K block of 16) the NS slices' [rows x 16] K-major
// core-matrix tiles (8 rows x 16 bytes per core matrix, the two K halves of a row group
// 128 bytes apart, row groups 256 bytes apart) lie back to back.  One pipeline stage of one
// operand is then one contiguous block, moved by a single bulk copy.  Row tiles: 128 columns
// of the model's g (A) and chunks of nw k points (B).

// element offset of (row, k-in-block kk) within one [rows x 16] core-matrix tile
__host__ __device__ __forceinline__ int tile16_off(int row, int kk) {
  return ((row >> 3) * 2 + (kk >> 3)) * 64 + (row & 7) * 8 + (kk & 7);
}

// Phase slices of the k points of a group as the B operand of stage A: rows k (chunks of nw,
// rows past nkc zero), (cos, sin) of 2 pi k.Re for r < nRe and nRe <= r < 2 nRe, K padded to
// Kp with zeros.  One thread per (k, 8 consecutive r).
__global__ void k_phase_slices_k(ModelDev M, MeshDev D, int64_t i0, int64_t nkc, int nrows, int nw, int ns, int Kp,
                                 __nv_bfloat16 *phik) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int R = M.nRge, n8 = Kp / 8, nkb = Kp / 16;
  if (t >= int64_t(nrows) * n8) return;
  const int k = int(t / n8), r0 = int(t % n8) * 8;
  long long N[8];
  int a0 = 0, a1 = 0, a2 = 0;
  if (k < nkc) D.km.unflat(D.ibzw_list[i0 + k], a0, a1, a2);
  for (int e = 0; e < 8; ++e) {
    const int r = r0 + e;
    N[e] = 0;
    if (k < nkc && r < 2 * R) {
      const int rr = r < R ? r : r - R;
      const int *Rv = M.Rge + 3 * rr;
      const double2 ph = mesh_phase(D.ktab, D.km, a0, a1, a2, Rv[0], Rv[1], Rv[2]);
      N[e] = fixed_round(r < R ? ph.x : ph.y, slice_top(ns));
    }
  }
  uint4 o[8];
  int_slices8(N, ns, o);
  const int kch = k / nw, row = k % nw, kb = r0 / 16;
  const size_t base = (size_t(kch) * nkb + kb) * ns;
  for (int sl = 0; sl < ns; ++sl)
    *reinterpret_cast<uint4 *>(phik + (base + sl) * (size_t(nw) * 16) + tile16_off(row, r0 % 16)) = o[sl];
}

// column j' = 2 col + part of T[k][col] = sum_Re e^{ik.Re} g[Re][col], col = (rp, m', n', alpha):
//   part 0 (real): rows r < nRe: Re g[r][col];  r >= nRe: -Im g[r-nRe][col]
//   part 1 (imag): rows r < nRe: Im g[r][col];  r >= nRe:  Re g[r-nRe][col]
__device__ __forceinline__ double g_operand(const ModelDev &M, int64_t ncol, int jp, int r) {
  const int R = M.nRge;
  const int64_t col = jp / 2;
  const double2 g = M.g_R[size_t(r < R ? r : r - R) * ncol + col];
  return r < R ? ((jp & 1) == 0 ? g.x : g.y) : ((jp & 1) == 0 ? -g.y : g.x);
}

// power-of-two scale of each g column j' (>= its largest entry; 1 for a zero column); one thread
// per column, so a warp reads 32 consecutive columns of each row of g (coalesced)
__global__ void k_g_scales(ModelDev M, int Ncols, double *gscale) {
  const int64_t jp64 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (jp64 >= Ncols) return;
  const int jp = int(jp64);
  const int64_t ncol = int64_t(M.nRgp) * M.nb * M.nb * M.nbr;
  double mx = 0.0;
  if (jp / 2 < ncol)
    for (int r = 0; r < 2 * M.nRge; ++r) mx = fmax(mx, fabs(g_operand(M, ncol, jp, r)));
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  gscale[jp] = mx > 0.0 ? ldexp(1.0, ex) : 1.0;
}

// Slices of the model's g as the A operand of stage A, pre-tiled by 128 columns: one thread per
// (column tile, K block, K half, row), 8 values each.  Columns past Ncols are zero rows.
__global__ void k_g_slices(ModelDev M, int ns, int Kp, int Ncols, int nct, const double *gscale, __nv_bfloat16 *gs) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int nkb = Kp / 16;
  if (t >= int64_t(nct) * nkb * 256) return;
  const int row = int(t & 127), half = int((t >> 7) & 1);
  const int64_t tk = t >> 8;
  const int kb = int(tk % nkb), ct = int(tk / nkb);
  const int jp = ct * kTcM + row;
  const int64_t ncol = int64_t(M.nRgp) * M.nb * M.nb * M.nbr;
  const bool live = jp < Ncols && jp / 2 < ncol;
  // rint(x 2^top / sigma) by integer operations (sigma = 2^ex, a power of two): the same integers
  // as the FP64 division, scaling and conversion, with no FP64 instruction
  const int ex = live ? int((__double_as_longlong(gscale[jp]) >> 52) & 0x7ff) - 1023 : 0;
  const int r0 = kb * 16 + half * 8;
  long long N[8];
  for (int e = 0; e < 8; ++e)
    N[e] = live && r0 + e < 2 * M.nRge ? fixed_round(g_operand(M, ncol, jp, r0 + e), slice_top(ns) - ex) : 0;
  uint4 o[8];
  int_slices8(N, ns, o);
  const size_t base = (size_t(ct) * nkb + kb) * ns;
  for (int sl = 0; sl < ns; ++sl)
    *reinterpret_cast<uint4 *>(gs + (base + sl) * (size_t(kTcM) * 16) + tile16_off(row, half * 8)) = o[sl];
}

// work items of a chunk: (k, 128-pair tile, column chunk); per k: ceil(npl/128) * nchunk(k)
// (also accumulates the issued tensor-core flops: 2 * 128 * columns * Kp per slice product)
__global__ void k_tc_items(ModelDev M, MeshDev D, int64_t i0, int64_t nkc, int nc_max, int Kp, int nprod,
                           int *nitem, unsigned long long *flops) {
  const int64_t kc = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (kc >= nkc) return;
  const int64_t i = i0 + kc;
  const int64_t npl = D.pair_ptr[i + 1] - D.pair_ptr[i];
  const int nk = round_up(2 * __popc(D.rmask[D.ibzw_list[i]]) * M.nb * M.nbr, 16);
  const int nch = (nk + nc_max - 1) / nc_max;
  const int ntile = int((npl + kTcM - 1) / kTcM);
  nitem[kc] = ntile * nch;
  atomicAdd(flops, 2ull * kTcM * (unsigned long long)nk * Kp * nprod * ntile);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: no swizzle, K-major; LBO = K-direction core-matrix stride,
// SBO = stride between 8-row groups (validated on sm_103a)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((addr & 0x3FFFFu) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
  return done != 0;
}

// wait for the completion of phase `phase` of an mbarrier; gives up after kWaitNs (the timer is
// read only once the first test has failed)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  if (mbar_try(mbar, phase)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try(mbar, phase)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

// The slice products of one K step of 16: A slice is (0-based) times B slice ls for every
// is + ls <= NS - 1, diagonal d = is + ls into accumulator min(d, NACC - 1) (NACC == 1: all into
// one), is-major.  ad0 / bd0: descriptors of slice 0 of A and B at this K step; slice i lies
// i * a16 (b16) 16-byte units further (the descriptor's address field counts 16-byte units and
// the shared window stays below 2^18 bytes, so adding to the descriptor moves the address).
// FIRST: the first K step, whose first product into each accumulator overwrites it.  Fully
// unrolled: a product costs the MMA and two 64-bit adds.
template <int NS, int NACC, bool FIRST>
__device__ __forceinline__ void slice_products(uint32_t tacc, uint32_t acc_cols, uint64_t ad0, uint64_t bd0,
                                               uint32_t a16, uint32_t b16, uint32_t idesc) {
#pragma unroll
  for (int is = 0; is < NS; ++is)
#pragma unroll
    for (int ls = 0; ls < NS - is; ++ls) {
      const int d = is + ls;
      const int acc = NACC == 1 ? 0 : (d < NACC - 1 ? d : NACC - 1);
      const bool first = FIRST && (NACC == 1 ? (is == 0 && ls == 0) :
                                   (acc < NACC - 1 ? (is == 0) : (is == 0 && ls == NACC - 1)));
      asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                   "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                   :: "r"(tacc + uint32_t(acc) * acc_cols), "l"(ad0 + uint64_t(is) * a16),
                      "l"(bd0 + uint64_t(ls) * b16), "r"(idesc), "r"(first ? 0u : 1u));
    }
}

// The same products with the A slices in tensor memory: slice is at column a_tm + 8 is (a
// 128 x 16 BF16 tile takes 8 columns of the 128 lanes).
template <int NS, int NACC, bool FIRST>
__device__ __forceinline__ void slice_products_tm(uint32_t tacc, uint32_t acc_cols, uint32_t a_tm, uint64_t bd0,
                                                  uint32_t b16, uint32_t idesc) {
#pragma unroll
  for (int is = 0; is < NS; ++is)
#pragma unroll
    for (int ls = 0; ls < NS - is; ++ls) {
      const int d = is + ls;
      const int acc = NACC == 1 ? 0 : (d < NACC - 1 ? d : NACC - 1);
      const bool first = FIRST && (NACC == 1 ? (is == 0 && ls == 0) :
                                   (acc < NACC - 1 ? (is == 0) : (is == 0 && ls == NACC - 1)));
      asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                   "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                   :: "r"(tacc + uint32_t(acc) * acc_cols), "r"(a_tm + uint32_t(8 * is)),
                      "l"(bd0 + uint64_t(ls) * b16), "r"(idesc), "r"(first ? 0u : 1u));
    }
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// core-matrix offset (bytes) of element (row, k) in a [rows x KC] K-major tile
template <int KC>
__device__ __forceinline__ uint32_t core_off(int row, int kgroup) {
  return uint32_t(((row >> 3) * (KC / 8) + kgroup) * 128 + (row & 7) * 16);
}

// 2^k as an FP32 number from the FP64 power of two 2^k (0 for 0 and below the FP32 normal
// range), by exponent arithmetic: no FP64 operation
__device__ __forceinline__ float pow2_float(double sigma) {
  const long long b = __double_as_longlong(sigma);
  const int k = int((b >> 52) & 0x7ff) - 1023;
  if (b == 0 || k < -126) return 0.f;
  return __int_as_float(k > 127 ? 0x7f800000 : (k + 127) << 23);
}

// Stage-B accumulator combination of 16 columns: the rounded tail plus the exact diagonals
// (each an exact FP32 multiple of its unit), summed by TwoSum into a float-float pair; the
// only rounding is that of the error sum, ~2^-48 of the result.  No FP64 operation: the FP64
// pipe is shared with the tensor pipe, and this runs beside the next products.
template <int NACC>
__device__ __forceinline__ void tmem_ff16(uint32_t ta, int nc, float *s, float *e) {
  for (int a = NACC - 1; a >= 0; --a) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(ta + uint32_t(a * nc)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (a == NACC - 1) {
      for (int j = 0; j < 16; ++j) {
        s[j] = __uint_as_float(v[j]);
        e[j] = 0.f;
      }
    } else {
      for (int j = 0; j < 16; ++j) {
        float t, u;
        ff_two_sum(s[j], __uint_as_float(v[j]), t, u);
        s[j] = t;
        e[j] = __fadd_rn(e[j], u);
      }
    }
  }
}

// the float-float sums s + e of 16 columns times their column scales, into C'[row][c0 + j]
__device__ __forceinline__ void store_ff16(const float *s, const float *e, const double *sc, float2 *dst, int nvalid) {
  for (int j = 0; j < 16; ++j)
    if (j < nvalid) {
      float h, l;
      ff_two_sum(s[j], e[j], h, l);
      const float f = pow2_float(sc[j]);
      dst[j] = make_float2(__fmul_rn(h, f), __fmul_rn(l, f));
    }
}

struct TcParams {
  int ns, nacc, Kp, Nmax, nc_max;   // Nmax: B rows per slice (columns of the real GEMM)
  int64_t i0, nkc, pair_base;       // stage B: first pair of the chunk
  int ncols, out_stride;            // stage A: live columns and the output row stride (float2)
  int withhold;                     // failure-path check: issue no MMA (so no barrier completes)
};

// KC: K per shared-memory stage (32: one CTA per SM; 16: two CTAs per SM share the SM's
// shared memory and tensor memory, one's epilogue overlapping the other's products).
// ST: shared-memory stages (copies run up to ST - 1 K blocks ahead of the MMAs).
template <int NS, int NACC, int KC, int ST>
__global__ void __launch_bounds__(kTcThreads, (KC == 16 && ST == 2) ? 2 : 1) k_vertex_gemm(ModelDev M, MeshDev D, TcParams P,
                                                               const int64_t *__restrict__ item_ptr,
                                                               const __nv_bfloat16 *__restrict__ phis,
                                                               const __nv_bfloat16 *__restrict__ bs,
                                                               const double *__restrict__ bscale, double *Cbuf,
                                                               int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[ST];
  __shared__ uint32_t tslot;
  __shared__ const __nv_bfloat16 *arow_s[kTcM];   // A row sources (nullptr: zero-filled row)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // once a CTA has recorded a timeout the remaining ones return without waiting in turn
  if (*reinterpret_cast<volatile int *>(err)) return;
  const int64_t item = blockIdx.x;
  int nc, n0, ncw, npt, a_row;   // a_row: this thread's A row (-1: zero-filled)
  const __nv_bfloat16 *bsk;      // B slices of this item
  const double *sc;              // column scales from n0
  double *crow;                  // this thread's output row from n0
  // which (k, 128-pair tile, column chunk)
  int64_t lo = 0, hi = P.nkc;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (item_ptr[mid] <= item) lo = mid; else hi = mid;
  }
  const int64_t kc = lo;
  const int64_t i = P.i0 + kc;
  const int k = D.ibzw_list[i];
  const int nk = round_up(2 * __popc(D.rmask[k]) * M.nb * M.nbr, 16);
  const int nch = (nk + P.nc_max - 1) / P.nc_max;
  nc = round_up((nk + nch - 1) / nch, 16);                   // balanced chunk width
  const int64_t local = item - item_ptr[kc];
  const int tile = int(local / nch), chunk = int(local % nch);
  n0 = chunk * nc;
  ncw = nk - n0 < nc ? nk - n0 : nc;                        // columns of this chunk (multiple of 16)
  const int64_t p0 = D.pair_ptr[i];
  const int64_t npl = D.pair_ptr[i + 1] - p0;
  const int64_t t0 = int64_t(tile) * kTcM;
  npt = int(npl - t0 < kTcM ? npl - t0 : kTcM);
  a_row = tid < npt ? D.pair_q[p0 + t0 + tid] : -1;
  bsk = bs + size_t(kc) * NS * P.Nmax * P.Kp;
  sc = bscale + kc * P.Nmax + n0;
  crow = Cbuf + (p0 + t0 + tid - P.pair_base) * P.Nmax + n0;
  // ST shared-memory stages, each NS x [128 x KC] (A) followed by NS x [nc_max x KC] (B)
  const size_t a_slice = size_t(kTcM) * KC * 2, b_slice = size_t(P.nc_max) * KC * 2;
  const size_t stage_bytes = size_t(NS) * (a_slice + b_slice);

  arow_s[tid] = a_row >= 0 ? phis + size_t(a_row) * NS * P.Kp : nullptr;   // read after the barrier below
  if (tid == 0) {
    for (int i = 0; i < ST; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[i])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const uint32_t ncols_alloc = NACC * nc <= 32 ? 32u : (NACC * nc <= 64 ? 64u : (NACC * nc <= 128 ? 128u :
                               (NACC * nc <= 256 ? 256u : 512u)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tslot)),
                 "r"(ncols_alloc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(ncw >> 3) << 17) | (uint32_t(kTcM >> 4) << 24);

  // asynchronous copies of the operands of K block kb into stage buf (one commit group).  A:
  // consecutive threads take consecutive 16-byte pieces of one row's slice, so a warp's
  // copies cover whole 32-byte sectors of 16 rows instead of half-sectors of 32.
  auto stage_load = [&](int buf, int kb) {
    unsigned char *sA = smem + buf * stage_bytes;
    unsigned char *sB = sA + NS * a_slice;
    constexpr int G = KC / 8;
    for (int c = tid; c < NS * kTcM * G; c += kTcThreads) {
      const int g = c % G, rs = c / G, row = rs % kTcM, s = rs / kTcM;
      const __nv_bfloat16 *src = arow_s[row];
      cp_async16(smem_u32(sA + s * a_slice + core_off<KC>(row, g)), (src ? src : phis) + size_t(s) * P.Kp + kb + g * 8,
                 src ? 16u : 0u);
    }
    for (int t = tid; t < NS * ncw * (KC / 8); t += kTcThreads) {
      const int s = t / (ncw * (KC / 8));
      const int rem = t % (ncw * (KC / 8));
      const int row = rem / (KC / 8), g = rem % (KC / 8);
      cp_async16(smem_u32(sB + s * b_slice + core_off<KC>(row, g)),
                 bsk + (size_t(s) * P.Nmax + n0 + row) * P.Kp + kb + g * 8, 16u);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  // Pipeline: the MMAs of block b are issued as soon as its operands have landed; the copies
  // of block b + ST - 1 go into the stage of block b - 1 once the MMAs of block b - 1 (its last
  // readers) have completed, so up to ST - 1 blocks of copies overlap the MMAs.
  const int nkb = P.Kp / KC;
  bool ok = true;
  int issued = -1;    // last K block whose MMAs were committed
  for (int p = 0; p < ST - 1 && p < nkb; ++p) stage_load(p, p * KC);
  for (int b = 0; b < nkb && ok; ++b) {
    const int buf = b % ST;
    // block b's copies have landed once at most min(ST - 2, nkb - 1 - b) later groups are pending
    const int later = (nkb - 1 - b) < (ST - 2) ? (nkb - 1 - b) : (ST - 2);
    if (later >= 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else if (later == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && !P.withhold) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const unsigned char *sA = smem + buf * stage_bytes;
      const unsigned char *sB = sA + NS * a_slice;
      // K-step-major order: every accumulator receives its products in the same sequence
      // whatever KC is, so the rounded tail accumulator (and the result) does not depend on
      // the tile shape
      const uint64_t ad0 = smem_desc(smem_u32(sA), 128u, (KC / 8) * 128u);
      const uint64_t bd0 = smem_desc(smem_u32(sB), 128u, (KC / 8) * 128u);
      const uint32_t a16 = uint32_t(a_slice >> 4), b16 = uint32_t(b_slice >> 4);
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {   // K step ks: 256 bytes (16 units) into each slice
        if (b == 0 && ks == 0)
          slice_products<NS, NACC, true>(taddr, uint32_t(nc), ad0, bd0, a16, b16, idesc);
        else
          slice_products<NS, NACC, false>(taddr, uint32_t(nc), ad0 + 16u * ks, bd0 + 16u * ks, a16, b16, idesc);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mbar[buf])) : "memory");
    }
    issued = b;
    const int nb = b + ST - 1;   // next block to copy, into the stage of block b - 1
    if (nb < nkb) {
      if (b >= 1) {
        // use (b - 1) / ST of that stage's barrier; the block agrees on the outcome, so a
        // timeout leaves the loop on every thread together
        const bool waited = mbar_wait(smem_u32(&mbar[(b - 1) % ST]), uint32_t(((b - 1) / ST) & 1));
        ok = __syncthreads_and(waited ? 1 : 0) != 0;
      }
      if (ok) stage_load(nb % ST, nb * KC);
    }
  }
  // no copy may still be in flight when the CTA leaves (after a timeout some can be)
  asm volatile("cp.async.wait_all;" ::: "memory");
  // the last commit tracks every MMA issued before it (after a timeout: the bounded second wait)
  {
    const bool waited = mbar_wait(smem_u32(&mbar[issued % ST]), uint32_t((issued / ST) & 1));
    if (!__syncthreads_and(waited ? 1 : 0)) ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    // accumulators -> float-float pairs -> C'[row][n0 + j]
    const int row = warp * 32 + lane;
    float2 *frow = reinterpret_cast<float2 *>(Cbuf) + (crow - Cbuf);
    for (int c0 = 0; c0 < ncw; c0 += 16) {
      float sm[16], er[16];
      tmem_ff16<NACC>(taddr + (uint32_t(warp * 32) << 16) + uint32_t(c0), nc, sm, er);
      if (row < npt) store_ff16(sm, er, sc + c0, frow + c0, ncw - c0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols_alloc));
}

// ---- warp-specialised persistent form (stage B rows: (k,q) pairs) ------------------------
// One CTA per SM walks the work items blockIdx.x, blockIdx.x + gridDim.x, ...  Roles:
//   warps 0-3  epilogue: tensor-memory lane quadrant w, int64 combination, FP64 stores;
//   warp 4     tensor-memory allocation; lane 0 issues every tcgen05.mma and commit;
//   warps 5-8  copies: cp.async of the A and B slices of K blocks of 16 into ST stages.
// Barriers: full[s] (128 copy threads arrive once their copies of stage s have landed),
// empty[s] (the MMA commit after the products that read stage s), accf[b] (the commit after
// an item's last products into accumulator buffer b), acce[b] (128 epilogue threads arrive
// once buffer b is read).  Two accumulator buffers of NACC x nc_max columns let the epilogue
// of one item run under the products of the next; ST - 2 stages of copies run ahead of the
// products.  Every wait is bounded; a timeout sets a CTA-wide abort flag and the error flag,
// each role leaves its loop, the copies and MMAs in flight are waited for (bounded) and the
// tensor memory is freed.
constexpr int kWsThreads = 288;
constexpr int kWsCopyThreads = 128;

struct WsItem {
  int nc, n0, ncw, npt;
  int64_t p0t0;   // first pair of the tile
  int kc;         // chunk-local k index
  int pad;
};
static_assert(sizeof(WsItem) == 4 * sizeof(int64_t), "work-item descriptor size");


// AND of v over the 128 epilogue threads (warps 0-3), named barrier 1
__device__ __forceinline__ bool epi_sync_and(bool v) {
  uint32_t r;
  asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.and.pred p, 1, 128, q;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(r) : "r"(v ? 1u : 0u) : "memory");
  return r != 0;
}

// descriptors of every work item of a chunk (one thread per k), so that the roles of the
// persistent kernel read one 32-byte record per item instead of searching item_ptr
__global__ void k_ws_items(ModelDev M, MeshDev D, TcParams P, const int64_t *item_ptr, WsItem *desc) {
  const int64_t kc = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (kc >= P.nkc) return;
  const int64_t i = P.i0 + kc;
  const int k = D.ibzw_list[i];
  const int nk = round_up(2 * __popc(D.rmask[k]) * M.nb * M.nbr, 16);
  const int nch = (nk + P.nc_max - 1) / P.nc_max;
  const int nc = round_up((nk + nch - 1) / nch, 16);
  const int64_t p0 = D.pair_ptr[i];
  const int64_t npl = D.pair_ptr[i + 1] - p0;
  const int64_t base = item_ptr[kc];
  const int64_t n = int64_t((npl + kTcM - 1) / kTcM) * nch;   // as counted by k_tc_items
  for (int64_t l = 0; l < n; ++l) {
    const int tile = int(l / nch), chunk = int(l % nch);
    WsItem w;
    w.kc = int(kc);
    w.nc = nc;
    w.n0 = chunk * nc;
    w.ncw = nk - w.n0 < nc ? nk - w.n0 : nc;
    const int64_t t0 = int64_t(tile) * kTcM;
    w.npt = int(npl - t0 < kTcM ? npl - t0 : kTcM);
    w.p0t0 = p0 + t0;
    w.pad = 0;
    desc[base + l] = w;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" :: "r"(mbar) : "memory");
}

template <int NS, int NACC, int ST>
__global__ void __launch_bounds__(kWsThreads, 1) k_vertex_gemm_ws(ModelDev M, MeshDev D, TcParams P, int64_t nitems,
                                                                  const WsItem *__restrict__ desc,
                                                                  const __nv_bfloat16 *__restrict__ phis,
                                                                  const __nv_bfloat16 *__restrict__ bs,
                                                                  const double *__restrict__ bscale, double *Cbuf,
                                                                  int *err) {
  constexpr int KC = 16;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[ST], empty[ST], accf[2], acce[2];
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (*reinterpret_cast<volatile int *>(err)) return;   // the whole CTA returns, before any barrier
  const size_t a_slice = size_t(kTcM) * KC * 2, b_slice = size_t(P.nc_max) * KC * 2;
  const size_t stage_bytes = size_t(NS) * (a_slice + b_slice);
  const int nkb = P.Kp / KC;
  if (tid == 0) {
    for (int i = 0; i < ST; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&full[i])), "r"(kWsCopyThreads));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[i])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&accf[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&acce[b])), "r"(kTcM));
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tslot;
  auto give_up = [&]() {
    abort_flag = 1;
    atomicExch(err, 1);
  };

  if (warp >= 5) {
    // ---------------- copies
    const int ct = tid - 5 * 32;               // 0..127
    const int g = ct & 1, r0 = ct >> 1;        // this thread's 16-byte piece and A rows r0, r0 + 64
    uint32_t it = 0;                           // K blocks issued so far (all items)
    bool ok = true;
    auto complete = [&](uint32_t j) {          // stage of block j has landed: publish it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&full[j % ST]));
    };
    // the next item's descriptor and A rows are fetched while the current item's copies go out
    WsItem w = blockIdx.x < nitems ? desc[blockIdx.x] : WsItem{};
    int q0 = r0 < w.npt ? D.pair_q[w.p0t0 + r0] : -1, q1 = r0 + 64 < w.npt ? D.pair_q[w.p0t0 + r0 + 64] : -1;
    for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const WsItem wn = item + gridDim.x < nitems ? desc[item + gridDim.x] : w;
      int q0n = -1, q1n = -1;
      const __nv_bfloat16 *src0 = q0 >= 0 ? phis + size_t(q0) * NS * P.Kp : nullptr;
      const __nv_bfloat16 *src1 = q1 >= 0 ? phis + size_t(q1) * NS * P.Kp : nullptr;
      const __nv_bfloat16 *bsk = bs + (size_t(w.kc) * NS * P.Nmax + w.n0) * P.Kp;
      const int kpre = nkb > 4 ? 4 : nkb - 1;
      for (int kb = 0; kb < nkb; ++kb) {
        if (kb == kpre && item + gridDim.x < nitems) {
          q0n = r0 < wn.npt ? D.pair_q[wn.p0t0 + r0] : -1;
          q1n = r0 + 64 < wn.npt ? D.pair_q[wn.p0t0 + r0 + 64] : -1;
        }
        const uint32_t slot = it % ST;
        if (it >= ST && !mbar_wait(smem_u32(&empty[slot]), ((it / ST) - 1) & 1)) {
          give_up();
          ok = false;
          break;
        }
        if (abort_flag) {
          ok = false;
          break;
        }
        unsigned char *sA = smem + slot * stage_bytes;
        unsigned char *sB = sA + NS * a_slice;
        const int k0 = kb * KC + g * 8;
        for (int sl = 0; sl < NS; ++sl) {
          cp_async16(smem_u32(sA + sl * a_slice + core_off<KC>(r0, g)), (src0 ? src0 : phis) + size_t(sl) * P.Kp + k0,
                     src0 ? 16u : 0u);
          cp_async16(smem_u32(sA + sl * a_slice + core_off<KC>(r0 + 64, g)),
                     (src1 ? src1 : phis) + size_t(sl) * P.Kp + k0, src1 ? 16u : 0u);
        }
        for (int rem = r0; rem < NS * w.ncw; rem += 64) {
          const int sl = rem / w.ncw, row = rem - sl * w.ncw;
          cp_async16(smem_u32(sB + sl * b_slice + core_off<KC>(row, g)),
                     bsk + (size_t(sl) * P.Nmax + row) * P.Kp + k0, 16u);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (it >= ST - 2) {                    // block it - (ST - 2) has landed once ST - 2 later groups remain
          asm volatile("cp.async.wait_group %0;" :: "n"(ST - 2) : "memory");
          complete(it - (ST - 2));
        }
        ++it;
      }
      w = wn;
      q0 = q0n;
      q1 = q1n;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (ok)
      for (uint32_t j = it >= ST - 2 ? it - (ST - 2) : 0; j < it; ++j) complete(j);
  } else if (warp == 4) {
    // ---------------- tensor-core products (one thread)
    if (lane == 0) {
      uint32_t it = 0, tcount = 0;
      uint64_t last_bar = 0;                   // barrier address + parity of the last commit
      uint32_t last_par = 0;
      bool any = false;
      WsItem wn = blockIdx.x < nitems ? desc[blockIdx.x] : WsItem{};
      for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        if (abort_flag) break;
        const WsItem w = wn;
        if (item + gridDim.x < nitems) wn = desc[item + gridDim.x];
        const uint32_t buf = tcount & 1;
        if (tcount >= 2 && !mbar_wait(smem_u32(&acce[buf]), ((tcount >> 1) - 1) & 1)) {
          give_up();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(w.ncw >> 3) << 17) |
                               (uint32_t(kTcM >> 4) << 24);
        const uint32_t tbase = taddr + buf * uint32_t(NACC * P.nc_max);
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
          const uint32_t slot = it % ST;
          if (!mbar_wait(smem_u32(&full[slot]), (it / ST) & 1) || abort_flag) {
            if (!abort_flag) give_up();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          if (!P.withhold) {
            const unsigned char *sA = smem + slot * stage_bytes;
            const unsigned char *sB = sA + NS * a_slice;
            const uint64_t ad0 = smem_desc(smem_u32(sA), 128u, (KC / 8) * 128u);
            const uint64_t bd0 = smem_desc(smem_u32(sB), 128u, (KC / 8) * 128u);
            if (kb == 0)
              slice_products<NS, NACC, true>(tbase, uint32_t(w.nc), ad0, bd0, uint32_t(a_slice >> 4),
                                             uint32_t(b_slice >> 4), idesc);
            else
              slice_products<NS, NACC, false>(tbase, uint32_t(w.nc), ad0, bd0, uint32_t(a_slice >> 4),
                                              uint32_t(b_slice >> 4), idesc);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&empty[slot])) : "memory");
            any = true;
            last_bar = smem_u32(&empty[slot]);
            last_par = (it / ST) & 1;
          }
          ++it;
        }
        if (!ok) break;
        if (!P.withhold) {
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(smem_u32(&accf[buf])) : "memory");
          last_bar = smem_u32(&accf[buf]);
          last_par = (tcount >> 1) & 1;
        }
        ++tcount;
      }
      // every MMA issued is complete before the tensor memory is freed
      if (any && !mbar_wait(uint32_t(last_bar), last_par)) give_up();
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 0-3: tensor-memory lanes 32w .. 32w + 31)
    const int row = warp * 32 + lane;
    uint32_t tcount = 0;
    WsItem wn = blockIdx.x < nitems ? desc[blockIdx.x] : WsItem{};
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
      const WsItem w = wn;
      if (item + gridDim.x < nitems) wn = desc[item + gridDim.x];
      const uint32_t buf = tcount & 1;
      const bool waited = mbar_wait(smem_u32(&accf[buf]), (tcount >> 1) & 1);
      // the four warps agree before leaving, so no warp reads a buffer another abandoned
      const bool ok = epi_sync_and(waited && !abort_flag);
      if (!ok) {
        if (!waited && !abort_flag) give_up();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const double *sc = bscale + w.kc * P.Nmax + w.n0;
      float2 *frow = reinterpret_cast<float2 *>(Cbuf) + (w.p0t0 + row - P.pair_base) * P.Nmax + w.n0;
      const uint32_t tbase = taddr + (uint32_t(warp * 32) << 16) + buf * uint32_t(NACC * P.nc_max);
      for (int c0 = 0; c0 < w.ncw; c0 += 16) {
        float sm[16], er[16];
        tmem_ff16<NACC>(tbase + uint32_t(c0), w.nc, sm, er);
        if (c0 + 16 >= w.ncw) {   // the last reads of this buffer are done: hand it back
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(smem_u32(&acce[buf]));
        }
        if (row < w.npt) store_ff16(sm, er, sc + c0, frow + c0, w.ncw - c0);
      }
      ++tcount;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 4) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(taddr));
}

// ---- stage A, persistent and warp-specialised, operand roles swapped ---------------------
// T[k][j'] = sum_r GS[j'][r] PhiK[k][r] with the rows of the contraction (tensor-memory
// lanes) on 128 columns j' of the model's g slices and its N dimension on a chunk of up to
// nw k points of the group.  The g slices (NS x Ncols x Kp, the large operand) then move from
// DRAM once per k chunk, and consecutive work items -- taken by neighbouring CTAs at the same
// time -- are the k chunks of one column tile, which share that tile through L2; the k phase
// slices of the group stay in L2.  Both operands are pre-tiled (k_g_slices,
// k_phase_slices_k), so a stage is two contiguous blocks: one thread moves them with two
// cp.async.bulk copies that complete on the stage's mbarrier (expect_tx), all ST stages in
// flight.  One accumulator set of NACC x nw (<= 480) tensor-memory columns; its epilogue (the
// diagonals summed by TwoSum into a float-float pair, scaled by the column's power of two,
// stored as two FP32 numbers) runs while the producer refills the stages.
// Roles: warps 0-3 epilogue (tensor-memory lane quadrant w), warp 4 tensor-memory allocation
// and (lane 0) every tcgen05.mma and commit, warp 5 lane 0 the bulk copies.  Barriers: full[s]
// (the producer's expect_tx arrival plus the bytes of its two copies), empty[s] (the MMA commit
// after the products that read stage s), accf (commit after an item's last products), acce
// (128 epilogue threads have read the accumulators).  Every wait is bounded; on a timeout the
// roles leave their loops, the producer waits (bounded) for its copies still in flight, the
// MMA thread for its last commit, and the tensor memory is freed.
constexpr int kSaThreads = 192;

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
               :: "r"(mbar), "r"(bytes) : "memory");
}

// bulk global -> shared copy of `bytes` (16-byte aligned addresses, a multiple of 16 bytes)
// completing on mbarrier `mbar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

template <int NS, int NACC, int ST, bool ATM>
__global__ void __launch_bounds__(kSaThreads, 1) k_stage_a_ws(TcParams P, int64_t nitems, int nkch,
                                                              const __nv_bfloat16 *__restrict__ gs,
                                                              const __nv_bfloat16 *__restrict__ phik,
                                                              const double *__restrict__ gscale, float2 *T,
                                                              int *err) {
  constexpr int KC = 16;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[ST], empty[ST], accf, acce;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (*reinterpret_cast<volatile int *>(err)) return;   // the whole CTA returns, before any barrier
  const int nw = P.nc_max;
  const uint32_t a_slice = uint32_t(kTcM) * KC * 2, b_slice = uint32_t(nw) * KC * 2;
  const uint32_t a_bytes = NS * a_slice, b_bytes = NS * b_slice;
  const uint32_t a_col0 = uint32_t(NACC * nw);   // ATM: two A buffers of 8 NS columns after the accumulators
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int nkb = P.Kp / KC;
  const int nkc = int(P.nkc);
  if (tid == 0) {
    for (int i = 0; i < ST; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&accf)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&acce)), "r"(kTcM));
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tslot;
  auto give_up = [&]() {
    abort_flag = 1;
    atomicExch(err, 1);
  };
  // item -> column tile ct, k chunk kch, first k k0, live k count nk, MMA width ncw
  auto decode = [&](int64_t item, int &ct, int &kch, int &k0, int &nk, int &ncw) {
    ct = int(item / nkch);
    kch = int(item - int64_t(ct) * nkch);
    k0 = kch * nw;
    nk = nkc - k0 < nw ? nkc - k0 : nw;
    ncw = round_up(nk, 16);
  };

  if (warp == 5) {
    // ---------------- bulk copies (one thread)
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      const unsigned char *gsb = reinterpret_cast<const unsigned char *>(gs);
      const unsigned char *pkb = reinterpret_cast<const unsigned char *>(phik);
      for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        int ct, kch, k0, nk, ncw;
        decode(item, ct, kch, k0, nk, ncw);
        const unsigned char *asrc = gsb + size_t(ct) * nkb * a_bytes;
        const unsigned char *bsrc = pkb + size_t(kch) * nkb * b_bytes;
        for (int kb = 0; kb < nkb; ++kb) {
          const uint32_t slot = it % ST;
          if (it >= ST && !mbar_wait(smem_u32(&empty[slot]), ((it / ST) - 1) & 1)) {
            give_up();
            ok = false;
            break;
          }
          if (abort_flag) {
            ok = false;
            break;
          }
          const uint32_t sA = smem_u32(smem + slot * stage_bytes);
          const uint32_t fb = smem_u32(&full[slot]);
          mbar_expect_tx(fb, stage_bytes);
          bulk_g2s(sA, asrc + size_t(kb) * a_bytes, a_bytes, fb);
          bulk_g2s(sA + a_bytes, bsrc + size_t(kb) * b_bytes, b_bytes, fb);
          ++it;
        }
      }
      // no copy may still be writing shared memory when the CTA leaves: wait (bounded) for the
      // stages issued last (on the normal path the MMA thread has consumed them already)
      for (uint32_t j = it >= ST ? it - ST : 0; j < it; ++j)
        if (!mbar_wait(smem_u32(&full[j % ST]), (j / ST) & 1)) give_up();
    }
    __syncwarp();
  } else if (warp == 4) {
    // ---------------- tensor-core products (one thread)
    if (lane == 0) {
      uint32_t it = 0, tcount = 0, last_bar = 0, last_par = 0;
      bool any = false;
      for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        if (abort_flag) break;
        int ct, kch, k0, nk, ncw;
        decode(item, ct, kch, k0, nk, ncw);
        if (tcount >= 1 && !mbar_wait(smem_u32(&acce), (tcount - 1) & 1)) {
          give_up();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(ncw >> 3) << 17) |
                               (uint32_t(kTcM >> 4) << 24);
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
          const uint32_t slot = it % ST;
          if (!mbar_wait(smem_u32(&full[slot]), (it / ST) & 1) || abort_flag) {
            if (!abort_flag) give_up();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          if (!P.withhold) {
            const unsigned char *sA = smem + slot * stage_bytes;
            const unsigned char *sB = sA + a_bytes;
            const uint64_t ad0 = smem_desc(smem_u32(sA), 128u, (KC / 8) * 128u);
            const uint64_t bd0 = smem_desc(smem_u32(sB), 128u, (KC / 8) * 128u);
            if (ATM) {
              // A slices into tensor-memory buffer it & 1 (each read once from shared memory
              // instead of once per product); the products of stage it - 2, the buffer's last
              // readers, have completed first
              if (it >= 2 && !mbar_wait(smem_u32(&empty[(it - 2) % ST]), ((it - 2) / ST) & 1)) {
                give_up();
                ok = false;
                break;
              }
              const uint32_t a_tm = taddr + a_col0 + (it & 1u) * uint32_t(8 * NS);
#pragma unroll
              for (int is = 0; is < NS; ++is)
                asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;"
                             :: "r"(a_tm + uint32_t(8 * is)), "l"(ad0 + uint64_t(is) * (a_slice >> 4)));
              if (kb == 0)
                slice_products_tm<NS, NACC, true>(taddr, uint32_t(nw), a_tm, bd0, b_slice >> 4, idesc);
              else
                slice_products_tm<NS, NACC, false>(taddr, uint32_t(nw), a_tm, bd0, b_slice >> 4, idesc);
            } else if (kb == 0) {
              slice_products<NS, NACC, true>(taddr, uint32_t(nw), ad0, bd0, a_slice >> 4, b_slice >> 4, idesc);
            } else {
              slice_products<NS, NACC, false>(taddr, uint32_t(nw), ad0, bd0, a_slice >> 4, b_slice >> 4, idesc);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&empty[slot])) : "memory");
            any = true;
            last_bar = smem_u32(&empty[slot]);
            last_par = (it / ST) & 1;
          }
          ++it;
        }
        if (!ok) break;
        if (!P.withhold) {
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(smem_u32(&accf)) : "memory");
          last_bar = smem_u32(&accf);
          last_par = tcount & 1;
        }
        ++tcount;
      }
      if (any && !mbar_wait(last_bar, last_par)) give_up();
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 0-3: tensor-memory lanes 32w .. 32w + 31 = columns j0 + row)
    const int row = warp * 32 + lane;
    uint32_t tcount = 0;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
      int ct, kch, k0, nk, ncw;
      decode(item, ct, kch, k0, nk, ncw);
      const int j = ct * kTcM + row;
      const bool live = j < P.ncols;
      const float f = live ? pow2_float(gscale[j]) : 0.f;
      const bool waited = mbar_wait(smem_u32(&accf), tcount & 1);
      const bool ok = epi_sync_and(waited && !abort_flag);
      if (!ok) {
        if (!waited && !abort_flag) give_up();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      float2 *out = T + size_t(k0) * P.out_stride + j;
      const uint32_t tb = taddr + (uint32_t(warp * 32) << 16);
      for (int c0 = 0; c0 < ncw; c0 += 16) {
        float sm[16], er[16];
        tmem_ff16<NACC>(tb + uint32_t(c0), nw, sm, er);
        if (c0 + 16 >= ncw) {   // the last reads of the accumulators: hand them back
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(smem_u32(&acce));
        }
        if (live)
          for (int c = 0; c < 16; ++c)
            if (c0 + c < nk) {
              float h, l;
              ff_two_sum(sm[c], er[c], h, l);
              out[size_t(c0 + c) * P.out_stride] = make_float2(__fmul_rn(h, f), __fmul_rn(l, f));
            }
      }
      ++tcount;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 4) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(taddr));
}
}  // namespace

int tc_kp(const ModelDev &M) { return round_up(2 * M.nRgp, kTcKc); }
int tc_nmax(const ModelDev &M) { return round_up(2 * M.nb * M.nb * M.nbr, 16); }
// Tile shapes a launch may use.  Every accumulator of a chunk must fit the CTA's tensor memory
// (NACC x width columns: all 512 with one CTA per SM, 256 with two) and the operand stages its
// shared memory.  Two CTAs per SM: K blocks of 16 in two stages.
int tc_nc_max(int ns) { return ns == 8 ? 64 : (ns == 7 ? 96 : 256); }
static int nacc_of(int ns) { return ns == 8 ? 6 : (ns == 7 ? 5 : 2); }
// Mixed mode: 4 slices (32-bit inputs, 10 products, two accumulators).  With 3 slices (24-bit
// inputs, 6 products) the Seebeck tensor of a 4-band case already missed the 1e-6 coefficient
// bound (1.06e-6), as did a contraction of length 686.
int tc_slices_for(int kp, bool fp64_grade) {
  if (!fp64_grade) return kp <= 1024 ? 4 : 0;
  return kp <= 256 ? 7 : (kp <= 816 ? 8 : 0);
}
static bool two_ctas(int kc, int st) { return kc == 16 && st == 2; }
static bool warp_specialised(int kc, int st) { return kc == 16 && st == 5; }
size_t tc_smem_bytes(int ns, int ncm, int kc, int st) {
  const size_t need = size_t(st) * (size_t(ns) * kTcM * kc * 2 + size_t(ns) * ncm * kc * 2);
  if (warp_specialised(kc, st)) return need;
  // two-CTA shapes ask for at least 96 KB so that no third CTA (whose tensor memory would not
  // fit) is placed on the SM
  return two_ctas(kc, st) && need < 96 * 1024 ? 96 * 1024 : need;
}
bool tc_nc_valid(int ns, int ncm, int kc, int st) {
  if (ncm < 16 || ncm % 16 != 0 || ncm > tc_nc_max(ns)) return false;
  if (!((kc == 32 && st == 2) || (kc == 16 && (st == 2 || st == 4 || st == 5)))) return false;
  if (tc_smem_bytes(ns, ncm, kc, st) > 200 * 1024 + 1024) return false;
  // the warp-specialised form double-buffers its accumulators in the 512 columns
  if (warp_specialised(kc, st)) return 2 * nacc_of(ns) * ncm <= 512;
  return !two_ctas(kc, st) || nacc_of(ns) * ncm <= 256;
}
std::vector<TcShape> tc_shape_candidates(int ns) {
  if (ns == 8) return {{48, 32, 2}, {64, 32, 2}, {32, 16, 2}, {64, 16, 4}, {32, 16, 5}};
  if (ns == 7) return {{48, 32, 2}, {64, 32, 2}, {96, 32, 2}, {48, 16, 2}, {96, 16, 4}, {48, 16, 5}};
  return {{64, 32, 2}, {128, 32, 2}, {256, 32, 2}, {128, 16, 2}, {256, 16, 4}, {64, 16, 5}, {128, 16, 5}};
}

int tc_kp_a(const ModelDev &M) { return round_up(2 * M.nRge, kTcKc); }
int tc_ncols_a(const ModelDev &M) { return round_up(2 * M.nRgp * M.nb * M.nb * M.nbr, 16); }

static int stage_a_nct(const ModelDev &M) { return (tc_ncols_a(M) + kTcM - 1) / kTcM; }
size_t tc_gs_elems_a(const ModelDev &M, int ns) { return size_t(ns) * stage_a_nct(M) * kTcM * tc_kp_a(M); }

cudaError_t launch_g_slices(const ModelDev &M, int ns, __nv_bfloat16 *gs, double *gscale, cudaStream_t st) {
  const int Ncols = tc_ncols_a(M), Kp = tc_kp_a(M), nct = stage_a_nct(M);
  EPHB_LAUNCH(k_g_scales, unsigned((int64_t(Ncols) + 127) / 128), 128, 0, st, M, Ncols, gscale);
  const int64_t n = int64_t(nct) * (Kp / 16) * 256;
  EPHB_LAUNCH(k_g_slices, unsigned((n + 255) / 256), 256, 0, st, M, ns, Kp, Ncols, nct, gscale, gs);
  return cudaGetLastError();
}

// Stage A on the tensor cores: the k phase slices of the group, then the persistent
// swapped-role contraction (k_stage_a_ws) into T[k][j'] as float-float pairs.  The k chunk
// width: the fewest chunks of at most (512 / NACC rounded down to 16) k points, balanced and
// rounded up to 16.
// chunk cap: the accumulators and (tensor-memory A form) two A buffers of 8 ns columns fit the
// 512 columns; both forms use the same chunks
static int stage_a_cap(int ns) { return ((512 - 16 * ns) / nacc_of(ns)) / 16 * 16; }
static int stage_a_chunk(int ns, int64_t nkc, int *nkch) {
  const int cap = stage_a_cap(ns);
  const int64_t n = (nkc + cap - 1) / cap;
  *nkch = int(n);
  return round_up(int((nkc + n - 1) / n), 16);
}
// rows of the phase-slice operand for any group of at most `chunk` k points: nkch x nw <=
// chunk + 16 nkch
size_t stage_a_phik_elems(const ModelDev &M, int ns, int64_t chunk) {
  const int cap = stage_a_cap(ns);
  const int64_t rows = chunk + 16 * ((chunk + cap - 1) / cap);
  return size_t(rows) * ns * tc_kp_a(M);
}
constexpr int kStageASt = 4;   // shared-memory stages of the stage-A pipeline

cudaError_t launch_stage_a_tc(const ModelDev &M, const MeshDev &D, int ns, int64_t i0, int64_t nkc,
                              __nv_bfloat16 *phik, const __nv_bfloat16 *gs, const double *gscale, double2 *T, int *err,
                              bool a_tmem, cudaStream_t st, double *flops_acc) {
  if (nkc <= 0) return cudaSuccess;
  if (ns != 7 && ns != 8) return cudaErrorInvalidValue;
  const int Kp = tc_kp_a(M), Ncols = tc_ncols_a(M);
  int nkch = 0;
  const int nw = stage_a_chunk(ns, nkc, &nkch);
  const int nrows = nkch * nw;
  const int64_t n = int64_t(nrows) * (Kp / 8);
  EPHB_LAUNCH(k_phase_slices_k, unsigned((n + 255) / 256), 256, 0, st, M, D, i0, nkc, nrows, nw, ns, Kp, phik);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TcParams P;
  P.ns = ns;
  P.nacc = nacc_of(ns);
  P.Kp = Kp;
  P.Nmax = Ncols;
  P.nc_max = nw;
  P.i0 = i0;
  P.nkc = nkc;
  P.pair_base = 0;
  P.ncols = 2 * M.nRgp * M.nb * M.nb * M.nbr;
  P.out_stride = P.ncols;
  P.withhold = 0;
  const int64_t nct = stage_a_nct(M);
  const int64_t nitems = nct * nkch;
  const size_t smem = size_t(kStageASt) * ns * (size_t(kTcM) * 16 * 2 + size_t(nw) * 16 * 2);
  int dev = 0, nsm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned grid = unsigned(nitems < nsm ? nitems : nsm);
  float2 *out = reinterpret_cast<float2 *>(T);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (r != cudaSuccess) return r;
    EPHB_LAUNCH(kern, grid, kSaThreads, smem, st, P, nitems, nkch, gs, phik, gscale, out, err);
    return cudaGetLastError();
  };
  if (a_tmem)
    e = ns == 8 ? go(k_stage_a_ws<8, 6, kStageASt, true>) : go(k_stage_a_ws<7, 5, kStageASt, true>);
  else
    e = ns == 8 ? go(k_stage_a_ws<8, 6, kStageASt, false>) : go(k_stage_a_ws<7, 5, kStageASt, false>);
  // issued MMA work: 128 columns x each chunk's width x Kp per slice product and column tile
  if (flops_acc) {
    double width = 0.0;
    for (int c = 0; c < nkch; ++c) width += round_up(int(std::min<int64_t>(nw, nkc - int64_t(c) * nw)), 16);
    *flops_acc += 2.0 * kTcM * width * Kp * (ns * (ns + 1) / 2) * double(nct);
  }
  return e;
}

cudaError_t launch_phase_slices(const ModelDev &M, const MeshDev &D, int ns, __nv_bfloat16 *phis,
                                __nv_bfloat16 *angle_tab, cudaStream_t st) {
  const int Kp = tc_kp(M);
  const int64_t n = D.nq * int64_t(Kp);
  const Mesh &q = D.qm;
  if (angle_tab && q.n[0] == q.n[1] && q.n[1] == q.n[2]) {
    EPHB_LAUNCH(k_phase_angle_table, unsigned((2 * q.n[0] + 127) / 128), 128, 0, st, q.n[0], ns, angle_tab);
    EPHB_LAUNCH(k_phase_slices_cubic, unsigned((n / 8 + 255) / 256), 256, 0, st, M, D, ns, Kp, angle_tab, phis);
  } else {
    EPHB_LAUNCH(k_phase_slices, unsigned((n + 255) / 256), 256, 0, st, M, D, ns, Kp, phis);
  }
  return cudaGetLastError();
}

cudaError_t launch_vertex_tc(const ModelDev &M, const MeshDev &D, int ns, int64_t i0, int64_t nkc, int64_t pair_base,
                             const double2 *A, const __nv_bfloat16 *phis, __nv_bfloat16 *bs, double *bscale,
                             int *nitem, int64_t *item_ptr, int64_t *scratch, int64_t scratch_elems,
                             int64_t *total_dev, double *Cbuf, int *err, cudaStream_t st, cudaEvent_t gemm0,
                             cudaEvent_t gemm1, int ncm, int kc, int stages, int withhold, int64_t *ws_desc,
                             int64_t ws_cap) {
  if (nkc <= 0) return cudaSuccess;
  if (!tc_nc_valid(ns, ncm, kc, stages)) return cudaErrorInvalidValue;
  const int Kp = tc_kp(M), Nmax = tc_nmax(M);
  {
    const size_t smem = b_slices_smem(M);
    cudaError_t r = cudaFuncSetAttribute(k_b_slices, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (r != cudaSuccess) return r;
    const int ngrp = b_slices_groups(M);
    EPHB_LAUNCH(k_b_slices, dim3(unsigned(nkc), unsigned(M.nb + 1), unsigned(ngrp)), 256, smem, st, M, D, i0, A, ns,
                Kp, Nmax, ngrp, bs, bscale);
  }
  const int nprod = ns * (ns + 1) / 2;
  EPHB_LAUNCH(k_tc_items, unsigned((nkc + 255) / 256), 256, 0, st, M, D, i0, nkc, ncm, Kp, nprod, nitem,
              reinterpret_cast<unsigned long long *>(total_dev + 1));
  cudaError_t e = exclusive_scan<int>(nitem, item_ptr, nkc, total_dev, scratch, scratch_elems, st);
  if (e != cudaSuccess) return e;
  int64_t nitems = 0;
  e = cudaMemcpyAsync(&nitems, total_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || nitems == 0) return e;
  TcParams P;
  P.ns = ns;
  P.nacc = nacc_of(ns);
  P.Kp = Kp;
  P.Nmax = Nmax;
  P.nc_max = ncm;
  P.i0 = i0;
  P.nkc = nkc;
  P.pair_base = pair_base;
  P.ncols = Nmax;
  P.out_stride = Nmax;
  P.withhold = withhold;
  const size_t smem = tc_smem_bytes(ns, ncm, kc, stages);
  if (gemm0) {
    e = cudaEventRecord(gemm0, st);
    if (e != cudaSuccess) return e;
  }
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (r != cudaSuccess) return r;
    EPHB_LAUNCH(kern, unsigned(nitems), kTcThreads, smem, st, M, D, P, item_ptr, phis, bs, bscale, Cbuf, err);
    return cudaGetLastError();
  };
  // persistent form: one CTA per SM
  auto go_ws = [&](auto kern) -> cudaError_t {
    if (nitems > ws_cap) return cudaErrorInvalidValue;
    WsItem *desc = reinterpret_cast<WsItem *>(ws_desc);
    EPHB_LAUNCH(k_ws_items, unsigned((nkc + 255) / 256), 256, 0, st, M, D, P, item_ptr, desc);
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (r != cudaSuccess) return r;
    int dev = 0, nsm = 0;
    r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (r != cudaSuccess) return r;
    const unsigned grid = unsigned(nitems < nsm ? nitems : nsm);
    EPHB_LAUNCH(kern, grid, kWsThreads, smem, st, M, D, P, nitems, desc, phis, bs, bscale, Cbuf, err);
    return cudaGetLastError();
  };
  if (warp_specialised(kc, stages))
    e = ns == 8 ? go_ws(k_vertex_gemm_ws<8, 6, 5>)
                : (ns == 7 ? go_ws(k_vertex_gemm_ws<7, 5, 5>) : go_ws(k_vertex_gemm_ws<4, 2, 5>));
  else if (ns == 8)
    e = kc == 32 ? go(k_vertex_gemm<8, 6, 32, 2>)
                 : (stages == 4 ? go(k_vertex_gemm<8, 6, 16, 4>) : go(k_vertex_gemm<8, 6, 16, 2>));
  else if (ns == 7)
    e = kc == 32 ? go(k_vertex_gemm<7, 5, 32, 2>)
                 : (stages == 4 ? go(k_vertex_gemm<7, 5, 16, 4>) : go(k_vertex_gemm<7, 5, 16, 2>));
  else
    e = kc == 32 ? go(k_vertex_gemm<4, 2, 32, 2>)
                 : (stages == 4 ? go(k_vertex_gemm<4, 2, 16, 4>) : go(k_vertex_gemm<4, 2, 16, 2>));
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e == cudaSuccess && gemm1) e = cudaEventRecord(gemm1, st);
  return e;
}

}  // namespace ephb
