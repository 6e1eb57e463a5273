// Transport-coefficient reduction that allocates no memory.
//
// Some callers may not allocate device memory when they need the coefficients: hosts that
// route every allocation through a pool of their own, and embedders that may only touch the
// buffers they were handed.  This entry point lets them turn response arrays they already
// own into the coefficient tensors.  Its only scratch is a file-scope __device__ array
// holding the per-block partial sums; every GPU that loads the library keeps that array
// until the process exits.
#include <mutex>

#include "ephb.h"
#include "internal.h"

namespace ephb {
namespace {

constexpr int kNaThreads = 256;
constexpr int64_t kNaChunk = 4096;                 // states (or modes) reduced by one block
constexpr int kNaMaxBlocks = 1024;                 // per kind (electron / phonon)
constexpr int kNaE = 36, kNaP = 18;
static_assert(int64_t(kNaMaxBlocks) * kNaChunk == EPHB_NOALLOC_MAX_ITEMS, "scratch bound and header disagree");

// Partial sums: [electron blocks][36] followed by [phonon blocks][18]; 442 KB.
static __device__ __align__(256) double g_noalloc_partials[kNaMaxBlocks * (kNaE + kNaP)];

struct NaParams {
  int64_t ns, nm;
  const double *eps, *vel, *wt, *I, *J;
  const double *w, *vph, *F, *G;
  double T, mu, Pe, Pph, omega_min;
  int nbe, nbp, nsym;
  double C[kMaxSym * 9];
};

__device__ inline double na_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block b < nbe reduces states [b*chunk, (b+1)*chunk); the others reduce phonon modes.
__global__ void __launch_bounds__(kNaThreads) k_na_partial(NaParams p, double *scratch) {
  __shared__ double ws[kNaThreads / 32][kNaE];
  double acc[kNaE];
  for (int j = 0; j < kNaE; ++j) acc[j] = 0.0;
  const double kT = kKbEVK * p.T;
  const bool electron = int(blockIdx.x) < p.nbe;
  const int b = electron ? int(blockIdx.x) : int(blockIdx.x) - p.nbe;
  const int64_t lo = int64_t(b) * kNaChunk;
  if (electron) {
    const int64_t hi = lo + kNaChunk < p.ns ? lo + kNaChunk : p.ns;
    for (int64_t s = lo + threadIdx.x; s < hi; s += kNaThreads) {
      if (p.wt[s] == 0.0) continue;
      const double f = 1.0 / (exp((p.eps[s] - p.mu) / kT) + 1.0);
      const double wff = p.wt[s] * f * (1.0 - f);
      const double d = p.eps[s] - p.mu;
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          const double vj = wff * p.vel[s * 3 + a] * p.J[s * 3 + c];
          const double vi = -wff * p.vel[s * 3 + a] * p.I[s * 3 + c];
          acc[a * 3 + c] += vj;
          acc[9 + a * 3 + c] += vi;
          acc[18 + a * 3 + c] += d * vj;
          acc[27 + a * 3 + c] += d * vi;
        }
    }
  } else {
    const int64_t hi = lo + kNaChunk < p.nm ? lo + kNaChunk : p.nm;
    for (int64_t t = lo + threadIdx.x; t < hi; t += kNaThreads) {
      const double w = p.w[t];
      if (!(w > p.omega_min)) continue;
      const double n = 1.0 / expm1(w / kT);
      const double wt = w * n * (1.0 + n);
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          acc[a * 3 + c] += -wt * p.vph[t * 3 + a] * p.G[t * 3 + c];
          acc[9 + a * 3 + c] += wt * p.vph[t * 3 + a] * p.F[t * 3 + c];
        }
    }
  }
  const int nacc = electron ? kNaE : kNaP;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < nacc; ++j) {
    const double v = na_warp_sum(acc[j]);
    if (lane == 0) ws[wid][j] = v;
  }
  __syncthreads();
  if (int(threadIdx.x) < nacc) {
    double s = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) s += ws[w][threadIdx.x];
    double *dst = electron ? scratch + size_t(b) * kNaE : scratch + size_t(kNaMaxBlocks) * kNaE + size_t(b) * kNaP;
    dst[threadIdx.x] = s;
  }
}

// out (72 doubles, ephb_coeffs order): sigma, sigmaS, S, alpha_el, kappa0_el, kappa_el, alpha_ph, kappa_ph
__global__ void k_na_final(NaParams p, const double *scratch, double *out) {
  __shared__ double M[kNaE + kNaP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < kNaE + kNaP; j += nw) {
    double s = 0.0;
    if (j < kNaE)
      for (int b = lane; b < p.nbe; b += 32) s += scratch[size_t(b) * kNaE + j];
    else
      for (int b = lane; b < p.nbp; b += 32) s += scratch[size_t(kNaMaxBlocks) * kNaE + size_t(b) * kNaP + (j - kNaE)];
    s = na_warp_sum(s);
    if (lane == 0) M[j] = s;
  }
  __syncthreads();
  // symmetrised electron tensors, one thread per (tensor, a, b): sum_S S M S^T (48 x 9 terms)
  __shared__ double t[4][9];
  const double sg[4] = {1.0, 1.0, -1.0, -1.0};
  if (threadIdx.x < 36) {
    const int c = threadIdx.x / 9, a = (threadIdx.x % 9) / 3, b = threadIdx.x % 3;
    double acc = 0.0;
    for (int o = 0; o < p.nsym; ++o) {
      const double *S = p.C + 9 * o;
      double s = 0.0;
      for (int e = 0; e < 3; ++e)
        for (int f = 0; f < 3; ++f) s += S[a * 3 + e] * M[9 * c + e * 3 + f] * S[b * 3 + f];
      acc += s;
    }
    t[c][a * 3 + b] = acc * sg[c] * p.Pe;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double *sig = t[0];
  double inv[9];
  inv[0] = sig[4] * sig[8] - sig[5] * sig[7];
  inv[1] = sig[2] * sig[7] - sig[1] * sig[8];
  inv[2] = sig[1] * sig[5] - sig[2] * sig[4];
  inv[3] = sig[5] * sig[6] - sig[3] * sig[8];
  inv[4] = sig[0] * sig[8] - sig[2] * sig[6];
  inv[5] = sig[2] * sig[3] - sig[0] * sig[5];
  inv[6] = sig[3] * sig[7] - sig[4] * sig[6];
  inv[7] = sig[1] * sig[6] - sig[0] * sig[7];
  inv[8] = sig[0] * sig[4] - sig[1] * sig[3];
  const double det = sig[0] * inv[0] + sig[1] * inv[3] + sig[2] * inv[6];
  double S[9], kel[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = 0.0;
      for (int c = 0; c < 3; ++c) v += inv[a * 3 + c] * t[1][c * 3 + b];
      S[a * 3 + b] = det != 0.0 ? v / det : 0.0;
    }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = 0.0;
      for (int c = 0; c < 3; ++c) v += t[2][a * 3 + c] * S[c * 3 + b];
      kel[a * 3 + b] = t[3][a * 3 + b] - v;
    }
  for (int j = 0; j < 9; ++j) {
    out[j] = t[0][j];
    out[9 + j] = t[1][j];
    out[18 + j] = S[j];
    out[27 + j] = t[2][j];
    out[36 + j] = t[3][j];
    out[45 + j] = kel[j];
    out[54 + j] = p.Pph * M[kNaE + j];
    out[63 + j] = p.Pph * M[kNaE + 9 + j];
  }
}

std::mutex g_na_mutex;
double *g_na_ptr[64] = {nullptr};   // device address of the scratch array, per device ordinal

}  // namespace
}  // namespace ephb

using namespace ephb;

extern "C" ephb_status ephb_transport_coefficients_noalloc(const ephb_coeff_inputs *in, double *out_dev,
                                                           void *cuda_stream) {
  if (!in || !out_dev) return EPHB_EINVAL;
  if (in->n_states < 0 || in->n_modes < 0 || in->n_states > EPHB_NOALLOC_MAX_ITEMS ||
      in->n_modes > EPHB_NOALLOC_MAX_ITEMS)
    return EPHB_EINVAL;   // more than EPHB_NOALLOC_MAX_ITEMS states or modes: the scratch would overflow
  if ((in->n_states > 0 && (!in->eps || !in->vel || !in->weight || !in->I || !in->J)) ||
      (in->n_modes > 0 && (!in->omega || !in->vph || !in->F || !in->G)))
    return EPHB_EINVAL;
  if (in->nsym < 1 || in->nsym > kMaxSym || !(in->T_K > 0) || !(in->volume_A3 > 0) || in->nk < 1 || in->nq < 1)
    return EPHB_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return EPHB_ECUDA;
  double *scratch = nullptr;
  {
    // first call on this device: look up the device address of the scratch array
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr) return EPHB_ECUDA;
      g_na_ptr[dev] = static_cast<double *>(ptr);
    }
    scratch = g_na_ptr[dev];
  }
  NaParams p;
  p.ns = in->n_states;
  p.nm = in->n_modes;
  p.eps = in->eps;
  p.vel = in->vel;
  p.wt = in->weight;
  p.I = in->I;
  p.J = in->J;
  p.w = in->omega;
  p.vph = in->vph;
  p.F = in->F;
  p.G = in->G;
  p.T = in->T_K;
  p.mu = in->mu_eV;
  const double V = in->volume_A3 * kAngstrom * kAngstrom * kAngstrom;
  const double kT = kKbEVK * in->T_K;
  p.Pe = in->spin_deg * kECharge / (V * double(in->nk) * kT);
  p.Pph = kECharge / (V * double(in->nq) * kT);
  p.omega_min = in->omega_min_eV;
  p.nbe = int((in->n_states + kNaChunk - 1) / kNaChunk);
  p.nbp = int((in->n_modes + kNaChunk - 1) / kNaChunk);
  p.nsym = in->nsym;
  for (int j = 0; j < in->nsym * 9; ++j) p.C[j] = in->sym_cart[j / 9][j % 9];
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (p.nbe + p.nbp > 0) {
    EPHB_LAUNCH(k_na_partial, unsigned(p.nbe + p.nbp), kNaThreads, 0, st, p, scratch);
    if (cudaGetLastError() != cudaSuccess) return EPHB_ECUDA;
  }
  EPHB_LAUNCH(k_na_final, 1, 512, 0, st, p, scratch, out_dev);
  if (cudaGetLastError() != cudaSuccess) return EPHB_ECUDA;
  return EPHB_OK;
}
