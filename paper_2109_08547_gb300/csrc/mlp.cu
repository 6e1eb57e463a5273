// Warm-start network: a fully connected net (tanh hidden layers, linear output) trained on
// converged solutions of the coupled BTE to propose the starting electron responses.
//
// Parameters are kept in FP32 (master copy, Adam moments) with a BF16 copy of the weights; in
// BF16 mode every matrix-product operand (weights, activations, back-propagated errors) is
// rounded to BF16 and the products accumulate in FP32.  FP32 mode skips the rounding (used to
// check the gradients tightly).  Loss: 1/(2N) sum_i |y_i - t_i|^2.  Every reduction runs in a
// fixed order, so a training run is bit-reproducible.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ephb.h"
#include "internal.h"

using namespace ephb;

namespace {

constexpr int kTile = 64;        // output tile (rows and columns) of the GEMM kernel
constexpr int kBK = 16;          // K step
constexpr int kGemmThreads = 256;
constexpr int kSplit = 152;      // split of the sample dimension for weight gradients

// C(i, j) = sum_k A(i, k) B(k, j) with A(i, k) = A[i sa_i + k sa_k], B(k, j) = B[k sb_k + j sb_j];
// blockIdx.z takes K range [z kc, (z+1) kc) and writes the partial C + z M N.
// EPI 0: C = acc (+ bias[j]); 1: C = tanh(acc + bias[j]); 2: C = acc * (1 - H(i,j)^2).
template <int EPI>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(int M, int N, int K, int kc, const float *__restrict__ A,
                                                       int64_t sa_i, int64_t sa_k, const float *__restrict__ Bm,
                                                       int64_t sb_k, int64_t sb_j, const float *__restrict__ bias,
                                                       const float *__restrict__ H, float *C, int round_bf16) {
  __shared__ float As[kBK][kTile + 1];
  __shared__ float Bs[kBK][kTile + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;     // 16 x 16 threads, 4 x 4 outputs each
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += kBK) {
    for (int t = tid; t < kBK * kTile; t += kGemmThreads) {
      const int kk = t / kTile, r = t % kTile;
      const int k = k0 + kk;
      float a = 0.f, b = 0.f;
      if (k < ke && i0 + r < M) a = A[int64_t(i0 + r) * sa_i + int64_t(k) * sa_k];
      if (k < ke && j0 + r < N) b = Bm[int64_t(k) * sb_k + int64_t(j0 + r) * sb_j];
      if (round_bf16) {
        a = __bfloat162float(__float2bfloat16_rn(a));
        b = __bfloat162float(__float2bfloat16_rn(b));
      }
      As[kk][r] = a;
      Bs[kk][r] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[u] = As[kk][ty + 16 * u];
        bv[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
  float *Cz = C + size_t(blockIdx.z) * M * N;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i >= M || j >= N) continue;
      float c = acc[u][v];
      if (EPI == 0 && bias) c += bias[j];
      if (EPI == 1) c = tanhf(c + bias[j]);
      if (EPI == 2) {
        const float h = H[int64_t(i) * N + j];
        c *= 1.f - h * h;
      }
      Cz[int64_t(i) * N + j] = c;
    }
}

// out[e] = sum_z part[z * n + e] (fixed order)
__global__ void k_sum_parts(int64_t n, int nz, const float *__restrict__ part, float *out) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= n) return;
  float s = 0.f;
  for (int z = 0; z < nz; ++z) s += part[size_t(z) * n + e];
  out[e] = s;
}

// column sums of D [N x O] in kSplit row chunks: part[z][o]
__global__ void k_colsum_parts(int64_t N, int O, const float *__restrict__ D, float *part) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  const int z = blockIdx.y;
  const int64_t rows = (N + kSplit - 1) / kSplit;
  const int64_t r0 = z * rows, r1 = r0 + rows < N ? r0 + rows : N;
  float s = 0.f;
  for (int64_t r = r0; r < r1; ++r) s += D[r * O + o];
  part[size_t(z) * O + o] = s;
}

// delta = (y - t) / N; per-block partial sums of |y - t|^2 (fixed block order)
__global__ void k_loss(int64_t n, float inv_n, const float *__restrict__ y, const float *__restrict__ t, float *delta,
                       float *part) {
  __shared__ float red[256];
  float s = 0.f;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const float d = y[e] - t[e];
    delta[e] = d * inv_n;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_adam(int64_t n, float lr, float b1, float b2, float eps, float c1, float c2, float *p,
                       const float *__restrict__ g, float *m, float *v) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= n) return;
  const float gg = g[e];
  const float mm = b1 * m[e] + (1.f - b1) * gg;
  const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
  m[e] = mm;
  v[e] = vv;
  p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// counter-based uniform in [0, 1): splitmix64 of (seed, index)
__device__ inline double uniform01(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return double(z >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_init_layer(int64_t nw, int64_t nb, float lim, uint64_t seed, uint64_t base, float *w, float *b) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e < nw) w[e] = float((2.0 * uniform01(seed, base + e) - 1.0) * lim);
  if (e < nb) b[e] = 0.f;
}

}  // namespace

struct ephb_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_in = 0, width = 0, depth = 0, n_out = 0;
  int round_bf16 = 1;
  std::vector<int> din, dout;
  std::vector<int64_t> woff, boff;
  int64_t nparam = 0, step = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  float *work = nullptr;   // activations, errors, partials
  size_t work_cap = 0;
  std::string err;
};

namespace {

ephb_status mfail(ephb_mlp *n, ephb_status s, const char *msg) {
  n->err = msg;
  return s;
}

#define MCK(x)                                                   \
  do {                                                           \
    cudaError_t e_ = (x);                                        \
    if (e_ != cudaSuccess) return mfail(net, EPHB_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

size_t work_floats(const ephb_mlp *net, int64_t n) {
  // activations h_0..h_depth, two error buffers, output, split-K partials, loss partials
  size_t acts = size_t(n) * net->n_in + size_t(n) * net->width * net->depth;
  size_t errs = 2 * size_t(n) * std::max(net->width, net->n_out);
  size_t outb = size_t(n) * net->n_out;
  size_t maxw = size_t(std::max(net->width, net->n_in)) * std::max(net->width, net->n_out);
  size_t parts = size_t(kSplit) * maxw + 1024;
  return acts + errs + outb + parts + 2048;
}

cudaError_t gemm(int epi, int M, int N, int K, int splits, const float *A, int64_t sa_i, int64_t sa_k,
                 const float *Bm, int64_t sb_k, int64_t sb_j, const float *bias, const float *H, float *C, int rb,
                 cudaStream_t st) {
  const int kc = (K + splits - 1) / splits;
  dim3 grid(unsigned((N + kTile - 1) / kTile), unsigned((M + kTile - 1) / kTile), unsigned(splits));
  if (epi == 0)
    EPHB_LAUNCH(k_gemm<0>, grid, kGemmThreads, 0, st, M, N, K, kc, A, sa_i, sa_k, Bm, sb_k, sb_j, bias, H, C, rb);
  else if (epi == 1)
    EPHB_LAUNCH(k_gemm<1>, grid, kGemmThreads, 0, st, M, N, K, kc, A, sa_i, sa_k, Bm, sb_k, sb_j, bias, H, C, rb);
  else
    EPHB_LAUNCH(k_gemm<2>, grid, kGemmThreads, 0, st, M, N, K, kc, A, sa_i, sa_k, Bm, sb_k, sb_j, bias, H, C, rb);
  return cudaGetLastError();
}

// forward pass into the work buffer; returns pointers to the activations and the output
cudaError_t forward(ephb_mlp *net, const float *x, int64_t n, std::vector<const float *> &h, float *&y) {
  const int L = net->depth + 1;
  float *w = net->work;
  h.assign(L, nullptr);
  h[0] = x;
  float *cur = w + size_t(n) * net->n_in;   // x is read in place; slot 0 of the work buffer stays free
  for (int l = 0; l < L; ++l) {
    const bool last = l == L - 1;
    float *out = last ? w + size_t(n) * net->n_in + size_t(n) * net->width * net->depth : cur;
    cudaError_t e = gemm(last ? 0 : 1, int(n), net->dout[l], net->din[l], 1, h[l], net->din[l], 1,
                         net->p + net->woff[l], 1, net->din[l], net->p + net->boff[l], nullptr, out, net->round_bf16,
                         net->stream);
    if (e != cudaSuccess) return e;
    if (!last) {
      h[l + 1] = out;
      cur = out + size_t(n) * net->width;
    } else {
      y = out;
    }
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

ephb_status ephb_mlp_create(ephb_mlp **out, int device, void *cuda_stream, int n_in, int width, int depth, int n_out,
                            uint64_t seed) {
  if (!out) return EPHB_EINVAL;
  *out = nullptr;
  if (n_in < 1 || width < 1 || depth < 0 || n_out < 1 || n_in > 4096 || width > 4096 || n_out > 4096)
    return EPHB_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return EPHB_ECUDA;
  if (device < 0 || device >= ndev) return EPHB_EINVAL;
  ephb_mlp *net = new (std::nothrow) ephb_mlp();
  if (!net) return EPHB_ENOMEM;
  net->device = device;
  net->n_in = n_in;
  net->width = width;
  net->depth = depth;
  net->n_out = n_out;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete net;
    return EPHB_ECUDA;
  }
  if (cuda_stream) {
    net->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete net;
      return EPHB_ECUDA;
    }
    net->own_stream = true;
  }
  const int L = depth + 1;
  int64_t o = 0;
  for (int l = 0; l < L; ++l) {
    const int a = l == 0 ? n_in : width, b = l == L - 1 ? n_out : width;
    net->din.push_back(a);
    net->dout.push_back(b);
    net->woff.push_back(o);
    o += int64_t(a) * b;
    net->boff.push_back(o);
    o += b;
  }
  net->nparam = o;
  bool ok = cudaMalloc(&net->p, o * sizeof(float)) == cudaSuccess && cudaMalloc(&net->g, o * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&net->m, o * sizeof(float)) == cudaSuccess && cudaMalloc(&net->v, o * sizeof(float)) == cudaSuccess;
  if (ok) ok = cudaMemsetAsync(net->m, 0, o * sizeof(float), net->stream) == cudaSuccess &&
               cudaMemsetAsync(net->v, 0, o * sizeof(float), net->stream) == cudaSuccess;
  uint64_t base = 0;
  for (int l = 0; l < L && ok; ++l) {
    const int64_t nw = int64_t(net->din[l]) * net->dout[l], nb = net->dout[l];
    const float lim = float(std::sqrt(6.0 / double(net->din[l] + net->dout[l])));
    const int64_t nmax = nw > nb ? nw : nb;
    EPHB_LAUNCH(k_init_layer, unsigned((nmax + 255) / 256), 256, 0, net->stream, nw, nb, lim, seed, base,
                net->p + net->woff[l], net->p + net->boff[l]);
    ok = cudaGetLastError() == cudaSuccess;
    base += uint64_t(nw);
  }
  if (ok) ok = cudaStreamSynchronize(net->stream) == cudaSuccess;
  if (!ok) {
    ephb_mlp_destroy(net);
    return EPHB_ECUDA;
  }
  *out = net;
  return EPHB_OK;
}

void ephb_mlp_destroy(ephb_mlp *net) {
  if (!net) return;
  cudaSetDevice(net->device);
  if (net->stream) cudaStreamSynchronize(net->stream);
  for (float *q : {net->p, net->g, net->m, net->v, net->work})
    if (q) cudaFree(q);
  if (net->own_stream) cudaStreamDestroy(net->stream);
  delete net;
}

const char *ephb_mlp_last_error(const ephb_mlp *net) { return net ? net->err.c_str() : "null network"; }

int64_t ephb_mlp_num_params(const ephb_mlp *net) { return net ? net->nparam : 0; }

ephb_status ephb_mlp_set_bf16(ephb_mlp *net, int on) {
  if (!net) return EPHB_EINVAL;
  net->round_bf16 = on ? 1 : 0;
  return EPHB_OK;
}

ephb_status ephb_mlp_get_params(ephb_mlp *net, float *host, int64_t n) {
  if (!net || !host || n != net->nparam) return EPHB_EINVAL;
  MCK(cudaSetDevice(net->device));
  MCK(cudaMemcpyAsync(host, net->p, n * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  MCK(cudaStreamSynchronize(net->stream));
  return EPHB_OK;
}

ephb_status ephb_mlp_set_params(ephb_mlp *net, const float *host, int64_t n) {
  if (!net || !host || n != net->nparam) return EPHB_EINVAL;
  MCK(cudaSetDevice(net->device));
  MCK(cudaMemcpyAsync(net->p, host, n * sizeof(float), cudaMemcpyHostToDevice, net->stream));
  MCK(cudaMemsetAsync(net->m, 0, n * sizeof(float), net->stream));
  MCK(cudaMemsetAsync(net->v, 0, n * sizeof(float), net->stream));
  MCK(cudaStreamSynchronize(net->stream));
  net->step = 0;
  return EPHB_OK;
}

static ephb_status ensure_work(ephb_mlp *net, int64_t n) {
  const size_t need = work_floats(net, n);
  if (need <= net->work_cap) return EPHB_OK;
  if (net->work) cudaFree(net->work);
  net->work = nullptr;
  net->work_cap = 0;
  MCK(cudaMalloc(&net->work, need * sizeof(float)));
  net->work_cap = need;
  return EPHB_OK;
}

ephb_status ephb_mlp_forward(ephb_mlp *net, const float *x_dev, int64_t n, float *y_dev) {
  if (!net || (!x_dev && n > 0) || (!y_dev && n > 0) || n < 0) return EPHB_EINVAL;
  if (n == 0) return EPHB_OK;
  MCK(cudaSetDevice(net->device));
  ephb_status s = ensure_work(net, n);
  if (s != EPHB_OK) return s;
  std::vector<const float *> h;
  float *y = nullptr;
  MCK(forward(net, x_dev, n, h, y));
  MCK(cudaMemcpyAsync(y_dev, y, size_t(n) * net->n_out * sizeof(float), cudaMemcpyDeviceToDevice, net->stream));
  MCK(cudaStreamSynchronize(net->stream));
  return EPHB_OK;
}

ephb_status ephb_mlp_loss_grad(ephb_mlp *net, const float *x_dev, const float *t_dev, int64_t n, float *loss_host,
                               float *grad_dev) {
  if (!net || !x_dev || !t_dev || n < 1) return EPHB_EINVAL;
  MCK(cudaSetDevice(net->device));
  ephb_status s = ensure_work(net, n);
  if (s != EPHB_OK) return s;
  cudaStream_t st = net->stream;
  const int L = net->depth + 1;
  std::vector<const float *> h;
  float *y = nullptr;
  MCK(forward(net, x_dev, n, h, y));
  // work layout after the forward pass: [x slot][h_1..h_depth][y][errA][errB][partials]
  float *errA = y + size_t(n) * net->n_out;
  float *errB = errA + size_t(n) * std::max(net->width, net->n_out);
  float *part = errB + size_t(n) * std::max(net->width, net->n_out);
  const int64_t ny = n * net->n_out;
  const int nlb = 256;
  EPHB_LAUNCH(k_loss, nlb, 256, 0, st, ny, 1.f / float(n), y, t_dev, errA, part);
  MCK(cudaGetLastError());
  float *lossp = part + size_t(kSplit) * size_t(std::max(net->width, net->n_in)) * std::max(net->width, net->n_out);
  MCK(cudaMemcpyAsync(lossp, part, nlb * sizeof(float), cudaMemcpyDeviceToDevice, st));
  float *delta = errA, *other = errB;
  for (int l = L - 1; l >= 0; --l) {
    const int a = net->din[l], b = net->dout[l];
    // dW_l = delta^T h_l  (split over samples, summed in order), db_l = column sums of delta
    const int splits = int(std::min<int64_t>(kSplit, (n + 255) / 256));
    MCK(gemm(0, b, a, int(n), splits, delta, 1, b, h[l], a, 1, nullptr, nullptr, part, net->round_bf16, st));
    EPHB_LAUNCH(k_sum_parts, unsigned((int64_t(a) * b + 255) / 256), 256, 0, st, int64_t(a) * b, splits, part,
                net->g + net->woff[l]);
    MCK(cudaGetLastError());
    EPHB_LAUNCH(k_colsum_parts, dim3(unsigned((b + 127) / 128), kSplit), 128, 0, st, n, b, delta, part);
    MCK(cudaGetLastError());
    EPHB_LAUNCH(k_sum_parts, unsigned((b + 255) / 256), 256, 0, st, int64_t(b), kSplit, part, net->g + net->boff[l]);
    MCK(cudaGetLastError());
    if (l > 0) {   // delta_{l-1} = (delta W_l) * (1 - h_l^2)
      MCK(gemm(2, int(n), a, b, 1, delta, b, 1, net->p + net->woff[l], a, 1, nullptr, h[l], other, net->round_bf16,
               st));
      std::swap(delta, other);
    }
  }
  if (grad_dev)
    MCK(cudaMemcpyAsync(grad_dev, net->g, net->nparam * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (loss_host) {
    std::vector<float> lp(nlb);
    MCK(cudaMemcpyAsync(lp.data(), lossp, nlb * sizeof(float), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    double sum = 0.0;
    for (float q : lp) sum += q;
    *loss_host = float(0.5 * sum / double(n));
  } else {
    MCK(cudaStreamSynchronize(st));
  }
  return EPHB_OK;
}

ephb_status ephb_mlp_train_step(ephb_mlp *net, const float *x_dev, const float *t_dev, int64_t n, float lr,
                                float *loss_host) {
  ephb_status s = ephb_mlp_loss_grad(net, x_dev, t_dev, n, loss_host, nullptr);
  if (s != EPHB_OK) return s;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  net->step += 1;
  const float c1 = float(1.0 - std::pow(0.9, double(net->step))), c2 = float(1.0 - std::pow(0.999, double(net->step)));
  EPHB_LAUNCH(k_adam, unsigned((net->nparam + 255) / 256), 256, 0, net->stream, net->nparam, lr, b1, b2, eps, c1, c2,
              net->p, net->g, net->m, net->v);
  MCK(cudaGetLastError());
  return EPHB_OK;
}

}  // extern "C"
