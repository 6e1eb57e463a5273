// The coupled e-ph iteration ("Coupled and decoupled BTEs": the phonon drag update, the
// electron loop against it, the Kelvin-Onsager step and the convergence test on the transport
// tensors) of every instance as one CUDA graph, launched once per solve.
//
// The host-driven loop (api.cu) reads a residual back after every FP64 sweep and every outer
// iteration to decide what to launch next.  Here those decisions are taken on the device:
// each loop is a WHILE conditional node and each choice a SWITCH node, and one-thread control
// kernels (k_gs_*) read the residuals that the coefficient kernels wrote and set the node
// conditions with cudaGraphSetConditional.  The graph holds one independent branch per
// instance, so the sweeps of all (T, mu, window) instances are in flight together from a
// single launch.  Within an instance the kernels and their order are the host loop's: the
// answers, sweep counts and iteration counts are bit-identical.
//
// Termination: every loop's control kernel counts its body executions and stops at the
// iteration limit (max_inner, max_outer), and also when %globaltimer has advanced past the
// time limit since the instance started (the instance is then flagged timed_out).
#include <cstring>
#include <vector>

#include "ephb.h"
#include "internal.h"

namespace ephb {
namespace {

__device__ inline unsigned long long gs_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline bool gs_out_of_time(GraphCtl *c, double limit_s) {
  if (double(gs_now() - c->t0) > limit_s * 1e9) {
    c->timed_out = 1;
    return true;
  }
  return false;
}

__global__ void k_gs_init(GraphCtl *c) {
  GraphCtl z;
  memset(&z, 0, sizeof(z));
  z.lambda = 1.0;
  z.t0 = gs_now();
  *c = z;
}

// Start of an outer iteration: which arithmetic the phonon-side terms use (the host loop's
// rule: FP32 while the outer residual is at or above kPh32Until, float-float after), the
// electron loop's tolerance, and the electron loop armed.
__global__ void k_gs_outer_head(GraphCtl *c, GraphOpts o, int has_switch, cudaGraphConditionalHandle h_ph,
                                cudaGraphConditionalHandle h_inner) {
  c->n_outer_body += 1;
  const bool late = gs_out_of_time(c, o.time_limit_s);
  int mode = 2;
  if (o.ph32_allowed) mode = (!c->outer_seen || c->residual >= kPh32Until) ? 0 : 1;
  c->ph_mode = mode;
  if (mode == 0) c->outer32 += 1;
  double tol_k = o.inner_tol;
  if (o.precision == EPHB_SOLVE_MIXED && o.level == EPHB_DRAGGED)
    tol_k = fmax(o.inner_tol, c->outer_seen ? 1e-2 * c->residual : 1e-2);
  c->tol_k = tol_k;
  if (o.precision == EPHB_SOLVE_MIXED) c->last_tol_k = tol_k;
  c->inner_it = 0;
  c->inner_ok = 0;
  if (!late) c->n_ph_body[mode] += 1;
  if (has_switch) cudaGraphSetConditional(h_ph, late ? 3u : unsigned(mode));   // 3: no body runs
  cudaGraphSetConditional(h_inner, late ? 0u : 1u);
}

// Electron loop of the dragless level (no outer iteration): arm it.
__global__ void k_gs_inner_start(GraphCtl *c, GraphOpts o, cudaGraphConditionalHandle h_inner) {
  c->tol_k = o.inner_tol;
  c->last_tol_k = o.inner_tol;
  c->inner_it = 0;
  c->inner_ok = 0;
  cudaGraphSetConditional(h_inner, 1u);
}

// After an FP64 sweep of the mixed loop: converged (or out of sweeps) -> the sweep's output is
// the answer (switch body 0 copies it); otherwise the FP32 corrections run (body 1).
__global__ void k_gs_inner_mixed(GraphCtl *c, const double *res, GraphOpts o, cudaGraphConditionalHandle h_sw,
                                 cudaGraphConditionalHandle h_inner) {
  c->n_inner_body += 1;
  const int it = c->inner_it + 1;
  c->inner_it = it;
  c->sweeps += 1;
  c->inner_total += 1;
  const bool conv = res[72] < c->tol_k;
  const bool stop = conv || it >= o.max_inner || gs_out_of_time(c, o.time_limit_s);
  if (conv) c->inner_ok = 1;
  if (!stop) c->sweeps32 += kCorrSweeps;
  const int sw = stop ? 0 : 1;
  c->n_in_body[sw] += 1;
  cudaGraphSetConditional(h_sw, unsigned(sw));
  cudaGraphSetConditional(h_inner, stop ? 0u : 1u);
}

// After one fused FP64 sweep: the sweep's own coefficient assembly sets sctl[0] when the loop
// is done (converged or max_inner sweeps).
__global__ void k_gs_inner_fp64(GraphCtl *c, const int *sctl, GraphOpts o, cudaGraphConditionalHandle h_inner) {
  c->n_inner_body += 1;
  const int it = c->inner_it + 1;
  c->inner_it = it;
  const bool stop = sctl[0] != 0 || it >= o.max_inner || gs_out_of_time(c, o.time_limit_s);
  cudaGraphSetConditional(h_inner, stop ? 0u : 1u);
}

// After the FP64 loop: an odd number of sweeps left the answer in the second buffer pair.
__global__ void k_gs_fp64_after(GraphCtl *c, const int *sctl, int64_t n3, const double *I2, const double *J2,
                                double *I, double *J) {
  const int done = sctl[1];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->sweeps += done;
    c->inner_total += done;
    c->inner_ok = sctl[2];
  }
  if (!(done & 1)) return;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n3; i += int64_t(gridDim.x) * blockDim.x) {
    I[i] = I2[i];
    J[i] = J2[i];
  }
}

// End of an outer iteration (after the KO step and the coefficients of the new state): the
// outer test of the host loop.
__global__ void k_gs_outer_tail(GraphCtl *c, const double *res, GraphOpts o, cudaGraphConditionalHandle h_outer) {
  const int outer = c->outer + 1;
  c->outer = outer;
  c->residual = res[73];
  c->outer_seen = 1;
  if (o.ko && res[75] != 0.0) c->lambda = res[74];
  const bool conv =
      o.level == EPHB_PARTIAL || (c->residual < o.tol && c->last_tol_k <= o.inner_tol && c->ph_mode != 0);
  if (conv && !c->timed_out) c->converged = 1;
  const bool go = !conv && outer < o.max_outer && !gs_out_of_time(c, o.time_limit_s);
  cudaGraphSetConditional(h_outer, go ? 1u : 0u);
}

__global__ void k_gs_dragless_tail(GraphCtl *c, const double *res) {
  c->outer = 1;
  c->residual = res[72];
  c->converged = c->inner_ok && !c->timed_out;
}

__global__ void k_gs_copy2(int64_t n, const double *a, const double *b, double *a_out, double *b_out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    a_out[i] = a[i];
    b_out[i] = b[i];
  }
}

__global__ void k_gs_copy(int64_t n, const double *a, double *out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = a[i];
}

__global__ void k_gs_zero(int64_t nwords, uint32_t *p) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nwords; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = 0u;
}

unsigned grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return unsigned(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// launched also for n = 0, so that a switch body made of it alone is never empty
cudaError_t copy2(int64_t n, const double *a, const double *b, double *ao, double *bo, cudaStream_t st) {
  EPHB_LAUNCH(k_gs_copy2, grid_for(n), 256, 0, st, n, a, b, ao, bo);
  return cudaGetLastError();
}

cudaError_t copy1(int64_t n, const double *a, double *o, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  EPHB_LAUNCH(k_gs_copy, grid_for(n), 256, 0, st, n, a, o);
  return cudaGetLastError();
}

cudaError_t zero_bytes(size_t bytes, void *p, cudaStream_t st) {
  const int64_t nw = int64_t(bytes / 4);
  if (nw == 0) return cudaSuccess;
  EPHB_LAUNCH(k_gs_zero, grid_for(nw), 256, 0, st, nw, static_cast<uint32_t *>(p));
  return cudaGetLastError();
}

#define GS_CK(call)                          \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)

// Captures launches from one stream into a given graph after given dependencies; end()
// returns the capture's leaf nodes.
struct Capture {
  cudaStream_t cs;
  long long k0 = 0;
  cudaError_t begin(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps) {
    k0 = launch_count();
    return cudaStreamBeginCaptureToGraph(cs, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                         cudaStreamCaptureModeRelaxed);
  }
  // kernels captured since begin() are added to *kcount
  cudaError_t end(std::vector<cudaGraphNode_t> &leaves, long long *kcount) {
    cudaStreamCaptureStatus stt;
    const cudaGraphNode_t *d = nullptr;
    size_t n = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &stt, nullptr, nullptr, &d, nullptr, &n);
    if (e == cudaSuccess && stt == cudaStreamCaptureStatusActive) leaves.assign(d, d + n);
    cudaGraph_t g2 = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g2);
    if (kcount) *kcount += launch_count() - k0;
    if (e != cudaSuccess) return e;
    if (stt != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    return e2;
  }
};

cudaError_t add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, unsigned size, cudaGraphNode_t *node,
                            cudaGraph_t *bodies) {
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};   // reserved fields zero
  std::memset(&p.conditional, 0, sizeof(p.conditional));
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = size;
  GS_CK(cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p));
  for (unsigned i = 0; i < size; ++i) bodies[i] = p.conditional.phGraph_out[i];
  return cudaSuccess;
}

struct InstBuilder {
  const ModelDev &M;
  const MeshDev &D;
  const GraphInst &g;
  const GraphOpts &o;
  cudaGraph_t root;
  Capture cap;
  GraphKernels &kc;
  bool mixed() const { return o.precision == EPHB_SOLVE_MIXED; }

  cudaError_t coefficients(double *prev, cudaStream_t st) {
    GS_CK(launch_e_partial(g.B, g.I, g.J, g.epart, st));
    GS_CK(launch_ph_partial(D, g.B, g.F, g.G, g.W_ph, g.inv_nnW, g.ppart, st));
    return launch_coeff_final(M, g.B, g.epart, g.ppart, g.res, prev, st);
  }

  // I, J, F, G at the start; the FP32 / float-float copies of the rates; the RTA tensors into prev_out
  cudaError_t prologue(cudaStream_t st) {
    EPHB_LAUNCH(k_gs_init, 1, 1, 0, st, g.ctl);
    GS_CK(cudaGetLastError());
    if (g.warm)
      GS_CK(launch_apply_warm(g.nst, g.I0, g.J0, g.warm, g.I, g.J, st));
    else
      GS_CK(copy2(g.nst * 3, g.I0, g.J0, g.I, g.J, st));
    GS_CK(copy1(g.nph * 3, g.F0, g.F, st));
    GS_CK(zero_bytes(size_t(g.nph) * 3 * sizeof(double), g.G, st));
    GS_CK(zero_bytes(kResLen * sizeof(double), g.prev_out, st));
    if (mixed()) GS_CK(launch_to_f32(g.nruns, g.run_w, g.run_w32, st));
    if (o.ph32_allowed) {
      GS_CK(launch_copy_f32(2 * g.n_entries, reinterpret_cast<const double *>(g.e_X),
                            reinterpret_cast<float *>(g.X32), st));
      GS_CK(launch_copy_f32(g.n_ph_entries, g.ph_Y, g.Y32, st));
      GS_CK(launch_copy_ff(2 * g.n_entries, reinterpret_cast<const double *>(g.e_X),
                           reinterpret_cast<float2 *>(g.Xff), st));
      GS_CK(launch_copy_ff(g.n_ph_entries, g.ph_Y, g.Yff, st));
    }
    return coefficients(g.prev_out, st);
  }

  // The electron loop's start: the coefficients of the current state (the loop's first
  // reference), then the drag term of the current F, G in the given arithmetic.
  cudaError_t inner_prologue(int drag_mode, cudaStream_t st) {
    GS_CK(zero_bytes(kResLen * sizeof(double), g.prev_in, st));
    GS_CK(coefficients(g.prev_in, st));
    if (drag_mode == 0) GS_CK(launch_drag_term32(D, g.B, g.Se, g.X32, g.FG32, g.seg_part, g.Dterm, st));
    if (drag_mode == 1) GS_CK(launch_drag_termff(D, g.B, g.Se, g.Xff, g.FGff, g.seg_part, g.Dterm, st));
    if (drag_mode == 2) GS_CK(launch_drag_term(D, g.B, g.Se, g.F, g.G, g.seg_part, g.Dterm, st));
    return cudaSuccess;
  }

  // FP64 loop only: the loop control words, the packed responses and the fused-assembly counter
  cudaError_t fp64_loop_setup(cudaStream_t st) {
    GS_CK(zero_bytes(4 * sizeof(int), g.sctl, st));
    GS_CK(launch_pack_ij(g.nst, g.I, g.J, g.IJ, st));
    return zero_bytes(sizeof(unsigned), g.fuse_ctr, st);
  }

  // phonon half of an outer iteration in arithmetic `mode` (0 FP32, 1 float-float, 2 FP64),
  // then the electron loop's start
  cudaError_t phonon_half(int mode, cudaStream_t st) {
    if (mode == 0) {
      GS_CK(launch_pack6_f32(g.nst, g.I, g.J, g.IJ32, st));
      GS_CK(launch_ph_sweep32(M, g.B, g.Sp, g.kinfo, g.Y32, g.IJ32, g.ph_part, g.Btv, st));
    } else if (mode == 1) {
      GS_CK(launch_pack6_ff(g.nst, g.I, g.J, g.IJff, st));
      GS_CK(launch_ph_sweepff(M, g.B, g.Sp, g.kinfo, g.Yff, g.IJff, g.ph_part, g.Btv, st));
    } else {
      GS_CK(launch_ph_sweep(M, g.B, g.Sp, g.kinfo, g.I, g.J, g.ph_part, g.Btv, st));
    }
    GS_CK(launch_ph_update(M, D, g.Btv, g.F0, g.inv_nnW, g.F, g.G, g.Afold, st));
    if (mode == 0) GS_CK(launch_pack6_f32(g.nph, g.F, g.G, g.FG32, st));
    if (mode == 1) GS_CK(launch_pack6_ff(g.nph, g.F, g.G, g.FGff, st));
    return inner_prologue(mode, st);
  }

  // The electron loop as a WHILE node after `deps` in `parent`; leaves <- the node (plus the
  // FP64 loop's buffer fix-up).
  cudaError_t electron_loop(cudaGraph_t parent, std::vector<cudaGraphNode_t> &leaves, bool drag,
                            cudaGraphConditionalHandle h_inner, cudaGraphConditionalHandle h_sw,
                            long long *after_count) {
    cudaGraphNode_t wn;
    cudaGraph_t body;
    GS_CK(add_conditional(parent, leaves, h_inner, cudaGraphCondTypeWhile, 1, &wn, &body));
    std::vector<cudaGraphNode_t> lb;
    const cudaStream_t st = cap.cs;
    GS_CK(cap.begin(body, {}));
    if (mixed()) {
      GS_CK(launch_self_sweep(M, g.B, g.Sr, g.run_col, g.run_w, g.I0, g.J0, g.inv_ffW, g.I, g.J, g.I2, g.J2,
                              drag ? g.Dterm : nullptr, g.seg_part, g.epart, nullptr, st));
      GS_CK(launch_coeff_final(M, g.B, g.epart, g.ppart, g.res, g.prev_in, st));
      EPHB_LAUNCH(k_gs_inner_mixed, 1, 1, 0, st, g.ctl, g.res, o, h_sw, h_inner);
      GS_CK(cudaGetLastError());
      GS_CK(cap.end(lb, &kc.inner_fixed));
      cudaGraphNode_t sn;
      cudaGraph_t sb[2];
      GS_CK(add_conditional(body, lb, h_sw, cudaGraphCondTypeSwitch, 2, &sn, sb));
      std::vector<cudaGraphNode_t> tmp;
      // 0: the sweep's output is the answer
      GS_CK(cap.begin(sb[0], {}));
      GS_CK(copy2(g.nst * 3, g.I2, g.J2, g.I, g.J, st));
      GS_CK(cap.end(tmp, &kc.in[0]));
      // 1: FP32 corrections d <- r + A d (kCorrSweeps, ping-pong), x <- x + d, and the
      // coefficients of the corrected x as the next sweep's reference
      GS_CK(cap.begin(sb[1], {}));
      GS_CK(launch_corr_init(g.nst, g.I2, g.I, g.J2, g.J, g.rI, g.rJ, g.dI, g.dJ, st));
      float *dA = g.dI, *dAJ = g.dJ, *dB = g.dI2, *dBJ = g.dJ2;
      for (int j = 0; j < kCorrSweeps; ++j) {
        GS_CK(launch_corr_sweep(M, g.nst, g.Sr, g.run_col, g.run_w32, g.inv_ffW, g.rI, g.rJ, dA, dAJ, g.part32, dB,
                                dBJ, st));
        std::swap(dA, dB);
        std::swap(dAJ, dBJ);
      }
      GS_CK(launch_corr_apply(g.nst, dA, dAJ, g.I, g.J, st));
      GS_CK(launch_e_partial(g.B, g.I, g.J, g.epart, st));
      GS_CK(launch_coeff_final(M, g.B, g.epart, g.ppart, g.res, g.prev_in, st));
      GS_CK(cap.end(tmp, &kc.in[1]));
      leaves.assign(1, wn);
      return cudaSuccess;
    }
    CoeffFuse fuse;
    fuse.ppart = g.ppart;
    fuse.res = g.res;
    fuse.prev = g.prev_in;
    fuse.ctl = g.sctl;
    fuse.max_sweeps = o.max_inner;
    fuse.tol = o.inner_tol;
    fuse.counter = g.fuse_ctr;
    GS_CK(launch_self_sweep(M, g.B, g.Sr, g.run_col, g.run_w, g.I0, g.J0, g.inv_ffW, g.I, g.J, g.I2, g.J2,
                            drag ? g.Dterm : nullptr, g.seg_part, g.epart, g.sctl, st, nullptr, nullptr, g.IJ, g.IJ2,
                            &fuse));
    EPHB_LAUNCH(k_gs_inner_fp64, 1, 1, 0, st, g.ctl, g.sctl, o, h_inner);
    GS_CK(cudaGetLastError());
    GS_CK(cap.end(lb, &kc.inner_fixed));
    leaves.assign(1, wn);
    GS_CK(cap.begin(parent, leaves));
    EPHB_LAUNCH(k_gs_fp64_after, grid_for(g.nst * 3), 256, 0, st, g.ctl, g.sctl, g.nst * 3, g.I2, g.J2, g.I, g.J);
    GS_CK(cudaGetLastError());
    return cap.end(leaves, after_count);   // runs once per electron loop
  }

  cudaError_t build() {
    const cudaStream_t st = cap.cs;
    std::vector<cudaGraphNode_t> L;
    GS_CK(cap.begin(root, {}));
    GS_CK(prologue(st));
    GS_CK(cap.end(L, &kc.prologue));
    cudaGraphConditionalHandle h_inner, h_sw = 0;
    GS_CK(cudaGraphConditionalHandleCreate(&h_inner, root, 0, 0));
    if (mixed()) GS_CK(cudaGraphConditionalHandleCreate(&h_sw, root, 0, 0));
    if (o.level == EPHB_DRAGLESS) {
      GS_CK(cap.begin(root, L));
      GS_CK(inner_prologue(-1, st));
      if (!mixed()) GS_CK(fp64_loop_setup(st));
      EPHB_LAUNCH(k_gs_inner_start, 1, 1, 0, st, g.ctl, o, h_inner);
      GS_CK(cudaGetLastError());
      GS_CK(cap.end(L, &kc.prologue));
      GS_CK(electron_loop(root, L, false, h_inner, h_sw, &kc.prologue));
      GS_CK(cap.begin(root, L));
      EPHB_LAUNCH(k_gs_dragless_tail, 1, 1, 0, st, g.ctl, g.res);
      GS_CK(cudaGetLastError());
      return cap.end(L, &kc.prologue);
    }
    // partial and dragged levels: the outer iteration
    cudaGraphConditionalHandle h_outer, h_ph = 0;
    GS_CK(cudaGraphConditionalHandleCreate(&h_outer, root, 1, cudaGraphCondAssignDefault));
    if (o.ph32_allowed) GS_CK(cudaGraphConditionalHandleCreate(&h_ph, root, 0, 0));
    cudaGraphNode_t on;
    cudaGraph_t ob;
    GS_CK(add_conditional(root, L, h_outer, cudaGraphCondTypeWhile, 1, &on, &ob));
    std::vector<cudaGraphNode_t> B;
    GS_CK(cap.begin(ob, {}));
    EPHB_LAUNCH(k_gs_outer_head, 1, 1, 0, st, g.ctl, o, o.ph32_allowed ? 1 : 0, h_ph, h_inner);
    GS_CK(cudaGetLastError());
    if (!o.ph32_allowed) GS_CK(phonon_half(2, st));
    GS_CK(cap.end(B, &kc.outer_fixed));
    if (o.ph32_allowed) {
      cudaGraphNode_t sn;
      cudaGraph_t sb[3];
      GS_CK(add_conditional(ob, B, h_ph, cudaGraphCondTypeSwitch, 3, &sn, sb));
      for (int m = 0; m < 3; ++m) {
        std::vector<cudaGraphNode_t> tmp;
        GS_CK(cap.begin(sb[m], {}));
        GS_CK(phonon_half(m, st));
        GS_CK(cap.end(tmp, &kc.ph[m]));
      }
      B.assign(1, sn);
    }
    if (!mixed()) {
      GS_CK(cap.begin(ob, B));
      GS_CK(fp64_loop_setup(st));
      GS_CK(cap.end(B, &kc.outer_fixed));
    }
    GS_CK(electron_loop(ob, B, true, h_inner, h_sw, &kc.outer_fixed));
    GS_CK(cap.begin(ob, B));
    if (o.ko) GS_CK(launch_ko(M, D, g.B, g.I, g.J, g.kpart, g.res, st));
    GS_CK(coefficients(g.prev_out, st));
    EPHB_LAUNCH(k_gs_outer_tail, 1, 1, 0, st, g.ctl, g.res, o, h_outer);
    GS_CK(cudaGetLastError());
    return cap.end(B, &kc.outer_fixed);
  }
};

}  // namespace

cudaError_t build_solve_graph(const ModelDev &M, const MeshDev &D, const std::vector<GraphInst> &insts,
                              const GraphOpts &o, cudaStream_t cs, cudaGraph_t *graph, cudaGraphExec_t *exec,
                              std::vector<GraphKernels> &kernels) {
  *graph = nullptr;
  *exec = nullptr;
  kernels.assign(insts.size(), GraphKernels{});
  const long long k0 = launch_count();
  cudaGraph_t root = nullptr;
  cudaError_t e = cudaGraphCreate(&root, 0);
  for (size_t i = 0; e == cudaSuccess && i < insts.size(); ++i) {
    InstBuilder b{M, D, insts[i], o, root, Capture{cs}, kernels[i]};
    e = b.build();
  }
  // the capture counted its launches; they run only when the graph does
  note_launches(int(k0 - launch_count()));
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, root, 0);
  if (e != cudaSuccess) {
    cudaStreamCaptureStatus stt;
    if (cudaStreamIsCapturing(cs, &stt) == cudaSuccess && stt != cudaStreamCaptureStatusNone) {
      cudaGraph_t g2 = nullptr;
      cudaStreamEndCapture(cs, &g2);
    }
    if (*exec) cudaGraphExecDestroy(*exec);
    *exec = nullptr;
    if (root) cudaGraphDestroy(root);
    return e;
  }
  *graph = root;
  return cudaSuccess;
}

}  // namespace ephb
