// Host runtime behind the C ABI (include/ephb.h): the context, its device buffers, the
// call sequencing and the iteration control of the coupled BTE.  All numerical work is
// enqueued as CUDA kernels on the context stream; the host only validates arguments,
// sizes buffers and reads back scalars (counts, residuals) that steer the next launch.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ephb.h"
#include "internal.h"

using namespace ephb;

namespace {
std::atomic<long long> g_launches{0};
}

void ephb::note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long ephb::launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

// Accumulates the device time between pairs of events recorded around one kind of kernel.
struct EventTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  double ms = 0.0;
  bool pending = false;
  cudaError_t init() {
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    return e;
  }
  cudaError_t start(cudaStream_t s) { return cudaEventRecord(a, s); }
  cudaError_t stop(cudaStream_t s) {
    pending = true;
    return cudaEventRecord(b, s);
  }
  // call after the stream has been synchronised past stop()
  cudaError_t collect() {
    if (!pending) return cudaSuccess;
    float t = 0.f;
    cudaError_t e = cudaEventElapsedTime(&t, a, b);
    ms += t;
    pending = false;
    return e;
  }
  ~EventTimer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

template <typename T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t count) {
    if (count <= n && p) return cudaSuccess;
    release();
    size_t c = count ? count : 1;
    cudaError_t e = cudaMalloc(&p, c * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      return e;
    }
    n = c;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

}  // namespace

namespace {

// Everything that belongs to one (T, mu, window) instance: its rate lists and its BTE state.
struct InstState {
  double T = 300, mu = 0, win_lo = 0, win_hi = 0;
  int64_t n_entries = 0, n_ph_entries = 0, n_tuples = 0;
  DBuf<int64_t> row_ptr, ph_row_ptr;
  DBuf<uint32_t> e_kpns, ph_kpn;
  DBuf<double2> e_X;
  DBuf<int> ph_st;
  DBuf<double> ph_Y;
  // BTE
  DBuf<double> st_eps, st_vel, st_ff, st_wt, W_e, inv_ffW, I0, J0, I, J, I2, J2, Bt, W_ph, inv_nnW, F0, F, G, Btv,
      seg_part, epart, ppart, kpart, res, prev_in, prev_out, prev_tmp, Dterm, run_w;
  // segments of the entry stream (drag term) and of the partner runs (self term)
  DBuf<int> nseg_row, eseg_row, rseg_row, run_flag;
  DBuf<int64_t> eseg_ptr, eseg_begin, rseg_ptr, rseg_begin, run_ptr, run_idx;
  DBuf<uint32_t> run_col;
  int64_t neseg = 0, nrseg = 0, nruns = 0;
  // segments of the phonon entry stream (phonon drag scatter) and their partial sums
  DBuf<int> pnseg_row, pseg_row;
  DBuf<int64_t> pseg_ptr, pseg_begin;
  DBuf<double> pseg_part;
  int64_t npseg = 0;
  DBuf<double> W_chimp;         // e-chimp part of the electron RTA rates [nst]
  DBuf<double> W_iso, W_iso_rep;   // ph-isotope part of the phonon RTA rates [nq][nbr], [n_qrep][nbr]
  DBuf<uint32_t> kcrd;
  DBuf<int2> kinfo;
  DBuf<int> sctl;               // device-driven sweep loop: stop flag, sweeps done, converged
  DBuf<unsigned long long> nzero;
  DBuf<float> warm;             // warm-start scale factors [nst][2]
  // mixed-precision electron loop: FP32 run weights, residual and correction vectors, partials
  DBuf<float> run_w32, rI, rJ, dI, dJ, dI2, dJ2, part32;
  DBuf<double2> IJ, IJ2;        // packed responses for the FP64 gathers
  DBuf<unsigned> fuse_ctr;      // blocks done in the fused finalisation
  bool have_f32 = false;
  DBuf<unsigned> vmaxb;
  DBuf<double> Afold;           // phonon fold at the q representatives [n_qrep][nbr][6]
  // mixed iteration, early outer iterations: FP32 copies of the instance's rates (X, Y) and of
  // the responses ([state][I | J]) and phonon deviations ([mode][F | G]); rebuilt per solve
  DBuf<float2> X32;
  DBuf<float> Y32, IJ32, FG32;
  // later outer iterations: float-float copies of the same (FP64-grade on the FP32 pipe)
  DBuf<float4> Xff;
  DBuf<float2> Yff, IJff, FGff;
  bool bte_ready = false, has_warm = false, solved = false;
  bool lists_pending = false;   // the instance's lists are to be derived from the union lists
  ephb_solve_info last{};       // the instance's last solve

  // after a deferred instance's solve: the lists and the sweep arrays go, the responses, the
  // RTA rates and the state tables (the coefficients' inputs) stay
  void release_lists() {
    row_ptr.release(); ph_row_ptr.release(); e_kpns.release(); ph_kpn.release(); e_X.release(); ph_st.release();
    ph_Y.release();
    seg_part.release(); Dterm.release(); run_w.release(); I2.release(); J2.release(); Btv.release();
    nseg_row.release(); eseg_row.release(); rseg_row.release(); run_flag.release(); eseg_ptr.release();
    eseg_begin.release(); rseg_ptr.release(); rseg_begin.release(); run_ptr.release(); run_idx.release();
    run_col.release();
    for (auto *b : {&run_w32, &rI, &rJ, &dI, &dJ, &dI2, &dJ2, &part32}) b->release();
    IJ.release();
    IJ2.release();
    X32.release(); Y32.release(); IJ32.release(); FG32.release();
    Xff.release(); Yff.release(); IJff.release(); FGff.release();
    pnseg_row.release(); pseg_row.release(); pseg_ptr.release(); pseg_begin.release(); pseg_part.release();
    have_f32 = false;
    lists_pending = true;
  }

  void release_all() {
    row_ptr.release(); ph_row_ptr.release(); e_kpns.release(); ph_kpn.release(); e_X.release(); ph_st.release();
    ph_Y.release();
    for (auto *b : {&st_eps, &st_vel, &st_ff, &st_wt, &W_e, &inv_ffW, &I0, &J0, &I, &J, &I2, &J2, &Bt, &W_ph,
                    &inv_nnW, &F0, &F, &G, &Btv, &seg_part, &epart, &ppart, &kpart, &res, &prev_in, &prev_out,
                    &prev_tmp, &Dterm, &run_w})
      b->release();
    nseg_row.release(); eseg_row.release(); rseg_row.release(); run_flag.release(); eseg_ptr.release();
    eseg_begin.release(); rseg_ptr.release(); rseg_begin.release(); run_ptr.release(); run_idx.release();
    run_col.release(); kcrd.release(); kinfo.release(); sctl.release(); nzero.release(); warm.release();
    vmaxb.release();
    for (auto *b : {&run_w32, &rI, &rJ, &dI, &dJ, &dI2, &dJ2, &part32}) b->release();
    IJ.release();
    IJ2.release();
    fuse_ctr.release();
    Afold.release();
    X32.release(); Y32.release(); IJ32.release(); FG32.release();
    Xff.release(); Yff.release(); IJff.release(); FGff.release();
    pnseg_row.release(); pseg_row.release(); pseg_ptr.release(); pseg_begin.release(); pseg_part.release();
    W_chimp.release();
    W_iso.release();
    W_iso_rep.release();
    bte_ready = has_warm = solved = have_f32 = lists_pending = false;
  }
};

}  // namespace

struct ephb_ctx : InstState {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int stage = 0;   // 1 model, 2 meshes, 3 rates, 4 solved

  ModelDev M;
  DBuf<int> Re, Rd, Rge, Rgp, sym_rot, sym_inv;
  DBuf<double2> H_R, D_R, g_R;
  DBuf<double> sym_cart, sym_pair;

  // meshes
  Mesh km{}, qm{};
  int ratio[3] = {1, 1, 1};
  double lo = 0, hi = 0, degen_tol = 1e-6, omega_min = 1e-4;
  int64_t n_ibzw = 0, n_pairs = 0;
  ephb_mesh_info minfo{};
  DBuf<double2> ktab, qtab, cvec, u;
  DBuf<double2> interp;          // Fourier sums of H / D and their gradients for a list chunk
  DBuf<double> eps, vel, w, vph;
  DBuf<uint8_t> egrp, pgrp;
  DBuf<uint32_t> amask, rmask;
  DBuf<int> qrep, qop, qstab, qflag, qlist, qrep_of;
  DBuf<int64_t> qpos;
  int64_t n_qrep = 0;
  DBuf<__nv_bfloat16> angle_tab;      // slices of cos, sin of the 2 pi j / n angles of a cubic q mesh
  DBuf<int> atom_perm, atom_shift;
  DBuf<int> rep, op, stab, flag, ibzw_list, ibzw_of, npairs, pair_q, pair_i, qcount, pq_rank;
  DBuf<int64_t> pos, pair_ptr, pair_off, qpair_ptr, scratch, scal;

  // rates (scratch shared by the instances)
  DBuf<int> cntE, cntPh;
  DBuf<int64_t> escan, phscan;
  DBuf<double2> Tbuf, Abuf;
  // tensor-core contraction: phase slices, B' slices and scales, work items, output scratch
  DBuf<__nv_bfloat16> phis, bslices;
  // stage A on tensor cores: k phase slices of a chunk, the model's g slices (made once per
  // model and slice count) and their column scales
  DBuf<__nv_bfloat16> phik, gslices;
  DBuf<double> gscale;
  int gslices_ns = 0;
  DBuf<double> bscale, Cbuf;
  DBuf<int> nitem, tc_err;
  DBuf<int64_t> item_ptr;
  DBuf<int64_t> ws_desc;   // work-item descriptors of the persistent contraction (4 int64 each)
  int64_t ws_cap = 0;
  DBuf<double> fk, nbq, wr;
  DBuf<double2> ut;
  DBuf<float4> cff, uff;   // float-float c(k) and u(q) of the tensor-core epilogue
  DBuf<float> eps32, w32;  // FP32 copies of the energies (delta-cutoff estimate)
  DBuf<unsigned long long> ucount;

  // T-independent vertex lists over the union of the instance windows (several instances)
  int64_t u_entries = 0, u_ph_entries = 0, u_tuples = 0;
  bool deferred = false;        // instances derive their lists when solved (memory bound)
  DBuf<int64_t> u_row_ptr, u_ph_row_ptr;
  DBuf<uint32_t> u_kpns, u_ph_kpn;
  DBuf<double2> u_X;
  DBuf<int> u_ph_st;
  DBuf<double> u_ph_V;
  // Anderson acceleration of the outer iteration: ring of phonon updates g and residuals f
  DBuf<double> and_g, and_f, and_part, and_dots;

  // instances: the one in use lives in the InstState base, the others in slots
  int ninst = 1, cur = 0;
  std::vector<InstState> slots = std::vector<InstState>(1);
  // tuning: column-chunk width of the tensor-core contraction (FP64-grade, mixed); 0 = not
  // tuned yet.  force_cols != 0 overrides the tuner.
  int tune_cols[3] = {0, 0, 0};   // [7 slices, 4 slices, 8 slices]
  int tune_kc[3] = {32, 32, 32};
  int tune_st[3] = {2, 2, 2};
  int force_cols = 0;
  int withhold_mma = 0;   // failure-path check (EPHB_TUNE_WITHHOLD_MMA)
  int force_defer = 0;    // EPHB_TUNE_DEFER_INSTANCES: derive instance lists at solve time always
  int stage_a_tmem = 0;   // EPHB_TUNE_STAGE_A_TMEM_A: stage A's A slices through tensor memory
  double *host_res = nullptr;   // pinned: kResLen doubles, then the sweep-loop control (4 ints)
  // charged impurities (e-chimp) and the Gaussian of the last rates call (their delta)
  ephb_impurities imp{};
  int iso_nat = 0;               // phonon-isotope channel: mass-variance parameter per atom
  double iso_g[4] = {0, 0, 0, 0};
  double delta_sigma = 0.0, delta_cut = 0.0;
  DBuf<double> chimp_part, chimp_qtf;
  // device-driven solve: the instantiated graph, the signature of what it was built from, the
  // kernels per body (launch counts), the capture stream and the per-instance control blocks
  cudaGraph_t sg_graph = nullptr;
  cudaGraphExec_t sg_exec = nullptr;
  std::vector<unsigned char> sg_sig;
  std::vector<GraphKernels> sg_kernels;
  cudaStream_t sg_cs = nullptr;
  DBuf<GraphCtl> sg_ctl;
  void drop_graph() {
    if (sg_exec) cudaGraphExecDestroy(sg_exec);
    if (sg_graph) cudaGraphDestroy(sg_graph);
    sg_exec = nullptr;
    sg_graph = nullptr;
    sg_sig.clear();
  }
};

namespace {

ephb_status fail(ephb_ctx *ctx, ephb_status s, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return s;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? EPHB_ENOMEM : EPHB_ECUDA,                \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

template <typename T>
cudaError_t upload(DBuf<T> &b, const T *src, size_t count, cudaStream_t st) {
  cudaError_t e = b.ensure(count);
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  e = cudaMemcpyAsync(b.p, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

int64_t read_i64(ephb_ctx *ctx, const int64_t *dptr, cudaError_t &e) {
  int64_t v = 0;
  e = cudaMemcpyAsync(&v, dptr, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return v;
}

MeshDev mesh_view(ephb_ctx *c) {
  MeshDev D;
  std::memset(&D, 0, sizeof(D));
  D.km = c->km;
  D.qm = c->qm;
  for (int d = 0; d < 3; ++d) D.ratio[d] = c->ratio[d];
  D.nk = c->km.size();
  D.nq = c->qm.size();
  D.ktab = c->ktab.p;
  D.qtab = c->qtab.p;
  D.eps = c->eps.p;
  D.cvec = c->cvec.p;
  D.vel = c->vel.p;
  D.egrp = c->egrp.p;
  D.amask = c->amask.p;
  D.rmask = c->rmask.p;
  D.qrep = c->qrep.p;
  D.qop = c->qop.p;
  D.qrep_of = c->qrep_of.p;
  D.qlist = c->qlist.p;
  D.qstab = c->qstab.p;
  D.n_qrep = c->n_qrep;
  D.w = c->w.p;
  D.u = c->u.p;
  D.vph = c->vph.p;
  D.pgrp = c->pgrp.p;
  D.rep = c->rep.p;
  D.op = c->op.p;
  D.stab = c->stab.p;
  D.ibzw_of = c->ibzw_of.p;
  D.ibzw_list = c->ibzw_list.p;
  D.n_ibzw = c->n_ibzw;
  D.pair_ptr = c->pair_ptr.p;
  D.pair_q = c->pair_q.p;
  D.pair_i = c->pair_i.p;
  D.qpair_ptr = c->qpair_ptr.p;
  D.pq_rank = c->pq_rank.p;
  D.n_pairs = c->n_pairs;
  D.omega_min = c->omega_min;
  D.degen_tol = c->degen_tol;
  return D;
}

BteDev bte_view(ephb_ctx *c) {
  BteDev B;
  std::memset(&B, 0, sizeof(B));
  B.nb = c->M.nb;
  B.nbr = c->M.nbr;
  B.nsym = c->M.nsym;
  B.nst = c->n_ibzw * c->M.nb;
  B.nq = c->qm.size();
  B.T = c->T;
  B.mu = c->mu;
  B.spin_deg = c->M.spin_deg;
  const double *L = c->M.lattice;
  double V = fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                  L[2] * (L[3] * L[7] - L[4] * L[6])) *
             kAngstrom * kAngstrom * kAngstrom;
  double kT = kKbEVK * c->T;
  B.Pe = c->M.spin_deg * kECharge / (V * double(c->km.size()) * kT);
  B.Pph = kECharge / (V * double(c->qm.size()) * kT);
  B.row_ptr = c->row_ptr.p;
  B.e_kpns = c->e_kpns.p;
  B.e_X = c->e_X.p;
  B.ph_row_ptr = c->ph_row_ptr.p;
  B.ph_st = c->ph_st.p;
  B.ph_kpn = c->ph_kpn.p;
  B.ph_Y = c->ph_Y.p;
  B.kcrd = c->kcrd.p;
  B.st_eps = c->st_eps.p;
  B.st_vel = c->st_vel.p;
  B.st_ff = c->st_ff.p;
  B.st_wt = c->st_wt.p;
  return B;
}

}  // namespace

extern "C" {

ephb_status ephb_create(ephb_ctx **out, int device, void *cuda_stream) {
  if (!out) return EPHB_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return EPHB_ECUDA;
  if (device < 0 || device >= ndev) return EPHB_EINVAL;
  ephb_ctx *ctx = new (std::nothrow) ephb_ctx();
  if (!ctx) return EPHB_ENOMEM;
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return EPHB_ECUDA;
  }
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return EPHB_ECUDA;
    }
    ctx->own_stream = true;
  }
  if (cudaMallocHost(&ctx->host_res, (kResLen + 2) * sizeof(double)) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return EPHB_ENOMEM;
  }
  *out = ctx;
  return EPHB_OK;
}

void ephb_destroy(ephb_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  ctx->Re.release(); ctx->Rd.release(); ctx->Rge.release(); ctx->Rgp.release(); ctx->sym_rot.release();
  ctx->sym_inv.release(); ctx->H_R.release(); ctx->D_R.release(); ctx->g_R.release(); ctx->sym_cart.release();
  ctx->sym_pair.release();
  ctx->ktab.release(); ctx->interp.release(); ctx->qtab.release(); ctx->cvec.release(); ctx->u.release(); ctx->eps.release();
  ctx->vel.release(); ctx->w.release(); ctx->vph.release(); ctx->egrp.release(); ctx->pgrp.release();
  ctx->qrep.release(); ctx->qop.release(); ctx->qstab.release(); ctx->qflag.release(); ctx->qlist.release();
  ctx->qrep_of.release(); ctx->qpos.release(); ctx->atom_perm.release();
  ctx->atom_shift.release(); ctx->angle_tab.release();
  ctx->amask.release(); ctx->rmask.release(); ctx->rep.release(); ctx->op.release(); ctx->stab.release(); ctx->flag.release();
  ctx->ibzw_list.release(); ctx->ibzw_of.release(); ctx->npairs.release(); ctx->pair_q.release();
  ctx->pair_i.release(); ctx->qcount.release(); ctx->pq_rank.release(); ctx->pos.release();
  ctx->pair_ptr.release(); ctx->pair_off.release(); ctx->qpair_ptr.release(); ctx->scratch.release(); ctx->scal.release();
  ctx->cntE.release(); ctx->cntPh.release(); ctx->escan.release(); ctx->phscan.release();
  ctx->Tbuf.release(); ctx->Abuf.release();
  ctx->phik.release(); ctx->gslices.release(); ctx->gscale.release();
  ctx->phis.release(); ctx->bslices.release(); ctx->bscale.release(); ctx->Cbuf.release(); ctx->nitem.release();
  ctx->tc_err.release(); ctx->item_ptr.release(); ctx->ws_desc.release(); ctx->fk.release(); ctx->nbq.release(); ctx->wr.release();
  ctx->ut.release(); ctx->ucount.release(); ctx->cff.release(); ctx->uff.release(); ctx->eps32.release();
  ctx->w32.release();
  ctx->u_row_ptr.release(); ctx->u_ph_row_ptr.release(); ctx->u_kpns.release(); ctx->u_ph_kpn.release();
  ctx->u_X.release(); ctx->u_ph_st.release(); ctx->u_ph_V.release();
  ctx->drop_graph();
  ctx->sg_ctl.release();
  ctx->chimp_part.release();
  ctx->chimp_qtf.release();
  if (ctx->sg_cs) cudaStreamDestroy(ctx->sg_cs);
  ctx->release_all();
  for (auto &sl : ctx->slots) sl.release_all();
  if (ctx->host_res) cudaFreeHost(ctx->host_res);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *ephb_last_error(const ephb_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ---------------------------------------------------------------------------------------
ephb_status ephb_set_wannier_model(ephb_ctx *ctx, const ephb_model *m) {
  if (!ctx) return EPHB_EINVAL;
  if (!m) return fail(ctx, EPHB_EINVAL, "model is NULL");
  CK(cudaSetDevice(ctx->device));
  if (m->nb < 1 || m->nb > kMaxBands) return fail(ctx, EPHB_EINVAL, "nb must be in [1, 8]");
  if (m->nat < 1 || 3 * m->nat > kMaxBranches) return fail(ctx, EPHB_EINVAL, "nat must be in [1, 4]");
  if (m->nb * m->nb * 3 * m->nat > 384)
    return fail(ctx, EPHB_EINVAL, "nb^2 * 3 nat must not exceed 384 (vertex tile of one k point)");
  if (m->nRe < 1 || m->nRd < 1 || m->nRge < 1 || m->nRgp < 1) return fail(ctx, EPHB_EINVAL, "empty R list");
  if (m->nRge > 4096) return fail(ctx, EPHB_EINVAL, "nRge > 4096 not supported");
  if (m->nsym < 1 || m->nsym > kMaxSym) return fail(ctx, EPHB_EINVAL, "nsym must be in [1, 48]");
  if (!m->mass_amu || !m->Re || !m->H_R || !m->Rd || !m->D_R || !m->Rge || !m->Rgp || !m->g_R || !m->sym_rot ||
      !m->sym_cart)
    return fail(ctx, EPHB_EINVAL, "NULL array in model");
  if (!(m->omega_ref_eV > 0) || !(m->spin_deg > 0) || !(m->bg_omega_ref_eV > 0) || !(m->bg_T_ref > 0) ||
      m->bg_rate_coeff < 0)
    return fail(ctx, EPHB_EINVAL, "bad scalar model parameter");
  for (int a = 0; a < m->nat; ++a)
    if (!(m->mass_amu[a] > 0)) return fail(ctx, EPHB_EINVAL, "masses must be positive");
  // lattice-vector components stay below 2^16, so mesh index x component sums fit 32 bits
  {
    const std::pair<const int32_t *, int> lists[4] = {{m->Re, m->nRe}, {m->Rd, m->nRd}, {m->Rge, m->nRge},
                                                      {m->Rgp, m->nRgp}};
    for (const auto &l : lists)
      for (int64_t i = 0; i < 3 * int64_t(l.second); ++i)
        if (l.first[i] > 65535 || l.first[i] < -65535)
          return fail(ctx, EPHB_EINVAL, "lattice-vector components must lie within +-65535");
  }
  // the operation list must be a group closed under inversion: find S^-1 for each S
  std::vector<int> inv(m->nsym, -1);
  for (int s = 0; s < m->nsym; ++s) {
    const int32_t *A = m->sym_rot + 9 * s;
    for (int t = 0; t < m->nsym && inv[s] < 0; ++t) {
      const int32_t *B = m->sym_rot + 9 * t;
      bool id = true;
      for (int i = 0; i < 3 && id; ++i)
        for (int j = 0; j < 3 && id; ++j) {
          int v = 0;
          for (int l = 0; l < 3; ++l) v += A[3 * i + l] * B[3 * l + j];
          id = v == (i == j ? 1 : 0);
        }
      if (id) inv[s] = t;
    }
    if (inv[s] < 0) return fail(ctx, EPHB_EINVAL, "symmetry operations are not closed under inversion");
  }
  // atom map of every operation: S tau_a = tau_{p(a)} + L_a with L_a a lattice vector (crystal
  // coordinates); the phonon eigenvectors at S q follow from those at q with it
  std::vector<int> aperm(size_t(m->nsym) * m->nat), ashift(size_t(m->nsym) * m->nat * 3);
  {
    double A[3][3], Ai[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[i][j] = m->lattice[i][j];
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                       A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (!(std::fabs(det) > 0)) return fail(ctx, EPHB_EINVAL, "singular lattice");
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
        Ai[i][j] = (A[i1][j1] * A[i2][j2] - A[i1][j2] * A[i2][j1]) / det;   // inverse: (A^-1)_ij
      }
    static const double zero[3] = {0, 0, 0};
    for (int s = 0; s < m->nsym; ++s) {
      const double *C = m->sym_cart + 9 * s;
      for (int a = 0; a < m->nat; ++a) {
        const double *ta = m->tau_cart ? m->tau_cart + 3 * a : zero;
        double p[3];
        for (int x = 0; x < 3; ++x) p[x] = C[3 * x] * ta[0] + C[3 * x + 1] * ta[1] + C[3 * x + 2] * ta[2];
        int found = -1;
        for (int b = 0; b < m->nat && found < 0; ++b) {
          const double *tb = m->tau_cart ? m->tau_cart + 3 * b : zero;
          double d[3] = {p[0] - tb[0], p[1] - tb[1], p[2] - tb[2]};
          double c[3];
          bool lattice_vec = true;
          for (int j = 0; j < 3; ++j) {
            c[j] = d[0] * Ai[0][j] + d[1] * Ai[1][j] + d[2] * Ai[2][j];
            if (std::fabs(c[j] - std::round(c[j])) > 1e-6) lattice_vec = false;
          }
          if (lattice_vec) {
            found = b;
            for (int j = 0; j < 3; ++j) ashift[(size_t(s) * m->nat + a) * 3 + j] = int(std::lround(c[j]));
          }
        }
        if (found < 0) return fail(ctx, EPHB_EINVAL, "a symmetry operation does not map the atoms onto each other");
        aperm[size_t(s) * m->nat + a] = found;
      }
    }
  }
  ModelDev &M = ctx->M;
  // the tile shapes tuned for the previous model stay valid while the contraction's shape is
  // the same (a model of equal dimensions with new values)
  const bool same_shape = ctx->stage >= 1 && M.nb == m->nb && M.nat == m->nat && M.nRge == m->nRge &&
                          M.nRgp == m->nRgp;
  M = ModelDev();
  M.nat = m->nat;
  M.nb = m->nb;
  M.nbr = 3 * m->nat;
  M.nRe = m->nRe;
  M.nRd = m->nRd;
  M.nRge = m->nRge;
  M.nRgp = m->nRgp;
  M.nsym = m->nsym;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M.lattice[3 * i + j] = m->lattice[i][j];
  M.omega_ref = m->omega_ref_eV;
  M.spin_deg = m->spin_deg;
  M.bg_coeff = m->bg_rate_coeff;
  M.bg_w = m->bg_omega_ref_eV;
  M.bg_T = m->bg_T_ref;
  double msum = 0;
  for (int a = 0; a < m->nat; ++a) {
    M.mass[a] = m->mass_amu[a];
    msum += m->mass_amu[a];
  }
  M.mass_mean = msum / m->nat;
  cudaStream_t st = ctx->stream;
  const size_t nb2 = size_t(m->nb) * m->nb, nbr2 = size_t(M.nbr) * M.nbr;
  CK(upload(ctx->Re, m->Re, size_t(m->nRe) * 3, st));
  CK(upload(ctx->Rd, m->Rd, size_t(m->nRd) * 3, st));
  CK(upload(ctx->Rge, m->Rge, size_t(m->nRge) * 3, st));
  CK(upload(ctx->Rgp, m->Rgp, size_t(m->nRgp) * 3, st));
  CK(upload(ctx->H_R, reinterpret_cast<const double2 *>(m->H_R), size_t(m->nRe) * nb2, st));
  CK(upload(ctx->D_R, reinterpret_cast<const double2 *>(m->D_R), size_t(m->nRd) * nbr2, st));
  CK(upload(ctx->g_R, reinterpret_cast<const double2 *>(m->g_R), size_t(m->nRge) * m->nRgp * nb2 * M.nbr, st));
  CK(upload(ctx->sym_rot, m->sym_rot, size_t(m->nsym) * 9, st));
  CK(upload(ctx->sym_cart, m->sym_cart, size_t(m->nsym) * 9, st));
  {
    std::vector<double> pair(81, 0.0);
    for (int o = 0; o < m->nsym; ++o) {
      const double *S = m->sym_cart + 9 * o;
      for (int ab = 0; ab < 9; ++ab)
        for (int ef = 0; ef < 9; ++ef) pair[ab * 9 + ef] += S[(ab / 3) * 3 + ef / 3] * S[(ab % 3) * 3 + ef % 3];
    }
    CK(upload(ctx->sym_pair, pair.data(), pair.size(), st));
  }
  CK(upload(ctx->sym_inv, inv.data(), inv.size(), st));
  CK(upload(ctx->atom_perm, aperm.data(), aperm.size(), st));
  CK(upload(ctx->atom_shift, ashift.data(), ashift.size(), st));
  M.Re = ctx->Re.p;
  M.Rd = ctx->Rd.p;
  M.Rge = ctx->Rge.p;
  M.Rgp = ctx->Rgp.p;
  M.H_R = ctx->H_R.p;
  M.D_R = ctx->D_R.p;
  M.g_R = ctx->g_R.p;
  M.sym_rot = ctx->sym_rot.p;
  M.sym_cart = ctx->sym_cart.p;
  M.sym_pair = ctx->sym_pair.p;
  M.sym_inv = ctx->sym_inv.p;
  M.atom_perm = ctx->atom_perm.p;
  M.atom_shift = ctx->atom_shift.p;
  ctx->stage = 1;
  if (!same_shape) ctx->tune_cols[0] = ctx->tune_cols[1] = ctx->tune_cols[2] = 0;   // a new shape is tuned again
  ctx->gslices_ns = 0;                          // and its g slices are made again
  ctx->bte_ready = false;
  return EPHB_OK;
}

// ---------------------------------------------------------------------------------------
ephb_status ephb_build_meshes_ibz(ephb_ctx *ctx, const ephb_mesh_opts *o, ephb_mesh_info *out) {
  if (!ctx) return EPHB_EINVAL;
  if (ctx->stage < 1) return fail(ctx, EPHB_ESTATE, "set_wannier_model must come first");
  if (!o) return fail(ctx, EPHB_EINVAL, "opts is NULL");
  CK(cudaSetDevice(ctx->device));
  for (int d = 0; d < 3; ++d) {
    if (o->kmesh[d] < 1 || o->qmesh[d] < 1 || o->kmesh[d] > 1023)
      return fail(ctx, EPHB_EINVAL, "mesh dimensions must be in [1, 1023]");
    if (o->kmesh[d] % o->qmesh[d] != 0) return fail(ctx, EPHB_EINVAL, "k mesh must be a multiple of the q mesh");
  }
  Mesh km{{o->kmesh[0], o->kmesh[1], o->kmesh[2]}}, qm{{o->qmesh[0], o->qmesh[1], o->qmesh[2]}};
  if (km.size() > (int64_t(1) << kKpBits)) return fail(ctx, EPHB_EINVAL, "k mesh larger than 2^21 points");
  if (ctx->M.nsym > 1 && !(km.n[0] == km.n[1] && km.n[1] == km.n[2] && qm.n[0] == qm.n[1] && qm.n[1] == qm.n[2]))
    return fail(ctx, EPHB_EINVAL, "symmetry reduction needs cubic (n x n x n) meshes");
  if (!(o->window_hi_eV >= o->window_lo_eV)) return fail(ctx, EPHB_EINVAL, "empty window");
  ctx->km = km;
  ctx->qm = qm;
  for (int d = 0; d < 3; ++d) ctx->ratio[d] = km.n[d] / qm.n[d];
  ctx->lo = o->window_lo_eV;
  ctx->hi = o->window_hi_eV;
  ctx->degen_tol = o->degen_tol_eV > 0 ? o->degen_tol_eV : 1e-6;
  ctx->omega_min = o->omega_min_eV > 0 ? o->omega_min_eV : 1e-4;
  const ModelDev &M = ctx->M;
  const int64_t nk = km.size(), nq = qm.size();
  const int nb = M.nb, nbr = M.nbr;
  cudaStream_t st = ctx->stream;
  EventTimer tm;
  CK(tm.init());
  CK(tm.start(st));
  CK(ctx->ktab.ensure(km.n[0] + km.n[1] + km.n[2]));
  CK(ctx->qtab.ensure(qm.n[0] + qm.n[1] + qm.n[2]));
  CK(ctx->eps.ensure(nk * nb));
  CK(ctx->cvec.ensure(nk * nb * nb));
  CK(ctx->vel.ensure(nk * nb * 3));
  CK(ctx->egrp.ensure(nk * nb * 2));
  CK(ctx->amask.ensure(nk));
  CK(ctx->rmask.ensure(nk));
  CK(ctx->w.ensure(nq * nbr));
  CK(ctx->u.ensure(nq * nbr * nbr));
  CK(ctx->vph.ensure(nq * nbr * 3));
  CK(ctx->pgrp.ensure(nq * nbr * 2));
  CK(ctx->rep.ensure(nk));
  CK(ctx->op.ensure(nk));
  CK(ctx->stab.ensure(nk));
  CK(ctx->flag.ensure(nk));
  CK(ctx->pos.ensure(nk));
  CK(ctx->ibzw_of.ensure(nk));
  CK(ctx->scal.ensure(16));
  int64_t scr = scan_scratch_elems(nk > nq ? nk : nq);
  CK(ctx->scratch.ensure(scr));
  CK(launch_phase_tables(ctx->ktab.p, km, st));
  CK(launch_phase_tables(ctx->qtab.p, qm, st));
  // Phonons: eigen-decompositions on the representatives of the q wedge, the rest by rotation
  CK(ctx->qrep.ensure(nq));
  CK(ctx->qop.ensure(nq));
  CK(ctx->qstab.ensure(nq));
  CK(ctx->qflag.ensure(nq));
  CK(ctx->qpos.ensure(nq));
  CK(ctx->qlist.ensure(nq));
  CK(ctx->qrep_of.ensure(nq));
  CK(launch_ibz(M, qm, ctx->qrep.p, ctx->qop.p, ctx->qstab.p, ctx->qflag.p, st));
  CK(exclusive_scan<int>(ctx->qflag.p, ctx->qpos.p, nq, ctx->scal.p + 0, ctx->scratch.p, ctx->scratch.n, st));
  CK(launch_compact(nq, ctx->qflag.p, ctx->qpos.p, ctx->qlist.p, st));
  CK(cudaMemcpyAsync(&ctx->n_qrep, ctx->scal.p + 0, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(launch_rep_index(nq, ctx->qlist.p, ctx->n_qrep, ctx->qrep_of.p, st));
  auto interp_for = [&](int64_t n, int nmat) {
    return ctx->interp.ensure(size_t(4) * nmat * nmat * size_t(std::min<int64_t>(n, interp_chunk())));
  };
  CK(interp_for(ctx->n_qrep, M.nbr));
  CK(launch_phonon_modes(M, qm, ctx->qlist.p, ctx->n_qrep, ctx->qtab.p, ctx->degen_tol, ctx->omega_min, ctx->w.p,
                         ctx->u.p, ctx->vph.p, ctx->pgrp.p, ctx->interp.p, st));
  CK(launch_phonons_from_rep(M, qm, ctx->qtab.p, ctx->qrep.p, ctx->qop.p, ctx->w.p, ctx->u.p, ctx->vph.p,
                             ctx->pgrp.p, st));
  // Electron bands: eigen-decompositions on the representatives of the wedge first; a point whose
  // representative has no band in the window takes the representative's energies and rotated
  // velocities (it holds no active state and no rate reads its eigenvectors); every other point
  // is decomposed itself.  Without symmetry every point is its own representative.
  CK(launch_ibz(M, km, ctx->rep.p, ctx->op.p, ctx->stab.p, ctx->flag.p, st));
  CK(exclusive_scan<int>(ctx->flag.p, ctx->pos.p, nk, ctx->scal.p + 0, ctx->scratch.p, ctx->scratch.n, st));
  CK(launch_compact(nk, ctx->flag.p, ctx->pos.p, ctx->ibzw_of.p, st));     // representatives (scratch use)
  int64_t n_rep = 0, n_own = 0;
  CK(cudaMemcpyAsync(&n_rep, ctx->scal.p + 0, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(interp_for(n_rep, M.nb));
  CK(launch_electron_bands(M, km, ctx->ibzw_of.p, n_rep, ctx->ktab.p, ctx->degen_tol, ctx->lo, ctx->hi, ctx->eps.p,
                           ctx->cvec.p, ctx->vel.p, ctx->egrp.p, ctx->amask.p, ctx->rmask.p, ctx->interp.p, st));
  CK(launch_bands_from_rep(M, km, ctx->rep.p, ctx->op.p, ctx->eps.p, ctx->vel.p, ctx->egrp.p, ctx->amask.p,
                           ctx->rmask.p, ctx->flag.p, st));
  CK(exclusive_scan<int>(ctx->flag.p, ctx->pos.p, nk, ctx->scal.p + 0, ctx->scratch.p, ctx->scratch.n, st));
  CK(launch_compact(nk, ctx->flag.p, ctx->pos.p, ctx->ibzw_of.p, st));     // points decomposed themselves
  CK(cudaMemcpyAsync(&n_own, ctx->scal.p + 0, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(interp_for(n_own, M.nb));
  CK(launch_electron_bands(M, km, ctx->ibzw_of.p, n_own, ctx->ktab.p, ctx->degen_tol, ctx->lo, ctx->hi, ctx->eps.p,
                           ctx->cvec.p, ctx->vel.p, ctx->egrp.p, ctx->amask.p, ctx->rmask.p, ctx->interp.p, st));
  CK(launch_ibzw_flag(nk, ctx->rep.p, ctx->amask.p, ctx->flag.p, st));
  CK(exclusive_scan<int>(ctx->flag.p, ctx->pos.p, nk, ctx->scal.p + 0, ctx->scratch.p, ctx->scratch.n, st));
  CK(launch_count_bits(ctx->amask.p, nk, ctx->scal.p + 1, st));
  CK(launch_count_reps(ctx->rep.p, nk, ctx->scal.p + 2, st));
  int64_t host_scal[3];
  CK(cudaMemcpyAsync(host_scal, ctx->scal.p, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->n_ibzw = host_scal[0];
  CK(ctx->ibzw_list.ensure(ctx->n_ibzw));
  CK(launch_ibzw_fill(nk, ctx->flag.p, ctx->pos.p, ctx->ibzw_list.p, ctx->ibzw_of.p, st));
  // pairs (k, q) with an active band at k+q, sorted by q within each k
  const int nch = pair_chunks(nq);
  const int64_t ncnt = ctx->n_ibzw * nch;
  CK(ctx->npairs.ensure(ncnt));
  CK(ctx->pair_off.ensure(ncnt + 1));
  CK(ctx->pair_ptr.ensure(ctx->n_ibzw + 1));
  MeshDev D = mesh_view(ctx);
  CK(launch_pair_count(D, ctx->npairs.p, st));
  CK(ctx->scratch.ensure(scan_scratch_elems(std::max<int64_t>(ncnt, nk))));
  CK(exclusive_scan<int>(ctx->npairs.p, ctx->pair_off.p, ncnt, ctx->pair_off.p + ncnt, ctx->scratch.p,
                         ctx->scratch.n, st));
  CK(launch_pair_ptr(ctx->n_ibzw, nch, ctx->pair_off.p, ctx->pair_ptr.p, st));
  cudaError_t e;
  ctx->n_pairs = read_i64(ctx, ctx->pair_ptr.p + ctx->n_ibzw, e);
  CK(e);
  CK(ctx->pair_q.ensure(ctx->n_pairs));
  CK(ctx->pair_i.ensure(ctx->n_pairs));
  CK(ctx->pq_rank.ensure(ctx->n_pairs));
  D = mesh_view(ctx);
  CK(launch_pair_fill(D, ctx->pair_off.p, ctx->pair_q.p, ctx->pair_i.p, st));
  CK(ctx->qcount.ensure(nq));
  CK(ctx->qpair_ptr.ensure(nq + 1));
  CK(launch_qpair_count(D, ctx->qcount.p, st));
  CK(exclusive_scan<int>(ctx->qcount.p, ctx->qpair_ptr.p, nq, ctx->qpair_ptr.p + nq, ctx->scratch.p,
                         ctx->scratch.n, st));
  D = mesh_view(ctx);
  CK(launch_qpair_fill(D, ctx->pq_rank.p, st));
  CK(tm.stop(st));
  CK(cudaStreamSynchronize(st));
  CK(tm.collect());
  ephb_mesh_info info;
  info.ms = tm.ms;
  info.nk = nk;
  info.nq = nq;
  info.n_active_states = host_scal[1];
  info.n_ibz = host_scal[2];
  info.n_ibz_window = ctx->n_ibzw;
  info.n_pairs = ctx->n_pairs;
  ctx->minfo = info;
  if (out) *out = info;
  ctx->stage = 2;
  ctx->bte_ready = false;
  return EPHB_OK;
}

// ---------------------------------------------------------------------------------------
namespace {

// Put instance i in the InstState base; the one there goes back to its slot.
void select_instance(ephb_ctx *ctx, int i) {
  if (i == ctx->cur) return;
  InstState &base = *ctx;
  std::swap(base, ctx->slots[ctx->cur]);
  std::swap(base, ctx->slots[i]);
  ctx->cur = i;
}

// n instances, every one without a solution; instance 0 in the base
void set_instances(ephb_ctx *ctx, int n) {
  select_instance(ctx, 0);
  while (int(ctx->slots.size()) > n) {
    ctx->slots.back().release_all();
    ctx->slots.pop_back();
  }
  ctx->slots.resize(n);
  ctx->ninst = n;
  ctx->bte_ready = ctx->has_warm = ctx->solved = false;
  for (int i = 1; i < n; ++i) ctx->slots[i].bte_ready = ctx->slots[i].has_warm = ctx->slots[i].solved = false;
}

// The lists just computed (vertex-only) become the union lists; each instance then takes the
// entries of its window with its occupation factors.
// The lists of the instance in the base from the union lists: its window, T and mu are set.
ephb_status derive_one(ephb_ctx *ctx) {
  cudaStream_t st = ctx->stream;
  const ModelDev &M = ctx->M;
  const int64_t nst = ctx->n_ibzw * M.nb, nph = ctx->qm.size() * M.nbr;
  ctx->n_tuples = ctx->u_tuples;
  ctx->bte_ready = false;
  MeshDev D = mesh_view(ctx);
  const InstWindow w{ctx->win_lo, ctx->win_hi};
  CK(launch_epi_tables(M, D, ctx->T, ctx->mu, ctx->fk.p, ctx->nbq.p, ctx->wr.p, ctx->ut.p, st));
  CK(launch_inst_count(M, D, w, ctx->u_row_ptr.p, ctx->u_kpns.p, ctx->u_ph_row_ptr.p, ctx->u_ph_st.p,
                       ctx->u_ph_kpn.p, ctx->cntE.p, ctx->cntPh.p, st));
  CK(ctx->row_ptr.ensure(nst + 1));
  CK(ctx->ph_row_ptr.ensure(nph + 1));
  CK(exclusive_scan<int>(ctx->cntE.p, ctx->row_ptr.p, nst, ctx->scal.p + 3, ctx->scratch.p, ctx->scratch.n, st));
  CK(exclusive_scan<int>(ctx->cntPh.p, ctx->ph_row_ptr.p, nph, ctx->scal.p + 4, ctx->scratch.p, ctx->scratch.n,
                         st));
  CK(cudaMemcpyAsync(ctx->row_ptr.p + nst, ctx->scal.p + 3, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(ctx->ph_row_ptr.p + nph, ctx->scal.p + 4, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  int64_t hs[2];
  CK(cudaMemcpyAsync(hs, ctx->scal.p + 3, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->n_entries = hs[0];
  ctx->n_ph_entries = hs[1];
  CK(ctx->e_kpns.ensure(ctx->n_entries));
  CK(ctx->e_X.ensure(ctx->n_entries));
  CK(ctx->ph_st.ensure(ctx->n_ph_entries));
  CK(ctx->ph_kpn.ensure(ctx->n_ph_entries));
  CK(ctx->ph_Y.ensure(ctx->n_ph_entries));
  CK(launch_inst_fill(M, D, w, ctx->fk.p, ctx->nbq.p, ctx->u_row_ptr.p, ctx->u_kpns.p, ctx->u_X.p,
                      ctx->u_ph_row_ptr.p, ctx->u_ph_st.p, ctx->u_ph_kpn.p, ctx->u_ph_V.p, ctx->row_ptr.p,
                      ctx->ph_row_ptr.p, ctx->e_kpns.p, ctx->e_X.p, ctx->ph_st.p, ctx->ph_kpn.p, ctx->ph_Y.p, st));
  ctx->lists_pending = false;
  return EPHB_OK;
}

// Entries of the electron and phonon lists of the instance in the base (its window), counted
// from the union lists without writing them.
ephb_status count_one(ephb_ctx *ctx, int64_t &ne, int64_t &nphe) {
  cudaStream_t st = ctx->stream;
  const ModelDev &M = ctx->M;
  const int64_t nst = ctx->n_ibzw * M.nb, nph = ctx->qm.size() * M.nbr;
  MeshDev D = mesh_view(ctx);
  const InstWindow w{ctx->win_lo, ctx->win_hi};
  CK(launch_inst_count(M, D, w, ctx->u_row_ptr.p, ctx->u_kpns.p, ctx->u_ph_row_ptr.p, ctx->u_ph_st.p,
                       ctx->u_ph_kpn.p, ctx->cntE.p, ctx->cntPh.p, st));
  CK(ctx->escan.ensure(nst + 1));
  CK(ctx->phscan.ensure(nph + 1));
  CK(exclusive_scan<int>(ctx->cntE.p, ctx->escan.p, nst, ctx->scal.p + 3, ctx->scratch.p, ctx->scratch.n, st));
  CK(exclusive_scan<int>(ctx->cntPh.p, ctx->phscan.p, nph, ctx->scal.p + 4, ctx->scratch.p, ctx->scratch.n, st));
  int64_t hs[2];
  CK(cudaMemcpyAsync(hs, ctx->scal.p + 3, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ne = hs[0];
  nphe = hs[1];
  return EPHB_OK;
}

// The lists just computed (vertex-only) become the union lists; each instance then takes the
// entries of its window with its occupation factors.  When the instances' lists together would
// not fit the free device memory (their entry counts with the solve's working arrays), each
// instance keeps only its window, T and mu here and derives its lists when it is solved; after
// its solve the lists and sweep arrays are released again (the responses, rates and
// coefficient inputs stay).
ephb_status derive_instances(ephb_ctx *ctx, const ephb_thermo *inst, int ninst) {
  const ModelDev &M = ctx->M;
  const int64_t nst = ctx->n_ibzw * M.nb, nph = ctx->qm.size() * M.nbr;
  std::swap(ctx->u_row_ptr, ctx->row_ptr);
  std::swap(ctx->u_ph_row_ptr, ctx->ph_row_ptr);
  std::swap(ctx->u_kpns, ctx->e_kpns);
  std::swap(ctx->u_ph_kpn, ctx->ph_kpn);
  std::swap(ctx->u_X, ctx->e_X);
  std::swap(ctx->u_ph_st, ctx->ph_st);
  std::swap(ctx->u_ph_V, ctx->ph_Y);
  ctx->u_entries = ctx->n_entries;
  ctx->u_ph_entries = ctx->n_ph_entries;
  ctx->u_tuples = ctx->n_tuples;
  CK(ctx->cntE.ensure(nst > 0 ? nst : 1));
  CK(ctx->cntPh.ensure(nph > 0 ? nph : 1));
  CK(ctx->scratch.ensure(scan_scratch_elems(nst > nph ? nst : nph)));
  CK(ctx->fk.ensure(size_t(ctx->km.size()) * M.nb));
  CK(ctx->nbq.ensure(size_t(nph)));
  CK(ctx->wr.ensure(size_t(nph)));
  CK(ctx->ut.ensure(size_t(nph) * M.nbr));
  // per instance: lists (20 B per electron entry, 16 B per phonon entry), sweep arrays and
  // run scratch (~28 B per electron entry) and the mixed iteration's FP32 and float-float
  // copies of the rates (24 B per electron entry, 12 B per phonon entry)
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  double need = 0.0;
  for (int i = 0; i < ninst; ++i) {
    select_instance(ctx, i);
    ctx->T = inst[i].T_K;
    ctx->mu = inst[i].mu_eV;
    const bool own = inst[i].window_lo_eV < inst[i].window_hi_eV;
    ctx->win_lo = own ? std::max(inst[i].window_lo_eV, ctx->lo) : ctx->lo;
    ctx->win_hi = own ? std::min(inst[i].window_hi_eV, ctx->hi) : ctx->hi;
    ctx->n_tuples = ctx->u_tuples;
    ctx->bte_ready = false;
    ctx->lists_pending = true;
    if (ninst > 1 && !ctx->force_defer) {
      int64_t ne = 0, nphe = 0;
      ephb_status r = count_one(ctx, ne, nphe);
      if (r != EPHB_OK) return r;
      need += 72.0 * double(ne) + 36.0 * double(nphe);
    }
  }
  const bool defer = ninst > 1 && (ctx->force_defer || need > 0.5 * double(free_b));
  for (int i = 0; i < ninst; ++i) {
    select_instance(ctx, i);
    if (!defer) {
      ephb_status r = derive_one(ctx);
      if (r != EPHB_OK) return r;
    }
  }
  ctx->deferred = defer;
  select_instance(ctx, 0);
  return EPHB_OK;
}

}  // namespace

ephb_status ephb_compute_transition_rates(ephb_ctx *ctx, const ephb_thermo *inst, int ninst, const ephb_delta *delta,
                                          ephb_precision precision, ephb_rates_info *out) {
  if (!ctx) return EPHB_EINVAL;
  if (ctx->stage < 2) return fail(ctx, EPHB_ESTATE, "build_meshes_ibz must come first");
  if (!inst || !delta) return fail(ctx, EPHB_EINVAL, "NULL argument");
  if (ninst < 1 || ninst > EPHB_MAX_INSTANCES) return fail(ctx, EPHB_EINVAL, "ninst out of range");
  if (precision != EPHB_FP64 && precision != EPHB_FP64_SLICED && precision != EPHB_SPLIT_BF16)
    return fail(ctx, EPHB_EINVAL, "precision must be EPHB_FP64, EPHB_FP64_SLICED or EPHB_SPLIT_BF16");
  if (delta->kind != EPHB_DELTA_GAUSS && delta->kind != EPHB_DELTA_TETRA)
    return fail(ctx, EPHB_EINVAL, "delta kind must be EPHB_DELTA_GAUSS or EPHB_DELTA_TETRA");
  if (delta->kind == EPHB_DELTA_GAUSS && (!(delta->sigma_eV > 0) || !(delta->cutoff_sigmas > 0)))
    return fail(ctx, EPHB_EINVAL, "sigma and cutoff must be positive");
  ctx->delta_sigma = delta->sigma_eV;
  ctx->delta_cut = delta->cutoff_sigmas;
  // exact FP32 sums of the accumulated slice diagonals bound the contraction length
  if (precision == EPHB_FP64_SLICED && tc_slices_for(tc_kp(ctx->M), true) == 0)
    return fail(ctx, EPHB_EINVAL, "EPHB_FP64_SLICED needs 2 nRgp <= 816");
  if (precision == EPHB_SPLIT_BF16 && tc_slices_for(tc_kp(ctx->M), false) == 0)
    return fail(ctx, EPHB_EINVAL, "EPHB_SPLIT_BF16 needs 2 nRgp <= 1024");
  bool windowed = false;
  for (int i = 0; i < ninst; ++i) {
    if (!(inst[i].T_K > 0)) return fail(ctx, EPHB_EINVAL, "T must be positive");
    if (inst[i].window_lo_eV < inst[i].window_hi_eV &&
        (inst[i].window_lo_eV > ctx->lo || inst[i].window_hi_eV < ctx->hi))
      windowed = true;
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const ModelDev &M = ctx->M;
  const int nb = M.nb, nbr = M.nbr;
  const int64_t nq = ctx->qm.size();
  // several instances (or a window narrower than the meshes'): one T-independent vertex pass
  // over the mesh window, then the rate lists of every instance from it
  const bool multi = ninst > 1 || windowed;
  ctx->deferred = false;
  set_instances(ctx, ninst);
  ctx->T = inst->T_K;
  ctx->mu = inst->mu_eV;
  ctx->win_lo = ctx->lo;
  ctx->win_hi = ctx->hi;
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  RateParams rp;
  rp.T = inst->T_K;
  rp.mu = inst->mu_eV;
  rp.tetra = delta->kind == EPHB_DELTA_TETRA ? 1 : 0;
  const double sig = rp.tetra ? 1.0 : delta->sigma_eV;   // unused with the tetrahedron weights
  rp.sigma = sig;
  rp.cut = rp.tetra ? 0.0 : delta->cutoff_sigmas * sig;
  rp.inv_sigma = 1.0 / sig;
  rp.gnorm = 1.0 / (sig * std::sqrt(2.0 * kPi));
  auto ff_split = [](double v) {
    const float h = float(v);
    return make_float2(h, float(v - double(h)));
  };
  rp.inv_sigma_ff = ff_split(rp.inv_sigma);
  rp.gnorm_ff = ff_split(rp.gnorm);
  rp.inv_Nq_pref = 2.0 * kPi / (kHbarEVs * double(nq));
  rp.y_scale = double(nq) / double(ctx->km.size());
  rp.vertex_only = multi ? 1 : 0;
  rp.rot_fp32 = precision == EPHB_SPLIT_BF16 ? 1 : 0;   // mixed mode: FP32 rotations in the epilogue
  const int64_t np = ctx->n_pairs;
  CK(ctx->cntE.ensure(np * nb));
  CK(ctx->cntPh.ensure(np * nbr));
  CK(ctx->escan.ensure(np * nb));
  CK(ctx->phscan.ensure(np * nbr));
  CK(ctx->ucount.ensure(8));
  MeshDev D = mesh_view(ctx);
  // FP32 copies of the energies for the FP32 estimate of the delta-cutoff decisions
  CK(ctx->eps32.ensure(size_t(ctx->km.size()) * nb));
  CK(ctx->w32.ensure(size_t(nq) * nbr));
  CK(launch_to_f32(int64_t(ctx->km.size()) * nb, ctx->eps.p, ctx->eps32.p, st));
  CK(launch_to_f32(int64_t(nq) * nbr, ctx->w.p, ctx->w32.p, st));
  rp.eps32 = ctx->eps32.p;
  rp.w32 = ctx->w32.p;
  CK(launch_rate_count(M, D, rp, ctx->cntE.p, ctx->cntPh.p, ctx->ucount.p, st));
  int64_t big = np * (nb > nbr ? nb : nbr);
  CK(ctx->scratch.ensure(scan_scratch_elems(big)));
  CK(exclusive_scan<int>(ctx->cntE.p, ctx->escan.p, np * nb, ctx->scal.p + 3, ctx->scratch.p, ctx->scratch.n, st));
  CK(exclusive_scan<int>(ctx->cntPh.p, ctx->phscan.p, np * nbr, ctx->scal.p + 4, ctx->scratch.p, ctx->scratch.n,
                         st));
  int64_t hs[2];
  unsigned long long ntup = 0;
  CK(cudaMemcpyAsync(hs, ctx->scal.p + 3, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ntup, ctx->ucount.p, sizeof(ntup), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->n_entries = hs[0];
  ctx->n_ph_entries = hs[1];
  ctx->n_tuples = int64_t(ntup);
  CK(ctx->e_kpns.ensure(ctx->n_entries));
  CK(ctx->e_X.ensure(ctx->n_entries));
  CK(ctx->ph_st.ensure(ctx->n_ph_entries));
  CK(ctx->ph_kpn.ensure(ctx->n_ph_entries));
  CK(ctx->ph_Y.ensure(ctx->n_ph_entries));
  CK(ctx->row_ptr.ensure(ctx->n_ibzw * nb + 1));
  CK(ctx->ph_row_ptr.ensure(nq * nbr + 1));
  CK(launch_row_ptrs(D, nb, nbr, ctx->escan.p, ctx->phscan.p, ctx->n_entries, ctx->n_ph_entries, ctx->row_ptr.p,
                     ctx->ph_row_ptr.p, st));
  // stage A / B in chunks of irreducible-window k points
  const size_t per_k = stage_a_T_elems(M);
  int64_t chunk = int64_t((size_t(3) << 29) / (2 * per_k * sizeof(double2)));
  if (chunk < 1) chunk = 1;
  if (chunk > ctx->n_ibzw) chunk = ctx->n_ibzw;
  if (chunk > 0) {
    CK(ctx->Tbuf.ensure(size_t(chunk) * per_k));
    CK(ctx->Abuf.ensure(size_t(chunk) * stage_a_A_elems(M)));
  }
  EventTimer ta, tb, tc, tg;
  CK(ta.init());
  CK(tb.init());
  CK(tc.init());
  CK(tg.init());
  const bool tensor = precision != EPHB_FP64;
  const int ns = tensor ? tc_slices_for(tc_kp(M), precision == EPHB_FP64_SLICED) : 0;
  const int tslot = ns == 8 ? 2 : (ns == 7 ? 0 : 1);   // tuned tile shape per slicing (4 slices: 1)
  const int ncm = tensor && ctx->force_cols ? std::min(ctx->force_cols, tc_nc_max(ns)) : 0;   // 0: tuned width
  int autotuned = 0;
  // stage A on the tensor cores too, always in the FP64-grade form (its error would add to the
  // mixed mode's), while its contraction length keeps the diagonal sums exact
  const int ns_a = tc_slices_for(tc_kp_a(M), true);
  const bool tensor_a = tensor && ns_a != 0;
  double tensor_flops_a = 0.0;
  std::vector<int64_t> hpp;
  int Nmax = 0;
  const int64_t kMaxChunkPairs = 1 << 20;   // bound of the contraction scratch (pairs x Nmax doubles)
  if (tensor) {
    // phase slices of the whole q mesh, the pair pointers (to bound chunks by pairs) and scratch
    Nmax = tc_nmax(M);
    const int Kp = tc_kp(M);
    CK(ctx->phis.ensure(size_t(nq) * ns * Kp));
    CK(ctx->angle_tab.ensure(size_t(2) * 1024 * 8));
    CK(launch_phase_slices(M, D, ns, ctx->phis.p, ctx->angle_tab.p, st));
    hpp.resize(ctx->n_ibzw + 1);
    CK(cudaMemcpyAsync(hpp.data(), ctx->pair_ptr.p, hpp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(ctx->bslices.ensure(size_t(chunk) * ns * Nmax * Kp));
    CK(ctx->bscale.ensure(size_t(chunk) * Nmax));
    CK(ctx->nitem.ensure(chunk));
    CK(ctx->item_ptr.ensure(chunk));
    CK(ctx->Cbuf.ensure(size_t(std::min<int64_t>(np, kMaxChunkPairs)) * Nmax));
    // work items of a chunk: at most (pairs / 128 + k points) tiles, each in at most Nmax / 16
    // column chunks
    ctx->ws_cap = (std::min<int64_t>(np, kMaxChunkPairs) / 128 + chunk) * ((Nmax + 15) / 16);
    CK(ctx->ws_desc.ensure(size_t(ctx->ws_cap) * 4));
    CK(ctx->tc_err.ensure(1));
    if (tensor_a) {   // g slices once per model; k phase slices per chunk
      const size_t gsz = tc_gs_elems_a(M, ns_a);
      if (ctx->gslices_ns != ns_a || ctx->gslices.n < gsz) {
        CK(ctx->gslices.ensure(gsz));
        CK(ctx->gscale.ensure(tc_ncols_a(M)));
        CK(launch_g_slices(M, ns_a, ctx->gslices.p, ctx->gscale.p, st));
        ctx->gslices_ns = ns_a;
      }
      CK(ctx->phik.ensure(stage_a_phik_elems(M, ns_a, chunk)));
    }
    CK(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), st));
    CK(cudaMemsetAsync(ctx->scal.p + 7, 0, sizeof(int64_t), st));
    CK(ctx->scratch.ensure(scan_scratch_elems(chunk > big ? chunk : big)));
    // occupation / prefactor / eigenvector tables of the rate epilogue
    CK(ctx->fk.ensure(size_t(ctx->km.size()) * nb));
    CK(ctx->nbq.ensure(size_t(nq) * nbr));
    CK(ctx->wr.ensure(size_t(nq) * nbr));
    CK(ctx->ut.ensure(size_t(nq) * nbr * nbr));
    CK(launch_epi_tables(M, D, rp.T, rp.mu, ctx->fk.p, ctx->nbq.p, ctx->wr.p, ctx->ut.p, st));
    if (tensor) {
      CK(ctx->cff.ensure(size_t(ctx->km.size()) * M.nb * M.nb));
      CK(ctx->uff.ensure(size_t(ctx->qm.size()) * M.nbr * M.nbr));
      CK(launch_ff_tables(M, D, ctx->ut.p, ctx->cff.p, ctx->uff.p, st));
    }
  }
  // Stage A runs on groups of up to `chunk` k points (all of them when the buffers allow), so
  // its contraction sees many k tiles per launch; stage B then walks the group in sub-chunks
  // whose pairs fit the contraction scratch, reading the group's stage-A output at its offset.
  int64_t a0 = 0, a_end = 0;
  for (int64_t i0 = 0; i0 < ctx->n_ibzw;) {
    if (i0 >= a_end) {
      a0 = i0;
      a_end = ctx->n_ibzw - i0 < chunk ? ctx->n_ibzw : i0 + chunk;
      const int64_t na = a_end - a0;
      CK(ta.start(st));
      if (tensor_a) {
        CK(launch_stage_a_tc(M, D, ns_a, a0, na, ctx->phik.p, ctx->gslices.p, ctx->gscale.p, ctx->Tbuf.p,
                             ctx->tc_err.p, ctx->stage_a_tmem != 0, st, &tensor_flops_a));
        CK(launch_stage_a2(M, D, a0, na, ctx->Tbuf.p, ctx->Abuf.p, true, st));
      } else {
        CK(launch_stage_a(M, D, a0, na, ctx->Tbuf.p, ctx->Abuf.p, st));
      }
      CK(ta.stop(st));
    }
    int64_t nkc = a_end - i0;
    if (tensor) {   // also keep the chunk's pairs within the contraction scratch
      while (nkc > 1 && hpp[i0 + nkc] - hpp[i0] > kMaxChunkPairs) nkc = (nkc + 1) / 2;
      if (hpp[i0 + nkc] - hpp[i0] > kMaxChunkPairs)
        return fail(ctx, EPHB_EINVAL, "one irreducible k has more pairs than the contraction scratch holds");
    }
    const double2 *Achunk = ctx->Abuf.p + size_t(i0 - a0) * stage_a_A_elems(M);
    CK(tb.start(st));
    if (!tensor) {
      CK(launch_stage_b_rates(M, D, rp, i0, nkc, Achunk, ctx->escan.p, ctx->phscan.p, ctx->e_kpns.p,
                              ctx->e_X.p, ctx->ph_st.p, ctx->ph_kpn.p, ctx->ph_Y.p, st));
      CK(tb.stop(st));
    } else {
      auto contract = [&](cudaEvent_t e0, cudaEvent_t e1, int width, int kc, int stages) {
        return launch_vertex_tc(M, D, ns, i0, nkc, hpp[i0], Achunk, ctx->phis.p, ctx->bslices.p,
                                ctx->bscale.p, ctx->nitem.p, ctx->item_ptr.p, ctx->scratch.p, ctx->scratch.n,
                                ctx->scal.p + 6, ctx->Cbuf.p, ctx->tc_err.p, st, e0, e1, width, kc, stages,
                                ctx->withhold_mma, ctx->ws_desc.p, ctx->ws_cap);
      };
      int &tuned = ctx->tune_cols[tslot];
      int &tuned_kc = ctx->tune_kc[tslot];
      int &tuned_st = ctx->tune_st[tslot];
      if (ncm == 0 && tuned == 0) {
        // autotune on this chunk: time the GEMM at every candidate tile shape and keep the
        // fastest (the contraction is the same for every shape, so the last run stands)
        float best = 3.4e38f;
        for (const TcShape &sh : tc_shape_candidates(ns)) {
          EventTimer tt;
          CK(tt.init());
          CK(contract(tt.a, tt.b, sh.width, sh.kc, sh.stages));
          tt.pending = true;
          CK(cudaStreamSynchronize(st));
          CK(tt.collect());
          if (tt.ms < best) {
            best = float(tt.ms);
            tuned = sh.width;
            tuned_kc = sh.kc;
            tuned_st = sh.stages;
          }
        }
        autotuned = 1;
      } else {
        CK(contract(tg.a, tg.b, ncm ? ncm : tuned, ncm ? 32 : tuned_kc, ncm ? 2 : tuned_st));
        tg.pending = true;
      }
      CK(tb.stop(st));
      CK(tc.start(st));
      CK(launch_vertex_epilogue(M, D, rp, hpp[i0], hpp[i0 + nkc], hpp[i0], ctx->Cbuf.p, Nmax, ctx->fk.p,
                                ctx->nbq.p, ctx->wr.p, ctx->ut.p, ctx->cff.p, ctx->uff.p, ctx->escan.p,
                                ctx->phscan.p, ctx->e_kpns.p, ctx->e_X.p, ctx->ph_st.p, ctx->ph_kpn.p, ctx->ph_Y.p,
                                st));
      CK(tc.stop(st));
    }
    CK(cudaStreamSynchronize(st));
    CK(ta.collect());
    CK(tb.collect());
    CK(tc.collect());
    CK(tg.collect());
    i0 += nkc;
  }
  double tensor_flops = 0.0;
  if (tensor) {
    int herr = 0;
    int64_t tfl = 0;
    CK(cudaMemcpyAsync(&herr, ctx->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tfl, ctx->scal.p + 7, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) return fail(ctx, EPHB_ETIMEOUT, "a tensor-core wait gave up (vertex contraction)");
    tensor_flops = double(tfl);
  }
  unsigned long long cnt[5];
  CK(cudaMemcpyAsync(cnt, ctx->ucount.p, sizeof(cnt), cudaMemcpyDeviceToHost, st));
  if (multi) {
    ephb_status r = derive_instances(ctx, inst, ninst);
    if (r != EPHB_OK) return r;
  }
  CK(cudaEventRecord(ev1, st));
  CK(cudaEventSynchronize(ev1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (out) {
    out->n_tuples = ctx->n_tuples;
    out->n_entries = ctx->n_entries;
    out->n_ph_entries = ctx->n_ph_entries;
    out->n_pairs = np;
    out->ms = ms;
    out->ms_stage_a = ta.ms;
    out->ms_stage_b = tb.ms;
    const double ncol = double(M.nRgp) * M.nb * M.nb * M.nbr;
    out->stage_a_flops = 8.0 * double(ctx->n_ibzw) * M.nRge * ncol + 8.0 * double(cnt[3]) * ncol;
    out->stage_b_flops = double(cnt[2]);
    out->ms_epilogue = tc.ms;
    out->tensor_flops = tensor_flops;
    out->tensor_flops_a = tensor_flops_a;
    out->rot_flops = double(cnt[4]);
    out->ms_gemm = tg.ms;
    out->tc_cols = tensor ? (ncm ? ncm : ctx->tune_cols[tslot]) : 0;
    out->tc_kblock = tensor ? (ncm ? 32 : ctx->tune_kc[tslot]) : 0;
    out->tc_stages = tensor ? (ncm ? 2 : ctx->tune_st[tslot]) : 0;
    out->autotuned = autotuned;
  }
  ctx->stage = 3;
  return EPHB_OK;
}

// ---------------------------------------------------------------------------------------
namespace {

ephb_status bte_setup(ephb_ctx *ctx) {
  const ModelDev &M = ctx->M;
  cudaStream_t st = ctx->stream;
  const int64_t nst = ctx->n_ibzw * M.nb, nph = ctx->qm.size() * M.nbr, nk = ctx->km.size();
  CK(ctx->st_eps.ensure(nst));
  CK(ctx->st_vel.ensure(nst * 3));
  CK(ctx->st_ff.ensure(nst));
  CK(ctx->st_wt.ensure(nst));
  CK(ctx->kcrd.ensure(nk));
  CK(ctx->kinfo.ensure(nk));
  CK(ctx->W_e.ensure(nst));
  CK(ctx->inv_ffW.ensure(nst));
  for (auto *b : {&ctx->I0, &ctx->J0, &ctx->I, &ctx->J, &ctx->I2, &ctx->J2}) CK(b->ensure(nst * 3));
  CK(ctx->Bt.ensure(nph));
  CK(ctx->W_ph.ensure(nph));
  CK(ctx->inv_nnW.ensure(nph));
  for (auto *b : {&ctx->F0, &ctx->F, &ctx->G}) CK(b->ensure(nph * 3));
  CK(ctx->Btv.ensure(nph * 6));
  CK(ctx->Afold.ensure(size_t(ctx->n_qrep > 0 ? ctx->n_qrep : 1) * M.nbr * 6));
  CK(ctx->epart.ensure(size_t(coeff_partials()) * 36));
  CK(ctx->ppart.ensure(size_t(coeff_partials()) * 18));
  CK(ctx->kpart.ensure(size_t(coeff_partials()) * 9));
  for (auto *b : {&ctx->res, &ctx->prev_in, &ctx->prev_out, &ctx->prev_tmp}) CK(b->ensure(kResLen));
  CK(ctx->sctl.ensure(4));
  MeshDev D = mesh_view(ctx);
  CK(launch_state_setup(M, D, ctx->T, ctx->mu, ctx->win_lo, ctx->win_hi, ctx->st_eps.p, ctx->st_vel.p, ctx->st_ff.p, ctx->st_wt.p,
                        ctx->kcrd.p, ctx->kinfo.p, st));
  BteDev B = bte_view(ctx);
  CK(ctx->nzero.ensure(1));
  CK(cudaMemsetAsync(ctx->nzero.p, 0, sizeof(unsigned long long), st));
  const double *W_add = nullptr;
  if (ctx->imp.n_species > 0) {   // e-chimp rates join W^RTA (Matthiessen's rule)
    if (!(ctx->delta_sigma > 0) || !(ctx->delta_cut > 0))
      return fail(ctx, EPHB_EINVAL, "charged impurities need the Gaussian width of the rates call");
    CK(ctx->W_chimp.ensure(nst));
    CK(ctx->chimp_part.ensure(size_t(chimp_partials())));
    CK(ctx->chimp_qtf.ensure(1));
    const double *L = M.lattice;   // rows: the lattice vectors (Angstrom)
    const double det3 = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                        L[2] * (L[3] * L[7] - L[4] * L[6]);
    const double V = fabs(det3) * kAngstrom * kAngstrom * kAngstrom;
    ChimpParams cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.nspec = ctx->imp.n_species;
    for (int i = 0; i < cp.nspec; ++i) {
      cp.n_m3[i] = ctx->imp.n_cm3[i] * 1e6;
      cp.Z[i] = ctx->imp.Z[i];
    }
    cp.eps_r = ctx->imp.eps_r;
    cp.V = V;
    // reciprocal vectors (1/m): the rows of 2 pi (L^-1)^T, (L^-1)^T[r][c] = cofactor(r, c) / det L
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        const double cof = L[r1 * 3 + c1] * L[r2 * 3 + c2] - L[r1 * 3 + c2] * L[r2 * 3 + c1];
        cp.rec[r][c] = 2.0 * kPi * cof / det3 / kAngstrom;
      }
    cp.sigma = ctx->delta_sigma;
    cp.cut_sigmas = ctx->delta_cut;
    cp.gnorm = 1.0 / (ctx->delta_sigma * sqrt(2.0 * kPi));
    cp.pref = 2.0 * kPi / (kHbarEVs * double(nk));
    cp.win_lo = ctx->win_lo;
    cp.win_hi = ctx->win_hi;
    const double kT_J = kKbEVK * kECharge * ctx->T;
    const double ff_scale = M.spin_deg * kECharge * kECharge / (kT_J * double(nk) * V * 8.8541878128e-12 * cp.eps_r);
    CK(launch_chimp_rates(D, B, cp, ctx->eps.p, nk * M.nb, ff_scale, ctx->chimp_part.p, ctx->chimp_qtf.p,
                          ctx->W_chimp.p, st));
    W_add = ctx->W_chimp.p;
  }
  CK(launch_rta_electron(B, ctx->W_e.p, ctx->inv_ffW.p, ctx->I0.p, ctx->J0.p, ctx->nzero.p, st, W_add));
  CK(launch_ph_rowsum(B, ctx->Bt.p, st));
  const double *W_ph_add = nullptr;
  if (ctx->iso_nat > 0) {   // ph-isotope rates join W^RTA_sq (Matthiessen's rule)
    if (ctx->iso_nat != M.nat) return fail(ctx, EPHB_EINVAL, "isotope parameters for a different number of atoms");
    if (!(ctx->delta_sigma > 0) || !(ctx->delta_cut > 0))
      return fail(ctx, EPHB_EINVAL, "isotope scattering needs the Gaussian width of the rates call");
    CK(ctx->W_iso.ensure(nph));
    CK(ctx->W_iso_rep.ensure(size_t(ctx->n_qrep > 0 ? ctx->n_qrep : 1) * M.nbr));
    IsoParams ip;
    std::memset(&ip, 0, sizeof(ip));
    for (int a = 0; a < ctx->iso_nat; ++a) ip.g[a] = ctx->iso_g[a];
    ip.sigma = ctx->delta_sigma;
    ip.cut_sigmas = ctx->delta_cut;
    ip.gnorm = 1.0 / (ctx->delta_sigma * sqrt(2.0 * kPi));
    ip.pref = kPi / (2.0 * kHbarEVs * double(ctx->qm.size()));
    CK(launch_iso_rates(M, D, ip, ctx->W_iso_rep.p, ctx->W_iso.p, st));
    W_ph_add = ctx->W_iso.p;
  }
  CK(launch_rta_phonon(M, D, B, ctx->Bt.p, ctx->W_ph.p, ctx->inv_nnW.p, ctx->F0.p, st, W_ph_add));
  // partner runs of the electron rows (self term), then segments of the entry stream
  // (drag term) and of the run stream (self term)
  const int64_t ne = ctx->n_entries;
  CK(ctx->run_flag.ensure(ne));
  CK(ctx->run_idx.ensure(ne));
  CK(ctx->run_ptr.ensure(nst + 1));
  CK(ctx->scratch.ensure(scan_scratch_elems(ne > nst ? ne : nst)));
  CK(launch_build_runs(B, ne, ctx->kinfo.p, ctx->run_flag.p, ctx->run_idx.p, ctx->scratch.p, ctx->scratch.n,
                       ctx->run_ptr.p, nullptr, nullptr, ctx->nruns, ctx->scal.p + 5, st));
  CK(ctx->run_col.ensure(ctx->nruns));
  CK(ctx->run_w.ensure(ctx->nruns));
  CK(launch_fill_runs(B, ne, ctx->nruns, ctx->kinfo.p, ctx->run_flag.p, ctx->run_idx.p, ctx->run_ptr.p,
                      ctx->run_col.p, ctx->run_w.p, st));
  CK(ctx->nseg_row.ensure(nst));
  CK(ctx->eseg_ptr.ensure(nst + 1));
  CK(ctx->rseg_ptr.ensure(nst + 1));
  CK(launch_build_segments(nst, ctx->row_ptr.p, ctx->nseg_row.p, ctx->eseg_ptr.p, ctx->scratch.p, ctx->scratch.n,
                           ctx->neseg, st));
  CK(ctx->eseg_row.ensure(ctx->neseg));
  CK(ctx->eseg_begin.ensure(ctx->neseg));
  CK(launch_fill_segments(nst, ctx->row_ptr.p, ctx->eseg_ptr.p, ctx->eseg_row.p, ctx->eseg_begin.p, st));
  CK(launch_build_segments(nst, ctx->run_ptr.p, ctx->nseg_row.p, ctx->rseg_ptr.p, ctx->scratch.p, ctx->scratch.n,
                           ctx->nrseg, st));
  CK(ctx->rseg_row.ensure(ctx->nrseg));
  CK(ctx->rseg_begin.ensure(ctx->nrseg));
  CK(launch_fill_segments(nst, ctx->run_ptr.p, ctx->rseg_ptr.p, ctx->rseg_row.p, ctx->rseg_begin.p, st));
  CK(ctx->pnseg_row.ensure(nph));
  CK(ctx->pseg_ptr.ensure(nph + 1));
  CK(ctx->scratch.ensure(scan_scratch_elems(nph)));
  CK(launch_build_segments(nph, ctx->ph_row_ptr.p, ctx->pnseg_row.p, ctx->pseg_ptr.p, ctx->scratch.p,
                           ctx->scratch.n, ctx->npseg, st));
  CK(ctx->pseg_row.ensure(ctx->npseg));
  CK(ctx->pseg_begin.ensure(ctx->npseg));
  CK(launch_fill_segments(nph, ctx->ph_row_ptr.p, ctx->pseg_ptr.p, ctx->pseg_row.p, ctx->pseg_begin.p, st));
  CK(ctx->pseg_part.ensure(size_t(ctx->npseg) * 6));
  CK(ctx->seg_part.ensure(size_t(ctx->neseg > ctx->nrseg ? ctx->neseg : ctx->nrseg) * 6));
  CK(ctx->Dterm.ensure(nst * 6));
  CK(cudaMemsetAsync(ctx->Dterm.p, 0, nst * 6 * sizeof(double), st));
  ctx->bte_ready = true;
  ctx->have_f32 = false;
  return EPHB_OK;
}

SweepSegs entry_segs(ephb_ctx *c) {
  SweepSegs S;
  std::memset(&S, 0, sizeof(S));
  S.nseg = c->neseg;
  S.seg_row = c->eseg_row.p;
  S.seg_begin = c->eseg_begin.p;
  S.seg_ptr = c->eseg_ptr.p;
  S.row_ptr = c->row_ptr.p;
  return S;
}

SweepSegs run_segs(ephb_ctx *c) {
  SweepSegs S;
  std::memset(&S, 0, sizeof(S));
  S.nseg = c->nrseg;
  S.seg_row = c->rseg_row.p;
  S.seg_begin = c->rseg_begin.p;
  S.seg_ptr = c->rseg_ptr.p;
  S.row_ptr = c->run_ptr.p;
  return S;
}

SweepSegs ph_segs(ephb_ctx *c) {
  SweepSegs S;
  std::memset(&S, 0, sizeof(S));
  S.nseg = c->npseg;
  S.seg_row = c->pseg_row.p;
  S.seg_begin = c->pseg_begin.p;
  S.seg_ptr = c->pseg_ptr.p;
  S.row_ptr = c->ph_row_ptr.p;
  return S;
}

// Recompute the requested partial sums, finalise the tensors against `prev` and read `res`.
ephb_status coefficients_to_host(ephb_ctx *ctx, double *prev, bool electron = true, bool phonon = true) {
  MeshDev D = mesh_view(ctx);
  BteDev B = bte_view(ctx);
  if (electron) CK(launch_e_partial(B, ctx->I.p, ctx->J.p, ctx->epart.p, ctx->stream));
  if (phonon)
    CK(launch_ph_partial(D, B, ctx->F.p, ctx->G.p, ctx->W_ph.p, ctx->inv_nnW.p, ctx->ppart.p, ctx->stream));
  CK(launch_coeff_final(ctx->M, B, ctx->epart.p, ctx->ppart.p, ctx->res.p, prev, ctx->stream));
  CK(cudaMemcpyAsync(ctx->host_res, ctx->res.p, kResLen * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return EPHB_OK;
}

}  // namespace

constexpr int kSweepBatch = 8;   // electron sweeps queued per host round trip
static_assert(kAndMaxSlots == EPHB_MAX_ACCEL_DEPTH + 1, "Anderson ring size");

namespace {

// Anderson weights over the n ring slots (newest: slot `head`) from their weighted Gram
// matrix H: alpha_head = 1 - sum gamma, alpha_j = gamma_j, gamma the least-squares solution of
// min |f_head - sum_j gamma_j (f_head - f_j)| (normal equations, partial pivoting, a 1e-12
// relative ridge).  False when the system is singular or the weights are out of bounds.
bool anderson_weights(const double (&H)[kAndMaxSlots][kAndMaxSlots], int n, int head, double *alpha) {
  int idx[kAndMaxSlots];
  int m = 0;
  for (int j = 0; j < n; ++j)
    if (j != head) idx[m++] = j;
  for (int j = 0; j < kAndMaxSlots; ++j) alpha[j] = 0.0;
  alpha[head] = 1.0;
  if (m == 0) return true;
  double A[kAndMaxSlots][kAndMaxSlots + 1];
  const double hh = H[head][head];
  double tr = 0.0;
  for (int a = 0; a < m; ++a) {
    for (int c = 0; c < m; ++c)
      A[a][c] = hh - H[head][idx[a]] - H[head][idx[c]] + H[idx[a]][idx[c]];
    A[a][m] = hh - H[head][idx[a]];
    tr += A[a][a];
  }
  if (!(tr > 0) || !std::isfinite(tr)) return false;
  for (int a = 0; a < m; ++a) A[a][a] += 1e-12 * tr / m;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (!(fabs(A[piv][c]) > 1e-14 * tr)) return false;
    if (piv != c)
      for (int k = 0; k <= m; ++k) std::swap(A[c][k], A[piv][k]);
    for (int r = c + 1; r < m; ++r) {
      const double fct = A[r][c] / A[c][c];
      for (int k = c; k <= m; ++k) A[r][k] -= fct * A[c][k];
    }
  }
  double gam[kAndMaxSlots];
  for (int r = m - 1; r >= 0; --r) {
    double v = A[r][m];
    for (int k = r + 1; k < m; ++k) v -= A[r][k] * gam[k];
    gam[r] = v / A[r][r];
  }
  double sg = 0.0, l1 = 0.0;
  for (int a = 0; a < m; ++a) {
    if (!std::isfinite(gam[a])) return false;
    sg += gam[a];
    l1 += fabs(gam[a]);
  }
  if (l1 > 1e3) return false;
  for (int a = 0; a < m; ++a) alpha[idx[a]] = gam[a];
  alpha[head] = 1.0 - sg;
  return true;
}

// The coupled solve of the instance in the InstState base.
ephb_status solve_one(ephb_ctx *ctx, const ephb_solve_opts *o, ephb_solve_info *out) {
  cudaStream_t st = ctx->stream;
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  ephb_status s = EPHB_OK;
  if (!ctx->bte_ready) {   // RTA terms, runs and segments depend on the rate lists only
    s = bte_setup(ctx);
    if (s != EPHB_OK) return s;
  }
  const ModelDev &M = ctx->M;
  const int64_t nst = ctx->n_ibzw * M.nb, nph = ctx->qm.size() * M.nbr;
  const double tol = o->tol, inner_tol = o->inner_tol > 0 ? o->inner_tol : 0.1 * o->tol;
  if (o->warm_start && ctx->has_warm) {   // learned start I = I0 + a_I k_B J0, J = J0 (1 + a_J)
    CK(launch_apply_warm(nst, ctx->I0.p, ctx->J0.p, ctx->warm.p, ctx->I.p, ctx->J.p, st));
  } else {
    CK(cudaMemcpyAsync(ctx->I.p, ctx->I0.p, nst * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->J.p, ctx->J0.p, nst * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaMemcpyAsync(ctx->F.p, ctx->F0.p, nph * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(ctx->G.p, 0, nph * 3 * sizeof(double), st));
  CK(cudaMemsetAsync(ctx->prev_out.p, 0, kResLen * sizeof(double), st));
  s = coefficients_to_host(ctx, ctx->prev_out.p);   // RTA; prev_out <- RTA tensors
  if (s != EPHB_OK) return s;
  MeshDev D = mesh_view(ctx);
  BteDev B = bte_view(ctx);
  int outer = 0, inner_total = 0;
  int64_t sweeps = 0;
  bool converged = o->level == EPHB_RTA;
  double residual = 0.0, lambda = 1.0;
  bool outer_seen = false;   // an outer residual exists (mixed precision's inexact inner solves)
  double last_tol_k = 0.0;   // tolerance of the last electron loop (mixed precision)
  EventTimer te, tp, td;
  EventTimer tsw[kSweepBatch];   // the self-term kernel of each queued sweep
  EventTimer tc32;               // FP32 correction sweeps (mixed precision)
  int64_t sweeps32 = 0;
  CK(tc32.init());
  CK(te.init());
  CK(tp.init());
  CK(td.init());
  for (auto &t : tsw) CK(t.init());

  // Mixed precision: each FP64 sweep x' = b + A x gives the residual (and the convergence test,
  // the same as the plain loop's); then kCorrSweeps FP32 sweeps of d <- r + A d, r = x' - x,
  // and x <- x + d, before the next FP64 sweep.
  // Mixed precision, dragged level: while the outer residual is above kPh32Until the phonon
  // scatter and the drag term run in FP32 (their error is far below the residual of those
  // iterations); the solve ends only after an outer iteration with both in FP64.
  const bool ph32_allowed = o->precision == EPHB_SOLVE_MIXED && o->level == EPHB_DRAGGED;
  bool ph32 = false;
  int outer32 = 0;
  if (ph32_allowed) {
    CK(ctx->X32.ensure(ctx->n_entries));
    CK(ctx->Y32.ensure(ctx->n_ph_entries));
    CK(ctx->IJ32.ensure(nst * 6));
    CK(ctx->FG32.ensure(nph * 6));
    CK(launch_copy_f32(2 * ctx->n_entries, reinterpret_cast<const double *>(ctx->e_X.p),
                       reinterpret_cast<float *>(ctx->X32.p), st));
    CK(launch_copy_f32(ctx->n_ph_entries, ctx->ph_Y.p, ctx->Y32.p, st));
    CK(ctx->Xff.ensure(ctx->n_entries));
    CK(ctx->Yff.ensure(ctx->n_ph_entries));
    CK(ctx->IJff.ensure(nst * 6));
    CK(ctx->FGff.ensure(nph * 6));
    CK(launch_copy_ff(2 * ctx->n_entries, reinterpret_cast<const double *>(ctx->e_X.p),
                      reinterpret_cast<float2 *>(ctx->Xff.p), st));
    CK(launch_copy_ff(ctx->n_ph_entries, ctx->ph_Y.p, ctx->Yff.p, st));
  }

  // Anderson acceleration (dragged level): ring of the last m+1 phonon updates g_j and
  // residuals f_j = g_j - x_j over x = (F, G); from the third outer iteration on the electrons
  // are solved against x = sum_j alpha_j g_j, alpha minimising |sum_j alpha_j f_j| (F and G
  // halves weighted by the first residual's) subject to sum_j alpha_j = 1.
  const int and_m = o->level == EPHB_DRAGGED ? o->accel_depth : 0;
  const int and_R = and_m + 1;
  const int64_t half = nph * 3;
  int and_n = 0, and_head = 0;
  double and_H[kAndMaxSlots][kAndMaxSlots] = {};
  double and_wF = 0.0, and_wG = 0.0;
  if (and_m > 0) {
    CK(ctx->and_g.ensure(size_t(and_R) * 2 * half));
    CK(ctx->and_f.ensure(size_t(and_R) * 2 * half));
    CK(ctx->and_part.ensure(and_part_len()));
    CK(ctx->and_dots.ensure(2 * kAndMaxSlots));
  }
  // g is in ring slot and_head; x = (F, G) is the iterate the electrons were solved against
  auto anderson_step = [&]() -> ephb_status {
    double *g = ctx->and_g.p + size_t(and_head) * 2 * half;
    double *f = ctx->and_f.p + size_t(and_head) * 2 * half;
    CK(launch_and_resid(half, g, ctx->F.p, ctx->G.p, f, st));
    and_n = std::min(and_n + 1, and_R);
    CK(launch_and_dots(half, f, ctx->and_f.p, 2 * half, and_n, ctx->and_part.p, ctx->and_dots.p, st));
    double hd[2 * kAndMaxSlots];
    CK(cudaMemcpyAsync(hd, ctx->and_dots.p, 2 * and_n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (and_wF == 0.0) {
      and_wF = hd[2 * and_head] > 0 ? 1.0 / hd[2 * and_head] : 1.0;
      and_wG = hd[2 * and_head + 1] > 0 ? 1.0 / hd[2 * and_head + 1] : 1.0;
    }
    for (int j = 0; j < and_n; ++j) and_H[and_head][j] = and_H[j][and_head] = and_wF * hd[2 * j] + and_wG * hd[2 * j + 1];
    AndCoef al{};
    al.a[and_head] = 1.0;
    if (!anderson_weights(and_H, and_n, and_head, al.a)) {   // keep only the newest entry
      for (int j = 0; j < kAndMaxSlots; ++j) al.a[j] = j == and_head ? 1.0 : 0.0;
      if (and_head != 0) {
        CK(cudaMemcpyAsync(ctx->and_g.p, g, 2 * half * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ctx->and_f.p, f, 2 * half * sizeof(double), cudaMemcpyDeviceToDevice, st));
        and_H[0][0] = and_H[and_head][and_head];
        al.a[0] = 1.0;
        al.a[and_head] = 0.0;
      }
      and_n = 1;
      and_head = 0;
    }
    CK(launch_and_mix(half, ctx->and_g.p, 2 * half, and_n, al, ctx->F.p, ctx->G.p, st));
    and_head = (and_head + 1) % and_R;
    return EPHB_OK;
  };

  auto inner_loop_mixed = [&](int drag, bool &ok) -> ephb_status {
    ok = false;
    // inexact inner solves while the outer iteration is far from converged: the electron loop
    // stops at 1e-2 of the last outer residual, but never before inner_tol, so the final outer
    // iterations (residual near tol) still bring the electrons to inner_tol
    const double tol_k = o->level != EPHB_DRAGGED ? inner_tol
                                                  : std::max(inner_tol, outer_seen ? 1e-2 * residual : 1e-2);
    last_tol_k = tol_k;
    const int64_t n3 = nst * 3;
    if (!ctx->have_f32) {
      CK(ctx->run_w32.ensure(ctx->nruns));
      for (auto *b : {&ctx->rI, &ctx->rJ, &ctx->dI, &ctx->dJ, &ctx->dI2, &ctx->dJ2}) CK(b->ensure(n3));
      CK(ctx->part32.ensure(size_t(ctx->nrseg) * 6));
      CK(launch_to_f32(ctx->nruns, ctx->run_w.p, ctx->run_w32.p, st));
      ctx->have_f32 = true;
    }
    CK(cudaMemsetAsync(ctx->prev_in.p, 0, kResLen * sizeof(double), st));
    ephb_status r = coefficients_to_host(ctx, ctx->prev_in.p, true, true);
    if (r != EPHB_OK) return r;
    if (drag) {
      CK(td.start(st));
      if (ph32)
        CK(launch_drag_term32(D, B, entry_segs(ctx), ctx->X32.p, ctx->FG32.p, ctx->seg_part.p, ctx->Dterm.p, st));
      else if (ph32_allowed)
        CK(launch_drag_termff(D, B, entry_segs(ctx), ctx->Xff.p, ctx->FGff.p, ctx->seg_part.p, ctx->Dterm.p, st));
      else
        CK(launch_drag_term(D, B, entry_segs(ctx), ctx->F.p, ctx->G.p, ctx->seg_part.p, ctx->Dterm.p, st));
      CK(td.stop(st));
    }
    const SweepSegs S = run_segs(ctx);
    for (int it = 1; it <= o->max_inner; ++it) {
      CK(te.start(st));
      CK(launch_self_sweep(M, B, S, ctx->run_col.p, ctx->run_w.p, ctx->I0.p, ctx->J0.p, ctx->inv_ffW.p, ctx->I.p,
                           ctx->J.p, ctx->I2.p, ctx->J2.p, drag ? ctx->Dterm.p : nullptr, ctx->seg_part.p,
                           ctx->epart.p, nullptr, st, tsw[0].a, tsw[0].b));
      tsw[0].pending = true;
      CK(launch_coeff_final(ctx->M, B, ctx->epart.p, ctx->ppart.p, ctx->res.p, ctx->prev_in.p, st));
      CK(te.stop(st));
      CK(cudaMemcpyAsync(ctx->host_res, ctx->res.p, kResLen * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      CK(te.collect());
      CK(td.collect());
      CK(tsw[0].collect());
      CK(tc32.collect());
      ++sweeps;
      ++inner_total;
      if (ctx->host_res[72] < tol_k) {   // x' is the answer
        std::swap(ctx->I.p, ctx->I2.p);
        std::swap(ctx->J.p, ctx->J2.p);
        B = bte_view(ctx);
        ok = true;
        return EPHB_OK;
      }
      if (it == o->max_inner) {
        std::swap(ctx->I.p, ctx->I2.p);
        std::swap(ctx->J.p, ctx->J2.p);
        B = bte_view(ctx);
        return EPHB_OK;
      }
      CK(tc32.start(st));
      CK(launch_corr_init(nst, ctx->I2.p, ctx->I.p, ctx->J2.p, ctx->J.p, ctx->rI.p, ctx->rJ.p, ctx->dI.p, ctx->dJ.p,
                          st));
      float *dA = ctx->dI.p, *dAJ = ctx->dJ.p, *dB = ctx->dI2.p, *dBJ = ctx->dJ2.p;
      for (int j = 0; j < kCorrSweeps; ++j) {
        CK(launch_corr_sweep(M, nst, S, ctx->run_col.p, ctx->run_w32.p, ctx->inv_ffW.p, ctx->rI.p, ctx->rJ.p, dA,
                             dAJ, ctx->part32.p, dB, dBJ, st));
        std::swap(dA, dB);
        std::swap(dAJ, dBJ);
      }
      sweeps32 += kCorrSweeps;
      CK(launch_corr_apply(nst, dA, dAJ, ctx->I.p, ctx->J.p, st));
      CK(tc32.stop(st));
      // coefficients of the corrected x become the reference of the next FP64 sweep's test
      // (on the device: the next sweep's read-back is the next host round trip)
      CK(launch_e_partial(B, ctx->I.p, ctx->J.p, ctx->epart.p, st));
      CK(launch_coeff_final(ctx->M, B, ctx->epart.p, ctx->ppart.p, ctx->res.p, ctx->prev_in.p, st));
    }
    return EPHB_OK;
  };

  auto inner_loop = [&](int drag, bool &ok) -> ephb_status {
    if (o->precision == EPHB_SOLVE_MIXED) return inner_loop_mixed(drag, ok);
    ok = false;
    CK(cudaMemsetAsync(ctx->prev_in.p, 0, kResLen * sizeof(double), st));
    ephb_status r = coefficients_to_host(ctx, ctx->prev_in.p, true, true);
    if (r != EPHB_OK) return r;
    if (drag) {   // F, G are fixed for this electron loop: its drag term is computed once
      CK(td.start(st));
      CK(launch_drag_term(D, B, entry_segs(ctx), ctx->F.p, ctx->G.p, ctx->seg_part.p, ctx->Dterm.p, st));
      CK(td.stop(st));
    }
    // Sweeps are queued in batches without a host round trip each: the coefficient kernel
    // advances the sweep counter and sets the stop flag (converged or max_inner reached), after
    // which the queued kernels return at once.
    const SweepSegs S = run_segs(ctx);
    int *hctl = reinterpret_cast<int *>(ctx->host_res + kResLen);
    CK(cudaMemsetAsync(ctx->sctl.p, 0, 4 * sizeof(int), st));
    CK(ctx->IJ.ensure(nst * 3));
    CK(ctx->IJ2.ensure(nst * 3));
    CK(launch_pack_ij(nst, ctx->I.p, ctx->J.p, ctx->IJ.p, st));
    // the sweep writes the electron partial sums and, in its last block, the coefficients
    // (the phonon partials are unchanged in the electron loop)
    CK(ctx->fuse_ctr.ensure(1));
    CK(cudaMemsetAsync(ctx->fuse_ctr.p, 0, sizeof(unsigned), st));
    CoeffFuse fuse;
    fuse.ppart = ctx->ppart.p;
    fuse.res = ctx->res.p;
    fuse.prev = ctx->prev_in.p;
    fuse.ctl = ctx->sctl.p;
    fuse.max_sweeps = o->max_inner;
    fuse.tol = inner_tol;
    fuse.counter = ctx->fuse_ctr.p;
    int queued = 0;
    for (;;) {
      const int nb = std::min(kSweepBatch, o->max_inner - queued);
      CK(te.start(st));
      for (int j = 0; j < nb; ++j) {
        CK(launch_self_sweep(M, B, S, ctx->run_col.p, ctx->run_w.p, ctx->I0.p, ctx->J0.p, ctx->inv_ffW.p, ctx->I.p,
                             ctx->J.p, ctx->I2.p, ctx->J2.p, drag ? ctx->Dterm.p : nullptr, ctx->seg_part.p,
                             ctx->epart.p, ctx->sctl.p, st, tsw[j].a, tsw[j].b, ctx->IJ.p, ctx->IJ2.p, &fuse));
        tsw[j].pending = true;
      }
      CK(te.stop(st));
      queued += nb;
      CK(cudaMemcpyAsync(ctx->host_res, ctx->res.p, kResLen * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(hctl, ctx->sctl.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      CK(te.collect());
      CK(td.collect());
      for (int j = 0; j < nb; ++j) CK(tsw[j].collect());
      if (hctl[0] || queued >= o->max_inner) break;
    }
    const int done = hctl[1];
    sweeps += done;
    inner_total += done;
    if (done & 1) {   // the last sweep wrote the second buffer pair
      std::swap(ctx->I.p, ctx->I2.p);
      std::swap(ctx->J.p, ctx->J2.p);
      std::swap(ctx->IJ.p, ctx->IJ2.p);
    }
    B = bte_view(ctx);
    ok = hctl[2] != 0;
    return EPHB_OK;
  };

  if (o->level == EPHB_DRAGLESS) {
    bool ok;
    s = inner_loop(0, ok);
    if (s != EPHB_OK) return s;
    converged = ok;
    outer = 1;
    residual = ctx->host_res[72];
  } else if (o->level == EPHB_DRAGGED || o->level == EPHB_PARTIAL) {
    for (outer = 1; outer <= o->max_outer; ++outer) {
      ph32 = ph32_allowed && (!outer_seen || residual >= kPh32Until);
      outer32 += ph32 ? 1 : 0;
      CK(tp.start(st));
      if (ph32) {
        CK(launch_pack6_f32(nst, ctx->I.p, ctx->J.p, ctx->IJ32.p, st));
        CK(launch_ph_sweep32(M, B, ph_segs(ctx), ctx->kinfo.p, ctx->Y32.p, ctx->IJ32.p, ctx->pseg_part.p, ctx->Btv.p,
                             st));
      } else if (ph32_allowed) {
        CK(launch_pack6_ff(nst, ctx->I.p, ctx->J.p, ctx->IJff.p, st));
        CK(launch_ph_sweepff(M, B, ph_segs(ctx), ctx->kinfo.p, ctx->Yff.p, ctx->IJff.p, ctx->pseg_part.p, ctx->Btv.p,
                             st));
      } else {
        CK(launch_ph_sweep(M, B, ph_segs(ctx), ctx->kinfo.p, ctx->I.p, ctx->J.p, ctx->pseg_part.p, ctx->Btv.p, st));
      }
      CK(tp.stop(st));
      if (and_m > 0 && outer >= 2) {   // the update goes to the ring, the mix to (F, G)
        double *g = ctx->and_g.p + size_t(and_head) * 2 * half;
        CK(launch_ph_update(M, D, ctx->Btv.p, ctx->F0.p, ctx->inv_nnW.p, g, g + half, ctx->Afold.p, st));
        s = anderson_step();
        if (s != EPHB_OK) return s;
      } else {
        CK(launch_ph_update(M, D, ctx->Btv.p, ctx->F0.p, ctx->inv_nnW.p, ctx->F.p, ctx->G.p, ctx->Afold.p, st));
      }
      if (ph32) CK(launch_pack6_f32(nph, ctx->F.p, ctx->G.p, ctx->FG32.p, st));
      else if (ph32_allowed) CK(launch_pack6_ff(nph, ctx->F.p, ctx->G.p, ctx->FGff.p, st));
      bool ok;
      s = inner_loop(1, ok);
      if (s != EPHB_OK) return s;
      CK(tp.collect());
      // the KO step keeps lambda in res[74] (res[75]: applied); the coefficient read-back
      // below brings both to the host with the residual, so the step needs no round trip
      if (o->ko_correction) CK(launch_ko(M, D, B, ctx->I.p, ctx->J.p, ctx->kpart.p, ctx->res.p, st));
      s = coefficients_to_host(ctx, ctx->prev_out.p);
      if (s != EPHB_OK) return s;
      if (o->ko_correction && ctx->host_res[75] != 0.0) lambda = ctx->host_res[74];
      residual = ctx->host_res[73];
      outer_seen = true;
      // an outer iteration whose electron loop stopped early does not end the iteration
      if (o->level == EPHB_PARTIAL || (residual < tol && last_tol_k <= inner_tol && !ph32)) {
        converged = true;
        break;
      }
    }
    if (outer > o->max_outer) outer = o->max_outer;
  }
  unsigned long long nzero = 0;
  CK(cudaMemcpyAsync(&nzero, ctx->nzero.p, sizeof(nzero), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(ev1, st));
  CK(cudaEventSynchronize(ev1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (out) {
    out->outer_iters = outer;
    out->inner_iters_total = inner_total;
    out->converged = converged ? 1 : 0;
    out->n_zero_rate_states = int(nzero);
    out->residual = residual;
    out->lambda = lambda;
    out->n_sweeps = sweeps;
    out->ms = ms;
    out->ms_e_sweep = te.ms;
    double ms_self = 0.0;
    for (auto &t : tsw) ms_self += t.ms;
    out->ms_self_kernel = ms_self;
    out->n_sweeps32 = sweeps32;
    out->ms_corr = tc32.ms;
    out->outer_iters32 = outer32;
    // FP64 work of one self-term sweep: 6 multiply-adds per run (+ two 3x3 rotations with symmetry)
    out->e_sweep_flops = double(ctx->nruns) * (ctx->M.nsym > 1 ? 12.0 + 36.0 : 12.0);
    out->ms_ph_sweep = tp.ms;
    // per electron sweep: the entry stream (k'|n|s word + X+,X-) plus the per-row arrays
    // per electron sweep: the run stream (partner word + weight) plus the per-row arrays
    // (segment pointer, I0, J0, 1/(f(1-f)W), drag term, new I, J)
    out->e_sweep_bytes = 12.0 * double(ctx->nruns) + double(nst) * (8.0 + 20.0 * 8.0);
    out->ms_drag = td.ms;
    out->n_runs = ctx->nruns;
  }
  ctx->solved = true;
  if (!converged) return fail(ctx, EPHB_ENOCONV, "iteration limit reached before the tolerance");
  return EPHB_OK;
}

// ---- device-driven solve: every instance's coupled iteration in one CUDA graph launch

constexpr double kGraphTimeLimitS = 600.0;   // a device loop running longer stops (EPHB_ETIMEOUT)

void sig_bytes(std::vector<unsigned char> &sig, const void *v, size_t n) {
  const unsigned char *p = static_cast<const unsigned char *>(v);
  sig.insert(sig.end(), p, p + n);
}
#define sig_add(sig, v) sig_bytes((sig), &(v), sizeof(v))

// The buffers of the instance in the base sized for the device-driven solve, and everything
// its capture reads gathered into one record.
ephb_status graph_prepare(ephb_ctx *ctx, const GraphOpts &go, int slot, GraphInst &g) {
  if (!ctx->bte_ready) {
    ephb_status s = bte_setup(ctx);
    if (s != EPHB_OK) return s;
  }
  const ModelDev &M = ctx->M;
  const int64_t nst = ctx->n_ibzw * M.nb, nph = ctx->qm.size() * M.nbr;
  const bool mixed = go.precision == EPHB_SOLVE_MIXED;
  if (mixed) {
    CK(ctx->run_w32.ensure(ctx->nruns));
    for (auto *b : {&ctx->rI, &ctx->rJ, &ctx->dI, &ctx->dJ, &ctx->dI2, &ctx->dJ2}) CK(b->ensure(nst * 3));
    CK(ctx->part32.ensure(size_t(ctx->nrseg) * 6));
  } else {
    CK(ctx->IJ.ensure(nst * 3));
    CK(ctx->IJ2.ensure(nst * 3));
    CK(ctx->fuse_ctr.ensure(1));
  }
  if (go.ph32_allowed) {
    CK(ctx->X32.ensure(ctx->n_entries));
    CK(ctx->Y32.ensure(ctx->n_ph_entries));
    CK(ctx->IJ32.ensure(nst * 6));
    CK(ctx->FG32.ensure(nph * 6));
    CK(ctx->Xff.ensure(ctx->n_entries));
    CK(ctx->Yff.ensure(ctx->n_ph_entries));
    CK(ctx->IJff.ensure(nst * 6));
    CK(ctx->FGff.ensure(nph * 6));
  }
  std::memset(&g, 0, sizeof(g));
  const BteDev B = bte_view(ctx);
  const SweepSegs Sr = run_segs(ctx), Se = entry_segs(ctx);
  std::memcpy(&g.B, &B, sizeof(B));
  std::memcpy(&g.Sr, &Sr, sizeof(Sr));
  std::memcpy(&g.Se, &Se, sizeof(Se));
  const SweepSegs Sp = ph_segs(ctx);
  std::memcpy(&g.Sp, &Sp, sizeof(Sp));
  g.ph_part = ctx->pseg_part.p;
  g.nst = nst;
  g.nph = nph;
  g.n_entries = ctx->n_entries;
  g.n_ph_entries = ctx->n_ph_entries;
  g.nruns = ctx->nruns;
  g.kinfo = ctx->kinfo.p;
  g.run_col = ctx->run_col.p;
  g.run_w = ctx->run_w.p;
  g.I0 = ctx->I0.p;
  g.J0 = ctx->J0.p;
  g.inv_ffW = ctx->inv_ffW.p;
  g.W_ph = ctx->W_ph.p;
  g.inv_nnW = ctx->inv_nnW.p;
  g.F0 = ctx->F0.p;
  g.ph_Y = ctx->ph_Y.p;
  g.e_X = ctx->e_X.p;
  g.I = ctx->I.p;
  g.J = ctx->J.p;
  g.I2 = ctx->I2.p;
  g.J2 = ctx->J2.p;
  g.F = ctx->F.p;
  g.G = ctx->G.p;
  g.Btv = ctx->Btv.p;
  g.Afold = ctx->Afold.p;
  g.Dterm = ctx->Dterm.p;
  g.seg_part = ctx->seg_part.p;
  g.epart = ctx->epart.p;
  g.ppart = ctx->ppart.p;
  g.kpart = ctx->kpart.p;
  g.res = ctx->res.p;
  g.prev_in = ctx->prev_in.p;
  g.prev_out = ctx->prev_out.p;
  if (mixed) {
    g.run_w32 = ctx->run_w32.p;
    g.rI = ctx->rI.p;
    g.rJ = ctx->rJ.p;
    g.dI = ctx->dI.p;
    g.dJ = ctx->dJ.p;
    g.dI2 = ctx->dI2.p;
    g.dJ2 = ctx->dJ2.p;
    g.part32 = ctx->part32.p;
  } else {
    g.sctl = ctx->sctl.p;
    g.fuse_ctr = ctx->fuse_ctr.p;
    g.IJ = ctx->IJ.p;
    g.IJ2 = ctx->IJ2.p;
  }
  if (go.ph32_allowed) {
    g.X32 = ctx->X32.p;
    g.Y32 = ctx->Y32.p;
    g.IJ32 = ctx->IJ32.p;
    g.FG32 = ctx->FG32.p;
    g.Xff = ctx->Xff.p;
    g.Yff = ctx->Yff.p;
    g.IJff = ctx->IJff.p;
    g.FGff = ctx->FGff.p;
  }
  g.warm = ctx->has_warm ? ctx->warm.p : nullptr;
  g.ctl = ctx->sg_ctl.p + slot;
  return EPHB_OK;
}

// Solves the instances `which` (their lists present) in one graph launch; infos[j] gets
// instance which[j]'s summary.  The graph is reused when everything it was built from is
// unchanged.
ephb_status graph_solve_set(ephb_ctx *ctx, const ephb_solve_opts *o, const std::vector<int> &which,
                            std::vector<ephb_solve_info> &infos, double &ms_launch, bool &reused) {
  GraphOpts go;
  std::memset(&go, 0, sizeof(go));
  go.level = o->level;
  go.precision = o->precision;
  go.ko = o->ko_correction ? 1 : 0;
  go.max_outer = o->max_outer;
  go.max_inner = o->max_inner;
  go.ph32_allowed = o->precision == EPHB_SOLVE_MIXED && o->level == EPHB_DRAGGED;
  go.tol = o->tol;
  go.inner_tol = o->inner_tol > 0 ? o->inner_tol : 0.1 * o->tol;
  go.time_limit_s = kGraphTimeLimitS;
  CK(ctx->sg_ctl.ensure(size_t(ctx->ninst)));
  std::vector<GraphInst> gi(which.size());
  std::vector<unsigned char> sig;
  sig_add(sig, go);
  sig_add(sig, ctx->M);
  const MeshDev D = mesh_view(ctx);
  sig_add(sig, D);
  for (size_t j = 0; j < which.size(); ++j) {
    select_instance(ctx, which[j]);
    GraphInst &g = gi[j];
    ephb_status s = graph_prepare(ctx, go, which[j], g);
    if (s != EPHB_OK) return s;
    // the warm start is applied only where asked for
    if (!o->warm_start) g.warm = nullptr;
    sig_add(sig, g);
  }
  reused = ctx->sg_exec && sig == ctx->sg_sig;
  if (!reused) {
    ctx->drop_graph();
    if (!ctx->sg_cs) CK(cudaStreamCreateWithFlags(&ctx->sg_cs, cudaStreamNonBlocking));
    cudaError_t e = build_solve_graph(ctx->M, D, gi, go, ctx->sg_cs, &ctx->sg_graph, &ctx->sg_exec, ctx->sg_kernels);
    if (e != cudaSuccess) {
      ctx->drop_graph();
      return fail(ctx, EPHB_ECUDA, std::string("building the solve graph: ") + cudaGetErrorString(e));
    }
    ctx->sg_sig = sig;
  }
  const cudaStream_t st = ctx->stream;
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  CK(cudaGraphLaunch(ctx->sg_exec, st));
  CK(cudaEventRecord(ev1, st));
  std::vector<GraphCtl> hc(ctx->ninst);
  CK(cudaMemcpyAsync(hc.data(), ctx->sg_ctl.p, sizeof(GraphCtl) * ctx->ninst, cudaMemcpyDeviceToHost, st));
  std::vector<unsigned long long> nzero(which.size(), 0ull);
  for (size_t j = 0; j < which.size(); ++j) {
    select_instance(ctx, which[j]);
    CK(cudaMemcpyAsync(&nzero[j], ctx->nzero.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  ms_launch = ms;
  infos.assign(which.size(), ephb_solve_info{});
  long long kernels = 0;
  bool late = false;
  for (size_t j = 0; j < which.size(); ++j) {
    const GraphCtl &c = hc[which[j]];
    const GraphKernels &k = ctx->sg_kernels[j];
    kernels += k.prologue + c.n_outer_body * k.outer_fixed + c.n_inner_body * k.inner_fixed;
    for (int m = 0; m < 3; ++m) kernels += c.n_ph_body[m] * k.ph[m];
    for (int b = 0; b < 2; ++b) kernels += c.n_in_body[b] * k.in[b];
    late = late || c.timed_out;
    select_instance(ctx, which[j]);
    ephb_solve_info &f = infos[j];
    f.outer_iters = c.outer;
    f.inner_iters_total = int(c.inner_total);
    f.converged = c.converged;
    f.n_zero_rate_states = int(nzero[j]);
    f.residual = c.residual;
    f.lambda = c.lambda;
    f.n_sweeps = c.sweeps;
    f.ms = ms;
    f.e_sweep_flops = double(ctx->nruns) * (ctx->M.nsym > 1 ? 12.0 + 36.0 : 12.0);
    f.e_sweep_bytes = 12.0 * double(ctx->nruns) + double(ctx->n_ibzw * ctx->M.nb) * (8.0 + 20.0 * 8.0);
    f.n_runs = ctx->nruns;
    f.n_sweeps32 = c.sweeps32;
    f.outer_iters32 = c.outer32;
    f.graph_launches = 1;
    f.graph_reused = reused ? 1 : 0;
    ctx->have_f32 = go.precision == EPHB_SOLVE_MIXED;
    ctx->solved = true;
  }
  note_launches(int(kernels));
  if (late) return fail(ctx, EPHB_ETIMEOUT, "a device-driven loop ran past its time limit");
  return EPHB_OK;
}

// ephb_solve_coupled_bte with opts->device_loop set.
ephb_status solve_graph(ephb_ctx *ctx, const ephb_solve_opts *o, ephb_solve_info *out) {
  ephb_solve_info sum{};
  sum.converged = 1;
  sum.lambda = 1.0;
  bool noconv = false;
  std::vector<std::vector<int>> sets;
  if (ctx->deferred) {
    for (int i = 0; i < ctx->ninst; ++i) sets.push_back({i});
  } else {
    sets.emplace_back();
    for (int i = 0; i < ctx->ninst; ++i) sets.back().push_back(i);
  }
  for (const auto &which : sets) {
    if (ctx->deferred) {
      select_instance(ctx, which[0]);
      if (ctx->lists_pending) {
        ephb_status d = derive_one(ctx);
        if (d != EPHB_OK) return d;
      }
    }
    std::vector<ephb_solve_info> infos;
    double ms = 0.0;
    bool reused = false;
    ephb_status r = graph_solve_set(ctx, o, which, infos, ms, reused);
    if (r != EPHB_OK) return r;
    sum.ms += ms;
    sum.graph_launches += 1;
    sum.graph_reused = reused ? 1 : 0;
    for (size_t j = 0; j < which.size(); ++j) {
      select_instance(ctx, which[j]);
      ephb_solve_info one = infos[j];
      if (!one.converged && o->warm_start && ctx->has_warm) {
        // the learned start did not converge: the plain RTA start decides (host-driven)
        ephb_solve_opts plain = *o;
        plain.warm_start = 0;
        plain.device_loop = 0;
        ephb_solve_info again{};
        ephb_status r2 = solve_one(ctx, &plain, &again);
        if (r2 != EPHB_OK && r2 != EPHB_ENOCONV) return r2;
        again.n_sweeps += one.n_sweeps;
        again.n_sweeps32 += one.n_sweeps32;
        again.inner_iters_total += one.inner_iters_total;
        again.ms += one.ms;
        sum.ms += again.ms - one.ms;
        one = again;
      }
      noconv = noconv || !one.converged;
      ctx->last = one;
      sum.outer_iters = std::max(sum.outer_iters, one.outer_iters);
      sum.inner_iters_total += one.inner_iters_total;
      sum.converged = sum.converged && one.converged;
      sum.n_zero_rate_states += one.n_zero_rate_states;
      sum.residual = std::max(sum.residual, one.residual);
      sum.lambda = one.lambda;
      sum.n_sweeps += one.n_sweeps;
      sum.e_sweep_bytes += one.e_sweep_bytes;
      sum.n_runs += one.n_runs;
      sum.n_sweeps32 += one.n_sweeps32;
      sum.outer_iters32 = std::max(sum.outer_iters32, one.outer_iters32);
      sum.e_sweep_flops += one.e_sweep_flops;
    }
    if (ctx->deferred) {
      CK(cudaStreamSynchronize(ctx->stream));
      ctx->release_lists();
      ctx->drop_graph();   // its buffers are gone
    }
  }
  select_instance(ctx, 0);
  if (out) *out = sum;
  ctx->stage = 4;
  if (noconv) return fail(ctx, EPHB_ENOCONV, "iteration limit reached before the tolerance");
  return EPHB_OK;
}

}  // namespace

ephb_status ephb_solve_coupled_bte(ephb_ctx *ctx, const ephb_solve_opts *o, ephb_solve_info *out) {
  if (!ctx) return EPHB_EINVAL;
  if (ctx->stage < 3) return fail(ctx, EPHB_ESTATE, "compute_transition_rates must come first");
  if (!o) return fail(ctx, EPHB_EINVAL, "opts is NULL");
  if (o->level < EPHB_RTA || o->level > EPHB_DRAGGED) return fail(ctx, EPHB_EINVAL, "bad level");
  if (!(o->tol > 0) || o->max_outer < 1 || o->max_inner < 1) return fail(ctx, EPHB_EINVAL, "bad tolerances");
  if (o->precision != EPHB_SOLVE_FP64 && o->precision != EPHB_SOLVE_MIXED)
    return fail(ctx, EPHB_EINVAL, "bad solve precision");
  if (o->accel_depth < 0 || o->accel_depth > EPHB_MAX_ACCEL_DEPTH)
    return fail(ctx, EPHB_EINVAL, "accel_depth outside 0..EPHB_MAX_ACCEL_DEPTH");
  if (o->device_loop != 0 && o->device_loop != 1) return fail(ctx, EPHB_EINVAL, "device_loop must be 0 or 1");
  if (o->device_loop && (o->accel_depth != 0 || o->level == EPHB_RTA))
    return fail(ctx, EPHB_EINVAL, "device_loop needs accel_depth 0 and a level other than EPHB_RTA");
  CK(cudaSetDevice(ctx->device));
  if (o->device_loop) return solve_graph(ctx, o, out);
  // every instance in turn; the summary adds up counts and times and keeps the worst residual
  ephb_solve_info sum{};
  sum.converged = 1;
  sum.lambda = 1.0;
  bool noconv = false;
  for (int i = 0; i < ctx->ninst; ++i) {
    select_instance(ctx, i);
    if (ctx->lists_pending) {
      ephb_status d = derive_one(ctx);
      if (d != EPHB_OK) return d;
    }
    ephb_solve_info one{};
    ephb_status r = solve_one(ctx, o, &one);
    if (r == EPHB_ENOCONV && o->warm_start && ctx->has_warm) {
      // the learned start did not converge: the plain RTA start decides
      ephb_solve_opts plain = *o;
      plain.warm_start = 0;
      ephb_solve_info again{};
      r = solve_one(ctx, &plain, &again);
      again.n_sweeps += one.n_sweeps;
      again.inner_iters_total += one.inner_iters_total;
      again.ms += one.ms;
      one = again;
    }
    if (r != EPHB_OK && r != EPHB_ENOCONV) return r;
    noconv = noconv || r == EPHB_ENOCONV;
    ctx->last = one;
    if (ctx->deferred) {
      CK(cudaStreamSynchronize(ctx->stream));
      ctx->release_lists();
    }
    sum.outer_iters = std::max(sum.outer_iters, one.outer_iters);
    sum.inner_iters_total += one.inner_iters_total;
    sum.converged = sum.converged && one.converged;
    sum.n_zero_rate_states += one.n_zero_rate_states;
    sum.residual = std::max(sum.residual, one.residual);
    sum.lambda = one.lambda;
    sum.n_sweeps += one.n_sweeps;
    sum.ms += one.ms;
    sum.ms_e_sweep += one.ms_e_sweep;
    sum.ms_ph_sweep += one.ms_ph_sweep;
    sum.e_sweep_bytes += one.e_sweep_bytes;
    sum.ms_drag += one.ms_drag;
    sum.n_runs += one.n_runs;
    sum.ms_self_kernel += one.ms_self_kernel;
    sum.n_sweeps32 += one.n_sweeps32;
    sum.ms_corr += one.ms_corr;
    sum.outer_iters32 = std::max(sum.outer_iters32, one.outer_iters32);
    sum.e_sweep_flops += one.e_sweep_flops;
  }
  select_instance(ctx, 0);
  if (out) *out = sum;
  ctx->stage = 4;
  if (noconv) return fail(ctx, EPHB_ENOCONV, "iteration limit reached before the tolerance");
  return EPHB_OK;
}

ephb_status ephb_set_impurities(ephb_ctx *ctx, const ephb_impurities *imp) {
  if (!ctx) return EPHB_EINVAL;
  ephb_impurities v{};
  if (imp && imp->n_species != 0) {
    if (imp->n_species < 0 || imp->n_species > EPHB_MAX_DOPANTS)
      return fail(ctx, EPHB_EINVAL, "n_species outside 0..EPHB_MAX_DOPANTS");
    if (!(imp->eps_r > 0)) return fail(ctx, EPHB_EINVAL, "eps_r must be positive");
    for (int i = 0; i < imp->n_species; ++i)
      if (!(imp->n_cm3[i] >= 0) || !std::isfinite(imp->Z[i]))
        return fail(ctx, EPHB_EINVAL, "concentrations must be non-negative and charges finite");
    v = *imp;
  }
  ctx->imp = v;
  // the RTA terms of every instance change
  ctx->bte_ready = false;
  for (auto &sl : ctx->slots) sl.bte_ready = false;
  return EPHB_OK;
}

ephb_status ephb_set_isotopes(ephb_ctx *ctx, const double *g, int nat) {
  if (!ctx) return EPHB_EINVAL;
  if (!g || nat == 0) {
    ctx->iso_nat = 0;
  } else {
    if (nat < 0 || nat > 4) return fail(ctx, EPHB_EINVAL, "nat outside 0..4");
    for (int a = 0; a < nat; ++a)
      if (!(g[a] >= 0) || !std::isfinite(g[a])) return fail(ctx, EPHB_EINVAL, "mass variances must be >= 0");
    ctx->iso_nat = nat;
    for (int a = 0; a < 4; ++a) ctx->iso_g[a] = a < nat ? g[a] : 0.0;
  }
  ctx->bte_ready = false;
  for (auto &sl : ctx->slots) sl.bte_ready = false;
  return EPHB_OK;
}

ephb_status ephb_transport_coefficients(ephb_ctx *ctx, int inst, ephb_coeffs *out) {
  if (!ctx) return EPHB_EINVAL;
  if (inst < 0 || inst >= ctx->ninst) return fail(ctx, EPHB_EINVAL, "inst out of range");
  if (!out) return fail(ctx, EPHB_EINVAL, "out is NULL");
  select_instance(ctx, inst);
  if (ctx->stage < 4 || !ctx->bte_ready) return fail(ctx, EPHB_ESTATE, "solve_coupled_bte must come first");
  CK(cudaSetDevice(ctx->device));
  ephb_status s = coefficients_to_host(ctx, ctx->prev_tmp.p);
  if (s != EPHB_OK) return s;
  const double *r = ctx->host_res;
  std::memcpy(out->sigma, r + 0, 9 * sizeof(double));
  std::memcpy(out->sigmaS, r + 9, 9 * sizeof(double));
  std::memcpy(out->alpha_el, r + 18, 9 * sizeof(double));
  std::memcpy(out->kappa0_el, r + 27, 9 * sizeof(double));
  std::memcpy(out->alpha_ph, r + 36, 9 * sizeof(double));
  std::memcpy(out->kappa_ph, r + 45, 9 * sizeof(double));
  std::memcpy(out->S, r + 54, 9 * sizeof(double));
  std::memcpy(out->kappa_el, r + 63, 9 * sizeof(double));
  return EPHB_OK;
}

// ---------------------------------------------------------------------------------------
int64_t ephb_num_states(const ephb_ctx *ctx) { return ctx ? ctx->n_ibzw * ctx->M.nb : 0; }

ephb_status ephb_state_features(ephb_ctx *ctx, int inst, float *feat_dev, int64_t n_states) {
  if (!ctx || !feat_dev) return EPHB_EINVAL;
  if (ctx->stage < 3) return fail(ctx, EPHB_ESTATE, "compute_transition_rates must come first");
  if (inst < 0 || inst >= ctx->ninst) return fail(ctx, EPHB_EINVAL, "inst out of range");
  if (n_states != ctx->n_ibzw * ctx->M.nb) return fail(ctx, EPHB_EINVAL, "n_states must be ephb_num_states()");
  CK(cudaSetDevice(ctx->device));
  select_instance(ctx, inst);
  if (ctx->lists_pending) {
    ephb_status d = derive_one(ctx);
    if (d != EPHB_OK) return d;
  }
  if (!ctx->bte_ready) {
    ephb_status s = bte_setup(ctx);
    if (s != EPHB_OK) return s;
  }
  CK(ctx->vmaxb.ensure(1));
  CK(launch_state_features(bte_view(ctx), ctx->W_e.p, ctx->vmaxb.p, feat_dev, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return EPHB_OK;
}

ephb_status ephb_state_targets(ephb_ctx *ctx, int inst, float *targ_dev, int64_t n_states) {
  if (!ctx || !targ_dev) return EPHB_EINVAL;
  if (inst < 0 || inst >= ctx->ninst) return fail(ctx, EPHB_EINVAL, "inst out of range");
  select_instance(ctx, inst);
  if (ctx->stage < 4 || !ctx->solved) return fail(ctx, EPHB_ESTATE, "the instance has no solution yet");
  if (n_states != ctx->n_ibzw * ctx->M.nb) return fail(ctx, EPHB_EINVAL, "n_states must be ephb_num_states()");
  CK(cudaSetDevice(ctx->device));
  CK(ctx->vmaxb.ensure(1));
  CK(launch_state_targets(bte_view(ctx), ctx->I.p, ctx->J.p, ctx->J0.p, ctx->vmaxb.p, targ_dev, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return EPHB_OK;
}

ephb_status ephb_set_warm_start(ephb_ctx *ctx, int inst, const float *scale_dev, int64_t n_states) {
  if (!ctx) return EPHB_EINVAL;
  if (ctx->stage < 3) return fail(ctx, EPHB_ESTATE, "compute_transition_rates must come first");
  if (inst < 0 || inst >= ctx->ninst) return fail(ctx, EPHB_EINVAL, "inst out of range");
  if (n_states != ctx->n_ibzw * ctx->M.nb) return fail(ctx, EPHB_EINVAL, "n_states must be ephb_num_states()");
  CK(cudaSetDevice(ctx->device));
  select_instance(ctx, inst);
  if (!scale_dev) {
    ctx->has_warm = false;
    return EPHB_OK;
  }
  CK(ctx->warm.ensure(size_t(n_states) * 2));
  CK(cudaMemcpyAsync(ctx->warm.p, scale_dev, size_t(n_states) * 2 * sizeof(float), cudaMemcpyDeviceToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->has_warm = true;
  return EPHB_OK;
}

ephb_status ephb_instance_solve_info(ephb_ctx *ctx, int inst, ephb_solve_info *out) {
  if (!ctx || !out) return EPHB_EINVAL;
  if (inst < 0 || inst >= ctx->ninst) return fail(ctx, EPHB_EINVAL, "inst out of range");
  *out = inst == ctx->cur ? ctx->last : ctx->slots[inst].last;
  return EPHB_OK;
}

ephb_status ephb_set_tuning(ephb_ctx *ctx, int key, int value) {
  if (!ctx) return EPHB_EINVAL;
  if (key == EPHB_TUNE_WITHHOLD_MMA) {
    ctx->withhold_mma = value ? 1 : 0;
    return EPHB_OK;
  }
  if (key == EPHB_TUNE_DEFER_INSTANCES) {
    ctx->force_defer = value ? 1 : 0;
    return EPHB_OK;
  }
  if (key == EPHB_TUNE_STAGE_A_TMEM_A) {
    ctx->stage_a_tmem = value ? 1 : 0;
    return EPHB_OK;
  }
  if (key != EPHB_TUNE_TC_COLS) return fail(ctx, EPHB_EINVAL, "unknown tuning key");
  if (value != 0 && (value < 16 || value % 16 != 0 || value > 256))
    return fail(ctx, EPHB_EINVAL, "column-chunk width must be 0 or a multiple of 16 in [16, 256]");
  ctx->force_cols = value;
  if (value == 0) ctx->tune_cols[0] = ctx->tune_cols[1] = ctx->tune_cols[2] = 0;   // tune again on the next call
  return EPHB_OK;
}

ephb_status ephb_select_instance(ephb_ctx *ctx, int inst) {
  if (!ctx) return EPHB_EINVAL;
  if (inst < 0 || inst >= ctx->ninst) return fail(ctx, EPHB_EINVAL, "inst out of range");
  select_instance(ctx, inst);
  return EPHB_OK;
}

int ephb_num_instances(const ephb_ctx *ctx) { return ctx ? ctx->ninst : 0; }

ephb_status ephb_get_device_array(ephb_ctx *ctx, int which, void **dptr, int64_t shape[4], int *dtype) {
  if (!ctx || !dptr || !shape || !dtype) return EPHB_EINVAL;
  const int64_t nk = ctx->km.size(), nq = ctx->qm.size(), nb = ctx->M.nb, nbr = ctx->M.nbr;
  const int64_t nst = ctx->n_ibzw * nb;
  for (int d = 0; d < 4; ++d) shape[d] = 1;
  int need = 2;
  void *p = nullptr;
  int dt = 0;
  switch (which) {
    case EPHB_ARR_EPS: p = ctx->eps.p; shape[0] = nk; shape[1] = nb; break;
    case EPHB_ARR_VEL: p = ctx->vel.p; shape[0] = nk; shape[1] = nb; shape[2] = 3; break;
    case EPHB_ARR_OMEGA: p = ctx->w.p; shape[0] = nq; shape[1] = nbr; break;
    case EPHB_ARR_VPH: p = ctx->vph.p; shape[0] = nq; shape[1] = nbr; shape[2] = 3; break;
    case EPHB_ARR_IBZ_REP: p = ctx->rep.p; shape[0] = nk; dt = 2; break;
    case EPHB_ARR_IBZ_OP: p = ctx->op.p; shape[0] = nk; dt = 2; break;
    case EPHB_ARR_IBZW_LIST: p = ctx->ibzw_list.p; shape[0] = ctx->n_ibzw; dt = 2; break;
    case EPHB_ARR_ACTIVE: p = ctx->amask.p; shape[0] = nk; dt = 4; break;
    case EPHB_ARR_PAIR_PTR: p = ctx->pair_ptr.p; shape[0] = ctx->n_ibzw + 1; dt = 3; break;
    case EPHB_ARR_PAIR_Q: p = ctx->pair_q.p; shape[0] = ctx->n_pairs; dt = 2; break;
    case EPHB_ARR_ROW_PTR: p = ctx->row_ptr.p; shape[0] = nst + 1; dt = 3; need = 3; break;
    case EPHB_ARR_ENTRY_KPNS: p = ctx->e_kpns.p; shape[0] = ctx->n_entries; dt = 4; need = 3; break;
    case EPHB_ARR_ENTRY_X: p = ctx->e_X.p; shape[0] = ctx->n_entries; shape[1] = 2; need = 3; break;
    case EPHB_ARR_W_E: p = ctx->W_e.p; shape[0] = nst; need = 4; break;
    case EPHB_ARR_W_PH: p = ctx->W_ph.p; shape[0] = nq; shape[1] = nbr; need = 4; break;
    case EPHB_ARR_I: p = ctx->I.p; shape[0] = nst; shape[1] = 3; need = 4; break;
    case EPHB_ARR_J: p = ctx->J.p; shape[0] = nst; shape[1] = 3; need = 4; break;
    case EPHB_ARR_F: p = ctx->F.p; shape[0] = nq; shape[1] = nbr; shape[2] = 3; need = 4; break;
    case EPHB_ARR_G: p = ctx->G.p; shape[0] = nq; shape[1] = nbr; shape[2] = 3; need = 4; break;
    case EPHB_ARR_STATE_EPS: p = ctx->st_eps.p; shape[0] = nst; need = 4; break;
    case EPHB_ARR_STATE_VEL: p = ctx->st_vel.p; shape[0] = nst; shape[1] = 3; need = 4; break;
    case EPHB_ARR_STATE_WEIGHT: p = ctx->st_wt.p; shape[0] = nst; need = 4; break;
    default: return fail(ctx, EPHB_EINVAL, "unknown array id");
  }
  if (ctx->stage < need || (need == 4 && !ctx->bte_ready)) return fail(ctx, EPHB_ESTATE, "array not computed yet");
  *dptr = p;
  *dtype = dt;
  return EPHB_OK;
}

int64_t ephb_kernel_launches(void) { return g_launches.load(); }

ephb_status ephb_copy_array_to_host(ephb_ctx *ctx, int which, void *host_dst, int64_t nbytes) {
  if (!ctx || !host_dst) return EPHB_EINVAL;
  void *p;
  int64_t shape[4];
  int dt;
  ephb_status s = ephb_get_device_array(ctx, which, &p, shape, &dt);
  if (s != EPHB_OK) return s;
  const int64_t esz[5] = {8, 16, 4, 8, 4};
  int64_t need = shape[0] * shape[1] * shape[2] * shape[3] * esz[dt];
  if (nbytes < need) return fail(ctx, EPHB_EINVAL, "destination too small");
  CK(cudaSetDevice(ctx->device));
  if (need > 0) {
    CK(cudaMemcpyAsync(host_dst, p, size_t(need), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return EPHB_OK;
}

}  // extern "C"

extern "C" ephb_status ephb_selftest_exp_ff(const double *y_dev, double *out_dev, int64_t n, void *cuda_stream) {
  if (n < 0 || (n > 0 && (!y_dev || !out_dev))) return EPHB_EINVAL;
  if (launch_selftest_exp_ff(y_dev, out_dev, n, static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess)
    return EPHB_ECUDA;
  return EPHB_OK;
}
