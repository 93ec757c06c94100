// C ABI of the learned proposal (declared in include/mcrt.h): the network
// object, its training steps, cell features, the second-moment tallies of a
// solve, and the per-cell proposal built from probabilities or from the
// network.  Host side only: validation, buffers and launches of learn.cu.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mcrt.h"
#include "ctx.h"
#include "mcrt_internal.h"

using namespace mcrt_host;

struct mcrt_mlp {
  int device = 0, K = 0;
  long long np = 0;
  int grid = 0;
  DevBuf theta, theta16, m1, m2, grad, partial, loss_partial, loss, nrm, errf, stat_partial, bsum;
  int t = 0;
  bool have_loss = false;
  cudaStream_t last_stream = nullptr;
  std::string err;
};

namespace {

int mfail(mcrt_mlp *m, int code, const std::string &msg) {
  if (m) m->err = msg;
  return code;
}

int mcuda_fail(mcrt_mlp *m, cudaError_t e, const char *where) {
  cudaGetLastError();
  return mfail(m, e == cudaErrorMemoryAllocation ? MCRT_E_OOM : MCRT_E_CUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

#define MK(call, where)                                      \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return mcuda_fail(m, e_, where); \
  } while (0)

void mlp_release(mcrt_mlp *m) {
  DevBuf *bufs[] = {&m->theta, &m->theta16, &m->m1, &m->m2, &m->grad, &m->partial,
                    &m->loss_partial, &m->loss, &m->nrm, &m->errf, &m->stat_partial, &m->bsum};
  for (DevBuf *b : bufs) release(*b);
}

long long ncells_of(const mcrt_ctx *ctx) {
  return (long long)ctx->grid.nx * ctx->grid.ny * ctx->grid.nz;
}

// Device error flag of the learned-proposal kernels, cleared on `s`.
int clear_lerr(mcrt_ctx *ctx, cudaStream_t s) {
  CK(ensure(ctx->lerr, sizeof(unsigned long long)), "alloc error flag");
  CK(cudaMemsetAsync(ctx->lerr.p, 0, sizeof(unsigned long long), s), "clear error flag");
  return MCRT_OK;
}

int read_lerr(mcrt_ctx *ctx, cudaStream_t s, unsigned long long *flag) {
  CK(cudaMemcpyAsync(flag, ctx->lerr.p, sizeof(*flag), cudaMemcpyDeviceToHost, s), "read error flag");
  CK(cudaStreamSynchronize(s), "sync");
  return MCRT_OK;
}

int ensure_cell_buffers(mcrt_ctx *ctx) {
  const size_t nc = (size_t)ncells_of(ctx), nb = ctx->nb, ng = ctx->ng;
  CK(ensure(ctx->cell_cn, nc * nb * sizeof(uint64_t)), "alloc cell proposal");
  CK(ensure(ctx->cell_cg, nc * nb * ng * sizeof(uint64_t)), "alloc cell proposal");
  CK(ensure(ctx->cell_hemi, nc * sizeof(uint32_t)), "alloc cell proposal");
  return MCRT_OK;
}

mcrt::FeatArgs feat_args(const mcrt_ctx *ctx, const int32_t *cells, long long n, float *out) {
  const mcrt_grid_desc &g = ctx->grid;
  mcrt::FeatArgs f;
  std::memset(&f, 0, sizeof(f));
  f.nx = g.nx;
  f.ny = g.ny;
  f.nz = g.nz;
  f.dx = g.lx / g.nx;
  f.dy = g.ly / g.ny;
  f.dz = g.lz / g.nz;
  f.h = 0.5 * g.ly;
  f.yf = (const double *)ctx->yf64.p;
  f.T_wall[0] = g.T_wall[0];
  f.T_wall[1] = g.T_wall[1];
  f.eps_wall[0] = g.eps_wall[0];
  f.eps_wall[1] = g.eps_wall[1];
  f.T_max = proposal_T_max(ctx);
  f.field64 = (const double2 *)ctx->field64.p;
  f.fpos32 = (const uint2 *)ctx->fpos32.p;
  f.kptab = (const float4 *)ctx->kptab.p;
  f.nT = ctx->nT;
  f.cells = cells;
  f.n = n;
  f.out = out;
  f.err = (unsigned long long *)ctx->lerr.p;
  return f;
}

int need_tables_and_fields(mcrt_ctx *ctx) {
  if (!ctx->have_kdist || !ctx->have_fields) return fail(ctx, MCRT_E_STATE, "set kdist and fields first");
  if (ctx->nT > 512) return fail(ctx, MCRT_E_UNSUPPORTED, "tables of at most 512 T nodes");
  return MCRT_OK;
}

}  // namespace

extern "C" {

int64_t mcrt_mlp_nparams(int K) { return K < 1 ? -1 : (int64_t)mcrt::mlp_nparams(K); }

int mcrt_mlp_create(int device, int K, mcrt_mlp **out) {
  if (!out) return MCRT_E_ARG;
  *out = nullptr;
  if (K < 1) return MCRT_E_ARG;
  if (K + 2 > mcrt::kMaxTrainOut) return MCRT_E_UNSUPPORTED;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MCRT_E_CUDA;
  }
  mcrt_mlp *m = new (std::nothrow) mcrt_mlp();
  if (!m) return MCRT_E_OOM;
  m->device = device;
  m->K = K;
  m->np = mcrt::mlp_nparams(K);
  DeviceGuard dg(device);
  if (!dg.ok) {
    delete m;
    return MCRT_E_CUDA;
  }
  m->grid = mcrt::mlp_train_grid();
  const size_t np = (size_t)m->np;
  cudaError_t e = cudaSuccess;
  DevBuf *f32[] = {&m->theta, &m->m1, &m->m2, &m->grad};
  for (DevBuf *b : f32)
    if (e == cudaSuccess) e = ensure(*b, np * sizeof(float));
  if (e == cudaSuccess) e = ensure(m->theta16, np * sizeof(__half));
  if (e == cudaSuccess) e = ensure(m->partial, (size_t)m->grid * np * sizeof(float));
  if (e == cudaSuccess) e = ensure(m->loss_partial, (size_t)m->grid * sizeof(double));
  if (e == cudaSuccess) e = ensure(m->loss, sizeof(double));
  if (e == cudaSuccess) e = ensure(m->nrm, 2 * MCRT_NFEAT * sizeof(float));
  if (e == cudaSuccess) e = ensure(m->errf, sizeof(unsigned long long));
  if (e == cudaSuccess) e = ensure(m->stat_partial, (size_t)m->grid * 4 * sizeof(double));
  if (e == cudaSuccess) e = ensure(m->bsum, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(m->errf.p, 0, sizeof(unsigned long long));
  for (DevBuf *b : f32)
    if (e == cudaSuccess) e = cudaMemset(b->p, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->theta16.p, 0, np * sizeof(__half));
  if (e == cudaSuccess) {
    float nrm[2 * MCRT_NFEAT];
    for (int i = 0; i < MCRT_NFEAT; ++i) {
      nrm[i] = 0.f;
      nrm[MCRT_NFEAT + i] = 1.f;
    }
    e = cudaMemcpy(m->nrm.p, nrm, sizeof(nrm), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    mlp_release(m);
    delete m;
    return e == cudaErrorMemoryAllocation ? MCRT_E_OOM : MCRT_E_CUDA;
  }
  *out = m;
  return MCRT_OK;
}

int mcrt_mlp_set_params(mcrt_mlp *m, const float *theta, const float *feat_mean,
                        const float *feat_inv_std) {
  if (!m) return MCRT_E_ARG;
  if (!theta || !feat_mean || !feat_inv_std) return mfail(m, MCRT_E_ARG, "null argument");
  for (long long j = 0; j < m->np; ++j)
    if (!std::isfinite(theta[j])) return mfail(m, MCRT_E_ARG, "non-finite parameter");
  for (int i = 0; i < MCRT_NFEAT; ++i)
    if (!std::isfinite(feat_mean[i]) || !std::isfinite(feat_inv_std[i]))
      return mfail(m, MCRT_E_ARG, "non-finite normalisation");
  DeviceGuard dg(m->device);
  if (!dg.ok) return mfail(m, MCRT_E_CUDA, "cudaSetDevice");
  const size_t np = (size_t)m->np;
  MK(cudaMemcpy(m->theta.p, theta, np * sizeof(float), cudaMemcpyHostToDevice), "copy theta");
  float nrm[2 * MCRT_NFEAT];
  std::memcpy(nrm, feat_mean, MCRT_NFEAT * sizeof(float));
  std::memcpy(nrm + MCRT_NFEAT, feat_inv_std, MCRT_NFEAT * sizeof(float));
  MK(cudaMemcpy(m->nrm.p, nrm, sizeof(nrm), cudaMemcpyHostToDevice), "copy normalisation");
  MK(cudaMemset(m->m1.p, 0, np * sizeof(float)), "reset Adam");
  MK(cudaMemset(m->m2.p, 0, np * sizeof(float)), "reset Adam");
  MK(mcrt::launch_theta_to_half((const float *)m->theta.p, (__half *)m->theta16.p, m->np, nullptr),
     "theta to FP16");
  MK(cudaDeviceSynchronize(), "sync");
  m->t = 0;
  return MCRT_OK;
}

int mcrt_mlp_get_params(mcrt_mlp *m, float *theta, float *theta_used) {
  if (!m) return MCRT_E_ARG;
  if (!theta) return mfail(m, MCRT_E_ARG, "null theta");
  DeviceGuard dg(m->device);
  if (!dg.ok) return mfail(m, MCRT_E_CUDA, "cudaSetDevice");
  MK(cudaDeviceSynchronize(), "sync");
  const size_t np = (size_t)m->np;
  MK(cudaMemcpy(theta, m->theta.p, np * sizeof(float), cudaMemcpyDeviceToHost), "copy theta");
  if (theta_used) {
    std::vector<__half> h(np);
    MK(cudaMemcpy(h.data(), m->theta16.p, np * sizeof(__half), cudaMemcpyDeviceToHost), "copy theta16");
    for (size_t j = 0; j < np; ++j) theta_used[j] = __half2float(h[j]);
  }
  return MCRT_OK;
}

int mcrt_mlp_forward(mcrt_mlp *m, const float *feat, int64_t n, const float *p0, int p0_stride,
                     float mix, float *q_out, void *stream) {
  if (!m) return MCRT_E_ARG;
  if (n < 0 || (n > 0 && (!feat || !p0 || !q_out))) return mfail(m, MCRT_E_ARG, "bad arguments");
  if (p0_stride != 0 && p0_stride != m->K) return mfail(m, MCRT_E_ARG, "p0_stride must be 0 or K");
  if (!(mix >= 0.f && mix <= 1.f)) return mfail(m, MCRT_E_ARG, "mix outside [0, 1]");
  DeviceGuard dg(m->device);
  if (!dg.ok) return mfail(m, MCRT_E_CUDA, "cudaSetDevice");
  mcrt::MlpInferArgs a;
  std::memset(&a, 0, sizeof(a));
  a.theta16 = (const __half *)m->theta16.p;
  a.fmean = (const float *)m->nrm.p;
  a.finv = a.fmean + MCRT_NFEAT;
  a.K = m->K;
  a.feat = feat;
  a.n = n;
  a.p0 = p0;
  a.p0_stride = p0_stride;
  a.mix = mix;
  a.q_out = q_out;
  MK(mcrt::launch_mlp_infer(a, (cudaStream_t)stream), "forward");
  return MCRT_OK;
}

int mcrt_mlp_loss_grad(mcrt_mlp *m, const float *feat, const float *mom, const float *cost,
                       float c0, const float *p0, int p0_stride, const float *wgt, int mode,
                       int64_t n_data, const int32_t *idx, int64_t n, float mix, float *grad_out,
                       void *stream) {
  if (!m) return MCRT_E_ARG;
  if (mode != MCRT_LOSS_CELL && mode != MCRT_LOSS_BATCH) return mfail(m, MCRT_E_ARG, "bad loss mode");
  if (n < 1 || !feat || !mom || !p0) return mfail(m, MCRT_E_ARG, "bad arguments");
  if (n_data < 1 || (!idx && n > n_data)) return mfail(m, MCRT_E_ARG, "batch beyond the dataset");
  if (p0_stride != 0 && p0_stride != m->K) return mfail(m, MCRT_E_ARG, "p0_stride must be 0 or K");
  if (!(mix >= 0.f && mix <= 1.f)) return mfail(m, MCRT_E_ARG, "mix outside [0, 1]");
  if (!(c0 >= 0.f) || !std::isfinite(c0)) return mfail(m, MCRT_E_ARG, "c0 < 0");
  DeviceGuard dg(m->device);
  if (!dg.ok) return mfail(m, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  mcrt::MlpTrainArgs a;
  std::memset(&a, 0, sizeof(a));
  a.theta16 = (const __half *)m->theta16.p;
  a.fmean = (const float *)m->nrm.p;
  a.finv = a.fmean + MCRT_NFEAT;
  a.K = m->K;
  a.feat = feat;
  a.mom = mom;
  a.cost = cost;
  a.c0 = c0;
  a.p0 = p0;
  a.p0_stride = p0_stride;
  a.wgt = wgt;
  a.mode = mode;
  a.stat_partial = (double *)m->stat_partial.p;
  a.idx = idx;
  a.n_data = n_data;
  a.n = n;
  a.mix = mix;
  a.err = (unsigned long long *)m->errf.p;
  a.partial = (float *)m->partial.p;
  a.loss_partial = (double *)m->loss_partial.p;
  a.grid = m->grid;
  const double *bsum = nullptr;
  if (mode == MCRT_LOSS_BATCH) {
    // pass 0: the batch sums the per-sample multipliers depend on
    a.pass = 0;
    MK(mcrt::launch_mlp_train(a, s), "train step (batch sums)");
    MK(mcrt::launch_stat_reduce((const double *)m->stat_partial.p, m->grid, (double *)m->bsum.p, s),
       "batch sums");
    bsum = (const double *)m->bsum.p;
    a.bsum = bsum;
  }
  a.pass = 1;
  MK(mcrt::launch_mlp_train(a, s), "train step");
  MK(mcrt::launch_grad_reduce((const float *)m->partial.p, (const double *)m->loss_partial.p, m->grid,
                              m->np, bsum, (float *)m->grad.p, (double *)m->loss.p, s),
     "gradient reduction");
  if (grad_out)
    MK(cudaMemcpyAsync(grad_out, m->grad.p, (size_t)m->np * sizeof(float), cudaMemcpyDeviceToDevice, s),
       "copy gradient");
  m->have_loss = true;
  m->last_stream = s;
  return MCRT_OK;
}

int mcrt_mlp_adam_step(mcrt_mlp *m, const float *grad, float lr, float beta1, float beta2, float eps,
                       void *stream) {
  if (!m) return MCRT_E_ARG;
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return mfail(m, MCRT_E_ARG, "bad Adam hyper-parameters");
  DeviceGuard dg(m->device);
  if (!dg.ok) return mfail(m, MCRT_E_CUDA, "cudaSetDevice");
  m->t += 1;
  const float c1 = (float)(1.0 - std::pow((double)beta1, m->t));
  const float c2 = (float)(1.0 - std::pow((double)beta2, m->t));
  MK(mcrt::launch_adam((float *)m->theta.p, (__half *)m->theta16.p,
                       grad ? grad : (const float *)m->grad.p, (float *)m->m1.p, (float *)m->m2.p,
                       m->np, lr, beta1, beta2, eps, c1, c2, (cudaStream_t)stream),
     "Adam step");
  return MCRT_OK;
}

int mcrt_mlp_last_loss(mcrt_mlp *m, double *loss) {
  if (!m) return MCRT_E_ARG;
  if (!loss) return mfail(m, MCRT_E_ARG, "null loss");
  if (!m->have_loss) return mfail(m, MCRT_E_STATE, "no loss yet");
  DeviceGuard dg(m->device);
  if (!dg.ok) return mfail(m, MCRT_E_CUDA, "cudaSetDevice");
  unsigned long long flag = 0;
  MK(cudaMemcpyAsync(loss, m->loss.p, sizeof(double), cudaMemcpyDeviceToHost, m->last_stream), "read loss");
  MK(cudaMemcpyAsync(&flag, m->errf.p, sizeof(flag), cudaMemcpyDeviceToHost, m->last_stream), "read flag");
  MK(cudaStreamSynchronize(m->last_stream), "sync");
  if (flag) {
    MK(cudaMemset(m->errf.p, 0, sizeof(flag)), "clear flag");
    return mfail(m, MCRT_E_ARG, "a batch index outside the dataset (its sample was skipped)");
  }
  return MCRT_OK;
}

const char *mcrt_mlp_last_error(const mcrt_mlp *m) { return m ? m->err.c_str() : ""; }

int mcrt_mlp_destroy(mcrt_mlp *m) {
  if (!m) return MCRT_OK;
  {
    DeviceGuard dg(m->device);
    cudaDeviceSynchronize();
    mlp_release(m);
    cudaGetLastError();
  }
  delete m;
  return MCRT_OK;
}

int mcrt_cell_features(mcrt_ctx *ctx, const int32_t *cells, int64_t n, float *out, void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (n < 0 || (n > 0 && !out)) return fail(ctx, MCRT_E_ARG, "bad arguments");
  if (ctx->grid.xz_walls)
    return fail(ctx, MCRT_E_UNSUPPORTED, "the features assume a channel (periodic x and z)");
  if (!cells && n > ncells_of(ctx)) return fail(ctx, MCRT_E_ARG, "n beyond the grid");
  const int rc = need_tables_and_fields(ctx);
  if (rc != MCRT_OK) return rc;
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const int rce = clear_lerr(ctx, s);
  if (rce != MCRT_OK) return rce;
  CK(mcrt::launch_features(feat_args(ctx, cells, n, out), s), "features");
  unsigned long long flag = 0;
  const int rcr = read_lerr(ctx, s, &flag);
  if (rcr != MCRT_OK) return rcr;
  if (flag) return fail(ctx, MCRT_E_ARG, "cell index outside the grid");
  return MCRT_OK;
}

int mcrt_tally_moments(mcrt_ctx *ctx, const mcrt_solve_params *p, const int32_t *cells, int64_t n,
                       float *mom_out, float *cost_out, double *q_out, double *sigma_out,
                       void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (!p) return fail(ctx, MCRT_E_ARG, "null params");
  if (n < 0 || (n > 0 && (!cells || !mom_out || !cost_out))) return fail(ctx, MCRT_E_ARG, "bad arguments");
  if (p->precision != MCRT_FP32) return fail(ctx, MCRT_E_ARG, "tallies come from the FP32 solve");
  if (p->estimator != MCRT_EST_ERMC) return fail(ctx, MCRT_E_ARG, "tallies come from the emission-based solve");
  if (p->use_box) return fail(ctx, MCRT_E_ARG, "tallies need the whole grid (use_box = 0)");
  int b[6];
  const int rc0 = check_solve_params(ctx, p, b);
  if (rc0 != MCRT_OK) return rc0;
  if (ctx->nb * ctx->ng > mcrt::kMaxTallyK) return fail(ctx, MCRT_E_UNSUPPORTED, "more than 1024 spectral points");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const int rcp = ensure_plain_proposal(ctx, s);
  if (rcp != MCRT_OK) return rcp;
  const int rce = clear_lerr(ctx, s);
  if (rce != MCRT_OK) return rce;
  mcrt::TraceArgs a;
  fill_trace_args(ctx, p, b, &a);
  const long long nbox = a.ncells_box;
  if (!q_out) {
    CK(ensure(ctx->q, nbox * sizeof(double)), "alloc q");
    q_out = (double *)ctx->q.p;
  }
  a.q = q_out;
  a.sigma = sigma_out;
  a.steps_cell = nullptr;
  const long long P = mcrt::fp32_bricks_positions(a.bnx, a.bny, a.bnz);
  long long Pc = ((long long)ctx->scratch_mib << 20) / ((long long)p->rays_per_cell * (long long)sizeof(float));
  if (Pc < 1) Pc = 1;
  if (Pc > P) Pc = P;
  CK(ensure(ctx->ybuf, (size_t)Pc * p->rays_per_cell * sizeof(float)), "alloc sample scratch");
  CK(ensure(ctx->step_acc, (size_t)Pc * sizeof(unsigned long long)), "alloc step scratch");
  CK(ensure(ctx->ray_steps, (size_t)Pc * p->rays_per_cell * sizeof(unsigned)), "alloc step scratch");
  a.ybuf = (float *)ctx->ybuf.p;
  a.step_acc = (unsigned long long *)ctx->step_acc.p;
  a.ray_steps = (unsigned *)ctx->ray_steps.p;
  const int rl = setup_long_rays(ctx, Pc * (long long)p->rays_per_cell, &a);
  if (rl != MCRT_OK) return rl;
  mcrt::TallyArgs t;
  std::memset(&t, 0, sizeof(t));
  t.cells = cells;
  t.n = n;
  t.nx = a.nx;
  t.ny = a.ny;
  t.nz = a.nz;
  t.ybuf = a.ybuf;
  t.ray_steps = a.ray_steps;
  t.N = p->rays_per_cell;
  t.key0 = a.key0;
  t.key1 = a.key1;
  t.snapshot = a.snapshot;
  t.ray_off = p->ray_offset;
  t.cn = a.cn;
  t.cg = a.cg;
  t.cell_cn = a.cell_cn;
  t.cell_cg = a.cell_cg;
  t.cell_hemi = a.cell_hemi;
  t.nb = ctx->nb;
  t.ng = ctx->ng;
  t.m_out = mom_out;
  t.c_out = cost_out;
  t.err = (unsigned long long *)ctx->lerr.p;
  CK(cudaMemsetAsync(ctx->counters.p, 0, mcrt::NCOUNTERS * sizeof(unsigned long long), s), "clear counters");
  ctx->kev_chunks = 0;
  CK(cudaEventRecord(ctx->ev0, s), "event");
  int launches = 0;
  for (long long p0 = 0; p0 < P; p0 += Pc) {
    a.chunk_p0 = t.chunk_p0 = p0;
    a.chunk_p1 = t.chunk_p1 = p0 + Pc < P ? p0 + Pc : P;
    int kn = 0;
    CK(mcrt::launch_trace_fp32(a, ctx->min_blocks, ctx->steps_per_round, s, nullptr, &kn), "trace launch");
    CK(mcrt::launch_tally(t, s), "tally launch");
    launches += kn + 1;
  }
  CK(cudaEventRecord(ctx->ev1, s), "event");
  ctx->last_launches = launches;
  ctx->last_stream = s;
  ctx->solved = true;
  ctx->last_T_max = ctx->prop_T_max;
  unsigned long long c5 = 0, flag = 0;
  CK(cudaMemcpyAsync(&c5, (unsigned long long *)ctx->counters.p + 5, sizeof(c5), cudaMemcpyDeviceToHost, s),
     "read error flag");
  const int rcr = read_lerr(ctx, s, &flag);
  if (rcr != MCRT_OK) return rcr;
  if (c5) return fail(ctx, MCRT_E_TIMEOUT, "trace kernel stopped without progress");
  if (flag) return fail(ctx, MCRT_E_ARG, "cell index outside the grid");
  return MCRT_OK;
}

int mcrt_get_plain_probs(mcrt_ctx *ctx, float *p0) {
  if (!ctx) return MCRT_E_ARG;
  if (!p0) return fail(ctx, MCRT_E_ARG, "null p0");
  if (!ctx->have_kdist || !ctx->have_fields) return fail(ctx, MCRT_E_STATE, "set kdist and fields first");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  const int rc = ensure_plain_proposal(ctx, nullptr);
  if (rc != MCRT_OK) return rc;
  CK(cudaDeviceSynchronize(), "sync");
  std::memcpy(p0, ctx->p0_host.data(), ctx->p0_host.size() * sizeof(float));
  return MCRT_OK;
}

int mcrt_set_cell_proposal_probs(mcrt_ctx *ctx, const float *q, void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (!q) return fail(ctx, MCRT_E_ARG, "null q");
  if (!ctx->have_kdist) return fail(ctx, MCRT_E_STATE, "set_kdist first");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->have_cell_prop = false;
  int rc = ensure_cell_buffers(ctx);
  if (rc == MCRT_OK) rc = clear_lerr(ctx, s);
  if (rc != MCRT_OK) return rc;
  CK(mcrt::launch_quantize_cells(q, ncells_of(ctx), ctx->nb, ctx->ng, (unsigned long long *)ctx->cell_cn.p,
                                 (unsigned long long *)ctx->cell_cg.p, (unsigned *)ctx->cell_hemi.p,
                                 (unsigned long long *)ctx->lerr.p, s),
     "quantise");
  unsigned long long flag = 0;
  rc = read_lerr(ctx, s, &flag);
  if (rc != MCRT_OK) return rc;
  if (flag) return fail(ctx, MCRT_E_ARG, "a cell without positive spectral weight");
  ctx->have_cell_prop = true;
  return MCRT_OK;
}

int mcrt_set_spectral_proposal(mcrt_ctx *ctx, int mode, void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (mode != MCRT_SPECTRAL_LOCAL && mode != MCRT_SPECTRAL_HYBRID) return fail(ctx, MCRT_E_ARG, "bad mode");
  int rc = need_tables_and_fields(ctx);
  if (rc != MCRT_OK) return rc;
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  rc = ensure_plain_proposal(ctx, s);  // p0 of the hybrid
  if (rc != MCRT_OK) return rc;
  ctx->have_cell_prop = false;
  rc = ensure_cell_buffers(ctx);
  if (rc == MCRT_OK) rc = clear_lerr(ctx, s);
  if (rc != MCRT_OK) return rc;
  mcrt::SpectralArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = ncells_of(ctx);
  a.nb = ctx->nb;
  a.ng = ctx->ng;
  a.nT = ctx->nT;
  a.mode = mode;
  a.T_min = ctx->T_min_field;
  a.T_max = proposal_T_max(ctx);
  a.fpos32 = (const uint2 *)ctx->fpos32.p;
  a.field64 = (const double2 *)ctx->field64.p;
  a.ktab32 = (const float2 *)ctx->ktab32.p;
  a.btab32 = (const float2 *)ctx->btab32.p;
  a.w_g32 = (const float *)ctx->wg32.p;
  a.p0 = (const float *)ctx->p0_32.p;
  a.cell_cn = (unsigned long long *)ctx->cell_cn.p;
  a.cell_cg = (unsigned long long *)ctx->cell_cg.p;
  a.cell_hemi = (unsigned *)ctx->cell_hemi.p;
  a.err = (unsigned long long *)ctx->lerr.p;
  CK(mcrt::launch_spectral_proposal(a, s), "spectral proposal");
  unsigned long long flag = 0;
  rc = read_lerr(ctx, s, &flag);
  if (rc != MCRT_OK) return rc;
  if (flag) return fail(ctx, MCRT_E_ARG, "a cell without positive spectral weight");
  ctx->have_cell_prop = true;
  return MCRT_OK;
}

int mcrt_get_cell_proposal(mcrt_ctx *ctx, uint64_t *cn, uint64_t *cg, uint32_t *hemi) {
  if (!ctx) return MCRT_E_ARG;
  if (!cn || !cg || !hemi) return fail(ctx, MCRT_E_ARG, "null output");
  if (!ctx->have_cell_prop) return fail(ctx, MCRT_E_STATE, "no cell proposal");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  const size_t nc = (size_t)ncells_of(ctx), nb = ctx->nb, ng = ctx->ng;
  CK(cudaDeviceSynchronize(), "sync");
  CK(cudaMemcpy(cn, ctx->cell_cn.p, nc * nb * sizeof(uint64_t), cudaMemcpyDeviceToHost), "copy cn");
  CK(cudaMemcpy(cg, ctx->cell_cg.p, nc * nb * ng * sizeof(uint64_t), cudaMemcpyDeviceToHost), "copy cg");
  CK(cudaMemcpy(hemi, ctx->cell_hemi.p, nc * sizeof(uint32_t), cudaMemcpyDeviceToHost), "copy hemi");
  return MCRT_OK;
}

int mcrt_set_learned_proposal(mcrt_ctx *ctx, mcrt_mlp *m, float mix, void *stream) {
  if (!ctx) return MCRT_E_ARG;
  if (!m) return fail(ctx, MCRT_E_ARG, "null network");
  if (ctx->grid.xz_walls)
    return fail(ctx, MCRT_E_UNSUPPORTED, "the features assume a channel (periodic x and z)");
  if (!(mix > 0.f && mix <= 1.f)) return fail(ctx, MCRT_E_ARG, "mix outside (0, 1]");
  int rc = need_tables_and_fields(ctx);
  if (rc != MCRT_OK) return rc;
  if (m->K != ctx->nb * ctx->ng) return fail(ctx, MCRT_E_ARG, "network outputs differ from n_bands n_g");
  if (m->device != ctx->grid.device) return fail(ctx, MCRT_E_ARG, "network on another device");
  DeviceGuard dg(ctx->grid.device);
  if (!dg.ok) return fail(ctx, MCRT_E_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  rc = ensure_plain_proposal(ctx, s);
  if (rc == MCRT_OK) rc = ensure_cell_buffers(ctx);
  if (rc == MCRT_OK) rc = clear_lerr(ctx, s);
  if (rc != MCRT_OK) return rc;
  ctx->have_cell_prop = false;
  const long long nc = ncells_of(ctx);
  CK(ensure(ctx->feat, (size_t)nc * MCRT_NFEAT * sizeof(float)), "alloc features");
  CK(mcrt::launch_features(feat_args(ctx, nullptr, nc, (float *)ctx->feat.p), s), "features");
  mcrt::MlpInferArgs a;
  std::memset(&a, 0, sizeof(a));
  a.theta16 = (const __half *)m->theta16.p;
  a.fmean = (const float *)m->nrm.p;
  a.finv = a.fmean + MCRT_NFEAT;
  a.K = m->K;
  a.p0 = (const float *)ctx->p0_32.p;
  a.p0_stride = 0;
  a.mix = mix;
  a.nb = ctx->nb;
  a.ng = ctx->ng;
  a.err = (unsigned long long *)ctx->lerr.p;
  // the network's probabilities for a chunk of cells, then their integer
  // proposal: the FP64 quantisation runs in its own kernel, with more warps per
  // SM than the network's shared-memory tiles allow
  const long long chunk = nc < (1LL << 20) ? nc : (1LL << 20);
  const long long K = m->K, KO = K + 2;
  CK(ensure(ctx->qprop, (size_t)chunk * KO * sizeof(float)), "alloc network outputs");
  for (long long c0 = 0; c0 < nc; c0 += chunk) {
    const long long cnum = nc - c0 < chunk ? nc - c0 : chunk;
    a.feat = (const float *)ctx->feat.p + c0 * MCRT_NFEAT;
    a.n = cnum;
    a.q_out = (float *)ctx->qprop.p;
    CK(mcrt::launch_mlp_infer(a, s), "network");
    CK(mcrt::launch_quantize_cells((const float *)ctx->qprop.p, cnum, ctx->nb, ctx->ng,
                                   (unsigned long long *)ctx->cell_cn.p + c0 * ctx->nb,
                                   (unsigned long long *)ctx->cell_cg.p + c0 * K,
                                   (unsigned *)ctx->cell_hemi.p + c0, (unsigned long long *)ctx->lerr.p, s),
       "quantise");
  }
  unsigned long long flag = 0;
  rc = read_lerr(ctx, s, &flag);
  if (rc != MCRT_OK) return rc;
  if (flag) return fail(ctx, MCRT_E_ARG, "network gave a cell without positive spectral weight");
  ctx->have_cell_prop = true;
  return MCRT_OK;
}

}  // extern "C"
