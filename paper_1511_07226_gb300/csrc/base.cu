// The non-pipelined flexible methods on one GPU, as comparison baselines:
// FCG (Alg. 2), GCR (Alg. 9) and FGMRES (Alg. 13, classical Gram-Schmidt as
// printed).  Their reductions block: each iteration has two reduction phases
// whose results the very next kernel needs (FCG: gamma and the betas, then
// eta; GCR: the betas, then gamma and eta; FGMRES: the Gram-Schmidt
// coefficients, then the norm).  On one GPU "blocking" means a kernel
// boundary plus a last-block combine, with no host round trip.
#include "pfk_internal.cuh"
#include "solver.cuh"
#include "stencil.cuh"

#include <cmath>

namespace pfk {

constexpr int kBaseThreads = 128;
constexpr int kBaseBlocksPerSm = 6;
constexpr int kBaseStride = kBaseThreads + 1;
static_assert(kBaseBlocksPerSm <= kMaxBlocksPerSm, "partials are sized for kMaxBlocksPerSm blocks per SM");

// A CSR operator (stencil operators take the tiled walk).
struct CsrView {
  const int32_t* rowptr;
  const int32_t* colidx;
  const double* vals;
};

static CsrView csr_of(const pfk_operator* op) {
  CsrView A;
  A.rowptr = op->rowptr; A.colidx = op->colidx; A.vals = op->vals;
  return A;
}

// (A m)_r of a CSR operator.
__device__ __forceinline__ double base_row(const CsrView& A, const double* __restrict__ m, int64_t r) {
  double acc = 0.0;
  for (int32_t p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) acc = fma(A.vals[p], m[A.colidx[p]], acc);
  return acc;
}

// ---------------------------------------------------------------------------
// Building blocks
// ---------------------------------------------------------------------------

// x_i = x_{i-1} + alpha p_{i-1}, r_i = r_{i-1} - alpha s_{i-1} (slot of i-1).
__global__ void __launch_bounds__(kThreads) base_advance(double* __restrict__ x, double* __restrict__ r,
                                                         const double* __restrict__ P, const double* __restrict__ S,
                                                         int64_t N, const SolveCtl* ctl) {
  if (ctl->status != kRun) return;
  const double alpha = ctl->alpha;
  const size_t off = (size_t)(ctl->i % (ctl->mmax + 1)) * (size_t)N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    x[e] = fma(alpha, P[off + e], x[e]);
    r[e] = fma(-alpha, S[off + e], r[e]);
  }
}

// Dots of a vector v with r (<v, r>), of r with itself, and with the stored
// s_k of the window W_i (transposed through shared memory).  Mode FCG:
// v = u = B(r_i): convergence test on gamma_i = <u_i, r_i>, then the betas.
// Mode GCR: v = A u_i: the betas only.
enum { kDotsFcg = 0, kDotsGcr = 1 };

template <int NW>
__global__ void __launch_bounds__(kBaseThreads, kBaseBlocksPerSm) base_window_dots(const double* __restrict__ v,
                                                                                   const double* __restrict__ r,
                                                                                   const double* __restrict__ S,
                                                                                   int64_t N, SolveCtl* ctl,
                                                                                   double* partials, int mode) {
  if (ctl->status != kRun) return;
  constexpr int ND = NW + 2;
  constexpr int NWARPS = kBaseThreads / 32;
  __shared__ size_t s_off[NW];
  __shared__ double s_sk[NW * kBaseStride];
  __shared__ double s_v[kBaseThreads];
  __shared__ double s_red[NWARPS * ND];
  __shared__ double s_sum[ND];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = ctl->i + 1;
  const int nu = nu_window(i, ctl->mmax, ctl->truncation);
  const int slots = ctl->mmax + 1;
  if (threadIdx.x < nu) s_off[threadIdx.x] = (size_t)((i - nu + (int)threadIdx.x) % slots) * (size_t)N;
  __syncthreads();
  double* my = s_sk + threadIdx.x;
  const double* wv = s_v + warp * 32;
  const double* lrow = s_sk + lane * kBaseStride + warp * 32;
  double g0 = 0.0, g1 = 0.0, gw = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * kBaseThreads; base < N; base += (int64_t)gridDim.x * kBaseThreads) {
    const int64_t e = base + threadIdx.x;
    double vv = 0.0;
    if (e < N) {
      vv = v[e];
      const double rv = r[e];
      g0 = fma(vv, rv, g0);
      g1 = fma(rv, rv, g1);
#pragma unroll
      for (int j = 0; j < NW; ++j)
        if (j < nu) my[j * kBaseStride] = S[s_off[j] + e];
    } else {
#pragma unroll
      for (int j = 0; j < NW; ++j)
        if (j < nu) my[j * kBaseStride] = 0.0;
    }
    s_v[threadIdx.x] = vv;
    __syncwarp();
    if (lane < nu) {
      double c = gw;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) c = fma(wv[t], lrow[t], c);
      gw = c;
    }
    __syncwarp();
  }
  {
    const double w0 = warp_sum(g0), w1 = warp_sum(g1);
    const int nd = nu + 2;
    if (lane == 0) {
      s_red[warp * nd + 0] = w0;
      s_red[warp * nd + 1] = w1;
    }
    if (lane < nu) s_red[warp * nd + 2 + lane] = gw;
    __syncthreads();
  }
  if (!combine_block_partials_2l(s_red, nu + 2, partials, ND, &ctl->counter, ctl->gcounter, s_sum)) return;
  if (threadIdx.x != 0) return;
  const double* c = s_sum + 2;
  if (mode == kDotsFcg) {
    // Alg. 2: gamma_i = <u_i, r_i>, convergence, beta_{i,k} = -<u_i, s_k> / eta_k
    const double gamma = s_sum[0], rr = s_sum[1];
    ctl->it += 1;
    ctl->gamma = gamma;
    const double rho = cgcr_rho(ctl, gamma, rr);
    ctl->rho = rho;
    push_history(ctl, rho, sqrt(rr), nan(""), nan(""));
    if (!isfinite(rho)) { ctl->status = kNonFinite; return; }
    if (rho <= ctl->target) { ctl->status = kConverged; ctl->i = i; return; }
  }
  for (int jj = 0; jj < nu; ++jj) ctl->beta[jj] = -c[jj] / ctl->eta_ring[(i - nu + jj) % slots];
  ctl->nw = nu;
}

// p_i = u + sum_k beta_{i,k} p_k over W_i, into ring slot i.
template <int NW>
__global__ void __launch_bounds__(kThreads, 3) base_maxpy(const double* __restrict__ u, double* __restrict__ P,
                                                           int64_t N, const SolveCtl* ctl) {
  if (ctl->status != kRun) return;
  __shared__ double s_b[NW];
  __shared__ size_t s_off[NW];
  const int i = ctl->i + 1;
  const int nu = ctl->nw;
  const int slots = ctl->mmax + 1;
  if (threadIdx.x < nu) {
    s_b[threadIdx.x] = ctl->beta[threadIdx.x];
    s_off[threadIdx.x] = (size_t)((i - nu + (int)threadIdx.x) % slots) * (size_t)N;
  }
  __syncthreads();
  const size_t out = (size_t)(i % slots) * (size_t)N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    double p = u[e];
#pragma unroll 4
    for (int j = 0; j < nu; ++j) p = fma(s_b[j], P[s_off[j] + e], p);
    P[out + e] = p;
  }
}

// s = A p for p in ring slot `which` (0 = slot 0, 1 = slot i of the current
// iteration), with the dots <p, r>, <p, s>, <r, s>, <s, s>, <r, r>; the last
// block runs the mode's scalar step.
enum { kApplyFcgFill = 0, kApplyFcgEta = 1, kApplyGcrFill = 2, kApplyGcrFinal = 3 };

// The scalar step after s = A p and its five dots (last block, one thread).
__device__ __forceinline__ void base_apply_scalars(SolveCtl* ctl, int i, int slots, int mode, const double* s_sum) {
  const double pr = s_sum[0], ps = s_sum[1], rs = s_sum[2], ss = s_sum[3], rr = s_sum[4];
  if (mode == kApplyFcgFill) { cgcr_fill_scalars(ctl, pr, ps, rr); return; }        // gamma_0 = <u_0, r_0>, eta_0 = <p_0, s_0>
  if (mode == kApplyGcrFill) { cgcr_fill_scalars(ctl, rs, ss, rr); return; }        // gamma_0 = <r_0, s_0>, eta_0 = <s_0, s_0>
  if (mode == kApplyFcgEta) {
    // Alg. 2: eta_i = <p_i, s_i>, alpha_i = gamma_i / eta_i
    const double eta = ps;
    const double al = eta != 0.0 ? ctl->gamma / eta : nan("");
    ctl->i = i;
    ctl->eta = eta;
    ctl->alpha = al;
    ctl->eta_ring[i % slots] = eta;
    if (ctl->history && ctl->hist_len - 1 < ctl->hist_cap && ctl->hist_len >= 1) {
      ctl->history[(size_t)(ctl->hist_len - 1) * PFK_HISTORY_FIELDS + 2] = eta;
      ctl->history[(size_t)(ctl->hist_len - 1) * PFK_HISTORY_FIELDS + 3] = al;
    }
    if (eta <= 0.0) { ctl->status = kBreakdown; return; }
    if (ctl->it >= ctl->maxit) { ctl->status = kMaxit; return; }
    return;
  }
  // Alg. 9 (standard reading): gamma_i = <r_i, s_i>, eta_i = <s_i, s_i>; convergence,
  // then alpha_i = gamma_i / eta_i
  ctl->it += 1;
  ctl->i = i;
  ctl->gamma = rs;
  const double rho = cgcr_rho(ctl, rs, rr);
  ctl->rho = rho;
  const double al = ss != 0.0 ? rs / ss : nan("");
  push_history(ctl, rho, sqrt(rr), ss, al);
  if (!isfinite(rho)) { ctl->status = kNonFinite; return; }
  if (rho <= ctl->target) { ctl->status = kConverged; return; }
  ctl->eta = ss;
  ctl->alpha = al;
  ctl->eta_ring[i % slots] = ss;
  if (ss <= 0.0) { ctl->status = kBreakdown; return; }
  if (ctl->it >= ctl->maxit) { ctl->status = kMaxit; return; }
}

// CSR operators: one row per thread.
__global__ void __launch_bounds__(kThreads) base_apply_dots(CsrView A, double* __restrict__ P,
                                                            double* __restrict__ S, const double* __restrict__ r,
                                                            int64_t N, SolveCtl* ctl, double* partials, int mode) {
  if (ctl->status != kRun) return;
  const bool fill = (mode == kApplyFcgFill || mode == kApplyGcrFill);
  const int i = fill ? 0 : ctl->i + 1;
  const int slots = ctl->mmax + 1;
  const size_t off = (size_t)(i % slots) * (size_t)N;
  const double* p = P + off;
  double* s = S + off;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const double sv = base_row(A, p, e);
    s[e] = sv;
    const double pv = p[e], rv = r[e];
    acc[0] = fma(pv, rv, acc[0]);
    acc[1] = fma(pv, sv, acc[1]);
    acc[2] = fma(rv, sv, acc[2]);
    acc[3] = fma(sv, sv, acc[3]);
    acc[4] = fma(rv, rv, acc[4]);
  }
  __shared__ double s_red[(kThreads / 32) * 5];
  __shared__ double s_sum[5];
  if (!reduce_last_block<5>(acc, 5, partials, 5, &ctl->counter, s_red, s_sum)) return;
  if (threadIdx.x != 0) return;
  base_apply_scalars(ctl, i, slots, mode, s_sum);
}

// Stencil operators: the same step on the tiled z-marching walk (s = A p and
// the five dots in its epilogue, r prefetched one plane ahead).
struct BaseApplyEpi {
  double* __restrict__ s;
  const double* __restrict__ r;
  double acc[5];
  struct Pre {
    double r;
  };
  __device__ __forceinline__ Pre pre(int64_t c) const { return Pre{r[c]}; }
  __device__ __forceinline__ void operator()(int64_t c, double sv, double pv, const Pre& p) {
    s[c] = sv;
    acc[0] = fma(pv, p.r, acc[0]);
    acc[1] = fma(pv, sv, acc[1]);
    acc[2] = fma(p.r, sv, acc[2]);
    acc[3] = fma(sv, sv, acc[3]);
    acc[4] = fma(p.r, p.r, acc[4]);
  }
};

template <bool ADV>
__global__ void __launch_bounds__(kTileThreads) base_apply_dots_walk(TiledStencil<double, double> T,
                                                                     double* __restrict__ P, double* __restrict__ S,
                                                                     const double* __restrict__ r, int64_t N,
                                                                     SolveCtl* ctl, double* partials, int mode) {
  if (ctl->status != kRun) return;
  const bool fill = (mode == kApplyFcgFill || mode == kApplyGcrFill);
  const int i = fill ? 0 : ctl->i + 1;
  const int slots = ctl->mmax + 1;
  const size_t off = (size_t)(i % slots) * (size_t)N;
  BaseApplyEpi e{S + off, r, {0.0, 0.0, 0.0, 0.0, 0.0}};
  tiled_stencil_walk<double, double, ADV, 1>(T, P + off, e);
  __shared__ double s_red[(kTileThreads / 32) * 5];
  __shared__ double s_sum[5];
  if (!reduce_last_block<5>(e.acc, 5, partials, 5, &ctl->counter, s_red, s_sum)) return;
  if (threadIdx.x != 0) return;
  base_apply_scalars(ctl, i, slots, mode, s_sum);
}

static int base_template(int mmax) { return mmax <= 8 ? 8 : mmax <= 16 ? 16 : 32; }

static cudaError_t launch_window_dots(const SolveEnv& env, int tmpl, const double* v, const double* r,
                                      const double* S, int mode) {
  const int64_t need = (env.N + kBaseThreads - 1) / kBaseThreads;
  const int64_t cap = (int64_t)env.ctx->num_sms * kBaseBlocksPerSm;
  const int blocks = (int)(need < cap ? need : cap);
  if (!env.partials_fit_2l(blocks, tmpl + 2)) return cudaErrorInvalidValue;
  switch (tmpl) {
    case 8: base_window_dots<8><<<blocks, kBaseThreads, 0, env.st>>>(v, r, S, env.N, env.ctl, env.partials, mode); break;
    case 16: base_window_dots<16><<<blocks, kBaseThreads, 0, env.st>>>(v, r, S, env.N, env.ctl, env.partials, mode); break;
    default: base_window_dots<32><<<blocks, kBaseThreads, 0, env.st>>>(v, r, S, env.N, env.ctl, env.partials, mode); break;
  }
  return cudaGetLastError();
}

static cudaError_t launch_maxpy(const SolveEnv& env, int tmpl, const double* u, double* P) {
  const int blocks = stream_blocks(env.ctx, env.N, 4);
  switch (tmpl) {
    case 8: base_maxpy<8><<<blocks, kThreads, 0, env.st>>>(u, P, env.N, env.ctl); break;
    case 16: base_maxpy<16><<<blocks, kThreads, 0, env.st>>>(u, P, env.N, env.ctl); break;
    default: base_maxpy<32><<<blocks, kThreads, 0, env.st>>>(u, P, env.N, env.ctl); break;
  }
  return cudaGetLastError();
}

static cudaError_t launch_apply_dots(const SolveEnv& env, double* P, double* S, const double* r, int mode) {
  const pfk_operator* op = env.op;
  if (!op->rowptr) {
    TiledStencil<double, double> T;
    const bool adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
    const int slots = adv ? tiled_stencil_slots(base_apply_dots_walk<true>, env.ctx->num_sms)
                          : tiled_stencil_slots(base_apply_dots_walk<false>, env.ctx->num_sms);
    const int units = tiled_stencil_setup<double, double>(T, op, op->d, op->kx, op->ky, op->kz, slots);
    const int64_t cap = env.partials_cap / 5;
    const int blocks = (int)(units < cap ? units : cap);
    if (adv) base_apply_dots_walk<true><<<blocks, kTileThreads, 0, env.st>>>(T, P, S, r, env.N, env.ctl, env.partials, mode);
    else base_apply_dots_walk<false><<<blocks, kTileThreads, 0, env.st>>>(T, P, S, r, env.N, env.ctl, env.partials, mode);
    return cudaGetLastError();
  }
  const int blocks = stream_blocks(env.ctx, env.N, 2);
  if (!env.partials_fit(blocks, 5)) return cudaErrorInvalidValue;
  base_apply_dots<<<blocks, kThreads, 0, env.st>>>(csr_of(env.op), P, S, r, env.N, env.ctl, env.partials, mode);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FCG (Alg. 2)
// ---------------------------------------------------------------------------

class Fcg : public Method {
 public:
  int64_t workspace_doubles(int64_t N, int mmax) const override { return 3 * N + 2 * (int64_t)(mmax + 1) * N; }
  void bind(double* ws, int64_t N, int mmax) override {
    N_ = N; mmax_ = mmax;
    r_ = ws; u_ = r_ + N; tmp_ = u_ + N;
    P_ = tmp_ + N; S_ = P_ + (mmax + 1) * N;
  }
  double* scratch() override { return tmp_; }
  bool configure(const pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, int64_t N, int mode) override {
    persistent_ = mode != 1 && persistent_eligible(ctx, op, pc, PFK_FCG, 0, N);
    return persistent_;
  }
  cudaError_t fill(const SolveEnv& env, const double* b, double* x) override {
    cudaError_t e;
    if ((e = op_apply(env.op, x, r_, b, nullptr, env.st)) != cudaSuccess) return e;   // r_0 = b - A x_0
    if ((e = env.pc_apply(r_, P_, nullptr, nullptr)) != cudaSuccess) return e;       // p_0 = u_0 = B(r_0)
    return launch_apply_dots(env, P_, S_, r_, kApplyFcgFill);                          // s_0 = A p_0, gamma_0, eta_0
  }
  cudaError_t iteration(const SolveEnv& env, double* x) override {
    if (persistent_) {
      cudaError_t e = env.mark_pass(0);
      if (e != cudaSuccess) return e;
      e = launch_persistent(env, false, mmax_, x, r_, u_, nullptr, nullptr, nullptr, nullptr, P_, S_, nullptr,
                            nullptr, kPersistentIters);
      if (e != cudaSuccess) return e;
      return env.mark_pass(1);
    }
    const int* status = &env.ctl->status;
    const int tmpl = base_template(mmax_);
    cudaError_t e;
    base_advance<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, env.st>>>(x, r_, P_, S_, N_, env.ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = env.pc_apply(r_, u_, nullptr, status)) != cudaSuccess) return e;         // u_i = B(r_i)
    if ((e = env.mark_pass(0)) != cudaSuccess) return e;
    if ((e = launch_window_dots(env, tmpl, u_, r_, S_, kDotsFcg)) != cudaSuccess) return e;   // gamma_i, betas
    if ((e = launch_maxpy(env, tmpl, u_, P_)) != cudaSuccess) return e;                // p_i
    if ((e = launch_apply_dots(env, P_, S_, r_, kApplyFcgEta)) != cudaSuccess) return e;      // s_i, eta_i, alpha_i
    return env.mark_pass(1);
  }

 private:
  int64_t N_ = 0;
  int mmax_ = 0;
  bool persistent_ = false;
  double *r_ = nullptr, *u_ = nullptr, *tmp_ = nullptr, *P_ = nullptr, *S_ = nullptr;
};

// ---------------------------------------------------------------------------
// GCR (Alg. 9)
// ---------------------------------------------------------------------------

class Gcr : public Method {
 public:
  int64_t workspace_doubles(int64_t N, int mmax) const override { return 4 * N + 2 * (int64_t)(mmax + 1) * N; }
  void bind(double* ws, int64_t N, int mmax) override {
    N_ = N; mmax_ = mmax;
    r_ = ws; u_ = r_ + N; au_ = u_ + N; tmp_ = au_ + N;
    P_ = tmp_ + N; S_ = P_ + (mmax + 1) * N;
  }
  double* scratch() override { return tmp_; }
  cudaError_t fill(const SolveEnv& env, const double* b, double* x) override {
    cudaError_t e;
    if ((e = op_apply(env.op, x, r_, b, nullptr, env.st)) != cudaSuccess) return e;   // r_0
    if ((e = env.pc_apply(r_, P_, nullptr, nullptr)) != cudaSuccess) return e;       // p_0 = u_0 = B(r_0)
    return launch_apply_dots(env, P_, S_, r_, kApplyGcrFill);                          // s_0, gamma_0, eta_0
  }
  cudaError_t iteration(const SolveEnv& env, double* x) override {
    const int* status = &env.ctl->status;
    const int tmpl = base_template(mmax_);
    cudaError_t e;
    base_advance<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, env.st>>>(x, r_, P_, S_, N_, env.ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = env.pc_apply(r_, u_, nullptr, status)) != cudaSuccess) return e;         // u_i = B(r_i)
    if ((e = env.mark_pass(0)) != cudaSuccess) return e;
    if ((e = op_apply(env.op, u_, au_, nullptr, status, env.st)) != cudaSuccess) return e;   // A u_i
    if ((e = launch_window_dots(env, tmpl, au_, r_, S_, kDotsGcr)) != cudaSuccess) return e;  // betas
    if ((e = launch_maxpy(env, tmpl, u_, P_)) != cudaSuccess) return e;                // p_i
    if ((e = launch_apply_dots(env, P_, S_, r_, kApplyGcrFinal)) != cudaSuccess) return e;    // s_i, gamma, eta
    return env.mark_pass(1);
  }

 private:
  int64_t N_ = 0;
  int mmax_ = 0;
  double *r_ = nullptr, *u_ = nullptr, *au_ = nullptr, *tmp_ = nullptr, *P_ = nullptr, *S_ = nullptr;
};

// ---------------------------------------------------------------------------
// FGMRES (Alg. 13)
// ---------------------------------------------------------------------------

constexpr int kGm = PFK_MAX_MMAX;

struct FgState {
  double H[(kGm + 1) * kGm];
  double R[(kGm + 1) * kGm];
  double cs[kGm], sn[kGm];
  double g[kGm + 1];
  double y[kGm];
  double inv;
  int k;        // column being formed
  int ncols;
};

// beta = ||r_0||, convergence, g = beta e_0.
__global__ void __launch_bounds__(kThreads) fgb_fill_norm(const double* __restrict__ r, int64_t N, SolveCtl* ctl,
                                                          FgState* gs, double* partials) {
  double acc[1] = {0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    acc[0] = fma(r[e], r[e], acc[0]);
  __shared__ double s_red[kThreads / 32];
  __shared__ double s_sum[1];
  if (!reduce_last_block<1>(acc, 1, partials, 1, &ctl->counter, s_red, s_sum)) return;
  if (threadIdx.x != 0) return;
  const double beta = sqrt(s_sum[0]);
  if (!ctl->target_set) {
    ctl->rho0 = beta;
    ctl->target = fmax(ctl->rtol * beta, ctl->atol);
    ctl->target_set = 1;
  }
  push_history(ctl, beta, beta, nan(""), nan(""));
  ctl->rho = beta;
  ctl->i = 0;
  gs->g[0] = beta;
  gs->k = 0;
  gs->ncols = 0;
  gs->inv = beta != 0.0 ? 1.0 / beta : 0.0;
  if (!isfinite(beta)) ctl->status = kNonFinite;
  else if (beta <= ctl->target) ctl->status = kConverged;
  else if (ctl->it >= ctl->maxit) ctl->status = kMaxit;
  else ctl->status = kRun;
}

// slot k of P (k = gs->k) scaled by gs->inv in place, and copied to `cur`.
__global__ void __launch_bounds__(kThreads) fgb_scale(const double* __restrict__ src, double* __restrict__ P,
                                                      double* __restrict__ cur, int64_t N, const FgState* gs,
                                                      const int* status) {
  if (*status != kRun) return;
  const double inv = gs->inv;
  const size_t off = (size_t)gs->k * (size_t)N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (src ? src[e] : P[off + e]) * inv;
    P[off + e] = v;
    cur[e] = v;
  }
}

// z = A u_k, and u_k stored in slot k of U (CSR operators).
__global__ void __launch_bounds__(kThreads) fgb_apply_store(CsrView A, const double* __restrict__ ucur,
                                                            double* __restrict__ U, double* __restrict__ z, int64_t N,
                                                            const FgState* gs, const int* status) {
  if (*status != kRun) return;
  const size_t off = (size_t)gs->k * (size_t)N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    z[e] = base_row(A, ucur, e);
    U[off + e] = ucur[e];
  }
}

// Stencil operators: z = A u and the copy of u into U on the tiled walk.
struct FgStoreEpi {
  double* __restrict__ z;
  double* __restrict__ u;
  struct Pre {};
  __device__ __forceinline__ Pre pre(int64_t) const { return Pre{}; }
  __device__ __forceinline__ void operator()(int64_t c, double zv, double uv, const Pre&) const {
    z[c] = zv;
    u[c] = uv;
  }
};

template <bool ADV>
__global__ void __launch_bounds__(kTileThreads) fgb_apply_store_walk(TiledStencil<double, double> T,
                                                                     const double* __restrict__ ucur,
                                                                     double* __restrict__ U, double* __restrict__ z,
                                                                     int64_t N, const FgState* gs, const int* status) {
  if (*status != kRun) return;
  FgStoreEpi e{z, U + (size_t)gs->k * (size_t)N};
  tiled_stencil_walk<double, double, ADV, 1>(T, ucur, e);
}

static cudaError_t launch_apply_store(const SolveEnv& env, const double* ucur, double* U, double* z,
                                      const FgState* gs, const int* status) {
  const pfk_operator* op = env.op;
  if (!op->rowptr) {
    TiledStencil<double, double> T;
    const bool adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
    const int slots = adv ? tiled_stencil_slots(fgb_apply_store_walk<true>, env.ctx->num_sms)
                          : tiled_stencil_slots(fgb_apply_store_walk<false>, env.ctx->num_sms);
    const int units = tiled_stencil_setup<double, double>(T, op, op->d, op->kx, op->ky, op->kz, slots);
    if (adv) fgb_apply_store_walk<true><<<units, kTileThreads, 0, env.st>>>(T, ucur, U, z, env.N, gs, status);
    else fgb_apply_store_walk<false><<<units, kTileThreads, 0, env.st>>>(T, ucur, U, z, env.N, gs, status);
  } else {
    fgb_apply_store<<<stream_blocks(env.ctx, env.N, 8), kThreads, 0, env.st>>>(csr_of(op), ucur, U, z, env.N, gs,
                                                                               status);
  }
  return cudaGetLastError();
}

// Classical Gram-Schmidt coefficients h_{j,k} = <p_j, z_k>, j <= k (transposed dots).
template <int NW>
__global__ void __launch_bounds__(kBaseThreads, kBaseBlocksPerSm) fgb_dots(const double* __restrict__ z,
                                                                           const double* __restrict__ P, int64_t N,
                                                                           SolveCtl* ctl, FgState* gs,
                                                                           double* partials) {
  if (ctl->status != kRun) return;
  constexpr int ND = NW;
  constexpr int NWARPS = kBaseThreads / 32;
  __shared__ double s_pk[NW * kBaseStride];
  __shared__ double s_z[kBaseThreads];
  __shared__ double s_red[NWARPS * ND];
  __shared__ double s_sum[ND];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nk = gs->k + 1;           // p_0 .. p_k
  double* my = s_pk + threadIdx.x;
  const double* wz = s_z + warp * 32;
  const double* lrow = s_pk + lane * kBaseStride + warp * 32;
  double gw = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * kBaseThreads; base < N; base += (int64_t)gridDim.x * kBaseThreads) {
    const int64_t e = base + threadIdx.x;
    double zv = 0.0;
    if (e < N) {
      zv = z[e];
#pragma unroll
      for (int j = 0; j < NW; ++j)
        if (j < nk) my[j * kBaseStride] = P[(size_t)j * (size_t)N + e];
    } else {
#pragma unroll
      for (int j = 0; j < NW; ++j)
        if (j < nk) my[j * kBaseStride] = 0.0;
    }
    s_z[threadIdx.x] = zv;
    __syncwarp();
    if (lane < nk) {
      double c = gw;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) c = fma(wz[t], lrow[t], c);
      gw = c;
    }
    __syncwarp();
  }
  if (lane < nk) s_red[warp * nk + lane] = gw;
  __syncthreads();
  if (!combine_block_partials_2l(s_red, nk, partials, ND, &ctl->counter, ctl->gcounter, s_sum)) return;
  if (threadIdx.x != 0) return;
  for (int j = 0; j < nk; ++j) gs->H[j * kGm + gs->k] = s_sum[j];
}

// pbar = z_k - sum_j h_{j,k} p_j into slot k+1, and ||pbar||^2; the last block
// finishes column k: h_{k+1,k}, Givens, estimate, status.
template <int NW>
__global__ void __launch_bounds__(kThreads, 3) fgb_orth(const double* __restrict__ z, double* __restrict__ P,
                                                        int64_t N, SolveCtl* ctl, FgState* gs, int m,
                                                        double* partials) {
  if (ctl->status != kRun) return;
  __shared__ double s_h[NW];
  const int k = gs->k;
  const int nk = k + 1;
  if (threadIdx.x < nk) s_h[threadIdx.x] = gs->H[threadIdx.x * kGm + k];
  __syncthreads();
  const size_t out = (size_t)(k + 1) * (size_t)N;
  double acc[1] = {0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    double v = z[e];
#pragma unroll 4
    for (int j = 0; j < nk; ++j) v = fma(-s_h[j], P[(size_t)j * (size_t)N + e], v);
    if (k + 1 < m) P[out + e] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  __shared__ double s_red[kThreads / 32];
  __shared__ double s_sum[1];
  if (!reduce_last_block<1>(acc, 1, partials, 1, &ctl->counter, s_red, s_sum)) return;
  if (threadIdx.x != 0) return;
  const double h = sqrt(s_sum[0]);
  gs->H[(k + 1) * kGm + k] = h;
  ctl->it += 1;
  gs->ncols = k + 1;
  ctl->i = k + 1;
  for (int j = 0; j <= k + 1; ++j) gs->R[j * kGm + k] = gs->H[j * kGm + k];
  for (int j = 0; j < k; ++j) {
    const double a = gs->R[j * kGm + k], b = gs->R[(j + 1) * kGm + k];
    gs->R[j * kGm + k] = gs->cs[j] * a + gs->sn[j] * b;
    gs->R[(j + 1) * kGm + k] = -gs->sn[j] * a + gs->cs[j] * b;
  }
  const double a = gs->R[k * kGm + k], b = gs->R[(k + 1) * kGm + k];
  const double rr = hypot(a, b);
  const double c = rr != 0.0 ? a / rr : 1.0, s = rr != 0.0 ? b / rr : 0.0;
  gs->cs[k] = c;
  gs->sn[k] = s;
  gs->R[k * kGm + k] = rr;
  gs->R[(k + 1) * kGm + k] = 0.0;
  gs->g[k + 1] = -s * gs->g[k];
  gs->g[k] = c * gs->g[k];
  const double est = fabs(gs->g[k + 1]);
  ctl->rho = est;
  push_history(ctl, est, nan(""), nan(""), h);
  gs->inv = h != 0.0 ? 1.0 / h : 0.0;
  gs->k = k + 1;
  if (!isfinite(est)) { ctl->status = kNonFinite; return; }
  if (est <= ctl->target || h == 0.0) { ctl->status = kConverged; return; }
  if (k + 1 == m) { ctl->status = kCycleEnd; return; }
  if (ctl->it >= ctl->maxit) { ctl->status = kMaxit; return; }
}

__global__ void fgb_lsq(FgState* gs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n = gs->ncols;
  for (int j = n - 1; j >= 0; --j) {
    double s = gs->g[j];
    for (int l = j + 1; l < n; ++l) s -= gs->R[j * kGm + l] * gs->y[l];
    gs->y[j] = s / gs->R[j * kGm + j];
  }
}

__global__ void __launch_bounds__(kThreads) fgb_update_x(double* __restrict__ x, const double* __restrict__ U,
                                                         int64_t N, const FgState* gs) {
  const int n = gs->ncols;
  if (n == 0) return;
  __shared__ double s_y[kGm];
  if (threadIdx.x < n) s_y[threadIdx.x] = gs->y[threadIdx.x];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    double v = x[e];
    for (int j = 0; j < n; ++j) v = fma(s_y[j], U[(size_t)j * (size_t)N + e], v);
    x[e] = v;
  }
}

class Fgmres : public Method {
 public:
  int64_t workspace_doubles(int64_t N, int m) const override {
    return state_doubles() + 5 * N + (int64_t)(m + 1) * N + (int64_t)m * N;
  }
  void bind(double* ws, int64_t N, int m) override {
    N_ = N; m_ = m;
    gs_ = (FgState*)ws;
    double* v = ws + state_doubles();
    r_ = v; z_ = r_ + N; pcur_ = z_ + N; ucur_ = pcur_ + N; tmp_ = ucur_ + N;
    P_ = tmp_ + N; U_ = P_ + (int64_t)(m + 1) * N;
  }
  double* scratch() override { return tmp_; }
  int cycle_length() const override { return m_; }
  cudaError_t fill(const SolveEnv& env, const double* b, double* x) override {
    const int* status = &env.ctl->status;
    const int blocks = stream_blocks(env.ctx, N_, 2);
    if (!env.partials_fit(blocks, 1)) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = op_apply(env.op, x, r_, b, nullptr, env.st)) != cudaSuccess) return e;        // r_0
    fgb_fill_norm<<<blocks, kThreads, 0, env.st>>>(r_, N_, env.ctl, gs_, env.partials);      // beta
    fgb_scale<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, env.st>>>(r_, P_, pcur_, N_, gs_, status);  // p_0
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = env.pc_apply(pcur_, ucur_, nullptr, status)) != cudaSuccess) return e;       // u_0 = B(p_0)
    return launch_apply_store(env, ucur_, U_, z_, gs_, status);                            // z_0 = A u_0
  }
  cudaError_t iteration(const SolveEnv& env, double* x) override {
    (void)x;
    const int* status = &env.ctl->status;
    const int tmpl = base_template(m_ + 1);
    const int64_t need = (N_ + kBaseThreads - 1) / kBaseThreads;
    const int64_t cap = (int64_t)env.ctx->num_sms * kBaseBlocksPerSm;
    const int dblocks = (int)(need < cap ? need : cap);
    const int oblocks = stream_blocks(env.ctx, N_, 2);
    if (!env.partials_fit_2l(dblocks, tmpl) || !env.partials_fit(oblocks, 1)) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = env.mark_pass(0)) != cudaSuccess) return e;
    switch (tmpl) {
      case 8:
        fgb_dots<8><<<dblocks, kBaseThreads, 0, env.st>>>(z_, P_, N_, env.ctl, gs_, env.partials);
        fgb_orth<8><<<oblocks, kThreads, 0, env.st>>>(z_, P_, N_, env.ctl, gs_, m_, env.partials);
        break;
      case 16:
        fgb_dots<16><<<dblocks, kBaseThreads, 0, env.st>>>(z_, P_, N_, env.ctl, gs_, env.partials);
        fgb_orth<16><<<oblocks, kThreads, 0, env.st>>>(z_, P_, N_, env.ctl, gs_, m_, env.partials);
        break;
      default:
        fgb_dots<32><<<dblocks, kBaseThreads, 0, env.st>>>(z_, P_, N_, env.ctl, gs_, env.partials);
        fgb_orth<32><<<oblocks, kThreads, 0, env.st>>>(z_, P_, N_, env.ctl, gs_, m_, env.partials);
        break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = env.mark_pass(1)) != cudaSuccess) return e;
    fgb_scale<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, env.st>>>(nullptr, P_, pcur_, N_, gs_, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;                              // p_k = pbar / h
    if ((e = env.pc_apply(pcur_, ucur_, nullptr, status)) != cudaSuccess) return e;    // u_k = B(p_k)
    return launch_apply_store(env, ucur_, U_, z_, gs_, status);                          // z_k = A u_k
  }
  cudaError_t end_cycle(const SolveEnv& env, double* x) override {
    fgb_lsq<<<1, 32, 0, env.st>>>(gs_);
    fgb_update_x<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, env.st>>>(x, U_, N_, gs_);
    return cudaGetLastError();
  }

 private:
  static int64_t state_doubles() { return (int64_t)((sizeof(FgState) + 255) / 256 * 256 / sizeof(double)); }
  int64_t N_ = 0;
  int m_ = 0;
  FgState* gs_ = nullptr;
  double *r_ = nullptr, *z_ = nullptr, *pcur_ = nullptr, *ucur_ = nullptr, *tmp_ = nullptr;
  double *P_ = nullptr, *U_ = nullptr;
};

Method* make_fcg() { return new Fcg(); }
Method* make_gcr() { return new Gcr(); }
Method* make_fgmres() { return new Fgmres(); }

}  // namespace pfk
