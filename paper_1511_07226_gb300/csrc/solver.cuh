// Method interface shared by the solver drivers (internal).
#pragma once

#include "pfk_internal.cuh"

namespace pfk {

// Everything a method's kernels need besides its own vectors.
struct SolveEnv {
  pfk_context* ctx;
  const pfk_operator* op;
  const pfk_pc* pc;          // null = identity
  cudaStream_t st;
  SolveCtl* ctl;             // device control block
  double* partials;          // reduction partials of the method's kernels
  int64_t partials_cap;      // doubles available at `partials`
  int64_t N;

  // True if a launch of `blocks` blocks writing `stride` partials each fits.
  bool partials_fit(int blocks, int stride) const { return (int64_t)blocks * stride <= partials_cap; }
  // The same for a two-level combine (block rows plus one row per group).
  bool partials_fit_2l(int blocks, int stride) const {
    return blocks <= kCombineGroup * kMaxCombineGroups &&
           (int64_t)(blocks + (blocks + kCombineGroup - 1) / kCombineGroup) * stride <= partials_cap;
  }
  cudaEvent_t pass_ev0, pass_ev1;   // profiling: recorded around the fused pass (or null)

  // out = add + B(v); B = identity when pc is null.
  cudaError_t pc_apply(const double* v, double* out, const double* add, const int* status) const;
  // Records pass_ev0 (which = 0) or pass_ev1 (1) if profiling.
  cudaError_t mark_pass(int which) const;
};

// A Krylov method as a pipeline fill plus a replayable iteration.
class Method {
 public:
  virtual ~Method() {}
  // FP64 words of workspace for n unknowns and window/restart length mmax.
  virtual int64_t workspace_doubles(int64_t N, int mmax) const = 0;
  virtual void bind(double* ws, int64_t N, int mmax) = 0;
  // One length-N vector the driver may use between phases (true residual).
  virtual double* scratch() = 0;
  // (Re)start from x: pipeline fill and the scalars of iteration 0; sets ctl->status.
  virtual cudaError_t fill(const SolveEnv& env, const double* b, double* x) = 0;
  // One iteration; every kernel is a no-op once ctl->status != kRun.
  virtual cudaError_t iteration(const SolveEnv& env, double* x) = 0;
  // Called by the driver when an iteration group stopped with status kRun at
  // the end of a restart cycle (GMRES types); default: nothing.
  virtual cudaError_t end_cycle(const SolveEnv& env, double* x) { (void)env; (void)x; return cudaSuccess; }
  // Number of ring/Hessenberg columns (GMRES types restart after this many).
  virtual int cycle_length() const { return 0; }
  // Once per solve, before bind: picks the persistent single-launch form when
  // the method has one, the problem is eligible and `mode` allows it (0 auto,
  // 1 never, 2 required).  Returns whether it did.
  virtual bool configure(const pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, int64_t N, int mode) {
    (void)ctx; (void)op; (void)pc; (void)N; (void)mode;
    return false;
  }
  // Once per solve, before the graphs are captured (e.g. the PIPEFGMRES shift
  // estimate); may synchronise.  `dscalar` is a device scalar slot; the method
  // reports the shift it uses (NaN if none) in *host_sigma.
  virtual cudaError_t prepare(const SolveEnv& env, const double* b, double* dscalar, double* host_sigma) {
    (void)env; (void)b; (void)dscalar;
    *host_sigma = NAN;
    return cudaSuccess;
  }
};

// Persistent single-launch iterations (persistent.cu): eligibility, and one
// cooperative launch of up to `iters` PIPEFCG (pipelined) or FCG iterations.
// FCG passes w, m0, m1, n, Q, Z as null.
constexpr int kPersistentIters = 16;
bool persistent_eligible(const pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, int method, int naive_like,
                         int64_t N);
cudaError_t launch_persistent(const SolveEnv& env, bool pipelined, int mmax, double* x, double* r, double* u,
                              double* w, double* m0, double* m1, double* n, double* P, double* S, double* Q,
                              double* Z, int iters);

Method* make_pipefcg(bool naive);
Method* make_pipegcr_w();
Method* make_pipefcg_theta();
Method* make_pipegcr();
Method* make_pipefgmres(double sigma);
Method* make_fcg();
Method* make_gcr();
Method* make_fgmres();

// ---------------------------------------------------------------------------
// Scalar phase shared by the CG- and CR-type methods (runs in one thread of the
// last block of the kernel that completed the iteration's reduction)
// ---------------------------------------------------------------------------

// Truncation (Sec. 5): standard nu_i = min(i, nu_max); restart-style
// nu_i = ((i - 1) mod nu_max) + 1.
__device__ __forceinline__ int nu_window(int i, int mmax, int truncation) {
  return truncation == PFK_TRUNC_RESTART ? ((i - 1) % mmax) + 1 : (i < mmax ? i : mmax);
}

__device__ __forceinline__ void push_history(SolveCtl* c, double rho, double rn, double eta, double alpha) {
  if (c->history && c->hist_len < c->hist_cap) {
    double* h = c->history + (size_t)c->hist_len * PFK_HISTORY_FIELDS;
    h[0] = rho; h[1] = rn; h[2] = eta; h[3] = alpha;
  }
  c->hist_len += 1;
}

__device__ __forceinline__ double cgcr_rho(const SolveCtl* ctl, double gamma, double rr) {
  return ctl->norm == PFK_NORM_NATURAL ? sqrt(fabs(gamma)) : sqrt(rr);
}

// Pipeline fill: gamma_0, eta_0 (= delta_0 for Alg. 8, <s_0, s_0> for Alg. 11),
// ||r_0||^2 -> rho_0, target, alpha_0 = gamma_0 / eta_0 and the fill status.
__device__ __forceinline__ void cgcr_fill_scalars(SolveCtl* ctl, double gamma, double eta, double rr) {
  const double rho = cgcr_rho(ctl, gamma, rr);
  if (!ctl->target_set) {
    ctl->rho0 = rho;
    ctl->target = fmax(ctl->rtol * rho, ctl->atol);
    ctl->target_set = 1;
  }
  const double al = eta != 0.0 ? gamma / eta : nan("");
  push_history(ctl, rho, sqrt(rr), eta, al);
  ctl->rho = rho;
  ctl->gamma = gamma;
  ctl->eta = eta;
  ctl->alpha = al;
  ctl->i = 0;
  ctl->nw = 0;
  ctl->eta_ring[0] = eta;
  if (!isfinite(rho)) ctl->status = kNonFinite;
  else if (rho <= ctl->target) ctl->status = kConverged;
  else if (eta <= 0.0) ctl->status = kFillBreakdown;
  else ctl->status = kRun;
}

// Iteration i once its reduction is complete: gamma_i, delta_i, ||r_i||^2 and
// the window dots c[jj] = <v_i, s_k>, k = i - nu_i + jj (v = u for Alg. 8,
// w for Alg. 11).  Convergence test first (as in the listings' order), then
// beta_{i,k} = -c_k / eta_k, eta_i = delta_i - sum_k beta_{i,k}^2 eta_k (k
// ascending), alpha_i = gamma_i / eta_i; eta_i <= 0 is a norm breakdown.
__device__ __forceinline__ void cgcr_iteration_scalars(SolveCtl* ctl, int i, int nu, double gamma, double delta,
                                                       double rr, const double* c) {
  const int slots = ctl->mmax + 1;
  ctl->it += 1;
  ctl->i = i;
  ctl->gamma = gamma;
  ctl->delta = delta;
  const double rnorm = sqrt(rr);
  const double rho = cgcr_rho(ctl, gamma, rr);
  ctl->rho = rho;
  const int hslot = ctl->hist_len;
  push_history(ctl, rho, rnorm, nan(""), nan(""));
  if (!isfinite(rho)) { ctl->status = kNonFinite; return; }
  if (rho <= ctl->target) { ctl->status = kConverged; return; }
  double sumb = 0.0;
  for (int jj = 0; jj < nu; ++jj) {
    const int k = i - nu + jj;
    const double ek = ctl->eta_ring[k % slots];
    const double b = -c[jj] / ek;
    ctl->beta[jj] = b;
    sumb += b * b * ek;
  }
  const double eta = delta - sumb;
  const double al = eta != 0.0 ? gamma / eta : nan("");
  ctl->eta = eta;
  ctl->alpha = al;
  ctl->nw = nu;
  ctl->eta_ring[i % slots] = eta;
  if (ctl->history && hslot < ctl->hist_cap) {
    ctl->history[(size_t)hslot * PFK_HISTORY_FIELDS + 2] = eta;
    ctl->history[(size_t)hslot * PFK_HISTORY_FIELDS + 3] = al;
  }
  if (eta <= 0.0) { ctl->status = kBreakdown; return; }
  if (ctl->it >= ctl->maxit) { ctl->status = kMaxit; return; }
}

// cgcr_iteration_scalars by all threads of the (last) block: the nu window
// betas -c_k / eta_k (each a global load of eta_k and a division) are formed
// in parallel, one per thread, and thread 0 accumulates eta_i in the same k
// order; everything else is thread 0's, in the same statement order.  c is
// the window's dots in k order (shared or global memory); s_tmp holds 2 * cap
// + 1 doubles of shared memory, cap >= nu.
__device__ __forceinline__ void cgcr_iteration_scalars_block(SolveCtl* ctl, int i, int nu, double gamma, double delta,
                                                             double rr, const double* c, double* s_tmp, int cap) {
  int* s_go = (int*)(s_tmp + 2 * cap);
  if (threadIdx.x == 0) {
    ctl->it += 1;
    ctl->i = i;
    ctl->gamma = gamma;
    ctl->delta = delta;
    const double rnorm = sqrt(rr);
    const double rho = cgcr_rho(ctl, gamma, rr);
    ctl->rho = rho;
    s_go[1] = ctl->hist_len;
    push_history(ctl, rho, rnorm, nan(""), nan(""));
    s_go[0] = 1;
    if (!isfinite(rho)) { ctl->status = kNonFinite; s_go[0] = 0; }
    else if (rho <= ctl->target) { ctl->status = kConverged; s_go[0] = 0; }
  }
  __syncthreads();
  if (!s_go[0]) return;
  const int slots = ctl->mmax + 1;
  if ((int)threadIdx.x < nu) {
    const int k = i - nu + (int)threadIdx.x;
    const double ek = ctl->eta_ring[k % slots];
    const double b = -c[threadIdx.x] / ek;
    ctl->beta[threadIdx.x] = b;
    s_tmp[threadIdx.x] = b * b;
    s_tmp[cap + threadIdx.x] = ek;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sumb = 0.0;
  for (int jj = 0; jj < nu; ++jj) sumb = fma(s_tmp[jj], s_tmp[cap + jj], sumb);
  const double eta = delta - sumb;
  const double al = eta != 0.0 ? gamma / eta : nan("");
  const int hslot = s_go[1];
  ctl->eta = eta;
  ctl->alpha = al;
  ctl->nw = nu;
  ctl->eta_ring[i % slots] = eta;
  if (ctl->history && hslot < ctl->hist_cap) {
    ctl->history[(size_t)hslot * PFK_HISTORY_FIELDS + 2] = eta;
    ctl->history[(size_t)hslot * PFK_HISTORY_FIELDS + 3] = al;
  }
  if (eta <= 0.0) { ctl->status = kBreakdown; return; }
  if (ctl->it >= ctl->maxit) { ctl->status = kMaxit; return; }
}

}  // namespace pfk
