// Nested flexible Krylov solve as a preconditioner: the block upper-triangular
// preconditioner of the paper's Stokes experiment (Sec. 6, ex43),
//
//   B = [K_hat  B^T ; 0  S_hat]^-1:   y_p = S_hat^-1 v_p,
//                                      y_u = K_hat^-1 (v_u - B^T y_p),
//
// with S_hat diagonal and K_hat^-1 an inexact inner solve of the viscous block
// by a (pipelined) flexible Krylov method with Jacobi, from zero, ending at
// the inner tolerance, at the iteration limit or at a norm breakdown (no
// restarts, no true-residual check).  Every step runs on the device with its
// scalars in the inner solve's own control block, so an application is a
// fixed sequence of launches (pre, B^T SpMV, inner fill, inner_maxit inner
// iterations, post) that the outer solve's CUDA graph records like any other
// preconditioner; inner iterations after the inner solve stopped are no-ops.
#include "pfk_internal.cuh"
#include "solver.cuh"

#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

namespace pfk {

Method* make_inner_method(int method);
pfk_status create_pc(pfk_context* ctx, const pfk_operator* op, const pfk_pc_desc* desc, pfk_pc* pc);

struct NestedState {
  const pfk_operator* K = nullptr;    // viscous block (nu unknowns)
  const pfk_operator* Bt = nullptr;   // B^T on the full vector (zero pressure rows)
  int64_t N = 0, nu = 0;
  int maxit = 0;
  double* sinv = nullptr;             // 1 / S_hat (N - nu)
  double* y = nullptr;                // the application's result before `add` (N)
  double* t = nullptr;                // v - B^T y_p (N; the first nu entries are the inner rhs)
  double* ws = nullptr;               // inner method's vectors
  SolveCtl* ctl = nullptr;            // inner solve's control block
  double* partials = nullptr;
  int64_t partials_cap = 0;
  pfk_pc* jacobi = nullptr;           // inner preconditioner
  std::unique_ptr<Method> M;
};

// y_u = 0 (inner initial guess), y_p = S_hat^-1 v_p, and the inner control
// block reset.  When the outer solve is no longer running the inner target is
// set to +inf, so the inner fill reports convergence and the inner iterations
// do nothing.
__global__ void __launch_bounds__(kThreads) nested_pre_kernel(const double* __restrict__ v, double* __restrict__ y,
                                                              const double* __restrict__ sinv, int64_t N,
                                                              int64_t nu, SolveCtl* ictl,
                                                              const int* __restrict__ status) {
  const bool run = !status || *status == kRun;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ictl->status = kRun;
    ictl->it = 0;
    ictl->i = 0;
    ictl->nw = 0;
    ictl->hist_len = 0;
    ictl->counter = 0u;
    ictl->target_set = run ? 0 : 1;
    ictl->target = run ? 0.0 : INFINITY;
  }
  if (!run) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = e < nu ? 0.0 : sinv[e - nu] * v[e];
}

// out = add + y
__global__ void __launch_bounds__(kThreads) nested_post_kernel(const double* __restrict__ y,
                                                               const double* __restrict__ add,
                                                               double* __restrict__ out, int64_t N,
                                                               const int* __restrict__ status) {
  if (status && *status != kRun) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = add ? add[e] + y[e] : y[e];
}

cudaError_t nested_apply(const pfk_pc* pc, const double* v, double* out, const double* add, const int* status,
                         cudaStream_t st) {
  NestedState* S = (NestedState*)pc->nested;
  const int blocks = stream_blocks(pc->ctx, S->N, 8);
  nested_pre_kernel<<<blocks, kThreads, 0, st>>>(v, S->y, S->sinv, S->N, S->nu, S->ctl, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = op_apply(S->Bt, S->y, S->t, v, status, st)) != cudaSuccess) return e;     // t = v - B^T y
  SolveEnv env;
  env.ctx = pc->ctx;
  env.op = S->K;
  env.pc = S->jacobi;
  env.st = st;
  env.ctl = S->ctl;
  env.partials = S->partials;
  env.partials_cap = S->partials_cap;
  env.N = S->nu;
  env.pass_ev0 = env.pass_ev1 = nullptr;
  if ((e = S->M->fill(env, S->t, S->y)) != cudaSuccess) return e;                    // K y_u = t_u from 0
  for (int i = 0; i < S->maxit; ++i)
    if ((e = S->M->iteration(env, S->y)) != cudaSuccess) return e;
  nested_post_kernel<<<blocks, kThreads, 0, st>>>(S->y, add, out, S->N, status);
  return cudaGetLastError();
}

pfk_status create_nested_pc(pfk_context* ctx, const pfk_operator* K, const pfk_operator* Bt,
                            const double* schur_diag, const pfk_inner_solve* inner, pfk_pc* pc) {
  pc->ctx = ctx;
  pc->op = Bt;
  pc->kind = PFK_PC_BLOCK_UPPER;
  auto S = new (std::nothrow) NestedState();
  if (!S) return PFK_ERR_OOM;
  pc->nested = S;
  S->K = K;
  S->Bt = Bt;
  S->N = Bt->n;
  S->nu = K->n;
  S->maxit = inner->maxit;
  S->M.reset(make_inner_method(inner->method));
  if (!S->M) {
    set_error(ctx, "inner method must be one of the CG / CR types (FCG, PIPEFCG, PIPEFCG_THETA, GCR, PIPEGCR, "
                   "PIPEGCR_W)");
    return PFK_ERR_INVALID;
  }
  cudaStream_t st = ctx->stream;
  const int64_t N = S->N, nu = S->nu;
  PFK_CUDA(ctx, cudaMallocAsync((void**)&S->sinv, (size_t)(N - nu) * sizeof(double), st));
  std::vector<double> h(N - nu);
  for (int64_t i = 0; i < N - nu; ++i) {
    if (!(schur_diag[i] != 0.0) || !std::isfinite(schur_diag[i])) {
      set_error(ctx, "Schur diagonal entries must be finite and non-zero");
      return PFK_ERR_INVALID;
    }
    h[i] = 1.0 / schur_diag[i];
  }
  PFK_CUDA(ctx, cudaMemcpyAsync(S->sinv, h.data(), (size_t)(N - nu) * sizeof(double), cudaMemcpyHostToDevice, st));
  PFK_CUDA(ctx, cudaMallocAsync((void**)&S->y, (size_t)N * sizeof(double), st));
  PFK_CUDA(ctx, cudaMallocAsync((void**)&S->t, (size_t)N * sizeof(double), st));
  const int64_t wd = S->M->workspace_doubles(nu, inner->mmax);
  PFK_CUDA(ctx, cudaMallocAsync((void**)&S->ws, (size_t)wd * sizeof(double), st));
  S->M->bind(S->ws, nu, inner->mmax);
  S->partials_cap = ((int64_t)ctx->num_sms * kMaxBlocksPerSm + kMaxCombineGroups) * kPartialStride;
  PFK_CUDA(ctx, cudaMallocAsync((void**)&S->partials, (size_t)S->partials_cap * sizeof(double), st));
  PFK_CUDA(ctx, cudaMallocAsync((void**)&S->ctl, sizeof(SolveCtl), st));
  SolveCtl c;
  std::memset(&c, 0, sizeof(c));
  c.status = kRun;
  c.maxit = inner->maxit;
  c.mmax = inner->mmax;
  c.truncation = PFK_TRUNC_STANDARD;
  c.norm = PFK_NORM_NATURAL;
  c.rtol = inner->rtol;
  c.atol = 0.0;
  PFK_CUDA(ctx, cudaMemcpyAsync(S->ctl, &c, sizeof(SolveCtl), cudaMemcpyHostToDevice, st));
  S->jacobi = new (std::nothrow) pfk_pc();
  if (!S->jacobi) return PFK_ERR_OOM;
  S->jacobi->device = ctx->device;
  S->jacobi->stream = ctx->stream;
  pfk_pc_desc jd{};
  jd.kind = PFK_PC_JACOBI;
  pfk_status s = create_pc(ctx, K, &jd, S->jacobi);
  if (s != PFK_OK) return s;
  PFK_CUDA(ctx, cudaStreamSynchronize(st));
  return PFK_OK;
}

void destroy_nested(pfk_pc* pc) {
  NestedState* S = (NestedState*)pc->nested;
  if (!S) return;
  cudaStream_t st = pc->stream;
  for (void* p : {(void*)S->sinv, (void*)S->y, (void*)S->t, (void*)S->ws, (void*)S->ctl, (void*)S->partials})
    if (p) cudaFreeAsync(p, st);
  cudaStreamSynchronize(st);
  if (S->jacobi) pfk_destroy_preconditioner(S->jacobi);
  delete S;
  pc->nested = nullptr;
}

}  // namespace pfk
