// Solve driver: restarts, residual replacement and graph-replayed iterations.
//
// Host logic only (scalars and control); every vector operation is a kernel of
// the method object.  Per solve:
//   1. the pipeline fill and `graph_iters` iterations of the method are each
//      captured once into a CUDA graph (all scalars live in the device control
//      block, so the same graphs are valid for every restart and iteration);
//   2. fill graph, then iteration-graph launches, two in flight, with the
//      status words copied back asynchronously after each; iterations after
//      convergence are no-ops;
//   3. on convergence the true residual ||b - A x|| is checked (residual
//      replacement: restart from x with a tightened target when it fails); on a
//      norm breakdown the method restarts from x, flushing the pipeline
//      (Sec. 5: implementations detect norm breakdown and restart).
#include "pfk_internal.cuh"
#include "solver.cuh"

#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

namespace pfk {

cudaError_t SolveEnv::pc_apply(const double* v, double* out, const double* add, const int* status) const {
  if (pc) return pfk::pc_apply(pc, v, out, add, status, st);
  pfk_pc id;   // identity
  id.ctx = ctx;
  id.op = op;
  id.kind = PFK_PC_NONE;
  return pfk::pc_apply(&id, v, out, add, status, st);
}

cudaError_t SolveEnv::mark_pass(int which) const {
  cudaEvent_t e = which == 0 ? pass_ev0 : pass_ev1;
  if (!e) return cudaSuccess;
  return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
}

__global__ void ctl_restart_kernel(SolveCtl* ctl) {
  ctl->status = kRun;
  ctl->i = 0;
  ctl->nw = 0;
  ctl->counter = 0u;
}

static Method* make_method(int method, double sigma = NAN) {
  switch (method) {
    case PFK_PIPEFCG: return make_pipefcg(false);
    case PFK_PIPEFCG_NAIVE: return make_pipefcg(true);
    case PFK_PIPEGCR_W: return make_pipegcr_w();
    case PFK_PIPEFCG_THETA: return make_pipefcg_theta();
    case PFK_PIPEGCR: return make_pipegcr();
    case PFK_PIPEFGMRES: return make_pipefgmres(sigma);
    case PFK_FCG: return make_fcg();
    case PFK_GCR: return make_gcr();
    case PFK_FGMRES: return make_fgmres();
    default: return nullptr;
  }
}

// Methods usable as the inner solve of a nested preconditioner (device-only
// control: no restarts, no cycle ends).
Method* make_inner_method(int method) {
  switch (method) {
    case PFK_FCG:
    case PFK_PIPEFCG:
    case PFK_PIPEFCG_THETA:
    case PFK_GCR:
    case PFK_PIPEGCR:
    case PFK_PIPEGCR_W: return make_method(method);
    default: return nullptr;
  }
}

bool method_supported(int method) {
  std::unique_ptr<Method> m(make_method(method));
  return m != nullptr;
}

pfk_status solve_workspace_bytes(int method, int mmax, int64_t n, int64_t* bytes) {
  std::unique_ptr<Method> m(make_method(method));
  if (!m) return PFK_ERR_INVALID;
  *bytes = m->workspace_doubles(n, mmax) * (int64_t)sizeof(double);
  return PFK_OK;
}

namespace {

struct Graph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  int kernels = 0;
  ~Graph() {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
  }
};

template <typename F>
cudaError_t capture(cudaStream_t cs, Graph& out, F&& body) {
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t eb = body();
  e = cudaStreamEndCapture(cs, &out.g);
  if (eb != cudaSuccess) return eb;
  if (e != cudaSuccess) return e;
  size_t nn = 0;
  if ((e = cudaGraphGetNodes(out.g, nullptr, &nn)) != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn && (e = cudaGraphGetNodes(out.g, nodes.data(), &nn)) != cudaSuccess) return e;
  for (auto& n : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) out.kernels++;
  }
  return cudaGraphInstantiate(&out.x, out.g, 0);
}

struct Events {
  std::vector<cudaEvent_t> v;
  ~Events() {
    for (auto e : v)
      if (e) cudaEventDestroy(e);
  }
  cudaError_t make(int n, unsigned flags) {
    v.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
      cudaError_t e = cudaEventCreateWithFlags(&v[i], flags);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};

}  // namespace

pfk_status run_solve(pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, const pfk_solve_params* prm,
                     const double* b, double* x, pfk_solve_info* info) {
  cudaStream_t st = ctx->stream;
  const int64_t N = op->n;
  const int mmax = prm->mmax;
  std::unique_ptr<Method> M(make_method(prm->method, prm->sigma));
  if (!M) {
    set_error(ctx, "method not available");
    return PFK_ERR_INVALID;
  }
  if (prm->persistent < 0 || prm->persistent > 2) {
    set_error(ctx, "persistent must be 0 (auto), 1 (never) or 2 (required)");
    return PFK_ERR_INVALID;
  }
  if (!M->configure(ctx, op, pc, N, prm->persistent) && prm->persistent == 2) {
    set_error(ctx, "the persistent path needs PIPEFCG or FCG, an assembled CSR operator, Jacobi or no "
                   "preconditioner and n <= PFK_PERSISTENT_MAX_N");
    return PFK_ERR_INVALID;
  }
  // ---- workspace: control block | method vectors | partials | scalars | history ----
  // partials: room for any kernel of the solve (at most kMaxBlocksPerSm blocks
  // per SM, at most kPartialStride values per block); launches check it.
  const int64_t wd = M->workspace_doubles(N, mmax);
  // block rows of the largest reduction grid plus the two-level combine's group rows
  const int64_t pd = ((int64_t)ctx->num_sms * kMaxBlocksPerSm + kMaxCombineGroups) * kPartialStride;
  const int64_t sd = 64;
  const int hist_cap = prm->history ? prm->history_capacity : 0;
  const int64_t hd = (int64_t)hist_cap * PFK_HISTORY_FIELDS;
  const size_t ctl_bytes = (sizeof(SolveCtl) + 255) / 256 * 256;
  const size_t need = (size_t)(wd + pd + sd + hd) * sizeof(double) + ctl_bytes + 256;
  if (ctx->ws_bytes < need) {
    if (ctx->ws) cudaFreeAsync(ctx->ws, st);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    cudaError_t e = cudaMallocAsync(&ctx->ws, need, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(ctx, "out of device memory for the solve workspace");
      return PFK_ERR_OOM;
    }
    ctx->ws_bytes = need;
  }
  char* base = (char*)ctx->ws;
  SolveCtl* ctl = (SolveCtl*)base;
  double* ws = (double*)(base + ctl_bytes);
  double* partials = ws + wd;
  double* d_out = partials + pd;
  double* hist = hist_cap ? d_out + sd : nullptr;
  M->bind(ws, N, mmax);

  SolveCtl h;
  std::memset(&h, 0, sizeof(h));
  h.status = kRun;
  h.maxit = prm->maxit;
  h.mmax = mmax;
  h.truncation = prm->truncation;
  h.norm = prm->norm;
  h.rtol = prm->rtol;
  h.atol = prm->atol;
  h.history = hist;
  h.hist_cap = hist_cap;
  h.bar_timeout_ns = prm->barrier_timeout_us == 0 ? 2000000000ll
                     : prm->barrier_timeout_us < 0 ? 0ll : 1000ll * (long long)prm->barrier_timeout_us;
  PFK_CUDA(ctx, cudaMemcpyAsync(ctl, &h, sizeof(SolveCtl), cudaMemcpyHostToDevice, st));

  SolveEnv env;
  env.ctx = ctx;
  env.op = op;
  env.pc = pc;
  env.st = st;
  env.ctl = ctl;
  env.partials = partials;
  env.partials_cap = pd;
  env.N = N;
  env.pass_ev0 = env.pass_ev1 = nullptr;

  long long kernel_launches = 0;

  // ---- ||b|| ----
  double bnorm = 0.0;
  PFK_CUDA(ctx, dot_into(ctx, b, b, N, d_out, st));
  kernel_launches += 1;
  PFK_CUDA(ctx, cudaMemcpyAsync(&bnorm, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
  PFK_CUDA(ctx, cudaStreamSynchronize(st));
  bnorm = std::sqrt(bnorm);
  double sigma_used = NAN;
  PFK_CUDA(ctx, M->prepare(env, b, d_out, &sigma_used));
  const bool gmres = M->cycle_length() > 0;

  // ---- graphs: recorded on the library's own stream (the caller's may be the
  // legacy default stream, which cannot be captured), launched on the caller's ----
  const int K = prm->graph_iters > 0 ? prm->graph_iters : 8;
  const bool profile = prm->profile != 0;
  Events pev;
  if (profile) PFK_CUDA(ctx, pev.make(2 * K, cudaEventDefault));
  Graph gfill, giter;
  {
    SolveEnv cenv = env;
    cenv.st = ctx->cap_stream;
    cudaError_t e = capture(cenv.st, gfill, [&]() -> cudaError_t {
      ctl_restart_kernel<<<1, 1, 0, cenv.st>>>(ctl);
      cudaError_t e2 = cudaGetLastError();
      if (e2 != cudaSuccess) return e2;
      return M->fill(cenv, b, x);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "capture pipeline fill");
    e = capture(cenv.st, giter, [&]() -> cudaError_t {
      cudaError_t e2 = cudaSuccess;
      for (int g = 0; g < K && e2 == cudaSuccess; ++g) {
        SolveEnv ienv = cenv;
        if (profile) {
          ienv.pass_ev0 = pev.v[2 * g];
          ienv.pass_ev1 = pev.v[2 * g + 1];
        }
        e2 = M->iteration(ienv, x);
      }
      return e2;
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "capture iteration");
  }

  SolveCtl* hc = ctx->pinned;   // pinned status copies (owned by the context)
  Events ev, tev;
  PFK_CUDA(ctx, ev.make(2, cudaEventDisableTiming));
  PFK_CUDA(ctx, tev.make(2, cudaEventDefault));

  PFK_CUDA(ctx, cudaEventRecord(tev.v[0], st));

  const double goal = std::fmax(prm->rtol * bnorm, prm->atol);
  int restarts = 0, breakdowns = 0, replacements = 0;
  bool prev_breakdown = false;
  pfk_status result = PFK_OK;
  double rnorm_true = NAN;
  double target = NAN;
  double pass_ms = 0.0;
  double* scratch = M->scratch();

  auto true_residual = [&](double* out) -> cudaError_t {
    cudaError_t e = op_apply(op, x, scratch, b, nullptr, st);
    if (e != cudaSuccess) return e;
    e = dot_into(ctx, scratch, scratch, N, d_out, st);
    if (e != cudaSuccess) return e;
    kernel_launches += 2;
    e = cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    *out = std::sqrt(*out);
    return e;
  };
  // With profiling, one graph is in flight: after it completes, the event pairs
  // of the passes that did work (the first `done` of the K) are summed.
  auto collect = [&](int done) -> cudaError_t {
    for (int g = 0; g < done && g < K; ++g) {
      float ms = 0.f;
      cudaError_t e = cudaEventElapsedTime(&ms, pev.v[2 * g], pev.v[2 * g + 1]);
      if (e != cudaSuccess) return e;
      pass_ms += ms;
    }
    return cudaSuccess;
  };

  for (;;) {
    // ---- (re)start: pipeline fill ----
    PFK_CUDA(ctx, cudaGraphLaunch(gfill.x, st));
    kernel_launches += gfill.kernels;
    PFK_CUDA(ctx, cudaMemcpyAsync(&hc[0], ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st));
    PFK_CUDA(ctx, cudaStreamSynchronize(st));
    int status = hc[0].status;
    if (std::isnan(target)) target = hc[0].target;

    if (status == kRun) {
      if (hc[0].it >= prm->maxit) {
        status = kMaxit;
      } else if (!profile) {
        // ---- iterate: graph launches, two in flight ----
        int q = 0;
        PFK_CUDA(ctx, cudaGraphLaunch(giter.x, st));
        kernel_launches += giter.kernels;
        PFK_CUDA(ctx, cudaMemcpyAsync(&hc[q], ctl, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
        PFK_CUDA(ctx, cudaEventRecord(ev.v[q], st));
        for (;;) {
          PFK_CUDA(ctx, cudaGraphLaunch(giter.x, st));
          kernel_launches += giter.kernels;
          PFK_CUDA(ctx, cudaMemcpyAsync(&hc[q ^ 1], ctl, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
          PFK_CUDA(ctx, cudaEventRecord(ev.v[q ^ 1], st));
          PFK_CUDA(ctx, cudaEventSynchronize(ev.v[q]));
          if (hc[q].status != kRun) break;
          q ^= 1;
        }
      } else {
        int before = hc[0].passes;
        for (;;) {
          PFK_CUDA(ctx, cudaGraphLaunch(giter.x, st));
          kernel_launches += giter.kernels;
          PFK_CUDA(ctx, cudaMemcpyAsync(&hc[1], ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st));
          PFK_CUDA(ctx, cudaStreamSynchronize(st));
          PFK_CUDA(ctx, collect(hc[1].passes - before));
          before = hc[1].passes;
          if (hc[1].status != kRun) break;
        }
      }
      PFK_CUDA(ctx, cudaMemcpyAsync(&hc[0], ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st));
      PFK_CUDA(ctx, cudaStreamSynchronize(st));
      if (status == kRun) status = hc[0].status;
    }
    // GMRES types: least-squares solve over the cycle's valid columns and
    // x = x_0 + U y, whatever ended the cycle
    if (gmres && status != kNonFinite) {
      PFK_CUDA(ctx, M->end_cycle(env, x));
      kernel_launches += 2;
    }
    if (status == kCycleEnd) {
      prev_breakdown = false;
      continue;
    }

    if (status == kConverged) {
      double rt = 0.0;
      PFK_CUDA(ctx, true_residual(&rt));
      rnorm_true = rt;
      if (!prm->true_residual_check || rt <= goal) {
        result = PFK_OK;
        break;
      }
      if (restarts >= prm->max_restarts) {
        set_error(ctx, "true residual above the goal after max_restarts residual replacements");
        result = PFK_ERR_NOT_CONVERGED;
        break;
      }
      replacements += 1;
      restarts += 1;
      target *= 0.5 * goal / rt;
      PFK_CUDA(ctx, cudaMemcpyAsync(&ctl->target, &target, sizeof(double), cudaMemcpyHostToDevice, st));
      prev_breakdown = false;
      continue;
    }
    if (status == kBreakdown) {
      breakdowns += 1;
      const int i_since = hc[0].i;
      if ((i_since <= 1 && prev_breakdown) || restarts >= prm->max_restarts) {
        set_error(ctx, "norm breakdown persisted after restarting");
        result = PFK_ERR_BREAKDOWN;
        break;
      }
      restarts += 1;
      prev_breakdown = true;
      continue;
    }
    if (status == kFillBreakdown) {
      set_error(ctx, "norm breakdown in the pipeline fill (eta_0 <= 0)");
      result = PFK_ERR_BREAKDOWN;
      break;
    }
    if (status == kNonFinite) {
      set_error(ctx, "non-finite residual norm");
      result = PFK_ERR_BREAKDOWN;
      break;
    }
    if (status == kTimeout) {
      set_error(ctx, "a grid-barrier wait of the persistent kernel timed out");
      result = PFK_ERR_TIMEOUT;
      break;
    }
    if (status == kMaxit) {
      set_error(ctx, "maximum number of iterations reached");
      result = PFK_ERR_NOT_CONVERGED;
      break;
    }
    set_error(ctx, "unexpected device status");
    result = PFK_ERR_CUDA;
    break;
  }
  PFK_CUDA(ctx, cudaEventRecord(tev.v[1], st));
  if (result != PFK_OK || std::isnan(rnorm_true)) {
    double rt = 0.0;
    PFK_CUDA(ctx, true_residual(&rt));
    rnorm_true = rt;
  }
  PFK_CUDA(ctx, cudaMemcpyAsync(&hc[0], ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st));
  PFK_CUDA(ctx, cudaStreamSynchronize(st));
  float ms = 0.f;
  PFK_CUDA(ctx, cudaEventElapsedTime(&ms, tev.v[0], tev.v[1]));
  const int hl = hc[0].hist_len;
  if (prm->history && hist_cap > 0) {
    const int ncopy = hl < hist_cap ? hl : hist_cap;
    if (ncopy > 0)
      PFK_CUDA(ctx, cudaMemcpy(prm->history, hist, (size_t)ncopy * PFK_HISTORY_FIELDS * sizeof(double),
                               cudaMemcpyDeviceToHost));
  }
  if (info) {
    info->status = result;
    info->iterations = hc[0].it;
    info->restarts = restarts;
    info->breakdowns = breakdowns;
    info->replacements = replacements;
    info->history_len = hl;
    info->rho0 = hc[0].rho0;
    info->rho_final = hc[0].rho;
    info->rnorm_true = rnorm_true;
    info->bnorm = bnorm;
    info->time_ms = ms;
    info->pass_launches = hc[0].passes;
    info->kernel_launches = (int32_t)(kernel_launches > INT32_MAX ? INT32_MAX : kernel_launches);
    info->pass_bytes = hc[0].alg_bytes;
    info->pass_flops = hc[0].alg_flops;
    info->pass_ms = profile ? pass_ms : 0.0;
  }
  return result;
}

}  // namespace pfk
