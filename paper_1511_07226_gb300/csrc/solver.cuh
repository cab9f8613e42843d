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
};

Method* make_pipefcg(bool naive);

}  // namespace pfk
