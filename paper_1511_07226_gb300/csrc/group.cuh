// Grouped persistent PIPEFCG / PIPEGCR / PIPEFGMRES (group.cu): host interface used by the grouped
// batch entry point and by the serving loop.
#pragma once

#include "pfk_internal.cuh"

namespace pfk {

// Whether a system can run on the grouped kernel (stencil operator, PIPEFCG,
// PIPEGCR or PIPEFGMRES, NONE / JACOBI / FP64 or FP32 INNER_PCG
// preconditioner); *why says why not.
bool group_eligible(const pfk_operator* op, const pfk_pc_desc* pc, const pfk_solve_params* prm, const char** why);
// The method and preconditioner part of that test alone.
bool group_method_eligible(const pfk_pc_desc* pc, const pfk_solve_params* prm, const char** why);

// CTAs of a system with n cells and `rows` x-rows: `requested` if > 0, else
// about 4,096 cells per CTA; at most 64 and at most one per x-row.
int group_ctas(int64_t n, int64_t rows, int requested);

// Active systems of the grouped kernel and their launches, on one context's
// stream.  Not thread-safe: one host thread drives a runner.
class GroupRunner {
 public:
  GroupRunner();
  ~GroupRunner();
  GroupRunner(const GroupRunner&) = delete;
  GroupRunner& operator=(const GroupRunner&) = delete;

  // Device tables for up to max_slots systems (0: as many as CTAs fit).
  pfk_status init(pfk_context* ctx, int max_slots);
  // CTAs one cooperative launch can hold, and those not taken by active systems.
  int capacity_ctas() const;
  int free_ctas() const;
  bool any_active() const;
  // Device bytes admit() allocates for a system.
  static int64_t workspace_bytes(int64_t n, int mmax, int nblk);
  // Makes a system active with nblk CTAs: b_dev / x_dev are device vectors the
  // caller keeps alive until release (x holds x0 and receives the solution);
  // hist_dev (or null) a device history of hist_cap entries.  PFK_ERR_BUSY if
  // its CTAs do not fit now.
  pfk_status admit(const pfk_operator* op, const pfk_pc_desc* pc, const pfk_solve_params* prm, const double* b_dev,
                   double* x_dev, int nblk, double* hist_dev, int hist_cap, int* slot);
  // One cooperative launch advancing every active system by at most `iters`
  // steps, then the systems' states read back (synchronises the stream).
  pfk_status step(int iters);
  bool done(int slot) const;
  // The solve summary of a finished system (time_ms and kernel_launches are
  // left to the caller).
  void info(int slot, pfk_solve_info* out) const;
  // Frees the system's workspace (stream-ordered) and its CTAs.
  void release(int slot);
  int launches() const;
  double kernel_ms() const;

 private:
  struct Impl;
  Impl* m_;
};

}  // namespace pfk
