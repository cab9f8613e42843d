// PIPEFGMRES (Alg. 15, constant shift sigma, eq. pipefgmresz) on one GPU.
//
// A restart cycle is a pipeline fill followed by passes k = 1 .. m-1:
//
//  fill   r_0 = b - A x_0, beta = ||r_0|| (its reduction also checks convergence),
//         p_0 = r_0 / beta, u_0 = B(p_0), zbar_0 = A u_0 - sigma p_0 fused with
//         the dots of Hessenberg column 0 (<p_0, zbar_0>, ||zbar_0||^2), then
//         qbar_0 = B(zbar_0), wbar_0 = A qbar_0;
//  pass k (fgmres_pass<NW>) one HBM pass that forms
//           p_k = (zbar_{k-1} - sum_j hbar_{j,k-1} p_j) / hbar_{k,k-1},
//           u_k = (qbar_{k-1} - sum_j u_j hbar_{j,k-1}) / hbar_{k,k-1},
//           zbar_k = (wbar_{k-1} - sum_j h_{j,k-1} zbar_j) / h_{k,k-1},
//         accumulates the dots of column k (<p_j, zbar_k>, j <= k, and
//         ||zbar_k||^2; the p_j read by the MAXPY are kept on chip), and in the
//         last block computes column k of H, t = ||zbar_k||^2 - sum hbar^2
//         (breakdown if t < 0), hbar_{k+1,k} = sqrt(t), one Givens rotation and
//         the least-squares residual estimate |g_{k+1}| (convergence test);
//         then qbar_k = B(zbar_k) and wbar_k = A qbar_k.
//  end    y from the rotated triangular system, x = x_0 + sum_j y_j u_j.
//
// The reduction of pass k is in flight while B and A run (Sec. 5.3).
// Division by hbar_{k,k-1} is done as a multiplication by its reciprocal,
// computed once per column.
#include "pfk_internal.cuh"
#include "solver.cuh"

#include <cmath>

namespace pfk {

constexpr int kGm = PFK_MAX_MMAX;   // largest restart length

// Device state of the current restart cycle.
struct GmresState {
  double H[(kGm + 1) * kGm];    // H[j * kGm + k]: shifted Hessenberg (h)
  double Hb[(kGm + 1) * kGm];   // unshifted (hbar)
  double R[(kGm + 1) * kGm];    // H with the Givens rotations applied
  double cs[kGm], sn[kGm];
  double g[kGm + 1];
  double y[kGm];
  double sigma;
  double beta0;
  double inv;                   // 1 / hbar_{k,k-1} for the next pass
  int k;                        // column formed by the next pass
  int ncols;                    // valid columns of the cycle
};

struct FgArgs {
  double* P;     // m vectors p_0 .. p_{m-1}
  double* U;     // m vectors u_0, tilde-u_1 .. tilde-u_{m-1}
  double* Zb;    // m vectors zbar_0 ..
  const double* qb;
  const double* wb;
  double* zc;    // copy of zbar_k for the preconditioner
  int64_t N;
  int m;
  SolveCtl* ctl;
  GmresState* gs;
  double* partials;
};

// Column k of H from its dots (hb[j] = <p_j, zbar_k>, j <= k; zz = ||zbar_k||^2),
// Givens update and status.  One thread.
__device__ void fgmres_column(SolveCtl* ctl, GmresState* gs, int k, int m, const double* hb, double zz) {
  const double sigma = gs->sigma;
  double tsum = 0.0;
  for (int j = 0; j <= k; ++j) {
    gs->Hb[j * kGm + k] = hb[j];
    gs->H[j * kGm + k] = hb[j];
    tsum += hb[j] * hb[j];
  }
  gs->H[k * kGm + k] = hb[k] + sigma;
  const double t = zz - tsum;
  if (!(t >= 0.0)) {
    ctl->i = k + 1;     // breakdown while forming column k: columns 0 .. k-1 valid
    gs->ncols = k;
    ctl->status = isfinite(t) ? kBreakdown : kNonFinite;
    return;
  }
  const double hsub = sqrt(t);
  gs->Hb[(k + 1) * kGm + k] = hsub;
  gs->H[(k + 1) * kGm + k] = hsub;
  ctl->it += 1;
  gs->ncols = k + 1;
  ctl->i = k + 1;
  // Givens: apply the previous rotations to column k, then zero its subdiagonal
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
  push_history(ctl, est, nan(""), t, hsub);
  gs->inv = hsub != 0.0 ? 1.0 / hsub : 0.0;
  gs->k = k + 1;
  if (!isfinite(est)) { ctl->status = kNonFinite; return; }
  if (est <= ctl->target || t == 0.0) { ctl->status = kConverged; return; }
  if (k + 1 == m) { ctl->status = kCycleEnd; return; }
  if (ctl->it >= ctl->maxit) { ctl->status = kMaxit; return; }
}

constexpr int kFgThreads = 128;
constexpr int kFgBlocksPerSm = 6;
constexpr int kFgStride = kFgThreads + 1;
static_assert(kFgBlocksPerSm <= kMaxBlocksPerSm, "partials are sized for kMaxBlocksPerSm blocks per SM");

template <int NW>
__global__ void __launch_bounds__(kFgThreads, kFgBlocksPerSm) fgmres_pass(FgArgs a) {
  SolveCtl* ctl = a.ctl;
  if (ctl->status != kRun) return;
  GmresState* gs = a.gs;
  constexpr int ND = NW + 2;
  constexpr int NWARPS = kFgThreads / 32;
  __shared__ double s_hb[NW], s_h[NW];
  __shared__ double s_pk[NW * kFgStride];
  __shared__ double s_z[kFgThreads];
  __shared__ double s_red[NWARPS * ND];
  __shared__ double s_sum[ND];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = gs->k;                 // column formed here; window j < k
  const double inv = gs->inv;
  const int64_t N = a.N;
  if (threadIdx.x < k) {
    s_hb[threadIdx.x] = gs->Hb[threadIdx.x * kGm + (k - 1)];
    s_h[threadIdx.x] = gs->H[threadIdx.x * kGm + (k - 1)];
  }
  __syncthreads();
  const size_t koff = (size_t)k * (size_t)N;
  const size_t km1 = (size_t)(k - 1) * (size_t)N;
  double* my_pk = s_pk + threadIdx.x;
  const double* warp_z = s_z + warp * 32;
  const double* lane_row = s_pk + lane * kFgStride + warp * 32;
  double gz = 0.0, gp = 0.0, gw = 0.0;   // ||zbar_k||^2, <p_k, zbar_k>, lane-owned <p_lane, zbar_k>

  for (int64_t base = (int64_t)blockIdx.x * kFgThreads; base < N; base += (int64_t)gridDim.x * kFgThreads) {
    const int64_t e = base + threadIdx.x;
    double zk = 0.0;
    if (e < N) {
      double p = a.Zb[km1 + e], u = a.qb[e], z = a.wb[e];
#pragma unroll
      for (int j = 0; j < NW; ++j) {
        if (j < k) {
          const size_t o = (size_t)j * (size_t)N + e;
          const double pj = a.P[o];
          p = fma(-s_hb[j], pj, p);
          u = fma(-s_hb[j], a.U[o], u);
          z = fma(-s_h[j], a.Zb[o], z);
          my_pk[j * kFgStride] = pj;
        }
      }
      p *= inv;
      u *= inv;
      zk = z * inv;
      a.P[koff + e] = p;
      a.U[koff + e] = u;
      a.Zb[koff + e] = zk;
      a.zc[e] = zk;
      gz = fma(zk, zk, gz);
      gp = fma(p, zk, gp);
    } else {
#pragma unroll
      for (int j = 0; j < NW; ++j)
        if (j < k) my_pk[j * kFgStride] = 0.0;
    }
    s_z[threadIdx.x] = zk;
    __syncwarp();
    if (lane < k) {
      double c = gw;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) c = fma(warp_z[t], lane_row[t], c);
      gw = c;
    }
    __syncwarp();
  }
  {
    const double wz = warp_sum(gz), wp = warp_sum(gp);
    const int nd = k + 2;
    if (lane == 0) {
      s_red[warp * nd + 0] = wz;
      s_red[warp * nd + 1 + k] = wp;    // hb[k] = <p_k, zbar_k>
    }
    if (lane < k) s_red[warp * nd + 1 + lane] = gw;
    __syncthreads();
  }
  if (!combine_block_partials_2l(s_red, k + 2, a.partials, ND, &ctl->counter, ctl->gcounter, s_sum)) return;
  if (threadIdx.x != 0) return;
  // traffic: zbar_{k-1}, qbar, wbar and 3k window vectors read, p_k, u_k,
  // zbar_k written; FP64: 3k MAXPY FMAs, 3 scalings, k + 2 dot FMAs
  ctl->passes += 1;
  ctl->alg_bytes += 8.0 * (double)N * (double)(3 + 3 * k + 4);
  ctl->alg_flops += (double)N * (2.0 * (3 * k + k + 2) + 3.0);
  fgmres_column(ctl, gs, k, a.m, s_sum + 1, s_sum[0]);
}

// beta = ||r_0||: history, target, convergence; g = beta e_0.
__global__ void __launch_bounds__(kThreads) fgmres_fill_norm(const double* __restrict__ r, int64_t N, SolveCtl* ctl,
                                                             GmresState* gs, double* partials) {
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
  gs->beta0 = beta;
  gs->g[0] = beta;
  gs->k = 0;
  gs->ncols = 0;
  gs->inv = beta != 0.0 ? 1.0 / beta : 0.0;
  if (!isfinite(beta)) ctl->status = kNonFinite;
  else if (beta <= ctl->target) ctl->status = kConverged;
  else if (ctl->it >= ctl->maxit) ctl->status = kMaxit;    // no column of this cycle may start
  else ctl->status = kRun;
}

// p_0 = r_0 / beta (reciprocal multiply).
__global__ void __launch_bounds__(kThreads) fgmres_scale(const double* __restrict__ r, double* __restrict__ p0,
                                                         int64_t N, const GmresState* gs, const int* status) {
  if (*status != kRun) return;
  const double inv = gs->inv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    p0[e] = r[e] * inv;
}

// zbar_0 = (A u_0) - sigma p_0 in place, with the dots of column 0.
__global__ void __launch_bounds__(kThreads) fgmres_fill_col0(const double* __restrict__ p0, double* __restrict__ z0,
                                                             int64_t N, SolveCtl* ctl, GmresState* gs, int m,
                                                             double* partials) {
  if (ctl->status != kRun) return;
  const double sigma = gs->sigma;
  double acc[2] = {0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const double pv = p0[e];
    const double zv = fma(-sigma, pv, z0[e]);
    z0[e] = zv;
    acc[0] = fma(zv, zv, acc[0]);
    acc[1] = fma(pv, zv, acc[1]);
  }
  __shared__ double s_red[(kThreads / 32) * 2];
  __shared__ double s_sum[2];
  if (!reduce_last_block<2>(acc, 2, partials, 2, &ctl->counter, s_red, s_sum)) return;
  if (threadIdx.x != 0) return;
  fgmres_column(ctl, gs, 0, m, s_sum + 1, s_sum[0]);
}

// End of a cycle: back substitution R y = g on the ncols valid columns.
__global__ void fgmres_lsq(GmresState* gs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n = gs->ncols;
  for (int j = n - 1; j >= 0; --j) {
    double s = gs->g[j];
    for (int l = j + 1; l < n; ++l) s -= gs->R[j * kGm + l] * gs->y[l];
    gs->y[j] = s / gs->R[j * kGm + j];
  }
}

// x = x_0 + sum_j y_j u_j over the valid columns.
__global__ void __launch_bounds__(kThreads) fgmres_update_x(double* __restrict__ x, const double* __restrict__ U,
                                                            int64_t N, const GmresState* gs) {
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

__global__ void fgmres_set_sigma(GmresState* gs, double sigma) { gs->sigma = sigma; }

static int fg_template(int m) { return m <= 8 ? 8 : m <= 16 ? 16 : 32; }

class PipeFgmres : public Method {
 public:
  explicit PipeFgmres(double sigma) : sigma_(sigma) {}

  int64_t workspace_doubles(int64_t N, int m) const override {
    return state_doubles() + 5 * N + 3 * (int64_t)m * N;
  }

  void bind(double* ws, int64_t N, int m) override {
    N_ = N;
    m_ = m;
    gs_ = (GmresState*)ws;
    double* v = ws + state_doubles();
    r_ = v; qb_ = r_ + N; wb_ = qb_ + N; tmp_ = wb_ + N; zc_ = tmp_ + N;
    P_ = zc_ + N;
    U_ = P_ + (int64_t)m * N;
    Zb_ = U_ + (int64_t)m * N;
  }

  double* scratch() override { return tmp_; }
  int cycle_length() const override { return m_; }

  // sigma: given, or estimated by 10 power iterations on v -> A B(v) from
  // v = b / ||b|| (sigma = ||A B(v)|| at the last step, ||v|| = 1).
  cudaError_t prepare(const SolveEnv& env, const double* b, double* dscalar, double* host_sigma) override {
    double sigma = sigma_;
    if (std::isnan(sigma)) {
      cudaError_t e;
      double nrm = 0.0;
      if ((e = dot_into(env.ctx, b, b, N_, dscalar, env.st)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(&nrm, dscalar, sizeof(double), cudaMemcpyDeviceToHost, env.st)) != cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(env.st)) != cudaSuccess) return e;
      nrm = std::sqrt(nrm);
      if ((e = scale_into(env, b, r_, nrm > 0.0 ? 1.0 / nrm : 0.0)) != cudaSuccess) return e;
      for (int it = 0; it < 10; ++it) {
        if ((e = env.pc_apply(r_, tmp_, nullptr, nullptr)) != cudaSuccess) return e;
        if ((e = op_apply(env.op, tmp_, qb_, nullptr, nullptr, env.st)) != cudaSuccess) return e;
        if ((e = dot_into(env.ctx, qb_, qb_, N_, dscalar, env.st)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&nrm, dscalar, sizeof(double), cudaMemcpyDeviceToHost, env.st)) != cudaSuccess)
          return e;
        if ((e = cudaStreamSynchronize(env.st)) != cudaSuccess) return e;
        nrm = std::sqrt(nrm);
        if ((e = scale_into(env, qb_, r_, nrm > 0.0 ? 1.0 / nrm : 0.0)) != cudaSuccess) return e;
      }
      sigma = nrm;
    }
    *host_sigma = sigma;
    fgmres_set_sigma<<<1, 1, 0, env.st>>>(gs_, sigma);
    return cudaGetLastError();
  }

  cudaError_t fill(const SolveEnv& env, const double* b, double* x) override {
    cudaStream_t st = env.st;
    const int* status = &env.ctl->status;
    cudaError_t e;
    const int blocks = stream_blocks(env.ctx, N_, 2);
    if (!env.partials_fit(blocks, 2)) return cudaErrorInvalidValue;
    if ((e = op_apply(env.op, x, r_, b, nullptr, st)) != cudaSuccess) return e;   // r_0 = b - A x_0
    fgmres_fill_norm<<<blocks, kThreads, 0, st>>>(r_, N_, env.ctl, gs_, env.partials);
    fgmres_scale<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, st>>>(r_, P_, N_, gs_, status);   // p_0
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = env.pc_apply(P_, U_, nullptr, status)) != cudaSuccess) return e;               // u_0 = B(p_0)
    if ((e = op_apply(env.op, U_, Zb_, nullptr, status, st)) != cudaSuccess) return e;      // A u_0
    fgmres_fill_col0<<<blocks, kThreads, 0, st>>>(P_, Zb_, N_, env.ctl, gs_, m_, env.partials);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = env.pc_apply(Zb_, qb_, nullptr, status)) != cudaSuccess) return e;            // qbar_0
    return op_apply(env.op, qb_, wb_, nullptr, status, st);                                 // wbar_0
  }

  cudaError_t iteration(const SolveEnv& env, double* x) override {
    (void)x;
    FgArgs a;
    a.P = P_; a.U = U_; a.Zb = Zb_; a.qb = qb_; a.wb = wb_; a.zc = zc_;
    a.N = N_; a.m = m_; a.ctl = env.ctl; a.gs = gs_; a.partials = env.partials;
    const int tmpl = fg_template(m_);
    const int64_t need = (N_ + kFgThreads - 1) / kFgThreads;
    const int64_t cap = (int64_t)env.ctx->num_sms * kFgBlocksPerSm;
    const int blocks = (int)(need < cap ? need : cap);
    if (!env.partials_fit_2l(blocks, tmpl + 2)) return cudaErrorInvalidValue;
    cudaError_t e = env.mark_pass(0);
    if (e != cudaSuccess) return e;
    switch (tmpl) {
      case 8: fgmres_pass<8><<<blocks, kFgThreads, 0, env.st>>>(a); break;
      case 16: fgmres_pass<16><<<blocks, kFgThreads, 0, env.st>>>(a); break;
      default: fgmres_pass<32><<<blocks, kFgThreads, 0, env.st>>>(a); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = env.mark_pass(1)) != cudaSuccess) return e;
    const int* status = &env.ctl->status;
    // qbar_k = B(zbar_k), wbar_k = A qbar_k (zbar_k also written to zc by the pass,
    // so the graph's pointers are the same for every k)
    if ((e = env.pc_apply(zc_, qb_, nullptr, status)) != cudaSuccess) return e;
    return op_apply(env.op, qb_, wb_, nullptr, status, env.st);
  }

  cudaError_t end_cycle(const SolveEnv& env, double* x) override {
    fgmres_lsq<<<1, 32, 0, env.st>>>(gs_);
    fgmres_update_x<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, env.st>>>(x, U_, N_, gs_);
    return cudaGetLastError();
  }

 private:
  static int64_t state_doubles() { return (int64_t)((sizeof(GmresState) + 255) / 256 * 256 / sizeof(double)); }
  cudaError_t scale_into(const SolveEnv& env, const double* src, double* dst, double s);

  double sigma_;
  int64_t N_ = 0;
  int m_ = 0;
  GmresState* gs_ = nullptr;
  double *r_ = nullptr, *qb_ = nullptr, *wb_ = nullptr, *tmp_ = nullptr, *zc_ = nullptr;
  double *P_ = nullptr, *U_ = nullptr, *Zb_ = nullptr;
};

__global__ void scale_kernel(const double* __restrict__ src, double* __restrict__ dst, int64_t N, double s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e] * s;
}

cudaError_t PipeFgmres::scale_into(const SolveEnv& env, const double* src, double* dst, double s) {
  scale_kernel<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, env.st>>>(src, dst, N_, s);
  return cudaGetLastError();
}

Method* make_pipefgmres(double sigma) { return new PipeFgmres(sigma); }

}  // namespace pfk
