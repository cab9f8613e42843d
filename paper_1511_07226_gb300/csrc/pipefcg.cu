// PIPEFCG (Alg. 8), naive PIPEFCG (Alg. 7) and PIPEGCR_w (Alg. 12) on one GPU.
//
// Alg. 12 keeps exactly the vectors of Alg. 8 (x, r, tilde-u, w recurred with
// z, m = tilde-u + B(w - r), n = A m, and the p, s, q, z histories); what
// changes is the left operand of every inner product -- w_i instead of
// tilde-u_i: gamma_i = <r_i, w_i>, delta_i = <w_i, w_i>, beta_{i,k} =
// -<w_i, s_k>/eta_k -- and the fill's gamma_0 = <r_0, s_0>, eta_0 = <s_0, s_0>
// (s_0 = A p_0 = w_0, q_0 = B(s_0) = m_0, z_0 = A q_0 = n_0).  The same pass
// serves both, selecting the left operand per element.
//
// The projection repair of eq. (proj) (theta variant) adds <r_i, w_i> to the
// pass's reduction; the scalar phase forms theta_i = <r_i, w_i>/<r_i, r_i> and a
// small kernel writes the preconditioner input t = w_i - theta_i r_i and
// theta_i u_i (added back by the preconditioner's epilogue).  On one GPU the
// extra inner product rides on the pass's reduction; nothing blocks.
//
// One iteration i is three kernel groups, all reading their scalars from the
// device control block (no host synchronisation, capturable in a CUDA graph):
//
//  1. pipefcg_pass<NW>  one HBM pass that
//       - finishes iteration i-1's four MAXPYs
//           p_{i-1} = u_{i-1} + sum beta_{i-1,k} p_k,  s, q, z likewise,
//         over the window W_{i-1} and writes them into ring slot (i-1) mod (mmax+1),
//       - advances x_i, r_i, u_i (= tilde-u_i), w_i with alpha_{i-1},
//       - accumulates the partial sums of gamma_i = <u_i, r_i>,
//         delta_i = <u_i, w_i>, ||r_i||^2 and <u_i, s_k> for every s_k of
//         W_{i-1} and s_{i-1} (the s_k read by the MAXPY are kept on chip, so
//         the window is read from HBM once),
//       - writes the preconditioner input t = w_i - r_i (eq. BwMinusR),
//       - and, in the last block to finish, combines the partial sums in a fixed
//         order and computes beta_{i,k} = -<u_i, s_k>/eta_k,
//         eta_i = delta_i - sum beta_{i,k}^2 eta_k, alpha_i = gamma_i/eta_i and the
//         convergence / breakdown status (the single reduction phase of Alg. 8);
//  2. the preconditioner, m_i = u_i + B(w_i - r_i) (Alg. 7: m_i = B(w_i));
//  3. the operator, n_i = A m_i.
//
// The reduction of step 1 is "in flight" (its scalars are not needed) while
// steps 2 and 3 run: the overlap the paper obtains with MPI_Iallreduce becomes
// the absence of any host round trip between the passes.  The statement-level
// arithmetic is the listing's; only kernel boundaries are moved: the MAXPYs of
// iteration i-1 are deferred into the pass that starts iteration i.
#include "pfk_internal.cuh"
#include "solver.cuh"

#include <cmath>

namespace pfk {

struct FcgArgs {
  double* x;
  double* r;
  double* u;
  double* w;
  const double* m;
  const double* n;
  double* t;
  double* P;
  double* S;
  double* Q;
  double* Z;
  int64_t N;
  int mmax;
  int naive;
  int gcrw;          // Alg. 12: inner products against w_i instead of tilde-u_i
  int theta;         // eq. (proj): also <r_i, w_i>; t is written by theta_prep_kernel
  SolveCtl* ctl;
  double* partials;
};

// Threads per block of the fused pass and resident blocks per SM (24 warps per
// SM).  Each thread handles one element per tile.  The history values s_k
// read by the MAXPYs are parked in shared memory, one row per window slot and
// one column per thread, and after the advance each warp computes the window
// dot products transposed: lane j sums u_e s_{k_j,e} over the warp's 32
// elements e.  So every thread holds one window accumulator instead of nu, the
// FP64 instruction count is unchanged, and register use stays low.
constexpr int kPassThreads = 128;
constexpr int kPassBlocksPerSm = 6;
constexpr int kSkStride = kPassThreads + 1;   // padding: conflict-free row reads
static_assert(kPassBlocksPerSm <= kMaxBlocksPerSm, "partials are sized for kMaxBlocksPerSm blocks per SM");
static_assert(PFK_MAX_MMAX + 5 <= kPartialStride, "partials are sized for kPartialStride values per block");

template <int NW>
__global__ void __launch_bounds__(kPassThreads, kPassBlocksPerSm) pipefcg_pass(FcgArgs a) {
  SolveCtl* ctl = a.ctl;
  if (ctl->status != kRun) return;
  constexpr int ND = NW + 5;
  constexpr int NWARPS = kPassThreads / 32;
  __shared__ double s_beta[NW];
  __shared__ size_t s_off[NW];
  __shared__ double s_red[NWARPS * ND];
  __shared__ double s_sum[ND];
  __shared__ double s_sk[NW * kSkStride];
  __shared__ double s_u[kPassThreads];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int iprev = ctl->i;      // i - 1
  const int nwp = ctl->nw;       // |W_{i-1}|
  const double alpha = ctl->alpha;
  const int slots = a.mmax + 1;
  const int64_t N = a.N;
  if (threadIdx.x < nwp) {
    const int k = iprev - nwp + (int)threadIdx.x;
    s_beta[threadIdx.x] = ctl->beta[threadIdx.x];
    s_off[threadIdx.x] = (size_t)(k % slots) * (size_t)N;
  }
  __syncthreads();
  const size_t coff = (size_t)(iprev % slots) * (size_t)N;
  double* my_sk = s_sk + threadIdx.x;
  const double* warp_u = s_u + warp * 32;
  const double* lane_row = s_sk + lane * kSkStride + warp * 32;

  // per-thread sums of gamma, delta, ||r||^2, <u, s_{i-1}>, <r, w> (theta
  // variant); lane-owned window sum
  double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0, g4 = 0.0, gw = 0.0;

  for (int64_t base = (int64_t)blockIdx.x * kPassThreads; base < N; base += (int64_t)gridDim.x * kPassThreads) {
    const int64_t e = base + threadIdx.x;
    double un = 0.0;
    if (e < N) {
      const double u0 = a.u[e], w0 = a.w[e];
      double p = u0, s = w0, q = a.m[e], z = a.n[e];
#pragma unroll
      for (int j = 0; j < NW; ++j) {
        if (j < nwp) {
          const size_t o = s_off[j] + e;
          const double b = s_beta[j];
          const double sv = a.S[o];
          p = fma(b, a.P[o], p);
          s = fma(b, sv, s);
          q = fma(b, a.Q[o], q);
          z = fma(b, a.Z[o], z);
          my_sk[j * kSkStride] = sv;
        }
      }
      a.P[coff + e] = p;
      a.S[coff + e] = s;
      a.Q[coff + e] = q;
      a.Z[coff + e] = z;
      const double xn = fma(alpha, p, a.x[e]);
      const double rn = fma(-alpha, s, a.r[e]);
      un = fma(-alpha, q, u0);
      const double wn = fma(-alpha, z, w0);
      a.x[e] = xn;
      a.r[e] = rn;
      a.u[e] = un;
      a.w[e] = wn;
      if (!a.naive && !a.theta) a.t[e] = wn - rn;
      if (a.theta) g4 = fma(rn, wn, g4);
      const double lv = a.gcrw ? wn : un;   // left operand of the inner products
      g0 = fma(lv, rn, g0);
      g1 = fma(lv, wn, g1);
      g2 = fma(rn, rn, g2);
      g3 = fma(lv, s, g3);
      un = lv;
    } else {
#pragma unroll
      for (int j = 0; j < NW; ++j)
        if (j < nwp) my_sk[j * kSkStride] = 0.0;
    }
    s_u[threadIdx.x] = un;
    __syncwarp();
    if (lane < nwp) {
      double c = gw;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) c = fma(warp_u[t], lane_row[t], c);
      gw = c;
    }
    __syncwarp();
  }

  // block partials: scalars by warp reduction, window sums straight from their lanes
  {
    const double w0 = warp_sum(g0), w1 = warp_sum(g1), w2 = warp_sum(g2), w3 = warp_sum(g3);
    const int nd = nwp + 4 + (a.theta ? 1 : 0);
    if (lane == 0) {
      s_red[warp * nd + 0] = w0;
      s_red[warp * nd + 1] = w1;
      s_red[warp * nd + 2] = w2;
      s_red[warp * nd + 3] = w3;
    }
    if (a.theta) {
      const double w4 = warp_sum(g4);
      if (lane == 0) s_red[warp * nd + 4 + nwp] = w4;
    }
    if (lane < nwp) s_red[warp * nd + 4 + lane] = gw;
    __syncthreads();
  }
  if (!combine_block_partials_2l(s_red, nwp + 4 + (a.theta ? 1 : 0), a.partials, ND, &ctl->counter, ctl->gcounter,
                                 s_sum))
    return;

  // ---- scalar phase of iteration i (the last block; s_red is free again) ----
  const int i = iprev + 1;
  const double gamma = s_sum[0], delta = s_sum[1], rr = s_sum[2];
  if (threadIdx.x == 0) {
    // algorithmic traffic of this pass: u, w, m, n, x, r and 4 nu_{i-1} history
    // vectors read; p, s, q, z, x, r, u, w (and t) written.  FP64 flops: 4 nu
    // MAXPY FMAs, 4 advance FMAs, nu + 4 dot FMAs, and the subtraction for t.
    ctl->passes += 1;
    ctl->alg_bytes += 8.0 * (double)N * (double)(4 * nwp + 14 + ((a.naive || a.theta) ? 0 : 1));
    ctl->alg_flops += (double)N * (2.0 * (5 * nwp + 8 + (a.theta ? 1 : 0)) + ((a.naive || a.theta) ? 0.0 : 1.0));
    if (a.theta) ctl->theta = rr > 0.0 ? s_sum[4 + nwp] / rr : 1.0;
  }
  const int nu = nu_window(i, a.mmax, ctl->truncation);
  // window dots in order k = i-1-nwp .. i-1 (W_{i-1}, then s_{i-1}); W_i is
  // the last nu of them
  static_assert(NWARPS * ND >= 3 * NW + 2, "scalar-phase scratch fits in s_red");
  double* s_cw = s_red;              // NW + 1 window dots
  double* s_tmp = s_red + NW + 1;    // 2 NW + 1
  if ((int)threadIdx.x <= nwp) s_cw[threadIdx.x] = (int)threadIdx.x < nwp ? s_sum[4 + threadIdx.x] : s_sum[3];
  __syncthreads();
  cgcr_iteration_scalars_block(ctl, i, nu, gamma, delta, rr, s_cw + (nwp + 1 - nu), s_tmp, NW);
}

// Pipeline fill dots: gamma_0 = <u_0, r_0>, delta_0 = <u_0, w_0>, ||r_0||^2,
// then eta_0 = delta_0, alpha_0 = gamma_0 / eta_0 and the fill status.  For
// Alg. 12 `u` is w_0 = s_0: gamma_0 = <r_0, s_0>, eta_0 = <s_0, s_0>.
__global__ void __launch_bounds__(kThreads) pipefcg_fill_dots(const double* __restrict__ u,
                                                              const double* __restrict__ r,
                                                              const double* __restrict__ w, int64_t N,
                                                              SolveCtl* ctl, double* partials) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const double uv = u[e], rv = r[e];
    acc[0] = fma(uv, rv, acc[0]);
    acc[1] = fma(uv, w[e], acc[1]);
    acc[2] = fma(rv, rv, acc[2]);
  }
  __shared__ double s_red[(kThreads / 32) * 3];
  __shared__ double s_sum[3];
  if (!reduce_last_block<3>(acc, 3, partials, 3, &ctl->counter, s_red, s_sum)) return;
  if (threadIdx.x != 0) return;
  // eta_0 = delta_0 (Alg. 8)
  cgcr_fill_scalars(ctl, s_sum[0], s_sum[1], s_sum[2]);
}

// eq. (proj) variant: t = w - theta r and tu = theta u (the preconditioner adds tu).
__global__ void __launch_bounds__(kThreads) theta_prep_kernel(const double* __restrict__ w,
                                                              const double* __restrict__ r,
                                                              const double* __restrict__ u, double* __restrict__ t,
                                                              double* __restrict__ tu, int64_t N,
                                                              const SolveCtl* ctl) {
  if (ctl->status != kRun) return;
  const double th = ctl->theta;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    t[e] = fma(-th, r[e], w[e]);
    tu[e] = th * u[e];
  }
}

template <int NW>
static cudaError_t launch_pass(const FcgArgs& a, int blocks, cudaStream_t st) {
  pipefcg_pass<NW><<<blocks, kPassThreads, 0, st>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_pass_any(const FcgArgs& a, int nw_template, int blocks, cudaStream_t st) {
  switch (nw_template) {
    case 4: return launch_pass<4>(a, blocks, st);
    case 8: return launch_pass<8>(a, blocks, st);
    case 16: return launch_pass<16>(a, blocks, st);
    default: return launch_pass<32>(a, blocks, st);
  }
}

int pipefcg_template(int mmax) { return mmax <= 4 ? 4 : mmax <= 8 ? 8 : mmax <= 16 ? 16 : 32; }

// --------------------------------------------------------------------------
// Method object
// --------------------------------------------------------------------------

class PipeFcg : public Method {
 public:
  PipeFcg(bool naive, bool gcrw, bool theta = false) : naive_(naive), gcrw_(gcrw), theta_(theta) {}

  int64_t workspace_doubles(int64_t N, int mmax) const override {
    return 7 * N + 4 * (int64_t)(mmax + 1) * N;
  }

  void bind(double* ws, int64_t N, int mmax) override {
    N_ = N;
    mmax_ = mmax;
    r_ = ws; u_ = r_ + N; w_ = u_ + N; m_ = w_ + N; n_ = m_ + N; t_ = n_ + N; tmp_ = t_ + N;
    P_ = tmp_ + N;
    S_ = P_ + (mmax + 1) * N;
    Q_ = S_ + (mmax + 1) * N;
    Z_ = Q_ + (mmax + 1) * N;
  }

  double* scratch() override { return tmp_; }

  bool configure(const pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, int64_t N, int mode) override {
    persistent_ = mode != 1 && persistent_eligible(ctx, op, pc, PFK_PIPEFCG, naive_ || gcrw_ || theta_, N);
    return persistent_;
  }

  cudaError_t fill(const SolveEnv& env, const double* b, double* x) override {
    cudaStream_t st = env.st;
    cudaError_t e;
    if ((e = op_apply(env.op, x, r_, b, nullptr, st)) != cudaSuccess) return e;          // r_0 = b - A x_0
    if ((e = env.pc_apply(r_, u_, nullptr, nullptr)) != cudaSuccess) return e;           // u_0 = B(r_0)
    if ((e = op_apply(env.op, u_, w_, nullptr, nullptr, st)) != cudaSuccess) return e;  // w_0 = A p_0, p_0 = u_0
    if ((e = env.pc_apply(w_, m_, nullptr, nullptr)) != cudaSuccess) return e;           // m_0 = B(w_0)
    if ((e = op_apply(env.op, m_, n_, nullptr, nullptr, st)) != cudaSuccess) return e;   // n_0 = A m_0
    const int blocks = stream_blocks(env.ctx, N_, 2);
    if (!env.partials_fit(blocks, 3)) return cudaErrorInvalidValue;
    pipefcg_fill_dots<<<blocks, kThreads, 0, st>>>(gcrw_ ? w_ : u_, r_, w_, N_, env.ctl, env.partials);
    return cudaGetLastError();
  }

  cudaError_t iteration(const SolveEnv& env, double* x) override {
    if (persistent_) {
      // m alternates between m_ (even iterations, written by the fill) and t_
      cudaError_t e = env.mark_pass(0);
      if (e != cudaSuccess) return e;
      e = launch_persistent(env, true, mmax_, x, r_, u_, w_, m_, t_, n_, P_, S_, Q_, Z_, kPersistentIters);
      if (e != cudaSuccess) return e;
      return env.mark_pass(1);
    }
    FcgArgs a;
    a.x = x; a.r = r_; a.u = u_; a.w = w_; a.m = m_; a.n = n_; a.t = t_;
    a.P = P_; a.S = S_; a.Q = Q_; a.Z = Z_;
    a.N = N_; a.mmax = mmax_; a.naive = naive_ ? 1 : 0; a.gcrw = gcrw_ ? 1 : 0; a.theta = theta_ ? 1 : 0;
    a.ctl = env.ctl; a.partials = env.partials;
    const int tmpl = pipefcg_template(mmax_);
    cudaError_t e = env.mark_pass(0);
    if (e != cudaSuccess) return e;
    const int64_t need = (N_ + kPassThreads - 1) / kPassThreads;
    const int64_t cap = (int64_t)env.ctx->num_sms * kPassBlocksPerSm;
    const int blocks = (int)(need < cap ? need : cap);
    if (!env.partials_fit_2l(blocks, tmpl + 5)) return cudaErrorInvalidValue;
    e = launch_pass_any(a, tmpl, blocks, env.st);
    if (e != cudaSuccess) return e;
    if ((e = env.mark_pass(1)) != cudaSuccess) return e;
    const int* status = &env.ctl->status;
    if (naive_) {
      e = env.pc_apply(w_, m_, nullptr, status);                 // m_i = B(w_i)          (Alg. 7)
    } else if (theta_) {
      theta_prep_kernel<<<stream_blocks(env.ctx, N_, 8), kThreads, 0, env.st>>>(w_, r_, u_, t_, tmp_, N_, env.ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      e = env.pc_apply(t_, m_, tmp_, status);                    // m_i = theta u_i + B(w_i - theta r_i)
    } else {
      e = env.pc_apply(t_, m_, u_, status);                      // m_i = u_i + B(w_i - r_i) (Alg. 8)
    }
    if (e != cudaSuccess) return e;
    return op_apply(env.op, m_, n_, nullptr, status, env.st);    // n_i = A m_i
  }

 private:
  bool naive_;
  bool gcrw_;
  bool theta_;
  bool persistent_ = false;
  int64_t N_ = 0;
  int mmax_ = 0;
  double *r_ = nullptr, *u_ = nullptr, *w_ = nullptr, *m_ = nullptr, *n_ = nullptr, *t_ = nullptr,
         *tmp_ = nullptr;
  double *P_ = nullptr, *S_ = nullptr, *Q_ = nullptr, *Z_ = nullptr;
};

Method* make_pipefcg(bool naive) { return new PipeFcg(naive, false); }
Method* make_pipegcr_w() { return new PipeFcg(false, true); }
Method* make_pipefcg_theta() { return new PipeFcg(false, false, true); }

}  // namespace pfk
