// PIPEGCR (Alg. 11) on one GPU.
//
// Iteration i is three kernel groups reading their scalars from the device
// control block (capturable in one CUDA graph):
//
//  1. pipegcr_advance<NW>: the deferred MAXPYs of iteration i-1
//       p_{i-1} = u_{i-1} + sum beta_{i-1,k} p_k,  s_{i-1} = w_{i-1} + ...,
//       q_{i-1} = m_{i-1} + ...
//     into ring slot (i-1) mod (mmax+1), then x_i, r_i and u_i (tilde-u) with
//     alpha_{i-1};
//  2. the iteration's single reduction with w_i = A u_i: gamma_i = <r_i, w_i>,
//     delta_i = <w_i, w_i>, ||r_i||^2 and <w_i, s_k> for the nu_i stored s_k,
//     and the preconditioner input t = w_i - r_i; the last block computes beta,
//     eta_i, alpha_i and the status.  For a stencil operator this is two
//     kernels -- the tiled z-marching walk (w, t and the three scalar dots,
//     handed over in the control block) and a streaming pass over w and the
//     window (pipegcr_window_dots) -- because the fused one-kernel form,
//     pipegcr_apply_dots (kept for CSR operators), is latency-bound;
//  3. the preconditioner, m_i = u_i + B(w_i - r_i).
//
// Unlike Alg. 8 the operator product w_i = A u_i is explicit, so the
// reduction overlaps only the preconditioner (Sec. 4.2).
#include "pfk_internal.cuh"
#include "solver.cuh"
#include "stencil.cuh"

namespace pfk {

struct GcrArgs {
  double* x;
  double* r;
  double* u;
  double* w;
  const double* m;
  double* t;
  double* P;
  double* S;
  double* Q;
  int64_t N;
  int mmax;
  SolveCtl* ctl;
  double* partials;
};

constexpr int kGcrThreads = 128;
constexpr int kGcrBlocksPerSm = 6;
constexpr int kGcrStride = kGcrThreads + 1;
static_assert(kGcrBlocksPerSm <= kMaxBlocksPerSm, "partials are sized for kMaxBlocksPerSm blocks per SM");

template <int NW>
__global__ void __launch_bounds__(kThreads, 3) pipegcr_advance(GcrArgs a) {
  SolveCtl* ctl = a.ctl;
  if (ctl->status != kRun) return;
  __shared__ double s_beta[NW];
  __shared__ size_t s_off[NW];
  const int iprev = ctl->i;
  const int nwp = ctl->nw;
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
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const double u0 = a.u[e];
    double p = u0, s = a.w[e], q = a.m[e];
#pragma unroll 4
    for (int j = 0; j < nwp; ++j) {
      const size_t o = s_off[j] + e;
      const double b = s_beta[j];
      p = fma(b, a.P[o], p);
      s = fma(b, a.S[o], s);
      q = fma(b, a.Q[o], q);
    }
    a.P[coff + e] = p;
    a.S[coff + e] = s;
    a.Q[coff + e] = q;
    a.x[e] = fma(alpha, p, a.x[e]);
    a.r[e] = fma(-alpha, s, a.r[e]);
    a.u[e] = fma(-alpha, q, u0);
  }
}

// Operator row value (A u)_r of a CSR operator (stencils take the tiled walk
// below).
struct OpView {
  const int32_t* rowptr;
  const int32_t* colidx;
  const double* vals;
};

__device__ __forceinline__ double op_row_csr(const OpView& A, const double* __restrict__ m, int64_t r) {
  double acc = 0.0;
  for (int32_t p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) acc = fma(A.vals[p], m[A.colidx[p]], acc);
  return acc;
}

// CSR operators: warps walk "chunks" of 32 consecutive rows.  Each chunk's w
// values and stored s_k values are staged in shared memory and lane jj of the
// warp sums w_e s_{k_jj,e} over the chunk (the same transposed window dot as
// in the PIPEFCG pass).
template <int NW>
__global__ void __launch_bounds__(kGcrThreads, kGcrBlocksPerSm) pipegcr_apply_dots(GcrArgs a, OpView A) {
  SolveCtl* ctl = a.ctl;
  if (ctl->status != kRun) return;
  constexpr int ND = NW + 3;
  constexpr int NWARPS = kGcrThreads / 32;
  __shared__ size_t s_off[NW];
  __shared__ double s_sk[NW * kGcrStride];
  __shared__ double s_w[kGcrThreads];
  __shared__ double s_red[NWARPS * ND];
  __shared__ double s_sum[ND];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = ctl->i + 1;
  const int nu = nu_window(i, a.mmax, ctl->truncation);
  const int slots = a.mmax + 1;
  const int64_t N = a.N;
  if (threadIdx.x < nu) {
    const int k = i - nu + (int)threadIdx.x;
    s_off[threadIdx.x] = (size_t)(k % slots) * (size_t)N;
  }
  __syncthreads();
  double* my_sk = s_sk + threadIdx.x;
  const double* warp_w = s_w + warp * 32;
  const double* lane_row = s_sk + lane * kGcrStride + warp * 32;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0, gw = 0.0;

  const int64_t nchunks = (N + 31) / 32;
  const int64_t gwarps = (int64_t)gridDim.x * NWARPS;
  for (int64_t ch0 = (int64_t)blockIdx.x * NWARPS; ch0 < nchunks; ch0 += gwarps) {
    // all warps of the block iterate together (block-uniform trip count)
    const int64_t ch = ch0 + warp;
    double wv = 0.0;
    bool valid = false;
    int64_t c = 0;
    if (ch < nchunks) {
      c = ch * 32 + lane;
      if (c < N) {
        valid = true;
        wv = op_row_csr(A, a.u, c);
      }
    }
    if (valid) {
      const double rv = a.r[c];
      // the window's s_k values, eight loads in flight at a time, parked in
      // shared memory for the transposed dots
#pragma unroll
      for (int j0 = 0; j0 < NW; j0 += 8) {
        double sv[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          sv[jj] = (j0 + jj < nu) ? __ldg(&a.S[s_off[j0 + jj] + c]) : 0.0;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (j0 + jj < nu) my_sk[(j0 + jj) * kGcrStride] = sv[jj];
      }
      a.w[c] = wv;
      a.t[c] = wv - rv;
      g0 = fma(rv, wv, g0);
      g1 = fma(wv, wv, g1);
      g2 = fma(rv, rv, g2);
    } else {
#pragma unroll
      for (int j = 0; j < NW; ++j)
        if (j < nu) my_sk[j * kGcrStride] = 0.0;
    }
    s_w[threadIdx.x] = valid ? wv : 0.0;
    __syncwarp();
    if (lane < nu) {
      double cacc = gw;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) cacc = fma(warp_w[t], lane_row[t], cacc);
      gw = cacc;
    }
    __syncwarp();
  }
  {
    const double w0 = warp_sum(g0), w1 = warp_sum(g1), w2 = warp_sum(g2);
    const int nd = nu + 3;
    if (lane == 0) {
      s_red[warp * nd + 0] = w0;
      s_red[warp * nd + 1] = w1;
      s_red[warp * nd + 2] = w2;
    }
    if (lane < nu) s_red[warp * nd + 3 + lane] = gw;
    __syncthreads();
  }
  if (!combine_block_partials_2l(s_red, nu + 3, a.partials, ND, &ctl->counter, ctl->gcounter, s_sum)) return;
  if (threadIdx.x == 0) {
    // algorithmic traffic of the iteration's two kernels: advance reads u, w, m,
    // x, r and 3 nu_{i-1} history vectors, writes p, s, q, x, r, u; the apply
    // reads u, r, the operator (4 coefficient arrays for a stencil) and nu_i s_k,
    // writes w and t.  FP64: 3 nu_{i-1} + 3 + 7 (stencil) + nu_i + 3 FMAs, 1 sub.
    const int nwp = ctl->nw;
    ctl->passes += 1;
    ctl->alg_bytes += 8.0 * (double)N * (double)((5 + 3 * nwp + 6) + (2 + nu + 2));
    ctl->alg_flops += (double)N * (2.0 * (3 * nwp + 3 + nu + 3) + 1.0);
  }
  static_assert(NWARPS * ND >= 2 * NW + 1, "scalar-phase scratch fits in s_red");
  cgcr_iteration_scalars_block(ctl, i, nu, s_sum[0], s_sum[1], s_sum[2], s_sum + 3, s_red, NW);
}

// ---- stencil operators: w = A u by the tiled walk, then the window dots ----

// Epilogue of the walk: w = A u, t = w - r, and per-thread <r, w>, <w, w>, <r, r>.
struct GcrApplyEpi {
  double* __restrict__ w;
  double* __restrict__ t;
  const double* __restrict__ r;
  double g0, g1, g2;
  struct Pre {
    double r;
  };
  __device__ __forceinline__ Pre pre(int64_t c) const { return Pre{r[c]}; }
  __device__ __forceinline__ void operator()(int64_t c, double wv, double, const Pre& p) {
    w[c] = wv;
    t[c] = wv - p.r;
    g0 = fma(p.r, wv, g0);
    g1 = fma(wv, wv, g1);
    g2 = fma(p.r, p.r, g2);
  }
};

template <bool ADV>
__global__ void __launch_bounds__(kTileThreads) pipegcr_apply_walk(TiledStencil<double, double> T, GcrArgs a) {
  SolveCtl* ctl = a.ctl;
  if (ctl->status != kRun) return;
  GcrApplyEpi e{a.w, a.t, a.r, 0.0, 0.0, 0.0};
  tiled_stencil_walk<double, double, ADV, 1>(T, a.u, e);
  double acc[3] = {e.g0, e.g1, e.g2};
  __shared__ double smem[(kTileThreads / 32) * 3];
  __shared__ double sums[3];
  if (reduce_last_block<3>(acc, 3, a.partials, 3, &ctl->counter, smem, sums) && threadIdx.x == 0) {
    ctl->pend[0] = sums[0];
    ctl->pend[1] = sums[1];
    ctl->pend[2] = sums[2];
  }
}

// <w_i, s_k> over the window, one register accumulator per window slot and
// thread (independent FMAs, no shared-memory staging); the last block adds the
// walk's gamma, delta, ||r||^2 and runs the scalar phase of iteration i.
constexpr int kWinBlocksPerSm = 5;   // 93 registers at NW = 32

template <int NW>
__global__ void __launch_bounds__(kGcrThreads, kWinBlocksPerSm) pipegcr_window_dots(GcrArgs a, int stencil_flops) {
  SolveCtl* ctl = a.ctl;
  if (ctl->status != kRun) return;
  constexpr int NWARPS = kGcrThreads / 32;
  __shared__ size_t s_off[NW];
  __shared__ double s_red[NWARPS * NW];
  __shared__ double s_sum[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = ctl->i + 1;
  const int nu = nu_window(i, a.mmax, ctl->truncation);
  const int slots = a.mmax + 1;
  const int64_t N = a.N;
  if (threadIdx.x < nu) {
    const int k = i - nu + (int)threadIdx.x;
    s_off[threadIdx.x] = (size_t)(k % slots) * (size_t)N;
  }
  __syncthreads();
  double acc[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) acc[j] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * kGcrThreads + threadIdx.x; e < N; e += (int64_t)gridDim.x * kGcrThreads) {
    const double wv = __ldg(&a.w[e]);
#pragma unroll
    for (int j = 0; j < NW; ++j)
      if (j < nu) acc[j] = fma(wv, __ldg(&a.S[s_off[j] + e]), acc[j]);
  }
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    if (j < nu) {
      const double v = warp_sum(acc[j]);
      if (lane == 0) s_red[warp * nu + j] = v;
    }
  }
  __syncthreads();
  if (!combine_block_partials_2l(s_red, nu, a.partials, NW, &ctl->counter, ctl->gcounter, s_sum)) return;
  if (threadIdx.x == 0) {
    // algorithmic traffic of the iteration's kernels: advance reads u, w, m, x,
    // r and 3 nu_{i-1} history vectors, writes p, s, q, x, r, u; the walk reads
    // u, r and the 4 coefficient arrays, writes w and t; the window pass reads w
    // and nu_i s_k.  FP64: 3 nu_{i-1} + 3 (advance) + 7 (stencil) + 3 + nu_i FMAs, 1 sub.
    const int nwp = ctl->nw;
    ctl->passes += 1;
    ctl->alg_bytes += 8.0 * (double)N * (double)((5 + 3 * nwp + 6) + (2 + 4 + 2) + (1 + nu));
    ctl->alg_flops += (double)N * (2.0 * (3 * nwp + 3 + stencil_flops + nu + 3) + 1.0);
  }
  static_assert(NWARPS * NW >= 2 * NW + 1, "scalar-phase scratch fits in s_red");
  cgcr_iteration_scalars_block(ctl, i, nu, ctl->pend[0], ctl->pend[1], ctl->pend[2], s_sum, s_red, NW);
}

// Fill: gamma_0 = <r_0, w_0> with w_0 = A u_0 = s_0, eta_0 = <s_0, s_0>, ||r_0||^2.
__global__ void __launch_bounds__(kThreads) pipegcr_fill_dots(const double* __restrict__ r,
                                                              const double* __restrict__ w, int64_t N,
                                                              SolveCtl* ctl, double* partials) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const double rv = r[e], wv = w[e];
    acc[0] = fma(rv, wv, acc[0]);
    acc[1] = fma(wv, wv, acc[1]);
    acc[2] = fma(rv, rv, acc[2]);
  }
  __shared__ double s_red[(kThreads / 32) * 3];
  __shared__ double s_sum[3];
  if (!reduce_last_block<3>(acc, 3, partials, 3, &ctl->counter, s_red, s_sum)) return;
  if (threadIdx.x != 0) return;
  cgcr_fill_scalars(ctl, s_sum[0], s_sum[1], s_sum[2]);
}

static int gcr_template(int mmax) { return mmax <= 8 ? 8 : mmax <= 16 ? 16 : 32; }

class PipeGcr : public Method {
 public:
  int64_t workspace_doubles(int64_t N, int mmax) const override { return 6 * N + 3 * (int64_t)(mmax + 1) * N; }

  void bind(double* ws, int64_t N, int mmax) override {
    N_ = N;
    mmax_ = mmax;
    r_ = ws; u_ = r_ + N; w_ = u_ + N; m_ = w_ + N; t_ = m_ + N; tmp_ = t_ + N;
    P_ = tmp_ + N;
    S_ = P_ + (mmax + 1) * N;
    Q_ = S_ + (mmax + 1) * N;
  }

  double* scratch() override { return tmp_; }

  cudaError_t fill(const SolveEnv& env, const double* b, double* x) override {
    cudaStream_t st = env.st;
    cudaError_t e;
    if ((e = op_apply(env.op, x, r_, b, nullptr, st)) != cudaSuccess) return e;          // r_0 = b - A x_0
    if ((e = env.pc_apply(r_, u_, nullptr, nullptr)) != cudaSuccess) return e;           // u_0 = B(r_0), p_0 = u_0
    if ((e = op_apply(env.op, u_, w_, nullptr, nullptr, st)) != cudaSuccess) return e;  // s_0 = A p_0 (kept as w)
    if ((e = env.pc_apply(w_, m_, nullptr, nullptr)) != cudaSuccess) return e;           // q_0 = B(s_0) (kept as m)
    const int blocks = stream_blocks(env.ctx, N_, 2);
    if (!env.partials_fit(blocks, 3)) return cudaErrorInvalidValue;
    pipegcr_fill_dots<<<blocks, kThreads, 0, st>>>(r_, w_, N_, env.ctl, env.partials);
    return cudaGetLastError();
  }

  cudaError_t iteration(const SolveEnv& env, double* x) override {
    GcrArgs a;
    a.x = x; a.r = r_; a.u = u_; a.w = w_; a.m = m_; a.t = t_;
    a.P = P_; a.S = S_; a.Q = Q_;
    a.N = N_; a.mmax = mmax_; a.ctl = env.ctl; a.partials = env.partials;
    const pfk_operator* op = env.op;
    OpView A;
    A.rowptr = op->rowptr; A.colidx = op->colidx; A.vals = op->vals;
    const bool stencil = op->rowptr == nullptr;
    const bool adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
    const int tmpl = gcr_template(mmax_);
    const int ablocks = stream_blocks(env.ctx, N_, 4);
    const int64_t chunks = (N_ + 31) / 32;
    const int64_t need = (chunks + kGcrThreads / 32 - 1) / (kGcrThreads / 32);
    const int64_t cap = (int64_t)env.ctx->num_sms * kGcrBlocksPerSm;
    const int dblocks = (int)(need < cap ? need : cap);
    if (!env.partials_fit_2l(dblocks, tmpl + 3)) return cudaErrorInvalidValue;
    cudaError_t e = env.mark_pass(0);
    if (e != cudaSuccess) return e;
    if (stencil) {
      TiledStencil<double, double> T;
      const int slots = adv ? tiled_stencil_slots(pipegcr_apply_walk<true>, env.ctx->num_sms)
                            : tiled_stencil_slots(pipegcr_apply_walk<false>, env.ctx->num_sms);
      const int units = tiled_stencil_setup<double, double>(T, op, op->d, op->kx, op->ky, op->kz, slots);
      const int64_t wcap = env.partials_cap / 3;
      const int wblocks = (int)(units < wcap ? units : wcap);
      const int64_t wneed = (N_ + kGcrThreads - 1) / kGcrThreads;
      const int64_t wslots = (int64_t)env.ctx->num_sms * kWinBlocksPerSm;
      const int sblocks = (int)(wneed < wslots ? wneed : wslots);
      if (!env.partials_fit_2l(sblocks, tmpl)) return cudaErrorInvalidValue;
      switch (tmpl) {
        case 8: pipegcr_advance<8><<<ablocks, kThreads, 0, env.st>>>(a); break;
        case 16: pipegcr_advance<16><<<ablocks, kThreads, 0, env.st>>>(a); break;
        default: pipegcr_advance<32><<<ablocks, kThreads, 0, env.st>>>(a); break;
      }
      if (adv) pipegcr_apply_walk<true><<<wblocks, kTileThreads, 0, env.st>>>(T, a);
      else pipegcr_apply_walk<false><<<wblocks, kTileThreads, 0, env.st>>>(T, a);
      const int sf = adv ? 10 : 7;
      switch (tmpl) {
        case 8: pipegcr_window_dots<8><<<sblocks, kGcrThreads, 0, env.st>>>(a, sf); break;
        case 16: pipegcr_window_dots<16><<<sblocks, kGcrThreads, 0, env.st>>>(a, sf); break;
        default: pipegcr_window_dots<32><<<sblocks, kGcrThreads, 0, env.st>>>(a, sf); break;
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = env.mark_pass(1)) != cudaSuccess) return e;
      return env.pc_apply(t_, m_, u_, &env.ctl->status);   // m_i = B(w_i - r_i) + u_i
    }
    switch (tmpl) {
      case 8:
        pipegcr_advance<8><<<ablocks, kThreads, 0, env.st>>>(a);
        pipegcr_apply_dots<8><<<dblocks, kGcrThreads, 0, env.st>>>(a, A);
        break;
      case 16:
        pipegcr_advance<16><<<ablocks, kThreads, 0, env.st>>>(a);
        pipegcr_apply_dots<16><<<dblocks, kGcrThreads, 0, env.st>>>(a, A);
        break;
      default:
        pipegcr_advance<32><<<ablocks, kThreads, 0, env.st>>>(a);
        pipegcr_apply_dots<32><<<dblocks, kGcrThreads, 0, env.st>>>(a, A);
        break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = env.mark_pass(1)) != cudaSuccess) return e;
    return env.pc_apply(t_, m_, u_, &env.ctl->status);   // m_i = B(w_i - r_i) + u_i
  }

 private:
  int64_t N_ = 0;
  int mmax_ = 0;
  double *r_ = nullptr, *u_ = nullptr, *w_ = nullptr, *m_ = nullptr, *t_ = nullptr, *tmp_ = nullptr;
  double *P_ = nullptr, *S_ = nullptr, *Q_ = nullptr;
};

Method* make_pipegcr() { return new PipeGcr(); }

}  // namespace pfk
