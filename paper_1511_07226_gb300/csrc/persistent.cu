// Persistent single-launch iterations for small systems: PIPEFCG (Alg. 8) and
// FCG (Alg. 2) with an assembled CSR operator and the Jacobi (or identity)
// preconditioner, many iterations per launch.
//
// At a few thousand unknowns (the 64 x 64 problem with inclusions) the whole
// Krylov state sits in L2 and an iteration is nothing but its dependency
// chain: every kernel boundary and every reduction that some later step waits
// for costs a fixed latency.  Here one cooperative launch runs up to `iters`
// iterations; the blocks own fixed rows and meet at grid barriers (bounded
// waits), so the cost of a dependency is one barrier instead of a kernel
// boundary plus a last-block combine.
//
//  * PIPEFCG: one barrier per iteration.  The pass (deferred MAXPYs of
//    iteration i-1, advance of x, r, u, w, the dot partials of gamma_i,
//    delta_i and <u_i, s_k>) and the Jacobi preconditioner m_i = u_i +
//    D^-1 (w_i - r_i) are row-local; only n_i = A m_i reads other blocks' rows
//    and needs the barrier.  The reduction's partial sums are written before
//    the same barrier, and after it every block combines them itself (in one
//    fixed order, so every block gets bitwise the same scalars) while its
//    operator rows are in flight: the reduction is hidden behind the operator
//    application exactly as the reordering of Alg. 8 allows (Sec. 3.2.3).
//    m and the partials alternate between two buffers, so a block that runs
//    ahead into the next pass never overwrites what a slower block still reads.
//  * FCG: the same data and arithmetic per statement, but Alg. 2's blocking
//    dependencies need three barriers per iteration: gamma_i and the betas
//    before p_i, every p_i before s_i = A p_i, eta_i before the next advance.
//
// Rows are split in chunks of 32 over the blocks; four threads share a row and
// split the direction window between them (k = q, q + 4, ... for thread q of
// the row), so the four warps of a block spread the FP64 work over the SM's
// four sub-partitions.  The quad sums are combined by a fixed shuffle tree, so
// every run is bitwise reproducible.  Block 0 keeps the control block up to
// date (status, counters, history) for the host driver.
#include "pfk_internal.cuh"
#include "solver.cuh"

#include <cmath>

namespace pfk {

constexpr int kPerThreads = 128;
constexpr int kPerRows = 32;                // rows of a chunk (4 threads per row)
constexpr int kPerNd = PFK_MAX_MMAX + 4;    // largest partial row (gamma, delta, ||r||^2, c_{i-1}, window)
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;
constexpr int kMaxPerBlocks = 192;          // grid cap (the partial rows live in shared memory: 54 KB)

struct PersistArgs {
  const int32_t* rowptr;
  const int32_t* colidx;
  const double* vals;
  const double* dinv;      // Jacobi D^-1, or null for the identity
  int64_t N;
  int mmax;
  int iters;               // iterations per launch (at most)
  int nchunks;
  double* x;
  double* r;
  double* u;
  double* w;
  double* m0;              // m of even iterations (the fill writes m_0 here)
  double* m1;              // m of odd iterations
  double* n;
  double* P;
  double* S;
  double* Q;
  double* Z;
  SolveCtl* ctl;
  double* partials;        // PIPEFCG: [2][grid][kPerNd]; FCG: [grid][kPerNd] then [grid]
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch (all blocks resident).  Arrival on a
// counter; the last arrival resets it and bumps the generation the others
// wait on.  The wait is bounded: on time-out the block raises bar_abort, and a
// raised bar_abort ends every other wait.  Returns false in that case.
__device__ __forceinline__ bool grid_barrier(SolveCtl* ctl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire(&ctl->bar_gen);
    __threadfence();
    int ok = 1;
    if (atomicAdd(&ctl->bar_count, 1u) == gridDim.x - 1) {
      ctl->bar_count = 0u;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire(&ctl->bar_gen) == g) {
        if (ld_acquire(&ctl->bar_abort)) { ok = 0; break; }
        if (global_ns() - t0 > kBarrierTimeoutNs) {
          atomicExch(&ctl->bar_abort, 1u);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum over the 32 rows of a chunk of a value held by thread q = j % 4 of each
// row (lanes q, q + 4, ..., q + 28 of a warp), then over the block's four
// warps in order: red[j] for j < nd.  `v` is this thread's value of column
// (4 * slot + q); call with every thread.  smem: 4 * nd doubles.
__device__ __forceinline__ double quad_col_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

// Copies the block rows partials[0 .. nb * kPerNd) (16-byte aligned, a
// multiple of 16 bytes) into shared memory with asynchronous 16-byte copies
// issued by all threads at once (cp.async, completed by wait_partials), so one
// L2 round trip brings every row instead of one per load.
__device__ __forceinline__ void fetch_partials(const double* partials, int nb, double* s_part) {
  const int chunks = nb * (kPerNd / 2);
  for (int c = threadIdx.x; c < chunks; c += kPerThreads) {
    const unsigned int dst = (unsigned int)__cvta_generic_to_shared(s_part + 2 * c);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(partials + 2 * c) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void wait_partials() {
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
}

// Sums the fetched rows s_part[b * kPerNd + j], b < nb, j < nd, in a fixed
// order (lane l of warp w: rows l, l + 32, ... of columns w, w + 4, ..., then a
// fixed shuffle tree) into out[j] (shared memory).  Every block that calls it
// gets bitwise the same sums.
__device__ __forceinline__ void sum_partials(const double* s_part, int nb, int nd, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < nd; j += kPerThreads / 32) {
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) a += s_part[b * kPerNd + j];
    a = warp_sum(a);
    if (lane == 0) out[j] = a;
  }
  __syncthreads();
}

// Writes this block's partial row: column j of the block = sum over its
// threads' values vals(j).  acc[s] is this thread's sum for column 4 s + q of
// the window part; sc[0..3] the scalar columns (held by q = 0 threads, zero
// elsewhere).  Layout: [sc0, sc1, sc2, sc3, window 0 .. nw-1].
template <int NWQ>
__device__ __forceinline__ void write_pipefcg_row(const double (&sc)[4], const double (&acc)[NWQ], int nw,
                                                  double* s_red, double* row) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = lane & 3;
  // scalars: full warp sums (only q = 0 lanes hold them)
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double v = warp_sum(sc[c]);
    if (lane == 0) s_red[warp * kPerNd + c] = v;
  }
#pragma unroll
  for (int s = 0; s < NWQ; ++s) {
    const double v = quad_col_sum(acc[s]);
    const int j = 4 * s + q;
    if (lane < 4 && j < nw) s_red[warp * kPerNd + 4 + j] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 4 + nw; j += blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kPerThreads / 32; ++w) v += s_red[w * kPerNd + j];
    row[j] = v;
  }
}

// Scalars every block keeps for itself (identical in all blocks).
struct PerState {
  int status, it, i, nw, hist_len;
  int go;
  double alpha, gamma, delta, eta, rho;
  double beta[PFK_MAX_MMAX];
  double eta_ring[PFK_MAX_MMAX + 1];
  double sums[kPerNd];
  double cw[PFK_MAX_MMAX + 1];
  double tmp[2 * PFK_MAX_MMAX + 2];
};

__device__ __forceinline__ void load_state(PerState* st, const SolveCtl* ctl) {
  if (threadIdx.x == 0) {
    st->status = ctl->status;
    st->it = ctl->it;
    st->i = ctl->i;
    st->nw = ctl->nw;
    st->hist_len = ctl->hist_len;
    st->alpha = ctl->alpha;
    st->gamma = ctl->gamma;
    st->delta = ctl->delta;
    st->eta = ctl->eta;
    st->rho = ctl->rho;
  }
  for (int j = threadIdx.x; j < PFK_MAX_MMAX; j += blockDim.x) st->beta[j] = ctl->beta[j];
  for (int j = threadIdx.x; j <= PFK_MAX_MMAX; j += blockDim.x) st->eta_ring[j] = ctl->eta_ring[j];
  __syncthreads();
}

// History entry of block 0 (the others only keep the count).
__device__ __forceinline__ void per_push_history(PerState* st, SolveCtl* ctl, double rho, double rn, double eta,
                                                 double alpha) {
  if (blockIdx.x == 0 && ctl->history && st->hist_len < ctl->hist_cap) {
    double* h = ctl->history + (size_t)st->hist_len * PFK_HISTORY_FIELDS;
    h[0] = rho; h[1] = rn; h[2] = eta; h[3] = alpha;
  }
  st->hist_len += 1;
}

// Block 0 copies the state back to the control block (after each iteration).
__device__ __forceinline__ void store_state(const PerState* st, SolveCtl* ctl, int nbeta) {
  if (blockIdx.x != 0) return;
  for (int j = threadIdx.x; j < nbeta; j += blockDim.x) ctl->beta[j] = st->beta[j];
  if (threadIdx.x == 0) {
    ctl->status = st->status;
    ctl->it = st->it;
    ctl->i = st->i;
    ctl->nw = st->nw;
    ctl->hist_len = st->hist_len;
    ctl->alpha = st->alpha;
    ctl->gamma = st->gamma;
    ctl->delta = st->delta;
    ctl->eta = st->eta;
    ctl->rho = st->rho;
    const int slots = ctl->mmax + 1;
    ctl->eta_ring[st->i % slots] = st->eta_ring[st->i % slots];
  }
}

__device__ __forceinline__ double csr_row(const PersistArgs& a, const double* m, int64_t e) {
  double acc = 0.0;
  const int32_t end = a.rowptr[e + 1];
  for (int32_t p = a.rowptr[e]; p < end; ++p) acc = fma(a.vals[p], __ldcg(&m[a.colidx[p]]), acc);
  return acc;
}

// ---------------------------------------------------------------------------
// PIPEFCG
// ---------------------------------------------------------------------------

template <int NW>
__global__ void __launch_bounds__(kPerThreads) pipefcg_persistent(PersistArgs a) {
  constexpr int NWQ = NW / 4;
  extern __shared__ double s_part[];     // the grid's partial rows, nb * kPerNd
  __shared__ PerState st;
  __shared__ double s_red[(kPerThreads / 32) * kPerNd];
  __shared__ size_t s_off[NW];
  SolveCtl* ctl = a.ctl;
  load_state(&st, ctl);
  const int q = threadIdx.x & 3;
  const int rowi = threadIdx.x >> 2;
  const int slots = a.mmax + 1;
  const int64_t N = a.N;
  const int nb = gridDim.x;

  for (int g = 0; g < a.iters; ++g) {
    if (st.status != kRun) break;
    const int iprev = st.i, i = iprev + 1;
    const int nwp = st.nw;
    const double alpha = st.alpha;
    const double* mprev = (iprev & 1) ? a.m1 : a.m0;
    double* mnew = (i & 1) ? a.m1 : a.m0;
    double* part = a.partials + (size_t)(i & 1) * nb * kPerNd;
    if ((int)threadIdx.x < nwp) s_off[threadIdx.x] = (size_t)((iprev - nwp + (int)threadIdx.x) % slots) * (size_t)N;
    __syncthreads();
    const size_t coff = (size_t)(iprev % slots) * (size_t)N;

    double sc[4] = {0.0, 0.0, 0.0, 0.0};   // gamma_i, delta_i, ||r_i||^2, <u_i, s_{i-1}>
    double acc[NWQ];
#pragma unroll
    for (int s = 0; s < NWQ; ++s) acc[s] = 0.0;

    // ---- pass: MAXPYs of iteration i-1, advance, Jacobi, dot partials ----
    for (int c = blockIdx.x; c < a.nchunks; c += nb) {
      const int64_t e = (int64_t)c * kPerRows + rowi;
      const bool valid = e < N;
      double sp = 0.0, ss = 0.0, sq = 0.0, sz = 0.0;
      double skv[NWQ];
#pragma unroll
      for (int s = 0; s < NWQ; ++s) {
        const int j = 4 * s + q;
        skv[s] = 0.0;
        if (valid && j < nwp) {
          const size_t o = s_off[j] + e;
          const double b = st.beta[j];
          const double sv = __ldcg(&a.S[o]);
          sp = fma(b, __ldcg(&a.P[o]), sp);
          ss = fma(b, sv, ss);
          sq = fma(b, __ldcg(&a.Q[o]), sq);
          sz = fma(b, __ldcg(&a.Z[o]), sz);
          skv[s] = sv;
        }
      }
      sp += __shfl_xor_sync(0xffffffffu, sp, 1);
      ss += __shfl_xor_sync(0xffffffffu, ss, 1);
      sq += __shfl_xor_sync(0xffffffffu, sq, 1);
      sz += __shfl_xor_sync(0xffffffffu, sz, 1);
      sp += __shfl_xor_sync(0xffffffffu, sp, 2);
      ss += __shfl_xor_sync(0xffffffffu, ss, 2);
      sq += __shfl_xor_sync(0xffffffffu, sq, 2);
      sz += __shfl_xor_sync(0xffffffffu, sz, 2);
      if (valid) {
        const double u0 = __ldcg(&a.u[e]), w0 = __ldcg(&a.w[e]);
        const double p = u0 + sp, s = w0 + ss, qv = __ldcg(&mprev[e]) + sq, z = __ldcg(&a.n[e]) + sz;
        const double xn = fma(alpha, p, __ldcg(&a.x[e]));
        const double rn = fma(-alpha, s, __ldcg(&a.r[e]));
        const double un = fma(-alpha, qv, u0);
        const double wn = fma(-alpha, z, w0);
        const double t = wn - rn;                            // B's input w_i - r_i (eq. BwMinusR)
        const double y = a.dinv ? __dmul_rn(__ldcg(&a.dinv[e]), t) : t;
        if (q == 0) {
          a.P[coff + e] = p;
          a.S[coff + e] = s;
          a.Q[coff + e] = qv;
          a.Z[coff + e] = z;
          a.x[e] = xn;
          a.r[e] = rn;
          a.u[e] = un;
          a.w[e] = wn;
          mnew[e] = __dadd_rn(un, y);                        // m_i = u_i + B(w_i - r_i)
          sc[0] = fma(un, rn, sc[0]);
          sc[1] = fma(un, wn, sc[1]);
          sc[2] = fma(rn, rn, sc[2]);
          sc[3] = fma(un, s, sc[3]);
        }
#pragma unroll
        for (int s2 = 0; s2 < NWQ; ++s2) acc[s2] = fma(un, skv[s2], acc[s2]);
      }
    }
    write_pipefcg_row<NWQ>(sc, acc, nwp, s_red, part + (size_t)blockIdx.x * kPerNd);

    if (!grid_barrier(ctl)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->status = kTimeout;
      return;
    }

    // ---- the pass's partial rows in flight while n_i = A m_i (own rows) is
    // formed, then their combine ----
    fetch_partials(part, nb, s_part);
    for (int c = blockIdx.x; c < a.nchunks; c += nb) {
      const int64_t e = (int64_t)c * kPerRows + rowi;
      if (e < N && q == 0) a.n[e] = csr_row(a, mnew, e);
    }
    wait_partials();
    sum_partials(s_part, nb, 4 + nwp, st.sums);

    // ---- scalar phase of iteration i (Alg. 8), the same in every block ----
    const int nu = nu_window(i, a.mmax, ctl->truncation);
    if (threadIdx.x == 0) {
      const double gamma = st.sums[0], delta = st.sums[1], rr = st.sums[2];
      st.it += 1;
      st.i = i;
      st.gamma = gamma;
      st.delta = delta;
      const double rho = ctl->norm == PFK_NORM_NATURAL ? sqrt(fabs(gamma)) : sqrt(rr);
      st.rho = rho;
      per_push_history(&st, ctl, rho, sqrt(rr), nan(""), nan(""));
      st.go = 1;
      if (!isfinite(rho)) { st.status = kNonFinite; st.go = 0; }
      else if (rho <= ctl->target) { st.status = kConverged; st.go = 0; }
    }
    // window dots in order k = i-1-nwp .. i-1 (W_{i-1}, then s_{i-1}); W_i is the last nu
    if ((int)threadIdx.x <= nwp) st.cw[threadIdx.x] = (int)threadIdx.x < nwp ? st.sums[4 + threadIdx.x] : st.sums[3];
    __syncthreads();
    if (st.go) {
      const double* cwin = st.cw + (nwp + 1 - nu);
      if ((int)threadIdx.x < nu) {
        const int k = i - nu + (int)threadIdx.x;
        const double ek = st.eta_ring[k % slots];
        const double bb = -cwin[threadIdx.x] / ek;
        st.tmp[threadIdx.x] = bb;
        st.tmp[PFK_MAX_MMAX + 1 + threadIdx.x] = ek;
      }
      __syncthreads();
      if ((int)threadIdx.x < nu) st.beta[threadIdx.x] = st.tmp[threadIdx.x];
      if (threadIdx.x == 0) {
        double sumb = 0.0;
        for (int jj = 0; jj < nu; ++jj) {
          const double bb = st.tmp[jj];
          sumb = fma(bb * bb, st.tmp[PFK_MAX_MMAX + 1 + jj], sumb);
        }
        const double eta = st.delta - sumb;
        const double al = eta != 0.0 ? st.gamma / eta : nan("");
        st.eta = eta;
        st.alpha = al;
        st.nw = nu;
        st.eta_ring[i % slots] = eta;
        if (blockIdx.x == 0 && ctl->history && st.hist_len - 1 < ctl->hist_cap) {
          ctl->history[(size_t)(st.hist_len - 1) * PFK_HISTORY_FIELDS + 2] = eta;
          ctl->history[(size_t)(st.hist_len - 1) * PFK_HISTORY_FIELDS + 3] = al;
        }
        if (eta <= 0.0) st.status = kBreakdown;
        else if (st.it >= ctl->maxit) st.status = kMaxit;
      }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->passes += 1;
      // pass words per row: u, w, m, n, x, r, D^-1 and 4 nu history read; p, s,
      // q, z, x, r, u, w, m written.  FP64 flops: 4 nu MAXPY, 4 advance and
      // nu + 4 dot FMAs, the Jacobi product and two additions.
      ctl->alg_bytes += 8.0 * (double)N * (double)(4 * nwp + 16);
      ctl->alg_flops += (double)N * (2.0 * (5 * nwp + 8) + 3.0);
    }
    store_state(&st, ctl, st.go ? nu : 0);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// FCG
// ---------------------------------------------------------------------------

template <int NW>
__global__ void __launch_bounds__(kPerThreads) fcg_persistent(PersistArgs a) {
  constexpr int NWQ = NW / 4;
  extern __shared__ double s_part[];     // the grid's partial rows, nb * kPerNd
  __shared__ PerState st;
  __shared__ double s_red[(kPerThreads / 32) * kPerNd];
  __shared__ size_t s_off[NW];
  SolveCtl* ctl = a.ctl;
  load_state(&st, ctl);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = lane & 3;
  const int rowi = threadIdx.x >> 2;
  const int slots = a.mmax + 1;
  const int64_t N = a.N;
  const int nb = gridDim.x;
  double* red1 = a.partials;                             // [nb][kPerNd]: gamma, ||r||^2, -, -, window dots
  double* red3 = a.partials + (size_t)nb * kPerNd;       // [nb][kPerNd]: eta

  for (int g = 0; g < a.iters; ++g) {
    if (st.status != kRun) break;
    const int iprev = st.i, i = iprev + 1;
    const double alpha = st.alpha;
    const int nu = nu_window(i, a.mmax, ctl->truncation);
    if ((int)threadIdx.x < nu) s_off[threadIdx.x] = (size_t)((i - nu + (int)threadIdx.x) % slots) * (size_t)N;
    __syncthreads();
    const size_t poff = (size_t)(iprev % slots) * (size_t)N;

    // ---- x_i, r_i, u_i = B(r_i) (Jacobi), gamma_i, ||r_i||^2, <u_i, s_k> ----
    double sc[4] = {0.0, 0.0, 0.0, 0.0};
    double acc[NWQ];
#pragma unroll
    for (int s = 0; s < NWQ; ++s) acc[s] = 0.0;
    for (int c = blockIdx.x; c < a.nchunks; c += nb) {
      const int64_t e = (int64_t)c * kPerRows + rowi;
      if (e >= N) continue;
      const double xn = fma(alpha, __ldcg(&a.P[poff + e]), __ldcg(&a.x[e]));
      const double rn = fma(-alpha, __ldcg(&a.S[poff + e]), __ldcg(&a.r[e]));
      const double un = a.dinv ? __ldcg(&a.dinv[e]) * rn : rn;
      if (q == 0) {
        a.x[e] = xn;
        a.r[e] = rn;
        a.u[e] = un;
        sc[0] = fma(un, rn, sc[0]);
        sc[1] = fma(rn, rn, sc[1]);
      }
#pragma unroll
      for (int s = 0; s < NWQ; ++s) {
        const int j = 4 * s + q;
        if (j < nu) acc[s] = fma(un, __ldcg(&a.S[s_off[j] + e]), acc[s]);
      }
    }
    write_pipefcg_row<NWQ>(sc, acc, nu, s_red, red1 + (size_t)blockIdx.x * kPerNd);
    if (!grid_barrier(ctl)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->status = kTimeout;
      return;
    }
    fetch_partials(red1, nb, s_part);
    wait_partials();
    sum_partials(s_part, nb, 4 + nu, st.sums);
    // Alg. 2: gamma_i, convergence, beta_{i,k} = -<u_i, s_k> / eta_k
    if (threadIdx.x == 0) {
      const double gamma = st.sums[0], rr = st.sums[1];
      st.it += 1;
      st.gamma = gamma;
      const double rho = ctl->norm == PFK_NORM_NATURAL ? sqrt(fabs(gamma)) : sqrt(rr);
      st.rho = rho;
      per_push_history(&st, ctl, rho, sqrt(rr), nan(""), nan(""));
      st.go = 1;
      if (!isfinite(rho)) { st.status = kNonFinite; st.go = 0; }
      else if (rho <= ctl->target) { st.status = kConverged; st.i = i; st.go = 0; }
    }
    __syncthreads();
    if (!st.go) {
      store_state(&st, ctl, 0);
      break;
    }
    if ((int)threadIdx.x < nu) st.beta[threadIdx.x] = -st.sums[4 + threadIdx.x] / st.eta_ring[(i - nu + (int)threadIdx.x) % slots];
    __syncthreads();

    // ---- p_i = u_i + sum beta_{i,k} p_k into ring slot i ----
    const size_t ioff = (size_t)(i % slots) * (size_t)N;
    for (int c = blockIdx.x; c < a.nchunks; c += nb) {
      const int64_t e = (int64_t)c * kPerRows + rowi;
      const bool valid = e < N;
      double sp = 0.0;
#pragma unroll
      for (int s = 0; s < NWQ; ++s) {
        const int j = 4 * s + q;
        if (valid && j < nu) sp = fma(st.beta[j], __ldcg(&a.P[s_off[j] + e]), sp);
      }
      sp += __shfl_xor_sync(0xffffffffu, sp, 1);
      sp += __shfl_xor_sync(0xffffffffu, sp, 2);
      if (valid && q == 0) a.P[ioff + e] = __ldcg(&a.u[e]) + sp;
    }
    if (!grid_barrier(ctl)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->status = kTimeout;
      return;
    }

    // ---- s_i = A p_i, eta_i = <p_i, s_i> ----
    double ps = 0.0;
    for (int c = blockIdx.x; c < a.nchunks; c += nb) {
      const int64_t e = (int64_t)c * kPerRows + rowi;
      if (e < N && q == 0) {
        const double sv = csr_row(a, a.P + ioff, e);
        a.S[ioff + e] = sv;
        ps = fma(__ldcg(&a.P[ioff + e]), sv, ps);
      }
    }
    {
      const double v = warp_sum(ps);
      if (lane == 0) s_red[warp] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kPerThreads / 32; ++w) t += s_red[w];
        red3[(size_t)blockIdx.x * kPerNd] = t;
      }
    }
    if (!grid_barrier(ctl)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->status = kTimeout;
      return;
    }
    fetch_partials(red3, nb, s_part);
    wait_partials();
    sum_partials(s_part, nb, 1, st.sums);
    if (threadIdx.x == 0) {
      // Alg. 2: eta_i = <p_i, s_i>, alpha_i = gamma_i / eta_i
      const double eta = st.sums[0];
      const double al = eta != 0.0 ? st.gamma / eta : nan("");
      st.i = i;
      st.eta = eta;
      st.alpha = al;
      st.nw = nu;
      st.eta_ring[i % slots] = eta;
      if (blockIdx.x == 0 && ctl->history && st.hist_len - 1 < ctl->hist_cap && st.hist_len >= 1) {
        ctl->history[(size_t)(st.hist_len - 1) * PFK_HISTORY_FIELDS + 2] = eta;
        ctl->history[(size_t)(st.hist_len - 1) * PFK_HISTORY_FIELDS + 3] = al;
      }
      if (eta <= 0.0) st.status = kBreakdown;
      else if (st.it >= ctl->maxit) st.status = kMaxit;
    }
    __syncthreads();
    store_state(&st, ctl, nu);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int persistent_template(int mmax) { return mmax <= 4 ? 4 : mmax <= 8 ? 8 : mmax <= 16 ? 16 : 32; }

// Blocks of the persistent launch: one per 32-row chunk up to one per SM (the
// grid must be co-resident for the barriers; one block per SM keeps every
// SM's FP64 units in use and the barrier short).
int persistent_blocks(const pfk_context* ctx, int64_t N) {
  const int64_t chunks = (N + kPerRows - 1) / kPerRows;
  const int64_t cap = ctx->num_sms < kMaxPerBlocks ? ctx->num_sms : kMaxPerBlocks;
  return (int)(chunks < cap ? chunks : cap);
}

bool persistent_eligible(const pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, int method, int naive_like,
                         int64_t N) {
  if (naive_like) return false;
  if (method != PFK_PIPEFCG && method != PFK_FCG) return false;
  if (!op->rowptr) return false;
  if (pc && pc->kind != PFK_PC_NONE && pc->kind != PFK_PC_JACOBI) return false;
  if (pc && pc->kind == PFK_PC_JACOBI && !op->csr_dinv && !op->dinv) return false;
  return N >= 1 && N <= PFK_PERSISTENT_MAX_N && persistent_blocks(ctx, N) >= 1;
}

int64_t persistent_partials(const pfk_context* ctx, int64_t N) {
  return 2 * (int64_t)persistent_blocks(ctx, N) * kPerNd;
}

template <int NW>
static cudaError_t launch_one(bool pipelined, const PersistArgs& a, int blocks, cudaStream_t st) {
  void* fn = pipelined ? (void*)pipefcg_persistent<NW> : (void*)fcg_persistent<NW>;
  const int smem = blocks * kPerNd * (int)sizeof(double);
  cudaError_t e = pipelined ? cudaFuncSetAttribute(pipefcg_persistent<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                            : cudaFuncSetAttribute(fcg_persistent<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kPerThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PersistArgs args = a;
  void* params[] = {&args};
  return cudaLaunchKernelExC(&cfg, fn, params);
}

cudaError_t launch_persistent(const SolveEnv& env, bool pipelined, int mmax, double* x, double* r, double* u,
                              double* w, double* m0, double* m1, double* n, double* P, double* S, double* Q,
                              double* Z, int iters) {
  const pfk_operator* op = env.op;
  PersistArgs a;
  a.rowptr = op->rowptr;
  a.colidx = op->colidx;
  a.vals = op->vals;
  // the D^-1 the Jacobi preconditioner applies (pc_apply's choice)
  a.dinv = (env.pc && env.pc->kind == PFK_PC_JACOBI) ? (op->csr_dinv ? op->csr_dinv : op->dinv) : nullptr;
  a.N = env.N;
  a.mmax = mmax;
  a.iters = iters;
  a.nchunks = (int)((env.N + kPerRows - 1) / kPerRows);
  a.x = x; a.r = r; a.u = u; a.w = w; a.m0 = m0; a.m1 = m1; a.n = n;
  a.P = P; a.S = S; a.Q = Q; a.Z = Z;
  a.ctl = env.ctl;
  // partial rows start on a 16-byte boundary (asynchronous 16-byte copies)
  const size_t mis = ((uintptr_t)env.partials & 15u) / sizeof(double);
  a.partials = env.partials + (mis ? 2 - mis : 0);
  const int blocks = persistent_blocks(env.ctx, env.N);
  if (!env.partials_fit(2 * blocks + 1, kPerNd)) return cudaErrorInvalidValue;
  switch (persistent_template(mmax)) {
    case 4: return launch_one<4>(pipelined, a, blocks, env.st);
    case 8: return launch_one<8>(pipelined, a, blocks, env.st);
    case 16: return launch_one<16>(pipelined, a, blocks, env.st);
    default: return launch_one<32>(pipelined, a, blocks, env.st);
  }
}

}  // namespace pfk
