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
// every run is bitwise reproducible.  A block's rows of every vector and ring
// slot, and its CSR rows, stay in shared memory for the whole launch (loaded
// at the start, written back at the end); within a launch only m_i / p_i
// (read by other blocks' operator rows) and the partial rows go through
// global memory, the partial rows fetched with asynchronous 16-byte copies.
// On this GPU an FP64 instruction costs its sub-partition tens of
// nanoseconds whatever its active lanes, so the reductions and the scalar
// phase are arranged to keep such instructions few and off one warp's chain.
// Block 0 keeps the control block up to date (status, counters, history) for
// the host driver.
#include "pfk_internal.cuh"
#include "solver.cuh"

#include <cmath>

namespace pfk {

constexpr int kPerThreads = 128;
constexpr int kPerRows = 32;                // rows of a chunk (4 threads per row)
constexpr int kPerNd = PFK_MAX_MMAX + 4;    // largest partial row (gamma, delta, ||r||^2, c_{i-1}, window)
constexpr int kMaxPerBlocks = 192;          // grid cap (the fetched partial rows take nb x 288 bytes)
constexpr int kPerSmemLimit = 220 * 1024;   // dynamic shared memory of one block (of 227 KB)

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

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void red_add_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier of a cooperative launch (all blocks resident).  Arrival on a
// counter (acquire-release: the block's writes, ordered before thread 0 by the
// block barrier, are released; the last arrival acquires everyone's); the last
// arrival resets the counter and bumps the generation with a release, the
// others wait for it with acquire loads.  The wait is bounded (the control
// block's bar_timeout_ns, 2 s by default): on time-out the block raises
// bar_abort, and a raised bar_abort ends every other wait.
// Returns false in that case.
__device__ __forceinline__ bool grid_barrier(SolveCtl* ctl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire(&ctl->bar_gen);
    int ok = 1;
    if (atom_add_acq_rel(&ctl->bar_count, 1u) == gridDim.x - 1) {
      ctl->bar_count = 0u;
      red_add_release(&ctl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      const long long budget = ctl->bar_timeout_ns;
      while (ld_acquire(&ctl->bar_gen) == g) {
        if (ld_acquire(&ctl->bar_abort)) { ok = 0; break; }
        if (budget <= 0 || global_ns() - t0 > (unsigned long long)budget) {
          atomicExch(&ctl->bar_abort, 1u);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum of a value over the eight rows a warp holds, for the thread position q
// of a row: lanes q, q + 4, ..., q + 28 (a fixed shuffle tree; every lane gets
// the sum of its own q).  Call with all 32 lanes.
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
// order into out[j] (shared memory).  Each FP64 instruction costs a
// sub-partition tens of nanoseconds whatever its lane count, so the work is
// spread over (column, row group) tasks that keep all lanes busy: task t of
// the block sums rows g, g + G, g + 2G, ... of column j (t = g * nd + j, G =
// the groups that fit in the block's threads, at most 4), then thread j adds
// the G group sums in group order.  Every block gets bitwise the same sums.
__device__ __forceinline__ void sum_partials(const double* s_part, int nb, int nd, double* out, double* s_grp) {
  int G = kPerThreads / nd;
  G = G < 1 ? 1 : (G > 4 ? 4 : G);
  for (int t = threadIdx.x; t < G * nd; t += kPerThreads) {
    const int g = t / nd, j = t - g * nd;
    double a = 0.0;
    for (int b = g; b < nb; b += G) a += s_part[b * kPerNd + j];
    s_grp[t] = a;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nd; j += kPerThreads) {
    double a = s_grp[j];
    for (int g = 1; g < G; ++g) a += s_grp[g * nd + j];
    out[j] = a;
  }
  __syncthreads();
}

// Writes this block's partial row: column j of the block = sum over its
// threads' values.  Thread q of a row holds scalar column q in scq (its own
// product, computed from the row's values every thread of the row has) and
// window columns 4 s + q in acc[s].  Layout: [scalar 0..3, window 0 .. nw-1].
// Each column is summed over the warp's rows by three shuffle steps (lanes of
// equal q), then over the four warps in order.
template <int NWQ>
__device__ __forceinline__ void write_pipefcg_row(double scq, const double (&acc)[NWQ], int nw, double* s_red,
                                                  double* row) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = lane & 3;
  {
    const double v = quad_col_sum(scq);
    if (lane < 4) s_red[warp * kPerNd + q] = v;
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
  int truncation, norm, maxit, hist_cap;   // copies of the control block's constants
  double target;
  double* history;
  int passes;                              // work counters of this launch (block 0 adds them at the end)
  double alg_bytes, alg_flops;
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
    st->truncation = ctl->truncation;
    st->norm = ctl->norm;
    st->maxit = ctl->maxit;
    st->hist_cap = ctl->hist_cap;
    st->target = ctl->target;
    st->history = ctl->history;
    st->passes = 0;
    st->alg_bytes = 0.0;
    st->alg_flops = 0.0;
  }
  for (int j = threadIdx.x; j < PFK_MAX_MMAX; j += blockDim.x) st->beta[j] = ctl->beta[j];
  for (int j = threadIdx.x; j <= PFK_MAX_MMAX; j += blockDim.x) st->eta_ring[j] = ctl->eta_ring[j];
  __syncthreads();
}

// History entry of block 0 (the others only keep the count).
__device__ __forceinline__ void per_push_history(PerState* st, SolveCtl* ctl, double rho, double rn, double eta,
                                                 double alpha) {
  if (blockIdx.x == 0 && st->history && st->hist_len < st->hist_cap) {
    double* h = st->history + (size_t)st->hist_len * PFK_HISTORY_FIELDS;
    h[0] = rho; h[1] = rn; h[2] = eta; h[3] = alpha;
  }
  st->hist_len += 1;
}

// Block 0 copies the state back to the control block (after each iteration).
__device__ __forceinline__ void store_state(const PerState* st, SolveCtl* ctl, int nbeta, int slots) {
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
    ctl->eta_ring[st->i % slots] = st->eta_ring[st->i % slots];
  }
}

// Block 0 adds the launch's work counters to the control block (at exit).
__device__ __forceinline__ void store_counters(const PerState* st, SolveCtl* ctl) {
  if (blockIdx.x != 0 || threadIdx.x != 0 || st->passes == 0) return;
  ctl->passes += st->passes;
  ctl->alg_bytes += st->alg_bytes;
  ctl->alg_flops += st->alg_flops;
}

// ---------------------------------------------------------------------------
// Rows resident in shared memory
// ---------------------------------------------------------------------------

// The block's rows of every vector it owns stay in shared memory for the whole
// launch (loaded at the start, written back at the end): block b owns the
// 32-row chunks b, b + nb, ...; local row l = (local chunk) * 32 + row in
// chunk.  Vector v sits at base[v * pitch + l], ring g slot k at
// base[(nvec + g * slots + k) * pitch + l]; pitch = rows + 1 keeps the four
// threads of a row (which read four different slots) on different banks.
// Only what other blocks read goes through global memory within a launch:
// m_i (PIPEFCG) or p_i (FCG) for the operator rows, and the partial sums.
struct Resident {
  double* base;
  int rows, pitch, nvec, slots;
  __device__ __forceinline__ double* vec(int v) const { return base + (size_t)v * pitch; }
  __device__ __forceinline__ double* ring(int g, int k) const { return base + (size_t)(nvec + g * slots + k) * pitch; }
};

// Global index of local row l (or -1 past the end).
__device__ __forceinline__ int64_t own_row(int l, int nb, int64_t N) {
  const int64_t c = (int64_t)blockIdx.x + (int64_t)(l / kPerRows) * nb;
  const int64_t e = c * kPerRows + (l % kPerRows);
  return e < N ? e : -1;
}

// Copies the block's rows between global vectors (gv[v], rings gr[g] of
// `slots` slots of length N) and the resident copy; to_smem selects the
// direction.  Vectors given as null are skipped (zero in shared memory).
__device__ __forceinline__ void resident_copy(const Resident& R, double* const* gv, double* const* gr, int nrings,
                                              int nb, int64_t N, bool to_smem) {
  for (int l = threadIdx.x; l < R.rows; l += blockDim.x) {
    const int64_t e = own_row(l, nb, N);
    for (int v = 0; v < R.nvec; ++v) {
      double* s = R.vec(v) + l;
      if (to_smem) *s = (e >= 0 && gv[v]) ? __ldcg(&gv[v][e]) : 0.0;
      else if (e >= 0 && gv[v]) gv[v][e] = *s;
    }
    for (int g = 0; g < nrings; ++g)
      for (int k = 0; k < R.slots; ++k) {
        double* s = R.ring(g, k) + l;
        double* gp = gr[g] + (size_t)k * (size_t)N;
        if (to_smem) *s = e >= 0 ? __ldcg(&gp[e]) : 0.0;
        else if (e >= 0) gp[e] = *s;
      }
  }
  __syncthreads();
}

// The CSR rows of the block's chunks, staged in shared memory when they fit
// (rowptr relative to the chunk's first entry, column indices, values), so the
// operator rows cost one round of loads (the input values) per iteration.
struct CsrStage {
  int* rp;        // [chunks][kPerRows + 1]
  int* ci;
  double* va;
  int cap;        // entries available
  int staged;     // 1 if every chunk fits
};

__device__ __forceinline__ void stage_csr(const PersistArgs& a, CsrStage& cs, int cpb, int nb) {
  __shared__ int s_fit;
  if (threadIdx.x == 0) {
    int total = 0;
    for (int lc = 0; lc < cpb; ++lc) {
      const int64_t c = (int64_t)blockIdx.x + (int64_t)lc * nb;
      if (c * kPerRows >= a.N) break;
      const int64_t e0 = c * kPerRows, e1 = min(e0 + kPerRows, a.N);
      total += a.rowptr[e1] - a.rowptr[e0];
    }
    s_fit = total <= cs.cap ? 1 : 0;
  }
  __syncthreads();
  cs.staged = s_fit;
  if (!cs.staged) return;
  int off = 0;
  for (int lc = 0; lc < cpb; ++lc) {
    const int64_t c = (int64_t)blockIdx.x + (int64_t)lc * nb;
    int* rp = cs.rp + lc * (kPerRows + 1);
    if (c * kPerRows >= a.N) {
      for (int t = threadIdx.x; t <= kPerRows; t += blockDim.x) rp[t] = off;
      continue;
    }
    const int64_t e0 = c * kPerRows, e1 = min(e0 + kPerRows, a.N);
    const int32_t base = a.rowptr[e0];
    for (int t = threadIdx.x; t <= kPerRows; t += blockDim.x) {
      const int64_t e = min(e0 + t, e1);
      rp[t] = off + (a.rowptr[e] - base);
    }
    const int cnt = a.rowptr[e1] - base;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      cs.ci[off + t] = a.colidx[base + t];
      cs.va[off + t] = a.vals[base + t];
    }
    off += cnt;
  }
  __syncthreads();
}

// (A m)_e for global row e = local row l: entries in column order, fused
// multiply-adds from zero (the same arithmetic as the CSR operator kernel).
__device__ __forceinline__ double csr_row(const PersistArgs& a, const CsrStage& cs, const double* m, int64_t e,
                                          int l) {
  double acc = 0.0;
  if (cs.staged) {
    const int* rp = cs.rp + (l / kPerRows) * (kPerRows + 1) + (l % kPerRows);
    for (int p = rp[0]; p < rp[1]; ++p) acc = fma(cs.va[p], __ldcg(&m[cs.ci[p]]), acc);
  } else {
    const int32_t end = a.rowptr[e + 1];
    for (int32_t p = a.rowptr[e]; p < end; ++p) acc = fma(a.vals[p], __ldcg(&m[a.colidx[p]]), acc);
  }
  return acc;
}

// Dynamic shared memory of a launch: resident rows, staged CSR, partial rows.
struct PerLayout {
  int cpb, rows, pitch, nvec, nrings, slots, csr_cap;
  size_t resident_doubles, csr_bytes, part_doubles;
  __host__ __device__ size_t bytes() const {
    return resident_doubles * sizeof(double) + part_doubles * sizeof(double) + csr_bytes;
  }
};

__host__ __device__ __forceinline__ PerLayout per_layout(int64_t N, int nb, int slots, bool pipelined) {
  PerLayout L;
  const int64_t nchunks = (N + kPerRows - 1) / kPerRows;
  L.cpb = (int)((nchunks + nb - 1) / nb);
  L.rows = L.cpb * kPerRows;
  L.pitch = L.rows + 1;
  L.nvec = pipelined ? 7 : 4;          // x, r, u, w, m, n, D^-1  |  x, r, u, D^-1
  L.nrings = pipelined ? 4 : 2;        // P, S, Q, Z              |  P, S
  L.slots = slots;
  L.resident_doubles = (size_t)(L.nvec + L.nrings * slots) * L.pitch;
  L.part_doubles = (size_t)nb * kPerNd;
  L.csr_cap = L.rows * 8;              // staged entries (a 5- or 7-point row fits)
  L.csr_bytes = ((size_t)L.cpb * (kPerRows + 1) * sizeof(int) + 15) / 16 * 16 +
                ((size_t)L.csr_cap * (sizeof(int) + sizeof(double)) + 15) / 16 * 16;
  return L;
}

// ---------------------------------------------------------------------------
// PIPEFCG
// ---------------------------------------------------------------------------

template <int NW>
__global__ void __launch_bounds__(kPerThreads) pipefcg_persistent(PersistArgs a) {
  constexpr int NWQ = NW / 4;
  extern __shared__ __align__(16) double s_dyn[];
  __shared__ PerState st;
  __shared__ double s_red[(kPerThreads / 32) * kPerNd];
  SolveCtl* ctl = a.ctl;
  const int q = threadIdx.x & 3;
  const int rowi = threadIdx.x >> 2;
  const int slots = a.mmax + 1;
  const int64_t N = a.N;
  const int nb = gridDim.x;
  const PerLayout L = per_layout(N, nb, slots, true);
  double* s_part = s_dyn;                                          // nb * kPerNd
  const Resident R{s_dyn + L.part_doubles, L.rows, L.pitch, L.nvec, slots};
  CsrStage cs;
  {
    char* cb = (char*)(s_dyn + L.part_doubles + L.resident_doubles);
    cs.rp = (int*)cb;
    cs.va = (double*)(cb + (((size_t)L.cpb * (kPerRows + 1) * sizeof(int) + 15) / 16 * 16));
    cs.ci = (int*)(cs.va + L.csr_cap);
    cs.cap = L.csr_cap;
  }
  load_state(&st, ctl);
  if (st.status != kRun) return;   // a launch queued behind the one that finished
  {
    double* gm = (st.i & 1) ? a.m1 : a.m0;
    double* gv[7] = {a.x, a.r, a.u, a.w, gm, a.n, const_cast<double*>(a.dinv)};
    double* gr[4] = {a.P, a.S, a.Q, a.Z};
    resident_copy(R, gv, gr, 4, nb, N, true);
  }
  stage_csr(a, cs, L.cpb, nb);
  double* sx = R.vec(0);
  double* sr = R.vec(1);
  double* su = R.vec(2);
  double* sw = R.vec(3);
  double* sm = R.vec(4);
  double* sn = R.vec(5);
  const double* sd = R.vec(6);
  const bool jacobi = a.dinv != nullptr;

  for (int g = 0; g < a.iters; ++g) {
    if (st.status != kRun) break;
    const int iprev = st.i, i = iprev + 1;
    const int nwp = st.nw;
    const double alpha = st.alpha;
    double* mnew = (i & 1) ? a.m1 : a.m0;
    double* part = a.partials + (size_t)(i & 1) * nb * kPerNd;
    const int cslot = iprev % slots;

    double scq = 0.0;   // thread q of a row: gamma_i, delta_i, ||r_i||^2, <u_i, s_{i-1}> for q = 0..3
    double acc[NWQ];
#pragma unroll
    for (int s = 0; s < NWQ; ++s) acc[s] = 0.0;

    // ---- pass: MAXPYs of iteration i-1, advance, Jacobi, dot partials ----
    for (int lc = 0; lc < L.cpb; ++lc) {
      const int l = lc * kPerRows + rowi;
      const int64_t e = own_row(l, nb, N);
      const bool valid = e >= 0;
      double sp = 0.0, ss = 0.0, sq = 0.0, sz = 0.0;
      double skv[NWQ];
#pragma unroll
      for (int s = 0; s < NWQ; ++s) {
        const int j = 4 * s + q;
        skv[s] = 0.0;
        if (valid && j < nwp) {
          const int k = (iprev - nwp + j) % slots;
          const double b = st.beta[j];
          const double sv = R.ring(1, k)[l];
          sp = fma(b, R.ring(0, k)[l], sp);
          ss = fma(b, sv, ss);
          sq = fma(b, R.ring(2, k)[l], sq);
          sz = fma(b, R.ring(3, k)[l], sz);
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
      double un = 0.0, p = 0.0, s = 0.0, qv = 0.0, z = 0.0, xn = 0.0, rn = 0.0, wn = 0.0, mn = 0.0;
      if (valid) {
        const double u0 = su[l], w0 = sw[l];
        p = u0 + sp;
        s = w0 + ss;
        qv = sm[l] + sq;
        z = sn[l] + sz;
        xn = fma(alpha, p, sx[l]);
        rn = fma(-alpha, s, sr[l]);
        un = fma(-alpha, qv, u0);
        wn = fma(-alpha, z, w0);
        const double t = wn - rn;                            // B's input w_i - r_i (eq. BwMinusR)
        const double y = jacobi ? __dmul_rn(sd[l], t) : t;
        mn = __dadd_rn(un, y);                               // m_i = u_i + B(w_i - r_i)
        const double lf = q == 2 ? rn : un, rt = q == 0 ? rn : q == 1 ? wn : q == 2 ? rn : s;
        scq = fma(lf, rt, scq);
      }
      __syncwarp();   // every lane of the row has read the old values before thread 0 of the row writes
      if (valid && q == 0) {
        R.ring(0, cslot)[l] = p;
        R.ring(1, cslot)[l] = s;
        R.ring(2, cslot)[l] = qv;
        R.ring(3, cslot)[l] = z;
        sx[l] = xn;
        sr[l] = rn;
        su[l] = un;
        sw[l] = wn;
        sm[l] = mn;
        mnew[e] = mn;
      }
#pragma unroll
      for (int s2 = 0; s2 < NWQ; ++s2) acc[s2] = fma(un, skv[s2], acc[s2]);
    }
    write_pipefcg_row<NWQ>(scq, acc, nwp, s_red, part + (size_t)blockIdx.x * kPerNd);

    if (!grid_barrier(ctl)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->status = kTimeout;
      return;
    }

    // ---- the pass's partial rows in flight while n_i = A m_i (own rows) is
    // formed, then their combine ----
    fetch_partials(part, nb, s_part);
    for (int lc = 0; lc < L.cpb; ++lc) {
      const int l = lc * kPerRows + rowi;
      const int64_t e = own_row(l, nb, N);
      if (e >= 0 && q == 0) sn[l] = csr_row(a, cs, mnew, e, l);
    }
    wait_partials();
    sum_partials(s_part, nb, 4 + nwp, st.sums, s_red);

    // ---- scalar phase of iteration i (Alg. 8), the same in every block ----
    // Warp 1 (thread 32) forms rho_i and the convergence verdict and writes the
    // history while warp 0 forms the betas, eta_i and alpha_i (used only when
    // the iteration goes on): the two chains run on different sub-partitions.
    const int nu = nu_window(i, a.mmax, st.truncation);
    if (threadIdx.x == 32) {
      const double gamma = st.sums[0], rr = st.sums[2];
      const double rho = st.norm == PFK_NORM_NATURAL ? sqrt(fabs(gamma)) : sqrt(rr);
      st.rho = rho;
      per_push_history(&st, ctl, rho, st.history ? sqrt(rr) : nan(""), nan(""), nan(""));
      st.go = !isfinite(rho) ? -1 : (rho <= st.target ? 0 : 1);
    }
    if (threadIdx.x < 32) {
      // window dots in order k = i-1-nwp .. i-1 (W_{i-1}, then s_{i-1}); W_i is the last nu
      const int jj = (int)threadIdx.x;
      double term = 0.0;
      if (jj < nu) {
        const int c = nwp + 1 - nu + jj;
        const double cv = c < nwp ? st.sums[4 + c] : st.sums[3];
        const double ek = st.eta_ring[(i - nu + jj) % slots];
        const double bb = -cv / ek;
        st.beta[jj] = bb;
        term = (bb * bb) * ek;
      }
      // sum of beta^2 eta over the window: a fixed shuffle tree
      term = warp_sum(term);
      if (jj == 0) {
        const double eta = st.sums[1] - term;
        st.eta = eta;
        st.alpha = eta != 0.0 ? st.sums[0] / eta : nan("");
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      st.it += 1;
      st.i = i;
      st.gamma = st.sums[0];
      st.delta = st.sums[1];
      if (st.go < 0) { st.status = kNonFinite; st.go = 0; }
      else if (st.go == 0) st.status = kConverged;
      else {
        st.nw = nu;
        st.eta_ring[i % slots] = st.eta;
        if (blockIdx.x == 0 && st.history && st.hist_len - 1 < st.hist_cap) {
          st.history[(size_t)(st.hist_len - 1) * PFK_HISTORY_FIELDS + 2] = st.eta;
          st.history[(size_t)(st.hist_len - 1) * PFK_HISTORY_FIELDS + 3] = st.alpha;
        }
        if (st.eta <= 0.0) st.status = kBreakdown;
        else if (st.it >= st.maxit) st.status = kMaxit;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      st.passes += 1;
      // pass words per row: u, w, m, n, x, r, D^-1 and 4 nu history read; p, s,
      // q, z, x, r, u, w, m written.  FP64 flops: 4 nu MAXPY, 4 advance and
      // nu + 4 dot FMAs, the Jacobi product and two additions.
      st.alg_bytes += 8.0 * (double)N * (double)(4 * nwp + 16);
      st.alg_flops += (double)N * (2.0 * (5 * nwp + 8) + 3.0);
    }
    store_state(&st, ctl, st.go ? nu : 0, slots);
    __syncthreads();
  }
  {
    double* gm = (st.i & 1) ? a.m1 : a.m0;
    double* gv[7] = {a.x, a.r, a.u, a.w, gm, a.n, nullptr};
    double* gr[4] = {a.P, a.S, a.Q, a.Z};
    resident_copy(R, gv, gr, 4, nb, N, false);
  }
  store_counters(&st, ctl);
}

// ---------------------------------------------------------------------------
// FCG
// ---------------------------------------------------------------------------

template <int NW>
__global__ void __launch_bounds__(kPerThreads) fcg_persistent(PersistArgs a) {
  constexpr int NWQ = NW / 4;
  extern __shared__ __align__(16) double s_dyn[];
  __shared__ PerState st;
  __shared__ double s_red[(kPerThreads / 32) * kPerNd];
  SolveCtl* ctl = a.ctl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = lane & 3;
  const int rowi = threadIdx.x >> 2;
  const int slots = a.mmax + 1;
  const int64_t N = a.N;
  const int nb = gridDim.x;
  const PerLayout L = per_layout(N, nb, slots, false);
  double* s_part = s_dyn;
  const Resident R{s_dyn + L.part_doubles, L.rows, L.pitch, L.nvec, slots};
  CsrStage cs;
  {
    char* cb = (char*)(s_dyn + L.part_doubles + L.resident_doubles);
    cs.rp = (int*)cb;
    cs.va = (double*)(cb + (((size_t)L.cpb * (kPerRows + 1) * sizeof(int) + 15) / 16 * 16));
    cs.ci = (int*)(cs.va + L.csr_cap);
    cs.cap = L.csr_cap;
  }
  double* red1 = a.partials;                             // [nb][kPerNd]: gamma, ||r||^2, -, -, window dots
  double* red3 = a.partials + (size_t)nb * kPerNd;       // [nb][kPerNd]: eta
  load_state(&st, ctl);
  if (st.status != kRun) return;   // a launch queued behind the one that finished
  {
    double* gv[4] = {a.x, a.r, a.u, const_cast<double*>(a.dinv)};
    double* gr[2] = {a.P, a.S};
    resident_copy(R, gv, gr, 2, nb, N, true);
  }
  stage_csr(a, cs, L.cpb, nb);
  double* sx = R.vec(0);
  double* sr = R.vec(1);
  double* su = R.vec(2);
  const double* sd = R.vec(3);
  const bool jacobi = a.dinv != nullptr;

  for (int g = 0; g < a.iters; ++g) {
    if (st.status != kRun) break;
    const int iprev = st.i, i = iprev + 1;
    const double alpha = st.alpha;
    const int nu = nu_window(i, a.mmax, st.truncation);
    const int pslot = iprev % slots, islot = i % slots;

    // ---- x_i, r_i, u_i = B(r_i) (Jacobi), gamma_i, ||r_i||^2, <u_i, s_k> ----
    double scq = 0.0;   // thread q of a row: gamma_i (q = 0), ||r_i||^2 (q = 1)
    double acc[NWQ];
#pragma unroll
    for (int s = 0; s < NWQ; ++s) acc[s] = 0.0;
    for (int lc = 0; lc < L.cpb; ++lc) {
      const int l = lc * kPerRows + rowi;
      const bool valid = own_row(l, nb, N) >= 0;
      double xn = 0.0, rn = 0.0, un = 0.0;
      if (valid) {
        xn = fma(alpha, R.ring(0, pslot)[l], sx[l]);
        rn = fma(-alpha, R.ring(1, pslot)[l], sr[l]);
        un = jacobi ? __dmul_rn(sd[l], rn) : rn;
        if (q < 2) scq = fma(q == 0 ? un : rn, rn, scq);
#pragma unroll
        for (int s = 0; s < NWQ; ++s) {
          const int j = 4 * s + q;
          if (j < nu) acc[s] = fma(un, R.ring(1, (i - nu + j) % slots)[l], acc[s]);
        }
      }
      __syncwarp();   // every lane of the row has read x, r before thread 0 of the row writes
      if (valid && q == 0) {
        sx[l] = xn;
        sr[l] = rn;
        su[l] = un;
      }
    }
    write_pipefcg_row<NWQ>(scq, acc, nu, s_red, red1 + (size_t)blockIdx.x * kPerNd);
    if (!grid_barrier(ctl)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->status = kTimeout;
      return;
    }
    fetch_partials(red1, nb, s_part);
    wait_partials();
    sum_partials(s_part, nb, 4 + nu, st.sums, s_red);
    // Alg. 2: gamma_i, convergence (thread 32), beta_{i,k} = -<u_i, s_k> / eta_k
    // (warp 0, used only when the iteration goes on)
    if (threadIdx.x == 32) {
      const double gamma = st.sums[0], rr = st.sums[1];
      st.it += 1;
      st.gamma = gamma;
      const double rho = st.norm == PFK_NORM_NATURAL ? sqrt(fabs(gamma)) : sqrt(rr);
      st.rho = rho;
      per_push_history(&st, ctl, rho, st.history ? sqrt(rr) : nan(""), nan(""), nan(""));
      st.go = 1;
      if (!isfinite(rho)) { st.status = kNonFinite; st.go = 0; }
      else if (rho <= st.target) { st.status = kConverged; st.i = i; st.go = 0; }
    }
    if ((int)threadIdx.x < nu) st.beta[threadIdx.x] = -st.sums[4 + threadIdx.x] / st.eta_ring[(i - nu + (int)threadIdx.x) % slots];
    __syncthreads();
    if (!st.go) {
      store_state(&st, ctl, 0, slots);
      break;
    }

    // ---- p_i = u_i + sum beta_{i,k} p_k into ring slot i (resident and global) ----
    double* gp = a.P + (size_t)islot * (size_t)N;
    for (int lc = 0; lc < L.cpb; ++lc) {
      const int l = lc * kPerRows + rowi;
      const int64_t e = own_row(l, nb, N);
      const bool valid = e >= 0;
      double sp = 0.0;
#pragma unroll
      for (int s = 0; s < NWQ; ++s) {
        const int j = 4 * s + q;
        if (valid && j < nu) sp = fma(st.beta[j], R.ring(0, (i - nu + j) % slots)[l], sp);
      }
      sp += __shfl_xor_sync(0xffffffffu, sp, 1);
      sp += __shfl_xor_sync(0xffffffffu, sp, 2);
      if (valid && q == 0) {
        const double p = su[l] + sp;
        R.ring(0, islot)[l] = p;
        gp[e] = p;
      }
    }
    if (!grid_barrier(ctl)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->status = kTimeout;
      return;
    }

    // ---- s_i = A p_i, eta_i = <p_i, s_i> ----
    double ps = 0.0;
    for (int lc = 0; lc < L.cpb; ++lc) {
      const int l = lc * kPerRows + rowi;
      const int64_t e = own_row(l, nb, N);
      if (e >= 0 && q == 0) {
        const double sv = csr_row(a, cs, gp, e, l);
        R.ring(1, islot)[l] = sv;
        ps = fma(R.ring(0, islot)[l], sv, ps);
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
    sum_partials(s_part, nb, 1, st.sums, s_red);
    if (threadIdx.x == 0) {
      // Alg. 2: eta_i = <p_i, s_i>, alpha_i = gamma_i / eta_i
      const double eta = st.sums[0];
      const double al = eta != 0.0 ? st.gamma / eta : nan("");
      st.i = i;
      st.eta = eta;
      st.alpha = al;
      st.nw = nu;
      st.eta_ring[i % slots] = eta;
      if (blockIdx.x == 0 && st.history && st.hist_len - 1 < st.hist_cap && st.hist_len >= 1) {
        st.history[(size_t)(st.hist_len - 1) * PFK_HISTORY_FIELDS + 2] = eta;
        st.history[(size_t)(st.hist_len - 1) * PFK_HISTORY_FIELDS + 3] = al;
      }
      if (eta <= 0.0) st.status = kBreakdown;
      else if (st.it >= st.maxit) st.status = kMaxit;
    }
    __syncthreads();
    store_state(&st, ctl, nu, slots);
    __syncthreads();
  }
  {
    double* gv[4] = {a.x, a.r, a.u, nullptr};
    double* gr[2] = {a.P, a.S};
    resident_copy(R, gv, gr, 2, nb, N, false);
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

static size_t persistent_smem(const pfk_context* ctx, int64_t N, int mmax, bool pipelined) {
  return per_layout(N, persistent_blocks(ctx, N), mmax + 1, pipelined).bytes();
}

bool persistent_eligible(const pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, int method, int naive_like,
                         int64_t N) {
  if (naive_like) return false;
  if (method != PFK_PIPEFCG && method != PFK_FCG) return false;
  if (!op->rowptr) return false;
  if (pc && pc->kind != PFK_PC_NONE && pc->kind != PFK_PC_JACOBI) return false;
  if (pc && pc->kind == PFK_PC_JACOBI && !op->csr_dinv && !op->dinv) return false;
  if (N < 1 || N > PFK_PERSISTENT_MAX_N || persistent_blocks(ctx, N) < 1) return false;
  // the rows of the largest window must fit in shared memory
  return persistent_smem(ctx, N, PFK_MAX_MMAX, true) <= kPerSmemLimit;
}

template <int NW>
static cudaError_t launch_one(bool pipelined, const PersistArgs& a, int blocks, cudaStream_t st) {
  void* fn = pipelined ? (void*)pipefcg_persistent<NW> : (void*)fcg_persistent<NW>;
  const int smem = (int)per_layout(a.N, blocks, a.mmax + 1, pipelined).bytes();
  if (smem > kPerSmemLimit) return cudaErrorInvalidValue;
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
