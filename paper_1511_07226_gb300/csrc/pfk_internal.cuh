// Internal declarations of the pfk library (not part of the C ABI).
//
// Layout in HBM: every vector is a contiguous FP64 array of n entries in cell
// order i + nx (j + ny k), 256-byte aligned (cudaMalloc).  Direction histories
// (p, s, q, z for PIPEFCG) are rings of (mmax + 1) such vectors stored back to
// back, slot of direction k = k mod (mmax + 1).  Scalars of the iteration live
// in a device control block (SolveCtl) so that every kernel of an iteration has
// the same arguments and one captured CUDA graph can be replayed.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pfk.h"

namespace pfk {

constexpr int kThreads = 256;          // threads per block of the streaming kernels
constexpr int kMaxBlocksPerSm = 8;     // upper bound of every reduction kernel's grid, per SM
constexpr int kPartialStride = PFK_MAX_MMAX + 8;   // upper bound of values per block in a reduction
constexpr int kCombineGroup = 32;      // blocks per group of the two-level combine
constexpr int kMaxCombineGroups = 64;  // groups it supports (grids of up to 2,048 blocks)

// Status codes kept in SolveCtl::status.
enum DevStatus : int {
  kRun = 0,
  kConverged = 1,
  kBreakdown = 2,       // eta_i <= 0 (or t < 0): restart from x
  kMaxit = 3,
  kFillBreakdown = 4,   // eta_0 <= 0 in a pipeline fill
  kNonFinite = 5,
  kCycleEnd = 6,        // GMRES types: restart length reached
  kTimeout = 7,         // a bounded grid-barrier wait of a persistent kernel ran out
};

// Device control block of one solve.
struct SolveCtl {
  int status;
  int it;          // iterations so far (all restarts)
  int i;           // index of the last completed iteration since the last (re)start
  int nw;          // size of the window W_i whose betas are in beta[]
  int hist_len;
  int hist_cap;
  int maxit;
  int mmax;
  int truncation;
  int norm;
  int target_set;
  int pad0;
  double target;
  double rtol, atol;
  double rho0, rho;
  double alpha, gamma, delta, eta;
  double beta[PFK_MAX_MMAX];
  double eta_ring[PFK_MAX_MMAX + 1];
  double* history;         // device buffer hist_cap * PFK_HISTORY_FIELDS
  unsigned int counter;    // arrival counter of the last-block reduction
  unsigned int gcounter[kMaxCombineGroups];   // per-group arrival counters of the two-level combine
  int passes;              // fused passes that did work
  double alg_bytes;        // their algorithmic HBM bytes
  double alg_flops;        // their FP64 flops (FMA = 2)
  double theta;            // projection coefficient <r_i, w_i>/<r_i, r_i> (eq. proj variant)
  double pend[3];          // reduction results handed from one kernel to the next (PIPEGCR apply)
  unsigned int bar_count;  // grid barrier of the persistent kernels: arrivals,
  unsigned int bar_gen;    // generation (bumped by the last arrival),
  unsigned int bar_abort;  // set when a wait timed out (every block then leaves)
  unsigned int bar_pad;
  long long bar_timeout_ns;  // bound of each barrier wait (<= 0: no wait allowed)
};

// Control block of a preconditioner application (inner iterations).
struct PcCtl {
  int ok;                  // last inner iteration whose x update happens (k, or
                           // earlier when <D^-1 r, r> or <s, p> hit exactly 0)
  int pad;
  double gamma, eta;
  double alpha[64];
  double beta[64];
  unsigned int counter;
  unsigned int pad1;
  long long calls;         // noisy preconditioner: applications so far
  double scale;            // noisy preconditioner: eta ||v|| / ||xi_j|| of the current application
  long long row;           // noisy preconditioner: j mod count of the current application
};

}  // namespace pfk

// ---------------------------------------------------------------------------
// Opaque handle types of the C ABI
// ---------------------------------------------------------------------------

struct pfk_context {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;    // library-owned, only used to record CUDA graphs
  int num_sms = 0;
  std::string err;
  // cached workspace of pfk_solve (grown on demand)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* scratch_partials = nullptr;   // reduction partials for standalone calls
  unsigned int* scratch_counter = nullptr;
  double* scratch_out = nullptr;
  pfk::SolveCtl* pinned = nullptr;      // host-pinned status copies of pfk_solve
  // block sizes autotuned by pfk_solve_batched, keyed by (mmax template, log2 of
  // the largest system, count bucket, preconditioner precision + 2 x inner iterations)
  std::map<std::tuple<int, int, int, int>, int> batched_tuned;
};

struct pfk_operator {
  pfk_context* ctx = nullptr;   // used while the context lives; destruction uses `device`
  int device = 0;
  cudaStream_t stream = nullptr;
  int kind = 0;
  int storage = 0;
  int nx = 0, ny = 0, nz = 0, ndim = 0;
  int64_t n = 0;
  // stencil, FP64: diagonal, +x/+y/+z face coefficients (0 on the boundary), D^-1
  double* d = nullptr;
  double* kx = nullptr;
  double* ky = nullptr;
  double* kz = nullptr;
  double* dinv = nullptr;
  double adv[3] = {0, 0, 0};    // h |v_d|
  int upw[3] = {0, 0, 0};       // -1: upwind at -e_d (v_d > 0), +1: at +e_d, 0: none
  double gersh = 0.0;           // max_i sum_j |a_ij| / a_ii
  // reduced-precision copies (created on demand by preconditioners)
  float* d32 = nullptr;
  float* kx32 = nullptr;
  float* ky32 = nullptr;
  float* kz32 = nullptr;
  float* dinv32 = nullptr;
  __nv_bfloat16* d16 = nullptr;
  __nv_bfloat16* kx16 = nullptr;
  __nv_bfloat16* ky16 = nullptr;
  __nv_bfloat16* kz16 = nullptr;
  __nv_bfloat16* dinv16 = nullptr;
  // CSR (kind CSR, or stencil with storage CSR)
  int64_t nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  double* vals = nullptr;
  double* csr_dinv = nullptr;
};

struct pfk_pc {
  pfk_context* ctx = nullptr;   // used while the context lives; destruction uses `device`
  int device = 0;
  cudaStream_t stream = nullptr;
  const pfk_operator* op = nullptr;
  int kind = 0;
  int inner = 0;
  int precision = 0;
  double lo = 0.0, hi = 0.0;
  // scratch of the inner iterations (FP64 or FP32 depending on precision)
  void* buf = nullptr;
  size_t buf_bytes = 0;
  pfk::PcCtl* ctl = nullptr;
  double* partials = nullptr;
  int partials_cap = 0;         // doubles in `partials` (bounds the grid of the reduction kernels)
  // noisy preconditioner: the noise bank (count x n) and 1 / ||xi_j||
  double noise_eta = 0.0;
  double* bank = nullptr;
  double* bank_inv_norm = nullptr;
  int bank_count = 0;
  void* nested = nullptr;       // block upper-triangular preconditioner state (nested.cu)
};

namespace pfk {

// ---------------------------------------------------------------------------
// Error handling helpers (host)
// ---------------------------------------------------------------------------
void set_error(pfk_context* ctx, const std::string& msg);
pfk_status cuda_fail(pfk_context* ctx, cudaError_t e, const char* what);

#define PFK_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return pfk::cuda_fail(ctx, e_, #call); \
  } while (0)

// Grid size of the streaming kernels: a fixed function of n and the SM count,
// so reductions are combined in the same order on every run.
int stream_blocks(const pfk_context* ctx, int64_t n, int blocks_per_sm = 2);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sums over rows: out[j] = sum_{b < nrows} rows[b * stride + j], j < nd, by
// all threads of the block.  The loads come from L2 (~0.4 us each) while the
// rest of the GPU may idle, so they are issued many at a time: for nd <= 4
// thread t takes rows t, t + T, ... (all nd values of a row, four rows per
// step); otherwise lane l of warp w takes values l and l + 32 of rows w,
// w + nwarps, ... (a coalesced row per load, eight rows per step).  Each
// thread adds its rows in increasing order, then a fixed shuffle tree (nd <=
// 4) or the warps in order combine them: the sums are deterministic.  smem
// holds nwarps * nd doubles; out may be shared or global memory.
__device__ __forceinline__ void sum_rows(const double* rows, int nrows, int nd, int stride, double* smem,
                                         double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (nd <= 4) {
    const int T = blockDim.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int b = threadIdx.x;
    for (; b + 3 * T < nrows; b += 4 * T) {
      double t[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) t[u][q] = q < nd ? __ldcg(&rows[(size_t)(b + u * T) * stride + q]) : 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += t[u][q];
    }
    for (; b < nrows; b += T)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nd) acc[q] += __ldcg(&rows[(size_t)b * stride + q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q < nd) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) smem[warp * nd + q] = v;
      }
    }
  } else {
    constexpr int U = 8;
    for (int jc = 0; jc < nd; jc += 64) {
      const int j0 = jc + lane, j1 = jc + lane + 32;
      const bool h0 = j0 < nd, h1 = j1 < nd;
      double a0 = 0.0, a1 = 0.0;
      int b = warp;
      for (; b + (U - 1) * nwarps < nrows; b += U * nwarps) {
        double t0[U], t1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const double* row = rows + (size_t)(b + u * nwarps) * stride;
          t0[u] = h0 ? __ldcg(row + j0) : 0.0;
          t1[u] = h1 ? __ldcg(row + j1) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          a0 += t0[u];
          a1 += t1[u];
        }
      }
      for (; b < nrows; b += nwarps) {
        const double* row = rows + (size_t)b * stride;
        if (h0) a0 += __ldcg(row + j0);
        if (h1) a1 += __ldcg(row + j1);
      }
      if (h0) smem[warp * nd + j0] = a0;
      if (h1) smem[warp * nd + j1] = a1;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nd; j += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nwarps; ++w) v += smem[w * nd + j];
    out[j] = v;
  }
  __syncthreads();
}

// Writes this block's row partials[blockIdx.x * stride + j] = sum_w smem[w *
// nd + j] (smem[w * nd + j]: warp w's sum of value j).
__device__ __forceinline__ void write_block_row(const double* smem, int nd, double* partials, int stride) {
  const int nwarps = blockDim.x >> 5;
  for (int j = threadIdx.x; j < nd; j += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nwarps; ++w) v += smem[w * nd + j];
    partials[(size_t)blockIdx.x * stride + j] = v;
  }
}

// Arrival at `counter` after this block's writes; true in the block that
// arrives as number `count` (all its threads), which then sees every earlier
// arrival's writes.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int count) {
  __shared__ unsigned int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == count - 1) ? 1u : 0u;
  __syncthreads();
  const bool last = s_last != 0u;
  if (last) __threadfence();
  return last;
}

// Second half of reduce_last_block, for kernels that prepare the per-warp
// partial sums themselves: smem[w * nd + j] holds warp w's sum of value j.
// Writes this block's partial sums, then the last block to arrive combines all
// blocks' partials in a fixed order (sum_rows) into sums[j] and returns true.
// smem is reused.
__device__ __forceinline__ bool combine_block_partials(double* smem, int nd, double* partials, int stride,
                                                       unsigned int* counter, double* sums) {
  write_block_row(smem, nd, partials, stride);
  if (!arrive_last(counter, gridDim.x)) return false;
  sum_rows(partials, gridDim.x, nd, stride, smem, sums);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Two-level variant for the large reductions: the last block of each group of
// kCombineGroup consecutive blocks sums the group's rows (sum_rows, block
// order) into group row nb + g while other blocks still compute; the last
// group to finish sums the group rows in group order into sums.  The serial
// tail is one group's rows plus the group rows instead of all nb rows.
// partials holds (nb + ceil(nb / kCombineGroup)) * stride doubles; gcounter
// one zero counter per group (left zero); nb <= kCombineGroup *
// kMaxCombineGroups.
__device__ __forceinline__ bool combine_block_partials_2l(double* smem, int nd, double* partials, int stride,
                                                          unsigned int* counter, unsigned int* gcounter,
                                                          double* sums) {
  const int nb = gridDim.x;
  const int g = blockIdx.x / kCombineGroup;
  const int gb0 = g * kCombineGroup;
  const int gn = min(kCombineGroup, nb - gb0);
  const int ng = (nb + kCombineGroup - 1) / kCombineGroup;
  write_block_row(smem, nd, partials, stride);
  if (!arrive_last(&gcounter[g], (unsigned int)gn)) return false;
  sum_rows(partials + (size_t)gb0 * stride, gn, nd, stride, smem, partials + (size_t)(nb + g) * stride);
  if (threadIdx.x == 0) gcounter[g] = 0u;
  if (!arrive_last(counter, (unsigned int)ng)) return false;
  sum_rows(partials + (size_t)nb * stride, ng, nd, stride, smem, sums);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Block-level partial sums of `nd` accumulators, written to
// partials[blockIdx.x * stride + j]; then the last block to arrive combines all
// blocks' partials in a fixed order (lane-strided over blocks, then a fixed
// shuffle tree) into sums[j] (shared memory of the last block).
// Returns true in the last block (all its threads).  `smem` must hold
// (kThreads / 32) * nd doubles; sums must hold nd doubles.
template <int ND>
__device__ __forceinline__ bool reduce_last_block(const double (&acc)[ND], int nd, double* partials, int stride,
                                                  unsigned int* counter, double* smem, double* sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    if (j < nd) {
      double v = warp_sum(acc[j]);
      if (lane == 0) smem[warp * nd + j] = v;
    }
  }
  __syncthreads();
  return combine_block_partials(smem, nd, partials, stride, counter, sums);
}

// ---------------------------------------------------------------------------
// Kernel launchers shared between translation units
// ---------------------------------------------------------------------------

// y = A x (FP64).  If `status` is non-null the kernel does nothing when
// *status != kRun.  If `bsub` is non-null computes y = bsub - A x.
cudaError_t op_apply(const pfk_operator* op, const double* x, double* y, const double* bsub, const int* status,
                     cudaStream_t st);

// out = add + B(v) (add may be null).  `status` as above.
cudaError_t pc_apply(const pfk_pc* pc, const double* v, double* out, const double* add, const int* status,
                     cudaStream_t st);

// Nested block preconditioner (nested.cu).
cudaError_t nested_apply(const pfk_pc* pc, const double* v, double* out, const double* add, const int* status,
                         cudaStream_t st);
void destroy_nested(pfk_pc* pc);

// Sum of squares / dot products into a device scalar (deterministic order).
cudaError_t dot_into(pfk_context* ctx, const double* a, const double* b, int64_t n, double* out, cudaStream_t st);

}  // namespace pfk
