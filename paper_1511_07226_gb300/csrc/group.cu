// Grouped persistent PIPEFCG / PIPEGCR / PIPEFGMRES: several stencil systems
// advanced together by one cooperative launch, each system by its own group
// of CTAs.
//
// A system of n cells belongs to a group of C CTAs (by default about 4,096
// cells per CTA, at most kGrpMaxCtas); the CTA of rank q owns a contiguous
// range of the grid's x-rows (a row is a (j, k) pair) and with them those
// cells of every vector.  The system's PIPEFCG solve (Alg. 8) runs on the
// group alone: the pipeline fill, the fused pass (the deferred MAXPYs of the
// previous iteration, the advance of x, r, u, w, the dots gamma_i, delta_i,
// ||r_i||^2 and the window dots <u_i, s_k>), the preconditioner (none,
// Jacobi, or k inner Jacobi-PCG iterations, Alg. 3, in FP64 or FP32) and
// the operator.  PIPEGCR (Alg. 11) splits the pass in two: the deferred MAXPYs
// with the advance of x, r, u, then w_i = A u_i with the dots gamma_i =
// <r_i, w_i>, delta_i = <w_i, w_i>, ||r_i||^2 and <w_i, s_k>.  PIPEFGMRES
// (Alg. 15) forms p_k, u_k, zbar_k and the dots of Hessenberg column k in one
// pass; every CTA keeps the Givens rotations, and a restart cycle ends with
// the least-squares solution and x = x_0 + U y.
//
// A reduction writes one partial row per CTA; the CTAs meet at the system's
// own barrier (an arrival counter and a generation word of that system, with
// bounded waits) and every CTA sums the rows in rank order, so all CTAs of
// the group hold bitwise the same scalars and run the scalar phase
// themselves.  An operator application that reads other CTAs' rows
// (the stencil's neighbouring planes) first waits at the system's barrier for
// its input vector to be complete.  Nothing waits for another system.
//
// The solve is resumable: a launch advances each system by at most `iters`
// steps (a step is an iteration, a pipeline fill or a PIPEFGMRES cycle start
// with its first column) and leaves its scalars in
// the system's state record, so the host can retire finished systems and
// admit new ones between launches (continuous batching).  Restarts on norm
// breakdown and residual replacement (the true-residual check at
// convergence) follow the single-system driver (Sec. 5).  A system's
// arithmetic depends only on its own data and its CTA count, never on the
// other systems of the launch, so its result is bitwise the same alone or in
// any batch.  With C = 1 this is the one-block-per-system batched solve.
#include "group.cuh"
#include "pfk_internal.cuh"
#include "solver.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

namespace pfk {

pfk_status ensure_reduced_copies(pfk_operator* op, int precision);

constexpr int kGrpThreads = 256;
constexpr int kGrpNW = PFK_MAX_MMAX;         // window buffer of the pass (columns)
constexpr int kGrpNd = PFK_MAX_MMAX + 4;     // longest partial row
constexpr int kGrpMaxCtas = 64;              // CTAs of one system
constexpr int kGrpCellsPerCta = 4096;        // default group size: cells per CTA
constexpr int kGrpMaxInner = 64;             // inner PCG iterations

enum GrpPhase { kGStart = 0, kGFill = 1, kGIter = 2, kGDone = 3 };

struct GrpParams {
  int method;                 // PFK_PIPEFCG, PFK_PIPEGCR or PFK_PIPEFGMRES
  int mmax, truncation, norm, maxit, max_restarts, true_check;
  double rtol, atol;
  int pc_kind, pc_inner;
  int pc_fp32, pad_p;         // inner PCG in FP32 (vectors and coefficient copies)
  long long bar_timeout_ns;   // bound of each barrier wait (<= 0: no wait allowed)
  double sigma;               // PIPEFGMRES shift; NaN: estimated at the start
};

// Barrier words of one system (reset by the host at admission).
struct GrpBar {
  unsigned int count, gen, abort, pad;
};

// Solve state of one system, kept in device memory between launches.  During
// a launch every CTA of the group holds an identical copy in shared memory;
// rank 0 writes it back at the end.
struct GrpState {
  int phase, status, result;
  int it, i, nw, restarts, breakdowns, replacements, hist_len, prev_bd, target_set;
  int steps, pad;
  double alpha, gamma, delta, eta, target, rho0, rho, bnorm, goal, rtrue;
  double beta[PFK_MAX_MMAX];
  double eta_ring[PFK_MAX_MMAX + 1];
  // PIPEFGMRES: the shift, and the current restart cycle's Givens rotations,
  // rotated right-hand side g and previous Hessenberg column (hbar and h)
  double sigma, gm_inv;
  double gm_cs[PFK_MAX_MMAX], gm_sn[PFK_MAX_MMAX], gm_g[PFK_MAX_MMAX + 1];
  double gm_hb[PFK_MAX_MMAX + 1], gm_h[PFK_MAX_MMAX + 1];
  int gm_k, gm_ncols;      // column the next pass forms; valid columns of the cycle
};
static_assert(sizeof(GrpState) % 8 == 0, "GrpState is copied as 8-byte words");

struct GrpSys {
  int nx, ny, nz, ndim;
  int64_t n;
  const double* d;
  const double* kx;
  const double* ky;
  const double* kz;
  const double* dinv;
  const float* d32;   // FP32 coefficient copies (FP32 inner PCG)
  const float* kx32;
  const float* ky32;
  const float* kz32;
  const float* dinv32;
  double a0, a1, a2;
  int u0, u1, u2;
  int adv;            // any advection weight non-zero
  int nblk;           // CTAs of the group
  int pad0;
  const double* b;
  double* x;
  double* ws;         // r, u, w, m, n, t, tmp, then rings P, S, Q, Z of mmax + 1 slots
                      // (PIPEFGMRES: r, qbar, wbar at 0, n, 2n; then p_j, u_j, zbar_j at 7n)
  double* pcws;       // inner PCG: r, p, s, x
  double* part;       // [2][nblk][kGrpNd] partial rows
  double* gm;         // PIPEFGMRES: rotated Hessenberg columns R [(m+1) x m] (rank 0 writes)
  double* hist;
  int hist_cap, pad;
  GrpParams P;
  GrpState* state;
  GrpBar* bar;
};

namespace {

// What a CTA keeps for its system during a launch (shared memory).
struct GrpCta {
  GrpState st;
  double red[8];                 // results of group sums
  double pg, pbeta;              // inner PCG scalars
  double palpha[kGrpMaxInner];
  double s_beta[kGrpNW];
  double s_h[kGrpNW];            // PIPEFGMRES: h_{j,k-1} of the pass
  double s_y[kGrpNW];            // PIPEFGMRES: least-squares solution of the cycle
  double s_col[kGrpNW + 1];      // PIPEFGMRES: the column being rotated
  double s_tot[kGrpNd];
  size_t s_off[kGrpNW];
  int last_x, par, rank, nblk, abort, pad;
  int64_t row_lo, row_hi;        // the CTA's x-rows [row_lo, row_hi)
};

__device__ __forceinline__ unsigned long long grp_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int grp_ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int grp_atom_add(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void grp_red_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of the system's group.  Arrival on the system's counter
// (acquire-release: the CTA's writes, ordered before thread 0 by the block
// barrier, are released; the last arrival acquires everyone's); the last
// arrival resets the counter and bumps the generation with a release, the
// others wait for it with acquire loads, at most bar_timeout_ns.  A wait that
// runs out raises the system's abort word, and a raised abort word makes
// every later barrier of the system return at once; the CTA then records the
// abort and the step loop stops.  One CTA: a block barrier.
__device__ void grp_barrier(const GrpSys& S, GrpCta* g) {
  __syncthreads();
  if (g->nblk == 1) return;
  if (threadIdx.x == 0) {
    int ok = !g->abort && !grp_ld_acquire(&S.bar->abort);
    if (ok) {
      const unsigned int gen = grp_ld_acquire(&S.bar->gen);
      if (grp_atom_add(&S.bar->count, 1u) == (unsigned int)g->nblk - 1u) {
        S.bar->count = 0u;
        grp_red_release(&S.bar->gen, 1u);
      } else {
        const unsigned long long t0 = grp_ns();
        const long long budget = S.P.bar_timeout_ns;
        while (grp_ld_acquire(&S.bar->gen) == gen) {
          if (grp_ld_acquire(&S.bar->abort)) { ok = 0; break; }
          if (budget <= 0 || grp_ns() - t0 > (unsigned long long)budget) {
            atomicExch(&S.bar->abort, 1u);
            ok = 0;
            break;
          }
        }
      }
    }
    if (!ok) g->abort = 1;
  }
  __syncthreads();
}

// Sums ND values over the system's cells into g->red[0..ND): per CTA a fixed
// warp tree and the warps in order; with several CTAs each writes its row of
// partials, and after the system's barrier every CTA adds the rows in rank
// order.  All threads of the CTA must call it.
template <int ND>
__device__ void grp_sum(const GrpSys& S, GrpCta* g, const double (&v)[ND], double* s_red) {
  constexpr int NWARP = kGrpThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int par = g->par;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const double s = warp_sum(v[j]);
    if (lane == 0) s_red[warp * ND + j] = s;
  }
  __syncthreads();
  if (threadIdx.x < ND) {
    double s = 0.0;
    for (int w = 0; w < NWARP; ++w) s += s_red[w * ND + threadIdx.x];
    if (g->nblk == 1) g->red[threadIdx.x] = s;
    else S.part[((size_t)par * g->nblk + g->rank) * kGrpNd + threadIdx.x] = s;
  }
  if (g->nblk == 1) {
    __syncthreads();
    return;
  }
  grp_barrier(S, g);
  if (threadIdx.x < ND) {
    const double* p = S.part + (size_t)par * g->nblk * kGrpNd + threadIdx.x;
    double s = 0.0;
    for (int b = 0; b < g->nblk; ++b) s += __ldcg(p + (size_t)b * kGrpNd);
    g->red[threadIdx.x] = s;
  }
  if (threadIdx.x == 0) g->par = par ^ 1;
  __syncthreads();
}

// The CTA's cells (contiguous: whole x-rows).  Call sites unroll these loops
// (more loads in flight per thread; the accumulation order is unchanged).
#define GRP_ELEMS(S, g, e)                                                                          \
  for (int64_t e = (g)->row_lo * (S).nx + threadIdx.x, e_end_ = (g)->row_hi * (S).nx; e < e_end_;  \
       e += kGrpThreads)

// The CTA's x-rows, one per warp; (i, j, k) and the cell index c.
#define GRP_ROWS(S, g, c, i, j, k)                                                                  \
  for (int64_t row_ = (g)->row_lo + (threadIdx.x >> 5); row_ < (g)->row_hi; row_ += kGrpThreads / 32) \
    for (int j = (int)(row_ % (S).ny), k = (int)(row_ / (S).ny), i = (int)(threadIdx.x & 31); i < (S).nx; \
         i += 32)                                                                                    \
      for (int64_t c = row_ * (S).nx + i, once_ = 1; once_; once_ = 0)

// The operator's coefficients in the arithmetic type V of a kernel phase: the
// FP64 arrays, or the FP32 copies of the FP32 inner preconditioner.
template <typename V>
struct GrpCoef {
  const V* d;
  const V* kx;
  const V* ky;
  const V* kz;
  const V* dinv;
};

// (A m)_c for cell c = (i, j, k): diffusion faces and upwind advection, fused
// multiply-adds in a fixed order, in V.  m is written by other CTAs during the
// launch, so its loads go to L2 (never a stale L1 line).
template <typename V>
__device__ __forceinline__ V grp_row_t(const GrpSys& S, const GrpCoef<V>& A, const V* m, int64_t c, int i, int j,
                                       int k) {
  const int64_t sxy = (int64_t)S.nx * S.ny;
  if (!S.adv) {
    // pure diffusion: the same products without the zero advection weights
    // (adding +0 to a coefficient changes nothing)
    V acc = A.d[c] * __ldcg(m + c);
    if (i > 0) acc = fma(-A.kx[c - 1], __ldcg(m + c - 1), acc);
    if (i < S.nx - 1) acc = fma(-A.kx[c], __ldcg(m + c + 1), acc);
    if (j > 0) acc = fma(-A.ky[c - S.nx], __ldcg(m + c - S.nx), acc);
    if (j < S.ny - 1) acc = fma(-A.ky[c], __ldcg(m + c + S.nx), acc);
    if (S.ndim == 3) {
      if (k > 0) acc = fma(-A.kz[c - sxy], __ldcg(m + c - sxy), acc);
      if (k < S.nz - 1) acc = fma(-A.kz[c], __ldcg(m + c + sxy), acc);
    }
    return acc;
  }
  const V a0 = (V)S.a0, a1 = (V)S.a1, a2 = (V)S.a2;
  V acc = A.d[c] * __ldcg(m + c);
  if (i > 0) acc = fma(-(A.kx[c - 1] + (S.u0 == -1 ? a0 : V(0))), __ldcg(m + c - 1), acc);
  if (i < S.nx - 1) acc = fma(-(A.kx[c] + (S.u0 == 1 ? a0 : V(0))), __ldcg(m + c + 1), acc);
  if (j > 0) acc = fma(-(A.ky[c - S.nx] + (S.u1 == -1 ? a1 : V(0))), __ldcg(m + c - S.nx), acc);
  if (j < S.ny - 1) acc = fma(-(A.ky[c] + (S.u1 == 1 ? a1 : V(0))), __ldcg(m + c + S.nx), acc);
  if (S.ndim == 3) {
    if (k > 0) acc = fma(-(A.kz[c - sxy] + (S.u2 == -1 ? a2 : V(0))), __ldcg(m + c - sxy), acc);
    if (k < S.nz - 1) acc = fma(-(A.kz[c] + (S.u2 == 1 ? a2 : V(0))), __ldcg(m + c + sxy), acc);
  }
  return acc;
}

__device__ __forceinline__ GrpCoef<double> grp_coef64(const GrpSys& S) {
  return GrpCoef<double>{S.d, S.kx, S.ky, S.kz, S.dinv};
}

__device__ __forceinline__ double grp_row(const GrpSys& S, const double* m, int64_t c, int i, int j, int k) {
  return grp_row_t<double>(S, grp_coef64(S), m, c, i, j, k);
}

// y = A m, or y = bsub - A m, on the CTA's cells.  m must be complete on
// every CTA of the group (the caller passed a system barrier since it was
// last written).
__device__ void grp_apply(const GrpSys& S, GrpCta* g, const double* m, double* y, const double* bsub) {
  #pragma unroll 2
  GRP_ROWS(S, g, c, i, j, k) {
    const double v = grp_row(S, m, c, i, j, k);
    y[c] = bsub ? bsub[c] - v : v;
  }
  __syncthreads();
}

// Inner Jacobi-PCG in V (FP64, or FP32 vectors and coefficient copies with
// the inner products of FP32 values accumulated in FP64): out = add + x_k.
template <typename V>
__device__ void grp_pcg(const GrpSys& S, GrpCta* g, const GrpCoef<V>& A, const double* v, double* out,
                        const double* add, double* s_red) {
  const int64_t n = S.n;
  V* r = (V*)S.pcws;
  V* p = r + n;
  V* s = p + n;
  V* x = s + n;
  const V* dinv = A.dinv;
  const int kk = S.P.pc_inner;
  {
    // r_0 = v; gamma_0 = <D^-1 r_0, r_0>
    double acc[1] = {0.0};
    #pragma unroll 4
    GRP_ELEMS(S, g, e) {
      const V rv = (V)v[e];
      r[e] = rv;
      const V z = dinv[e] * rv;
      acc[0] += (double)z * (double)rv;
    }
    grp_sum<1>(S, g, acc, s_red);
    if (threadIdx.x == 0) {
      g->pg = g->red[0];
      g->last_x = g->pg == 0.0 ? 0 : kk;
    }
    __syncthreads();
  }
  if (g->last_x > 0) {
    // p_0 = D^-1 r_0, s_0 = A p_0, eta_0 = <s_0, p_0>
    #pragma unroll 4
    GRP_ELEMS(S, g, e) p[e] = dinv[e] * r[e];
    grp_barrier(S, g);
    double acc[1] = {0.0};
    #pragma unroll 2
    GRP_ROWS(S, g, c, i, j, k) {
      const V sv = grp_row_t<V>(S, A, p, c, i, j, k);
      s[c] = sv;
      acc[0] += (double)sv * (double)p[c];
    }
    grp_sum<1>(S, g, acc, s_red);
    if (threadIdx.x == 0) {
      if (g->red[0] == 0.0) g->last_x = 0;
      else g->palpha[0] = g->pg / g->red[0];
    }
    __syncthreads();
  }
  for (int it = 1; it < kk; ++it) {
    if (it > g->last_x) break;
    {
      // r_i = r_{i-1} - alpha_{i-1} s_{i-1}; gamma_i
      const V al = (V)g->palpha[it - 1];
      double acc[1] = {0.0};
      #pragma unroll 4
      GRP_ELEMS(S, g, e) {
        const V rv = r[e] - al * s[e];
        r[e] = rv;
        const V z = dinv[e] * rv;
        acc[0] += (double)z * (double)rv;
      }
      grp_sum<1>(S, g, acc, s_red);
      if (threadIdx.x == 0) {
        const double gn = g->red[0];
        if (gn == 0.0) {
          g->last_x = it;
        } else {
          g->pbeta = gn / g->pg;
          g->pg = gn;
        }
      }
      __syncthreads();
    }
    {
      // x_i = x_{i-1} + alpha_{i-1} p_{i-1}; p_i = D^-1 r_i + beta_i p_{i-1}
      const V al = (V)g->palpha[it - 1];
      const V be = (V)g->pbeta;
      const bool do_p = it < g->last_x;
      #pragma unroll 4
      GRP_ELEMS(S, g, e) {
        const V po = p[e];
        x[e] = (it == 1 ? V(0) : x[e]) + al * po;
        if (do_p) p[e] = dinv[e] * r[e] + be * po;
      }
      if (!do_p) {
        __syncthreads();
        break;
      }
      grp_barrier(S, g);
    }
    {
      // s_i = A p_i, eta_i
      double acc[1] = {0.0};
      #pragma unroll 2
      GRP_ROWS(S, g, c, i, j, k) {
        const V sv = grp_row_t<V>(S, A, p, c, i, j, k);
        s[c] = sv;
        acc[0] += (double)sv * (double)p[c];
      }
      grp_sum<1>(S, g, acc, s_red);
      if (threadIdx.x == 0) {
        if (g->red[0] == 0.0) g->last_x = it;
        else g->palpha[it] = g->pg / g->red[0];
      }
      __syncthreads();
    }
  }
  const int last_x = g->last_x;
  const V al = (V)g->palpha[kk - 1];
  #pragma unroll 4
  GRP_ELEMS(S, g, e) {
    double y;
    if (last_x == 0) y = 0.0;
    else if (kk <= last_x) y = (double)((kk == 1 ? V(0) : x[e]) + al * p[e]);
    else y = (double)x[e];
    out[e] = add ? add[e] + y : y;
  }
  grp_barrier(S, g);
}

// out = add + B(v) on the CTA's cells (v and add: this CTA's own cells, already
// written); ends with a system barrier, so out may feed an operator.  Inner
// PCG in the statement order of Alg. 3 with x_0 = 0 and the same guards as the
// single-system preconditioner (an exactly zero <D^-1 r, r> or <s, p> stops
// the updates of x).
__device__ void grp_pc(const GrpSys& S, GrpCta* g, const double* v, double* out, const double* add, double* s_red) {
  const GrpParams& P = S.P;
  if (P.pc_kind != PFK_PC_INNER_PCG) {
    #pragma unroll 4
    GRP_ELEMS(S, g, e) {
      // B(v) = D^-1 v and add + B(v): two roundings (no fused multiply-add)
      const double y = P.pc_kind == PFK_PC_JACOBI ? __dmul_rn(S.dinv[e], v[e]) : v[e];
      out[e] = add ? __dadd_rn(add[e], y) : y;
    }
    grp_barrier(S, g);
    return;
  }
  if (P.pc_fp32) grp_pcg<float>(S, g, GrpCoef<float>{S.d32, S.kx32, S.ky32, S.kz32, S.dinv32}, v, out, add, s_red);
  else grp_pcg<double>(S, g, grp_coef64(S), v, out, add, s_red);
}

__device__ __forceinline__ double grp_rho(const GrpParams& P, double gamma, double rr) {
  return P.norm == PFK_NORM_NATURAL ? sqrt(fabs(gamma)) : sqrt(rr);
}

__device__ __forceinline__ void grp_push_history(const GrpSys& S, GrpCta* g, double rho, double rn, double eta,
                                                 double al) {
  GrpState* st = &g->st;
  if (g->rank == 0 && S.hist && st->hist_len < S.hist_cap) {
    double* h = S.hist + (size_t)st->hist_len * PFK_HISTORY_FIELDS;
    h[0] = rho; h[1] = rn; h[2] = eta; h[3] = al;
  }
  st->hist_len += 1;
}

// Scalar phase of iteration i (thread 0 of every CTA): convergence test on
// rho_i first (the listings' order), then beta_{i,k} = -c_k / eta_k for the
// window k = i - nu_i .. i - 1 (cw(jj) gives c for k = i - nu_i + jj), eta_i =
// delta_i - sum_k beta_{i,k}^2 eta_k (k ascending), alpha_i = gamma_i / eta_i;
// eta_i <= 0 is a norm breakdown.
template <typename CW>
__device__ void grp_scalar_phase(const GrpSys& S, GrpCta* g, int i, double gamma, double delta, double rr,
                                 const CW& cw) {
  const GrpParams& P = S.P;
  GrpState* st = &g->st;
  const int slots = P.mmax + 1;
  st->it += 1;
  st->i = i;
  st->gamma = gamma;
  st->delta = delta;
  const double rho = grp_rho(P, gamma, rr);
  st->rho = rho;
  const int hslot = st->hist_len;
  grp_push_history(S, g, rho, sqrt(rr), nan(""), nan(""));
  if (!isfinite(rho)) {
    st->status = kNonFinite;
    return;
  }
  if (rho <= st->target) {
    st->status = kConverged;
    return;
  }
  const int nu = nu_window(i, P.mmax, P.truncation);
  double sumb = 0.0;
  for (int jj = 0; jj < nu; ++jj) {
    const double ek = st->eta_ring[(i - nu + jj) % slots];
    const double bb = -cw(jj) / ek;
    st->beta[jj] = bb;
    sumb += bb * bb * ek;
  }
  const double eta = delta - sumb;
  const double al = eta != 0.0 ? gamma / eta : nan("");
  st->eta = eta;
  st->alpha = al;
  st->nw = nu;
  st->eta_ring[i % slots] = eta;
  if (g->rank == 0 && S.hist && hslot < S.hist_cap) {
    S.hist[(size_t)hslot * PFK_HISTORY_FIELDS + 2] = eta;
    S.hist[(size_t)hslot * PFK_HISTORY_FIELDS + 3] = al;
  }
  if (eta <= 0.0) st->status = kBreakdown;
  else if (st->it >= P.maxit) st->status = kMaxit;
}

// Combines a CTA's partial row (nd values in s_row, shared) over the group
// into g->s_tot: directly with one CTA, else through the partial rows and the
// system's barrier, summed in rank order.
__device__ void grp_combine_row(const GrpSys& S, GrpCta* g, int nd, const double* s_warp) {
  const int par = g->par;
  if (threadIdx.x < nd) {
    double v = 0.0;
    for (int w = 0; w < kGrpThreads / 32; ++w) v += s_warp[w * nd + threadIdx.x];
    if (g->nblk == 1) g->s_tot[threadIdx.x] = v;
    else S.part[((size_t)par * g->nblk + g->rank) * kGrpNd + threadIdx.x] = v;
  }
  if (g->nblk > 1) {
    grp_barrier(S, g);
    if (threadIdx.x < nd) {
      const double* pp = S.part + (size_t)par * g->nblk * kGrpNd + threadIdx.x;
      double v = 0.0;
      for (int b = 0; b < g->nblk; ++b) v += __ldcg(pp + (size_t)b * kGrpNd);
      g->s_tot[threadIdx.x] = v;
    }
    if (threadIdx.x == 0) g->par = par ^ 1;
  }
  __syncthreads();
}

// The fused pass of iteration i (the same statements as the single-system
// pass: the deferred MAXPYs p, s, q, z of iteration i-1 from u, w, m, n and
// the window; x, r, u, w advanced with alpha_{i-1}; t = w - r; the dots
// gamma, delta, ||r||^2, <u, s_{i-1}> and <u, s_k> for the rest of the
// window), then the group sum and the scalar phase in every CTA.
__device__ void grp_pass(const GrpSys& S, GrpCta* g, double* smem) {
  constexpr int T = kGrpThreads;
  GrpState* st = &g->st;
  const int64_t n = S.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* vr = S.ws;
  double* vu = vr + n;
  double* vw = vu + n;
  const double* vm = vw + n;
  const double* vn = vm + n;
  double* vt = (double*)vn + n;
  const int slots = S.P.mmax + 1;
  double* Pr = S.ws + 7 * n;
  double* Sr = Pr + (int64_t)slots * n;
  double* Qr = Sr + (int64_t)slots * n;
  double* Zr = Qr + (int64_t)slots * n;
  const int iprev = st->i;
  const int nwp = st->nw;
  const double alpha = st->alpha;
  // shared layout: s_sk[kGrpNW][T + 1] | s_u[T] | partial sums of the warps
  double* s_sk = smem;
  double* s_u = s_sk + kGrpNW * (T + 1);
  double* s_red = s_u + T;
  if (threadIdx.x < nwp) {
    g->s_off[threadIdx.x] = (size_t)((iprev - nwp + (int)threadIdx.x) % slots) * (size_t)n;
    g->s_beta[threadIdx.x] = st->beta[threadIdx.x];
  }
  __syncthreads();
  const size_t coff = (size_t)(iprev % slots) * (size_t)n;
  double* my = s_sk + threadIdx.x;
  const double* wu = s_u + warp * 32;
  const double* lrow = s_sk + lane * (T + 1) + warp * 32;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0, gw = 0.0;
  const int64_t e_lo = g->row_lo * S.nx, e_hi = g->row_hi * S.nx;
  for (int64_t base = e_lo; base < e_hi; base += T) {
    const int64_t e = base + threadIdx.x;
    double un = 0.0;
    if (e < e_hi) {
      const double u0 = vu[e], w0 = vw[e];
      double p = u0, s = w0, q = vm[e], z = vn[e];
#pragma unroll 4
      for (int jj = 0; jj < nwp; ++jj) {
        const size_t o = g->s_off[jj] + e;
        const double bb = g->s_beta[jj];
        const double sv = Sr[o];
        p = fma(bb, Pr[o], p);
        s = fma(bb, sv, s);
        q = fma(bb, Qr[o], q);
        z = fma(bb, Zr[o], z);
        my[jj * (T + 1)] = sv;
      }
      Pr[coff + e] = p;
      Sr[coff + e] = s;
      Qr[coff + e] = q;
      Zr[coff + e] = z;
      const double xn = fma(alpha, p, S.x[e]);
      const double rn = fma(-alpha, s, vr[e]);
      un = fma(-alpha, q, u0);
      const double wn = fma(-alpha, z, w0);
      S.x[e] = xn;
      vr[e] = rn;
      vu[e] = un;
      vw[e] = wn;
      vt[e] = wn - rn;
      g0 = fma(un, rn, g0);
      g1 = fma(un, wn, g1);
      g2 = fma(rn, rn, g2);
      g3 = fma(un, s, g3);
    } else {
      for (int jj = 0; jj < nwp; ++jj) my[jj * (T + 1)] = 0.0;
    }
    s_u[threadIdx.x] = un;
    __syncwarp();
    if (lane < nwp) {
      double c = gw;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) c = fma(wu[t], lrow[t], c);
      gw = c;
    }
    __syncwarp();
  }
  // partial row of the CTA: gamma, delta, rr, <u, s_{i-1}>, window dots
  const int nd = nwp + 4;
  {
    const double a0 = warp_sum(g0), a1 = warp_sum(g1), a2 = warp_sum(g2), a3 = warp_sum(g3);
    if (lane == 0) {
      s_red[warp * nd + 0] = a0;
      s_red[warp * nd + 1] = a1;
      s_red[warp * nd + 2] = a2;
      s_red[warp * nd + 3] = a3;
    }
    if (lane < nwp) s_red[warp * nd + 4 + lane] = gw;
  }
  __syncthreads();
  grp_combine_row(S, g, nd, s_red);
  if (threadIdx.x == 0) {
    // the window dots of iteration i: <u_i, s_k> for the previous window's
    // slots (columns 4..) and the new s_{i-1} (column 3)
    const double* tot = g->s_tot;
    const int i = iprev + 1;
    const int nu = nu_window(i, S.P.mmax, S.P.truncation);
    const int off = nwp + 1 - nu;
    grp_scalar_phase(S, g, i, tot[0], tot[1], tot[2], [&](int jj) {
      const int src = off + jj;
      return src < nwp ? tot[4 + src] : tot[3];
    });
  }
  __syncthreads();
}

// PIPEGCR (Alg. 11), first part of iteration i: the deferred MAXPYs of
// iteration i-1 (p, s, q from u, w, m and the window) into ring slot i-1,
// then x_i, r_i and u_i with alpha_{i-1}; ends at the system's barrier (the
// operator reads the neighbours' u_i next).
__device__ void grp_gcr_advance(const GrpSys& S, GrpCta* g) {
  GrpState* st = &g->st;
  const int64_t n = S.n;
  double* vr = S.ws;
  double* vu = vr + n;
  const double* vw = vu + n;
  const double* vm = vw + n;
  const int slots = S.P.mmax + 1;
  double* Pr = S.ws + 7 * n;
  double* Sr = Pr + (int64_t)slots * n;
  double* Qr = Sr + (int64_t)slots * n;
  const int iprev = st->i;
  const int nwp = st->nw;
  const double alpha = st->alpha;
  if (threadIdx.x < nwp) {
    g->s_off[threadIdx.x] = (size_t)((iprev - nwp + (int)threadIdx.x) % slots) * (size_t)n;
    g->s_beta[threadIdx.x] = st->beta[threadIdx.x];
  }
  __syncthreads();
  const size_t coff = (size_t)(iprev % slots) * (size_t)n;
  #pragma unroll 4
  GRP_ELEMS(S, g, e) {
    const double u0 = vu[e];
    double p = u0, sv = vw[e], q = vm[e];
#pragma unroll 4
    for (int jj = 0; jj < nwp; ++jj) {
      const size_t o = g->s_off[jj] + e;
      const double bb = g->s_beta[jj];
      p = fma(bb, Pr[o], p);
      sv = fma(bb, Sr[o], sv);
      q = fma(bb, Qr[o], q);
    }
    Pr[coff + e] = p;
    Sr[coff + e] = sv;
    Qr[coff + e] = q;
    S.x[e] = fma(alpha, p, S.x[e]);
    vr[e] = fma(-alpha, sv, vr[e]);
    vu[e] = fma(-alpha, q, u0);
  }
  grp_barrier(S, g);
}

// PIPEGCR, second part: w_i = A u_i on the CTA's rows and t = w_i - r_i; the
// iteration's one reduction -- gamma_i = <r_i, w_i>, delta_i = <w_i, w_i>,
// ||r_i||^2 and <w_i, s_k> for the window k = i - nu_i .. i - 1 (transposed
// through shared memory as in the PIPEFCG pass) -- and the scalar phase.
__device__ void grp_gcr_dots(const GrpSys& S, GrpCta* g, double* smem) {
  constexpr int T = kGrpThreads;
  GrpState* st = &g->st;
  const int64_t n = S.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* vr = S.ws;
  const double* vu = vr + n;
  double* vw = (double*)vu + n;
  double* vt = S.ws + 5 * n;
  const int slots = S.P.mmax + 1;
  const double* Sr = S.ws + 7 * n + (int64_t)slots * n;
  const int i = st->i + 1;
  const int nu = nu_window(i, S.P.mmax, S.P.truncation);
  #pragma unroll 2
  GRP_ROWS(S, g, c, ii, j, k) {
    const double wv = grp_row(S, vu, c, ii, j, k);
    vw[c] = wv;
    vt[c] = wv - vr[c];
  }
  if (threadIdx.x < nu) g->s_off[threadIdx.x] = (size_t)((i - nu + (int)threadIdx.x) % slots) * (size_t)n;
  __syncthreads();
  double* s_sk = smem;
  double* s_w = s_sk + kGrpNW * (T + 1);
  double* s_red = s_w + T;
  double* my = s_sk + threadIdx.x;
  const double* ww = s_w + warp * 32;
  const double* lrow = s_sk + lane * (T + 1) + warp * 32;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0, gw = 0.0;
  const int64_t e_lo = g->row_lo * S.nx, e_hi = g->row_hi * S.nx;
  for (int64_t base = e_lo; base < e_hi; base += T) {
    const int64_t e = base + threadIdx.x;
    double wv = 0.0;
    if (e < e_hi) {
      wv = vw[e];
      const double rv = vr[e];
      g0 = fma(rv, wv, g0);
      g1 = fma(wv, wv, g1);
      g2 = fma(rv, rv, g2);
      for (int jj = 0; jj < nu; ++jj) my[jj * (T + 1)] = Sr[g->s_off[jj] + e];
    } else {
      for (int jj = 0; jj < nu; ++jj) my[jj * (T + 1)] = 0.0;
    }
    s_w[threadIdx.x] = wv;
    __syncwarp();
    if (lane < nu) {
      double c = gw;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) c = fma(ww[t], lrow[t], c);
      gw = c;
    }
    __syncwarp();
  }
  const int nd = nu + 4;
  {
    const double a0 = warp_sum(g0), a1 = warp_sum(g1), a2 = warp_sum(g2);
    if (lane == 0) {
      s_red[warp * nd + 0] = a0;
      s_red[warp * nd + 1] = a1;
      s_red[warp * nd + 2] = a2;
      s_red[warp * nd + 3] = 0.0;
    }
    if (lane < nu) s_red[warp * nd + 4 + lane] = gw;
  }
  __syncthreads();
  grp_combine_row(S, g, nd, s_red);
  if (threadIdx.x == 0) {
    const double* tot = g->s_tot;
    grp_scalar_phase(S, g, i, tot[0], tot[1], tot[2], [&](int jj) { return tot[4 + jj]; });
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// PIPEFGMRES (Alg. 15, constant shift sigma, eq. pipefgmresz).  Vectors: r at
// ws, qbar at ws + n, wbar at ws + 2n, the true-residual scratch at ws + 6n,
// then the cycle's p_j, u_j and zbar_j (m each).  Every CTA keeps the
// rotations, g and the last column itself (identical in all CTAs); rank 0
// writes the rotated columns R for the end of the cycle.
// ---------------------------------------------------------------------------

// Column k of H from its dots (hb[j] = <p_j, zbar_k>, j <= k; zz =
// ||zbar_k||^2): hbar and h = hbar + sigma e_k, t = zz - sum hbar^2 (norm
// breakdown if t < 0), hbar_{k+1,k} = sqrt(t), the previous rotations and a
// new one, the least-squares residual estimate |g_{k+1}| and the status.
// Thread 0.
__device__ void grp_gm_column(const GrpSys& S, GrpCta* g, int k, const double* hb, double zz) {
  GrpState* st = &g->st;
  const int m = S.P.mmax;
  double tsum = 0.0;
  for (int j = 0; j <= k; ++j) {
    st->gm_hb[j] = hb[j];
    st->gm_h[j] = hb[j];
    tsum += hb[j] * hb[j];
  }
  st->gm_h[k] = hb[k] + st->sigma;
  const double t = zz - tsum;
  if (!(t >= 0.0)) {
    st->i = k + 1;     // columns 0 .. k-1 are valid
    st->gm_ncols = k;
    st->status = isfinite(t) ? kBreakdown : kNonFinite;
    return;
  }
  const double hsub = sqrt(t);
  st->gm_hb[k + 1] = hsub;
  st->gm_h[k + 1] = hsub;
  st->it += 1;
  st->gm_ncols = k + 1;
  st->i = k + 1;
  double* col = g->s_col;
  for (int j = 0; j <= k + 1; ++j) col[j] = st->gm_h[j];
  for (int j = 0; j < k; ++j) {
    const double a = col[j], b = col[j + 1];
    col[j] = st->gm_cs[j] * a + st->gm_sn[j] * b;
    col[j + 1] = -st->gm_sn[j] * a + st->gm_cs[j] * b;
  }
  const double a = col[k], b = col[k + 1];
  const double rr = hypot(a, b);
  const double c = rr != 0.0 ? a / rr : 1.0, sn = rr != 0.0 ? b / rr : 0.0;
  st->gm_cs[k] = c;
  st->gm_sn[k] = sn;
  col[k] = rr;
  col[k + 1] = 0.0;
  if (g->rank == 0)
    for (int j = 0; j <= k + 1; ++j) S.gm[j * m + k] = col[j];
  st->gm_g[k + 1] = -sn * st->gm_g[k];
  st->gm_g[k] = c * st->gm_g[k];
  const double est = fabs(st->gm_g[k + 1]);
  st->rho = est;
  grp_push_history(S, g, est, nan(""), t, hsub);
  st->gm_inv = hsub != 0.0 ? 1.0 / hsub : 0.0;
  st->gm_k = k + 1;
  if (!isfinite(est)) st->status = kNonFinite;
  else if (est <= st->target || t == 0.0) st->status = kConverged;
  else if (k + 1 == m) st->status = kCycleEnd;
  else if (st->it >= S.P.maxit) st->status = kMaxit;
  else st->status = kRun;
}

// Cycle start: r_0 = b - A x_0 and beta = ||r_0|| (history, target,
// convergence); if the cycle runs, p_0 = r_0 / beta, u_0 = B(p_0), zbar_0 =
// A u_0 - sigma p_0 with the dots of column 0, and column 0.
__device__ void grp_gm_fill(const GrpSys& S, GrpCta* g, double* smem) {
  GrpState* st = &g->st;
  const int64_t n = S.n;
  const int m = S.P.mmax;
  double* r = S.ws;
  double* P0 = S.ws + 7 * n;
  double* U0 = P0 + (int64_t)m * n;
  double* Z0 = U0 + (int64_t)m * n;
  grp_apply(S, g, S.x, r, S.b);
  {
    double acc[1] = {0.0};
    GRP_ELEMS(S, g, e) acc[0] = fma(r[e], r[e], acc[0]);
    grp_sum<1>(S, g, acc, smem);
  }
  if (threadIdx.x == 0) {
    const double beta = sqrt(g->red[0]);
    if (!st->target_set) {
      st->rho0 = beta;
      st->target = fmax(S.P.rtol * beta, S.P.atol);
      st->target_set = 1;
    }
    grp_push_history(S, g, beta, beta, nan(""), nan(""));
    st->rho = beta;
    st->i = 0;
    st->gm_g[0] = beta;
    st->gm_k = 0;
    st->gm_ncols = 0;
    st->gm_inv = beta != 0.0 ? 1.0 / beta : 0.0;
    if (!isfinite(beta)) st->status = kNonFinite;
    else if (beta <= st->target) st->status = kConverged;
    else if (st->it >= S.P.maxit) st->status = kMaxit;
    else st->status = kRun;
  }
  __syncthreads();
  if (st->status != kRun) return;
  const double inv = st->gm_inv;
  GRP_ELEMS(S, g, e) P0[e] = r[e] * inv;
  grp_pc(S, g, P0, U0, nullptr, smem);       // u_0 = B(p_0)
  grp_apply(S, g, U0, Z0, nullptr);          // A u_0
  const double sigma = st->sigma;
  double acc[2] = {0.0, 0.0};
#pragma unroll 4
  GRP_ELEMS(S, g, e) {
    const double pv = P0[e];
    const double zv = fma(-sigma, pv, Z0[e]);
    Z0[e] = zv;
    acc[0] = fma(zv, zv, acc[0]);
    acc[1] = fma(pv, zv, acc[1]);
  }
  grp_sum<2>(S, g, acc, smem);
  if (threadIdx.x == 0) grp_gm_column(S, g, 0, &g->red[1], g->red[0]);
  __syncthreads();
}

// Pass k >= 1: p_k = (zbar_{k-1} - sum_j hbar_{j,k-1} p_j) / hbar_{k,k-1},
// u_k = (qbar - sum_j hbar_{j,k-1} u_j) / hbar_{k,k-1}, zbar_k = (wbar -
// sum_j h_{j,k-1} zbar_j) / hbar_{k,k-1} (reciprocal multiply), with the dots
// <p_j, zbar_k> (j <= k; the p_j read by the MAXPY transposed through shared
// memory as in the PIPEFCG pass) and ||zbar_k||^2, then column k.
__device__ void grp_gm_pass(const GrpSys& S, GrpCta* g, double* smem) {
  constexpr int T = kGrpThreads;
  GrpState* st = &g->st;
  const int64_t n = S.n;
  const int m = S.P.mmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = st->gm_k;
  const double inv = st->gm_inv;
  double* P = S.ws + 7 * n;
  double* U = P + (int64_t)m * n;
  double* Zb = U + (int64_t)m * n;
  const double* qb = S.ws + n;
  const double* wb = S.ws + 2 * n;
  if (threadIdx.x < k) {
    g->s_beta[threadIdx.x] = st->gm_hb[threadIdx.x];
    g->s_h[threadIdx.x] = st->gm_h[threadIdx.x];
  }
  __syncthreads();
  const size_t koff = (size_t)k * (size_t)n, km1 = (size_t)(k - 1) * (size_t)n;
  double* s_sk = smem;
  double* s_z = s_sk + kGrpNW * (T + 1);
  double* s_red = s_z + T;
  double* my = s_sk + threadIdx.x;
  const double* wz = s_z + warp * 32;
  const double* lrow = s_sk + lane * (T + 1) + warp * 32;
  double gz = 0.0, gp = 0.0, gw = 0.0;
  const int64_t e_lo = g->row_lo * S.nx, e_hi = g->row_hi * S.nx;
  for (int64_t base = e_lo; base < e_hi; base += T) {
    const int64_t e = base + threadIdx.x;
    double zk = 0.0;
    if (e < e_hi) {
      double p = Zb[km1 + e], u = qb[e], z = wb[e];
#pragma unroll 4
      for (int j = 0; j < k; ++j) {
        const size_t o = (size_t)j * (size_t)n + e;
        const double pj = P[o];
        p = fma(-g->s_beta[j], pj, p);
        u = fma(-g->s_beta[j], U[o], u);
        z = fma(-g->s_h[j], Zb[o], z);
        my[j * (T + 1)] = pj;
      }
      p *= inv;
      u *= inv;
      zk = z * inv;
      P[koff + e] = p;
      U[koff + e] = u;
      Zb[koff + e] = zk;
      gz = fma(zk, zk, gz);
      gp = fma(p, zk, gp);
    } else {
      for (int j = 0; j < k; ++j) my[j * (T + 1)] = 0.0;
    }
    s_z[threadIdx.x] = zk;
    __syncwarp();
    if (lane < k) {
      double c = gw;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) c = fma(wz[t], lrow[t], c);
      gw = c;
    }
    __syncwarp();
  }
  const int nd = k + 2;     // ||zbar_k||^2, <p_j, zbar_k> for j = 0 .. k
  {
    const double a0 = warp_sum(gz), a1 = warp_sum(gp);
    if (lane == 0) {
      s_red[warp * nd + 0] = a0;
      s_red[warp * nd + 1 + k] = a1;
    }
    if (lane < k) s_red[warp * nd + 1 + lane] = gw;
  }
  __syncthreads();
  grp_combine_row(S, g, nd, s_red);
  if (threadIdx.x == 0) grp_gm_column(S, g, k, g->s_tot + 1, g->s_tot[0]);
  __syncthreads();
}

// qbar = B(zbar_k), wbar = A qbar (the next pass's inputs).
__device__ void grp_gm_precondition(const GrpSys& S, GrpCta* g, double* smem, int k) {
  const int64_t n = S.n;
  const int m = S.P.mmax;
  const double* Zk = S.ws + 7 * n + 2 * (int64_t)m * n + (int64_t)k * n;
  double* qb = S.ws + n;
  double* wb = S.ws + 2 * n;
  grp_pc(S, g, Zk, qb, nullptr, smem);
  grp_apply(S, g, qb, wb, nullptr);
}

// End of a cycle: back substitution R y = g on the valid columns (every CTA,
// from the columns rank 0 wrote), x = x_0 + sum_j y_j u_j; ends at the
// system's barrier (x then feeds an operator).
__device__ void grp_gm_end_cycle(const GrpSys& S, GrpCta* g) {
  GrpState* st = &g->st;
  const int nc = st->gm_ncols;
  if (nc == 0) return;
  const int m = S.P.mmax;
  const int64_t n = S.n;
  grp_barrier(S, g);
  if (threadIdx.x == 0) {
    for (int j = nc - 1; j >= 0; --j) {
      double s = st->gm_g[j];
      for (int l = j + 1; l < nc; ++l) s -= __ldcg(&S.gm[j * m + l]) * g->s_y[l];
      g->s_y[j] = s / __ldcg(&S.gm[j * m + j]);
    }
  }
  __syncthreads();
  const double* U = S.ws + 7 * n + (int64_t)m * n;
#pragma unroll 4
  GRP_ELEMS(S, g, e) {
    double v = S.x[e];
    for (int j = 0; j < nc; ++j) v = fma(g->s_y[j], U[(size_t)j * (size_t)n + e], v);
    S.x[e] = v;
  }
  grp_barrier(S, g);
}

// The shift sigma when none is given: 10 power iterations on v -> A B(v)
// from v = b / ||b|| (sigma = ||A B(v)|| at the last step).
__device__ void grp_gm_sigma(const GrpSys& S, GrpCta* g, double* smem) {
  GrpState* st = &g->st;
  if (!isnan(S.P.sigma)) {
    if (threadIdx.x == 0) st->sigma = S.P.sigma;
    __syncthreads();
    return;
  }
  const int64_t n = S.n;
  double* v = S.ws;
  double* t = S.ws + 6 * n;
  double* q = S.ws + n;
  double nrm = st->bnorm;
  {
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    GRP_ELEMS(S, g, e) v[e] = S.b[e] * inv;
  }
  for (int it = 0; it < 10; ++it) {
    grp_pc(S, g, v, t, nullptr, smem);
    grp_apply(S, g, t, q, nullptr);
    double acc[1] = {0.0};
    GRP_ELEMS(S, g, e) acc[0] = fma(q[e], q[e], acc[0]);
    grp_sum<1>(S, g, acc, smem);
    nrm = sqrt(g->red[0]);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    GRP_ELEMS(S, g, e) v[e] = q[e] * inv;
    __syncthreads();
  }
  if (threadIdx.x == 0) st->sigma = nrm;
  __syncthreads();
}

// Pipeline fill (Alg. 8 / Alg. 11, before the loop) from the current x.
__device__ void grp_fill(const GrpSys& S, GrpCta* g, double* smem) {
  GrpState* st = &g->st;
  const int64_t n = S.n;
  double* vr = S.ws;
  double* vu = vr + n;
  double* vw = vu + n;
  double* vm = vw + n;
  double* vn = vm + n;
  double* s_red = smem;
  const bool gcr = S.P.method == PFK_PIPEGCR;
  grp_apply(S, g, S.x, vr, S.b);             // r_0 = b - A x_0
  grp_pc(S, g, vr, vu, nullptr, s_red);      // u_0 = B(r_0) = p_0
  grp_apply(S, g, vu, vw, nullptr);          // w_0 = A p_0 (Alg. 11: s_0)
  grp_pc(S, g, vw, vm, nullptr, s_red);      // m_0 = B(w_0) (Alg. 11: q_0)
  if (!gcr) grp_apply(S, g, vm, vn, nullptr);   // n_0 = A m_0
  // Alg. 8: gamma_0 = <u_0, r_0>, eta_0 = delta_0 = <u_0, w_0>;
  // Alg. 11: gamma_0 = <r_0, s_0>, eta_0 = <s_0, s_0>; and ||r_0||^2
  double acc[3] = {0.0, 0.0, 0.0};
  #pragma unroll 4
  GRP_ELEMS(S, g, e) {
    const double a = gcr ? vw[e] : vu[e];
    acc[0] = fma(a, vr[e], acc[0]);
    acc[1] = fma(a, vw[e], acc[1]);
    acc[2] = fma(vr[e], vr[e], acc[2]);
  }
  grp_sum<3>(S, g, acc, s_red);
  if (threadIdx.x == 0) {
    const GrpParams& P = S.P;
    const double gamma = g->red[0], eta = g->red[1], rr = g->red[2];
    const double rho = grp_rho(P, gamma, rr);
    if (!st->target_set) {
      st->rho0 = rho;
      st->target = fmax(P.rtol * rho, P.atol);
      st->target_set = 1;
    }
    const double al = eta != 0.0 ? gamma / eta : nan("");
    grp_push_history(S, g, rho, sqrt(rr), eta, al);
    st->rho = rho;
    st->gamma = gamma;
    st->eta = eta;
    st->alpha = al;
    st->i = 0;
    st->nw = 0;
    st->eta_ring[0] = eta;
    if (!isfinite(rho)) st->status = kNonFinite;
    else if (rho <= st->target) st->status = kConverged;
    else if (eta <= 0.0) st->status = kFillBreakdown;
    else if (st->it >= P.maxit) st->status = kMaxit;
    else st->status = kRun;
  }
  __syncthreads();
}

// ||b - A x||_2 into g->red[0] (x complete on the group).
__device__ void grp_true_residual(const GrpSys& S, GrpCta* g, double* smem) {
  double* tmp = S.ws + 6 * S.n;
  grp_apply(S, g, S.x, tmp, S.b);
  double acc[1] = {0.0};
  #pragma unroll 4
  GRP_ELEMS(S, g, e) acc[0] = fma(tmp[e], tmp[e], acc[0]);
  grp_sum<1>(S, g, acc, smem);
  if (threadIdx.x == 0) g->red[0] = sqrt(g->red[0]);
  __syncthreads();
}

// What follows a cycle that stopped (status != kRun), as in the
// single-system driver: at convergence the true residual decides between
// acceptance and a residual replacement (restart with the target tightened by
// 0.5 goal / ||b - A x||); a norm breakdown restarts unless it persisted.
__device__ void grp_after_cycle(const GrpSys& S, GrpCta* g, double* smem) {
  GrpState* st = &g->st;
  const GrpParams& P = S.P;
  const int status = st->status;
  if (status == kConverged) {
    grp_true_residual(S, g, smem);
    if (threadIdx.x == 0) {
      const double rt = g->red[0];
      st->rtrue = rt;
      if (!P.true_check || rt <= st->goal) {
        st->result = PFK_OK;
        st->phase = kGDone;
      } else if (st->restarts >= P.max_restarts) {
        st->result = PFK_ERR_NOT_CONVERGED;
        st->phase = kGDone;
      } else {
        st->replacements += 1;
        st->restarts += 1;
        st->target *= 0.5 * st->goal / rt;
        st->prev_bd = 0;
        st->phase = kGFill;
      }
    }
  } else if (status == kBreakdown) {
    if (threadIdx.x == 0) {
      st->breakdowns += 1;
      if ((st->i <= 1 && st->prev_bd) || st->restarts >= P.max_restarts) {
        st->result = PFK_ERR_BREAKDOWN;
        st->phase = kGDone;
      } else {
        st->restarts += 1;
        st->prev_bd = 1;
        st->phase = kGFill;
      }
    }
  } else if (threadIdx.x == 0) {
    st->result = status == kMaxit ? PFK_ERR_NOT_CONVERGED : PFK_ERR_BREAKDOWN;
    st->phase = kGDone;
  }
  __syncthreads();
}

// One launch: CTA blockIdx.x serves system blk[blockIdx.x].x as rank
// blk[blockIdx.x].y of its group and advances it by at most `iters` steps.
__global__ void __launch_bounds__(kGrpThreads, 3)
    grouped_pipefcg(const GrpSys* __restrict__ systems, const int2* __restrict__ blk, int iters) {
  extern __shared__ double smem[];
  __shared__ GrpCta g;
  const int2 me = blk[blockIdx.x];
  const GrpSys S = systems[me.x];
  {
    const unsigned long long* src = (const unsigned long long*)S.state;
    unsigned long long* dst = (unsigned long long*)&g.st;
    for (int w = threadIdx.x; w < (int)(sizeof(GrpState) / 8); w += kGrpThreads) dst[w] = __ldcg(src + w);
  }
  if (threadIdx.x == 0) {
    g.rank = me.y;
    g.nblk = S.nblk;
    g.par = 0;
    g.abort = 0;
    const int64_t rows = (int64_t)S.ny * S.nz;
    g.row_lo = rows * me.y / S.nblk;
    g.row_hi = rows * (me.y + 1) / S.nblk;
  }
  __syncthreads();
  GrpState* st = &g.st;
  if (st->phase == kGDone) return;
  const int64_t n = S.n;
  if (st->phase == kGStart) {
    double acc[1] = {0.0};
    GRP_ELEMS(S, (&g), e) acc[0] = fma(S.b[e], S.b[e], acc[0]);
    grp_sum<1>(S, &g, acc, smem);
    if (threadIdx.x == 0) {
      st->bnorm = sqrt(g.red[0]);
      st->goal = fmax(S.P.rtol * st->bnorm, S.P.atol);
      st->rtrue = nan("");
      st->phase = kGFill;
    }
    __syncthreads();
    if (S.P.method == PFK_PIPEFGMRES) grp_gm_sigma(S, &g, smem);
  }
  for (int step = 0; step < iters && st->phase != kGDone && !g.abort; ++step) {
    if (threadIdx.x == 0) st->steps += 1;
    if (S.P.method == PFK_PIPEFGMRES) {
      // a step: the cycle start with column 0, or pass k; then B and A for
      // the next pass, or the end of the cycle
      if (st->phase == kGFill) grp_gm_fill(S, &g, smem);
      else grp_gm_pass(S, &g, smem);
      if (st->status == kRun) {
        grp_gm_precondition(S, &g, smem, st->gm_k - 1);
        if (threadIdx.x == 0) st->phase = kGIter;
        __syncthreads();
        continue;
      }
      if (st->status != kNonFinite) grp_gm_end_cycle(S, &g);
      if (st->status == kCycleEnd) {
        if (threadIdx.x == 0) {
          st->prev_bd = 0;
          st->phase = kGFill;
        }
        __syncthreads();
      } else {
        grp_after_cycle(S, &g, smem);
      }
      continue;
    }
    if (st->phase == kGFill) {
      grp_fill(S, &g, smem);
      if (threadIdx.x == 0 && st->status == kRun) st->phase = kGIter;
      __syncthreads();
      if (st->status != kRun) grp_after_cycle(S, &g, smem);
      continue;
    }
    const bool gcr = S.P.method == PFK_PIPEGCR;
    if (gcr) {
      grp_gcr_advance(S, &g);
      grp_gcr_dots(S, &g, smem);
    } else {
      grp_pass(S, &g, smem);
    }
    if (st->status != kRun) {
      grp_after_cycle(S, &g, smem);
      continue;
    }
    double* vu = S.ws + n;
    double* vm = S.ws + 3 * n;
    double* vn = S.ws + 4 * n;
    double* vt = S.ws + 5 * n;
    grp_pc(S, &g, vt, vm, vu, smem);        // m_i = u_i + B(w_i - r_i)
    if (!gcr) grp_apply(S, &g, vm, vn, nullptr);   // n_i = A m_i (Alg. 8)
  }
  if (st->phase == kGDone && !g.abort && (isnan(st->rtrue) || st->result != PFK_OK)) {
    grp_true_residual(S, &g, smem);
    if (threadIdx.x == 0) st->rtrue = g.red[0];
    __syncthreads();
  }
  if (g.rank != 0) return;
  if (threadIdx.x == 0 && (g.abort || grp_ld_acquire(&S.bar->abort))) {
    st->phase = kGDone;
    st->result = PFK_ERR_TIMEOUT;
  }
  __syncthreads();
  {
    const unsigned long long* src = (const unsigned long long*)&g.st;
    unsigned long long* dst = (unsigned long long*)S.state;
    for (int w = threadIdx.x; w < (int)(sizeof(GrpState) / 8); w += kGrpThreads) dst[w] = src[w];
  }
}

size_t grp_smem_bytes() {
  return ((size_t)kGrpNW * (kGrpThreads + 1) + kGrpThreads + (size_t)(kGrpThreads / 32) * kGrpNd) * sizeof(double);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host: slots, admission and launches
// ---------------------------------------------------------------------------

bool group_method_eligible(const pfk_pc_desc* pcd, const pfk_solve_params* prm, const char** why) {
  const char* w = nullptr;
  if (!prm || (prm->method != PFK_PIPEFCG && prm->method != PFK_PIPEGCR && prm->method != PFK_PIPEFGMRES))
    w = "the grouped solve runs PFK_PIPEFCG, PFK_PIPEGCR or PFK_PIPEFGMRES";
  else if (prm->mmax < 1 || prm->mmax > PFK_MAX_MMAX) w = "mmax out of range";
  else if (pcd && !(pcd->kind == PFK_PC_NONE || pcd->kind == PFK_PC_JACOBI ||
                    (pcd->kind == PFK_PC_INNER_PCG && (pcd->precision == PFK_FP64 || pcd->precision == PFK_FP32) &&
                     pcd->inner_iters >= 1 && pcd->inner_iters <= kGrpMaxInner)))
    w = "the grouped solve supports NONE, JACOBI and FP64 / FP32 INNER_PCG preconditioners";
  if (why) *why = w;
  return w == nullptr;
}

bool group_eligible(const pfk_operator* op, const pfk_pc_desc* pcd, const pfk_solve_params* prm, const char** why) {
  if (!op || !op->d || op->rowptr) {
    if (why) *why = "the grouped solve needs matrix-free stencil operators";
    return false;
  }
  if (op->n > INT32_MAX) {
    if (why) *why = "system too large for the grouped solve";
    return false;
  }
  return group_method_eligible(pcd, prm, why);
}

// CTAs of a system at about `cells` cells each, at most kGrpMaxCtas and at
// most one per x-row (a group's CTAs own whole rows).
static int group_ctas_cells(int64_t n, int64_t rows, int64_t cells) {
  int64_t c = (n + cells - 1) / cells;
  c = std::min<int64_t>(c, kGrpMaxCtas);
  c = std::min<int64_t>(c, rows);
  return (int)std::max<int64_t>(c, 1);
}

int group_ctas(int64_t n, int64_t rows, int requested) {
  if (requested > 0) return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)requested, kGrpMaxCtas, rows}));
  return group_ctas_cells(n, rows, kGrpCellsPerCta);
}

// Cells per CTA chosen by timing (ctas_per_system = -1), per device, size
// bucket (ceil log2 of the batch's largest system), method and
// preconditioner (kind, inner iterations, precision); kept for the process.
static std::mutex g_tuned_mu;
static std::map<std::tuple<int, int, int, int, int, int>, int64_t> g_tuned_cells;

struct GroupRunner::Impl {
  pfk_context* ctx = nullptr;
  cudaStream_t st = nullptr;
  int max_slots = 0;
  int max_ctas = 0;         // CTAs the GPU holds at once (the cooperative launch's limit)
  int used_ctas = 0;
  GrpSys* dsys = nullptr;
  GrpState* dstate = nullptr;
  GrpBar* dbar = nullptr;
  int2* dblk = nullptr;
  GrpState* hstate = nullptr;   // pinned
  std::vector<GrpSys> hsys;
  std::vector<int> active;      // slot -> 1 if active
  std::vector<void*> mem;       // slot -> workspace allocation
  std::vector<int2> hblk;
  bool map_dirty = true;
  int launches = 0;
  double kernel_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

GroupRunner::GroupRunner() : m_(new Impl) {}

GroupRunner::~GroupRunner() {
  Impl& M = *m_;
  for (size_t s = 0; s < M.mem.size(); ++s)
    if (M.mem[s]) cudaFreeAsync(M.mem[s], M.st);
  if (M.st) cudaStreamSynchronize(M.st);
  if (M.dsys) cudaFree(M.dsys);
  if (M.dstate) cudaFree(M.dstate);
  if (M.dbar) cudaFree(M.dbar);
  if (M.dblk) cudaFree(M.dblk);
  if (M.hstate) cudaFreeHost(M.hstate);
  if (M.ev0) cudaEventDestroy(M.ev0);
  if (M.ev1) cudaEventDestroy(M.ev1);
  delete m_;
}

pfk_status GroupRunner::init(pfk_context* ctx, int max_slots) {
  Impl& M = *m_;
  M.ctx = ctx;
  M.st = ctx->stream;
  cudaSetDevice(ctx->device);
  const size_t smem = grp_smem_bytes();
  PFK_CUDA(ctx, cudaFuncSetAttribute(grouped_pipefcg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PFK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grouped_pipefcg, kGrpThreads, smem));
  if (per_sm < 1) {
    set_error(ctx, "the grouped kernel does not fit on an SM");
    return PFK_ERR_INVALID;
  }
  M.max_ctas = per_sm * ctx->num_sms;
  M.max_slots = max_slots > 0 ? max_slots : M.max_ctas;
  PFK_CUDA(ctx, cudaMalloc((void**)&M.dsys, sizeof(GrpSys) * M.max_slots));
  PFK_CUDA(ctx, cudaMalloc((void**)&M.dstate, sizeof(GrpState) * M.max_slots));
  PFK_CUDA(ctx, cudaMalloc((void**)&M.dbar, sizeof(GrpBar) * M.max_slots));
  PFK_CUDA(ctx, cudaMalloc((void**)&M.dblk, sizeof(int2) * M.max_ctas));
  PFK_CUDA(ctx, cudaMallocHost((void**)&M.hstate, sizeof(GrpState) * M.max_slots));
  PFK_CUDA(ctx, cudaEventCreate(&M.ev0));
  PFK_CUDA(ctx, cudaEventCreate(&M.ev1));
  M.hsys.assign(M.max_slots, GrpSys{});
  M.active.assign(M.max_slots, 0);
  M.mem.assign(M.max_slots, nullptr);
  return PFK_OK;
}

int GroupRunner::capacity_ctas() const { return m_->max_ctas; }
int GroupRunner::free_ctas() const { return m_->max_ctas - m_->used_ctas; }
int GroupRunner::launches() const { return m_->launches; }
double GroupRunner::kernel_ms() const { return m_->kernel_ms; }
bool GroupRunner::any_active() const { return m_->used_ctas > 0; }

int64_t GroupRunner::workspace_bytes(int64_t n, int mmax, int nblk) {
  const int64_t slots = mmax + 1;
  return (int64_t)sizeof(double) *
             ((7 + 4 * slots) * n + 4 * n + 2 * (int64_t)nblk * kGrpNd + (int64_t)(mmax + 1) * mmax) +
         256;
}

pfk_status GroupRunner::admit(const pfk_operator* op, const pfk_pc_desc* pcd, const pfk_solve_params* prm,
                              const double* b_dev, double* x_dev, int nblk, double* hist_dev, int hist_cap,
                              int* slot_out) {
  Impl& M = *m_;
  pfk_context* ctx = M.ctx;
  *slot_out = -1;
  const char* why = nullptr;
  if (!group_eligible(op, pcd, prm, &why)) {
    set_error(ctx, why);
    return PFK_ERR_INVALID;
  }
  if (nblk < 1 || nblk > kGrpMaxCtas) {
    set_error(ctx, "CTAs per system out of range");
    return PFK_ERR_INVALID;
  }
  if (nblk > M.max_ctas - M.used_ctas) return PFK_ERR_BUSY;
  int slot = -1;
  for (int s = 0; s < M.max_slots; ++s)
    if (!M.active[s]) {
      slot = s;
      break;
    }
  if (slot < 0) return PFK_ERR_BUSY;
  const int64_t n = op->n;
  const bool fp32 = pcd && pcd->kind == PFK_PC_INNER_PCG && pcd->precision == PFK_FP32;
  if (fp32) {
    const pfk_status cs = ensure_reduced_copies(const_cast<pfk_operator*>(op), PFK_FP32);
    if (cs != PFK_OK) return cs;
  }
  void* mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, workspace_bytes(n, prm->mmax, nblk), M.st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    set_error(ctx, "out of device memory for the grouped solve's workspace");
    return PFK_ERR_OOM;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocAsync (grouped workspace)");
  GrpSys S{};
  S.nx = op->nx; S.ny = op->ny; S.nz = op->nz; S.ndim = op->ndim; S.n = n;
  S.d = op->d; S.kx = op->kx; S.ky = op->ky; S.kz = op->kz; S.dinv = op->dinv;
  S.d32 = op->d32; S.kx32 = op->kx32; S.ky32 = op->ky32; S.kz32 = op->kz32; S.dinv32 = op->dinv32;
  S.a0 = op->adv[0]; S.a1 = op->adv[1]; S.a2 = op->adv[2];
  S.u0 = op->upw[0]; S.u1 = op->upw[1]; S.u2 = op->upw[2];
  S.adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
  S.nblk = nblk;
  S.b = b_dev;
  S.x = x_dev;
  S.ws = (double*)mem;
  S.pcws = S.ws + (7 + 4 * (int64_t)(prm->mmax + 1)) * n;
  S.part = S.pcws + 4 * n;
  S.gm = S.part + 2 * (int64_t)nblk * kGrpNd;
  S.hist = hist_dev;
  S.hist_cap = hist_dev ? hist_cap : 0;
  GrpParams& P = S.P;
  P.method = prm->method;
  P.mmax = prm->mmax; P.truncation = prm->truncation; P.norm = prm->norm; P.maxit = prm->maxit;
  P.max_restarts = prm->max_restarts; P.true_check = prm->true_residual_check;
  P.rtol = prm->rtol; P.atol = prm->atol;
  P.pc_kind = pcd ? pcd->kind : PFK_PC_NONE;
  P.pc_inner = pcd ? pcd->inner_iters : 0;
  P.pc_fp32 = fp32 ? 1 : 0;
  P.sigma = prm->sigma;
  P.bar_timeout_ns = prm->barrier_timeout_us == 0 ? 2000000000LL
                     : prm->barrier_timeout_us < 0 ? 0LL
                                                   : (long long)prm->barrier_timeout_us * 1000LL;
  S.state = M.dstate + slot;
  S.bar = M.dbar + slot;
  GrpState s0{};
  s0.phase = kGStart;
  s0.status = kRun;
  s0.rtrue = NAN;
  s0.sigma = NAN;
  M.hsys[slot] = S;
  M.hstate[slot] = s0;
  PFK_CUDA(ctx, cudaMemcpyAsync(M.dsys + slot, &M.hsys[slot], sizeof(GrpSys), cudaMemcpyHostToDevice, M.st));
  PFK_CUDA(ctx, cudaMemcpyAsync(M.dstate + slot, &M.hstate[slot], sizeof(GrpState), cudaMemcpyHostToDevice, M.st));
  PFK_CUDA(ctx, cudaMemsetAsync(M.dbar + slot, 0, sizeof(GrpBar), M.st));
  M.mem[slot] = mem;
  M.active[slot] = 1;
  M.used_ctas += nblk;
  M.map_dirty = true;
  *slot_out = slot;
  return PFK_OK;
}

pfk_status GroupRunner::step(int iters) {
  Impl& M = *m_;
  pfk_context* ctx = M.ctx;
  if (M.used_ctas == 0) return PFK_OK;
  if (M.map_dirty) {
    M.hblk.clear();
    for (int s = 0; s < M.max_slots; ++s)
      if (M.active[s])
        for (int q = 0; q < M.hsys[s].nblk; ++q) M.hblk.push_back(make_int2(s, q));
    PFK_CUDA(ctx, cudaMemcpyAsync(M.dblk, M.hblk.data(), sizeof(int2) * M.hblk.size(), cudaMemcpyHostToDevice,
                                  M.st));
    M.map_dirty = false;
  }
  const int grid = (int)M.hblk.size();
  const GrpSys* a0 = M.dsys;
  const int2* a1 = M.dblk;
  int a2 = iters;
  void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2};
  PFK_CUDA(ctx, cudaEventRecord(M.ev0, M.st));
  PFK_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)grouped_pipefcg, dim3(grid), dim3(kGrpThreads), args,
                                            grp_smem_bytes(), M.st));
  PFK_CUDA(ctx, cudaEventRecord(M.ev1, M.st));
  int hi = 0;
  for (int s = 0; s < M.max_slots; ++s)
    if (M.active[s]) hi = s + 1;
  PFK_CUDA(ctx, cudaMemcpyAsync(M.hstate, M.dstate, sizeof(GrpState) * hi, cudaMemcpyDeviceToHost, M.st));
  PFK_CUDA(ctx, cudaStreamSynchronize(M.st));
  float ms = 0.f;
  PFK_CUDA(ctx, cudaEventElapsedTime(&ms, M.ev0, M.ev1));
  M.kernel_ms += ms;
  M.launches += 1;
  return PFK_OK;
}

bool GroupRunner::done(int slot) const {
  const Impl& M = *m_;
  return M.active[slot] && M.hstate[slot].phase == kGDone;
}

void GroupRunner::info(int slot, pfk_solve_info* I) const {
  const Impl& M = *m_;
  const GrpState& s = M.hstate[slot];
  std::memset(I, 0, sizeof(*I));
  I->status = s.phase == kGDone ? s.result : PFK_PENDING;
  I->iterations = s.it;
  I->restarts = s.restarts;
  I->breakdowns = s.breakdowns;
  I->replacements = s.replacements;
  I->history_len = s.hist_len;
  I->rho0 = s.rho0;
  I->rho_final = s.rho;
  I->rnorm_true = s.rtrue;
  I->bnorm = s.bnorm;
  I->pass_launches = M.hsys[slot].nblk;
}

void GroupRunner::release(int slot) {
  Impl& M = *m_;
  if (!M.active[slot]) return;
  cudaFreeAsync(M.mem[slot], M.st);
  M.mem[slot] = nullptr;
  M.active[slot] = 0;
  M.used_ctas -= M.hsys[slot].nblk;
  M.map_dirty = true;
}

}  // namespace pfk

using namespace pfk;

extern "C" pfk_status pfk_solve_grouped(pfk_context* ctx, int nsys, const pfk_operator* const* ops,
                                        const pfk_pc_desc* pcd, const pfk_solve_params* prm, const double* const* b,
                                        double* const* x, int ptrs_on_device, int ctas_per_system,
                                        pfk_solve_info* infos) {
  if (!ctx || !ops || !prm || !b || !x || nsys <= 0) {
    set_error(ctx, "invalid argument");
    return PFK_ERR_INVALID;
  }
  if (ctas_per_system < -1 || ctas_per_system > kGrpMaxCtas) {
    set_error(ctx, "ctas_per_system must be -1 (tuned), 0 (automatic) or 1..64");
    return PFK_ERR_INVALID;
  }
  for (int j = 0; j < nsys; ++j) {
    const char* why = nullptr;
    if (!group_eligible(ops[j], pcd, prm, &why)) {
      set_error(ctx, why);
      return PFK_ERR_INVALID;
    }
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  GroupRunner R;
  pfk_status ps = R.init(ctx, 0);
  if (ps != PFK_OK) return ps;
  std::vector<int> nblk(nsys);
  auto rows_of = [&](int j) { return (int64_t)ops[j]->ny * ops[j]->nz; };
  for (int j = 0; j < nsys; ++j) {
    nblk[j] = group_ctas(ops[j]->n, rows_of(j), ctas_per_system > 0 ? ctas_per_system : 0);
    if (nblk[j] > R.capacity_ctas()) {
      set_error(ctx, "a system needs more CTAs than the GPU holds at once");
      return PFK_ERR_INVALID;
    }
  }
  // device copies of host x / b, and the history
  const bool host = !ptrs_on_device;
  const int hcap = prm->history ? prm->history_capacity : 0;
  int64_t ntot = 0;
  for (int j = 0; j < nsys; ++j) ntot += ops[j]->n;
  char* arena = nullptr;
  const size_t bytes = sizeof(double) * ((host ? 2 * ntot : 0) + (int64_t)nsys * hcap * PFK_HISTORY_FIELDS) + 64;
  PFK_CUDA(ctx, cudaMallocAsync((void**)&arena, bytes, st));
  struct Free {
    char* p; cudaStream_t s;
    ~Free() { if (p) { cudaFreeAsync(p, s); cudaStreamSynchronize(s); } }
  } guard{arena, st};
  std::vector<const double*> bd(nsys);
  std::vector<double*> xd(nsys);
  double* dhist = (double*)arena + (host ? 2 * ntot : 0);
  {
    int64_t off = 0;
    for (int j = 0; j < nsys; ++j) {
      const int64_t n = ops[j]->n;
      if (host) {
        double* xb = (double*)arena + 2 * off;
        PFK_CUDA(ctx, cudaMemcpyAsync(xb, x[j], n * sizeof(double), cudaMemcpyHostToDevice, st));
        PFK_CUDA(ctx, cudaMemcpyAsync(xb + n, b[j], n * sizeof(double), cudaMemcpyHostToDevice, st));
        xd[j] = xb;
        bd[j] = xb + n;
        off += n;
      } else {
        xd[j] = x[j];
        bd[j] = b[j];
      }
    }
  }
  if (hcap) PFK_CUDA(ctx, cudaMemsetAsync(dhist, 0xff, sizeof(double) * (size_t)nsys * hcap * PFK_HISTORY_FIELDS, st));
  if (ctas_per_system == -1) {
    // tuned group size: per candidate, the systems that fit one launch run
    // their start and fill, then two timed steps; x is restored afterwards
    int64_t nmax = 0;
    for (int j = 0; j < nsys; ++j) nmax = std::max(nmax, ops[j]->n);
    const auto key = std::make_tuple(ctx->device, (int)std::ceil(std::log2((double)std::max<int64_t>(nmax, 2))),
                                     (int)prm->method, pcd ? (int)pcd->kind : 0, pcd ? (int)pcd->inner_iters : 0,
                                     pcd ? (int)pcd->precision : 0);
    int64_t cells = 0;
    {
      std::lock_guard<std::mutex> lk(g_tuned_mu);
      auto f = g_tuned_cells.find(key);
      if (f != g_tuned_cells.end()) cells = f->second;
    }
    if (cells == 0) {
      double* xsave = nullptr;
      PFK_CUDA(ctx, cudaMallocAsync((void**)&xsave, sizeof(double) * (size_t)ntot, st));
      struct FreeX {
        double* p; cudaStream_t s;
        ~FreeX() { if (p) cudaFreeAsync(p, s); }
      } xguard{xsave, st};
      {
        int64_t off = 0;
        for (int j = 0; j < nsys; ++j) {
          PFK_CUDA(ctx, cudaMemcpyAsync(xsave + off, xd[j], ops[j]->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
          off += ops[j]->n;
        }
      }
      double best = -1.0;
      for (int64_t cand : {2048, 4096, 8192, 16384}) {
        GroupRunner T;
        ps = T.init(ctx, 0);
        if (ps != PFK_OK) return ps;
        std::vector<int> slots;
        double work = 0.0;
        for (int j = 0; j < nsys; ++j) {
          const int c = group_ctas_cells(ops[j]->n, rows_of(j), cand);
          if (c > T.free_ctas()) break;
          int sl = -1;
          ps = T.admit(ops[j], pcd, prm, bd[j], xd[j], c, nullptr, 0, &sl);
          if (ps != PFK_OK) return ps;
          slots.push_back(sl);
          work += (double)ops[j]->n;
        }
        if (slots.empty()) continue;
        if ((ps = T.step(1)) != PFK_OK) return ps;
        const double t0 = T.kernel_ms();
        if ((ps = T.step(2)) != PFK_OK) return ps;
        const double rate = work / std::max(T.kernel_ms() - t0, 1e-6);
        if (rate > best) {
          best = rate;
          cells = cand;
        }
        for (int sl : slots) T.release(sl);
        int64_t off = 0;
        for (int j = 0; j < nsys; ++j) {
          PFK_CUDA(ctx, cudaMemcpyAsync(xd[j], xsave + off, ops[j]->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
          off += ops[j]->n;
        }
      }
      PFK_CUDA(ctx, cudaStreamSynchronize(st));
      if (cells == 0) cells = kGrpCellsPerCta;
      std::lock_guard<std::mutex> lk(g_tuned_mu);
      g_tuned_cells[key] = cells;
    }
    for (int j = 0; j < nsys; ++j) nblk[j] = group_ctas_cells(ops[j]->n, rows_of(j), cells);
  }
  // admission in the given order; iterations chunked so that finished
  // systems make room for the next ones
  std::vector<int> slot_of(nsys, -1), state(nsys, 0);   // 0 queued, 1 active, 2 done
  std::vector<pfk_solve_info> out(nsys);
  int next = 0, finished = 0;
  const int iters = 8;
  while (finished < nsys) {
    while (next < nsys && nblk[next] <= R.free_ctas()) {
      int s = -1;
      ps = R.admit(ops[next], pcd, prm, bd[next], xd[next], nblk[next],
                   hcap ? dhist + (size_t)next * hcap * PFK_HISTORY_FIELDS : nullptr, hcap, &s);
      if (ps == PFK_ERR_BUSY) break;
      if (ps != PFK_OK) return ps;
      slot_of[next] = s;
      state[next] = 1;
      ++next;
    }
    ps = R.step(iters);
    if (ps != PFK_OK) return ps;
    for (int j = 0; j < nsys; ++j)
      if (state[j] == 1 && R.done(slot_of[j])) {
        R.info(slot_of[j], &out[j]);
        R.release(slot_of[j]);
        state[j] = 2;
        ++finished;
      }
  }
  if (host)
    for (int j = 0; j < nsys; ++j)
      PFK_CUDA(ctx, cudaMemcpyAsync(x[j], xd[j], ops[j]->n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (hcap)
    PFK_CUDA(ctx, cudaMemcpyAsync(prm->history, dhist, sizeof(double) * (size_t)nsys * hcap * PFK_HISTORY_FIELDS,
                                  cudaMemcpyDeviceToHost, st));
  PFK_CUDA(ctx, cudaStreamSynchronize(st));
  pfk_status first = PFK_OK;
  for (int j = 0; j < nsys; ++j) {
    out[j].time_ms = R.kernel_ms();
    out[j].kernel_launches = R.launches();
    if (first == PFK_OK && out[j].status != PFK_OK) first = (pfk_status)out[j].status;
    if (infos) infos[j] = out[j];
  }
  if (first == PFK_ERR_TIMEOUT) set_error(ctx, "a group-barrier wait of the grouped kernel timed out");
  else if (first != PFK_OK) set_error(ctx, "at least one system of the batch did not converge");
  return first;
}
