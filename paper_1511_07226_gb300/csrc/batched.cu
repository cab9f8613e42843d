// Batched PIPEFCG: many independent stencil systems in one persistent launch.
//
// Each thread block owns one system for the whole solve: pipeline fill
// (Alg. 8, before the loop), iterations (the same fused pass as the
// single-system kernel: deferred MAXPYs, advance, window dots transposed
// through shared memory), the preconditioner (Jacobi or inner Jacobi-PCG,
// Alg. 3, FP64 or FP32) and the operator, restarts on norm breakdown and the
// true-residual check (residual replacement) -- all with block-level
// reductions and __syncthreads, because the whole system belongs to the
// block.  Blocks take systems from an atomic work counter, largest first, and
// never wait for one another, so there is no grid barrier and nothing to time
// out.  A system's arithmetic does not depend on the rest of the batch.
#include "pfk_internal.cuh"
#include "solver.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <vector>

namespace pfk {

pfk_status ensure_reduced_copies(pfk_operator* op, int precision);

struct BatchSys {
  int nx, ny, nz, ndim;
  int64_t n;
  const double* d;
  const double* kx;
  const double* ky;
  const double* kz;
  const double* dinv;
  const float* d32;
  const float* kx32;
  const float* ky32;
  const float* kz32;
  const float* dinv32;
  double a0, a1, a2;
  int u0, u1, u2;
  int adv;         // any advection weight non-zero
  const double* b;
  double* x;
  double* ws;      // r, u, w, m, n, t, tmp, then rings p, s, q, z of mmax+1 slots
  void* pcws;      // preconditioner scratch: r, p, s, x (double or float)
  double* hist;
  int hist_cap;
};

struct BatchOut {
  int status, it, restarts, breakdowns, replacements, hist_len;
  double rho0, rho, rnorm_true, bnorm;
};

struct BatchParams {
  int mmax, truncation, norm, maxit, max_restarts, true_check;
  double rtol, atol;
  int pc_kind, pc_inner, pc_prec;
};

// Scalars of the block's current system (shared memory).
struct BlkState {
  int status, it, i, nw, restarts, breakdowns, replacements, hist_len, prev_bd, target_set;
  int last_x;                       // inner PCG: last iteration whose x update happens
  double alpha, gamma, delta, eta, target, rho0, rho, bnorm, goal, rtrue;
  double pg, palpha[64], pbeta;     // inner PCG scalars
  double beta[PFK_MAX_MMAX];
  double eta_ring[PFK_MAX_MMAX + 1];
  double red[8];                    // results of block reductions
};

// ---------------------------------------------------------------------------
// Block helpers
// ---------------------------------------------------------------------------

// Sums nd values over the block (fixed order: warp tree, then warps in order)
// into st->red[0..nd-1]; all threads must call it.
template <int ND>
__device__ __forceinline__ void block_sum(const double (&v)[ND], double* smem, BlkState* st) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const double s = warp_sum(v[j]);
    if (lane == 0) smem[warp * ND + j] = s;
  }
  __syncthreads();
  if (threadIdx.x < ND) {
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += smem[w * ND + threadIdx.x];
    st->red[threadIdx.x] = s;
  }
  __syncthreads();
}

template <typename V, typename C>
__device__ __forceinline__ V cvt(C v) { return (V)v; }

// (A m)_c for cell c = (i, j, k), operator coefficients of type C, arithmetic V.
// m is not __restrict__: it is written during the launch, so its loads must
// stay coherent ones that the block barriers order, not read-only-cache loads.
template <typename V, typename C>
__device__ __forceinline__ V sys_row(const BatchSys& S, const C* d, const C* kx, const C* ky, const C* kz,
                                     const V* m, int64_t c, int i, int j, int k) {
  const int64_t sxy = (int64_t)S.nx * S.ny;
  if (!S.adv) {
    // pure diffusion: the same products without the zero advection weights
    // (adding +0 to a coefficient changes nothing)
    V acc = (V)d[c] * m[c];
    if (i > 0) acc = fma(-(V)kx[c - 1], m[c - 1], acc);
    if (i < S.nx - 1) acc = fma(-(V)kx[c], m[c + 1], acc);
    if (j > 0) acc = fma(-(V)ky[c - S.nx], m[c - S.nx], acc);
    if (j < S.ny - 1) acc = fma(-(V)ky[c], m[c + S.nx], acc);
    if (S.ndim == 3) {
      if (k > 0) acc = fma(-(V)kz[c - sxy], m[c - sxy], acc);
      if (k < S.nz - 1) acc = fma(-(V)kz[c], m[c + sxy], acc);
    }
    return acc;
  }
  const V a0 = (V)S.a0, a1 = (V)S.a1, a2 = (V)S.a2;
  V acc = (V)d[c] * m[c];
  if (i > 0) acc = fma(-((V)kx[c - 1] + (S.u0 == -1 ? a0 : V(0))), m[c - 1], acc);
  if (i < S.nx - 1) acc = fma(-((V)kx[c] + (S.u0 == 1 ? a0 : V(0))), m[c + 1], acc);
  if (j > 0) acc = fma(-((V)ky[c - S.nx] + (S.u1 == -1 ? a1 : V(0))), m[c - S.nx], acc);
  if (j < S.ny - 1) acc = fma(-((V)ky[c] + (S.u1 == 1 ? a1 : V(0))), m[c + S.nx], acc);
  if (S.ndim == 3) {
    if (k > 0) acc = fma(-((V)kz[c - sxy] + (S.u2 == -1 ? a2 : V(0))), m[c - sxy], acc);
    if (k < S.nz - 1) acc = fma(-((V)kz[c] + (S.u2 == 1 ? a2 : V(0))), m[c + sxy], acc);
  }
  return acc;
}

// One x-row per warp; (j, k) from the row.
#define SYS_ROWS(S, c, i, j, k)                                                                       \
  for (int row_ = (int)(threadIdx.x >> 5), j = 0, k = 0;                                             \
       row_ < (S).ny * (S).nz && ((j = row_ % (S).ny), (k = row_ / (S).ny), true);                   \
       row_ += (int)(blockDim.x >> 5))                                                               \
    for (int i = (int)(threadIdx.x & 31); i < (S).nx; i += 32)                                        \
      for (int64_t c = (int64_t)row_ * (S).nx + i, once_ = 1; once_; once_ = 0)

#define SYS_ELEMS(n, e) for (int64_t e = threadIdx.x; e < (n); e += blockDim.x)

// y = A m (FP64), or y = b - A m if bsub.
__device__ void sys_apply(const BatchSys& S, const double* m, double* y, const double* bsub) {
  SYS_ROWS(S, c, i, j, k) {
    const double v = sys_row<double, double>(S, S.d, S.kx, S.ky, S.kz, m, c, i, j, k);
    y[c] = bsub ? bsub[c] - v : v;
  }
  __syncthreads();
}

// out = add + B(v) for the batch's preconditioner (Jacobi, or inner PCG with
// V = double / float and matching coefficient copies).  Mirrors the
// single-system inner PCG: same guards, same statement order.
template <typename V>
__device__ void sys_pcg(const BatchSys& S, const BatchParams& P, const V* dinvv, const V* dv, const V* kxv,
                        const V* kyv, const V* kzv, const double* v, double* out, const double* add, double* smem,
                        BlkState* st) {
  const int64_t n = S.n;
  V* base = (V*)S.pcws;
  V* r = base;
  V* p = base + n;
  V* s = base + 2 * n;
  V* x = base + 3 * n;
  const int kk = P.pc_inner;
  // r_0 = v; gamma_0 = <D^-1 r, r>
  {
    V acc = V(0);
    SYS_ELEMS(n, e) {
      const V rv = (V)v[e];
      r[e] = rv;
      acc += (dinvv[e] * rv) * rv;
    }
    double a[1] = {(double)acc};
    block_sum<1>(a, smem, st);
    if (threadIdx.x == 0) {
      st->pg = st->red[0];
      st->last_x = st->pg == 0.0 ? 0 : kk;
    }
    __syncthreads();
  }
  if (st->last_x > 0) {
    // p_0 = D^-1 r_0, s_0 = A p_0, eta_0 = <s_0, p_0>
    SYS_ELEMS(n, e) p[e] = dinvv[e] * r[e];
    __syncthreads();
    V acc = V(0);
    SYS_ROWS(S, c, i, j, k) {
      const V sv = sys_row<V, V>(S, dv, kxv, kyv, kzv, p, c, i, j, k);
      s[c] = sv;
      acc += sv * p[c];
    }
    double a[1] = {(double)acc};
    block_sum<1>(a, smem, st);
    if (threadIdx.x == 0) {
      if (st->red[0] == 0.0) st->last_x = 0;
      else st->palpha[0] = st->pg / st->red[0];
    }
    __syncthreads();
  }
  for (int it = 1; it < kk; ++it) {
    if (it > st->last_x) break;
    {
      // r_i = r_{i-1} - alpha_{i-1} s_{i-1}; gamma_i
      const V al = (V)st->palpha[it - 1];
      V acc = V(0);
      SYS_ELEMS(n, e) {
        const V rv = r[e] - al * s[e];
        r[e] = rv;
        acc += (dinvv[e] * rv) * rv;
      }
      double a[1] = {(double)acc};
      block_sum<1>(a, smem, st);
      if (threadIdx.x == 0) {
        const double g = st->red[0];
        if (g == 0.0) st->last_x = it;
        else {
          st->pbeta = g / st->pg;
          st->pg = g;
        }
      }
      __syncthreads();
    }
    {
      // x_i = x_{i-1} + alpha_{i-1} p_{i-1}; p_i = D^-1 r_i + beta_i p_{i-1}
      const V al = (V)st->palpha[it - 1];
      const V be = (V)st->pbeta;
      const bool do_p = it < st->last_x;
      SYS_ELEMS(n, e) {
        const V po = p[e];
        x[e] = (it == 1 ? V(0) : x[e]) + al * po;
        if (do_p) p[e] = dinvv[e] * r[e] + be * po;
      }
      __syncthreads();
      if (!do_p) break;
    }
    {
      // s_i = A p_i, eta_i
      V acc = V(0);
      SYS_ROWS(S, c, i, j, k) {
        const V sv = sys_row<V, V>(S, dv, kxv, kyv, kzv, p, c, i, j, k);
        s[c] = sv;
        acc += sv * p[c];
      }
      double a[1] = {(double)acc};
      block_sum<1>(a, smem, st);
      if (threadIdx.x == 0) {
        if (st->red[0] == 0.0) st->last_x = it;
        else st->palpha[it] = st->pg / st->red[0];
      }
      __syncthreads();
    }
  }
  const int last_x = st->last_x;
  const V al = (V)st->palpha[kk - 1];
  SYS_ELEMS(n, e) {
    double y;
    if (last_x == 0) y = 0.0;
    else if (kk <= last_x) y = (double)((kk == 1 ? V(0) : x[e]) + al * p[e]);
    else y = (double)x[e];
    out[e] = add ? add[e] + y : y;
  }
  __syncthreads();
}

__device__ void sys_pc(const BatchSys& S, const BatchParams& P, const double* v, double* out, const double* add,
                       double* smem, BlkState* st) {
  if (P.pc_kind == PFK_PC_NONE || P.pc_kind == PFK_PC_JACOBI) {
    SYS_ELEMS(S.n, e) {
      // B(v) = D^-1 v and add + B(v): two roundings (no fused multiply-add)
      const double y = P.pc_kind == PFK_PC_JACOBI ? __dmul_rn(S.dinv[e], v[e]) : v[e];
      out[e] = add ? __dadd_rn(add[e], y) : y;
    }
    __syncthreads();
    return;
  }
  if (P.pc_prec == PFK_FP64) sys_pcg<double>(S, P, S.dinv, S.d, S.kx, S.ky, S.kz, v, out, add, smem, st);
  else sys_pcg<float>(S, P, S.dinv32, S.d32, S.kx32, S.ky32, S.kz32, v, out, add, smem, st);
}

__device__ void blk_push_history(const BatchSys& S, BlkState* st, double rho, double rn, double eta, double al) {
  if (S.hist && st->hist_len < S.hist_cap) {
    double* h = S.hist + (size_t)st->hist_len * PFK_HISTORY_FIELDS;
    h[0] = rho; h[1] = rn; h[2] = eta; h[3] = al;
  }
  st->hist_len += 1;
}

__device__ __forceinline__ double blk_rho(const BatchParams& P, double gamma, double rr) {
  return P.norm == PFK_NORM_NATURAL ? sqrt(fabs(gamma)) : sqrt(rr);
}

// The fused pass of iteration i for one system (block-level) and its scalar
// phase, as in the single-system pipefcg_pass.
template <int NW>
__device__ void sys_pass(const BatchSys& S, const BatchParams& P, double* smem, BlkState* st) {
  const int64_t n = S.n;
  const int T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* vr = S.ws;
  double* vu = vr + n;
  double* vw = vu + n;
  const double* vm = vw + n;
  const double* vn = vm + n;
  double* vt = (double*)vn + n;
  const int slots = P.mmax + 1;
  double* Pr = S.ws + 7 * n;
  double* Sr = Pr + (int64_t)slots * n;
  double* Qr = Sr + (int64_t)slots * n;
  double* Zr = Qr + (int64_t)slots * n;
  const int iprev = st->i;
  const int nwp = st->nw;
  const double alpha = st->alpha;
  // shared layout: s_sk[NW][T+1] | s_u[T] | scratch for block sums
  double* s_sk = smem;
  double* s_u = s_sk + NW * (T + 1);
  double* s_red = s_u + T;
  __shared__ size_t s_off[NW];
  __shared__ double s_beta[NW];
  if (threadIdx.x < nwp) {
    s_off[threadIdx.x] = (size_t)((iprev - nwp + (int)threadIdx.x) % slots) * (size_t)n;
    s_beta[threadIdx.x] = st->beta[threadIdx.x];
  }
  __syncthreads();
  const size_t coff = (size_t)(iprev % slots) * (size_t)n;
  double* my = s_sk + threadIdx.x;
  const double* wu = s_u + warp * 32;
  const double* lrow = s_sk + lane * (T + 1) + warp * 32;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0, gw = 0.0;
  for (int64_t base = 0; base < n; base += T) {
    const int64_t e = base + threadIdx.x;
    double un = 0.0;
    if (e < n) {
      const double u0 = vu[e], w0 = vw[e];
      double p = u0, s = w0, q = vm[e], z = vn[e];
#pragma unroll 4
      for (int j = 0; j < nwp; ++j) {
        const size_t o = s_off[j] + e;
        const double bb = s_beta[j];
        const double sv = Sr[o];
        p = fma(bb, Pr[o], p);
        s = fma(bb, sv, s);
        q = fma(bb, Qr[o], q);
        z = fma(bb, Zr[o], z);
        my[j * (T + 1)] = sv;
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
      for (int j = 0; j < nwp; ++j) my[j * (T + 1)] = 0.0;
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
  // block sums: gamma, delta, rr, <u, s_{i-1}>, window dots
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
  __shared__ double s_tot[PFK_MAX_MMAX + 4];
  if (threadIdx.x < nd) {
    double v = 0.0;
    for (int w = 0; w < T / 32; ++w) v += s_red[w * nd + threadIdx.x];
    s_tot[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int i = iprev + 1;
    const double gamma = s_tot[0], delta = s_tot[1], rr = s_tot[2];
    st->it += 1;
    st->i = i;
    st->gamma = gamma;
    const double rho = blk_rho(P, gamma, rr);
    st->rho = rho;
    const int hslot = st->hist_len;
    blk_push_history(S, st, rho, sqrt(rr), nan(""), nan(""));
    if (!isfinite(rho)) st->status = kNonFinite;
    else if (rho <= st->target) st->status = kConverged;
    else {
      const int nu = nu_window(i, P.mmax, P.truncation);
      const int off = nwp + 1 - nu;
      double sumb = 0.0;
      for (int jj = 0; jj < nu; ++jj) {
        const int src = off + jj;
        const double cc = src < nwp ? s_tot[4 + src] : s_tot[3];
        const double ek = st->eta_ring[(i - nu + jj) % slots];
        const double bb = -cc / ek;
        st->beta[jj] = bb;
        sumb += bb * bb * ek;
      }
      const double eta = delta - sumb;
      const double al = eta != 0.0 ? gamma / eta : nan("");
      st->eta = eta;
      st->alpha = al;
      st->nw = nu;
      st->eta_ring[i % slots] = eta;
      if (S.hist && hslot < S.hist_cap) {
        S.hist[(size_t)hslot * PFK_HISTORY_FIELDS + 2] = eta;
        S.hist[(size_t)hslot * PFK_HISTORY_FIELDS + 3] = al;
      }
      if (eta <= 0.0) st->status = kBreakdown;
      else if (st->it >= P.maxit) st->status = kMaxit;
    }
  }
  __syncthreads();
}

template <int NW>
__device__ void sys_solve(const BatchSys& S, const BatchParams& P, double* smem, BlkState* st, BatchOut* out) {
  const int64_t n = S.n;
  double* vr = S.ws;
  double* vu = vr + n;
  double* vw = vu + n;
  double* vm = vw + n;
  double* vn = vm + n;
  double* vt = vn + n;
  double* tmp = vt + n;
  if (threadIdx.x == 0) {
    st->it = 0; st->restarts = 0; st->breakdowns = 0; st->replacements = 0; st->hist_len = 0;
    st->prev_bd = 0; st->target_set = 0; st->status = kRun; st->rtrue = nan("");
  }
  {
    double acc[1] = {0.0};
    SYS_ELEMS(n, e) acc[0] = fma(S.b[e], S.b[e], acc[0]);
    block_sum<1>(acc, smem, st);
    if (threadIdx.x == 0) {
      st->bnorm = sqrt(st->red[0]);
      st->goal = fmax(P.rtol * st->bnorm, P.atol);
    }
    __syncthreads();
  }
  int result = PFK_OK;
  for (int guard = 0; guard < 100000; ++guard) {
    // ---- pipeline fill (Alg. 8) ----
    sys_apply(S, S.x, vr, S.b);                 // r_0 = b - A x_0
    sys_pc(S, P, vr, vu, nullptr, smem, st);    // u_0 = B(r_0) = p_0
    sys_apply(S, vu, vw, nullptr);              // w_0 = A p_0
    sys_pc(S, P, vw, vm, nullptr, smem, st);    // m_0 = B(w_0)
    sys_apply(S, vm, vn, nullptr);              // n_0 = A m_0
    {
      double acc[3] = {0.0, 0.0, 0.0};
      SYS_ELEMS(n, e) {
        acc[0] = fma(vu[e], vr[e], acc[0]);
        acc[1] = fma(vu[e], vw[e], acc[1]);
        acc[2] = fma(vr[e], vr[e], acc[2]);
      }
      block_sum<3>(acc, smem, st);
      if (threadIdx.x == 0) {
        const double gamma = st->red[0], eta = st->red[1], rr = st->red[2];
        const double rho = blk_rho(P, gamma, rr);
        if (!st->target_set) {
          st->rho0 = rho;
          st->target = fmax(P.rtol * rho, P.atol);
          st->target_set = 1;
        }
        const double al = eta != 0.0 ? gamma / eta : nan("");
        blk_push_history(S, st, rho, sqrt(rr), eta, al);
        st->rho = rho; st->gamma = gamma; st->eta = eta; st->alpha = al;
        st->i = 0; st->nw = 0; st->eta_ring[0] = eta;
        if (!isfinite(rho)) st->status = kNonFinite;
        else if (rho <= st->target) st->status = kConverged;
        else if (eta <= 0.0) st->status = kFillBreakdown;
        else if (st->it >= P.maxit) st->status = kMaxit;
        else st->status = kRun;
      }
      __syncthreads();
    }
    // ---- iterations ----
    while (st->status == kRun) {
      sys_pass<NW>(S, P, smem, st);
      if (st->status != kRun) break;
      sys_pc(S, P, vt, vm, vu, smem, st);       // m_i = u_i + B(w_i - r_i)
      sys_apply(S, vm, vn, nullptr);            // n_i = A m_i
    }
    const int status = st->status;
    if (status == kConverged) {
      sys_apply(S, S.x, tmp, S.b);
      double acc[1] = {0.0};
      SYS_ELEMS(n, e) acc[0] = fma(tmp[e], tmp[e], acc[0]);
      block_sum<1>(acc, smem, st);
      if (threadIdx.x == 0) {
        const double rt = sqrt(st->red[0]);
        st->rtrue = rt;
        if (!P.true_check || rt <= st->goal) {
          st->status = -100;    // accepted
        } else if (st->restarts >= P.max_restarts) {
          st->status = -102;    // true residual stagnates above the goal
        } else {
          st->replacements += 1;
          st->restarts += 1;
          st->target *= 0.5 * st->goal / rt;
          st->prev_bd = 0;
          st->status = kRun;
        }
      }
      __syncthreads();
      if (st->status == -100) { result = PFK_OK; break; }
      if (st->status == -102) { result = PFK_ERR_NOT_CONVERGED; break; }
      continue;
    }
    if (status == kBreakdown) {
      if (threadIdx.x == 0) {
        st->breakdowns += 1;
        if ((st->i <= 1 && st->prev_bd) || st->restarts >= P.max_restarts) {
          st->status = -101;
        } else {
          st->restarts += 1;
          st->prev_bd = 1;
          st->status = kRun;
        }
      }
      __syncthreads();
      if (st->status == -101) { result = PFK_ERR_BREAKDOWN; break; }
      continue;
    }
    result = (status == kMaxit) ? PFK_ERR_NOT_CONVERGED : PFK_ERR_BREAKDOWN;
    break;
  }
  if (isnan(st->rtrue) || result != PFK_OK) {
    sys_apply(S, S.x, tmp, S.b);
    double acc[1] = {0.0};
    SYS_ELEMS(n, e) acc[0] = fma(tmp[e], tmp[e], acc[0]);
    block_sum<1>(acc, smem, st);
    if (threadIdx.x == 0) st->rtrue = sqrt(st->red[0]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out->status = result;
    out->it = st->it;
    out->restarts = st->restarts;
    out->breakdowns = st->breakdowns;
    out->replacements = st->replacements;
    out->hist_len = st->hist_len;
    out->rho0 = st->rho0;
    out->rho = st->rho;
    out->rnorm_true = st->rtrue;
    out->bnorm = st->bnorm;
  }
  __syncthreads();
}

// At most 64 registers, so that two blocks of 512 threads (or four of 256)
// share an SM: the kernel is latency-bound, and 32 warps per SM (the limit the
// window buffer's shared memory sets at 512 threads) hide more of it than 16
// (measured about 7 % faster on the 512-system batch than the 92-register build).
template <int NW>
__global__ void __launch_bounds__(512, 2) batched_pipefcg(const BatchSys* __restrict__ systems, const int* __restrict__ order, int nsys,
                                BatchParams P, int* next, BatchOut* outs) {
  extern __shared__ double smem[];
  __shared__ BlkState st;
  __shared__ int s_sys;
  for (;;) {
    if (threadIdx.x == 0) s_sys = atomicAdd(next, 1);
    __syncthreads();
    const int q = s_sys;
    __syncthreads();
    if (q >= nsys) return;
    const int sid = order[q];
    const BatchSys S = systems[sid];
    sys_solve<NW>(S, P, smem, &st, &outs[sid]);
  }
}

static size_t batch_smem(int nw, int T) { return ((size_t)nw * (T + 1) + T + (size_t)(T / 32) * (nw + 4)) * sizeof(double); }

static int batch_template(int mmax) { return mmax <= 8 ? 8 : mmax <= 16 ? 16 : mmax <= 24 ? 24 : 32; }

template <int NW>
static cudaError_t launch_batch(int blocks, int T, size_t smem, cudaStream_t st, const BatchSys* sys,
                                const int* order, int nsys, const BatchParams& P, int* next, BatchOut* outs) {
  cudaError_t e = cudaFuncSetAttribute(batched_pipefcg<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  batched_pipefcg<NW><<<blocks, T, smem, st>>>(sys, order, nsys, P, next, outs);
  return cudaGetLastError();
}

static cudaError_t launch_any(int tmpl, int blocks, int T, size_t smem, cudaStream_t st, const BatchSys* sys,
                              const int* order, int nsys, const BatchParams& P, int* next, BatchOut* outs) {
  switch (tmpl) {
    case 8: return launch_batch<8>(blocks, T, smem, st, sys, order, nsys, P, next, outs);
    case 16: return launch_batch<16>(blocks, T, smem, st, sys, order, nsys, P, next, outs);
    case 24: return launch_batch<24>(blocks, T, smem, st, sys, order, nsys, P, next, outs);
    default: return launch_batch<32>(blocks, T, smem, st, sys, order, nsys, P, next, outs);
  }
}

static int blocks_per_sm(int tmpl, int T, size_t smem) {
  int nb = 0;
  cudaError_t e;
  // the occupancy query honours the kernel's dynamic shared-memory limit
  // (48 KB by default): raise it to this launch's size first
  switch (tmpl) {
    case 8: e = cudaFuncSetAttribute(batched_pipefcg<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); break;
    case 16: e = cudaFuncSetAttribute(batched_pipefcg<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); break;
    case 24: e = cudaFuncSetAttribute(batched_pipefcg<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); break;
    default: e = cudaFuncSetAttribute(batched_pipefcg<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  switch (tmpl) {
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_pipefcg<8>, T, smem); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_pipefcg<16>, T, smem); break;
    case 24: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_pipefcg<24>, T, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_pipefcg<32>, T, smem); break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace pfk

using namespace pfk;

extern "C" pfk_status pfk_solve_batched(pfk_context* ctx, int nsys, const pfk_operator* const* ops,
                                        const pfk_pc_desc* pcd, const pfk_solve_params* prm, const double* const* b,
                                        double* const* x, int ptrs_on_device, int block_threads,
                                        pfk_solve_info* infos) {
  if (!ctx || !ops || !prm || !b || !x || nsys <= 0) {
    set_error(ctx, "invalid argument");
    return PFK_ERR_INVALID;
  }
  if (prm->method != PFK_PIPEFCG || prm->mmax < 1 || prm->mmax > PFK_MAX_MMAX) {
    set_error(ctx, "batched solve supports PFK_PIPEFCG with 1 <= mmax <= PFK_MAX_MMAX");
    return PFK_ERR_INVALID;
  }
  if (block_threads != 0 && (block_threads < 64 || block_threads > 512 || block_threads % 32)) {
    set_error(ctx, "block_threads must be 0 or a multiple of 32 in [64, 512]");
    return PFK_ERR_INVALID;
  }
  BatchParams P;
  P.mmax = prm->mmax; P.truncation = prm->truncation; P.norm = prm->norm; P.maxit = prm->maxit;
  P.max_restarts = prm->max_restarts; P.true_check = prm->true_residual_check;
  P.rtol = prm->rtol; P.atol = prm->atol;
  P.pc_kind = pcd ? pcd->kind : PFK_PC_NONE;
  P.pc_inner = pcd ? pcd->inner_iters : 0;
  P.pc_prec = pcd ? pcd->precision : PFK_FP64;
  if (!(P.pc_kind == PFK_PC_NONE || P.pc_kind == PFK_PC_JACOBI ||
        (P.pc_kind == PFK_PC_INNER_PCG && (P.pc_prec == PFK_FP64 || P.pc_prec == PFK_FP32) && P.pc_inner >= 1 &&
         P.pc_inner <= 64))) {
    set_error(ctx, "batched solve supports NONE, JACOBI and INNER_PCG (FP64 or FP32) preconditioners");
    return PFK_ERR_INVALID;
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const int slots = P.mmax + 1;
  const bool fp32 = P.pc_kind == PFK_PC_INNER_PCG && P.pc_prec == PFK_FP32;
  std::vector<BatchSys> hs(nsys);
  std::vector<int64_t> wsoff(nsys), pcoff(nsys);
  int64_t wtot = 0, ptot = 0, nmax = 0;
  for (int j = 0; j < nsys; ++j) {
    const pfk_operator* op = ops[j];
    if (!op || !op->d || op->rowptr) {
      set_error(ctx, "batched solve needs matrix-free stencil operators");
      return PFK_ERR_INVALID;
    }
    if (fp32) {
      pfk_status s = ensure_reduced_copies(const_cast<pfk_operator*>(op), PFK_FP32);
      if (s != PFK_OK) return s;
    }
    const int64_t n = op->n;
    nmax = std::max(nmax, n);
    wsoff[j] = wtot;
    wtot += (7 + 4 * (int64_t)slots) * n;
    pcoff[j] = ptot;
    ptot += 4 * n;   // doubles (enough for float too)
  }
  const int hcap = prm->history ? prm->history_capacity : 0;
  // device arena: workspaces | pc scratch | x copies | b copies (host path) | history | descriptors | outs | order | counter
  const bool host = !ptrs_on_device;
  int64_t ntot = 0;
  for (int j = 0; j < nsys; ++j) ntot += ops[j]->n;
  const size_t bytes = sizeof(double) * (size_t)(wtot + ptot + (host ? 2 * ntot : 0) + (int64_t)nsys * hcap * 4) +
                       sizeof(BatchSys) * nsys + sizeof(BatchOut) * nsys + sizeof(int) * (nsys + 64) + 1024;
  char* arena = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&arena, bytes, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocAsync (batch arena)");
  struct Free {
    char* p; cudaStream_t s;
    ~Free() { if (p) { cudaFreeAsync(p, s); cudaStreamSynchronize(s); } }
  } guard{arena, st};
  double* dws = (double*)arena;
  double* dpc = dws + wtot;
  double* dxb = dpc + ptot;
  double* dhist = dxb + (host ? 2 * ntot : 0);
  BatchSys* dsys = (BatchSys*)(dhist + (int64_t)nsys * hcap * 4);
  BatchOut* douts = (BatchOut*)(dsys + nsys);
  int* dorder = (int*)(douts + nsys);
  int* dnext = dorder + nsys;
  int64_t xo = 0;
  for (int j = 0; j < nsys; ++j) {
    const pfk_operator* op = ops[j];
    BatchSys& S = hs[j];
    S.nx = op->nx; S.ny = op->ny; S.nz = op->nz; S.ndim = op->ndim; S.n = op->n;
    S.d = op->d; S.kx = op->kx; S.ky = op->ky; S.kz = op->kz; S.dinv = op->dinv;
    S.d32 = op->d32; S.kx32 = op->kx32; S.ky32 = op->ky32; S.kz32 = op->kz32; S.dinv32 = op->dinv32;
    S.a0 = op->adv[0]; S.a1 = op->adv[1]; S.a2 = op->adv[2];
    S.u0 = op->upw[0]; S.u1 = op->upw[1]; S.u2 = op->upw[2];
    S.adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
    S.ws = dws + wsoff[j];
    S.pcws = dpc + pcoff[j];
    S.hist = hcap ? dhist + (int64_t)j * hcap * 4 : nullptr;
    S.hist_cap = hcap;
    if (host) {
      double* xb = dxb + 2 * xo;
      PFK_CUDA(ctx, cudaMemcpyAsync(xb, x[j], op->n * sizeof(double), cudaMemcpyHostToDevice, st));
      PFK_CUDA(ctx, cudaMemcpyAsync(xb + op->n, b[j], op->n * sizeof(double), cudaMemcpyHostToDevice, st));
      S.x = xb;
      S.b = xb + op->n;
      xo += op->n;
    } else {
      S.x = x[j];
      S.b = b[j];
    }
  }
  // largest systems first (longest-processing-time order)
  std::vector<int> order(nsys);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return ops[a]->n > ops[c]->n; });
  PFK_CUDA(ctx, cudaMemcpyAsync(dsys, hs.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, st));
  PFK_CUDA(ctx, cudaMemcpyAsync(dorder, order.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));

  const int tmpl = batch_template(P.mmax);
  auto smem_of = [&](int T) { return batch_smem(tmpl, T); };
  auto valid_T = [&](int T) { return smem_of(T) <= 227 * 1024; };
  int T = block_threads;
  const int lg = (int)std::ceil(std::log2((double)std::max<int64_t>(nmax, 2)));
  const auto key = std::make_tuple(tmpl, lg, nsys >= 4 * ctx->num_sms ? 2 : (nsys >= ctx->num_sms ? 1 : 0),
                                   (int)fp32 + 2 * P.pc_inner);
  if (T == 0) {
    auto it = ctx->batched_tuned.find(key);
    if (it != ctx->batched_tuned.end()) T = it->second;
  }
  std::vector<double> xsave;
  if (T == 0) {
    // autotune: a short trial (maxit 3, all systems) per candidate; x and the
    // workspace are restored afterwards by re-copying x
    BatchParams Pt = P;
    Pt.maxit = 3;
    Pt.true_check = 0;
    std::vector<std::vector<double>> x0(nsys);
    for (int j = 0; j < nsys; ++j) {
      x0[j].resize(ops[j]->n);
      PFK_CUDA(ctx, cudaMemcpyAsync(x0[j].data(), hs[j].x, ops[j]->n * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    PFK_CUDA(ctx, cudaStreamSynchronize(st));
    cudaEvent_t t0, t1;
    PFK_CUDA(ctx, cudaEventCreate(&t0));
    PFK_CUDA(ctx, cudaEventCreate(&t1));
    float best = 1e30f;
    for (int cand : {128, 256, 512}) {
      if (!valid_T(cand)) continue;
      const int bps = blocks_per_sm(tmpl, cand, smem_of(cand));
      if (bps < 1) continue;
      const int blocks = std::min(nsys, bps * ctx->num_sms);
      PFK_CUDA(ctx, cudaMemsetAsync(dnext, 0, sizeof(int), st));
      PFK_CUDA(ctx, cudaEventRecord(t0, st));
      PFK_CUDA(ctx, launch_any(tmpl, blocks, cand, smem_of(cand), st, dsys, dorder, nsys, Pt, dnext, douts));
      PFK_CUDA(ctx, cudaEventRecord(t1, st));
      PFK_CUDA(ctx, cudaEventSynchronize(t1));
      float ms = 0.f;
      PFK_CUDA(ctx, cudaEventElapsedTime(&ms, t0, t1));
      if (ms < best) {
        best = ms;
        T = cand;
      }
      for (int j = 0; j < nsys; ++j)
        PFK_CUDA(ctx, cudaMemcpyAsync(hs[j].x, x0[j].data(), ops[j]->n * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (T == 0) {
      set_error(ctx, "no block size fits the batched kernel");
      return PFK_ERR_INVALID;
    }
    ctx->batched_tuned[key] = T;
  }
  if (!valid_T(T)) {
    set_error(ctx, "block_threads too large for the window's shared memory");
    return PFK_ERR_INVALID;
  }
  const int bps = blocks_per_sm(tmpl, T, smem_of(T));
  if (bps < 1) {
    set_error(ctx, "batched kernel does not fit on an SM with this block size");
    return PFK_ERR_INVALID;
  }
  const int blocks = std::min(nsys, bps * ctx->num_sms);
  cudaEvent_t t0, t1;
  PFK_CUDA(ctx, cudaEventCreate(&t0));
  PFK_CUDA(ctx, cudaEventCreate(&t1));
  PFK_CUDA(ctx, cudaMemsetAsync(dnext, 0, sizeof(int), st));
  PFK_CUDA(ctx, cudaEventRecord(t0, st));
  PFK_CUDA(ctx, launch_any(tmpl, blocks, T, smem_of(T), st, dsys, dorder, nsys, P, dnext, douts));
  PFK_CUDA(ctx, cudaEventRecord(t1, st));
  std::vector<BatchOut> hout(nsys);
  PFK_CUDA(ctx, cudaMemcpyAsync(hout.data(), douts, sizeof(BatchOut) * nsys, cudaMemcpyDeviceToHost, st));
  if (host)
    for (int j = 0; j < nsys; ++j)
      PFK_CUDA(ctx, cudaMemcpyAsync(x[j], hs[j].x, ops[j]->n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (hcap)
    PFK_CUDA(ctx, cudaMemcpyAsync(prm->history, dhist, sizeof(double) * (size_t)nsys * hcap * 4,
                                  cudaMemcpyDeviceToHost, st));
  PFK_CUDA(ctx, cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  pfk_status first = PFK_OK;
  for (int j = 0; j < nsys; ++j) {
    if (first == PFK_OK && hout[j].status != PFK_OK) first = (pfk_status)hout[j].status;
    if (infos) {
      pfk_solve_info& I = infos[j];
      std::memset(&I, 0, sizeof(I));
      I.status = hout[j].status;
      I.iterations = hout[j].it;
      I.restarts = hout[j].restarts;
      I.breakdowns = hout[j].breakdowns;
      I.replacements = hout[j].replacements;
      I.history_len = hout[j].hist_len;
      I.rho0 = hout[j].rho0;
      I.rho_final = hout[j].rho;
      I.rnorm_true = hout[j].rnorm_true;
      I.bnorm = hout[j].bnorm;
      I.time_ms = ms;
      I.pass_launches = T;
      I.kernel_launches = 1;
    }
  }
  if (first != PFK_OK) set_error(ctx, "at least one system of the batch did not converge");
  return first;
}
