// Preconditioners B of the flexible methods (Sec. 2; notation table Sec. 3).
//
//  * Jacobi:     B(v) = D^-1 v.
//  * Inner PCG:  k iterations of Alg. 3 (M^-1 = D^-1) on A y = v from y = 0,
//                the inner solver of the paper's block-Jacobi experiments
//                (Sec. 6, "5 iterations of Jacobi-preconditioned CG").
//                Three kernels per inner iteration:
//                  A_i  r_i = r_{i-1} - alpha_{i-1} s_{i-1}, partial gamma_i = <D^-1 r_i, r_i>
//                  B_i  x_i = x_{i-1} + alpha_{i-1} p_{i-1}, p_i = D^-1 r_i + beta_i p_{i-1}
//                  C_i  s_i = A p_i, partial eta_i = <s_i, p_i>
//                each ending in a device-side last-block combine of its partial
//                sums, so no host synchronisation happens inside B.
//  * Chebyshev:  k sweeps of Chebyshev acceleration of Jacobi over [lo, hi]
//                (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
//                Alg. 12.1), one fused kernel per sweep.
//
// Precision variants (spec mixed precision): vectors V = double or
// float, coefficient storage C = double, float or bfloat16.  Inner products of
// the FP32 variants accumulate per thread in FP32 and are combined across
// threads and blocks in FP64.
#include "pfk_internal.cuh"
#include "stencil.cuh"
#include "stencil_tma.cuh"

#include <cmath>
#include <type_traits>

namespace pfk {

pfk_status ensure_reduced_copies(pfk_operator* op, int precision);

template <typename C>
__device__ __forceinline__ double to_d(C v) { return (double)v; }
template <>
__device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <typename V, typename C>
__device__ __forceinline__ V cv(C v) { return (V)v; }
template <>
__device__ __forceinline__ float cv<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename V, typename C>
struct StencilT {
  const C* d;
  const C* kx;
  const C* ky;
  const C* kz;
  const C* dinv;
  int nx, ny, nz, ndim;
  V a0, a1, a2;
  int u0, u1, u2;
  int64_t n;
};

#define GRID_LOOP(c, n) \
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < (n); c += (int64_t)gridDim.x * blockDim.x)

#define SKIP_IF_DONE(status) \
  if ((status) && *(status) != kRun) return;

// ---------------------------------------------------------------------------
// Jacobi / identity
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads) jacobi_kernel(const double* __restrict__ dinv, const double* __restrict__ v,
                                                          const double* __restrict__ add, double* __restrict__ out,
                                                          int64_t n, const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  // product and sum rounded separately (no fused multiply-add), as B(v) = D^-1 v
  // and add + B(v) are two operations
  GRID_LOOP(c, n) {
    double y = dinv ? __dmul_rn(dinv[c], v[c]) : v[c];
    out[c] = add ? __dadd_rn(add[c], y) : y;
  }
}

// ---------------------------------------------------------------------------
// Noisy preconditioner (toy experiment, Fig. FCGtoy)
// ---------------------------------------------------------------------------

// ||v||; the last block picks the bank row j = calls mod count, the scale
// eta ||v|| / ||xi_j|| and advances the application counter.
__global__ void __launch_bounds__(kThreads) noisy_norm_kernel(const double* __restrict__ v, int64_t n, double eta,
                                                              const double* __restrict__ inv_norm, int count,
                                                              PcCtl* ctl, double* partials,
                                                              const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  double acc[1] = {0.0};
  GRID_LOOP(c, n) acc[0] = fma(v[c], v[c], acc[0]);
  __shared__ double smem[kThreads / 32];
  __shared__ double sums[1];
  if (reduce_last_block<1>(acc, 1, partials, 1, &ctl->counter, smem, sums) && threadIdx.x == 0) {
    const long long j = ctl->calls % count;
    ctl->row = j;
    ctl->scale = eta * sqrt(sums[0]) * inv_norm[j];
    ctl->calls += 1;
  }
}

// out = add + v + scale xi_row
__global__ void __launch_bounds__(kThreads) noisy_apply_kernel(const double* __restrict__ v,
                                                               const double* __restrict__ bank, int64_t n,
                                                               const PcCtl* ctl, const double* __restrict__ add,
                                                               double* __restrict__ out,
                                                               const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  const double s = ctl->scale;
  const double* xi = bank + (size_t)ctl->row * (size_t)n;
  GRID_LOOP(c, n) {
    const double y = fma(s, xi[c], v[c]);
    out[c] = add ? add[c] + y : y;
  }
}

// 1 / ||xi_j|| for every bank row (one block per row, fixed order).
__global__ void __launch_bounds__(kThreads) noisy_row_norms_kernel(const double* __restrict__ bank, int64_t n,
                                                                   double* __restrict__ inv_norm,
                                                                   int* __restrict__ bad) {
  const double* xi = bank + (size_t)blockIdx.x * (size_t)n;
  double acc = 0.0;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) acc = fma(xi[c], xi[c], acc);
  __shared__ double sm[kThreads / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
    if (!(s > 0.0)) atomicExch(bad, 1);
    inv_norm[blockIdx.x] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Inner Jacobi-PCG
// ---------------------------------------------------------------------------

// A_0 and B_0 in one launch (neither needs the other's result):
// r_0 = v (not stored: A_1 reads v), p_0 = D^-1 r_0, gamma_0 = <D^-1 r_0, r_0>;
// finalize: stop at once (B(v) = 0) if gamma_0 == 0 (then v and p_0 are zero).
template <typename V, typename C>
__global__ void __launch_bounds__(kThreads) pcg_first_kernel(StencilT<V, C> A, const double* __restrict__ v,
                                                             V* __restrict__ p0, PcCtl* ctl, int k,
                                                             double* partials, const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  V accv = V(0);
  GRID_LOOP(c, A.n) {
    const V rv = (V)v[c];
    const V z = cv<V, C>(A.dinv[c]) * rv;
    p0[c] = z;
    accv += z * rv;
  }
  double acc[1] = {(double)accv};
  __shared__ double smem[kThreads / 32];
  __shared__ double sums[1];
  if (reduce_last_block<1>(acc, 1, partials, 1, &ctl->counter, smem, sums) && threadIdx.x == 0) {
    const double g = sums[0];
    ctl->gamma = g;
    ctl->ok = (g == 0.0) ? 0 : k;
  }
}

// A_i (i >= 1).  r_i = r_{i-1} - alpha_{i-1} s_{i-1} (r_0 = v).
// Finalize: beta_i = gamma_i / gamma_{i-1} (stop if gamma_i == 0).
template <typename V, typename C>
__global__ void __launch_bounds__(kThreads) pcg_a_kernel(StencilT<V, C> A, const double* __restrict__ v,
                                                         V* __restrict__ r, const V* __restrict__ s, PcCtl* ctl,
                                                         int i, double* partials, const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  const int last_x = ctl->ok;
  if (i > last_x) return;
  const V alpha = (V)ctl->alpha[i - 1];
  V accv = V(0);
  GRID_LOOP(c, A.n) {
    const V rv = (i == 1 ? (V)v[c] : r[c]) - alpha * s[c];
    r[c] = rv;
    accv += (cv<V, C>(A.dinv[c]) * rv) * rv;
  }
  double acc[1] = {(double)accv};
  __shared__ double smem[kThreads / 32];
  __shared__ double sums[1];
  if (reduce_last_block<1>(acc, 1, partials, 1, &ctl->counter, smem, sums) && threadIdx.x == 0) {
    const double g = sums[0];
    if (g == 0.0) {
      ctl->ok = i;
    } else {
      ctl->beta[i] = g / ctl->gamma;
      ctl->gamma = g;
    }
  }
}

// B_i (i >= 1).  x_i = x_{i-1} + alpha_{i-1} p_{i-1} (while i <= last_x);
//                p_i = D^-1 r_i + beta_i p_{i-1} (while i < last_x).
template <typename V, typename C>
__global__ void __launch_bounds__(kThreads) pcg_b_kernel(StencilT<V, C> A, const V* __restrict__ r,
                                                         const V* __restrict__ pold, V* __restrict__ pnew,
                                                         V* __restrict__ x, PcCtl* ctl, int i,
                                                         const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  const int last_x = ctl->ok;
  if (i > last_x) return;                  // x_i is not formed (and neither is p_i)
  const bool do_p = i < last_x;
  const V alpha = (V)ctl->alpha[i - 1];
  const V beta = (V)ctl->beta[i];
  GRID_LOOP(c, A.n) {
    const V po = pold[c];
    x[c] = (i == 1 ? V(0) : x[c]) + alpha * po;
    if (do_p) pnew[c] = cv<V, C>(A.dinv[c]) * r[c] + beta * po;
  }
}

// C_i.  s_i = A p_i, eta_i = <s_i, p_i>; finalize alpha_i = gamma_i / eta_i
// (stop if eta_i == 0).  Tiled z-marching stencil walk.
template <typename V>
struct PcgCEpi {
  V* __restrict__ s;
  V acc;
  struct Pre {};
  __device__ __forceinline__ Pre pre(int64_t) const { return Pre{}; }
  __device__ __forceinline__ void operator()(int64_t c, V sv, V pv, const Pre&) {
    s[c] = sv;
    acc += sv * pv;
  }
};

template <typename V, typename C, bool ADV>
__global__ void __launch_bounds__(kTileThreads) pcg_c_kernel(TiledStencil<V, C> T, const V* __restrict__ p,
                                                             V* __restrict__ s, PcCtl* ctl, int i, double* partials,
                                                             const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  if (!(i < ctl->ok)) return;
  PcgCEpi<V> e{s, V(0)};
  tiled_stencil_walk<V, C, ADV, tiled_width<V, C>()>(T, p, e);
  double acc[1] = {(double)e.acc};
  __shared__ double smem[kTileThreads / 32];
  __shared__ double sums[1];
  if (reduce_last_block<1>(acc, 1, partials, 1, &ctl->counter, smem, sums) && threadIdx.x == 0) {
    const double eta = sums[0];
    if (eta == 0.0) {
      ctl->ok = i;
    } else {
      ctl->eta = eta;
      ctl->alpha[i] = ctl->gamma / eta;
    }
  }
}

// F.  x_k = x_{k-1} + alpha_{k-1} p_{k-1} if the loop reached iteration k;
//     out = add + x.
template <typename V, typename C>
__global__ void __launch_bounds__(kThreads) pcg_final_kernel(int64_t n, const V* __restrict__ p,
                                                             const V* __restrict__ x, const double* __restrict__ add,
                                                             double* __restrict__ out, const PcCtl* ctl, int k,
                                                             const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  const int last_x = ctl->ok;
  const V alpha = (V)ctl->alpha[k - 1];
  GRID_LOOP(c, n) {
    double y;
    if (last_x == 0) {
      y = 0.0;
    } else if (k <= last_x) {
      y = (double)((k == 1 ? V(0) : x[c]) + alpha * p[c]);
    } else {
      y = (double)x[c];
    }
    out[c] = add ? add[c] + y : y;
  }
}

// ---------------------------------------------------------------------------
// Chebyshev-Jacobi
// ---------------------------------------------------------------------------

// Sweep 0 setup: r_0 = v, d_0 = (D^-1 r_0) / theta, as a product with the
// host-computed 1 / theta (a per-element FP64 division costs a dozen FP64
// instructions).
template <typename V, typename C>
__global__ void __launch_bounds__(kThreads) cheb_init_kernel(StencilT<V, C> A, const double* __restrict__ v,
                                                             V* __restrict__ r, V* __restrict__ dvec, V inv_theta,
                                                             const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  GRID_LOOP(c, A.n) {
    V rv = (V)v[c];
    r[c] = rv;
    dvec[c] = (cv<V, C>(A.dinv[c]) * rv) * inv_theta;
  }
}

// Sweep j (j + 1 < k): x_{j+1} = x_j + d_j; r_{j+1} = r_j - A d_j;
// d_{j+1} = c1 d_j + c2 D^-1 r_{j+1} (tiled stencil walk over d_j).
template <typename V, typename C>
struct ChebEpi {
  const C* __restrict__ dinv;
  V* __restrict__ dn;
  V* __restrict__ r;
  V* __restrict__ x;
  int first;
  V c1, c2;
  struct Pre {
    V x, r, dinv;
  };
  __device__ __forceinline__ Pre pre(int64_t c) const {
    return Pre{first ? V(0) : x[c], r[c], ld_coef<V, C>(dinv, c)};
  }
  __device__ __forceinline__ void operator()(int64_t c, V ad, V dc, const Pre& p) const {
    x[c] = p.x + dc;
    const V rv = p.r - ad;
    r[c] = rv;
    dn[c] = c1 * dc + c2 * (p.dinv * rv);
  }
};

template <typename V, typename C, bool ADV>
__global__ void __launch_bounds__(kTileThreads, 3) cheb_sweep_kernel(TiledStencil<V, C> T, const C* __restrict__ dinv,
                                                                  const V* __restrict__ dj, V* __restrict__ dn,
                                                                  V* __restrict__ r, V* __restrict__ x, int j, V c1,
                                                                  V c2, const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  ChebEpi<V, C> e{dinv, dn, r, x, j == 0, c1, c2};
  tiled_stencil_walk<V, C, ADV, tiled_width<V, C>()>(T, dj, e);
}

// Last sweep: out = add + x_{k-1} + d_{k-1} (no operator application).
template <typename V>
__global__ void __launch_bounds__(kThreads) cheb_last_kernel(int64_t n, const V* __restrict__ dj,
                                                             const V* __restrict__ x, int first,
                                                             const double* __restrict__ add,
                                                             double* __restrict__ out,
                                                             const int* __restrict__ status) {
  SKIP_IF_DONE(status);
  GRID_LOOP(c, n) {
    const V xv = (first ? V(0) : x[c]) + dj[c];
    out[c] = add ? add[c] + (double)xv : (double)xv;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

bool tma_make_map(CUtensorMap* map, const void* base, CUtensorMapDataType type, int es, int nx, int ny, int nz,
                  int box_w, int box_h) {
  auto fn = tma_encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * es, (cuuint64_t)nx * ny * es};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return fn(map, type, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Maps of the operator's coefficient arrays and the walked input m (and, for
// the Chebyshev sweep, dinv, r, x).  False if any map cannot be made.
template <typename C>
static bool tma_maps(TmaMaps& M, const pfk_operator* op, const float* m, const C* d, const C* kx, const C* ky,
                     const C* kz, const C* dinv, const float* r, const float* x) {
  const int nx = op->nx, ny = op->ny, nz = op->nz, es = (int)sizeof(C);
  const CUtensorMapDataType ct = sizeof(C) == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  bool ok = tma_make_map(&M.m, m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, nz, kTmaMW, kTmaMH) &&
            tma_make_map(&M.kx, kx, ct, es, nx, ny, nz, kTmaMW, kTileY) &&
            tma_make_map(&M.ky, ky, ct, es, nx, ny, nz, kTileX, kTmaKyH) &&
            tma_make_map(&M.d, d, ct, es, nx, ny, nz, kTileX, kTileY) &&
            tma_make_map(&M.kz, kz, ct, es, nx, ny, nz, kTileX, kTileY);
  if (ok && dinv)
    ok = tma_make_map(&M.dinv, dinv, ct, es, nx, ny, nz, kTileX, kTileY) &&
         tma_make_map(&M.r, r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, nz, kTileX, kTileY) &&
         tma_make_map(&M.x, x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, nz, kTileX, kTileY);
  return ok;
}

// Resident blocks of a TMA walk kernel (its dynamic shared memory included).
template <typename K>
static int tma_slots(K kernel, int smem, int num_sms) {
  static const int per_sm = [&]() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kTileThreads, smem) != cudaSuccess) {
      cudaGetLastError();
      b = 1;
    }
    return b < 1 ? 1 : b;
  }();
  return per_sm * num_sms;
}

// Work decomposition (32 x 8 tiles, z-chunks sized to the resident blocks) and
// the operator's advection weights.
static TmaWalkArgs tma_args(const pfk_operator* op, int slots, const int* status, int* err) {
  TmaWalkArgs a{};
  a.nx = op->nx; a.ny = op->ny; a.nz = op->nz;
  a.tiles_x = (op->nx + kTileX - 1) / kTileX;
  a.tiles_y = (op->ny + kTileY - 1) / kTileY;
  a.zc = tiled_stencil_zc(a.tiles_x * a.tiles_y, op->nz, slots);
  a.zchunks = (op->nz + a.zc - 1) / a.zc;
  a.a0 = (float)op->adv[0]; a.a1 = (float)op->adv[1]; a.a2 = (float)op->adv[2];
  a.up0 = op->upw[0] < 0 ? -1 : 1; a.up1 = op->upw[1] < 0 ? -1 : 1; a.up2 = op->upw[2] < 0 ? -1 : 1;
  a.status = status;
  a.err = err;
  return a;
}

template <typename C, bool CHEB>
static cudaError_t tma_launch(const TmaMaps& M, TmaWalkArgs a, const pfk_operator* op, cudaStream_t st) {
  using L = TmaStage<float, C, CHEB ? 3 : 0>;
  const bool adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
  const int slots = adv ? tma_slots(tma_walk_kernel<C, true, CHEB>, L::smem, op->ctx->num_sms)
                        : tma_slots(tma_walk_kernel<C, false, CHEB>, L::smem, op->ctx->num_sms);
  const TmaWalkArgs d = tma_args(op, slots, a.status, a.err);
  a.tiles_x = d.tiles_x; a.tiles_y = d.tiles_y; a.zc = d.zc; a.zchunks = d.zchunks;
  a.nx = d.nx; a.ny = d.ny; a.nz = d.nz;
  a.a0 = d.a0; a.a1 = d.a1; a.a2 = d.a2; a.up0 = d.up0; a.up1 = d.up1; a.up2 = d.up2;
  const int units = a.tiles_x * a.tiles_y * a.zchunks;
  if (adv) tma_walk_kernel<C, true, CHEB><<<units, kTileThreads, L::smem, st>>>(M, a);
  else tma_walk_kernel<C, false, CHEB><<<units, kTileThreads, L::smem, st>>>(M, a);
  return cudaGetLastError();
}

template <typename V, typename C>
static StencilT<V, C> make_stencil(const pfk_operator* op, const C* d, const C* kx, const C* ky, const C* kz,
                                   const C* dinv) {
  StencilT<V, C> A;
  A.d = d; A.kx = kx; A.ky = ky; A.kz = kz; A.dinv = dinv;
  A.nx = op->nx; A.ny = op->ny; A.nz = op->nz; A.ndim = op->ndim;
  A.a0 = (V)op->adv[0]; A.a1 = (V)op->adv[1]; A.a2 = (V)op->adv[2];
  A.u0 = op->upw[0]; A.u1 = op->upw[1]; A.u2 = op->upw[2];
  A.n = op->n;
  return A;
}

template <typename V, typename C>
static cudaError_t inner_pcg(const pfk_pc* pc, StencilT<V, C> A, const double* v, double* out, const double* add,
                             const int* status, cudaStream_t st) {
  const int64_t n = A.n;
  V* base = (V*)pc->buf;
  V* r = base;
  V* s = base + n;
  V* x = base + 2 * n;
  V* p[2] = {base + 3 * n, base + 4 * n};
  const int k = pc->inner;
  const int blocks = stream_blocks(pc->ctx, n, 8);
  const int sblocks = stream_blocks(pc->ctx, n, 8);
  TiledStencil<V, C> T;
  const pfk_operator* op = pc->op;
  const bool adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
  const int slots = adv ? tiled_stencil_slots(pcg_c_kernel<V, C, true>, pc->ctx->num_sms)
                        : tiled_stencil_slots(pcg_c_kernel<V, C, false>, pc->ctx->num_sms);
  const int units = tiled_stencil_setup<V, C>(T, op, A.d, A.kx, A.ky, A.kz, slots);
  const int tblocks = units < pc->partials_cap ? units : pc->partials_cap;
  PcCtl* ctl = pc->ctl;
  pcg_first_kernel<V, C><<<blocks, kThreads, 0, st>>>(A, v, p[0], ctl, k, pc->partials, status);
  // reduced precision on an aligned 3-D grid: the TMA-pipelined walk
  bool tma = false;
  TmaMaps maps[2];
  if constexpr (std::is_same<V, float>::value) {
    tma = tma_walk_usable(op->nx, op->nz, {p[0], p[1], s, A.d, A.kx, A.ky, A.kz}) &&
          tma_maps<C>(maps[0], op, p[0], A.d, A.kx, A.ky, A.kz, nullptr, nullptr, nullptr) &&
          tma_maps<C>(maps[1], op, p[1], A.d, A.kx, A.ky, A.kz, nullptr, nullptr, nullptr);
  }
  auto pcg_c = [&](const V* pv, int i) {
    if constexpr (std::is_same<V, float>::value) {
      if (tma) {
        TmaWalkArgs a{};
        a.s = s;
        a.ctl = ctl;
        a.i = i;
        a.partials = pc->partials;
        a.status = status;
        a.err = (int*)pc->ctx->scratch_counter + 3;
        tma_launch<C, false>(maps[pv == p[0] ? 0 : 1], a, op, st);
        return;
      }
    }
    if (T.adv) pcg_c_kernel<V, C, true><<<tblocks, kTileThreads, 0, st>>>(T, pv, s, ctl, i, pc->partials, status);
    else pcg_c_kernel<V, C, false><<<tblocks, kTileThreads, 0, st>>>(T, pv, s, ctl, i, pc->partials, status);
  };
  pcg_c(p[0], 0);
  for (int i = 1; i < k; ++i) {
    pcg_a_kernel<V, C><<<blocks, kThreads, 0, st>>>(A, v, r, s, ctl, i, pc->partials, status);
    pcg_b_kernel<V, C><<<sblocks, kThreads, 0, st>>>(A, r, p[(i - 1) & 1], p[i & 1], x, ctl, i, status);
    pcg_c(p[i & 1], i);
  }
  pcg_final_kernel<V, C><<<sblocks, kThreads, 0, st>>>(n, p[(k - 1) & 1], x, add, out, ctl, k, status);
  return cudaGetLastError();
}

template <typename V, typename C>
static cudaError_t chebyshev(const pfk_pc* pc, StencilT<V, C> A, const double* v, double* out, const double* add,
                             const int* status, cudaStream_t st) {
  const int64_t n = A.n;
  V* base = (V*)pc->buf;
  V* r = base;
  V* x = base + n;
  V* dv[2] = {base + 2 * n, base + 3 * n};
  const int k = pc->inner;
  const int sblocks = stream_blocks(pc->ctx, n, 8);
  const double theta = (pc->hi + pc->lo) / 2.0, delta = (pc->hi - pc->lo) / 2.0;
  const double sigma1 = theta / delta;
  double rho = 1.0 / sigma1;
  TiledStencil<V, C> T;
  const pfk_operator* op = pc->op;
  const bool adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
  const int slots = adv ? tiled_stencil_slots(cheb_sweep_kernel<V, C, true>, pc->ctx->num_sms)
                        : tiled_stencil_slots(cheb_sweep_kernel<V, C, false>, pc->ctx->num_sms);
  const int units = tiled_stencil_setup<V, C>(T, op, A.d, A.kx, A.ky, A.kz, slots);
  // reduced precision on an aligned 3-D grid: the TMA-pipelined walk
  bool tma = false;
  TmaMaps maps[2];
  if constexpr (std::is_same<V, float>::value) {
    tma = tma_walk_usable(op->nx, op->nz, {dv[0], dv[1], r, x, A.d, A.kx, A.ky, A.kz, A.dinv}) &&
          tma_maps<C>(maps[0], op, dv[0], A.d, A.kx, A.ky, A.kz, A.dinv, r, x) &&
          tma_maps<C>(maps[1], op, dv[1], A.d, A.kx, A.ky, A.kz, A.dinv, r, x);
  }
  cheb_init_kernel<V, C><<<sblocks, kThreads, 0, st>>>(A, v, r, dv[0], (V)(1.0 / theta), status);
  for (int j = 0; j + 1 < k; ++j) {
    const double rho_new = 1.0 / (2.0 * sigma1 - rho);
    const V c1 = (V)(rho_new * rho), c2 = (V)(2.0 * rho_new / delta);
    if constexpr (std::is_same<V, float>::value) {
      if (tma) {
        TmaWalkArgs a{};
        a.dn = dv[(j + 1) & 1];
        a.r = r;
        a.x = x;
        a.first = j == 0;
        a.c1 = c1;
        a.c2 = c2;
        a.status = status;
        a.err = (int*)pc->ctx->scratch_counter + 3;
        tma_launch<C, true>(maps[j & 1], a, op, st);
        rho = rho_new;
        continue;
      }
    }
    if (T.adv)
      cheb_sweep_kernel<V, C, true><<<units, kTileThreads, 0, st>>>(T, A.dinv, dv[j & 1], dv[(j + 1) & 1], r, x, j,
                                                                    c1, c2, status);
    else
      cheb_sweep_kernel<V, C, false><<<units, kTileThreads, 0, st>>>(T, A.dinv, dv[j & 1], dv[(j + 1) & 1], r, x, j,
                                                                     c1, c2, status);
    rho = rho_new;
  }
  cheb_last_kernel<V><<<sblocks, kThreads, 0, st>>>(n, dv[(k - 1) & 1], x, k == 1, add, out, status);
  return cudaGetLastError();
}

cudaError_t pc_apply(const pfk_pc* pc, const double* v, double* out, const double* add, const int* status,
                     cudaStream_t st) {
  if (pc->kind == PFK_PC_BLOCK_UPPER) return nested_apply(pc, v, out, add, status, st);
  const pfk_operator* op = pc->op;
  const int64_t n = op->n;
  if (pc->kind == PFK_PC_NONE || pc->kind == PFK_PC_JACOBI) {
    const double* dinv = pc->kind == PFK_PC_NONE ? nullptr : (op->rowptr && op->csr_dinv ? op->csr_dinv : op->dinv);
    jacobi_kernel<<<stream_blocks(pc->ctx, n, 8), kThreads, 0, st>>>(dinv, v, add, out, n, status);
    return cudaGetLastError();
  }
  if (pc->kind == PFK_PC_NOISY) {
    const int blocks = stream_blocks(pc->ctx, n, 2);
    noisy_norm_kernel<<<blocks, kThreads, 0, st>>>(v, n, pc->noise_eta, pc->bank_inv_norm, pc->bank_count, pc->ctl,
                                                   pc->partials, status);
    noisy_apply_kernel<<<stream_blocks(pc->ctx, n, 8), kThreads, 0, st>>>(v, pc->bank, n, pc->ctl, add, out,
                                                                          status);
    return cudaGetLastError();
  }
  if (pc->kind == PFK_PC_INNER_PCG) {
    if (pc->precision == PFK_FP64)
      return inner_pcg<double, double>(pc, make_stencil<double, double>(op, op->d, op->kx, op->ky, op->kz, op->dinv),
                                       v, out, add, status, st);
    if (pc->precision == PFK_FP32)
      return inner_pcg<float, float>(pc, make_stencil<float, float>(op, op->d32, op->kx32, op->ky32, op->kz32,
                                                                    op->dinv32), v, out, add, status, st);
    return inner_pcg<float, __nv_bfloat16>(pc, make_stencil<float, __nv_bfloat16>(op, op->d16, op->kx16, op->ky16,
                                                                                   op->kz16, op->dinv16),
                                           v, out, add, status, st);
  }
  // Chebyshev
  if (pc->precision == PFK_FP64)
    return chebyshev<double, double>(pc, make_stencil<double, double>(op, op->d, op->kx, op->ky, op->kz, op->dinv), v,
                                     out, add, status, st);
  if (pc->precision == PFK_FP32)
    return chebyshev<float, float>(pc, make_stencil<float, float>(op, op->d32, op->kx32, op->ky32, op->kz32,
                                                                  op->dinv32), v, out, add, status, st);
  return chebyshev<float, __nv_bfloat16>(pc, make_stencil<float, __nv_bfloat16>(op, op->d16, op->kx16, op->ky16,
                                                                                op->kz16, op->dinv16),
                                         v, out, add, status, st);
}

pfk_status create_noisy_pc(pfk_context* ctx, const pfk_operator* op, double eta, const double* bank, int count,
                           int bank_on_device, pfk_pc* pc) {
  pc->ctx = ctx;
  pc->op = op;
  pc->kind = PFK_PC_NOISY;
  pc->noise_eta = eta;
  pc->bank_count = count;
  const int64_t n = op->n;
  cudaStream_t st = ctx->stream;
  const size_t bytes = (size_t)count * (size_t)n * sizeof(double);
  PFK_CUDA(ctx, cudaMallocAsync((void**)&pc->bank, bytes, st));
  PFK_CUDA(ctx, cudaMemcpyAsync(pc->bank, bank, bytes, bank_on_device ? cudaMemcpyDeviceToDevice
                                                                        : cudaMemcpyHostToDevice, st));
  PFK_CUDA(ctx, cudaMallocAsync((void**)&pc->bank_inv_norm, (size_t)count * sizeof(double) + sizeof(int), st));
  int* bad = (int*)(pc->bank_inv_norm + count);
  PFK_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), st));
  noisy_row_norms_kernel<<<count, kThreads, 0, st>>>(pc->bank, n, pc->bank_inv_norm, bad);
  PFK_CUDA(ctx, cudaGetLastError());
  PFK_CUDA(ctx, cudaMallocAsync((void**)&pc->ctl, sizeof(PcCtl), st));
  PFK_CUDA(ctx, cudaMemsetAsync(pc->ctl, 0, sizeof(PcCtl), st));
  pc->partials_cap = ctx->num_sms * 8;
  PFK_CUDA(ctx, cudaMallocAsync((void**)&pc->partials, (size_t)pc->partials_cap * sizeof(double), st));
  int hbad = 0;
  PFK_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PFK_CUDA(ctx, cudaStreamSynchronize(st));
  if (hbad) {
    set_error(ctx, "a noise bank row has zero norm");
    return PFK_ERR_INVALID;
  }
  return PFK_OK;
}

pfk_status create_pc(pfk_context* ctx, const pfk_operator* op, const pfk_pc_desc* desc, pfk_pc* pc) {
  pc->ctx = ctx;
  pc->op = op;
  pc->kind = desc->kind;
  pc->inner = desc->inner_iters;
  pc->precision = desc->precision;
  const bool stencil = op->d != nullptr;
  if (pc->kind < PFK_PC_NONE || pc->kind > PFK_PC_CHEBYSHEV) {   // PFK_PC_NOISY has its own constructor
    set_error(ctx, "unknown preconditioner kind");
    return PFK_ERR_INVALID;
  }
  if ((pc->kind == PFK_PC_INNER_PCG || pc->kind == PFK_PC_CHEBYSHEV)) {
    if (!stencil) {
      set_error(ctx, "inner-iteration preconditioners need a stencil operator");
      return PFK_ERR_INVALID;
    }
    if (pc->inner < 1 || pc->inner > 64) {
      set_error(ctx, "inner_iters must be in [1, 64]");
      return PFK_ERR_INVALID;
    }
    if (pc->precision < PFK_FP64 || pc->precision > PFK_BF16_COEF_FP32) {
      set_error(ctx, "unknown precision");
      return PFK_ERR_INVALID;
    }
    pfk_status s = ensure_reduced_copies(const_cast<pfk_operator*>(op), pc->precision);
    if (s != PFK_OK) return s;
    const size_t esz = pc->precision == PFK_FP64 ? sizeof(double) : sizeof(float);
    pc->buf_bytes = 5 * (size_t)op->n * esz;
    PFK_CUDA(ctx, cudaMallocAsync(&pc->buf, pc->buf_bytes, ctx->stream));
    PFK_CUDA(ctx, cudaMallocAsync((void**)&pc->ctl, sizeof(PcCtl), ctx->stream));
    PFK_CUDA(ctx, cudaMemsetAsync(pc->ctl, 0, sizeof(PcCtl), ctx->stream));
    const int units = tiled_stencil_max_units(op->nx, op->ny, op->nz);
    pc->partials_cap = ctx->num_sms * 8 > units ? ctx->num_sms * 8 : units;
    PFK_CUDA(ctx, cudaMallocAsync((void**)&pc->partials, (size_t)pc->partials_cap * sizeof(double), ctx->stream));
    if (pc->kind == PFK_PC_CHEBYSHEV) {
      if (desc->cheb_lo == 0.0 && desc->cheb_hi == 0.0) {
        pc->lo = 0.1 * op->gersh;
        pc->hi = 1.1 * op->gersh;
      } else {
        pc->lo = desc->cheb_lo;
        pc->hi = desc->cheb_hi;
      }
      if (!(pc->hi > pc->lo) || !(pc->lo > 0.0)) {
        set_error(ctx, "Chebyshev bounds must satisfy 0 < lo < hi");
        return PFK_ERR_INVALID;
      }
    }
  } else if (pc->kind == PFK_PC_JACOBI && !stencil && !op->csr_dinv) {
    set_error(ctx, "Jacobi needs the operator diagonal");
    return PFK_ERR_INVALID;
  }
  PFK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PFK_OK;
}

}  // namespace pfk

// ---------------------------------------------------------------------------
// Allocation-free inner Jacobi-PCG application (pfk_pc_apply_inner_pcg_noalloc)
//
// For callers that must not allocate device memory when they apply the
// preconditioner.  The scratch of the inner iterations (five work vectors, the
// per-block partial sums and the control block) lives in one file-scope device
// array instead of pfk_pc's cudaMalloc'd buffers; the kernels are the same.
// The array exists once per GPU that loads the library and stays allocated
// until the process exits.  Host code cannot use the array's name as a device
// address: its address is fetched per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------

#include <mutex>

namespace pfk {

constexpr int64_t kNoallocMaxN = PFK_NOALLOC_MAX_N;
// One partial sum per block of the inner PCG's reduction kernels: pcg_first and
// pcg_a launch up to 8 blocks per SM (stream_blocks(ctx, n, 8)), never more
// than one block per 256 unknowns, and the stencil walk is capped at this
// count; a call whose grid would exceed it is rejected.
constexpr int64_t kNoallocPartials = 2048;
constexpr int64_t kNoallocCtlDoubles = (sizeof(PcCtl) + sizeof(double) - 1) / sizeof(double);
constexpr int64_t kNoallocDoubles = 5 * kNoallocMaxN + kNoallocPartials + kNoallocCtlDoubles;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

constexpr int kNoallocMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static double* g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of g_noalloc_scratch on ctx's device (looked up once per device).
static pfk_status noalloc_scratch(pfk_context* ctx, double** out) {
  if (ctx->device < 0 || ctx->device >= kNoallocMaxDevices) {
    set_error(ctx, "device index too large for the allocation-free entry point");
    return PFK_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[ctx->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress (static scratch)");
    g_noalloc_addr[ctx->device] = (double*)p;
  }
  *out = g_noalloc_addr[ctx->device];
  return PFK_OK;
}

}  // namespace pfk

extern "C" pfk_status pfk_pc_apply_inner_pcg_noalloc(pfk_context* ctx, const pfk_operator* op, int inner_iters,
                                                      const double* v, double* y) {
  using namespace pfk;
  if (!ctx || !op || !v || !y) {
    set_error(ctx, "NULL argument");
    return PFK_ERR_INVALID;
  }
  if (v == y) {
    set_error(ctx, "v and y must not overlap");
    return PFK_ERR_INVALID;
  }
  if (!op->d) {
    set_error(ctx, "the allocation-free inner PCG needs a stencil operator");
    return PFK_ERR_INVALID;
  }
  if (inner_iters < 1 || inner_iters > 64) {
    set_error(ctx, "inner_iters must be in [1, 64]");
    return PFK_ERR_INVALID;
  }
  if (op->n > kNoallocMaxN) {
    set_error(ctx, "operator size exceeds PFK_NOALLOC_MAX_N (262144 unknowns), the capacity of the static "
                   "scratch of the allocation-free entry point");
    return PFK_ERR_INVALID;
  }
  if (stream_blocks(ctx, op->n, 8) > kNoallocPartials) {
    set_error(ctx, "the inner PCG's reduction grid on this GPU exceeds the 2048 partial sums of the static "
                   "scratch of the allocation-free entry point");
    return PFK_ERR_INVALID;
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  double* scratch = nullptr;
  pfk_status s = noalloc_scratch(ctx, &scratch);
  if (s != PFK_OK) return s;
  pfk_pc tmp;
  tmp.ctx = ctx;
  tmp.op = op;
  tmp.kind = PFK_PC_INNER_PCG;
  tmp.inner = inner_iters;
  tmp.precision = PFK_FP64;
  tmp.buf = scratch;
  tmp.buf_bytes = 5 * (size_t)op->n * sizeof(double);
  tmp.partials = scratch + 5 * kNoallocMaxN;
  tmp.partials_cap = (int)kNoallocPartials;
  tmp.ctl = (PcCtl*)(scratch + 5 * kNoallocMaxN + kNoallocPartials);
  // the control block keeps the previous call's values: its arrival counter
  // must start at zero
  PFK_CUDA(ctx, cudaMemsetAsync(tmp.ctl, 0, sizeof(PcCtl), ctx->stream));
  const StencilT<double, double> A = make_stencil<double, double>(op, op->d, op->kx, op->ky, op->kz, op->dinv);
  e = inner_pcg<double, double>(&tmp, A, v, y, nullptr, nullptr, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "inner PCG kernels");
  PFK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PFK_OK;
}
