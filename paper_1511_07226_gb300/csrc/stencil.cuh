// Tiled z-marching application of the 7-point (3D) / 5-point (2D)
// finite-volume stencil (A of every listing; T_spmv of the Sec. 8 model).
//
// A block of 32 x 8 threads owns a 32 x 8 tile of an x-y plane and walks a
// chunk of consecutive z planes.  Each thread keeps its column's values of the
// input vector at k - 1, k, k + 1 (and kz at k - 1) in registers, takes the
// x neighbours from its warp neighbours (shuffles) and the y neighbours from a
// double-buffered shared-memory copy of the plane, so every input array is read
// from HBM once; only the tile edges are re-read (from L2).  One block-wide
// barrier per plane.
//
// The epilogue functor receives (cell index, (A m)_c, m_c, pre) for every
// cell of the domain, where pre = epi.pre(c) was loaded one plane ahead
// together with the stencil's own operands (the epilogue's extra inputs are
// prefetched too); it may accumulate per-thread partial sums.
#pragma once

#include "pfk_internal.cuh"

#include <cmath>

namespace pfk {

constexpr int kTileX = 32;
constexpr int kTileY = 8;
constexpr int kTileThreads = kTileX * kTileY;

template <typename V, typename C>
struct TiledStencil {
  const C* d;
  const C* kx;
  const C* ky;
  const C* kz;
  int nx, ny, nz;
  int tiles_x, tiles_y, zc, zchunks;   // work decomposition: tiles_x * tiles_y * zchunks units of zc planes
  V a0, a1, a2;                        // upwind weights h |v_d| (0: no advection along d)
  int up0, up1, up2;                   // side of the upwind neighbour: -1 (v_d > 0) or +1
  bool adv;                            // any weight non-zero
};

template <typename V, typename C>
__device__ __forceinline__ V ld_coef(const C* p, int64_t c) {
  return (V)p[c];
}
template <>
__device__ __forceinline__ float ld_coef<float, __nv_bfloat16>(const __nv_bfloat16* p, int64_t c) {
  return __bfloat162float(p[c]);
}

// Values of one plane that a thread needs for its W cells: the input at
// k + 1 and the coefficients at k of each cell, and the tile-edge neighbours
// that come from global memory (x edges: lane 0 of segment 0 and lane 31 of
// segment W - 1; y edges: rows 0 and kTileY - 1).
template <typename V, int W, typename Pre>
struct PlaneVals {
  Pre e[W];                 // the epilogue's prefetched inputs
  V mup[W], d[W], kx[W], ky[W], kz[W];
  V mxm, kxm, mxp;          // m at i - 1 and kx at i - 1 (left edge), m at i + 1 (right edge)
  V mym[W], kym[W], myp[W]; // m and ky at j - 1, m at j + 1 (rows 0 / kTileY - 1)
};

template <typename V, typename C, int W, typename Epi>
__device__ __forceinline__ void load_plane(const TiledStencil<V, C>& A, const V* __restrict__ m, int64_t c0, int k,
                                           int i0, int j, int tx, int ty, int64_t sxy, bool jin, const Epi& epi,
                                           PlaneVals<V, W, typename Epi::Pre>& p) {
  p.mxm = p.kxm = p.mxp = V(0);
#pragma unroll
  for (int w = 0; w < W; ++w) {
    p.mup[w] = p.d[w] = p.kx[w] = p.ky[w] = p.kz[w] = V(0);
    p.mym[w] = p.kym[w] = p.myp[w] = V(0);
    const int i = i0 + kTileX * w;
    if (!jin || i >= A.nx) continue;
    const int64_t c = c0 + kTileX * w;
    p.e[w] = epi.pre(c);
    if (k + 1 < A.nz) p.mup[w] = m[c + sxy];
    p.d[w] = ld_coef<V, C>(A.d, c);
    p.kx[w] = ld_coef<V, C>(A.kx, c);
    p.ky[w] = ld_coef<V, C>(A.ky, c);
    if (A.nz > 1) p.kz[w] = ld_coef<V, C>(A.kz, c);
    if (w == 0 && tx == 0 && i > 0) {
      p.mxm = m[c - 1];
      p.kxm = ld_coef<V, C>(A.kx, c - 1);
    }
    if (w == W - 1 && tx == kTileX - 1 && i + 1 < A.nx) p.mxp = m[c + 1];
    if (ty == 0 && j > 0) {
      p.mym[w] = m[c - A.nx];
      p.kym[w] = ld_coef<V, C>(A.ky, c - A.nx);
    }
    if (ty == kTileY - 1 && j + 1 < A.ny) p.myp[w] = m[c + A.nx];
  }
}

// Walks every work unit assigned to this block; all threads of the block must
// call it (it contains block-wide barriers).  A tile is W segments of 32
// consecutive x cells by kTileY rows; lane tx of row ty owns cells
// x0 + tx + 32 w.  The loads of plane k + 1 are issued before plane k is
// computed, so HBM latency overlaps a whole plane step.  ADV: the operator has
// an upwind advection part (am* / ap* non-zero).
template <typename V, typename C, bool ADV, int W, typename Epi>
__device__ __forceinline__ void tiled_stencil_walk(const TiledStencil<V, C>& A, const V* __restrict__ m, Epi& epi) {
  constexpr int TW = kTileX * W;
  __shared__ V sm_m[2][kTileY][TW + 1];
  __shared__ V sm_ky[2][kTileY][TW + 1];
  const int tx = threadIdx.x & (kTileX - 1);
  const int ty = threadIdx.x / kTileX;
  const int64_t sxy = (int64_t)A.nx * A.ny;
  const int tiles_x = (A.nx + TW - 1) / TW;
  const int units = tiles_x * A.tiles_y * A.zchunks;
  int buf = 0;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int tile = u % (tiles_x * A.tiles_y);
    const int chunk = u / (tiles_x * A.tiles_y);
    const int i0 = (tile % tiles_x) * TW + tx;
    const int j = (tile / tiles_x) * kTileY + ty;
    const int z0 = chunk * A.zc;
    const int z1 = min(A.nz, z0 + A.zc);
    const bool jin = j < A.ny;
    const int64_t col0 = (int64_t)j * A.nx + i0;
    V mdn[W], mc[W], kzdn[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      mdn[w] = mc[w] = kzdn[w] = V(0);
      const int64_t col = col0 + kTileX * w;
      if (jin && i0 + kTileX * w < A.nx) {
        if (z0 > 0) {
          mdn[w] = m[col + (int64_t)(z0 - 1) * sxy];
          kzdn[w] = ld_coef<V, C>(A.kz, col + (int64_t)(z0 - 1) * sxy);
        }
        mc[w] = m[col + (int64_t)z0 * sxy];
      }
    }
    PlaneVals<V, W, typename Epi::Pre> cur, nxt;
    load_plane<V, C, W>(A, m, col0 + (int64_t)z0 * sxy, z0, i0, j, tx, ty, sxy, jin, epi, cur);
    for (int k = z0; k < z1; ++k) {
      const int64_t c0 = col0 + (int64_t)k * sxy;
      if (k + 1 < z1) load_plane<V, C, W>(A, m, c0 + sxy, k + 1, i0, j, tx, ty, sxy, jin, epi, nxt);
      // x neighbours from the warp: lane - 1 / lane + 1 of the same segment,
      // lane 31 / lane 0 of the neighbouring segment, or the tile edge
      V mxm[W], kxm[W], mxp[W];
#pragma unroll
      for (int w = 0; w < W; ++w) {
        mxm[w] = __shfl_up_sync(0xffffffffu, mc[w], 1);
        kxm[w] = __shfl_up_sync(0xffffffffu, cur.kx[w], 1);
        mxp[w] = __shfl_down_sync(0xffffffffu, mc[w], 1);
      }
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const V prev_m = __shfl_sync(0xffffffffu, w > 0 ? mc[w > 0 ? w - 1 : 0] : V(0), kTileX - 1);
        const V prev_k = __shfl_sync(0xffffffffu, w > 0 ? cur.kx[w > 0 ? w - 1 : 0] : V(0), kTileX - 1);
        const V next_m = __shfl_sync(0xffffffffu, w + 1 < W ? mc[w + 1 < W ? w + 1 : 0] : V(0), 0);
        if (tx == 0) {
          mxm[w] = w == 0 ? cur.mxm : prev_m;
          kxm[w] = w == 0 ? cur.kxm : prev_k;
        }
        if (tx == kTileX - 1) mxp[w] = w == W - 1 ? cur.mxp : next_m;
      }
      // y neighbours through shared memory
#pragma unroll
      for (int w = 0; w < W; ++w) {
        sm_m[buf][ty][tx + kTileX * w] = mc[w];
        sm_ky[buf][ty][tx + kTileX * w] = cur.ky[w];
      }
      __syncthreads();
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int i = i0 + kTileX * w;
        if (!jin || i >= A.nx) continue;
        const int xs = tx + kTileX * w;
        const V mym = ty > 0 ? sm_m[buf][ty - 1][xs] : cur.mym[w];
        const V kym = ty > 0 ? sm_ky[buf][ty - 1][xs] : cur.kym[w];
        const V myp = ty < kTileY - 1 ? sm_m[buf][ty + 1][xs] : cur.myp[w];
        // neighbours outside the domain are zero (loads skipped) and the
        // +x / +y / +z coefficients are zero on the far boundary, so the
        // diffusion terms need no guards
        V acc = cur.d[w] * mc[w];
        acc -= kxm[w] * mxm[w];
        acc -= cur.kx[w] * mxp[w];
        acc -= kym * mym;
        acc -= cur.ky[w] * myp;
        if (A.nz > 1) {
          acc -= kzdn[w] * mdn[w];
          acc -= cur.kz[w] * cur.mup[w];
        }
        if (ADV) {
          // one upwind neighbour per direction (the other side's weight is
          // zero): select it, then one FMA; a neighbour outside the domain is
          // the zero ghost value
          const V ux = A.up0 < 0 ? (i > 0 ? mxm[w] : V(0)) : (i + 1 < A.nx ? mxp[w] : V(0));
          const V uy = A.up1 < 0 ? (j > 0 ? mym : V(0)) : (j + 1 < A.ny ? myp : V(0));
          acc -= A.a0 * ux;
          acc -= A.a1 * uy;
          if (A.nz > 1) {
            const V uz = A.up2 < 0 ? (k > 0 ? mdn[w] : V(0)) : (k + 1 < A.nz ? cur.mup[w] : V(0));
            acc -= A.a2 * uz;
          }
        }
        epi(c0 + kTileX * w, acc, mc[w], cur.e[w]);
      }
      buf ^= 1;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        mdn[w] = mc[w];
        mc[w] = cur.mup[w];
        kzdn[w] = cur.kz[w];
      }
      cur = nxt;
    }
  }
}

// Host: the tile decomposition of an operator.  One block per work unit (a
// tile and a chunk of zc consecutive planes).  zc is chosen against the
// number of blocks the GPU holds at once (`slots`): time ~ waves x (zc + 1/2)
// (half a plane for the priming loads), so the last wave is not mostly empty.
inline int tiled_stencil_zc(int tiles, int nz, int slots) {
  if (nz < 4) return nz;
  int best = nz;
  double best_cost = 1e300;
  const int zmax = nz < 32 ? nz : 32;
  for (int zc = 2; zc <= zmax; ++zc) {
    const double units = (double)tiles * (double)((nz + zc - 1) / zc);
    const double cost = std::ceil(units / (double)slots) * (zc + 0.5);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = zc;
    }
  }
  return best;
}

inline int tiled_stencil_tiles(int nx, int ny, int w) {
  return ((nx + kTileX * w - 1) / (kTileX * w)) * ((ny + kTileY - 1) / kTileY);
}

// Upper bound of the unit count of any decomposition (zc >= 2, one cell per thread).
inline int tiled_stencil_max_units(int nx, int ny, int nz) {
  return tiled_stencil_tiles(nx, ny, 1) * (nz < 4 ? 1 : (nz + 1) / 2);
}

// Blocks of `kernel` (kTileThreads threads) resident on the whole GPU.
template <typename K>
int tiled_stencil_slots(K kernel, int num_sms) {
  static const int per_sm = [&]() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kTileThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      b = 1;
    }
    return b < 1 ? 1 : b;
  }();
  return per_sm * num_sms;
}

// Cells per thread along x: FP64 walks are bound by the FP64 pipe (one cell
// per thread keeps registers low); the FP32 walk with FP32 coefficients is
// bound by memory latency (two cells per thread double the loads in flight;
// measured 1.35x faster at 256^3).  With BF16 coefficients two cells per
// thread measured slower (register pressure), so it keeps one.
template <typename V, typename C>
__host__ __device__ constexpr int tiled_width() { return (sizeof(V) == 8 || sizeof(C) == 2) ? 1 : 2; }

template <typename V, typename C>
int tiled_stencil_setup(TiledStencil<V, C>& A, const pfk_operator* op, const C* d, const C* kx, const C* ky,
                        const C* kz, int slots) {
  A.d = d; A.kx = kx; A.ky = ky; A.kz = kz;
  A.nx = op->nx; A.ny = op->ny; A.nz = op->nz;
  constexpr int W = tiled_width<V, C>();
  A.tiles_x = (op->nx + kTileX * W - 1) / (kTileX * W);
  A.tiles_y = (op->ny + kTileY - 1) / kTileY;
  A.zc = tiled_stencil_zc(A.tiles_x * A.tiles_y, op->nz, slots);
  A.zchunks = (op->nz + A.zc - 1) / A.zc;
  A.a0 = (V)op->adv[0];
  A.a1 = (V)op->adv[1];
  A.a2 = (V)op->adv[2];
  A.up0 = op->upw[0] < 0 ? -1 : 1;
  A.up1 = op->upw[1] < 0 ? -1 : 1;
  A.up2 = op->upw[2] < 0 ? -1 : 1;
  A.adv = op->adv[0] != 0.0 || op->adv[1] != 0.0 || op->adv[2] != 0.0;
  return A.tiles_x * A.tiles_y * A.zchunks;
}

}  // namespace pfk
