// TMA-pipelined stencil walk for the reduced-precision preconditioners (FP32
// vectors; FP32 or BF16 coefficients).
//
// The register walk of stencil.cuh keeps one plane of loads in flight per
// thread; with 4- and 2-byte operands that is too few bytes to cover HBM
// latency (ncu: 2.6-3.5 TB/s).  Here the tensor memory accelerator stages the
// operands of whole planes of a 32 x 8 tile in shared memory, four planes
// ahead: one thread issues cp.async.bulk.tensor copies per array and plane
// into a ring of kTmaStages stages, each completed through an mbarrier
// transaction count, and the block computes plane k from stages k-1, k, k+1.
// Halos come in the copies themselves (the input box spans x0-8..x0+39 and
// j0-1..j0+8; out-of-range parts are filled with zeros by the copy engine,
// which is exactly the Dirichlet ghost value; the ghost planes -1 and nz are
// zeroed in shared memory instead of copied), so the arithmetic needs no
// neighbour exchange and no boundary guards.  Every
// TMA x coordinate is a multiple of 8 elements (16 bytes).  Waits are bounded:
// a block whose copies do not arrive in time writes NaN to its outputs, sets
// an error word and returns after a bounded wait for its copies in flight.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <initializer_list>

#include "pfk_internal.cuh"
#include "stencil.cuh"

namespace pfk {

constexpr int kTmaStages = 4;
constexpr int kTmaHalo = 8;                         // x halo: keeps x coordinates 16-byte aligned
constexpr int kTmaMW = kTileX + 2 * kTmaHalo;       // 48: width of the input and kx boxes
constexpr int kTmaMH = kTileY + 2;                  // 10: height of the input box
constexpr int kTmaKyH = kTileY + 1;                 // 9: height of the ky box
constexpr unsigned kTmaSpinLimit = 1u << 22;        // polls of one wait (with back-off: ~0.3 s)

__host__ __device__ constexpr int tma_align128(int b) { return (b + 127) / 128 * 128; }

// Byte layout of one stage (all offsets 128-byte aligned).  NE extra arrays
// for the epilogue: dinv (C), r (V), x (V) for the Chebyshev sweep.
template <typename V, typename C, int NE>
struct TmaStage {
  static constexpr int m_bytes = kTmaMH * kTmaMW * (int)sizeof(V);
  static constexpr int kx_bytes = kTileY * kTmaMW * (int)sizeof(C);
  static constexpr int ky_bytes = kTmaKyH * kTileX * (int)sizeof(C);
  static constexpr int c_bytes = kTileY * kTileX * (int)sizeof(C);   // d, kz, dinv
  static constexpr int v_bytes = kTileY * kTileX * (int)sizeof(V);   // r, x
  static constexpr int off_m = 0;
  static constexpr int off_kx = off_m + tma_align128(m_bytes);
  static constexpr int off_ky = off_kx + tma_align128(kx_bytes);
  static constexpr int off_d = off_ky + tma_align128(ky_bytes);
  static constexpr int off_kz = off_d + tma_align128(c_bytes);
  static constexpr int off_dinv = off_kz + tma_align128(c_bytes);
  static constexpr int off_r = off_dinv + (NE ? tma_align128(c_bytes) : 0);
  static constexpr int off_x = off_r + (NE ? tma_align128(v_bytes) : 0);
  static constexpr int bytes = off_x + (NE ? tma_align128(v_bytes) : 0);
  // bytes the copies of one stage deliver (the mbarrier's transaction count)
  static constexpr unsigned tx_bytes =
      (unsigned)(m_bytes + kx_bytes + ky_bytes + 2 * c_bytes + (NE ? c_bytes + 2 * v_bytes : 0));
  static constexpr int smem = kTmaStages * bytes + 128;     // + room to align the base to 128 bytes
};

__device__ __forceinline__ unsigned tma_smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tma_mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tma_smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void tma_mbar_expect(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tma_smem_u32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool tma_mbar_try(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(tma_smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// False if the phase did not complete within kTmaSpinLimit polls.
__device__ __forceinline__ bool tma_mbar_wait(uint64_t* b, unsigned parity) {
  for (unsigned it = 0; it < kTmaSpinLimit; ++it) {
    if (tma_mbar_try(b, parity)) return true;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(tma_smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tma_smem_u32(bar))
      : "memory");
}

struct TmaMaps {
  CUtensorMap m, kx, ky, d, kz, dinv, r, x;
};

struct TmaWalkArgs {
  int nx, ny, nz, tiles_x, tiles_y, zc, zchunks;
  float a0, a1, a2;
  int up0, up1, up2;
  // outputs / scalars
  float* s;            // pcg_c: s = A p
  float* dn;           // Chebyshev: next direction
  float* r;            // Chebyshev: residual (read from the stage, written here)
  float* x;            // Chebyshev: iterate (read from the stage, written here)
  int first;           // Chebyshev: x_j = 0
  float c1, c2;
  PcCtl* ctl;          // pcg_c: scalars
  int i;               // pcg_c: inner iteration
  double* partials;
  const int* status;
  int* err;            // set when a wait gives up
};

// CHEB = false: s = A p and <s, p> (inner PCG); CHEB = true: one Chebyshev sweep.
template <typename C, bool ADV, bool CHEB>
__global__ void __launch_bounds__(kTileThreads) tma_walk_kernel(const __grid_constant__ TmaMaps maps, TmaWalkArgs a) {
  using V = float;
  constexpr int NE = CHEB ? 3 : 0;
  using L = TmaStage<V, C, NE>;
  if (a.status && *a.status != kRun) return;
  if (!CHEB && !(a.i < a.ctl->ok)) return;
  extern __shared__ __align__(128) unsigned char tma_smem_raw[];
  __shared__ __align__(8) uint64_t bars[kTmaStages];
  unsigned char* tma_smem = tma_smem_raw + ((128u - (tma_smem_u32(tma_smem_raw) & 127u)) & 127u);
  const int tx = threadIdx.x & (kTileX - 1);
  const int ty = threadIdx.x / kTileX;
  const int u = blockIdx.x;                                   // one work unit per block
  const int tile = u % (a.tiles_x * a.tiles_y);
  const int chunk = u / (a.tiles_x * a.tiles_y);
  const int x0 = (tile % a.tiles_x) * kTileX;
  const int j0 = (tile / a.tiles_x) * kTileY;
  const int z0 = chunk * a.zc;
  const int z1 = min(a.nz, z0 + a.zc);
  const int P0 = z0 - 1;                                      // first plane staged
  const int nplanes = (z1 - z0) + 2;                          // planes z0-1 .. z1
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTmaStages; ++s) tma_mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int p) {
    const int s = (p - P0) % kTmaStages;
    unsigned char* st = tma_smem + s * L::bytes;
    uint64_t* bar = &bars[s];
    if (p < 0 || p >= a.nz) {
      // the ghost planes below and above the grid: only their input values and
      // kz are read, and both are zero (Dirichlet ghost, no face)
      V* m = (V*)(st + L::off_m);
      for (int e = 0; e < kTmaMH * kTmaMW; ++e) m[e] = V(0);
      C* kz = (C*)(st + L::off_kz);
      for (int e = 0; e < kTileY * kTileX; ++e) kz[e] = C(0.0f);
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tma_smem_u32(bar)) : "memory");
      return;
    }
    tma_mbar_expect(bar, L::tx_bytes);
    tma_load_3d(st + L::off_m, &maps.m, x0 - kTmaHalo, j0 - 1, p, bar);
    tma_load_3d(st + L::off_kx, &maps.kx, x0 - kTmaHalo, j0, p, bar);
    tma_load_3d(st + L::off_ky, &maps.ky, x0, j0 - 1, p, bar);
    tma_load_3d(st + L::off_d, &maps.d, x0, j0, p, bar);
    tma_load_3d(st + L::off_kz, &maps.kz, x0, j0, p, bar);
    if (CHEB) {
      tma_load_3d(st + L::off_dinv, &maps.dinv, x0, j0, p, bar);
      tma_load_3d(st + L::off_r, &maps.r, x0, j0, p, bar);
      tma_load_3d(st + L::off_x, &maps.x, x0, j0, p, bar);
    }
  };
  const int prime = nplanes < kTmaStages ? nplanes : kTmaStages;
  if (threadIdx.x == 0)
    for (int t = 0; t < prime; ++t) issue(P0 + t);
  int issued = prime;                                         // planes P0 .. P0 + issued - 1 are in flight or done
  int waited = 0;                                             // planes P0 .. P0 + waited - 1 are complete
  auto wait_upto = [&](int p) -> bool {                       // wait for planes up to p (uniform result)
    bool ok = true;
    while (P0 + waited <= p) {
      const int q = P0 + waited;
      const int s = (q - P0) % kTmaStages;
      const unsigned parity = (unsigned)(((q - P0) / kTmaStages) & 1);
      ok = tma_mbar_wait(&bars[s], parity) && ok;
      ++waited;
    }
    return __syncthreads_and(ok) != 0;
  };
  const int i = x0 + tx, j = j0 + ty;
  const bool in = i < a.nx && j < a.ny;
  const int64_t sxy = (int64_t)a.nx * a.ny;
  V dot = V(0);                                               // per-thread <s, p> (FP32, as the register walk)
  bool ok = wait_upto(z0);
  for (int k = z0; k < z1 && ok; ++k) {
    ok = wait_upto(k + 1);
    if (!ok) break;
    const unsigned char* sp = tma_smem + ((k - 1 - P0) % kTmaStages) * L::bytes;
    const unsigned char* sc = tma_smem + ((k - P0) % kTmaStages) * L::bytes;
    const unsigned char* sn = tma_smem + ((k + 1 - P0) % kTmaStages) * L::bytes;
    if (in) {
      const V* m = (const V*)(sc + L::off_m);
      const C* kx = (const C*)(sc + L::off_kx);
      const C* ky = (const C*)(sc + L::off_ky);
      const int mi = (ty + 1) * kTmaMW + tx + kTmaHalo;
      const V mc = m[mi];
      const V mxm = m[mi - 1], mxp = m[mi + 1], mym = m[mi - kTmaMW], myp = m[mi + kTmaMW];
      const V mdn = ((const V*)(sp + L::off_m))[mi];
      const V mup = ((const V*)(sn + L::off_m))[mi];
      const int ci = ty * kTileX + tx;
      const V kxc = ld_coef<V, C>(kx, ty * kTmaMW + tx + kTmaHalo);
      const V kxm = ld_coef<V, C>(kx, ty * kTmaMW + tx + kTmaHalo - 1);
      const V kyc = ld_coef<V, C>(ky, (ty + 1) * kTileX + tx);
      const V kym = ld_coef<V, C>(ky, ty * kTileX + tx);
      const V kzc = ld_coef<V, C>((const C*)(sc + L::off_kz), ci);
      const V kzm = ld_coef<V, C>((const C*)(sp + L::off_kz), ci);
      const V dc = ld_coef<V, C>((const C*)(sc + L::off_d), ci);
      V acc = dc * mc;
      acc -= kxm * mxm;
      acc -= kxc * mxp;
      acc -= kym * mym;
      acc -= kyc * myp;
      acc -= kzm * mdn;
      acc -= kzc * mup;
      if (ADV) {
        acc -= a.a0 * (a.up0 < 0 ? mxm : mxp);
        acc -= a.a1 * (a.up1 < 0 ? mym : myp);
        acc -= a.a2 * (a.up2 < 0 ? mdn : mup);
      }
      const int64_t c = (int64_t)k * sxy + (int64_t)j * a.nx + i;
      if (CHEB) {
        const V xo = a.first ? V(0) : ((const V*)(sc + L::off_x))[ci];
        a.x[c] = xo + mc;
        const V rv = ((const V*)(sc + L::off_r))[ci] - acc;
        a.r[c] = rv;
        a.dn[c] = a.c1 * mc + a.c2 * (ld_coef<V, C>((const C*)(sc + L::off_dinv), ci) * rv);
      } else {
        a.s[c] = acc;
        dot += acc * mc;
      }
    }
    __syncthreads();                                          // every thread is done with plane k-1's stage
    if (issued < nplanes) {
      if (threadIdx.x == 0) issue(P0 + issued);               // plane k+3 into plane k-1's stage
      ++issued;
    }
  }
  if (!ok) {
    // copies did not arrive: mark the outputs, report, and wait (bounded) for
    // the copies still in flight before the block's shared memory is released
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    for (int k = z0; k < z1; ++k)
      if (in) {
        const int64_t c = (int64_t)k * sxy + (int64_t)j * a.nx + i;
        if (CHEB) a.r[c] = nanf("");
        else a.s[c] = nanf("");
      }
    while (waited < issued) {
      const int q = P0 + waited;
      tma_mbar_wait(&bars[(q - P0) % kTmaStages], (unsigned)(((q - P0) / kTmaStages) & 1));
      ++waited;
    }
    if (!CHEB) dot = nanf("");
  }
  if (!CHEB) {
    // block partials of <s, p>, last block finalises alpha (as pcg_c_kernel)
    double accd[1] = {(double)dot};
    __shared__ double smem[kTileThreads / 32];
    __shared__ double sums[1];
    if (reduce_last_block<1>(accd, 1, a.partials, 1, &a.ctl->counter, smem, sums) && threadIdx.x == 0) {
      const double eta = sums[0];
      if (eta == 0.0) {
        a.ctl->ok = a.i;
      } else {
        a.ctl->eta = eta;
        a.ctl->alpha[a.i] = a.ctl->gamma / eta;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn();

// 3-D tiled map over an nx x ny x nz array of element size es; false if the
// encoder is unavailable or rejects the map.
bool tma_make_map(CUtensorMap* map, const void* base, CUtensorMapDataType type, int es, int nx, int ny, int nz,
                  int box_w, int box_h);

// The TMA walk applies to 3-D grids whose x extent keeps every row 16-byte
// aligned for 2- and 4-byte elements, with 16-byte aligned arrays.
inline bool tma_walk_usable(int nx, int nz, std::initializer_list<const void*> arrays) {
  if (nz < 2 || nx % 8 != 0 || !tma_encode_fn()) return false;
  for (const void* p : arrays)
    if (!p || ((uintptr_t)p & 15u)) return false;
  return true;
}

}  // namespace pfk
