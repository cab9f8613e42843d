// C ABI entry points (include/pfk.h): argument checking, handle lifetime and
// host <-> device staging.  All compute is in the kernels of the other files.
#include "pfk_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

namespace pfk {

pfk_status create_stencil(pfk_context* ctx, const pfk_operator_desc* desc, pfk_operator* op);
pfk_status create_csr(pfk_context* ctx, const pfk_operator_desc* desc, pfk_operator* op);
pfk_status create_pc(pfk_context* ctx, const pfk_operator* op, const pfk_pc_desc* desc, pfk_pc* pc);
pfk_status create_noisy_pc(pfk_context* ctx, const pfk_operator* op, double eta, const double* bank, int count,
                           int bank_on_device, pfk_pc* pc);
pfk_status create_nested_pc(pfk_context* ctx, const pfk_operator* K, const pfk_operator* Bt,
                            const double* schur_diag, const pfk_inner_solve* inner, pfk_pc* pc);
pfk_status run_solve(pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, const pfk_solve_params* prm,
                     const double* b, double* x, pfk_solve_info* info);
pfk_status solve_workspace_bytes(int method, int mmax, int64_t n, int64_t* bytes);
bool method_supported(int method);
cudaError_t fp64_probe(pfk_context* ctx, int iters, double* tflops, double* ms_out);

static thread_local std::string g_thread_error;

void set_error(pfk_context* ctx, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_thread_error = msg;
}

pfk_status cuda_fail(pfk_context* ctx, cudaError_t e, const char* what) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s failed: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  cudaGetLastError();
  set_error(ctx, buf);
  return e == cudaErrorMemoryAllocation ? PFK_ERR_OOM : PFK_ERR_CUDA;
}

}  // namespace pfk

using namespace pfk;

#define CHECK_ARG(ctx, cond, msg)            \
  do {                                       \
    if (!(cond)) {                           \
      set_error(ctx, msg);                   \
      return PFK_ERR_INVALID;                \
    }                                        \
  } while (0)

extern "C" {

int pfk_abi_version(void) { return PFK_ABI_VERSION; }

const char* pfk_last_error(const pfk_context* ctx) {
  return ctx ? ctx->err.c_str() : g_thread_error.c_str();
}

pfk_status pfk_create_context(int device, void* cuda_stream, pfk_context** out) {
  CHECK_ARG(nullptr, out != nullptr, "ctx output pointer is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
  CHECK_ARG(nullptr, device >= 0 && device < count, "no such CUDA device");
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
  pfk_context* ctx = new (std::nothrow) pfk_context();
  if (!ctx) return PFK_ERR_OOM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if ((e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) {
    delete ctx;
    return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
  }
  // scratch for standalone reductions: partials of up to 8 blocks per SM, a counter pair, outputs
  const size_t np = (size_t)ctx->num_sms * 8 + 64;
  if ((e = cudaMalloc((void**)&ctx->scratch_partials, np * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc((void**)&ctx->scratch_counter, 4 * sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMalloc((void**)&ctx->scratch_out, 8 * sizeof(double))) != cudaSuccess) {
    pfk_destroy_context(ctx);
    return cuda_fail(nullptr, e, "cudaMalloc (context scratch)");
  }
  if ((e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    pfk_destroy_context(ctx);
    return cuda_fail(nullptr, e, "cudaStreamCreate (capture stream)");
  }
  if ((e = cudaMallocHost((void**)&ctx->pinned, 2 * sizeof(SolveCtl))) != cudaSuccess) {
    pfk_destroy_context(ctx);
    return cuda_fail(nullptr, e, "cudaMallocHost (status words)");
  }
  // stream-ordered: no device-wide synchronisation, so a context can be created
  // while another thread records a CUDA graph
  if ((e = cudaMemsetAsync(ctx->scratch_counter, 0, 4 * sizeof(unsigned int), ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
    pfk_destroy_context(ctx);
    return cuda_fail(nullptr, e, "cudaMemsetAsync (context scratch)");
  }
  *out = ctx;
  return PFK_OK;
}

pfk_status pfk_destroy_context(pfk_context* ctx) {
  if (!ctx) return PFK_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFreeAsync(ctx->ws, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->scratch_partials) cudaFree(ctx->scratch_partials);
  if (ctx->scratch_counter) cudaFree(ctx->scratch_counter);
  if (ctx->scratch_out) cudaFree(ctx->scratch_out);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
  return PFK_OK;
}

pfk_status pfk_create_operator(pfk_context* ctx, const pfk_operator_desc* desc, pfk_operator** out) {
  CHECK_ARG(ctx, ctx && desc && out, "NULL argument");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  pfk_operator* op = new (std::nothrow) pfk_operator();
  if (!op) return PFK_ERR_OOM;
  op->ctx = ctx;
  op->device = ctx->device;
  op->stream = ctx->stream;
  op->kind = desc->kind;
  op->storage = desc->storage;
  pfk_status s;
  if (desc->kind == PFK_STENCIL5_2D || desc->kind == PFK_STENCIL7_3D) {
    bool ok = desc->nx > 0 && desc->ny > 0 && desc->eta != nullptr &&
              (desc->kind == PFK_STENCIL5_2D ? desc->nz == 1 || desc->nz == 0 : desc->nz > 0) &&
              (desc->storage == PFK_STORAGE_MATRIX_FREE || desc->storage == PFK_STORAGE_CSR);
    for (int d = 0; d < 3; ++d) ok = ok && std::isfinite(desc->vel[d]);
    if (!ok) {
      delete op;
      set_error(ctx, "invalid stencil description");
      return PFK_ERR_INVALID;
    }
    s = create_stencil(ctx, desc, op);
  } else if (desc->kind == PFK_CSR) {
    if (!(desc->n > 0 && desc->n < INT32_MAX && desc->nnz >= 0 && desc->rowptr &&
          (desc->nnz == 0 || (desc->colidx && desc->vals)))) {
      delete op;
      set_error(ctx, "invalid CSR description");
      return PFK_ERR_INVALID;
    }
    s = create_csr(ctx, desc, op);
  } else {
    delete op;
    set_error(ctx, "unknown operator kind");
    return PFK_ERR_INVALID;
  }
  if (s != PFK_OK) {
    pfk_destroy_operator(op);
    return s;
  }
  *out = op;
  return PFK_OK;
}

pfk_status pfk_destroy_operator(pfk_operator* op) {
  if (!op) return PFK_OK;
  // the operator may outlive its context (e.g. finalisation order in a
  // garbage-collected binding): use the device recorded at creation only
  // (and the stream it was created on, which must outlive it); the frees are
  // stream-ordered, so destroying an operator does not synchronise the device
  cudaSetDevice(op->device);
  cudaStreamSynchronize(op->stream);
  void* ptrs[] = {op->d, op->kx, op->ky, op->kz, op->dinv, op->d32, op->kx32, op->ky32, op->kz32, op->dinv32,
                  op->d16, op->kx16, op->ky16, op->kz16, op->dinv16, op->rowptr, op->colidx, op->vals,
                  op->csr_dinv};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, op->stream);
  cudaStreamSynchronize(op->stream);
  delete op;
  return PFK_OK;
}

pfk_status pfk_operator_size(const pfk_operator* op, int64_t* n) {
  CHECK_ARG(nullptr, op && n, "NULL argument");
  *n = op->n;
  return PFK_OK;
}

pfk_status pfk_operator_apply(pfk_context* ctx, const pfk_operator* op, const double* x, double* y) {
  CHECK_ARG(ctx, ctx && op && x && y, "NULL argument");
  CHECK_ARG(ctx, x != y, "x and y must not overlap");
  cudaSetDevice(ctx->device);
  PFK_CUDA(ctx, op_apply(op, x, y, nullptr, nullptr, ctx->stream));
  PFK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PFK_OK;
}

pfk_status pfk_create_preconditioner(pfk_context* ctx, const pfk_operator* op, const pfk_pc_desc* desc,
                                     pfk_pc** out) {
  CHECK_ARG(ctx, ctx && op && desc && out, "NULL argument");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  pfk_pc* pc = new (std::nothrow) pfk_pc();
  if (!pc) return PFK_ERR_OOM;
  pc->device = ctx->device;
  pc->stream = ctx->stream;
  pfk_status s = create_pc(ctx, op, desc, pc);
  if (s != PFK_OK) {
    pfk_destroy_preconditioner(pc);
    return s;
  }
  *out = pc;
  return PFK_OK;
}

pfk_status pfk_create_noisy_preconditioner(pfk_context* ctx, const pfk_operator* op, double eta, const double* bank,
                                           int count, int bank_on_device, pfk_pc** out) {
  CHECK_ARG(ctx, ctx && op && bank && out, "NULL argument");
  CHECK_ARG(ctx, eta >= 0.0 && count >= 1, "noisy preconditioner needs eta >= 0 and count >= 1");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  pfk_pc* pc = new (std::nothrow) pfk_pc();
  if (!pc) return PFK_ERR_OOM;
  pc->device = ctx->device;
  pc->stream = ctx->stream;
  pfk_status s = create_noisy_pc(ctx, op, eta, bank, count, bank_on_device, pc);
  if (s != PFK_OK) {
    pfk_destroy_preconditioner(pc);
    return s;
  }
  *out = pc;
  return PFK_OK;
}

pfk_status pfk_create_block_preconditioner(pfk_context* ctx, const pfk_operator* K, const pfk_operator* Bt,
                                           const double* schur_diag, const pfk_inner_solve* inner, pfk_pc** out) {
  CHECK_ARG(ctx, ctx && K && Bt && schur_diag && inner && out, "NULL argument");
  CHECK_ARG(ctx, Bt->n > K->n, "Bt must be N x N with N larger than K's size");
  CHECK_ARG(ctx, inner->mmax >= 1 && inner->mmax <= PFK_MAX_MMAX, "inner mmax out of range");
  CHECK_ARG(ctx, inner->maxit >= 1 && inner->rtol >= 0.0, "inner maxit must be >= 1 and rtol >= 0");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  pfk_pc* pc = new (std::nothrow) pfk_pc();
  if (!pc) return PFK_ERR_OOM;
  pc->device = ctx->device;
  pc->stream = ctx->stream;
  pfk_status s = create_nested_pc(ctx, K, Bt, schur_diag, inner, pc);
  if (s != PFK_OK) {
    pfk_destroy_preconditioner(pc);
    return s;
  }
  *out = pc;
  return PFK_OK;
}

pfk_status pfk_destroy_preconditioner(pfk_pc* pc) {
  if (!pc) return PFK_OK;
  if (pc->nested) destroy_nested(pc);
  // as for operators: never dereference the (possibly destroyed) context
  cudaSetDevice(pc->device);
  cudaStreamSynchronize(pc->stream);
  if (pc->buf) cudaFreeAsync(pc->buf, pc->stream);
  if (pc->ctl) cudaFreeAsync(pc->ctl, pc->stream);
  if (pc->partials) cudaFreeAsync(pc->partials, pc->stream);
  if (pc->bank) cudaFreeAsync(pc->bank, pc->stream);
  if (pc->bank_inv_norm) cudaFreeAsync(pc->bank_inv_norm, pc->stream);
  cudaStreamSynchronize(pc->stream);
  delete pc;
  return PFK_OK;
}

pfk_status pfk_pc_apply(pfk_context* ctx, const pfk_pc* pc, const double* v, double* y) {
  CHECK_ARG(ctx, ctx && pc && v && y, "NULL argument");
  CHECK_ARG(ctx, v != y, "v and y must not overlap");
  cudaSetDevice(ctx->device);
  PFK_CUDA(ctx, pc_apply(pc, v, y, nullptr, nullptr, ctx->stream));
  PFK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PFK_OK;
}

pfk_status pfk_pc_workspace_bytes(const pfk_pc* pc, int64_t* bytes) {
  CHECK_ARG(nullptr, pc && bytes, "NULL argument");
  *bytes = (int64_t)pc->buf_bytes;
  return PFK_OK;
}

pfk_status pfk_default_params(pfk_solve_params* p) {
  CHECK_ARG(nullptr, p != nullptr, "NULL argument");
  std::memset(p, 0, sizeof(*p));
  p->method = PFK_PIPEFCG;
  p->mmax = 30;
  p->truncation = PFK_TRUNC_STANDARD;
  p->norm = PFK_NORM_NATURAL;
  p->rtol = 1e-8;
  p->atol = 0.0;
  p->maxit = 10000;
  p->max_restarts = 20;
  p->sigma = NAN;
  p->true_residual_check = 1;
  p->graph_iters = 8;
  return PFK_OK;
}

int pfk_method_storage_vectors(int method, int mmax) {
  switch (method) {
    case PFK_PIPEFCG:
    case PFK_PIPEFCG_NAIVE:
    case PFK_PIPEGCR_W:
    case PFK_PIPEFCG_THETA: return 4 * mmax + 11;
    case PFK_FCG: return mmax + 6;
    case PFK_GCR: return 2 * mmax + 7;
    case PFK_PIPEGCR: return 2 * mmax + 7 + mmax + 2;
    case PFK_FGMRES: return 2 * mmax + 2;
    case PFK_PIPEFGMRES: return 4 * mmax + 2;
    default: return -1;
  }
}

pfk_status pfk_solve_workspace_bytes(int method, int mmax, int64_t n, int64_t* bytes) {
  CHECK_ARG(nullptr, bytes && n > 0 && mmax >= 1 && mmax <= PFK_MAX_MMAX, "invalid argument");
  return solve_workspace_bytes(method, mmax, n, bytes);
}

pfk_status pfk_solve(pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, const pfk_solve_params* params,
                     const double* b, double* x, int ptr_on_device, pfk_solve_info* info) {
  CHECK_ARG(ctx, ctx && op && params && b && x, "NULL argument");
  CHECK_ARG(ctx, params->mmax >= 1 && params->mmax <= PFK_MAX_MMAX, "mmax out of range [1, PFK_MAX_MMAX]");
  CHECK_ARG(ctx, params->maxit >= 0, "maxit < 0");
  CHECK_ARG(ctx, params->rtol >= 0.0 && params->atol >= 0.0, "negative tolerance");
  CHECK_ARG(ctx, params->truncation == PFK_TRUNC_STANDARD || params->truncation == PFK_TRUNC_RESTART,
            "unknown truncation");
  CHECK_ARG(ctx, params->norm == PFK_NORM_NATURAL || params->norm == PFK_NORM_UNPRECONDITIONED, "unknown norm");
  CHECK_ARG(ctx, !params->history || params->history_capacity >= 0, "negative history capacity");
  // a nested block preconditioner is built from the blocks (K, B^T), not from
  // the outer operator: it must match the outer operator's size
  CHECK_ARG(ctx, !pc || pc->op == op || (pc->kind == PFK_PC_BLOCK_UPPER && pc->op->n == op->n),
            "preconditioner was built for another operator");
  if (!method_supported(params->method)) {
    set_error(ctx, "method not available");
    return PFK_ERR_INVALID;
  }
  cudaSetDevice(ctx->device);
  const int64_t n = op->n;
  if (info) std::memset(info, 0, sizeof(*info));
  const double* bd = b;
  double* xd = x;
  double* stage = nullptr;
  if (!ptr_on_device) {
    cudaError_t e = cudaMallocAsync((void**)&stage, 2 * n * sizeof(double), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocAsync (staging)");
    PFK_CUDA(ctx, cudaMemcpyAsync(stage, b, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    PFK_CUDA(ctx, cudaMemcpyAsync(stage + n, x, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    bd = stage;
    xd = stage + n;
  }
  pfk_status s = run_solve(ctx, op, pc, params, bd, xd, info);
  if (!ptr_on_device) {
    if (s == PFK_OK || s == PFK_ERR_NOT_CONVERGED || s == PFK_ERR_BREAKDOWN)
      cudaMemcpyAsync(x, xd, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    cudaFreeAsync(stage, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess && s == PFK_OK) return cuda_fail(ctx, e, "copy back");
  }
  return s;
}

pfk_status pfk_probe_fp64_fma(pfk_context* ctx, int iters, double* tflops, double* ms) {
  CHECK_ARG(ctx, ctx != nullptr, "NULL context");
  CHECK_ARG(ctx, tflops != nullptr && ms != nullptr, "NULL output pointer");
  CHECK_ARG(ctx, iters >= 1 && iters <= (1 << 24), "iters must be in [1, 2^24]");
  cudaSetDevice(ctx->device);
  PFK_CUDA(ctx, fp64_probe(ctx, iters, tflops, ms));
  return PFK_OK;
}

}  // extern "C"
