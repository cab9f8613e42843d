// Serving loop: continuous batching of independent solves (host runtime).
//
// Requests are copied at submission and queued in arrival order.  Requests
// the grouped kernel can run (stencil, PIPEFCG / PIPEGCR / PIPEFGMRES, NONE /
// JACOBI / inner-PCG preconditioner) with at most group_max_n unknowns go to the group queue:
// one scheduler thread with its own stream and pfk_context keeps them in a
// GroupRunner, each with its own group of CTAs, and advances all of them by a
// few steps per cooperative launch; between launches it publishes the
// finished ones and admits queued ones while their CTAs fit (and the memory
// budget allows).  The other requests go to worker threads, each with its own
// CUDA stream and pfk_context, which admit the next request (the head of the
// queue, or with PFK_SERVE_SMALLEST_FIRST the queued request with the fewest
// unknowns) when the device-memory budget allows (memory of the active solves
// is accounted from each request's estimate), run the whole solve through the
// graph-replayed single-system path, publish the result and release the
// memory.  Kernels of both kinds run concurrently on the GPU.  Nothing in a
// solve depends on the others, so results are bitwise those of the same
// request solved alone (by pfk_solve_grouped with the same CTA count, or by
// pfk_solve).
#include "group.cuh"
#include "pfk_internal.cuh"

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace pfk {
void set_error(pfk_context* ctx, const std::string& msg);
}

using namespace pfk;

namespace {

using Clock = std::chrono::steady_clock;

struct Item {
  uint64_t ticket = 0;
  pfk_operator_desc desc{};
  std::vector<double> eta, vals, b, x;
  std::vector<int32_t> rowptr, colidx;
  pfk_pc_desc pc{};
  pfk_solve_params prm{};
  int64_t n = 0;
  int64_t bytes = 0;
  Clock::time_point t_submit;
  double latency_ms = 0.0;
  pfk_solve_info info{};
  pfk_status status = PFK_PENDING;
  std::string err;
  bool done = false;
  bool grouped = false;   // served by the grouped kernel
  int nblk = 0;           // its CTAs
};

}  // namespace

struct pfk_server {
  int device = 0;
  int64_t budget = 0;
  int64_t in_use = 0;
  int active = 0;
  int capacity = 0;
  int order = PFK_SERVE_FIFO;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<std::shared_ptr<Item>> queue;    // whole-GPU requests
  std::deque<std::shared_ptr<Item>> gqueue;   // grouped requests
  int64_t group_max_n = 0;
  int group_ctas = 0;
  std::thread group_thread;
  cudaStream_t gstream = nullptr;
  pfk_context* gctx = nullptr;
  std::unordered_map<uint64_t, std::shared_ptr<Item>> items;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::thread> workers;
  // per worker: stream and context, created before any worker starts and
  // destroyed after all have stopped, so that no context set-up or teardown
  // runs while a worker records a CUDA graph
  std::vector<cudaStream_t> streams;
  std::vector<pfk_context*> ctxs;
};

namespace {

// Device bytes a request holds while active: operator coefficients (and the
// preconditioner's reduced copies), preconditioner scratch, the solve
// workspace, reduction partials and host-staging buffers.
int64_t estimate_bytes(const Item& it, int num_sms) {
  const int64_t n = it.n;
  int64_t op = 0;
  if (it.desc.kind == PFK_CSR) op = it.desc.nnz * 12 + (n + 1) * 4 + n * 8;
  else op = 5 * n * 8;
  int64_t pc = 0;
  if (it.pc.kind == PFK_PC_INNER_PCG || it.pc.kind == PFK_PC_CHEBYSHEV) {
    const int64_t es = it.pc.precision == PFK_FP64 ? 8 : 4;
    pc = 5 * n * es + (it.pc.precision == PFK_FP32 ? 5 * n * 4 : it.pc.precision == PFK_BF16_COEF_FP32 ? 5 * n * 2 : 0);
  }
  int64_t ws = 0;
  if (pfk_solve_workspace_bytes(it.prm.method, it.prm.mmax, n, &ws) != PFK_OK) ws = 0;
  const int64_t partials = (int64_t)num_sms * kMaxBlocksPerSm * kPartialStride * 8 + 64 * 1024;
  return op + pc + ws + partials + 2 * n * 8;
}

// Device bytes of a grouped request: operator coefficients, the grouped
// workspace, and its device x and b.
int64_t estimate_group_bytes(const Item& it) {
  return 5 * it.n * 8 + GroupRunner::workspace_bytes(it.n, it.prm.mmax, it.nblk) + 2 * it.n * 8;
}

// The request admitted next from queue q (not empty; srv->mu held).
std::deque<std::shared_ptr<Item>>::iterator next_request(pfk_server* srv, std::deque<std::shared_ptr<Item>>& q) {
  auto best = q.begin();
  if (srv->order == PFK_SERVE_SMALLEST_FIRST)
    for (auto p = q.begin(); p != q.end(); ++p)
      if ((*p)->n < (*best)->n) best = p;
  return best;
}

std::deque<std::shared_ptr<Item>>::iterator next_request(pfk_server* srv) { return next_request(srv, srv->queue); }

// Publishes a finished request (srv->mu not held).
void publish(pfk_server* srv, const std::shared_ptr<Item>& it, pfk_status st, const pfk_solve_info& info,
             const std::string& err) {
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    it->status = st;
    it->err = err;
    it->info = info;
    it->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - it->t_submit).count();
    it->done = true;
    it->eta.clear();
    it->eta.shrink_to_fit();
    it->b.clear();
    it->b.shrink_to_fit();
    srv->in_use -= it->bytes;
    srv->active -= 1;
  }
  srv->cv_done.notify_all();
  srv->cv_work.notify_all();
}

// The grouped requests' scheduler: admits queued requests while their CTAs
// and memory fit, advances every active one by kGroupSteps steps per
// cooperative launch, publishes the finished ones.
void group_main(pfk_server* srv) {
  constexpr int kGroupSteps = 8;
  cudaSetDevice(srv->device);
  pfk_context* ctx = srv->gctx;
  GroupRunner R;
  const bool ok = ctx && R.init(ctx, 0) == PFK_OK;
  const std::string init_err = ok ? std::string() : (ctx ? pfk_last_error(ctx) : "no context for grouped requests");
  struct Active {
    std::shared_ptr<Item> it;
    pfk_operator* op = nullptr;
    double* xb = nullptr;     // device x then b
    int slot = -1;
    Clock::time_point t0;
  };
  std::vector<Active> act;
  for (;;) {
    std::vector<std::shared_ptr<Item>> take;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      int free_ctas = ok ? R.free_ctas() : 1 << 30;
      // the next queued request fits: its CTAs are free and its memory fits
      // the budget (or nothing at all is active)
      auto fits = [&]() {
        if (srv->gqueue.empty()) return false;
        const auto& cand = *next_request(srv, srv->gqueue);
        if (ok && cand->nblk > free_ctas) return false;
        return (srv->active == 0 && take.empty()) || srv->in_use + cand->bytes <= srv->budget;
      };
      srv->cv_work.wait(lk, [&] { return srv->stop || !act.empty() || fits(); });
      if (srv->stop) break;
      while (fits()) {
        const auto pos = next_request(srv, srv->gqueue);
        const auto cand = *pos;
        take.push_back(cand);
        free_ctas -= cand->nblk;
        srv->in_use += cand->bytes;
        srv->active += 1;
        srv->gqueue.erase(pos);
      }
    }
    for (auto& it : take) {
      if (!ok) {
        pfk_solve_info info{};
        info.status = PFK_ERR_CUDA;
        publish(srv, it, PFK_ERR_CUDA, info, init_err);
        continue;
      }
      Active a;
      a.it = it;
      a.t0 = Clock::now();
      pfk_status st = pfk_create_operator(ctx, &it->desc, &a.op);
      if (st == PFK_OK) {
        cudaError_t e = cudaMallocAsync((void**)&a.xb, 2 * it->n * sizeof(double), ctx->stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(a.xb, it->x.data(), it->n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(a.xb + it->n, it->b.data(), it->n * sizeof(double), cudaMemcpyHostToDevice,
                              ctx->stream);
        st = e == cudaSuccess ? PFK_OK : cuda_fail(ctx, e, "grouped request buffers");
      }
      if (st == PFK_OK)
        st = R.admit(a.op, &it->pc, &it->prm, a.xb + it->n, a.xb, it->nblk, nullptr, 0, &a.slot);
      if (st != PFK_OK) {
        const std::string err = pfk_last_error(ctx);
        if (a.xb) cudaFreeAsync(a.xb, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        pfk_destroy_operator(a.op);
        pfk_solve_info info{};
        info.status = st;
        publish(srv, it, st, info, err);
        continue;
      }
      act.push_back(a);
    }
    if (act.empty()) continue;
    const pfk_status sst = R.step(kGroupSteps);
    for (size_t k = 0; k < act.size();) {
      Active& a = act[k];
      const bool fin = sst != PFK_OK || R.done(a.slot);
      if (!fin) {
        ++k;
        continue;
      }
      pfk_solve_info info{};
      pfk_status st = sst;
      std::string err;
      if (sst == PFK_OK) {
        R.info(a.slot, &info);
        st = (pfk_status)info.status;
        info.time_ms = std::chrono::duration<double, std::milli>(Clock::now() - a.t0).count();
        if (cudaMemcpyAsync(a.it->x.data(), a.xb, a.it->n * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream) != cudaSuccess)
          st = PFK_ERR_CUDA;
      } else {
        info.status = sst;
        err = pfk_last_error(ctx);
      }
      R.release(a.slot);
      cudaFreeAsync(a.xb, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      pfk_destroy_operator(a.op);
      if (st == PFK_ERR_TIMEOUT) err = "a group-barrier wait of the grouped kernel timed out";
      else if (st != PFK_OK && err.empty()) err = "the grouped solve did not converge";
      if (info.status == PFK_OK) info.status = st;
      publish(srv, a.it, st, info, err);
      act[k] = act.back();
      act.pop_back();
    }
  }
  // stopping: active grouped requests are finished first
  while (!act.empty() && ok) {
    if (R.step(kGroupSteps) != PFK_OK) break;
    for (size_t k = 0; k < act.size();) {
      if (!R.done(act[k].slot)) {
        ++k;
        continue;
      }
      pfk_solve_info info{};
      R.info(act[k].slot, &info);
      cudaMemcpyAsync(act[k].it->x.data(), act[k].xb, act[k].it->n * sizeof(double), cudaMemcpyDeviceToHost,
                      ctx->stream);
      R.release(act[k].slot);
      cudaFreeAsync(act[k].xb, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      pfk_destroy_operator(act[k].op);
      const pfk_status st = (pfk_status)info.status;
      publish(srv, act[k].it, st, info, st == PFK_OK ? "" : "the grouped solve did not converge");
      act[k] = act.back();
      act.pop_back();
    }
  }
  // a launch failed while stopping: the rest end with its error
  const std::string err = ctx ? pfk_last_error(ctx) : "no context for grouped requests";
  for (auto& a : act) {
    R.release(a.slot);
    if (a.xb) cudaFreeAsync(a.xb, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    pfk_destroy_operator(a.op);
    pfk_solve_info info{};
    info.status = PFK_ERR_CUDA;
    publish(srv, a.it, PFK_ERR_CUDA, info, err);
  }
}

void worker_main(pfk_server* srv, int index) {
  cudaSetDevice(srv->device);
  pfk_context* ctx = srv->ctxs[index];
  for (;;) {
    std::shared_ptr<Item> it;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv_work.wait(lk, [&] {
        if (srv->stop) return true;
        if (srv->queue.empty()) return false;
        const auto& next = *next_request(srv);
        return srv->active == 0 || srv->in_use + next->bytes <= srv->budget;
      });
      if (srv->stop) break;
      const auto pos = next_request(srv);
      it = *pos;
      srv->queue.erase(pos);
      srv->in_use += it->bytes;
      srv->active += 1;
    }
    pfk_status st = PFK_ERR_CUDA;
    pfk_solve_info info{};
    std::string err;
    if (ctx) {
      pfk_operator* op = nullptr;
      pfk_pc* pc = nullptr;
      st = pfk_create_operator(ctx, &it->desc, &op);
      if (st == PFK_OK && it->pc.kind != PFK_PC_NONE) st = pfk_create_preconditioner(ctx, op, &it->pc, &pc);
      if (st == PFK_OK) st = pfk_solve(ctx, op, pc, &it->prm, it->b.data(), it->x.data(), 0, &info);
      pfk_destroy_preconditioner(pc);
      pfk_destroy_operator(op);
      // the workspace belongs to this request's budget: give it back
      if (ctx->ws) {
        cudaFreeAsync(ctx->ws, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
      }
    }
    if (st != PFK_OK && info.status == PFK_OK) info.status = st;
    if (st != PFK_OK) err = ctx ? pfk_last_error(ctx) : "worker has no context";
    publish(srv, it, st, info, err);
  }
}

void release_workers(pfk_server* srv) {
  for (pfk_context* c : srv->ctxs)
    if (c) pfk_destroy_context(c);
  for (cudaStream_t s : srv->streams)
    if (s) cudaStreamDestroy(s);
  srv->ctxs.clear();
  srv->streams.clear();
  if (srv->gctx) pfk_destroy_context(srv->gctx);
  if (srv->gstream) cudaStreamDestroy(srv->gstream);
  srv->gctx = nullptr;
  srv->gstream = nullptr;
}

}  // namespace

extern "C" {

pfk_status pfk_server_create(pfk_context* ctx, const pfk_server_params* params, pfk_server** out) {
  if (!ctx || !out) {
    set_error(ctx, "NULL argument");
    return PFK_ERR_INVALID;
  }
  *out = nullptr;
  pfk_server* srv = new (std::nothrow) pfk_server();
  if (!srv) return PFK_ERR_OOM;
  srv->device = ctx->device;
  const int workers = params && params->workers > 0 ? params->workers : 4;
  srv->capacity = params && params->queue_capacity > 0 ? params->queue_capacity : 4096;
  if (params && params->order != PFK_SERVE_FIFO && params->order != PFK_SERVE_SMALLEST_FIRST) {
    delete srv;
    set_error(ctx, "unknown admission order");
    return PFK_ERR_INVALID;
  }
  srv->order = params ? params->order : PFK_SERVE_FIFO;
  const int32_t gmax = params ? params->group_max_n : 0;
  srv->group_max_n = gmax == 0 ? 110592 : (gmax < 0 ? 0 : gmax);
  srv->group_ctas = params ? params->group_ctas : 0;
  if (srv->group_ctas < 0 || srv->group_ctas > 64) {
    delete srv;
    set_error(ctx, "group_ctas must be 0 (automatic) or 1..64");
    return PFK_ERR_INVALID;
  }
  int64_t budget = params ? params->memory_budget : 0;
  if (budget <= 0) {
    size_t fr = 0, tot = 0;
    cudaSetDevice(ctx->device);
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete srv;
      set_error(ctx, "cudaMemGetInfo failed");
      return PFK_ERR_CUDA;
    }
    budget = (int64_t)(0.8 * (double)fr);
  }
  srv->budget = budget;
  cudaSetDevice(ctx->device);
  for (int w = 0; w < workers; ++w) {
    cudaStream_t s = nullptr;
    pfk_context* c = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    pfk_status ps = e == cudaSuccess ? pfk_create_context(ctx->device, s, &c) : PFK_ERR_CUDA;
    srv->streams.push_back(s);
    srv->ctxs.push_back(c);
    if (ps != PFK_OK) {
      release_workers(srv);
      delete srv;
      set_error(ctx, "could not create the worker streams and contexts");
      return ps;
    }
  }
  if (srv->group_max_n > 0) {
    cudaError_t e = cudaStreamCreateWithFlags(&srv->gstream, cudaStreamNonBlocking);
    pfk_status ps = e == cudaSuccess ? pfk_create_context(ctx->device, srv->gstream, &srv->gctx) : PFK_ERR_CUDA;
    if (ps != PFK_OK) {
      release_workers(srv);
      delete srv;
      set_error(ctx, "could not create the grouped requests' stream and context");
      return ps;
    }
  }
  for (int w = 0; w < workers; ++w) srv->workers.emplace_back(worker_main, srv, w);
  if (srv->group_max_n > 0) srv->group_thread = std::thread(group_main, srv);
  *out = srv;
  return PFK_OK;
}

pfk_status pfk_submit(pfk_server* srv, const pfk_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket || !req->b) {
    set_error(nullptr, "NULL argument");
    return PFK_ERR_INVALID;
  }
  auto it = std::make_shared<Item>();
  it->desc = req->op;
  it->pc = req->pc;
  it->prm = req->params;
  it->prm.history = nullptr;
  it->prm.history_capacity = 0;
  it->prm.profile = 0;
  int64_t n = 0;
  if (req->op.kind == PFK_STENCIL5_2D || req->op.kind == PFK_STENCIL7_3D) {
    if (!req->op.eta || req->op.eta_on_device || req->op.nx <= 0 || req->op.ny <= 0) {
      set_error(nullptr, "requests need host stencil coefficients");
      return PFK_ERR_INVALID;
    }
    n = (int64_t)req->op.nx * req->op.ny * (req->op.kind == PFK_STENCIL5_2D ? 1 : req->op.nz);
    if (n <= 0) {
      set_error(nullptr, "invalid stencil size");
      return PFK_ERR_INVALID;
    }
    it->eta.assign(req->op.eta, req->op.eta + n);
    it->desc.eta = it->eta.data();
  } else if (req->op.kind == PFK_CSR) {
    if (req->op.csr_on_device || !req->op.rowptr || req->op.n <= 0 || req->op.nnz < 0 ||
        (req->op.nnz > 0 && (!req->op.colidx || !req->op.vals))) {
      set_error(nullptr, "requests need host CSR arrays (row pointers, columns, values)");
      return PFK_ERR_INVALID;
    }
    if (req->op.rowptr[0] != 0 || req->op.rowptr[req->op.n] != req->op.nnz) {
      set_error(nullptr, "CSR row pointers must run from 0 to nnz");
      return PFK_ERR_INVALID;
    }
    n = req->op.n;
    it->rowptr.assign(req->op.rowptr, req->op.rowptr + n + 1);
    it->colidx.assign(req->op.colidx, req->op.colidx + req->op.nnz);
    it->vals.assign(req->op.vals, req->op.vals + req->op.nnz);
    it->desc.rowptr = it->rowptr.data();
    it->desc.colidx = it->colidx.data();
    it->desc.vals = it->vals.data();
  } else {
    set_error(nullptr, "unknown operator kind");
    return PFK_ERR_INVALID;
  }
  if (it->prm.mmax < 1 || it->prm.mmax > PFK_MAX_MMAX) {
    set_error(nullptr, "mmax out of range");
    return PFK_ERR_INVALID;
  }
  it->n = n;
  it->b.assign(req->b, req->b + n);
  if (req->x0) it->x.assign(req->x0, req->x0 + n);
  else it->x.assign(n, 0.0);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, srv->device);
  if (srv->group_max_n > 0 && n <= srv->group_max_n && it->desc.kind != PFK_CSR && it->desc.storage == 0) {
    it->grouped = group_method_eligible(&it->pc, &it->prm, nullptr);
    if (it->grouped) {
      const int64_t rows = (int64_t)it->desc.ny * (it->desc.kind == PFK_STENCIL5_2D ? 1 : it->desc.nz);
      it->nblk = group_ctas(n, rows, srv->group_ctas);
    }
  }
  it->bytes = it->grouped ? estimate_group_bytes(*it) : estimate_bytes(*it, sms);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if ((int)srv->items.size() >= srv->capacity) {
      set_error(nullptr, "server queue is full");
      return PFK_ERR_BUSY;
    }
    it->ticket = srv->next_ticket++;
    it->t_submit = Clock::now();
    srv->items[it->ticket] = it;
    (it->grouped ? srv->gqueue : srv->queue).push_back(it);
    *ticket = it->ticket;
  }
  srv->cv_work.notify_all();
  return PFK_OK;
}

pfk_status pfk_poll(pfk_server* srv, uint64_t ticket, double* x_out, pfk_solve_info* info, double* latency_ms,
                    int wait_ms) {
  if (!srv) {
    set_error(nullptr, "NULL argument");
    return PFK_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto f = srv->items.find(ticket);
  if (f == srv->items.end()) {
    set_error(nullptr, "unknown or already collected ticket");
    return PFK_ERR_INVALID;
  }
  std::shared_ptr<Item> it = f->second;
  if (!it->done) {
    if (wait_ms == 0) return PFK_PENDING;
    if (wait_ms < 0) srv->cv_done.wait(lk, [&] { return it->done; });
    else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return it->done; }))
      return PFK_PENDING;
  }
  if (x_out) std::memcpy(x_out, it->x.data(), sizeof(double) * it->n);
  if (info) *info = it->info;
  if (latency_ms) *latency_ms = it->latency_ms;
  if (it->status != PFK_OK) set_error(nullptr, it->err);
  srv->items.erase(ticket);
  return it->status;
}

pfk_status pfk_server_destroy(pfk_server* srv) {
  if (!srv) return PFK_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->queue.clear();
    srv->gqueue.clear();
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  if (srv->group_thread.joinable()) srv->group_thread.join();
  release_workers(srv);
  delete srv;
  return PFK_OK;
}

}  // extern "C"
