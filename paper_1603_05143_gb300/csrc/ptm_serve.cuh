// Serving runtime of libptm.so: continuous batching of MD frames that arrive at
// any time (part of ptm.cu's translation unit).
//
// One scheduler thread per server owns every CUDA call of the server.  Frames
// wait in a FIFO; a frame is admitted when its device bytes fit the HBM budget
// beside the frames already on the device.  Whenever a stream slot is free, all
// admitted frames not yet launched (up to max_batch_frames, and up to
// max_batch_atoms atoms unless a single frame is larger) become one batch:
// inputs are copied in, one persistent launch classifies them, outputs are
// copied back, and an event marks completion.  Frames that arrive while batches
// run join the next batch as soon as memory and a slot free up, and the slots'
// streams overlap on the device.  Device memory comes from a reuse pool, so no
// cudaFree (which synchronises the device) happens while serving.
#pragma once
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Size-class pool of device blocks (powers of two from 4 KiB); blocks return to
// the pool and are reused, and are released only when the pool is destroyed.
struct DevicePool {
  std::multimap<size_t, void *> free_blocks;
  std::vector<void *> all;
  static size_t cls(size_t bytes) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    return c;
  }
  cudaError_t alloc(size_t bytes, void **p) {
    const size_t c = cls(bytes);
    auto it = free_blocks.find(c);
    if (it != free_blocks.end()) { *p = it->second; free_blocks.erase(it); return cudaSuccess; }
    cudaError_t e = cudaMalloc(p, c);
    if (e == cudaSuccess) all.push_back(*p);
    return e;
  }
  void release(size_t bytes, void *p) { if (p) free_blocks.emplace(cls(bytes), p); }
  ~DevicePool() { for (void *p : all) cudaFree(p); }
};

struct Request {
  uint64_t ticket = 0;
  ptm_frame frame{};         // host pointers
  ptm_outputs out{};         // host pointers
  size_t bytes = 0;          // device bytes while in flight (inputs, outputs, workspace share)
  double t_submit = 0, t_start = 0, t_done = 0;
  int64_t batch = -1;
  int state = 0;             // 0 queued, 1 launched, 2 done
  ptm_status status = PTM_OK;
  // device copies
  void *dpos = nullptr; int8_t *dsp = nullptr; void *dout = nullptr;
  size_t pos_bytes = 0, out_bytes = 0;
};

struct InFlight {
  std::vector<Request *> reqs;
  ptm_batch *batch = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t done = nullptr;
  int slot = 0;
  bool fail = false;               // fault injection: report this batch as failed
};

constexpr size_t kOutBytesPerAtom = 1 + 1 + 4 + 4 + 16 + 36 + 60 + 4 + 12;

size_t request_bytes(const ptm_frame &f) {
  const size_t n = (size_t)f.n_atoms;
  const size_t pos = n * 3 * (f.pos_dtype == PTM_F64 ? 8 : 4);
  const size_t ws = n * (f.pos_dtype == PTM_F64 ? 32 : 16) + 20 * n + 8 * (4 * n + 64) + sizeof(FrameDesc) +
                    sizeof(ShiftTables) + 4096 +
                    n * 8 * PTM_KNN + 28 * n + 768 +
                    (f.ordering == PTM_ORDER_TOPOLOGICAL ? n * 4 + topo_side_bytes(n) + 1024 : 0);
  return pos + n + n * kOutBytesPerAtom + ws;
}

}  // namespace

struct ptm_server {
  ptm_context *ctx = nullptr;
  size_t budget = 0, in_use = 0;
  int max_batch = 64, nslots = 4;   // batches in flight (4 streams: 220 M atoms/s capacity against 203 M with 2)
  int64_t max_batch_atoms = 4 << 20;
  ptm_tuning tuning{};
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  std::vector<void *> staging;       // pinned host staging per slot (descriptors)
  size_t staging_bytes = 0;
  std::deque<Request *> queue;
  std::vector<InFlight *> inflight;
  std::unordered_map<uint64_t, Request *> reqs;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  int64_t next_batch = 0;
  DevicePool pool;
  std::string error;
  // host-side fault injection (ptm_server_inject)
  bool hold_next = false;          // the next launched batch's completion goes unseen ...
  InFlight *held = nullptr;        // ... while it is held here
  int fail_next = 0;               // batches still to report as failed
};

namespace {

// Launch one batch of admitted requests on slot `slot` (scheduler thread only).
ptm_status launch_batch(ptm_server *S, std::vector<Request *> &rs, int slot, InFlight **out) {
  ptm_context *ctx = S->ctx;
  cudaStream_t st = S->streams[slot];
  const int nf = (int)rs.size();
  std::vector<ptm_frame> frames(nf);
  std::vector<ptm_outputs> outs(nf);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < nf; i++) {
    Request *r = rs[i];
    const size_t n = (size_t)r->frame.n_atoms;
    r->pos_bytes = n * 3 * (r->frame.pos_dtype == PTM_F64 ? 8 : 4);
    r->out_bytes = n * kOutBytesPerAtom + 64;      // + alignment of the float outputs
    if (e == cudaSuccess) e = S->pool.alloc(r->pos_bytes, &r->dpos);
    if (e == cudaSuccess && r->frame.species) e = S->pool.alloc(n, (void **)&r->dsp);
    if (e == cudaSuccess) e = S->pool.alloc(r->out_bytes, &r->dout);
    if (e != cudaSuccess) break;
    e = cudaMemcpyAsync(r->dpos, r->frame.positions, r->pos_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && r->frame.species) e = cudaMemcpyAsync(r->dsp, r->frame.species, n, cudaMemcpyHostToDevice, st);
    frames[i] = r->frame;
    frames[i].positions = r->dpos;
    frames[i].species = r->frame.species ? r->dsp : nullptr;
    unsigned char *o = (unsigned char *)r->dout;
    ptm_outputs &d = outs[i];
    d.structure = r->out.structure ? (int8_t *)o : nullptr; o += n;
    d.alloy = r->out.alloy ? (int8_t *)o : nullptr; o += n;
    o = (unsigned char *)(((uintptr_t)o + 15) & ~(uintptr_t)15);
    d.rmsd = r->out.rmsd ? (float *)o : nullptr; o += 4 * n;
    d.scale = r->out.scale ? (float *)o : nullptr; o += 4 * n;
    d.quat = r->out.quat ? (float *)o : nullptr; o += 16 * n;
    d.strain = r->out.strain ? (float *)o : nullptr; o += 36 * n;
    d.correspondence = r->out.correspondence ? (int32_t *)o : nullptr; o += 60 * n;
    d.von_mises = r->out.von_mises ? (float *)o : nullptr; o += 4 * n;
    d.rodrigues = r->out.rodrigues ? (float *)o : nullptr;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "serve: inputs");
  InFlight *F = new InFlight();
  F->reqs = rs;
  F->slot = slot;
  ptm_batch *b = new ptm_batch();
  b->ctx = ctx;
  b->nframes = nf;
  b->owns_block = false;
  if (S->tuning.cell_factor > 0) b->cell_factor = S->tuning.cell_factor;
  if (S->tuning.tile_atoms > 0) b->tile_atoms = (S->tuning.tile_atoms + 31) / 32 * 32;
  if (S->tuning.blocks_per_sm > 0) b->blocks_per_sm = S->tuning.blocks_per_sm;
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  BatchPlan P;
  ptm_status rsn = batch_plan(nf, frames.data(), b->cell_factor, P);
  if (rsn != PTM_OK) { delete b; delete F; return rsn; }
  b->f64 = P.f64; b->ntotal = P.ntotal; b->ncell = P.ncell;
  F->ws_bytes = batch_workspace_bytes(nf, P.ntotal, P.ncell, P.f64, P.topo);
  e = S->pool.alloc(F->ws_bytes, &F->ws);
  for (int i = 0; i < 5 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&b->ev[i], cudaEventDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->done, cudaEventDisableTiming);
  if (e != cudaSuccess) { batch_free(b); delete F; return cuda_fail(ctx, e, "serve: workspace"); }
  b->block = F->ws;
  batch_layout(b, (unsigned char *)F->ws, P, outs.data());
  if ((e = batch_side_init(b)) != cudaSuccess) { batch_free(b); delete F; return cuda_fail(ctx, e, "serve: streams"); }
  // descriptors through this slot's pinned staging (free: the slot's previous batch is done)
  const size_t need = (sizeof(FrameDesc) + sizeof(ShiftTables) + sizeof(BinParams) + 2 * sizeof(int64_t) +
                       sizeof(int)) * nf;
  unsigned char *hs = (unsigned char *)S->staging[slot];
  if (need > S->staging_bytes) { batch_free(b); delete F; return PTM_ERR_INVALID_ARG; }
  unsigned char *h_tab = hs + sizeof(FrameDesc) * nf, *h_bp = h_tab + sizeof(ShiftTables) * nf;
  unsigned char *h_off = h_bp + sizeof(BinParams) * nf;
  unsigned char *h_soff = h_off + sizeof(int64_t) * nf, *h_sfr = h_soff + sizeof(int64_t) * nf;
  std::memcpy(hs, P.hd.data(), sizeof(FrameDesc) * nf);
  std::memcpy(h_tab, P.tabs.data(), sizeof(ShiftTables) * nf);
  std::memcpy(h_bp, P.hb.data(), sizeof(BinParams) * nf);
  std::memcpy(h_off, P.off.data(), sizeof(int64_t) * nf);
  std::memcpy(h_soff, P.small_off.data(), sizeof(int64_t) * P.small_off.size());
  std::memcpy(h_sfr, P.small_frames.data(), sizeof(int) * P.small_frames.size());
  e = cudaMemcpyAsync(b->d_descs, hs, sizeof(FrameDesc) * nf, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_tabs, h_tab, sizeof(ShiftTables) * nf, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_bp, h_bp, sizeof(BinParams) * nf, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_atom_off, h_off, sizeof(int64_t) * nf, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && b->nsmall)
    e = cudaMemcpyAsync(b->d_small_off, h_soff, sizeof(int64_t) * b->nsmall, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && b->nsmall)
    e = cudaMemcpyAsync(b->d_small_frames, h_sfr, sizeof(int) * b->nsmall, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) { batch_free(b); delete F; return cuda_fail(ctx, e, "serve: descriptors"); }
  rsn = batch_enqueue(b, st);
  if (rsn != PTM_OK) { batch_free(b); delete F; return rsn; }
  for (int i = 0; i < nf && e == cudaSuccess; i++) {
    Request *r = rs[i];
    const size_t n = (size_t)r->frame.n_atoms;
    const ptm_outputs &d = outs[i];
    if (r->out.structure) e = cudaMemcpyAsync(r->out.structure, d.structure, n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->out.alloy) e = cudaMemcpyAsync(r->out.alloy, d.alloy, n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->out.rmsd) e = cudaMemcpyAsync(r->out.rmsd, d.rmsd, 4 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->out.scale) e = cudaMemcpyAsync(r->out.scale, d.scale, 4 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->out.quat) e = cudaMemcpyAsync(r->out.quat, d.quat, 16 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->out.strain) e = cudaMemcpyAsync(r->out.strain, d.strain, 36 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->out.correspondence)
      e = cudaMemcpyAsync(r->out.correspondence, d.correspondence, 60 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->out.von_mises) e = cudaMemcpyAsync(r->out.von_mises, d.von_mises, 4 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r->out.rodrigues) e = cudaMemcpyAsync(r->out.rodrigues, d.rodrigues, 12 * n, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(F->done, st);
  if (e != cudaSuccess) { batch_free(b); delete F; return cuda_fail(ctx, e, "serve: outputs"); }
  F->batch = b;
  *out = F;
  return PTM_OK;
}

void retire(ptm_server *S, InFlight *F, ptm_status status) {
  const double t = now_s();
  for (Request *r : F->reqs) {
    S->pool.release(r->pos_bytes, r->dpos);
    if (r->dsp) S->pool.release((size_t)r->frame.n_atoms, r->dsp);
    S->pool.release(r->out_bytes, r->dout);
    r->dpos = r->dout = nullptr;
    r->dsp = nullptr;
  }
  S->pool.release(F->ws_bytes, F->ws);
  cudaEventDestroy(F->done);
  batch_free(F->batch);
  std::lock_guard<std::mutex> lock(S->mu);
  for (Request *r : F->reqs) {
    S->in_use -= r->bytes;
    r->t_done = t;
    r->status = status;
    r->state = 2;
  }
  S->slot_busy[F->slot] = false;
  S->cv_done.notify_all();
}

void serve_loop(ptm_server *S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lock(S->mu);
  for (;;) {
    // completions: a batch whose event reports an error (or that a test marked
    // as failed) completes with PTM_ERR_CUDA instead of waiting for ever
    std::vector<std::pair<InFlight *, ptm_status>> finished;
    for (size_t i = 0; i < S->inflight.size();) {
      InFlight *F = S->inflight[i];
      const cudaError_t q = F == S->held ? cudaErrorNotReady : cudaEventQuery(F->done);
      if (q == cudaErrorNotReady) { i++; continue; }
      ptm_status st = PTM_OK;
      if (q != cudaSuccess || F->fail) {
        st = PTM_ERR_CUDA;
        S->error = std::string("serve: batch completion failed: ") +
                   (q != cudaSuccess ? cudaGetErrorString(q) : "injected by ptm_server_inject");
        if (q != cudaSuccess) cudaGetLastError();
      }
      finished.push_back({F, st});
      S->inflight.erase(S->inflight.begin() + i);
    }
    if (!finished.empty()) {
      lock.unlock();
      for (auto &fs : finished) retire(S, fs.first, fs.second);
      lock.lock();
      continue;
    }
    if (S->stop && S->queue.empty() && S->inflight.empty()) break;
    // admission + launch on a free slot
    int slot = -1;
    for (int i = 0; i < S->nslots; i++) if (!S->slot_busy[i]) { slot = i; break; }
    std::vector<Request *> take;
    int64_t batch_atoms = 0;
    if (slot >= 0) {
      while (!S->queue.empty() && (int)take.size() < S->max_batch) {
        Request *r = S->queue.front();
        if (r->bytes > S->budget) {                 // can never fit
          S->queue.pop_front();
          r->status = PTM_ERR_OUT_OF_MEMORY;
          r->state = 2;
          r->t_done = now_s();
          S->cv_done.notify_all();
          continue;
        }
        if (S->in_use + r->bytes > S->budget) break;
        if (!take.empty() && r->frame.pos_dtype != take[0]->frame.pos_dtype) break;
        if (!take.empty() && batch_atoms + r->frame.n_atoms > S->max_batch_atoms) break;
        batch_atoms += r->frame.n_atoms;
        S->queue.pop_front();
        S->in_use += r->bytes;
        take.push_back(r);
      }
    }
    if (!take.empty()) {
      S->slot_busy[slot] = true;
      const int64_t bid = S->next_batch++;
      const double t = now_s();
      for (Request *r : take) { r->state = 1; r->t_start = t; r->batch = bid; }
      lock.unlock();
      InFlight *F = nullptr;
      ptm_status rs = launch_batch(S, take, slot, &F);
      if (rs != PTM_OK) cudaStreamSynchronize(S->streams[slot]);   // copies may be in flight
      lock.lock();
      if (rs == PTM_OK) {
        if (S->hold_next) { S->held = F; S->hold_next = false; }
        if (S->fail_next > 0) { F->fail = true; S->fail_next--; }
        S->inflight.push_back(F);
      } else {
        S->error = S->ctx->last_error;
        for (Request *r : take) {
          S->in_use -= r->bytes;
          r->status = rs;
          r->state = 2;
          r->t_done = now_s();
          if (r->dpos) S->pool.release(r->pos_bytes, r->dpos);
          if (r->dsp) S->pool.release((size_t)r->frame.n_atoms, r->dsp);
          if (r->dout) S->pool.release(r->out_bytes, r->dout);
          r->dpos = r->dout = nullptr;
          r->dsp = nullptr;
        }
        S->slot_busy[slot] = false;
        S->cv_done.notify_all();
      }
      continue;
    }
    // nothing to launch: wait for a submission or poll in-flight work
    S->cv_work.wait_for(lock, std::chrono::microseconds(S->inflight.empty() ? 2000 : 50));
  }
}

}  // namespace

extern "C" ptm_status ptm_server_create(ptm_context *ctx, const ptm_server_options *opt, ptm_server **out) {
  if (!ctx || !out) return PTM_ERR_INVALID_ARG;
  *out = nullptr;
  CK(cudaSetDevice(ctx->device));
  ptm_server *S = new (std::nothrow) ptm_server();
  if (!S) return PTM_ERR_OUT_OF_MEMORY;
  S->ctx = ctx;
  S->budget = (opt && opt->hbm_budget_bytes) ? opt->hbm_budget_bytes : ctx->budget;
  if (opt && opt->max_batch_frames > 0) S->max_batch = opt->max_batch_frames;
  if (opt && opt->streams > 0) S->nslots = std::min(opt->streams, 8);
  if (opt && opt->max_batch_atoms > 0) S->max_batch_atoms = opt->max_batch_atoms;
  if (opt) S->tuning = opt->tuning;
  S->staging_bytes = (sizeof(FrameDesc) + sizeof(ShiftTables) + sizeof(BinParams) + 2 * sizeof(int64_t) +
                      sizeof(int)) * (size_t)S->max_batch;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < S->nslots && e == cudaSuccess; i++) {
    cudaStream_t st = nullptr;
    void *h = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&h, S->staging_bytes);
    S->streams.push_back(st);
    S->staging.push_back(h);
    S->slot_busy.push_back(false);
  }
  if (e != cudaSuccess) {
    ptm_status rs = cuda_fail(ctx, e, "ptm_server_create");
    for (auto st : S->streams) if (st) cudaStreamDestroy(st);
    for (auto h : S->staging) if (h) cudaFreeHost(h);
    delete S;
    return rs;
  }
  S->worker = std::thread(serve_loop, S);
  *out = S;
  return PTM_OK;
}

extern "C" ptm_status ptm_submit(ptm_server *S, const ptm_frame *frame, const ptm_outputs *out, uint64_t *ticket) {
  if (!S || !frame || !out || !ticket) return PTM_ERR_INVALID_ARG;
  if (frame->n_atoms < 1 || frame->n_atoms >= (1ll << 31) || !frame->positions) return PTM_ERR_INVALID_ARG;
  if (frame->pos_dtype != PTM_F32 && frame->pos_dtype != PTM_F64) return PTM_ERR_INVALID_ARG;
  if (frame->ordering != PTM_ORDER_EUCLIDEAN && frame->ordering != PTM_ORDER_TOPOLOGICAL) return PTM_ERR_INVALID_ARG;
  if (!finite_cell(frame->cell)) return PTM_ERR_INVALID_ARG;
  Request *r = new (std::nothrow) Request();
  if (!r) return PTM_ERR_OUT_OF_MEMORY;
  r->frame = *frame;
  r->out = *out;
  r->bytes = request_bytes(*frame);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) { delete r; return PTM_ERR_INVALID_ARG; }
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
  }
  S->cv_work.notify_one();
  return PTM_OK;
}

extern "C" ptm_status ptm_poll(ptm_server *S, uint64_t ticket, int *done) {
  if (!S || !done) return PTM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return PTM_ERR_NOT_FOUND;
  *done = it->second->state == 2;
  return *done ? it->second->status : PTM_OK;
}

extern "C" ptm_status ptm_wait(ptm_server *S, uint64_t ticket, int timeout_ms) {
  if (!S) return PTM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return PTM_ERR_NOT_FOUND;
  Request *r = it->second;
  const auto pred = [&] { return r->state == 2; };
  if (timeout_ms < 0) S->cv_done.wait(lock, pred);
  else if (!S->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) return PTM_ERR_TIMEOUT;
  return r->status;
}

extern "C" ptm_status ptm_ticket_info(ptm_server *S, uint64_t ticket, double *times, int64_t *batch) {
  if (!S) return PTM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return PTM_ERR_NOT_FOUND;
  const Request *r = it->second;
  if (times) { times[0] = r->t_submit; times[1] = r->t_start; times[2] = r->t_done; }
  if (batch) *batch = r->batch;
  return PTM_OK;
}

extern "C" ptm_status ptm_release(ptm_server *S, uint64_t ticket) {
  if (!S) return PTM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return PTM_ERR_NOT_FOUND;
  if (it->second->state != 2) return PTM_ERR_BUSY;
  delete it->second;
  S->reqs.erase(it);
  return PTM_OK;
}

extern "C" ptm_status ptm_server_inject(ptm_server *S, int fault) {
  if (!S) return PTM_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    switch (fault) {
      case PTM_FAULT_HOLD_NEXT: S->hold_next = true; break;
      case PTM_FAULT_RELEASE_HELD: S->hold_next = false; S->held = nullptr; break;
      case PTM_FAULT_FAIL_NEXT: S->fail_next++; break;
      default: return PTM_ERR_INVALID_ARG;
    }
  }
  S->cv_work.notify_all();
  return PTM_OK;
}

extern "C" ptm_status ptm_server_destroy(ptm_server *S) {
  if (!S) return PTM_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
    S->hold_next = false;          // a held completion is seen again, so the drain ends
    S->held = nullptr;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();       // drains queued and in-flight work
  cudaSetDevice(S->ctx->device);
  for (auto st : S->streams) cudaStreamDestroy(st);
  for (auto h : S->staging) cudaFreeHost(h);
  for (auto &kv : S->reqs) delete kv.second;
  delete S;
  cudaGetLastError();
  return PTM_OK;
}
