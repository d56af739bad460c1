// Continuous-batching server for elastance and mobility solves.
//
// Worker threads each own a context and a non-blocking CUDA stream; a request
// runs on one worker from start to finish, so the solves of different requests
// overlap on the device.  Admission is by device-memory footprint: a request
// starts only when a worker is free and its workspace fits under the cap
// together with the requests in flight.  The queue is first-in first-out,
// except that a request that fits may pass the head of the queue when the
// head does not fit yet, at most kMaxPass times per head request.  With
// batching on (bie_server_batching), a worker that takes a request also takes
// queued requests of the same kind and options (up to the batch limits) and
// solves them together as one block-diagonal system (the batched solves).
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/bie2d.h"
#include "bie_internal.cuh"

namespace {

constexpr int kMaxPass = 64;
using Clock = std::chrono::steady_clock;

struct Job {
  bie_request req;
  int64_t ticket = 0;
  size_t need = 0;
  std::vector<int> bs;  // body_start (host copy)
  Clock::time_point t_submit;
  double seconds = 0.0;
  int status = BIE_OK;
  bie_info info{};
  bool done = false;
};

}  // namespace

struct bie_server {
  int device = 0;
  size_t cap = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::unordered_map<int64_t, Job*> jobs;
  size_t inflight = 0, peak = 0;
  int64_t next_ticket = 1, completed = 0;
  int head_passed = 0;
  bool stopping = false;
  int max_batch = 1;                  // requests a worker may solve together
  int max_request_nodes = 16384;      // larger requests are solved alone
  int max_batch_nodes = 262144;       // nodes of one batch
  int64_t batches = 0;                // batched solves run (two or more requests)
  std::vector<std::thread> workers;
};

namespace {

// Pick the next job a free worker may run (mu held); nullptr if none fits.
Job* pick(bie_server* s) {
  if (s->queue.empty()) return nullptr;
  auto fits = [&](const Job* j) { return s->cap == 0 || s->inflight == 0 || s->inflight + j->need <= s->cap; };
  if (fits(s->queue.front())) {
    Job* j = s->queue.front();
    s->queue.pop_front();
    s->head_passed = 0;
    return j;
  }
  if (s->head_passed >= kMaxPass) return nullptr;  // the head waits for memory; nobody passes it now
  for (auto it = s->queue.begin() + 1; it != s->queue.end(); ++it) {
    if (fits(*it)) {
      Job* j = *it;
      s->queue.erase(it);
      s->head_passed += 1;
      return j;
    }
  }
  return nullptr;
}

bool batchable(const bie_server* s, const Job* j) {
  return j->req.density == nullptr && j->req.opts.fmm_order == 0 && j->bs.back() <= s->max_request_nodes;
}

bool same_batch(const Job* a, const Job* b) {
  return a->req.kind == b->req.kind && memcmp(&a->req.opts, &b->req.opts, sizeof(bie_opts)) == 0 &&
         (a->req.geom.interior_pt != nullptr) == (b->req.geom.interior_pt != nullptr);
}

// After pick: more queued requests to solve together with `first` (mu held),
// in queue order, while the batch's workspace fits under the cap.  Returns
// the bytes to reserve for the whole batch.
size_t grow_batch(bie_server* s, Job* first, std::vector<Job*>& batch) {
  batch.assign(1, first);
  size_t need = first->need;
  if (s->max_batch <= 1 || !batchable(s, first)) return need;
  std::vector<int> bs(first->bs), pb{0, (int)first->bs.size() - 1};
  int nodes = first->bs.back();
  for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < s->max_batch;) {
    Job* c = *it;
    if (!batchable(s, c) || !same_batch(first, c) || nodes + c->bs.back() > s->max_batch_nodes) {
      ++it;
      continue;
    }
    std::vector<int> bs2(bs), pb2(pb);
    const int off = bs2.back();
    for (size_t i = 1; i < c->bs.size(); ++i) bs2.push_back(off + c->bs[i]);
    pb2.push_back(pb2.back() + (int)c->bs.size() - 1);
    const int N = (int)bs2.size() - 1, P = (int)pb2.size() - 1;
    const size_t need2 = bie::workspace_bytes_batch(first->req.kind, bs2.data(), N, pb2.data(), P, &first->req.opts);
    if (s->cap && s->inflight + need2 > s->cap) break;  // the batch would not fit
    batch.push_back(c);
    bs.swap(bs2);
    pb.swap(pb2);
    nodes += c->bs.back();
    need = need2;
    it = s->queue.erase(it);
  }
  return need;
}

void finish(bie_server* s, Job* j, int status, const bie_info& info) {
  j->status = status;
  j->info = info;
  j->seconds = std::chrono::duration<double>(Clock::now() - j->t_submit).count();
  j->done = true;
  s->completed += 1;
}

void worker_main(bie_server* s) {
  cudaSetDevice(s->device);
  bie_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  const bool ok = bie_create(&ctx, s->device, 0) == BIE_OK &&
                  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
  std::vector<Job*> batch;
  std::vector<bie_geometry> geoms;
  std::vector<const double*> loads;
  std::vector<double*> outs;
  std::vector<bie_info> infos;
  std::vector<int> status;
  auto solo = [&](Job* b, bie_info* info) -> int {
    const bie_request& r = b->req;
    if (r.kind == BIE_KIND_LAPLACE)
      return elastance_solve(ctx, &r.geom, r.load, r.out, r.density, &r.opts, info, stream);
    return mobility_solve(ctx, &r.geom, r.load, r.out, r.density, &r.opts, info, stream);
  };
  for (;;) {
    Job* j = nullptr;
    size_t reserved = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return (s->stopping && s->queue.empty()) || (j = pick(s)) != nullptr; });
      if (!j) break;
      reserved = grow_batch(s, j, batch);
      s->inflight += reserved;
      if (s->inflight > s->peak) s->peak = s->inflight;
      if (batch.size() > 1) s->batches += 1;
    }
    const int P = (int)batch.size();
    infos.assign(P, bie_info{});
    status.assign(P, BIE_ERR_CUDA);
    if (ok) {
      const bie_opts* opts = &j->req.opts;
      if (P == 1) {
        status[0] = solo(j, &infos[0]);
      } else {
        geoms.clear();
        loads.clear();
        outs.clear();
        for (Job* b : batch) {
          geoms.push_back(b->req.geom);
          loads.push_back(b->req.load);
          outs.push_back(b->req.out);
        }
        const int rc = j->req.kind == BIE_KIND_LAPLACE
                           ? elastance_solve_batch(ctx, P, geoms.data(), loads.data(), outs.data(), opts,
                                                   infos.data(), status.data(), stream)
                           : mobility_solve_batch(ctx, P, geoms.data(), loads.data(), outs.data(), opts,
                                                  infos.data(), status.data(), stream);
        if (rc < 0) {
          // one bad request must fail alone: solve the batch's requests one by one
          cudaStreamSynchronize(stream);
          for (int p = 0; p < P; ++p) status[p] = solo(batch[p], &infos[p]);
        }
      }
      // memory follows the requests in flight: hand the workspace back to the pool
      bie::release_workspace(ctx, stream);
      cudaStreamSynchronize(stream);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->inflight -= reserved;
      for (int p = 0; p < P; ++p) finish(s, batch[p], status[p], infos[p]);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
  if (ctx) bie_destroy(ctx);
}

bool is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int bie_server_create(bie_server** out, int device, int workers, size_t hbm_cap_bytes) {
  if (!out || workers < 1 || workers > 256) return BIE_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  bie_server* s = new bie_server();
  s->device = device;
  s->cap = hbm_cap_bytes;
  for (int w = 0; w < workers; ++w) s->workers.emplace_back(worker_main, s);
  *out = s;
  return BIE_OK;
}

int bie_server_submit(bie_server* s, const bie_request* req, int64_t* ticket) {
  if (!s || !req || !ticket) return BIE_ERR_INVALID;
  const bie_geometry& g = req->geom;
  if ((req->kind != BIE_KIND_LAPLACE && req->kind != BIE_KIND_STOKES) || g.n_bodies < 1 || !g.body_start ||
      !req->load || !req->out)
    return BIE_ERR_INVALID;
  // body_start (host or device) sizes the workspace
  std::vector<int> bs(g.n_bodies + 1);
  if (is_device(g.body_start)) {
    cudaSetDevice(s->device);
    if (cudaMemcpy(bs.data(), g.body_start, bs.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return BIE_ERR_CUDA;
  } else {
    std::copy(g.body_start, g.body_start + g.n_bodies + 1, bs.begin());
  }
  if (bs[g.n_bodies] < 8) return BIE_ERR_INVALID;
  for (int i = 0; i < g.n_bodies; ++i)
    if (bs[i + 1] < bs[i]) return BIE_ERR_INVALID;
  cudaSetDevice(s->device);
  const size_t need = bie::workspace_bytes_for(req->kind, bs.data(), g.n_bodies, req->opts.restart);
  if (s->cap && need > s->cap) return BIE_ERR_NOMEM;
  Job* j = new Job();
  j->req = *req;
  j->need = need;
  j->bs.swap(bs);
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
      delete j;
      return BIE_ERR_INVALID;
    }
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    *ticket = j->ticket;
  }
  s->cv_work.notify_one();
  return BIE_OK;
}

int bie_server_wait(bie_server* s, int64_t ticket, bie_info* info, double* seconds) {
  if (!s) return BIE_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return BIE_ERR_INVALID;
  Job* j = it->second;
  s->cv_done.wait(lk, [&] { return j->done; });
  const int status = j->status;
  if (info) *info = j->info;
  if (seconds) *seconds = j->seconds;
  s->jobs.erase(it);
  delete j;
  return status;
}

int bie_server_batching(bie_server* s, int max_batch, int max_request_nodes, int64_t* batches) {
  if (!s || max_batch < 0 || max_batch > 65535 || max_request_nodes < 0) return BIE_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (max_batch > 0) s->max_batch = max_batch;
  if (max_request_nodes > 0) s->max_request_nodes = max_request_nodes;
  if (batches) *batches = s->batches;
  return BIE_OK;
}

int bie_server_stats(bie_server* s, int64_t* completed, size_t* inflight, size_t* peak) {
  if (!s) return BIE_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (inflight) *inflight = s->inflight;
  if (peak) *peak = s->peak;
  return BIE_OK;
}

void bie_server_destroy(bie_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
}

}  // extern "C"
