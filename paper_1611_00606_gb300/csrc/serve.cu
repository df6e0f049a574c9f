// Serving: continuous batching of k-point requests on one plan.
//
// hs_submit() queues a request and returns a ticket.  A scheduler thread
// admits queued requests in arrival order whenever the request's exact device
// footprint (its workspace plus its H and S) fits in the plan's HBM budget
// next to the requests already running, and a stream slot is free.  Each
// admitted request gets a workspace from a dedicated stream-ordered memory
// pool and its own stream, so requests that arrive while others run are
// admitted as memory frees up and their kernels overlap on the device.  A
// host callback on the request's stream marks completion; the scheduler then
// returns the workspace to the pool.  Every request runs the same kernels with
// the same reduction order as hs_assemble, so its H and S are bitwise the same
// alone and in any mix.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <new>

#include "plan.h"

namespace {

constexpr int kAtomsBatchMax = 16;  // requests per grouped per-atom launch

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  int64_t ticket = 0;
  const double2* A = nullptr;
  const double2* B = nullptr;
  int ld = 0;
  const double* U = nullptr;
  int N_G = 0;
  double2* H = nullptr;
  double2* S = nullptr;
  size_t fp = 0;
  size_t inflight_at_admit = 0;
  double t_submit = 0, t_admit = 0;
  std::atomic<double> t_done{0.0};
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e_in = nullptr;
  Workspace ws;
  std::atomic<int> gpu_done{0};
  int state = 0;  // 0 queued, 1 running, 2 finished (resources returned)
  int rc = HS_OK;
  ServeState* owner = nullptr;
};

}  // namespace

struct ServeState {
  hs_plan_s* plan = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<int64_t, Request*> reqs;
  std::vector<Request*> running;
  std::vector<cudaStream_t> free_streams;
  size_t in_use = 0;
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  cudaMemPool_t pool = nullptr;
  cudaStream_t batch_stream = nullptr;  // grouped per-atom launches (split form)
  AtomsGraph* graph = nullptr;
  uint64_t batches = 0, batched_requests = 0;
  static constexpr int kMaxRunning = 16;
  static constexpr size_t kMaxQueue = 1u << 16;
};

namespace {

void CUDART_CB on_done(void* arg) {
  Request* r = (Request*)arg;
  ServeState* S = r->owner;  // r may be retired as soon as gpu_done is set
  r->t_done.store(now_s());
  r->gpu_done.store(1);
  S->cv.notify_all();  // no CUDA calls and no locks in a host callback
}

int take_stream(ServeState* S, Request* r) {
  if (S->free_streams.empty()) {
    cudaStream_t st;
    HS_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    S->free_streams.push_back(st);
  }
  r->st = S->free_streams.back();
  S->free_streams.pop_back();
  HS_CUDA_TRY(cudaEventCreate(&r->e0));
  HS_CUDA_TRY(cudaEventCreate(&r->e1));
  HS_CUDA_TRY(cudaEventRecord(r->e0, r->st));
  return HS_OK;
}

int finish_launch(Request* r) {
  HS_CUDA_TRY(cudaEventRecord(r->e1, r->st));
  HS_CUDA_TRY(cudaLaunchHostFunc(r->st, on_done, r));
  return HS_OK;
}

// Launch one admitted request on its own stream (FP64 form).
int launch(ServeState* S, Request* r) {
  hs_plan_s* p = S->plan;
  int rc = take_stream(S, r);
  if (rc != HS_OK) return rc;
  rc = p->ws_alloc(r->ws, r->N_G, p->N_f, r->st, true);
  if (rc != HS_OK) return rc;
  rc = p->enqueue(r->A, r->B, r->ld, r->U, r->N_G, r->H, r->S, r->ws, r->st, false);
  if (rc != HS_OK) return rc;
  return finish_launch(r);
}

// Split form: the requests admitted in one pass share one grouped per-atom launch.
// Each request slices its inputs on its own stream; the batch stream waits for all
// of them, replays the plan's graph (grouped MODE_ATOMS kernel over every request's
// atoms), and each request stream waits for it before its own slicing of Z, Y, X,
// its contractions and its mirror.  Returns per-request codes in rcs.
void launch_batch(ServeState* S, std::vector<Request*>& batch, std::vector<int>& rcs) {
  hs_plan_s* p = S->plan;
  rcs.assign(batch.size(), HS_OK);
  std::vector<AtomsJob> jobs;
  std::vector<Request*> ready;
  for (size_t i = 0; i < batch.size(); ++i) {
    Request* r = batch[i];
    int rc = take_stream(S, r);
    if (rc == HS_OK) rc = p->ws_alloc(r->ws, r->N_G, p->N_f, r->st, true);
    if (rc == HS_OK) rc = p->split_inputs(r->A, r->B, r->ld, r->U, r->N_G, r->ws, r->st);
    if (rc == HS_OK && cudaEventCreateWithFlags(&r->e_in, cudaEventDisableTiming) != cudaSuccess)
      rc = HS_ECUDA;
    if (rc == HS_OK && cudaEventRecord(r->e_in, r->st) != cudaSuccess) rc = HS_ECUDA;
    rcs[i] = rc;
    if (rc == HS_OK) {
      jobs.push_back(AtomsJob{&r->ws, r->N_G});
      ready.push_back(r);
    }
  }
  if (ready.empty()) return;
  int rc = HS_OK;
  cudaEvent_t e_atoms = nullptr;
  if (!S->batch_stream &&
      cudaStreamCreateWithFlags(&S->batch_stream, cudaStreamNonBlocking) != cudaSuccess)
    rc = HS_ECUDA;
  if (rc == HS_OK && !S->graph && !(S->graph = hs_atoms_graph_new())) rc = HS_ENOMEM;
  for (Request* r : ready)
    if (rc == HS_OK && cudaStreamWaitEvent(S->batch_stream, r->e_in, 0) != cudaSuccess)
      rc = HS_ECUDA;
  if (rc == HS_OK) rc = p->split_atoms(jobs.data(), (int)jobs.size(), S->batch_stream, S->graph);
  if (rc == HS_OK && cudaEventCreateWithFlags(&e_atoms, cudaEventDisableTiming) != cudaSuccess)
    rc = HS_ECUDA;
  if (rc == HS_OK && cudaEventRecord(e_atoms, S->batch_stream) != cudaSuccess) rc = HS_ECUDA;
  if (rc == HS_OK) {
    S->batches += 1;
    S->batched_requests += ready.size();
  }
  for (size_t i = 0, k = 0; i < batch.size(); ++i) {
    if (rcs[i] != HS_OK) continue;
    Request* r = ready[k++];
    int rr = rc;
    if (rr == HS_OK && cudaStreamWaitEvent(r->st, e_atoms, 0) != cudaSuccess) rr = HS_ECUDA;
    if (rr == HS_OK) rr = p->split_outputs(r->A, r->ld, r->N_G, r->H, r->S, r->ws, r->st, false);
    if (rr == HS_OK && hs_launch_mirror(r->H, r->N_G, r->N_G, r->st) != cudaSuccess) rr = HS_ECUDA;
    if (rr == HS_OK) rr = finish_launch(r);
    rcs[i] = rr;
  }
  if (e_atoms) cudaEventDestroy(e_atoms);  // released once its waits are satisfied
}

void finish(ServeState* S, Request* r) {
  hs_plan_s* p = S->plan;
  if (r->e_in) {
    cudaEventDestroy(r->e_in);
    r->e_in = nullptr;
  }
  if (r->ws.Z || r->ws.W2) p->ws_free(r->ws, r->st);
  if (r->st) S->free_streams.push_back(r->st);
  S->in_use -= r->fp;
  r->state = 2;
}

void scheduler(ServeState* S) {
  cudaSetDevice(S->plan->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // harvest completed requests
    for (size_t i = 0; i < S->running.size();) {
      Request* r = S->running[i];
      if (r->gpu_done.load()) {
        int err = S->plan->check_device_error();
        if (err != HS_OK) r->rc = err;
        finish(S, r);
        S->running[i] = S->running.back();
        S->running.pop_back();
      } else {
        ++i;
      }
    }
    // admit in arrival order: the head blocks until it fits (FIFO fairness)
    std::vector<Request*> batch;
    while (!S->queue.empty() && (int)(S->running.size() + batch.size()) < ServeState::kMaxRunning &&
           (int)batch.size() < kAtomsBatchMax) {
      Request* r = S->queue.front();
      if (S->plan->budget && S->in_use + r->fp > S->plan->budget) break;
      S->queue.pop_front();
      S->in_use += r->fp;
      r->inflight_at_admit = S->in_use;
      r->t_admit = now_s();
      r->state = 1;
      batch.push_back(r);
    }
    if (!batch.empty()) {
      std::vector<int> rcs(batch.size(), HS_OK);
      if (S->plan->precision == HS_SPLIT_BF16) {
        launch_batch(S, batch, rcs);
      } else {
        for (size_t i = 0; i < batch.size(); ++i) rcs[i] = launch(S, batch[i]);
      }
      for (size_t i = 0; i < batch.size(); ++i) {
        Request* r = batch[i];
        if (rcs[i] != HS_OK) {
          cudaGetLastError();
          r->rc = rcs[i];
          if (r->st) cudaStreamSynchronize(r->st);
          finish(S, r);
        } else {
          S->running.push_back(r);
        }
      }
    }
    S->cv.notify_all();
    if (S->stop && S->running.empty()) break;
    S->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

ServeState* ensure_serve(hs_plan_s* p) {
  if (p->serve) return p->serve;
  ServeState* S = new (std::nothrow) ServeState();
  if (!S) return nullptr;
  S->plan = p;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = p->device;
  if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
    cudaGetLastError();
    S->pool = nullptr;
  } else {
    uint64_t keep = UINT64_MAX;  // keep freed blocks for the next request
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  p->serve = S;
  S->th = std::thread(scheduler, S);
  return S;
}

}  // namespace

// Workspaces of serving requests come from the plan's own pool when it exists.
cudaMemPool_t hs_serve_pool(hs_plan_s* p) { return p->serve ? p->serve->pool : nullptr; }

bool hs_plan_s::serve_busy() {
  if (!serve) return false;
  std::lock_guard<std::mutex> lk(serve->mu);
  return !serve->queue.empty() || !serve->running.empty();
}

void hs_plan_s::serve_shutdown() {
  ServeState* S = serve;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    // queued requests that never started are cancelled
    for (Request* r : S->queue) {
      r->rc = HS_ECUDA;
      r->state = 2;
    }
    S->queue.clear();
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->th.joinable()) S->th.join();
  // every stream is back in the pool; wait for their host callbacks to return
  for (cudaStream_t st : S->free_streams) cudaStreamSynchronize(st);
  for (auto& kv : S->reqs) {
    Request* r = kv.second;
    if (r->e0) cudaEventDestroy(r->e0);
    if (r->e1) cudaEventDestroy(r->e1);
    delete r;
  }
  if (S->batch_stream) {
    cudaStreamSynchronize(S->batch_stream);
    cudaStreamDestroy(S->batch_stream);
  }
  hs_atoms_graph_free(S->graph);
  for (cudaStream_t st : S->free_streams) cudaStreamDestroy(st);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  delete S;
  serve = nullptr;
}

extern "C" int hs_submit(hs_plan_t p, const hs_z* A, const hs_z* B, int ld_AB, const double* U,
                         int N_G, hs_z* H, hs_z* S, int64_t* ticket) {
  if (!p || !A || !B || !U || !H || !S || !ticket || H == S) return HS_EINVAL;
  if (p->real) return HS_ENOTSUP;  // serving takes complex requests only
  if (N_G < 1 || N_G > p->N_G_max || ld_AB < p->N_A * p->N_L) return HS_EINVAL;
  size_t fp;
  {
    std::lock_guard<std::mutex> lk(p->mu);
    if (!p->t_valid) return HS_EINVAL;  // hs_set_t first
    fp = p->ws_bytes(N_G, p->N_f) + (size_t)2 * 16 * N_G * (size_t)N_G;
    if (p->budget && fp > p->budget) return HS_ENOMEM;
    if (!ensure_serve(p)) return HS_ENOMEM;
  }
  ServeState* SS = p->serve;
  Request* r = new (std::nothrow) Request();
  if (!r) return HS_ENOMEM;
  r->A = (const double2*)A;
  r->B = (const double2*)B;
  r->ld = ld_AB;
  r->U = U;
  r->N_G = N_G;
  r->H = (double2*)H;
  r->S = (double2*)S;
  r->fp = fp;
  r->owner = SS;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(SS->mu);
    if (SS->queue.size() >= ServeState::kMaxQueue) {
      delete r;
      return HS_EBUSY;
    }
    r->ticket = SS->next_ticket++;
    SS->reqs[r->ticket] = r;
    SS->queue.push_back(r);
  }
  SS->cv.notify_all();
  *ticket = r->ticket;
  return HS_OK;
}

extern "C" int hs_poll(hs_plan_t p, int64_t ticket, int64_t timeout_us, hs_info* info) {
  if (!p || !p->serve) return HS_EINVAL;
  ServeState* S = p->serve;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return HS_EINVAL;
  Request* r = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(
                                                              timeout_us > 0 ? timeout_us : 0);
  while (r->state != 2) {
    if (timeout_us == 0) return HS_PENDING;
    if (timeout_us > 0) {
      if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && r->state != 2)
        return HS_ETIMEDOUT;
    } else {
      S->cv.wait_for(lk, std::chrono::milliseconds(10));
    }
  }
  const int rc = r->rc;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->n_fallback = p->N_f;
    info->slices = p->slices;
    float ms = 0.f;
    if (r->e0 && r->e1 && cudaEventElapsedTime(&ms, r->e0, r->e1) == cudaSuccess)
      info->ms_total = ms;
    else
      cudaGetLastError();
    info->ms_queue = 1e3 * (r->t_admit - r->t_submit);
    info->ms_latency = 1e3 * (r->t_done.load() - r->t_submit);
    info->inflight_bytes = (double)r->inflight_at_admit;
  }
  if (r->e0) cudaEventDestroy(r->e0);
  if (r->e1) cudaEventDestroy(r->e1);
  S->reqs.erase(it);
  delete r;
  return rc;
}
