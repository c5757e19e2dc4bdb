// tmd_serve.cu -- serving: admission by device-memory budget, resident
// buffers, continuous batching.
//
// tmd_submit queues a request.  A driver thread admits queued requests in
// arrival order while the memory budget and the slot table allow, gives each
// admitted frame resident output buffers (and, for frames in host memory,
// copies the compressed streams into resident device buffers on a copy
// stream; device-resident frames are decoded in place), and launches every
// frame whose inputs are ready in the next batch -- one launch chain over all
// of them -- on one of two compute streams, so a new batch starts while the
// previous one still runs.  Buffers stay resident until tmd_release; tmd_poll
// hands out the decoded buffers.  The decoded bytes of a
// frame depend only on the frame, never on the batch it ran in.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "tmd_api_internal.h"

namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

enum class ReqState { kQueued, kCopying, kRunning, kDone, kFailed };

struct Request {
  uint64_t id = 0;
  tmd_frame_in src;           // caller's frame
  tmd_frame_in in;            // frame as decoded: the caller's (device sources) or a copy
  bool borrow = false;        // device source: decoded in place, no copy
  tmd_frame_out out;          // resident outputs
  void* mem = nullptr;        // one allocation holding inputs and outputs
  size_t bytes = 0;           // budget charge (buffers + scratch estimate)
  ReqState state = ReqState::kQueued;
  cudaEvent_t copied = nullptr;
  int batch = -1;
  int err = TMD_OK;
};

struct Batch {
  std::vector<uint64_t> ids;
  void* scratch = nullptr;
  void* dev_record = nullptr;
  cudaEvent_t done = nullptr;
  int stream = 0;
};

}  // namespace

struct TmdServer {
  tmd_handle* h = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread driver;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<uint64_t> queue;                 // submitted, not admitted
  std::map<uint64_t, Request> reqs;
  std::vector<Batch*> running;
  uint64_t used = 0;                          // bytes charged by admitted requests
  uint32_t active = 0;                        // admitted, not released
  cudaStream_t copy = nullptr;
  cudaStream_t compute[2] = {nullptr, nullptr};
  bool busy[2] = {false, false};          // a batch is running on compute[i]
  void* record[2] = {nullptr, nullptr};   // pinned launch record per compute stream
  size_t record_bytes[2] = {0, 0};
  std::string err;

  void run();
};

namespace {

// Byte layout of a request's resident buffers (inputs then outputs).
struct ReqLayout {
  size_t off[23];
  size_t native, row_start, att_count, status, total;
};

const size_t kElem[23] = {1, 1, 1, 2, 4, 2, 2, 2, 1, 1, 1, 1, 1, 2, 4, 4, 2, 4, 2, 2, 1, 1, 1};
// length kind of each field: 0 track, 1 attached, 2 difference, 3 bin, 4 unattached
const int kKind[23] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 4, 4, 4, 4, 4, 4, 4};

const void** field_ptr(tmd_frame_in& f, int i) {
  const void** p[23] = {(const void**)&f.qpt, (const void**)&f.row, (const void**)&f.slice,
                        (const void**)&f.pad, (const void**)&f.time, (const void**)&f.ncl,
                        (const void**)&f.qtot_a, (const void**)&f.qmax_a,
                        (const void**)&f.flags_a, (const void**)&f.sigma_pad_a,
                        (const void**)&f.sigma_time_a, (const void**)&f.row_diff,
                        (const void**)&f.slice_leg_diff, (const void**)&f.pad_res,
                        (const void**)&f.time_res, (const void**)&f.n_unatt,
                        (const void**)&f.pad_diff_u, (const void**)&f.time_diff_u,
                        (const void**)&f.qtot_u, (const void**)&f.qmax_u,
                        (const void**)&f.flags_u, (const void**)&f.sigma_pad_u,
                        (const void**)&f.sigma_time_u};
  return p[i];
}

size_t field_len(const tmd_frame_in& f, int i) {
  switch (kKind[i]) {
    case 0: return f.n_tracks;
    case 1: return f.n_attached;
    case 2: return (size_t)f.n_attached - f.n_tracks;
    case 3: return TMD_NBIN;
    default: return f.n_unattached;
  }
}

ReqLayout req_layout(const tmd_frame_in& f) {
  ReqLayout L;
  size_t o = 0;
  for (int i = 0; i < 23; i++) {
    L.off[i] = o;
    o += up256(field_len(f, i) * kElem[i]);
  }
  L.native = o;
  o += up256(((size_t)f.n_attached + f.n_unattached) * TMD_REC_BYTES);
  L.row_start = o;
  o += up256(4 * (TMD_NBIN + 1));
  L.att_count = o;
  o += up256(4 * TMD_NBIN);
  L.status = o;
  o += 256;
  L.total = o;
  return L;
}

}  // namespace

void TmdServer::run() {
  cudaSetDevice(h->device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    bool progressed = false;
    // 1. admit queued requests in order while budget and slots allow
    while (!queue.empty()) {
      Request& r = reqs[queue.front()];
      if (active >= h->max_slots || used + r.bytes > h->mem_budget) break;
      queue.pop_front();
      const ReqLayout L = req_layout(r.src);
      const size_t mem_bytes = r.borrow ? L.total - L.native : L.total;
      if (cudaMallocAsync(&r.mem, mem_bytes, copy) != cudaSuccess) {
        cudaGetLastError();
        r.state = ReqState::kFailed;
        r.err = TMD_ERR_NOMEM;
        cv_done.notify_all();
        continue;
      }
      used += r.bytes;
      active++;
      // inputs: host sources are copied into the request's buffer, device
      // sources are decoded in place; outputs follow the inputs (or start
      // the buffer when the inputs are borrowed)
      char* base = static_cast<char*>(r.mem);
      char* obase = r.borrow ? base - L.native : base;
      r.in = r.src;
      if (!r.borrow) {
        for (int i = 0; i < 23; i++) {
          const size_t nb = field_len(r.src, i) * kElem[i];
          const void* s = *field_ptr(r.src, i);
          *field_ptr(r.in, i) = nb ? base + L.off[i] : nullptr;
          if (nb) cudaMemcpyAsync(base + L.off[i], s, nb, cudaMemcpyDefault, copy);
        }
      }
      r.out.native = reinterpret_cast<uint8_t*>(obase + L.native);
      r.out.row_start = reinterpret_cast<uint32_t*>(obase + L.row_start);
      r.out.att_count = reinterpret_cast<uint32_t*>(obase + L.att_count);
      r.out.status = reinterpret_cast<uint32_t*>(obase + L.status);
      cudaEventCreateWithFlags(&r.copied, cudaEventDisableTiming);
      cudaEventRecord(r.copied, copy);
      r.state = ReqState::kCopying;
      progressed = true;
    }
    // 2. batch every request whose copy has finished
    std::vector<uint64_t> ready;
    for (auto& kv : reqs)
      if (kv.second.state == ReqState::kCopying && cudaEventQuery(kv.second.copied) == cudaSuccess)
        ready.push_back(kv.first);
    const int free_stream = !busy[0] ? 0 : (!busy[1] ? 1 : -1);
    if (!ready.empty() && free_stream >= 0) {
      std::vector<tmd_frame_in> ins;
      std::vector<tmd_frame_out> outs;
      for (uint64_t id : ready) {
        ins.push_back(reqs[id].in);
        outs.push_back(reqs[id].out);
      }
      size_t sb = 0, rb = 0;
      tmd_call_sizes((uint32_t)ins.size(), ins.data(), nullptr, &sb, &rb);
      Batch* b = new Batch();
      b->ids = ready;
      b->stream = free_stream;
      cudaStream_t cs = compute[free_stream];
      int rc = TMD_OK;
      if (record_bytes[free_stream] < rb) {  // the stream is idle: safe to regrow
        if (record[free_stream]) cudaFreeHost(record[free_stream]);
        record[free_stream] = nullptr;
        record_bytes[free_stream] = 0;
        if (cudaMallocHost(&record[free_stream], 2 * rb) == cudaSuccess)
          record_bytes[free_stream] = 2 * rb;
        else
          cudaGetLastError();
      }
      if (!record[free_stream] || cudaMallocAsync(&b->scratch, sb, cs) != cudaSuccess ||
          cudaMallocAsync(&b->dev_record, rb, cs) != cudaSuccess) {
        cudaGetLastError();
        rc = TMD_ERR_NOMEM;
      }
      if (rc == TMD_OK)
        rc = tmd_enqueue(h, (uint32_t)ins.size(), ins.data(), outs.data(), nullptr, nullptr,
                         b->scratch, record[free_stream], b->dev_record, cs, false, nullptr);
      cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
      cudaEventRecord(b->done, cs);
      if (b->scratch) cudaFreeAsync(b->scratch, cs);
      if (b->dev_record) cudaFreeAsync(b->dev_record, cs);
      b->scratch = b->dev_record = nullptr;
      for (uint64_t id : ready) {
        Request& r = reqs[id];
        r.state = rc == TMD_OK ? ReqState::kRunning : ReqState::kFailed;
        r.err = rc;
      }
      busy[free_stream] = true;
      running.push_back(b);
      progressed = true;
    }
    // 3. retire finished batches
    for (size_t i = 0; i < running.size();) {
      Batch* b = running[i];
      if (cudaEventQuery(b->done) == cudaSuccess) {
        for (uint64_t id : b->ids) {
          auto it = reqs.find(id);
          if (it != reqs.end() && it->second.state == ReqState::kRunning)
            it->second.state = ReqState::kDone;
        }
        cudaEventDestroy(b->done);
        busy[b->stream] = false;
        delete b;
        running.erase(running.begin() + i);
        progressed = true;
        cv_done.notify_all();
      } else {
        i++;
      }
    }
    if (!progressed) {
      // wait for a submit/release, or poll the GPU again shortly
      cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

// The handle's server, started on first use; nullptr (with the handle's
// error set) if its allocation, streams or driver thread cannot be made.
static TmdServer* server_of(tmd_handle* h) {
  if (h->server) return h->server;
  TmdServer* s = new (std::nothrow) TmdServer();
  if (!s) {
    tmd_set_error(h, TMD_ERR_NOMEM, "server allocation failed");
    return nullptr;
  }
  s->h = h;
  cudaSetDevice(h->device);
  if (cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->compute[0], cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->compute[1], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    for (cudaStream_t st : {s->copy, s->compute[0], s->compute[1]})
      if (st) cudaStreamDestroy(st);
    delete s;
    tmd_set_error(h, TMD_ERR_CUDA, "server streams could not be created");
    return nullptr;
  }
  // keep freed pool memory resident instead of returning it to the driver
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  try {
    s->driver = std::thread([s] { s->run(); });
  } catch (...) {
    for (cudaStream_t st : {s->copy, s->compute[0], s->compute[1]}) cudaStreamDestroy(st);
    delete s;
    tmd_set_error(h, TMD_ERR_NOMEM, "server thread could not be started");
    return nullptr;
  }
  h->server = s;
  return s;
}

void tmd_serve_shutdown(tmd_handle* h) {
  TmdServer* s = h->server;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->driver.joinable()) s->driver.join();
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  for (Batch* b : s->running) {
    if (b->done) cudaEventDestroy(b->done);
    delete b;
  }
  for (void* r : s->record)
    if (r) cudaFreeHost(r);
  for (auto& kv : s->reqs) {
    if (kv.second.copied) cudaEventDestroy(kv.second.copied);
    if (kv.second.mem) cudaFree(kv.second.mem);
  }
  cudaStreamDestroy(s->copy);
  cudaStreamDestroy(s->compute[0]);
  cudaStreamDestroy(s->compute[1]);
  delete s;
  h->server = nullptr;
}

extern "C" int tmd_submit(tmd_handle* h, const tmd_frame_in* in, uint64_t* req_id) {
  if (!h || !in || !req_id) return TMD_ERR_ARG;
  // validate the frame as it will be decoded (resident outputs are aligned)
  tmd_frame_out probe;
  static uint32_t dummy[4];
  probe.native = reinterpret_cast<uint8_t*>(dummy);
  probe.row_start = probe.att_count = probe.status = dummy;
  int rc = tmd_validate_frame(h, in, &probe);
  if (rc != TMD_OK) return rc;
  const ReqLayout L = req_layout(*in);
  size_t sb = 0, rb = 0;
  tmd_call_sizes(1, in, nullptr, &sb, &rb);
  // device-resident frames are decoded where they are (no copy)
  cudaPointerAttributes pa;
  bool borrow = false;
  if (cudaPointerGetAttributes(&pa, in->n_unatt) == cudaSuccess)
    borrow = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
  else
    cudaGetLastError();
  const uint64_t bytes = (borrow ? L.total - L.native : L.total) + sb;
  if (bytes > h->mem_budget)
    return tmd_set_error(h, TMD_ERR_BUDGET, "frame needs %llu bytes, the budget is %llu",
                         (unsigned long long)bytes, (unsigned long long)h->mem_budget);
  TmdServer* s = server_of(h);
  if (!s) return TMD_ERR_NOMEM;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Request r;
    r.id = s->next_id++;
    r.src = *in;
    r.borrow = borrow;
    r.bytes = bytes;
    *req_id = r.id;
    s->reqs[r.id] = r;
    s->queue.push_back(r.id);
  }
  s->cv_work.notify_all();
  return TMD_OK;
}

extern "C" int tmd_poll(tmd_handle* h, uint64_t req_id, uint32_t timeout_us, tmd_frame_out* out) {
  if (!h || !out) return TMD_ERR_ARG;
  TmdServer* s = h->server;
  if (!s) return tmd_set_error(h, TMD_ERR_STATE, "unknown request %llu", (unsigned long long)req_id);
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
  for (;;) {
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end())
      return tmd_set_error(h, TMD_ERR_STATE, "unknown request %llu", (unsigned long long)req_id);
    if (it->second.state == ReqState::kDone) {
      *out = it->second.out;
      return TMD_OK;
    }
    if (it->second.state == ReqState::kFailed)
      return tmd_set_error(h, it->second.err, "request %llu failed", (unsigned long long)req_id);
    if (std::chrono::steady_clock::now() >= deadline) return TMD_PENDING;
    s->cv_done.wait_until(lk, deadline);
  }
}

extern "C" int tmd_release(tmd_handle* h, uint64_t req_id) {
  if (!h) return TMD_ERR_ARG;
  TmdServer* s = h->server;
  if (!s) return tmd_set_error(h, TMD_ERR_STATE, "unknown request %llu", (unsigned long long)req_id);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end())
      return tmd_set_error(h, TMD_ERR_STATE, "unknown request %llu", (unsigned long long)req_id);
    Request& r = it->second;
    if (r.state == ReqState::kQueued) {
      for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if (*q == req_id) { s->queue.erase(q); break; }
    } else if (r.state == ReqState::kCopying || r.state == ReqState::kRunning) {
      return tmd_set_error(h, TMD_ERR_STATE, "request %llu is still being decoded",
                           (unsigned long long)req_id);
    } else {
      if (r.mem) {
        cudaSetDevice(h->device);
        cudaFreeAsync(r.mem, s->copy);
        s->used -= r.bytes;
        s->active--;
      }
      if (r.copied) cudaEventDestroy(r.copied);
    }
    s->reqs.erase(it);
  }
  s->cv_work.notify_all();
  return TMD_OK;
}
