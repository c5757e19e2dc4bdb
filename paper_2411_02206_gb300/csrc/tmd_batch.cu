// tmd_batch.cu -- batched decoding captured in a CUDA graph.
//
// The multi-frame schedule: one launch record covers all frames of the batch,
// every kernel of the chain spans the work items of all frames (the persistent
// decoders pull (frame, warp-task) and (frame, chunk) items from global
// counters), and the chain -- record upload, scratch clear, the kernels on
// their two streams with the event edges between them -- is captured once
// and replayed with one cudaGraphLaunch.  Small frames therefore
// share waves with large ones instead of each paying a launch sequence and a
// tail of its own.
#include <vector>

#include "tmd_api_internal.h"

struct tmd_batch {
  tmd_handle* h = nullptr;
  uint32_t n = 0;
  void* scratch = nullptr;
  void* host_record = nullptr;
  void* dev_record = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t aux = nullptr;  // second branch of the captured chain
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~tmd_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (aux) cudaStreamDestroy(aux);
    for (cudaEvent_t e : {fork, join})
      if (e) cudaEventDestroy(e);
    if (scratch) cudaFree(scratch);
    if (dev_record) cudaFree(dev_record);
    if (host_record) cudaFreeHost(host_record);
  }
};

extern "C" int tmd_batch_create(tmd_handle* h, uint32_t n, const tmd_frame_in* in,
                                const tmd_frame_out* out, tmd_batch** out_batch) {
  if (!h || !out_batch) return TMD_ERR_ARG;
  *out_batch = nullptr;
  if (n == 0 || !in || !out) return tmd_set_error(h, TMD_ERR_ARG, "empty batch");
  for (uint32_t f = 0; f < n; f++) {
    const int rc = tmd_validate_frame(h, &in[f], &out[f]);
    if (rc != TMD_OK) return rc;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return tmd_set_error(h, TMD_ERR_CUDA, "device");
  size_t scratch_bytes = 0, record_bytes = 0;
  tmd_call_sizes(n, in, nullptr, &scratch_bytes, &record_bytes);
  tmd_batch* b = new (std::nothrow) tmd_batch();
  if (!b) return tmd_set_error(h, TMD_ERR_NOMEM, "batch");
  b->h = h;
  b->n = n;
  if (cudaMalloc(&b->scratch, scratch_bytes) != cudaSuccess ||
      cudaMalloc(&b->dev_record, record_bytes) != cudaSuccess ||
      cudaMallocHost(&b->host_record, record_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return tmd_set_error(h, TMD_ERR_NOMEM, "batch allocation (%zu bytes) failed", scratch_bytes);
  }
  int rc = tmd_cuda_check(h, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "stream");
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking), "stream");
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming), "event");
  if (rc != TMD_OK) { delete b; return rc; }
  rc = tmd_cuda_check(h, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal),
                      "begin capture");
  if (rc == TMD_OK) {
    // no timing events inside the graph; the fork/join events become edges
    const ChainStreams cs{b->aux, b->fork, b->join};
    rc = tmd_enqueue(h, n, in, out, nullptr, nullptr, b->scratch, b->host_record, b->dev_record,
                     b->cap, false, &cs);
    const int rc2 = tmd_cuda_check(h, cudaStreamEndCapture(b->cap, &b->graph), "end capture");
    if (rc == TMD_OK) rc = rc2;
  }
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
  if (rc != TMD_OK) {
    delete b;
    return rc;
  }
  *out_batch = b;
  return TMD_OK;
}

extern "C" int tmd_batch_launch(tmd_batch* b, void* stream) {
  if (!b) return TMD_ERR_ARG;
  tmd_handle* h = b->h;
  if (cudaSetDevice(h->device) != cudaSuccess) return tmd_set_error(h, TMD_ERR_CUDA, "device");
  return tmd_cuda_check(h, cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)),
                        "graph launch");
}

extern "C" int tmd_batch_destroy(tmd_batch* b) {
  if (!b) return TMD_ERR_ARG;
  cudaSetDevice(b->h->device);
  cudaDeviceSynchronize();  // a replay may still be running on the caller's stream
  delete b;
  return TMD_OK;
}
