// tmd_tune.cu -- tuning parameters and the autotuner.
//
// The parameters only change how the work is laid out (the staging-round
// variant of the track decoder, the store pattern of the record scatter, the
// second stream of the unattached decode, and how many blocks per SM the
// persistent decoders start); every setting produces identical output.  tmd_autotune
// times the decode chain on the caller's frames for each candidate, keeps the
// fastest, and stores it in the autotune cache (a small JSON file keyed by the
// GPU name and SM count) when the handle was created with one.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tmd_api_internal.h"

namespace {

struct Param {
  const char* name;
  int tmd_handle::*field;
  int lo, hi;
};
const Param kParams[] = {
    {"decode_variant", &tmd_handle::tune_decode_variant, 0, 1},
    {"scatter_variant", &tmd_handle::tune_scatter_variant, 0, 1},
    {"overlap", &tmd_handle::tune_overlap, 0, 2},
    {"unatt_variant", &tmd_handle::tune_unatt_variant, 0, 1},
    {"decode_blocks_per_sm", &tmd_handle::tune_decode_bps, 0, 64},
    {"unatt_blocks_per_sm", &tmd_handle::tune_unatt_bps, 0, 64},
    {"rans_overlap", &tmd_handle::tune_rans_overlap, 0, 1},
    {"coded_overlap", &tmd_handle::tune_coded_overlap, 0, 2},
};

std::string device_key(const tmd_handle* h) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, h->device) != cudaSuccess) return "unknown";
  char buf[320];
  snprintf(buf, sizeof buf, "%s|%d", p.name, h->sms);
  return buf;
}

}  // namespace

extern "C" int tmd_tune_set(tmd_handle* h, const char* key, int value) {
  if (!h || !key) return TMD_ERR_ARG;
  for (const Param& p : kParams) {
    if (strcmp(p.name, key) == 0) {
      if (value < p.lo || value > p.hi)
        return tmd_set_error(h, TMD_ERR_ARG, "%s must be in [%d, %d]", key, p.lo, p.hi);
      h->*(p.field) = value;
      return TMD_OK;
    }
  }
  return tmd_set_error(h, TMD_ERR_ARG, "unknown tuning parameter '%s'", key);
}

extern "C" int tmd_tune_get(tmd_handle* h, const char* key, int* value) {
  if (!h || !key || !value) return TMD_ERR_ARG;
  for (const Param& p : kParams) {
    if (strcmp(p.name, key) == 0) {
      *value = h->*(p.field);
      return TMD_OK;
    }
  }
  return tmd_set_error(h, TMD_ERR_ARG, "unknown tuning parameter '%s'", key);
}

void tmd_tune_load(tmd_handle* h) {
  FILE* f = fopen(h->autotune_cache.c_str(), "r");
  if (!f) return;
  char buf[4096];
  const size_t n = fread(buf, 1, sizeof buf - 1, f);
  fclose(f);
  buf[n] = 0;
  const std::string key = "\"" + device_key(h) + "\"";
  const char* at = strstr(buf, key.c_str());
  if (!at) return;
  for (const Param& p : kParams) {
    const std::string pk = std::string("\"") + p.name + "\":";
    const char* q = strstr(at, pk.c_str());
    int v = 0;
    if (q && sscanf(q + pk.size(), " %d", &v) == 1 && v >= p.lo && v <= p.hi) h->*(p.field) = v;
  }
}

static int time_chain(tmd_handle* h, uint32_t n, const tmd_frame_in* in, const tmd_frame_out* out,
                      cudaStream_t st, float* ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return tmd_set_error(h, TMD_ERR_CUDA, "event create");
  int rc = tmd_launch(h, n, in, out, nullptr, nullptr, st);  // warm-up
  const int reps = 3;
  if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventRecord(a, st), "event");
  for (int r = 0; r < reps && rc == TMD_OK; r++) rc = tmd_launch(h, n, in, out, nullptr, nullptr, st);
  if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventRecord(b, st), "event");
  if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventSynchronize(b), "event sync");
  float t = 0.0f;
  if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventElapsedTime(&t, a, b), "elapsed");
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  return rc;
}

extern "C" int tmd_autotune(tmd_handle* h, uint32_t n, const tmd_frame_in* in,
                            const tmd_frame_out* out, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (n == 0 || !in || !out) return tmd_set_error(h, TMD_ERR_ARG, "no frames to tune on");
  for (uint32_t f = 0; f < n; f++) {
    const int rc = tmd_validate_frame(h, &in[f], &out[f]);
    if (rc != TMD_OK) return rc;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool prof = h->prof.on;
  h->prof.on = false;
  // coordinate descent: each parameter in turn, the others at their best
  struct Axis {
    int tmd_handle::*field;
    std::vector<int> values;
  };
  const Axis axes[] = {
      {&tmd_handle::tune_decode_variant, {0, 1}},
      {&tmd_handle::tune_scatter_variant, {0, 1}},
      {&tmd_handle::tune_overlap, {0, 1, 2}},
      {&tmd_handle::tune_unatt_variant, {0, 1}},
      {&tmd_handle::tune_unatt_bps, {0, 1, 2, 3, 4}},
  };
  h->tune_decode_bps = 0;
  float best = 1e30f;
  int rc = time_chain(h, n, in, out, st, &best);
  for (const Axis& ax : axes) {
    int keep = h->*(ax.field);
    for (int v : ax.values) {
      if (rc != TMD_OK) break;
      if (v == keep) continue;
      h->*(ax.field) = v;
      float ms = 0;
      rc = time_chain(h, n, in, out, st, &ms);
      if (rc == TMD_OK && ms < best) { best = ms; keep = v; }
    }
    h->*(ax.field) = keep;
  }
  h->prof.on = prof;
  if (rc != TMD_OK) return rc;
  if (!h->autotune_cache.empty()) {
    FILE* f = fopen(h->autotune_cache.c_str(), "w");
    if (f) {
      fprintf(f, "{\"%s\": {", device_key(h).c_str());
      for (const Param& p : kParams) fprintf(f, "\"%s\": %d, ", p.name, h->*(p.field));
      fprintf(f, "\"chain_ms\": %.4f}}\n", best);
      fclose(f);
    }
  }
  return TMD_OK;
}
