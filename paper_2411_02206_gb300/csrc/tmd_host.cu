// tmd_host.cu -- decoding from host buffers.
//
// tmd_decode_frame_host: one cudaMemcpyAsync per input stream into
// handle-owned device memory, the decode chain, and the copies of the native
// list, row offsets and status back to the host buffers; synchronous.
//
// tmd_decode_host_stream: the same for a sequence of frames, pipelined the
// way Sec. 4 of arXiv:2411.02206 runs several decoding instances on streams
// to hide the transfers (Fig. 2): kPipeSlots device slots; frame i's inputs
// go up on a host-to-device copy stream while earlier frames are decoded on
// the compute stream and their results come back on a device-to-host copy
// stream.  A slot is refilled only after the results of the frame that last
// used it have left; with three slots the upload of frame i waits for the
// download of frame i - 3, so both copy directions stay busy.
//
// tmd_decode_coded_host_stream runs the same pipeline for coded frames: one
// upload of the coded bytes per frame, then entropy decoding and track-model
// decoding on the compute stream.
#include <algorithm>
#include <cstring>

#include "tmd_api_internal.h"

namespace {

size_t up(size_t x) { return (x + 255) / 256 * 256; }

struct Field {
  const void* src;
  size_t bytes;
  const void** dst;
};

// The input streams of a frame (host pointers in `in`, device pointers to be
// set in `d`), in tmd_frame_in order.
int input_fields(const tmd_frame_in* in, tmd_frame_in* d, Field (&fs)[23]) {
  const size_t nt = in->n_tracks, na = in->n_attached, nu = in->n_unattached;
  *d = *in;
  const Field f[23] = {
      {in->qpt, nt, (const void**)&d->qpt}, {in->row, nt, (const void**)&d->row},
      {in->slice, nt, (const void**)&d->slice}, {in->pad, 2 * nt, (const void**)&d->pad},
      {in->time, 4 * nt, (const void**)&d->time}, {in->ncl, 2 * nt, (const void**)&d->ncl},
      {in->qtot_a, 2 * na, (const void**)&d->qtot_a}, {in->qmax_a, 2 * na, (const void**)&d->qmax_a},
      {in->flags_a, na, (const void**)&d->flags_a},
      {in->sigma_pad_a, na, (const void**)&d->sigma_pad_a},
      {in->sigma_time_a, na, (const void**)&d->sigma_time_a},
      {in->row_diff, na - nt, (const void**)&d->row_diff},
      {in->slice_leg_diff, na - nt, (const void**)&d->slice_leg_diff},
      {in->pad_res, 2 * (na - nt), (const void**)&d->pad_res},
      {in->time_res, 4 * (na - nt), (const void**)&d->time_res},
      {in->n_unatt, 4 * (size_t)TMD_NBIN, (const void**)&d->n_unatt},
      {in->pad_diff_u, 2 * nu, (const void**)&d->pad_diff_u},
      {in->time_diff_u, 4 * nu, (const void**)&d->time_diff_u},
      {in->qtot_u, 2 * nu, (const void**)&d->qtot_u}, {in->qmax_u, 2 * nu, (const void**)&d->qmax_u},
      {in->flags_u, nu, (const void**)&d->flags_u},
      {in->sigma_pad_u, nu, (const void**)&d->sigma_pad_u},
      {in->sigma_time_u, nu, (const void**)&d->sigma_time_u}};
  for (int i = 0; i < 23; i++) fs[i] = f[i];
  return na < nt ? TMD_ERR_ARG : TMD_OK;
}

// Device bytes of one frame: inputs, then native, row_start, att_count, status.
size_t frame_bytes(const tmd_frame_in* in) {
  tmd_frame_in d;
  Field fs[23];
  input_fields(in, &d, fs);
  size_t need = 0;
  for (const Field& f : fs) need += up(f.bytes);
  const size_t n = (size_t)in->n_attached + in->n_unattached;
  return need + up(n * TMD_REC_BYTES) + up(4 * (TMD_NBIN + 1)) + up(4 * TMD_NBIN) + 256;
}

// Enqueue the input copies of `in` into device memory at p (on st) and fill
// the device-side descriptors.
int place_frame(tmd_handle* h, const tmd_frame_in* in, char* p, cudaStream_t st,
                tmd_frame_in* d, tmd_frame_out* o) {
  Field fs[23];
  if (input_fields(in, d, fs) != TMD_OK)
    return tmd_set_error(h, TMD_ERR_ARG, "n_attached < n_tracks");
  for (const Field& f : fs) {
    *f.dst = f.bytes ? p : nullptr;
    if (f.bytes) {
      if (!f.src) return tmd_set_error(h, TMD_ERR_ARG, "host input array is NULL");
      const cudaError_t e = cudaMemcpyAsync(p, f.src, f.bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return tmd_cuda_check(h, e, "H2D copy");
    }
    p += up(f.bytes);
  }
  const size_t native_bytes = ((size_t)in->n_attached + in->n_unattached) * TMD_REC_BYTES;
  o->native = reinterpret_cast<uint8_t*>(p);
  p += up(native_bytes);
  o->row_start = reinterpret_cast<uint32_t*>(p);
  p += up(4 * (TMD_NBIN + 1));
  o->att_count = reinterpret_cast<uint32_t*>(p);
  p += up(4 * TMD_NBIN);
  o->status = reinterpret_cast<uint32_t*>(p);
  return tmd_validate_frame(h, d, o);
}

// Enqueue the result copies of a decoded frame back to the host buffers.
int fetch_frame(tmd_handle* h, const tmd_frame_in* in, const tmd_frame_out* o,
                const tmd_frame_out* out, cudaStream_t st) {
  const size_t native_bytes = ((size_t)in->n_attached + in->n_unattached) * TMD_REC_BYTES;
  struct Back { void* dst; const void* src; size_t bytes; };
  const Back bs[] = {{out->native, o->native, native_bytes},
                     {out->row_start, o->row_start, 4 * (TMD_NBIN + 1)},
                     {out->att_count, o->att_count, 4 * (size_t)TMD_NBIN},
                     {out->status, o->status, 4}};
  for (const Back& b : bs) {
    if (!b.dst || !b.bytes) continue;
    const cudaError_t e = cudaMemcpyAsync(b.dst, b.src, b.bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return tmd_cuda_check(h, e, "D2H copy");
  }
  return TMD_OK;
}

int grow(tmd_handle* h, void** buf, size_t* have, size_t need) {
  if (need <= *have) return TMD_OK;
  if (*buf) {
    cudaDeviceSynchronize();
    cudaFree(*buf);
  }
  *buf = nullptr;
  *have = 0;
  if (cudaMalloc(buf, need) != cudaSuccess) {
    cudaGetLastError();
    return tmd_set_error(h, TMD_ERR_NOMEM, "staging allocation of %zu bytes failed", need);
  }
  *have = need;
  return TMD_OK;
}

}  // namespace

extern "C" int tmd_decode_frame_host(tmd_handle* h, const tmd_frame_in* in,
                                     const tmd_frame_out* out, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (!in || !out) return tmd_set_error(h, TMD_ERR_ARG, "null descriptor");
  if (in->n_attached < in->n_tracks) return tmd_set_error(h, TMD_ERR_ARG, "n_attached < n_tracks");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaSetDevice(h->device) != cudaSuccess) return tmd_set_error(h, TMD_ERR_CUDA, "cudaSetDevice");
  int rc = grow(h, &h->stage, &h->stage_bytes, frame_bytes(in));
  if (rc != TMD_OK) return rc;
  tmd_frame_in d;
  tmd_frame_out o;
  if ((rc = place_frame(h, in, static_cast<char*>(h->stage), st, &d, &o)) != TMD_OK) return rc;
  if ((rc = tmd_launch(h, 1, &d, &o, nullptr, nullptr, st)) != TMD_OK) return rc;
  if ((rc = fetch_frame(h, in, &o, out, st)) != TMD_OK) return rc;
  return tmd_cuda_check(h, cudaStreamSynchronize(st), "stream synchronize");
}

namespace {

// Copy streams and slot events of the host pipelines, made on first use.
int pipe_streams(tmd_handle* h) {
  if (h->h2d) return TMD_OK;
  int rc = TMD_OK;
  if ((rc = tmd_cuda_check(h, cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking),
                           "stream")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking),
                           "stream")) != TMD_OK)
    return rc;
  for (int s = 0; s < tmd_handle::kPipeSlots; s++)
    for (cudaEvent_t* e : {&h->pipe_in[s], &h->pipe_dec[s], &h->pipe_out[s]})
      if ((rc = tmd_cuda_check(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming),
                               "event")) != TMD_OK)
        return rc;
  return TMD_OK;
}

// Device bytes of one coded frame's slot: the coded bytes, then the outputs.
size_t coded_slot_bytes(const tmd_coded_frame& c) {
  const size_t n = (size_t)c.n_attached + c.n_unattached;
  return up(c.bytes) + up(n * TMD_REC_BYTES) + up(4 * (TMD_NBIN + 1)) + up(4 * TMD_NBIN) + 256;
}

}  // namespace

extern "C" int tmd_decode_coded_host_stream(tmd_handle* h, uint32_t n, const tmd_coded_frame* in,
                                            const tmd_frame_out* out, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (n == 0) return TMD_OK;
  if (!in || !out) return tmd_set_error(h, TMD_ERR_ARG, "null frame arrays");
  for (uint32_t i = 0; i < n; i++) {
    if (in[i].n_attached < in[i].n_tracks)
      return tmd_set_error(h, TMD_ERR_ARG, "frame %u: n_attached < n_tracks", i);
    if (!in[i].data || in[i].bytes < TMD_RANS_HEADER_BYTES)
      return tmd_set_error(h, TMD_ERR_ARG, "frame %u: no coded frame", i);
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return tmd_set_error(h, TMD_ERR_CUDA, "cudaSetDevice");
  cudaStream_t comp = static_cast<cudaStream_t>(stream);
  int rc = pipe_streams(h);
  if (rc != TMD_OK) return rc;
  size_t need = 0;
  for (uint32_t i = 0; i < n; i++) need = std::max(need, coded_slot_bytes(in[i]));
  const int slots = (int)std::min<uint32_t>(n, tmd_handle::kPipeSlots);
  for (int s = 0; s < slots; s++)
    if ((rc = grow(h, &h->pipe_buf[s], &h->pipe_bytes[s], need)) != TMD_OK) return rc;
  if ((rc = tmd_cuda_check(h, cudaEventRecord(h->pipe_dec[0], comp), "event")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->h2d, h->pipe_dec[0], 0), "wait")) != TMD_OK)
    return rc;
  for (uint32_t i = 0; i < n && rc == TMD_OK; i++) {
    const int s = (int)(i % slots);
    const tmd_coded_frame& c = in[i];
    const size_t nrec = (size_t)c.n_attached + c.n_unattached;
    char* p = static_cast<char*>(h->pipe_buf[s]);
    tmd_frame_out o;
    o.native = reinterpret_cast<uint8_t*>(p + up(c.bytes));
    o.row_start = reinterpret_cast<uint32_t*>(p + up(c.bytes) + up(nrec * TMD_REC_BYTES));
    o.att_count = o.row_start + up(4 * (TMD_NBIN + 1)) / 4;
    o.status = o.att_count + up(4 * TMD_NBIN) / 4;
    tmd_frame_in counts{};
    counts.n_tracks = c.n_tracks;
    counts.n_attached = c.n_attached;
    counts.n_unattached = c.n_unattached;
    if (i >= (uint32_t)slots)
      rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->h2d, h->pipe_out[s], 0), "wait");
    if (rc == TMD_OK)
      rc = tmd_cuda_check(h, cudaMemcpyAsync(p, c.data, c.bytes, cudaMemcpyHostToDevice, h->h2d),
                          "H2D copy");
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventRecord(h->pipe_in[s], h->h2d), "event");
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaStreamWaitEvent(comp, h->pipe_in[s], 0), "wait");
    if (rc == TMD_OK)
      rc = tmd_decode_coded_frame(h, p, c.bytes, c.n_tracks, c.n_attached, c.n_unattached, &o,
                                  comp);
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventRecord(h->pipe_dec[s], comp), "event");
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->d2h, h->pipe_dec[s], 0), "wait");
    if (rc == TMD_OK) rc = fetch_frame(h, &counts, &o, &out[i], h->d2h);
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventRecord(h->pipe_out[s], h->d2h), "event");
  }
  const int rc2 = tmd_cuda_check(h, cudaStreamSynchronize(h->d2h), "stream synchronize");
  const int rc3 = tmd_cuda_check(h, cudaStreamSynchronize(comp), "stream synchronize");
  return rc != TMD_OK ? rc : (rc2 != TMD_OK ? rc2 : rc3);
}

extern "C" int tmd_decode_host_stream(tmd_handle* h, uint32_t n, const tmd_frame_in* in,
                                      const tmd_frame_out* out, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (n == 0) return TMD_OK;
  if (!in || !out) return tmd_set_error(h, TMD_ERR_ARG, "null frame arrays");
  for (uint32_t i = 0; i < n; i++)
    if (in[i].n_attached < in[i].n_tracks)
      return tmd_set_error(h, TMD_ERR_ARG, "frame %u: n_attached < n_tracks", i);
  if (cudaSetDevice(h->device) != cudaSuccess) return tmd_set_error(h, TMD_ERR_CUDA, "cudaSetDevice");
  cudaStream_t comp = static_cast<cudaStream_t>(stream);
  int rc = pipe_streams(h);
  if (rc != TMD_OK) return rc;
  size_t need = 0;
  for (uint32_t i = 0; i < n; i++) need = std::max(need, frame_bytes(&in[i]));
  const int slots = (int)std::min<uint32_t>(n, tmd_handle::kPipeSlots);
  for (int s = 0; s < slots; s++)
    if ((rc = grow(h, &h->pipe_buf[s], &h->pipe_bytes[s], need)) != TMD_OK) return rc;
  // the caller's stream sees the slots only after earlier work on it
  if ((rc = tmd_cuda_check(h, cudaEventRecord(h->pipe_dec[0], comp), "event")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->h2d, h->pipe_dec[0], 0), "wait")) != TMD_OK)
    return rc;
  for (uint32_t i = 0; i < n && rc == TMD_OK; i++) {
    const int s = (int)(i % slots);
    tmd_frame_in d;
    tmd_frame_out o;
    if (i >= (uint32_t)slots)
      rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->h2d, h->pipe_out[s], 0), "wait");
    if (rc == TMD_OK)
      rc = place_frame(h, &in[i], static_cast<char*>(h->pipe_buf[s]), h->h2d, &d, &o);
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventRecord(h->pipe_in[s], h->h2d), "event");
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaStreamWaitEvent(comp, h->pipe_in[s], 0), "wait");
    if (rc == TMD_OK) rc = tmd_launch(h, 1, &d, &o, nullptr, nullptr, comp);
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventRecord(h->pipe_dec[s], comp), "event");
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->d2h, h->pipe_dec[s], 0), "wait");
    if (rc == TMD_OK) rc = fetch_frame(h, &in[i], &o, &out[i], h->d2h);
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaEventRecord(h->pipe_out[s], h->d2h), "event");
  }
  const int rc2 = tmd_cuda_check(h, cudaStreamSynchronize(h->d2h), "stream synchronize");
  const int rc3 = tmd_cuda_check(h, cudaStreamSynchronize(comp), "stream synchronize");
  return rc != TMD_OK ? rc : (rc2 != TMD_OK ? rc2 : rc3);
}
