// tmd_host.cu -- end-to-end decode from host buffers: one cudaMemcpyAsync per
// input stream into handle-owned device memory, the decode chain, and the
// copies of the native list, row offsets and status back to the host.
#include <cstring>

#include "tmd_api_internal.h"

namespace {
size_t up(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

extern "C" int tmd_decode_frame_host(tmd_handle* h, const tmd_frame_in* in,
                                     const tmd_frame_out* out, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (!in || !out) return tmd_set_error(h, TMD_ERR_ARG, "null descriptor");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nt = in->n_tracks, na = in->n_attached, nu = in->n_unattached;
  if (na < nt) return tmd_set_error(h, TMD_ERR_ARG, "n_attached < n_tracks");
  struct Field { const void* src; size_t bytes; const void** dst; };
  tmd_frame_in d = *in;
  Field fs[] = {
      {in->qpt, nt, (const void**)&d.qpt}, {in->row, nt, (const void**)&d.row},
      {in->slice, nt, (const void**)&d.slice}, {in->pad, 2 * nt, (const void**)&d.pad},
      {in->time, 4 * nt, (const void**)&d.time}, {in->ncl, 2 * nt, (const void**)&d.ncl},
      {in->qtot_a, 2 * na, (const void**)&d.qtot_a}, {in->qmax_a, 2 * na, (const void**)&d.qmax_a},
      {in->flags_a, na, (const void**)&d.flags_a}, {in->sigma_pad_a, na, (const void**)&d.sigma_pad_a},
      {in->sigma_time_a, na, (const void**)&d.sigma_time_a},
      {in->row_diff, na - nt, (const void**)&d.row_diff},
      {in->slice_leg_diff, na - nt, (const void**)&d.slice_leg_diff},
      {in->pad_res, 2 * (na - nt), (const void**)&d.pad_res},
      {in->time_res, 4 * (na - nt), (const void**)&d.time_res},
      {in->n_unatt, 4 * (size_t)TMD_NBIN, (const void**)&d.n_unatt},
      {in->pad_diff_u, 2 * nu, (const void**)&d.pad_diff_u},
      {in->time_diff_u, 4 * nu, (const void**)&d.time_diff_u},
      {in->qtot_u, 2 * nu, (const void**)&d.qtot_u}, {in->qmax_u, 2 * nu, (const void**)&d.qmax_u},
      {in->flags_u, nu, (const void**)&d.flags_u}, {in->sigma_pad_u, nu, (const void**)&d.sigma_pad_u},
      {in->sigma_time_u, nu, (const void**)&d.sigma_time_u}};
  size_t need = 0;
  for (const Field& f : fs) need += up(f.bytes);
  const size_t native_bytes = (na + nu) * TMD_REC_BYTES;
  need += up(native_bytes) + up(4 * (TMD_NBIN + 1)) + up(4 * TMD_NBIN) + 256;
  if (cudaSetDevice(h->device) != cudaSuccess) return tmd_set_error(h, TMD_ERR_CUDA, "cudaSetDevice");
  if (need > h->stage_bytes) {
    if (h->stage) {
      cudaDeviceSynchronize();
      cudaFree(h->stage);
    }
    h->stage = nullptr;
    h->stage_bytes = 0;
    if (cudaMalloc(&h->stage, need) != cudaSuccess) {
      cudaGetLastError();
      return tmd_set_error(h, TMD_ERR_NOMEM, "staging allocation of %zu bytes failed", need);
    }
    h->stage_bytes = need;
  }
  char* p = static_cast<char*>(h->stage);
  for (const Field& f : fs) {
    *f.dst = f.bytes ? p : nullptr;
    if (f.bytes) {
      if (!f.src) return tmd_set_error(h, TMD_ERR_ARG, "host input array is NULL");
      const cudaError_t e = cudaMemcpyAsync(p, f.src, f.bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return tmd_cuda_check(h, e, "H2D copy");
    }
    p += up(f.bytes);
  }
  tmd_frame_out o;
  o.native = reinterpret_cast<uint8_t*>(p);
  p += up(native_bytes);
  o.row_start = reinterpret_cast<uint32_t*>(p);
  p += up(4 * (TMD_NBIN + 1));
  o.att_count = reinterpret_cast<uint32_t*>(p);
  p += up(4 * TMD_NBIN);
  o.status = reinterpret_cast<uint32_t*>(p);
  int rc = tmd_validate_frame(h, &d, &o);
  if (rc != TMD_OK) return rc;
  rc = tmd_launch(h, 1, &d, &o, nullptr, nullptr, st);
  if (rc != TMD_OK) return rc;
  struct Back { void* dst; const void* src; size_t bytes; };
  const Back bs[] = {{out->native, o.native, native_bytes},
                     {out->row_start, o.row_start, 4 * (TMD_NBIN + 1)},
                     {out->att_count, o.att_count, 4 * (size_t)TMD_NBIN},
                     {out->status, o.status, 4}};
  for (const Back& b : bs) {
    if (!b.dst || !b.bytes) continue;
    const cudaError_t e = cudaMemcpyAsync(b.dst, b.src, b.bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return tmd_cuda_check(h, e, "D2H copy");
  }
  return tmd_cuda_check(h, cudaStreamSynchronize(st), "stream synchronize");
}
