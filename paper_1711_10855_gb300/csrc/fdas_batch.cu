// fdas_batch.cu -- many spectra of uneven lengths in one persistent launch (declared in
// include/fdas.h): the batch object, its CUDA-graph launch and the segment-length autotuner.
//
// A batch holds one template bank for the largest |z| of its spectra (a spectrum with a smaller
// zmax uses the middle rows of the same bank: the templates depend on z only) and a device table
// of per-spectrum descriptors.  One launch of the descriptor-driven kernel correlates every
// spectrum with its templates; the flattened (spectrum, segment group, template) work is split
// into equal contiguous ranges over the SMs, so uneven lengths do not unbalance the grid.
// Segment lengths without that kernel (256, 1024, 4096, 8192) run one single-spectrum launch per
// spectrum instead, in order on the stream (as a CUDA graph of those launches with use_graph).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "fdas.h"
#include "fdas_internal.h"

struct fdas_batch {
  int device = 0, sm_count = 0;
  int count = 0;
  int L = 0, m = 0, h = 0, V = 0, zstep = 1, zmax_bank = 0, Z_bank = 0, G = 0;
  std::vector<int64_t> n_bins;
  std::vector<int> zmax;
  int64_t units = 0;
  float2* d_templates = nullptr;
  double2* d_taps = nullptr;
  float2* d_twist = nullptr;
  int* d_status = nullptr;
  fdas::SpecDesc* d_descs = nullptr;
  fdas::SpecDesc* h_descs = nullptr;   // pinned staging of the descriptor table
  bool built = false;
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // completion of the last work this batch enqueued (fdas_batch_destroy waits on it, not on the
  // whole device)
  cudaEvent_t done = nullptr;
  // per-spectrum launches (G == 0): the pointers the graph was captured with
  std::vector<const float*> cap_specs;
  std::vector<float*> cap_planes;
};

namespace {

thread_local int g_batch_error = FDAS_OK;

void free_batch(fdas_batch* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->done) cudaEventDestroy(b->done);
  cudaFree(b->d_templates);
  cudaFree(b->d_taps);
  cudaFree(b->d_twist);
  cudaFree(b->d_status);
  cudaFree(b->d_descs);
  if (b->h_descs) cudaFreeHost(b->h_descs);
  delete b;
}

// Record the batch's completion event after work enqueued on `st` (not while `st` is being
// captured into a CUDA graph: a captured record is no event the host can wait on).
int note_work(fdas_batch* b, cudaStream_t st, cudaError_t launch) {
  if (launch != cudaSuccess) return FDAS_ERR_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FDAS_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return FDAS_OK;
  return cudaEventRecord(b->done, st) == cudaSuccess ? FDAS_OK : FDAS_ERR_CUDA;
}

fdas::BatchParams batch_params(const fdas_batch* b) {
  fdas::BatchParams q;
  std::memset(&q, 0, sizeof(q));
  q.templates = b->d_templates;
  q.twist = b->d_twist;
  q.status = b->d_status;
  q.descs = b->d_descs;
  q.count = b->count;
  q.units = b->units;
  q.unit_list = nullptr;
  q.V = b->V;
  q.h = b->h;
  return q;
}

// One single-spectrum launch per spectrum (segment lengths without the descriptor-driven
// kernel); spectrum i uses rows z_off_i.. of the shared bank.
cudaError_t launch_per_spectrum(const fdas_batch* b, const float* const* d_spectra, float* const* d_planes,
                                cudaStream_t st) {
  for (int i = 0; i < b->count; ++i) {
    const fdas::SpecDesc& d = b->h_descs[i];
    fdas::ConvParams q;
    std::memset(&q, 0, sizeof(q));
    q.spectrum = reinterpret_cast<const float2*>(d_spectra[i]);
    q.templates = b->d_templates + (size_t)d.z_off * b->L;
    q.twist = b->d_twist;
    q.plane = d_planes[i];
    q.status = b->d_status;
    q.n_bins = d.n_bins;
    q.nseg = d.nseg;
    q.units = 0;
    q.Z = d.Z;
    q.V = b->V;
    q.h = b->h;
    CUtensorMap map;
    if (fdas::encode_spectrum_map(&map, d_spectra[i], d.n_bins, b->L) != FDAS_OK) return cudaErrorInvalidValue;
    const cudaError_t e = fdas::launch_convolve(b->L, &map, q, b->sm_count, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_any(const fdas_batch* b, const float* const* d_spectra, float* const* d_planes,
                       cudaStream_t st) {
  if (b->G == 0) return launch_per_spectrum(b, d_spectra, d_planes, st);
  return fdas::launch_batch(b->L, batch_params(b), b->sm_count, st);
}

}  // namespace

extern "C" {

int fdas_batch_last_error(void) { return g_batch_error; }

fdas_batch* fdas_batch_create(int count, const int64_t* n_bins, const int* zmax, int zstep, int seg_len,
                              int tmpl_len) {
  g_batch_error = FDAS_OK;
  if (count < 1 || count > (1 << 20) || !n_bins || !zmax || zstep < 1) {
    g_batch_error = FDAS_ERR_INVALID;
    return nullptr;
  }
  int zmax_bank = 0;
  for (int i = 0; i < count; ++i) {
    const int rc = fdas::validate_geometry(n_bins[i], zmax[i], zstep, seg_len, tmpl_len);
    if (rc != FDAS_OK) {
      g_batch_error = rc;
      return nullptr;
    }
    if (zmax[i] > zmax_bank) zmax_bank = zmax[i];
  }
  const int G = fdas::batch_segments_per_cta(seg_len);   // 0: one launch per spectrum
  int ndev = 0, dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    g_batch_error = FDAS_ERR_NO_DEVICE;
    return nullptr;
  }
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    g_batch_error = FDAS_ERR_CUDA;
    return nullptr;
  }
  if (major != 10 || minor != 3) {
    g_batch_error = FDAS_ERR_UNSUPPORTED;
    return nullptr;
  }
  fdas_batch* b = new (std::nothrow) fdas_batch();
  if (!b) {
    g_batch_error = FDAS_ERR_ALLOC;
    return nullptr;
  }
  b->device = dev;
  b->sm_count = sms;
  b->count = count;
  b->L = seg_len;
  b->m = tmpl_len;
  b->h = tmpl_len / 2;
  b->V = seg_len - tmpl_len;
  b->zstep = zstep;
  b->zmax_bank = zmax_bank;
  b->Z_bank = 2 * (zmax_bank / zstep) + 1;
  b->G = G;
  b->n_bins.assign(n_bins, n_bins + count);
  b->zmax.assign(zmax, zmax + count);
  const size_t ntap = (size_t)tmpl_len + 1;
  if (cudaMalloc(&b->d_templates, sizeof(float2) * (size_t)b->Z_bank * b->L) != cudaSuccess ||
      cudaMalloc(&b->d_taps, sizeof(double2) * (size_t)b->Z_bank * ntap) != cudaSuccess ||
      cudaMalloc(&b->d_twist, sizeof(float2) * (size_t)b->L) != cudaSuccess ||
      cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_descs, sizeof(fdas::SpecDesc) * (size_t)count) != cudaSuccess ||
      cudaHostAlloc(&b->h_descs, sizeof(fdas::SpecDesc) * (size_t)count, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    g_batch_error = FDAS_ERR_ALLOC;
    return nullptr;
  }
  if (cudaMemsetAsync(b->d_status, 0, sizeof(int), 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
    free_batch(b);
    g_batch_error = FDAS_ERR_CUDA;
    return nullptr;
  }
  // static part of the descriptor table: sizes, template rows and unit ranges
  int64_t base = 0;
  for (int i = 0; i < count; ++i) {
    fdas::SpecDesc& d = b->h_descs[i];
    std::memset(&d, 0, sizeof(d));
    d.n_bins = n_bins[i];
    d.nseg = (n_bins[i] + b->V - 1) / b->V;
    d.ngroups = G > 0 ? (d.nseg + G - 1) / G : d.nseg;
    d.Z = 2 * (zmax[i] / zstep) + 1;
    d.z_off = (zmax_bank - zmax[i]) / zstep;
    d.unit_base = base;
    base += d.ngroups * d.Z;
  }
  b->units = base;
  return b;
}

int fdas_batch_templates_build(fdas_batch* b, fdas_stream_t stream) {
  if (!b) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int rc = note_work(
      b, st, fdas::build_templates_into(b->d_taps, b->d_templates, b->d_twist, b->zmax_bank, b->zstep, b->L, b->m, st));
  if (rc != FDAS_OK) return rc;
  b->built = true;
  return FDAS_OK;
}

int fdas_batch_convolve_power(fdas_batch* b, const float* const* d_spectra, float* const* d_planes, int use_graph,
                              fdas_stream_t stream) {
  if (!b || !d_spectra || !d_planes) return FDAS_ERR_INVALID;
  if (!b->built) return FDAS_ERR_NOT_BUILT;
  for (int i = 0; i < b->count; ++i) {
    if (!d_spectra[i] || !d_planes[i]) return FDAS_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_spectra[i]) & 15u) || (reinterpret_cast<uintptr_t>(d_planes[i]) & 15u))
      return FDAS_ERR_ALIGN;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the pinned staging may still feed a previous call's copy: wait for it on this stream's order
  if (cudaStreamSynchronize(st) != cudaSuccess) return FDAS_ERR_CUDA;
  for (int i = 0; i < b->count; ++i) {
    b->h_descs[i].spec = reinterpret_cast<const float2*>(d_spectra[i]);
    b->h_descs[i].plane = d_planes[i];
  }
  if (b->G > 0 && cudaMemcpyAsync(b->d_descs, b->h_descs, sizeof(fdas::SpecDesc) * (size_t)b->count,
                                   cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FDAS_ERR_CUDA;
  if (!use_graph) return note_work(b, st, launch_any(b, d_spectra, d_planes, st));
  if (b->G == 0 && b->graph_exec &&
      (!std::equal(b->cap_specs.begin(), b->cap_specs.end(), d_spectra) ||
       !std::equal(b->cap_planes.begin(), b->cap_planes.end(), d_planes))) {
    // per-spectrum launches hold the pointers as parameters: new pointers need a new graph
    cudaGraphExecDestroy(b->graph_exec);
    cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
  }
  if (!b->graph_exec) {
    // capture once; the persistent launch's parameters (table address, sizes) never change
    if (cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return FDAS_ERR_CUDA;
    const cudaError_t le = launch_any(b, d_spectra, d_planes, b->capture_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->capture_stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return FDAS_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&b->graph_exec, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      b->graph_exec = nullptr;
      return FDAS_ERR_CUDA;
    }
    b->graph = g;
    b->cap_specs.assign(d_spectra, d_spectra + b->count);
    b->cap_planes.assign(d_planes, d_planes + b->count);
  }
  return note_work(b, st, cudaGraphLaunch(b->graph_exec, st));
}

int fdas_batch_check(fdas_batch* b, fdas_stream_t stream) {
  if (!b) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int status = 0;
  if (cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FDAS_ERR_CUDA;
  if (status != 0) {
    if (cudaMemsetAsync(b->d_status, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      return FDAS_ERR_CUDA;
    return FDAS_ERR_TIMEOUT;
  }
  return FDAS_OK;
}

int fdas_batch_destroy(fdas_batch* b) {
  if (!b) return FDAS_OK;
  if (b->done) cudaEventSynchronize(b->done);   // the batch's last enqueued work, not the whole device
  free_batch(b);
  return FDAS_OK;
}

int fdas_batch_info(const fdas_batch* b, int* seg_len, int* z_bank, int64_t* units, int* segments_per_cta) {
  if (!b) return FDAS_ERR_INVALID;
  if (seg_len) *seg_len = b->L;
  if (z_bank) *z_bank = b->Z_bank;
  if (units) *units = b->units;
  if (segments_per_cta) *segments_per_cta = b->G;
  return FDAS_OK;
}

int fdas_batch_autotune(int count, const int64_t* n_bins, const int* zmax, int zstep, int tmpl_len,
                        const int* seg_len_candidates, int n_candidates, const float* const* d_spectra,
                        float* const* d_planes, fdas_stream_t stream, int* best_seg_len, float* ms_out) {
  if (!seg_len_candidates || n_candidates < 1 || !best_seg_len) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float best = -1.f;
  *best_seg_len = 0;
  for (int c = 0; c < n_candidates; ++c) {
    if (ms_out) ms_out[c] = -1.f;
    fdas_batch* b = fdas_batch_create(count, n_bins, zmax, zstep, seg_len_candidates[c], tmpl_len);
    if (!b) continue;   // this segment length cannot serve the batch (tmpl_len > L/2)
    int rc = fdas_batch_templates_build(b, stream);
    if (rc == FDAS_OK) rc = fdas_batch_convolve_power(b, d_spectra, d_planes, 0, stream);   // warm-up
    float ms = 0.f;
    if (rc == FDAS_OK) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      const int reps = 3;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == FDAS_OK; ++r)
        rc = launch_any(b, d_spectra, d_planes, st) == cudaSuccess ? FDAS_OK : FDAS_ERR_CUDA;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = FDAS_ERR_CUDA;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    if (rc == FDAS_OK) rc = fdas_batch_check(b, stream);
    fdas_batch_destroy(b);
    if (rc != FDAS_OK) return rc;
    if (ms_out) ms_out[c] = ms;
    if (best < 0.f || ms < best) {
      best = ms;
      *best_seg_len = seg_len_candidates[c];
    }
  }
  return *best_seg_len ? FDAS_OK : FDAS_ERR_INVALID;
}

}  // extern "C"
