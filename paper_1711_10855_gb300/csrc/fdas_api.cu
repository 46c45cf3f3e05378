// fdas_api.cu -- the C ABI of libfdas (declared in include/fdas.h): plan life cycle, argument
// validation, the FP64 template-bank build (step a1) and the launch of the fused kernel.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include <cuda.h>
#include <cuda_runtime.h>

#include "fdas.h"
#include "fdas_device.cuh"
#include "fdas_internal.h"

struct fdas_plan {
  int device = 0;
  int sm_count = 0;
  int64_t n_bins = 0;
  int zmax = 0, zstep = 1, L = 0, m = 0, h = 0, V = 0, Z = 0;
  int64_t nseg = 0;
  int n1 = 0;                        // lanes per transform group for this L
  float2* d_templates = nullptr;     // Z x L complex64, IFFT first-pass layout
  double2* d_taps = nullptr;         // Z x (m+1) complex128 normalised taps
  float2* d_twist = nullptr;         // L complex64 inter-pass twiddles, same layout
  int* d_status = nullptr;
  bool built = false;
  const void* map_ptr = nullptr;     // spectrum pointer the cached tensor map describes
  CUtensorMap map;
  // tensor-core variant (fdas_convolve_power_tc), allocated on its first call
  float2* tc_bank = nullptr;         // Z x L natural-order template spectra
  float2* tc_seg = nullptr;          // nseg x L forward segment spectra of the current call
  unsigned char* tc_mats = nullptr;  // DFT matrices, BF16 then FP16
  unsigned* tc_tmax = nullptr;
  bool tc_ready = false;
  // completion of the last work this plan enqueued (fdas_destroy and the introspection calls wait
  // on it instead of on the whole device)
  cudaEvent_t done = nullptr;
};

namespace {

thread_local int g_last_error = FDAS_OK;

constexpr int kGLPoints = 16;
__constant__ double c_gl_x[kGLPoints];   // Gauss-Legendre nodes on [-1, 1]
__constant__ double c_gl_w[kGLPoints];   // and weights

// Gauss-Legendre nodes and weights by Newton iteration on the Legendre polynomial P_n, using
// the three-term recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1} and
// P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).
void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// The quadrature rule, computed once per process (a function-local static is initialised
// exactly once even when several host threads build plans at the same time).
struct GLTable {
  double x[kGLPoints], w[kGLPoints];
  GLTable() { gauss_legendre(kGLPoints, x, w); }
};
const GLTable& gl_table() {
  static const GLTable table;
  return table;
}

// a1, part 1: raw response H_q(z) = int_0^1 exp(i pi (z u^2 - (z+2q) u)) du by composite
// 16-point Gauss-Legendre quadrature (panels short enough that the phase turns by at most
// ~4 rad per panel), then normalisation to unit L2 norm over q = -h..h.  One block per z.
__global__ void taps_kernel(double2* taps, int zmax, int zstep, int h) {
  const int zi = blockIdx.x;
  const double z = (double)(-zmax + zi * zstep);
  const int ntap = 2 * h + 1;
  double2* row = taps + (size_t)zi * ntap;
  double part = 0.0;
  for (int j = threadIdx.x; j < ntap; j += blockDim.x) {
    const double q = (double)(j - h);
    const double b = z + 2.0 * q;
    const int panels = (int)ceil(3.14159265358979323846 * (fabs(z) + 2.0 * fabs(q) + 1.0) / 4.0) + 1;
    const double width = 1.0 / panels;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < panels; ++k) {
      const double mid = (k + 0.5) * width;
      double pr = 0.0, pi = 0.0;
#pragma unroll
      for (int g = 0; g < kGLPoints; ++g) {
        const double u = mid + 0.5 * width * c_gl_x[g];
        double sn, cs;
        sincospi(z * u * u - b * u, &sn, &cs);
        pr += c_gl_w[g] * cs;
        pi += c_gl_w[g] * sn;
      }
      re += pr;
      im += pi;
    }
    re *= 0.5 * width;
    im *= 0.5 * width;
    row[j] = make_double2(re, im);
    part += re * re + im * im;
  }
  __shared__ double red[256];
  red[threadIdx.x] = part;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double scale = 1.0 / sqrt(red[0]);
  for (int j = threadIdx.x; j < ntap; j += blockDim.x) {
    const double2 v = row[j];
    row[j] = make_double2(v.x * scale, v.y * scale);
  }
}

// Float offset of the real part of element k in the pair-major structure-of-arrays layout
// (lane k1 = k % n1, k2 = k / n1; pair p = k2/2 of lane k1 is the float4 at p*n1 + k1 holding
// re(2p), re(2p+1), im(2p), im(2p+1)); the imaginary part is 2 floats further.  n1 = 0 is the
// interleaved natural order, where the imaginary part is the next float.
__host__ __device__ __forceinline__ int pair_layout_re(int k, int n1) {
  if (n1 == 0) return 2 * k;   // natural order (L >= 4096)
  const int k1 = k % n1, k2 = k / n1;
  return ((k2 >> 1) * n1 + k1) * 4 + (k2 & 1);
}

// a1, part 2: T_z[k] = (1/L) sum_{j=0}^{m} conj(Hn_{j-h}) exp(+i 2pi k j / L) in FP64 (the
// conjugated template placed at circular index q + h, so that the correlation's valid outputs
// are the first V of each segment), rounded to complex64 and stored in the kernel layout.
// grid (L/256, Z), 256 threads; dynamic shared memory L double2 of exp(+i 2pi j / L).
__global__ void spectra_kernel(const double2* taps, float2* templates, int L, int h, int n1) {
  extern __shared__ double2 e_tab[];
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)j / (double)L, &sn, &cs);
    e_tab[j] = make_double2(cs, sn);
  }
  __syncthreads();
  const int zi = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  const int ntap = 2 * h + 1;
  const double2* row = taps + (size_t)zi * ntap;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < ntap; ++j) {
    const double2 hq = row[j];
    const double2 e = e_tab[(int)(((long long)k * j) % L)];
    re += hq.x * e.x + hq.y * e.y;   // Re(conj(h) e)
    im += hq.x * e.y - hq.y * e.x;   // Im(conj(h) e)
  }
  float* dst = reinterpret_cast<float*>(templates + (size_t)zi * L);
  const int off = pair_layout_re(k, n1);
  dst[off] = (float)(re / L);
  dst[off + (n1 ? 2 : 1)] = (float)(im / L);
}

// Inter-pass twiddles exp(+i 2pi n2 k1 / L), n2 < N2 = L/n1, k1 < n1: lane k1's pair j holds
// n2 = j and n2 = j + N2/2 (float4 at j*n1 + k1: re, re, im, im).  n1 = 0 (L >= 4096): the
// natural table exp(-2 pi i t / L).
__global__ void twist_kernel(float2* tw, int L, int n1) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L) return;
  if (n1 == 0) {   // L >= 4096: W[t] = exp(-2 pi i t / L) for the Stockham passes
    double sn, cs;
    sincospi(2.0 * (double)idx / (double)L, &sn, &cs);
    tw[idx] = make_float2((float)cs, (float)-sn);
    return;
  }
  const int k1 = idx % n1, n2 = idx / n1;
  const int h2 = L / n1 / 2;
  double sn, cs;
  sincospi(2.0 * (double)(((long long)n2 * k1) % L) / (double)L, &sn, &cs);
  float* dst = reinterpret_cast<float*>(tw);
  const int off = ((n2 % h2) * n1 + k1) * 4 + n2 / h2;
  dst[off] = (float)cs;
  dst[off + 2] = (float)sn;
}

// Failure-detection self test: one thread waits, with the given bound, on an mbarrier whose
// phase nothing completes, and records the timeout in the status word exactly as the fused
// kernel does.  The wait ends by itself; the context stays usable.
__global__ void wait_selftest_kernel(int* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  fdas::mbar_init(&bar, 1);
  fdas::fence_barrier_init();
  if (!fdas::mbar_wait(&bar, 0, limit_ns)) atomicOr(status, fdas::kStatusTimeout);
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

int validate(int64_t n_bins, int zmax, int zstep, int seg_len, int tmpl_len) {
  if (n_bins < 4 || n_bins % 4 != 0 || n_bins > (int64_t(1) << 30)) return FDAS_ERR_INVALID;
  if (zstep < 1 || zmax < 0 || zmax % zstep != 0) return FDAS_ERR_INVALID;
  if (2 * (int64_t)(zmax / zstep) + 1 > 65535) return FDAS_ERR_INVALID;
  if (!is_pow2(seg_len) || seg_len < FDAS_MIN_SEG_LEN || seg_len > FDAS_MAX_SEG_LEN) return FDAS_ERR_INVALID;
  if (tmpl_len < 4 || tmpl_len % 4 != 0 || tmpl_len > seg_len / 2) return FDAS_ERR_INVALID;
  return FDAS_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn lookup_encode_fn() {
  void* ptr = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<EncodeTiledFn>(ptr);
}
EncodeTiledFn get_encode_fn() {
  static const EncodeTiledFn fn = lookup_encode_fn();   // looked up once, thread-safe
  return fn;
}

// Record the plan's completion event after work enqueued on `st` (skipped while the stream is
// being captured into a CUDA graph: a captured record is not an event the host can wait on).
int note_work(fdas_plan* p, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FDAS_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return FDAS_OK;
  return cudaEventRecord(p->done, st) == cudaSuccess ? FDAS_OK : FDAS_ERR_CUDA;
}
int enqueued(fdas_plan* p, cudaStream_t st, cudaError_t launch) {
  if (launch != cudaSuccess) return FDAS_ERR_CUDA;
  return note_work(p, st);
}

// 1-D tensor map over the spectrum: n_bins elements of 8 bytes, box of min(L, 256) elements,
// zero fill outside [0, n_bins).
int make_spectrum_map(fdas_plan* p, const void* d_spectrum) {
  if (p->L >= 4096) return FDAS_OK;   // the L >= 4096 kernels read the spectrum directly
  if (p->map_ptr == d_spectrum) return FDAS_OK;
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return FDAS_ERR_CUDA;
  cuuint64_t gdim[1] = {(cuuint64_t)p->n_bins};
  cuuint64_t gstride[1] = {0};
  cuuint32_t box[1] = {(cuuint32_t)(p->L < 256 ? p->L : 256)};
  cuuint32_t estride[1] = {1};
  CUresult r = enc(&p->map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 1, const_cast<void*>(d_spectrum), gdim, gstride, box,
                   estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    p->map_ptr = nullptr;
    return FDAS_ERR_CUDA;
  }
  p->map_ptr = d_spectrum;
  return FDAS_OK;
}

void free_tc_memory(fdas_plan* p) {
  cudaFree(p->tc_bank);
  cudaFree(p->tc_seg);
  cudaFree(p->tc_mats);
  cudaFree(p->tc_tmax);
  p->tc_bank = nullptr;
  p->tc_seg = nullptr;
  p->tc_mats = nullptr;
  p->tc_tmax = nullptr;
  p->tc_ready = false;
}

void free_plan_memory(fdas_plan* p) {
  free_tc_memory(p);
  if (p->done) cudaEventDestroy(p->done);
  p->done = nullptr;
  cudaFree(p->d_templates);
  cudaFree(p->d_taps);
  cudaFree(p->d_twist);
  cudaFree(p->d_status);
  p->d_templates = nullptr;
  p->d_taps = nullptr;
  p->d_twist = nullptr;
  p->d_status = nullptr;
}

}  // namespace

extern "C" {

const char* fdas_error_string(int code) {
  switch (code) {
    case FDAS_OK: return "ok";
    case FDAS_ERR_INVALID: return "invalid argument";
    case FDAS_ERR_ALIGN: return "misaligned pointer";
    case FDAS_ERR_NOT_BUILT: return "templates not built (call fdas_templates_build first)";
    case FDAS_ERR_ALLOC: return "device allocation failed";
    case FDAS_ERR_CUDA: return "CUDA runtime or launch error";
    case FDAS_ERR_NO_DEVICE: return "no CUDA device";
    case FDAS_ERR_UNSUPPORTED: return "device is not compute capability 10.3 (GB300)";
    case FDAS_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    default: return "unknown fdas status";
  }
}

int fdas_last_error(void) { return g_last_error; }

fdas_plan* fdas_plan_create(int64_t n_bins, int zmax, int zstep, int seg_len, int tmpl_len) {
  g_last_error = FDAS_OK;
  int rc = validate(n_bins, zmax, zstep, seg_len, tmpl_len);
  if (rc != FDAS_OK) {
    g_last_error = rc;
    return nullptr;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    g_last_error = FDAS_ERR_NO_DEVICE;
    return nullptr;
  }
  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    g_last_error = FDAS_ERR_CUDA;
    return nullptr;
  }
  if (major != 10 || minor != 3) {
    g_last_error = FDAS_ERR_UNSUPPORTED;
    return nullptr;
  }
  fdas_plan* p = new (std::nothrow) fdas_plan();
  if (!p) {
    g_last_error = FDAS_ERR_ALLOC;
    return nullptr;
  }
  p->device = dev;
  p->sm_count = sms;
  p->n_bins = n_bins;
  p->zmax = zmax;
  p->zstep = zstep;
  p->L = seg_len;
  p->m = tmpl_len;
  p->h = tmpl_len / 2;
  p->V = seg_len - tmpl_len;
  p->Z = 2 * (zmax / zstep) + 1;
  p->nseg = (n_bins + p->V - 1) / p->V;
  p->n1 = fdas::conv_group_threads(seg_len);
  const size_t ntap = (size_t)tmpl_len + 1;
  if (cudaMalloc(&p->d_templates, sizeof(float2) * (size_t)p->Z * p->L) != cudaSuccess ||
      cudaMalloc(&p->d_taps, sizeof(double2) * (size_t)p->Z * ntap) != cudaSuccess ||
      cudaMalloc(&p->d_twist, sizeof(float2) * (size_t)p->L) != cudaSuccess ||
      cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    free_plan_memory(p);
    delete p;
    g_last_error = FDAS_ERR_ALLOC;
    return nullptr;
  }
  // cleared before any stream can use the plan (a non-blocking stream is not ordered after
  // default-stream work)
  if (cudaMemsetAsync(p->d_status, 0, sizeof(int), 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) {
    free_plan_memory(p);
    delete p;
    g_last_error = FDAS_ERR_CUDA;
    return nullptr;
  }
  return p;
}

int fdas_templates_build(fdas_plan* p, fdas_stream_t stream) {
  if (!p) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (fdas::build_templates_into(p->d_taps, p->d_templates, p->d_twist, p->zmax, p->zstep, p->L, p->m, st) !=
      cudaSuccess)
    return FDAS_ERR_CUDA;
  p->built = true;
  p->tc_ready = false;   // the tensor-core variant copies the bank again on its next call
  return note_work(p, st);
}

int fdas_convolve_power(fdas_plan* p, const float* d_spectrum, float* d_plane, fdas_stream_t stream) {
  if (!p || !d_spectrum || !d_plane) return FDAS_ERR_INVALID;
  if (!p->built) return FDAS_ERR_NOT_BUILT;
  if ((reinterpret_cast<uintptr_t>(d_spectrum) & 15u) || (reinterpret_cast<uintptr_t>(d_plane) & 15u))
    return FDAS_ERR_ALIGN;
  int rc = make_spectrum_map(p, d_spectrum);
  if (rc != FDAS_OK) return rc;
  fdas::ConvParams q;
  q.spectrum = reinterpret_cast<const float2*>(d_spectrum);
  q.templates = p->d_templates;
  q.twist = p->d_twist;
  q.plane = d_plane;
  q.status = p->d_status;
  q.n_bins = p->n_bins;
  q.nseg = p->nseg;
  q.units = 0;
  q.Z = p->Z;
  q.V = p->V;
  q.h = p->h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return enqueued(p, st, fdas::launch_convolve(p->L, &p->map, q, p->sm_count, st));
}

int fdas_plan_group_segments(const fdas_plan* p) {
  if (!p) return FDAS_ERR_INVALID;
  const int G = fdas::batch_segments_per_cta(p->L);
  return G > 0 ? G : FDAS_ERR_INVALID;
}

int fdas_convolve_power_units_masked(fdas_plan* p, const float* d_spectrum, float* d_plane,
                                     const int32_t* d_units, const uint16_t* d_masks, int64_t n_units,
                                     fdas_stream_t stream) {
  if (!p || !d_spectrum || !d_plane || !d_units || n_units < 1) return FDAS_ERR_INVALID;
  if (!p->built) return FDAS_ERR_NOT_BUILT;
  if (fdas::batch_segments_per_cta(p->L) == 0) return FDAS_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(d_spectrum) & 15u) || (reinterpret_cast<uintptr_t>(d_plane) & 15u) ||
      (reinterpret_cast<uintptr_t>(d_units) & 3u) || (reinterpret_cast<uintptr_t>(d_masks) & 1u))
    return FDAS_ERR_ALIGN;
  fdas::ConvParams q;
  q.spectrum = reinterpret_cast<const float2*>(d_spectrum);
  q.templates = p->d_templates;
  q.twist = p->d_twist;
  q.plane = d_plane;
  q.status = p->d_status;
  q.n_bins = p->n_bins;
  q.nseg = p->nseg;
  q.units = 0;
  q.Z = p->Z;
  q.V = p->V;
  q.h = p->h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return enqueued(p, st, fdas::launch_units(p->L, q, d_units, d_masks, n_units, p->sm_count, st));
}

int fdas_convolve_power_units_device_count(fdas_plan* p, const float* d_spectrum, float* d_plane,
                                           const int32_t* d_units, const uint16_t* d_masks, const int64_t* d_count,
                                           int64_t max_units, fdas_stream_t stream) {
  if (!p || !d_spectrum || !d_plane || !d_units || !d_count || max_units < 1) return FDAS_ERR_INVALID;
  if (!p->built) return FDAS_ERR_NOT_BUILT;
  if (fdas::batch_segments_per_cta(p->L) == 0) return FDAS_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(d_spectrum) & 15u) || (reinterpret_cast<uintptr_t>(d_plane) & 15u) ||
      (reinterpret_cast<uintptr_t>(d_units) & 3u) || (reinterpret_cast<uintptr_t>(d_masks) & 1u) ||
      (reinterpret_cast<uintptr_t>(d_count) & 7u))
    return FDAS_ERR_ALIGN;
  fdas::ConvParams q;
  q.spectrum = reinterpret_cast<const float2*>(d_spectrum);
  q.templates = p->d_templates;
  q.twist = p->d_twist;
  q.plane = d_plane;
  q.status = p->d_status;
  q.n_bins = p->n_bins;
  q.nseg = p->nseg;
  q.units = 0;
  q.Z = p->Z;
  q.V = p->V;
  q.h = p->h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return enqueued(p, st, fdas::launch_units(p->L, q, d_units, d_masks, max_units, p->sm_count, st, d_count));
}

int fdas_convolve_power_units(fdas_plan* p, const float* d_spectrum, float* d_plane, const int32_t* d_units,
                              int64_t n_units, fdas_stream_t stream) {
  return fdas_convolve_power_units_masked(p, d_spectrum, d_plane, d_units, nullptr, n_units, stream);
}

namespace {
int convolve_pairs(fdas_plan* p, const float* d_spectrum, float* d_plane, const int32_t* d_pairs,
                   const int64_t* d_count, int64_t n_pairs, fdas_stream_t stream) {
  if (!p || !d_spectrum || !d_plane || !d_pairs || n_pairs < 1) return FDAS_ERR_INVALID;
  if (!p->built) return FDAS_ERR_NOT_BUILT;
  if (!fdas::pairs_supported(p->L)) return FDAS_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(d_spectrum) & 15u) || (reinterpret_cast<uintptr_t>(d_plane) & 15u) ||
      (reinterpret_cast<uintptr_t>(d_pairs) & 3u) || (reinterpret_cast<uintptr_t>(d_count) & 7u))
    return FDAS_ERR_ALIGN;
  fdas::PairParams q;
  q.spec = reinterpret_cast<const float2*>(d_spectrum);
  q.plane = d_plane;
  q.templates = p->d_templates;
  q.twist = p->d_twist;
  q.status = p->d_status;
  q.pairs = d_pairs;
  q.pair_count = d_count;
  q.n_pairs = n_pairs;
  q.n_bins = p->n_bins;
  q.nseg = p->nseg;
  q.Z = p->Z;
  q.V = p->V;
  q.h = p->h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return enqueued(p, st, fdas::launch_pairs(p->L, q, p->sm_count, st));
}
}  // namespace

int fdas_convolve_power_pairs(fdas_plan* p, const float* d_spectrum, float* d_plane, const int32_t* d_pairs,
                              int64_t n_pairs, fdas_stream_t stream) {
  return convolve_pairs(p, d_spectrum, d_plane, d_pairs, nullptr, n_pairs, stream);
}

int fdas_convolve_power_pairs_device_count(fdas_plan* p, const float* d_spectrum, float* d_plane,
                                           const int32_t* d_pairs, const int64_t* d_count, int64_t max_pairs,
                                           fdas_stream_t stream) {
  if (!d_count) return FDAS_ERR_INVALID;
  return convolve_pairs(p, d_spectrum, d_plane, d_pairs, d_count, max_pairs, stream);
}

int fdas_segment_spectra(fdas_plan* p, const float* d_spectrum, float* d_out, fdas_stream_t stream) {
  if (!p || !d_spectrum || !d_out) return FDAS_ERR_INVALID;
  if (!p->built) return FDAS_ERR_NOT_BUILT;
  if ((reinterpret_cast<uintptr_t>(d_spectrum) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 15u))
    return FDAS_ERR_ALIGN;
  int rc = make_spectrum_map(p, d_spectrum);
  if (rc != FDAS_OK) return rc;
  fdas::SegParams q;
  q.twist = p->d_twist;
  q.spectrum_in = reinterpret_cast<const float2*>(d_spectrum);
  q.out = reinterpret_cast<float2*>(d_out);
  q.status = p->d_status;
  q.n_bins = p->n_bins;
  q.nseg = p->nseg;
  q.V = p->V;
  q.h = p->h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return enqueued(p, st, fdas::launch_segment_spectra(p->L, &p->map, q, p->sm_count, st));
}

namespace {

// The tensor-core variant's workspace, allocated and filled on the first call after a template
// build: natural-order bank, its max |Re|, |Im|, the four sets of DFT matrices, the segment
// spectra.
int tc_ensure_ready(fdas_plan* p, cudaStream_t st) {
  if (p->tc_ready) return FDAS_OK;
  free_tc_memory(p);
  const int mb = fdas::tc_matrices_bytes();
  if (cudaMalloc(&p->tc_bank, sizeof(float2) * (size_t)p->Z * p->L) != cudaSuccess ||
      cudaMalloc(&p->tc_seg, sizeof(float2) * (size_t)p->nseg * p->L) != cudaSuccess ||
      cudaMalloc(&p->tc_mats, 4 * (size_t)mb) != cudaSuccess ||
      cudaMalloc(&p->tc_tmax, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    free_tc_memory(p);
    return FDAS_ERR_ALLOC;
  }
  if (fdas::launch_tc_prepare(p->d_templates, p->Z, p->tc_bank, p->tc_tmax, p->tc_mats, st) != cudaSuccess)
    return FDAS_ERR_CUDA;
  p->tc_ready = true;
  return FDAS_OK;
}

fdas::TcParams tc_params(const fdas_plan* p, const float* d_spectrum, int precision, bool forward) {
  const int mb = fdas::tc_matrices_bytes();
  fdas::TcParams q;
  q.seg = p->tc_seg;
  q.seg_out = p->tc_seg;
  q.spectrum = reinterpret_cast<const float2*>(d_spectrum);
  q.bank = p->tc_bank;
  q.twist = p->d_twist;
  q.mats = p->tc_mats + (size_t)mb * ((forward ? 2 : 0) + (precision == FDAS_TC_FP16 ? 1 : 0));
  q.tmax = p->tc_tmax;
  q.plane = nullptr;
  q.status = p->d_status;
  q.n_bins = p->n_bins;
  q.nseg = p->nseg;
  q.units = forward ? (p->nseg + 3) / 4 : p->nseg * (int64_t)((p->Z + 3) / 4);
  q.Z = p->Z;
  q.V = p->V;
  q.h = p->h;
  return q;
}

int tc_validate(fdas_plan* p, const void* a, const void* b, int precision) {
  if (!p || !a || !b || (precision != FDAS_TC_BF16 && precision != FDAS_TC_FP16)) return FDAS_ERR_INVALID;
  if (!p->built) return FDAS_ERR_NOT_BUILT;
  if (p->L != 2048) return FDAS_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(a) & 15u) || (reinterpret_cast<uintptr_t>(b) & 15u)) return FDAS_ERR_ALIGN;
  return FDAS_OK;
}

}  // namespace

int fdas_convolve_power_tc(fdas_plan* p, const float* d_spectrum, float* d_plane, int precision,
                           fdas_stream_t stream) {
  int rc = tc_validate(p, d_spectrum, d_plane, precision);
  if (rc != FDAS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if ((rc = tc_ensure_ready(p, st)) != FDAS_OK) return rc;
  if (fdas::launch_tc(tc_params(p, d_spectrum, precision, true), precision, true, p->sm_count, st) != cudaSuccess)
    return FDAS_ERR_CUDA;
  fdas::TcParams q = tc_params(p, d_spectrum, precision, false);
  q.plane = d_plane;
  return enqueued(p, st, fdas::launch_tc(q, precision, false, p->sm_count, st));
}

int fdas_segment_spectra_tc(fdas_plan* p, const float* d_spectrum, float* d_out, int precision,
                            fdas_stream_t stream) {
  int rc = tc_validate(p, d_spectrum, d_out, precision);
  if (rc != FDAS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if ((rc = tc_ensure_ready(p, st)) != FDAS_OK) return rc;
  fdas::TcParams q = tc_params(p, d_spectrum, precision, true);
  q.seg_out = reinterpret_cast<float2*>(d_out);
  return enqueued(p, st, fdas::launch_tc(q, precision, true, p->sm_count, st));
}

int fdas_check(fdas_plan* p, fdas_stream_t stream) {
  if (!p) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int status = 0;
  if (cudaMemcpyAsync(&status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FDAS_ERR_CUDA;
  if (status != 0) {
    // cleared in the stream's order, before the call returns
    if (cudaMemsetAsync(p->d_status, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      return FDAS_ERR_CUDA;
    return (status & fdas::kStatusTimeout) ? FDAS_ERR_TIMEOUT : FDAS_ERR_INVALID;
  }
  return FDAS_OK;
}

int fdas_selftest_wait_timeout(fdas_plan* p, int64_t limit_ns, fdas_stream_t stream) {
  if (!p || limit_ns < 1000 || limit_ns > 2000000000LL) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return enqueued(p, st, fdas::launch_wait_selftest(p->d_status, limit_ns, st));
}

int fdas_destroy(fdas_plan* p) {
  if (!p) return FDAS_OK;
  if (p->done) cudaEventSynchronize(p->done);   // the plan's last enqueued work, not the whole device
  free_plan_memory(p);
  delete p;
  return FDAS_OK;
}

int fdas_plan_dims(const fdas_plan* p, int* Z, int* V, int64_t* nseg) {
  if (!p) return FDAS_ERR_INVALID;
  if (Z) *Z = p->Z;
  if (V) *V = p->V;
  if (nseg) *nseg = p->nseg;
  return FDAS_OK;
}

int fdas_template_taps(fdas_plan* p, int z_idx, double* host_out) {
  if (!p || !host_out || z_idx < 0 || z_idx >= p->Z) return FDAS_ERR_INVALID;
  if (!p->built) return FDAS_ERR_NOT_BUILT;
  const size_t ntap = (size_t)p->m + 1;
  if (cudaEventSynchronize(p->done) != cudaSuccess) return FDAS_ERR_CUDA;
  if (cudaMemcpy(host_out, p->d_taps + (size_t)z_idx * ntap, sizeof(double2) * ntap, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return FDAS_ERR_CUDA;
  return FDAS_OK;
}

int fdas_template_spectrum(fdas_plan* p, int z_idx, float* host_out) {
  if (!p || !host_out || z_idx < 0 || z_idx >= p->Z) return FDAS_ERR_INVALID;
  if (!p->built) return FDAS_ERR_NOT_BUILT;
  if (cudaEventSynchronize(p->done) != cudaSuccess) return FDAS_ERR_CUDA;
  float2* tmp = static_cast<float2*>(std::malloc(sizeof(float2) * (size_t)p->L));
  if (!tmp) return FDAS_ERR_ALLOC;
  if (cudaMemcpy(tmp, p->d_templates + (size_t)z_idx * p->L, sizeof(float2) * (size_t)p->L,
                 cudaMemcpyDeviceToHost) != cudaSuccess) {
    std::free(tmp);
    return FDAS_ERR_CUDA;
  }
  const float* f = reinterpret_cast<const float*>(tmp);
  for (int k = 0; k < p->L; ++k) {
    const int off = pair_layout_re(k, p->n1);
    host_out[2 * k] = f[off];
    host_out[2 * k + 1] = f[off + (p->n1 ? 2 : 1)];
  }
  std::free(tmp);
  return FDAS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Helpers for the allocation-free entry point (fdas_static.cu): the same validation, template
// build kernels and tensor-map encoding as the plan-based calls above, on caller-given memory.
// ---------------------------------------------------------------------------------------
namespace fdas {

int validate_geometry(int64_t n_bins, int zmax, int zstep, int seg_len, int tmpl_len) {
  return validate(n_bins, zmax, zstep, seg_len, tmpl_len);
}

cudaError_t build_templates_into(double2* taps, float2* templates, float2* twist, int zmax, int zstep, int L,
                                 int m, cudaStream_t st) {
  const GLTable& gl = gl_table();
  cudaError_t e = cudaMemcpyToSymbolAsync(c_gl_x, gl.x, sizeof(gl.x), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_gl_w, gl.w, sizeof(gl.w), 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const int Z = 2 * (zmax / zstep) + 1, h = m / 2, n1 = conv_group_threads(L);
  taps_kernel<<<Z, 256, 0, st>>>(taps, zmax, zstep, h);
  const size_t tab = sizeof(double2) * (size_t)L;
  e = cudaFuncSetAttribute(spectra_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab);
  if (e != cudaSuccess) return e;
  spectra_kernel<<<dim3((L + 255) / 256, Z), 256, tab, st>>>(taps, templates, L, h, n1);
  twist_kernel<<<(L + 255) / 256, 256, 0, st>>>(twist, L, n1);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* status, int64_t limit_ns, cudaStream_t st) {
  wait_selftest_kernel<<<1, 1, 0, st>>>(status, (unsigned long long)limit_ns);
  return cudaGetLastError();
}

int encode_spectrum_map(CUtensorMap* map, const void* d_spectrum, int64_t n_bins, int L) {
  if (L >= 4096) return FDAS_OK;   // the L >= 4096 kernels read the spectrum directly
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return FDAS_ERR_CUDA;
  cuuint64_t gdim[1] = {(cuuint64_t)n_bins};
  cuuint64_t gstride[1] = {0};
  cuuint32_t box[1] = {(cuuint32_t)(L < 256 ? L : 256)};
  cuuint32_t estride[1] = {1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 1, const_cast<void*>(d_spectrum), gdim, gstride, box,
                   estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? FDAS_OK : FDAS_ERR_CUDA;
}

}  // namespace fdas
