// fdas_static.cu -- fdas_convolve_power_static: the fused correlation without any device
// allocation (declared in include/fdas.h).  The template bank, FP64 taps, twiddle table and
// status word live in one file-scope device array instead of plan memory; fdas_static_check
// reads (and clears) that status word, fdas_static_selftest_wait_timeout exercises it.
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "fdas.h"
#include "fdas_internal.h"

namespace {

// The scratch array.  In host code `g_static_scratch` is only a host-side stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_static_scratch[FDAS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;

struct DeviceScratch {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_static_scratch on this device
  int sm_count = 0;
  bool have_bank = false;          // geometry of the template bank currently in the array
  int zmax = -1, zstep = -1, L = -1, m = -1;
};

DeviceScratch g_dev[kMaxDevices];
std::mutex g_mutex;

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// The array's device address on the current device, looked up once per device (with that device
// current), and the device's SM count.  Returns FDAS_OK or an error code; g_mutex must be held.
int device_scratch(DeviceScratch** out) {
  int ndev = 0, dev = 0, major = 0, minor = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return FDAS_ERR_NO_DEVICE;
  }
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FDAS_ERR_CUDA;
  DeviceScratch& s = g_dev[dev];
  if (!s.ready) {
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
      return FDAS_ERR_CUDA;
    if (major != 10 || minor != 3) return FDAS_ERR_UNSUPPORTED;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return FDAS_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FDAS_ERR_CUDA;
    s.base = static_cast<unsigned char*>(ptr);
    s.sm_count = sms;
    s.ready = true;
  }
  *out = &s;
  return FDAS_OK;
}

// Layout of the array: status word (its own 256 bytes, at a fixed place so that it survives
// calls with other geometries) | template spectra | taps | twiddles.
constexpr size_t kOffStatus = 0;
constexpr size_t kOffBank = 256;

}  // namespace

extern "C" int fdas_convolve_power_static(int64_t n_bins, int zmax, int zstep, int seg_len, int tmpl_len,
                                          const float* d_spectrum, float* d_plane, fdas_stream_t stream) {
  int rc = fdas::validate_geometry(n_bins, zmax, zstep, seg_len, tmpl_len);
  if (rc != FDAS_OK) return rc;
  const int L = seg_len, m = tmpl_len, h = m / 2, V = L - m;
  const int Z = 2 * (zmax / zstep) + 1;
  const size_t off_tmpl = kOffBank;
  const size_t off_taps = off_tmpl + round256(sizeof(float2) * (size_t)Z * L);
  const size_t off_twist = off_taps + round256(sizeof(double2) * (size_t)Z * (m + 1));
  const size_t need = off_twist + round256(sizeof(float2) * (size_t)L);
  if (need > (size_t)FDAS_STATIC_SCRATCH_BYTES) return FDAS_ERR_INVALID;
  if (!d_spectrum || !d_plane) return FDAS_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(d_spectrum) & 15u) || (reinterpret_cast<uintptr_t>(d_plane) & 15u))
    return FDAS_ERR_ALIGN;

  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceScratch* sp = nullptr;
  if ((rc = device_scratch(&sp)) != FDAS_OK) return rc;
  DeviceScratch& s = *sp;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float2* templates = reinterpret_cast<float2*>(s.base + off_tmpl);
  double2* taps = reinterpret_cast<double2*>(s.base + off_taps);
  float2* twist = reinterpret_cast<float2*>(s.base + off_twist);
  int* status = reinterpret_cast<int*>(s.base + kOffStatus);

  if (!s.have_bank || s.zmax != zmax || s.zstep != zstep || s.L != L || s.m != m) {
    s.have_bank = false;
    if (fdas::build_templates_into(taps, templates, twist, zmax, zstep, L, m, st) != cudaSuccess)
      return FDAS_ERR_CUDA;
    s.have_bank = true;
    s.zmax = zmax;
    s.zstep = zstep;
    s.L = L;
    s.m = m;
  }

  CUtensorMap map;
  rc = fdas::encode_spectrum_map(&map, d_spectrum, n_bins, L);
  if (rc != FDAS_OK) return rc;
  fdas::ConvParams q;
  q.spectrum = reinterpret_cast<const float2*>(d_spectrum);
  q.templates = templates;
  q.twist = twist;
  q.plane = d_plane;
  q.status = status;
  q.n_bins = n_bins;
  q.nseg = (n_bins + V - 1) / V;
  q.units = 0;
  q.Z = Z;
  q.V = V;
  q.h = h;
  return fdas::launch_convolve(L, &map, q, s.sm_count, st) == cudaSuccess ? FDAS_OK : FDAS_ERR_CUDA;
}

extern "C" int fdas_static_check(fdas_stream_t stream) {
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceScratch* sp = nullptr;
  int rc = device_scratch(&sp);
  if (rc != FDAS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* status = reinterpret_cast<int*>(sp->base + kOffStatus);
  int word = 0;
  if (cudaMemcpyAsync(&word, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FDAS_ERR_CUDA;
  if (word == 0) return FDAS_OK;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return FDAS_ERR_CUDA;
  return (word & fdas::kStatusTimeout) ? FDAS_ERR_TIMEOUT : FDAS_ERR_INVALID;
}

extern "C" int fdas_static_selftest_wait_timeout(int64_t limit_ns, fdas_stream_t stream) {
  if (limit_ns < 1000 || limit_ns > 2000000000LL) return FDAS_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceScratch* sp = nullptr;
  int rc = device_scratch(&sp);
  if (rc != FDAS_OK) return rc;
  int* status = reinterpret_cast<int*>(sp->base + kOffStatus);
  return fdas::launch_wait_selftest(status, limit_ns, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FDAS_OK
             : FDAS_ERR_CUDA;
}
