// fdas_convolve_big.cu -- the fused correlation (steps a2..a7 of Eq. 2 by overlap-and-save,
// Section 2) for segment lengths 4096 and 8192.
//
// One CTA of 512 threads owns a segment at a time: it loads the segment (zeros outside [0, n)),
// transforms it (forward, Eq. 3 sign) into shared memory once, and then for every template z
// multiplies by T_z, inverse-transforms and stores |y|^2 of the first V outputs.  Transforms are
// Stockham autosort FFTs in shared memory (ping-pong between two L-point buffers): radix-4
// passes, plus one radix-2 pass when log2 L is odd.  Pass p combines sub-transforms of length Ns
// into length R*Ns: butterfly j (j < L/R) reads elements j + r*L/R, multiplies element r by
// W^(r*k*L/(R*Ns)) (k = j mod Ns, W = exp(-+2 pi i / L) from the plan's twiddle table), takes the
// R-point DFT and writes element r to (j - k)*R + k + r*Ns.  The first pass of an inverse
// transform reads X*T directly and the last pass writes powers to the plane, so each template
// costs log_4 L passes over shared memory.  Templates are stored in natural order.
#include <cuda_runtime.h>

#include "fdas_device.cuh"
#include "fdas_internal.h"

namespace fdas {
namespace {

constexpr int kBigThreads = 512;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// W^t for the forward transform (DIR = -1), its conjugate for the inverse (DIR = +1).
template <int DIR>
__device__ __forceinline__ float2 twiddle(const float2* W, int t) {
  float2 w = __ldg(W + t);
  if (DIR > 0) w.y = -w.y;
  return w;
}

// One radix-4 pass with sub-transform length Ns.
template <int L, int DIR, class Load, class Store>
__device__ __forceinline__ void pass4(int Ns, const float2* W, Load load, Store store) {
  for (int j = threadIdx.x; j < L / 4; j += kBigThreads) {
    const int k = j & (Ns - 1);
    const int t = k * (L / (4 * Ns));
    float2 v0 = load(j), v1 = load(j + L / 4), v2 = load(j + L / 2), v3 = load(j + 3 * L / 4);
    if (Ns > 1) {
      v1 = cmulf(v1, twiddle<DIR>(W, t));
      v2 = cmulf(v2, twiddle<DIR>(W, 2 * t));
      v3 = cmulf(v3, twiddle<DIR>(W, 3 * t));
    }
    const float2 a0 = make_float2(v0.x + v2.x, v0.y + v2.y), a1 = make_float2(v0.x - v2.x, v0.y - v2.y);
    const float2 a2 = make_float2(v1.x + v3.x, v1.y + v3.y), a3 = make_float2(v1.x - v3.x, v1.y - v3.y);
    const float2 y0 = make_float2(a0.x + a2.x, a0.y + a2.y), y2 = make_float2(a0.x - a2.x, a0.y - a2.y);
    // forward: y1 = a1 - i a3, y3 = a1 + i a3; inverse: the two swap
    const float2 ym = make_float2(a1.x + a3.y, a1.y - a3.x), yp = make_float2(a1.x - a3.y, a1.y + a3.x);
    const int d = ((j - k) << 2) + k;
    store(d, y0);
    store(d + Ns, DIR < 0 ? ym : yp);
    store(d + 2 * Ns, y2);
    store(d + 3 * Ns, DIR < 0 ? yp : ym);
  }
}

// The final radix-2 pass (Ns = L/2, so k = j and the twiddle index is j).
template <int L, int DIR, class Load, class Store>
__device__ __forceinline__ void pass2(const float2* W, Load load, Store store) {
  for (int j = threadIdx.x; j < L / 2; j += kBigThreads) {
    const float2 v0 = load(j), v1 = cmulf(load(j + L / 2), twiddle<DIR>(W, j));
    store(j, make_float2(v0.x + v1.x, v0.y + v1.y));
    store(j + L / 2, make_float2(v0.x - v1.x, v0.y - v1.y));
  }
}

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

// A whole L-point transform: `first` supplies the input, `last` consumes the output (natural
// order); b0 / b1 are the ping-pong buffers.  Ends with a CTA barrier.
template <int L, int DIR, class First, class Last>
__device__ __forceinline__ void stockham(float2* b0, float2* b1, const float2* W, First first, Last last) {
  constexpr int P4 = ilog2c(L) / 2;
  constexpr bool R2 = (ilog2c(L) & 1) != 0;
  constexpr int P = P4 + (R2 ? 1 : 0);
  auto ld = [](const float2* b) { return [b](int i) { return b[i]; }; };
  auto st = [](float2* b) { return [b](int i, float2 v) { b[i] = v; }; };
  static_for<P>([&](auto pp) {
    constexpr int p = decltype(pp)::value;
    float2* src = (p % 2 == 1) ? b0 : b1;
    float2* dst = (p % 2 == 0) ? b0 : b1;
    if constexpr (p < P4) {
      constexpr int Ns = 1 << (2 * p);
      if constexpr (p == 0 && p == P - 1) pass4<L, DIR>(Ns, W, first, last);
      else if constexpr (p == 0) pass4<L, DIR>(Ns, W, first, st(dst));
      else if constexpr (p == P - 1) pass4<L, DIR>(Ns, W, ld(src), last);
      else pass4<L, DIR>(Ns, W, ld(src), st(dst));
    } else {
      pass2<L, DIR>(W, ld(src), last);
    }
    __syncthreads();
  });
}

template <int L>
__global__ void __launch_bounds__(kBigThreads, 1) convolve_big_kernel(const ConvParams p) {
  extern __shared__ __align__(16) float2 sbig[];
  float2* X = sbig;
  float2* b0 = sbig + L;
  float2* b1 = sbig + 2 * L;
  const float2* W = p.twist;
  for (int64_t s = blockIdx.x; s < p.nseg; s += gridDim.x) {
    const int64_t x0 = s * (int64_t)p.V - p.h;
    // a2 + a3: the segment (zeros outside [0, n)), forward transform into X
    stockham<L, -1>(
        b0, b1, W,
        [&](int i) {
          const int64_t r = x0 + i;
          return (r >= 0 && r < p.n_bins) ? __ldg(p.spectrum + r) : make_float2(0.f, 0.f);
        },
        [&](int i, float2 v) { X[i] = v; });
    const int64_t segbase = s * (int64_t)p.V;
    const int64_t lim64 = p.n_bins - segbase < (int64_t)p.V ? p.n_bins - segbase : (int64_t)p.V;
    const int lim = (int)lim64;
    for (int z = 0; z < p.Z; ++z) {
      const float2* T = p.templates + (size_t)z * L;
      float* row = p.plane + (size_t)z * p.n_bins + segbase;
      // a4 + a5 + a6 + a7: X*T_z, inverse transform, keep n < V, store |y|^2
      stockham<L, +1>(
          b0, b1, W, [&](int i) { return cmulf(X[i], __ldg(T + i)); },
          [&](int i, float2 v) {
            if (i < lim) __stcs(row + i, fmaf(v.x, v.x, v.y * v.y));
          });
    }
  }
}

// Forward transforms only (a2 + a3), natural order, for tests of the FFT.
template <int L>
__global__ void __launch_bounds__(kBigThreads, 1) segment_spectra_big_kernel(const SegParams p) {
  extern __shared__ __align__(16) float2 sbig[];
  float2* b0 = sbig;
  float2* b1 = sbig + L;
  for (int64_t s = blockIdx.x; s < p.nseg; s += gridDim.x) {
    const int64_t x0 = s * (int64_t)p.V - p.h;
    float2* out = p.out + (size_t)s * L;
    stockham<L, -1>(
        b0, b1, p.twist,
        [&](int i) {
          const int64_t r = x0 + i;
          return (r >= 0 && r < p.n_bins) ? __ldg(p.spectrum_in + r) : make_float2(0.f, 0.f);
        },
        [&](int i, float2 v) { out[i] = v; });
  }
}

template <int L>
cudaError_t launch_big(const ConvParams& p, int sm_count, cudaStream_t st) {
  constexpr size_t smem = 3 * (size_t)L * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(convolve_big_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int per_sm = (int)(227 * 1024 / smem) > 0 ? (int)(227 * 1024 / smem) : 1;
  const int64_t grid = p.nseg < (int64_t)per_sm * sm_count ? p.nseg : (int64_t)per_sm * sm_count;
  convolve_big_kernel<L><<<(unsigned)grid, kBigThreads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_seg_big(const SegParams& p, int sm_count, cudaStream_t st) {
  constexpr size_t smem = 2 * (size_t)L * sizeof(float2);
  cudaError_t e =
      cudaFuncSetAttribute(segment_spectra_big_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = p.nseg < (int64_t)sm_count ? p.nseg : (int64_t)sm_count;
  segment_spectra_big_kernel<L><<<(unsigned)grid, kBigThreads, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_convolve_big(int L, const ConvParams& p, int sm_count, cudaStream_t st) {
  switch (L) {
    case 4096: return launch_big<4096>(p, sm_count, st);
    case 8192: return launch_big<8192>(p, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_segment_spectra_big(int L, const SegParams& p, int sm_count, cudaStream_t st) {
  switch (L) {
    case 4096: return launch_seg_big<4096>(p, sm_count, st);
    case 8192: return launch_seg_big<8192>(p, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdas
