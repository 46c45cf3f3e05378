// fdas_convolve_big.cu -- the fused correlation (steps a2..a7 of Eq. 2 by overlap-and-save,
// Section 2) for segment lengths 4096 and 8192.
//
// One CTA of L/16 threads owns a segment at a time: it loads the segment (zeros outside [0, n)),
// transforms it (forward, Eq. 3 sign) into shared memory once, and then for every template z
// multiplies by T_z, inverse-transforms and stores |y|^2 of the first V outputs.  Transforms are
// Stockham autosort FFTs in shared memory (ping-pong between two L-point buffers): radix-16
// passes (each thread one 16-point DFT in registers), plus one radix-2 pass when log16 L is not
// whole.  Pass p combines sub-transforms of length Ns into length R*Ns: butterfly j (j < L/R)
// reads elements j + r*L/R, multiplies element r by W^(r*k*L/(R*Ns)) (k = j mod Ns,
// W = exp(-+2 pi i / L), from a quarter-period table in shared memory staged from the plan's
// twiddle table), takes the R-point DFT and writes element r to (j - k)*R + k + r*Ns.  The first
// pass of an inverse transform reads X*T directly and the last pass writes powers to the plane.
// Shared buffers hold element i at i + i/16, so the stride-16 writes of the first pass spread
// over the banks.  Templates are stored in natural order.
#include <cuda_runtime.h>

#include "fdas_device.cuh"
#include "fdas_internal.h"

namespace fdas {
namespace {

constexpr int kRadix = 16;

__host__ __device__ constexpr int padded(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

template <int L>
struct BigCfg {
  static constexpr int NT = L / kRadix;                 // threads per CTA
  static constexpr int P16 = ilog2c(L) / 4;             // radix-16 passes
  static constexpr bool R2 = (ilog2c(L) % 4) == 1;      // one radix-2 pass after them
  static constexpr int P = P16 + (R2 ? 1 : 0);
  static constexpr int BUF = padded(L);                 // padded buffer length (float2)
  static_assert(ilog2c(L) % 4 == 0 || R2, "L = 16^p or 2 * 16^p");
};

// W^t for the forward transform (DIR = -1), its conjugate for the inverse (DIR = +1), from the
// quarter-period table Q[u] = W^u, u < L/4 (at padded(u)): W^(u + q L/4) = (-i)^q W^u.
template <int L, int DIR>
__device__ __forceinline__ float2 twiddle(const float2* Q, int t) {
  const float2 b = Q[padded(t & (L / 4 - 1))];   // the table is bank-padded like the buffers
  const int q = (t / (L / 4)) & 3;
  float2 w = (q & 1) ? make_float2(b.y, -b.x) : b;   // -i * b for odd quadrants
  if (q & 2) w = make_float2(-w.x, -w.y);
  if (DIR > 0) w.y = -w.y;
  return w;
}

// One radix-R pass with sub-transform length Ns (R = 16 or 2).
template <int L, int R, int DIR, class Load, class Store>
__device__ __forceinline__ void pass_r(int Ns, const float2* Q, Load load, Store store) {
  constexpr int NT = BigCfg<L>::NT, LOGR = ilog2c(R);
  for (int j = threadIdx.x; j < L / R; j += NT) {
    const int k = j & (Ns - 1);
    const int t = k * (L / (R * Ns));
    float2 v[R];
    static_for<R>([&](auto rr) {
      constexpr int r = decltype(rr)::value;
      v[bitrev(r, LOGR)] = load(j + r * (L / R));
    });
    if (Ns > 1) {
      // W^(r t) for r = 1..R-1 from W^t by products of depth <= 4 (one table read per butterfly:
      // reading every power would put a half-warp's stride-16r indices on one bank)
      float2 w[R];
      w[1] = twiddle<L, DIR>(Q, t);
      static_for<R - 2>([&](auto ii) {
        constexpr int r = decltype(ii)::value + 2;
        constexpr int hi = 1 << (ilog2c(r));      // largest power of two <= r
        if constexpr (hi == r) w[r] = cmul(w[r / 2], w[r / 2]);
        else w[r] = cmul(w[hi], w[r - hi]);
      });
      static_for<R - 1>([&](auto ii) {
        constexpr int r = decltype(ii)::value + 1;
        v[bitrev(r, LOGR)] = cmul(v[bitrev(r, LOGR)], w[r]);
      });
    }
    fft_dit<R, DIR>(v);
    const int d = (j - k) * R + k;
    static_for<R>([&](auto rr) {
      constexpr int r = decltype(rr)::value;
      store(d + r * Ns, v[r]);
    });
  }
}

// A whole L-point transform: `first` supplies the input, `last` consumes the output (natural
// order); b0 / b1 are the padded ping-pong buffers.  Ends with a CTA barrier.
template <int L, int DIR, class First, class Last>
__device__ __forceinline__ void stockham(float2* b0, float2* b1, const float2* Q, First first, Last last) {
  using C = BigCfg<L>;
  auto ld = [](const float2* b) { return [b](int i) { return b[padded(i)]; }; };
  auto st = [](float2* b) { return [b](int i, float2 v) { b[padded(i)] = v; }; };
  static_for<C::P>([&](auto pp) {
    constexpr int p = decltype(pp)::value;
    float2* src = (p % 2 == 1) ? b0 : b1;
    float2* dst = (p % 2 == 0) ? b0 : b1;
    if constexpr (p < C::P16) {
      constexpr int Ns = 1 << (4 * p);
      if constexpr (p == 0) pass_r<L, kRadix, DIR>(Ns, Q, first, st(dst));
      else if constexpr (p == C::P - 1) pass_r<L, kRadix, DIR>(Ns, Q, ld(src), last);
      else pass_r<L, kRadix, DIR>(Ns, Q, ld(src), st(dst));
    } else {
      pass_r<L, 2, DIR>(L / 2, Q, ld(src), last);
    }
    __syncthreads();
  });
}

// The first L/4 entries of the plan's twiddle table into shared memory.
template <int L>
__device__ __forceinline__ void stage_quarter(float2* Q, const float2* twist) {
  for (int u = threadIdx.x; u < L / 4; u += BigCfg<L>::NT) Q[padded(u)] = __ldg(twist + u);
  __syncthreads();
}

template <int L>
__global__ void __launch_bounds__(BigCfg<L>::NT) convolve_big_kernel(const ConvParams p) {
  using C = BigCfg<L>;
  extern __shared__ __align__(16) float2 sbig[];
  float2* X = sbig;
  float2* b0 = sbig + C::BUF;
  float2* b1 = sbig + 2 * C::BUF;
  float2* Q = sbig + 3 * C::BUF;
  stage_quarter<L>(Q, p.twist);
  for (int64_t s = blockIdx.x; s < p.nseg; s += gridDim.x) {
    const int64_t x0 = s * (int64_t)p.V - p.h;
    // a2 + a3: the segment (zeros outside [0, n)), forward transform into X
    stockham<L, -1>(
        b0, b1, Q,
        [&](int i) {
          const int64_t r = x0 + i;
          return (r >= 0 && r < p.n_bins) ? __ldg(p.spectrum + r) : make_float2(0.f, 0.f);
        },
        [&](int i, float2 v) { X[padded(i)] = v; });
    const int64_t segbase = s * (int64_t)p.V;
    const int64_t lim64 = p.n_bins - segbase < (int64_t)p.V ? p.n_bins - segbase : (int64_t)p.V;
    const int lim = (int)lim64;
    for (int z = 0; z < p.Z; ++z) {
      const float2* T = p.templates + (size_t)z * L;
      float* row = p.plane + (size_t)z * p.n_bins + segbase;
      // a4 + a5 + a6 + a7: X*T_z, inverse transform, keep n < V, store |y|^2
      stockham<L, +1>(
          b0, b1, Q, [&](int i) { return cmul(X[padded(i)], __ldg(T + i)); },
          [&](int i, float2 v) {
            if (i < lim) __stcs(row + i, fmaf(v.x, v.x, v.y * v.y));
          });
    }
  }
}

// Forward transforms only (a2 + a3), natural order, for tests of the FFT.
template <int L>
__global__ void __launch_bounds__(BigCfg<L>::NT) segment_spectra_big_kernel(const SegParams p) {
  using C = BigCfg<L>;
  extern __shared__ __align__(16) float2 sbig[];
  float2* b0 = sbig;
  float2* b1 = sbig + C::BUF;
  float2* Q = sbig + 2 * C::BUF;
  stage_quarter<L>(Q, p.twist);
  for (int64_t s = blockIdx.x; s < p.nseg; s += gridDim.x) {
    const int64_t x0 = s * (int64_t)p.V - p.h;
    float2* out = p.out + (size_t)s * L;
    stockham<L, -1>(
        b0, b1, Q,
        [&](int i) {
          const int64_t r = x0 + i;
          return (r >= 0 && r < p.n_bins) ? __ldg(p.spectrum_in + r) : make_float2(0.f, 0.f);
        },
        [&](int i, float2 v) { out[i] = v; });
  }
}

template <int L>
cudaError_t launch_big(const ConvParams& p, int sm_count, cudaStream_t st) {
  using C = BigCfg<L>;
  constexpr size_t smem = (3 * (size_t)C::BUF + padded(L / 4)) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(convolve_big_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, convolve_big_kernel<L>, C::NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t grid = p.nseg < (int64_t)per_sm * sm_count ? p.nseg : (int64_t)per_sm * sm_count;
  convolve_big_kernel<L><<<(unsigned)grid, C::NT, smem, st>>>(p);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_seg_big(const SegParams& p, int sm_count, cudaStream_t st) {
  using C = BigCfg<L>;
  constexpr size_t smem = (2 * (size_t)C::BUF + padded(L / 4)) * sizeof(float2);
  cudaError_t e =
      cudaFuncSetAttribute(segment_spectra_big_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = p.nseg < (int64_t)sm_count ? p.nseg : (int64_t)sm_count;
  segment_spectra_big_kernel<L><<<(unsigned)grid, C::NT, smem, st>>>(p);
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
