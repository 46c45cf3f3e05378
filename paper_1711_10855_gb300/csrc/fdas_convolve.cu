// fdas_convolve.cu -- the fused FDAS correlation kernel for sm_103a.
//
// One launch computes the whole f-fdot power plane (Adamek et al. 2017, Section 1 Eq. 2, by
// the overlap-and-save method of Section 2):
//
//   a2  TMA (cp.async.bulk.tensor, zero fill outside [0, n_bins)) brings each segment's L bins
//       A[s*V - h .. s*V - h + L) into shared memory,
//   a3  forward FFT of the segment, kept in shared memory for all Z templates,
//   a4  for every template z: multiply by the template spectrum T_z (streamed from L2 into a
//       ring of shared-memory slots by bulk copies),
//   a5  inverse FFT,
//   a6  keep outputs n < V (the template is placed so that circular wrap-around lands in the
//       last m outputs),
//   a7  |y|^2 stored with streaming (evict-first) stores into plane[z][s*V + n].
//
// Transform of length L = N1 * N2 by a group of N1 lanes, N2 points per lane (four-step):
//   pass 1: each lane k1 holds Y[k1 + N1*k2], k2 < N2, and does an N2-point DFT in registers,
//   twist:  multiply by exp(SIGN i 2pi n2 k1 / L),
//   exchange through a padded shared-memory tile (C = N2/N1 rounds of N1 x N1),
//   pass 2: lane t holds column n2 = r*N1 + t and does an N1-point DFT in registers; output
//           index n = n2 + N2*n1, so lane t ends with every n = t (mod N1).
// The paper's design (Section 2: shuffle stage for N <= 32, shared memory above) is replaced
// by two register passes and a single shared-memory exchange per transform.
//
// Work decomposition: a CTA of 8 warps owns G consecutive segments at a time ("group"); the
// flattened (group, z) list is split into contiguous equal ranges, one per CTA (grid = #SMs),
// so every CTA does the same number of inverse transforms.  P warps share a segment and take
// alternate templates.
#include <cstdio>

#include "fdas_device.cuh"
#include "fdas_internal.h"

namespace fdas {

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <int L_, int N1_, int P_>
struct ConvCfg {
  static constexpr int L = L_;
  static constexpr int N1 = N1_;
  static constexpr int N2 = L / N1;
  static constexpr int F = 32 / N1;        // transform groups per warp
  static constexpr int W = 8;              // compute warps per CTA
  static constexpr int P = P_;             // warps sharing one segment
  static constexpr int G = F * W / P;      // segments resident per CTA
  static constexpr int R = 4;              // template ring slots
  static constexpr int C = N2 / N1;        // exchange rounds
  static constexpr int LOG_N1 = ilog2(N1);
  static constexpr int LOG_N2 = ilog2(N2);
  static constexpr int TR_PITCH = N1 + 1;  // float2 per exchange-tile row (bank-conflict padding)
  static constexpr int TR_GROUP = N1 * TR_PITCH;
  static constexpr int TR_WARP = F * TR_GROUP;
  static constexpr int BOX = L < 256 ? L : 256;   // TMA box (elements of 8 bytes)
  static constexpr size_t OFF_X = 0;
  static constexpr size_t OFF_T = OFF_X + (size_t)G * L * 8;
  static constexpr size_t OFF_TW = OFF_T + (size_t)R * L * 8;
  static constexpr size_t OFF_TR = OFF_TW + (size_t)L * 8;
  static constexpr size_t OFF_BAR = align_up(OFF_TR + (size_t)W * TR_WARP * 8, 128);
  static constexpr size_t SMEM = OFF_BAR + 256;
  static_assert(N1 * N2 == L && N2 % N1 == 0 && 32 % N1 == 0, "bad decomposition");
  static_assert(L % BOX == 0, "segment must be whole boxes");
  static_assert(SMEM <= 232448, "shared memory budget");
};

// ---------------------------------------------------------------------------------------
// Shared per-lane pieces of the transform
// ---------------------------------------------------------------------------------------

// Element k = k1 + N1*k2 of a segment spectrum / template / twiddle table lives at this
// float2 index of its L-entry buffer (pairs k2 = 2p, 2p+1 of one lane are adjacent: float4).
template <class Cfg>
__device__ __forceinline__ int layout_index(int k1, int k2) {
  return ((k2 >> 1) * Cfg::N1 + k1) * 2 + (k2 & 1);
}

// v[n2] *= tw[n2][k1] (CONJ: by its conjugate), n2 = 1..N2-1.
template <class Cfg, bool CONJ>
__device__ __forceinline__ void apply_twist(float2 (&v)[Cfg::N2], const float2* __restrict__ stw, int k1) {
  static_for<Cfg::N2 / 2>([&](auto pp) {
    constexpr int p = decltype(pp)::value;
    const float4 w = reinterpret_cast<const float4*>(stw)[p * Cfg::N1 + k1];
    if constexpr (p > 0) {
      v[2 * p] = CONJ ? cmul_conj_b(v[2 * p], make_float2(w.x, w.y)) : cmul(v[2 * p], make_float2(w.x, w.y));
    }
    v[2 * p + 1] =
        CONJ ? cmul_conj_b(v[2 * p + 1], make_float2(w.z, w.w)) : cmul(v[2 * p + 1], make_float2(w.z, w.w));
  });
}

// Pass 1 result v[n2] (lane k1) -> exchange -> pass 2 per column; calls out(r, n1, value)
// with the transform's output at n = r*N1 + k1 + N2*n1 held by this lane.
template <class Cfg, int SIGN, class Out>
__device__ __forceinline__ void exchange_and_pass2(float2 (&v)[Cfg::N2], float2* tr, int k1, Out&& out) {
  static_for<Cfg::C>([&](auto rr) {
    constexpr int r = decltype(rr)::value;
    __syncwarp();
    static_for<Cfg::N1>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      tr[i * Cfg::TR_PITCH + k1] = v[r * Cfg::N1 + i];
    });
    __syncwarp();
    float2 u[Cfg::N1];
    static_for<Cfg::N1>([&](auto jj) {
      constexpr int j = decltype(jj)::value;
      u[j] = tr[k1 * Cfg::TR_PITCH + bitrev(j, Cfg::LOG_N1)];
    });
    fft_dit<Cfg::N1, SIGN>(u);
    static_for<Cfg::N1>([&](auto nn) {
      constexpr int n1 = decltype(nn)::value;
      out(std::integral_constant<int, r>{}, std::integral_constant<int, n1>{}, u[n1]);
    });
  });
}

// Forward FFT (Eq. 3) of one segment held in natural order in sx; calls
// out(r, n1, X[r*N1 + k1 + N2*n1]).
template <class Cfg, class Out>
__device__ __forceinline__ void forward_transform(const float2* sx, const float2* __restrict__ stw, float2* tr,
                                                  int k1, Out&& out) {
  float2 v[Cfg::N2];
  static_for<Cfg::N2>([&](auto kk) {
    constexpr int k2 = decltype(kk)::value;
    v[bitrev(k2, Cfg::LOG_N2)] = sx[k1 + Cfg::N1 * k2];
  });
  fft_dit<Cfg::N2, -1>(v);
  apply_twist<Cfg, true>(v, stw, k1);
  exchange_and_pass2<Cfg, -1>(v, tr, k1, out);
}

// Device status word: set bit 0 when a bounded wait gave up.
__device__ __forceinline__ void report_timeout(int* status, volatile int* abort_flag) {
  *abort_flag = 1;
  atomicOr(status, 1);
}

// ---------------------------------------------------------------------------------------
// The fused kernel
// ---------------------------------------------------------------------------------------
template <class Cfg>
__global__ void __launch_bounds__(256, 1)
    fdas_convolve_kernel(const __grid_constant__ CUtensorMap spec_map, const ConvParams p) {
  constexpr int L = Cfg::L, N1 = Cfg::N1, R = Cfg::R, P = Cfg::P, G = Cfg::G;
  extern __shared__ __align__(1024) unsigned char smem[];
  float2* sX = reinterpret_cast<float2*>(smem + Cfg::OFF_X);
  float2* sT = reinterpret_cast<float2*>(smem + Cfg::OFF_T);
  float2* sTw = reinterpret_cast<float2*>(smem + Cfg::OFF_TW);
  float2* sTr = reinterpret_cast<float2*>(smem + Cfg::OFF_TR);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::OFF_BAR);
  uint64_t* segbar = full + R;
  uint64_t* twbar = segbar + 1;
  int64_t* issued_pos = reinterpret_cast<int64_t*>(twbar + 1);   // [R] last position issued per slot
  unsigned* cnt = reinterpret_cast<unsigned*>(issued_pos + R);      // [R] consumer arrivals per slot
  volatile int* abort_flag = reinterpret_cast<volatile int*>(cnt + R);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gw = lane / N1, k1 = lane % N1;
  const int par = warp % P;
  const int seg_slot = (warp / P) * Cfg::F + gw;
  float2* myX = sX + seg_slot * L;
  float2* myTr = sTr + warp * Cfg::TR_WARP + gw * Cfg::TR_GROUP;

  const int64_t U = p.units;
  const int64_t u0 = (int64_t)blockIdx.x * U / gridDim.x;
  const int64_t u1 = ((int64_t)blockIdx.x + 1) * U / gridDim.x;
  const int64_t npos = u1 - u0;
  if (npos <= 0) return;

  if (tid == 0) {
    for (int r = 0; r < R; ++r) {
      mbar_init(&full[r], 1);
      cnt[r] = 0u;
      issued_pos[r] = -1;
    }
    mbar_init(segbar, 1);
    mbar_init(twbar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();

  auto issue_template = [&](int64_t i) {
    const int slot = (int)(i % R);
    const int64_t z = (u0 + i) % p.Z;
    issued_pos[slot] = i;
    mbar_arrive_expect_tx(&full[slot], L * 8);
    bulk_g2s(sT + (size_t)slot * L, p.templates + (size_t)z * L, L * 8, &full[slot]);
  };
  if (tid == 0) {
    mbar_arrive_expect_tx(twbar, L * 8);
    bulk_g2s(sTw, p.twist, L * 8, twbar);
    const int64_t first = npos < R ? npos : R;
    for (int64_t i = 0; i < first; ++i) issue_template(i);
  }
  // `alive` is CTA-uniform: it only changes through __syncthreads_and.
  int alive = __syncthreads_and(mbar_wait(twbar, 0) ? 1 : 0);
  if (!alive && tid == 0) report_timeout(p.status, abort_flag);

  uint32_t seg_phase = 0;
  bool seg_in_flight = false;
  const int64_t g_first = u0 / p.Z, g_last = (u1 - 1) / p.Z;
  for (int64_t grp = g_first; grp <= g_last; ++grp) {
    const int64_t a = (grp * p.Z > u0 ? grp * p.Z : u0) - u0;
    const int64_t b = ((grp + 1) * p.Z < u1 ? (grp + 1) * p.Z : u1) - u0;
    // every warp is done with the previous group's spectra before they are overwritten
    alive = __syncthreads_and(alive && !*abort_flag);
    if (!alive) break;
    if (tid == 0) {
      mbar_arrive_expect_tx(segbar, G * L * 8);
      for (int j = 0; j < G; ++j) {
        const int64_t x0 = (grp * G + j) * (int64_t)p.V - p.h;
        for (int bx = 0; bx < L / Cfg::BOX; ++bx)
          tma_load_1d(sX + (size_t)j * L + bx * Cfg::BOX, &spec_map, (int32_t)(x0 + bx * Cfg::BOX), segbar);
      }
    }
    seg_in_flight = true;
    alive = __syncthreads_and(mbar_wait(segbar, seg_phase) ? 1 : 0);
    if (!alive) {
      if (tid == 0) report_timeout(p.status, abort_flag);
      break;
    }
    seg_in_flight = false;
    seg_phase ^= 1u;
    if (par == 0) {
      // a3: forward FFT in place; X[n] goes to the slot of the inverse transform's first pass
      forward_transform<Cfg>(myX, sTw, myTr, k1, [&](auto rr, auto nn, float2 val) {
        constexpr int k2p = decltype(rr)::value + Cfg::C * decltype(nn)::value;
        myX[layout_index<Cfg>(k1, k2p)] = val;
      });
    }
    __syncthreads();

    const int64_t s = grp * G + seg_slot;
    const int64_t segbase = s * (int64_t)p.V;
    const int64_t lim64 = p.n_bins - segbase < (int64_t)p.V ? p.n_bins - segbase : (int64_t)p.V;
    const int lim = lim64 > 0 ? (int)lim64 : 0;   // outputs n < lim of this segment are stored
    int64_t i = a + (((par - a) % P) + P) % P;
    for (; i < b; i += P) {
      const int slot = (int)(i % R);
      // warp-uniform bounded wait for the template of position i
      int ok = *abort_flag ? 0 : (mbar_wait(&full[slot], (uint32_t)((i / R) & 1)) ? 1 : 0);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) report_timeout(p.status, abort_flag);
        break;
      }
      const int64_t z = (u0 + i) % p.Z;
      const float2* st = sT + (size_t)slot * L;

      // a4: Y = X * T in the first pass's register order (bit-reversed for the DIT)
      float2 v[Cfg::N2];
      static_for<Cfg::N2 / 2>([&](auto pp) {
        constexpr int q = decltype(pp)::value;
        const float4 x = reinterpret_cast<const float4*>(myX)[q * N1 + k1];
        const float4 t = reinterpret_cast<const float4*>(st)[q * N1 + k1];
        v[bitrev(2 * q, Cfg::LOG_N2)] = cmul(make_float2(x.x, x.y), make_float2(t.x, t.y));
        v[bitrev(2 * q + 1, Cfg::LOG_N2)] = cmul(make_float2(x.z, x.w), make_float2(t.z, t.w));
      });
      // release the template slot; the last of the W/P consumers refills it R positions ahead
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        const unsigned old = atomicAdd(&cnt[slot], 1u);
        if ((old + 1u) % (unsigned)(Cfg::W / P) == 0u) {
          __threadfence_block();
          if (i + R < npos) {
            fence_proxy_async_smem();
            issue_template(i + R);
          }
        }
      }
      // a5: inverse FFT
      fft_dit<Cfg::N2, +1>(v);
      apply_twist<Cfg, false>(v, sTw, k1);
      float* row = p.plane + z * p.n_bins + segbase;
      exchange_and_pass2<Cfg, +1>(v, myTr, k1, [&](auto rr, auto nn, float2 y) {
        // a6 + a7: keep n < V (and inside the spectrum), store |y|^2
        const int n = decltype(rr)::value * N1 + k1 + Cfg::N2 * decltype(nn)::value;
        if (n < lim) __stcs(row + n, power(y));
      });
    }
  }

  // After a timeout, wait (bounded) for this CTA's copies still in flight before exiting.
  __syncthreads();
  if (tid == 0 && (*abort_flag || !alive)) {
    for (int r = 0; r < R; ++r)
      if (issued_pos[r] >= 0) (void)mbar_wait(&full[r], (uint32_t)((issued_pos[r] / R) & 1));
    if (seg_in_flight) (void)mbar_wait(segbar, seg_phase);
  }
}

// Forward transforms only (steps a2 + a3), natural-order output, for tests of the FFT.
template <class Cfg>
__global__ void __launch_bounds__(256, 1)
    fdas_segment_spectra_kernel(const __grid_constant__ CUtensorMap spec_map, const SegParams p) {
  constexpr int L = Cfg::L, N1 = Cfg::N1;
  constexpr int GS = 8 * Cfg::F;   // segments per CTA (one per transform group)
  extern __shared__ __align__(1024) unsigned char smem[];
  float2* sX = reinterpret_cast<float2*>(smem);
  float2* sTw = sX + (size_t)GS * L;
  float2* sTr = sTw + L;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + align_up(((size_t)GS * L + L + 8 * Cfg::TR_WARP) * 8, 128));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gw = lane / N1, k1 = lane % N1;
  const int slot = warp * Cfg::F + gw;
  const int64_t s0 = (int64_t)blockIdx.x * GS;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, (GS + 1) * L * 8);
    bulk_g2s(sTw, p.twist, L * 8, bar);
    for (int j = 0; j < GS; ++j) {
      const int64_t x0 = (s0 + j) * (int64_t)p.V - p.h;
      for (int bx = 0; bx < L / Cfg::BOX; ++bx)
        tma_load_1d(sX + (size_t)j * L + bx * Cfg::BOX, &spec_map, (int32_t)(x0 + bx * Cfg::BOX), bar);
    }
  }
  const int ok = __syncthreads_and(mbar_wait(bar, 0) ? 1 : 0);
  if (!ok) {
    if (tid == 0) {
      atomicOr(p.status, 1);
      (void)mbar_wait(bar, 0);   // bounded wait for copies still in flight
    }
    return;
  }
  const int64_t s = s0 + slot;
  float2* dst = p.out + s * L;
  const bool valid = s < p.nseg;
  forward_transform<Cfg>(sX + (size_t)slot * L, sTw, sTr + warp * Cfg::TR_WARP + gw * Cfg::TR_GROUP, k1,
                         [&](auto rr, auto nn, float2 val) {
                           const int n = decltype(rr)::value * N1 + k1 + Cfg::N2 * decltype(nn)::value;
                           if (valid) dst[n] = val;
                         });
}

// ---------------------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------------------
int conv_group_threads(int L) { return L <= 512 ? 16 : 32; }

template <class Cfg>
static cudaError_t launch_conv_cfg(const CUtensorMap* map, const ConvParams& p, int sm_count, cudaStream_t st) {
  auto kern = fdas_convolve_kernel<Cfg>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
  if (e != cudaSuccess) return e;
  ConvParams q = p;
  const int64_t ngroups = (p.nseg + Cfg::G - 1) / Cfg::G;
  q.units = ngroups * p.Z;
  const int64_t grid = q.units < sm_count ? q.units : sm_count;
  kern<<<(unsigned)grid, 256, Cfg::SMEM, st>>>(*map, q);
  return cudaGetLastError();
}

template <class Cfg>
static cudaError_t launch_seg_cfg(const CUtensorMap* map, const SegParams& p, cudaStream_t st) {
  constexpr int GS = 8 * Cfg::F;
  constexpr size_t smem = align_up(((size_t)GS * Cfg::L + Cfg::L + 8 * Cfg::TR_WARP) * 8, 128) + 64;
  auto kern = fdas_segment_spectra_kernel<Cfg>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = (p.nseg + GS - 1) / GS;
  kern<<<(unsigned)grid, 256, smem, st>>>(*map, p);
  return cudaGetLastError();
}

using Cfg256 = ConvCfg<256, 16, 1>;
using Cfg512 = ConvCfg<512, 16, 1>;
using Cfg1024 = ConvCfg<1024, 32, 1>;
using Cfg2048 = ConvCfg<2048, 32, 2>;

cudaError_t launch_convolve(int L, const CUtensorMap* map, const ConvParams& p, int sm_count, cudaStream_t st) {
  switch (L) {
    case 256: return launch_conv_cfg<Cfg256>(map, p, sm_count, st);
    case 512: return launch_conv_cfg<Cfg512>(map, p, sm_count, st);
    case 1024: return launch_conv_cfg<Cfg1024>(map, p, sm_count, st);
    case 2048: return launch_conv_cfg<Cfg2048>(map, p, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_segment_spectra(int L, const CUtensorMap* map, const SegParams& p, int, cudaStream_t st) {
  switch (L) {
    case 256: return launch_seg_cfg<Cfg256>(map, p, st);
    case 512: return launch_seg_cfg<Cfg512>(map, p, st);
    case 1024: return launch_seg_cfg<Cfg1024>(map, p, st);
    case 2048: return launch_seg_cfg<Cfg2048>(map, p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdas
