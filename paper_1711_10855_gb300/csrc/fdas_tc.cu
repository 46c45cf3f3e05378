// fdas_tc.cu -- the correlation (Eq. 2 by overlap-and-save, Section 2) with the inverse segment
// transforms as DFT-matrix contractions on the tensor cores (tcgen05.mma kind::f16, BF16 or FP16
// operands split into hi + lo parts, FP32 accumulation in TMEM), for segment length 2048.
//
// For segment s and template z, Y[k] = X_s[k] T_z[k] and y[n] = sum_k Y[k] exp(+2 pi i k n / L)
// (the 1/L is folded into T).  With k = k1 + 32 k2 and n = n2 + 64 n1 (k1, n1 < 32; k2, n2 < 64):
//   stage 1  Z[n2][k1] = sum_k2 w64^(n2 k2) Y[k1 + 32 k2]      (a 64-point DFT per k1)
//   twist    Z'[n2][k1] = Z[n2][k1] w2048^(k1 n2)
//   stage 2  y[n2 + 64 n1] = sum_k1 Z'[n2][k1] w32^(k1 n1)     (a 32-point DFT per n2)
// Each complex product is one real GEMM on [Re | Im] blocks.  Every operand is split as
// x = hi + lo (hi = round(x), lo = round(x - hi)) and D = A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// One CTA per SM walks units (segment s, 4 templates).  Stage 1: A = W1, the 64-point DFT matrix
// with rows 2 n2 (Re) and 2 n2 + 1 (Im) and K = (Re k2 | Im k2); B = the products Y, rows
// 32 zl + k1 (template zl of the unit), same K; D1 is 128 lanes (n2, Re / Im) by 128 columns
// (zl, k1).  The stage-1 epilogue pairs each Re lane with its Im neighbour by a shuffle, twists,
// and writes A2 (two 128-row tiles: 2 templates x 64 n2, K = (Re k1 | Im k1)) in 16-byte rows.
// Stage 2: A = A2, B = W2 (rows Re n1 | Im n1), D2 columns (Re n1 | Im n1); its epilogue stores
// |y|^2 of the outputs n < V.  Y and A2 have their own shared buffers, so the stage-2 MMAs of a
// unit run while the CTA forms the next unit's Y, and the next stage-1 MMAs while it stores
// the powers.  Operands sit in shared memory in the K-major no-swizzle layout: element (r, k)
// at (k / 8) * lbo + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes.
//
// The forward segment transforms (Eq. 3 sign) use the same kernel with the conjugate matrices
// and twist: Y is the time-domain segment (A[s V - h + j], zero outside [0, n)), a unit is 4
// segments, and the stage-2 epilogue stores the complex spectrum X_s in natural order.
//
// FP16 keeps 5 exponent bits: Y is scaled by 2^-e per segment (inverse: bound = max |X_s| max |T|;
// forward: bound = max |A| over the unit's segments; bound 2^-e in [2^10, 2^11)) and stage-1
// results by 2^-6 (folded into the twist) before they are split; the outputs are scaled back.
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fdas.h"
#include "fdas_internal.h"
#include "fdas_umma.cuh"

namespace fdas {
namespace {

constexpr int kTL = 2048, kTN2 = 64, kTNV = 32, kTZ = 4;   // L = 32 x 64
constexpr int kTcThreads = 512, kTcWarps = kTcThreads / 32;
constexpr int kLbo128 = 16 * 128;   // K-chunk stride of a 128-row matrix
constexpr int kLbo64 = 8 * 128;     // K-chunk stride of a 64-row matrix
// A2 K-chunks 2064 B apart (not 2048): in the stage-1 epilogue's 16-byte stores the Re lanes and
// the Im lanes of a quarter-warp write chunks 4 apart, which then fall in different bank halves
constexpr int kLboA2 = 16 * 128 + 16;
constexpr int kW1Bytes = 128 * 128 * 2, kW2Bytes = 64 * 64 * 2, kYBytes = 128 * 128 * 2, kA2Tile = 8 * kLboA2;
constexpr int kOffW1h = 0, kOffW1l = kOffW1h + kW1Bytes, kOffW2h = kOffW1l + kW1Bytes, kOffW2l = kOffW2h + kW2Bytes;
// twist w2048^(k1 n2) for the k1 pair (2j, 2j+1) at float4 j * 64 + n2: (re, re, im, im)
constexpr int kOffTw = kOffW2l + kW2Bytes;
constexpr int kOffY = kOffTw + kTL * 8;              // Y hi | lo
constexpr int kOffA2 = kOffY + 2 * kYBytes;          // A2 tiles: hi 0, hi 1, lo 0, lo 1
constexpr int kOffMisc = kOffA2 + 4 * kA2Tile;       // mbarriers, TMEM slot, reduction scratch
constexpr int kTcSmem = kOffMisc + 128;
constexpr int kMatBytes = 2 * kW1Bytes + 2 * kW2Bytes;   // W1 hi, W1 lo, W2 hi, W2 lo
static_assert(kTcSmem <= 232448, "shared memory");

__host__ __device__ constexpr int canon(int r, int k, int lbo) {
  return (k >> 3) * lbo + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

template <int PREC>
struct TcType;
template <>
struct TcType<0> {
  using T = __nv_bfloat16;
  using T2 = __nv_bfloat162;
  static constexpr uint32_t fmt = 1;
  __device__ static T cvt(float x) { return __float2bfloat16_rn(x); }
  __device__ static float back(T x) { return __bfloat162float(x); }
  __device__ static T2 cvt2(float2 x) { return __float22bfloat162_rn(x); }
  __device__ static float2 back2(T2 x) { return __bfloat1622float2(x); }
};
template <>
struct TcType<1> {
  using T = __half;
  using T2 = __half2;
  static constexpr uint32_t fmt = 0;
  __device__ static T cvt(float x) { return __float2half_rn(x); }
  __device__ static float back(T x) { return __half2float(x); }
  __device__ static T2 cvt2(float2 x) { return __float22half2_rn(x); }
  __device__ static float2 back2(T2 x) { return __half22float2(x); }
};

// Eight consecutive K elements of one row (16 bytes of a core-matrix row), hi and lo parts.
template <int PREC>
__device__ __forceinline__ void split_store8(unsigned char* hi, unsigned char* lo, int off, const float* x) {
  using TT = TcType<PREC>;
  union {
    typename TT::T2 h[4];
    uint4 u;
  } H, Lo;
#pragma unroll
  for (int j = 0; j < 4; ++j) {   // pairs: packed conversions and a packed subtraction
    const float2 x2 = make_float2(x[2 * j], x[2 * j + 1]);
    H.h[j] = TT::cvt2(x2);
    Lo.h[j] = TT::cvt2(sub2(x2, TT::back2(H.h[j])));
  }
  *reinterpret_cast<uint4*>(hi + off) = H.u;
  *reinterpret_cast<uint4*>(lo + off) = Lo.u;
}

template <int PREC>
__device__ __forceinline__ void split_store1(unsigned char* hi, unsigned char* lo, int off, float x) {
  using TT = TcType<PREC>;
  const typename TT::T h = TT::cvt(x);
  *reinterpret_cast<typename TT::T*>(hi + off) = h;
  *reinterpret_cast<typename TT::T*>(lo + off) = TT::cvt(x - TT::back(h));
}

// e with bound 2^-e in [2^10, 2^11) for a positive finite bound (0 otherwise), clamped to
// [-50, 50] so that the scale 2^-e and the power scale 2^(2 (e + 6)) stay normal FP32 numbers.
__device__ __forceinline__ int fp16_exponent(float bound) {
  if (!(bound > 0.f) || !(bound < 3.0e38f)) return 0;
  const int e = ilogbf(bound) - 10;
  return e < -50 ? -50 : (e > 50 ? 50 : e);
}

__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// DFT matrices in the operand layout (hi and lo), built in FP64, angles 2 pi j / N with j reduced
// mod N and sign d = +1 (inverse) or -1 (forward): W1 rows r = 2 n2 + part (part 0: Re, 1: Im),
// K = 128 (Re k2 | Im k2): row 2 n2 = (cos | -d sin), row 2 n2 + 1 = (d sin | cos) of
// 2 pi n2 k2 / 64; W2 rows n < 64 (Re n1 | Im n1), K = 64 (Re k1 | Im k1): row n1 =
// (cos | -d sin), row 32 + n1 = (d sin | cos) of 2 pi n1 k1 / 32.
template <int PREC, bool FWD>
__global__ void tc_matrices_kernel(unsigned char* mats) {
  constexpr double d = FWD ? -1.0 : 1.0;
  unsigned char* w1h = mats;
  unsigned char* w1l = mats + kW1Bytes;
  unsigned char* w2h = mats + 2 * kW1Bytes;
  unsigned char* w2l = w2h + kW2Bytes;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 128 * 128 + 64 * 64; idx += gridDim.x * blockDim.x) {
    if (idx < 128 * 128) {
      const int r = idx / 128, k = idx % 128;
      const int n2 = r >> 1, im_row = r & 1, k2 = k & 63;
      double sn, cs;
      sincospi(2.0 * (double)((n2 * k2) % 64) / 64.0, &sn, &cs);
      sn *= d;
      const double v = im_row == 0 ? (k < 64 ? cs : -sn) : (k < 64 ? sn : cs);
      split_store1<PREC>(w1h, w1l, canon(r, k, kLbo128), (float)v);
    } else {
      const int j = idx - 128 * 128;
      const int n = j / 64, k = j % 64;
      const int n1 = n % kTNV, k1 = k & 31;
      double sn, cs;
      sincospi(2.0 * (double)((n1 * k1) % 32) / 32.0, &sn, &cs);
      sn *= d;
      const double v = n < kTNV ? (k < 32 ? cs : -sn) : (k < 32 ? sn : cs);
      split_store1<PREC>(w2h, w2l, canon(n, k, kLbo64), (float)v);
    }
  }
}

// Natural-order template bank from the plan's bank (pair-major layout of the N1 = 32
// decomposition, element k = k1 + 32 k2 at float offset ((k2/2) 32 + k1) 4 + k2 % 2, Im +2),
// and max |Re|, |Im| over it (for the FP16 scale; non-negative floats order as unsigned).
__global__ void tc_bank_kernel(const float2* bank, int Z, float2* nat, unsigned* tmax) {
  const int64_t total = (int64_t)Z * kTL;
  unsigned m = 0u;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = idx / kTL;
    const int k = (int)(idx % kTL), k1 = k & 31, k2 = k >> 5;
    const float* f = reinterpret_cast<const float*>(bank + z * kTL);
    const int off = ((k2 >> 1) * 32 + k1) * 4 + (k2 & 1);
    const float2 v = make_float2(f[off], f[off + 2]);
    nat[idx] = v;
    m = max(m, __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y))));
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(tmax, m);
}

template <int PREC, bool FWD>
__global__ void __launch_bounds__(kTcThreads, 1) tc_convolve_kernel(const TcParams p) {
  using TT = TcType<PREC>;
  constexpr uint32_t kIdesc1 = tc_idesc(TT::fmt, 128, 128), kIdesc2 = tc_idesc(TT::fmt, 128, 2 * kTNV);
  extern __shared__ __align__(1024) unsigned char sm[];
  const float4* sTw = reinterpret_cast<const float4*>(sm + kOffTw);
  unsigned char* sY = sm + kOffY;
  unsigned char* sA2 = sm + kOffA2;
  uint64_t* bar1 = reinterpret_cast<uint64_t*>(sm + kOffMisc);        // stage-1 MMAs done
  uint64_t* bar2 = bar1 + 1;                                           // stage-2 MMAs done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffMisc + 16);
  unsigned* sRed = reinterpret_cast<unsigned*>(sm + kOffMisc + 32);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int64_t U = p.units;
  const int64_t u0 = (int64_t)blockIdx.x * U / gridDim.x, u1 = ((int64_t)blockIdx.x + 1) * U / gridDim.x;
  if (u1 <= u0) return;
  // DFT matrices, and the twist in k1 pairs (times 2^-6 for FP16; conjugated for the forward
  // pass), once per CTA
  {
    const uint4* src = reinterpret_cast<const uint4*>(p.mats);
    uint4* dst = reinterpret_cast<uint4*>(sm + kOffW1h);
    for (int i = tid; i < kMatBytes / 16; i += kTcThreads) dst[i] = __ldg(src + i);
    // the plan's table holds w2048^(k1 n2) at float ((n2 % 32) * 32 + k1) * 4 + n2 / 32, Im + 2
    const float* tw = reinterpret_cast<const float*>(p.twist);
    float4* tdst = reinterpret_cast<float4*>(sm + kOffTw);
    const float s2 = PREC == 1 ? 0.015625f : 1.f, s2i = FWD ? -s2 : s2;
    for (int i = tid; i < kTL / 2; i += kTcThreads) {
      const int j = i >> 6, n2 = i & 63;
      const int off0 = ((n2 & 31) * 32 + 2 * j) * 4 + (n2 >> 5), off1 = off0 + 4;   // k1 = 2j, 2j + 1
      tdst[i] = make_float4(__ldg(tw + off0) * s2, __ldg(tw + off1) * s2, __ldg(tw + off0 + 2) * s2i,
                            __ldg(tw + off1 + 2) * s2i);
    }
  }
  if (tid == 0) {
    mbar_init(bar1, 1);
    mbar_init(bar2, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, 256);   // D1: columns 0..127; D2: 128..255 (two 64-column tiles)
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tm = *tslot;
  const uint32_t tm_lane = tm + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t aW1h = smem_u32(sm + kOffW1h), aW1l = smem_u32(sm + kOffW1l);
  const uint32_t aW2h = smem_u32(sm + kOffW2h), aW2l = smem_u32(sm + kOffW2l);
  const uint32_t aY = smem_u32(sY), aA2 = smem_u32(sA2);
  // inverse: unit u = (segment u / CZ, templates 4 (u % CZ) ..); forward: segments 4u .. 4u + 3
  const int CZ = FWD ? 1 : (p.Z + kTZ - 1) / kTZ;
  const float tmax = __uint_as_float(*p.tmax);
  uint32_t ph1 = 0, ph2 = 0;
  bool pend1 = false, pend2 = false;
  bool ok = true;
  int64_t cur_s = -1;
  float s1 = 1.f, post_next = 1.f;

  // FP16: the per-segment scale, when unit u starts a new segment (CTA-uniform; has barriers)
  auto setup = [&](int64_t u) {
    const int64_t s = u / CZ;
    if constexpr (PREC == 1 && FWD) {
      // max |Re|, |Im| over the unit's inputs A[4u V - h .. (4u + 3) V - h + L)
      const int64_t r0 = 4 * u * (int64_t)p.V - p.h;
      const int64_t len = 3 * (int64_t)p.V + kTL;
      unsigned m = 0u;
      for (int64_t i = tid; i < len; i += kTcThreads) {
        const int64_t r = r0 + i;
        if (r >= 0 && r < p.n_bins) {
          const float2 v = __ldg(p.spectrum + r);
          m = max(m, __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y))));
        }
      }
      m = __reduce_max_sync(0xffffffffu, m);
      if (tid == 0) *sRed = 0u;
      __syncthreads();
      if (lane == 0) atomicMax(sRed, m);
      __syncthreads();
      const int e = fp16_exponent(__uint_as_float(*sRed));
      s1 = ldexpf(1.f, -e);
      post_next = ldexpf(1.f, e + 6);
    } else if constexpr (PREC == 1) {
      if (s != cur_s) {
        const float4* xs = reinterpret_cast<const float4*>(p.seg + s * kTL);
        unsigned m = 0u;
        for (int i = tid; i < kTL / 2; i += kTcThreads) {
          const float4 v = __ldg(xs + i);
          m = max(m, __float_as_uint(fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)))));
        }
        m = __reduce_max_sync(0xffffffffu, m);
        if (tid == 0) *sRed = 0u;
        __syncthreads();
        if (lane == 0) atomicMax(sRed, m);
        __syncthreads();
        const int e = fp16_exponent(__uint_as_float(*sRed) * tmax);
        s1 = ldexpf(1.f, -e);
        post_next = ldexpf(1.f, 2 * (e + 6));
      }
    }
    cur_s = s;
  };

  // Y of unit u into the stage-1 B operand: row 32 zl + k1, K = (Re k2 | Im k2); templates
  // beyond Z give zero rows.  A warp task is (zl, eight k2 = 8c..8c+7) with k1 = lane.
  auto form_y = [&](int64_t u) {
    const int64_t s = u / CZ;
    const int z0 = (int)(u % CZ) * kTZ;
    const int nz = FWD ? (p.nseg - 4 * u < kTZ ? (int)(p.nseg - 4 * u) : kTZ) : (p.Z - z0 < kTZ ? p.Z - z0 : kTZ);
    const float2* X = FWD ? nullptr : p.seg + s * kTL;
    for (int task = warp; task < kTZ * 8; task += kTcWarps) {
      const int zl = task >> 3, c = task & 7, k1 = lane;
      float re[8], im[8];
      if (FWD && zl < nz) {
        // segment 4u + zl, time index j = k1 + 32 k2
        const int64_t r0 = (4 * u + zl) * (int64_t)p.V - p.h + k1 + 256 * c;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t r = r0 + 32 * j;
          const float2 a = (r >= 0 && r < p.n_bins) ? __ldg(p.spectrum + r) : make_float2(0.f, 0.f);
          re[j] = a.x;
          im[j] = a.y;
          if constexpr (PREC == 1) {
            re[j] *= s1;
            im[j] *= s1;
          }
        }
      } else if (!FWD && zl < nz) {
        const float2* T = p.bank + (size_t)(z0 + zl) * kTL;
        float2 t[8], x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          t[j] = __ldg(T + k1 + 32 * (8 * c + j));
          x[j] = __ldg(X + k1 + 32 * (8 * c + j));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          re[j] = fmaf(x[j].x, t[j].x, -x[j].y * t[j].y);
          im[j] = fmaf(x[j].x, t[j].y, x[j].y * t[j].x);
          if constexpr (PREC == 1) {
            re[j] *= s1;
            im[j] *= s1;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) re[j] = im[j] = 0.f;
      }
      const int row = 32 * zl + k1;
      split_store8<PREC>(sY, sY + kYBytes, canon(row, 8 * c, kLbo128), re);
      split_store8<PREC>(sY, sY + kYBytes, canon(row, 64 + 8 * c, kLbo128), im);
    }
  };

  auto sync_for_mma = [&]() {
    fence_proxy_async_smem();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
  };

  auto issue_stage1 = [&]() {
    if (tid == 0) {
      const uint64_t ah = umma_desc(aW1h, kLbo128, 128), al = umma_desc(aW1l, kLbo128, 128);
      const uint64_t bh = umma_desc(aY, kLbo128, 128), bl = umma_desc(aY + kYBytes, kLbo128, 128);
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const uint64_t o = (uint64_t)((ks * 2 * kLbo128) >> 4);
        umma_f16(tm, ah + o, bh + o, kIdesc1, ks > 0 ? 1u : 0u);
        umma_f16(tm, ah + o, bl + o, kIdesc1, 1u);
        umma_f16(tm, al + o, bh + o, kIdesc1, 1u);
      }
      umma_commit(bar1);
    }
    pend1 = true;
  };

  auto issue_stage2 = [&](int ntiles) {
    if (tid == 0) {
      const uint64_t bh = umma_desc(aW2h, kLbo64, 128), bl = umma_desc(aW2l, kLbo64, 128);
      for (int t = 0; t < ntiles; ++t) {
        const uint64_t ah = umma_desc(aA2 + t * kA2Tile, kLboA2, 128);
        const uint64_t al = umma_desc(aA2 + (2 + t) * kA2Tile, kLboA2, 128);
        const uint32_t d = tm + 128 + 64 * t;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t oa = (uint64_t)((ks * 2 * kLboA2) >> 4), ob = (uint64_t)((ks * 2 * kLbo64) >> 4);
          umma_f16(d, ah + oa, bh + ob, kIdesc2, ks > 0 ? 1u : 0u);
          umma_f16(d, ah + oa, bl + ob, kIdesc2, 1u);
          umma_f16(d, al + oa, bh + ob, kIdesc2, 1u);
        }
      }
      umma_commit(bar2);
    }
    pend2 = true;
  };

  // bounded wait on a commit barrier (one polling thread), then a CTA barrier
  auto wait_bar = [&](uint64_t* bar, uint32_t& ph, bool& pend) -> bool {
    const int good = __syncthreads_and(tid == 0 ? (mbar_wait(bar, ph) ? 1 : 0) : 1);
    tmem_fence_after_sync();
    if (good) {
      ph ^= 1u;
      pend = false;
    }
    return good != 0;
  };

  // stage-1 epilogue: warp (quadrant q, template zl = warp / 4): lane = (n2 = 16 q + lane / 2,
  // part = lane % 2), 32 columns k1.  The Re lane sends Re Z and receives -Im Z from its Im
  // neighbour, which sends -Im Z and receives Re Z:
  //   Re Z' = Re Z tw.re + (-Im Z) tw.im,  Im Z' = Im Z tw.re + Re Z tw.im.
  auto epilogue1 = [&](int nz) {
    const int q = warp & 3, zl = warp >> 2;
    const int n2 = 16 * q + (lane >> 1), part = lane & 1;
    float o[32];
    if (zl < nz) {
      float v[32];
      tmem_ld16(tm_lane + 32 * zl, *reinterpret_cast<float(*)[16]>(v));
      tmem_ld16(tm_lane + 32 * zl + 16, *reinterpret_cast<float(*)[16]>(v + 16));
      tmem_wait_ld();
      const float send = part ? -1.f : 1.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {   // k1 = 2j, 2j + 1 as packed pairs
        const float2 v2 = make_float2(v[2 * j], v[2 * j + 1]);
        const float2 sv = mul2(v2, make_float2(send, send));
        const float2 w2 = make_float2(__shfl_xor_sync(0xffffffffu, sv.x, 1), __shfl_xor_sync(0xffffffffu, sv.y, 1));
        const float4 tw = sTw[j * 64 + n2];
        const float2 o2 = fma2(w2, make_float2(tw.z, tw.w), mul2(v2, make_float2(tw.x, tw.y)));
        o[2 * j] = o2.x;
        o[2 * j + 1] = o2.y;
      }
    } else {
#pragma unroll
      for (int k1 = 0; k1 < 32; ++k1) o[k1] = 0.f;
    }
    const int row2 = 64 * (zl & 1) + n2;
    unsigned char* hi = sA2 + (zl >> 1) * kA2Tile;
    unsigned char* lo = sA2 + (2 + (zl >> 1)) * kA2Tile;
#pragma unroll
    for (int c = 0; c < 4; ++c) split_store8<PREC>(hi, lo, canon(row2, 32 * part + 8 * c, kLboA2), o + 8 * c);
  };

  // stage-2 epilogue: warp (half g of n1, tile t, quadrant q): template 2t + q/2,
  // n2 = 32 (q % 2) + lane, n1 = 16 g .. 16 g + 15
  auto epilogue2 = [&](int64_t u, int nz, float post) {
    const int64_t s = u / CZ;
    const int z0 = (int)(u % CZ) * kTZ;
    const int g = warp >> 3, t = (warp >> 2) & 1, q = warp & 3;
    const int zl = 2 * t + (q >> 1), n2 = 32 * (q & 1) + lane;
    if (FWD && zl < nz) {
      float re[16], im[16];
      const uint32_t col = tm_lane + 128 + 64 * t + 16 * g;
      tmem_ld16(col, re);
      tmem_ld16(col + 32, im);
      tmem_wait_ld();
      float2* out = p.seg_out + (4 * u + zl) * kTL;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float2 v = make_float2(re[j], im[j]);
        if constexpr (PREC == 1) v = make_float2(v.x * post, v.y * post);
        out[n2 + kTN2 * (16 * g + j)] = v;
      }
    } else if (!FWD && zl < nz) {
      float re[16], im[16];
      const uint32_t col = tm_lane + 128 + 64 * t + 16 * g;   // Re y(n1) at n1, Im y(n1) at 32 + n1
      tmem_ld16(col, re);
      tmem_ld16(col + 32, im);
      tmem_wait_ld();
      float* row = p.plane + (size_t)(z0 + zl) * p.n_bins + s * (int64_t)p.V;
      const int64_t lim64 = p.n_bins - s * (int64_t)p.V < (int64_t)p.V ? p.n_bins - s * (int64_t)p.V : (int64_t)p.V;
#pragma unroll
      for (int j = 0; j < 16; j += 2) {   // n1 pairs: packed |y|^2
        const float2 r2 = make_float2(re[j], re[j + 1]), i2 = make_float2(im[j], im[j + 1]);
        float2 pw = fma2(r2, r2, mul2(i2, i2));
        if constexpr (PREC == 1) pw = mul2(pw, make_float2(post, post));
        const int n = n2 + kTN2 * (16 * g + j);
        if (n < lim64) __stcs(row + n, pw.x);
        if (n + kTN2 < lim64) __stcs(row + n + kTN2, pw.y);
      }
    }
  };

  // software pipeline: stage 2 of unit u runs while Y of unit u + 1 is formed, and stage 1 of
  // unit u + 1 while the powers of unit u are stored
  setup(u0);
  form_y(u0);
  float post_cur = post_next;
  sync_for_mma();
  issue_stage1();
  for (int64_t u = u0; u < u1; ++u) {
    const int z0 = (int)(u % CZ) * kTZ;
    const int nz = FWD ? (p.nseg - 4 * u < kTZ ? (int)(p.nseg - 4 * u) : kTZ) : (p.Z - z0 < kTZ ? p.Z - z0 : kTZ);
    if (!(ok = wait_bar(bar1, ph1, pend1))) break;
    epilogue1(nz);
    sync_for_mma();
    issue_stage2((nz + 1) / 2);
    const float post_u = post_cur;
    if (u + 1 < u1) {
      setup(u + 1);
      form_y(u + 1);
      post_cur = post_next;
      sync_for_mma();
      issue_stage1();
    }
    if (!(ok = wait_bar(bar2, ph2, pend2))) break;
    epilogue2(u, nz, post_u);
    tmem_fence_before_sync();
  }
  if (!ok && tid == 0) {
    atomicOr(p.status, 1);
    // bounded waits for the MMAs still in flight
    if (pend1) (void)mbar_wait(bar1, ph1);
    if (pend2) (void)mbar_wait(bar2, ph2);
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tm, 256);
}

}  // namespace

int tc_matrices_bytes() { return kMatBytes; }

cudaError_t launch_tc_prepare(const float2* bank, int Z, float2* nat, unsigned* tmax, unsigned char* mats,
                              cudaStream_t st) {
  if (cudaMemsetAsync(tmax, 0, sizeof(unsigned), st) != cudaSuccess) return cudaGetLastError();
  tc_bank_kernel<<<1024, 256, 0, st>>>(bank, Z, nat, tmax);
  tc_matrices_kernel<0, false><<<80, 256, 0, st>>>(mats);
  tc_matrices_kernel<1, false><<<80, 256, 0, st>>>(mats + kMatBytes);
  tc_matrices_kernel<0, true><<<80, 256, 0, st>>>(mats + 2 * kMatBytes);
  tc_matrices_kernel<1, true><<<80, 256, 0, st>>>(mats + 3 * kMatBytes);
  return cudaGetLastError();
}

cudaError_t launch_tc(const TcParams& p, int precision, bool forward, int sm_count, cudaStream_t st) {
  auto kern = forward ? (precision == 1 ? tc_convolve_kernel<1, true> : tc_convolve_kernel<0, true>)
                      : (precision == 1 ? tc_convolve_kernel<1, false> : tc_convolve_kernel<0, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e != cudaSuccess) return e;
  const int64_t grid = p.units < sm_count ? p.units : sm_count;
  kern<<<(unsigned)grid, kTcThreads, kTcSmem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace fdas
