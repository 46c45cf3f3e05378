// fdas_tc.cu -- the correlation (Eq. 2 by overlap-and-save, Section 2) with the inverse segment
// transforms as DFT-matrix contractions on the tensor cores (tcgen05.mma kind::f16, BF16 or FP16
// operands split into hi + lo parts, FP32 accumulation in TMEM), for segment length 2048.
//
// For segment s and template z, Y[k] = X_s[k] T_z[k] and y[n] = sum_k Y[k] exp(+2 pi i k n / L)
// (the 1/L is folded into T).  With k = k1 + 32 k2 and n = n2 + 64 n1 (k1, n1 < 32; k2, n2 < 64):
//   stage 1  Z[k1][n2] = sum_k2 Y[k1 + 32 k2] w64^(k2 n2)      (a 64-point DFT per k1)
//   twist    Z'[k1][n2] = Z[k1][n2] w2048^(k1 n2)
//   stage 2  y[n2 + 64 n1] = sum_k1 Z'[k1][n2] w32^(k1 n1)     (a 32-point DFT per n2)
// Each complex product is one real GEMM on [Re | Im] blocks: rows of A are [Re x | Im x], rows of
// B^T are [cos | -sin] and [sin | cos] of the DFT matrix.  Every operand is split as
// x = hi + lo (hi = round(x), lo = round(x - hi)) and D = A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// One CTA per SM walks units (segment s, 4 templates): A1 = 4 templates x 32 k1 = 128 rows by
// K = 128, B1 = 128 x 128 (N = [Re | Im] of n2); the stage-1 epilogue applies the twist and
// writes A2 as two 128-row tiles (2 templates x 64 n2) by K = 64; stage 2 has N = 64 (Re and Im
// of n1 < 32).  The stage-2 epilogue stores |y|^2 of the outputs n < V.  Operands sit in
// shared memory in the K-major no-swizzle layout: element (r, k) of a matrix with R rows at
// (k / 8) * (R / 8) * 128 + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes.
//
// FP16 keeps 5 exponent bits: Y is scaled by 2^-e per segment (max |X_s| max |T| 2^-e <= 2^11)
// and stage-1 results by 2^-6 before they are split; the powers are scaled back.
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
constexpr int kB1Bytes = 128 * 128 * 2, kB2Bytes = 64 * 64 * 2, kA1Bytes = 128 * 128 * 2, kA2Tile = 128 * 64 * 2;
constexpr int kLbo128 = 16 * 128;   // K-chunk stride of a 128-row matrix
constexpr int kLbo64 = 8 * 128;     // K-chunk stride of a 64-row matrix
constexpr int kOffB1h = 0, kOffB1l = kOffB1h + kB1Bytes, kOffB2h = kOffB1l + kB1Bytes, kOffB2l = kOffB2h + kB2Bytes;
constexpr int kOffX = kOffB2l + kB2Bytes;            // 2048 float2
constexpr int kOffTw = kOffX + kTL * 8;              // the plan's twist table (2048 float2)
constexpr int kOffA = kOffTw + kTL * 8;              // A1 hi | lo, later A2 tiles hi | lo
constexpr int kOffMisc = kOffA + 2 * kA1Bytes;       // mbarrier, TMEM slot, reduction scratch
constexpr int kTcSmem = kOffMisc + 128;
constexpr int kMatBytes = 2 * kB1Bytes + 2 * kB2Bytes;   // B1 hi, B1 lo, B2 hi, B2 lo
static_assert(2 * kA2Tile * 2 <= 2 * kA1Bytes, "A2 tiles must fit in the A1 area");
static_assert(kTcSmem <= 227 * 1024, "shared memory");

__host__ __device__ constexpr int canon(int r, int k, int lbo) {
  return (k >> 3) * lbo + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

template <int PREC>
struct TcType;
template <>
struct TcType<0> {
  using T = __nv_bfloat16;
  static constexpr uint32_t fmt = 1;
  __device__ static T cvt(float x) { return __float2bfloat16_rn(x); }
  __device__ static float back(T x) { return __bfloat162float(x); }
};
template <>
struct TcType<1> {
  using T = __half;
  static constexpr uint32_t fmt = 0;
  __device__ static T cvt(float x) { return __float2half_rn(x); }
  __device__ static float back(T x) { return __half2float(x); }
};

template <int PREC>
__device__ __forceinline__ void split_store(unsigned char* hi, unsigned char* lo, int off, float x) {
  using TT = TcType<PREC>;
  const typename TT::T h = TT::cvt(x);
  *reinterpret_cast<typename TT::T*>(hi + off) = h;
  *reinterpret_cast<typename TT::T*>(lo + off) = TT::cvt(x - TT::back(h));
}

__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// DFT matrices in the operand layout (hi and lo), built in FP64: B1 rows n < 128 (Re n2 | Im n2),
// K = 128 (Re k2 | Im k2); B2 rows n < 64 (Re n1 | Im n1), K = 64 (Re k1 | Im k1).
template <int PREC>
__global__ void tc_matrices_kernel(unsigned char* mats) {
  unsigned char* b1h = mats;
  unsigned char* b1l = mats + kB1Bytes;
  unsigned char* b2h = mats + 2 * kB1Bytes;
  unsigned char* b2l = b2h + kB2Bytes;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 128 * 128 + 64 * 64; idx += gridDim.x * blockDim.x) {
    if (idx < 128 * 128) {
      const int n = idx / 128, k = idx % 128;
      const int n2 = n & 63, k2 = k & 63;
      double sn, cs;
      sincospi(2.0 * (double)((n2 * k2) % 64) / 64.0, &sn, &cs);
      const double v = n < 64 ? (k < 64 ? cs : -sn) : (k < 64 ? sn : cs);
      split_store<PREC>(b1h, b1l, canon(n, k, kLbo128), (float)v);
    } else {
      const int j = idx - 128 * 128;
      const int n = j / 64, k = j % 64;
      const int n1 = n % kTNV, k1 = k & 31;
      double sn, cs;
      sincospi(2.0 * (double)((n1 * k1) % 32) / 32.0, &sn, &cs);
      const double v = n < kTNV ? (k < 32 ? cs : -sn) : (k < 32 ? sn : cs);
      split_store<PREC>(b2h, b2l, canon(n, k, kLbo64), (float)v);
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

template <int PREC>
__global__ void __launch_bounds__(256, 1) tc_convolve_kernel(const TcParams p) {
  using TT = TcType<PREC>;
  constexpr uint32_t kIdesc1 = tc_idesc(TT::fmt, 128, 128), kIdesc2 = tc_idesc(TT::fmt, 128, 2 * kTNV);
  extern __shared__ __align__(1024) unsigned char sm[];
  float2* sX = reinterpret_cast<float2*>(sm + kOffX);
  const float* sTw = reinterpret_cast<const float*>(sm + kOffTw);
  unsigned char* sA = sm + kOffA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffMisc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffMisc + 8);
  unsigned* sRed = reinterpret_cast<unsigned*>(sm + kOffMisc + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int64_t U = p.units;
  const int64_t u0 = (int64_t)blockIdx.x * U / gridDim.x, u1 = ((int64_t)blockIdx.x + 1) * U / gridDim.x;
  if (u1 <= u0) return;
  // DFT matrices and the twist table, once per CTA
  {
    const uint4* src = reinterpret_cast<const uint4*>(p.mats);
    uint4* dst = reinterpret_cast<uint4*>(sm + kOffB1h);
    for (int i = tid; i < kMatBytes / 16; i += 256) dst[i] = __ldg(src + i);
    const float4* tw = reinterpret_cast<const float4*>(p.twist);
    float4* tdst = reinterpret_cast<float4*>(sm + kOffTw);
    for (int i = tid; i < kTL / 2; i += 256) tdst[i] = __ldg(tw + i);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, 256);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tm = *tslot;
  const uint32_t tm_lane = tm + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t aB1h = smem_u32(sm + kOffB1h), aB1l = smem_u32(sm + kOffB1l);
  const uint32_t aB2h = smem_u32(sm + kOffB2h), aB2l = smem_u32(sm + kOffB2l);
  const uint32_t aA = smem_u32(sA);
  const int CZ = (p.Z + kTZ - 1) / kTZ;
  const float tmax = __uint_as_float(*p.tmax);
  uint32_t phase = 0;
  bool ok = true;
  int64_t cur_s = -1;
  float s1 = 1.f, post = 1.f;
  const float s2 = PREC == 1 ? 0.015625f : 1.f;   // 2^-6 before the stage-2 split (FP16)

  auto wait_mma = [&]() -> bool {
    const int good = __syncthreads_and(tid == 0 ? (mbar_wait(bar, phase) ? 1 : 0) : 1);
    phase ^= 1u;
    tmem_fence_after_sync();
    return good != 0;
  };

  for (int64_t u = u0; u < u1 && ok; ++u) {
    const int64_t s = u / CZ;
    const int z0 = (int)(u % CZ) * kTZ;
    const int nz = p.Z - z0 < kTZ ? p.Z - z0 : kTZ;
    if (s != cur_s) {
      const float4* xs = reinterpret_cast<const float4*>(p.seg + s * kTL);
      float4* xd = reinterpret_cast<float4*>(sX);
      unsigned m = 0u;
      for (int i = tid; i < kTL / 2; i += 256) {
        const float4 v = __ldg(xs + i);
        xd[i] = v;
        m = max(m, __float_as_uint(fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)))));
      }
      if (PREC == 1) {
        m = __reduce_max_sync(0xffffffffu, m);
        if (tid == 0) *sRed = 0u;
        __syncthreads();
        if (lane == 0) atomicMax(sRed, m);
        __syncthreads();
        // 2^-e with max|X| max|T| 2^-e <= 2^11
        const float bound = __uint_as_float(*sRed) * tmax;
        int e = 0;
        if (bound > 2048.f) e = ilogbf(bound) - 10;
        s1 = ldexpf(1.f, -e);
        post = ldexpf(1.f, 2 * (e + 6));
      }
      cur_s = s;
      __syncthreads();
    }
    // A1: row 32 zl + k1, K = (Re k2 | Im k2); templates beyond Z give zero rows
    for (int idx = tid; idx < kTZ * kTL; idx += 256) {
      const int zl = idx / kTL, k = idx % kTL, k1 = k & 31, k2 = k >> 5;
      float2 y = make_float2(0.f, 0.f);
      if (zl < nz) {
        const float2 t = __ldg(p.bank + (size_t)(z0 + zl) * kTL + k);
        const float2 x = sX[k];
        y = make_float2(fmaf(x.x, t.x, -x.y * t.y) * s1, fmaf(x.x, t.y, x.y * t.x) * s1);
      }
      const int row = 32 * zl + k1;
      split_store<PREC>(sA, sA + kA1Bytes, canon(row, k2, kLbo128), y.x);
      split_store<PREC>(sA, sA + kA1Bytes, canon(row, 64 + k2, kLbo128), y.y);
    }
    fence_proxy_async_smem();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (tid == 0) {
      const uint64_t ah = umma_desc(aA, kLbo128, 128), al = umma_desc(aA + kA1Bytes, kLbo128, 128);
      const uint64_t bh = umma_desc(aB1h, kLbo128, 128), bl = umma_desc(aB1l, kLbo128, 128);
      for (int ks = 0; ks < 8; ++ks) {
        const uint64_t o = (uint64_t)((ks * 2 * kLbo128) >> 4);
        umma_f16(tm, ah + o, bh + o, kIdesc1, ks > 0 ? 1u : 0u);
        umma_f16(tm, ah + o, bl + o, kIdesc1, 1u);
        umma_f16(tm, al + o, bh + o, kIdesc1, 1u);
      }
      umma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    // stage-1 epilogue: warp (quadrant q = template zl, half h of n2); twist, split into A2
    {
      const int zl = warp & 3, h = warp >> 2, k1 = lane;
      unsigned char* a2h = sA + (zl >> 1) * kA2Tile;
      unsigned char* a2l = sA + 2 * kA2Tile + (zl >> 1) * kA2Tile;
      for (int c = 0; c < 2; ++c) {
        const int nb = 32 * h + 16 * c;
        float re[16], im[16];
        tmem_ld16(tm_lane + nb, re);
        tmem_ld16(tm_lane + 64 + nb, im);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n2 = nb + j;
          const int toff = ((n2 & 31) * 32 + k1) * 4 + (n2 >> 5);
          const float twr = sTw[toff], twi = sTw[toff + 2];
          float zr = fmaf(re[j], twr, -im[j] * twi) * s2, zi = fmaf(re[j], twi, im[j] * twr) * s2;
          if (zl >= nz) zr = zi = 0.f;
          const int row2 = 64 * (zl & 1) + n2;
          split_store<PREC>(a2h, a2l, canon(row2, k1, kLbo128), zr);
          split_store<PREC>(a2h, a2l, canon(row2, 32 + k1, kLbo128), zi);
        }
      }
    }
    fence_proxy_async_smem();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const int ntiles = (nz + 1) / 2;
    if (tid == 0) {
      const uint64_t bh = umma_desc(aB2h, kLbo64, 128), bl = umma_desc(aB2l, kLbo64, 128);
      for (int t = 0; t < ntiles; ++t) {
        const uint64_t ah = umma_desc(aA + t * kA2Tile, kLbo128, 128);
        const uint64_t al = umma_desc(aA + 2 * kA2Tile + t * kA2Tile, kLbo128, 128);
        const uint32_t d = tm + 128 + 64 * t;
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t oa = (uint64_t)((ks * 2 * kLbo128) >> 4), ob = (uint64_t)((ks * 2 * kLbo64) >> 4);
          umma_f16(d, ah + oa, bh + ob, kIdesc2, ks > 0 ? 1u : 0u);
          umma_f16(d, ah + oa, bl + ob, kIdesc2, 1u);
          umma_f16(d, al + oa, bh + ob, kIdesc2, 1u);
        }
      }
      umma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    // stage-2 epilogue: warp (tile t, quadrant q): template 2t + q/2, n2 = 32 (q % 2) + lane
    {
      const int t = warp >> 2, q = warp & 3;
      const int zl = 2 * t + (q >> 1), n2 = 32 * (q & 1) + lane;
      if (t < ntiles) {
        float re[32], im[32];
        const uint32_t col = tm_lane + 128 + 64 * t;   // columns: Re y(n1) at n1, Im y(n1) at 32 + n1
        tmem_ld16(col, *reinterpret_cast<float(*)[16]>(re));
        tmem_ld16(col + 16, *reinterpret_cast<float(*)[16]>(re + 16));
        tmem_ld16(col + 32, *reinterpret_cast<float(*)[16]>(im));
        tmem_ld16(col + 48, *reinterpret_cast<float(*)[16]>(im + 16));
        tmem_wait_ld();
        if (zl < nz) {
          float* row = p.plane + (size_t)(z0 + zl) * p.n_bins + s * (int64_t)p.V;
          const int64_t lim64 = p.n_bins - s * (int64_t)p.V < (int64_t)p.V ? p.n_bins - s * (int64_t)p.V : (int64_t)p.V;
#pragma unroll
          for (int n1 = 0; n1 < kTNV; ++n1) {
            const int n = n2 + kTN2 * n1;
            if (n < lim64) __stcs(row + n, fmaf(re[n1], re[n1], im[n1] * im[n1]) * post);
          }
        }
      }
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
  }
  if (!ok && tid == 0) {
    atomicOr(p.status, 1);
    (void)mbar_wait(bar, phase ^ 1u);   // bounded wait for the MMAs still in flight
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tm, 256);
}

}  // namespace

int tc_matrices_bytes() { return kMatBytes; }

cudaError_t launch_tc_prepare(const float2* bank, int Z, float2* nat, unsigned* tmax, unsigned char* mats_bf16,
                              unsigned char* mats_fp16, cudaStream_t st) {
  if (cudaMemsetAsync(tmax, 0, sizeof(unsigned), st) != cudaSuccess) return cudaGetLastError();
  tc_bank_kernel<<<1024, 256, 0, st>>>(bank, Z, nat, tmax);
  tc_matrices_kernel<0><<<80, 256, 0, st>>>(mats_bf16);
  tc_matrices_kernel<1><<<80, 256, 0, st>>>(mats_fp16);
  return cudaGetLastError();
}

cudaError_t launch_tc(const TcParams& p, int precision, int sm_count, cudaStream_t st) {
  auto kern = precision == 1 ? tc_convolve_kernel<1> : tc_convolve_kernel<0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e != cudaSuccess) return e;
  const int64_t grid = p.units < sm_count ? p.units : sm_count;
  kern<<<(unsigned)grid, 256, kTcSmem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace fdas
