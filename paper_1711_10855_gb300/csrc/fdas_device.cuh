// fdas_device.cuh -- device building blocks of the fused FDAS kernel (sm_103a).
//
//  * compile-time twiddle factors (cos/sin of 2*pi*j/M from a Taylor series on [0, pi/4]),
//  * an in-register radix-2 decimation-in-time FFT whose butterflies are written as fused
//    multiply-adds (the rotation w*b is c*(b + i*t*b) with t = tan or cot of the angle, so a
//    butterfly with a non-trivial twiddle is 6 FMAs and one with w in {1, +-i} is 4 adds),
//  * mbarrier / bulk-copy (TMA) wrappers whose waits are bounded in time.
//
// The DFT sign follows Eq. 3 of Adamek et al. 2017: forward X_m = sum_n x_n e^{-i2pi nm/N}
// (SIGN = -1); the inverse transform used after the template multiply has SIGN = +1 and no
// 1/N (the 1/L is folded into the stored template spectra).
#pragma once

#include <cstdint>
#include <utility>

#include <cuda_runtime.h>

namespace fdas {

// ---------------------------------------------------------------------------------------
// Compile-time trigonometry
// ---------------------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double taylor_sin(double x) {   // |x| <= pi/4
  double x2 = x * x, term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / (double)((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {   // |x| <= pi/4
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / (double)((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}

struct CosSin {
  double c, s;
};

// cos and sin of 2*pi*j/M for integer j and M a power of two, with the quadrant and the
// octant reduced exactly in integers.
__host__ __device__ constexpr CosSin cossin_2pi(long long j, long long M) {
  j %= M;
  if (j < 0) j += M;
  if (M == 1) return {1.0, 0.0};
  if (M == 2) return j == 0 ? CosSin{1.0, 0.0} : CosSin{-1.0, 0.0};
  const long long q = (4 * j) / M;        // quadrant
  const long long r = 4 * j - q * M;      // angle within the quadrant = (pi/2) * r / M
  double c = 0.0, s = 0.0;
  if (2 * r <= M) {
    const double phi = (kPi / 2.0) * (double)r / (double)M;
    c = taylor_cos(phi);
    s = taylor_sin(phi);
  } else {
    const double phi = (kPi / 2.0) * (double)(M - r) / (double)M;
    c = taylor_sin(phi);
    s = taylor_cos(phi);
  }
  switch (q) {
    case 0: return {c, s};
    case 1: return {-s, c};
    case 2: return {-c, -s};
    default: return {s, -c};
  }
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr double cabsd(double x) { return x < 0 ? -x : x; }

// ---------------------------------------------------------------------------------------
// Compile-time loops
// ---------------------------------------------------------------------------------------
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------------------
// Complex helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul_conj_b(float2 a, float2 b) {   // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float power(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// ---------------------------------------------------------------------------------------
// Radix-2 DIT butterfly a' = a + w b, b' = a - w b with w = exp(SIGN * i * 2*pi*J/M)
// ---------------------------------------------------------------------------------------
template <int J, int M, int SIGN>
__device__ __forceinline__ void butterfly(float2& a, float2& b) {
  constexpr CosSin cs = cossin_2pi(J, M);
  constexpr double wc = cs.c;
  constexpr double ws = SIGN * cs.s;
  if constexpr (J == 0) {
    const float2 t = a;
    a = make_float2(t.x + b.x, t.y + b.y);
    b = make_float2(t.x - b.x, t.y - b.y);
  } else if constexpr (4 * J == M) {
    // w = SIGN * i:  w*b = SIGN * (-b.y, b.x)
    const float2 t = a;
    if constexpr (SIGN > 0) {
      a = make_float2(t.x - b.y, t.y + b.x);
      b = make_float2(t.x + b.y, t.y - b.x);
    } else {
      a = make_float2(t.x + b.y, t.y - b.x);
      b = make_float2(t.x - b.y, t.y + b.x);
    }
  } else if constexpr (cabsd(wc) >= cabsd(ws)) {
    // w*b = c * (b.x - t b.y, b.y + t b.x), t = tan
    constexpr float t = (float)(ws / wc);
    constexpr float c = (float)wc;
    const float ur = fmaf(-t, b.y, b.x);
    const float ui = fmaf(t, b.x, b.y);
    const float2 s = a;
    a = make_float2(fmaf(c, ur, s.x), fmaf(c, ui, s.y));
    b = make_float2(fmaf(-c, ur, s.x), fmaf(-c, ui, s.y));
  } else {
    // w*b = s * (ct b.x - b.y, ct b.y + b.x), ct = cot
    constexpr float ct = (float)(wc / ws);
    constexpr float sn = (float)ws;
    const float ur = fmaf(ct, b.x, -b.y);
    const float ui = fmaf(ct, b.y, b.x);
    const float2 s = a;
    a = make_float2(fmaf(sn, ur, s.x), fmaf(sn, ui, s.y));
    b = make_float2(fmaf(-sn, ur, s.x), fmaf(-sn, ui, s.y));
  }
}

template <int N, int SIGN, int S, int I>
__device__ __forceinline__ void stage_butterfly(float2 (&v)[N]) {
  constexpr int span = 1 << S;
  constexpr int blk = (I / span) * (2 * span);
  constexpr int j = I % span;
  butterfly<j, 2 * span, SIGN>(v[blk + j], v[blk + j + span]);
}
template <int N, int SIGN, int S, int... I>
__device__ __forceinline__ void fft_stage(float2 (&v)[N], std::integer_sequence<int, I...>) {
  (stage_butterfly<N, SIGN, S, I>(v), ...);
}
template <int N, int SIGN, int... S>
__device__ __forceinline__ void fft_stages(float2 (&v)[N], std::integer_sequence<int, S...>) {
  (fft_stage<N, SIGN, S>(v, std::make_integer_sequence<int, N / 2>{}), ...);
}

// In-register DFT of N points: on entry v[i] = x[bitrev(i)], on exit v[m] = X[m] =
// sum_n x[n] exp(SIGN * i * 2*pi*n*m/N)  (Eq. 3 for SIGN = -1).
template <int N, int SIGN>
__device__ __forceinline__ void fft_dit(float2 (&v)[N]) {
  fft_stages<N, SIGN>(v, std::make_integer_sequence<int, ilog2(N)>{});
}

// ---------------------------------------------------------------------------------------
// Packed pairs: two complex numbers as structure-of-arrays in two 64-bit register pairs,
// processed by the sm_100+ packed FP32 instructions (add/mul/fma .f32x2): one instruction does
// the same operation on both members, which halves the issue slots of the transform.
// ---------------------------------------------------------------------------------------
struct cp2 {
  float2 re;   // (a.re, b.re)
  float2 im;   // (a.im, b.im)
};

__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Element-wise complex products of two pairs (4 packed instructions).
__device__ __forceinline__ cp2 cmul2(const cp2& a, const cp2& b) {
  return cp2{fma2(a.re, b.re, mul2(make_float2(-a.im.x, -a.im.y), b.im)), fma2(a.re, b.im, mul2(a.im, b.re))};
}
__device__ __forceinline__ cp2 cmul2_conj(const cp2& a, const cp2& b) {   // a * conj(b)
  return cp2{fma2(a.re, b.re, mul2(a.im, b.im)), fma2(a.im, b.re, mul2(make_float2(-a.re.x, -a.re.y), b.im))};
}
__device__ __forceinline__ float2 power2(const cp2& a) { return fma2(a.re, a.re, mul2(a.im, a.im)); }
__device__ __forceinline__ cp2 cp2_from(float4 v) { return cp2{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 cp2_to(const cp2& v) { return make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }

// Packed DIT butterfly on two pairs: a' = a + w b, b' = a - w b, w = exp(SIGN i 2pi J/M), the
// same twiddle for both members.  Same FMA forms as the scalar butterfly.
template <int J, int M, int SIGN>
__device__ __forceinline__ void butterfly2(cp2& a, cp2& b) {
  constexpr CosSin cs = cossin_2pi(J, M);
  constexpr double wc = cs.c;
  constexpr double ws = SIGN * cs.s;
  if constexpr (J == 0) {
    const cp2 t = a;
    a = cp2{add2(t.re, b.re), add2(t.im, b.im)};
    b = cp2{sub2(t.re, b.re), sub2(t.im, b.im)};
  } else if constexpr (4 * J == M) {
    const cp2 t = a;
    if constexpr (SIGN > 0) {   // w b = (-b.im, b.re)
      a = cp2{sub2(t.re, b.im), add2(t.im, b.re)};
      b = cp2{add2(t.re, b.im), sub2(t.im, b.re)};
    } else {                    // w b = (b.im, -b.re)
      a = cp2{add2(t.re, b.im), sub2(t.im, b.re)};
      b = cp2{sub2(t.re, b.im), add2(t.im, b.re)};
    }
  } else if constexpr (cabsd(wc) >= cabsd(ws)) {
    constexpr float t = (float)(ws / wc);
    constexpr float c = (float)wc;
    const float2 ur = fma2(bc(-t), b.im, b.re);
    const float2 ui = fma2(bc(t), b.re, b.im);
    const cp2 s = a;
    a = cp2{fma2(bc(c), ur, s.re), fma2(bc(c), ui, s.im)};
    b = cp2{fma2(bc(-c), ur, s.re), fma2(bc(-c), ui, s.im)};
  } else {
    constexpr float ct = (float)(wc / ws);
    constexpr float sn = (float)ws;
    const float2 ur = fma2(bc(ct), b.re, make_float2(-b.im.x, -b.im.y));
    const float2 ui = fma2(bc(ct), b.im, b.re);
    const cp2 s = a;
    a = cp2{fma2(bc(sn), ur, s.re), fma2(bc(sn), ui, s.im)};
    b = cp2{fma2(bc(-sn), ur, s.re), fma2(bc(-sn), ui, s.im)};
  }
}

template <int N, int SIGN, int S, int I>
__device__ __forceinline__ void stage_butterfly2(cp2 (&v)[N]) {
  constexpr int span = 1 << S;
  constexpr int blk = (I / span) * (2 * span);
  constexpr int j = I % span;
  butterfly2<j, 2 * span, SIGN>(v[blk + j], v[blk + j + span]);
}
template <int N, int SIGN, int S, int... I>
__device__ __forceinline__ void fft_stage2(cp2 (&v)[N], std::integer_sequence<int, I...>) {
  (stage_butterfly2<N, SIGN, S, I>(v), ...);
}
template <int N, int SIGN, int... S>
__device__ __forceinline__ void fft_stages2(cp2 (&v)[N], std::integer_sequence<int, S...>) {
  (fft_stage2<N, SIGN, S>(v, std::make_integer_sequence<int, N / 2>{}), ...);
}

// Two independent N-point DFTs in lockstep ("columns" a and b of each pair):
// on entry v[i] = (a[bitrev(i)], b[bitrev(i)]), on exit v[m] = (A[m], B[m]).
template <int N, int SIGN>
__device__ __forceinline__ void fft_pair_columns(cp2 (&v)[N]) {
  fft_stages2<N, SIGN>(v, std::make_integer_sequence<int, ilog2(N)>{});
}

template <int N, int SIGN, int J>
__device__ __forceinline__ void last_stage_scalar(cp2 (&v)[N / 2]) {
  float2 a = make_float2(v[J].re.x, v[J].im.x);
  float2 b = make_float2(v[J].re.y, v[J].im.y);
  butterfly<J, N, SIGN>(a, b);
  v[J] = cp2{make_float2(a.x, b.x), make_float2(a.y, b.y)};
}
template <int N, int SIGN, int... J>
__device__ __forceinline__ void last_stage_all(cp2 (&v)[N / 2], std::integer_sequence<int, J...>) {
  (last_stage_scalar<N, SIGN, J>(v), ...);
}

// One N-point DFT held as N/2 pairs v[i] = (x[bitrev(i)], x[bitrev(i + N/2)]): the first
// log2(N)-1 stages are two N/2-point DFTs in lockstep (packed), the last stage pairs the two
// members of each pair (scalar FMA butterflies).  On exit v[j] = (X[j], X[j + N/2]).
template <int N, int SIGN>
__device__ __forceinline__ void fft_split_pairs(cp2 (&v)[N / 2]) {
  fft_stages2<N / 2, SIGN>(v, std::make_integer_sequence<int, ilog2(N) - 1>{});
  last_stage_all<N, SIGN>(v, std::make_integer_sequence<int, N / 2>{});
}

// ---------------------------------------------------------------------------------------
// mbarrier and bulk asynchronous copies (TMA), with time-bounded waits
// ---------------------------------------------------------------------------------------
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; false if limit_ns elapsed first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}
// 1-D bulk copy global -> shared, completion counted in bytes on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 1-D tiled tensor copy global -> shared of one box starting at element x (may be negative or
// beyond the extent: those elements are zero-filled).  x * element size must be a multiple of
// 16 bytes.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* tmap, int32_t x, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], "
      "[%3];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(smem_u32(bar))
      : "memory");
}


// ---------------------------------------------------------------------------------------
// Tensor memory (TMEM, sm_100+): 128 lanes x 512 columns of 32-bit cells per SM, a store
// separate from shared memory.  Warp w of a CTA may access lanes [32*(w%4), 32*(w%4)+32);
// with the 32x32b shape lane i of the warp reads/writes TMEM lane 32*(w%4)+i, consecutive
// columns.  An address is (lane << 16) | column, offset from the base tcgen05.alloc returns.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {   // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {   // whole warp
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 consecutive 32-bit columns of this lane (asynchronous: tmem_wait_ld before use).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
        "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]), "f"(r[8]), "f"(r[9]),
      "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15])
      : "memory");
}

}  // namespace fdas
