// fdas_zband.cu -- the learned z-band proposal (declared in include/fdas.h): a 1-D convolutional
// network over the z = 0 power spectrum that predicts which templates of the z grid are worth
// correlating near each block of bins, with hand-written training (FP32 forward, backward,
// Adam) and inference (a fused tcgen05 kernel: FP16 weights and activations, FP32
// accumulation), and the conversion of its proposals into a work list for the correlation
// kernel.  The paper has no counterpart; the full search stays the reference against which
// recall is measured.
//
// Network (window width Wd, hop Wd/2, C = 32 channels, k = 9, dilations 1, 4, 16, zero padding
// 4 x dilation):
//   x_r = min(|A_r|^2 ln 2 / median |A|^2, 64)   (one scale for the whole spectrum)
//   window w = x over bins [w*hop - Wd/4, w*hop + 3Wd/4), 0 outside [0, n)
//   a1 = conv_1(x; W1, b1), a2 = conv_4(relu(a1); W2, b2), a3 = conv_16(relu(a2); W3, b3)
//     conv_d(in; W, b)[o][t] = b[o] + sum_{i,k} W[o][i][k] in[i][t + (k - 4) d]
//   m[c] = max over t in [Wd/4, 3Wd/4) of relu(a3[c][t]),   logits = Wl m + bl  (Z outputs)
//   loss = mean BCE-with-logits(logits, target)
// The central positions' receptive field (+-84 = 4 (1 + 4 + 16)) stays inside the window
// (Wd >= 4 x 84), so the logits of window w are those of the layers run once over the
// zero-extended x and max-pooled over the block [w*hop, (w+1)*hop): the inference kernel
// computes that form, without the overlap.
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fdas.h"
#include "fdas_internal.h"
#include "fdas_umma.cuh"

namespace {

constexpr int kC = 32;          // channels
constexpr int kK = 9;           // kernel taps
constexpr int kPad = 4;
constexpr int kTile = 128;      // positions per conv block
constexpr int kDil1 = 1, kDil2 = 4, kDil3 = 16;    // layer dilations
constexpr int kRF = kPad * (kDil1 + kDil2 + kDil3);   // receptive field of a layer-3 position

// Flat parameter layout (floats).
struct Layout {
  int W1, b1, W2, b2, W3, b3, Wl, bl, total;
  explicit Layout(int Z) {
    W1 = 0;
    b1 = W1 + kC * 1 * kK;
    W2 = b1 + kC;
    b2 = W2 + kC * kC * kK;
    W3 = b2 + kC;
    b3 = W3 + kC * kC * kK;
    Wl = b3 + kC;
    bl = Wl + Z * kC;
    total = bl + Z;
  }
};

constexpr float kXCap = 64.f;   // input cap: x_r = min(|A_r|^2 ln 2 / median |A|^2, 64)
constexpr int kSelBlocks = 2048; // grid cap of the median's first pass
constexpr int kSelBlocks12 = 304; // and of its second and third (2 blocks per SM of a GB300)

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// Exact lower median of |A_r|^2 (rank (n-1)/2) by radix selection on the FP32 bit patterns
// (non-negative floats order as unsigned integers): three passes over the spectrum histogram the
// top 8 bits (sign and exponent: most values share a few bins, so each warp counts into its own
// copy), then the next 12 bits of the values matching the digit found so far, then the last 12;
// after each pass one block finds the digit holding the rank (a block scan of the histogram).
// scale = ln 2 / median.
constexpr int kSelBins0 = 256, kSelBins = 4096;
constexpr int kSelPer = 8;   // complex values per thread and pass iteration (four 16-byte loads)
struct SelectState {
  long long k;                 // rank of the median among the values matching `prefix`
  unsigned prefix, mask;       // bits fixed so far and their mask
  unsigned hist0[kSelBins0];   // bits 31..24
  unsigned hist1[kSelBins];    // bits 23..12 of the values matching digit 0
  unsigned hist2[kSelBins];    // bits 11..0 of the values matching digits 0 and 1
};

__device__ __forceinline__ float power_of(const float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// PASS 0: top 8 bits of every value (one histogram per warp, summed at the end); PASS 1, 2: the
// next 12 bits of the values whose higher bits equal st->prefix.  Values are read in 16-byte pairs from the first 16-byte boundary (an
// 8-byte aligned spectrum's first value is counted on its own); the tail element by element.
template <int PASS>
__global__ void __launch_bounds__(256) select_pass_kernel(const float2* spec, int64_t n, SelectState* st) {
  constexpr int NB = PASS == 0 ? kSelBins0 : kSelBins;
  constexpr int SHIFT = PASS == 0 ? 24 : (PASS == 1 ? 12 : 0);
  constexpr int COPIES = PASS == 0 ? 8 : 1;   // per-warp histograms in pass 0
  __shared__ unsigned h[COPIES * NB];
  for (int i = threadIdx.x; i < COPIES * NB; i += 256) h[i] = 0u;
  const unsigned prefix = PASS == 0 ? 0u : st->prefix, mask = PASS == 0 ? 0u : st->mask;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  unsigned* hw = h + (COPIES > 1 ? (threadIdx.x >> 5) * NB : 0);
  auto count = [&](float2 a, bool valid) {
    unsigned bucket = 0xFFFFFFFFu;
    if (valid) {
      const unsigned bits = __float_as_uint(power_of(a));
      if ((bits & mask) == prefix) bucket = (bits >> SHIFT) & (unsigned)(NB - 1);
    }
    // one shared atomic per distinct bucket of the warp
    const unsigned peers = __match_any_sync(0xffffffffu, bucket);
    if (bucket != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&hw[bucket], (unsigned)__popc(peers));
  };
  const int off = (reinterpret_cast<uintptr_t>(spec) & 15u) ? 1 : 0;
  if (off && blockIdx.x == 0 && threadIdx.x < 32)
    count(threadIdx.x == 0 ? __ldg(spec) : make_float2(0.f, 0.f), threadIdx.x == 0 && n > 0);
  spec += off;
  n -= off;
  const int64_t step = (int64_t)gridDim.x * 256 * kSelPer;
  for (int64_t base = (int64_t)blockIdx.x * 256 * kSelPer; base < n; base += step) {
    // thread t reads the pairs (base + 2(t + 256 j), +1), j < kSelPer / 2: coalesced 16-byte loads
    float4 v[kSelPer / 2];
#pragma unroll
    for (int j = 0; j < kSelPer / 2; ++j) {
      const int64_t r = base + 2 * ((int64_t)threadIdx.x + 256 * j);
      v[j] = r + 1 < n ? __ldg(reinterpret_cast<const float4*>(spec + r))
                       : make_float4(r < n ? spec[r].x : 0.f, r < n ? spec[r].y : 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kSelPer / 2; ++j) {
      const int64_t r = base + 2 * ((int64_t)threadIdx.x + 256 * j);
      count(make_float2(v[j].x, v[j].y), r < n);
      count(make_float2(v[j].z, v[j].w), r + 1 < n);
    }
  }
  __syncthreads();
  unsigned* out = PASS == 0 ? st->hist0 : (PASS == 1 ? st->hist1 : st->hist2);
  for (int i = threadIdx.x; i < NB; i += 256) {
    unsigned c = 0u;
#pragma unroll
    for (int w = 0; w < COPIES; ++w) c += h[w * NB + i];
    if (c) atomicAdd(&out[i], c);
  }
}

// One block of 256 threads: the digit of histogram PASS holding rank st->k (thread t owns the
// bins [t*NB/256, (t+1)*NB/256); a block scan of their sums leaves exactly one thread whose range
// holds the rank), appended to st->prefix; after the last digit, scale = ln 2 / median.
template <int PASS>
__global__ void __launch_bounds__(256) select_digit_kernel(SelectState* st, float* scale) {
  constexpr int NB = PASS == 0 ? kSelBins0 : kSelBins;
  constexpr int SHIFT = PASS == 0 ? 24 : (PASS == 1 ? 12 : 0);
  constexpr int per = NB / 256;
  __shared__ long long wsum[8];
  const unsigned* hist = PASS == 0 ? st->hist0 : (PASS == 1 ? st->hist1 : st->hist2);
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  unsigned c[per];
  long long own = 0;
#pragma unroll
  for (int i = 0; i < per; ++i) {
    c[i] = hist[t * per + i];
    own += c[i];
  }
  long long inc = own;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += y;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  long long excl = inc - own;
  for (int i = 0; i < wid; ++i) excl += wsum[i];
  const long long k = st->k;
  if (k >= excl && k < excl + own) {
    long long r = k - excl;
    int d = t * per;
#pragma unroll
    for (int i = 0; i < per - 1; ++i)
      if (d == t * per + i && r >= (long long)c[i]) {
        r -= c[i];
        ++d;
      }
    const unsigned prefix = (PASS == 0 ? 0u : st->prefix) | ((unsigned)d << SHIFT);
    st->k = r;
    st->prefix = prefix;
    st->mask = PASS == 0 ? 0xFF000000u : (PASS == 1 ? 0xFFFFF000u : 0xFFFFFFFFu);
    if (PASS == 2) {
      const float med = __uint_as_float(prefix);
      *scale = med > 0.f ? 0.69314718055994531f / med : 0.f;
    }
  }
}

__global__ void __launch_bounds__(256) select_init_kernel(SelectState* st, int64_t n) {
  if (threadIdx.x == 0) {
    st->k = (n - 1) / 2;
    st->prefix = 0u;
    st->mask = 0u;
  }
  for (int i = threadIdx.x; i < kSelBins0; i += 256) st->hist0[i] = 0u;
  for (int i = threadIdx.x; i < kSelBins; i += 256) {
    st->hist1[i] = 0u;
    st->hist2[i] = 0u;
  }
}

__device__ __forceinline__ float power_x(const float2* spec, int64_t n, int64_t r, float scale) {
  if (r < 0 || r >= n) return 0.f;
  return fminf(power_of(spec[r]) * scale, kXCap);
}

// Windows of x: window w covers bins [w*hop - Wd/4, w*hop + 3Wd/4), 0 outside [0, n).
__global__ void spectrum_windows_kernel(const float2* spec, int64_t n, const float* scale, int Wd, int hop,
                                        float* x) {
  const int64_t w = blockIdx.x;
  const int64_t r0 = w * hop - Wd / 4;
  const float sc = *scale;
  for (int t = threadIdx.x; t < Wd; t += blockDim.x) x[w * Wd + t] = power_x(spec, n, r0 + t, sc);
}

// pre[b][o][t] = bias[o] + sum_{i,k} W[o][i][k] * in(b, i, t + (k - 4) D); in = x (CIN = 1) or
// relu(prev pre-activation).  Block: 128 positions of one window, all 32 output channels;
// thread (o = tid/8, t = tid%8 + 8j).
template <int CIN, int D>
constexpr size_t conv_fwd_smem() {
  return sizeof(float) * ((size_t)CIN * (kTile + 2 * kPad * D) + (size_t)kC * CIN * kK);
}

template <int CIN, bool RELU_IN, typename WT, int D>
__global__ void __launch_bounds__(256) conv_fwd_kernel(const float* in, const WT* W, const WT* bias, float* pre,
                                                       int Wd) {
  constexpr int S = kTile + 2 * kPad * D;   // staged positions: the tile and its halo
  extern __shared__ float dyn[];
  float (*sIn)[S] = reinterpret_cast<float (*)[S]>(dyn);
  float* sW = dyn + (size_t)CIN * S;
  const int b = blockIdx.y, t0 = blockIdx.x * kTile;
  for (int idx = threadIdx.x; idx < kC * CIN * kK; idx += blockDim.x) sW[idx] = to_f(W[idx]);
  for (int idx = threadIdx.x; idx < CIN * S; idx += blockDim.x) {
    const int i = idx / S, tt = idx % S;
    const int t = t0 + tt - kPad * D;
    float v = (t >= 0 && t < Wd) ? in[((size_t)b * CIN + i) * Wd + t] : 0.f;
    if (RELU_IN) v = fmaxf(v, 0.f);
    sIn[i][tt] = v;
  }
  __syncthreads();
  const int o = threadIdx.x >> 3, tl = threadIdx.x & 7;
  float acc[kTile / 8];
  const float bo = to_f(bias[o]);
#pragma unroll
  for (int j = 0; j < kTile / 8; ++j) acc[j] = bo;
  for (int i = 0; i < CIN; ++i) {
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      const float w = sW[(o * CIN + i) * kK + k];
#pragma unroll
      for (int j = 0; j < kTile / 8; ++j) acc[j] = fmaf(w, sIn[i][tl + 8 * j + k * D], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kTile / 8; ++j) pre[((size_t)b * kC + o) * Wd + t0 + tl + 8 * j] = acc[j];
}

// Pooling over the central half and the linear head: one block per window.
template <typename WT>
__global__ void pool_head_kernel(const float* a3, const WT* Wl, const WT* bl, int Wd, int Z, float* m_out,
                                 int* arg_out, float* logits) {
  const int b = blockIdx.x;
  __shared__ float sm[kC];
  const int lo = Wd / 4, hi = 3 * Wd / 4;
  // 8 threads per channel, then combine (first maximum on ties)
  const int c = threadIdx.x >> 3, l = threadIdx.x & 7;
  float best = -1.f;
  int barg = lo;
  for (int t = lo + l; t < hi; t += 8) {
    const float v = fmaxf(a3[((size_t)b * kC + c) * Wd + t], 0.f);
    if (v > best) {
      best = v;
      barg = t;
    }
  }
  for (int off = 4; off > 0; off >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, best, off, 8);
    const int oa = __shfl_down_sync(0xffffffffu, barg, off, 8);
    if (ov > best || (ov == best && oa < barg)) {
      best = ov;
      barg = oa;
    }
  }
  if (l == 0) {
    sm[c] = best;
    if (m_out) m_out[b * kC + c] = best;
    if (arg_out) arg_out[b * kC + c] = barg;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < Z; j += blockDim.x) {
    float s = to_f(bl[j]);
#pragma unroll 8
    for (int cc = 0; cc < kC; ++cc) s = fmaf(to_f(Wl[j * kC + cc]), sm[cc], s);
    logits[(size_t)b * Z + j] = s;
  }
}

// dlog = (sigmoid(l) - target) / (B*Z); loss_part[warp] = that warp's sum of BCE terms / (B*Z),
// summed afterwards in a fixed order (sum_fixed_kernel), so the loss is the same on every run.
__global__ void bce_grad_kernel(const float* logits, const float* target, int count, float* dlog, float* loss_part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float term = 0.f;
  if (i < count) {
    const float l = logits[i], t = target[i];
    dlog[i] = (1.f / (1.f + expf(-l)) - t) / (float)count;
    term = fmaxf(l, 0.f) - l * t + log1pf(expf(-fabsf(l)));
  }
  for (int off = 16; off > 0; off >>= 1) term += __shfl_down_sync(0xffffffffu, term, off);
  if ((threadIdx.x & 31) == 0 && i < count) loss_part[i >> 5] = term / (float)count;   // warps with a term
}

// out = sum of part[0..n) in a fixed order: thread t adds part[t], part[t + 1024], ... in turn,
// then a fixed-shape tree over the 1024 threads.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) sum_fixed_kernel(const float* part, int n, float* out) {
  __shared__ float s[1024];
  float a = 0.f;
  for (int j = threadIdx.x; j < n; j += 1024) a += part[j];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// out[j] = sum over blk = 0, 1, ..., nblk-1 (in that order) of part[blk * stride + j], j < n: the
// fixed-order reduction of per-block weight-gradient partials.
__global__ void reduce_partials_kernel(const float* part, int nblk, int stride, int n, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float a = 0.f;
  for (int blk = 0; blk < nblk; ++blk) a += part[(size_t)blk * stride + j];
  out[j] = a;
}

// Head backward: dWl[j][c] = sum_b dlog[b][j] m[b][c], dbl[j] = sum_b dlog[b][j].
__global__ void head_bwd_weights_kernel(const float* dlog, const float* m, int B, int Z, float* dWl, float* dbl) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Z * (kC + 1)) return;
  const int j = idx / (kC + 1), c = idx % (kC + 1);
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dlog[(size_t)b * Z + j] * (c < kC ? m[b * kC + c] : 1.f);
  if (c < kC) dWl[j * kC + c] = s;
  else dbl[j] = s;
}

// dm[b][c] = sum_j dlog[b][j] Wl[j][c]; then da3 = dm at the pooled position if a3 > 0 there.
__global__ void head_bwd_data_kernel(const float* dlog, const float* Wl, const int* arg, const float* a3, int Z,
                                     int Wd, float* da3) {
  const int b = blockIdx.x, c = threadIdx.x;
  if (c >= kC) return;
  float s = 0.f;
  for (int j = 0; j < Z; ++j) s = fmaf(dlog[(size_t)b * Z + j], Wl[j * kC + c], s);
  const int t = arg[b * kC + c];
  const size_t at = ((size_t)b * kC + c) * Wd + t;
  da3[at] = a3[at] > 0.f ? s : 0.f;
}

// dIn_pre[b][i][t] = (prev_pre > 0) * sum_{o,k} W[o][i][k] dOut[b][o][t - (k - 4) D].
template <int D>
constexpr size_t bwd_data_smem() {
  return sizeof(float) * ((size_t)kC * (kTile + 2 * kPad * D) + (size_t)kC * kC * kK);
}

template <int D>
__global__ void __launch_bounds__(256) conv_bwd_data_kernel(const float* dout, const float* W, const float* prev_pre,
                                                            float* din, int Wd) {
  constexpr int S = kTile + 2 * kPad * D;
  extern __shared__ float dyn[];
  float (*sD)[S] = reinterpret_cast<float (*)[S]>(dyn);
  float* sW = dyn + (size_t)kC * S;
  const int b = blockIdx.y, t0 = blockIdx.x * kTile;
  for (int idx = threadIdx.x; idx < kC * kC * kK; idx += blockDim.x) sW[idx] = W[idx];
  for (int idx = threadIdx.x; idx < kC * S; idx += blockDim.x) {
    const int o = idx / S, tt = idx % S;
    const int t = t0 + tt - kPad * D;
    sD[o][tt] = (t >= 0 && t < Wd) ? dout[((size_t)b * kC + o) * Wd + t] : 0.f;
  }
  __syncthreads();
  const int i = threadIdx.x >> 3, tl = threadIdx.x & 7;
  float acc[kTile / 8];
#pragma unroll
  for (int j = 0; j < kTile / 8; ++j) acc[j] = 0.f;
  for (int o = 0; o < kC; ++o) {
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      const float w = sW[(o * kC + i) * kK + k];
      // dOut index t - (k - 4) D = (t0 + tl + 8j) - (k - 4) D -> tile offset tl + 8j + (8 - k) D
#pragma unroll
      for (int j = 0; j < kTile / 8; ++j) acc[j] = fmaf(w, sD[o][tl + 8 * j + (2 * kPad - k) * D], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kTile / 8; ++j) {
    const size_t at = ((size_t)b * kC + i) * Wd + t0 + tl + 8 * j;
    din[at] = prev_pre[at] > 0.f ? acc[j] : 0.f;
  }
}

// Partials of one block (tile, b): part[blk][(o*CIN + i)*9 + k] = sum_{t in tile} in(b, i, t + (k - 4) D)
// * dOut[b][o][t] and part[blk][C*CIN*9 + o] = sum_{t in tile} dOut[b][o][t], blk = b*tiles + tile;
// reduce_partials_kernel then sums them over blocks in a fixed order (no floating-point atomics, so
// one seed gives one network).  Thread handles (o = tid/8) and i in {tid%8, tid%8 + 8, ...}.
template <int CIN, int D>
constexpr size_t bwd_weight_smem() {
  return sizeof(float) * ((size_t)CIN * (kTile + 2 * kPad * D) + (size_t)kC * kTile);
}

template <int CIN, bool RELU_IN, int D>
__global__ void __launch_bounds__(256) conv_bwd_weight_kernel(const float* in, const float* dout, int Wd,
                                                              float* part) {
  constexpr int S = kTile + 2 * kPad * D;
  extern __shared__ float dyn[];
  float (*sIn)[S] = reinterpret_cast<float (*)[S]>(dyn);
  float (*sD)[kTile] = reinterpret_cast<float (*)[kTile]>(dyn + (size_t)CIN * S);
  const int b = blockIdx.y, t0 = blockIdx.x * kTile;
  for (int idx = threadIdx.x; idx < CIN * S; idx += blockDim.x) {
    const int i = idx / S, tt = idx % S;
    const int t = t0 + tt - kPad * D;
    float v = (t >= 0 && t < Wd) ? in[((size_t)b * CIN + i) * Wd + t] : 0.f;
    if (RELU_IN) v = fmaxf(v, 0.f);
    sIn[i][tt] = v;
  }
  for (int idx = threadIdx.x; idx < kC * kTile; idx += blockDim.x) {
    const int o = idx / kTile, tt = idx % kTile;
    sD[o][tt] = dout[((size_t)b * kC + o) * Wd + t0 + tt];
  }
  __syncthreads();
  const int o = threadIdx.x >> 3, l = threadIdx.x & 7;
  for (int i = l; i < CIN; i += 8) {
    float acc[kK];
#pragma unroll
    for (int k = 0; k < kK; ++k) acc[k] = 0.f;
    for (int t = 0; t < kTile; ++t) {
      const float d = sD[o][t];
#pragma unroll
      for (int k = 0; k < kK; ++k) acc[k] = fmaf(sIn[i][t + k * D], d, acc[k]);
    }
    float* dst = part + ((size_t)b * gridDim.x + blockIdx.x) * ((size_t)kC * CIN * kK + kC);
#pragma unroll
    for (int k = 0; k < kK; ++k) dst[(o * CIN + i) * kK + k] = acc[k];
  }
  if (l == 0) {
    float s = 0.f;
    for (int t = 0; t < kTile; ++t) s += sD[o][t];
    part[((size_t)b * gridDim.x + blockIdx.x) * ((size_t)kC * CIN * kK + kC) + (size_t)kC * CIN * kK + o] = s;
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_half_kernel(const float* p, __half* h, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) h[i] = __float2half_rn(p[i]);
}

// Proposal -> correlation work list.  Segment j of group g (G segments of V bins: outputs
// [(gG+j)V, (gG+j+1)V)) is proposed for template z if any window whose central bins
// [w*hop, (w+1)*hop) meet the bins its outputs can draw on, [(gG+j)V - h, (gG+j+1)V + h), has
// sigmoid(logit_z) >= threshold; mask[g][z] holds those G bits and unit (g, z) is listed when
// any is set.
__global__ void group_flags_kernel(const float* logits, int n_win, int Z, float logit_thr, int hop, int64_t seg_bins,
                                   int G, int h, int n_groups, uint16_t* masks, int* counts) {
  const int g = blockIdx.x;
  const int64_t lo = (int64_t)g * G * seg_bins - h, hi = ((int64_t)g + 1) * G * seg_bins + h;
  int w0 = (int)((lo > 0 ? lo : 0) / hop);
  int w1 = (int)((hi + hop - 1) / hop);
  if (w1 > n_win) w1 = n_win;
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int z = threadIdx.x; z < Z; z += blockDim.x) {
    unsigned m = 0u;
    for (int w = w0; w < w1; ++w) {
      if (!(logits[(size_t)w * Z + z] >= logit_thr)) continue;
      const int64_t b0 = (int64_t)w * hop, b1 = b0 + hop;   // the window's central bins
      for (int j = 0; j < G; ++j) {
        const int64_t s0 = ((int64_t)g * G + j) * seg_bins - h, s1 = ((int64_t)g * G + j + 1) * seg_bins + h;
        if (b0 < s1 && b1 > s0) m |= 1u << j;
      }
    }
    masks[(size_t)g * Z + z] = (uint16_t)m;
    if (m) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) counts[g] = cnt;
}

// Proposal -> pair list.  Segment s has the outputs [s*V, (s+1)*V) (seg_bins = V) and draws on
// the inputs [s*V - h, (s+1)*V + h).  A template q is proposed for it by a block w (central bins
// [w*hop, (w+1)*hop)) that meets its outputs with sigmoid(logit) >= threshold, or by a block that
// meets only the inputs beyond them with sigmoid(logit) >= reach_threshold (a signal there must be
// strong for its response to reach the segment's outputs); pair (s, z) is listed when a template
// within z_halo of z is proposed.  One block per segment: the two maxima per template, the
// proposed flags in shared memory (Z ints), then the dilation.  mask[s][z] = 1 for a listed pair.
__global__ void segment_flags_kernel(const float* logits, int n_win, int Z, float logit_thr, float logit_reach,
                                     int z_halo, int hop, int64_t seg_bins, int h, uint16_t* masks, int* counts) {
  extern __shared__ int sflag[];
  const int64_t s = blockIdx.x;
  const int64_t o0 = s * seg_bins, o1 = (s + 1) * seg_bins;   // outputs
  const int64_t r0 = o0 - h, r1 = o1 + h;                     // inputs
  auto clampw = [&](int64_t w) { return (int)(w < 0 ? 0 : (w > n_win ? n_win : w)); };
  const int wr0 = clampw((r0 > 0 ? r0 : 0) / hop), wr1 = clampw((r1 + hop - 1) / hop);
  const int wo0 = clampw(o0 / hop), wo1 = clampw((o1 + hop - 1) / hop);
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  for (int z = threadIdx.x; z < Z; z += blockDim.x) {
    float own = -INFINITY, reach = -INFINITY;   // NaN logits never list
    for (int w = wr0; w < wr1; ++w) {
      const float v = logits[(size_t)w * Z + z];
      if (w >= wo0 && w < wo1) own = fmaxf(own, v);
      else reach = fmaxf(reach, v);
    }
    sflag[z] = (own >= logit_thr || reach >= logit_reach) ? 1 : 0;
  }
  __syncthreads();
  for (int z = threadIdx.x; z < Z; z += blockDim.x) {
    const int a = z - z_halo > 0 ? z - z_halo : 0, b = z + z_halo < Z - 1 ? z + z_halo : Z - 1;
    bool f = false;
    for (int q = a; q <= b && !f; ++q) f = sflag[q] != 0;
    masks[(size_t)s * Z + z] = f ? 1 : 0;
    if (f) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) counts[s] = cnt;
}

// Exclusive scan of per-group counts and the total: one block of 1024 threads, thread t owning
// the contiguous chunk [t c, (t+1) c) of the groups; chunk sums are scanned with warp shuffles.
__global__ void __launch_bounds__(1024) scan_counts_kernel(const int* counts, int n_groups, int64_t* offsets,
                                                           int64_t* total) {
  __shared__ int64_t warp_excl[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int chunk = (n_groups + 1023) / 1024;
  const int b = tid * chunk < n_groups ? tid * chunk : n_groups;
  const int e = b + chunk < n_groups ? b + chunk : n_groups;
  int64_t own = 0;
  for (int g = b; g < e; ++g) own += counts[g];
  int64_t incl = own;   // inclusive scan over the warp
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) warp_excl[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int64_t ws = warp_excl[lane];
    int64_t wi = ws;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += y;
    }
    warp_excl[lane] = wi - ws;
  }
  __syncthreads();
  int64_t run = warp_excl[wid] + incl - own;
  for (int g = b; g < e; ++g) {
    offsets[g] = run;
    run += counts[g];
  }
  if (tid == 1023) *total = run;
}

// units[offset_g + k] = g*Z + z for the k-th proposed z of group g (increasing z), and its
// segment mask when out_masks is set: one block of 256 threads per group, each unit placed by
// the popcount of the proposed templates before it.
__global__ void __launch_bounds__(256) write_units_kernel(const uint16_t* masks, const int64_t* offsets, int Z,
                                                          int32_t* units, uint16_t* out_masks) {
  __shared__ int warp_cnt[8];
  const int g = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t base = offsets[g];
  for (int z0 = 0; z0 < Z; z0 += 256) {
    const int z = z0 + (int)threadIdx.x;
    const unsigned mz = z < Z ? masks[(size_t)g * Z + z] : 0u;
    const bool f = mz != 0u;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_cnt[wid] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      before += i < wid ? warp_cnt[i] : 0;
      all += warp_cnt[i];
    }
    if (f) {
      const int64_t at = base + before + __popc(m & ((1u << lane) - 1u));
      units[at] = (int32_t)((int64_t)g * Z + z);
      if (out_masks) out_masks[at] = (uint16_t)mz;
    }
    base += all;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Fused inference over a whole spectrum on the tensor cores (tcgen05.mma kind::f16: FP16
// weights and activations, FP32 accumulation in TMEM).  A CTA holds the weights once and runs
// two independent groups of 4 warps, each with its own activation slot, half of the TMEM
// allocation, mbarrier and named barriers, so one group's MMAs overlap the other's epilogues.
// Group g of CTA b walks blocks w = 2b + g, 2b + g + 2*gridDim.x, ...; block w owns output
// positions [w*hop, (w+1)*hop) and recomputes the +-84-position halo its three layers need
// (dilations 1, 4, 16):
//   x   at P0-84 + j, j < 128*T1 + 8     (prefetched into registers one block ahead)
//   h1  at P0-80 + r, r < 128*T2 + 32    (layer 1 as an im2col GEMM: K = 9 taps padded to 16)
//   h2  at P0-64 + r, r < hop + 128      (layer 2: T2 = T3 + 1 M-tiles of 128 positions)
//   h3  at P0 + r,    r < hop            (layer 3: T3 = hop/128 M-tiles), max-pooled per channel
// Activations sit in shared memory "chunk-planar": channel chunk j (8 channels, 16 B) of
// position row r at plane j, offset 16*r.  A K-major no-swizzle operand whose rows are
// positions is then one descriptor per (tap k, K-half c): start row + k d, LBO = plane size,
// SBO = 128 B -- the im2col of a dilated k = 9 convolution costs no copies.
// ---------------------------------------------------------------------------------------
constexpr int kMaxHop = 512;
constexpr int kT3max = kMaxHop / 128;
constexpr int kT2max = kT3max + 1;
constexpr int kT1max = kT2max + 1;
constexpr int kNP1 = 128 * kT2max + 8 * kDil2;  // h1 rows (plane height)
constexpr int kNP2 = 128 * kT2max;              // h2 rows (plane height)
constexpr int kNA1 = 128 * kT1max;              // im2col rows of layer 1
constexpr int kNX = kNA1 + 8;                   // staged x values
constexpr int kGroupThreads = 128;
constexpr int kXPer = (kNX + kGroupThreads - 1) / kGroupThreads;   // prefetched x per thread
constexpr int kZStage = 256;                    // head weights staged in shared memory up to this Z
constexpr uint32_t kPlaneH1 = kNP1 * 16, kPlaneH2 = kNP2 * 16, kPlaneA1 = kNA1 * 16;
constexpr int kOffW1 = 0;                       // layer-1 weights: 2 K-chunks x 512 B
constexpr int kOffW2 = kOffW1 + 1024;           // 9 taps x 4 K-chunks x 512 B
constexpr int kOffW3 = kOffW2 + 9 * 2048;
constexpr int kOffWl = kOffW3 + 9 * 2048;       // head weights [Z][32] FP16
constexpr int kOffBl = kOffWl + kZStage * kC * 2;
constexpr int kOffBias = kOffBl + kZStage * 4;  // b1, b2, b3 (FP32 values of the FP16 copy)
constexpr int kOffSlot = kOffBias + 3 * kC * 4; // two activation slots
constexpr int kSlotH1 = 0;                      // also holds the staged x (dead before h1 is written)
constexpr int kSlotH2 = 4 * kPlaneH1;           // also holds the layer-1 im2col (dead before h2)
constexpr int kSlotBytes = kSlotH2 + 4 * kPlaneH2;
constexpr int kOffGroup = kOffSlot + 2 * kSlotBytes;   // per group: channel maxima, mbarrier
constexpr int kGroupMisc = 256;
constexpr int kOffTslot = kOffGroup + 2 * kGroupMisc;
constexpr int kProposeSmem = kOffTslot + 16;
constexpr uint32_t kIdesc = fdas::umma_idesc_f16(128, kC);
constexpr uint32_t kTmemCols = 512;             // 256 columns per group (<= 6 x 32 used)
static_assert(kDil1 == 1, "layer 1 is an im2col of adjacent x values");
static_assert(8 * kDil3 <= 128 && 8 * kDil2 <= 128, "each layer's halo fits in one extra 128-row tile");
static_assert(2 * kPlaneA1 <= 4 * kPlaneH2, "im2col must fit in the h2 planes");
static_assert(kNX * 4 <= (int)(4 * kPlaneH1), "staged x must fit in the h1 planes");
static_assert(32 * kT1max <= (int)kTmemCols / 2, "accumulators must fit a group's TMEM half");
static_assert(kOffSlot % 128 == 0 && kSlotBytes % 128 == 0, "slot alignment");
static_assert(kProposeSmem <= 227 * 1024, "shared memory");

struct ProposeParams {
  const float2* spec;
  int64_t n;
  const float* scale;       // ln 2 / median |A|^2 (device scalar)
  const __half* w;          // FP16 parameter vector (Layout order)
  int oW1, ob1, oW2, ob2, oW3, ob3, oWl, obl;
  int Z, hop;
  int64_t n_blocks;
  float* logits;            // n_blocks x Z
  int* status;              // bit 0: a bounded wait gave up
};

// B operand (weights) of one tap in the K-major no-swizzle layout: rows o (N = 32), K = in-ch.
__device__ __forceinline__ int wb_off(int o, int i) { return (i >> 3) * 512 + (o >> 3) * 128 + (o & 7) * 16 + (i & 7) * 2; }

// Named barrier of one 128-thread group (ids 1, 2; id 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory"); }
__device__ __forceinline__ int group_all(int g, int v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.and.pred q, %2, 128, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(v), "r"(g + 1)
      : "memory");
  return r;
}

template <int HOP>
__global__ void __launch_bounds__(256, 1) propose_kernel(const ProposeParams p) {
  static_assert(HOP % 128 == 0 && HOP <= kMaxHop, "hop");
  using namespace fdas;
  extern __shared__ __align__(1024) unsigned char sm[];
  __half* sW1 = reinterpret_cast<__half*>(sm + kOffW1);
  __half* sW2 = reinterpret_cast<__half*>(sm + kOffW2);
  __half* sW3 = reinterpret_cast<__half*>(sm + kOffW3);
  __half* sWl = reinterpret_cast<__half*>(sm + kOffWl);
  float* sBl = reinterpret_cast<float*>(sm + kOffBl);
  float* sBias = reinterpret_cast<float*>(sm + kOffBias);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffTslot);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 2, q = warp & 3, gt = tid & (kGroupThreads - 1);
  unsigned char* slot = sm + kOffSlot + g * kSlotBytes;
  float* sX = reinterpret_cast<float*>(slot + kSlotH1);
  unsigned char* sH1 = slot + kSlotH1;
  unsigned char* sH2 = slot + kSlotH2;
  unsigned char* sA1 = slot + kSlotH2;
  unsigned* sMax = reinterpret_cast<unsigned*>(sm + kOffGroup + g * kGroupMisc);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffGroup + g * kGroupMisc + 128);
  const bool wl_staged = p.Z <= kZStage;

  // weights into the B layouts (FP16) and the head; biases as FP32 values of the FP16 copy
  for (int idx = tid; idx < kC * 16; idx += 256) {
    const int o = idx >> 4, k = idx & 15;
    sW1[wb_off(o, k) / 2] = k < kK ? p.w[p.oW1 + o * kK + k] : __float2half_rn(0.f);
  }
  for (int idx = tid; idx < kK * kC * kC; idx += 256) {
    const int k = idx / (kC * kC), o = (idx / kC) % kC, i = idx % kC;
    sW2[k * 1024 + wb_off(o, i) / 2] = p.w[p.oW2 + (o * kC + i) * kK + k];
    sW3[k * 1024 + wb_off(o, i) / 2] = p.w[p.oW3 + (o * kC + i) * kK + k];
  }
  if (wl_staged) {
    for (int idx = tid; idx < p.Z * kC; idx += 256) sWl[idx] = p.w[p.oWl + idx];
    for (int j = tid; j < p.Z; j += 256) sBl[j] = __half2float(p.w[p.obl + j]);
  }
  if (tid < kC) {
    sBias[tid] = __half2float(p.w[p.ob1 + tid]);
    sBias[kC + tid] = __half2float(p.w[p.ob2 + tid]);
    sBias[2 * kC + tid] = __half2float(p.w[p.ob3 + tid]);
  }
  if (gt == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, kTmemCols);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tm = *tslot + 256u * g;
  const uint32_t tm_lane = tm + ((uint32_t)(32 * q) << 16);
  const uint32_t aW1 = smem_u32(sW1), aW2 = smem_u32(sW2), aW3 = smem_u32(sW3);
  const uint32_t aH1 = smem_u32(sH1), aH2 = smem_u32(sH2), aA1 = smem_u32(sA1);
  const float sc = *p.scale;
  constexpr int T3 = HOP / 128, T2 = T3 + 1, T1 = T2 + 1;
  constexpr int nx = 128 * T1 + 8;
  uint32_t phase = 0;
  bool ok = true;

  // x values of block w's staging window into registers (all loads issued before any use)
  float2 xa[kXPer];
  auto load_x = [&](int64_t P0) {
#pragma unroll
    for (int e = 0; e < kXPer; ++e) {
      const int j = gt + kGroupThreads * e;
      const int64_t r = P0 - kRF + j;
      xa[e] = (j < nx && r >= 0 && r < p.n) ? __ldg(p.spec + r) : make_float2(0.f, 0.f);
    }
  };
  // wait for this group's committed MMAs: one thread polls (bounded), the others sleep in the
  // group's hardware barrier
  auto wait_mma = [&]() -> bool {
    const int good = group_all(g, gt == 0 ? (mbar_wait(bar, phase) ? 1 : 0) : 1);
    phase ^= 1u;
    tmem_fence_after_sync();
    return good != 0;
  };
  auto sync_for_mma = [&]() {
    fence_proxy_async_smem();
    tmem_fence_before_sync();
    group_sync(g);
    tmem_fence_after_sync();
  };
  // accumulator tile t (lanes = rows 128t + 32q + lane) + bias -> relu -> FP16 planes, rows < limit.
  // The next tile's TMEM load is issued before this tile is converted (tcgen05.wait::ld waits for
  // every earlier load, so the wait comes first and the two buffers alternate).
  auto store_layer = [&](auto ntiles, int limit, const float* bias, unsigned char* dst, uint32_t plane) {
    constexpr int NT = decltype(ntiles)::value;
    float a[2][16], b[2][16];
    tmem_ld16(tm_lane, a[0]);
    tmem_ld16(tm_lane + 16, b[0]);
    static_for<NT>([&](auto tt) {
      constexpr int t = decltype(tt)::value, cur = t & 1;
      tmem_wait_ld();
      if constexpr (t + 1 < NT) {
        tmem_ld16(tm_lane + 32 * (t + 1), a[cur ^ 1]);
        tmem_ld16(tm_lane + 32 * (t + 1) + 16, b[cur ^ 1]);
      }
      const int r = 128 * t + 32 * q + lane;
      if (r < limit) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          __half2 h[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = 8 * j + 2 * e;
            const float v0 = c < 16 ? a[cur][c] : b[cur][c - 16], v1 = c + 1 < 16 ? a[cur][c + 1] : b[cur][c - 15];
            h[e] = __floats2half2_rn(fmaxf(v0 + bias[c], 0.f), fmaxf(v1 + bias[c + 1], 0.f));
          }
          *reinterpret_cast<uint4*>(dst + j * plane + r * 16) = *reinterpret_cast<uint4*>(h);
        }
      }
    });
  };
  // one k = 9 convolution layer with dilation D: NT M-tiles, A rows start at 128t + kD in the
  // source planes; tiles innermost, so consecutive MMAs feed independent accumulators.  A
  // descriptor's start address is its low field, so every operand is a base descriptor plus a
  // constant.
  auto issue_conv = [&](auto ntiles, auto dil, uint32_t src, uint32_t plane, uint32_t wts) {
    constexpr int NT = decltype(ntiles)::value, D = decltype(dil)::value;
    const uint64_t a0 = umma_desc(src, plane, 128), b0 = umma_desc(wts, 512, 128);
    static_for<kK>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      static_for<2>([&](auto cc) {
        constexpr int c = decltype(cc)::value;
        const uint64_t bd = b0 + (uint64_t)((k * 2048 + c * 1024) >> 4);
        const uint64_t ac = a0 + (uint64_t)(((uint32_t)(k * D) * 16 + 2u * c * plane) >> 4);
        static_for<NT>([&](auto tt) {
          constexpr int t = decltype(tt)::value;
          umma_f16(tm + 32 * t, ac + (uint64_t)(128 * t), bd, kIdesc, (k | c) != 0);
        });
      });
    });
    umma_commit(bar);
  };

  const int64_t wstep = 2 * (int64_t)gridDim.x;
  int64_t w = 2 * (int64_t)blockIdx.x + g;
  if (w < p.n_blocks) load_x(w * HOP);
  for (; w < p.n_blocks; w += wstep) {
#pragma unroll
    for (int e = 0; e < kXPer; ++e) {
      const int j = gt + kGroupThreads * e;
      if (j < nx) sX[j] = fminf(power_of(xa[e]) * sc, kXCap);
    }
    if (gt < kC) sMax[gt] = 0u;
    group_sync(g);
    if (w + wstep < p.n_blocks) load_x((w + wstep) * HOP);   // next block, used next iteration
    // layer-1 im2col: row r (position P0-80+r) = x[r .. r+8], zero for K in [9, 16)
    for (int r = gt; r < 128 * T1; r += kGroupThreads) {
      __half2 h[8];
#pragma unroll
      for (int e = 0; e < 4; ++e) h[e] = __floats2half2_rn(sX[r + 2 * e], sX[r + 2 * e + 1]);
      h[4] = __floats2half2_rn(sX[r + 8], 0.f);
      h[5] = h[6] = h[7] = __floats2half2_rn(0.f, 0.f);
      *reinterpret_cast<uint4*>(sA1 + r * 16) = *reinterpret_cast<uint4*>(&h[0]);
      *reinterpret_cast<uint4*>(sA1 + kPlaneA1 + r * 16) = *reinterpret_cast<uint4*>(&h[4]);
    }
    sync_for_mma();
    if (gt == 0) {
      const uint64_t bd = umma_desc(aW1, 512, 128), a0 = umma_desc(aA1, kPlaneA1, 128);
      static_for<T1>([&](auto tt) {
        constexpr int t = decltype(tt)::value;
        umma_f16(tm + 32 * t, a0 + (uint64_t)(128 * t), bd, kIdesc, 0u);   // 128 rows x 16 B = 2048 B
      });
      umma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    store_layer(std::integral_constant<int, T1>{}, 128 * T2 + 8 * kDil2, sBias, sH1, kPlaneH1);
    sync_for_mma();
    if (gt == 0) issue_conv(std::integral_constant<int, T2>{}, std::integral_constant<int, kDil2>{}, aH1, kPlaneH1, aW2);
    if (!(ok = wait_mma())) break;
    store_layer(std::integral_constant<int, T2>{}, HOP + 8 * kDil3, sBias + kC, sH2, kPlaneH2);
    sync_for_mma();
    if (gt == 0) issue_conv(std::integral_constant<int, T3>{}, std::integral_constant<int, kDil3>{}, aH2, kPlaneH2, aW3);
    if (!(ok = wait_mma())) break;
    // layer 3: relu(acc + b3), channel maxima over the block: each thread keeps the maximum of
    // its rows, then one warp reduction per channel (non-negative floats order as unsigned)
    {
      float mx[kC];
#pragma unroll
      for (int c = 0; c < kC; ++c) mx[c] = 0.f;
      float a[2][16], b[2][16];
      tmem_ld16(tm_lane, a[0]);
      tmem_ld16(tm_lane + 16, b[0]);
      static_for<T3>([&](auto tt) {
        constexpr int t = decltype(tt)::value, cur = t & 1;
        tmem_wait_ld();
        if constexpr (t + 1 < T3) {
          tmem_ld16(tm_lane + 32 * (t + 1), a[cur ^ 1]);
          tmem_ld16(tm_lane + 32 * (t + 1) + 16, b[cur ^ 1]);
        }
#pragma unroll
        for (int c = 0; c < kC; ++c) mx[c] = fmaxf(mx[c], (c < 16 ? a[cur][c] : b[cur][c - 16]) + sBias[2 * kC + c]);
      });
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(mx[c], 0.f)));
        if (lane == c) atomicMax(&sMax[c], m);
      }
    }
    tmem_fence_before_sync();
    group_sync(g);
    // head: logits[w][j] = bl[j] + sum_c Wl[j][c] m[c]  (FP16 weights, FP32 sums)
    float mc[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) mc[c] = __uint_as_float(sMax[c]);
    for (int j = gt; j < p.Z; j += kGroupThreads) {
      const __half* wl = wl_staged ? sWl + j * kC : p.w + p.oWl + (size_t)j * kC;
      float s = wl_staged ? sBl[j] : __half2float(p.w[p.obl + j]);
#pragma unroll
      for (int c4 = 0; c4 < kC / 8; ++c4) {
        const uint4 u = *reinterpret_cast<const uint4*>(wl + 8 * c4);
        const __half2* h2 = reinterpret_cast<const __half2*>(&u);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = __half22float2(h2[e]);
          s = fmaf(f.x, mc[8 * c4 + 2 * e], s);
          s = fmaf(f.y, mc[8 * c4 + 2 * e + 1], s);
        }
      }
      p.logits[w * p.Z + j] = s;
    }
    group_sync(g);   // sMax and the staging area are reused by the next block
  }
  if (!ok && gt == 0) {
    atomicOr(p.status, 1);
    (void)mbar_wait(bar, phase ^ 1u);   // bounded wait for this group's MMAs still in flight
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(*tslot, kTmemCols);
}

}  // namespace

struct fdas_zband {
  int Wd = 0, Z = 0, max_batch = 0, sm_count = 0;
  Layout lay{0};
  float* p = nullptr;        // FP32 master parameters
  __half* ph = nullptr;      // FP16 copy for inference
  float* g = nullptr;        // gradients
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* a1 = nullptr;       // pre-activations [B][C][Wd]
  float* a2 = nullptr;
  float* a3 = nullptr;
  float* d1 = nullptr;       // gradient buffers [B][C][Wd]
  float* d2 = nullptr;
  float* pooled = nullptr;   // [B][C]
  int* arg = nullptr;        // [B][C]
  float* logits = nullptr;   // [B][Z]
  float* dlog = nullptr;     // [B][Z]
  float* loss = nullptr;     // device scalar
  float* loss_part = nullptr; // per-warp loss partials [ceil(B*Z / 32)]
  float* wpart = nullptr;    // weight-gradient partials [B * Wd/128][C*C*9 + C]
  SelectState* sel = nullptr; // median selection state
  float* scale = nullptr;    // ln 2 / median |A|^2
  int* status = nullptr;     // bit 0: a bounded wait of the inference kernel gave up
  int step = 0;
  // fdas_zband_propose as a CUDA graph of its launches, captured for these arguments
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  const void* cap_spec = nullptr;
  int64_t cap_n = 0;
  const void* cap_logits = nullptr;
  // the synchronous host accessors run on `own`; `done` marks the last work enqueued on the net
  // (they and fdas_zband_destroy wait for it, not for the whole device)
  cudaStream_t own = nullptr;
  cudaEvent_t done = nullptr;
};

namespace {
void free_zband(fdas_zband* z) {
  void* ptrs[] = {z->p,      z->ph,  z->g,      z->m,    z->v,         z->a1,     z->a2,
                  z->a3,     z->d1,  z->d2,     z->pooled, z->arg,    z->logits, z->dlog,
                  z->loss,   z->loss_part, z->wpart, z->sel, z->scale, z->status};
  for (void* q : ptrs) cudaFree(q);
  if (z->graph_exec) cudaGraphExecDestroy(z->graph_exec);
  if (z->graph) cudaGraphDestroy(z->graph);
  if (z->capture_stream) cudaStreamDestroy(z->capture_stream);
  if (z->own) cudaStreamDestroy(z->own);
  if (z->done) cudaEventDestroy(z->done);
  delete z;
}

// Record the net's completion event after work enqueued on `st` (not while `st` is being captured
// into a CUDA graph: a captured record is no event the host can wait on).
int note_work(fdas_zband* z, cudaStream_t st, cudaError_t launch) {
  if (launch != cudaSuccess) return FDAS_ERR_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FDAS_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return FDAS_OK;
  return cudaEventRecord(z->done, st) == cudaSuccess ? FDAS_OK : FDAS_ERR_CUDA;
}

// Host copy between the net's buffers and host memory on its own stream, after the net's last
// enqueued work; returns when the copy has completed.
int host_copy(fdas_zband* z, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  if (cudaStreamWaitEvent(z->own, z->done, 0) != cudaSuccess ||
      cudaMemcpyAsync(dst, src, bytes, kind, z->own) != cudaSuccess || cudaStreamSynchronize(z->own) != cudaSuccess)
    return FDAS_ERR_CUDA;
  return FDAS_OK;
}

// Layers 1..3, pooling and head on B windows `in` (FP32 activations; FP32 or FP16 weights).
cudaError_t forward(fdas_zband* z, const float* in, int B, bool half_weights, cudaStream_t st) {
  const Layout& L = z->lay;
  const dim3 grid(z->Wd / kTile, B);
  if (half_weights) {
    const __half* h = z->ph;
    conv_fwd_kernel<1, false, __half, kDil1>
        <<<grid, 256, conv_fwd_smem<1, kDil1>(), st>>>(in, h + L.W1, h + L.b1, z->a1, z->Wd);
    conv_fwd_kernel<kC, true, __half, kDil2>
        <<<grid, 256, conv_fwd_smem<kC, kDil2>(), st>>>(z->a1, h + L.W2, h + L.b2, z->a2, z->Wd);
    conv_fwd_kernel<kC, true, __half, kDil3>
        <<<grid, 256, conv_fwd_smem<kC, kDil3>(), st>>>(z->a2, h + L.W3, h + L.b3, z->a3, z->Wd);
    pool_head_kernel<__half><<<B, 256, 0, st>>>(z->a3, h + L.Wl, h + L.bl, z->Wd, z->Z, z->pooled, z->arg, z->logits);
  } else {
    const float* p = z->p;
    conv_fwd_kernel<1, false, float, kDil1>
        <<<grid, 256, conv_fwd_smem<1, kDil1>(), st>>>(in, p + L.W1, p + L.b1, z->a1, z->Wd);
    conv_fwd_kernel<kC, true, float, kDil2>
        <<<grid, 256, conv_fwd_smem<kC, kDil2>(), st>>>(z->a1, p + L.W2, p + L.b2, z->a2, z->Wd);
    conv_fwd_kernel<kC, true, float, kDil3>
        <<<grid, 256, conv_fwd_smem<kC, kDil3>(), st>>>(z->a2, p + L.W3, p + L.b3, z->a3, z->Wd);
    pool_head_kernel<float><<<B, 256, 0, st>>>(z->a3, p + L.Wl, p + L.bl, z->Wd, z->Z, z->pooled, z->arg, z->logits);
  }
  return cudaGetLastError();
}

// scale = ln 2 / median |A|^2 into `scale`: seven launches.
void launch_power_scale(const float2* spec, int64_t n, SelectState* sel, float* scale, cudaStream_t st) {
  select_init_kernel<<<1, 256, 0, st>>>(sel, n);
  const int64_t blocks = (n + 256 * kSelPer - 1) / (256 * kSelPer);
  const unsigned grid = (unsigned)(blocks < kSelBlocks ? blocks : kSelBlocks);
  // passes 1 and 2 flush up to 4096 bins per block: fewer, longer blocks
  const unsigned grid12 = (unsigned)(blocks < kSelBlocks12 ? blocks : kSelBlocks12);
  select_pass_kernel<0><<<grid, 256, 0, st>>>(spec, n, sel);
  select_digit_kernel<0><<<1, 256, 0, st>>>(sel, scale);
  select_pass_kernel<1><<<grid12, 256, 0, st>>>(spec, n, sel);
  select_digit_kernel<1><<<1, 256, 0, st>>>(sel, scale);
  select_pass_kernel<2><<<grid12, 256, 0, st>>>(spec, n, sel);
  select_digit_kernel<2><<<1, 256, 0, st>>>(sel, scale);
}
}  // namespace

extern "C" {

fdas_zband* fdas_zband_create(int window, int n_out, int max_batch) {
  // the window's quarter margins must hold the receptive field (the windowed and whole-sequence
  // forms then agree)
  if (window < 4 * kRF || window % kTile != 0 || window > (1 << 16) || n_out < 1 || n_out > 65535 ||
      max_batch < 1 || max_batch > 65535)
    return nullptr;
  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) || major != 10 || minor != 3) {
    cudaGetLastError();
    return nullptr;
  }
  constexpr auto kSmemAttr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (cudaFuncSetAttribute(conv_fwd_kernel<kC, true, float, kDil2>, kSmemAttr, (int)conv_fwd_smem<kC, kDil2>()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(conv_fwd_kernel<kC, true, float, kDil3>, kSmemAttr, (int)conv_fwd_smem<kC, kDil3>()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(conv_fwd_kernel<kC, true, __half, kDil2>, kSmemAttr, (int)conv_fwd_smem<kC, kDil2>()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(conv_fwd_kernel<kC, true, __half, kDil3>, kSmemAttr, (int)conv_fwd_smem<kC, kDil3>()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(conv_bwd_data_kernel<kDil2>, kSmemAttr, (int)bwd_data_smem<kDil2>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_bwd_data_kernel<kDil3>, kSmemAttr, (int)bwd_data_smem<kDil3>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_bwd_weight_kernel<kC, true, kDil2>, kSmemAttr, (int)bwd_weight_smem<kC, kDil2>()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(conv_bwd_weight_kernel<kC, true, kDil3>, kSmemAttr, (int)bwd_weight_smem<kC, kDil3>()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(propose_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProposeSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(propose_kernel<384>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProposeSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(propose_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProposeSmem) !=
          cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  fdas_zband* z = new (std::nothrow) fdas_zband();
  if (!z) return nullptr;
  z->Wd = window;
  z->Z = n_out;
  z->max_batch = max_batch;
  z->sm_count = sms;
  z->lay = Layout(n_out);
  const size_t P = (size_t)z->lay.total, B = (size_t)max_batch, act = B * kC * (size_t)window;
  bool ok = cudaMalloc(&z->p, P * 4) == cudaSuccess && cudaMalloc(&z->ph, P * 2) == cudaSuccess &&
            cudaMalloc(&z->g, P * 4) == cudaSuccess && cudaMalloc(&z->m, P * 4) == cudaSuccess &&
            cudaMalloc(&z->v, P * 4) == cudaSuccess && cudaMalloc(&z->a1, act * 4) == cudaSuccess &&
            cudaMalloc(&z->a2, act * 4) == cudaSuccess && cudaMalloc(&z->a3, act * 4) == cudaSuccess &&
            cudaMalloc(&z->d1, act * 4) == cudaSuccess && cudaMalloc(&z->d2, act * 4) == cudaSuccess &&
            cudaMalloc(&z->pooled, B * kC * 4) == cudaSuccess && cudaMalloc(&z->arg, B * kC * 4) == cudaSuccess &&
            cudaMalloc(&z->logits, B * (size_t)n_out * 4) == cudaSuccess &&
            cudaMalloc(&z->dlog, B * (size_t)n_out * 4) == cudaSuccess && cudaMalloc(&z->loss, 4) == cudaSuccess &&
            cudaMalloc(&z->loss_part, (B * (size_t)n_out + 31) / 32 * 4) == cudaSuccess &&
            cudaMalloc(&z->wpart, B * (size_t)(window / kTile) * ((size_t)kC * kC * kK + kC) * 4) == cudaSuccess &&
            cudaMalloc(&z->sel, sizeof(SelectState)) == cudaSuccess &&
            cudaMalloc(&z->scale, 4) == cudaSuccess && cudaMalloc(&z->status, 4) == cudaSuccess &&
            cudaStreamCreateWithFlags(&z->own, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&z->done, cudaEventDisableTiming) == cudaSuccess;
  if (!ok || cudaMemsetAsync(z->p, 0, P * 4, z->own) != cudaSuccess ||
      cudaMemsetAsync(z->ph, 0, P * 2, z->own) != cudaSuccess || cudaMemsetAsync(z->m, 0, P * 4, z->own) != cudaSuccess ||
      cudaMemsetAsync(z->v, 0, P * 4, z->own) != cudaSuccess || cudaMemsetAsync(z->status, 0, 4, z->own) != cudaSuccess ||
      cudaEventRecord(z->done, z->own) != cudaSuccess || cudaStreamSynchronize(z->own) != cudaSuccess) {
    cudaGetLastError();
    free_zband(z);
    return nullptr;
  }
  return z;
}

int fdas_zband_param_count(const fdas_zband* z) { return z ? z->lay.total : FDAS_ERR_INVALID; }

int fdas_zband_set_params(fdas_zband* z, const float* host_params) {
  if (!z || !host_params) return FDAS_ERR_INVALID;
  const int P = z->lay.total;
  if (host_copy(z, z->p, host_params, (size_t)P * 4, cudaMemcpyHostToDevice) != FDAS_OK) return FDAS_ERR_CUDA;
  to_half_kernel<<<(P + 255) / 256, 256, 0, z->own>>>(z->p, z->ph, P);
  cudaMemsetAsync(z->m, 0, (size_t)P * 4, z->own);
  cudaMemsetAsync(z->v, 0, (size_t)P * 4, z->own);
  z->step = 0;
  if (note_work(z, z->own, cudaGetLastError()) != FDAS_OK) return FDAS_ERR_CUDA;
  return cudaStreamSynchronize(z->own) == cudaSuccess ? FDAS_OK : FDAS_ERR_CUDA;
}

int fdas_zband_get_params(fdas_zband* z, float* host_params) {
  if (!z || !host_params) return FDAS_ERR_INVALID;
  return host_copy(z, host_params, z->p, (size_t)z->lay.total * 4, cudaMemcpyDeviceToHost);
}

int fdas_zband_get_adam(fdas_zband* z, float* host_m, float* host_v, int* host_step) {
  if (!z || !host_m || !host_v || !host_step) return FDAS_ERR_INVALID;
  const size_t bytes = (size_t)z->lay.total * 4;
  if (host_copy(z, host_m, z->m, bytes, cudaMemcpyDeviceToHost) != FDAS_OK ||
      host_copy(z, host_v, z->v, bytes, cudaMemcpyDeviceToHost) != FDAS_OK)
    return FDAS_ERR_CUDA;
  *host_step = z->step;
  return FDAS_OK;
}

int fdas_zband_set_adam(fdas_zband* z, const float* host_m, const float* host_v, int step) {
  if (!z || !host_m || !host_v || step < 0) return FDAS_ERR_INVALID;
  const size_t bytes = (size_t)z->lay.total * 4;
  if (host_copy(z, z->m, host_m, bytes, cudaMemcpyHostToDevice) != FDAS_OK ||
      host_copy(z, z->v, host_v, bytes, cudaMemcpyHostToDevice) != FDAS_OK)
    return FDAS_ERR_CUDA;
  z->step = step;
  return FDAS_OK;
}

int fdas_zband_train_step(fdas_zband* z, const float* d_windows, const float* d_targets, int batch, float lr,
                          float* host_loss, fdas_stream_t stream) {
  if (!z || !d_windows || !d_targets || batch < 1 || batch > z->max_batch || !(lr > 0.f)) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Layout& L = z->lay;
  const int B = batch, Wd = z->Wd, Z = z->Z, P = L.total;
  if (forward(z, d_windows, B, false, st) != cudaSuccess) return FDAS_ERR_CUDA;
  bce_grad_kernel<<<(B * Z + 255) / 256, 256, 0, st>>>(z->logits, d_targets, B * Z, z->dlog, z->loss_part);
  sum_fixed_kernel<<<1, 1024, 0, st>>>(z->loss_part, (B * Z + 31) / 32, z->loss);
  head_bwd_weights_kernel<<<(Z * (kC + 1) + 255) / 256, 256, 0, st>>>(z->dlog, z->pooled, B, Z, z->g + L.Wl,
                                                                       z->g + L.bl);
  const size_t act = (size_t)B * kC * Wd;
  cudaMemsetAsync(z->d1, 0, act * 4, st);
  head_bwd_data_kernel<<<B, kC, 0, st>>>(z->dlog, z->p + L.Wl, z->arg, z->a3, Z, Wd, z->d1);   // da3
  const dim3 grid(Wd / kTile, B);
  const int nblk = B * (Wd / kTile);
  // partials of layer `cin` inputs, then their fixed-order sum into the W and b slices (W then b
  // are adjacent in the parameter layout)
  auto reduce = [&](int cin, int w_off) {
    const int n = kC * cin * kK + kC;
    reduce_partials_kernel<<<(n + 255) / 256, 256, 0, st>>>(z->wpart, nblk, n, n, z->g + w_off);
  };
  conv_bwd_weight_kernel<kC, true, kDil3><<<grid, 256, bwd_weight_smem<kC, kDil3>(), st>>>(z->a2, z->d1, Wd, z->wpart);
  reduce(kC, L.W3);
  conv_bwd_data_kernel<kDil3><<<grid, 256, bwd_data_smem<kDil3>(), st>>>(z->d1, z->p + L.W3, z->a2, z->d2, Wd);   // da2
  conv_bwd_weight_kernel<kC, true, kDil2><<<grid, 256, bwd_weight_smem<kC, kDil2>(), st>>>(z->a1, z->d2, Wd, z->wpart);
  reduce(kC, L.W2);
  conv_bwd_data_kernel<kDil2><<<grid, 256, bwd_data_smem<kDil2>(), st>>>(z->d2, z->p + L.W2, z->a1, z->d1, Wd);   // da1
  conv_bwd_weight_kernel<1, false, kDil1><<<grid, 256, bwd_weight_smem<1, kDil1>(), st>>>(d_windows, z->d1, Wd, z->wpart);
  reduce(1, L.W1);
  z->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)z->step), c2 = 1.f - powf(b2, (float)z->step);
  adam_kernel<<<(P + 255) / 256, 256, 0, st>>>(z->p, z->g, z->m, z->v, P, lr, b1, b2, 1e-8f, c1, c2);
  to_half_kernel<<<(P + 255) / 256, 256, 0, st>>>(z->p, z->ph, P);
  if (note_work(z, st, cudaGetLastError()) != FDAS_OK) return FDAS_ERR_CUDA;
  if (host_loss) {
    if (cudaMemcpyAsync(host_loss, z->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FDAS_ERR_CUDA;
  }
  return FDAS_OK;
}

int fdas_zband_gradients(fdas_zband* z, float* host_grads) {
  if (!z || !host_grads) return FDAS_ERR_INVALID;
  return host_copy(z, host_grads, z->g, (size_t)z->lay.total * 4, cudaMemcpyDeviceToHost);
}

int fdas_zband_predict(fdas_zband* z, const float* d_windows, int batch, int half_weights, float* d_logits,
                       fdas_stream_t stream) {
  if (!z || !d_windows || !d_logits || batch < 1) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int b0 = 0; b0 < batch; b0 += z->max_batch) {
    const int B = batch - b0 < z->max_batch ? batch - b0 : z->max_batch;
    if (forward(z, d_windows + (size_t)b0 * z->Wd, B, half_weights != 0, st) != cudaSuccess) return FDAS_ERR_CUDA;
    if (cudaMemcpyAsync(d_logits + (size_t)b0 * z->Z, z->logits, (size_t)B * z->Z * 4, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
      return FDAS_ERR_CUDA;
  }
  return note_work(z, st, cudaGetLastError());
}

// The launches of one proposal (median passes, then the fused inference) on `st`.
static cudaError_t launch_propose(fdas_zband* z, const float* d_spectrum, int64_t n_bins, float* d_logits,
                                  cudaStream_t st) {
  const int hop = z->Wd / 2;
  const int64_t nb = (n_bins + hop - 1) / hop;
  launch_power_scale(reinterpret_cast<const float2*>(d_spectrum), n_bins, z->sel, z->scale, st);
  ProposeParams q;
  q.spec = reinterpret_cast<const float2*>(d_spectrum);
  q.n = n_bins;
  q.scale = z->scale;
  q.w = z->ph;
  q.oW1 = z->lay.W1;
  q.ob1 = z->lay.b1;
  q.oW2 = z->lay.W2;
  q.ob2 = z->lay.b2;
  q.oW3 = z->lay.W3;
  q.ob3 = z->lay.b3;
  q.oWl = z->lay.Wl;
  q.obl = z->lay.bl;
  q.Z = z->Z;
  q.hop = hop;
  q.n_blocks = nb;
  q.logits = d_logits;
  q.status = z->status;
  const int64_t pairs = (nb + 1) / 2;
  const unsigned grid = (unsigned)(pairs < z->sm_count ? pairs : z->sm_count);
  switch (hop) {
    case 256: propose_kernel<256><<<grid, 256, kProposeSmem, st>>>(q); break;
    case 384: propose_kernel<384><<<grid, 256, kProposeSmem, st>>>(q); break;
    default: propose_kernel<512><<<grid, 256, kProposeSmem, st>>>(q); break;
  }
  return cudaGetLastError();
}

int fdas_zband_propose(fdas_zband* z, const float* d_spectrum, int64_t n_bins, float* d_logits,
                       fdas_stream_t stream) {
  if (!z || !d_spectrum || !d_logits || n_bins < 1 || n_bins > (int64_t(1) << 30)) return FDAS_ERR_INVALID;
  const int hop = z->Wd / 2;
  if (hop % 128 != 0 || hop > kMaxHop) return FDAS_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(d_spectrum) & 7u) || (reinterpret_cast<uintptr_t>(d_logits) & 3u))
    return FDAS_ERR_ALIGN;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // eight launches replayed as one graph: captured again when the spectrum, its length or the
  // logits buffer change (the weights are read through fixed pointers, so training needs none)
  if (!(z->graph_exec && z->cap_spec == d_spectrum && z->cap_n == n_bins && z->cap_logits == d_logits)) {
    if (z->graph_exec) cudaGraphExecDestroy(z->graph_exec);
    if (z->graph) cudaGraphDestroy(z->graph);
    z->graph_exec = nullptr;
    z->graph = nullptr;
    if (!z->capture_stream && cudaStreamCreateWithFlags(&z->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
      z->capture_stream = nullptr;
      return FDAS_ERR_CUDA;
    }
    if (cudaStreamBeginCapture(z->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return FDAS_ERR_CUDA;
    const cudaError_t le = launch_propose(z, d_spectrum, n_bins, d_logits, z->capture_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(z->capture_stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return FDAS_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&z->graph_exec, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      z->graph_exec = nullptr;
      cudaGetLastError();
      return FDAS_ERR_CUDA;
    }
    z->graph = g;
    z->cap_spec = d_spectrum;
    z->cap_n = n_bins;
    z->cap_logits = d_logits;
  }
  return note_work(z, st, cudaGraphLaunch(z->graph_exec, st));
}

int fdas_zband_check(fdas_zband* z, fdas_stream_t stream) {
  if (!z) return FDAS_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int status = 0;
  if (cudaMemcpyAsync(&status, z->status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FDAS_ERR_CUDA;
  if (status != 0) {
    if (cudaMemsetAsync(z->status, 0, 4, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      return FDAS_ERR_CUDA;
    return FDAS_ERR_TIMEOUT;
  }
  return FDAS_OK;
}

int fdas_zband_spectrum_windows(const float* d_spectrum, int64_t n_bins, int window, int hop, float* d_windows,
                                int64_t n_windows, fdas_stream_t stream) {
  if (!d_spectrum || !d_windows || n_bins < 1 || n_bins > (int64_t(1) << 30) || window < 4 || window % 4 != 0 ||
      window > (1 << 16) || hop < 1 || n_windows < 1 || n_windows > (1 << 30))
    return FDAS_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d_spectrum) & 7u) return FDAS_ERR_ALIGN;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SelectState* sel = nullptr;
  float* scale = nullptr;
  if (cudaMallocAsync(&sel, sizeof(SelectState), st) != cudaSuccess) return FDAS_ERR_ALLOC;
  if (cudaMallocAsync(&scale, 4, st) != cudaSuccess) {
    cudaFreeAsync(sel, st);
    return FDAS_ERR_ALLOC;
  }
  launch_power_scale(reinterpret_cast<const float2*>(d_spectrum), n_bins, sel, scale, st);
  spectrum_windows_kernel<<<(unsigned)n_windows, 256, 0, st>>>(reinterpret_cast<const float2*>(d_spectrum), n_bins,
                                                               scale, window, hop, d_windows);
  const int rc = cudaGetLastError() == cudaSuccess ? FDAS_OK : FDAS_ERR_CUDA;
  cudaFreeAsync(sel, st);
  cudaFreeAsync(scale, st);
  return rc;
}

// Work-list scratch: offsets (int64, n_groups + 1), counts (int32, n_groups), segment masks
// (uint16, n_groups * Z), each 16-byte aligned.
static int64_t align16(int64_t x) { return (x + 15) & ~(int64_t)15; }
static int64_t units_scratch_bytes(int64_t n_groups, int Z) {
  return align16(8 * (n_groups + 1)) + align16(4 * n_groups) + align16(2 * n_groups * (int64_t)Z);
}

int64_t fdas_zband_work_units_scratch_bytes(int64_t n_groups, int Z) {
  if (n_groups < 1 || n_groups > (1 << 24) || Z < 1 || n_groups * (int64_t)Z > INT32_MAX) return FDAS_ERR_INVALID;
  return units_scratch_bytes(n_groups, Z);
}

int fdas_zband_work_units_masked(const float* d_logits, int64_t n_windows, int Z, float threshold, int hop,
                                 int64_t seg_bins, int G, int h, int64_t n_groups, int32_t* d_units,
                                 uint16_t* d_masks, void* d_scratch, int64_t* host_count, fdas_stream_t stream) {
  if (!d_logits || !d_units || (!host_count && !d_scratch) || n_windows < 1 || n_windows > (1 << 30) || Z < 1 ||
      !(threshold > 0.f && threshold < 1.f) || hop < 1 || seg_bins < 1 || G < 1 || G > 16 || h < 0 ||
      n_groups < 1 || n_groups > (1 << 24) || (int64_t)n_groups * Z > INT32_MAX ||
      seg_bins * G > (int64_t(1) << 40))
    return FDAS_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(d_scratch) & 15u) || (reinterpret_cast<uintptr_t>(d_masks) & 1u))
    return FDAS_ERR_ALIGN;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float logit_thr = logf(threshold / (1.f - threshold));
  const int64_t bytes = units_scratch_bytes(n_groups, Z);
  unsigned char* scratch = static_cast<unsigned char*>(d_scratch);
  const bool own = scratch == nullptr;
  if (own && cudaMallocAsync(reinterpret_cast<void**>(&scratch), (size_t)bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return FDAS_ERR_ALLOC;
  }
  int64_t* offsets = reinterpret_cast<int64_t*>(scratch);
  int* counts = reinterpret_cast<int*>(scratch + align16(8 * (n_groups + 1)));
  uint16_t* masks = reinterpret_cast<uint16_t*>(scratch + align16(8 * (n_groups + 1)) + align16(4 * n_groups));
  group_flags_kernel<<<(unsigned)n_groups, 256, 0, st>>>(d_logits, (int)n_windows, Z, logit_thr, hop, seg_bins, G,
                                                        h, (int)n_groups, masks, counts);
  scan_counts_kernel<<<1, 1024, 0, st>>>(counts, (int)n_groups, offsets, offsets + n_groups);
  write_units_kernel<<<(unsigned)n_groups, 256, 0, st>>>(masks, offsets, Z, d_units, d_masks);
  int rc = FDAS_OK;
  if (cudaGetLastError() != cudaSuccess) rc = FDAS_ERR_CUDA;
  else if (host_count && (cudaMemcpyAsync(host_count, offsets + n_groups, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                          cudaStreamSynchronize(st) != cudaSuccess))
    rc = FDAS_ERR_CUDA;
  if (own) cudaFreeAsync(scratch, st);
  return rc;
}

int fdas_zband_work_units(const float* d_logits, int64_t n_windows, int Z, float threshold, int hop,
                          int64_t group_bins, int h, int64_t n_groups, int32_t* d_units, void* d_scratch,
                          int64_t* host_count, fdas_stream_t stream) {
  // one segment of group_bins per group: the group's flag
  return fdas_zband_work_units_masked(d_logits, n_windows, Z, threshold, hop, group_bins, 1, h, n_groups, d_units,
                                      nullptr, d_scratch, host_count, stream);
}

int fdas_zband_work_pairs(const float* d_logits, int64_t n_windows, int Z, float threshold, float reach_threshold,
                          int z_halo, int hop, int64_t seg_bins, int h, int64_t n_seg, int32_t* d_pairs,
                          void* d_scratch, int64_t* host_count, fdas_stream_t stream) {
  if (!d_logits || !d_pairs || !d_scratch || n_windows < 1 || n_windows > (1 << 30) || Z < 1 || Z > 8192 ||
      !(threshold > 0.f && threshold < 1.f) || !(reach_threshold >= threshold && reach_threshold <= 1.f) ||
      z_halo < 0 || z_halo > Z || hop < 1 || seg_bins < 1 || h < 0 ||
      n_seg < 1 || n_seg > (1 << 24) || n_seg * (int64_t)Z > INT32_MAX || seg_bins > (int64_t(1) << 40))
    return FDAS_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(d_scratch) & 15u) || (reinterpret_cast<uintptr_t>(d_logits) & 3u) ||
      (reinterpret_cast<uintptr_t>(d_pairs) & 3u))
    return FDAS_ERR_ALIGN;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float logit_thr = logf(threshold / (1.f - threshold));
  const float logit_reach = reach_threshold < 1.f ? logf(reach_threshold / (1.f - reach_threshold)) : INFINITY;
  unsigned char* scratch = static_cast<unsigned char*>(d_scratch);
  int64_t* offsets = reinterpret_cast<int64_t*>(scratch);
  int* counts = reinterpret_cast<int*>(scratch + align16(8 * (n_seg + 1)));
  uint16_t* masks = reinterpret_cast<uint16_t*>(scratch + align16(8 * (n_seg + 1)) + align16(4 * n_seg));
  segment_flags_kernel<<<(unsigned)n_seg, 256, sizeof(int) * (size_t)Z, st>>>(
      d_logits, (int)n_windows, Z, logit_thr, logit_reach, z_halo, hop, seg_bins, h, masks, counts);
  scan_counts_kernel<<<1, 1024, 0, st>>>(counts, (int)n_seg, offsets, offsets + n_seg);
  write_units_kernel<<<(unsigned)n_seg, 256, 0, st>>>(masks, offsets, Z, d_pairs, nullptr);
  if (cudaGetLastError() != cudaSuccess) return FDAS_ERR_CUDA;
  if (host_count && (cudaMemcpyAsync(host_count, offsets + n_seg, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess))
    return FDAS_ERR_CUDA;
  return FDAS_OK;
}

int fdas_zband_destroy(fdas_zband* z) {
  if (!z) return FDAS_OK;
  if (z->done) cudaEventSynchronize(z->done);   // the net's last enqueued work, not the whole device
  free_zband(z);
  return FDAS_OK;
}

}  // extern "C"
