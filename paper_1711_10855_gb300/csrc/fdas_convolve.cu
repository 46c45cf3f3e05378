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
//   pass 1: lane k1 holds Y[k1 + N1*k2], k2 < N2, as N2/2 packed pairs and does its N2-point DFT
//           in registers (two N2/2-point DFTs in lockstep with packed f32x2 butterflies, then one
//           scalar stage joining them),
//   twist:  multiply by exp(SIGN i 2pi n2 k1 / L) (packed),
//   exchange: one shared-memory transposition of 16-byte pair entries through a padded tile,
//   pass 2: lane t holds two columns n2 (a packed pair) and runs two N1-point DFTs in lockstep;
//           output index n = n2 + N2*n1, so lane t ends with outputs n = t (mod N1).
// The paper's design (Section 2: shuffle stage for N <= 32, shared memory above, 4 elements per
// thread) is replaced by two register passes with compile-time FMA butterflies on packed pairs
// and a single shared-memory exchange per transform.
//
// Work decomposition: a CTA of 8 warps owns G consecutive segments at a time ("group"); the
// flattened (group, z) list is split into contiguous equal ranges, one per CTA (grid = #SMs),
// so every CTA does the same number of inverse transforms.  P warps share a segment and take
// alternate templates.
#include <cstdio>
#include <type_traits>

#include "fdas_device.cuh"
#include "fdas_internal.h"

// The decoupled work-list instantiation leaves the shared-ring loop of the kernel unreachable.
#pragma nv_diag_suppress 128

namespace fdas {

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <int L_, int N1_, int P_, int XR_, int R_ = 4>
struct ConvCfg {
  static constexpr int L = L_;
  static constexpr int N1 = N1_;           // lanes per transform
  static constexpr int N2 = L / N1;        // points per lane in pass 1
  static constexpr int H2 = N2 / 2;        // pass-1 pairs per lane
  static constexpr int F = 32 / N1;        // transform groups per warp
  static constexpr int W = 8;              // compute warps per CTA
  static constexpr int P = P_;             // warps sharing one segment
  static constexpr int G = F * W / P;      // segments resident per CTA
  static constexpr int R = R_;             // template ring slots
  static constexpr int C = N2 / N1;        // pass-2 columns per lane
  static constexpr int CP = C / 2;         // pass-2 column pairs per lane (= exchange row rounds)
  static constexpr int XR = XR_;           // exchange sub-rounds (lane halves writing in turn)
  static constexpr int XCOLS = N1 / XR;    // exchange tile columns per sub-round
  static constexpr int XPITCH = XCOLS + 1; // 16-byte entries per tile row (odd: conflict-free)
  static constexpr int XGROUP = N1 * XPITCH;
  static constexpr int XWARP = F * XGROUP;
  static constexpr int LOG_N1 = ilog2(N1);
  static constexpr int LOG_N2 = ilog2(N2);
  static constexpr int BOX = L < 256 ? L : 256;   // TMA box (elements of 8 bytes)
  static constexpr size_t OFF_X = 0;
  static constexpr size_t OFF_T = OFF_X + (size_t)G * L * 8;
  static constexpr size_t OFF_TW = OFF_T + (size_t)R * L * 8;
  static constexpr size_t OFF_XB = OFF_TW + (size_t)L * 8;
  static constexpr size_t OFF_BAR = align_up(OFF_XB + (size_t)W * XWARP * 16, 128);
  static constexpr size_t SMEM = OFF_BAR + 256;
  static_assert(N1 * N2 == L && C >= 2 && C % 2 == 0 && 32 % N1 == 0, "bad decomposition");
  static_assert(N1 % XR == 0 && XCOLS % 2 == 0, "bad exchange split");
  static_assert(L % BOX == 0, "segment must be whole boxes");
  static_assert(SMEM <= 232448, "shared memory budget");
};

// ---------------------------------------------------------------------------------------
// Shared per-lane pieces of the transform
//
// Buffer layout of a segment spectrum, a template spectrum and the twiddle table (L complex
// values each), "pair-major structure of arrays": lane k1 of the first pass owns the pairs
// p = 0..H2-1; pair p of lane k1 is the float4 at index p*N1 + k1 holding
// (re(e0), re(e1), im(e0), im(e1)).  For spectra and templates e0, e1 are the elements
// k = k1 + N1*(2p) and k1 + N1*(2p+1); for the twiddle table they are exp(+i 2pi n2 k1 / L)
// for n2 = p and p + H2.  One 128-bit load gives a packed pair ready for f32x2 arithmetic.
// ---------------------------------------------------------------------------------------

// Pass 1 of the inverse transform on entry: v[i] = (Y[k1 + N1*bitrev(i)], Y[k1 + N1*(bitrev(i)+1)]),
// i < H2 (bitrev over log2 N2 bits of an even index is < H2).  After fft_split_pairs:
// v[j] = (Z[j], Z[j + H2]) for the lane's N2-point DFT; the twist then multiplies by the
// twiddle pair of row j.
template <class Cfg, bool CONJ>
__device__ __forceinline__ void apply_twist2(cp2 (&v)[Cfg::H2], const float4* __restrict__ stw, int k1) {
  static_for<Cfg::H2>([&](auto jj) {
    constexpr int j = decltype(jj)::value;
    const cp2 w = cp2_from(stw[j * Cfg::N1 + k1]);
    v[j] = CONJ ? cmul2_conj(v[j], w) : cmul2(v[j], w);
  });
}

// Exchange + pass 2.  Lane k1's pair j = r*N1 + t holds columns n2 = t + N1*r and
// t + N1*(r + CP) of row k1; lane t gathers, for its column pair r, the entries of all N1 lanes
// and runs two N1-point DFTs in lockstep.  Round r moves rows j in [r*N1, (r+1)*N1) through a
// tile of N1 rows x XCOLS lanes (XR sub-rounds, lanes [h*XCOLS, (h+1)*XCOLS) writing in turn).
// out(r, n1, pair) receives (y[t + N1*r + N2*n1], y[t + N1*(r+CP) + N2*n1]).
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

template <class Cfg, int SIGN, class Out, class AfterReads = NoHook>
__device__ __forceinline__ void exchange_and_pass2(cp2 (&v)[Cfg::H2], float4* xb, int k1, Out&& out,
                                                   AfterReads&& after_reads = AfterReads{}) {
  static_for<Cfg::CP>([&](auto rr) {
    constexpr int r = decltype(rr)::value;
    cp2 u[Cfg::N1];
    static_for<Cfg::XR>([&](auto hh) {
      constexpr int h = decltype(hh)::value;
      __syncwarp();
      if (k1 / Cfg::XCOLS == h) {
        const int c = k1 - h * Cfg::XCOLS;
        static_for<Cfg::N1>([&](auto ii) {
          constexpr int i = decltype(ii)::value;
          xb[i * Cfg::XPITCH + c] = cp2_to(v[r * Cfg::N1 + i]);
        });
      }
      __syncwarp();
      static_for<Cfg::XCOLS>([&](auto cc) {
        constexpr int c = decltype(cc)::value;
        constexpr int src = h * Cfg::XCOLS + c;   // the writing lane k1'
        u[bitrev(src, Cfg::LOG_N1)] = cp2_from(xb[k1 * Cfg::XPITCH + c]);
      });
    });
    if constexpr (r == Cfg::CP - 1) after_reads();   // the tile is free once its last round is read
    fft_pair_columns<Cfg::N1, SIGN>(u);
    static_for<Cfg::N1>([&](auto nn) {
      constexpr int n1 = decltype(nn)::value;
      out(std::integral_constant<int, r>{}, std::integral_constant<int, n1>{}, u[n1]);
    });
  });
}

// Forward FFT (Eq. 3) of one segment held in natural order (complex64) in sx;
// out(r, n1, pair) receives (X[t + N1*r + N2*n1], X[t + N1*(r+CP) + N2*n1]).
template <class Cfg, class Twist, class Out>
__device__ __forceinline__ void forward_transform_with(const float2* sx, Twist&& twist_conj, float4* xb, int k1,
                                                       Out&& out) {
  cp2 v[Cfg::H2];
  static_for<Cfg::H2>([&](auto ii) {
    constexpr int i = decltype(ii)::value;
    constexpr int k2 = bitrev(i, Cfg::LOG_N2);
    const float2 a = sx[k1 + Cfg::N1 * k2];
    const float2 b = sx[k1 + Cfg::N1 * (k2 + 1)];
    v[i] = cp2{make_float2(a.x, b.x), make_float2(a.y, b.y)};
  });
  fft_split_pairs<Cfg::N2, -1>(v);
  twist_conj(v);
  exchange_and_pass2<Cfg, -1>(v, xb, k1, out);
}
template <class Cfg, class Out>
__device__ __forceinline__ void forward_transform(const float2* sx, const float4* __restrict__ stw, float4* xb,
                                                  int k1, Out&& out) {
  forward_transform_with<Cfg>(sx, [&](cp2 (&v)[Cfg::H2]) { apply_twist2<Cfg, true>(v, stw, k1); }, xb, k1, out);
}

// Twist with the twiddle pairs held in this lane's TMEM row (4 columns per pair, chunks of 4 pairs).
template <class Cfg, bool CONJ>
__device__ __forceinline__ void apply_twist_tmem(cp2 (&v)[Cfg::H2], uint32_t tw_addr) {
  static_assert(Cfg::H2 % 8 == 0, "twist chunking");
  static_for<Cfg::H2 / 8>([&](auto cc) {
    constexpr int c = decltype(cc)::value;
    float r0[16], r1[16];
    tmem_ld16(tw_addr + 32 * c, r0);
    tmem_ld16(tw_addr + 32 * c + 16, r1);
    tmem_wait_ld();
    static_for<4>([&](auto qq) {
      constexpr int q = decltype(qq)::value;
      const cp2 w0 = cp2{make_float2(r0[4 * q], r0[4 * q + 1]), make_float2(r0[4 * q + 2], r0[4 * q + 3])};
      const cp2 w1 = cp2{make_float2(r1[4 * q], r1[4 * q + 1]), make_float2(r1[4 * q + 2], r1[4 * q + 3])};
      v[8 * c + q] = CONJ ? cmul2_conj(v[8 * c + q], w0) : cmul2(v[8 * c + q], w0);
      v[8 * c + 4 + q] = CONJ ? cmul2_conj(v[8 * c + 4 + q], w1) : cmul2(v[8 * c + 4 + q], w1);
    });
  });
}

// Store X[n] (held by lane t = n mod N1) into the pair-major layout of the inverse transform.
template <class Cfg>
__device__ __forceinline__ void store_spectrum_element(float* sx, int t, int k2, float re, float im) {
  const int base = ((k2 >> 1) * Cfg::N1 + t) * 4 + (k2 & 1);
  sx[base] = re;
  sx[base + 2] = im;
}

// One arrival on a shared-memory consumer counter with acquire-release semantics at CTA scope: the
// caller's earlier reads of the slot (ordered within the warp by __syncwarp) happen before the
// arrival, and the last arriver's later refill of the slot happens after every other arrival.
// Returns the count before this arrival.
__device__ __forceinline__ unsigned arrive_count(unsigned* counter) {
  unsigned old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(smem_u32(counter)) : "memory");
  return old;
}

// Bounded wait for a template slot: the common case (already filled) costs one try_wait; the abort
// flag is read only when the slot is not ready, so one warp's timeout stops the others quickly.
__device__ __forceinline__ int wait_slot(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return 1;
  if (*abort_flag) return 0;
  return mbar_wait(bar, parity) ? 1 : 0;
}

// Device status word: set kStatusTimeout when a bounded wait gave up.
__device__ __forceinline__ void report_timeout(int* status, volatile int* abort_flag) {
  *abort_flag = 1;
  atomicOr(status, kStatusTimeout);
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
  float4* sXb = reinterpret_cast<float4*>(smem + Cfg::OFF_XB);
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
  float4* myXb = sXb + warp * Cfg::XWARP + gw * Cfg::XGROUP;
  const float4* stw4 = reinterpret_cast<const float4*>(sTw);

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
      // a3: forward FFT in place; X[n] goes to the pair-major layout of the inverse transform
      forward_transform<Cfg>(myX, stw4, myXb, k1, [&](auto rr, auto nn, const cp2& x) {
        constexpr int r = decltype(rr)::value, n1 = decltype(nn)::value;
        float* sx = reinterpret_cast<float*>(myX);
        store_spectrum_element<Cfg>(sx, k1, r + Cfg::C * n1, x.re.x, x.im.x);
        store_spectrum_element<Cfg>(sx, k1, r + Cfg::CP + Cfg::C * n1, x.re.y, x.im.y);
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
      const int ok = __all_sync(0xffffffffu, wait_slot(&full[slot], (uint32_t)((i / R) & 1), abort_flag));
      if (!ok) {
        if (lane == 0) report_timeout(p.status, abort_flag);
        break;
      }
      const int64_t z = (u0 + i) % p.Z;
      const float2* st = sT + (size_t)slot * L;

      // a4: Y = X * T, loaded as packed pairs in the first pass's bit-reversed order
      cp2 v[Cfg::H2];
      static_for<Cfg::H2>([&](auto pp) {
        constexpr int q = decltype(pp)::value;
        const cp2 x = cp2_from(reinterpret_cast<const float4*>(myX)[q * N1 + k1]);
        const cp2 t = cp2_from(reinterpret_cast<const float4*>(st)[q * N1 + k1]);
        v[bitrev(2 * q, Cfg::LOG_N2)] = cmul2(x, t);
      });
      // release the template slot; the last of the W/P consumers refills it R positions ahead
      __syncwarp();
      if (lane == 0) {
        const unsigned old = arrive_count(&cnt[slot]);
        if ((old + 1u) % (unsigned)(Cfg::W / P) == 0u) {
          if (i + R < npos) {
            fence_proxy_async_smem();
            issue_template(i + R);
          }
        }
      }
      // a5: inverse FFT
      fft_split_pairs<Cfg::N2, +1>(v);
      apply_twist2<Cfg, false>(v, stw4, k1);
      float* row = p.plane + z * p.n_bins + segbase;
      exchange_and_pass2<Cfg, +1>(v, myXb, k1, [&](auto rr, auto nn, const cp2& y) {
        // a6 + a7: keep n < V (and inside the spectrum), store |y|^2
        constexpr int r = decltype(rr)::value, n1 = decltype(nn)::value;
        const float2 pw = power2(y);
        const int n_lo = r * N1 + k1 + Cfg::N2 * n1;
        const int n_hi = n_lo + Cfg::CP * N1;
        if (n_lo < lim) __stcs(row + n_lo, pw.x);
        if (n_hi < lim) __stcs(row + n_hi, pw.y);
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

// ---------------------------------------------------------------------------------------
// Variant with the segment spectra and the twiddle table in tensor memory (one column pair per
// lane: N2 = 2*N1, i.e. L = 512 and 2048).  Every warp owns its own segment(s); the template of
// each position is read from the shared-memory ring by all 8 warps.  Per inverse transform the
// shared-memory traffic is the template (L*8 bytes) and the exchange (2*L*8 bytes); the
// spectrum and the twiddles come from TMEM, a separate store, which relieves the shared-memory
// bandwidth that otherwise co-limits the kernel with the FP32 pipe.
// ---------------------------------------------------------------------------------------
template <int L_, int N1_>
struct TmemCfg {
  static constexpr int L = L_;
  static constexpr int N1 = N1_;
  static constexpr int N2 = L / N1;
  static constexpr int H2 = N2 / 2;
  static constexpr int F = 32 / N1;
  static constexpr int W = 8;
  static constexpr int P = 1;
  static constexpr int G = F * W;          // segments resident per CTA: one group of lanes each
  static constexpr int R = 4;
  static constexpr int C = 2;
  static constexpr int CP = 1;
  static constexpr int XR = 1;
  static constexpr int XCOLS = N1;
  static constexpr int XPITCH = N1 + 1;
  static constexpr int XGROUP = N1 * XPITCH;
  static constexpr int XWARP = F * XGROUP;
  static constexpr int LOG_N1 = ilog2(N1);
  static constexpr int LOG_N2 = ilog2(N2);
  static constexpr int BOX = L < 256 ? L : 256;
  // per-warp shared region: staging of its segments, then its exchange tiles
  static constexpr size_t REGION = align_up(((size_t)F * L * 8 > (size_t)XWARP * 16) ? (size_t)F * L * 8
                                                                                     : (size_t)XWARP * 16, 128);
  static constexpr size_t OFF_T = 0;
  static constexpr size_t OFF_REG = OFF_T + (size_t)R * L * 8;
  static constexpr size_t OFF_BAR = align_up(OFF_REG + (size_t)W * REGION, 128);
  static constexpr size_t SMEM = OFF_BAR + 256;
  // TMEM columns of each quadrant: twiddles, then the spectra of its two warps
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr uint32_t COL_TW = 0;
  static constexpr uint32_t COL_X = 2 * N2;
  static_assert(N2 == 2 * N1 && 32 % N1 == 0, "one column pair per lane");
  static_assert(6 * N2 <= (int)TMEM_COLS, "TMEM columns");
  static_assert(SMEM <= 232448, "shared memory budget");
};

// Spectrum b holding flattened unit u (largest b with unit_base <= u).
__device__ __forceinline__ int find_spectrum(const BatchParams& p, int64_t u) {
  if (p.descs == nullptr) return 0;
  int lo = 0, hi = p.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.descs[mid].unit_base <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ SpecDesc spectrum_desc(const BatchParams& p, int b) {
  return p.descs == nullptr ? p.single : p.descs[b];
}

// Units to compute: all of them, or the list length (from device memory when the list was made on
// the device; the check kernel has bounded it by the list's capacity p.units).
__device__ __forceinline__ int64_t unit_total(const BatchParams& p) { return p.units; }
__device__ __forceinline__ int64_t unit_total(const ListParams& p) { return p.unit_count ? *p.unit_count : p.units; }

// NV: pass-2 output rows n1 < NV can hold valid outputs (NV >= ceil(V / N2)); rows n1 >= NV are
// dropped at compile time, which also removes the butterfly halves that only feed them.
//
// Work: units (spectrum b, segment group g, template z) flattened over all spectra; each CTA
// takes a contiguous equal range.  Segment s of spectrum b is brought in by one bulk copy of its
// part inside [0, n_b) (cp.async.bulk) and the rest of the L-bin window is zero-filled by the
// owning warp.
//
// DEC (work lists with segment masks only): the warps are decoupled.  Instead of the shared
// template ring, each warp walks only the positions where one of its segments is listed and
// brings that position's template into its own shared region by a bulk copy, issued as soon as
// the region's exchange tile has been read (so it lands while the warp finishes the previous
// transform).  The time of a group is then set by its busiest warp, not by the number of listed
// units: sparse masks cost about their share of (segment, template) pairs.
template <class Cfg, int NV, bool LIST, bool DEC = false>
__global__ void __launch_bounds__(256, 1)
    fdas_convolve_tmem_kernel(const std::conditional_t<LIST, ListParams, BatchParams> p) {
  static_assert(!DEC || LIST, "decoupled warps serve masked work lists");
  constexpr int L = Cfg::L, N1 = Cfg::N1, R = Cfg::R, G = Cfg::G, H2 = Cfg::H2, W = Cfg::W;
  extern __shared__ __align__(1024) unsigned char smem[];
  float2* sT = reinterpret_cast<float2*>(smem + Cfg::OFF_T);
  unsigned char* sReg = smem + Cfg::OFF_REG;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::OFF_BAR);
  uint64_t* segbar = full + R;
  int64_t* issued_pos = reinterpret_cast<int64_t*>(segbar + 1);
  unsigned* cnt = reinterpret_cast<unsigned*>(issued_pos + R);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(cnt + R);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(cnt + R + 1);
  // template-refill cursor (positions are issued in increasing order, one thread at a time)
  struct IssueCursor {
    int64_t u;          // unit of the next position to issue
    int64_t spec_end;   // first unit of the next spectrum
    int b, z, Z, z_off; // its spectrum, template index within it, that spectrum's Z and bank offset
  };
  IssueCursor* cur = reinterpret_cast<IssueCursor*>(smem + Cfg::OFF_BAR + 128);
  uint64_t* wbar = reinterpret_cast<uint64_t*>(smem + Cfg::OFF_BAR + 192);   // [W] per-warp template copies (DEC)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gw = lane / N1, k1 = lane % N1;
  float2* myRegion = reinterpret_cast<float2*>(sReg + (size_t)warp * Cfg::REGION);
  float2* mySeg = myRegion + (size_t)gw * L;
  float4* myXb = reinterpret_cast<float4*>(myRegion) + gw * Cfg::XGROUP;

  // a work list that failed its check (kStatusBadList, set by the preceding check kernel) is not
  // run
  if constexpr (LIST) {
    if (*reinterpret_cast<volatile const int*>(p.status) & kStatusBadList) return;
  }
  const int64_t U = unit_total(p);
  // flattened unit of list entry e (identity without a work list)
  auto unit_at = [&](int64_t e) -> int64_t {
    if constexpr (LIST) return (int64_t)__ldg(p.unit_list + e);
    else return e;
  };
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
    if constexpr (DEC)
      for (int w = 0; w < W; ++w) mbar_init(&wbar[w], 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem_row = *tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t tw_addr = tmem_row + Cfg::COL_TW;
  const uint32_t x_addr = tmem_row + Cfg::COL_X + (uint32_t)(warp >> 2) * (2 * Cfg::N2);

  // Template of CTA position i (unit u0 + i): bank row z_off_b + (u - unit_base_b) mod Z_b.  The
  // cursor walks units in order, so an issue costs a few shared-memory operations; a descriptor is
  // read from global memory only when the walk enters the next spectrum.
  auto issue_template = [&](int64_t i) {
    const int slot = (int)(i % R);
    issued_pos[slot] = i;
    int64_t zrow;
    if constexpr (LIST) zrow = cur->z_off + unit_at(u0 + i) % cur->Z;
    else zrow = cur->z_off + cur->z;
    mbar_arrive_expect_tx(&full[slot], L * 8);
    bulk_g2s(sT + (size_t)slot * L, p.templates + (size_t)zrow * L, L * 8, &full[slot]);
    if constexpr (LIST) return;   // single spectrum: the cursor's spectrum never changes
    cur->u += 1;
    cur->z = cur->z + 1 == cur->Z ? 0 : cur->z + 1;
    if (cur->u == cur->spec_end && cur->u < U) {
      const int nb = cur->b + 1;
      const SpecDesc dn = spectrum_desc(p, nb);
      cur->b = nb;
      cur->z = 0;
      cur->Z = dn.Z;
      cur->z_off = dn.z_off;
      cur->spec_end = nb + 1 < p.count ? spectrum_desc(p, nb + 1).unit_base : U;
    }
  };
  if (tid == 0 && !DEC) {
    const int b0 = find_spectrum(p, u0);
    const SpecDesc d0 = spectrum_desc(p, b0);
    cur->u = u0;
    cur->b = b0;
    cur->Z = d0.Z;
    cur->z_off = d0.z_off;
    cur->z = (int)((u0 - d0.unit_base) % d0.Z);
    cur->spec_end = b0 + 1 < p.count ? spectrum_desc(p, b0 + 1).unit_base : U;
    const int64_t first = npos < R ? npos : R;
    for (int64_t i = 0; i < first; ++i) issue_template(i);
  }
  // twiddle pairs of lane k1 into this quadrant's TMEM rows (one warp per quadrant)
  if (warp < 4) {
    const float4* tw4 = reinterpret_cast<const float4*>(p.twist);
    static_for<H2 / 4>([&](auto cc) {
      constexpr int c = decltype(cc)::value;
      float r[16];
      static_for<4>([&](auto qq) {
        constexpr int q = decltype(qq)::value;
        const float4 w = __ldg(tw4 + (4 * c + q) * N1 + k1);
        r[4 * q] = w.x;
        r[4 * q + 1] = w.y;
        r[4 * q + 2] = w.z;
        r[4 * q + 3] = w.w;
      });
      tmem_st16(tw_addr + 16 * c, r);
    });
    tmem_wait_st();
  }
  // release template slot `slot` of position i; the last of the W consumers refills it R positions
  // ahead
  auto release_slot = [&](int64_t i, int slot) {
    __syncwarp();
    if (lane == 0) {
      const unsigned old = arrive_count(&cnt[slot]);
      if ((old + 1u) % (unsigned)W == 0u) {
        if (i + R < npos) {
          fence_proxy_async_smem();
          issue_template(i + R);
        }
      }
    }
  };
  tmem_fence_before_sync();
  int alive = 1;
  uint32_t seg_phase = 0;
  bool seg_in_flight = false;
  uint32_t w_phase = 0;        // DEC: parity of this warp's next template copy
  bool w_in_flight = false;    // DEC: a copy into this warp's region not yet waited for
  int64_t u = u0;
  while (u < u1) {
    // the segment group holding entry u (a run of list entries with the same group)
    const int64_t uu = unit_at(u);
    const int b = find_spectrum(p, uu);
    const SpecDesc d = spectrum_desc(p, b);
    const int64_t grp = (uu - d.unit_base) / d.Z;
    const int64_t z_first = (uu - d.unit_base) % d.Z;
    int64_t grp_end;
    if constexpr (LIST) {
      grp_end = u + 1;
      while (grp_end < u1 && unit_at(grp_end) / d.Z == grp) ++grp_end;
    } else {
      grp_end = d.unit_base + (grp + 1) * d.Z;
    }
    const int64_t a = u - u0;
    const int64_t bpos = (grp_end < u1 ? grp_end : u1) - u0;
    u = u0 + bpos;
    // every warp is done with its region (previous exchanges) before segments land in it
    alive = __syncthreads_and(alive && !*abort_flag);
    tmem_fence_after_sync();
    if (!alive) break;
    if (tid == 0) {
      // a2: bulk copies of the in-range part of every segment of the group
      uint32_t bytes = 0;
      for (int j = 0; j < G; ++j) {
        const int64_t x0 = (grp * G + j) * (int64_t)p.V - p.h;
        const int64_t c0 = x0 > 0 ? x0 : 0;
        const int64_t c1 = x0 + L < d.n_bins ? x0 + L : d.n_bins;
        if (c1 > c0) bytes += (uint32_t)((c1 - c0) * 8);
      }
      mbar_arrive_expect_tx(segbar, bytes);
      for (int j = 0; j < G; ++j) {
        float2* dst = reinterpret_cast<float2*>(sReg + (size_t)(j / Cfg::F) * Cfg::REGION) + (size_t)(j % Cfg::F) * L;
        const int64_t x0 = (grp * G + j) * (int64_t)p.V - p.h;
        const int64_t c0 = x0 > 0 ? x0 : 0;
        const int64_t c1 = x0 + L < d.n_bins ? x0 + L : d.n_bins;
        if (c1 > c0) bulk_g2s(dst + (c0 - x0), d.spec + c0, (uint32_t)((c1 - c0) * 8), segbar);
      }
    }
    {
      // zeros outside [0, n_b) in this lane group's window
      const int64_t x0 = (grp * G + warp * Cfg::F + gw) * (int64_t)p.V - p.h;
      const int64_t lo = x0 < 0 ? (-x0 < L ? -x0 : L) : 0;                           // [0, lo) below 0
      const int64_t hi = d.n_bins - x0 < L ? (d.n_bins - x0 > 0 ? d.n_bins - x0 : 0) : L;  // [hi, L) beyond n
      for (int e = k1; e < L; e += N1)
        if (e < lo || e >= hi) mySeg[e] = make_float2(0.f, 0.f);
    }
    seg_in_flight = true;
    alive = __syncthreads_and(mbar_wait(segbar, seg_phase) ? 1 : 0);
    if (!alive) {
      if (tid == 0) report_timeout(p.status, abort_flag);
      break;
    }
    seg_in_flight = false;
    seg_phase ^= 1u;

    // a3: forward FFT of this lane group's segment; X pairs (k2 = 2p, 2p+1) go to TMEM
    {
      float xr[16];
      forward_transform_with<Cfg>(
          mySeg, [&](cp2 (&v)[H2]) { apply_twist_tmem<Cfg, true>(v, tw_addr); }, myXb, k1,
          [&](auto, auto nn, const cp2& x) {
            constexpr int n1 = decltype(nn)::value;   // pair p = n1
            xr[4 * (n1 & 3)] = x.re.x;
            xr[4 * (n1 & 3) + 1] = x.re.y;
            xr[4 * (n1 & 3) + 2] = x.im.x;
            xr[4 * (n1 & 3) + 3] = x.im.y;
            if constexpr ((n1 & 3) == 3) tmem_st16(x_addr + 4 * (n1 - 3), xr);
          });
      tmem_wait_st();
    }

    const int64_t s = grp * G + warp * Cfg::F + gw;
    const int64_t segbase = s * (int64_t)p.V;
    const int64_t lim64 = d.n_bins - segbase < (int64_t)p.V ? d.n_bins - segbase : (int64_t)p.V;
    const int lim = lim64 > 0 ? (int)lim64 : 0;
    if constexpr (DEC) {
      // this warp's segment bits of list position i (warp-uniform)
      auto warp_bits = [&](int64_t i) -> unsigned {
        return ((unsigned)__ldg(p.unit_mask + u0 + i) >> (warp * Cfg::F)) & ((1u << Cfg::F) - 1u);
      };
      auto next_active = [&](int64_t i) {
        while (i < bpos && warp_bits(i) == 0u) ++i;
        return i;
      };
      // template of position i into this warp's region (lane 0; the region's earlier generic
      // accesses are ordered before the asynchronous copy)
      auto fetch = [&](int64_t i) {
        __syncwarp();
        if (lane == 0) {
          fence_proxy_async_smem();
          const int64_t zrow = unit_at(u0 + i) % d.Z;
          mbar_arrive_expect_tx(&wbar[warp], L * 8);
          bulk_g2s(myRegion, p.templates + (size_t)zrow * L, L * 8, &wbar[warp]);
        }
        w_in_flight = true;
      };
      int64_t i = next_active(a);
      if (i < bpos) fetch(i);
      while (i < bpos) {
        const int ok = __all_sync(0xffffffffu, wait_slot(&wbar[warp], w_phase, abort_flag));
        if (!ok) {   // the copy stays in flight: the exit path waits for it (bounded)
          if (lane == 0) report_timeout(p.status, abort_flag);
          break;
        }
        w_in_flight = false;
        w_phase ^= 1u;
        const int64_t z = unit_at(u0 + i) % d.Z;
        const int lim_z = ((warp_bits(i) >> gw) & 1u) ? lim : 0;
        const float4* st4 = reinterpret_cast<const float4*>(myRegion);
        cp2 v[H2];
        static_for<H2 / 8>([&](auto cc) {
          constexpr int c = decltype(cc)::value;
          float x0[16], x1[16];
          tmem_ld16(x_addr + 32 * c, x0);
          tmem_ld16(x_addr + 32 * c + 16, x1);
          float4 t[8];
          static_for<8>([&](auto qq) {
            constexpr int q = decltype(qq)::value;
            t[q] = st4[(8 * c + q) * N1 + k1];
          });
          tmem_wait_ld();
          static_for<8>([&](auto qq) {
            constexpr int q = decltype(qq)::value;
            constexpr int pp = 8 * c + q;
            const float* xs = q < 4 ? &x0[4 * q] : &x1[4 * (q - 4)];
            const cp2 x = cp2{make_float2(xs[0], xs[1]), make_float2(xs[2], xs[3])};
            v[bitrev(2 * pp, Cfg::LOG_N2)] = cmul2(x, cp2_from(t[q]));
          });
        });
        const int64_t inext = next_active(i + 1);
        fft_split_pairs<Cfg::N2, +1>(v);
        apply_twist_tmem<Cfg, false>(v, tw_addr);
        float* row = d.plane + z * d.n_bins + segbase;
        exchange_and_pass2<Cfg, +1>(
            v, myXb, k1,
            [&](auto, auto nn, const cp2& y) {
              constexpr int n1 = decltype(nn)::value;
              if constexpr (n1 < NV) {
                const float2 pw = power2(y);
                const int n_lo = k1 + Cfg::N2 * n1;
                const int n_hi = n_lo + N1;
                if (n_lo < lim_z) __stcs(row + n_lo, pw.x);
                if (n_hi < lim_z) __stcs(row + n_hi, pw.y);
              }
            },
            [&]() {
              if (inext < bpos) fetch(inext);
            });
        i = inext;
      }
      // after a timeout the abort flag is set: every warp leaves at the group barrier above
      tmem_fence_before_sync();
      continue;
    }
    for (int64_t i = a; i < bpos; ++i) {
      const int slot = (int)(i % R);
      const int ok = __all_sync(0xffffffffu, wait_slot(&full[slot], (uint32_t)((i / R) & 1), abort_flag));
      if (!ok) {
        if (lane == 0) report_timeout(p.status, abort_flag);
        break;
      }
      // row of this position: consecutive templates without a list, the entry's own with one
      int64_t z;
      if constexpr (LIST) z = unit_at(u0 + i) % d.Z;
      else z = z_first + (int64_t)(i - a);
      const float4* st4 = reinterpret_cast<const float4*>(sT + (size_t)slot * L);
      // a masked list entry: a warp none of whose segments is listed skips the transform (it still
      // releases the slot); lanes of an unlisted segment store nothing
      bool warp_on = true, group_on = true;
      if constexpr (LIST) {
        if (p.unit_mask) {
          const unsigned wm = ((unsigned)__ldg(p.unit_mask + u0 + i) >> (warp * Cfg::F)) & ((1u << Cfg::F) - 1u);
          warp_on = wm != 0u;
          group_on = ((wm >> gw) & 1u) != 0u;
        }
      }

      if (!warp_on) {   // the slot is released unread
        release_slot(i, slot);
        continue;
      }
      const int lim_z = group_on ? lim : 0;

      // a4: Y = X (TMEM) * T (shared ring), packed pairs in bit-reversed order, four pairs per
      // chunk (a sweep of equivalent orderings timed this one 0.5% faster than eight)
      cp2 v[H2];
      static_for<H2 / 4>([&](auto cc) {
        constexpr int c = decltype(cc)::value;
        float x0[16];
        tmem_ld16(x_addr + 16 * c, x0);
        float4 t[4];
        static_for<4>([&](auto qq) {
          constexpr int q = decltype(qq)::value;
          t[q] = st4[(4 * c + q) * N1 + k1];
        });
        tmem_wait_ld();
        static_for<4>([&](auto qq) {
          constexpr int q = decltype(qq)::value;
          constexpr int pp = 4 * c + q;
          const cp2 x = cp2{make_float2(x0[4 * q], x0[4 * q + 1]), make_float2(x0[4 * q + 2], x0[4 * q + 3])};
          v[bitrev(2 * pp, Cfg::LOG_N2)] = cmul2(x, cp2_from(t[q]));
        });
      });
      release_slot(i, slot);
      // a5: inverse FFT
      fft_split_pairs<Cfg::N2, +1>(v);
      apply_twist_tmem<Cfg, false>(v, tw_addr);
      float* row = d.plane + z * d.n_bins + segbase;
      exchange_and_pass2<Cfg, +1>(v, myXb, k1, [&](auto, auto nn, const cp2& y) {
        // a6 + a7: keep n < V (and inside the spectrum), store |y|^2
        constexpr int n1 = decltype(nn)::value;
        if constexpr (n1 < NV) {
          const float2 pw = power2(y);
          const int n_lo = k1 + Cfg::N2 * n1;
          const int n_hi = n_lo + N1;
          if (n_lo < lim_z) __stcs(row + n_lo, pw.x);
          if (n_hi < lim_z) __stcs(row + n_hi, pw.y);
        }
      });
    }
    tmem_fence_before_sync();
  }

  // After a timeout, wait (bounded) for this CTA's copies still in flight; always free TMEM.
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (tid == 0 && (*abort_flag || !alive)) {
    for (int r = 0; r < R; ++r)
      if (issued_pos[r] >= 0) (void)mbar_wait(&full[r], (uint32_t)((issued_pos[r] / R) & 1));
    if (seg_in_flight) (void)mbar_wait(segbar, seg_phase);
  }
  if constexpr (DEC) {
    if (lane == 0 && w_in_flight) (void)mbar_wait(&wbar[warp], w_phase);   // bounded
  }
  if (warp == 0) tmem_dealloc(*tmem_slot, Cfg::TMEM_COLS);
}

// Pair-list kernel (one transform per warp, L = 2048).  The listed (segment s, template z) pairs,
// entries s*Z + z in ascending order, are cut into equal contiguous ranges, one per warp of the
// grid, so a sparse list costs about its share of the full plane's transforms whatever its
// layout.  The warps are independent: a warp whose range enters a new segment brings it into its
// shared region (bulk copy of the part inside [0, n), zero fill of the rest) and runs the forward
// transform (Eq. 3) into its TMEM columns; for every pair it brings the template into the same
// region (bulk copy, issued as soon as the previous transform's exchange tile has been read when
// the next pair has the same segment), multiplies, runs the inverse transform and stores |y|^2
// for the segment's valid outputs (Section 2, overlap-and-save).  One mbarrier per warp serves
// both kinds of copy, at most one of them in flight.
template <class Cfg, int NV>
__global__ void __launch_bounds__(256, 1) fdas_convolve_pairs_kernel(const PairParams p) {
  static_assert(Cfg::F == 1, "one transform per warp");
  constexpr int L = Cfg::L, N1 = Cfg::N1, H2 = Cfg::H2, W = Cfg::W;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* wbar = reinterpret_cast<uint64_t*>(smem + (size_t)W * Cfg::REGION);   // [W]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(wbar + W);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wbar + W) + 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, k1 = lane;
  float2* myRegion = reinterpret_cast<float2*>(smem + (size_t)warp * Cfg::REGION);
  float4* myXb = reinterpret_cast<float4*>(myRegion);
  uint64_t* bar = &wbar[warp];

  // a list that failed its check (kStatusBadList, set by the preceding check kernel) is not run
  if (*reinterpret_cast<volatile const int*>(p.status) & kStatusBadList) return;
  const int64_t P = p.pair_count ? *p.pair_count : p.n_pairs;
  const int64_t NW = (int64_t)gridDim.x * W;
  const int64_t cta0 = (int64_t)blockIdx.x * W;
  if ((cta0 + W) * P / NW == cta0 * P / NW) return;   // no pair for this CTA (uniform)
  const int64_t e0 = (cta0 + warp) * P / NW, e1 = (cta0 + warp + 1) * P / NW;

  if (tid == 0) {
    for (int w = 0; w < W; ++w) mbar_init(&wbar[w], 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem_row = *tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t tw_addr = tmem_row + Cfg::COL_TW;
  const uint32_t x_addr = tmem_row + Cfg::COL_X + (uint32_t)(warp >> 2) * (2 * Cfg::N2);
  // twiddle pairs of lane k1 into this quadrant's TMEM rows (one warp per quadrant)
  if (warp < 4) {
    const float4* tw4 = reinterpret_cast<const float4*>(p.twist);
    static_for<H2 / 4>([&](auto cc) {
      constexpr int c = decltype(cc)::value;
      float r[16];
      static_for<4>([&](auto qq) {
        constexpr int q = decltype(qq)::value;
        const float4 w = __ldg(tw4 + (4 * c + q) * N1 + k1);
        r[4 * q] = w.x;
        r[4 * q + 1] = w.y;
        r[4 * q + 2] = w.z;
        r[4 * q + 3] = w.w;
      });
      tmem_st16(tw_addr + 16 * c, r);
    });
    tmem_wait_st();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();

  uint32_t phase = 0;
  bool in_flight = false;   // a copy into this warp's region not yet waited for (warp-uniform)
  // bounded wait for the copy in flight; false after a timeout (the copy stays marked in flight)
  auto wait_copy = [&]() -> bool {
    const int ok = __all_sync(0xffffffffu, wait_slot(bar, phase, abort_flag));
    if (!ok) {
      if (lane == 0) report_timeout(p.status, abort_flag);
      return false;
    }
    in_flight = false;
    phase ^= 1u;
    return true;
  };
  // template z into the region (its earlier generic accesses are ordered before the copy)
  auto fetch_template = [&](int z) {
    __syncwarp();
    if (lane == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, L * 8);
      bulk_g2s(myRegion, p.templates + (size_t)z * L, L * 8, bar);
    }
    in_flight = true;
  };

  int64_t cur_s = -1;
  for (int64_t e = e0; e < e1; ++e) {
    const int32_t u = __ldg(p.pairs + e);   // checked: 0 <= u < nseg*Z <= 2^31 - 1
    const int s32 = u / p.Z;                 // 32-bit division
    const int64_t s = s32;
    const int z = u - s32 * p.Z;
    if (s != cur_s) {
      // a2: the segment's window A[sV - h, sV - h + L): bulk copy of its part inside [0, n) (even
      // bounds: n and h are multiples of 4, so every copy is whole 16-byte units), zeros elsewhere
      const int64_t x0 = s * (int64_t)p.V - p.h;
      const int64_t c0 = x0 > 0 ? x0 : 0;
      const int64_t c1 = x0 + L < p.n_bins ? x0 + L : p.n_bins;
      __syncwarp();
      if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (uint32_t)((c1 - c0) * 8));
        bulk_g2s(myRegion + (c0 - x0), p.spec + c0, (uint32_t)((c1 - c0) * 8), bar);
      }
      in_flight = true;
      for (int i = k1; i < L; i += N1)
        if (x0 + i < c0 || x0 + i >= c1) myRegion[i] = make_float2(0.f, 0.f);
      if (!wait_copy()) break;
      __syncwarp();
      // a3: forward FFT of the segment; X pairs (k2 = 2p, 2p+1) go to TMEM
      float xr[16];
      forward_transform_with<Cfg>(
          myRegion, [&](cp2 (&v)[H2]) { apply_twist_tmem<Cfg, true>(v, tw_addr); }, myXb, k1,
          [&](auto, auto nn, const cp2& x) {
            constexpr int n1 = decltype(nn)::value;
            xr[4 * (n1 & 3)] = x.re.x;
            xr[4 * (n1 & 3) + 1] = x.re.y;
            xr[4 * (n1 & 3) + 2] = x.im.x;
            xr[4 * (n1 & 3) + 3] = x.im.y;
            if constexpr ((n1 & 3) == 3) tmem_st16(x_addr + 4 * (n1 - 3), xr);
          });
      tmem_wait_st();
      cur_s = s;
      fetch_template(z);
    }
    if (!wait_copy()) break;
    // the next pair's template is fetched during this transform when it has the same segment
    int znext = -1;
    if (e + 1 < e1) {
      const int32_t un = __ldg(p.pairs + e + 1);
      if (un / p.Z == s32) znext = un - s32 * p.Z;
    }
    // a4: Y = X (TMEM) * T (this warp's region), packed pairs in bit-reversed order
    const float4* st4 = reinterpret_cast<const float4*>(myRegion);
    cp2 v[H2];
    static_for<H2 / 4>([&](auto cc) {
      constexpr int c = decltype(cc)::value;
      float x0[16];
      tmem_ld16(x_addr + 16 * c, x0);
      float4 t[4];
      static_for<4>([&](auto qq) {
        constexpr int q = decltype(qq)::value;
        t[q] = st4[(4 * c + q) * N1 + k1];
      });
      tmem_wait_ld();
      static_for<4>([&](auto qq) {
        constexpr int q = decltype(qq)::value;
        constexpr int pp = 4 * c + q;
        const cp2 x = cp2{make_float2(x0[4 * q], x0[4 * q + 1]), make_float2(x0[4 * q + 2], x0[4 * q + 3])};
        v[bitrev(2 * pp, Cfg::LOG_N2)] = cmul2(x, cp2_from(t[q]));
      });
    });
    // a5: inverse FFT; a6 + a7: keep n < V inside the spectrum, store |y|^2
    fft_split_pairs<Cfg::N2, +1>(v);
    apply_twist_tmem<Cfg, false>(v, tw_addr);
    const int64_t segbase = s * (int64_t)p.V;
    const int64_t lim64 = p.n_bins - segbase < (int64_t)p.V ? p.n_bins - segbase : (int64_t)p.V;
    const int lim = (int)lim64;
    float* row = p.plane + (int64_t)z * p.n_bins + segbase;
    exchange_and_pass2<Cfg, +1>(
        v, myXb, k1,
        [&](auto, auto nn, const cp2& y) {
          constexpr int n1 = decltype(nn)::value;
          if constexpr (n1 < NV) {
            const float2 pw = power2(y);
            const int n_lo = k1 + Cfg::N2 * n1;
            const int n_hi = n_lo + N1;
            if (n_lo < lim) __stcs(row + n_lo, pw.x);
            if (n_hi < lim) __stcs(row + n_hi, pw.y);
          }
        },
        [&]() {
          if (znext >= 0) fetch_template(znext);
        });
  }

  // a copy still in flight after a timeout: wait for it (bounded); always free TMEM
  if (lane == 0 && in_flight) (void)mbar_wait(bar, phase);
  __syncwarp();
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(*tmem_slot, Cfg::TMEM_COLS);
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
  float4* sXb = reinterpret_cast<float4*>(sTw + L);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + align_up(((size_t)GS * L + L) * 8 + (size_t)8 * Cfg::XWARP * 16, 128));
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
      atomicOr(p.status, kStatusTimeout);
      (void)mbar_wait(bar, 0);   // bounded wait for copies still in flight
    }
    return;
  }
  const int64_t s = s0 + slot;
  float2* dst = p.out + s * L;
  const bool valid = s < p.nseg;
  forward_transform<Cfg>(sX + (size_t)slot * L, reinterpret_cast<const float4*>(sTw),
                         sXb + warp * Cfg::XWARP + gw * Cfg::XGROUP, k1, [&](auto rr, auto nn, const cp2& x) {
                           const int n = decltype(rr)::value * N1 + k1 + Cfg::N2 * decltype(nn)::value;
                           if (valid) {
                             dst[n] = make_float2(x.re.x, x.im.x);
                             dst[n + Cfg::CP * N1] = make_float2(x.re.y, x.im.y);
                           }
                         });
}

// ---------------------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------------------
int conv_group_threads(int L) { return L <= 256 ? 8 : (L <= 1024 ? 16 : (L <= 2048 ? 32 : 0)); }

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
  constexpr size_t smem = align_up(((size_t)GS * Cfg::L + Cfg::L) * 8 + (size_t)8 * Cfg::XWARP * 16, 128) + 64;
  static_assert(smem <= 232448, "shared memory budget of the segment-spectra kernel");
  auto kern = fdas_segment_spectra_kernel<Cfg>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = (p.nseg + GS - 1) / GS;
  kern<<<(unsigned)grid, 256, smem, st>>>(*map, p);
  return cudaGetLastError();
}

using Cfg256 = ConvCfg<256, 8, 1, 1>;
using Cfg512 = ConvCfg<512, 16, 1, 1>;
using Cfg1024 = ConvCfg<1024, 16, 2, 1>;
using Cfg2048 = ConvCfg<2048, 32, 4, 1, 2>;

template <class Cfg, int NV>
static cudaError_t launch_tmem_nv(const ListParams& p, int sm_count, cudaStream_t st) {
  // the work-list variant is a separate instantiation (with its own parameter type): the
  // full-plane code stays free of it
  const int64_t grid = p.units < sm_count ? p.units : sm_count;
  if (p.unit_list && p.unit_mask) {
    auto kern = fdas_convolve_tmem_kernel<Cfg, NV, true, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, 256, Cfg::SMEM, st>>>(p);
  } else if (p.unit_list) {
    auto kern = fdas_convolve_tmem_kernel<Cfg, NV, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, 256, Cfg::SMEM, st>>>(p);
  } else {
    auto kern = fdas_convolve_tmem_kernel<Cfg, NV, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, 256, Cfg::SMEM, st>>>(static_cast<const BatchParams&>(p));
  }
  return cudaGetLastError();
}

// Smallest instantiated NV >= ceil(V / N2): N1*3/4, N1*7/8 or N1.
template <class Cfg>
static cudaError_t launch_tmem_cfg(const ListParams& p, int sm_count, cudaStream_t st) {
  const int rows = (p.V + Cfg::N2 - 1) / Cfg::N2;
  if (rows <= Cfg::N1 * 3 / 4) return launch_tmem_nv<Cfg, Cfg::N1 * 3 / 4>(p, sm_count, st);
  if (rows <= Cfg::N1 * 7 / 8) return launch_tmem_nv<Cfg, Cfg::N1 * 7 / 8>(p, sm_count, st);
  return launch_tmem_nv<Cfg, Cfg::N1>(p, sm_count, st);
}

int batch_segments_per_cta(int L) {
  switch (L) {
    case 512: return TmemCfg<512, 16>::G;
    case 2048: return TmemCfg<2048, 32>::G;
    default: return 0;
  }
}

static cudaError_t launch_desc(int L, const ListParams& p, int sm_count, cudaStream_t st) {
  switch (L) {
    case 512: return launch_tmem_cfg<TmemCfg<512, 16>>(p, sm_count, st);
    case 2048: return launch_tmem_cfg<TmemCfg<2048, 32>>(p, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch(int L, const BatchParams& p, int sm_count, cudaStream_t st) {
  ListParams q;
  static_cast<BatchParams&>(q) = p;
  return launch_desc(L, q, sm_count, st);
}

// Single spectrum: the descriptor-driven kernel with an inline one-entry table where it exists.
static cudaError_t launch_single_desc(int L, const ConvParams& p, int sm_count, cudaStream_t st) {
  const int G = batch_segments_per_cta(L);
  BatchParams q;
  q.templates = p.templates;
  q.twist = p.twist;
  q.status = p.status;
  q.descs = nullptr;
  q.count = 1;
  q.single.spec = p.spectrum;
  q.single.plane = p.plane;
  q.single.n_bins = p.n_bins;
  q.single.nseg = p.nseg;
  q.single.unit_base = 0;
  q.single.ngroups = (p.nseg + G - 1) / G;
  q.single.Z = p.Z;
  q.single.z_off = 0;
  q.units = q.single.ngroups * p.Z;
  q.unit_list = nullptr;
  q.V = p.V;
  q.h = p.h;
  return launch_batch(L, q, sm_count, st);
}

// A work list is usable when its entries are strictly increasing and inside [0, limit): that
// bounds every template row, segment and plane row the kernel touches.  Otherwise kStatusBadList.
// With d_count the length is read from device memory and must lie in [0, n] (n = the list's capacity).
__global__ void check_units_kernel(const int32_t* units, int64_t n, int64_t limit, int* status,
                                   const int64_t* d_count) {
  if (d_count) {
    const int64_t c = *d_count;
    if (c < 0 || c > n) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusBadList);
      return;
    }
    n = c;
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = units[e];
    if (u < 0 || u >= limit || (e > 0 && (int64_t)units[e - 1] >= u)) atomicOr(status, kStatusBadList);
  }
}

cudaError_t launch_units(int L, const ConvParams& p, const int32_t* units, const uint16_t* masks, int64_t n_units,
                         int sm_count, cudaStream_t st, const int64_t* d_count) {
  const int G = batch_segments_per_cta(L);
  if (G == 0 || n_units < 1) return cudaErrorInvalidValue;
  const int64_t ngroups = (p.nseg + G - 1) / G;
  {
    const int64_t blocks = (n_units + 255) / 256;
    const unsigned grid = (unsigned)(blocks < 4LL * sm_count ? blocks : 4LL * sm_count);
    check_units_kernel<<<grid, 256, 0, st>>>(units, n_units, ngroups * p.Z, p.status, d_count);
  }
  ListParams q;
  q.templates = p.templates;
  q.twist = p.twist;
  q.status = p.status;
  q.descs = nullptr;
  q.count = 1;
  q.single.spec = p.spectrum;
  q.single.plane = p.plane;
  q.single.n_bins = p.n_bins;
  q.single.nseg = p.nseg;
  q.single.unit_base = 0;
  q.single.ngroups = ngroups;
  q.single.Z = p.Z;
  q.single.z_off = 0;
  q.units = n_units;
  q.unit_list = units;
  q.unit_mask = masks;
  q.unit_count = d_count;   // with a device count, n_units is the list's capacity (grid: every SM)
  q.V = p.V;
  q.h = p.h;
  return launch_desc(L, q, sm_count, st);
}

bool pairs_supported(int L) { return L == 2048; }

template <class Cfg, int NV>
static cudaError_t launch_pairs_nv(const PairParams& p, int sm_count, cudaStream_t st) {
  constexpr size_t smem = (size_t)Cfg::W * Cfg::REGION + 128;
  static_assert(smem <= 232448, "shared memory budget of the pair-list kernel");
  auto kern = fdas_convolve_pairs_kernel<Cfg, NV>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // every SM when the length is on the device; otherwise no more CTAs than W-pair shares
  const int64_t need = (p.n_pairs + Cfg::W - 1) / Cfg::W;
  const int64_t grid = p.pair_count || need > sm_count ? sm_count : need;
  kern<<<(unsigned)grid, 256, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_pairs(int L, const PairParams& p, int sm_count, cudaStream_t st) {
  if (!pairs_supported(L) || p.n_pairs < 1) return cudaErrorInvalidValue;
  {
    const int64_t blocks = (p.n_pairs + 255) / 256;
    const unsigned grid = (unsigned)(blocks < 4LL * sm_count ? blocks : 4LL * sm_count);
    check_units_kernel<<<grid, 256, 0, st>>>(p.pairs, p.n_pairs, p.nseg * p.Z, p.status, p.pair_count);
  }
  // two instantiations (compile time): rows pruned to 3/4 (m >= L/4), or none pruned
  using Cfg = TmemCfg<2048, 32>;
  const int rows = (p.V + Cfg::N2 - 1) / Cfg::N2;
  if (rows <= Cfg::N1 * 3 / 4) return launch_pairs_nv<Cfg, Cfg::N1 * 3 / 4>(p, sm_count, st);
  return launch_pairs_nv<Cfg, Cfg::N1>(p, sm_count, st);
}

cudaError_t launch_convolve(int L, const CUtensorMap* map, const ConvParams& p, int sm_count, cudaStream_t st) {
  switch (L) {
    case 256: return launch_conv_cfg<Cfg256>(map, p, sm_count, st);
    case 512: return launch_single_desc(512, p, sm_count, st);
    case 1024: return launch_conv_cfg<Cfg1024>(map, p, sm_count, st);
    case 2048: return launch_single_desc(2048, p, sm_count, st);
    case 4096:
    case 8192: return launch_convolve_big(L, p, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_segment_spectra(int L, const CUtensorMap* map, const SegParams& p, int sm_count, cudaStream_t st) {
  switch (L) {
    case 256: return launch_seg_cfg<Cfg256>(map, p, st);
    case 512: return launch_seg_cfg<Cfg512>(map, p, st);
    case 1024: return launch_seg_cfg<Cfg1024>(map, p, st);
    case 2048: return launch_seg_cfg<ConvCfg<2048, 32, 2, 2>>(map, p, st);   // two-round exchange fits
    case 4096:
    case 8192: return launch_segment_spectra_big(L, p, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdas
