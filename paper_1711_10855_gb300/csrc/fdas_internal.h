// fdas_internal.h -- declarations shared by the translation units of libfdas.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace fdas {

// Bits of a device status word.
constexpr int kStatusTimeout = 1;   // a bounded device wait gave up
constexpr int kStatusBadList = 2;   // a work list failed its check and was not run

// Parameters of the fused correlation kernel (steps a2..a7).
struct ConvParams {
  const float2* spectrum;   // n_bins complex64 (read by bulk copies in the descriptor-driven kernel)
  const float2* templates;  // Z x L template spectra, per-template layout of the IFFT's first pass
  const float2* twist;      // L inter-pass twiddles exp(+i 2pi n2 k1 / L), same layout
  float* plane;             // Z x n_bins output, row pitch n_bins
  int* status;              // device status word (kStatusTimeout | kStatusBadList)
  int64_t n_bins;
  int64_t nseg;             // ceil(n_bins / V)
  int64_t units;            // (number of segment groups) x Z
  int Z, V, h;
};

// One spectrum of a batch, as the persistent kernel reads it (device table or inline).
struct SpecDesc {
  const float2* spec;       // n_bins complex64, 16-byte aligned
  float* plane;             // Z x n_bins float32, row pitch n_bins
  int64_t n_bins;
  int64_t nseg;             // ceil(n_bins / V)
  int64_t unit_base;        // first flattened (segment group, template) unit of this spectrum
  int64_t ngroups;          // ceil(nseg / G), G = segments resident per CTA
  int Z;                    // templates of this spectrum
  int z_off;                // template-bank row of its first template
};

// Parameters of the descriptor-driven fused kernel (TMEM variant): one or many spectra.
struct BatchParams {
  const float2* templates;  // Z_bank x L template spectra (pair-major layout)
  const float2* twist;      // L inter-pass twiddles (pair-major layout)
  int* status;              // device status word (kStatusTimeout | kStatusBadList)
  const SpecDesc* descs;    // device table of `count` spectra, or nullptr: use `single`
  SpecDesc single;
  int count;
  int64_t units;            // total units over all spectra (or entries of unit_list)
  const int32_t* unit_list; // single spectrum only: ascending units g*Z + z to compute, or nullptr: all
  int V, h;
  // with unit_list: per entry, bit j = segment j of the unit's group is computed (nullptr: all)
  const uint16_t* unit_mask = nullptr;
};

// The work-list instantiation's parameters: a BatchParams plus the list length in device memory
// (read by the kernel), or nullptr: `units` entries.  A separate type keeps the full-plane kernel's
// parameters, and so its code, free of the work-list fields.
struct ListParams : BatchParams {
  const int64_t* unit_count = nullptr;
};

// Parameters of the pair-list kernel: one spectrum restricted to a list of (segment s, template
// z) pairs, entries s*Z + z in ascending order, cut into equal contiguous ranges, one per warp.
struct PairParams {
  const float2* spec;       // n_bins complex64, 16-byte aligned
  float* plane;             // Z x n_bins float32, row pitch n_bins
  const float2* templates;  // Z x L template spectra (pair-major layout)
  const float2* twist;      // L inter-pass twiddles (pair-major layout)
  int* status;              // device status word (kStatusTimeout | kStatusBadList)
  const int32_t* pairs;     // ascending entries s*Z + z
  const int64_t* pair_count;  // list length in device memory (checked), or nullptr: n_pairs
  int64_t n_pairs;          // entries, or the list's capacity with pair_count
  int64_t n_bins;
  int64_t nseg;             // ceil(n_bins / V)
  int Z, V, h;
};

// Parameters of the forward-transform-only kernel (steps a2 + a3, for tests).
struct SegParams {
  const float2* twist;
  const float2* spectrum_in; // n_bins complex64 (read directly by the L >= 4096 kernel)
  float2* out;              // nseg x L, natural order
  int* status;
  int64_t n_bins;
  int64_t nseg;
  int V, h;
};

// Threads per transform group (N1) used for segment length L; the template bank and the
// twiddle table are stored in the layout of that decomposition (element k = k1 + N1*k2 at
// ((k2/2)*N1 + k1)*2 + k2%2).  0 for L >= 4096: natural order, and the twiddle table holds
// exp(-2 pi i t / L), t < L (shared-memory Stockham kernel, fdas_convolve_big.cu).
int conv_group_threads(int L);

// Segments resident per CTA of the descriptor-driven kernel for segment length L, or 0 if L has
// no descriptor-driven kernel (then only the single-spectrum plan path serves it).
int batch_segments_per_cta(int L);
// Descriptor-driven launch (L with batch_segments_per_cta(L) > 0).
cudaError_t launch_batch(int L, const BatchParams& p, int sm_count, cudaStream_t stream);
// Single spectrum restricted to a work list of units g*Z + z (ascending).
cudaError_t launch_units(int L, const ConvParams& p, const int32_t* units, const uint16_t* masks, int64_t n_units, int sm_count,
                         cudaStream_t stream, const int64_t* d_count = nullptr);

// Whether segment length L has the pair-list kernel (one transform per warp: L = 2048).
bool pairs_supported(int L);
// Single spectrum restricted to a list of pairs s*Z + z (checked on the device first).
cudaError_t launch_pairs(int L, const PairParams& p, int sm_count, cudaStream_t stream);

// Launch helpers (defined in fdas_convolve.cu).  Return a cudaError_t from the launch.
cudaError_t launch_convolve(int L, const CUtensorMap* spec_map, const ConvParams& p, int sm_count,
                            cudaStream_t stream);
cudaError_t launch_segment_spectra(int L, const CUtensorMap* spec_map, const SegParams& p,
                                   int sm_count, cudaStream_t stream);
// Tensor-core variant for L = 2048 (fdas_tc.cu): inverse transforms as DFT-matrix contractions.
struct TcParams {
  const float2* seg;        // nseg x 2048 forward segment spectra, natural order (inverse pass)
  float2* seg_out;          // the same, written by the forward pass
  const float2* spectrum;   // n_bins complex64 (forward pass)
  const float2* bank;       // Z x 2048 template spectra, natural order
  const float2* twist;      // the plan's twist table (pair-major layout, N1 = 32)
  const unsigned char* mats;  // DFT matrices of the precision and direction, operand layout (hi, lo)
  const unsigned* tmax;     // bits of max |Re|, |Im| over the bank
  float* plane;
  int* status;
  int64_t n_bins;
  int64_t nseg;
  int64_t units;            // inverse: nseg x ceil(Z / 4); forward: ceil(nseg / 4)
  int Z, V, h;
};
// Bytes of one set of DFT matrices; the workspace holds four sets: inverse BF16, inverse FP16,
// forward BF16, forward FP16.
int tc_matrices_bytes();
cudaError_t launch_tc_prepare(const float2* bank, int Z, float2* nat, unsigned* tmax, unsigned char* mats,
                              cudaStream_t stream);
// forward = true: the segment transforms (spectrum -> seg_out); false: the correlation (seg -> plane).
cudaError_t launch_tc(const TcParams& p, int precision, bool forward, int sm_count, cudaStream_t stream);

// Segment lengths 4096 and 8192 (fdas_convolve_big.cu); no tensor map.
cudaError_t launch_convolve_big(int L, const ConvParams& p, int sm_count, cudaStream_t stream);
cudaError_t launch_segment_spectra_big(int L, const SegParams& p, int sm_count, cudaStream_t stream);

}  // namespace fdas

namespace fdas {
// Used by the allocation-free entry point (defined in fdas_api.cu).
int validate_geometry(int64_t n_bins, int zmax, int zstep, int seg_len, int tmpl_len);
cudaError_t build_templates_into(double2* taps, float2* templates, float2* twist, int zmax, int zstep, int L,
                                 int m, cudaStream_t st);
int encode_spectrum_map(CUtensorMap* map, const void* d_spectrum, int64_t n_bins, int L);
// One thread waits, for at most limit_ns, on a barrier nothing completes and sets kStatusTimeout.
cudaError_t launch_wait_selftest(int* status, int64_t limit_ns, cudaStream_t st);
}  // namespace fdas
