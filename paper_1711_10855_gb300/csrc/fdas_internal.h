// fdas_internal.h -- declarations shared by the two translation units of libfdas.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace fdas {

// Parameters of the fused correlation kernel (steps a2..a7).
struct ConvParams {
  const float2* templates;  // Z x L template spectra, per-template layout of the IFFT's first pass
  const float2* twist;      // L inter-pass twiddles exp(+i 2pi n2 k1 / L), same layout
  float* plane;             // Z x n_bins output, row pitch n_bins
  int* status;              // device status word (bit 0: a bounded wait gave up)
  int64_t n_bins;
  int64_t nseg;             // ceil(n_bins / V)
  int64_t units;            // (number of segment groups) x Z
  int Z, V, h;
};

// Parameters of the forward-transform-only kernel (steps a2 + a3, for tests).
struct SegParams {
  const float2* twist;
  float2* out;              // nseg x L, natural order
  int* status;
  int64_t n_bins;
  int64_t nseg;
  int V, h;
};

// Threads per transform group (N1) used for segment length L; the template bank and the
// twiddle table are stored in the layout of that decomposition (element k = k1 + N1*k2 at
// ((k2/2)*N1 + k1)*2 + k2%2).
int conv_group_threads(int L);

// Launch helpers (defined in fdas_convolve.cu).  Return a cudaError_t from the launch.
cudaError_t launch_convolve(int L, const CUtensorMap* spec_map, const ConvParams& p, int sm_count,
                            cudaStream_t stream);
cudaError_t launch_segment_spectra(int L, const CUtensorMap* spec_map, const SegParams& p,
                                   int sm_count, cudaStream_t stream);

}  // namespace fdas

namespace fdas {
// Used by the allocation-free entry point (defined in fdas_api.cu).
int validate_geometry(int64_t n_bins, int zmax, int zstep, int seg_len, int tmpl_len);
cudaError_t build_templates_into(double2* taps, float2* templates, float2* twist, int zmax, int zstep, int L,
                                 int m, cudaStream_t st);
int encode_spectrum_map(CUtensorMap* map, const void* d_spectrum, int64_t n_bins, int L);
}  // namespace fdas
