// fslbm_noalloc.cu -- mass balance of caller-owned device arrays that
// allocates nothing: the partial sums live in a fixed array of the library.
// For callers that cannot allocate device memory while they run (a framework
// that owns the GPU's memory through its own pool; loops where the device-wide
// synchronisation of cudaMalloc/cudaFree would stall other streams).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fslbm.h"
#include "fslbm_dev.cuh"

// Scratch for the per-block partial sums: one FP64 partial per block of
// FSLBM_NOALLOC_CELLS_PER_BLOCK cells, FSLBM_NOALLOC_MAX_BLOCKS of them
// (32 KiB).  Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) double g_noalloc_partials[FSLBM_NOALLOC_MAX_BLOCKS];

// Device address of the scratch array, per device ordinal (NULL = not looked
// up yet).  Host code must not hand g_noalloc_partials itself to a kernel: on
// the host that name is a stand-in, not a device address.
static void* g_scratch_addr[64];

namespace {

constexpr int kMaxBlocks = FSLBM_NOALLOC_MAX_BLOCKS;
constexpr long long kCellsPerBlock = FSLBM_NOALLOC_CELLS_PER_BLOCK;
constexpr int kMaxDevices = 64;

template <int P>
__global__ void __launch_bounds__(256) k_noalloc_partials(const uint8_t* __restrict__ flags,
                                                          const typename fsl::Form<P>::S* __restrict__ f,
                                                          const double* __restrict__ m, long long n,
                                                          double* __restrict__ partials) {
  using R = typename fsl::Form<P>::R;
  __shared__ double red[8];
  const long long lo = (long long)blockIdx.x * kCellsPerBlock;
  const long long hi = lo + kCellsPerBlock < n ? lo + kCellsPerBlock : n;
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const uint8_t k = flags[i] & fsl::KIND;
    if (k == fsl::LIQ) {
      R r = R(0);
#pragma unroll
      for (int q = 0; q < 19; ++q) r += fsl::ldq<P>(f, (size_t)q * (size_t)n + (size_t)i, q);
      s += fsl::rho_full<fsl::Form<P>::SH>(r);
    } else if (k == fsl::IFC) {
      s += m[i];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0)
    partials[blockIdx.x] = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
}

__global__ void __launch_bounds__(256) k_noalloc_final(const double* __restrict__ partials, int nb, double lost,
                                                       double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s += partials[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0)
    *out = (((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]))) + lost;
}

}  // namespace

extern "C" int fslbm_mass_balance_noalloc(const uint8_t* flags, const void* f_post, int precision, const double* m,
                                          long long n_cells, double lost, double* mass_out, void* stream) {
  if (!flags || !f_post || !m || !mass_out || n_cells <= 0) return FSLBM_ERR_ARG;
  if (precision < FSLBM_F64 || precision > FSLBM_F16) return FSLBM_ERR_ARG;
  const long long nb = (n_cells + kCellsPerBlock - 1) / kCellsPerBlock;
  if (nb > kMaxBlocks) return FSLBM_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSLBM_ERR_CUDA;
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr) return FSLBM_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
  }
  double* partials = (double*)g_scratch_addr[dev];
  cudaStream_t st = (cudaStream_t)stream;
  // each launch's own status (cudaLaunchKernel returns it): an earlier error
  // of unrelated work is neither reported as this call's nor cleared by it
  int nbi = (int)nb;
  long long n = n_cells;
  const void* fp = f_post;
  void* a1[] = {(void*)&flags, (void*)&fp, (void*)&m, (void*)&n, (void*)&partials};
  const void* kern = precision == FSLBM_F64   ? (const void*)k_noalloc_partials<fsl::P64>
                     : precision == FSLBM_F32 ? (const void*)k_noalloc_partials<fsl::P32>
                                              : (const void*)k_noalloc_partials<fsl::P16>;
  cudaError_t e = cudaLaunchKernel(kern, dim3(nbi), dim3(256), a1, 0, st);
  if (e == cudaSuccess) {
    void* a2[] = {(void*)&partials, (void*)&nbi, (void*)&lost, (void*)&mass_out};
    e = cudaLaunchKernel((const void*)k_noalloc_final, dim3(1), dim3(256), a2, 0, st);
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();  // the failed launch recorded its own error there
    return FSLBM_ERR_CUDA;
  }
  return FSLBM_OK;
}
