// fslbm_kernels.h -- launchers shared by the translation units of the library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fslbm_dev.cuh"

namespace fsl {

// Programmatic dependent launch.  Every kernel of the step starts with
// pdl_begin(): wait until the previous kernel of the stream has completed and
// its writes are visible (a no-op when launched without the attribute), then
// allow the next kernel to be launched, so that its launch and block
// scheduling overlap this kernel instead of following it.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launch with the programmatic-stream-serialization attribute
template <typename... KArgs, typename... Args>
inline int launch_k(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                    Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// the segment scan (fslbm_step.cu): the list of the 32-cell x segments that
// hold fluid, with their kind masks, and the step's interface cells
int launch_segments(const Par& p, const uint8_t* flags, int* seglist, int* segcount, int* ilist, int* cnt, int cap,
                    int* err, cudaStream_t st);

// zero the per-step counters cnt[0..7] and cnt[9] (one small kernel, so that
// the whole step is a chain of kernels)
int launch_reset(int* cnt, cudaStream_t st);

// how the bulk kernel reaches its pulled values (fslbm_bulk_loads)
enum BulkMode { BULK_PLAIN = 0, BULK_TMA = 1, BULK_ASYNC = 2, BULK_PAIRS = 3 };

// a second stream of the handle and two events: the interface geometry (and,
// beside the pair kernel, the interface kernel) runs on it beside the bulk
// kernel (fork after the segment scan, join before the interface kernel or
// the conversions)
struct Fork {
  cudaStream_t side;
  cudaEvent_t fork, join;
};

// bulk_mode: BulkMode (FP32/FP16 only for the staged modes); tmap: tensor map
// of v.fin for BULK_TMA; fork: NULL to run every kernel on st
template <int P>
int launch_step_kernels(const Par& p, const View<P>& v, cudaStream_t st, int bulk_blocks, int iface_blocks,
                        int* seglist, int* segcount, void* timing_handle, int bulk_mode, const CUtensorMap* tmap,
                        const Fork* fork);

// staged bulk kernels (fslbm_staged.cu): TMA shape test, tensor map of a
// population buffer, launchers
bool tma_shape_ok(const Par& p, int prec);
bool tma_encode(const Par& p, int prec, const void* base, CUtensorMap* map);
template <int P>
int launch_bulk_tma(const Par& p, const View<P>& v, const CUtensorMap* map, cudaStream_t st, int bulk_blocks,
                    const int* seglist, const int* segcount);
template <int P>
int launch_bulk_async(const Par& p, const View<P>& v, cudaStream_t st, int bulk_blocks, const int* seglist,
                      const int* segcount);

// bulk kernel with two x-adjacent cells per lane (fslbm_pairs.cu): shape
// test (nx even) and launcher (FP32/FP16)
bool pairs_shape_ok(const Par& p);
template <int P>
int launch_bulk_pairs(const Par& p, const View<P>& v, cudaStream_t st, int bulk_blocks, const int* seglist,
                      const int* segcount, bool shared);

// records timing event k of the handle's current step (host side, fslbm_api.cu)
int fslbm_mark(void* handle, int k);

template <int P>
int launch_conversions(const Par& p, const View<P>& v, cudaStream_t st, int list_blocks, int coop_blocks,
                       const MassReduce& mr);
// one cooperative launch of the conversion kernel's grid barrier on `blocks`
// blocks, waiting for `extra` blocks more than exist (self-check)
int launch_barrier_check(unsigned* ctr, int* err, int blocks, unsigned extra, cudaStream_t st);
// resident blocks per SM of the fused conversion kernel (0: not usable)
template <int P>
int convert_blocks_per_sm();

int launch_reduce(const double* in, long long n, double* tmp, int tmp_blocks, const double* add, double* out,
                  cudaStream_t st);

// state set-up and read-back (fslbm_state.cu)
template <int P>
int launch_init_pre(const Par& p, const View<P>& v, const double* f, const double* phi, const double* rho_in,
                    const double* u_in, const double* noise, double* keep_f0, cudaStream_t st);
template <int P>
int launch_init_post(const Par& p, const View<P>& v, const double* f, const double* m, const double* phi,
                     cudaStream_t st);
int launch_prepare_flags(const Par& p, uint8_t* flags, int* err, cudaStream_t st);
template <int P>
int launch_fields(const Par& p, const View<P>& v, unsigned mask, void* const* out, cudaStream_t st);
template <int P>
int launch_total_mass(const Par& p, const View<P>& v, double* partials, long long nparts, double* tmp,
                      int tmp_blocks, double* out, cudaStream_t st);

}  // namespace fsl
