// fslbm_staged.cu -- bulk stream-collide with the pulled values staged in
// shared memory ahead of use.
//
// Both kernels do the work of k_bulk (liquid cells of the fluid-segment list,
// one warp per 32-cell x segment, Eq. lbe1 pull, wall closures, Eq. lbe2
// collision, per-warp FP64 partial sums) with the same arithmetic, so their results are identical to it; they
// differ in how the 19 pulled values of a segment reach the warp.
//
// k_bulk_async  every lane copies the 19 values it will consume, f_q(x - c_q),
//          into its own shared-memory slots with cp.async, STAGES segments
//          ahead of use (FP16: the aligned 32-bit word holding the value), and
//          waits only for its own copies (cp.async.wait_group).  The copies of
//          the next segments are in flight while the warp collides this one,
//          without registers held for them.
// k_bulk_tma  lane 0 copies the 19 rows of a segment by tensor-map bulk copies
//          (cp.async.bulk.tensor) into a per-warp ring completed on mbarriers.
//          Row q is the box of 32 + 2H cells of population q starting at
//          (x0 - H, y - c_qy, z - c_qz); H is 16 bytes of elements, so every
//          copy starts on a 16-byte boundary, and lane l finds f_q(x - c_q) at
//          box offset H + l - c_qx.  Boxes reaching past a face read the fill
//          value (zero), which no cell uses.  Every mbarrier wait is bounded in
//          time: on expiry the kernel records ERRB_TMA, waits (bounded again)
//          for the copies it still has in flight, and returns.
// In both, cells on the faces or next to a wall, and non-liquid cells, take
// the general path of k_bulk from global memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "fslbm_dev.cuh"
#include "fslbm_kernels.h"
#include "fslbm_pull.cuh"

namespace fsl {

constexpr int TMA_STAGES = 2;
constexpr int TMA_WARPS = 4;                            // warps per block (128 threads)
constexpr unsigned long long TMA_WAIT_NS = 1000000000;  // 1 s per wait

// A tensor copy writes to a 128-byte aligned shared-memory address: rows sit
// at a pitch of a multiple of 128 bytes (FP32: 160-byte rows at 256, FP16:
// 96-byte rows at 128).
template <int P>
struct TmaGeom {
  using S = typename Form<P>::S;
  static constexpr int H = 16 / (int)sizeof(S);                // halo cells (16 bytes)
  static constexpr int BOXW = 32 + 2 * H;                      // cells per row box
  static constexpr int ROWB = BOXW * (int)sizeof(S);           // bytes per row (multiple of 16)
  static constexpr int PITCH = (ROWB + 127) / 128 * 128;       // row pitch in shared memory
  static constexpr int STAGE = 19 * PITCH;                     // bytes per segment
  static constexpr int SMEM = TMA_WARPS * TMA_STAGES * STAGE;  // dynamic shared memory per block
  static constexpr int BLOCKS = P == P32 ? 5 : 8;              // resident blocks per SM (shared memory)
  static_assert(ROWB % 16 == 0 && PITCH % 128 == 0 && STAGE % 128 == 0, "TMA row alignment");
  static_assert((H * (int)sizeof(S)) % 16 == 0, "box x origin x0 - H must be a 16-byte boundary");
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// order this thread's earlier shared-memory accesses before later async-proxy (TMA) ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the completion of the phase with the given parity, at most TMA_WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < (1u << 30); ++it) {
    if (mbar_test(bar, parity)) return true;
    if ((it & 63u) == 63u && global_ns() - t0 > TMA_WAIT_NS) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_row(void* dst, const CUtensorMap* map, int x, int y, int z, int q,
                                        uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(q), "r"(smem_u32(bar))
      : "memory");
}

template <int P, int q>
__device__ __forceinline__ typename Form<P>::R ld_row(const unsigned char* row, int idx) {
  using S = typename Form<P>::S;
  const S s = reinterpret_cast<const S*>(row)[idx];
  if constexpr (P == P16) return __half2float(s);
  else return s;
}

template <int P>
__global__ void __launch_bounds__(128, TmaGeom<P>::BLOCKS) k_bulk_tma(Par p, View<P> v, const __grid_constant__ CUtensorMap tmap,
                                                   const int* __restrict__ seglist,
                                                   const int* __restrict__ segcount) {
  pdl_begin();
  using R = typename Form<P>::R;
  using G = TmaGeom<P>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[TMA_WARPS][TMA_STAGES];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wbuf = smem + warp * (TMA_STAGES * G::STAGE);
  const int nseg = *((volatile const int*)segcount);
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const size_t N = (size_t)p.N;
  // the ring must start on a 128-byte boundary; if not, copy nothing and report
  if (smem_u32(smem) & 127u) {
    if (threadIdx.x == 0) atomicOr(v.err, ERRB_TMA);
    return;
  }
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < TMA_STAGES; ++s) mbar_init(&bars[warp][s], 1);
    mbar_fence_init();
    fence_proxy_async();
  }
  __syncwarp();

  // lane 0: start the copies of segment si into stage s
  auto issue = [&](int si, int s) {
    const int4 sd = reinterpret_cast<const int4*>(seglist)[si];
    const int x0 = sd.x, y = sd.y, z = sd.z;
    uint64_t* bar = &bars[warp][s];
    mbar_expect_tx(bar, 19u * (unsigned)G::ROWB);
    unsigned char* dst = wbuf + s * G::STAGE;
#pragma unroll
    for (int q = 0; q < 19; ++q) tma_row(dst + q * G::PITCH, &tmap, x0 - G::H, y - cy(q), z - cz(q), q, bar);
  };
  unsigned pending = 0u;  // stages with copies in flight (lane 0's view)
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < TMA_STAGES; ++s)
      if (gw + s * nw < nseg) {
        issue(gw + s * nw, s);
        pending |= 1u << s;
      }
  }

  double msum = 0.0;
  unsigned parity = 0u;  // bit s: parity of the next phase of stage s
  int stage = 0;
  bool failed = false;
  for (int si = gw; si < nseg; si += nw) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[warp][stage], (parity >> stage) & 1u));
    if (!ok) {
      failed = true;
      break;
    }
    parity ^= 1u << stage;
    pending &= ~(1u << stage);
    const unsigned char* buf = wbuf + stage * G::STAGE;

    const int4 sd = reinterpret_cast<const int4*>(seglist)[si];
    const int x = sd.x + lane, y = sd.y, z = sd.z;
    const long long rowstart = (long long)sd.w - sd.x;  // index of x = 0 in this row
    const bool in = x < p.nx;
    const long long i = FSL_CK_IF(p, in, rowstart + x, p.N);
    const uint8_t fl = in ? v.flags[i] : (uint8_t)GAS;
    const uint8_t k = fl & KIND;
    R f[19];
    const bool fast = k == LIQ && !(fl & NEARB) && x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1 && z > 0 &&
                      z < p.nz - 1;
    if (fast) {
#define FSL_LDS(q) f[q] = ld_row<P, q>(buf + q * G::PITCH, G::H + lane - cx(q));
      FSL_LDS(0) FSL_LDS(1) FSL_LDS(2) FSL_LDS(3) FSL_LDS(4) FSL_LDS(5) FSL_LDS(6) FSL_LDS(7) FSL_LDS(8)
      FSL_LDS(9) FSL_LDS(10) FSL_LDS(11) FSL_LDS(12) FSL_LDS(13) FSL_LDS(14) FSL_LDS(15) FSL_LDS(16)
      FSL_LDS(17) FSL_LDS(18)
#undef FSL_LDS
    }
    __syncwarp();
    // every lane has read the stage: refill it with the segment STAGES ahead
    if (lane == 0 && si + TMA_STAGES * nw < nseg) {
      fence_proxy_async();
      issue(si + TMA_STAGES * nw, stage);
      pending |= 1u << stage;
    }
    stage = stage + 1 == TMA_STAGES ? 0 : stage + 1;
    if (k != LIQ) continue;
    if (!fast) {
      unsigned wallm, gasm;
      f[0] = ld<P, 0>(v.fin, (size_t)i);
      pull_general<P>(p, v, x, y, z, f, wallm, gasm);
      if (gasm) atomicOr(v.err, ERRB_STATE);  // liquid must not touch gas
      wallm |= gasm;
      if (wallm) {
        R own[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) own[q] = ldq<P>(v.fin, (size_t)q * N + (size_t)i, q);
        wall_links<P>(p, v, i, wallm, 0u, own, f);
      }
    }
    R rho, ux, uy, uz;
    collide<R, Form<P>::SH>(p, f, rho, ux, uy, uz);
    if (rho_bad<Form<P>::SH>(rho)) atomicOr(v.err, ERRB_UNSTABLE);
    if (speed_bad(p, ux, uy, uz)) atomicOr(v.err, ERRB_SPEED);
#define FSL_ST(q) st<P, q>(v.fout, (size_t)q * N + (size_t)i, f[q]);
    FSL_ST(0) FSL_ST(1) FSL_ST(2) FSL_ST(3) FSL_ST(4) FSL_ST(5) FSL_ST(6) FSL_ST(7) FSL_ST(8)
    FSL_ST(9) FSL_ST(10) FSL_ST(11) FSL_ST(12) FSL_ST(13) FSL_ST(14) FSL_ST(15) FSL_ST(16)
    FSL_ST(17) FSL_ST(18)
#undef FSL_ST
    if (owned(p, x, y, z)) msum += rho_full<Form<P>::SH>(rho);
  }
  if (failed && lane == 0) {
    atomicOr(v.err, ERRB_TMA);
    // let the copies still in flight land before the block's shared memory is released
    for (int s = 0; s < TMA_STAGES; ++s)
      if (pending & (1u << s)) mbar_wait(&bars[warp][s], (parity >> s) & 1u);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, o);
  if (lane == 0) v.partials[gw] = msum;
}


// ---------------------------------------------------------------------------
// k_bulk_async
// ---------------------------------------------------------------------------
constexpr int AS_STAGES = 2;
constexpr int AS_WARPS = 4;
constexpr int AS_SMEM = AS_WARPS * AS_STAGES * 20 * 32 * 4;  // 19 value slots + 1 flag slot per lane

__device__ __forceinline__ void cp_async4(unsigned dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory"); }

template <int P>
__global__ void __launch_bounds__(128, 8) k_bulk_async(Par p, View<P> v, const int* __restrict__ seglist,
                                                     const int* __restrict__ segcount) {
  pdl_begin();
  using R = typename Form<P>::R;
  using S = typename Form<P>::S;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // slot (stage, k) of this lane: k = 0..18 values, 19 the word holding its flag
  const unsigned base = smem_u32(smem) + (unsigned)(warp * AS_STAGES * 20 * 128 + lane * 4);
  const uint32_t* slots = reinterpret_cast<const uint32_t*>(smem) + warp * AS_STAGES * 20 * 32 + lane;
  const int nseg = *((volatile const int*)segcount);
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const size_t N = (size_t)p.N;
  const long long sy = p.nx, sz = (long long)p.nx * p.ny;

  // all lanes: start the copies of segment si (if any) into stage stg, one commit group
  auto issue = [&](int si, int stg) {
    if (si < nseg) {
      const int4 sd = reinterpret_cast<const int4*>(seglist)[si];
      const int x = sd.x + lane, y = sd.y, z = sd.z;
      const long long rowstart = (long long)sd.w - sd.x;  // index of x = 0 in this row
      const bool in = x < p.nx;
      const long long i = FSL_CK_IF(p, in, rowstart + x, p.N);
      const bool xm = x >= 1, xp = x < p.nx - 1, ym = y >= 1, yp = y < p.ny - 1, zm = z >= 1, zp = z < p.nz - 1;
      const unsigned dst = base + (unsigned)(stg * 20 * 128);
      // the flag word (the flag array is padded to a multiple of 4 bytes)
      cp_async4(dst + 19 * 128, v.flags + ((in ? i : rowstart) & ~3LL), true);
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const int ccx = cx(q), ccy = cy(q), ccz = cz(q);
        bool ok = in;
        if (ccx == 1) ok = ok && xm;
        if (ccx == -1) ok = ok && xp;
        if (ccy == 1) ok = ok && ym;
        if (ccy == -1) ok = ok && yp;
        if (ccz == 1) ok = ok && zm;
        if (ccz == -1) ok = ok && zp;
        const long long e = (long long)q * (long long)N + (ok ? FSL_CK(p, i - (ccx + sy * ccy + sz * ccz), p.N) : 0LL);
        if constexpr (P == P16) {
          cp_async4(dst + q * 128, reinterpret_cast<const uint32_t*>(v.fin) + (e >> 1), ok);
        } else {
          cp_async4(dst + q * 128, v.fin + e, ok);
        }
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s0 = 0; s0 < AS_STAGES; ++s0) issue(gw + s0 * nw, s0);

  double msum = 0.0;
  int stg = 0;  // (not "st": that name is the store helper)
  for (int si = gw; si < nseg; si += nw) {
    cp_async_wait<AS_STAGES - 1>();  // this lane's copies of segment si have landed
    const uint32_t* sl = slots + stg * 20 * 32;
    const int4 sd = reinterpret_cast<const int4*>(seglist)[si];
    const int x = sd.x + lane, y = sd.y, z = sd.z;
    const long long rowstart = (long long)sd.w - sd.x;  // index of x = 0 in this row
    const bool in = x < p.nx;
    const long long i = FSL_CK_IF(p, in, rowstart + x, p.N);
    const uint8_t fl = in ? (uint8_t)(sl[19 * 32] >> (8 * (int)(i & 3))) : (uint8_t)GAS;
    const uint8_t k = fl & KIND;
    R f[19];
    const bool fast = k == LIQ && !(fl & NEARB) && x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1 && z > 0 &&
                      z < p.nz - 1;
    if (fast) {
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const uint32_t w = sl[q * 32];
        if constexpr (P == P16) {
          const long long e = (long long)q * (long long)N + i - (cx(q) + sy * cy(q) + sz * cz(q));
          const unsigned short hb = (unsigned short)(w >> (16 * (int)(e & 1)));
          f[q] = __half2float(__ushort_as_half(hb));
        } else {
          f[q] = __uint_as_float(w);
        }
      }
    }
    if (k == LIQ) {
      if (!fast) {
        unsigned wallm, gasm;
        f[0] = ld<P, 0>(v.fin, (size_t)i);
        pull_general<P>(p, v, x, y, z, f, wallm, gasm);
        if (gasm) atomicOr(v.err, ERRB_STATE);  // liquid must not touch gas
        wallm |= gasm;
        if (wallm) {
          R own[19];
#pragma unroll
          for (int q = 0; q < 19; ++q) own[q] = ldq<P>(v.fin, (size_t)q * N + (size_t)i, q);
          wall_links<P>(p, v, i, wallm, 0u, own, f);
        }
      }
      R rho, ux, uy, uz;
      collide<R, Form<P>::SH>(p, f, rho, ux, uy, uz);
      if (rho_bad<Form<P>::SH>(rho)) atomicOr(v.err, ERRB_UNSTABLE);
      if (speed_bad(p, ux, uy, uz)) atomicOr(v.err, ERRB_SPEED);
#define FSL_ST(q) st<P, q>(v.fout, (size_t)q * N + (size_t)i, f[q]);
      FSL_ST(0) FSL_ST(1) FSL_ST(2) FSL_ST(3) FSL_ST(4) FSL_ST(5) FSL_ST(6) FSL_ST(7) FSL_ST(8)
      FSL_ST(9) FSL_ST(10) FSL_ST(11) FSL_ST(12) FSL_ST(13) FSL_ST(14) FSL_ST(15) FSL_ST(16)
      FSL_ST(17) FSL_ST(18)
#undef FSL_ST
      if (owned(p, x, y, z)) msum += rho_full<Form<P>::SH>(rho);
    }
    // the slots of this stage have been read (their values are consumed above)
    issue(si + AS_STAGES * nw, stg);
    stg = stg + 1 == AS_STAGES ? 0 : stg + 1;
  }
  cp_async_wait<0>();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, o);
  if (lane == 0) v.partials[gw] = msum;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess && ptr)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

template <int P>
static bool shape_ok(const Par& p) {
  using G = TmaGeom<P>;
  return (p.nx % G::H) == 0 && p.nx >= G::BOXW;
}

bool tma_shape_ok(const Par& p, int prec) {
  if (prec == P32) return shape_ok<P32>(p);
  if (prec == P16) return shape_ok<P16>(p);
  return false;  // FP64 is bound by its arithmetic, not by its loads
}

bool tma_encode(const Par& p, int prec, const void* base, CUtensorMap* map) {
  if (!tma_shape_ok(p, prec) || ((uintptr_t)base & 15u) != 0u) return false;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const int elem = prec == P32 ? 4 : 2;
  const int H = 16 / elem;
  cuuint64_t dims[4] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz, 19};
  cuuint64_t strides[3] = {(cuuint64_t)p.nx * elem, (cuuint64_t)p.nx * p.ny * elem, (cuuint64_t)p.N * elem};
  cuuint32_t box[4] = {(cuuint32_t)(32 + 2 * H), 1, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, prec == P32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int P>
int launch_bulk_tma(const Par& p, const View<P>& v, const CUtensorMap* map, cudaStream_t st, int bulk_blocks,
                    const int* seglist, const int* segcount) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_bulk_tma<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmaGeom<P>::SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_bulk_tma<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
      return 1;
    attr = true;
  }
  return launch_k(k_bulk_tma<P>, bulk_blocks, 128, TmaGeom<P>::SMEM, st, p, v, *map, seglist, segcount);
}

template <int P>
int launch_bulk_async(const Par& p, const View<P>& v, cudaStream_t st, int bulk_blocks, const int* seglist,
                      const int* segcount) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_bulk_async<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, AS_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_bulk_async<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
      return 1;
    attr = true;
  }
  return launch_k(k_bulk_async<P>, bulk_blocks, 128, AS_SMEM, st, p, v, seglist, segcount);
}

template int launch_bulk_async<P32>(const Par&, const View<P32>&, cudaStream_t, int, const int*, const int*);
template int launch_bulk_async<P16>(const Par&, const View<P16>&, cudaStream_t, int, const int*, const int*);

template int launch_bulk_tma<P32>(const Par&, const View<P32>&, const CUtensorMap*, cudaStream_t, int, const int*,
                                  const int*);
template int launch_bulk_tma<P16>(const Par&, const View<P16>&, const CUtensorMap*, cudaStream_t, int, const int*,
                                  const int*);

}  // namespace fsl
