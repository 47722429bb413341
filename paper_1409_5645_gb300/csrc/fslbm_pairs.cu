// fslbm_pairs.cu -- bulk stream-collide with two x-adjacent cells per lane.
//
// k_bulk_pairs does the work of k_bulk (liquid cells of the fluid-segment
// list, Eq. lbe1 pull with half-way bounce-back at non-periodic faces,
// Eq. lbe2 collision, per-warp FP64 partial sums of the liquid density) with
// the same arithmetic per cell, so the populations it produces equal
// k_bulk's bit for bit.
// It differs in how the pulled values reach the lanes: each half-warp takes
// one 32-cell segment of the list, and lane l of it the cells x0 + 2l and
// x0 + 2l + 1, whose values of one population sit in one aligned word of a
// row (FP16: 32 bits, FP32: 64 bits).  The nine populations without an x
// component are pulled one word per pair, the ten shifted along x one value
// per cell, and the 19 results are stored one word per pair: 28 loads and 19
// stores per two cells instead of 38 and 38.  The collisions of the two cells
// run together in packed FP32x2 instructions (one instruction per operation
// of both cells).  A source beyond a non-periodic face is replaced by the
// cell's own slot of the opposite population (half-way bounce-back).
// A segment holding a liquid cell that needs the general pull (next to a WALL
// cell, on a periodic face, CLI link fractions or a moving wall on a face)
// takes the general path of k_bulk for its liquid cells.  Lattices with odd
// nx (rows not word-aligned) use k_bulk.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fslbm_dev.cuh"
#include "fslbm_kernels.h"
#include "fslbm_pull.cuh"

namespace fsl {

constexpr unsigned FULL = 0xffffffffu;

// resident blocks of 128 threads per SM (the register budget of a lane
// holding two cells: 80 registers in FP16, 96 in FP32); the grid is one
// resident wave
#ifndef FSL_PAIRS_BLOCKS16
#define FSL_PAIRS_BLOCKS16 6
#endif
#ifndef FSL_PAIRS_BLOCKS32
#define FSL_PAIRS_BLOCKS32 5
#endif
template <int P>
constexpr int pairs_blocks() { return P == P16 ? FSL_PAIRS_BLOCKS16 : FSL_PAIRS_BLOCKS32; }
// blocks per SM in the launch when the interface kernels run beside it on
// the side stream: fewer than resident, so that their blocks find room
// (measured on the 512x256x256 dam break: FP32 at 3 of 5 and FP16 at 4 of 6
// gave the shortest step)
#ifndef FSL_PAIRS_GRID16
#define FSL_PAIRS_GRID16 4
#endif
#ifndef FSL_PAIRS_GRID32
#define FSL_PAIRS_GRID32 3
#endif
template <int P>
constexpr int pairs_grid() { return P == P16 ? FSL_PAIRS_GRID16 : FSL_PAIRS_GRID32; }

// A word holding the values of two x-adjacent cells (lo: the even cell).
template <int P>
struct PairWord;

template <>
struct PairWord<P16> {
  using W = unsigned;
  static __device__ __forceinline__ W load(const __half* base, unsigned k) {
    return __ldg(reinterpret_cast<const unsigned*>(base + k));
  }
  // two single values into one word (lo: element ka, hi: element kb)
  static __device__ __forceinline__ W load2(const __half* base, unsigned ka, unsigned kb) {
    const unsigned a = __ldg(reinterpret_cast<const unsigned short*>(base + ka));
    const unsigned b = __ldg(reinterpret_cast<const unsigned short*>(base + kb));
    return a | (b << 16);
  }
  static __device__ __forceinline__ W zero() { return 0u; }
  static __device__ __forceinline__ float2 unpack(W w) {
    __half2 h;
    memcpy(&h, &w, 4);
    return __half22float2(h);
  }
  // rounded as the scalar store rounds each value
  static __device__ __forceinline__ W pack(float2 v) {
    const __half2 h = __floats2half2_rn(v.x, v.y);
    W w;
    memcpy(&w, &h, 4);
    return w;
  }
  static __device__ __forceinline__ void store(__half* base, unsigned k, W w) { *reinterpret_cast<unsigned*>(base + k) = w; }
  static __device__ __forceinline__ void store_lo(__half* base, unsigned k, W w) {
    *reinterpret_cast<unsigned short*>(base + k) = (unsigned short)(w & 0xffffu);
  }
  static __device__ __forceinline__ void store_hi(__half* base, unsigned k, W w) {
    *reinterpret_cast<unsigned short*>(base + k + 1) = (unsigned short)(w >> 16);
  }
};

template <>
struct PairWord<P32> {
  using W = float2;
  static __device__ __forceinline__ W load(const float* base, unsigned k) {
    return __ldg(reinterpret_cast<const float2*>(base + k));
  }
  static __device__ __forceinline__ W load2(const float* base, unsigned ka, unsigned kb) {
    return make_float2(__ldg(base + ka), __ldg(base + kb));
  }
  static __device__ __forceinline__ W zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 unpack(W w) { return w; }
  static __device__ __forceinline__ W pack(float2 v) { return v; }
  static __device__ __forceinline__ void store(float* base, unsigned k, W w) { *reinterpret_cast<float2*>(base + k) = w; }
  static __device__ __forceinline__ void store_lo(float* base, unsigned k, W w) { base[k] = w.x; }
  static __device__ __forceinline__ void store_hi(float* base, unsigned k, W w) { base[k + 1] = w.y; }
};

// ---------------------------------------------------------------------------
// The TRT collision of k_bulk (collide<float, SH> of fslbm_dev.cuh) for two
// cells at once, in the packed FP32 instructions of sm_100 and later
// (add/mul/fma.rn.f32x2): every operation of the scalar collision, in the same
// order and with the same rounding, on the pair (lo, hi), so each half equals
// the scalar result bit for bit while the pair costs one instruction per
// operation.  On return rho holds sum f (minus 1: the stored deviations) and
// usq_out |u|^2 of the pre-collision state.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <int q>
__device__ __forceinline__ float2 cdot2(float2 ux, float2 uy, float2 uz) {
  float2 s = bc2(0.f);
  if (cx(q) == 1) s = add2(s, ux);
  if (cx(q) == -1) s = sub2(s, ux);
  if (cy(q) == 1) s = add2(s, uy);
  if (cy(q) == -1) s = sub2(s, uy);
  if (cz(q) == 1) s = add2(s, uz);
  if (cz(q) == -1) s = sub2(s, uz);
  return s;
}

template <bool SH>
__device__ __forceinline__ void collide_x2(const Par& p, float2 (&f)[19], float2& rho, float2& usq_out) {
  float2 r = f[0], jx = bc2(0.f), jy = bc2(0.f), jz = bc2(0.f);
#pragma unroll
  for (int q = 1; q < 19; ++q) r = add2(r, f[q]);
#pragma unroll
  for (int q = 1; q < 19; ++q) {
    if (cx(q) == 1) jx = add2(jx, f[q]);
    if (cx(q) == -1) jx = sub2(jx, f[q]);
    if (cy(q) == 1) jy = add2(jy, f[q]);
    if (cy(q) == -1) jy = sub2(jy, f[q]);
    if (cz(q) == 1) jz = add2(jz, f[q]);
    if (cz(q) == -1) jz = sub2(jz, f[q]);
  }
  const float2 r0 = p.compressible ? (SH ? add2(bc2(1.f), r) : r) : bc2(1.f);
  const float2 ir0 = p.compressible ? make_float2(1.f / r0.x, 1.f / r0.y) : bc2(1.f);
  const float2 Ux = mul2(jx, ir0), Uy = mul2(jy, ir0), Uz = mul2(jz, ir0);
  const float gx = (float)p.g[0], gy = (float)p.g[1], gz = (float)p.g[2];
  const float2 ux = fma2(bc2(0.5f), bc2(gx), Ux), uy = fma2(bc2(0.5f), bc2(gy), Uy),
               uz = fma2(bc2(0.5f), bc2(gz), Uz);
  const float ilm = (float)p.inv_lam_m;
  const float2 vx = fma2(bc2(-gx), bc2(ilm), Ux), vy = fma2(bc2(-gy), bc2(ilm), Uy),
               vz = fma2(bc2(-gz), bc2(ilm), Uz);
  const float2 usq = fma2(uz, uz, fma2(uy, uy, mul2(ux, ux)));
  const float2 lp = bc2((float)p.lam_p), lm = bc2((float)p.lam_m);
  const float2 nl = bc2(p.linear_eq ? 0.f : 1.f);
  const float2 k0 = mul2(mul2(bc2(1.5f * wq<float>(0)), r0), nl);
  const float2 k1 = mul2(mul2(bc2(1.5f * wq<float>(1)), r0), nl);
  const float2 k7 = mul2(mul2(bc2(1.5f * wq<float>(7)), r0), nl);
  // the momentum-exact weights of e^- (as in collide)
  constexpr float m7f = 1.f / 12.f;
  constexpr float m1f = (1.f - 8.f * m7f) * 0.5f;
  const float2 m1 = mul2(bc2(m1f), r0), m7 = mul2(bc2(m7f), r0);
  float2 out[19];
  {
    const float2 ep = fma2(k0, neg2(usq), mul2(bc2(wq<float>(0)), r));
    out[0] = fma2(lp, sub2(f[0], ep), f[0]);
  }
#define FSL_PAIR2(q)                                                                     \
  {                                                                                      \
    constexpr int qb = inv(q);                                                           \
    const float2 kq = q <= 6 ? k1 : k7, mq = q <= 6 ? m1 : m7;                           \
    const float2 cu = cdot2<q>(ux, uy, uz), cv = cdot2<q>(vx, vy, vz);                   \
    const float2 ep = fma2(kq, fma2(mul2(bc2(3.f), cu), cu, neg2(usq)), mul2(bc2(wq<float>(q)), r)); \
    const float2 em = mul2(mq, cv);                                                      \
    const float2 np = fma2(bc2(0.5f), add2(f[q], f[qb]), neg2(ep));                      \
    const float2 nm = fma2(bc2(0.5f), sub2(f[q], f[qb]), neg2(em));                      \
    out[q] = fma2(lm, nm, fma2(lp, np, f[q]));                                           \
    out[qb] = fma2(neg2(lm), nm, fma2(lp, np, f[qb]));                                   \
  }
  FSL_PAIR2(1) FSL_PAIR2(3) FSL_PAIR2(5) FSL_PAIR2(7) FSL_PAIR2(9)
  FSL_PAIR2(11) FSL_PAIR2(13) FSL_PAIR2(15) FSL_PAIR2(17)
#undef FSL_PAIR2
#pragma unroll
  for (int q = 0; q < 19; ++q) f[q] = out[q];
  rho = r;
  usq_out = usq;
}

// k_bulk's test for a liquid cell whose sources are plain offsets or lie
// beyond a non-periodic face (bounce-back from its own slots)
__device__ __forceinline__ bool fast_cell(const Par& p, uint8_t fl, int x, int y, int z) {
  const bool ax = x == 0 || x == p.nx - 1, ay = y == 0 || y == p.ny - 1, az = z == 0 || z == p.nz - 1;
  if ((fl & KIND) != LIQ) return false;
  if (p.has_wd || p.has_uw) return !(fl & NEARB) && !ax && !ay && !az;
  return !(fl & NEARW) && !(ax && p.px) && !(ay && p.py) && !(az && p.pz);
}

// the general pull of k_bulk for one liquid cell (walls, periodic faces, CLI)
template <int P>
__device__ __forceinline__ void general_cell(const Par& p, const View<P>& v, long long i, int x, int y, int z,
                                             typename Form<P>::R (&f)[19]) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
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

// One liquid cell of a segment that needs the general pull, as k_bulk
// treats it; returns its density for the mass balance (0 if not owned).
template <int P>
__device__ __noinline__ double slow_cell(const Par& p, const View<P>& v, long long i, int x, int y, int z,
                                         uint8_t fl) {
  using R = typename Form<P>::R;
  constexpr bool SH = Form<P>::SH;
  const size_t N = (size_t)p.N;
  const long long sy = p.nx, sz = (long long)p.nx * p.ny;
  R f[19];
  if (fast_cell(p, fl, x, y, z)) {
    // plain offsets, bounce-back beyond a non-periodic face
    const bool ax0 = x == 0, ax1 = x == p.nx - 1, ay0 = y == 0, ay1 = y == p.ny - 1, az0 = z == 0,
               az1 = z == p.nz - 1;
    f[0] = ld<P, 0>(v.fin, (size_t)i);
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      const bool bbq = (cx(q) == 1 && ax0) || (cx(q) == -1 && ax1) || (cy(q) == 1 && ay0) || (cy(q) == -1 && ay1) ||
                       (cz(q) == 1 && az0) || (cz(q) == -1 && az1);
      f[q] = bbq ? ldq<P>(v.fin, (size_t)inv(q) * N + (size_t)i, inv(q))
                 : ldq<P>(v.fin, (size_t)q * N + (size_t)FSL_CK(p, i - (cx(q) + sy * cy(q) + sz * cz(q)), p.N), q);
    }
  } else {
    general_cell<P>(p, v, i, x, y, z, f);
  }
  R rho, ux, uy, uz;
  collide<R, SH>(p, f, rho, ux, uy, uz);
  if (rho_bad<SH>(rho)) atomicOr(v.err, ERRB_UNSTABLE);
  if (speed_bad(p, ux, uy, uz)) atomicOr(v.err, ERRB_SPEED);
#pragma unroll
  for (int q = 0; q < 19; ++q) stq<P>(v.fout, (size_t)q * N + (size_t)i, q, f[q]);
  return owned(p, x, y, z) ? rho_full<SH>(rho) : 0.0;
}

// The pulled values of population q for the pair (xa, xa + 1) of a row.  A
// population without an x component is one aligned word of the source row
// (or, beyond a y or z face, of the pair's own slots of the opposite
// population); one with an x component is shifted by one cell against the
// word grid and takes two single-value loads, each from the cell's own slot
// of the opposite population where its source lies beyond a face.  All loads
// are independent of one another.
template <int P, int q>
__device__ __forceinline__ typename PairWord<P>::W pull_pair(const Par& p, const typename Form<P>::S* fin, unsigned N,
                                                            unsigned ia, unsigned sy, unsigned sz, int xa, int y,
                                                            int z) {
  using PW = PairWord<P>;
  // the source row beyond a y or z face: bounce-back
  const bool bb = (cy(q) == 1 && y == 0) || (cy(q) == -1 && y == p.ny - 1) || (cz(q) == 1 && z == 0) ||
                  (cz(q) == -1 && z == p.nz - 1);
  // 32-bit element indices (19 N < 2^32): the offsets wrap modulo 2^32 to the
  // in-range result
  const unsigned own_k = (unsigned)inv(q) * N + ia;
  const unsigned src_k = (unsigned)q * N + ia - (unsigned)cx(q) - sy * (unsigned)cy(q) - sz * (unsigned)cz(q);
  if constexpr (cx(q) == 0) {
    return PW::load(fin, (unsigned)FSL_CK_WORD(p, bb ? own_k : src_k, (unsigned)(bb ? inv(q) : q) * N, N));
  } else {
    const bool bba = bb || (cx(q) == 1 && xa == 0);           // the even cell's source beyond the x face
    const bool bbb = bb || (cx(q) == -1 && xa + 2 == p.nx);   // the odd cell's
    return PW::load2(fin, (unsigned)FSL_CK_CELL(p, bba ? own_k : src_k, (unsigned)(bba ? inv(q) : q) * N, N),
                     (unsigned)FSL_CK_CELL(p, bbb ? own_k + 1 : src_k + 1, (unsigned)(bbb ? inv(q) : q) * N, N));
  }
}

// nparts: the mass-balance partial slots of the bulk kernels (one per warp of
// k_bulk's grid); the slots beyond this grid's warps are zeroed
template <int P>
__global__ void __launch_bounds__(128, pairs_blocks<P>()) k_bulk_pairs(Par p, View<P> v,
                                                                      const int* __restrict__ seglist,
                                                                      const int* __restrict__ segcount, int nparts) {
  pdl_begin();
  using R = typename Form<P>::R;
  using PW = PairWord<P>;
  using W = typename PW::W;
  constexpr bool SH = Form<P>::SH;
  const int nseg = *((volatile const int*)segcount);
  const int lane = threadIdx.x & 31, hl = lane & 15;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned Nu = (unsigned)p.N, syu = (unsigned)p.nx, szu = (unsigned)(p.nx * p.ny);
  double msum = 0.0;
  // records and masks of the segment list (see k_segments); the next round's
  // are loaded one round ahead, so a round's population loads depend on no
  // load of its own
  const int nsx = (p.nx + 31) >> 5;
  const uint4* masks = reinterpret_cast<const uint4*>(seglist) + (long long)nsx * p.ny * p.nz;
  int si = 2 * gw + (lane >> 4);
  int4 sd_n = make_int4(0, 0, 0, 0);
  uint4 sm_n = make_uint4(0u, 0u, 0u, 0u);
  if (si < nseg) {
    sd_n = reinterpret_cast<const int4*>(seglist)[si];
    sm_n = masks[si];
  }
  for (int base = 2 * gw; base < nseg; base += 2 * nw, si += 2 * nw) {  // the same count of rounds on every lane
    const bool act = si < nseg;
    const int4 sd = sd_n;
    const uint4 sm = sm_n;  // liquid, interface, liquid needing the general pull
    if (si + 2 * nw < nseg) {
      sd_n = reinterpret_cast<const int4*>(seglist)[si + 2 * nw];
      sm_n = masks[si + 2 * nw];
    }
    const int x0 = sd.x, y = sd.y, z = sd.z;
    const int xa = x0 + 2 * hl;
    const unsigned bits = act ? (sm.x >> (2 * hl)) & 3u : 0u;
    const long long ia = FSL_CK_WORD_IF(p, bits != 0u, (long long)sd.w + 2 * hl, p.N);  // the even cell of the pair
    const bool la = bits & 1u, lb = (bits >> 1) & 1u;
    const bool hslow = act && sm.z != 0u;               // uniform over the half-warp
    const bool hwork = act && sm.x != 0u && !hslow;     // the pair path serves this half
    if (hwork && (la || lb)) {
      const unsigned iau = (unsigned)ia;
      W w[19];
#define FSL_PP(q) w[q] = pull_pair<P, q>(p, v.fin, Nu, iau, syu, szu, xa, y, z);
      FSL_PP(0) FSL_PP(1) FSL_PP(2) FSL_PP(3) FSL_PP(4) FSL_PP(5) FSL_PP(6) FSL_PP(7) FSL_PP(8)
      FSL_PP(9) FSL_PP(10) FSL_PP(11) FSL_PP(12) FSL_PP(13) FSL_PP(14) FSL_PP(15) FSL_PP(16)
      FSL_PP(17) FSL_PP(18)
#undef FSL_PP
      {
        float2 f[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q] = PW::unpack(w[q]);
        float2 rho, usq;
        collide_x2<SH>(p, f, rho, usq);
        if ((la && rho_bad<SH>(rho.x)) || (lb && rho_bad<SH>(rho.y))) atomicOr(v.err, ERRB_UNSTABLE);
        if (p.umax2 > 0.0) {  // (speed_bad)
          const float um2 = (float)p.umax2;
          if ((la && usq.x > um2) || (lb && usq.y > um2)) atomicOr(v.err, ERRB_SPEED);
        }
        if (la && owned(p, xa, y, z)) msum += rho_full<SH>(rho.x);
        if (lb && owned(p, xa + 1, y, z)) msum += rho_full<SH>(rho.y);
#pragma unroll
        for (int q = 0; q < 19; ++q) w[q] = PW::pack(f[q]);
        if (la && lb) {
#pragma unroll
          for (int q = 0; q < 19; ++q) PW::store(v.fout, (unsigned)q * Nu + iau, w[q]);
        } else if (la) {
#pragma unroll
          for (int q = 0; q < 19; ++q) PW::store_lo(v.fout, (unsigned)q * Nu + iau, w[q]);
        } else if (lb) {
#pragma unroll
          for (int q = 0; q < 19; ++q) PW::store_hi(v.fout, (unsigned)q * Nu + iau, w[q]);
        }
      }
    }
    if (hslow && (la || lb)) {
      // the general path of k_bulk, one cell after the other (out of line: rare)
      const unsigned fl2 = (unsigned)*reinterpret_cast<const unsigned short*>(v.flags + ia);
      if (la) msum += slow_cell<P>(p, v, ia, xa, y, z, (uint8_t)(fl2 & 0xffu));
      if (lb) msum += slow_cell<P>(p, v, ia + 1, xa + 1, y, z, (uint8_t)(fl2 >> 8));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) msum += __shfl_down_sync(FULL, msum, o);
  if (lane == 0) v.partials[gw] = msum;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (nw + t < nparts) v.partials[nw + t] = 0.0;
}

// rows word-aligned (nx even) and the population arrays indexable in 32 bits
bool pairs_shape_ok(const Par& p) { return (p.nx & 1) == 0 && 19LL * p.N < (1LL << 32); }

template <int P>
int launch_bulk_pairs(const Par& p, const View<P>& v, cudaStream_t st, int bulk_blocks, const int* seglist,
                      const int* segcount, bool shared) {
  if constexpr (P == P64) {
    return 1;
  } else {
    // bulk_blocks is 8 resident blocks per SM of k_bulk; one resident wave
    // here, or fewer blocks beside the interface kernels (shared)
    const int grid = bulk_blocks / 8 * (shared ? pairs_grid<P>() : pairs_blocks<P>());
    return launch_k(k_bulk_pairs<P>, grid, 128, 0, st, p, v, seglist, segcount, bulk_blocks * 4);
  }
}

template int launch_bulk_pairs<P64>(const Par&, const View<P64>&, cudaStream_t, int, const int*, const int*, bool);
template int launch_bulk_pairs<P32>(const Par&, const View<P32>&, cudaStream_t, int, const int*, const int*, bool);
template int launch_bulk_pairs<P16>(const Par&, const View<P16>&, cudaStream_t, int, const int*, const int*, bool);

}  // namespace fsl
