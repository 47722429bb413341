// fslbm_step.cu -- the stream-collide kernels of one FSLBM time step.
//
// k_bulk   one thread per cell over the whole lattice.  Liquid cells pull their
//          19 populations (Eq. lbe1), apply half-way bounce-back / CLI at walls,
//          collide (Eq. lbe2) and store; interface cells are compacted into a
//          list by warp ballot; gas cells read one flag byte and stop.  The
//          liquid density is reduced per block for the mass balance.
// k_iface  one thread per interface cell (grid-stride over the list): pulls,
//          rebuilds the populations arriving from gas cells by the FSK rule
//          (Eq. koerner) or the FSL rule (Eq. closure, Table 1, D = 0) with the
//          link fraction from the height-function plane (Sec. 2.2, Sec. 5),
//          exchanges mass with its neighbours (Sec. 2.3), collides, stores, and
//          marks fill / empty conversions into compact lists.
// Both read f~(t) from fin and write f~(t+1) to fout; they touch disjoint cells.
#include "fslbm_dev.cuh"
#include "fslbm_kernels.h"

namespace fsl {

// ---------------------------------------------------------------------------
// warp-aggregated append of `pred` lanes' values to list[*count ...]
// (all 32 lanes of the warp must call it)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_append(bool pred, int value, int* list, int* count, int cap, int* err) {
  unsigned bal = __ballot_sync(0xffffffffu, pred);
  if (!bal) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(bal) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) {
    int k = base + __popc(bal & ((1u << lane) - 1u));
    if (k < cap) list[k] = value;
    else atomicOr(err, ERRB_OVERFLOW);
  }
}

// deterministic block sum of a double (blockDim.x == 128)
__device__ __forceinline__ double block_sum128(double v) {
  __shared__ double red[4];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) s = (red[0] + red[1]) + (red[2] + red[3]);
  __syncthreads();
  return s;
}

template <class R>
__device__ __forceinline__ R phi_at(const Par& p, const R* __restrict__ phin, long long j, uint8_t kj) {
  if (kj == LIQ) return R(1);
  if (kj == IFC) return phin[j];
  if (kj == GAS && p.freeze) return phin[j];
  return R(0);
}

// ---------------------------------------------------------------------------
// General pull for a cell next to a wall, a face or gas.  Fills f[q] from
// fluid sources and returns masks of wall and gas sources.
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ void pull_general(const Par& p, const View<P>& v, int x, int y, int z,
                                             typename Form<P>::R (&f)[19], unsigned& wallm, unsigned& gasm) {
  const size_t N = (size_t)p.N;
  wallm = 0u;
  gasm = 0u;
#pragma unroll
  for (int q = 1; q < 19; ++q) {
    long long s = nbr(p, x, y, z, -cx(q), -cy(q), -cz(q));
    uint8_t ks = kind_at(v.flags, s);
    if (is_fluid(ks)) f[q] = ldq<P>(v.fin, (size_t)q * N + (size_t)s, q);
    else if (ks == WALL) { wallm |= 1u << q; f[q] = 0; }
    else { gasm |= 1u << q; f[q] = 0; }
  }
}

// Wall closure for the links in wallm (needs the cell's own f~ and the
// pulled values): half-way bounce-back f_q = f~_p(x), p = qbar, or CLI with
// kappa = (1 - 2 dw)/(1 + 2 dw): f_q = f~_p(x) + kappa (f~_p(x - c_p) - f~_q(x)),
// where f~_p(x - c_p) is the value pulled along p (used only if that source is
// fluid).
template <int P>
__device__ __forceinline__ void wall_links(const Par& p, const View<P>& v, long long i, unsigned wallm,
                                           unsigned gasm, const typename Form<P>::R (&own)[19],
                                           typename Form<P>::R (&f)[19]) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
#pragma unroll
  for (int q = 1; q < 19; ++q) {
    if (!(wallm & (1u << q))) continue;
    const int pq = inv(q);
    R val = own[pq];
    if (p.has_wd) {
      R dw = (R)v.wd[(size_t)pq * N + (size_t)i];
      bool up_fluid = !((wallm | gasm) & (1u << pq));
      if (dw >= R(0) && up_fluid) {
        R kap = (R(1) - R(2) * dw) / (R(1) + R(2) * dw);
        val = val + kap * (f[pq] - own[q]);
      }
    }
    f[q] = val;
  }
}

// ---------------------------------------------------------------------------
// k_bulk
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128) k_bulk(Par p, View<P> v) {
  using R = typename Form<P>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const bool in = x < p.nx;
  const long long i = (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
  const uint8_t fl = in ? v.flags[i] : (uint8_t)GAS;
  const uint8_t k = fl & KIND;
  warp_append(k == IFC, (int)i, v.ilist, &v.cnt[0], v.cap, v.err);

  double msum = 0.0;
  if (k == LIQ) {
    const size_t N = (size_t)p.N;
    R f[19];
    const bool fast = !(fl & NEARB) && x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1 && z > 0 &&
                      z < p.nz - 1;
    if (fast) {
      const long long sy = p.nx, sz = (long long)p.nx * p.ny;
#define FSL_LD(q) f[q] = ld<P, q>(v.fin, (size_t)q * N + (size_t)(i - (cx(q) + sy * cy(q) + sz * cz(q))));
      FSL_LD(0) FSL_LD(1) FSL_LD(2) FSL_LD(3) FSL_LD(4) FSL_LD(5) FSL_LD(6) FSL_LD(7) FSL_LD(8)
      FSL_LD(9) FSL_LD(10) FSL_LD(11) FSL_LD(12) FSL_LD(13) FSL_LD(14) FSL_LD(15) FSL_LD(16)
      FSL_LD(17) FSL_LD(18)
#undef FSL_LD
    } else {
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
    collide<R>(p, f, rho, ux, uy, uz);
    if (!(rho > R(0)) || !(rho < R(1e30))) atomicOr(v.err, ERRB_UNSTABLE);
#define FSL_ST(q) st<P, q>(v.fout, (size_t)q * N + (size_t)i, f[q]);
    FSL_ST(0) FSL_ST(1) FSL_ST(2) FSL_ST(3) FSL_ST(4) FSL_ST(5) FSL_ST(6) FSL_ST(7) FSL_ST(8)
    FSL_ST(9) FSL_ST(10) FSL_ST(11) FSL_ST(12) FSL_ST(13) FSL_ST(14) FSL_ST(15) FSL_ST(16)
    FSL_ST(17) FSL_ST(18)
#undef FSL_ST
    msum = (double)rho;
  }
  double s = block_sum128(msum);
  if (threadIdx.x == 0) {
    long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    v.partials[b] = s;
  }
}

// ---------------------------------------------------------------------------
// Geometry of an interface cell from phi(t) (Sec. 2.2, Sec. 5): Parker-Youngs
// gradient, then height functions over 3x3 columns of 7 cells along the
// dominant axis; if every column is closed (liquid at its liquid end, gas at
// its gas end, no wall) the normal, the plane offset
// d = |n_a| (H(0,0) - 3.5) and the curvature come from the heights, else the
// normalised Parker-Youngs normal and the plane cutting the cell's own fill.
// ---------------------------------------------------------------------------
template <class R>
__device__ void geometry(const Par& p, const uint8_t* __restrict__ flags, const R* __restrict__ phin,
                         int x, int y, int z, R phic, R (&n)[3], R& d, R& kap, bool& ok) {
  R g0 = R(0), g1 = R(0), g2 = R(0);
#pragma unroll 1
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll 1
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        long long j = nbr(p, x, y, z, dx, dy, dz);
        uint8_t kj = kind_at(flags, j);
        R pj = (kj == WALL) ? phic : phi_at<R>(p, phin, j, kj);
        int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
        if (dx) g0 += R(dx * (2 - ay) * (2 - az)) * pj;
        if (dy) g1 += R(dy * (2 - az) * (2 - ax)) * pj;
        if (dz) g2 += R(dz * (2 - ax) * (2 - ay)) * pj;
      }
  n[0] = -g0; n[1] = -g1; n[2] = -g2;
  kap = R(0);
  R nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  if (!(nn > R(1e-24))) {
    ok = false;
    d = R(0);
    n[0] = R(0); n[1] = R(0); n[2] = R(1);
    return;
  }
  ok = true;
  int a = 0;
  R na = fabs(n[0]);
  if (fabs(n[1]) > na) { a = 1; na = fabs(n[1]); }
  if (fabs(n[2]) > na) { a = 2; }
  const int s = (a == 0 ? n[0] : (a == 1 ? n[1] : n[2])) > R(0) ? 1 : -1;
  const int b = (a == 0) ? 1 : 0;  // the third axis is the remaining one
  R H[9];
  bool closed = true;
#pragma unroll 1
  for (int ib = -1; ib <= 1 && closed; ++ib)
#pragma unroll 1
    for (int ic = -1; ic <= 1 && closed; ++ic) {
      R sum = R(0);
#pragma unroll 1
      for (int k = -3; k <= 3; ++k) {
        int o0 = (a == 0) ? k : ((b == 0) ? ib : ic);
        int o1 = (a == 1) ? k : ((b == 1) ? ib : ic);
        int o2 = (a == 2) ? k : ((b == 2) ? ib : ic);
        long long j = nbr(p, x, y, z, o0, o1, o2);
        uint8_t kj = kind_at(flags, j);
        if (kj == WALL) { closed = false; break; }
        if (k == -3 * s && kj != LIQ) { closed = false; break; }
        if (k == 3 * s && kj != GAS) { closed = false; break; }
        sum += phi_at<R>(p, phin, j, kj);
      }
      H[(ib + 1) * 3 + (ic + 1)] = sum;
    }
  if (closed) {
    R Hb = R(0.5) * (H[7] - H[1]);
    R Hc = R(0.5) * (H[5] - H[3]);
    R v0 = (a == 0) ? R(s) : ((b == 0) ? -Hb : -Hc);
    R v1 = (a == 1) ? R(s) : ((b == 1) ? -Hb : -Hc);
    R v2 = (a == 2) ? R(s) : ((b == 2) ? -Hb : -Hc);
    R len = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    n[0] = v0 / len; n[1] = v1 / len; n[2] = v2 / len;
    R nabs = fabs(a == 0 ? n[0] : (a == 1 ? n[1] : n[2]));
    d = nabs * (H[4] - R(3.5));
    if (p.sigma != 0.0) {
      R Hbb = H[7] - R(2) * H[4] + H[1];
      R Hcc = H[5] - R(2) * H[4] + H[3];
      R Hbc = R(0.25) * (H[8] - H[6] - H[2] + H[0]);
      R q2 = R(1) + Hb * Hb + Hc * Hc;
      R num = Hbb * (R(1) + Hc * Hc) + Hcc * (R(1) + Hb * Hb) - R(2) * Hb * Hc * Hbc;
      kap = -num / (q2 * sqrt(q2));
    }
  } else {
    R len = sqrt(nn);
    n[0] /= len; n[1] /= len; n[2] /= len;
    d = plic_offset<R>(n[0], n[1], n[2], phic);
  }
}

// ---------------------------------------------------------------------------
// k_iface
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128) k_iface(Par p, View<P> v, int bulk_blocks) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
  const int count = min(*((volatile int*)&v.cnt[0]), v.cap);
  const int stride = gridDim.x * blockDim.x;
  const int rounds = (count + stride - 1) / stride;
  double msum = 0.0;
  for (int r = 0; r < rounds; ++r) {
    const int li = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = li < count;
    bool fill = false, empty = false;
    int icell = 0;
    if (act) {
      const long long i = v.ilist[li];
      icell = (int)i;
      int x, y, z;
      coords(p, i, x, y, z);
      R own[19], f[19];
#pragma unroll
      for (int q = 0; q < 19; ++q) own[q] = ldq<P>(v.fin, (size_t)q * N + (size_t)i, q);
      R rt, utx, uty, utz;
      moments_post<R>(p, own, rt, utx, uty, utz);
      f[0] = own[0];
      unsigned wallm, gasm;
      pull_general<P>(p, v, x, y, z, f, wallm, gasm);
      const R phic = v.phin[i];
      // mass exchange (Sec. 2.3) with the pulled values, before any rebuild
      double dm = 0.0;
      if (!p.freeze) {
#pragma unroll
        for (int q = 1; q < 19; ++q) {
          if ((wallm | gasm) & (1u << q)) continue;
          long long s = nbr(p, x, y, z, -cx(q), -cy(q), -cz(q));
          uint8_t ks = v.flags[s] & KIND;
          R sw = (ks == LIQ) ? R(1) : R(0.5) * (phic + v.phin[s]);
          dm += (double)(sw * (f[q] - own[inv(q)]));
        }
      }
      if (wallm) wall_links<P>(p, v, i, wallm, gasm, own, f);
      if (gasm) {
        R n[3], d, kap;
        bool ok;
        geometry<R>(p, v.flags, v.phin, x, y, z, phic, n, d, kap, ok);
        R rb = R(p.rho_G);
        if (p.sigma != 0.0) rb = rb + R(3.0 * p.sigma) * kap;
        const R r0b = p.compressible ? rb : R(1);
        const R r0t = p.compressible ? rt : R(1);
        const R usq = utx * utx + uty * uty + utz * utz;
        const R lp = R(p.lam_p);
#pragma unroll
        for (int q = 1; q < 19; ++q) {
          if (!(gasm & (1u << q))) continue;
          const int pq = inv(q);  // boundary link: x + c_p is gas, missing f_pbar = f_q
          R eb = eplus_q<R>(p, pq, rb, r0b, utx, uty, utz, usq);
          bool up_fluid = !((wallm | gasm) & (1u << pq));
          if (p.rule == 0 || !up_fluid) {
            f[q] = -own[pq] + R(2) * eb;  // FSK, Eq. koerner
          } else {
            R dl = R(0.5);
            if (ok) {
              R cn = R(cx(pq)) * n[0] + R(cy(pq)) * n[1] + R(cz(pq)) * n[2];
              if (cn > R(0)) {
                dl = d / cn;
                dl = dl < R(p.delta_min) ? R(p.delta_min) : (dl > R(1) ? R(1) : dl);
              }
            }
            R et = eplus_q<R>(p, pq, rt, r0t, utx, uty, utz, usq);
            R nplus = (R(0.5) * (own[pq] + own[q]) - et) * R(p.inv_1plp);
            R C = lp * (R(0.5) + dl) - R(2) * lp;
            f[q] = (R(0.5) - dl) * own[pq] + R(0.5) * own[q] + (dl - R(1)) * f[pq] + C * nplus + eb;
          }
        }
      }
      R rho, ux, uy, uz;
      collide<R>(p, f, rho, ux, uy, uz);
      if (!(rho > R(0)) || !(rho < R(1e30))) atomicOr(v.err, ERRB_UNSTABLE);
#pragma unroll
      for (int q = 0; q < 19; ++q) stq<P>(v.fout, (size_t)q * N + (size_t)i, q, f[q]);
      double mm = v.m[i];
      if (!p.freeze) {
        mm = mm + dm;
        v.m[i] = mm;
        v.phout[i] = (R)(mm / (double)rho);
        fill = mm > (1.0 + p.eps) * (double)rho;
        empty = !fill && (mm < -p.eps * (double)rho);
      }
      msum += mm;
    }
    warp_append(fill, icell, v.flist, &v.cnt[1], v.cap, v.err);
    warp_append(empty, icell, v.elist, &v.cnt[2], v.cap, v.err);
  }
  double s = block_sum128(msum);
  if (threadIdx.x == 0) v.partials[bulk_blocks + blockIdx.x] = s;
}

// ---------------------------------------------------------------------------
// Fixed-order reduction of the block partials: out[b] = sum of chunk b.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ in, long long n, long long chunk,
                                                double* __restrict__ out, const double* add, double* final_out) {
  __shared__ double red[8];
  long long lo = (long long)blockIdx.x * chunk;
  long long hi = lo + chunk < n ? lo + chunk : n;
  double s = 0.0;
  for (long long k = lo + threadIdx.x; k < hi; k += blockDim.x) s += in[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
    out[blockIdx.x] = t;
    if (final_out) *final_out = t + (add ? *add : 0.0);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int P>
int launch_step_kernels(const Par& p, const View<P>& v, cudaStream_t st, int iface_blocks, void* timing_handle) {
  dim3 blk(128, 1, 1);
  dim3 grd((unsigned)((p.nx + 127) / 128), (unsigned)p.ny, (unsigned)p.nz);
  int bulk_blocks = (int)(grd.x * grd.y * grd.z);
  k_bulk<P><<<grd, blk, 0, st>>>(p, v);
  if (timing_handle && fslbm_mark_between(timing_handle)) return 1;
  k_iface<P><<<iface_blocks, 128, 0, st>>>(p, v, bulk_blocks);
  return (int)cudaGetLastError();
}

int launch_reduce(const double* in, long long n, double* tmp, int tmp_blocks, const double* add, double* out,
                  cudaStream_t st) {
  long long chunk = (n + tmp_blocks - 1) / tmp_blocks;
  if (chunk < 1) chunk = 1;
  int nb = (int)((n + chunk - 1) / chunk);
  if (nb < 1) nb = 1;
  k_reduce<<<nb, 256, 0, st>>>(in, n, chunk, tmp, nullptr, nullptr);
  k_reduce<<<1, 256, 0, st>>>(tmp, nb, nb, tmp + tmp_blocks, add, out);
  return (int)cudaGetLastError();
}

template int launch_step_kernels<P64>(const Par&, const View<P64>&, cudaStream_t, int, void*);
template int launch_step_kernels<P32>(const Par&, const View<P32>&, cudaStream_t, int, void*);
template int launch_step_kernels<P16>(const Par&, const View<P16>&, cudaStream_t, int, void*);

}  // namespace fsl
