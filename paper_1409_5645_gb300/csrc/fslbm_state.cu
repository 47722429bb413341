// fslbm_state.cu -- state set-up, field read-back and the full mass balance.
#include "fslbm_dev.cuh"
#include "fslbm_kernels.h"

namespace fsl {

// Populations from the caller (pre-collision f, or f^eq(rho,u) + noise) ->
// collide -> stored f~(t); m = phi rho, phi = m/rho on interface cells.
template <int P>
__global__ void k_init_pre(Par p, View<P> v, const double* __restrict__ fin, const double* __restrict__ phi,
                           const double* __restrict__ rho_in, const double* __restrict__ u_in,
                           const double* __restrict__ noise, double* __restrict__ keep_f0) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t k = v.flags[i] & KIND;
    R* phA = const_cast<R*>(v.phin);
    if (!is_fluid(k)) {
      v.m[i] = 0.0;
      phA[i] = (k == GAS && p.freeze && phi) ? (R)phi[i] : R(0);
      continue;
    }
    double fd[19];
    if (fin) {
#pragma unroll
      for (int q = 0; q < 19; ++q) fd[q] = fin[(size_t)q * N + i];
    } else {
      // equilibrium at (rho, u), u^eq = u (Eq. eqEven / eqOdd)
      double r = rho_in[i], u0 = u_in[3 * i], u1 = u_in[3 * i + 1], u2 = u_in[3 * i + 2];
      double r0 = p.compressible ? r : 1.0;
      double usq = u0 * u0 + u1 * u1 + u2 * u2;
      fd[0] = eplus<double, 0>(p, r, r0, u0, u1, u2, usq);
#define FSL_EQ(q) fd[q] = eplus<double, q>(p, r, r0, u0, u1, u2, usq) + eminus<double, q>(r0, u0, u1, u2);
      FSL_EQ(1) FSL_EQ(2) FSL_EQ(3) FSL_EQ(4) FSL_EQ(5) FSL_EQ(6) FSL_EQ(7) FSL_EQ(8) FSL_EQ(9)
      FSL_EQ(10) FSL_EQ(11) FSL_EQ(12) FSL_EQ(13) FSL_EQ(14) FSL_EQ(15) FSL_EQ(16) FSL_EQ(17) FSL_EQ(18)
#undef FSL_EQ
      if (noise) {
#pragma unroll
        for (int q = 0; q < 19; ++q) fd[q] += noise[(size_t)q * N + i];
      }
    }
    double rs = 0.0;
#pragma unroll
    for (int q = 0; q < 19; ++q) rs += fd[q];
    if (keep_f0) {
#pragma unroll
      for (int q = 0; q < 19; ++q) keep_f0[(size_t)q * N + i] = fd[q];
    }
    if (k == IFC) {
      double mm = (phi ? phi[i] : 1.0) * rs;
      v.m[i] = mm;
      phA[i] = (R)(mm / rs);
    } else {
      v.m[i] = rs;
      phA[i] = R(1);
    }
    R f[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) f[q] = to_arith<P>(fd[q], q);
    R rho, ux, uy, uz;
    collide<R, Form<P>::SH>(p, f, rho, ux, uy, uz);
#pragma unroll
    for (int q = 0; q < 19; ++q) stq<P>(const_cast<typename Form<P>::S*>(v.fin), (size_t)q * N + i, q, f[q]);
  }
}

template <int P>
__global__ void k_init_post(Par p, View<P> v, const double* __restrict__ fpost, const double* __restrict__ m,
                            const double* __restrict__ phi) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t k = v.flags[i] & KIND;
    R* phA = const_cast<R*>(v.phin);
    if (!is_fluid(k)) {
      v.m[i] = 0.0;
      phA[i] = (k == GAS && p.freeze && phi) ? (R)phi[i] : R(0);
      continue;
    }
#pragma unroll
    for (int q = 0; q < 19; ++q)
      stq<P>(const_cast<typename Form<P>::S*>(v.fin), (size_t)q * N + i, q, to_arith<P>(fpost[(size_t)q * N + i], q));
    v.m[i] = (k == IFC) ? m[i] : 0.0;
    phA[i] = (k == IFC) ? (R)phi[i] : R(1);
  }
}

// NEARB bit (a link ends in a wall or past a face) and invariant checks.
__global__ void k_prepare_flags(Par p, uint8_t* flags, int* err) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t k = flags[i] & KIND;
    if (k != LIQ && k != IFC && k != GAS && k != WALL) { atomicOr(err, ERRB_STATE); continue; }
    int x, y, z;
    coords(p, i, x, y, z);
    bool nearb = false, nearw = false, gas = false;
#pragma unroll
    for (int q = 1; q < 19; ++q) {
      long long j = nbr(p, x, y, z, cx(q), cy(q), cz(q));
      uint8_t kj = kind_at(flags, j);
      nearb |= (kj == WALL);
      nearw |= (j >= 0 && kj == WALL);
      gas |= (kj == GAS);
    }
    if (k == LIQ && gas) atomicOr(err, ERRB_STATE);
    flags[i] = (uint8_t)(k | (nearb ? NEARB : 0) | (nearw ? NEARW : 0));
  }
}

template <int P>
__global__ void k_fields(Par p, View<P> v, unsigned mask, uint8_t* oflags, double* of, double* om, double* ophi,
                         double* orho, double* ou) {
  using R = typename Form<P>::R;
  const size_t N = (size_t)p.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
       i += (long long)gridDim.x * blockDim.x) {
    uint8_t k = v.flags[i] & KIND;
    bool fl = is_fluid(k);
    constexpr bool SH = Form<P>::SH;
    R f[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) f[q] = fl ? ldq<P>(v.fin, (size_t)q * N + i, q) : R(0);
    R rho = R(0), ux = R(0), uy = R(0), uz = R(0);
    if (fl) moments_post<R, SH>(p, f, rho, ux, uy, uz);
    const double rhof = fl ? rho_full<SH>(rho) : 0.0;
    if (oflags) oflags[i] = k;
    if (of) {
#pragma unroll
      for (int q = 0; q < 19; ++q) of[(size_t)q * N + i] = fl ? ldq_full<P>(v.fin, (size_t)q * N + i, q) : 0.0;
    }
    if (om) om[i] = k == IFC ? v.m[i] : (k == LIQ ? rhof : 0.0);
    if (ophi) {
      double ph = 0.0;
      if (k == LIQ) ph = 1.0;
      else if (k == IFC || (k == GAS && p.freeze)) ph = (double)v.phin[i];
      ophi[i] = ph;
    }
    if (orho) orho[i] = rhof;
    if (ou) { ou[3 * i] = (double)ux; ou[3 * i + 1] = (double)uy; ou[3 * i + 2] = (double)uz; }
  }
}

// M = sum_liquid rho + sum_interface m: per-block partials in cell order.
template <int P>
__global__ void __launch_bounds__(256) k_mass_partials(Par p, View<P> v, double* __restrict__ partials,
                                                       long long per_block) {
  using R = typename Form<P>::R;
  __shared__ double red[8];
  const size_t N = (size_t)p.N;
  long long lo = (long long)blockIdx.x * per_block;
  long long hi = lo + per_block < p.N ? lo + per_block : p.N;
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    uint8_t k = v.flags[i] & KIND;
    if (!p.owned_all) {
      int x, y, z;
      coords(p, i, x, y, z);
      if (!owned(p, x, y, z)) continue;
    }
    if (k == LIQ) {
      R r = R(0);
#pragma unroll
      for (int q = 0; q < 19; ++q) r += ldq<P>(v.fin, (size_t)q * N + i, q);
      s += rho_full<Form<P>::SH>(r);
    } else if (k == IFC) {
      s += v.m[i];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0)
    partials[blockIdx.x] = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
}

static int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}

template <int P>
int launch_init_pre(const Par& p, const View<P>& v, const double* f, const double* phi, const double* rho_in,
                    const double* u_in, const double* noise, double* keep_f0, cudaStream_t st) {
  k_init_pre<P><<<grid_for(p.N, 128), 128, 0, st>>>(p, v, f, phi, rho_in, u_in, noise, keep_f0);
  return (int)cudaGetLastError();
}
template <int P>
int launch_init_post(const Par& p, const View<P>& v, const double* f, const double* m, const double* phi,
                     cudaStream_t st) {
  k_init_post<P><<<grid_for(p.N, 128), 128, 0, st>>>(p, v, f, m, phi);
  return (int)cudaGetLastError();
}
int launch_prepare_flags(const Par& p, uint8_t* flags, int* err, cudaStream_t st) {
  k_prepare_flags<<<grid_for(p.N, 256), 256, 0, st>>>(p, flags, err);
  return (int)cudaGetLastError();
}
template <int P>
int launch_fields(const Par& p, const View<P>& v, unsigned mask, void* const* out, cudaStream_t st) {
  void* ptr[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int k = 0;
  for (int b = 0; b < 6; ++b)
    if (mask & (1u << b)) ptr[b] = out[k++];
  k_fields<P><<<grid_for(p.N, 128), 128, 0, st>>>(p, v, mask, (uint8_t*)ptr[0], (double*)ptr[1], (double*)ptr[2],
                                                   (double*)ptr[3], (double*)ptr[4], (double*)ptr[5]);
  return (int)cudaGetLastError();
}
template <int P>
int launch_total_mass(const Par& p, const View<P>& v, double* partials, long long nparts, double* tmp,
                      int tmp_blocks, double* out, cudaStream_t st) {
  long long per = (p.N + nparts - 1) / nparts;
  if (per < 1) per = 1;
  long long nb = (p.N + per - 1) / per;
  k_mass_partials<P><<<(int)nb, 256, 0, st>>>(p, v, partials, per);
  return launch_reduce(partials, nb, tmp, tmp_blocks, v.lost, out, st);
}

#define FSL_INST(P)                                                                                          \
  template int launch_init_pre<P>(const Par&, const View<P>&, const double*, const double*, const double*,  \
                                  const double*, const double*, double*, cudaStream_t);                     \
  template int launch_init_post<P>(const Par&, const View<P>&, const double*, const double*, const double*, \
                                   cudaStream_t);                                                           \
  template int launch_fields<P>(const Par&, const View<P>&, unsigned, void* const*, cudaStream_t);          \
  template int launch_total_mass<P>(const Par&, const View<P>&, double*, long long, double*, int, double*,  \
                                    cudaStream_t);
FSL_INST(P64)
FSL_INST(P32)
FSL_INST(P16)
#undef FSL_INST

}  // namespace fsl
