// Control and observables: the list-rebuild decision (which also flips the current half of
// the double-buffered molecule arrays), deterministic FP64 reductions, the COM density
// profile and the thermodynamic-force iteration, and the FP64 export of centres of mass.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace adress {

// Rebuild decision after a mapping: rebuild when a centre moved more than skin/2 since the
// last build (it could have changed class or found a new partner), when the widest
// molecule makes max(rc_cg, rc_at + 2 ext) + 2 disp exceed the list cutoff, or when the
// host asked for it (the resolution region moved).  The mapping
// just written becomes current; the maxima are reset for the next mapping.
__global__ void k_decide(const __grid_constant__ Sys s, Bufs b, DecideArgs da) {
  static_assert(kExtSlots == 32, "one slot per lane");
  // launched as a programmatic dependent of the mapping kernel: its launch overlaps the
  // mapping's last blocks, and this wait returns once that grid has completed and its
  // writes are visible
  asm volatile("griddepcontrol.wait;" ::: "memory");
  Ctrl* c = b.ctrl;
  const int l = threadIdx.x;
  const unsigned me = __reduce_max_sync(0xffffffffu, c->ext_slot[0][l]);
  const unsigned mdd = __reduce_max_sync(0xffffffffu, c->ext_slot[1][l]);
  c->ext_slot[0][l] = 0u;
  c->ext_slot[1][l] = 0u;
  if (l != 0) return;
  const float e = sqrtf(__uint_as_float(me));
  const float md = sqrtf(__uint_as_float(mdd));
  const double cut = fmax(s.rc_cg, s.rc_at + 2.0 * (double)e);
  const int rb = da.force || c->force_rebuild || (md > 0.5 * s.skin) || (cut + 2.0 * md > s.r_list);
  if (cut > s.r_list) set_error(c, ADRESS_ERR_EXTENT, (int)(e * 1000));
  c->rebuild = rb;
  c->ext_now = e;
  if (rb) c->rebuilds += 1;
  if (da.advance) c->step += 1;
  c->parity ^= 1;
  if (da.use_h) cudaGraphSetConditional(da.h, (unsigned int)rb);
}

cudaError_t launch_decide(const Sys& s, const Bufs& b, DecideArgs da, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(32);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_decide, s, b, da);
}

// ---- deterministic FP64 reductions: per-block partials, then one fixed-order block ----

template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* part, int slot) {
  __shared__ double sm[32][NV];
#pragma unroll
  for (int j = 0; j < NV; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) sm[w][j] = v[j];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double acc = 0.0;
      for (int q = 0; q < nw; ++q) acc += sm[q][j];
      part[(size_t)slot * NV + j] = acc;
    }
  }
}

__global__ void __launch_bounds__(1024) k_reduce_parts(const double* part, int nparts, int nv,
                                                       double* out) {
  __shared__ double sm[32][8];
  double acc[8];
  for (int j = 0; j < nv; ++j) acc[j] = 0.0;
  for (int p = threadIdx.x; p < nparts; p += blockDim.x)
    for (int j = 0; j < nv; ++j) acc[j] += part[(size_t)p * nv + j];
  for (int j = 0; j < nv; ++j)
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if ((threadIdx.x & 31) == 0)
    for (int j = 0; j < nv; ++j) sm[threadIdx.x >> 5][j] = acc[j];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = 0; j < nv; ++j) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sm[q][j];
      out[j] = t;
    }
}

template <int NA>
__global__ void __launch_bounds__(256) k_kinetic(const __grid_constant__ Sys s, Bufs b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < s.N) {
    const double m = s.mass[i % NA];
    for (int d = 0; d < 3; ++d) {
      double u = b.v[(size_t)d * s.N + i];
      v[0] += 0.5 * m * u * u;
      v[1 + d] = m * u;
    }
  }
  block_partials<4>(v, b.part, blockIdx.x);
}

// Centre-of-mass x in double exactly as R = sum_k m_k (x_0 + minimg(x_k - x_0)) / M, wrapped.
template <int NA>
__device__ double com_x64(const Sys& s, const Box& B, const double* x, int a) {
  const double x0 = x[a * NA];
  double acc = 0.0;
  for (int k = 0; k < NA; ++k) acc += s.mass[k] * (x0 + minimg_cmp(x[a * NA + k] - x0, B.L[0], B.halfL[0]));
  double r = acc / s.Mtot;
  r -= B.L[0] * floor(r / B.L[0]);
  if (r >= B.L[0]) r -= B.L[0];
  return r;
}

// Distance of molecule a's centre of mass (in double, from x, as the definition forms it) to
// the nearest resolution centre (the first of equal distances).
template <int NA>
__device__ double center_d64(const Sys& s, const Box& B, const Bufs& b, int a) {
  const size_t N = (size_t)s.N;
  double R[3];
  for (int d = 0; d < 3; ++d) {
    const double x0 = b.x[d * N + a * NA];
    double acc = 0.0;
    for (int k = 0; k < NA; ++k) acc += s.mass[k] * (x0 + minimg_cmp(b.x[d * N + a * NA + k] - x0, B.L[d], B.halfL[d]));
    double r = acc / s.Mtot;
    r -= B.L[d] * floor(r / B.L[d]);
    if (r >= B.L[d]) r -= B.L[d];
    R[d] = r;
  }
  double best = INFINITY;
  for (int k = 0; k < s.n_centers; ++k) {
    const double4_32a C = b.cen64[k];
    const double t0 = minimg_cmp(R[0] - C.x, B.L[0], B.halfL[0]);
    const double t1 = minimg_cmp(R[1] - C.y, B.L[1], B.halfL[1]);
    const double t2 = minimg_cmp(R[2] - C.z, B.L[2], B.halfL[2]);
    const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(t0, t0), __dmul_rn(t1, t1)), __dmul_rn(t2, t2)));
    if (r < best) best = r;
  }
  return best;
}

// COM histogram folded about the slab centre: bin floor(|dxc| / tf_dx), integer atomics
// (one histogram of tf_n bins per box).  The FP32 path takes |dxc| from its float mapping
// and recomputes it in double for the few molecules within 1e-4 of a bin edge, so the bin
// is the one the double value gives.  A single box counts into shared memory first.
template <int NA>
__global__ void __launch_bounds__(1024) k_density(const __grid_constant__ Sys s, Bufs b) {
  extern __shared__ unsigned hs[];
  const bool multi = s.nbox > 1;
  if (!multi) {
    for (int k = threadIdx.x; k < s.tf_n; k += blockDim.x) hs[k] = 0u;
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd((unsigned long long*)b.nsamples, 1ull);
  const int cur = b.ctrl->parity;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < s.M; a += gridDim.x * blockDim.x) {
    const Box& B = box_of(s, b, a);
    int k;
    if (s.fp64) {
      k = (int)floor(fabs(b.dxc64[cur][a]) / s.tf_dx);
    } else {
      const float u = fabsf(b.molf[cur][a].x) * s.f.tf_inv_dx, fr = u - floorf(u);
      k = (int)floorf(u);
      if (fr < 1e-4f || fr > 1.f - 1e-4f)
        k = (int)floor((s.n_centers > 0 ? center_d64<NA>(s, B, b, a)
                                        : fabs(minimg_cmp(com_x64<NA>(s, B, b.x, a) - B.xc, B.L[0], B.halfL[0]))) /
                       s.tf_dx);
    }
    if (k < s.tf_n) {
      if (multi) atomicAdd(&b.hist[B.tf0 + k], 1ull);
      else atomicAdd(&hs[k], 1u);
    }
  }
  if (!multi) {
    __syncthreads();
    for (int k = threadIdx.x; k < s.tf_n; k += blockDim.x)
      if (hs[k]) atomicAdd(&b.hist[k], (unsigned long long)hs[k]);
  }
}

// Thermodynamic-force iteration on the accumulated profile, one block per box (tf_n nodes):
// rho_k = counts_k / (nsamples V_k) (V_k: 2 dx Ly Lz, or the shells around the resolution
// centres), g_k = (rho_k - rho_{k-1})/dx, g_0 = 0,
// three-point moving average, tf_k -= alpha g_k on hybrid-layer nodes, then the box's
// histogram is cleared (the sample count is cleared by the launcher afterwards).
__global__ void k_tf_update(const __grid_constant__ Sys s, Bufs b, double alpha) {
  extern __shared__ double g[];
  const Box& B = s.nbox > 1 ? b.boxes[blockIdx.x] : s.bx;
  const int n = s.tf_n, o = B.tf0;
  const double ns = (double)(*b.nsamples);
  // bin volume: two slabs, or a spherical shell around each resolution centre
  auto vol = [&](int k) {
    const double dx = s.tf_dx;
    return s.n_centers > 0
               ? ns * s.n_centers * 4.0 / 3.0 * M_PI * ((k + 1.0) * (k + 1.0) * (k + 1.0) - (double)k * k * k) * dx * dx * dx
               : ns * 2.0 * dx * B.L[1] * B.L[2];
  };
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double gk = 0.0;
    if (k > 0 && ns > 0) gk = ((double)b.hist[o + k] / vol(k) - (double)b.hist[o + k - 1] / vol(k - 1)) / s.tf_dx;
    g[k] = gk;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double sum = 0.0;
    int cnt = 0;
    for (int q = k - 1; q <= k + 1; ++q)
      if (q >= 0 && q < n) {
        sum += g[q];
        ++cnt;
      }
    const double dk = k * s.tf_dx;
    if (ns > 0 && dk >= B.d_at && dk <= B.d_at + B.d_hy) {
      double t = b.tf64[o + k] - alpha * sum / cnt;
      b.tf64[o + k] = t;
      b.tf32[o + k] = (float)t;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) b.hist[o + k] = 0ull;
}

// FP64 centres of mass of the current positions (computed from x as the definition
// states) and the resolution values the force kernels use.
__global__ void k_clear_samples(long long* n) { *n = 0; }

template <int NA>
__global__ void k_export_com(const __grid_constant__ Sys s, Bufs b, double* com, double* w) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= s.M) return;
  const Box& B = box_of(s, b, a);
  const size_t N = (size_t)s.N;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < 3; ++d) {
    const double x0 = b.x[d * N + a * NA];
    for (int k = 0; k < NA; ++k)
      acc[d] += s.mass[k] * (x0 + minimg_cmp(b.x[d * N + a * NA + k] - x0, B.L[d], B.halfL[d]));
    double r = acc[d] / s.Mtot;
    r -= B.L[d] * floor(r / B.L[d]);
    if (r >= B.L[d]) r -= B.L[d];
    com[(size_t)d * s.M + a] = r;
  }
  if (w) {
    const int cur = b.ctrl->parity;
    w[a] = s.fp64 ? b.com64[cur][a].w : (double)__int_as_float(b.com_fx[cur][a].w);
  }
}

// COM pair-distance histogram (numerator of the radial distribution function): every pair
// a < b of the same box with minimum-image distance r < nbins dr adds one to bin
// floor(r / dr) of its box.  All pairs, tiled: a block owns 256 molecules a and streams the
// molecules b >= its first one (up to the end of the last box it touches) through shared
// memory.  A float test with a margin discards the distant pairs; the rest are decided in
// double with explicitly rounded products and sums (no contraction), the operations the
// oracle performs, so bins are the oracle's.  One box counts into shared memory first.
constexpr int kRdfTile = 256;
__global__ void __launch_bounds__(kRdfTile) k_rdf(const __grid_constant__ Sys s, Bufs b, const double* __restrict__ com,
                                                  int nbins, double dr, float lim2, unsigned long long* counts) {
  extern __shared__ unsigned rh[];
  __shared__ double sx[kRdfTile], sy[kRdfTile], sz[kRdfTile];
  __shared__ float fx[kRdfTile], fy[kRdfTile], fz[kRdfTile];
  __shared__ int sbox[kRdfTile];
  const bool multi = s.nbox > 1;
  const int M = s.M;
  if (!multi)
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) rh[k] = 0u;
  const int i0 = blockIdx.x * kRdfTile;
  const int a = i0 + threadIdx.x;
  const bool live = a < M;
  const int ac = live ? a : M - 1;
  const Box& B = box_of(s, b, ac);
  const int mybox = multi ? b.mol_box[ac] : 0;
  int jend = M;
  if (multi) {
    const Box& BL = b.boxes[b.mol_box[min(i0 + kRdfTile, M) - 1]];
    jend = BL.mol0 + BL.nmol;
  }
  const double xa = com[ac], ya = com[(size_t)M + ac], za = com[2 * (size_t)M + ac];
  const float xaf = (float)xa, yaf = (float)ya, zaf = (float)za;
  const float Lx = (float)B.L[0], Ly = (float)B.L[1], Lz = (float)B.L[2];
  const float hx = 0.5f * Lx, hy = 0.5f * Ly, hz = 0.5f * Lz;
  for (int j0 = i0; j0 < jend; j0 += kRdfTile) {
    __syncthreads();
    const int j = j0 + threadIdx.x;
    if (j < jend) {
      const double X = com[j], Y = com[(size_t)M + j], Z = com[2 * (size_t)M + j];
      sx[threadIdx.x] = X;
      sy[threadIdx.x] = Y;
      sz[threadIdx.x] = Z;
      fx[threadIdx.x] = (float)X;
      fy[threadIdx.x] = (float)Y;
      fz[threadIdx.x] = (float)Z;
      sbox[threadIdx.x] = multi ? b.mol_box[j] : 0;
    }
    __syncthreads();
    if (!live) continue;
    const int n = min(kRdfTile, jend - j0);
    for (int q = max(0, a + 1 - j0); q < n; ++q) {
      float dx = xaf - fx[q], dy = yaf - fy[q], dz = zaf - fz[q];
      dx = dx > hx ? dx - Lx : (dx < -hx ? dx + Lx : dx);
      dy = dy > hy ? dy - Ly : (dy < -hy ? dy + Ly : dy);
      dz = dz > hz ? dz - Lz : (dz < -hz ? dz + Lz : dz);
      if (dx * dx + dy * dy + dz * dz >= lim2) continue;
      if (multi && sbox[q] != mybox) continue;
      const double ex = minimg_cmp(xa - sx[q], B.L[0], B.halfL[0]);
      const double ey = minimg_cmp(ya - sy[q], B.L[1], B.halfL[1]);
      const double ez = minimg_cmp(za - sz[q], B.L[2], B.halfL[2]);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
      const int k = (int)floor(sqrt(r2) / dr);
      if (k < nbins) {
        if (multi) atomicAdd(&counts[(size_t)mybox * nbins + k], 1ull);
        else atomicAdd(&rh[k], 1u);
      }
    }
  }
  if (!multi) {
    __syncthreads();
    for (int k = threadIdx.x; k < nbins; k += blockDim.x)
      if (rh[k]) atomicAdd(&counts[k], (unsigned long long)rh[k]);
  }
}

// ---- launchers -----------------------------------------------------------------------


cudaError_t launch_energy_reduce(const Sys& s, const Bufs& b, int nparts, int nvals, cudaStream_t st) {
  k_reduce_parts<<<1, 1024, 0, st>>>(b.part, nparts, nvals, b.result);
  return cudaGetLastError();
}

cudaError_t launch_kinetic(const Sys& s, const Bufs& b, cudaStream_t st) {
  const int blocks = ceil_div(s.N, 256);
  switch (s.NA) {
    case 1: k_kinetic<1><<<blocks, 256, 0, st>>>(s, b); break;
    case 2: k_kinetic<2><<<blocks, 256, 0, st>>>(s, b); break;
    case 3: k_kinetic<3><<<blocks, 256, 0, st>>>(s, b); break;
    default: k_kinetic<4><<<blocks, 256, 0, st>>>(s, b); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_energy_reduce(s, b, blocks, 4, st);
}

cudaError_t launch_density(const Sys& s, const Bufs& b, int, cudaStream_t st) {
  const int blocks = std::min(ceil_div(s.M, 1024), 2 * 152);
  const size_t smem = s.nbox > 1 ? 0 : sizeof(unsigned) * std::max(1, s.tf_n);
  switch (s.NA) {
    case 1: k_density<1><<<blocks, 1024, smem, st>>>(s, b); break;
    case 2: k_density<2><<<blocks, 1024, smem, st>>>(s, b); break;
    case 3: k_density<3><<<blocks, 1024, smem, st>>>(s, b); break;
    default: k_density<4><<<blocks, 1024, smem, st>>>(s, b); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_tf_update(const Sys& s, const Bufs& b, double alpha, cudaStream_t st) {
  if (s.tf_n <= 0) return cudaSuccess;
  k_tf_update<<<s.nbox, 256, sizeof(double) * s.tf_n, st>>>(s, b, alpha);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_clear_samples<<<1, 1, 0, st>>>(b.nsamples);
  return cudaGetLastError();
}

cudaError_t launch_rdf(const Sys& s, const Bufs& b, const double* com, int nbins, double dr,
                       unsigned long long* counts, cudaStream_t st) {
  const double rmax = nbins * dr;
  const float lim2 = (float)((rmax + 1e-3 * (1.0 + rmax)) * (rmax + 1e-3 * (1.0 + rmax)));
  const size_t smem = s.nbox > 1 ? 0 : sizeof(unsigned) * nbins;
  k_rdf<<<ceil_div(s.M, kRdfTile), kRdfTile, smem, st>>>(s, b, com, nbins, dr, lim2, counts);
  return cudaGetLastError();
}

cudaError_t launch_export_com(const Sys& s, const Bufs& b, int, double* com, double* w, cudaStream_t st) {
  const int blocks = ceil_div(s.M, 256);
  switch (s.NA) {
    case 1: k_export_com<1><<<blocks, 256, 0, st>>>(s, b, com, w); break;
    case 2: k_export_com<2><<<blocks, 256, 0, st>>>(s, b, com, w); break;
    case 3: k_export_com<3><<<blocks, 256, 0, st>>>(s, b, com, w); break;
    default: k_export_com<4><<<blocks, 256, 0, st>>>(s, b, com, w); break;
  }
  return cudaGetLastError();
}

}  // namespace adress
