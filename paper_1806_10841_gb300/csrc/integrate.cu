// Per-molecule kernels: first half of velocity Verlet, centre-of-mass mapping and the
// resolution function; the list-rebuild decision; FP64 reductions; the COM density
// profile and the thermodynamic-force iteration.
#include <math.h>

#include "internal.cuh"

namespace adress {

// First half kick + drift + wrap (when `integrate`), then the molecule's centre of mass
// R = sum m_k (x_0 + minimg(x_k - x_0)) / M wrapped into the box, the signed distance
// dxc = minimg(R_x - x_c), the resolution value l(|dxc|) (1 / squared cosine / 0,
// Sec. "Force interpolation") and the COM-relative atom offsets used by the force
// kernels.  One thread per molecule; the atoms of a molecule are contiguous so a warp
// reads 32*na consecutive doubles per component.
template <class P, int NA>
__global__ void __launch_bounds__(256) k_com(Sys s, Bufs b, int integrate) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  float ext = 0.f, disp2 = 0.f;
  if (a < s.M) {
    const int N = s.N;
    double xl[NA][3];
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const int i = a * NA + k;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double x = b.x[(size_t)d * N + i];
        if (integrate) {
          double fv = P::fp64 ? ((const double*)b.f)[(size_t)d * N + i]
                              : (double)((const float*)b.f)[(size_t)d * N + i];
          double v = b.v[(size_t)d * N + i];
          v = fma(0.5 * s.dt * s.inv_mass[k], fv, v);
          x = fma(s.dt, v, x);
          if (x < 0.0) x += s.L[d];
          if (x >= s.L[d]) x -= s.L[d];
          b.v[(size_t)d * N + i] = v;
          b.x[(size_t)d * N + i] = x;
        }
        xl[k][d] = x;
      }
    }
    // minimum-image unwrap relative to atom 0, then the mass-weighted mean offset c
    const double x0[3] = {xl[0][0], xl[0][1], xl[0][2]};
    double c[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = NA - 1; k >= 0; --k)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double dl = k ? minimg_cmp(xl[k][d] - xl[0][d], s.L[d], s.halfL[d]) : 0.0;
        xl[k][d] = dl;
        c[d] = fma(s.frac[k], dl, c[d]);
      }
    double R[3];
    unsigned int X[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double r = x0[d] + c[d];
      if (r < 0.0) r += s.L[d];
      if (r >= s.L[d]) r -= s.L[d];
      R[d] = r;
      X[d] = (unsigned int)(unsigned long long)llrint(r * s.fx_inv[d]);
    }
    const double dxc = minimg_cmp(R[0] - s.xc, s.L[0], s.halfL[0]);
    const double dd = fabs(dxc);
    double w;
    float wf;
    if (P::fp64) {
      if (dd < s.d_at) w = 1.0;
      else if (dd >= s.d_at + s.d_hy) w = 0.0;
      else {
        double cs = cos((dd - s.d_at) * s.pi_half_over_dhy);
        w = cs * cs;
      }
      wf = (float)w;
    } else {
      if (dd < s.d_at) wf = 1.f;
      else if (dd >= s.d_at + s.d_hy) wf = 0.f;
      else {
        float cs = cosf((float)((dd - s.d_at) * s.pi_half_over_dhy));
        wf = cs * cs;
      }
      w = (double)wf;
    }
    // COM-relative offsets o_k = (x_0 + minimg(x_k - x_0)) - R_unwrapped = dl_k - c
    float e2 = 0.f;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const int i = a * NA + k;
      double o0 = xl[k][0] - c[0], o1 = xl[k][1] - c[1], o2 = xl[k][2] - c[2];
      float q0 = (float)o0, q1 = (float)o1, q2 = (float)o2;
      e2 = fmaxf(e2, q0 * q0 + q1 * q1 + q2 * q2);
      if (P::fp64) b.off64[i] = make_double4_32a(o0, o1, o2, 0.0);
      else b.off32[i] = make_float4(q0, q1, q2, 0.f);
    }
    ext = sqrtf(e2);
    b.com64[a] = make_double4_32a(R[0], R[1], R[2], w);
    b.dxc64[a] = dxc;
    if (!P::fp64) b.molf[a] = make_float2((float)dxc, wf);
    int4 cf = make_int4((int)X[0], (int)X[1], (int)X[2], __float_as_int(wf));
    b.com_fx[a] = cf;
    int4 ref = b.com_ref[a];
    float d0 = (float)(int)(X[0] - (unsigned)ref.x) * s.fx_scale[0];
    float d1 = (float)(int)(X[1] - (unsigned)ref.y) * s.fx_scale[1];
    float d2 = (float)(int)(X[2] - (unsigned)ref.z) * s.fx_scale[2];
    disp2 = d0 * d0 + d1 * d1 + d2 * d2;
  }
  unsigned int e = __reduce_max_sync(0xffffffffu, __float_as_uint(ext));
  unsigned int dm = __reduce_max_sync(0xffffffffu, __float_as_uint(disp2));
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&b.ctrl->maxext, e);
    atomicMax(&b.ctrl->maxdisp2, dm);
  }
}

// Rebuild decision for this step: rebuild when a centre moved more than skin/2 since the
// last build (it could have changed class or found a new partner) or when the widest
// molecule makes max(rc_cg, rc_at + 2 ext) + 2 disp exceed the list cutoff.
__global__ void k_decide(Sys s, Ctrl* c, int force, int advance, cudaGraphConditionalHandle h,
                         int use_h) {
  const float ext = __uint_as_float(c->maxext);
  const float md = sqrtf(__uint_as_float(c->maxdisp2));
  const double cut = fmax(s.rc_cg, s.rc_at + 2.0 * (double)ext);
  int rb = force || (md > 0.5 * s.skin) || (cut + 2.0 * md > s.r_list);
  if (cut > s.r_list) set_error(c, ADRESS_ERR_EXTENT, (int)(ext * 1000));
  c->rebuild = rb;
  c->ext_now = ext;
  c->maxext = 0u;
  c->maxdisp2 = 0u;
  if (rb) c->rebuilds += 1;
  if (advance) c->step += 1;
  if (use_h) cudaGraphSetConditional(h, (unsigned int)rb);
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
__global__ void __launch_bounds__(256) k_kinetic(Sys s, Bufs b) {
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

// COM histogram folded about the slab centre: bin floor(|dxc| / tf_dx), integer atomics.
__global__ void k_density(Sys s, Bufs b) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a == 0) atomicAdd((unsigned long long*)b.nsamples, 1ull);
  if (a >= s.M) return;
  const double d = fabs(b.dxc64[a]);
  const int k = (int)floor(d / s.tf_dx);
  if (k < s.tf_n) atomicAdd(&b.hist[k], 1ull);
}

// Thermodynamic-force iteration on the accumulated profile (one block, tf_n nodes):
// rho_k = counts_k / (nsamples 2 dx Ly Lz), g_k = (rho_k - rho_{k-1})/dx, g_0 = 0,
// three-point moving average, tf_k -= alpha g_k on hybrid-layer nodes, then reset.
__global__ void k_tf_update(Sys s, Bufs b, double alpha) {
  extern __shared__ double g[];
  const int n = s.tf_n;
  const double ns = (double)(*b.nsamples);
  const double vol = ns * 2.0 * s.tf_dx * s.L[1] * s.L[2];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double gk = 0.0;
    if (k > 0 && ns > 0) gk = ((double)b.hist[k] / vol - (double)b.hist[k - 1] / vol) / s.tf_dx;
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
    if (ns > 0 && dk >= s.d_at && dk <= s.d_at + s.d_hy) {
      double t = b.tf64[k] - alpha * sum / cnt;
      b.tf64[k] = t;
      b.tf32[k] = (float)t;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) b.hist[k] = 0ull;
  if (threadIdx.x == 0) *b.nsamples = 0;
}

__global__ void k_export_com(Sys s, Bufs b, double* com, double* w) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= s.M) return;
  double4_32a r = b.com64[a];
  com[a] = r.x;
  com[(size_t)s.M + a] = r.y;
  com[2 * (size_t)s.M + a] = r.z;
  w[a] = r.w;
}

// ---- launchers -----------------------------------------------------------------------

template <class P>
static cudaError_t launch_com_p(const Sys& s, const Bufs& b, int integrate, cudaStream_t st) {
  const int blocks = ceil_div(s.M, 256);
  switch (s.NA) {
    case 1: k_com<P, 1><<<blocks, 256, 0, st>>>(s, b, integrate); break;
    case 2: k_com<P, 2><<<blocks, 256, 0, st>>>(s, b, integrate); break;
    case 3: k_com<P, 3><<<blocks, 256, 0, st>>>(s, b, integrate); break;
    default: k_com<P, 4><<<blocks, 256, 0, st>>>(s, b, integrate); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_com(const Sys& s, const Bufs& b, int precision, int integrate, cudaStream_t st) {
  return precision == ADRESS_FP64 ? launch_com_p<P64>(s, b, integrate, st)
                                  : launch_com_p<P32>(s, b, integrate, st);
}

cudaError_t launch_decide(const Sys& s, const Bufs& b, int force, int advance,
                          cudaGraphConditionalHandle h, int use_h, cudaStream_t st) {
  k_decide<<<1, 1, 0, st>>>(s, b.ctrl, force, advance, h, use_h);
  return cudaGetLastError();
}

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
  k_density<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b);
  return cudaGetLastError();
}

cudaError_t launch_tf_update(const Sys& s, const Bufs& b, double alpha, cudaStream_t st) {
  if (s.tf_n <= 0) return cudaSuccess;
  k_tf_update<<<1, 256, sizeof(double) * s.tf_n, st>>>(s, b, alpha);
  return cudaGetLastError();
}

cudaError_t launch_export_com(const Sys& s, const Bufs& b, double* com, double* w, cudaStream_t st) {
  k_export_com<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b, com, w);
  return cudaGetLastError();
}

}  // namespace adress
