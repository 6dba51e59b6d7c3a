// Force kernel of the AdResS step.  Work item t is one molecule; a group of four
// consecutive threads handles it, thread g owning atom g.  Items 0..n_hr-1 are
// high-resolution candidates (atomistic or hybrid at the last list build), the rest are
// coarse-grained molecules:
//  - high-resolution item: each thread sums, for its atom i and every listed neighbour
//    molecule b, the interpolated pair force of Eq. 1 (Sec. "Force interpolation"):
//      w_ab sum_j f^WCA(r_ij) + (1 - w_ab) (m_i/M) F^CG(|R_ab|) R_ab/|R_ab|,
//    w_ab = l_a l_b, the AT part only when w_ab > 0, the CG part only when w_ab < 1;
//  - coarse-grained item (l_a = 0, so w_ab = 0): the four threads split the neighbour
//    list, sum F^CG on the centre and combine it with warp shuffles; each thread takes
//    the mass fraction m_g/M of it.
// Then every thread adds its atom's bonded terms (FENE + WCA, never interpolated, same
// section) and the thermodynamic force in the hybrid layer (Sec. "Free energy corrections
// and the thermodynamic force").  In step mode it also adds the Langevin force and applies
// the second half kick, so the total force never makes an extra trip through memory.
// Each atom's force is written exactly once by its owner: no atomics, deterministic.
#include <math.h>

#include "internal.cuh"

namespace adress {

template <class P>
struct Prec;

template <>
struct Prec<P64> {
  using real = double;
  struct V3 {
    double x, y, z;
  };
  static __device__ __forceinline__ double4_32a com(const Bufs& b, int a) { return b.com64[a]; }
  static __device__ __forceinline__ double w(const double4_32a& c) { return c.w; }
  static __device__ __forceinline__ V3 dR(const Sys& s, const double4_32a& A, const double4_32a& B) {
    return {minimg_cmp(A.x - B.x, s.L[0], s.halfL[0]), minimg_cmp(A.y - B.y, s.L[1], s.halfL[1]),
            minimg_cmp(A.z - B.z, s.L[2], s.halfL[2])};
  }
  static __device__ __forceinline__ double4_32a off(const Bufs& b, int i) { return b.off64[i]; }
  static __device__ __forceinline__ double dxc(const Bufs& b, int a) { return b.dxc64[a]; }
  static __device__ __forceinline__ double cg(const Bufs& b, int cg_n, double r, double inv_dr, double* V) {
    const double u = r * inv_dr;
    int k = (int)u;
    if (k > cg_n - 1) k = cg_n - 1;
    const double t = u - k;
    *V = b.cgV64[k] * (1.0 - t) + b.cgV64[k + 1] * t;
    return b.cgF64[k] * (1.0 - t) + b.cgF64[k + 1] * t;
  }
  static __device__ __forceinline__ double tf(const Bufs& b, int k) { return b.tf64[k]; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};

template <>
struct Prec<P32> {
  using real = float;
  struct V3 {
    float x, y, z;
  };
  static __device__ __forceinline__ int4 com(const Bufs& b, int a) { return b.com_fx[a]; }
  static __device__ __forceinline__ float w(const int4& c) { return __int_as_float(c.w); }
  // exact integer difference of fixed-point centres (periodic wrap for free), then float
  static __device__ __forceinline__ V3 dR(const Sys& s, const int4& A, const int4& B) {
    return {(float)(int)((unsigned)A.x - (unsigned)B.x) * s.fx_scale[0],
            (float)(int)((unsigned)A.y - (unsigned)B.y) * s.fx_scale[1],
            (float)(int)((unsigned)A.z - (unsigned)B.z) * s.fx_scale[2]};
  }
  static __device__ __forceinline__ float4 off(const Bufs& b, int i) { return b.off32[i]; }
  static __device__ __forceinline__ float dxc(const Bufs& b, int a) { return b.molf[a].x; }
  static __device__ __forceinline__ float cg(const Bufs& b, int cg_n, float r, float inv_dr, float* V) {
    const float u = r * inv_dr;
    int k = (int)u;
    if (k > cg_n - 1) k = cg_n - 1;
    const float t = u - (float)k;
    const float2 lo = b.cgFV32[k], hi = b.cgFV32[k + 1];
    *V = fmaf(t, hi.y - lo.y, lo.y);
    return fmaf(t, hi.x - lo.x, lo.x);
  }
  static __device__ __forceinline__ float tf(const Bufs& b, int k) { return b.tf32[k]; }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
};

template <class P, int NA, bool STEP, bool ENERGY>
__global__ void __launch_bounds__(kForceBlock) k_forces(Sys s, Bufs b) {
  using Q = Prec<P>;
  using real = typename Q::real;
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x & 3;
  const unsigned gmask = 0xFu << (lane & ~3);
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const bool live = t < s.M;
  const bool own = live && g < NA;
  const int M = s.M;

  const real eps = (real)s.eps, sig2 = (real)s.sig2, rc_at2 = (real)s.rc_at2, rc_cg2 = (real)s.rc_cg2;
  const real inv_dr = (real)s.cg_inv_dr;
  const float ext = b.ctrl->ext_now;
  const real reach_at2 = (real)((s.rc_at + 2.0 * (double)ext) * (s.rc_at + 2.0 * (double)ext));
  const real frac_g = (real)s.frac[g < NA ? g : 0];

  real fx = 0, fy = 0, fz = 0;
  double e_at = 0.0, e_cg = 0.0, e_b = 0.0, vir = 0.0;

  const int a = live ? b.items[t] : 0;
  const int i = a * NA + (g < NA ? g : 0);
  const auto Ca = Q::com(b, a);
  const real wa = Q::w(Ca);
  const auto oi = Q::off(b, i);
  const int nnb = live ? b.nn[t] : 0;

  if (t < b.ctrl->n_hr) {
    // ---- high-resolution item: Eq. 1 for atom i against every neighbour ----
    for (int q = 0; q < nnb; ++q) {
      const int m = b.nbr[(size_t)q * M + t];
      const auto Cb = Q::com(b, m);
      const auto R = Q::dR(s, Ca, Cb);
      const real r2 = R.x * R.x + R.y * R.y + R.z * R.z;
      const real wab = wa * Q::w(Cb);
      if (own && wab > (real)0 && r2 < reach_at2) {
        const real px = R.x + (real)oi.x, py = R.y + (real)oi.y, pz = R.z + (real)oi.z;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          const auto oj = Q::off(b, m * NA + j);
          const real dx = px - (real)oj.x, dy = py - (real)oj.y, dz = pz - (real)oj.z;
          const real d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < rc_at2) {
            const real ir2 = (real)1 / d2;
            const real sr2 = sig2 * ir2;
            const real sr6 = sr2 * sr2 * sr2;
            const real fr = (real)24 * eps * ((real)2 * sr6 * sr6 - sr6) * ir2 * wab;
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
            if (ENERGY) {
              e_at += 0.5 * (double)wab * (double)((real)4 * eps * (sr6 * sr6 - sr6) + eps);
              vir += 0.5 * (double)(fr * d2);
            }
          }
        }
      }
      if (own && wab < (real)1 && r2 < rc_cg2) {
        const real r = Q::sqrt_(r2);
        real V;
        const real F = Q::cg(b, s.cg_n, r, inv_dr, &V);
        const real c = ((real)1 - wab) * F / r;
        fx += frac_g * c * R.x;
        fy += frac_g * c * R.y;
        fz += frac_g * c * R.z;
        if (ENERGY && g == 0) {
          e_cg += 0.5 * (double)(((real)1 - wab) * V);
          vir += 0.5 * (double)(c * r2);
        }
      }
    }
  } else {
    // ---- coarse-grained item: neighbour list split over the group ----
    if (live && g == 0 && wa != (real)0) set_error(b.ctrl, ADRESS_ERR_STATE, a);
    real Fx = 0, Fy = 0, Fz = 0;
    for (int q = g; q < nnb; q += kGroup) {
      const int m = b.nbr[(size_t)q * M + t];
      const auto Cb = Q::com(b, m);
      const auto R = Q::dR(s, Ca, Cb);
      const real r2 = R.x * R.x + R.y * R.y + R.z * R.z;
      if (r2 < rc_cg2) {
        const real r = Q::sqrt_(r2);
        real V;
        const real F = Q::cg(b, s.cg_n, r, inv_dr, &V);
        const real c = F / r;
        Fx += c * R.x;
        Fy += c * R.y;
        Fz += c * R.z;
        if (ENERGY) {
          e_cg += 0.5 * (double)V;
          vir += 0.5 * (double)(c * r2);
        }
      }
    }
    Fx += __shfl_xor_sync(gmask, Fx, 1);
    Fy += __shfl_xor_sync(gmask, Fy, 1);
    Fz += __shfl_xor_sync(gmask, Fz, 1);
    Fx += __shfl_xor_sync(gmask, Fx, 2);
    Fy += __shfl_xor_sync(gmask, Fy, 2);
    Fz += __shfl_xor_sync(gmask, Fz, 2);
    fx = frac_g * Fx;
    fy = frac_g * Fy;
    fz = frac_g * Fz;
  }

  if (own) {
    // ---- bonded terms of atom g (FENE + WCA on listed intramolecular pairs) ----
    const real R02 = (real)s.fene_r02, K = (real)s.fene_k;
#pragma unroll
    for (int q = 0; q < kMaxBonds; ++q) {
      if (q >= s.nb) break;
      const int p0 = s.bonds[2 * q], p1 = s.bonds[2 * q + 1];
      if (g != p0 && g != p1) continue;
      const int other = g == p0 ? p1 : p0;
      const auto oo = Q::off(b, a * NA + other);
      const real dx = (real)oi.x - (real)oo.x, dy = (real)oi.y - (real)oo.y, dz = (real)oi.z - (real)oo.z;
      const real d2 = dx * dx + dy * dy + dz * dz;
      if (d2 >= R02) {
        set_error(b.ctrl, ADRESS_ERR_BOND_BROKEN, a);
        continue;
      }
      const real gg = (real)1 - d2 / R02;
      real fr = -K / gg;
      double V = 0.0;
      if (ENERGY) V = -0.5 * (double)K * (double)R02 * log((double)gg);
      if (s.intra_wca && d2 < rc_at2) {
        const real ir2 = (real)1 / d2;
        const real sr2 = sig2 * ir2;
        const real sr6 = sr2 * sr2 * sr2;
        fr += (real)24 * eps * ((real)2 * sr6 * sr6 - sr6) * ir2;
        if (ENERGY) V += (double)((real)4 * eps * (sr6 * sr6 - sr6) + eps);
      }
      fx += fr * dx;
      fy += fr * dy;
      fz += fr * dz;
      if (ENERGY && g == p0) {
        e_b += V;
        vir += (double)(fr * d2);
      }
    }
    // ---- thermodynamic force in the hybrid layer ----
    if (s.tf_n > 0) {
      const real dxc = Q::dxc(b, a);
      const real d = dxc < (real)0 ? -dxc : dxc;
      if (d >= (real)s.d_at && d < (real)(s.d_at + s.d_hy)) {
        const real u = d * (real)s.tf_inv_dx;
        const int k = (int)u;
        real F = 0;
        if (k + 1 < s.tf_n) {
          const real tt = u - (real)k;
          F = Q::tf(b, k) * ((real)1 - tt) + Q::tf(b, k + 1) * tt;
        } else if (k + 1 == s.tf_n && u == (real)k) {
          F = Q::tf(b, k);
        }
        fx += frac_g * (dxc < (real)0 ? -F : F);
      }
    }
    const size_t N = (size_t)s.N;
    if (STEP) {
      // ---- Langevin force with the half-step velocity, then the second half kick ----
      const double m = s.mass[g], hdt_m = 0.5 * s.dt * s.inv_mass[g];
      unsigned long long c[4] = {(unsigned long long)i, (unsigned long long)s.replica, 0ull, 0ull};
      philox4x64_10(c, s.seed, (unsigned long long)b.ctrl->step);
      const double vx = b.v[i], vy = b.v[N + i], vz = b.v[2 * N + i];
      const double amp = sqrt(24.0 * s.gamma * s.kT * m / s.dt);
      if (P::fp64) {
        const double k53 = 1.0 / 9007199254740992.0;
        fx += -s.gamma * m * vx + amp * ((double)(c[0] >> 11) * k53 - 0.5);
        fy += -s.gamma * m * vy + amp * ((double)(c[1] >> 11) * k53 - 0.5);
        fz += -s.gamma * m * vz + amp * ((double)(c[2] >> 11) * k53 - 0.5);
      } else {
        const float k24 = 1.0f / 16777216.0f, gm = (float)(s.gamma * m), af = (float)amp;
        fx += -gm * (float)vx + af * ((float)(unsigned)(c[0] >> 40) * k24 - 0.5f);
        fy += -gm * (float)vy + af * ((float)(unsigned)(c[1] >> 40) * k24 - 0.5f);
        fz += -gm * (float)vz + af * ((float)(unsigned)(c[2] >> 40) * k24 - 0.5f);
      }
      b.v[i] = fma(hdt_m, (double)fx, vx);
      b.v[N + i] = fma(hdt_m, (double)fy, vy);
      b.v[2 * N + i] = fma(hdt_m, (double)fz, vz);
    }
    real* fo = (real*)b.f;
    fo[i] = fx;
    fo[N + i] = fy;
    fo[2 * N + i] = fz;
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) set_error(b.ctrl, ADRESS_ERR_NONFINITE, i);
  }

  if (ENERGY) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e_at += __shfl_xor_sync(0xffffffffu, e_at, o);
      e_cg += __shfl_xor_sync(0xffffffffu, e_cg, o);
      e_b += __shfl_xor_sync(0xffffffffu, e_b, o);
      vir += __shfl_xor_sync(0xffffffffu, vir, o);
    }
    if (lane == 0) {
      const size_t wid = (size_t)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
      b.part[wid * 4 + 0] = e_at;
      b.part[wid * 4 + 1] = e_cg;
      b.part[wid * 4 + 2] = e_b;
      b.part[wid * 4 + 3] = vir;
    }
  }
}

template <class P, int NA>
static void launch_fp(const Sys& s, const Bufs& b, int step_mode, int energy, cudaStream_t st) {
  const int blocks = ceil_div((long long)s.M * kGroup, kForceBlock);
  if (step_mode) {
    if (energy) k_forces<P, NA, true, true><<<blocks, kForceBlock, 0, st>>>(s, b);
    else k_forces<P, NA, true, false><<<blocks, kForceBlock, 0, st>>>(s, b);
  } else {
    if (energy) k_forces<P, NA, false, true><<<blocks, kForceBlock, 0, st>>>(s, b);
    else k_forces<P, NA, false, false><<<blocks, kForceBlock, 0, st>>>(s, b);
  }
}

template <class P>
static void launch_p(const Sys& s, const Bufs& b, int step_mode, int energy, cudaStream_t st) {
  switch (s.NA) {
    case 1: launch_fp<P, 1>(s, b, step_mode, energy, st); break;
    case 2: launch_fp<P, 2>(s, b, step_mode, energy, st); break;
    case 3: launch_fp<P, 3>(s, b, step_mode, energy, st); break;
    default: launch_fp<P, 4>(s, b, step_mode, energy, st); break;
  }
}

cudaError_t launch_forces(const Sys& s, const Bufs& b, int precision, int step_mode, int energy,
                          cudaStream_t st) {
  if (precision == ADRESS_FP64) launch_p<P64>(s, b, step_mode, energy, st);
  else launch_p<P32>(s, b, step_mode, energy, st);
  return cudaGetLastError();
}

}  // namespace adress
