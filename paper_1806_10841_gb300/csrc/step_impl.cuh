// The MD-step kernels of the AdResS library (templates; instantiated by step.cu for the
// WCA model and by step_ljrf.cu for the water-like Lennard-Jones + reaction-field model).
//
// One group of four consecutive threads handles one molecule (work item t), thread g
// owning atom g.  Kernels:
//   k_map      positions -> centre of mass, resolution value, COM-relative offsets
//   k_prologue first half kick + drift + wrap, then k_map's mapping
//   k_step     forces of Eq. 1 (Sec. "Force interpolation") + bonded (never interpolated)
//              + thermodynamic force (Sec. "Free energy corrections and the thermodynamic
//              force") and, by MODE:
//                MODE_FORCES   store the conservative force
//                MODE_LAST     + Langevin force, second half kick, store v and f
//                MODE_FUSED    + Langevin force, second half kick of this step, first half
//                              kick and drift of the next, wrap, and the next mapping
//                              (written to the other half of the double-buffered
//                              molecule arrays), so a step is one kernel.
//
// GB300 has 1.2 TFLOP/s of FP64 against ~70 TFLOP/s of FP32, so the FP32 mixed path keeps
// its FP64 work to the state update itself (kick and drift FMAs on double x and v):
// conversions, periodic wraps and the centre-of-mass mapping run on the integer pipes
// using the bit patterns of the doubles, and every pair force is FP32.  Positions enter
// the pair kernel as exact 32-bit fixed-point centres (so minimum-image differences are
// plain integer subtractions) plus float offsets.
#pragma once
#include <math.h>

#include "internal.cuh"

namespace adress {

constexpr int MODE_FORCES = 0;
constexpr int MODE_LAST = 1;
constexpr int MODE_FUSED = 2;

// ---------------- bit-level conversions (integer pipes) -------------------------------

// Exact float -> double for finite floats (float denormals become signed zeros).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned long long sg = (unsigned long long)(b >> 31) << 63;
  const unsigned long long m = (unsigned long long)(b & 0x7fffffu) << 29;
  const unsigned long long d = e ? (sg | ((unsigned long long)(e + 896u) << 52) | m) : sg;
  return __longlong_as_double((long long)d);
}

// double -> float rounding half away from zero (ties only differ from round-to-nearest-even).
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned sg = (unsigned)(bits >> 63) << 31;
  const unsigned long long a = (bits & 0x7fffffffffffffffull) + 0x10000000ull;
  const int e = (int)(a >> 52) - 896;
  if (e <= 0) return __uint_as_float(sg);
  if (e >= 255) return __uint_as_float(sg | 0x7f800000u);
  return __uint_as_float(sg | ((unsigned)e << 23) | (unsigned)((a >> 29) & 0x7fffffu));
}

// Rare path of the periodic wrap, kept out of line so the common path has no FP64 add.
static __device__ __noinline__ double wrap_slow(double y, double L) {
  if (y < 0.0) y += L;
  if (y >= L) y -= L;
  return y;
}

// y wrapped into [0, L): compare the bit patterns (non-negative doubles order like their bits).
__device__ __forceinline__ double wrap_bits(double y, double L, long long Lbits) {
  const long long bits = __double_as_longlong(y);
  if (bits < 0 || bits >= Lbits) y = wrap_slow(y, L);
  return y;
}

// Parameters as the pair loop's real type (float copies precomputed on the host).
template <class T>
__device__ __forceinline__ T par(double d, float f);
template <>
__device__ __forceinline__ double par<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float par<float>(double, float f) { return f; }

// floor(x 2^32 / L) for 0 <= x < L from the bits of x: the 53-bit significand times
// K = floor(2^q / L) (exact 128-bit product, high word kept), shifted by the exponent.
__device__ __forceinline__ unsigned fixed32(double x, unsigned long long K, int q) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = q - 44 - (e - 1023);
  const unsigned long long hi = __umul64hi(M, K);
  return (e == 0 || sh >= 64 || sh < 0) ? 0u : (unsigned)(hi >> sh);
}

// ---------------- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------------------
__device__ __forceinline__ void philox4x32_10(unsigned c[4], unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const unsigned lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// ---------------- precision policies for the pair loop --------------------------------

template <class P>
struct Prec;

template <>
struct Prec<P64> {
  using real = double;
  struct V3 {
    double x, y, z;
  };
  static __device__ __forceinline__ double4_32a com(const Bufs& b, int cur, int a) { return b.com64[cur][a]; }
  static __device__ __forceinline__ double w(const double4_32a& c) { return c.w; }
  static __device__ __forceinline__ V3 dR(const Box& X, const double4_32a& A, const double4_32a& B) {
    return {minimg_cmp(A.x - B.x, X.L[0], X.halfL[0]), minimg_cmp(A.y - B.y, X.L[1], X.halfL[1]),
            minimg_cmp(A.z - B.z, X.L[2], X.halfL[2])};
  }
  static __device__ __forceinline__ double4_32a off(const Bufs& b, int cur, int i) { return b.off64[cur][i]; }
  static __device__ __forceinline__ double cg(const Bufs& b, int cg_n, double r, double inv_dr, double* V) {
    const double u = r * inv_dr;
    int k = (int)u;
    if (k > cg_n - 1) k = cg_n - 1;
    const double t = u - k;
    *V = b.cgV64[k] * (1.0 - t) + b.cgV64[k + 1] * t;
    return b.cgF64[k] * (1.0 - t) + b.cgF64[k + 1] * t;
  }
  static __device__ __forceinline__ double tf(const Bufs& b, int k) { return b.tf64[k]; }
  static __device__ __forceinline__ double fec(const Bufs& b, int k) { return b.fec64[k]; }
  static __device__ __forceinline__ double sin_(double x) { return sin(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
  static __device__ __forceinline__ double acos_(double x) { return acos(x); }
  static __device__ __forceinline__ double div_(double a, double x) { return a / x; }
};

template <>
struct Prec<P32> {
  using real = float;
  struct V3 {
    float x, y, z;
  };
  static __device__ __forceinline__ int4 com(const Bufs& b, int cur, int a) { return b.com_fx[cur][a]; }
  static __device__ __forceinline__ float w(const int4& c) { return __int_as_float(c.w); }
  // exact integer difference of fixed-point centres (periodic wrap for free), then float
  static __device__ __forceinline__ V3 dR(const Box& X, const int4& A, const int4& B) {
    return {(float)(int)((unsigned)A.x - (unsigned)B.x) * X.fx_scale[0],
            (float)(int)((unsigned)A.y - (unsigned)B.y) * X.fx_scale[1],
            (float)(int)((unsigned)A.z - (unsigned)B.z) * X.fx_scale[2]};
  }
  static __device__ __forceinline__ float4 off(const Bufs& b, int cur, int i) { return b.off32[cur][i]; }
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
  static __device__ __forceinline__ float fec(const Bufs& b, int k) { return b.fec32[k]; }
  static __device__ __forceinline__ float sin_(float x) { return sinf(x); }
  // hardware approximations (a few ulp): the FP32 path's error budget is 2e-5 relative
  static __device__ __forceinline__ float sqrt_(float x) { return x * rsqrtf(x); }
  static __device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float acos_(float x) { return acosf(x); }
  static __device__ __forceinline__ float div_(float a, float x) { return __fdividef(a, x); }
};

// ---------------- mapping of a molecule (group of four lanes) --------------------------

__device__ __forceinline__ double shfl_d(unsigned mask, double v, int src) {
  return __hiloint2double(__shfl_sync(mask, __double2hiint(v), src), __shfl_sync(mask, __double2loint(v), src));
}
__device__ __forceinline__ double shfl_xor_d(unsigned mask, double v, int o) {
  return __hiloint2double(__shfl_xor_sync(mask, __double2hiint(v), o), __shfl_xor_sync(mask, __double2loint(v), o));
}

// Centre of mass in double exactly as R = sum_k m_k (x_0 + minimg(x_k - x_0)) / M, then
// wrapped; all lanes of the group get the x component.  Used where a decision must be
// taken in FP64 (region boundaries).
template <int NA>
__device__ __forceinline__ double com_x_fp64(const Sys& s, const Box& B, unsigned gmask, int base, int g, double xk) {
  const double x0 = shfl_d(gmask, xk, base);
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    const double xkk = shfl_d(gmask, xk, base + k);
    acc += s.mass[k] * (x0 + minimg_cmp(xkk - x0, B.L[0], B.halfL[0]));
  }
  double r = acc / s.Mtot;
  r -= B.L[0] * floor(r / B.L[0]);
  if (r >= B.L[0]) r -= B.L[0];
  return r;
}

// Nearest resolution centre of a molecule (self-adjusting geometry): the group's four lanes
// take every fourth centre, then reduce (distance, index) so that the first of equal
// distances wins, as the definition states.  FP32: from the fixed-point centres.
__device__ __forceinline__ float nearest_center32(const Sys& s, const Box& B, const Bufs& b, unsigned gmask, int g,
                                                  const unsigned R[3], int& kmin) {
  float best = INFINITY;
  int kb = 0x7fffffff;
  for (int k = g; k < s.n_centers; k += 4) {
    const int4 C = b.cen32[k];
    const float r = sqrtf(pair_r2((float)(int)(R[0] - (unsigned)C.x) * B.fx_scale[0],
                                  (float)(int)(R[1] - (unsigned)C.y) * B.fx_scale[1],
                                  (float)(int)(R[2] - (unsigned)C.z) * B.fx_scale[2]));
    if (r < best) {
      best = r;
      kb = k;
    }
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    const float ob = __shfl_xor_sync(gmask, best, o);
    const int ok = __shfl_xor_sync(gmask, kb, o);
    if (ob < best || (ob == best && ok < kb)) {
      best = ob;
      kb = ok;
    }
  }
  kmin = kb;
  return best;
}

// FP64: from a double centre of mass, the sum of squares in the definition's order.
__device__ __forceinline__ double nearest_center64(const Sys& s, const Box& B, const Bufs& b, unsigned gmask, int g,
                                                   const double R[3], int& kmin) {
  double best = INFINITY;
  int kb = 0x7fffffff;
  for (int k = g; k < s.n_centers; k += 4) {
    const double4_32a C = b.cen64[k];
    const double t0 = minimg_cmp(R[0] - C.x, B.L[0], B.halfL[0]);
    const double t1 = minimg_cmp(R[1] - C.y, B.L[1], B.halfL[1]);
    const double t2 = minimg_cmp(R[2] - C.z, B.L[2], B.halfL[2]);
    const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(t0, t0), __dmul_rn(t1, t1)), __dmul_rn(t2, t2)));
    if (r < best) {
      best = r;
      kb = k;
    }
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    const double ob = shfl_xor_d(gmask, best, o);
    const int ok = __shfl_xor_sync(gmask, kb, o);
    if (ob < best || (ob == best && ok < kb)) {
      best = ob;
      kb = ok;
    }
  }
  kmin = kb;
  return best;
}

// Centre of mass in double exactly as the definition forms it (all lanes of the group get it).
template <int NA>
__device__ __forceinline__ void com_fp64(const Sys& s, const Box& B, unsigned gmask, int base, const double x[3],
                                         double R[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double x0 = shfl_d(gmask, x[d], base);
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const double xkk = shfl_d(gmask, x[d], base + k);
      acc += s.mass[k] * (x0 + minimg_cmp(xkk - x0, B.L[d], B.halfL[d]));
    }
    double r = acc / s.Mtot;
    r -= B.L[d] * floor(r / B.L[d]);
    if (r >= B.L[d]) r -= B.L[d];
    R[d] = r;
  }
}

// Map one molecule: fixed-point centre, resolution value, offsets, region flag.
// P32: integer fixed-point arithmetic (exact, periodic) on the bits of the doubles.
template <int NA>
__device__ __forceinline__ void map_group32(const Sys& s, const Box& B, const Bufs& b, int nxt, int a, int g, unsigned gmask,
                                            int base, bool live, const double x[3], const int4 ref, float& ext2,
                                            float& disp2) {
  const bool own = live && g < NA;
  unsigned Pk[3], P0[3], R[3];
  int o32[3];
  float cs[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Pk[d] = fixed32(x[d], B.fxK[d], B.fxq[d]);
    P0[d] = __shfl_sync(gmask, Pk[d], base);
    const int dl = own ? (int)(Pk[d] - P0[d]) : 0;
    o32[d] = dl;
    cs[d] = s.f.frac[g < NA ? g : 0] * (float)dl;
    if (!own) cs[d] = 0.f;
    cs[d] += __shfl_xor_sync(gmask, cs[d], 1);
    cs[d] += __shfl_xor_sync(gmask, cs[d], 2);
    const int c32 = __float2int_rn(cs[d]);
    o32[d] -= c32;
    R[d] = P0[d] + (unsigned)c32;
  }
  float4 o = make_float4((float)o32[0] * B.fx_scale[0], (float)o32[1] * B.fx_scale[1],
                         (float)o32[2] * B.fx_scale[2], 0.f);
  if (own) {
    b.off32[nxt][a * NA + g] = o;
    ext2 = fmaxf(ext2, o.x * o.x + o.y * o.y + o.z * o.z);
  }
  // signed x distance to the slab centre (spheres: distance to the nearest centre); region
  // decided in FP64 near a boundary
  int kmin = 0;
  const float dxc = s.n_centers > 0 ? nearest_center32(s, B, b, gmask, g, R, kmin)
                                    : (float)(int)(R[0] - B.xc32) * B.fx_scale[0];
  float dd = fabsf(dxc);
  const bool near = fabsf(dd - B.d_at_f) < B.near_at || fabsf(dd - B.d_hyend_f) < B.near_hyend;
  int region;  // 0 AT, 1 hybrid, 2 CG
  if (__any_sync(gmask, live && near)) {
    double dxd;
    if (s.n_centers > 0) {
      double R64[3];
      com_fp64<NA>(s, B, gmask, base, x, R64);
      int k64;
      dxd = nearest_center64(s, B, b, gmask, g, R64, k64);
    } else {
      const double rx = com_x_fp64<NA>(s, B, gmask, base, g, x[0]);
      dxd = fabs(minimg_cmp(rx - B.xc, B.L[0], B.halfL[0]));
    }
    region = dxd < B.d_at ? 0 : (dxd >= B.d_at + B.d_hy ? 2 : 1);
  } else {
    region = dd < B.d_at_f ? 0 : (dd >= B.d_hyend_f ? 2 : 1);
  }
  if (live && g == 0) {
    float w = region == 0 ? 1.f : 0.f;
    if (region == 1) {
      const float c = cosf((dd - B.d_at_f) * B.pi_half_over_dhy_f);
      w = c * c;
    }
    if (s.lam_uniform_on) {
      w = s.f.lam_uniform;
      region = 0;  // no hybrid-layer forces
    }
    b.com_fx[nxt][a] = make_int4((int)R[0], (int)R[1], (int)R[2], __float_as_int(w));
    b.molf[nxt][a] = make_float2(dxc, region == 1 ? 1.f : 0.f);
    if (s.n_centers > 0) b.kcen[nxt][a] = kmin;
    const float d0 = (float)(int)(R[0] - (unsigned)ref.x) * B.fx_scale[0];
    const float d1 = (float)(int)(R[1] - (unsigned)ref.y) * B.fx_scale[1];
    const float d2 = (float)(int)(R[2] - (unsigned)ref.z) * B.fx_scale[2];
    disp2 = d0 * d0 + d1 * d1 + d2 * d2;
  }
}

// P64: the plain double-precision mapping (the FP64 reference path).
template <int NA>
__device__ __forceinline__ void map_group64(const Sys& s, const Box& B, const Bufs& b, int nxt, int a, int g, unsigned gmask,
                                            int base, bool live, const double x[3], const int4 ref, float& ext2,
                                            float& disp2) {
  const bool own = live && g < NA;
  double dl[3], c[3], R[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double x0 = shfl_d(gmask, x[d], base);
    dl[d] = own ? minimg_cmp(x[d] - x0, B.L[d], B.halfL[d]) : 0.0;
    double cs = own ? s.frac[g] * dl[d] : 0.0;
    cs += shfl_xor_d(gmask, cs, 1);
    cs += shfl_xor_d(gmask, cs, 2);
    c[d] = cs;
    double r = x0 + cs;
    if (r < 0.0) r += B.L[d];
    if (r >= B.L[d]) r -= B.L[d];
    R[d] = r;
  }
  if (own) {
    const double o0 = dl[0] - c[0], o1 = dl[1] - c[1], o2 = dl[2] - c[2];
    b.off64[nxt][a * NA + g] = make_double4_32a(o0, o1, o2, 0.0);
    ext2 = fmaxf(ext2, (float)(o0 * o0 + o1 * o1 + o2 * o2));
  }
  int kmin = 0;
  const double dxc = s.n_centers > 0 ? nearest_center64(s, B, b, gmask, g, R, kmin)
                                     : minimg_cmp(R[0] - B.xc, B.L[0], B.halfL[0]);
  if (live && g == 0) {
    const double dd = fabs(dxc);
    double w;
    if (dd < B.d_at) w = 1.0;
    else if (dd >= B.d_at + B.d_hy) w = 0.0;
    else {
      const double cs = cos((dd - B.d_at) * B.pi_half_over_dhy);
      w = cs * cs;
    }
    if (s.lam_uniform_on) w = s.lam_uniform;
    b.com64[nxt][a] = make_double4_32a(R[0], R[1], R[2], w);
    b.dxc64[nxt][a] = dxc;
    if (s.n_centers > 0) b.kcen[nxt][a] = kmin;
    unsigned X[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = (unsigned)(unsigned long long)llrint(R[d] * B.fx_inv[d]);
    b.com_fx[nxt][a] = make_int4((int)X[0], (int)X[1], (int)X[2], __float_as_int((float)w));
    const float d0 = (float)(int)(X[0] - (unsigned)ref.x) * B.fx_scale[0];
    const float d1 = (float)(int)(X[1] - (unsigned)ref.y) * B.fx_scale[1];
    const float d2 = (float)(int)(X[2] - (unsigned)ref.z) * B.fx_scale[2];
    disp2 = d0 * d0 + d1 * d1 + d2 * d2;
  }
}

// Block maximum of the molecule extent and of the displacement since the last list
// build, merged into the control block with one fire-and-forget atomic per block (no
// fence, no returned value, so blocks retire at once) into slot blockIdx mod kExtSlots:
// spread over 32 slots the blocks' atomics rarely meet at one address (one address for
// all blocks cost ~2 us of the fused step at 800k atoms); the decide kernel folds them.
__device__ __forceinline__ void publish_extent(const Bufs& b, float ext2, float disp2) {
  __shared__ unsigned red[2][kMaxForceBlock / 32];
  const unsigned e = __reduce_max_sync(0xffffffffu, __float_as_uint(ext2));
  const unsigned dm = __reduce_max_sync(0xffffffffu, __float_as_uint(disp2));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = e;
    red[1][w] = dm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned me = red[0][0], md = red[1][0];
#pragma unroll
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      me = max(me, red[0][k]);
      md = max(md, red[1][k]);
    }
    atomicMax(&b.ctrl->ext_slot[0][blockIdx.x & (kExtSlots - 1)], me);
    atomicMax(&b.ctrl->ext_slot[1][blockIdx.x & (kExtSlots - 1)], md);
  }
}

// ---------------- k_map / k_prologue ---------------------------------------------------

// The decide kernel that follows a mapping kernel may be scheduled once every block of the
// mapping has started (it waits for the mapping grid's completion itself).
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;"); }

template <class P, int NA, bool INTEGRATE, bool MULTI>
__global__ void __launch_bounds__(kMaxForceBlock) k_prologue(const __grid_constant__ Sys s, Bufs b) {
  allow_dependent_launch();
  const int lane = threadIdx.x & 31, g = threadIdx.x & 3, base = lane & ~3;
  const unsigned gmask = 0xFu << base;
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const bool live = a < s.M;
  const int i = (live ? a : 0) * NA + (g < NA ? g : 0);
  const int nxt = b.ctrl->parity ^ 1;
  const Box& B = box_t<MULTI>(s, b, live ? a : 0);
  const size_t N = (size_t)s.N;
  const int4 ref = live && g == 0 ? b.com_ref[a] : make_int4(0, 0, 0, 0);  // centre at the last build
  double x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    x[d] = b.x[d * N + i];
    if (INTEGRATE && live && g < NA) {
      const double fv = P::fp64 ? ((const double*)b.f)[d * N + i] : f2d_bits(((const float*)b.f)[d * N + i]);
      const double v = fma(s.hdt_m[g], fv, b.v[d * N + i]);
      x[d] = P::fp64 ? [&] {
        double y = fma(s.dt, v, x[d]);
        if (y < 0.0) y += B.L[d];
        if (y >= B.L[d]) y -= B.L[d];
        return y;
      }()
                     : wrap_bits(fma(s.dt, v, x[d]), B.L[d], B.Lbits[d]);
      b.v[d * N + i] = v;
      b.x[d * N + i] = x[d];
    }
  }
  float ext2 = 0.f, disp2 = 0.f;
  if (P::fp64) map_group64<NA>(s, B, b, nxt, a, g, gmask, base, live, x, ref, ext2, disp2);
  else map_group32<NA>(s, B, b, nxt, a, g, gmask, base, live, x, ref, ext2, disp2);
  publish_extent(b, ext2, disp2);
}

// ---------------- k_step ----------------------------------------------------------------

// MODEL 0: WCA between atoms of different molecules (the tetrahedral fluid);
// MODEL 1: Lennard-Jones + reaction-field Coulomb per site pair (the water-like fluid).
// Resident blocks per SM the FP32 kernels are compiled for (48 registers for the single-box
// WCA model: more warps to hide the neighbour-load latency, measured 3% faster than the
// unbounded 55; the batched and water variants keep 64).
template <class P, int MODEL, bool MULTI>
constexpr int step_min_blocks() {
  return P::fp64 ? 1 : (MODEL == 0 && !MULTI ? 10 : 8);
}

template <class P, int NA, int MODE, bool ENERGY, bool MULTI, int MODEL, bool HS>
__global__ void __launch_bounds__(kMaxForceBlock, step_min_blocks<P, MODEL, MULTI>()) k_step(const __grid_constant__ Sys s, Bufs b) {
  using Q = Prec<P>;
  using real = typename Q::real;
  if (MODE == MODE_FUSED) allow_dependent_launch();
  const int lane = threadIdx.x & 31, g = threadIdx.x & 3, base = lane & ~3;
  const unsigned gmask = 0xFu << base;
  // SPLIT > 1 (water): a high-resolution item takes SPLIT groups of four lanes in the same
  // warp, group `sub` every SPLIT-th neighbour from slot `sub`; CG items keep one group.
  constexpr int SPLIT = MODEL == 1 ? kSplitWater : 1;
  static_assert(SPLIT == 1 || SPLIT == 2 || SPLIT == 4, "lane groups per item");
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  int t = gtid >> 2, sub = 0;
  if (SPLIT > 1) {
    const int n_hr0 = b.ctrl->n_hr;
    if (gtid < kGroup * SPLIT * n_hr0) {
      t = gtid / (kGroup * SPLIT);
      sub = (gtid >> 2) & (SPLIT - 1);
    } else {
      t = n_hr0 + ((gtid - kGroup * SPLIT * n_hr0) >> 2);
    }
  }
  const bool live_item = t < s.M;
  const bool live = live_item && sub == 0;  // the group that integrates and maps the molecule
  const bool own = live && g < NA;
  const bool own_pair = live_item && g < NA;  // lanes that evaluate pair forces
  const int cur = b.ctrl->parity;
  // the first list slot this lane reads is fetched together with the item, before the count
  // is known (slots below the capacity lie inside the list array; the value is used only
  // when the count covers the slot)
  const bool hr_item = t < b.ctrl->n_hr;
  const int j0 = hr_item ? sub : g;
  const int m_first = live_item && j0 < s.cap ? b.nbr[(size_t)t * s.cap + j0] : 0;

  const real eps = par<real>(s.eps, s.f.eps), sig2 = par<real>(s.sig2, s.f.sig2);
  const real rc_at2 = par<real>(s.rc_at2, s.f.rc_at2), rc_cg2 = par<real>(s.rc_cg2, s.f.rc_cg2);
  const real inv_dr = par<real>(s.cg_inv_dr, s.f.cg_inv_dr);
  const real reach = par<real>(s.rc_at, s.f.rc_at) + (real)2 * (real)b.ctrl->ext_now;
  const real reach_at2 = reach * reach;
  const int gg0 = g < NA ? g : 0;
  const real frac_g = par<real>(s.frac[gg0], s.f.frac[gg0]);
  // MODEL 1: this atom's row of the site-pair coefficients
  real c12r[NA], c6r[NA], qqr[NA];
  real krf2 = 0;
  if (MODEL == 1) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      c12r[j] = par<real>(s.c12[gg0][j], s.f.c12[gg0][j]);
      c6r[j] = par<real>(s.c6[gg0][j], s.f.c6[gg0][j]);
      qqr[j] = par<real>(s.qq[gg0][j], s.f.qq[gg0][j]);
    }
    krf2 = par<real>(2.0 * s.krf, s.f.krf2);
  }

  real fx = 0, fy = 0, fz = 0;
  double e_at = 0.0, e_cg = 0.0, e_b = 0.0, vir = 0.0;

  const int a = live_item ? b.items[t] : 0;
  const Box& B = box_t<MULTI>(s, b, a);
  // centre at the last list build, for the displacement the next mapping reports: fetched
  // now so that its latency hides behind the force loops
  const int4 ref = MODE == MODE_FUSED && live && g == 0 ? b.com_ref[a] : make_int4(0, 0, 0, 0);
  const int i = a * NA + (g < NA ? g : 0);
  const auto Ca = Q::com(b, cur, a);
  const real wa = Q::w(Ca);
  const auto oi = Q::off(b, cur, i);
  const int nnb = live_item ? b.nn[t] : 0;
  // energy interpolation: a hybrid molecule sums its unweighted pair energies (AT per atom
  // lane, CG on lane 0 of its group) for the drift force
  constexpr bool hs = HS;
  const bool drift = hs && wa > (real)0 && wa < (real)1 && !s.lam_uniform_on;
  real dv = 0;
  // slow-force weight at this time level (1 without multiple time stepping)
  real sw = 1;
  if (s.respa_n > 1) sw = b.ctrl->step % s.respa_n == 0 ? (real)s.respa_n : (real)0;
  const bool slow = sw != (real)0 || ENERGY;

  if (hr_item) {
    // high-resolution item: Eq. 1 for atom i against every listed neighbour (of this lane
    // group's share); the next neighbour's index and centre are fetched while the current
    // one is evaluated
    int m_n = 0;
    auto C_n = Ca;
    if (sub < nnb) {
      m_n = m_first;
      C_n = Q::com(b, cur, m_n);
    }
    for (int q = sub; q < nnb; q += SPLIT) {
      const int m = m_n;
      const auto Cb = C_n;
      if (q + SPLIT < nnb) {
        m_n = b.nbr[(size_t)t * s.cap + q + SPLIT];
        C_n = Q::com(b, cur, m_n);
      }
      const auto R = Q::dR(B, Ca, Cb);
      const real r2 = pair_r2(R.x, R.y, R.z);
      const real wab = hs ? (real)0.5 * (wa + Q::w(Cb)) : wa * Q::w(Cb);
      if (own_pair && wab > (real)0 && r2 < reach_at2) {
        const real px = R.x + (real)oi.x, py = R.y + (real)oi.y, pz = R.z + (real)oi.z;
        typename P::off_t oj[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) oj[j] = Q::off(b, cur, m * NA + j);
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          const real dx = px - (real)oj[j].x, dy = py - (real)oj[j].y, dz = pz - (real)oj[j].z;
          const real d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < rc_at2) {
            real fr;
            if (MODEL == 0) {
              const real ir2 = Q::rcp_(d2);
              const real sr2 = sig2 * ir2;
              const real sr6 = sr2 * sr2 * sr2;
              fr = (real)24 * eps * ((real)2 * sr6 * sr6 - sr6) * ir2 * wab;
              if (ENERGY) e_at += 0.5 * (double)wab * (double)((real)4 * eps * (sr6 * sr6 - sr6) + eps);
              if (drift) dv += (real)4 * eps * (sr6 * sr6 - sr6) + eps;
            } else {
              // LJ (c12 r^-12 - c6 r^-6, shifted) + reaction field q_i q_j f (1/r + k_rf r^2 - c_rf);
              // the LJ term only for partner sites that have one with some site (water: O)
              const real ir = Q::rsqrt_(d2);
              const real ir2 = ir * ir;
              real flj = 0, vlj = 0;
              if ((s.lj_cols >> j) & 1) {
                const real ir6 = ir2 * ir2 * ir2;
                flj = ((real)12 * c12r[j] * ir6 - (real)6 * c6r[j]) * ir6 * ir2;
                if (ENERGY || drift) vlj = (c12r[j] * ir6 - c6r[j]) * ir6;
              }
              fr = (flj + qqr[j] * (ir2 * ir - krf2)) * wab;
              if (ENERGY)
                e_at += 0.5 * (double)wab *
                        ((double)vlj + s.vsh[gg0][j] + (double)qqr[j] * ((double)ir + s.krf * (double)d2 - s.crf));
              if (drift)
                dv += vlj + par<real>(s.vsh[gg0][j], s.f.vsh[gg0][j]) +
                      qqr[j] * (ir + par<real>(s.krf, s.f.krf) * d2 - par<real>(s.crf, s.f.crf));
            }
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
            if (ENERGY) vir += 0.5 * (double)(fr * d2);
          }
        }
      }
      if (own_pair && wab < (real)1 && r2 < rc_cg2 && slow) {
        const real r = Q::sqrt_(r2);
        real V = 0;
        const real F = s.cg_mode ? (real)b.fpair[(size_t)t * s.cap + q] : Q::cg(b, s.cg_n, r, inv_dr, &V);
        const real fw = ((real)1 - wab) * F;
        const real c = Q::div_(fw * sw, r);
        fx += frac_g * c * R.x;
        fy += frac_g * c * R.y;
        fz += frac_g * c * R.z;
        if (ENERGY && g == 0) {
          e_cg += 0.5 * (double)(((real)1 - wab) * V);
          vir += 0.5 * (double)(Q::div_(fw, r) * r2);
        }
        if (drift && g == 0) dv -= sw * V;
      }
    }
    if (SPLIT > 1) {  // the groups' shares of the force (energies are summed per warp)
      const unsigned mk = SPLIT == 2 ? 0xFFu << (lane & 24) : 0xFFFFu << (lane & 16);
#pragma unroll
      for (int o = kGroup; o < kGroup * SPLIT; o <<= 1) {
        fx += __shfl_xor_sync(mk, fx, o);
        fy += __shfl_xor_sync(mk, fy, o);
        fz += __shfl_xor_sync(mk, fz, o);
        if (hs) dv += __shfl_xor_sync(mk, dv, o);
      }
    }
    if (hs) {  // V_AT_a - V_CG_a = half the group's sum (every pair is listed from both sides)
      dv += __shfl_xor_sync(gmask, dv, 1);
      dv += __shfl_xor_sync(gmask, dv, 2);
      dv *= (real)0.5;
    }
  } else {
    // coarse-grained item (l_a = 0, so w_ab = 0): neighbour list split over the group
    if (live && g == 0 && wa != (real)0) set_error(b.ctrl, ADRESS_ERR_STATE, a);
    real Fx = 0, Fy = 0, Fz = 0;
    auto C_n = Ca;
    const int nnb_cg = slow ? nnb : 0;  // no CG force at inner levels of multiple time stepping
    // centres of the next two neighbours in flight (long lists: the water-like fluid)
    if (g < nnb_cg) C_n = Q::com(b, cur, m_first);
    auto C_n2 = Ca;
    if (g + kGroup < nnb_cg) C_n2 = Q::com(b, cur, b.nbr[(size_t)t * s.cap + g + kGroup]);
    for (int q = g; q < nnb_cg; q += kGroup) {
      const auto Cb = C_n;
      C_n = C_n2;
      if (q + 2 * kGroup < nnb_cg) C_n2 = Q::com(b, cur, b.nbr[(size_t)t * s.cap + q + 2 * kGroup]);
      const auto R = Q::dR(B, Ca, Cb);
      const real r2 = pair_r2(R.x, R.y, R.z);
      if (r2 < rc_cg2) {
        const real r = Q::sqrt_(r2);
        real V = 0;
        const real F = s.cg_mode ? (real)b.fpair[(size_t)t * s.cap + q] : Q::cg(b, s.cg_n, r, inv_dr, &V);
        const real c = Q::div_(F, r);
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
    const real fs = frac_g * sw;
    fx = fs * Fx;
    fy = fs * Fy;
    fz = fs * Fz;
  }

  // own state for the update, fetched before the bonded terms so the loads overlap them
  const size_t N = (size_t)s.N;
  double xo[3] = {0.0, 0.0, 0.0}, vo[3] = {0.0, 0.0, 0.0};
  if (MODE != MODE_FORCES && own) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      vo[d] = b.v[d * N + i];
      if (MODE == MODE_FUSED) xo[d] = b.x[d * N + i];
    }
  }

  if (own) {
    // bonded terms of atom g: harmonic bonds and angles, or FENE + WCA, on the listed
    // intramolecular pairs
    const real R02 = par<real>(s.fene_r02, s.f.fene_r02), K = par<real>(s.fene_k, s.f.fene_k);
    // each lane walks its own atom's bonds (bond order), so a warp runs as many bond bodies
    // as an atom has bonds, not as the molecule has
    const unsigned bw = s.bond_word[gg0];
    if (s.bond_model == 1) {
      const real kb = par<real>(s.bond_k, s.f.bond_k), r0 = par<real>(s.bond_r0, s.f.bond_r0);
#pragma unroll
      for (int q = 0; q < kMaxBonds; ++q) {
        if (q >= s.bmax) break;
        if (q >= (int)(bw >> 28)) continue;
        const int e = (bw >> (4 * q)) & 15;
        const auto oo = Q::off(b, cur, a * NA + (e & 7));
        const real dx = (real)oi.x - (real)oo.x, dy = (real)oi.y - (real)oo.y, dz = (real)oi.z - (real)oo.z;
        const real d2 = dx * dx + dy * dy + dz * dz;
        const real ird = Q::rsqrt_(d2);
        const real dl = d2 * ird;
        const real fr = -kb * (dl - r0) * ird;  // V = k/2 (r - r0)^2
        fx += fr * dx;
        fy += fr * dy;
        fz += fr * dz;
        if (ENERGY && (e & 8)) {
          e_b += 0.5 * (double)kb * (double)(dl - r0) * (double)(dl - r0);
          vir += (double)(fr * d2);
        }
      }
      // harmonic angles (i, vertex j, k): V = k/2 (theta - theta0)^2; the force on i is
      // dV/dtheta (v/(|u||v|) - cos(theta) u/|u|^2) / sin(theta), u = x_i - x_j, v = x_k - x_j,
      // likewise on k, and minus their sum on the vertex
      const real ka = par<real>(s.angle_k, s.f.angle_k), th0 = par<real>(s.angle_theta0, s.f.angle_theta0);
#pragma unroll
      for (int q = 0; q < kMaxAngles; ++q) {
        if (q >= s.n_angles) break;
        const int ai = s.angles[3 * q], aj = s.angles[3 * q + 1], ak = s.angles[3 * q + 2];
        if (g != ai && g != aj && g != ak) continue;
        const auto Oi = Q::off(b, cur, a * NA + ai), Oj = Q::off(b, cur, a * NA + aj), Ok = Q::off(b, cur, a * NA + ak);
        const real ux = (real)Oi.x - (real)Oj.x, uy = (real)Oi.y - (real)Oj.y, uz = (real)Oi.z - (real)Oj.z;
        const real vx = (real)Ok.x - (real)Oj.x, vy = (real)Ok.y - (real)Oj.y, vz = (real)Ok.z - (real)Oj.z;
        const real uu = ux * ux + uy * uy + uz * uz, vv = vx * vx + vy * vy + vz * vz;
        const real uv = ux * vx + uy * vy + uz * vz;
        const real iuv = Q::rsqrt_(uu * vv);
        real c = uv * iuv;
        c = c > (real)1 ? (real)1 : (c < (real)-1 ? (real)-1 : c);
        const real th = Q::acos_(c);
        const real s2 = (real)1 - c * c;
        const real gq = s2 > (real)0 ? ka * (th - th0) * Q::rsqrt_(s2) : (real)0;
        const real iu = Q::rcp_(uu), iv = Q::rcp_(vv);
        const real fix = gq * (vx * iuv - c * ux * iu), fiy = gq * (vy * iuv - c * uy * iu), fiz = gq * (vz * iuv - c * uz * iu);
        const real fkx = gq * (ux * iuv - c * vx * iv), fky = gq * (uy * iuv - c * vy * iv), fkz = gq * (uz * iuv - c * vz * iv);
        if (g == ai) {
          fx += fix;
          fy += fiy;
          fz += fiz;
        } else if (g == ak) {
          fx += fkx;
          fy += fky;
          fz += fkz;
        } else {
          fx -= fix + fkx;
          fy -= fiy + fky;
          fz -= fiz + fkz;
          if (ENERGY) {
            e_b += 0.5 * (double)ka * (double)(th - th0) * (double)(th - th0);
            vir += (double)(ux * fix + uy * fiy + uz * fiz + vx * fkx + vy * fky + vz * fkz);
          }
        }
      }
    } else {
#pragma unroll
    for (int q = 0; q < kMaxBonds; ++q) {
      if (q >= s.bmax) break;
      if (q >= (int)(bw >> 28)) continue;
      const int e = (bw >> (4 * q)) & 15;
      const auto oo = Q::off(b, cur, a * NA + (e & 7));
      const real dx = (real)oi.x - (real)oo.x, dy = (real)oi.y - (real)oo.y, dz = (real)oi.z - (real)oo.z;
      const real d2 = dx * dx + dy * dy + dz * dz;
      if (d2 >= R02) {
        set_error(b.ctrl, ADRESS_ERR_BOND_BROKEN, a);
        continue;
      }
      const real gg = (real)1 - Q::div_(d2, R02);
      real fr = Q::div_(-K, gg);
      double V = 0.0;
      if (ENERGY) V = -0.5 * (double)K * (double)R02 * log((double)gg);
      if (s.intra_wca && d2 < rc_at2) {
        const real ir2 = Q::rcp_(d2);
        const real sr2 = sig2 * ir2;
        const real sr6 = sr2 * sr2 * sr2;
        fr += (real)24 * eps * ((real)2 * sr6 * sr6 - sr6) * ir2;
        if (ENERGY) V += (double)((real)4 * eps * (sr6 * sr6 - sr6) + eps);
      }
      fx += fr * dx;
      fy += fr * dy;
      fz += fr * dz;
      if (ENERGY && (e & 8)) {
        e_b += V;
        vir += (double)(fr * d2);
      }
    }
    }
    // thermodynamic force on hybrid-layer molecules (region decided at mapping time), and
    // energy interpolation's drift force -(V_AT_a - V_CG_a - g(l_a)) l'(d) along grad d
    if (s.tf_n > 0 || hs) {
      real dxc;
      bool hy;
      if (P::fp64) {
        const double dd = b.dxc64[cur][a], ad = fabs(dd);
        dxc = (real)dd;
        hy = ad >= B.d_at && ad < B.d_at + B.d_hy && !s.lam_uniform_on;
      } else {
        const float2 mf = b.molf[cur][a];
        dxc = (real)mf.x;
        hy = mf.y != 0.f;
      }
      if (hy) {
        const real d = dxc < (real)0 ? -dxc : dxc;
        real F = 0;
        if (s.tf_n > 0) {
          const real u = d * par<real>(s.tf_inv_dx, s.f.tf_inv_dx);
          const int k = (int)u;
          if (k + 1 < s.tf_n) {
            const real tt = u - (real)k;
            F = Q::tf(b, B.tf0 + k) * ((real)1 - tt) + Q::tf(b, B.tf0 + k + 1) * tt;
          } else if (k + 1 == s.tf_n && u == (real)k) {
            F = Q::tf(b, B.tf0 + k);
          }
          F *= sw;
        }
        if (hs) {
          real gl = 0;
          if (s.fec_n > 0) {  // free-energy correction dDF/dl at l_a
            const real ul = wa * par<real>(s.fec_scale, s.f.fec_scale);
            const int kl = (int)ul;
            if (kl + 1 < s.fec_n) {
              const real tl = ul - (real)kl;
              gl = Q::fec(b, kl) * ((real)1 - tl) + Q::fec(b, kl + 1) * tl;
            } else {
              gl = Q::fec(b, s.fec_n - 1);
            }
          }
          // l'(d) = -(pi/(2 d_hy)) sin(pi (d - d_at)/d_hy)
          const real c = par<real>(B.pi_half_over_dhy, B.pi_half_over_dhy_f);
          const real sn = Q::sin_((real)2 * c * (d - par<real>(B.d_at, B.d_at_f)));
          F += (dv - sw * gl) * c * sn;
        }
        if (s.n_centers > 0) {
          // along the direction from the nearest centre
          const int kc = b.kcen[cur][a];
          real ux, uy, uz;
          if (P::fp64) {
            const double4_32a C = b.cen64[kc];
            const auto& R64 = Ca;
            ux = (real)minimg_cmp(R64.x - C.x, B.L[0], B.halfL[0]);
            uy = (real)minimg_cmp(R64.y - C.y, B.L[1], B.halfL[1]);
            uz = (real)minimg_cmp(R64.z - C.z, B.L[2], B.halfL[2]);
          } else {
            const int4 C = b.cen32[kc];
            const auto& R32 = Ca;
            ux = (real)((float)(int)((unsigned)R32.x - (unsigned)C.x) * B.fx_scale[0]);
            uy = (real)((float)(int)((unsigned)R32.y - (unsigned)C.y) * B.fx_scale[1]);
            uz = (real)((float)(int)((unsigned)R32.z - (unsigned)C.z) * B.fx_scale[2]);
          }
          const real fd = frac_g * Q::div_(F, d);
          fx += fd * ux;
          fy += fd * uy;
          fz += fd * uz;
        } else {
          fx += frac_g * (dxc < (real)0 ? -F : F);
        }
      }
    }
  }

  if (MODE == MODE_FORCES) {
    if (own) {
      real* fo = (real*)b.f;
      fo[i] = fx;
      fo[N + i] = fy;
      fo[2 * N + i] = fz;
    }
  } else {
    double x[3] = {0.0, 0.0, 0.0};
    if (own) {
      // Langevin force with the half-step velocity, noise keyed by (seed, time level n)
      const long long step = b.ctrl->step;
      const unsigned ia = (unsigned)(i - B.mol0 * NA);  // atom index within its replica
      unsigned c[4] = {ia, (unsigned)step, (unsigned)((unsigned long long)step >> 32), (unsigned)(2 * B.replica)};
      philox4x32_10(c, s.seed_lo, s.seed_hi);
      const double vx = vo[0], vy = vo[1], vz = vo[2];
      if (P::fp64) {
        unsigned lo[4] = {ia, (unsigned)step, (unsigned)((unsigned long long)step >> 32),
                          (unsigned)(2 * B.replica + 1)};
        philox4x32_10(lo, s.seed_lo, s.seed_hi);
        const double k53 = 1.0 / 9007199254740992.0, amp = s.amp[g], gm = s.gm[g];
        const double u0 = (double)(((unsigned long long)c[0] << 21) | (lo[0] >> 11)) * k53;
        const double u1 = (double)(((unsigned long long)c[1] << 21) | (lo[1] >> 11)) * k53;
        const double u2 = (double)(((unsigned long long)c[2] << 21) | (lo[2] >> 11)) * k53;
        fx += -gm * vx + amp * (u0 - 0.5);
        fy += -gm * vy + amp * (u1 - 0.5);
        fz += -gm * vz + amp * (u2 - 0.5);
      } else {
        const float k24 = 1.0f / 16777216.0f, af = s.ampf[g], gm = s.gmf[g];
        fx += -gm * d2f_bits(vx) + af * ((float)(c[0] >> 8) * k24 - 0.5f);
        fy += -gm * d2f_bits(vy) + af * ((float)(c[1] >> 8) * k24 - 0.5f);
        fz += -gm * d2f_bits(vz) + af * ((float)(c[2] >> 8) * k24 - 0.5f);
      }
      if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) set_error(b.ctrl, ADRESS_ERR_NONFINITE, i);
      const double h = s.hdt_m[g];
      const double fdx = P::fp64 ? (double)fx : f2d_bits((float)fx);
      const double fdy = P::fp64 ? (double)fy : f2d_bits((float)fy);
      const double fdz = P::fp64 ? (double)fz : f2d_bits((float)fz);
      if (MODE == MODE_LAST) {
        b.v[i] = fma(h, fdx, vx);
        b.v[N + i] = fma(h, fdy, vy);
        b.v[2 * N + i] = fma(h, fdz, vz);
        real* fo = (real*)b.f;
        fo[i] = fx;
        fo[N + i] = fy;
        fo[2 * N + i] = fz;
      } else {
        // second half kick of this step and first half kick of the next in one FMA,
        // then the drift; the force stays in registers
        const double h2 = s.dt_m[g];
        const double nvx = fma(h2, fdx, vx), nvy = fma(h2, fdy, vy), nvz = fma(h2, fdz, vz);
        double y0 = fma(s.dt, nvx, xo[0]), y1 = fma(s.dt, nvy, xo[1]), y2 = fma(s.dt, nvz, xo[2]);
        if (P::fp64) {
          if (y0 < 0.0) y0 += B.L[0];
          if (y0 >= B.L[0]) y0 -= B.L[0];
          if (y1 < 0.0) y1 += B.L[1];
          if (y1 >= B.L[1]) y1 -= B.L[1];
          if (y2 < 0.0) y2 += B.L[2];
          if (y2 >= B.L[2]) y2 -= B.L[2];
        } else {
          y0 = wrap_bits(y0, B.L[0], B.Lbits[0]);
          y1 = wrap_bits(y1, B.L[1], B.Lbits[1]);
          y2 = wrap_bits(y2, B.L[2], B.Lbits[2]);
        }
        b.v[i] = nvx;
        b.v[N + i] = nvy;
        b.v[2 * N + i] = nvz;
        b.x[i] = y0;
        b.x[N + i] = y1;
        b.x[2 * N + i] = y2;
        x[0] = y0;
        x[1] = y1;
        x[2] = y2;
      }
    }
    if (MODE == MODE_FUSED) {
      // the next step's mapping, into the other buffer half (lanes without an atom take atom 0)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double x0 = P::fp64 ? shfl_d(gmask, x[d], base) : shfl_d(gmask, x[d], base);
        if (!own) x[d] = x0;
      }
      float ext2 = 0.f, disp2 = 0.f;
      const int nxt = cur ^ 1;
      if (P::fp64) map_group64<NA>(s, B, b, nxt, a, g, gmask, base, live, x, ref, ext2, disp2);
      else map_group32<NA>(s, B, b, nxt, a, g, gmask, base, live, x, ref, ext2, disp2);
      publish_extent(b, ext2, disp2);
    }
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

// ---------------- launchers ----------------------------------------------------------

template <class P, int NA, int MODEL, bool HS>
static void launch_step_na(const Sys& s, const Bufs& b, int mode, int energy, cudaStream_t st) {
  const int blocks = ceil_div((long long)s.M * step_lanes(s), s.force_block);
  const bool multi = s.nbox > 1;
  switch (mode) {
    case MODE_FORCES:
      if (multi) {
        if (energy) k_step<P, NA, MODE_FORCES, true, true, MODEL, HS><<<blocks, s.force_block, 0, st>>>(s, b);
        else k_step<P, NA, MODE_FORCES, false, true, MODEL, HS><<<blocks, s.force_block, 0, st>>>(s, b);
      } else {
        if (energy) k_step<P, NA, MODE_FORCES, true, false, MODEL, HS><<<blocks, s.force_block, 0, st>>>(s, b);
        else k_step<P, NA, MODE_FORCES, false, false, MODEL, HS><<<blocks, s.force_block, 0, st>>>(s, b);
      }
      break;
    case MODE_LAST:
      if (multi) k_step<P, NA, MODE_LAST, false, true, MODEL, HS><<<blocks, s.force_block, 0, st>>>(s, b);
      else k_step<P, NA, MODE_LAST, false, false, MODEL, HS><<<blocks, s.force_block, 0, st>>>(s, b);
      break;
    default:
      if (multi) k_step<P, NA, MODE_FUSED, false, true, MODEL, HS><<<blocks, s.force_block, 0, st>>>(s, b);
      else k_step<P, NA, MODE_FUSED, false, false, MODEL, HS><<<blocks, s.force_block, 0, st>>>(s, b);
      break;
  }
}

}  // namespace adress
