// Internal declarations shared by the CUDA translation units of the AdResS library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/adress.h"

namespace adress {

constexpr int kMaxNA = 4;
constexpr int kMaxBonds = 6;
constexpr int kGroup = 4;  // threads per molecule in the force kernel

// Device control block: list-validity trackers, error word, counters.
struct Ctrl {
  unsigned int maxdisp2;  // float bits of the largest squared COM displacement since the last build
  unsigned int maxext;    // float bits of the largest atom-to-COM distance this step
  int rebuild;            // decision for the current step
  int err;                // first device error (adress_status), 0 = none
  int n_hr;               // high-resolution work items (first in `items`)
  int n_cg;
  long long step;         // time level of the state's forces
  int rebuilds;
  float ext_now;
  int max_nn;
  int err_info;
  int pad;
};

// Per-system constants, passed by value to every kernel.
struct Sys {
  int M, NA, N;
  double L[3], halfL[3];
  double fx_inv[3];    // 2^32 / L  (fixed-point COM)
  float fx_scale[3];   // L / 2^32
  float Lf[3];
  double xc, d_at, d_hy, d_hr;  // d_hr: high-resolution candidate bound at list build
  double pi_half_over_dhy;
  double mass[kMaxNA], inv_mass[kMaxNA], frac[kMaxNA], Mtot;
  double eps, sig2, rc_at2;
  int nb;
  int bonds[2 * kMaxBonds];
  double fene_k, fene_r02;
  int intra_wca;
  int cg_n;
  double cg_inv_dr, rc_cg2;
  int tf_n;
  double tf_inv_dx, tf_dx;
  double kT, gamma, dt;
  unsigned long long seed;
  long long replica;
  double skin, r_ext, r_list, r_list2, reach_at2;  // reach_at: rc_at + 2 r_ext
  double rc_at, rc_cg;
  int nc[3];
  int ncell;
  int cap;  // neighbour-list capacity per molecule
};

// Device buffers owned by the handle.
struct Bufs {
  // state (borrowed)
  double* x;
  double* v;
  void* f;
  // per molecule
  int4* com_fx;    // fixed-point COM (uint32 bits) + float bits of w
  int4* com_ref;   // fixed-point COM at the last list build
  double4_32a* com64;  // FP64 COM + w
  double* dxc64;   // signed x distance to the slab centre
  float2* molf;    // (dxc, w) in float
  // per atom
  double4_32a* off64;  // COM-relative atom offsets
  float4* off32;
  // lists
  int* mcell;       // Morton rank of each molecule's cell
  int* cell_count;  // [ncell]
  int* cell_fill;   // [ncell]
  int* cell_start;  // [ncell+1]
  int* sorted;      // molecules grouped by cell, cells in Morton order
  int* flag;        // [M] high-resolution candidate flag at sorted positions
  int* pos;         // [M] exclusive scan of flag
  int* items;       // [M] work items: high-resolution candidates first, then CG
  int* nn;          // [M] neighbour count per item
  int* nbr;         // [cap*M] neighbour molecule of item t in slot s at nbr[s*M + t]
  int* scan_tmp;    // block sums for device-wide scans
  const int* cell_rank;  // linear cell -> Morton rank
  const int* rank_cell;  // Morton rank -> linear cell
  // tables
  const double* cgF64;
  const double* cgV64;
  const float2* cgFV32;
  double* tf64;
  float* tf32;
  // reductions
  double* part;      // per-warp partials
  double* result;    // reduced results [8]
  unsigned long long* hist;  // density histogram [tf_n]
  long long* nsamples;
  Ctrl* ctrl;
};

__device__ __forceinline__ void set_error(Ctrl* c, int code, int info = 0) {
  if (atomicCAS(&c->err, 0, code) == 0) c->err_info = info;
}

// Minimum image for |d| < 1.5 L by comparison (no division).
__device__ __forceinline__ double minimg_cmp(double d, double L, double halfL) {
  if (d > halfL) d -= L;
  else if (d < -halfL) d += L;
  return d;
}

// ---- Philox4x64-10 (Salmon et al., SC'11): published multipliers and Weyl constants ----
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    unsigned long long lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
    unsigned long long lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
    unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// ---- precision policies --------------------------------------------------------------
struct P64 {
  using real = double;
  using off_t = double4_32a;
  using com_t = double4_32a;
  static constexpr bool fp64 = true;
};
struct P32 {
  using real = float;
  using off_t = float4;
  using com_t = int4;
  static constexpr bool fp64 = false;
};

// launchers (one per translation unit)
cudaError_t launch_com(const Sys& s, const Bufs& b, int precision, int integrate, cudaStream_t st);
cudaError_t launch_decide(const Sys& s, const Bufs& b, int force, int advance_step,
                          cudaGraphConditionalHandle h, int use_handle, cudaStream_t st);
cudaError_t launch_rebuild(const Sys& s, const Bufs& b, cudaStream_t st);
cudaError_t launch_forces(const Sys& s, const Bufs& b, int precision, int step_mode, int energy,
                          cudaStream_t st);
cudaError_t launch_energy_reduce(const Sys& s, const Bufs& b, int nparts, int nvals, cudaStream_t st);
cudaError_t launch_kinetic(const Sys& s, const Bufs& b, cudaStream_t st);
cudaError_t launch_density(const Sys& s, const Bufs& b, int precision, cudaStream_t st);
cudaError_t launch_tf_update(const Sys& s, const Bufs& b, double alpha, cudaStream_t st);
cudaError_t launch_export_com(const Sys& s, const Bufs& b, double* com, double* w, cudaStream_t st);

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

constexpr int kForceBlock = 128;
// Warps launched by the force kernel (one energy partial each).
inline int force_warps(const Sys& s) { return ceil_div((long long)s.M * kGroup, kForceBlock) * (kForceBlock / 32); }

}  // namespace adress
