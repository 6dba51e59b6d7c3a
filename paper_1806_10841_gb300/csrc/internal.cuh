// Internal declarations shared by the CUDA translation units of the AdResS library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/adress.h"

namespace adress {

constexpr int kMaxNA = 4;
constexpr int kMaxBonds = 6;
constexpr int kMaxAngles = 4;
constexpr int kMaxCenters = 1024;  // resolution centres of the self-adjusting geometry
constexpr int kGroup = 4;  // threads per molecule in the force kernel
// Default poll limit of a bounded mbarrier wait on tensor-core products: ~tens of ms, far
// beyond a 128x64x64 product.
constexpr unsigned kMmaWaitPolls = 1u << 22;

// Slots the mapping kernels' block maxima are spread over (see publish_extent).
constexpr int kExtSlots = 32;

// Device control block: list-validity trackers, error word, counters.
struct Ctrl {
  int rebuild;            // decision for the current step
  int err;                // first device error (adress_status), 0 = none
  int n_hr;               // high-resolution work items (first in `items`)
  int n_cg;
  long long step;         // time level of the state's forces
  int rebuilds;
  float ext_now;
  int max_nn;
  int err_info;
  int parity;          // which half of the double-buffered molecule arrays is current
  int n_dense;         // cells passed to the dense-cell list builder in this build
  int force_rebuild;   // set by the host (moved resolution centres), cleared by a list build
  // float bits of the last mapping's largest squared atom-to-COM distance [0] and largest
  // squared COM displacement since the last build [1], as block maxima spread over
  // kExtSlots slots (block b uses slot b mod kExtSlots); the decide kernel folds and clears them
  unsigned ext_slot[2][kExtSlots];
  int n_netc;  // candidate pairs of the network CG force from the last list build (Bufs::netc)
};

// Arguments of the rebuild decision taken after a mapping (k_decide in observe.cu): force a
// rebuild, advance the time level, set the graph conditional handle h.
struct DecideArgs {
  int force, advance, use_h;
  cudaGraphConditionalHandle h;
};

// Geometry of one periodic box (one replica): edges, fixed-point maps, slab and cells.
struct Box {
  double L[3], halfL[3];
  long long Lbits[3];           // bit patterns of L (wrap tests on the integer pipe)
  double fx_inv[3];             // 2^32 / L  (fixed-point COM)
  float fx_scale[3];            // L / 2^32
  unsigned long long fxK[3];    // floor(2^fxq / L), in [2^63, 2^64)
  int fxq[3];
  unsigned xc32;                // slab centre in 32-bit fixed point
  double xc, d_at, d_hy, d_hr;  // d_hr: high-resolution candidate bound at list build
  double pi_half_over_dhy;
  float d_at_f, d_hyend_f, pi_half_over_dhy_f, near_at, near_hyend;
  int nc[3];
  int ncell;   // cells of this box
  int cell0;   // first global cell index (and Morton rank) of this box
  int mol0;    // first molecule of this box
  int nmol;    // molecules of this box
  int index;   // position of this box in the batch
  int tf0;     // first entry of this box's thermodynamic-force table and density histogram
  long long replica;  // replica id (thermostat noise counter)
};

// Per-system constants, passed by value to every kernel.
struct Sys {
  int M, NA, N;
  int fp64;  // 1: FP64 path, 0: FP32 mixed path
  int nbox;  // 1: a single box (bx); > 1: batched replicas (Bufs::boxes, Bufs::mol_box)
  Box bx;
  double mass[kMaxNA], inv_mass[kMaxNA], frac[kMaxNA], Mtot;
  double hdt_m[kMaxNA];          // dt / (2 m)
  double amp[kMaxNA], gm[kMaxNA];  // Langevin: sqrt(24 gamma kT m / dt), gamma m
  float ampf[kMaxNA], gmf[kMaxNA];
  double eps, sig2, rc_at2;
  int nb;
  int bonds[2 * kMaxBonds];
  // the same bonds per atom, in bond order, one word per atom: entry q in bits 4q..4q+3 =
  // partner | 8 when the atom is the bond's first atom (which accounts its energy), the
  // count in bits 28..31; bmax the largest count
  unsigned bond_word[kMaxNA];
  int bmax;
  double fene_k, fene_r02;
  int intra_wca;
  int cg_n;
  double cg_inv_dr, rc_cg2;
  int tf_n;
  double tf_inv_dx, tf_dx;
  double kT, gamma, dt;
  unsigned long long seed;
  unsigned seed_lo, seed_hi;
  double skin, r_ext, r_list, r_list2, reach_at2;  // reach_at: rc_at + 2 r_ext
  // (rc_cg + skin)^2: list cutoff of pairs with a coarse-grained work item (weight 0 until
  // the next build, so only the CG force acts); pairs of two high-resolution items use r_list
  double r_cg_list2;
  double rc_at, rc_cg;
  int ncell;  // cells of all boxes
  int cap;  // neighbour-list capacity per molecule
  int force_block;  // threads per block of the mapping and force kernels
  int cg_mode;  // 0: tabulated F^CG, 1: learned network (pair forces in Bufs::fpair)
  double dt_m[kMaxNA];  // dt / m (both half kicks of a fused step)
  // water-like model (nb_model 1): site-pair Lennard-Jones c12 = 4 eps sigma^12,
  // c6 = 4 eps sigma^6, LJ energy shift, f q_i q_j; reaction field k_rf, c_rf
  int nb_model;
  double c12[kMaxNA][kMaxNA], c6[kMaxNA][kMaxNA], vsh[kMaxNA][kMaxNA], qq[kMaxNA][kMaxNA];
  double krf, crf;
  int lj_cols;  // bit j: some site has a Lennard-Jones term with site j
  // bonded: bond_model 0 FENE (+ WCA), 1 harmonic (bond_k, bond_r0); harmonic angles
  int bond_model;
  double bond_k, bond_r0;
  int n_angles;
  int angles[3 * kMaxAngles];
  double angle_k, angle_theta0;
  // self-adjusting geometry: n_centers > 0 makes the AT region the union of spheres of
  // radius d_at around the centres (Bufs::cen64 / cen32); d is the distance to the nearest
  int n_centers;
  // coupling: 0 force interpolation, 1 energy interpolation (pair weight (l_a + l_b)/2, drift
  // force); free-energy correction g(l) at fec_n nodes (Bufs::fec64 / fec32), fec_n - 1
  int scheme;
  int fec_n;
  double fec_scale;
  // Kirkwood thermodynamic integration: lam_uniform_on != 0 gives every molecule
  // l = lam_uniform (no thermodynamic or drift force; high-resolution items iff l > 0)
  int lam_uniform_on;
  double lam_uniform;
  // multiple time stepping (impulse r-RESPA): respa_n > 1 applies the slow forces (CG pairs,
  // thermodynamic force, CG share of the drift force) with weight respa_n at time levels
  // divisible by respa_n and skips them in between
  int respa_n;
  // float copies of the parameters the FP32 path uses (no run-time double->float work)
  struct {
    float eps, sig2, rc_at, rc_at2, rc_cg2, cg_inv_dr, fene_k, fene_r02;
    float tf_inv_dx;
    float frac[kMaxNA];
    float c12[kMaxNA][kMaxNA], c6[kMaxNA][kMaxNA], qq[kMaxNA][kMaxNA];
    float krf2, bond_k, bond_r0, angle_k, angle_theta0;
    float vsh[kMaxNA][kMaxNA], krf, crf, fec_scale, lam_uniform;
    float r_list2, r_cg_list2;  // the list cutoffs, for the list build
  } f;
};
static_assert(sizeof(Sys) <= 4096, "Sys is passed by value as a kernel parameter");

// Device buffers owned by the handle.
struct Bufs {
  // state (borrowed)
  double* x;
  double* v;
  void* f;
  // per molecule, double-buffered: [parity] is the mapping of the current positions
  int4* com_fx[2];         // fixed-point COM (uint32 bits) + float bits of w
  int4* com_ref;           // fixed-point COM at the last list build
  double4_32a* com64[2];   // FP64 path: COM + w
  double* dxc64[2];        // FP64 path: signed x distance to the slab centre (spheres: distance
                           // to the nearest centre)
  float2* molf[2];         // FP32 path: (signed x distance or distance to the nearest centre,
                           // 1 if in the hybrid layer)
  int* kcen[2];            // spheres: index of the nearest centre
  // per atom, double-buffered
  double4_32a* off64[2];   // COM-relative atom offsets (FP64 path)
  float4* off32[2];        // (FP32 path)
  // lists
  int* mcell;       // Morton rank of each molecule's cell
  int* cell_count;  // [ncell]
  int* cell_fill;   // [ncell]
  int* cell_start;  // [ncell+1]
  int* sorted;      // molecules grouped by cell, cells in Morton order, each cell in id order
  int* fill_tmp;    // [M] cell-grouped molecules in fill (arbitrary) order
  int4* scom;       // [M] fixed-point centres in `sorted` order (staged by the list build)
  int* flag;        // [M] high-resolution candidate flag at sorted positions
  int* pos;         // [M] exclusive scan of flag
  int* items;       // [M] work items: high-resolution candidates first, then CG
  int* item_of;     // [M] work item of each molecule
  int* nn;          // [M] neighbour count per item
  int* nbr;         // [M*cap] neighbour molecule of item t in slot q at nbr[t*cap + q]
  int* scan_tmp;    // block sums for device-wide scans
  const int* cell_rank;  // linear cell -> Morton rank
  // tables
  const double* cgF64;
  const double* cgV64;
  const float2* cgFV32;
  double* tf64;
  float* tf32;
  const double* fec64;  // [fec_n] free-energy correction dDF/dl (energy interpolation)
  const float* fec32;
  // reductions
  double* part;      // per-warp partials
  double* result;    // reduced results [8]
  unsigned long long* hist;  // density histogram [tf_n]
  long long* nsamples;
  Ctrl* ctrl;
  float* fpair;  // [M*cap] network CG pair force per list slot (CG mode 1)
  unsigned* pfrag;  // [pcap][10] normalised network inputs of this step's pairs as bf16 pairs:
                    // words 0-4 the ordering (d, s_a, s_b), 5-9 the ordering (d, s_b, s_a)
  int2* pslot;   // [pcap] the pair's two list slots
  int4* netc;    // [pcap] (CG mode 1) candidate pairs of the last build: slot, slot of the same
                 // pair in the partner's list, a, b
  unsigned* npair;  // pairs written this step
  long long pcap;   // pairs the buffers may hold (the allocation, or a smaller limit the host set)
  long long ncap;   // candidate records netc may hold (the allocation)
  unsigned wait_polls;  // poll limit of the tcgen05 evaluation's product waits (kMmaWaitPolls)
  // batched replicas (nbox > 1)
  const Box* boxes;    // [nbox]
  const int* mol_box;  // [M] box of each molecule
  const int* cell_box; // [ncell] box of each global cell rank
  int* dense_cells;     // [ncell] cells the dense-cell list builder handles
  const double4_32a* cen64;  // [n_centers] resolution centres (spheres)
  const int4* cen32;         // the same in 32-bit fixed point
  const int* nbr_cells; // [ncell][27] Morton ranks of each cell's neighbour cells (-1: none)
};

// Box of molecule a (the single box unless the system holds batched replicas).
__device__ __forceinline__ const Box& box_of(const Sys& s, const Bufs& b, int a) {
  return s.nbox > 1 ? b.boxes[b.mol_box[a]] : s.bx;
}
template <bool MULTI>
__device__ __forceinline__ const Box& box_t(const Sys& s, const Bufs& b, int a) {
  return MULTI ? b.boxes[b.mol_box[a]] : s.bx;
}

// Learned CG force: device parameter arrays (see mlp.cu).
struct MlpDevArgs {
  const float* P;
  const unsigned* W1p;
  const unsigned* W2p;
  const unsigned* W2Tp;
  const float* norm;
};
constexpr int kMlpNPar = 4865;   // 64*9 + 64 + 64*64 + 64 + 64 + 1
constexpr int kMlpNNorm = 19;    // in_mean[9], in_std[9], out_scale (the device copy adds 1/in_std[9])
constexpr int kMlpGradStride = 4868;

__device__ __forceinline__ void set_error(Ctrl* c, int code, int info = 0) {
  if (atomicCAS(&c->err, 0, code) == 0) c->err_info = info;
}

// Squared length of a COM separation with explicit roundings: every kernel that tests a
// pair against a cutoff forms it this way, so the force kernel and the network pair kernel
// decide alike for pairs on the cutoff.
__device__ __forceinline__ float pair_r2(float x, float y, float z) {
  return __fmaf_rn(z, z, __fmaf_rn(y, y, __fmul_rn(x, x)));
}
__device__ __forceinline__ double pair_r2(double x, double y, double z) {
  return __fma_rn(z, z, __fma_rn(y, y, __dmul_rn(x, x)));
}

// Minimum image for |d| < 1.5 L by comparison (no division).
__device__ __forceinline__ double minimg_cmp(double d, double L, double halfL) {
  if (d > halfL) d -= L;
  else if (d < -halfL) d += L;
  return d;
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
cudaError_t launch_com(const Sys& s, const Bufs& b, int precision, int integrate, cudaStream_t st,
                       DecideArgs da = DecideArgs{0, 0, 0, 0});
cudaError_t launch_rebuild(const Sys& s, const Bufs& b, cudaStream_t st);
// Rebuild decision after a mapping kernel (one thread); also flips the current half of the
// molecule arrays and, in a graph, sets the conditional of the rebuild node.
cudaError_t launch_decide(const Sys& s, const Bufs& b, DecideArgs da, cudaStream_t st);
cudaError_t launch_max_nn(const Sys& s, const Bufs& b, cudaStream_t st);
// The network force's candidate pairs of the current lists with their mirror slots
// (Bufs::netc, counted in Ctrl::n_netc, which the caller zeroes); launch_rebuild runs it in
// CG mode 1.
cudaError_t launch_net_candidates(const Sys& s, const Bufs& b, cudaStream_t st);
// out[i] = sum_{j<i} in[j] for i < n, *total = sum of all (n <= 8M)
cudaError_t device_exclusive_scan(const int* in, int* out, int n, int* tmp, int* total, cudaStream_t st);
// mode: 0 conservative forces, 1 last step of a run (thermostat + second half kick),
// 2 fused step (thermostat + both half kicks + drift + next mapping)
cudaError_t launch_step(const Sys& s, const Bufs& b, int precision, int mode, int energy, cudaStream_t st,
                        DecideArgs da = DecideArgs{0, 0, 0, 0});

cudaError_t launch_energy_reduce(const Sys& s, const Bufs& b, int nparts, int nvals, cudaStream_t st);
cudaError_t launch_kinetic(const Sys& s, const Bufs& b, cudaStream_t st);
cudaError_t launch_density(const Sys& s, const Bufs& b, int precision, cudaStream_t st);
cudaError_t launch_tf_update(const Sys& s, const Bufs& b, double alpha, cudaStream_t st);
cudaError_t launch_export_com(const Sys& s, const Bufs& b, int precision, double* com, double* w, cudaStream_t st);
// COM pair-distance histogram of the centres com [3][M] into counts [nbox][nbins] (added).
cudaError_t launch_rdf(const Sys& s, const Bufs& b, const double* com, int nbins, double dr,
                       unsigned long long* counts, cudaStream_t st);

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

cudaError_t mlp_forward(const MlpDevArgs& a, const float* feat, long long n, float* y, cudaStream_t st);
cudaError_t mlp_grad(const MlpDevArgs& a, const float* feat, const float* target, long long n, long long n_total,
                     float* part, float* grad, float* loss_acc, cudaStream_t st);
cudaError_t mlp_adam(const MlpDevArgs& a, float* mom, float* vel, const float* grad, float lr, int step,
                     cudaStream_t st);
cudaError_t mlp_pack(const MlpDevArgs& a, cudaStream_t st);
cudaError_t mlp_collect(const Sys& s, const Bufs& b, int pass, const int* offs, long long cap, long long base,
                        float* feat, float* target, int* ids, int* counts, cudaStream_t st);
cudaError_t mlp_pairs(const Sys& s, const Bufs& b, const MlpDevArgs& a, float* fpair, cudaStream_t st);
// Force-matched CG table from n samples (features [n][9], d = feature 0; targets [n]): bin
// width h, nb = ceil(rc / h) <= 4096 bins, bins with >= n_min samples; F, V device [cg_n + 1]
// on nodes k dr; *npop (device) = bins used.  acc [2 nb], cnt [nb] device scratch.
cudaError_t cg_fit(const float* feat, const float* target, long long n, double h, int nb, int n_min, int cg_n,
                   double dr, double rc, unsigned long long* acc, unsigned* cnt, double* F, double* V, int* npop,
                   cudaStream_t st);
cudaError_t mlp_gather(const float* feat, const float* target, long long n, long long start, long long cnt,
                       long long stride, float* feat_out, float* target_out, cudaStream_t st);

// Record the message returned by adress_last_error(NULL) and return the status.
adress_status set_global_error(adress_status s, const std::string& msg);

// Threads per block of the mapping and force kernels: 32, 64 or 128 (Sys::force_block).
// 128 is also the launch bound the kernels are compiled for (a bound of 256 costs them
// registers and ~4% time at 128 threads).
constexpr int kMaxForceBlock = 128;

// Threads per molecule the force kernel is launched with: four, or eight for the water-like
// model, whose high-resolution items split their neighbour lists over two lane groups.
// water-like model: a high-resolution work item takes kSplitWater groups of four lanes
constexpr int kSplitWater = 2;
inline int step_lanes(const Sys& s) { return s.nb_model == 1 ? kSplitWater * kGroup : kGroup; }

// Warps launched by the force kernel (one energy partial each).
inline int force_warps(const Sys& s) {
  return ceil_div((long long)s.M * step_lanes(s), s.force_block) * (s.force_block / 32);
}

}  // namespace adress
