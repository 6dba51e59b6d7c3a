// Host side of the C ABI declared in include/adress.h.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"

using namespace adress;

struct adress_ctx {
  Sys sys{};
  Bufs buf{};
  int precision = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  int device = 0;
  std::string err;
  bool bound = false;
  bool lists_built = false;
  std::vector<void*> allocs;
  int nparts = 0;
  // captured step graphs keyed by (steps, sample interval, TF update, alpha bits)
  std::map<std::tuple<int, int, int, uint64_t>, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs;
  bool eager = false;  // ADRESS_EAGER=1: launch kernel by kernel (for per-kernel profilers)
  // learned CG force
  float* mlp_P = nullptr;
  unsigned *mlp_W1p = nullptr, *mlp_W2p = nullptr, *mlp_W2Tp = nullptr;
  float *mlp_norm = nullptr, *mlp_mom = nullptr, *mlp_vel = nullptr, *mlp_grad = nullptr, *mlp_loss = nullptr;
  float* mlp_part = nullptr;
  long long mlp_part_blocks = 0;
  int mlp_step = 0;
  bool mlp_ready = false;
  float* smp_feat = nullptr;
  float* smp_target = nullptr;
  int* smp_ids = nullptr;
  long long smp_n = 0, smp_cap = 0;
  float *bat_feat = nullptr, *bat_target = nullptr;
  long long bat_cap = 0;
  int* mlp_counts = nullptr;  // [M + 1]
  int* mlp_offs = nullptr;    // [M + 1]
  MlpDevArgs mlp_args() const { return MlpDevArgs{mlp_P, mlp_W1p, mlp_W2p, mlp_W2Tp, mlp_norm}; }
};

static thread_local std::string g_init_error;
static constexpr int kMaxGraphSteps = 100;  // longest captured step graph

adress_status adress::set_global_error(adress_status s, const std::string& msg) {
  g_init_error = msg;
  return s;
}

static adress_status fail(adress_ctx* h, adress_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_init_error = msg;
  return s;
}

#define CUDA_OR_FAIL(h, call)                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail((h), ADRESS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

template <class T>
static cudaError_t dalloc(adress_ctx* h, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  *p = (T*)q;
  return cudaSuccess;
}

// Replace an owned device buffer by a new allocation of n elements (contents not kept).
template <class T>
static cudaError_t realloc_owned(adress_ctx* h, T** p, size_t n) {
  if (*p) {
    auto it = std::find(h->allocs.begin(), h->allocs.end(), (void*)*p);
    if (it != h->allocs.end()) h->allocs.erase(it);
    cudaFree(*p);
    *p = nullptr;
  }
  return dalloc(h, p, n);
}

static void free_graphs(adress_ctx* h) {
  for (auto& kv : h->graphs) {
    if (kv.second.second) cudaGraphExecDestroy(kv.second.second);
    if (kv.second.first) cudaGraphDestroy(kv.second.first);
  }
  h->graphs.clear();
}

// Host twin of the device fixed-point map: floor(x 2^32 / L) from the bits of x.
static unsigned fixed32_host(double x, unsigned long long K, int q) {
  unsigned long long bits;
  memcpy(&bits, &x, sizeof(bits));
  const int e = (int)((bits >> 52) & 0x7ff);
  const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = q - 44 - (e - 1023);
  const unsigned long long hi = (unsigned long long)(((unsigned __int128)M * K) >> 64);
  return (e == 0 || sh >= 64 || sh < 0) ? 0u : (unsigned)(hi >> sh);
}

static uint64_t morton3(uint64_t x, uint64_t y, uint64_t z) {
  uint64_t c = 0;
  for (int bit = 0; bit < 21; ++bit) {
    c |= ((x >> bit) & 1ull) << (3 * bit + 2);
    c |= ((y >> bit) & 1ull) << (3 * bit + 1);
    c |= ((z >> bit) & 1ull) << (3 * bit);
  }
  return c;
}

static int auto_capacity(const Sys& s) {
  const double vol = s.L[0] * s.L[1] * s.L[2];
  const double expect = 4.0 / 3.0 * M_PI * s.r_list * s.r_list * s.r_list * s.M / vol;
  int cap = (int)ceil(2.0 * expect + 16.0);
  cap = (cap + 3) & ~3;
  return std::min(cap, std::max(4, s.M - 1));
}

extern "C" {

const char* adress_status_string(adress_status s) {
  switch (s) {
    case ADRESS_OK: return "ok";
    case ADRESS_ERR_ARG: return "invalid argument";
    case ADRESS_ERR_CUDA: return "CUDA error";
    case ADRESS_ERR_LIST_OVERFLOW: return "neighbour list overflow";
    case ADRESS_ERR_NONFINITE: return "non-finite force";
    case ADRESS_ERR_BOND_BROKEN: return "FENE bond broken";
    case ADRESS_ERR_TIMEOUT: return "device wait timed out";
    case ADRESS_ERR_STATE: return "invalid state";
    case ADRESS_ERR_EXTENT: return "molecule wider than the list cutoff allows";
  }
  return "unknown status";
}

const char* adress_last_error(adress_handle h) { return h ? h->err.c_str() : g_init_error.c_str(); }

adress_status adress_init(const adress_config* c, void* stream, adress_handle* out) {
  if (!out) return fail(nullptr, ADRESS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!c) return fail(nullptr, ADRESS_ERR_ARG, "config is NULL");
  if (c->n_mols < 2) return fail(nullptr, ADRESS_ERR_ARG, "n_mols must be >= 2");
  if (c->atoms_per_mol < 1 || c->atoms_per_mol > kMaxNA)
    return fail(nullptr, ADRESS_ERR_ARG, "atoms_per_mol must be in 1..4");
  if ((long long)c->n_mols * c->atoms_per_mol > (1ll << 30))
    return fail(nullptr, ADRESS_ERR_ARG, "too many atoms");
  if (!c->mass) return fail(nullptr, ADRESS_ERR_ARG, "mass is NULL");
  for (int k = 0; k < c->atoms_per_mol; ++k)
    if (!(c->mass[k] > 0)) return fail(nullptr, ADRESS_ERR_ARG, "masses must be > 0");
  for (int d = 0; d < 3; ++d)
    if (!(c->box[d] > 0)) return fail(nullptr, ADRESS_ERR_ARG, "box edges must be > 0");
  if (c->n_bonds < 0 || c->n_bonds > kMaxBonds || (c->n_bonds > 0 && !c->bonds))
    return fail(nullptr, ADRESS_ERR_ARG, "n_bonds must be 0..6 with a bond array");
  for (int q = 0; q < 2 * c->n_bonds; ++q)
    if (c->bonds[q] < 0 || c->bonds[q] >= c->atoms_per_mol)
      return fail(nullptr, ADRESS_ERR_ARG, "bond index out of range");
  if (c->n_bonds > 0 && !(c->fene_r0 > 0)) return fail(nullptr, ADRESS_ERR_ARG, "fene_r0 must be > 0");
  if (!c->cg_F || !c->cg_V || c->cg_n < 1 || !(c->cg_dr > 0))
    return fail(nullptr, ADRESS_ERR_ARG, "CG table missing");
  if (c->rc_cg > c->cg_n * c->cg_dr * (1 + 1e-12))
    return fail(nullptr, ADRESS_ERR_ARG, "rc_cg beyond the CG table");
  if (c->tf_n < 0 || (c->tf_n > 0 && (!c->tf || !(c->tf_dx > 0))))
    return fail(nullptr, ADRESS_ERR_ARG, "thermodynamic-force table invalid");
  if (!(c->d_at_half >= 0) || !(c->d_hy >= 0)) return fail(nullptr, ADRESS_ERR_ARG, "slab widths must be >= 0");
  if (!(c->dt > 0) || c->gamma < 0 || c->kT < 0) return fail(nullptr, ADRESS_ERR_ARG, "dt, gamma, kT invalid");
  if (c->precision != ADRESS_FP64 && c->precision != ADRESS_FP32_MIXED)
    return fail(nullptr, ADRESS_ERR_ARG, "unknown precision");
  if (!(c->skin >= 0) || !(c->r_ext >= 0) || !(c->rc_at > 0) || !(c->rc_cg > 0))
    return fail(nullptr, ADRESS_ERR_ARG, "cutoffs invalid");

  adress_ctx* h = new adress_ctx();
  h->precision = c->precision;
  h->stream = (cudaStream_t)stream;
  {
    const char* ev = getenv("ADRESS_EAGER");
    h->eager = ev && ev[0] == '1';
  }
  cudaGetDevice(&h->device);
  Sys& s = h->sys;
  s.M = c->n_mols;
  s.NA = c->atoms_per_mol;
  s.N = s.M * s.NA;
  double Mtot = 0;
  for (int k = 0; k < s.NA; ++k) Mtot += c->mass[k];
  s.Mtot = Mtot;
  for (int k = 0; k < kMaxNA; ++k) {
    double m = k < s.NA ? c->mass[k] : 1.0;
    s.mass[k] = m;
    s.inv_mass[k] = 1.0 / m;
    s.frac[k] = k < s.NA ? m / Mtot : 0.0;
    s.hdt_m[k] = 0.5 * c->dt / m;
    s.amp[k] = sqrt(24.0 * c->gamma * c->kT * m / c->dt);
    s.gm[k] = c->gamma * m;
    s.ampf[k] = (float)s.amp[k];
    s.gmf[k] = (float)s.gm[k];
  }
  s.fp64 = c->precision == ADRESS_FP64;
  for (int d = 0; d < 3; ++d) {
    s.L[d] = c->box[d];
    s.halfL[d] = 0.5 * c->box[d];
    memcpy(&s.Lbits[d], &c->box[d], sizeof(double));
    s.fx_inv[d] = 4294967296.0 / c->box[d];
    s.fx_scale[d] = (float)(c->box[d] / 4294967296.0);
    s.Lf[d] = (float)c->box[d];
    int q = 63;
    while (ldexp(1.0, q) / c->box[d] < 9223372036854775808.0) ++q;  // 2^q / L >= 2^63
    while (ldexp(1.0, q) / c->box[d] >= 18446744073709551616.0) --q;
    s.fxq[d] = q;
    s.fxK[d] = (unsigned long long)(ldexp(1.0, q) / c->box[d]);
  }
  s.xc32 = fixed32_host(c->x_center - c->box[0] * floor(c->x_center / c->box[0]), s.fxK[0], s.fxq[0]);
  s.xc = c->x_center;
  s.d_at = c->d_at_half;
  s.d_hy = c->d_hy;
  s.d_hr = c->d_at_half + c->d_hy + 0.5 * c->skin;
  s.pi_half_over_dhy = c->d_hy > 0 ? 0.5 * M_PI / c->d_hy : 0.0;
  s.eps = c->wca_eps;
  s.sig2 = c->wca_sigma * c->wca_sigma;
  s.rc_at = c->rc_at;
  s.rc_at2 = c->rc_at * c->rc_at;
  s.nb = c->n_bonds;
  for (int q = 0; q < 2 * kMaxBonds; ++q) s.bonds[q] = q < 2 * c->n_bonds ? c->bonds[q] : 0;
  s.fene_k = c->fene_k;
  s.fene_r02 = c->fene_r0 * c->fene_r0;
  s.intra_wca = c->intra_wca;
  s.cg_n = c->cg_n;
  s.cg_inv_dr = 1.0 / c->cg_dr;
  s.rc_cg = c->rc_cg;
  s.rc_cg2 = c->rc_cg * c->rc_cg;
  s.tf_n = c->tf_n;
  s.tf_dx = c->tf_n > 0 ? c->tf_dx : 1.0;
  s.tf_inv_dx = 1.0 / s.tf_dx;
  s.kT = c->kT;
  s.gamma = c->gamma;
  s.dt = c->dt;
  s.seed = c->seed;
  s.seed_lo = (unsigned)(c->seed & 0xffffffffull);
  s.seed_hi = (unsigned)(c->seed >> 32);
  s.replica = c->replica;
  s.skin = c->skin;
  s.r_ext = c->r_ext;
  s.r_list = std::max(c->rc_cg, c->rc_at + 2.0 * c->r_ext) + c->skin;
  s.r_list2 = s.r_list * s.r_list;
  s.reach_at2 = (c->rc_at + 2.0 * c->r_ext) * (c->rc_at + 2.0 * c->r_ext);
  for (int d = 0; d < 3; ++d) {
    if (c->box[d] < 2.0 * s.r_list) {
      delete h;
      return fail(nullptr, ADRESS_ERR_ARG, "box edge shorter than twice the list cutoff");
    }
    s.nc[d] = std::max(1, (int)floor(c->box[d] / s.r_list));
  }
  if ((long long)s.nc[0] * s.nc[1] * s.nc[2] > 4096ll * 2048ll || s.M > 4096 * 2048 - 1) {
    delete h;
    return fail(nullptr, ADRESS_ERR_ARG, "too many cells or molecules for the device scans (max 8388607)");
  }
  if (c->tf_n > 4096) {
    delete h;
    return fail(nullptr, ADRESS_ERR_ARG, "tf_n must be <= 4096");
  }
  s.ncell = s.nc[0] * s.nc[1] * s.nc[2];
  for (int k = 0; k < kMaxNA; ++k) {
    s.dt_m[k] = c->dt / s.mass[k];
    s.f.frac[k] = (float)s.frac[k];
  }
  s.f.eps = (float)s.eps;
  s.f.sig2 = (float)s.sig2;
  s.f.rc_at = (float)s.rc_at;
  s.f.rc_at2 = (float)s.rc_at2;
  s.f.rc_cg2 = (float)s.rc_cg2;
  s.f.cg_inv_dr = (float)s.cg_inv_dr;
  s.f.fene_k = (float)s.fene_k;
  s.f.fene_r02 = (float)s.fene_r02;
  s.f.d_at = (float)s.d_at;
  s.f.d_hyend = (float)(s.d_at + s.d_hy);
  s.f.pi_half_over_dhy = (float)s.pi_half_over_dhy;
  s.f.tf_inv_dx = (float)s.tf_inv_dx;
  s.f.near_at = 1e-4f * (1.f + s.f.d_at);
  s.f.near_hyend = 1e-4f * (1.f + s.f.d_hyend);
  s.cap = c->max_neighbors > 0 ? std::min(c->max_neighbors, s.M - 1) : auto_capacity(s);

  // ---- device buffers ----
  Bufs& b = h->buf;
  const int M = s.M, N = s.N;
  h->nparts = std::max(force_warps(s), ceil_div(N, 256));
  cudaError_t e = cudaSuccess;
#define A(ptr, n)                                  \
  do {                                             \
    if (e == cudaSuccess) e = dalloc(h, &(ptr), (n)); \
  } while (0)
  A(b.com_ref, M);
  for (int p = 0; p < 2; ++p) {
    A(b.com_fx[p], M);
    if (h->precision == ADRESS_FP64) {
      A(b.com64[p], M);
      A(b.dxc64[p], M);
      A(b.off64[p], N);
    } else {
      A(b.molf[p], M);
      A(b.off32[p], N);
    }
  }
  A(b.mcell, M);
  A(b.cell_count, s.ncell);
  A(b.cell_fill, s.ncell);
  A(b.cell_start, s.ncell + 1);
  A(b.sorted, M);
  A(b.flag, M);
  A(b.pos, M + 1);
  A(b.items, M);
  A(b.item_of, M);
  A(b.nn, M);
  A(b.nbr, (size_t)s.cap * M);
  A(b.scan_tmp, 4096);
  int* cell_rank = nullptr;
  int* rank_cell = nullptr;
  A(cell_rank, s.ncell);
  A(rank_cell, s.ncell);
  b.cell_rank = cell_rank;
  b.rank_cell = rank_cell;
  double* cgF = nullptr;
  double* cgV = nullptr;
  float2* cgFV = nullptr;
  A(cgF, s.cg_n + 1);
  A(cgV, s.cg_n + 1);
  A(cgFV, s.cg_n + 1);
  b.cgF64 = cgF;
  b.cgV64 = cgV;
  b.cgFV32 = cgFV;
  A(b.tf64, std::max(1, s.tf_n));
  A(b.tf32, std::max(1, s.tf_n));
  A(b.part, (size_t)h->nparts * 4);
  A(b.result, 8);
  A(b.hist, std::max(1, s.tf_n));
  A(b.nsamples, 1);
  A(b.ctrl, 1);
#undef A
  if (e != cudaSuccess) {
    adress_destroy(h);
    return fail(nullptr, ADRESS_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }

  // ---- Morton ranks of cells ----
  std::vector<std::pair<uint64_t, int>> codes(s.ncell);
  for (int x = 0; x < s.nc[0]; ++x)
    for (int y = 0; y < s.nc[1]; ++y)
      for (int z = 0; z < s.nc[2]; ++z) {
        int lin = (x * s.nc[1] + y) * s.nc[2] + z;
        codes[lin] = {morton3(x, y, z), lin};
      }
  std::sort(codes.begin(), codes.end());
  std::vector<int> rank(s.ncell), rcell(s.ncell);
  for (int r = 0; r < s.ncell; ++r) {
    rank[codes[r].second] = r;
    rcell[r] = codes[r].second;
  }
  std::vector<float2> fv(s.cg_n + 1);
  for (int k = 0; k <= s.cg_n; ++k) fv[k] = make_float2((float)c->cg_F[k], (float)c->cg_V[k]);
  std::vector<double> tf(std::max(1, s.tf_n), 0.0);
  std::vector<float> tff(std::max(1, s.tf_n), 0.f);
  for (int k = 0; k < s.tf_n; ++k) {
    tf[k] = c->tf[k];
    tff[k] = (float)c->tf[k];
  }
  cudaStream_t st = h->stream;
#define H2D(dst, src, bytes)                                                                  \
  do {                                                                                        \
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(dst), (src), (bytes), cudaMemcpyHostToDevice, st); \
  } while (0)
  H2D(cell_rank, rank.data(), sizeof(int) * s.ncell);
  H2D(rank_cell, rcell.data(), sizeof(int) * s.ncell);
  H2D(cgF, c->cg_F, sizeof(double) * (s.cg_n + 1));
  H2D(cgV, c->cg_V, sizeof(double) * (s.cg_n + 1));
  H2D(cgFV, fv.data(), sizeof(float2) * (s.cg_n + 1));
  H2D(b.tf64, tf.data(), sizeof(double) * tf.size());
  H2D(b.tf32, tff.data(), sizeof(float) * tff.size());
#undef H2D
  if (e == cudaSuccess) e = cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.hist, 0, sizeof(unsigned long long) * std::max(1, s.tf_n), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.nsamples, 0, sizeof(long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.com_ref, 0, sizeof(int4) * M, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    std::string msg = std::string("init upload: ") + cudaGetErrorString(e);
    adress_destroy(h);
    return fail(nullptr, ADRESS_ERR_CUDA, msg);
  }
  *out = h;
  return ADRESS_OK;
}

adress_status adress_bind_state(adress_handle h, double* x, double* v, void* f) {
  if (!h) return ADRESS_ERR_ARG;
  if (!x || !v || !f) return fail(h, ADRESS_ERR_ARG, "state pointers must be non-NULL");
  h->buf.x = x;
  h->buf.v = v;
  h->buf.f = f;
  h->bound = true;
  h->lists_built = false;
  free_graphs(h);
  return ADRESS_OK;
}

static adress_status read_ctrl(adress_handle h, Ctrl* c) {
  CUDA_OR_FAIL(h, cudaMemcpyAsync(c, h->buf.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

// Map positions, rebuild lists; grow the capacity and redo while a list overflows.
static adress_status build_lists_sync(adress_handle h) {
  for (int attempt = 0; attempt < 4; ++attempt) {
    CUDA_OR_FAIL(h, launch_com(h->sys, h->buf, h->precision, 0, h->stream, DecideArgs{1, 0, 0, 0}));
    CUDA_OR_FAIL(h, launch_rebuild(h->sys, h->buf, h->stream));
    CUDA_OR_FAIL(h, launch_max_nn(h->sys, h->buf, h->stream));
    Ctrl c;
    adress_status st = read_ctrl(h, &c);
    if (st != ADRESS_OK) return st;
    if (c.err == ADRESS_ERR_LIST_OVERFLOW || c.max_nn > h->sys.cap) {
      int cap = ((int)ceil(c.max_nn * 1.5) + 8 + 3) & ~3;
      cap = std::min(cap, h->sys.M - 1);
      void* old = h->buf.nbr;
      int* nbr = nullptr;
      CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
      CUDA_OR_FAIL(h, dalloc(h, &nbr, (size_t)cap * h->sys.M));
      h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), old));
      cudaFree(old);
      h->buf.nbr = nbr;
      h->sys.cap = cap;
      if (h->buf.fpair) CUDA_OR_FAIL(h, realloc_owned(h, &h->buf.fpair, (size_t)cap * h->sys.M));
      free_graphs(h);
      int zero = 0;
      CUDA_OR_FAIL(h, cudaMemcpyAsync(&h->buf.ctrl->err, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
      continue;
    }
    if (c.err != 0) return fail(h, (adress_status)c.err, std::string("list build: ") +
                                                          adress_status_string((adress_status)c.err));
    h->lists_built = true;
    return ADRESS_OK;
  }
  return fail(h, ADRESS_ERR_LIST_OVERFLOW, "neighbour list capacity could not be grown enough");
}

adress_status adress_build_lists(adress_handle h) {
  if (!h) return ADRESS_ERR_ARG;
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  return build_lists_sync(h);
}

adress_status adress_compute_forces(adress_handle h, double* energies) {
  if (!h) return ADRESS_ERR_ARG;
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  adress_status st = build_lists_sync(h);
  if (st != ADRESS_OK) return st;
  if (h->sys.cg_mode) CUDA_OR_FAIL(h, mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, h->stream));
  CUDA_OR_FAIL(h, launch_step(h->sys, h->buf, h->precision, 0, energies != nullptr, h->stream));
  if (energies) {
    CUDA_OR_FAIL(h, launch_energy_reduce(h->sys, h->buf, force_warps(h->sys), 4, h->stream));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(energies, h->buf.result, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  }
  return ADRESS_OK;
}

// Capture `nsteps` steps into one graph:
//   prologue (half kick + drift + mapping) -> decide -> IF(rebuild){lists}
//   { fused step -> decide -> IF(rebuild){lists} } x (nsteps - 1)
//   last step (thermostat + second half kick, v and f stored)
// `decide` sets the conditional of the IF node that follows it.
static adress_status capture_steps(adress_handle h, int nsteps, int sample_every, int tf_update, double alpha,
                                   cudaGraph_t* gout, cudaGraphExec_t* xout) {
  cudaGraph_t g = nullptr;
  CUDA_OR_FAIL(h, cudaGraphCreate(&g, 0));
  std::vector<cudaGraphNode_t> deps;
  cudaStream_t cs = h->cap_stream;
  auto grab = [&](std::vector<cudaGraphNode_t>& into) -> cudaError_t {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &d, nullptr, &nd);
    if (e != cudaSuccess) return e;
    into.assign(d, d + nd);
    return cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, g, 0, 0);
    if (e != cudaSuccess) break;
    e = cudaStreamBeginCaptureToGraph(cs, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    const DecideArgs da{0, 1, 1, cond};  // the mapping kernel's last block sets the conditional
    cudaError_t le = cudaSuccess;
    if (k > 0 && h->sys.cg_mode) le = mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, cs);
    if (le == cudaSuccess)
      le = k == 0 ? launch_com(h->sys, h->buf, h->precision, 1, cs, da)
                  : launch_step(h->sys, h->buf, h->precision, 2, 0, cs, da);
    std::vector<cudaGraphNode_t> tail;
    cudaError_t ge = grab(tail);
    cudaGraph_t gg = g;
    e = cudaStreamEndCapture(cs, &gg);
    if (e == cudaSuccess) e = le;
    if (e == cudaSuccess) e = ge;
    if (e != cudaSuccess) break;

    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    e = cudaGraphAddNode(&cnode, g, tail.data(), nullptr, tail.size(), &cp);
    if (e != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    le = launch_rebuild(h->sys, h->buf, cs);
    cudaGraph_t bb = body;
    e = cudaStreamEndCapture(cs, &bb);
    if (e == cudaSuccess) e = le;
    if (e != cudaSuccess) break;
    deps.assign(1, cnode);
    // positions of time level k+1 are mapped and current here: sample the profile
    if (sample_every > 0 && (k + 1) % sample_every == 0) {
      e = cudaStreamBeginCaptureToGraph(cs, g, deps.data(), nullptr, deps.size(), cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) break;
      le = launch_density(h->sys, h->buf, h->precision, cs);
      ge = grab(deps);
      gg = g;
      e = cudaStreamEndCapture(cs, &gg);
      if (e == cudaSuccess) e = le;
      if (e == cudaSuccess) e = ge;
    }
  }
  if (e == cudaSuccess) {
    e = cudaStreamBeginCaptureToGraph(cs, g, deps.data(), nullptr, deps.size(), cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = cudaSuccess;
      if (h->sys.cg_mode) le = mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, cs);
      if (le == cudaSuccess) le = launch_step(h->sys, h->buf, h->precision, 1, 0, cs);
      if (le == cudaSuccess && tf_update) le = launch_tf_update(h->sys, h->buf, alpha, cs);
      cudaGraph_t gg = g;
      e = cudaStreamEndCapture(cs, &gg);
      if (e == cudaSuccess) e = le;
    }
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(h, ADRESS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(h, ADRESS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  *gout = g;
  *xout = x;
  return ADRESS_OK;
}

static adress_status launch_graph(adress_handle h, int n, int sample_every, int tf_update, double alpha) {
  uint64_t abits;
  memcpy(&abits, &alpha, sizeof(abits));
  const auto key = std::make_tuple(n, sample_every, tf_update, tf_update ? abits : 0ull);
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaGraph_t g;
    cudaGraphExec_t x;
    adress_status st = capture_steps(h, n, sample_every, tf_update, alpha, &g, &x);
    if (st != ADRESS_OK) return st;
    it = h->graphs.emplace(key, std::make_pair(g, x)).first;
  }
  CUDA_OR_FAIL(h, cudaGraphLaunch(it->second.second, h->stream));
  return ADRESS_OK;
}

adress_status adress_run(adress_handle h, int32_t nsteps, int32_t sample_every, int32_t tf_update, double alpha) {
  if (!h) return ADRESS_ERR_ARG;
  if (nsteps < 1 || nsteps > 1000 || sample_every < 0) return fail(h, ADRESS_ERR_ARG, "need 1 <= nsteps <= 1000, sample_every >= 0");
  if (!h->bound || !h->lists_built) return fail(h, ADRESS_ERR_STATE, "bind state and build lists first");
  if (h->eager) {
    for (int k = 0; k < nsteps; ++k) {
      const DecideArgs da{0, 1, 0, 0};
      if (k > 0 && h->sys.cg_mode) CUDA_OR_FAIL(h, mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, h->stream));
      if (k == 0) CUDA_OR_FAIL(h, launch_com(h->sys, h->buf, h->precision, 1, h->stream, da));
      else CUDA_OR_FAIL(h, launch_step(h->sys, h->buf, h->precision, 2, 0, h->stream, da));
      Ctrl c;
      adress_status st = read_ctrl(h, &c);
      if (st != ADRESS_OK) return st;
      if (c.rebuild) CUDA_OR_FAIL(h, launch_rebuild(h->sys, h->buf, h->stream));
      if (sample_every > 0 && (k + 1) % sample_every == 0)
        CUDA_OR_FAIL(h, launch_density(h->sys, h->buf, h->precision, h->stream));
    }
    if (h->sys.cg_mode) CUDA_OR_FAIL(h, mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, h->stream));
    CUDA_OR_FAIL(h, launch_step(h->sys, h->buf, h->precision, 1, 0, h->stream));
    if (tf_update) CUDA_OR_FAIL(h, launch_tf_update(h->sys, h->buf, alpha, h->stream));
    return ADRESS_OK;
  }
  return launch_graph(h, nsteps, sample_every, tf_update, alpha);
}

adress_status adress_step(adress_handle h, int32_t nsteps) {
  if (!h) return ADRESS_ERR_ARG;
  if (nsteps < 0) return fail(h, ADRESS_ERR_ARG, "nsteps < 0");
  if (!h->bound || !h->lists_built) return fail(h, ADRESS_ERR_STATE, "bind state and build lists first");
  if (nsteps == 0) return ADRESS_OK;
  if (h->eager) {
    for (int k = 0; k < nsteps; ++k) {
      const DecideArgs da{0, 1, 0, 0};
      if (k > 0 && h->sys.cg_mode) CUDA_OR_FAIL(h, mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, h->stream));
      if (k == 0) CUDA_OR_FAIL(h, launch_com(h->sys, h->buf, h->precision, 1, h->stream, da));
      else CUDA_OR_FAIL(h, launch_step(h->sys, h->buf, h->precision, 2, 0, h->stream, da));
      Ctrl c;
      adress_status st = read_ctrl(h, &c);
      if (st != ADRESS_OK) return st;
      if (c.rebuild) CUDA_OR_FAIL(h, launch_rebuild(h->sys, h->buf, h->stream));
    }
    if (h->sys.cg_mode) CUDA_OR_FAIL(h, mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, h->stream));
    CUDA_OR_FAIL(h, launch_step(h->sys, h->buf, h->precision, 1, 0, h->stream));
    return ADRESS_OK;
  }
  int left = nsteps;
  while (left > 0) {
    const int n = std::min(left, kMaxGraphSteps);
    adress_status st = launch_graph(h, n, 0, 0, 0.0);
    if (st != ADRESS_OK) return st;
    left -= n;
  }
  return ADRESS_OK;
}

adress_status adress_set_step(adress_handle h, int64_t step) {
  if (!h) return ADRESS_ERR_ARG;
  long long v = step;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(&h->buf.ctrl->step, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

adress_status adress_get_step(adress_handle h, int64_t* step) {
  if (!h || !step) return ADRESS_ERR_ARG;
  Ctrl c;
  adress_status st = read_ctrl(h, &c);
  if (st == ADRESS_OK) *step = c.step;
  return st;
}

adress_status adress_com_lambda(adress_handle h, double* com, double* w) {
  if (!h || !com || !w) return ADRESS_ERR_ARG;
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  CUDA_OR_FAIL(h, launch_com(h->sys, h->buf, h->precision, 0, h->stream, DecideArgs{0, 0, 0, 0}));
  CUDA_OR_FAIL(h, launch_export_com(h->sys, h->buf, h->precision, com, w, h->stream));
  return ADRESS_OK;
}

adress_status adress_kinetic(adress_handle h, double* out) {
  if (!h || !out) return ADRESS_ERR_ARG;
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  CUDA_OR_FAIL(h, launch_kinetic(h->sys, h->buf, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(out, h->buf.result, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

adress_status adress_density_accumulate(adress_handle h) {
  if (!h) return ADRESS_ERR_ARG;
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  CUDA_OR_FAIL(h, launch_com(h->sys, h->buf, h->precision, 0, h->stream, DecideArgs{0, 0, 0, 0}));
  CUDA_OR_FAIL(h, launch_density(h->sys, h->buf, h->precision, h->stream));
  return ADRESS_OK;
}

adress_status adress_density_get(adress_handle h, int64_t* counts, int32_t n, int64_t* nsamples) {
  if (!h || (!counts && n > 0) || n < 0 || n > h->sys.tf_n) return ADRESS_ERR_ARG;
  if (n > 0)
    CUDA_OR_FAIL(h, cudaMemcpyAsync(counts, h->buf.hist, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, h->stream));
  long long ns = 0;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(&ns, h->buf.nsamples, sizeof(ns), cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  if (nsamples) *nsamples = ns;
  return ADRESS_OK;
}

adress_status adress_density_reset(adress_handle h) {
  if (!h) return ADRESS_ERR_ARG;
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->buf.hist, 0, sizeof(unsigned long long) * std::max(1, h->sys.tf_n), h->stream));
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->buf.nsamples, 0, sizeof(long long), h->stream));
  return ADRESS_OK;
}

adress_status adress_tf_update(adress_handle h, double alpha) {
  if (!h) return ADRESS_ERR_ARG;
  CUDA_OR_FAIL(h, launch_tf_update(h->sys, h->buf, alpha, h->stream));
  return ADRESS_OK;
}

adress_status adress_set_tf(adress_handle h, const double* tf, int32_t n) {
  if (!h || n != h->sys.tf_n || (n > 0 && !tf)) return ADRESS_ERR_ARG;
  if (n == 0) return ADRESS_OK;
  std::vector<float> f(n);
  for (int k = 0; k < n; ++k) f[k] = (float)tf[k];
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->buf.tf64, tf, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->buf.tf32, f.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

adress_status adress_get_tf(adress_handle h, double* tf, int32_t n) {
  if (!h || n != h->sys.tf_n || (n > 0 && !tf)) return ADRESS_ERR_ARG;
  if (n == 0) return ADRESS_OK;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(tf, h->buf.tf64, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

adress_status adress_list_stats(adress_handle h, int64_t* out) {
  if (!h || !out) return ADRESS_ERR_ARG;
  CUDA_OR_FAIL(h, launch_max_nn(h->sys, h->buf, h->stream));
  Ctrl c;
  adress_status st = read_ctrl(h, &c);
  if (st != ADRESS_OK) return st;
  out[0] = c.n_hr;
  out[1] = c.n_cg;
  out[2] = c.rebuilds;
  out[3] = c.max_nn;
  out[4] = h->sys.cap;
  out[5] = h->sys.ncell;
  out[6] = 0;
  out[7] = 0;
  return ADRESS_OK;
}

adress_status adress_time_kernels(adress_handle h, int32_t reps, float* ms_out) {
  if (!h || !ms_out || reps < 1) return ADRESS_ERR_ARG;
  if (!h->bound || !h->lists_built) return fail(h, ADRESS_ERR_STATE, "bind state and build lists first");
  cudaEvent_t ev[4];
  for (int k = 0; k < 4; ++k) CUDA_OR_FAIL(h, cudaEventCreate(&ev[k]));
  double acc[4] = {0, 0, 0, 0};
  cudaError_t e = cudaSuccess;
  cudaStream_t st = h->stream;
  auto timed = [&](int which, auto&& launch) {
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
    acc[which] += t;
  };
  timed(0, [&] { return launch_com(h->sys, h->buf, h->precision, 1, st, DecideArgs{1, 1, 0, 0}); });
  timed(1, [&] { return launch_rebuild(h->sys, h->buf, st); });
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    if (h->sys.cg_mode && e == cudaSuccess) e = mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, st);
    timed(2, [&] { return launch_step(h->sys, h->buf, h->precision, 2, 0, st, DecideArgs{1, 1, 0, 0}); });
    timed(1, [&] { return launch_rebuild(h->sys, h->buf, st); });
  }
  if (h->sys.cg_mode && e == cudaSuccess) e = mlp_pairs(h->sys, h->buf, h->mlp_args(), h->buf.fpair, st);
  timed(3, [&] { return launch_step(h->sys, h->buf, h->precision, 1, 0, st); });
  for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
  if (e != cudaSuccess) return fail(h, ADRESS_ERR_CUDA, std::string("kernel timing: ") + cudaGetErrorString(e));
  ms_out[0] = (float)acc[0];
  ms_out[1] = (float)(acc[1] / (reps + 1));
  ms_out[2] = (float)(acc[2] / reps);
  ms_out[3] = (float)acc[3];
  return ADRESS_OK;
}

adress_status adress_list_export(adress_handle h, int32_t* items, int32_t* nn, int32_t* nbr) {
  if (!h || !items || !nn || !nbr) return ADRESS_ERR_ARG;
  if (!h->lists_built) return fail(h, ADRESS_ERR_STATE, "no lists built");
  const size_t M = (size_t)h->sys.M;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(items, h->buf.items, sizeof(int) * M, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(nn, h->buf.nn, sizeof(int) * M, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(nbr, h->buf.nbr, sizeof(int) * M * h->sys.cap, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

// ---------------- learned CG force ------------------------------------------------------

static adress_status mlp_alloc(adress_handle h) {
  if (h->mlp_P) return ADRESS_OK;
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_P, kMlpNPar));
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_W1p, 64 * 8));
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_W2p, 64 * 32));
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_W2Tp, 64 * 32));
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_norm, kMlpNNorm));
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_mom, kMlpNPar));
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_vel, kMlpNPar));
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_grad, kMlpNPar + 1));
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_loss, 1024));
  return ADRESS_OK;
}

static adress_status mlp_part_for(adress_handle h, long long n) {
  const long long blocks = (n + 63) / 64;
  if (blocks <= h->mlp_part_blocks) return ADRESS_OK;
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  CUDA_OR_FAIL(h, realloc_owned(h, &h->mlp_part, (size_t)blocks * kMlpGradStride));
  h->mlp_part_blocks = blocks;
  return ADRESS_OK;
}

adress_status adress_mlp_set(adress_handle h, const float* params, const float* norm) {
  if (!h || !params || !norm) return ADRESS_ERR_ARG;
  for (int k = 0; k < 9; ++k)
    if (!(norm[9 + k] > 0)) return fail(h, ADRESS_ERR_ARG, "input standard deviations must be > 0");
  adress_status st = mlp_alloc(h);
  if (st != ADRESS_OK) return st;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->mlp_P, params, sizeof(float) * kMlpNPar, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->mlp_norm, norm, sizeof(float) * kMlpNNorm, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->mlp_mom, 0, sizeof(float) * kMlpNPar, h->stream));
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->mlp_vel, 0, sizeof(float) * kMlpNPar, h->stream));
  CUDA_OR_FAIL(h, mlp_pack(h->mlp_args(), h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  h->mlp_step = 0;
  h->mlp_ready = true;
  return ADRESS_OK;
}

adress_status adress_mlp_get(adress_handle h, float* params, float* norm) {
  if (!h || !params || !norm) return ADRESS_ERR_ARG;
  if (!h->mlp_ready) return fail(h, ADRESS_ERR_STATE, "no network parameters set");
  CUDA_OR_FAIL(h, cudaMemcpyAsync(params, h->mlp_P, sizeof(float) * kMlpNPar, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(norm, h->mlp_norm, sizeof(float) * kMlpNNorm, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

adress_status adress_set_cg_mode(adress_handle h, int32_t mode) {
  if (!h || mode < 0 || mode > 1) return ADRESS_ERR_ARG;
  if (mode == 1) {
    if (!h->mlp_ready) return fail(h, ADRESS_ERR_STATE, "set the network parameters first");
    if (h->sys.NA != 4 && h->sys.NA != 3 && h->sys.NA != 2 && h->sys.NA != 1) return ADRESS_ERR_ARG;
    if (!h->buf.fpair) CUDA_OR_FAIL(h, dalloc(h, &h->buf.fpair, (size_t)h->sys.cap * h->sys.M));
  }
  if (h->sys.cg_mode != mode) free_graphs(h);
  h->sys.cg_mode = mode;
  return ADRESS_OK;
}

adress_status adress_mlp_collect(adress_handle h, int64_t cap, int64_t* n_total) {
  if (!h || cap < 1 || !n_total) return ADRESS_ERR_ARG;
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  adress_status st = build_lists_sync(h);
  if (st != ADRESS_OK) return st;
  const int M = h->sys.M;
  if (!h->mlp_counts) {
    CUDA_OR_FAIL(h, dalloc(h, &h->mlp_counts, M + 1));
    CUDA_OR_FAIL(h, dalloc(h, &h->mlp_offs, M + 1));
  }
  CUDA_OR_FAIL(h, mlp_collect(h->sys, h->buf, 0, nullptr, 0, 0, nullptr, nullptr, nullptr, h->mlp_counts, h->stream));
  CUDA_OR_FAIL(h, device_exclusive_scan(h->mlp_counts, h->mlp_offs, M, h->buf.scan_tmp, h->mlp_offs + M, h->stream));
  int found = 0;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(&found, h->mlp_offs + M, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  if (h->smp_cap < cap) {
    // grow, keeping the samples collected so far
    float *nf = nullptr, *nt = nullptr;
    int* ni = nullptr;
    CUDA_OR_FAIL(h, dalloc(h, &nf, (size_t)cap * 9));
    CUDA_OR_FAIL(h, dalloc(h, &nt, (size_t)cap));
    CUDA_OR_FAIL(h, dalloc(h, &ni, (size_t)cap * 2));
    if (h->smp_n > 0) {
      CUDA_OR_FAIL(h, cudaMemcpyAsync(nf, h->smp_feat, sizeof(float) * 9 * h->smp_n, cudaMemcpyDeviceToDevice, h->stream));
      CUDA_OR_FAIL(h, cudaMemcpyAsync(nt, h->smp_target, sizeof(float) * h->smp_n, cudaMemcpyDeviceToDevice, h->stream));
      CUDA_OR_FAIL(h, cudaMemcpyAsync(ni, h->smp_ids, sizeof(int) * 2 * h->smp_n, cudaMemcpyDeviceToDevice, h->stream));
      CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    }
    for (void* old : {(void*)h->smp_feat, (void*)h->smp_target, (void*)h->smp_ids})
      if (old) {
        h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), old));
        cudaFree(old);
      }
    h->smp_feat = nf;
    h->smp_target = nt;
    h->smp_ids = ni;
    h->smp_cap = cap;
  }
  CUDA_OR_FAIL(h, mlp_collect(h->sys, h->buf, 1, h->mlp_offs, h->smp_cap, h->smp_n, h->smp_feat, h->smp_target,
                              h->smp_ids, nullptr, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  h->smp_n = std::min<long long>(h->smp_cap, h->smp_n + found);
  *n_total = h->smp_n;
  return ADRESS_OK;
}

adress_status adress_mlp_samples(adress_handle h, float* feat, float* target, int32_t* ids, int64_t n) {
  if (!h || n < 0 || n > h->smp_n) return ADRESS_ERR_ARG;
  if (n == 0) return ADRESS_OK;
  if (feat) CUDA_OR_FAIL(h, cudaMemcpyAsync(feat, h->smp_feat, sizeof(float) * 9 * n, cudaMemcpyDeviceToHost, h->stream));
  if (target) CUDA_OR_FAIL(h, cudaMemcpyAsync(target, h->smp_target, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
  if (ids) CUDA_OR_FAIL(h, cudaMemcpyAsync(ids, h->smp_ids, sizeof(int) * 2 * n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

adress_status adress_mlp_load_samples(adress_handle h, const float* feat, const float* target, int64_t n) {
  if (!h || !feat || !target || n < 1) return ADRESS_ERR_ARG;
  if (h->smp_cap < n) {
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    CUDA_OR_FAIL(h, realloc_owned(h, &h->smp_feat, (size_t)n * 9));
    CUDA_OR_FAIL(h, realloc_owned(h, &h->smp_target, (size_t)n));
    CUDA_OR_FAIL(h, realloc_owned(h, &h->smp_ids, (size_t)n * 2));
    h->smp_cap = n;
  }
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->smp_feat, feat, sizeof(float) * 9 * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->smp_target, target, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->smp_ids, 0xff, sizeof(int) * 2 * n, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  h->smp_n = n;
  return ADRESS_OK;
}

adress_status adress_mlp_forward(adress_handle h, const float* feat, int64_t n, float* y) {
  if (!h || !feat || !y || n < 1) return ADRESS_ERR_ARG;
  if (!h->mlp_ready) return fail(h, ADRESS_ERR_STATE, "no network parameters set");
  CUDA_OR_FAIL(h, mlp_forward(h->mlp_args(), feat, n, y, h->stream));
  return ADRESS_OK;
}

adress_status adress_mlp_loss_grad(adress_handle h, const float* feat, const float* target, int64_t n, float* grad) {
  if (!h || !feat || !target || !grad || n < 1) return ADRESS_ERR_ARG;
  if (!h->mlp_ready) return fail(h, ADRESS_ERR_STATE, "no network parameters set");
  adress_status st = mlp_part_for(h, n);
  if (st != ADRESS_OK) return st;
  CUDA_OR_FAIL(h, mlp_grad(h->mlp_args(), feat, target, n, n, h->mlp_part, h->mlp_grad, nullptr, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(grad, h->mlp_grad, sizeof(float) * (kMlpNPar + 1), cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

static long long coprime_stride(long long n) {
  long long p = 1000003;  // prime; advance to the next value coprime with n
  auto gcd = [](long long a, long long b) {
    while (b) {
      long long t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  while (gcd(p, n) != 1) p += 2;
  return p % n == 0 ? 1 : p;
}

adress_status adress_mlp_train(adress_handle h, int32_t epochs, int32_t batch, float lr, float* loss) {
  if (!h || epochs < 1 || epochs > 1024 || batch < 16 || !(lr > 0)) return ADRESS_ERR_ARG;
  if (!h->mlp_ready) return fail(h, ADRESS_ERR_STATE, "no network parameters set");
  if (h->smp_n < batch) return fail(h, ADRESS_ERR_STATE, "fewer samples than one batch");
  adress_status st = mlp_part_for(h, batch);
  if (st != ADRESS_OK) return st;
  if (h->bat_cap < batch) {
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    CUDA_OR_FAIL(h, realloc_owned(h, &h->bat_feat, (size_t)batch * 9));
    CUDA_OR_FAIL(h, realloc_owned(h, &h->bat_target, (size_t)batch));
    h->bat_cap = batch;
  }
  const long long n = h->smp_n, nb = n / batch, stride = coprime_stride(n);
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->mlp_loss, 0, sizeof(float) * epochs, h->stream));
  for (int e = 0; e < epochs; ++e)
    for (long long bi = 0; bi < nb; ++bi) {
      CUDA_OR_FAIL(h, mlp_gather(h->smp_feat, h->smp_target, n, (e * nb + bi) * batch, batch, stride, h->bat_feat,
                                 h->bat_target, h->stream));
      CUDA_OR_FAIL(h, mlp_grad(h->mlp_args(), h->bat_feat, h->bat_target, batch, batch, h->mlp_part, h->mlp_grad,
                               h->mlp_loss + e, h->stream));
      CUDA_OR_FAIL(h, mlp_adam(h->mlp_args(), h->mlp_mom, h->mlp_vel, h->mlp_grad, lr, ++h->mlp_step, h->stream));
      CUDA_OR_FAIL(h, mlp_pack(h->mlp_args(), h->stream));
    }
  std::vector<float> acc(epochs);
  CUDA_OR_FAIL(h, cudaMemcpyAsync(acc.data(), h->mlp_loss, sizeof(float) * epochs, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  if (loss)
    for (int e = 0; e < epochs; ++e) loss[e] = acc[e] / (float)(nb * batch);
  return ADRESS_OK;
}

adress_status adress_check(adress_handle h) {
  if (!h) return ADRESS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, ADRESS_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  Ctrl c;
  adress_status st = read_ctrl(h, &c);
  if (st != ADRESS_OK) return st;
  if (c.err != 0) {
    int zero = 0;
    CUDA_OR_FAIL(h, cudaMemcpyAsync(&h->buf.ctrl->err, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    char msg[160];
    snprintf(msg, sizeof(msg), "device error: %s (info %d)", adress_status_string((adress_status)c.err),
             c.err_info);
    return fail(h, (adress_status)c.err, msg);
  }
  return ADRESS_OK;
}

void adress_destroy(adress_handle h) {
  if (!h) return;
  if (h->stream || h->bound) cudaStreamSynchronize(h->stream);
  free_graphs(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // extern "C"
