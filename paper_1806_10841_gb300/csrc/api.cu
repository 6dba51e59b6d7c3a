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
  // boxes (one per replica) and the cell arrays sized for ncell_cap cells
  std::vector<Box> boxes;
  Box* d_boxes = nullptr;
  int* mol_box = nullptr;
  int* cell_box = nullptr;
  int* cell_rank = nullptr;
  int* nbr_cells = nullptr;  // [ncell][27]
  int ncell_cap = 0;
  double4_32a* cen64 = nullptr;  // resolution centres (self-adjusting geometry)
  int4* cen32 = nullptr;
  double skin0 = 0.0;  // skin of the configuration (the autotuner scales it)
  // network pair buffers: pairs allocated, and the smaller limit set by adress_set_limit (0: none)
  long long pcap_alloc = 0, pcap_limit = 0;
  double cg_dr = 0.0;  // node spacing of the CG table
  // radial distribution function scratch
  double* rdf_com = nullptr;
  unsigned long long* rdf_counts = nullptr;
  size_t rdf_cap = 0;
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

// Pair buffers of the network CG force: every unordered listed pair at most once
// (sum of list lengths / 2 <= M cap / 2), plus 16 bytes of slack each for the evaluation's
// bulk copies, which round a ragged last tile up to 16 bytes.
static cudaError_t alloc_pair_buffers(adress_ctx* h) {
  Bufs& b = h->buf;
  const long long pcap = (long long)h->sys.M * h->sys.cap / 2 + 32;
  cudaError_t e = realloc_owned(h, &b.pfrag, (size_t)pcap * 10 + 4);
  if (e == cudaSuccess) e = realloc_owned(h, &b.pslot, (size_t)pcap + 2);
  if (e == cudaSuccess) e = realloc_owned(h, &b.netc, (size_t)pcap);
  if (e == cudaSuccess && !b.npair) e = dalloc(h, &b.npair, 1);
  if (e == cudaSuccess) {
    h->pcap_alloc = pcap;
    b.pcap = h->pcap_limit > 0 ? std::min(h->pcap_limit, pcap) : pcap;
    b.ncap = pcap;
  }
  return e;
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

// Expected neighbours of the densest box, doubled, as the initial list capacity.
static int auto_capacity(const Sys& s, const std::vector<Box>& boxes, const std::vector<int>& nmol) {
  double expect = 0.0;
  for (size_t k = 0; k < boxes.size(); ++k) {
    const Box& B = boxes[k];
    const double vol = B.L[0] * B.L[1] * B.L[2];
    expect = std::max(expect, 4.0 / 3.0 * M_PI * s.r_list * s.r_list * s.r_list * nmol[k] / vol);
  }
  int cap = (int)ceil(2.0 * expect + 16.0);
  cap = (cap + 3) & ~3;
  return std::min(cap, std::max(4, s.M - 1));
}

// Validation of one configuration; empty when valid.
static std::string config_error(const adress_config* c) {
  if (c->n_mols < 2) return "n_mols must be >= 2";
  if (c->atoms_per_mol < 1 || c->atoms_per_mol > kMaxNA) return "atoms_per_mol must be in 1..4";
  if ((long long)c->n_mols * c->atoms_per_mol > (1ll << 30)) return "too many atoms";
  if (!c->mass) return "mass is NULL";
  for (int k = 0; k < c->atoms_per_mol; ++k)
    if (!(c->mass[k] > 0)) return "masses must be > 0";
  for (int d = 0; d < 3; ++d)
    if (!(c->box[d] > 0)) return "box edges must be > 0";
  if (c->n_bonds < 0 || c->n_bonds > kMaxBonds || (c->n_bonds > 0 && !c->bonds))
    return "n_bonds must be 0..6 with a bond array";
  for (int q = 0; q < 2 * c->n_bonds; ++q)
    if (c->bonds[q] < 0 || c->bonds[q] >= c->atoms_per_mol) return "bond index out of range";
  for (int q = 0; q < c->n_bonds; ++q)
    if (c->bonds[2 * q] == c->bonds[2 * q + 1]) return "a bond joins an atom to itself";
  if (c->n_bonds > 0 && !(c->fene_r0 > 0)) return "fene_r0 must be > 0";
  if (!c->cg_F || !c->cg_V || c->cg_n < 1 || !(c->cg_dr > 0)) return "CG table missing";
  if (c->rc_cg > c->cg_n * c->cg_dr * (1 + 1e-12)) return "rc_cg beyond the CG table";
  if (c->tf_n < 0 || (c->tf_n > 0 && (!c->tf || !(c->tf_dx > 0)))) return "thermodynamic-force table invalid";
  if (c->tf_n > 4096) return "tf_n must be <= 4096";
  if (!(c->d_at_half >= 0) || !(c->d_hy >= 0)) return "slab widths must be >= 0";
  if (!(c->dt > 0) || c->gamma < 0 || c->kT < 0) return "dt, gamma, kT invalid";
  if (c->precision != ADRESS_FP64 && c->precision != ADRESS_FP32_MIXED) return "unknown precision";
  if (!(c->skin >= 0) || !(c->r_ext >= 0) || !(c->rc_at > 0) || !(c->rc_cg > 0)) return "cutoffs invalid";
  if (c->nb_model != 0 && c->nb_model != 1) return "nb_model must be 0 or 1";
  if (c->nb_model == 1) {
    if (c->atoms_per_mol != 3) return "nb_model 1 needs three atoms per molecule";
    if (!c->charge || !c->lj_eps || !c->lj_sigma) return "nb_model 1 needs charge, lj_eps and lj_sigma";
    for (int k = 0; k < c->atoms_per_mol; ++k)
      if (!(c->lj_eps[k] >= 0) || !(c->lj_sigma[k] >= 0) || !(c->charge[k] == c->charge[k]))
        return "lj_eps, lj_sigma must be >= 0 and charges finite";
    if (!(c->coulomb_f >= 0) || !(c->eps_rf >= 1)) return "coulomb_f must be >= 0 and eps_rf >= 1";
  }
  if (c->bond_model != 0 && c->bond_model != 1) return "bond_model must be 0 or 1";
  if (c->bond_model == 1 && (!(c->bond_k >= 0) || !(c->bond_r0 > 0))) return "bond_k >= 0 and bond_r0 > 0 needed";
  if (c->n_angles < 0 || c->n_angles > kMaxAngles || (c->n_angles > 0 && !c->angles)) return "n_angles must be 0..4 with an angle array";
  for (int q = 0; q < c->n_angles; ++q) {
    const int* t = c->angles + 3 * q;
    if (t[0] < 0 || t[1] < 0 || t[2] < 0 || t[0] >= c->atoms_per_mol || t[1] >= c->atoms_per_mol ||
        t[2] >= c->atoms_per_mol || t[0] == t[1] || t[1] == t[2] || t[0] == t[2])
      return "angle indices out of range or repeated";
  }
  if (c->n_angles > 0 && (!(c->angle_k >= 0) || !(c->angle_theta0 > 0) || !(c->angle_theta0 <= M_PI)))
    return "angle_k >= 0 and 0 < angle_theta0 <= pi needed";
  if (c->n_centers < 0 || c->n_centers > kMaxCenters || (c->n_centers > 0 && !c->centers))
    return "n_centers must be 0..1024 with a centre array";
  for (int q = 0; q < 3 * c->n_centers; ++q)
    if (!(c->centers[q] == c->centers[q]) || isinf(c->centers[q])) return "resolution centres must be finite";
  if (c->scheme != 0 && c->scheme != 1) return "scheme must be 0 (force) or 1 (energy interpolation)";
  if (c->fec_n < 0 || c->fec_n == 1 || c->fec_n > 4096 || (c->fec_n > 0 && !c->fec))
    return "fec_n must be 0 or 2..4096 with a table";
  if (c->fec_n > 0 && c->scheme != 1) return "the free-energy correction needs scheme 1";
  if (c->respa_n < 0 || c->respa_n > 64) return "respa_n must be 0..64";
  for (int k = 0; k < c->fec_n; ++k)
    if (!(c->fec[k] == c->fec[k]) || isinf(c->fec[k])) return "free-energy correction must be finite";
  return "";
}

// Replicas of a batch share the molecule model, the interaction, the tables' grids, the
// thermostat and the list parameters; they differ in size, box, slab and replica id.
static std::string shared_mismatch(const adress_config* a, const adress_config* c) {
  if (c->atoms_per_mol != a->atoms_per_mol) return "atoms_per_mol";
  for (int k = 0; k < a->atoms_per_mol; ++k)
    if (c->mass[k] != a->mass[k]) return "mass";
  if (c->wca_eps != a->wca_eps || c->wca_sigma != a->wca_sigma || c->rc_at != a->rc_at) return "WCA parameters";
  if (c->n_bonds != a->n_bonds || c->fene_k != a->fene_k || c->fene_r0 != a->fene_r0 ||
      c->intra_wca != a->intra_wca)
    return "bonded model";
  for (int q = 0; q < 2 * a->n_bonds; ++q)
    if (c->bonds[q] != a->bonds[q]) return "bond list";
  if (c->cg_n != a->cg_n || c->cg_dr != a->cg_dr || c->rc_cg != a->rc_cg) return "CG table grid";
  for (int k = 0; k <= a->cg_n; ++k)
    if (c->cg_F[k] != a->cg_F[k] || c->cg_V[k] != a->cg_V[k]) return "CG table";
  if (c->tf_n != a->tf_n || (a->tf_n > 0 && c->tf_dx != a->tf_dx)) return "thermodynamic-force grid";
  if (c->kT != a->kT || c->gamma != a->gamma || c->dt != a->dt || c->seed != a->seed) return "thermostat";
  if (c->skin != a->skin || c->r_ext != a->r_ext || c->max_neighbors != a->max_neighbors) return "list parameters";
  if (c->precision != a->precision) return "precision";
  if (c->nb_model != a->nb_model || c->coulomb_f != a->coulomb_f || c->eps_rf != a->eps_rf) return "nonbonded model";
  for (int k = 0; k < a->atoms_per_mol && a->nb_model == 1; ++k)
    if (c->charge[k] != a->charge[k] || c->lj_eps[k] != a->lj_eps[k] || c->lj_sigma[k] != a->lj_sigma[k])
      return "site parameters";
  if (c->bond_model != a->bond_model || c->bond_k != a->bond_k || c->bond_r0 != a->bond_r0 ||
      c->n_angles != a->n_angles || c->angle_k != a->angle_k || c->angle_theta0 != a->angle_theta0)
    return "bonded model";
  for (int q = 0; q < 3 * a->n_angles; ++q)
    if (c->angles[q] != a->angles[q]) return "angle list";
  if (c->scheme != a->scheme || c->fec_n != a->fec_n) return "coupling scheme";
  if (std::max(1, c->respa_n) != std::max(1, a->respa_n)) return "multiple time stepping";
  for (int k = 0; k < a->fec_n; ++k)
    if (c->fec[k] != a->fec[k]) return "free-energy correction";
  return "";
}

// Geometry of one box: edges, fixed-point maps and slab (cells are set by setup_cells).
static Box make_box(const adress_config* c, double skin) {
  Box B{};
  for (int d = 0; d < 3; ++d) {
    B.L[d] = c->box[d];
    B.halfL[d] = 0.5 * c->box[d];
    memcpy(&B.Lbits[d], &c->box[d], sizeof(double));
    B.fx_inv[d] = 4294967296.0 / c->box[d];
    B.fx_scale[d] = (float)(c->box[d] / 4294967296.0);
    int q = 63;
    while (ldexp(1.0, q) / c->box[d] < 9223372036854775808.0) ++q;  // 2^q / L >= 2^63
    while (ldexp(1.0, q) / c->box[d] >= 18446744073709551616.0) --q;
    B.fxq[d] = q;
    B.fxK[d] = (unsigned long long)(ldexp(1.0, q) / c->box[d]);
  }
  B.xc32 = fixed32_host(c->x_center - c->box[0] * floor(c->x_center / c->box[0]), B.fxK[0], B.fxq[0]);
  B.xc = c->x_center;
  B.d_at = c->d_at_half;
  B.d_hy = c->d_hy;
  B.d_hr = c->d_at_half + c->d_hy + 0.5 * skin;
  B.pi_half_over_dhy = c->d_hy > 0 ? 0.5 * M_PI / c->d_hy : 0.0;
  B.d_at_f = (float)B.d_at;
  B.d_hyend_f = (float)(B.d_at + B.d_hy);
  B.pi_half_over_dhy_f = (float)B.pi_half_over_dhy;
  B.near_at = 1e-4f * (1.f + B.d_at_f);
  B.near_hyend = 1e-4f * (1.f + B.d_hyend_f);
  B.replica = c->replica;
  return B;
}

// List cutoff r_list = max(rc_cg, rc_at + 2 r_ext) + skin and everything that follows from
// it: cells of edge >= r_list in every box (ranked in Morton order inside each box, boxes
// one after another), the high-resolution candidate bound, and the device copies.
static adress_status setup_cells(adress_ctx* h, double skin) {
  Sys& s = h->sys;
  Bufs& b = h->buf;
  const double r_list = std::max(s.rc_cg, s.rc_at + 2.0 * s.r_ext) + skin;
  for (const Box& B : h->boxes)
    for (int d = 0; d < 3; ++d)
      if (B.L[d] < 2.0 * r_list) return fail(h, ADRESS_ERR_ARG, "box edge shorter than twice the list cutoff");
  long long total = 0;
  for (Box& B : h->boxes) {
    for (int d = 0; d < 3; ++d) B.nc[d] = std::max(1, (int)floor(B.L[d] / r_list));
    B.ncell = B.nc[0] * B.nc[1] * B.nc[2];
    B.cell0 = (int)std::min<long long>(total, 1ll << 30);
    total += (long long)B.nc[0] * B.nc[1] * B.nc[2];
  }
  if (total > 4096ll * 2048ll) return fail(h, ADRESS_ERR_ARG, "too many cells for the device scans (max 8388608)");
  s.skin = skin;
  s.r_list = r_list;
  s.r_list2 = r_list * r_list;
  s.r_cg_list2 = (s.rc_cg + skin) * (s.rc_cg + skin);
  s.f.r_list2 = (float)s.r_list2;
  s.f.r_cg_list2 = (float)s.r_cg_list2;
  s.ncell = (int)total;
  // energy interpolation: a molecule within r_list of the hybrid layer may pair with a
  // hybrid one (weight (l_a + l_b)/2 > 0), so it is a high-resolution item too
  for (Box& B : h->boxes) B.d_hr = B.d_at + B.d_hy + (s.scheme == 1 ? r_list : 0.5 * skin);
  s.bx = h->boxes[0];

  cudaError_t e = cudaSuccess;
  if (s.ncell > h->ncell_cap) {
    int *cc = b.cell_count, *cf = b.cell_fill, *cs = b.cell_start;
    if (e == cudaSuccess) e = realloc_owned(h, &cc, s.ncell);
    if (e == cudaSuccess) e = realloc_owned(h, &cf, s.ncell);
    if (e == cudaSuccess) e = realloc_owned(h, &cs, s.ncell + 1);
    if (e == cudaSuccess) e = realloc_owned(h, &h->cell_rank, s.ncell);
    if (e == cudaSuccess && s.nbox > 1) e = realloc_owned(h, &h->cell_box, s.ncell);
    if (e == cudaSuccess) e = realloc_owned(h, &h->buf.dense_cells, s.ncell);
    if (e == cudaSuccess) e = realloc_owned(h, &h->nbr_cells, (size_t)s.ncell * 27);
    b.cell_count = cc;
    b.cell_fill = cf;
    b.cell_start = cs;
    if (e != cudaSuccess) return fail(h, ADRESS_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->ncell_cap = s.ncell;
  }
  // the list build expects zero cell counters (it leaves them zero after each build)
  e = cudaMemsetAsync(b.cell_count, 0, sizeof(int) * (size_t)s.ncell, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.cell_fill, 0, sizeof(int) * (size_t)s.ncell, h->stream);
  if (e != cudaSuccess) return fail(h, ADRESS_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  b.cell_rank = h->cell_rank;
  b.cell_box = h->cell_box;
  b.nbr_cells = h->nbr_cells;

  std::vector<int> rank(s.ncell), cbox(s.nbox > 1 ? s.ncell : 0);
  for (int k = 0; k < s.nbox; ++k) {
    const Box& B = h->boxes[k];
    std::vector<std::pair<uint64_t, int>> codes(B.ncell);
    for (int x = 0; x < B.nc[0]; ++x)
      for (int y = 0; y < B.nc[1]; ++y)
        for (int z = 0; z < B.nc[2]; ++z) {
          const int lin = (x * B.nc[1] + y) * B.nc[2] + z;
          codes[lin] = {morton3(x, y, z), lin};
        }
    std::sort(codes.begin(), codes.end());
    for (int r = 0; r < B.ncell; ++r) {
      rank[B.cell0 + codes[r].second] = B.cell0 + r;
      if (s.nbox > 1) cbox[B.cell0 + r] = k;
    }
  }
  // the 27 neighbour cells of every cell (by Morton rank), in the list order
  // (ox, oy, oz) = (j/9 - 1, (j/3)%3 - 1, j%3 - 1); -1 where a dimension has fewer than three
  // cells and the offset would repeat a cell
  std::vector<int> ncells((size_t)s.ncell * 27);
  for (int k = 0; k < s.nbox; ++k) {
    const Box& B = h->boxes[k];
    for (int x = 0; x < B.nc[0]; ++x)
      for (int y = 0; y < B.nc[1]; ++y)
        for (int z = 0; z < B.nc[2]; ++z) {
          const int r = rank[B.cell0 + (x * B.nc[1] + y) * B.nc[2] + z];
          for (int j = 0; j < 27; ++j) {
            const int o[3] = {j / 9 - 1, (j / 3) % 3 - 1, j % 3 - 1};
            const int c[3] = {x, y, z};
            int q[3];
            bool ok = true;
            for (int d = 0; d < 3; ++d) {
              const int lo = B.nc[d] >= 3 ? -1 : 0, hi = B.nc[d] >= 2 ? 1 : 0;
              ok = ok && o[d] >= lo && o[d] <= hi;
              q[d] = (c[d] + o[d] + B.nc[d]) % B.nc[d];
            }
            ncells[(size_t)r * 27 + j] = ok ? rank[B.cell0 + (q[0] * B.nc[1] + q[1]) * B.nc[2] + q[2]] : -1;
          }
        }
  }
  cudaStream_t st = h->stream;
  e = cudaMemcpyAsync(h->cell_rank, rank.data(), sizeof(int) * s.ncell, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->nbr_cells, ncells.data(), sizeof(int) * ncells.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && s.nbox > 1)
    e = cudaMemcpyAsync(h->cell_box, cbox.data(), sizeof(int) * s.ncell, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && s.nbox > 1)
    e = cudaMemcpyAsync(h->d_boxes, h->boxes.data(), sizeof(Box) * s.nbox, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
  if (e != cudaSuccess) return fail(h, ADRESS_ERR_CUDA, std::string("cell upload: ") + cudaGetErrorString(e));
  free_graphs(h);
  h->lists_built = false;
  return ADRESS_OK;
}

// Resolution centres wrapped into the box, in double and in 32-bit fixed point.
static adress_status upload_centers(adress_ctx* h, const double* c, int n) {
  const Box& B = h->boxes[0];
  std::vector<double4_32a> c64(n);
  std::vector<int4> c32(n);
  for (int k = 0; k < n; ++k) {
    double w[3];
    for (int d = 0; d < 3; ++d) {
      w[d] = c[3 * k + d] - B.L[d] * floor(c[3 * k + d] / B.L[d]);
      if (w[d] >= B.L[d]) w[d] -= B.L[d];
    }
    c64[k] = make_double4_32a(w[0], w[1], w[2], 0.0);
    c32[k] = make_int4((int)fixed32_host(w[0], B.fxK[0], B.fxq[0]), (int)fixed32_host(w[1], B.fxK[1], B.fxq[1]),
                       (int)fixed32_host(w[2], B.fxK[2], B.fxq[2]), 0);
  }
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->cen64, c64.data(), sizeof(double4_32a) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->cen32, c32.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

static adress_status init_impl(const adress_config* cfgs, int nbox, void* stream, adress_handle* out) {
  if (!out) return fail(nullptr, ADRESS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfgs) return fail(nullptr, ADRESS_ERR_ARG, "config is NULL");
  if (nbox < 1 || nbox > 65536) return fail(nullptr, ADRESS_ERR_ARG, "n_replicas must be in 1..65536");
  long long mtot = 0;
  for (int k = 0; k < nbox; ++k) {
    const std::string why = config_error(&cfgs[k]);
    if (!why.empty())
      return fail(nullptr, ADRESS_ERR_ARG, nbox > 1 ? "replica " + std::to_string(k) + ": " + why : why);
    if (k > 0) {
      const std::string what = shared_mismatch(&cfgs[0], &cfgs[k]);
      if (!what.empty())
        return fail(nullptr, ADRESS_ERR_ARG, "replica " + std::to_string(k) + " differs from replica 0 in " + what);
    }
    const double r_list = std::max(cfgs[k].rc_cg, cfgs[k].rc_at + 2.0 * cfgs[k].r_ext) + cfgs[k].skin;
    for (int d = 0; d < 3; ++d)
      if (cfgs[k].box[d] < 2.0 * r_list)
        return fail(nullptr, ADRESS_ERR_ARG,
                    (nbox > 1 ? "replica " + std::to_string(k) + ": " : std::string()) +
                        "box edge shorter than twice the list cutoff");
    mtot += cfgs[k].n_mols;
  }
  if (nbox > 1)
    for (int k = 0; k < nbox; ++k)
      if (cfgs[k].n_centers > 0)
        return fail(nullptr, ADRESS_ERR_ARG, "resolution centres are supported for single-system handles only");
  if (mtot > 4096 * 2048 - 1)
    return fail(nullptr, ADRESS_ERR_ARG, "too many molecules for the device scans (max 8388607)");
  const adress_config* c = &cfgs[0];

  adress_ctx* h = new adress_ctx();
  h->precision = c->precision;
  h->stream = (cudaStream_t)stream;
  {
    const char* ev = getenv("ADRESS_EAGER");
    h->eager = ev && ev[0] == '1';
  }
  cudaGetDevice(&h->device);
  Sys& s = h->sys;
  s.nbox = nbox;
  s.M = (int)mtot;
  s.NA = c->atoms_per_mol;
  s.N = s.M * s.NA;
  s.force_block = 128;
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
  s.eps = c->wca_eps;
  s.sig2 = c->wca_sigma * c->wca_sigma;
  s.rc_at = c->rc_at;
  s.rc_at2 = c->rc_at * c->rc_at;
  s.nb = c->n_bonds;
  for (int q = 0; q < 2 * kMaxBonds; ++q) s.bonds[q] = q < 2 * c->n_bonds ? c->bonds[q] : 0;
  // per-atom bond partners in bond order (bit 3: this atom is the bond's first atom)
  {
    int cnt[kMaxNA] = {0, 0, 0, 0};
    for (int g = 0; g < kMaxNA; ++g) s.bond_word[g] = 0;
    for (int q = 0; q < c->n_bonds; ++q) {
      const int p0 = c->bonds[2 * q], p1 = c->bonds[2 * q + 1];
      s.bond_word[p0] |= (unsigned)(p1 | 8) << (4 * cnt[p0]++);
      s.bond_word[p1] |= (unsigned)p0 << (4 * cnt[p1]++);
    }
    s.bmax = 0;
    for (int g = 0; g < kMaxNA; ++g) {
      s.bond_word[g] |= (unsigned)cnt[g] << 28;
      s.bmax = std::max(s.bmax, cnt[g]);
    }
  }
  s.fene_k = c->fene_k;
  s.fene_r02 = c->fene_r0 * c->fene_r0;
  s.intra_wca = c->intra_wca;
  s.cg_n = c->cg_n;
  s.cg_inv_dr = 1.0 / c->cg_dr;
  h->cg_dr = c->cg_dr;
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
  s.r_ext = c->r_ext;
  s.reach_at2 = (c->rc_at + 2.0 * c->r_ext) * (c->rc_at + 2.0 * c->r_ext);
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
  s.f.tf_inv_dx = (float)s.tf_inv_dx;
  s.nb_model = c->nb_model;
  if (c->nb_model == 1) {
    const double rc = c->rc_at;
    s.krf = (c->eps_rf - 1.0) / ((2.0 * c->eps_rf + 1.0) * rc * rc * rc);
    s.crf = 1.0 / rc + s.krf * rc * rc;
    for (int i = 0; i < s.NA; ++i)
      for (int j = 0; j < s.NA; ++j) {
        const double e = sqrt(c->lj_eps[i] * c->lj_eps[j]);
        const double sg = 0.5 * (c->lj_sigma[i] + c->lj_sigma[j]);
        const double s6 = sg * sg * sg * sg * sg * sg;
        s.c12[i][j] = 4.0 * e * s6 * s6;
        s.c6[i][j] = 4.0 * e * s6;
        const double ir6 = 1.0 / (rc * rc * rc * rc * rc * rc);
        s.vsh[i][j] = -(s.c12[i][j] * ir6 - s.c6[i][j]) * ir6;
        s.qq[i][j] = c->coulomb_f * c->charge[i] * c->charge[j];
        if (s.c12[i][j] != 0.0 || s.c6[i][j] != 0.0) s.lj_cols |= 1 << j;
        s.f.c12[i][j] = (float)s.c12[i][j];
        s.f.c6[i][j] = (float)s.c6[i][j];
        s.f.qq[i][j] = (float)s.qq[i][j];
      }
    s.f.krf2 = (float)(2.0 * s.krf);
    s.f.krf = (float)s.krf;
    s.f.crf = (float)s.crf;
    for (int i = 0; i < s.NA; ++i)
      for (int j = 0; j < s.NA; ++j) s.f.vsh[i][j] = (float)s.vsh[i][j];
  }
  s.scheme = c->scheme;
  s.fec_n = c->fec_n;
  s.fec_scale = c->fec_n > 1 ? (double)(c->fec_n - 1) : 0.0;
  s.f.fec_scale = (float)s.fec_scale;
  s.n_centers = c->n_centers;
  s.lam_uniform_on = 0;
  s.lam_uniform = 0.0;
  s.respa_n = std::max(1, c->respa_n);
  s.bond_model = c->bond_model;
  s.bond_k = c->bond_k;
  s.bond_r0 = c->bond_r0;
  s.n_angles = c->n_angles;
  for (int q = 0; q < 3 * kMaxAngles; ++q) s.angles[q] = q < 3 * c->n_angles ? c->angles[q] : 0;
  s.angle_k = c->angle_k;
  s.angle_theta0 = c->angle_theta0;
  s.f.bond_k = (float)c->bond_k;
  s.f.bond_r0 = (float)c->bond_r0;
  s.f.angle_k = (float)c->angle_k;
  s.f.angle_theta0 = (float)c->angle_theta0;

  std::vector<int> nmol(nbox);
  h->boxes.resize(nbox);
  int mol0 = 0;
  for (int k = 0; k < nbox; ++k) {
    Box& B = h->boxes[k];
    B = make_box(&cfgs[k], c->skin);
    B.mol0 = mol0;
    B.nmol = cfgs[k].n_mols;
    B.index = k;
    B.tf0 = k * s.tf_n;
    nmol[k] = cfgs[k].n_mols;
    mol0 += cfgs[k].n_mols;
  }
  h->skin0 = c->skin;
  s.r_list = std::max(c->rc_cg, c->rc_at + 2.0 * c->r_ext) + c->skin;
  s.cap = c->max_neighbors > 0 ? std::min(c->max_neighbors, s.M - 1) : auto_capacity(s, h->boxes, nmol);

  // ---- device buffers ----
  Bufs& b = h->buf;
  const int M = s.M, N = s.N;
  {
    int warps = 0;
    for (int blk = 32; blk <= kMaxForceBlock; blk *= 2)
      warps = std::max(warps, ceil_div((long long)M * step_lanes(s), blk) * (blk / 32));
    h->nparts = std::max(warps, ceil_div(N, 256));
  }
  const int ntf = std::max(1, nbox * s.tf_n);
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
    if (c->n_centers > 0) A(b.kcen[p], M);
  }
  A(b.mcell, M);
  A(b.sorted, M);
  A(b.fill_tmp, M);
  A(b.scom, M);
  A(b.flag, M);
  A(b.pos, M + 1);
  A(b.items, M);
  A(b.item_of, M);
  A(b.nn, M);
  A(b.nbr, (size_t)s.cap * M);
  A(b.scan_tmp, 4096);
  double* cgF = nullptr;
  double* cgV = nullptr;
  float2* cgFV = nullptr;
  A(cgF, s.cg_n + 1);
  A(cgV, s.cg_n + 1);
  A(cgFV, s.cg_n + 1);
  b.cgF64 = cgF;
  b.cgV64 = cgV;
  b.cgFV32 = cgFV;
  A(b.tf64, ntf);
  A(b.tf32, ntf);
  if (c->fec_n > 0) {
    double* f64 = nullptr;
    float* f32 = nullptr;
    A(f64, c->fec_n);
    A(f32, c->fec_n);
    b.fec64 = f64;
    b.fec32 = f32;
  }
  A(b.part, (size_t)h->nparts * 4);
  A(b.result, 8);
  A(b.hist, ntf);
  A(b.nsamples, 1);
  A(b.ctrl, 1);
  if (c->n_centers > 0) {
    A(h->cen64, c->n_centers);
    A(h->cen32, c->n_centers);
  }
  if (nbox > 1) {
    A(h->d_boxes, nbox);
    A(h->mol_box, M);
  }
#undef A
  b.boxes = h->d_boxes;
  b.mol_box = h->mol_box;
  b.wait_polls = kMmaWaitPolls;
  b.cen64 = h->cen64;
  b.cen32 = h->cen32;
  if (e != cudaSuccess) {
    adress_destroy(h);
    return fail(nullptr, ADRESS_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  {
    adress_status st = setup_cells(h, c->skin);
    if (st != ADRESS_OK) {
      const std::string msg = h->err;
      adress_destroy(h);
      return fail(nullptr, st, msg);
    }
  }

  std::vector<float2> fv(s.cg_n + 1);
  for (int k = 0; k <= s.cg_n; ++k) fv[k] = make_float2((float)c->cg_F[k], (float)c->cg_V[k]);
  std::vector<double> tf(ntf, 0.0);
  std::vector<float> tff(ntf, 0.f);
  std::vector<float> fecf(c->fec, c->fec + c->fec_n);  // staged until the stream synchronises
  for (int r = 0; r < nbox; ++r)
    for (int k = 0; k < s.tf_n; ++k) {
      tf[r * s.tf_n + k] = cfgs[r].tf[k];
      tff[r * s.tf_n + k] = (float)cfgs[r].tf[k];
    }
  std::vector<int> mb(nbox > 1 ? M : 0);
  for (int r = 0; r < nbox && nbox > 1; ++r)
    std::fill(mb.begin() + h->boxes[r].mol0, mb.begin() + h->boxes[r].mol0 + cfgs[r].n_mols, r);
  cudaStream_t st = h->stream;
#define H2D(dst, src, bytes)                                                                  \
  do {                                                                                        \
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(dst), (src), (bytes), cudaMemcpyHostToDevice, st); \
  } while (0)
  H2D(cgF, c->cg_F, sizeof(double) * (s.cg_n + 1));
  H2D(cgV, c->cg_V, sizeof(double) * (s.cg_n + 1));
  H2D(cgFV, fv.data(), sizeof(float2) * (s.cg_n + 1));
  H2D(b.tf64, tf.data(), sizeof(double) * tf.size());
  H2D(b.tf32, tff.data(), sizeof(float) * tff.size());
  if (c->fec_n > 0) {
    H2D(b.fec64, c->fec, sizeof(double) * c->fec_n);
    H2D(b.fec32, fecf.data(), sizeof(float) * c->fec_n);
  }
  if (nbox > 1) H2D(h->mol_box, mb.data(), sizeof(int) * M);
#undef H2D
  if (e == cudaSuccess) e = cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.hist, 0, sizeof(unsigned long long) * ntf, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.nsamples, 0, sizeof(long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.com_ref, 0, sizeof(int4) * M, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    std::string msg = std::string("init upload: ") + cudaGetErrorString(e);
    adress_destroy(h);
    return fail(nullptr, ADRESS_ERR_CUDA, msg);
  }
  if (c->n_centers > 0) {
    adress_status st2 = upload_centers(h, c->centers, c->n_centers);
    if (st2 != ADRESS_OK) {
      const std::string msg = h->err;
      adress_destroy(h);
      return fail(nullptr, st2, msg);
    }
  }
  *out = h;
  return ADRESS_OK;
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
  return init_impl(c, 1, stream, out);
}

adress_status adress_init_batch(const adress_config* cfgs, int32_t n_replicas, void* stream, adress_handle* out) {
  return init_impl(cfgs, n_replicas, stream, out);
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
      if (h->buf.fpair) {
        CUDA_OR_FAIL(h, realloc_owned(h, &h->buf.fpair, (size_t)cap * h->sys.M));
        CUDA_OR_FAIL(h, alloc_pair_buffers(h));
      }
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

adress_status adress_set_uniform_lambda(adress_handle h, int32_t on, double lambda) {
  if (!h) return ADRESS_ERR_ARG;
  if (on && !(lambda >= 0.0 && lambda <= 1.0)) return fail(h, ADRESS_ERR_ARG, "uniform lambda must be in [0, 1]");
  h->sys.lam_uniform_on = on ? 1 : 0;
  h->sys.lam_uniform = on ? lambda : 0.0;
  h->sys.f.lam_uniform = (float)h->sys.lam_uniform;
  free_graphs(h);
  h->lists_built = false;  // the work-item classes change
  return ADRESS_OK;
}

adress_status adress_kirkwood(adress_handle h, const double* lambdas, int32_t n, int32_t n_equil, int32_t n_samples,
                              int32_t every, double* dhdl) {
  if (!h || !lambdas || !dhdl || n < 1 || n_equil < 0 || n_samples < 1 || every < 1)
    return fail(h, ADRESS_ERR_ARG, "kirkwood needs lambdas, n >= 1, n_equil >= 0, n_samples >= 1, every >= 1");
  if (h->sys.scheme != 1) return fail(h, ADRESS_ERR_STATE, "Kirkwood integration needs energy interpolation");
  if (h->sys.cg_mode) return fail(h, ADRESS_ERR_STATE, "Kirkwood integration needs the tabulated CG energy");
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  for (int k = 0; k < n; ++k)
    if (!(lambdas[k] > 0.0 && lambdas[k] < 1.0)) return fail(h, ADRESS_ERR_ARG, "Kirkwood nodes must lie inside (0, 1)");
  adress_status st = ADRESS_OK;
  for (int k = 0; k < n && st == ADRESS_OK; ++k) {
    const double lam = lambdas[k];
    st = adress_set_uniform_lambda(h, 1, lam);
    if (st == ADRESS_OK) st = adress_compute_forces(h, nullptr);
    if (st == ADRESS_OK) st = adress_step(h, n_equil);
    double acc = 0.0;
    for (int j = 0; j < n_samples && st == ADRESS_OK; ++j) {
      double e[4];
      st = adress_step(h, every);
      if (st == ADRESS_OK) st = adress_compute_forces(h, e);
      acc += e[0] / lam - e[1] / (1.0 - lam);  // dH/dl = V_AT - V_CG
    }
    dhdl[k] = acc / ((double)n_samples * h->sys.M);
  }
  // back to position-dependent resolution, lists and forces of the current state
  const adress_status st2 = adress_set_uniform_lambda(h, 0, 0.0);
  if (st == ADRESS_OK) st = st2;
  if (st == ADRESS_OK) st = adress_compute_forces(h, nullptr);
  if (st == ADRESS_OK) st = adress_check(h);
  return st;
}

adress_status adress_set_centers(adress_handle h, const double* centers, int32_t n) {
  if (!h) return ADRESS_ERR_ARG;
  if (h->sys.n_centers == 0 || n != h->sys.n_centers || !centers)
    return fail(h, ADRESS_ERR_ARG, "set_centers needs the configured number of resolution centres");
  for (int q = 0; q < 3 * n; ++q)
    if (!(centers[q] == centers[q]) || isinf(centers[q])) return fail(h, ADRESS_ERR_ARG, "resolution centres must be finite");
  adress_status st = upload_centers(h, centers, n);
  if (st != ADRESS_OK) return st;
  // the work-item classes were decided for the old region: the next decision rebuilds the
  // lists (the flag stays set until a list build clears it)
  const int one = 1;
  CUDA_OR_FAIL(h, cudaMemcpyAsync(&h->buf.ctrl->force_rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

adress_status adress_rdf(adress_handle h, int32_t nbins, double dr, int64_t* counts) {
  if (!h) return ADRESS_ERR_ARG;
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  if (!counts || nbins < 1 || nbins > 4096 || !(dr > 0)) return fail(h, ADRESS_ERR_ARG, "need counts, 1 <= nbins <= 4096, dr > 0");
  for (const Box& B : h->boxes)
    for (int d = 0; d < 3; ++d)
      if (nbins * dr > B.halfL[d]) return fail(h, ADRESS_ERR_ARG, "nbins * dr exceeds half a box edge");
  const Sys& s = h->sys;
  if (!h->rdf_com) CUDA_OR_FAIL(h, dalloc(h, &h->rdf_com, (size_t)3 * s.M));
  const size_t n = (size_t)s.nbox * nbins;
  if (h->rdf_cap < n) {
    CUDA_OR_FAIL(h, realloc_owned(h, &h->rdf_counts, n));
    h->rdf_cap = n;
  }
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->rdf_counts, 0, sizeof(unsigned long long) * n, h->stream));
  CUDA_OR_FAIL(h, launch_export_com(s, h->buf, h->precision, h->rdf_com, nullptr, h->stream));
  CUDA_OR_FAIL(h, launch_rdf(s, h->buf, h->rdf_com, nbins, dr, h->rdf_counts, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(counts, h->rdf_counts, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
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
  if (!h || (!counts && n > 0) || n < 0 || n > h->sys.nbox * h->sys.tf_n) return ADRESS_ERR_ARG;
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
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->buf.hist, 0, sizeof(unsigned long long) * std::max(1, h->sys.nbox * h->sys.tf_n),
                                  h->stream));
  CUDA_OR_FAIL(h, cudaMemsetAsync(h->buf.nsamples, 0, sizeof(long long), h->stream));
  return ADRESS_OK;
}

adress_status adress_tf_update(adress_handle h, double alpha) {
  if (!h) return ADRESS_ERR_ARG;
  CUDA_OR_FAIL(h, launch_tf_update(h->sys, h->buf, alpha, h->stream));
  return ADRESS_OK;
}

adress_status adress_set_tf(adress_handle h, const double* tf, int32_t n) {
  if (!h || n != h->sys.nbox * h->sys.tf_n || (n > 0 && !tf)) return ADRESS_ERR_ARG;
  if (n == 0) return ADRESS_OK;
  std::vector<float> f(n);
  for (int k = 0; k < n; ++k) f[k] = (float)tf[k];
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->buf.tf64, tf, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->buf.tf32, f.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
  return ADRESS_OK;
}

adress_status adress_get_tf(adress_handle h, double* tf, int32_t n) {
  if (!h || n != h->sys.nbox * h->sys.tf_n || (n > 0 && !tf)) return ADRESS_ERR_ARG;
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

adress_status adress_set_tuning(adress_handle h, int32_t force_block, double skin) {
  if (!h) return ADRESS_ERR_ARG;
  if (force_block != 32 && force_block != 64 && force_block != 128)
    return fail(h, ADRESS_ERR_ARG, "force_block must be 32, 64 or 128");
  if (!(skin >= 0)) return fail(h, ADRESS_ERR_ARG, "skin must be >= 0");
  const double old_skin = h->sys.skin;
  adress_status st = setup_cells(h, skin);
  if (st != ADRESS_OK) {
    setup_cells(h, old_skin);
    return fail(h, st, "set_tuning: " + h->err);
  }
  h->sys.force_block = force_block;
  free_graphs(h);
  h->lists_built = false;
  return ADRESS_OK;
}

adress_status adress_get_tuning(adress_handle h, int32_t* force_block, double* skin) {
  if (!h) return ADRESS_ERR_ARG;
  if (force_block) *force_block = h->sys.force_block;
  if (skin) *skin = h->sys.skin;
  return ADRESS_OK;
}

adress_status adress_autotune(adress_handle h, int32_t nsteps, double* results, int32_t max_results,
                              int32_t* n_results) {
  if (!h) return ADRESS_ERR_ARG;
  if (nsteps < 1 || nsteps > kMaxGraphSteps) return fail(h, ADRESS_ERR_ARG, "nsteps must be in 1..100");
  if (!h->bound) return fail(h, ADRESS_ERR_STATE, "no state bound");
  if (n_results) *n_results = 0;
  Sys& s = h->sys;
  const size_t n3 = (size_t)3 * s.N;
  const size_t fbytes = n3 * (h->precision == ADRESS_FP64 ? sizeof(double) : sizeof(float));
  double *x0 = nullptr, *v0 = nullptr;
  void* f0 = nullptr;
  Ctrl c0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaMalloc(&x0, n3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&v0, n3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&f0, fbytes);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  auto cleanup = [&]() {
    cudaFree(x0);
    cudaFree(v0);
    cudaFree(f0);
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
  };
  if (e != cudaSuccess) {
    cleanup();
    return fail(h, ADRESS_ERR_CUDA, std::string("autotune scratch: ") + cudaGetErrorString(e));
  }
  cudaStream_t st = h->stream;
  e = cudaMemcpyAsync(x0, h->buf.x, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v0, h->buf.v, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f0, h->buf.f, fbytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c0, h->buf.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return fail(h, ADRESS_ERR_CUDA, std::string("autotune save: ") + cudaGetErrorString(e));
  }
  c0.err = 0;
  auto restore = [&]() -> cudaError_t {
    cudaError_t r = cudaMemcpyAsync(h->buf.x, x0, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(h->buf.v, v0, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(h->buf.f, f0, fbytes, cudaMemcpyDeviceToDevice, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(h->buf.ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    return r;
  };
  const double skin0 = h->skin0;
  const int block0 = s.force_block;
  const double cur_skin = s.skin;
  std::vector<double> skins;
  for (double m : {0.5, 0.75, 1.0, 1.25, 1.5, 2.0}) {
    const double sk = m * skin0;
    if (std::find(skins.begin(), skins.end(), sk) == skins.end()) skins.push_back(sk);
  }
  // each trial: capture + one warm-up run, then kAutotuneRuns timed runs; the trial's time
  // is their median and its spread their range
  constexpr int kAutotuneRuns = 5;
  int best_block = block0, rows = 0;
  double best_skin = cur_skin, best_med = 1e300, start_med = -1.0, start_min = 0.0;
  adress_status status = ADRESS_OK;
  for (double sk : skins) {
    for (int blk : {32, 64, 128}) {
      if (adress_set_tuning(h, blk, sk) != ADRESS_OK) continue;  // a box too small for this skin
      cudaError_t r = restore();
      if (r != cudaSuccess) {
        status = fail(h, ADRESS_ERR_CUDA, std::string("autotune restore: ") + cudaGetErrorString(r));
        break;
      }
      status = build_lists_sync(h);
      if (status == ADRESS_OK) status = launch_graph(h, nsteps, 0, 0, 0.0);  // capture + warm-up
      double t[kAutotuneRuns];
      for (int k = 0; k < kAutotuneRuns && status == ADRESS_OK; ++k) {
        if (cudaEventRecord(ev[0], st) != cudaSuccess) status = ADRESS_ERR_CUDA;
        if (status == ADRESS_OK) status = launch_graph(h, nsteps, 0, 0, 0.0);
        if (status == ADRESS_OK && cudaEventRecord(ev[1], st) != cudaSuccess) status = ADRESS_ERR_CUDA;
        float ms = 0.f;
        if (status == ADRESS_OK && cudaEventSynchronize(ev[1]) != cudaSuccess) status = ADRESS_ERR_CUDA;
        if (status == ADRESS_OK) cudaEventElapsedTime(&ms, ev[0], ev[1]);
        t[k] = ms / nsteps;
      }
      if (status == ADRESS_OK) status = adress_check(h);
      if (status != ADRESS_OK) break;
      std::sort(t, t + kAutotuneRuns);
      const double med = t[kAutotuneRuns / 2];
      if (results && rows < max_results) {
        results[5 * rows + 0] = blk;
        results[5 * rows + 1] = sk;
        results[5 * rows + 2] = med;
        results[5 * rows + 3] = t[0];
        results[5 * rows + 4] = t[kAutotuneRuns - 1];
      }
      ++rows;
      if (blk == block0 && sk == cur_skin) {
        start_med = med;
        start_min = t[0];
      }
      if (med < best_med) {
        best_med = med;
        best_block = blk;
        best_skin = sk;
      }
    }
    if (status != ADRESS_OK) break;
  }
  // keep the starting setting unless the best trial's median is below every run of it
  if (status == ADRESS_OK && start_med >= 0.0 && !(best_med < start_min)) {
    best_block = block0;
    best_skin = cur_skin;
  }
  if (n_results) *n_results = std::min(rows, std::max(0, max_results));
  adress_status st2 = adress_set_tuning(h, status == ADRESS_OK ? best_block : block0,
                                        status == ADRESS_OK ? best_skin : cur_skin);
  cudaError_t r = restore();
  cleanup();
  if (status != ADRESS_OK) return status;
  if (st2 != ADRESS_OK) return st2;
  if (r != cudaSuccess) return fail(h, ADRESS_ERR_CUDA, std::string("autotune restore: ") + cudaGetErrorString(r));
  return build_lists_sync(h);
}

adress_status adress_set_limit(adress_handle h, int32_t which, int64_t value) {
  if (!h) return ADRESS_ERR_ARG;
  switch (which) {
    case ADRESS_LIMIT_PAIR_CAPACITY:
      h->pcap_limit = value > 0 ? value : 0;
      if (h->pcap_alloc > 0) h->buf.pcap = h->pcap_limit > 0 ? std::min(h->pcap_limit, h->pcap_alloc) : h->pcap_alloc;
      break;
    case ADRESS_LIMIT_MMA_WAIT_POLLS:
      if (value > 0xFFFFFFFFll) return fail(h, ADRESS_ERR_ARG, "wait poll limit must be below 2^32");
      h->buf.wait_polls = value < 0 ? kMmaWaitPolls : (unsigned)value;
      break;
    default:
      return fail(h, ADRESS_ERR_ARG, "unknown limit");
  }
  free_graphs(h);  // captured launches hold the old values
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
  CUDA_OR_FAIL(h, dalloc(h, &h->mlp_norm, kMlpNNorm + 9));  // + 1/in_std
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
  float ext[kMlpNNorm + 9];
  memcpy(ext, norm, sizeof(float) * kMlpNNorm);
  for (int k = 0; k < 9; ++k) ext[kMlpNNorm + k] = (float)(1.0 / (double)norm[9 + k]);
  CUDA_OR_FAIL(h, cudaMemcpyAsync(h->mlp_norm, ext, sizeof(ext), cudaMemcpyHostToDevice, h->stream));
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
    if (h->sys.scheme == 1) return fail(h, ADRESS_ERR_STATE, "energy interpolation needs the tabulated CG energy");
    if (h->sys.NA != 4 && h->sys.NA != 3 && h->sys.NA != 2 && h->sys.NA != 1) return ADRESS_ERR_ARG;
    if (!h->buf.fpair) {
      CUDA_OR_FAIL(h, dalloc(h, &h->buf.fpair, (size_t)h->sys.cap * h->sys.M));
      CUDA_OR_FAIL(h, alloc_pair_buffers(h));
    }
  }
  if (h->sys.cg_mode != mode) free_graphs(h);
  h->sys.cg_mode = mode;
  // candidate pairs of the lists already built (later builds add them themselves)
  if (mode == 1 && h->lists_built) {
    CUDA_OR_FAIL(h, cudaMemsetAsync(&h->buf.ctrl->n_netc, 0, sizeof(int), h->stream));
    CUDA_OR_FAIL(h, launch_net_candidates(h->sys, h->buf, h->stream));
  }
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

adress_status adress_cg_fit(adress_handle h, double fit_dr, int32_t n_min, int32_t install, double* F, double* V) {
  if (!h || !(fit_dr > 0) || n_min < 1) return ADRESS_ERR_ARG;
  if (h->smp_n < 1) return fail(h, ADRESS_ERR_STATE, "cg_fit needs samples (adress_mlp_collect or adress_mlp_load_samples)");
  const Sys& s = h->sys;
  const double rc = s.rc_cg;
  const int nb = (int)ceil(rc / fit_dr);
  if (nb < 1 || nb > 4096) return fail(h, ADRESS_ERR_ARG, "cg_fit: rc_cg / fit_dr must be at most 4096 bins");
  const int n = s.cg_n + 1;
  unsigned long long* acc = nullptr;
  unsigned* cnt = nullptr;
  double *dF = nullptr, *dV = nullptr;
  int* npop = nullptr;
  cudaError_t e = cudaMalloc(&acc, sizeof(unsigned long long) * 2 * nb);
  if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(unsigned) * nb);
  if (e == cudaSuccess) e = cudaMalloc(&dF, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dV, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&npop, sizeof(int));
  std::vector<double> hF(n), hV(n);
  int np = 0;
  if (e == cudaSuccess)
    e = cg_fit(h->smp_feat, h->smp_target, h->smp_n, fit_dr, nb, n_min, s.cg_n, h->cg_dr, rc, acc, cnt, dF, dV,
               npop, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hF.data(), dF, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hV.data(), dV, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&np, npop, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && np > 0 && install) {
    std::vector<float2> fv(n);
    for (int k = 0; k < n; ++k) fv[k] = make_float2((float)hF[k], (float)hV[k]);
    e = cudaMemcpyAsync((void*)h->buf.cgF64, dF, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)h->buf.cgV64, dV, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void*)h->buf.cgFV32, fv.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  cudaFree(acc);
  cudaFree(cnt);
  cudaFree(dF);
  cudaFree(dV);
  cudaFree(npop);
  if (e != cudaSuccess) return fail(h, ADRESS_ERR_CUDA, std::string("cg_fit: ") + cudaGetErrorString(e));
  if (np == 0) return fail(h, ADRESS_ERR_STATE, "cg_fit: no bin holds n_min samples");
  if (F) memcpy(F, hF.data(), sizeof(double) * n);
  if (V) memcpy(V, hV.data(), sizeof(double) * n);
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
