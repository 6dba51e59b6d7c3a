// Neighbour search on the GPU: a linked-cell list over molecule centres of mass (the
// paper's linked-cell-list neighbour search, Sec. "Heterogeneous Spatial Domain
// Decomposition Algorithm", here on one GPU).  Cells are ranked in Morton order;
// molecules are counting-sorted by cell and each cell's members are then put in id order,
// so every list is deterministic; molecules are split into two work lists — high-resolution
// candidates (|dxc| < d_at + d_hy + skin/2) first, then coarse-grained molecules —
// and each work item gets a full Verlet list: partners within r_list when both are
// high-resolution items, within rc_cg + skin when either is coarse-grained (such a pair has
// weight 0 until the next build, so only the CG force, cut at rc_cg, acts between them;
// the lists stay symmetric).

// Staged candidate: centre + (molecule id | high-resolution flag in bit 31).
__device__ __forceinline__ int tag_id(int id, int hr) { return (int)((unsigned)id | ((unsigned)hr << 31)); }
__device__ __forceinline__ int id_of(int w) { return w & 0x7fffffff; }
#include <algorithm>

#include "internal.cuh"

namespace adress {

constexpr int kScanThreads = 512;
constexpr int kScanEPT = 4;
constexpr int kScanTile = kScanThreads * kScanEPT;

// Cell coordinate of a fixed-point coordinate X (X / 2^32 of the box edge): exact.
__device__ __forceinline__ int cell_of(unsigned int X, int nc) {
  return (int)(((unsigned long long)X * (unsigned long long)nc) >> 32);
}

// Cell populations.  cell_count and cell_fill are zero on entry: zeroed when allocated and
// again by k_rb_sortcell once this build no longer needs them.
__global__ void k_rb_count(const __grid_constant__ Sys s, Bufs b) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a == 0) {
    b.ctrl->n_dense = 0;
    b.ctrl->force_rebuild = 0;
    b.ctrl->n_netc = 0;
  }
  if (a >= s.M) return;
  const Box& B = box_of(s, b, a);
  const int4 C = b.com_fx[b.ctrl->parity][a];
  const int cx = cell_of((unsigned)C.x, B.nc[0]), cy = cell_of((unsigned)C.y, B.nc[1]),
            cz = cell_of((unsigned)C.z, B.nc[2]);
  const int r = b.cell_rank[B.cell0 + (cx * B.nc[1] + cy) * B.nc[2] + cz];
  b.mcell[a] = r;
  atomicAdd(&b.cell_count[r], 1);
}

// ---- exclusive scan in two launches: tile sums, then every block adds up the sums of the
// tiles before its own (at most kScanMaxTiles of them) and scans its tile ----

constexpr int kScanMaxTiles = 4096;

// Block-wide sum of v (every thread gets it).
__device__ __forceinline__ int block_sum(int v) {
  __shared__ int part[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  __syncthreads();  // part[] may still be read by a previous call
  if (lane == 0) part[w] = v;
  __syncthreads();
  int s = lane < (int)(blockDim.x >> 5) ? part[lane] : 0;
  return __reduce_add_sync(0xffffffffu, s);
}

// Block-wide exclusive scan of v; *total gets the block's sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[w] = incl;
  __syncthreads();
  if (w == 0) {
    int ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
    int wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    warp_sums[lane] = wi - ws;  // exclusive
    if (lane == 31) warp_sums[31] = wi;  // block total in the last slot (read below)
  }
  __syncthreads();
  const int excl = incl - v + (w ? warp_sums[w] : 0);
  if (total) *total = warp_sums[31];
  return excl;
}

// The warp-0 pass stores exclusive sums in slots 0..nw-1 and the total in slot 31; with 512
// threads nw = 16 <= 31, so they never clash.
static_assert(kScanThreads / 32 < 32, "scan block too large");

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int* in, int* tile_sums, int n) {
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanEPT;
  int sum = 0;
#pragma unroll
  for (int e = 0; e < kScanEPT; ++e) sum += (base + e < n) ? in[base + e] : 0;
  sum = block_sum(sum);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = sum;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* in, int* out, const int* tile_sums, int n,
                                                             int* grand) {
  int before = 0;
  for (int k = threadIdx.x; k < (int)blockIdx.x; k += blockDim.x) before += tile_sums[k];
  before = block_sum(before);
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanEPT;
  int v[kScanEPT], sum = 0;
#pragma unroll
  for (int e = 0; e < kScanEPT; ++e) {
    v[e] = (base + e < n) ? in[base + e] : 0;
    sum += v[e];
  }
  int total;
  int run = before + block_exclusive_scan(sum, &total);
#pragma unroll
  for (int e = 0; e < kScanEPT; ++e) {
    if (base + e < n) out[base + e] = run;
    run += v[e];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *grand = before + total;
}

static cudaError_t exclusive_scan(const int* in, int* out, int n, int* tmp, int* total, cudaStream_t st) {
  const int ntiles = std::max(1, ceil_div(n, kScanTile));
  if (ntiles > kScanMaxTiles) return cudaErrorInvalidValue;
  k_scan_sums<<<ntiles, kScanThreads, 0, st>>>(in, tmp, n);
  k_scan_apply<<<ntiles, kScanThreads, 0, st>>>(in, out, tmp, n, total);
  return cudaGetLastError();
}

__global__ void k_rb_fill(const __grid_constant__ Sys s, Bufs b) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= s.M) return;
  const int r = b.mcell[a];
  const int p = b.cell_start[r] + atomicAdd(&b.cell_fill[r], 1);
  b.fill_tmp[p] = a;
}

// Each molecule's position in its cell is the number of the cell's members with a smaller
// id (ids are distinct), so every cell's slice of `sorted` is in increasing id.  One thread
// per molecule; the molecule's high-resolution flag goes to the same position.  The cell
// counters, no longer needed by this build, are zeroed for the next one.
__global__ void k_rb_sortcell(const __grid_constant__ Sys s, Bufs b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  for (int c = p; c < s.ncell; c += gridDim.x * blockDim.x) {
    b.cell_count[c] = 0;
    b.cell_fill[c] = 0;
  }
  if (p >= s.M) return;
  const int a = b.fill_tmp[p], cur = b.ctrl->parity;
  const int r = b.mcell[a];
  const int ps = b.cell_start[r], pe = b.cell_start[r + 1];
  int rank = 0;
  for (int q = ps; q < pe; ++q) rank += b.fill_tmp[q] < a;
  b.sorted[ps + rank] = a;
  b.scom[ps + rank] = b.com_fx[cur][a];
  const double d = s.fp64 ? fabs(b.dxc64[cur][a]) : (double)fabsf(b.molf[cur][a].x);
  if (s.lam_uniform_on) b.flag[ps + rank] = s.lam_uniform > 0.0 ? 1 : 0;
  else b.flag[ps + rank] = d < box_of(s, b, a).d_hr + (s.fp64 ? 0.0 : 1e-3) ? 1 : 0;
}

// Work item of the molecule at sorted position k: high-resolution items first, then
// coarse-grained ones, each in sorted order (pos = exclusive scan of the flags).
__device__ __forceinline__ int item_at(const Sys& s, const Bufs& b, int k) {
  const int p = b.pos[k];
  return b.flag[k] ? p : b.pos[s.M] + (k - p);
}

// Stage candidates c0 .. c0 + nc - 1 of a 27-cell neighbourhood into st[0 .. nc): lane c < 27
// holds neighbour cell c's first sorted position `start`, its offset `pre` in the candidate
// list and the inclusive prefix `incl`.  All lanes copy, 32 candidates at a time; a lane finds
// the cell of its candidate k as the number of cells whose inclusive prefix is <= k (binary
// lifting over the monotone prefixes, five shuffles).
__device__ __forceinline__ void stage_window(const Bufs& b, int lane, int incl, int pre, int start, int c0, int nc,
                                             int4* st) {
  for (int k0 = 0; k0 < nc; k0 += 32) {
    const int k = c0 + k0 + lane;
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      const int probe = lo + step - 1;
      const int v = __shfl_sync(0xffffffffu, incl, probe < 27 ? probe : 26);
      if (probe < 27 && v <= k) lo += step;
    }
    const int c = lo < 27 ? lo : 26;
    const int s0 = __shfl_sync(0xffffffffu, start, c), p0 = __shfl_sync(0xffffffffu, pre, c);
    if (k0 + lane < nc) {
      const int g = s0 + (k - p0);
      const int4 C = b.scom[g];
      st[k0 + lane] = make_int4(C.x, C.y, C.z, tag_id(b.sorted[g], b.flag[g]));
    }
  }
  __syncwarp();
}

// One warp per cell (cells in Morton order).  Lanes 0..26 take the 27 neighbour cells in
// the fixed (ox, oy, oz) order, a warp scan gives each cell's offset in the candidate list,
// and the candidates (centre + id; each cell's members already in id order) are staged in
// shared memory once; each molecule of the cell then tests all candidates in parallel and
// appends its neighbours in candidate order with ballot/popc compaction.  A cell with more
// than kMaxCand candidates or 32 molecules is passed to k_rb_nbr_dense.
constexpr int kNbrWarps = 4;
constexpr int kMaxCand = 160;  // candidates staged at once (4 warps: 10 KB, 16 blocks per SM)
__global__ void __launch_bounds__(32 * kNbrWarps) k_rb_nbr(const __grid_constant__ Sys s, Bufs b) {
  __shared__ int4 stage[kNbrWarps][kMaxCand];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * kNbrWarps + w;
  if (r >= s.ncell) return;  // warp-uniform
  const Box& B = s.nbox > 1 ? b.boxes[b.cell_box[r]] : s.bx;
  int cnt = 0, start = 0;
  if (lane < 27) {
    const int rr = b.nbr_cells[(size_t)r * 27 + lane];
    if (rr >= 0) {
      start = b.cell_start[rr];
      cnt = b.cell_start[rr + 1] - start;
    }
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const int pre = incl - cnt;
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const int n_home = __shfl_sync(0xffffffffu, cnt, 13);
  const int home_start = __shfl_sync(0xffffffffu, start, 13);
  if (r == 0 && lane == 0) {
    const int n_hr = b.pos[s.M];
    b.ctrl->n_hr = n_hr;
    b.ctrl->n_cg = s.M - n_hr;
  }
  if (n_home == 0) return;
  if (total > kMaxCand || n_home > 32) {
    if (lane == 0) b.dense_cells[atomicAdd(&b.ctrl->n_dense, 1)] = r;
    return;
  }
  stage_window(b, lane, incl, pre, start, 0, total, stage[w]);
  // the home cell is neighbour 13: its molecules and their work items, recorded here
  const int home_pre = __shfl_sync(0xffffffffu, pre, 13);
  const int my_item = lane < n_home ? item_at(s, b, home_start + lane) : 0;
  if (lane < n_home) {
    const int a = id_of(stage[w][home_pre + lane].w);
    b.items[my_item] = a;
    b.item_of[a] = my_item;
  }
  const float rl2 = s.f.r_list2, rcl2 = s.f.r_cg_list2;
  for (int h = 0; h < n_home; ++h) {
    const int4 H = stage[w][home_pre + h];
    const int a = id_of(H.w);
    const int t = __shfl_sync(0xffffffffu, my_item, h);
    int count = 0;
    for (int k0 = 0; k0 < total; k0 += 32) {
      const int k = k0 + lane;
      bool hit = false;
      int m = 0;
      if (k < total) {
        const int4 D = stage[w][k];
        m = id_of(D.w);
        const float d0 = (float)(int)((unsigned)H.x - (unsigned)D.x) * B.fx_scale[0];
        const float d1 = (float)(int)((unsigned)H.y - (unsigned)D.y) * B.fx_scale[1];
        const float d2 = (float)(int)((unsigned)H.z - (unsigned)D.z) * B.fx_scale[2];
        hit = m != a && d0 * d0 + d1 * d1 + d2 * d2 < ((H.w & D.w) < 0 ? rl2 : rcl2);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int p = count + __popc(bal & ((1u << lane) - 1u));
        if (p < s.cap) b.nbr[(size_t)t * s.cap + p] = m;
      }
      count += __popc(bal);
    }
    if (lane == 0) {
      b.nn[t] = count < s.cap ? count : s.cap;
      b.com_ref[a] = make_int4(H.x, H.y, H.z, 0);
      if (count > s.cap) set_error(b.ctrl, ADRESS_ERR_LIST_OVERFLOW, count);
    }
  }
}

// Dense cells (those k_rb_nbr passed on): kHomeParts warps per listed cell, each taking
// batches of 32 of its molecules (one per lane), persistent grid.  Candidates (centre + id)
// are staged in shared memory kMaxCand at a time by all lanes; each lane then walks the staged
// window for its own molecule and appends its neighbours in candidate order (the order of
// the ballot compaction in k_rb_nbr): the same lists for any density.
constexpr int kHomeParts = 4;  // warps that share one dense cell's home molecules
__global__ void __launch_bounds__(32 * kNbrWarps) k_rb_nbr_dense(const __grid_constant__ Sys s, Bufs b) {
  __shared__ int4 stage[kNbrWarps][kMaxCand];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_dense = b.ctrl->n_dense;
  const int4* com = b.com_fx[b.ctrl->parity];
  const float rl2 = s.f.r_list2, rcl2 = s.f.r_cg_list2;
  // task = (dense cell, part): part j takes the home batches j, j + kHomeParts, ... so that
  // the molecules of one dense cell are shared by kHomeParts warps
  for (int task = blockIdx.x * kNbrWarps + w; task < n_dense * kHomeParts; task += gridDim.x * kNbrWarps) {
    const int di = task / kHomeParts, part = task % kHomeParts;
    const int r = b.dense_cells[di];
    const Box& B = s.nbox > 1 ? b.boxes[b.cell_box[r]] : s.bx;
    int cnt = 0, start = 0;
    if (lane < 27) {
      const int rr = b.nbr_cells[(size_t)r * 27 + lane];
      if (rr >= 0) {
        start = b.cell_start[rr];
        cnt = b.cell_start[rr + 1] - start;
      }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int pre = incl - cnt;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int n_home = __shfl_sync(0xffffffffu, cnt, 13);
    const int home_start = __shfl_sync(0xffffffffu, start, 13);
    for (int hb = part * 32; hb < n_home; hb += kHomeParts * 32) {
      // this lane's home molecule (lanes past the cell's end take none)
      const bool mine = hb + lane < n_home;
      const int kh = home_start + hb + (mine ? lane : 0);
      const int a = b.sorted[kh];
      const int4 C = com[a];
      const int H = tag_id(a, b.flag[kh]);
      const int tt = mine ? item_at(s, b, kh) : 0;
      if (mine) {
        b.items[tt] = a;
        b.item_of[a] = tt;
      }
      int count = 0;
      int* row = b.nbr + (size_t)tt * s.cap;
      for (int c0 = 0; c0 < total; c0 += kMaxCand) {
        const int nc = min(kMaxCand, total - c0);
        __syncwarp();  // the previous window is no longer read
        stage_window(b, lane, incl, pre, start, c0, nc, stage[w]);
        if (mine) {
#pragma unroll 4
          for (int k = 0; k < nc; ++k) {
            const int4 D = stage[w][k];
            const int m = id_of(D.w);
            const float d0 = (float)(int)((unsigned)C.x - (unsigned)D.x) * B.fx_scale[0];
            const float d1 = (float)(int)((unsigned)C.y - (unsigned)D.y) * B.fx_scale[1];
            const float d2 = (float)(int)((unsigned)C.z - (unsigned)D.z) * B.fx_scale[2];
            if (m != a && d0 * d0 + d1 * d1 + d2 * d2 < ((H & D.w) < 0 ? rl2 : rcl2)) {
              if (count < s.cap) row[count] = m;
              ++count;
            }
          }
        }
      }
      if (mine) {
        b.nn[tt] = count < s.cap ? count : s.cap;
        b.com_ref[a] = make_int4(C.x, C.y, C.z, 0);
        if (count > s.cap) set_error(b.ctrl, ADRESS_ERR_LIST_OVERFLOW, count);
      }
    }
  }
}

cudaError_t launch_net_candidates(const Sys& s, const Bufs& b, cudaStream_t st);

// Largest neighbour count of the last build (host-side capacity check only).
__global__ void k_max_nn(const __grid_constant__ Sys s, const Bufs b) {
  int m = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s.M; t += gridDim.x * blockDim.x) m = max(m, b.nn[t]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(&b.ctrl->max_nn, m);
}

cudaError_t launch_max_nn(const Sys& s, const Bufs& b, cudaStream_t st) {
  cudaMemsetAsync(&b.ctrl->max_nn, 0, sizeof(int), st);
  k_max_nn<<<64, 256, 0, st>>>(s, b);
  return cudaGetLastError();
}

cudaError_t device_exclusive_scan(const int* in, int* out, int n, int* tmp, int* total, cudaStream_t st) {
  return exclusive_scan(in, out, n, tmp, total, st);
}

cudaError_t launch_rebuild(const Sys& s, const Bufs& b, cudaStream_t st) {
  cudaError_t e;
  k_rb_count<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b);
  if ((e = exclusive_scan(b.cell_count, b.cell_start, s.ncell, b.scan_tmp, b.cell_start + s.ncell, st)) !=
      cudaSuccess)
    return e;
  k_rb_fill<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b);
  k_rb_sortcell<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b);
  if ((e = exclusive_scan(b.flag, b.pos, s.M, b.scan_tmp, b.pos + s.M, st)) != cudaSuccess) return e;
  k_rb_nbr<<<ceil_div(s.ncell, kNbrWarps), 32 * kNbrWarps, 0, st>>>(s, b);
  k_rb_nbr_dense<<<std::min(ceil_div((long long)s.ncell * kHomeParts, kNbrWarps), 152 * 16), 32 * kNbrWarps, 0, st>>>(s, b);
  if (s.cg_mode && b.netc) return launch_net_candidates(s, b, st);
  return cudaGetLastError();
}

}  // namespace adress
