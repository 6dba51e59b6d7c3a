// Neighbour search on the GPU: a linked-cell list over molecule centres of mass (the
// paper's linked-cell-list neighbour search, Sec. "Heterogeneous Spatial Domain
// Decomposition Algorithm", here on one GPU).  Cells are ranked in Morton order;
// molecules are counting-sorted by cell, each cell's members put in id order so every
// list is deterministic; molecules are split into two work lists — high-resolution
// candidates (|dxc| < d_at + d_hy + skin/2) first, then coarse-grained molecules —
// and each work item gets a full Verlet list of molecules within r_list.
#include "internal.cuh"

namespace adress {

constexpr int kScanThreads = 512;
constexpr int kScanEPT = 4;
constexpr int kScanTile = kScanThreads * kScanEPT;

// Cell coordinate of a fixed-point coordinate X (X / 2^32 of the box edge): exact.
__device__ __forceinline__ int cell_of(unsigned int X, int nc) {
  return (int)(((unsigned long long)X * (unsigned long long)nc) >> 32);
}

__global__ void k_rb_zero(Sys s, Bufs b) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < s.ncell; c += gridDim.x * blockDim.x) {
    b.cell_count[c] = 0;
    b.cell_fill[c] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) b.ctrl->max_nn = 0;
}

__global__ void k_rb_count(Sys s, Bufs b) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= s.M) return;
  const int4 C = b.com_fx[b.ctrl->parity][a];
  const int cx = cell_of((unsigned)C.x, s.nc[0]), cy = cell_of((unsigned)C.y, s.nc[1]),
            cz = cell_of((unsigned)C.z, s.nc[2]);
  const int r = b.cell_rank[(cx * s.nc[1] + cy) * s.nc[2] + cz];
  b.mcell[a] = r;
  atomicAdd(&b.cell_count[r], 1);
}

// ---- exclusive scan: tiles of 2048 ints, a single-block scan of tile sums, add back ----

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

// Correct block_exclusive_scan's use of slot 31: the warp-0 pass stores exclusive sums in
// slots 0..nw-1 and the total in slot 31; with 512 threads nw = 16 <= 31, so they never clash.
static_assert(kScanThreads / 32 < 32, "scan block too large");

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int* in, int* out, int* tile_sums, int n) {
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanEPT;
  int v[kScanEPT], sum = 0;
#pragma unroll
  for (int e = 0; e < kScanEPT; ++e) {
    v[e] = (base + e < n) ? in[base + e] : 0;
    sum += v[e];
  }
  int total;
  int run = block_exclusive_scan(sum, &total);
#pragma unroll
  for (int e = 0; e < kScanEPT; ++e) {
    if (base + e < n) out[base + e] = run;
    run += v[e];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block: exclusive scan of up to 1024*4 tile sums in place; total -> *grand.
__global__ void __launch_bounds__(1024) k_scan_top(int* tile_sums, int ntiles, int* grand) {
  const int base = threadIdx.x * 4;
  int v[4], sum = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    v[e] = (base + e < ntiles) ? tile_sums[base + e] : 0;
    sum += v[e];
  }
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) ws[w] = incl;
  __syncthreads();
  if (w == 0) {
    int x = ws[lane], xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    ws[lane] = xi - x;
    if (lane == 31) *grand = xi;
  }
  __syncthreads();
  int run = incl - sum + ws[w];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (base + e < ntiles) tile_sums[base + e] = run;
    run += v[e];
  }
}

__global__ void k_scan_add(int* out, const int* tile_sums, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_sums[i / kScanTile];
}

static cudaError_t exclusive_scan(const int* in, int* out, int n, int* tmp, int* total, cudaStream_t st) {
  const int ntiles = ceil_div(n, kScanTile);
  k_scan_tiles<<<ntiles, kScanThreads, 0, st>>>(in, out, tmp, n);
  k_scan_top<<<1, 1024, 0, st>>>(tmp, ntiles, total);
  k_scan_add<<<ceil_div(n, 256), 256, 0, st>>>(out, tmp, n);
  return cudaGetLastError();
}

__global__ void k_rb_fill(Sys s, Bufs b) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= s.M) return;
  const int r = b.mcell[a];
  const int p = b.cell_start[r] + atomicAdd(&b.cell_fill[r], 1);
  b.sorted[p] = a;
}

// Members of each cell in increasing molecule id (insertion sort; cells hold a few).
__global__ void k_rb_sort(Sys s, Bufs b) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s.ncell) return;
  const int lo = b.cell_start[r], hi = b.cell_start[r + 1];
  for (int i = lo + 1; i < hi; ++i) {
    const int key = b.sorted[i];
    int j = i - 1;
    while (j >= lo && b.sorted[j] > key) {
      b.sorted[j + 1] = b.sorted[j];
      --j;
    }
    b.sorted[j + 1] = key;
  }
}

__global__ void k_rb_flag(Sys s, Bufs b) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= s.M) return;
  const int a = b.sorted[k], cur = b.ctrl->parity;
  const double d = s.fp64 ? fabs(b.dxc64[cur][a]) : (double)fabsf(b.molf[cur][a].x);
  b.flag[k] = d < s.d_hr + (s.fp64 ? 0.0 : 1e-3) ? 1 : 0;
}

__global__ void k_rb_items(Sys s, Bufs b) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_hr = b.pos[s.M];
  if (k == 0) {
    b.ctrl->n_hr = n_hr;
    b.ctrl->n_cg = s.M - n_hr;
  }
  if (k >= s.M) return;
  const int a = b.sorted[k];
  const int p = b.pos[k];
  if (b.flag[k]) b.items[p] = a;
  else b.items[n_hr + (k - p)] = a;
}

// Full Verlet list of work item t: every other molecule whose centre lies within r_list,
// scanning the 27 neighbour cells (fewer when a dimension has < 3 cells) in fixed order.
__global__ void __launch_bounds__(128) k_rb_nbr(Sys s, Bufs b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.M) return;
  const int a = b.items[t];
  const int4* com = b.com_fx[b.ctrl->parity];
  const int4 C = com[a];
  b.com_ref[a] = C;
  const int c0 = cell_of((unsigned)C.x, s.nc[0]), c1 = cell_of((unsigned)C.y, s.nc[1]),
            c2 = cell_of((unsigned)C.z, s.nc[2]);
  const float rl2 = (float)s.r_list2;
  int cnt = 0;
  const int lo0 = s.nc[0] >= 3 ? -1 : 0, lo1 = s.nc[1] >= 3 ? -1 : 0, lo2 = s.nc[2] >= 3 ? -1 : 0;
  const int hi0 = s.nc[0] >= 2 ? 1 : 0, hi1 = s.nc[1] >= 2 ? 1 : 0, hi2 = s.nc[2] >= 2 ? 1 : 0;
  for (int o0 = lo0; o0 <= hi0; ++o0) {
    const int x = (c0 + o0 + s.nc[0]) % s.nc[0];
    for (int o1 = lo1; o1 <= hi1; ++o1) {
      const int y = (c1 + o1 + s.nc[1]) % s.nc[1];
      for (int o2 = lo2; o2 <= hi2; ++o2) {
        const int z = (c2 + o2 + s.nc[2]) % s.nc[2];
        const int r = b.cell_rank[(x * s.nc[1] + y) * s.nc[2] + z];
        const int pe = b.cell_start[r + 1];
        for (int p = b.cell_start[r]; p < pe; ++p) {
          const int m = b.sorted[p];
          if (m == a) continue;
          const int4 D = com[m];
          const float d0 = (float)(int)((unsigned)C.x - (unsigned)D.x) * s.fx_scale[0];
          const float d1 = (float)(int)((unsigned)C.y - (unsigned)D.y) * s.fx_scale[1];
          const float d2 = (float)(int)((unsigned)C.z - (unsigned)D.z) * s.fx_scale[2];
          if (d0 * d0 + d1 * d1 + d2 * d2 < rl2) {
            if (cnt < s.cap) b.nbr[(size_t)cnt * s.M + t] = m;
            ++cnt;
          }
        }
      }
    }
  }
  b.nn[t] = cnt < s.cap ? cnt : s.cap;
  atomicMax(&b.ctrl->max_nn, cnt);
  if (cnt > s.cap) set_error(b.ctrl, ADRESS_ERR_LIST_OVERFLOW, cnt);
}

cudaError_t launch_rebuild(const Sys& s, const Bufs& b, cudaStream_t st) {
  cudaError_t e;
  k_rb_zero<<<ceil_div(s.ncell, 256) < 1024 ? ceil_div(s.ncell, 256) : 1024, 256, 0, st>>>(s, b);
  k_rb_count<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b);
  if ((e = exclusive_scan(b.cell_count, b.cell_start, s.ncell, b.scan_tmp, b.cell_start + s.ncell, st)) !=
      cudaSuccess)
    return e;
  k_rb_fill<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b);
  k_rb_sort<<<ceil_div(s.ncell, 256), 256, 0, st>>>(s, b);
  k_rb_flag<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b);
  if ((e = exclusive_scan(b.flag, b.pos, s.M, b.scan_tmp, b.pos + s.M, st)) != cudaSuccess) return e;
  k_rb_items<<<ceil_div(s.M, 256), 256, 0, st>>>(s, b);
  k_rb_nbr<<<ceil_div(s.M, 128), 128, 0, st>>>(s, b);
  return cudaGetLastError();
}

}  // namespace adress
