// Network evaluation of the MD step on the 5th-generation tensor cores (tcgen05): the same
// 9 -> 64 -> 64 -> 1 SiLU network as k_mlp_eval, with both layers' products issued by one
// thread as 128-row MMAs whose accumulators live in tensor memory (TMEM).
//
// A tile is 64 pairs in both orderings: rows r < 64 hold pair p0 + r with features (d, s_a,
// s_b), rows r >= 64 the same pairs with (d, s_b, s_a).  Per tile: the pair buffer's bf16
// inputs go to shared memory (A1, K padded to 16), one MMA gives layer 1 into TMEM columns
// 0..63; each thread reads its row back (tcgen05.ld), adds the bias, applies SiLU and writes
// the bf16 activations to shared memory (A2); four MMAs (K = 64) give layer 2 into columns
// 64..127; each thread forms its row's output w3 . silu(z2 + b2) + b3, and the pair force is
// the mean over the two orderings times the output scale, written to both list slots.  The
// layer-2 products of a tile are issued together with the layer-1 product of the block's
// next tile, so a tile costs one barrier wait.
// Waits on the MMA completion barrier are bounded: on expiry the kernel records a timeout
// status and every block leaves after freeing its TMEM.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "umma.cuh"

namespace adress {

namespace {

constexpr int kTcH = 64, kTcIn = 9;
constexpr int kTcOb1 = kTcH * kTcIn, kTcOb2 = kTcOb1 + kTcH + kTcH * kTcH, kTcOw3 = kTcOb2 + kTcH,
              kTcOb3 = kTcOw3 + kTcH, kTcOW2 = kTcOb1 + kTcH;
constexpr uint32_t kWaitPolls = kMmaWaitPolls;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float tanh_hw(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// z sigma(z) = h (1 + tanh h) with h = z/2, as in the warp-MMA evaluation.  The products
// deliver h directly: weights and biases enter halved (exact in bf16 and fp32), and each
// bias rides in the product as three bf16 terms (hi + lo + lo2, the fp32 value to its last
// bit) against three input columns of ones.
__device__ __forceinline__ float silu_half(float h) { return fmaf(h, tanh_hw(h), h); }

__device__ __forceinline__ uint16_t bf16_bits(float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&b);
}
// v as hi + lo + lo2 in bf16 (each the rounding of what the previous ones leave)
__device__ __forceinline__ void split3(float v, uint16_t (&h)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    h[k] = bf16_bits(v);
    v -= __uint_as_float((uint32_t)h[k] << 16);
  }
}

// byte offset of the 16-byte chunk (row r, K chunk kc) in a K-major no-swizzle operand with
// nk chunks of 8 elements per row
__device__ __forceinline__ uint32_t chunk_off(int r, int kc, int nk) {
  return (uint32_t)((r >> 3) * (nk * 128) + kc * 128 + (r & 7) * 16);
}

struct __align__(1024) TcSmem {
  uint8_t A1[128 * 16 * 2];  // 128 rows x 16 bf16: 9 inputs, three ones (bias), zeros
  uint8_t A2[128 * 64 * 2];  // 128 rows x 64 bf16
  uint8_t A2b[128 * 16 * 2];  // 128 rows x 16 bf16: three ones (bias of layer 2), zeros
  uint8_t B1[64 * 16 * 2];   // W1 / 2: 64 outputs x 16 inputs (K-major), b1 / 2 in columns 9..11
  uint8_t B2[64 * 64 * 2];   // W2 / 2: 64 outputs x 64 inputs
  uint8_t B2b[64 * 16 * 2];  // b2 / 2 in columns 0..2
  float w3[kTcH];
  float y[128];
  // pair-buffer rows (inputs, list slots) of three tiles, filled by bulk copies: a tile's
  // rows land while an earlier tile is evaluated
  struct alignas(16) In {
    unsigned frag[64 * 10];
    int2 slot[64];
  } in[3];
  uint64_t mbin[3];
  uint64_t mbar;
  uint32_t taddr;
  int abort;
};

__global__ void __launch_bounds__(128, 4) k_mlp_eval_tc(const float* __restrict__ P, const float* __restrict__ norm,
                                                        const unsigned* __restrict__ pfrag,
                                                        const int2* __restrict__ pslot, const unsigned* npair,
                                                        long long pcap, long long nslot, uint32_t polls,
                                                        float* __restrict__ fpair, Ctrl* ctrl) {
  __shared__ TcSmem S;
  const int tid = threadIdx.x, warp = tid >> 5;
  // operands that do not change, in the K-major core-matrix layout: halved weights from the
  // fp32 master (the same bf16 values, halved, as the packed copies of the other kernels),
  // halved biases split in three, and the columns of ones that multiply them
  for (int i = tid; i < 64 * 8; i += 128) {  // W2 / 2: row n, chunk kc = inputs 8 kc .. 8 kc + 7
    const int n = i >> 3, kc = i & 7;
    alignas(16) uint16_t e[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) e[k] = bf16_bits(0.5f * P[kTcOW2 + n * kTcH + 8 * kc + k]);
    *reinterpret_cast<uint4*>(S.B2 + chunk_off(n, kc, 8)) = *reinterpret_cast<const uint4*>(e);
  }
  if (tid < kTcH) {
    const int n = tid;
    alignas(16) uint16_t e[16] = {};
    uint16_t hb[3];
#pragma unroll
    for (int k = 0; k < kTcIn; ++k) e[k] = bf16_bits(0.5f * P[n * kTcIn + k]);
    split3(0.5f * P[kTcOb1 + n], hb);
    e[9] = hb[0], e[10] = hb[1], e[11] = hb[2];
    *reinterpret_cast<uint4*>(S.B1 + chunk_off(n, 0, 2)) = *reinterpret_cast<const uint4*>(e);
    *reinterpret_cast<uint4*>(S.B1 + chunk_off(n, 1, 2)) = *reinterpret_cast<const uint4*>(e + 8);
    split3(0.5f * P[kTcOb2 + n], hb);
    *reinterpret_cast<uint4*>(S.B2b + chunk_off(n, 0, 2)) = make_uint4(hb[0] | (uint32_t)hb[1] << 16, hb[2], 0u, 0u);
    *reinterpret_cast<uint4*>(S.B2b + chunk_off(n, 1, 2)) = make_uint4(0u, 0u, 0u, 0u);
    S.w3[n] = P[kTcOw3 + n];
  }
  // A2b: ones in columns 0..2 of every row
  *reinterpret_cast<uint4*>(S.A2b + chunk_off(tid, 0, 2)) = make_uint4(0x3F803F80u, 0x3F80u, 0u, 0u);
  *reinterpret_cast<uint4*>(S.A2b + chunk_off(tid, 1, 2)) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    S.abort = 0;
    umma::mbar_init(&S.mbar, 1);
    for (int k = 0; k < 3; ++k) umma::mbar_init(&S.mbin[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    umma::alloc(&S.taddr, 128);
    umma::relinquish();
  }
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = S.taddr;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  const float b3 = P[kTcOb3], scale = norm[2 * kTcIn];
  constexpr uint32_t idesc = umma::idesc_bf16_f32(128, 64);
  const uint32_t a1 = umma::smem_u32(S.A1), a2 = umma::smem_u32(S.A2), a2b = umma::smem_u32(S.A2b),
                 bw1 = umma::smem_u32(S.B1), bw2 = umma::smem_u32(S.B2), bw2b = umma::smem_u32(S.B2b);
  // the pair buffer holds at most pcap pairs: a count beyond it (an overflow the feature
  // kernel has reported) is clamped so that no tile reads past the buffer
  const long long np = min((long long)*npair, pcap);
  const long long ntiles = (np + 63) / 64;
  uint32_t phase = 0;

  // The block's j-th tile is blockIdx.x + j gridDim.x; its pair-buffer rows go to in[j % 3]
  // (barrier phase (j / 3) & 1).  Thread 0 requests tile j + 2 once every thread is past
  // tile j - 1, the last user of that buffer.  The copy of a ragged last tile is rounded up to
  // 16 bytes (the buffers are allocated with that much slack); its missing rows read as zero.
  long long issued = 0, landed = 0;  // tiles requested (thread 0) / seen landed (each thread)
  auto request = [&](long long j) {
    const long long p0 = ((long long)blockIdx.x + j * gridDim.x) * 64;
    if (p0 >= np) return;
    const uint32_t n = (uint32_t)min(64LL, np - p0);
    const uint32_t bf = (40u * n + 15u) & ~15u, bs = (8u * n + 15u) & ~15u;
    uint64_t* mb = &S.mbin[j % 3];
    umma::mbar_arrive_expect_tx(mb, bf + bs);
    umma::bulk_g2s(S.in[j % 3].frag, pfrag + p0 * 10, bf, mb);
    umma::bulk_g2s(S.in[j % 3].slot, pslot + p0, bs, mb);
    issued = j + 1;
  };
  // inputs of tile j's row tid: pair p0 + (tid & 63), ordering tid >> 6 (words 5u .. 5u + 4),
  // then ones in columns 9..11 (the bias terms of W1's chunk 1)
  auto stage_inputs = [&](long long j) {
    if (umma::mbar_wait(&S.mbin[j % 3], (uint32_t)((j / 3) & 1), kWaitPolls))
      landed = j + 1;
    else
      atomicExch(&S.abort, 1);
    const long long p = ((long long)blockIdx.x + j * gridDim.x) * 64 + (tid & 63);
    const int u = tid >> 6;
    uint4 c0 = make_uint4(0u, 0u, 0u, 0u), c1 = make_uint4(0x3F800000u, 0x3F803F80u, 0u, 0u);
    if (p < np) {
      const unsigned* r = S.in[j % 3].frag + (tid & 63) * 10 + 5 * u;
      c0 = make_uint4(r[0], r[1], r[2], r[3]);
      c1.x |= r[4] & 0xFFFFu;
    }
    *reinterpret_cast<uint4*>(S.A1 + chunk_off(tid, 0, 2)) = c0;
    *reinterpret_cast<uint4*>(S.A1 + chunk_off(tid, 1, 2)) = c1;
  };
  // make the shared-memory writes and TMEM reads of all threads precede what thread 0 issues
  auto sync_for_issue = [&]() {
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
  };
  // wait for every product issued so far; false once any thread of the block gave up
  // (`polls` bounds these waits; the drain wait before the TMEM is freed keeps kWaitPolls)
  auto wait_products = [&]() -> bool {
    if (!umma::mbar_wait(&S.mbar, phase, polls)) atomicExch(&S.abort, 1);
    phase ^= 1u;
    umma::fence_after_sync();
    __syncthreads();
    return S.abort == 0;
  };

  // pipeline: layer 1 of the first tile alone, then per tile one barrier wait for layer 2
  // of this tile together with layer 1 of the next
  long long tile = blockIdx.x, j = 0;
  if (tid == 0) {
    request(0);
    request(1);
  }
  if (tile < ntiles) {
    stage_inputs(0);
    sync_for_issue();
    if (tid == 0) {
      umma::fence_after_sync();
      umma::mma_bf16(tmem, umma::desc(a1, 128, 256), umma::desc(bw1, 128, 256), idesc, 0u);
      umma::commit(&S.mbar);
    }
    if (!wait_products()) tile = ntiles;
  }
  while (tile < ntiles) {
    const long long p0 = tile * 64, next = tile + gridDim.x;
    const bool has_next = next < ntiles;
    // layer 1 (TMEM columns 0..63) -> SiLU -> bf16 activations of row tid
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float z[32];
      umma::ld32(tmem + lane_base + 32 * half, z);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const auto act = [&](int k) { return silu_half(z[8 * c + k]); };
        const uint4 q = make_uint4(pack2(act(0), act(1)), pack2(act(2), act(3)), pack2(act(4), act(5)),
                                   pack2(act(6), act(7)));
        *reinterpret_cast<uint4*>(S.A2 + chunk_off(tid, 4 * half + c, 8)) = q;
      }
    }
    if (has_next) stage_inputs(j + 1);
    sync_for_issue();
    if (tid == 0) {
      request(j + 2);
      umma::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma::mma_bf16(tmem + 64, umma::desc(a2 + 256 * kk, 128, 1024), umma::desc(bw2 + 256 * kk, 128, 1024), idesc,
                       kk > 0 ? 1u : 0u);
      umma::mma_bf16(tmem + 64, umma::desc(a2b, 128, 256), umma::desc(bw2b, 128, 256), idesc, 1u);
      if (has_next) umma::mma_bf16(tmem, umma::desc(a1, 128, 256), umma::desc(bw1, 128, 256), idesc, 0u);
      umma::commit(&S.mbar);
    }
    if (!wait_products()) break;
    // layer 2 (columns 64..127) -> SiLU -> output weight: this row's network output
    float acc = 0.f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float z[32];
      umma::ld32(tmem + lane_base + 64 + 32 * half, z);
#pragma unroll
      for (int c = 0; c < 32; ++c) acc = fmaf(S.w3[32 * half + c], silu_half(z[c]), acc);
    }
    S.y[tid] = acc + b3;
    __syncthreads();
    if (tid < 64 && p0 + tid < np) {
      const float fv = 0.5f * scale * (S.y[tid] + S.y[tid + 64]);
      const int2 sl = S.in[j % 3].slot[tid];
      if (sl.x >= 0 && sl.x < nslot) fpair[sl.x] = fv;
      if (sl.y >= 0 && sl.y < nslot) fpair[sl.y] = fv;
    }
    tile = next;
    ++j;
  }
  if (S.abort) {
    if (tid == 0) set_error(ctrl, ADRESS_ERR_TIMEOUT, 2);
    // give the products still in flight a second bounded wait before their TMEM is freed
    umma::mbar_wait(&S.mbar, phase ^ 1u, kWaitPolls);
  }
  // bulk copies still in flight (after an abort) land before the block's shared memory is
  // released
  if (tid == 0)
    for (long long k = landed; k < issued; ++k) umma::mbar_wait(&S.mbin[k % 3], (uint32_t)((k / 3) & 1), kWaitPolls);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::dealloc(tmem, 128);
}

}  // namespace

cudaError_t launch_mlp_eval_tc(const Sys& s, const MlpDevArgs& a, const Bufs& b, float* fpair, cudaStream_t st) {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    // four blocks per SM (the register bound of the kernel keeps a fifth out), 4 x 128 TMEM
    // columns = all 512; two or three per SM were 20 and 7 us slower per evaluation
    grid = 4 * sms;
  }
  k_mlp_eval_tc<<<grid, 128, 0, st>>>(a.P, a.norm, b.pfrag, b.pslot, b.npair, b.pcap,
                                       (long long)s.M * s.cap, b.wait_polls, fpair,
                                       b.ctrl);
  return cudaGetLastError();
}

}  // namespace adress
