// Learned coarse-grained pair force: a 9 -> 64 -> 64 -> 1 SiLU network of the COM
// distance and eight orientation invariants, trained by force matching on atomistic pair
// forces, replacing the tabulated F^CG of Eq. 1 (Sec. "Force interpolation": the CG force
// acts between the molecules' centres of mass).
//
// Features of a pair (a, b): e = (R_b - R_a)/d, d = |R_b - R_a|; the four projections of
// a's atoms on e and of b's atoms on -e, each sorted ascending.  Target: the atomistic
// force on a from b projected on -e (positive = repulsive).  Network: x = (feat - mean)/std,
// h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), y = w3.h2 + b3, force = out_scale * y; the
// pair force is the mean over the two orderings of (s_a, s_b), so it is the same for both
// molecules and Newton's third law holds exactly.
//
// Tensor cores: warp-level BF16 mma (m16n8k16) with FP32 accumulation.  The layer-1
// accumulators of a 16-sample tile are, element for element, the A fragments of layer 2,
// so activations never leave registers in the forward pass.  Weights are BF16 copies of
// FP32 master weights; the backward pass propagates deltas with the same tensor-core
// product and forms the weight gradients as BF16 tensor-core products over the samples of
// a block, with FP32 accumulation, per-block partials and a fixed-order reduction.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <stdlib.h>
#include <string.h>

#include "internal.cuh"

namespace adress {

cudaError_t launch_mlp_eval_tc(const Sys& s, const MlpDevArgs& a, const Bufs& b, float* fpair, cudaStream_t st);

// ---------------- parameters ----------------------------------------------------------
// Flat FP32 master vector: [W1 (64 x 9) | b1 (64) | W2 (64 x 64) | b2 (64) | w3 (64) | b3]
constexpr int kH = 64;
constexpr int kIn = 9;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH, ob3 = ow3 + kH;
constexpr int kNPar = ob3 + 1;  // 4865
constexpr int kGradStride = kMlpGradStride;  // per-block partial record (params + loss, padded)
static_assert(kNPar == kMlpNPar, "parameter layout");

struct MlpDev {
  const float* P;       // master parameters (FP32)
  const unsigned* W1p;  // W1 as bf16 pairs, K padded to 16: [64][8]
  const unsigned* W2p;  // W2 as bf16 pairs: [64 out][32 in-pairs]
  const unsigned* W2Tp; // W2 transposed as bf16 pairs: [64 in][32 out-pairs]
  const float* norm;    // in_mean[9], in_std[9], out_scale, 1/in_std[9]
};

// What the forward pass reads: operand copies, biases, output weights and the input
// normalisation, in global memory or staged in shared memory.
struct MlpView {
  const unsigned* W1p;
  const unsigned* W2p;
  const float *b1, *b2, *w3;
  float b3;
  const float* mean;
  const float* inv_std;
};
// Loads of the view's arrays.  From shared memory they go through volatile ld.shared so
// that the compiler reloads them per tile instead of hoisting all 80 words per lane out of
// the pair loop into registers (which would cut the kernel's occupancy to a quarter).
struct LdGlobal {
  static __device__ __forceinline__ unsigned u(const unsigned* p) { return *p; }
  static __device__ __forceinline__ float f(const float* p) { return *p; }
};
struct LdShared {
  static __device__ __forceinline__ unsigned u(const unsigned* p) {
    unsigned v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
  }
  static __device__ __forceinline__ float f(const float* p) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
  }
};

__device__ __forceinline__ MlpView view_of(const MlpDev& m) {
  return MlpView{m.W1p, m.W2p, m.P + ob1, m.P + ob2, m.P + ow3, m.P[ob3], m.norm, m.norm + 2 * kIn + 1};
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}
// SiLU z sigma(z) and its derivative, sigma(z) = 1 / (1 + e^-z) from the hardware base-2
// exponential and reciprocal approximations (a few ulp, far below the bfloat16 resolution of
// the activations; e^-z = inf gives sigma = 0).  An IEEE division here was most of the
// instructions of the network evaluation.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// e^-z = 2^(-z log2 e)
__device__ __forceinline__ float exp_neg(float z) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(z * -1.4426950408889634f));
  return r;
}
__device__ __forceinline__ float silu_f(float z) { return z * rcp_approx(1.0f + exp_neg(z)); }
// The MD evaluation's SiLU: z sigma(z) = (z/2) (1 + tanh(z/2)) with the hardware tanh
// approximation (absolute error about 2^-11): one special-function operation instead of two,
// the pipe that bounds the network evaluation; the error stays below the bfloat16 resolution
// the first layer's activations are rounded to.
__device__ __forceinline__ float tanh_approx(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float silu_t(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_approx(h), h);
}
__device__ __forceinline__ float dsilu_f(float z) {
  const float sg = rcp_approx(1.0f + exp_neg(z));
  return sg * (1.0f + z * (1.0f - sg));
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + C, FP32 accumulate.
__device__ __forceinline__ void mma16816(float d[4], const unsigned a[4], unsigned b0, unsigned b1, const float c[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%11,%12,%13};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]),
        "f"(c[3]));
}

// Forward of one 16-sample tile held by a warp.  Lane = 4 g + tg; the lane's A fragment of
// the normalised inputs covers rows g, g+8 and columns 2tg, 2tg+1, 2tg+8, 2tg+9.
// Outputs: z1, z2 (pre-activations, D layout: n-tile j holds columns 8j + 2tg, +1 of rows g
// (elements 0, 1) and g+8 (elements 2, 3)), y for rows g and g+8 (all four lanes of a group).
struct Tile {
  float z1[8][4], z2[8][4];
};

template <class LD = LdGlobal>
__device__ __forceinline__ void tile_forward(const MlpView& m, const unsigned ax[4], Tile& T, float& y_g, float& y_g8) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  const float* b1 = m.b1;
  const float* b2 = m.b2;
  const float* w3 = m.w3;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int o = 8 * j + 2 * tg;
    const float c0 = LD::f(b1 + o), c1 = LD::f(b1 + o + 1);
    const float c[4] = {c0, c1, c0, c1};
    mma16816(T.z1[j], ax, LD::u(m.W1p + (8 * j + g) * 8 + tg), LD::u(m.W1p + (8 * j + g) * 8 + tg + 4), c);
  }
  unsigned a2[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    a2[kk][0] = pack_bf16(silu_f(T.z1[2 * kk][0]), silu_f(T.z1[2 * kk][1]));
    a2[kk][1] = pack_bf16(silu_f(T.z1[2 * kk][2]), silu_f(T.z1[2 * kk][3]));
    a2[kk][2] = pack_bf16(silu_f(T.z1[2 * kk + 1][0]), silu_f(T.z1[2 * kk + 1][1]));
    a2[kk][3] = pack_bf16(silu_f(T.z1[2 * kk + 1][2]), silu_f(T.z1[2 * kk + 1][3]));
  }
  float pg = 0.f, pg8 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int o = 8 * j + 2 * tg;
    const float c0 = LD::f(b2 + o), c1 = LD::f(b2 + o + 1);
    float c[4] = {c0, c1, c0, c1};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma16816(c, a2[kk], LD::u(m.W2p + (8 * j + g) * 32 + 8 * kk + tg), LD::u(m.W2p + (8 * j + g) * 32 + 8 * kk + tg + 4), c);
#pragma unroll
    for (int e = 0; e < 4; ++e) T.z2[j][e] = c[e];
    const float w0 = LD::f(w3 + o), w1 = LD::f(w3 + o + 1);
    pg += w0 * silu_f(c[0]) + w1 * silu_f(c[1]);
    pg8 += w0 * silu_f(c[2]) + w1 * silu_f(c[3]);
  }
  pg += __shfl_xor_sync(0xffffffffu, pg, 1);
  pg += __shfl_xor_sync(0xffffffffu, pg, 2);
  pg8 += __shfl_xor_sync(0xffffffffu, pg8, 1);
  pg8 += __shfl_xor_sync(0xffffffffu, pg8, 2);
  y_g = pg + m.b3;
  y_g8 = pg8 + m.b3;
}

// Forward of one 16-sample tile returning only the outputs (no pre-activations kept), with
// the layer-2 column tiles evaluated two at a time to bound the registers in flight.
template <class LD>
__device__ __forceinline__ void tile_forward_y(const MlpView& m, const unsigned ax[4], float& y_g, float& y_g8) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  unsigned a2[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    float z[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * kk + h;
      const int o = 8 * j + 2 * tg;
      const float c0 = LD::f(m.b1 + o), c1 = LD::f(m.b1 + o + 1);
      const float c[4] = {c0, c1, c0, c1};
      mma16816(z[h], ax, LD::u(m.W1p + (8 * j + g) * 8 + tg), LD::u(m.W1p + (8 * j + g) * 8 + tg + 4), c);
    }
    a2[kk][0] = pack_bf16(silu_f(z[0][0]), silu_f(z[0][1]));
    a2[kk][1] = pack_bf16(silu_f(z[0][2]), silu_f(z[0][3]));
    a2[kk][2] = pack_bf16(silu_f(z[1][0]), silu_f(z[1][1]));
    a2[kk][3] = pack_bf16(silu_f(z[1][2]), silu_f(z[1][3]));
  }
  float pg = 0.f, pg8 = 0.f;
#pragma unroll 2
  for (int j = 0; j < 8; ++j) {
    const int o = 8 * j + 2 * tg;
    const float c0 = LD::f(m.b2 + o), c1 = LD::f(m.b2 + o + 1);
    float c[4] = {c0, c1, c0, c1};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma16816(c, a2[kk], LD::u(m.W2p + (8 * j + g) * 32 + 8 * kk + tg),
               LD::u(m.W2p + (8 * j + g) * 32 + 8 * kk + tg + 4), c);
    const float w0 = LD::f(m.w3 + o), w1 = LD::f(m.w3 + o + 1);
    pg += w0 * silu_f(c[0]) + w1 * silu_f(c[1]);
    pg8 += w0 * silu_f(c[2]) + w1 * silu_f(c[3]);
  }
  pg += __shfl_xor_sync(0xffffffffu, pg, 1);
  pg += __shfl_xor_sync(0xffffffffu, pg, 2);
  pg8 += __shfl_xor_sync(0xffffffffu, pg8, 1);
  pg8 += __shfl_xor_sync(0xffffffffu, pg8, 2);
  y_g = pg + m.b3;
  y_g8 = pg8 + m.b3;
}

// Forward of two 16-sample tiles at once (the two orderings of 16 pairs): every weight
// fragment is loaded once (as one 64-bit word from the staged W1q / W2q layouts) and feeds
// both tiles' products.  Outputs y for rows g and g + 8 of each tile.
struct MlpViewQ {
  const uint2* W1q;  // [(8 j + g) * 4 + tg] = W1p words tg, tg + 4 of row 8 j + g
  const uint2* W2q;  // [(8 j + g) * 16 + 4 kk + tg] = W2p words 8 kk + tg, 8 kk + tg + 4
  const float *b1, *b2, *w3;
  float b3;
};
__device__ __forceinline__ uint2 lds_u2(const uint2* p) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}
__device__ __forceinline__ void tile_forward_y2(const MlpViewQ& m, const unsigned ax0[4], const unsigned ax1[4],
                                                float y[2][2]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  unsigned a2[2][4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    float z[2][2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * kk + h;
      const int o = 8 * j + 2 * tg;
      const float c0 = LdShared::f(m.b1 + o), c1 = LdShared::f(m.b1 + o + 1);
      const float c[4] = {c0, c1, c0, c1};
      const uint2 wq = lds_u2(m.W1q + (8 * j + g) * 4 + tg);
      mma16816(z[0][h], ax0, wq.x, wq.y, c);
      mma16816(z[1][h], ax1, wq.x, wq.y, c);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      a2[u][kk][0] = pack_bf16(silu_t(z[u][0][0]), silu_t(z[u][0][1]));
      a2[u][kk][1] = pack_bf16(silu_t(z[u][0][2]), silu_t(z[u][0][3]));
      a2[u][kk][2] = pack_bf16(silu_t(z[u][1][0]), silu_t(z[u][1][1]));
      a2[u][kk][3] = pack_bf16(silu_t(z[u][1][2]), silu_t(z[u][1][3]));
    }
  }
  float p[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 2
  for (int j = 0; j < 8; ++j) {
    const int o = 8 * j + 2 * tg;
    const float c0 = LdShared::f(m.b2 + o), c1 = LdShared::f(m.b2 + o + 1);
    float c[2][4] = {{c0, c1, c0, c1}, {c0, c1, c0, c1}};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint2 wq = lds_u2(m.W2q + (8 * j + g) * 16 + 4 * kk + tg);
      mma16816(c[0], a2[0][kk], wq.x, wq.y, c[0]);
      mma16816(c[1], a2[1][kk], wq.x, wq.y, c[1]);
    }
    const float w0 = LdShared::f(m.w3 + o), w1 = LdShared::f(m.w3 + o + 1);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      p[u][0] += w0 * silu_t(c[u][0]) + w1 * silu_t(c[u][1]);
      p[u][1] += w0 * silu_t(c[u][2]) + w1 * silu_t(c[u][3]);
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float v = p[u][r];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      y[u][r] = v + m.b3;
    }
}

// A fragment of normalised inputs from a [16][9] feature tile (row stride 9 floats).
template <class LD = LdGlobal>
__device__ __forceinline__ void input_fragment(const MlpView& m, const float* f16x9, unsigned ax[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  float v[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int k = (c < 2 ? 2 * tg + c : 2 * tg + 8 + (c - 2));
      const int row = g + 8 * r;
      v[r][c] = k < kIn ? (f16x9[row * kIn + k] - LD::f(m.mean + k)) * LD::f(m.inv_std + k) : 0.f;
    }
  ax[0] = pack_bf16(v[0][0], v[0][1]);
  ax[1] = pack_bf16(v[1][0], v[1][1]);
  ax[2] = pack_bf16(v[0][2], v[0][3]);
  ax[3] = pack_bf16(v[1][2], v[1][3]);
}

// ---------------- forward over a feature array ------------------------------------------
// y[n] = network output (before out_scale); rows past n are padding.
__global__ void __launch_bounds__(128) k_mlp_forward(MlpDev m, const float* __restrict__ feat, long long n,
                                                     float* __restrict__ y) {
  __shared__ float tile[4][16 * kIn];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = ((long long)blockIdx.x * 4 + w) * 16;
  for (int e = lane; e < 16 * kIn; e += 32) {
    const long long s = base + e / kIn;
    tile[w][e] = s < n ? feat[s * kIn + e % kIn] : 0.f;
  }
  __syncwarp();
  const MlpView mv = view_of(m);
  unsigned ax[4];
  input_fragment(mv, tile[w], ax);
  float yg, yg8;
  tile_forward_y<LdGlobal>(mv, ax, yg, yg8);
  const int g = lane >> 2, tg = lane & 3;
  if (tg == 0) {
    if (base + g < n) y[base + g] = yg;
    if (base + g + 8 < n) y[base + g + 8] = yg8;
  }
}

// ---------------- loss and gradient of one block of 64 samples ---------------------------
// Writes the block's partial gradient (sum over its samples of dL/dparam with
// L = (1/n_total) sum (y - t/out_scale)^2) and loss partial to part[blockIdx.x].
__global__ void __launch_bounds__(128) k_mlp_grad(MlpDev m, const float* __restrict__ feat,
                                                  const float* __restrict__ target, long long n, long long n_total,
                                                  float* __restrict__ part) {
  __shared__ float ftile[4][16 * kIn];
  __shared__ __nv_bfloat16 sd2[64][kH + 8];  // delta of layer 2 [sample][out]
  __shared__ __nv_bfloat16 sh1[64][kH + 8];  // h1 [sample][in]
  __shared__ __nv_bfloat16 sd1[64][kH + 8];  // delta of layer 1 [sample][out]
  __shared__ __nv_bfloat16 sx[64][16 + 8];   // normalised inputs [sample][k]
  __shared__ float sb[4][3][kH];             // per-warp partials of gb1, gb2, gw3
  __shared__ float sl[4][2];                 // per-warp gb3 and loss
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  const long long base = ((long long)blockIdx.x * 4 + w) * 16;
  const float inv_scale = 1.0f / m.norm[2 * kIn];
  for (int e = lane; e < 16 * kIn; e += 32) {
    const long long s = base + e / kIn;
    ftile[w][e] = s < n ? feat[s * kIn + e % kIn] : 0.f;
  }
  __syncwarp();
  const MlpView mv = view_of(m);
  unsigned ax[4];
  input_fragment(mv, ftile[w], ax);
  Tile T;
  float yg, yg8;
  tile_forward(mv, ax, T, yg, yg8);
  const bool vg = base + g < n, vg8 = base + g + 8 < n;
  const float rg = vg ? yg - target[base + g] * inv_scale : 0.f;
  const float rg8 = vg8 ? yg8 - target[base + g + 8] * inv_scale : 0.f;
  const float dyg = 2.f * rg / (float)n_total, dyg8 = 2.f * rg8 / (float)n_total;
  // layer 2 deltas, bias / w3 partials, and stores for the weight-gradient products
  const float* w3 = m.P + ow3;
  float pb2[8][2], pw3[8][2];
  unsigned ad2[4][4];
  float d2v[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int o = 8 * j + 2 * tg;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float dy = e < 2 ? dyg : dyg8;
      d2v[j][e] = dy * w3[o + (e & 1)] * dsilu_f(T.z2[j][e]);
    }
    pb2[j][0] = d2v[j][0] + d2v[j][2];
    pb2[j][1] = d2v[j][1] + d2v[j][3];
    pw3[j][0] = dyg * silu_f(T.z2[j][0]) + dyg8 * silu_f(T.z2[j][2]);
    pw3[j][1] = dyg * silu_f(T.z2[j][1]) + dyg8 * silu_f(T.z2[j][3]);
    const int r0 = 16 * w + g;
    sd2[r0][o] = __float2bfloat16_rn(d2v[j][0]);
    sd2[r0][o + 1] = __float2bfloat16_rn(d2v[j][1]);
    sd2[r0 + 8][o] = __float2bfloat16_rn(d2v[j][2]);
    sd2[r0 + 8][o + 1] = __float2bfloat16_rn(d2v[j][3]);
    sh1[r0][o] = __float2bfloat16_rn(silu_f(T.z1[j][0]));
    sh1[r0][o + 1] = __float2bfloat16_rn(silu_f(T.z1[j][1]));
    sh1[r0 + 8][o] = __float2bfloat16_rn(silu_f(T.z1[j][2]));
    sh1[r0 + 8][o + 1] = __float2bfloat16_rn(silu_f(T.z1[j][3]));
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    ad2[kk][0] = pack_bf16(d2v[2 * kk][0], d2v[2 * kk][1]);
    ad2[kk][1] = pack_bf16(d2v[2 * kk][2], d2v[2 * kk][3]);
    ad2[kk][2] = pack_bf16(d2v[2 * kk + 1][0], d2v[2 * kk + 1][1]);
    ad2[kk][3] = pack_bf16(d2v[2 * kk + 1][2], d2v[2 * kk + 1][3]);
  }
  // delta of layer 1 = (delta2 W2) * silu'(z1): a 16 x 64 x 64 tensor-core product
  float pb1[8][2];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma16816(c, ad2[kk], m.W2Tp[(8 * j + g) * 32 + 8 * kk + tg], m.W2Tp[(8 * j + g) * 32 + 8 * kk + tg + 4], c);
    const int o = 8 * j + 2 * tg;
#pragma unroll
    for (int e = 0; e < 4; ++e) c[e] *= dsilu_f(T.z1[j][e]);
    pb1[j][0] = c[0] + c[2];
    pb1[j][1] = c[1] + c[3];
    const int r0 = 16 * w + g;
    sd1[r0][o] = __float2bfloat16_rn(c[0]);
    sd1[r0][o + 1] = __float2bfloat16_rn(c[1]);
    sd1[r0 + 8][o] = __float2bfloat16_rn(c[2]);
    sd1[r0 + 8][o + 1] = __float2bfloat16_rn(c[3]);
  }
  // normalised inputs (bf16) for the W1 gradient
  {
    const int r0 = 16 * w + g;
    const __nv_bfloat162* a0 = reinterpret_cast<const __nv_bfloat162*>(&ax[0]);
    const __nv_bfloat162* a1 = reinterpret_cast<const __nv_bfloat162*>(&ax[1]);
    const __nv_bfloat162* a2 = reinterpret_cast<const __nv_bfloat162*>(&ax[2]);
    const __nv_bfloat162* a3 = reinterpret_cast<const __nv_bfloat162*>(&ax[3]);
    sx[r0][2 * tg] = a0->x;
    sx[r0][2 * tg + 1] = a0->y;
    sx[r0 + 8][2 * tg] = a1->x;
    sx[r0 + 8][2 * tg + 1] = a1->y;
    sx[r0][2 * tg + 8] = a2->x;
    sx[r0][2 * tg + 9] = a2->y;
    sx[r0 + 8][2 * tg + 8] = a3->x;
    sx[r0 + 8][2 * tg + 9] = a3->y;
  }
  // warp reductions of the bias / w3 partials over the 16 samples (across groups g)
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int off = 4; off < 32; off <<= 1) {
        pb1[j][e] += __shfl_xor_sync(0xffffffffu, pb1[j][e], off);
        pb2[j][e] += __shfl_xor_sync(0xffffffffu, pb2[j][e], off);
        pw3[j][e] += __shfl_xor_sync(0xffffffffu, pw3[j][e], off);
      }
  if (g == 0)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        sb[w][0][8 * j + 2 * tg + e] = pb1[j][e];
        sb[w][1][8 * j + 2 * tg + e] = pb2[j][e];
        sb[w][2][8 * j + 2 * tg + e] = pw3[j][e];
      }
  float pgb3 = (tg == 0) ? dyg + dyg8 : 0.f, pl = (tg == 0) ? rg * rg + rg8 * rg8 : 0.f;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    pgb3 += __shfl_xor_sync(0xffffffffu, pgb3, off);
    pl += __shfl_xor_sync(0xffffffffu, pl, off);
  }
  if (lane == 0) {
    sl[w][0] = pgb3;
    sl[w][1] = pl;
  }
  __syncthreads();

  float* out = part + (size_t)blockIdx.x * kGradStride;
  // W2 gradient rows o in [16w, 16w + 16): sum over the block's 64 samples of d2[s][o] h1[s][k]
  {
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
    const int o0 = 16 * w;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int s0 = 16 * ks;
      unsigned a[4];
      a[0] = pack_bf16(__bfloat162float(sd2[s0 + 2 * tg][o0 + g]), __bfloat162float(sd2[s0 + 2 * tg + 1][o0 + g]));
      a[1] = pack_bf16(__bfloat162float(sd2[s0 + 2 * tg][o0 + g + 8]), __bfloat162float(sd2[s0 + 2 * tg + 1][o0 + g + 8]));
      a[2] = pack_bf16(__bfloat162float(sd2[s0 + 2 * tg + 8][o0 + g]), __bfloat162float(sd2[s0 + 2 * tg + 9][o0 + g]));
      a[3] = pack_bf16(__bfloat162float(sd2[s0 + 2 * tg + 8][o0 + g + 8]),
                       __bfloat162float(sd2[s0 + 2 * tg + 9][o0 + g + 8]));
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const unsigned b0 = pack_bf16(__bfloat162float(sh1[s0 + 2 * tg][8 * j + g]),
                                      __bfloat162float(sh1[s0 + 2 * tg + 1][8 * j + g]));
        const unsigned b1 = pack_bf16(__bfloat162float(sh1[s0 + 2 * tg + 8][8 * j + g]),
                                      __bfloat162float(sh1[s0 + 2 * tg + 9][8 * j + g]));
        mma16816(acc[j], a, b0, b1, acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * j + 2 * tg;
      out[oW2 + (o0 + g) * kH + k] = acc[j][0];
      out[oW2 + (o0 + g) * kH + k + 1] = acc[j][1];
      out[oW2 + (o0 + g + 8) * kH + k] = acc[j][2];
      out[oW2 + (o0 + g + 8) * kH + k + 1] = acc[j][3];
    }
  }
  // W1 gradient rows o in [16w, 16w + 16): sum over samples of d1[s][o] x[s][k], k < 9
  {
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    const int o0 = 16 * w;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int s0 = 16 * ks;
      unsigned a[4];
      a[0] = pack_bf16(__bfloat162float(sd1[s0 + 2 * tg][o0 + g]), __bfloat162float(sd1[s0 + 2 * tg + 1][o0 + g]));
      a[1] = pack_bf16(__bfloat162float(sd1[s0 + 2 * tg][o0 + g + 8]), __bfloat162float(sd1[s0 + 2 * tg + 1][o0 + g + 8]));
      a[2] = pack_bf16(__bfloat162float(sd1[s0 + 2 * tg + 8][o0 + g]), __bfloat162float(sd1[s0 + 2 * tg + 9][o0 + g]));
      a[3] = pack_bf16(__bfloat162float(sd1[s0 + 2 * tg + 8][o0 + g + 8]),
                       __bfloat162float(sd1[s0 + 2 * tg + 9][o0 + g + 8]));
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const unsigned b0 = pack_bf16(__bfloat162float(sx[s0 + 2 * tg][8 * j + g]),
                                      __bfloat162float(sx[s0 + 2 * tg + 1][8 * j + g]));
        const unsigned b1 = pack_bf16(__bfloat162float(sx[s0 + 2 * tg + 8][8 * j + g]),
                                      __bfloat162float(sx[s0 + 2 * tg + 9][8 * j + g]));
        mma16816(acc[j], a, b0, b1, acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 8 * j + 2 * tg + (e & 1), o = o0 + g + (e >= 2 ? 8 : 0);
        if (k < kIn) out[oW1 + o * kIn + k] = acc[j][e];
      }
  }
  for (int o = threadIdx.x; o < kH; o += blockDim.x) {
    out[ob1 + o] = sb[0][0][o] + sb[1][0][o] + sb[2][0][o] + sb[3][0][o];
    out[ob2 + o] = sb[0][1][o] + sb[1][1][o] + sb[2][1][o] + sb[3][1][o];
    out[ow3 + o] = sb[0][2][o] + sb[1][2][o] + sb[2][2][o] + sb[3][2][o];
  }
  if (threadIdx.x == 0) {
    out[ob3] = sl[0][0] + sl[1][0] + sl[2][0] + sl[3][0];
    out[kNPar] = sl[0][1] + sl[1][1] + sl[2][1] + sl[3][1];
  }
}

// Fixed-order sum of the block partials: grad [kNPar + 1] (last entry: sum of squared
// residuals, also added to *loss_acc when given).
__global__ void k_mlp_grad_reduce(const float* part, int nblk, float* grad, float* loss_acc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kNPar) return;
  float acc = 0.f;
  for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * kGradStride + p];
  grad[p] = acc;
  if (p == kNPar && loss_acc) *loss_acc += acc;
}

// Adam on the FP32 master parameters.
__global__ void k_mlp_adam(float* P, float* mom, float* vel, const float* grad, float lr, float b1c, float b2c) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNPar) return;
  const float gr = grad[p];
  const float mo = 0.9f * mom[p] + 0.1f * gr;
  const float ve = 0.999f * vel[p] + 0.001f * gr * gr;
  mom[p] = mo;
  vel[p] = ve;
  P[p] -= lr * (mo / b1c) / (sqrtf(ve / b2c) + 1e-8f);
}

// BF16 operand copies of W1 (K padded to 16), W2 and W2 transposed, from the master.
__global__ void k_mlp_pack(const float* P, unsigned* W1p, unsigned* W2p, unsigned* W2Tp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kH * 8) {
    const int o = t / 8, kp = t % 8;
    const float lo = 2 * kp < kIn ? P[oW1 + o * kIn + 2 * kp] : 0.f;
    const float hi = 2 * kp + 1 < kIn ? P[oW1 + o * kIn + 2 * kp + 1] : 0.f;
    W1p[t] = pack_bf16(lo, hi);
  }
  if (t < kH * 32) {
    const int r = t / 32, kp = t % 32;
    W2p[t] = pack_bf16(P[oW2 + r * kH + 2 * kp], P[oW2 + r * kH + 2 * kp + 1]);
    W2Tp[t] = pack_bf16(P[oW2 + (2 * kp) * kH + r], P[oW2 + (2 * kp + 1) * kH + r]);
  }
}

// ---------------- features of a pair from the current mapping --------------------------

__device__ __forceinline__ void sort4f(float v[4]) {
  float a = fminf(v[0], v[1]), b = fmaxf(v[0], v[1]), c = fminf(v[2], v[3]), d = fmaxf(v[2], v[3]);
  const float lo = fminf(a, c), hi = fmaxf(b, d), m1 = fmaxf(a, c), m2 = fminf(b, d);
  v[0] = lo;
  v[1] = fminf(m1, m2);
  v[2] = fmaxf(m1, m2);
  v[3] = hi;
}

// COM-relative offset of atom i in the current mapping, as float (either path's layout).
template <bool F64>
__device__ __forceinline__ float4 offset_f(const Bufs& b, int cur, int i) {
  if (F64) {
    const double4_32a o = b.off64[cur][i];
    return make_float4((float)o.x, (float)o.y, (float)o.z, 0.f);
  }
  return b.off32[cur][i];
}

// Features of (a, b) with e from a to b; feat[9].  Atoms beyond na project to 0 (padding).
// The first molecule's centre A and atom offsets oa[] come from the caller.
template <int NA, bool F64>
__device__ __forceinline__ void pair_features32(const Box& X, const int4 A, const float4 (&oa)[NA], const Bufs& b,
                                                int cur, int bb, float feat[9]) {
  const int4 B = b.com_fx[cur][bb];
  const float ex = (float)(int)((unsigned)B.x - (unsigned)A.x) * X.fx_scale[0];
  const float ey = (float)(int)((unsigned)B.y - (unsigned)A.y) * X.fx_scale[1];
  const float ez = (float)(int)((unsigned)B.z - (unsigned)A.z) * X.fx_scale[2];
  const float d = sqrtf(ex * ex + ey * ey + ez * ez), id = 1.f / d;
  float sa[4] = {0.f, 0.f, 0.f, 0.f}, sb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    const float4 ob = offset_f<F64>(b, cur, bb * NA + k);
    sa[k] = (oa[k].x * ex + oa[k].y * ey + oa[k].z * ez) * id;
    sb[k] = -(ob.x * ex + ob.y * ey + ob.z * ez) * id;
  }
  if (NA == 4) {
    sort4f(sa);
    sort4f(sb);
  } else {
    for (int i = 1; i < NA; ++i)
      for (int j = i; j > 0 && sa[j - 1] > sa[j]; --j) {
        const float t = sa[j]; sa[j] = sa[j - 1]; sa[j - 1] = t;
      }
    for (int i = 1; i < NA; ++i)
      for (int j = i; j > 0 && sb[j - 1] > sb[j]; --j) {
        const float t = sb[j]; sb[j] = sb[j - 1]; sb[j - 1] = t;
      }
  }
  feat[0] = d;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    feat[1 + k] = sa[k];
    feat[5 + k] = sb[k];
  }
}

template <int NA, bool F64>
__device__ __forceinline__ void pair_features32(const Sys& s, const Bufs& b, int cur, int a, int bb, float feat[9]) {
  float4 oa[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) oa[k] = offset_f<F64>(b, cur, a * NA + k);
  pair_features32<NA, F64>(box_of(s, b, a), b.com_fx[cur][a], oa, b, cur, bb, feat);
}

// Atomistic force on a from b projected on -e (the force-matching target), FP32.
template <int NA, bool F64>
__device__ __forceinline__ float pair_target32(const Sys& s, const Bufs& b, int cur, int a, int bb) {
  const int4 A = b.com_fx[cur][a], B = b.com_fx[cur][bb];
  const Box& X = box_of(s, b, a);
  const float Rx = (float)(int)((unsigned)A.x - (unsigned)B.x) * X.fx_scale[0];
  const float Ry = (float)(int)((unsigned)A.y - (unsigned)B.y) * X.fx_scale[1];
  const float Rz = (float)(int)((unsigned)A.z - (unsigned)B.z) * X.fx_scale[2];
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    const float4 oi = offset_f<F64>(b, cur, a * NA + i);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const float4 oj = offset_f<F64>(b, cur, bb * NA + j);
      const float dx = Rx + oi.x - oj.x, dy = Ry + oi.y - oj.y, dz = Rz + oi.z - oj.z;
      const float d2 = dx * dx + dy * dy + dz * dz;
      if (d2 < s.f.rc_at2) {
        float fr;
        if (s.nb_model == 1) {
          // Lennard-Jones + reaction field of the site pair (the water-like model)
          const float ir2 = 1.f / d2, ir = sqrtf(ir2), ir6 = ir2 * ir2 * ir2;
          fr = (12.f * s.f.c12[i][j] * ir6 - 6.f * s.f.c6[i][j]) * ir6 * ir2 + s.f.qq[i][j] * (ir2 * ir - s.f.krf2);
        } else {
          const float ir2 = 1.f / d2, sr2 = s.f.sig2 * ir2, sr6 = sr2 * sr2 * sr2;
          fr = 24.f * s.f.eps * (2.f * sr6 * sr6 - sr6) * ir2;
        }
        Fx += fr * dx;
        Fy += fr * dy;
        Fz += fr * dz;
      }
    }
  }
  const float r = sqrtf(Rx * Rx + Ry * Ry + Rz * Rz);
  return (Fx * Rx + Fy * Ry + Fz * Rz) / r;
}

// Count (pass 0) or write (pass 1) the samples of every work item: pairs with a < b, COM
// distance below rc_cg.  Writing uses per-item offsets from an exclusive scan, so the
// sample order is deterministic (item order, then list order).
template <int NA, bool F64>
__global__ void k_mlp_collect(const __grid_constant__ Sys s, Bufs b, int pass, const int* offs, long long cap, long long base, float* feat,
                              float* target, int* ids, int* counts) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.M) return;
  const int cur = b.ctrl->parity;
  const int a = b.items[t];
  const int n = b.nn[t];
  int c = 0;
  long long o = pass ? base + offs[t] : 0;
  for (int q = 0; q < n; ++q) {
    const int m = b.nbr[(size_t)t * s.cap + q];
    if (m <= a) continue;
    const int4 A = b.com_fx[cur][a], B = b.com_fx[cur][m];
    const Box& X = box_of(s, b, a);
    const float dx = (float)(int)((unsigned)B.x - (unsigned)A.x) * X.fx_scale[0];
    const float dy = (float)(int)((unsigned)B.y - (unsigned)A.y) * X.fx_scale[1];
    const float dz = (float)(int)((unsigned)B.z - (unsigned)A.z) * X.fx_scale[2];
    if (dx * dx + dy * dy + dz * dz >= s.f.rc_cg2) continue;
    if (pass && o < cap) {
      float f[9];
      pair_features32<NA, F64>(s, b, cur, a, m, f);
#pragma unroll
      for (int k = 0; k < 9; ++k) feat[o * 9 + k] = f[k];
      target[o] = pair_target32<NA, F64>(s, b, cur, a, m);
      ids[2 * o] = a;
      ids[2 * o + 1] = m;
    }
    ++c;
    ++o;
  }
  if (!pass) counts[t] = c;
}

// ---------------- pair forces for the dynamics -------------------------------------------
// Every list slot (t, q) whose pair needs a CG force (COM distance < rc_cg and w_ab < 1, the
// force kernel's test in its own precision and arithmetic) gets the symmetrised network
// force in fpair[t cap + q].  At each list build k_net_candidates records every pair that may
// need the network before the next build, once (from the molecule with the smaller id), with
// its slot and the mirror slot in the partner's list.  Per step k_mlp_feat tests the
// candidates, computes the features of those that need the network and appends them to a
// pair buffer (one atomic per warp; the buffer order varies between runs, the values do
// not); the evaluation kernel (k_mlp_eval_tc on tcgen05, or k_mlp_eval below: 16 pairs per
// warp tile, both orderings as two tensor-core tiles, weights staged in shared memory) then
// writes the force to both slots.

// The first molecule's centre (FP64 or fixed-point, by path) is passed in.
template <bool F64>
struct Centre;
template <>
struct Centre<true> {
  double4_32a c;
};
template <>
struct Centre<false> {
  int4 c;
};

template <bool F64>
__device__ __forceinline__ Centre<F64> centre_of(const Bufs& b, int cur, int a) {
  if constexpr (F64)
    return {b.com64[cur][a]};
  else
    return {b.com_fx[cur][a]};
}

template <bool F64>
__device__ __forceinline__ bool needs_network(const Sys& s, const Box& X, const Bufs& b, int cur, const Centre<F64>& CA,
                                              int m) {
  if constexpr (F64) {
    const double4_32a A = CA.c, B = b.com64[cur][m];
    const double r2 = pair_r2(minimg_cmp(A.x - B.x, X.L[0], X.halfL[0]), minimg_cmp(A.y - B.y, X.L[1], X.halfL[1]),
                              minimg_cmp(A.z - B.z, X.L[2], X.halfL[2]));
    return A.w * B.w < 1.0 && r2 < s.rc_cg2;
  } else {
    const int4 A = CA.c, B = b.com_fx[cur][m];
    const float r2 = pair_r2((float)(int)((unsigned)A.x - (unsigned)B.x) * X.fx_scale[0],
                             (float)(int)((unsigned)A.y - (unsigned)B.y) * X.fx_scale[1],
                             (float)(int)((unsigned)A.z - (unsigned)B.z) * X.fx_scale[2]);
    return __int_as_float(A.w) * __int_as_float(B.w) < 1.f && r2 < s.f.rc_cg2;
  }
}

// Both orderings of a pair's features, normalised (mean, 1/std in sn) and packed as bf16
// pairs the way the evaluation kernels read their A operands.
__device__ __forceinline__ void pack_pair_inputs(const float f[9], const float (*sn)[kIn], unsigned* out) {
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int w = 0; w < 5; ++w) {
      float v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * w + h;
        const int src = (u == 0 || k == 0) ? k : (k < 5 ? k + 4 : k - 4);
        v[h] = k < kIn ? (f[src < kIn ? src : 0] - sn[0][k < kIn ? k : 0]) * sn[1][k < kIn ? k : 0] : 0.f;
      }
      out[5 * u + w] = pack_bf16(v[0], v[1]);
    }
}

// A molecule deep in the atomistic region at the list build: it keeps lambda = 1 until the
// next build (its centre moves by less than skin/2 before then).  thr = d_at - skin/2 - 1e-3
// of the molecule's box (as float for the FP32 path, whose distances are floats).
template <bool F64>
__device__ __forceinline__ bool deep_atomistic(const Sys& s, const Bufs& b, int cur, int a, double thr, float thr_f) {
  if (s.lam_uniform_on) return s.lam_uniform >= 1.0;
  if constexpr (F64)
    return fabs(b.dxc64[cur][a]) < thr;
  else
    return fabsf(b.molf[cur][a].x) < thr_f;
}

// Candidate pairs of the network force, built with the lists: every
// listed slot (t, q) whose molecule pair a = items[t] < m is within rc_cg + skin and is not
// made of two deep-atomistic molecules.  Until the next build every pair that needs the
// network (weight below 1, centres within rc_cg) is among them: the centres move by less
// than skin/2 each, and a pair of deep-atomistic molecules keeps weight 1.  Records (slot,
// mirror slot, a, m); four lanes per work item, one atomic per warp (the order varies between
// runs, the set does not).
template <bool F64>
__global__ void __launch_bounds__(128) k_net_candidates(const __grid_constant__ Sys s, Bufs b) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 2, g = threadIdx.x & 3;
  const int lane = threadIdx.x & 31;
  const bool live = t < s.M;
  const int cur = b.ctrl->parity;
  const int a = live ? b.items[t] : 0;
  const int n = live ? b.nn[t] : 0;
  const Box& X = box_of(s, b, a);
  // the threshold once per thread (neighbours share the box of the work item); the FP32
  // path forms it from float parameters (skin = sqrt(r_cg_list2) - rc_cg), off the FP64 pipe
  const double thr = F64 ? X.d_at - 0.5 * s.skin - 1e-3 : 0.0;
  const float thr_f = X.d_at_f - 0.5f * (sqrtf(s.f.r_cg_list2) - sqrtf(s.f.rc_cg2)) - 1e-3f;
  const bool deep_a = live && deep_atomistic<F64>(s, b, cur, a, thr, thr_f);
  const int* row = b.nbr + (size_t)t * s.cap;
  auto candidate = [&](int m) -> bool {
    if (m <= a || (deep_a && deep_atomistic<F64>(s, b, cur, m, thr, thr_f))) return false;
    if constexpr (F64) {
      const double4_32a A = b.com64[cur][a], B = b.com64[cur][m];
      return pair_r2(minimg_cmp(A.x - B.x, X.L[0], X.halfL[0]), minimg_cmp(A.y - B.y, X.L[1], X.halfL[1]),
                     minimg_cmp(A.z - B.z, X.L[2], X.halfL[2])) < s.r_cg_list2;
    } else {
      const int4 A = b.com_fx[cur][a], B = b.com_fx[cur][m];
      return pair_r2((float)(int)((unsigned)A.x - (unsigned)B.x) * X.fx_scale[0],
                     (float)(int)((unsigned)A.y - (unsigned)B.y) * X.fx_scale[1],
                     (float)(int)((unsigned)A.z - (unsigned)B.z) * X.fx_scale[2]) < s.f.r_cg_list2;
    }
  };
  unsigned long long sel = 0ull;
  int cnt = 0;
  for (int q = g, j = 0; q < n; q += 4, ++j)
    if (candidate(row[q])) {
      ++cnt;
      if (j < 64) sel |= 1ull << j;
    }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  int base = 0;
  if (lane == 31 && incl > 0) base = atomicAdd(&b.ctrl->n_netc, incl);
  base = __shfl_sync(0xffffffffu, base, 31);
  long long p = (long long)base + (incl - cnt);
  if (cnt == 0) return;
  int qx = g + 256;  // where the search for candidates beyond the mask resumes
  for (int left = cnt; left > 0; --left) {
    int q;
    if (sel) {
      q = g + 4 * (__ffsll((long long)sel) - 1);
      sel &= sel - 1;
    } else {
      for (q = qx; q < n; q += 4)
        if (candidate(row[q])) break;
      if (q >= n) return;  // not reached: the first walk counted this slot
      qx = q + 4;
    }
    if (p >= b.ncap) {  // not reached: at most one record per unordered listed pair
      set_error(b.ctrl, ADRESS_ERR_LIST_OVERFLOW, (int)p);
      return;
    }
    // the mirror slot: where a sits in m's list (the lists are symmetric)
    const int m = row[q], tb = b.item_of[m], nb = b.nn[tb];
    const int* rb = b.nbr + (size_t)tb * s.cap;
    int found = -1;
    for (int qq = 0; qq < nb; ++qq)
      if (rb[qq] == a) {
        found = qq;
        break;
      }
    if (found < 0) set_error(b.ctrl, ADRESS_ERR_STATE, a);
    b.netc[p] = make_int4(t * s.cap + q, found < 0 ? -1 : tb * s.cap + found, a, m);
    ++p;
  }
}

cudaError_t launch_net_candidates(const Sys& s, const Bufs& b, cudaStream_t st) {
  const int blocks = ceil_div((long long)s.M * 4, 128);
  if (s.fp64) k_net_candidates<true><<<blocks, 128, 0, st>>>(s, b);
  else k_net_candidates<false><<<blocks, 128, 0, st>>>(s, b);
  return cudaGetLastError();
}

// Pairs that need the network this step, from the candidates of the last build: the force
// kernel's test (centres within rc_cg, weight below 1) in its own precision and arithmetic,
// then the pair's features, normalised bf16 inputs of both orderings and its two list slots
// appended to the pair buffer (one atomic per warp).  One thread per candidate, persistent grid.
template <int NA, bool F64>
__global__ void __launch_bounds__(128) k_mlp_feat(const __grid_constant__ Sys s, Bufs b, const float* __restrict__ norm) {
  // multiple time stepping: the network gives a slow (CG) force, needed only at outer time
  // levels; elsewhere no pair is written and the evaluation kernel finds nothing to do
  if (s.respa_n > 1 && b.ctrl->step % s.respa_n != 0) return;
  __shared__ float sn[2][kIn];
  if (threadIdx.x < kIn) {
    sn[0][threadIdx.x] = norm[threadIdx.x];
    sn[1][threadIdx.x] = norm[2 * kIn + 1 + threadIdx.x];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int cur = b.ctrl->parity;
  const long long nc = min((long long)b.ctrl->n_netc, b.ncap);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); k0 < nc; k0 += stride) {
    const long long k = k0 + lane;
    int4 rec = make_int4(0, 0, 0, 0);
    bool need = false;
    if (k < nc) {
      rec = b.netc[k];
      need = needs_network<F64>(s, box_of(s, b, rec.z), b, cur, centre_of<F64>(b, cur, rec.z), rec.w);
    }
    // the features first, so that their gathers overlap the warp's atomic below
    float f[9];
    if (need) pair_features32<NA, F64>(s, b, cur, rec.z, rec.w, f);
    const unsigned bal = __ballot_sync(0xffffffffu, need);
    unsigned base = 0;
    if (lane == 0 && bal) base = atomicAdd(b.npair, (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!need) continue;
    const long long p = (long long)base + __popc(bal & ((1u << lane) - 1u));
    if (p >= b.pcap) {
      set_error(b.ctrl, ADRESS_ERR_LIST_OVERFLOW, (int)p);
      continue;
    }
    pack_pair_inputs(f, sn, b.pfrag + p * 10);
    b.pslot[p] = make_int2(rec.x, rec.y);
  }
}

__global__ void __launch_bounds__(128, 8) k_mlp_eval(MlpDev m, const unsigned* __restrict__ pfrag,
                                                     const int2* __restrict__ pslot, const unsigned* npair,
                                                     long long pcap, long long nslot, float* __restrict__ fpair) {
  __shared__ float yo[4][2][16];
  __shared__ uint2 sW1[kH * 4], sW2[kH * 16];
  __shared__ float sB[3 * kH];
  for (int i = threadIdx.x; i < kH * 16; i += blockDim.x) {
    const int r = i >> 4, kk = (i >> 2) & 3, tg = i & 3;
    sW2[i] = make_uint2(m.W2p[r * 32 + 8 * kk + tg], m.W2p[r * 32 + 8 * kk + tg + 4]);
  }
  for (int i = threadIdx.x; i < kH * 4; i += blockDim.x) {
    const int r = i >> 2, tg = i & 3;
    sW1[i] = make_uint2(m.W1p[r * 8 + tg], m.W1p[r * 8 + tg + 4]);
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    sB[i] = m.P[ob1 + i];
    sB[kH + i] = m.P[ob2 + i];
    sB[2 * kH + i] = m.P[ow3 + i];
  }
  __syncthreads();
  const MlpViewQ mq{sW1, sW2, sB, sB + kH, sB + 2 * kH, m.P[ob3]};
  const float scale = m.norm[2 * kIn];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  const long long np = min((long long)*npair, pcap);  // clamped to the buffer (see k_mlp_eval_tc)
  const long long ntiles = (np + 15) / 16;
  for (long long tile = (long long)blockIdx.x * 4 + w; tile < ntiles; tile += (long long)gridDim.x * 4) {
    const long long p0 = tile * 16;
    // A fragments straight from the pair buffer: rows g, g + 8; words tg (columns 2tg, 2tg+1)
    // and, for tg = 0, word 4 (columns 8, 9); the other column words are zero padding
    unsigned ax0[4] = {0u, 0u, 0u, 0u}, ax1[4] = {0u, 0u, 0u, 0u};
    if (p0 + g < np) {
      const unsigned* r = pfrag + (p0 + g) * 10;
      ax0[0] = r[tg];
      ax1[0] = r[5 + tg];
      if (tg == 0) {
        ax0[2] = r[4];
        ax1[2] = r[9];
      }
    }
    if (p0 + g + 8 < np) {
      const unsigned* r = pfrag + (p0 + g + 8) * 10;
      ax0[1] = r[tg];
      ax1[1] = r[5 + tg];
      if (tg == 0) {
        ax0[3] = r[4];
        ax1[3] = r[9];
      }
    }
    float y[2][2];
    tile_forward_y2(mq, ax0, ax1, y);
    if (tg == 0) {
      yo[w][0][g] = y[0][0];
      yo[w][0][g + 8] = y[0][1];
      yo[w][1][g] = y[1][0];
      yo[w][1][g + 8] = y[1][1];
    }
    __syncwarp();
    if (lane < 16 && p0 + lane < np) {
      const float fv = 0.5f * scale * (yo[w][0][lane] + yo[w][1][lane]);
      const int2 sl = pslot[p0 + lane];
      if (sl.x >= 0 && sl.x < nslot) fpair[sl.x] = fv;
      if (sl.y >= 0 && sl.y < nslot) fpair[sl.y] = fv;
    }
    __syncwarp();
  }
}

// Training batch `cnt` samples starting at `start` of a fixed permutation of the n
// samples: sample (start + i) * stride mod n (stride coprime with n).
__global__ void k_mlp_gather(const float* feat, const float* target, long long n, long long start, long long cnt,
                             long long stride, float* fo, float* to) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const long long src = (long long)(((unsigned long long)(start + i) * (unsigned long long)stride) % (unsigned long long)n);
#pragma unroll
  for (int k = 0; k < kIn; ++k) fo[i * kIn + k] = feat[src * kIn + k];
  to[i] = target[src];
}

// ---------------- force-matched CG table ---------------------------------------------------
// The CG force of Eq. 1 acts between centres of mass (Sec. "Force interpolation").  Its
// force-matched table is the mean, per distance bin, of the atomistic pair force projected on
// the COM axis over the collected samples (features[0] = COM distance d, target = that force):
//   bin j = floor(d / h) (d < rc), mean_j = sum / count for bins with count >= n_min;
//   F_raw(r) linear between the centres (j + 1/2) h of those bins, constant beyond the first
//   and the last;  F(r_k) = F_raw(r_k) - F_raw(rc) for r_k = k dr < rc, 0 from rc on;
//   V(r_k) = sum_{m >= k} (F_m + F_{m+1}) dr / 2  (trapezoid rule from rc down to r_k).
// Sums are exact integers: each target is scaled by 2^48 and split into a high part
// (>> 24) and a low part (24 bits), summed with 64-bit integer atomics (order-independent,
// so the table is deterministic); the mean is formed from them in double.

constexpr double kFitScale = 281474976710656.0;  // 2^48

__global__ void k_fit_bins(const float* __restrict__ feat, const float* __restrict__ target, long long n, double h,
                           int nb, unsigned long long* __restrict__ acc, unsigned* __restrict__ cnt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)feat[i * kIn];
    if (!(d >= 0.0)) continue;
    const double u = d / h;
    if (u >= (double)nb) continue;
    const int j = (int)u;
    const long long q = llrint((double)target[i] * kFitScale);
    atomicAdd(&acc[2 * j], (unsigned long long)(q >> 24));
    atomicAdd(&acc[2 * j + 1], (unsigned long long)(q & 0xFFFFFFll));
    atomicAdd(&cnt[j], 1u);
  }
}

constexpr int kFitMaxBins = 4096;

// One block: means of the populated bins (compacted in bin order by a block scan), node
// values by linear interpolation between their centres, the shift to F(rc) = 0, and V by the
// trapezoid sum (one thread, from rc down, the definition's order).
__global__ void __launch_bounds__(1024) k_fit_table(const unsigned long long* __restrict__ acc,
                                                    const unsigned* __restrict__ cnt, int nb, double h, int n_min,
                                                    int cg_n, double dr, double rc, double* __restrict__ F,
                                                    double* __restrict__ V, int* __restrict__ npop_out) {
  __shared__ double pc[kFitMaxBins], pm[kFitMaxBins];
  __shared__ int wsum[32], npop;
  constexpr int per = kFitMaxBins / 1024;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int flag[per], cntp = 0;
#pragma unroll
  for (int e = 0; e < per; ++e) {
    const int j = t * per + e;
    flag[e] = j < nb && cnt[j] >= (unsigned)n_min;
    cntp += flag[e];
  }
  int incl = cntp;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int x = wsum[lane];
    int xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += v;
    }
    wsum[lane] = xi - x;
    if (lane == 31) npop = xi;
  }
  __syncthreads();
  int pos = incl - cntp + wsum[w];
#pragma unroll
  for (int e = 0; e < per; ++e) {
    const int j = t * per + e;
    if (flag[e]) {
      const double sum = (double)(long long)acc[2 * j] * (1.0 / 16777216.0) + (double)(long long)acc[2 * j + 1] / kFitScale;
      pc[pos] = __dmul_rn(__dadd_rn((double)j, 0.5), h);
      pm[pos] = sum / (double)cnt[j];
      ++pos;
    }
  }
  __syncthreads();
  const int np = npop;
  if (t == 0) *npop_out = np;
  if (np == 0) return;
  // F_raw(r): clamped linear interpolation between the populated centres
  auto raw = [&](double r) -> double {
    if (r <= pc[0]) return pm[0];
    if (r >= pc[np - 1]) return pm[np - 1];
    int lo = 0, hi = np - 1;  // pc[lo] < r < pc[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pc[mid] <= r) lo = mid;
      else hi = mid;
    }
    const double slope = __ddiv_rn(__dsub_rn(pm[hi], pm[lo]), __dsub_rn(pc[hi], pc[lo]));
    return __dadd_rn(__dmul_rn(slope, __dsub_rn(r, pc[lo])), pm[lo]);
  };
  const double f_rc = raw(rc);
  for (int k = t; k <= cg_n; k += blockDim.x) {
    const double r = __dmul_rn((double)k, dr);
    F[k] = r < rc ? __dsub_rn(raw(r), f_rc) : 0.0;
  }
  __syncthreads();
  if (t == 0) {
    double v = 0.0;
    V[cg_n] = 0.0;
    for (int k = cg_n - 1; k >= 0; --k) {
      v = __dadd_rn(v, __dmul_rn(__dmul_rn(0.5, __dadd_rn(F[k], F[k + 1])), dr));
      V[k] = v;
    }
  }
}

cudaError_t cg_fit(const float* feat, const float* target, long long n, double h, int nb, int n_min, int cg_n,
                   double dr, double rc, unsigned long long* acc, unsigned* cnt, double* F, double* V, int* npop,
                   cudaStream_t st) {
  if (nb > kFitMaxBins) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 2 * nb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * nb, st);
  if (e != cudaSuccess) return e;
  const long long blocks = std::min<long long>((n + 255) / 256, 152 * 8);
  if (n > 0) k_fit_bins<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, st>>>(feat, target, n, h, nb, acc, cnt);
  k_fit_table<<<1, 1024, 0, st>>>(acc, cnt, nb, h, n_min, cg_n, dr, rc, F, V, npop);
  return cudaGetLastError();
}

// ---------------- launchers ------------------------------------------------------------

cudaError_t mlp_gather(const float* feat, const float* target, long long n, long long start, long long cnt,
                       long long stride, float* fo, float* to, cudaStream_t st) {
  k_mlp_gather<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(feat, target, n, start, cnt, stride, fo, to);
  return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpDevArgs& a, const float* feat, long long n, float* y, cudaStream_t st) {
  const MlpDev m{a.P, a.W1p, a.W2p, a.W2Tp, a.norm};
  const long long tiles = (n + 15) / 16;
  k_mlp_forward<<<(unsigned)((tiles + 3) / 4), 128, 0, st>>>(m, feat, n, y);
  return cudaGetLastError();
}

cudaError_t mlp_grad(const MlpDevArgs& a, const float* feat, const float* target, long long n, long long n_total,
                     float* part, float* grad, float* loss_acc, cudaStream_t st) {
  const MlpDev m{a.P, a.W1p, a.W2p, a.W2Tp, a.norm};
  const int nblk = (int)((n + 63) / 64);
  k_mlp_grad<<<nblk, 128, 0, st>>>(m, feat, target, n, n_total, part);
  k_mlp_grad_reduce<<<(kNPar + 1 + 255) / 256, 256, 0, st>>>(part, nblk, grad, loss_acc);
  return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpDevArgs& a, float* mom, float* vel, const float* grad, float lr, int step,
                     cudaStream_t st) {
  const float b1c = 1.f - powf(0.9f, (float)step), b2c = 1.f - powf(0.999f, (float)step);
  k_mlp_adam<<<(kNPar + 255) / 256, 256, 0, st>>>((float*)a.P, mom, vel, grad, lr, b1c, b2c);
  return cudaGetLastError();
}

cudaError_t mlp_pack(const MlpDevArgs& a, cudaStream_t st) {
  k_mlp_pack<<<(kH * 32 + 255) / 256, 256, 0, st>>>(a.P, (unsigned*)a.W1p, (unsigned*)a.W2p, (unsigned*)a.W2Tp);
  return cudaGetLastError();
}

cudaError_t mlp_collect(const Sys& s, const Bufs& b, int pass, const int* offs, long long cap, long long base,
                        float* feat, float* target, int* ids, int* counts, cudaStream_t st) {
  const int blocks = ceil_div(s.M, 128);
#define COLLECT(NA_)                                                                                       \
  (s.fp64 ? k_mlp_collect<NA_, true><<<blocks, 128, 0, st>>>(s, b, pass, offs, cap, base, feat, target, ids, counts) \
          : k_mlp_collect<NA_, false><<<blocks, 128, 0, st>>>(s, b, pass, offs, cap, base, feat, target, ids, counts))
  switch (s.NA) {
    case 1: COLLECT(1); break;
    case 2: COLLECT(2); break;
    case 3: COLLECT(3); break;
    default: COLLECT(4); break;
  }
#undef COLLECT
  return cudaGetLastError();
}

cudaError_t mlp_pairs(const Sys& s, const Bufs& b, const MlpDevArgs& a, float* fpair, cudaStream_t st) {
  const MlpDev m{a.P, a.W1p, a.W2p, a.W2Tp, a.norm};
  cudaError_t e = cudaMemsetAsync(b.npair, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  // persistent grid for the candidates (their count is on the device): 22 blocks per SM,
  // about two waves of the 10 that the kernel's 48 registers let reside (11, 16, 20, 33 and
  // 44 blocks per SM measured slower at 800k atoms)
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    blocks = 22 * sms;
  }
#define FEAT(NA_)                                                       \
  (s.fp64 ? k_mlp_feat<NA_, true><<<blocks, 128, 0, st>>>(s, b, a.norm) \
          : k_mlp_feat<NA_, false><<<blocks, 128, 0, st>>>(s, b, a.norm))
  switch (s.NA) {
    case 1: FEAT(1); break;
    case 2: FEAT(2); break;
    case 3: FEAT(3); break;
    default: FEAT(4); break;
  }
#undef FEAT
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the tcgen05 / TMEM evaluation (mlp_tc.cu), unless ADRESS_MLP_KERNEL=mma selects the
  // warp-level MMA kernel below (same network, same results to rounding order)
  static int tc = -1;
  if (tc < 0) {
    const char* v = getenv("ADRESS_MLP_KERNEL");
    tc = v && strcmp(v, "mma") == 0 ? 0 : 1;
  }
  if (tc) return launch_mlp_eval_tc(s, a, b, fpair, st);
  // persistent grid: as many blocks as fit on the device at once
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_eval, 128, 0) != cudaSuccess || per_sm < 1)
      per_sm = 4;
    grid = per_sm * sms;
  }
  k_mlp_eval<<<grid, 128, 0, st>>>(m, b.pfrag, b.pslot, b.npair, b.pcap, (long long)s.M * s.cap, fpair);
  return cudaGetLastError();
}

}  // namespace adress
