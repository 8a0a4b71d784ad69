// Learned initializer of multi-direct forcing: a multilayer perceptron maps each
// Lagrangian point's local velocity-deficit stencil to the force of the first MDF
// iteration; the plain iterations (Sec. 2.2, MDF) then run from it as before.  No
// counterpart in the paper (the MDF itself is named there, Sec. 1 and 2.2).
//
// Features of point k of a particle (27): the deficit U_b - u_b* (u_b* = D_I u*, the
// velocity the first interpolation gathers) at points k-4 .. k+4 of the same circle,
// each as (normal, tangent, 0) components in the frame of point k (normal = unit
// offset from the centre, tangent = normal rotated by +90 degrees).  Output (3): the
// force in that frame (the third component is unused in 2D).  Spheres: the point and
// its 8 nearest neighbours on the sphere in the point's (normal, t1, t2) frame (below).
//
// Parameters (FP32, row-major), kMlpParams floats:
//   W1 [27][64], b1 [64], W2 [64][64], b2 [64], W3 [64][3], b3 [3], in_scale, out_scale
// hidden layers ReLU; the network sees features * in_scale and its output is scaled by
// out_scale.
//
// Kernels: features (for the step and for training samples), tensor-core inference
// (mma.sync m16n8k16, FP16 operands, FP32 accumulation, one warp per 16 points) and
// FP32 training: forward, backward, weight gradients, Adam.
#include <algorithm>
#include <cstdint>
#include <string>

#include "common.cuh"
#include "launch.h"
#include "mlp.h"

namespace ibmlbm {

constexpr int kIn = kMlpIn, kH = kMlpH, kOut = kMlpOut;
constexpr int oW1 = 0, ob1 = oW1 + kIn * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kOut, oInS = ob3 + kOut, oOutS = oInS + 1;
static_assert(oOutS + 1 == kMlpParams, "parameter layout");

// ------------------------------------------------------------------ features
// frame of point k: unit offset n from the centre and t = n rotated by +90 degrees
__device__ __forceinline__ void point_frame(const float* ref_f, int k, float& nx, float& ny) {
  const float rx = ref_f[2 * k], ry = ref_f[2 * k + 1];
  const float inv = rsqrtf(rx * rx + ry * ry);
  nx = rx * inv;
  ny = ry * inv;
}

__device__ __forceinline__ void features_2d(const float* Ub, const float* ubs, const float* ref_f,
                                            int nl, long long base, int k, float (&x)[kIn]) {
  float nx, ny;
  point_frame(ref_f, k, nx, ny);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    int kk = k + j - 4;
    kk = kk < 0 ? kk + nl : (kk >= nl ? kk - nl : kk);
    const long long b = base + kk;
    const float dx = Ub[2 * b] - ubs[2 * b], dy = Ub[2 * b + 1] - ubs[2 * b + 1];
    x[3 * j] = dx * nx + dy * ny;
    x[3 * j + 1] = -dx * ny + dy * nx;
    x[3 * j + 2] = 0.0f;
  }
}

// 3D (spheres): the deficit at point k and at its 8 stencil neighbours (frame3, nbr3:
// the 8 nearest other points of the reference sphere ordered by azimuth about the
// normal), each as (normal, t1, t2) components in the frame of point k.  Output (3):
// the force in that frame.
__device__ __forceinline__ void features_3d(const IbmArgs& A, long long base, int k, float (&x)[kIn]) {
  const float* F = A.frame3 + 9 * k;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int kk = j == 0 ? k : A.nbr3[8 * k + j - 1];
    const long long b = base + kk;
    const float d0 = A.Ub[3 * b] - A.ubs[3 * b], d1 = A.Ub[3 * b + 1] - A.ubs[3 * b + 1],
                d2 = A.Ub[3 * b + 2] - A.ubs[3 * b + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[3 * j + a] = d0 * F[3 * a] + d1 * F[3 * a + 1] + d2 * F[3 * a + 2];
  }
}

// training samples of the last step: features and the step's total force F_b in the
// frame of each point (thread per point)
__global__ void mlp_samples_kernel(IbmArgs A, float* __restrict__ X, float* __restrict__ Y) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= A.npts) return;
  const int k = (int)(b % A.nl);
  float x[kIn];
  if (A.D == 3) {
    features_3d(A, b - k, k, x);
    const float* F = A.frame3 + 9 * k;
    const float Fx = A.Fb[3 * b], Fy = A.Fb[3 * b + 1], Fz = A.Fb[3 * b + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) Y[b * kOut + a] = Fx * F[3 * a] + Fy * F[3 * a + 1] + Fz * F[3 * a + 2];
  } else {
    features_2d(A.Ub, A.ubs, A.ref_f, A.nl, b - k, k, x);
    float nx, ny;
    point_frame(A.ref_f, k, nx, ny);
    const float Fx = A.Fb[2 * b], Fy = A.Fb[2 * b + 1];
    Y[b * kOut] = Fx * nx + Fy * ny;
    Y[b * kOut + 1] = -Fx * ny + Fy * nx;
    Y[b * kOut + 2] = 0.0f;
  }
#pragma unroll
  for (int c = 0; c < kIn; ++c) X[b * kIn + c] = x[c];
}

// ------------------------------------------------------------------ inference
__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// transposed FP16 weights in shared memory: WT[n][k] (k contiguous), K padded to a
// multiple of 16 (+8 against bank conflicts), N padded to a multiple of 8
constexpr int kK1 = 32, kP1 = kK1 + 8;  // layer 1: K = 27 -> 32
constexpr int kK2 = 64, kP2 = kK2 + 8;
constexpr int kN3 = 8;                 // layer 3: N = 3 -> 8
constexpr int kInferWarps = 8;
constexpr int kXP = kK1 + 8;           // staged feature rows (halves)

// the weights as the kernels keep them in shared memory (built once per parameter set
// by mlp_image_kernel, copied in 16-byte pieces)
struct __align__(16) WeightImage {
  __half w1[kH * kP1];
  __half w2[kH * kP2];
  __half w3[kN3 * kP2];
  float b1[kH], b2[kH], b3[kN3];
};
static_assert(sizeof(WeightImage) % 16 == 0, "image copied as uint4");

struct InferSmem {
  WeightImage W;
  __half x[kInferWarps][16 * kXP];
};

// B fragment (k16 x n8) of a transposed weight matrix at k-block kb, n-tile nt
__device__ __forceinline__ void b_frag(const __half* WT, int pitch, int kb, int nt, int lane, uint32_t& b0,
                                       uint32_t& b1) {
  const int gid = lane >> 2, tig = lane & 3;
  const __half* r = WT + (nt * 8 + gid) * pitch + kb * 16 + tig * 2;
  b0 = *reinterpret_cast<const uint32_t*>(r);
  b1 = *reinterpret_cast<const uint32_t*>(r + 8);
}

// transposed FP16 weights and FP32 biases from the parameter vector
__device__ void build_image(WeightImage& I, const float* __restrict__ P) {
  for (int t = threadIdx.x; t < kH * kP1; t += blockDim.x) {
    const int n = t / kP1, k = t % kP1;
    I.w1[t] = __float2half_rn(k < kIn ? P[oW1 + k * kH + n] : 0.0f);
  }
  for (int t = threadIdx.x; t < kH * kP2; t += blockDim.x) {
    const int n = t / kP2, k = t % kP2;
    I.w2[t] = __float2half_rn(k < kH ? P[oW2 + k * kH + n] : 0.0f);
  }
  for (int t = threadIdx.x; t < kN3 * kP2; t += blockDim.x) {
    const int n = t / kP2, k = t % kP2;
    I.w3[t] = __float2half_rn(k < kH && n < kOut ? P[oW3 + k * kOut + n] : 0.0f);
  }
  for (int t = threadIdx.x; t < kH; t += blockDim.x) {
    I.b1[t] = P[ob1 + t];
    I.b2[t] = P[ob2 + t];
  }
  for (int t = threadIdx.x; t < kN3; t += blockDim.x) I.b3[t] = t < kOut ? P[ob3 + t] : 0.0f;
}

__global__ void mlp_image_kernel(const float* __restrict__ P, WeightImage* img) { build_image(*img, P); }

__device__ __forceinline__ void copy_image(WeightImage& dst, const WeightImage* __restrict__ src) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(&dst);
  for (int t = threadIdx.x; t < (int)(sizeof(WeightImage) / 16); t += blockDim.x) d4[t] = s4[t];
}

// the three layers for the 16 feature rows staged in xs (FP16, already scaled); returns
// the outputs of rows gid and gid + 8 at columns 2 tig, 2 tig + 1
__device__ __forceinline__ void mlp_rows(const InferSmem& S, const __half* xs, int lane, float (&o)[4]) {
  const int gid = lane >> 2, tig = lane & 3;
  float h[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float c0 = S.W.b1[nt * 8 + tig * 2], c1 = S.W.b1[nt * 8 + tig * 2 + 1];
    h[nt][0] = c0;
    h[nt][1] = c1;
    h[nt][2] = c0;
    h[nt][3] = c1;
  }
#pragma unroll
  for (int kb = 0; kb < kK1 / 16; ++kb) {
    const __half* r0 = xs + gid * kXP + kb * 16 + tig * 2;
    const __half* r1 = xs + (gid + 8) * kXP + kb * 16 + tig * 2;
    const uint32_t a0 = *reinterpret_cast<const uint32_t*>(r0), a1 = *reinterpret_cast<const uint32_t*>(r1);
    const uint32_t a2 = *reinterpret_cast<const uint32_t*>(r0 + 8), a3 = *reinterpret_cast<const uint32_t*>(r1 + 8);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t b0, b1;
      b_frag(S.W.w1, kP1, kb, nt, lane, b0, b1);
      mma16816(h[nt], a0, a1, a2, a3, b0, b1);
    }
  }
  // layer 2: the accumulator layout of layer 1 is the A operand layout of layer 2
  float g[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float c0 = S.W.b2[nt * 8 + tig * 2], c1 = S.W.b2[nt * 8 + tig * 2 + 1];
    g[nt][0] = c0;
    g[nt][1] = c1;
    g[nt][2] = c0;
    g[nt][3] = c1;
  }
#pragma unroll
  for (int kb = 0; kb < kK2 / 16; ++kb) {
    const uint32_t a0 = pack_half2(fmaxf(h[2 * kb][0], 0.f), fmaxf(h[2 * kb][1], 0.f));
    const uint32_t a1 = pack_half2(fmaxf(h[2 * kb][2], 0.f), fmaxf(h[2 * kb][3], 0.f));
    const uint32_t a2 = pack_half2(fmaxf(h[2 * kb + 1][0], 0.f), fmaxf(h[2 * kb + 1][1], 0.f));
    const uint32_t a3 = pack_half2(fmaxf(h[2 * kb + 1][2], 0.f), fmaxf(h[2 * kb + 1][3], 0.f));
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t b0, b1;
      b_frag(S.W.w2, kP2, kb, nt, lane, b0, b1);
      mma16816(g[nt], a0, a1, a2, a3, b0, b1);
    }
  }
  o[0] = S.W.b3[tig * 2];
  o[1] = S.W.b3[tig * 2 + 1];
  o[2] = o[0];
  o[3] = o[1];
#pragma unroll
  for (int kb = 0; kb < kK2 / 16; ++kb) {
    const uint32_t a0 = pack_half2(fmaxf(g[2 * kb][0], 0.f), fmaxf(g[2 * kb][1], 0.f));
    const uint32_t a1 = pack_half2(fmaxf(g[2 * kb][2], 0.f), fmaxf(g[2 * kb][3], 0.f));
    const uint32_t a2 = pack_half2(fmaxf(g[2 * kb + 1][0], 0.f), fmaxf(g[2 * kb + 1][1], 0.f));
    const uint32_t a3 = pack_half2(fmaxf(g[2 * kb + 1][2], 0.f), fmaxf(g[2 * kb + 1][3], 0.f));
    uint32_t b0, b1;
    b_frag(S.W.w3, kP2, kb, 0, lane, b0, b1);
    mma16816(o, a0, a1, a2, a3, b0, b1);
  }
}

// The three layers for 32 feature rows (two m16 tiles, rows t * 16 + r of xs): every B
// fragment read from shared memory feeds both tiles.  The first layer's outputs are
// packed to the second layer's A fragments right away (half the registers of the FP32
// accumulators), and the third layer takes the second layer's columns two n-tiles at a
// time, so the second layer's accumulators are never all live.  o[t]: the outputs of
// rows t * 16 + gid and t * 16 + gid + 8 at columns 2 tig, 2 tig + 1.
__device__ __forceinline__ void mlp_rows32(const WeightImage& W, const __half* xs, int lane, float (&o)[2][4]) {
  const int gid = lane >> 2, tig = lane & 3;
  uint32_t a2[2][kK2 / 16][4];  // layer 2 A fragments (ReLU of layer 1, FP16)
  {
    float h[2][8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float c0 = W.b1[nt * 8 + tig * 2], c1 = W.b1[nt * 8 + tig * 2 + 1];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        h[t][nt][0] = c0;
        h[t][nt][1] = c1;
        h[t][nt][2] = c0;
        h[t][nt][3] = c1;
      }
    }
#pragma unroll
    for (int kb = 0; kb < kK1 / 16; ++kb) {
      uint32_t a[2][4];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const __half* r0 = xs + (t * 16 + gid) * kXP + kb * 16 + tig * 2;
        const __half* r1 = r0 + 8 * kXP;
        a[t][0] = *reinterpret_cast<const uint32_t*>(r0);
        a[t][1] = *reinterpret_cast<const uint32_t*>(r1);
        a[t][2] = *reinterpret_cast<const uint32_t*>(r0 + 8);
        a[t][3] = *reinterpret_cast<const uint32_t*>(r1 + 8);
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b0, b1;
        b_frag(W.w1, kP1, kb, nt, lane, b0, b1);
#pragma unroll
        for (int t = 0; t < 2; ++t) mma16816(h[t][nt], a[t][0], a[t][1], a[t][2], a[t][3], b0, b1);
      }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int kb = 0; kb < kK2 / 16; ++kb) {
        a2[t][kb][0] = pack_half2(fmaxf(h[t][2 * kb][0], 0.f), fmaxf(h[t][2 * kb][1], 0.f));
        a2[t][kb][1] = pack_half2(fmaxf(h[t][2 * kb][2], 0.f), fmaxf(h[t][2 * kb][3], 0.f));
        a2[t][kb][2] = pack_half2(fmaxf(h[t][2 * kb + 1][0], 0.f), fmaxf(h[t][2 * kb + 1][1], 0.f));
        a2[t][kb][3] = pack_half2(fmaxf(h[t][2 * kb + 1][2], 0.f), fmaxf(h[t][2 * kb + 1][3], 0.f));
      }
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    o[t][0] = W.b3[tig * 2];
    o[t][1] = W.b3[tig * 2 + 1];
    o[t][2] = o[t][0];
    o[t][3] = o[t][1];
  }
  // layer 2 by pairs of n-tiles (2 k3, 2 k3 + 1), each pair then one k-block of layer 3
#pragma unroll
  for (int k3 = 0; k3 < kK2 / 16; ++k3) {
    float g[2][2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int nt = 2 * k3 + q;
      const float c0 = W.b2[nt * 8 + tig * 2], c1 = W.b2[nt * 8 + tig * 2 + 1];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        g[t][q][0] = c0;
        g[t][q][1] = c1;
        g[t][q][2] = c0;
        g[t][q][3] = c1;
      }
    }
#pragma unroll
    for (int kb = 0; kb < kK2 / 16; ++kb)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        uint32_t b0, b1;
        b_frag(W.w2, kP2, kb, 2 * k3 + q, lane, b0, b1);
#pragma unroll
        for (int t = 0; t < 2; ++t)
          mma16816(g[t][q], a2[t][kb][0], a2[t][kb][1], a2[t][kb][2], a2[t][kb][3], b0, b1);
      }
    uint32_t b0, b1;
    b_frag(W.w3, kP2, k3, 0, lane, b0, b1);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const uint32_t x0 = pack_half2(fmaxf(g[t][0][0], 0.f), fmaxf(g[t][0][1], 0.f));
      const uint32_t x1 = pack_half2(fmaxf(g[t][0][2], 0.f), fmaxf(g[t][0][3], 0.f));
      const uint32_t x2 = pack_half2(fmaxf(g[t][1][0], 0.f), fmaxf(g[t][1][1], 0.f));
      const uint32_t x3 = pack_half2(fmaxf(g[t][1][2], 0.f), fmaxf(g[t][1][3], 0.f));
      mma16816(o[t], x0, x1, x2, x3, b0, b1);
    }
  }
}

// Inference on an array of feature rows X [n][27] -> Y [n][3] (testing the kernel).
__global__ void __launch_bounds__(kInferWarps * 32) mlp_infer_kernel(const float* __restrict__ P,
                                                                    const float* __restrict__ X, long long n,
                                                                    float* __restrict__ Y) {
  __shared__ InferSmem S;
  build_image(S.W, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float ins = P[oInS], outs = P[oOutS];
  __half* xs = S.x[w];
  for (long long r0 = ((long long)blockIdx.x * kInferWarps + w) * 16; r0 < n;
       r0 += (long long)gridDim.x * kInferWarps * 16) {
    if (lane < 16) {
      const long long r = r0 + lane;
#pragma unroll
      for (int c = 0; c < kK1; ++c)
        xs[lane * kXP + c] = __float2half_rn(r < n && c < kIn ? X[r * kIn + c] * ins : 0.0f);
    }
    __syncwarp();
    float o[4];
    mlp_rows(S, xs, lane, o);
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const long long r = r0 + gid + 8 * half;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = tig * 2 + c;
        if (r < n && col < kOut) Y[r * kOut + col] = o[2 * half + c] * outs;
      }
    }
    __syncwarp();
  }
}

// In a time step, after the first interpolation: the first MDF force of every point is
// the network's prediction from its deficit stencil (replacing 2 (U_b - u_b*)).  One
// warp per particle: the particle's deficits are staged in shared memory once, then
// its points go through the network 32 at a time (two m16 tiles sharing every weight
// fragment), lane r building the feature row of point r of the pass and storing it as
// four 16-byte words.
constexpr int kMaxNl = 256;  // points per particle the step kernel stages

__global__ void __launch_bounds__(kInferWarps * 32) mlp_step_kernel(IbmArgs A, const float* __restrict__ P,
                                                                   const WeightImage* __restrict__ img) {
  __shared__ WeightImage W;
  __shared__ __align__(16) __half xs32[kInferWarps][32 * kXP];  // the 32 feature rows of a pass
  __shared__ float dsm[kInferWarps][2 * kMaxNl];
  __shared__ float frame[2 * kMaxNl];
  copy_image(W, img);
  for (int k = threadIdx.x; k < A.nl; k += blockDim.x) {
    float nx, ny;
    point_frame(A.ref_f, k, nx, ny);
    frame[2 * k] = nx;
    frame[2 * k + 1] = ny;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const float ins = P[oInS], outs = P[oOutS];
  const int nl = A.nl;
  __half* xs = xs32[w];
  float* d = dsm[w];
  // up to 32 points a particle: lane k holds point k's deficit of the warp's next
  // particle, loaded while the network runs on the current one
  const int stride = gridDim.x * kInferWarps;
  const bool pre = nl <= 32;
  float nxt[2] = {0.0f, 0.0f};
  auto fetch = [&](int i) {
    if (!pre || i >= A.np || lane >= nl) return;
    const long long b = (long long)i * nl + lane;
    const float2 U = reinterpret_cast<const float2*>(A.Ub)[b], u = reinterpret_cast<const float2*>(A.ubs)[b];
    nxt[0] = U.x - u.x;
    nxt[1] = U.y - u.y;
  };
  fetch(blockIdx.x * kInferWarps + w);
  for (int i = blockIdx.x * kInferWarps + w; i < A.np; i += stride) {
    const long long base = (long long)i * nl;
    if (pre) {
      if (lane < nl) {
        d[2 * lane] = nxt[0];
        d[2 * lane + 1] = nxt[1];
      }
      fetch(i + stride);
    } else {
      for (int k = lane; k < nl; k += 32) {
        const long long b = base + k;
        d[2 * k] = A.Ub[2 * b] - A.ubs[2 * b];
        d[2 * k + 1] = A.Ub[2 * b + 1] - A.ubs[2 * b + 1];
      }
    }
    __syncwarp();
    for (int r0 = 0; r0 < nl; r0 += 32) {
      {
        const int k = r0 + lane;
        uint32_t wd[kK1 / 2];  // the row as 16 words of two halves
#pragma unroll
        for (int q = 0; q < kK1 / 2; ++q) wd[q] = 0u;
        if (k < nl) {
          const float nx = frame[2 * k], ny = frame[2 * k + 1];
          float x[kIn];
#pragma unroll
          for (int j = 0; j < 9; ++j) {
            int kk = k + j - 4;
            kk = kk < 0 ? kk + nl : (kk >= nl ? kk - nl : kk);
            const float dx = d[2 * kk], dy = d[2 * kk + 1];
            x[3 * j] = (dx * nx + dy * ny) * ins;
            x[3 * j + 1] = (-dx * ny + dy * nx) * ins;
            x[3 * j + 2] = 0.0f;
          }
#pragma unroll
          for (int q = 0; q < kK1 / 2; ++q)
            wd[q] = pack_half2(2 * q < kIn ? x[2 * q] : 0.0f, 2 * q + 1 < kIn ? x[2 * q + 1] : 0.0f);
        }
        uint4* row = reinterpret_cast<uint4*>(xs + lane * kXP);
#pragma unroll
        for (int q = 0; q < kK1 / 8; ++q) row[q] = make_uint4(wd[4 * q], wd[4 * q + 1], wd[4 * q + 2], wd[4 * q + 3]);
      }
      __syncwarp();
      float o[2][4];
      mlp_rows32(W, xs, lane, o);
      if (tig == 0) {  // columns 0 and 1: normal and tangential force
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int k = r0 + t * 16 + gid + 8 * half;
            if (k >= nl) continue;
            const long long b = base + k;
            const float nx = frame[2 * k], ny = frame[2 * k + 1];
            const float fn = o[t][2 * half] * outs, ft = o[t][2 * half + 1] * outs;
            const float Fx = fn * nx - ft * ny, Fy = fn * ny + ft * nx;
            A.dFb[2 * b] = Fx;
            A.dFb[2 * b + 1] = Fy;
            A.Fb[2 * b] = Fx;
            A.Fb[2 * b + 1] = Fy;
          }
      }
      __syncwarp();
    }
  }
}

// 3D: the same replacement of the first MDF force, point-parallel: a warp takes 16
// points at a time (grid stride), gathers their stencils from global memory (the
// deficits of a sphere's points stay in L1/L2 between the warp's rows), runs them
// through the network and writes F_b = dF_b back in the global frame.
__global__ void __launch_bounds__(kInferWarps * 32) mlp_step3_kernel(IbmArgs A, const float* __restrict__ P,
                                                                    const WeightImage* __restrict__ img) {
  __shared__ InferSmem S;
  copy_image(S.W, img);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const float ins = P[oInS], outs = P[oOutS];
  __half* xs = S.x[w];
  for (long long r0 = ((long long)blockIdx.x * kInferWarps + w) * 16; r0 < A.npts;
       r0 += (long long)gridDim.x * kInferWarps * 16) {
    if (lane < 16) {
      const long long b = r0 + lane;
      if (b < A.npts) {
        const int k = (int)(b % A.nl);
        float x[kIn];
        features_3d(A, b - k, k, x);
#pragma unroll
        for (int c = 0; c < kK1; ++c) xs[lane * kXP + c] = __float2half_rn(c < kIn ? x[c] * ins : 0.0f);
      } else {
#pragma unroll
        for (int c = 0; c < kK1; ++c) xs[lane * kXP + c] = __float2half_rn(0.0f);
      }
    }
    __syncwarp();
    float o[4];
    mlp_rows(S, xs, lane, o);
    // column 2 (t2 component) sits in the lane with tig = 1 of the same row group
    const float c2a = __shfl_down_sync(0xffffffffu, o[0], 1), c2b = __shfl_down_sync(0xffffffffu, o[2], 1);
    if (tig == 0) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const long long b = r0 + gid + 8 * half;
        if (b >= A.npts) continue;
        const int k = (int)(b % A.nl);
        const float* F = A.frame3 + 9 * k;
        const float fl[3] = {o[2 * half] * outs, o[2 * half + 1] * outs, (half ? c2b : c2a) * outs};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float v = fl[0] * F[c] + fl[1] * F[3 + c] + fl[2] * F[6 + c];
          A.dFb[3 * b + c] = v;
          A.Fb[3 * b + c] = v;
        }
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ training (FP32)
// forward, thread per sample: H1, H2 (after ReLU) and Y kept for the backward pass
__global__ void __launch_bounds__(128) mlp_fwd_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                      int B, float* __restrict__ H1, float* __restrict__ H2,
                                                      float* __restrict__ Y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  float x[kIn], h1[kH];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = X[(long long)s * kIn + i];
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float a = P[ob1 + j];
#pragma unroll
    for (int i = 0; i < kIn; ++i) a += x[i] * P[oW1 + i * kH + j];
    h1[j] = fmaxf(a, 0.0f);
    H1[(long long)s * kH + j] = h1[j];
  }
  float y[kOut];
#pragma unroll
  for (int o = 0; o < kOut; ++o) y[o] = P[ob3 + o];
  for (int j = 0; j < kH; ++j) {
    float a = P[ob2 + j];
#pragma unroll
    for (int i = 0; i < kH; ++i) a += h1[i] * P[oW2 + i * kH + j];
    a = fmaxf(a, 0.0f);
    H2[(long long)s * kH + j] = a;
#pragma unroll
    for (int o = 0; o < kOut; ++o) y[o] += a * P[oW3 + j * kOut + o];
  }
#pragma unroll
  for (int o = 0; o < kOut; ++o) Y[(long long)s * kOut + o] = y[o];
}

// backward through the activations, thread per sample.  Loss: mean over the samples of
// the squared error summed over the outputs.  Writes dY, dH2 and dH1 (pre-activation
// gradients) and adds the sample's squared error to *loss.
__global__ void __launch_bounds__(128) mlp_bwd_kernel(const float* __restrict__ P, const float* __restrict__ T,
                                                      int B, const float* __restrict__ H1,
                                                      const float* __restrict__ H2, const float* __restrict__ Y,
                                                      float* __restrict__ dY, float* __restrict__ dH2,
                                                      float* __restrict__ dH1, double* loss) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  float dy[kOut];
  double se = 0.0;
#pragma unroll
  for (int o = 0; o < kOut; ++o) {
    const float e = Y[(long long)s * kOut + o] - T[(long long)s * kOut + o];
    se += (double)e * e;
    dy[o] = 2.0f * e / (float)B;
    dY[(long long)s * kOut + o] = dy[o];
  }
  atomicAdd(loss, se / B);
  float d2[kH];
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float a = 0.0f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) a += dy[o] * P[oW3 + j * kOut + o];
    d2[j] = H2[(long long)s * kH + j] > 0.0f ? a : 0.0f;
    dH2[(long long)s * kH + j] = d2[j];
  }
  for (int i = 0; i < kH; ++i) {
    float a = 0.0f;
#pragma unroll
    for (int j = 0; j < kH; ++j) a += d2[j] * P[oW2 + i * kH + j];
    dH1[(long long)s * kH + i] = H1[(long long)s * kH + i] > 0.0f ? a : 0.0f;
  }
}

// weight gradients, thread per parameter, summed over the batch in sample order
__global__ void __launch_bounds__(128) mlp_wgrad_kernel(const float* __restrict__ X, int B,
                                                        const float* __restrict__ H1, const float* __restrict__ H2,
                                                        const float* __restrict__ dY, const float* __restrict__ dH2,
                                                        const float* __restrict__ dH1, float* __restrict__ G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= oInS) return;
  const float *A = nullptr, *D = nullptr;
  int ai = 0, di = 0, an = 0, dn = 0;
  if (p < ob1) {  // W1[i][j]
    A = X; an = kIn; ai = p / kH; D = dH1; dn = kH; di = p % kH;
  } else if (p < oW2) {
    D = dH1; dn = kH; di = p - ob1;
  } else if (p < ob2) {
    A = H1; an = kH; ai = (p - oW2) / kH; D = dH2; dn = kH; di = (p - oW2) % kH;
  } else if (p < oW3) {
    D = dH2; dn = kH; di = p - ob2;
  } else if (p < ob3) {
    A = H2; an = kH; ai = (p - oW3) / kOut; D = dY; dn = kOut; di = (p - oW3) % kOut;
  } else {
    D = dY; dn = kOut; di = p - ob3;
  }
  float g = 0.0f;
  for (int s = 0; s < B; ++s) {
    const float d = D[(long long)s * dn + di];
    g += A ? A[(long long)s * an + ai] * d : d;
  }
  G[p] = g;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8), step t >= 1; the two scales are not trained
__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                                float* __restrict__ V, long long t, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= oInS) return;
  const float b1 = 0.9f, b2 = 0.999f;
  const float m = b1 * M[p] + (1.0f - b1) * G[p];
  const float v = b2 * V[p] + (1.0f - b2) * G[p] * G[p];
  M[p] = m;
  V[p] = v;
  const float mh = m / (1.0f - powf(b1, (float)t)), vh = v / (1.0f - powf(b2, (float)t));
  P[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// ------------------------------------------------------------------ launchers
size_t mlp_scratch_floats(int B) { return (size_t)B * (2 * kH + kOut + 2 * kH + kOut) + 8; }

cudaError_t launch_mlp_samples(const IbmArgs& A, float* X, float* Y, cudaStream_t s) {
  if (A.npts == 0) return cudaSuccess;
  mlp_samples_kernel<<<(unsigned)((A.npts + 127) / 128), 128, 0, s>>>(A, X, Y);
  return cudaGetLastError();
}

int mlp_max_points() { return kMaxNl; }
size_t mlp_image_bytes() { return sizeof(WeightImage); }

cudaError_t launch_mlp_image(const float* P, void* img, cudaStream_t s) {
  mlp_image_kernel<<<1, 256, 0, s>>>(P, static_cast<WeightImage*>(img));
  return cudaGetLastError();
}

cudaError_t launch_mlp_step(const IbmArgs& A, const float* P, const void* img, cudaStream_t s) {
  if (A.D == 3) {
    if (A.npts == 0) return cudaSuccess;
    const long long groups = (A.npts + 15) / 16;
    const unsigned grid = (unsigned)std::min<long long>((groups + kInferWarps - 1) / kInferWarps, 152LL * 8);
    mlp_step3_kernel<<<grid, kInferWarps * 32, 0, s>>>(A, P, static_cast<const WeightImage*>(img));
    return cudaGetLastError();
  }
  if (A.np == 0) return cudaSuccess;
  static int resident = 0;  // blocks the GPU holds at once: each warp then walks its particles
  if (resident == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_step_kernel, kInferWarps * 32, 0);
    if (e != cudaSuccess) return e;
    resident = std::max(1, sms * per_sm);
  }
  const unsigned grid = (unsigned)std::min((A.np + kInferWarps - 1) / kInferWarps, resident);
  mlp_step_kernel<<<grid, kInferWarps * 32, 0, s>>>(A, P, static_cast<const WeightImage*>(img));
  return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const float* P, const float* X, long long n, float* Y, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const long long tiles = (n + 15) / 16;
  const unsigned grid = (unsigned)min((tiles + kInferWarps - 1) / kInferWarps, (long long)152 * 8);
  mlp_infer_kernel<<<grid, kInferWarps * 32, 0, s>>>(P, X, n, Y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* P, const float* X, const float* T, int B, float* G, double* d_loss,
                            float* scratch, cudaStream_t s) {
  float* H1 = scratch;
  float* H2 = H1 + (size_t)B * kH;
  float* Y = H2 + (size_t)B * kH;
  float* dH1 = Y + (size_t)B * kOut;
  float* dH2 = dH1 + (size_t)B * kH;
  float* dY = dH2 + (size_t)B * kH;
  const unsigned g = (unsigned)((B + 127) / 128);
  cudaError_t e = cudaMemsetAsync(d_loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  mlp_fwd_kernel<<<g, 128, 0, s>>>(P, X, B, H1, H2, Y);
  mlp_bwd_kernel<<<g, 128, 0, s>>>(P, T, B, H1, H2, Y, dY, dH2, dH1, d_loss);
  mlp_wgrad_kernel<<<(oInS + 127) / 128, 128, 0, s>>>(X, B, H1, H2, dY, dH2, dH1, G);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* P, const float* G, float* M, float* V, long long t, float lr,
                            cudaStream_t s) {
  mlp_adam_kernel<<<(oInS + 255) / 256, 256, 0, s>>>(P, G, M, V, t, lr);
  return cudaGetLastError();
}

}  // namespace ibmlbm

// ------------------------------------------------------------------ C ABI
#include "ibmlbm.h"

extern "C" {

int32_t ibm_lbm_mlp_param_count(void) { return ibmlbm::kMlpParams; }

int ibm_lbm_mlp_scratch_size(int32_t batch, size_t* bytes) {
  if (batch <= 0 || !bytes) {
    ibmlbm::set_last_error("batch must be positive and bytes non-NULL");
    return IBMLBM_ERR_INVALID_ARG;
  }
  *bytes = sizeof(float) * ibmlbm::mlp_scratch_floats(batch) + sizeof(double) + 256;
  return IBMLBM_OK;
}

int ibm_lbm_mlp_grad(const float* d_params, const float* d_X, const float* d_T, int32_t batch, float* d_grad,
                     double* h_loss, void* d_scratch, size_t scratch_bytes, void* stream) {
  size_t need = 0;
  if (ibm_lbm_mlp_scratch_size(batch, &need) != IBMLBM_OK) return IBMLBM_ERR_INVALID_ARG;
  if (!d_params || !d_X || !d_T || !d_grad || !d_scratch || scratch_bytes < need ||
      reinterpret_cast<uintptr_t>(d_scratch) % 16) {
    ibmlbm::set_last_error("mlp_grad: NULL pointer or scratch too small / misaligned");
    return IBMLBM_ERR_INVALID_ARG;
  }
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* d_loss = reinterpret_cast<double*>(d_scratch);
  float* scr = reinterpret_cast<float*>(static_cast<char*>(d_scratch) + 256);
  cudaError_t e = ibmlbm::launch_mlp_grad(d_params, d_X, d_T, batch, d_grad, d_loss, scr, s);
  if (e == cudaSuccess && h_loss) e = cudaMemcpyAsync(h_loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && h_loss) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ibmlbm::set_last_error(std::string("mlp_grad: ") + cudaGetErrorString(e));
    return IBMLBM_ERR_CUDA;
  }
  return IBMLBM_OK;
}

int ibm_lbm_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t t, float lr,
                     void* stream) {
  if (!d_params || !d_grad || !d_m || !d_v || t < 1) {
    ibmlbm::set_last_error("mlp_adam: NULL pointer or t < 1");
    return IBMLBM_ERR_INVALID_ARG;
  }
  const cudaError_t e = ibmlbm::launch_mlp_adam(d_params, d_grad, d_m, d_v, t, lr, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    ibmlbm::set_last_error(std::string("mlp_adam: ") + cudaGetErrorString(e));
    return IBMLBM_ERR_CUDA;
  }
  return IBMLBM_OK;
}

int ibm_lbm_mlp_infer(const float* d_params, const float* d_X, int64_t n, float* d_Y, void* stream) {
  if (!d_params || (n > 0 && (!d_X || !d_Y)) || n < 0) {
    ibmlbm::set_last_error("mlp_infer: NULL pointer or n < 0");
    return IBMLBM_ERR_INVALID_ARG;
  }
  const cudaError_t e = ibmlbm::launch_mlp_infer(d_params, d_X, n, d_Y, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    ibmlbm::set_last_error(std::string("mlp_infer: ") + cudaGetErrorString(e));
    return IBMLBM_ERR_CUDA;
  }
  return IBMLBM_OK;
}

}  // extern "C"
