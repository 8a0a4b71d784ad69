// Immersed-boundary kernels (Sec. 2.2, Sec. 4) and the particle update (Sec. 2.3).
//
// Multi-direct forcing, iteration m = 1..M, per particle:
//   interpolation  u_b = sum delta(x - X_b) (u* + dt f_IB / (2 rho_f))   (Eq. 7, 12, 47)
//                  dF_b = 2 rho_f (U_b - u_b) / dt, F_b += dF_b           (Eq. 10)
//   spreading      f_IB += sum_b dF_b delta(x - X_b) dV                    (Eq. 11, 13, 48)
// Each particle's node box lives in shared memory: 2D one warp per particle, 3D one
// block per sphere, with one interpolation and one spreading launch per iteration.
// The box cells reach f_IB with one global atomic per cell.
// Gathering u* + f_IB/2 equals the paper's u^(m-1) = u^(m-2) + dt D_E dF/(2 rho_f)
// by linearity, so no separate velocity field is updated between iterations.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "launch.h"
#include "pdf_access.cuh"

namespace ibmlbm {

// 4-point regularised delta function (Fig. 2b; Peskin's form)
__device__ __forceinline__ float delta4(float r) {
  const float a = fabsf(r);
  if (a <= 1.0f) return 0.125f * (3.0f - 2.0f * a + sqrtf(fmaxf(0.0f, 1.0f + 4.0f * a - 4.0f * a * a)));
  if (a <= 2.0f) return 0.125f * (5.0f - 2.0f * a - sqrtf(fmaxf(0.0f, -7.0f + 12.0f * a - 4.0f * a * a)));
  return 0.0f;
}

// 3-point regularised delta function (Fig. 2b; the form of Roma, Peskin and Berger,
// used with drs = 1.9 in Sec. 2.2)
__device__ __forceinline__ float delta3(float r) {
  const float a = fabsf(r);
  if (a <= 0.5f) return (1.0f + sqrtf(fmaxf(0.0f, 1.0f - 3.0f * a * a))) * (1.0f / 3.0f);
  if (a <= 1.5f) return (5.0f - 3.0f * a - sqrtf(fmaxf(0.0f, -2.0f + 6.0f * a - 3.0f * a * a))) * (1.0f / 6.0f);
  return 0.0f;
}

__device__ __forceinline__ float delta_w(int kind, float r) { return kind == 3 ? delta3(r) : delta4(r); }

// The weights of the four support nodes along one axis, at offsets (t - 1) - f from
// the point (t = 0..3, f as support_first gives it).  At these four offsets every
// branch of a delta function takes the same square root, so one suffices:
//   4-point (f in [0, 1)), q = sqrt(1 + 4 f - 4 f^2):
//     (3 - 2f - q) / 8, (3 - 2f + q) / 8, (1 + 2f + q) / 8, (1 + 2f - q) / 8;
//   3-point (f in [-1/2, 1/2)), q = sqrt(1 - 3 f^2):
//     (2 - 3f - q) / 6, (1 + q) / 3, (2 + 3f - q) / 6, 0.
// (Substituting |r| = 1 + f, f, 1 - f, 2 - f into the two branches of each function.)
__device__ __forceinline__ void delta_weights(int kind, float f, float (&w)[4]) {
  if (kind == 3) {
    const float q = sqrtf(fmaxf(0.0f, 1.0f - 3.0f * f * f));
    w[0] = (2.0f - 3.0f * f - q) * (1.0f / 6.0f);
    w[1] = (1.0f + q) * (1.0f / 3.0f);
    w[2] = (2.0f + 3.0f * f - q) * (1.0f / 6.0f);
    w[3] = 0.0f;
  } else {
    const float q = sqrtf(fmaxf(0.0f, 1.0f + 4.0f * f - 4.0f * f * f));
    w[0] = 0.125f * (3.0f - 2.0f * f - q);
    w[1] = 0.125f * (3.0f - 2.0f * f + q);
    w[2] = 0.125f * (1.0f + 2.0f * f + q);
    w[3] = 0.125f * (1.0f + 2.0f * f - q);
  }
}

// First support node along one axis of a fixed-point coordinate X, and fr such that
// the offset of support node t (t = 0..3) from X is (t - 1) - fr: 4-point nodes
// floor(X)-1 .. floor(X)+2 (fr = frac X); 3-point nodes round(X)-1 .. round(X)+1
// (fr = X - round X), whose fourth node then carries weight zero.
__device__ __forceinline__ int support_first(int kind, long long X, float& fr) {
  if (kind == 3) {
    const long long r = X + (1LL << 31);  // X + 1/2
    fr = fix_frac(r) - 0.5f;
    return fix_anchor(r) - 1;
  }
  fr = fix_frac(X);
  return fix_anchor(X) - 1;
}

// 2D kernels with one warp per particle and the particle's node box in shared memory
// (kIbmWarps particles per block, no block-wide barrier).  A box cell holds both
// components (float2); rows are box_pitch(S) cells apart, so the 4 x 4 support of a
// point falls on 16 different bank pairs.  In the later interpolations the box
// reaches shared memory through cp.async, so all of a warp's loads are in flight at
// once.  f_IB is stored interleaved in 2D ([N][2]).
constexpr int kIbmWarps = 8;

__device__ __forceinline__ void cp_async8(float2* dst, const float2* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// 16 bytes, or 16 zero bytes when pred is false
__device__ __forceinline__ void cp_async16z(void* dst, const void* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// floats of shared memory per warp: the box [S][P] float2, then
//   interpolation, mode 1: f_IB of the box [S][P] float2;
//   spreading: the point table, weights [32][kTw] and (F_x, F_y, first cell) [32] float4.
constexpr int kTw = 9;  // the 4 + 4 one-dimensional weights of a point (+1 against bank conflicts)
__host__ __device__ inline int interp2_warp_floats(int mode, int S) {
  return 2 * S * box_pitch(S) * (mode == 0 ? 1 : 2);
}
__host__ __device__ inline int spread2_warp_floats(int S) { return 2 * S * box_pitch(S) + 32 * kTw + 32 * 4; }

size_t ibm_box2_smem(int box) {
  const int a = interp2_warp_floats(1, box), c = spread2_warp_floats(box);
  return sizeof(float) * (size_t)kIbmWarps * (size_t)max(a, c);
}

// Warps per block of a single run's 2D interpolation and spreading: kIbmWarps, fewer
// for particles whose boxes would not fit 227 KB of shared memory per block (one warp
// per particle either way; the kernels take the count from blockDim).
int ibm2_warps(int box) {
  const size_t per = sizeof(float) * (size_t)max(interp2_warp_floats(1, box), spread2_warp_floats(box));
  int w = kIbmWarps;
  while (w > 1 && per * w > 227 * 1024) --w;
  return w;
}
size_t ibm2_smem(int box) {
  const int a = interp2_warp_floats(1, box), c = spread2_warp_floats(box);
  return sizeof(float) * (size_t)ibm2_warps(box) * (size_t)max(a, c);
}

// box node (row r, column c) -> grid node; false beyond a wall
__device__ __forceinline__ bool box_node(const Geo& g, int ox, int oy, int r, int c, int& gx, int& gy) {
  gx = ox + c;
  gy = oy + r;
  bool ok = true;
  if (gx < 0 || gx >= g.nx) {
    if (g.per[0]) gx = ((gx % g.nx) + g.nx) % g.nx; else ok = false;
  }
  if (gy < 0 || gy >= g.ny) {
    if (g.per[1]) gy = ((gy % g.ny) + g.ny) % g.ny; else ok = false;
  }
  return ok;
}

// Interpolation (Eq. 47), iteration m.
//   MODE 0 (m = 1, or m = 0: box only, when no forcing iteration runs): u* (Eq. 5) of
//     every node of the particle's box from the PDFs (AA-parity addressing), kept in
//     the particle's box buffer for the later iterations and the interior sums;
//   MODE 1 (m >= 2): the box buffer plus f_IB/2; with m < 0 the same gather after the
//     last iteration only records the residual U_b - D_I u^(M).
// Lane k then interpolates point k from shared memory.  Box nodes beyond a wall hold
// zero, which drops them from the sum.
// wf: floats of shared memory per warp (0: this mode's need for the box).  A kernel
// whose warps go on to other particles independently passes one stride for all.
// NU: box nodes a lane takes per round in MODE 0, all loaded before any is reduced
// (four measured faster in the batch's fused launches, two everywhere else).
template <int SC, int PARITY, int MODE, int ST, int NU = 2>
__device__ __forceinline__ void interp2_body(const IbmArgs& A, int m, unsigned blk, int wf = 0) {
  extern __shared__ __align__(16) float smem_i[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int slot = (int)blk * (int)(blockDim.x >> 5) + wib;  // warps per block: blockDim
  if (slot >= A.np) return;  // whole warp
  const int i = A.order[slot];
  const int S = SC ? SC : A.box, P = box_pitch(S), cells = S * P;
  __syncwarp();  // the warp's shared memory is free (a particle before may have used it)
  float2* box = reinterpret_cast<float2*>(smem_i + (size_t)wib * (wf ? wf : interp2_warp_floats(MODE, S)));
  float2* aux = box + cells;
  float2* ub = reinterpret_cast<float2*>(A.ubox) + (size_t)i * cells;
  // the first point of this lane is loaded before the box, so both latencies overlap
  const bool has0 = m != 0 && lane < A.nl;
  const long long b0 = (long long)i * A.nl + lane;
  long long X0x = 0, X0y = 0;
  float U0x = 0.0f, U0y = 0.0f;
  if (has0) {
    X0x = A.Xb[b0 * 2];
    X0y = A.Xb[b0 * 2 + 1];
    U0x = A.Ub[b0 * 2];
    U0y = A.Ub[b0 * 2 + 1];
  }
  const int ox = fix_anchor(A.Xcf[(long long)i * 2 + 0]) - A.rcell - 2;
  const int oy = fix_anchor(A.Xcf[(long long)i * 2 + 1]) - A.rcell - 2;
  int ash = 0;  // MODE 1: offset of the f_IB rows in the buffer (aux[r P + c + ash] is node (ox + c, oy + r))
  if (MODE == 0) {
    // Only the nodes within R + 2 sqrt(2) of the centre are needed: every support node
    // of a point on the circle (at most 2 nodes from it along each axis) and the
    // interior the momentum sums use.  The box corners beyond hold zero.
    const float fx = fix_frac(A.Xcf[(long long)i * 2 + 0]), fy = fix_frac(A.Xcf[(long long)i * 2 + 1]);
    const float Rn = A.radius_f + 2.8285f + 0.01f, Rn2 = Rn * Rn;
    const int c0 = A.rcell + 2;  // box column / row of the anchor node
    // NU box nodes per lane and round
    for (int t0 = lane; t0 < S * S; t0 += 32 * NU) {
      float fa[NU][9];
      bool ok[NU];
#pragma unroll
      for (int k = 0; k < NU; ++k) {
        const int t = t0 + 32 * k;
        ok[k] = false;
        if (t >= S * S) continue;
        const int r = t / S, c = t - r * S;
        const float dx = (float)(c - c0) - fx, dy = (float)(r - c0) - fy;
        if (dx * dx + dy * dy > Rn2) continue;
        int gx, gy;
        ok[k] = box_node(A.g, ox, oy, r, c, gx, gy);
        if (!ok[k]) continue;
        const long long n = (long long)gx + (long long)A.g.nx * gy;
        if (PARITY == 1 && gx >= 1 && gx <= A.g.nx - 2 && gy >= 1 && gy <= A.g.ny - 2)
          load_pdfs<Lat<2>, PARITY, ST, true>(A.g, A.f, gx, gy, 0, n, fa[k]);  // fixed offsets
        else
          load_pdfs<Lat<2>, PARITY, ST>(A.g, A.f, gx, gy, 0, n, fa[k]);
      }
#pragma unroll
      for (int k = 0; k < NU; ++k) {
        const int t = t0 + 32 * k;
        if (t >= S * S) continue;
        const int r = t / S, c = t - r * S;
        float2 v = make_float2(0.0f, 0.0f);
        if (ok[k]) {
          float us[3], s1;
          moments<Lat<2>>(fa[k], us, s1);
          v = make_float2(us[0], us[1]);
        }
        box[r * P + c] = v;
        ub[r * P + c] = v;
      }
    }
    __syncwarp();
    if (m == 0) return;  // box u* only (no multi-direct forcing iteration this step)
  } else {
    for (int q = lane; q < cells / 2; q += 32) cp_async16(box + 2 * q, ub + 2 * q);
    const float2* fib2 = reinterpret_cast<const float2*>(A.fib);
    // Where the box's rows lie inside the domain along x (and rows hold an even number
    // of nodes, so that a pair of nodes starting at an even node is 16-byte aligned),
    // f_IB comes two nodes per copy; a box starting at an odd node keeps its rows one
    // cell on in the buffer (ash), the spare cells of the row pitch taking the extra node.
    if (A.g.nx % 2 == 0 && P >= S + 2 && ox >= 0 && ox + S <= A.g.nx - 1) {
      ash = ox & 1;
      const int base = ox - ash, nch = (S + ash + 1) / 2;
      for (int t = lane; t < S * nch; t += 32) {
        const int r = t / nch, j = t - r * nch;
        int gy = oy + r;
        bool ok = true;
        if (gy < 0 || gy >= A.g.ny) {
          if (A.g.per[1]) gy = ((gy % A.g.ny) + A.g.ny) % A.g.ny;
          else ok = false;
        }
        const long long n = ok ? (long long)(base + 2 * j) + (long long)A.g.nx * gy : 0;
        cp_async16z(aux + r * P + 2 * j, fib2 + n, ok && IBMLBM_CHK(n + 1, A.g.N));
      }
    } else {
      for (int t = lane; t < S * S; t += 32) {
        const int r = t / S, c = t - r * S;
        int gx, gy;
        const bool ok = box_node(A.g, ox, oy, r, c, gx, gy);
        const long long n = ok ? (long long)gx + (long long)A.g.nx * gy : 0;
        cp_async8(aux + r * P + c, fib2 + n, ok && IBMLBM_CHK(n, A.g.N));
      }
    }
    cp_async_wait_all();
    __syncwarp();
  }
  for (int k = lane; k < A.nl; k += 32) {
    const long long b = (long long)i * A.nl + k;
    const bool first = k == lane;
    const long long Xx = first ? X0x : A.Xb[b * 2], Xy = first ? X0y : A.Xb[b * 2 + 1];
    const float Ux = first ? U0x : A.Ub[b * 2], Uy = first ? U0y : A.Ub[b * 2 + 1];
    float rx, ry;
    const int lx0 = support_first(A.delta_kind, Xx, rx) - ox, ly0 = support_first(A.delta_kind, Xy, ry) - oy;
    float acc0 = 0.0f, acc1 = 0.0f;
    if (lx0 < 0 || ly0 < 0 || lx0 + 3 >= S || ly0 + 3 >= S) {
      atomicOr(A.status, ST_CAPACITY);
    } else {
      float wx[4], wyv[4];
      delta_weights(A.delta_kind, rx, wx);
      delta_weights(A.delta_kind, ry, wyv);
#pragma unroll
      for (int sy = 0; sy < 4; ++sy) {
        const float wy = wyv[sy];
        const int o = (ly0 + sy) * P + lx0;
        float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
        for (int sx = 0; sx < 4; ++sx) {
          float2 v = box[o + sx];
          if (MODE == 1) {
            const float2 h = aux[o + ash + sx];
            v.x += 0.5f * h.x;
            v.y += 0.5f * h.y;
          }
          a0 += wx[sx] * v.x;
          a1 += wx[sx] * v.y;
        }
        acc0 += wy * a0;
        acc1 += wy * a1;
      }
    }
    if (m < 0) {  // residual pass after the last iteration: r_b = U_b - D_I u^(M)
      A.res[b * 2] = Ux - acc0;
      A.res[b * 2 + 1] = Uy - acc1;
      continue;
    }
    const float d0 = 2.0f * (Ux - acc0), d1 = 2.0f * (Uy - acc1);
    A.dFb[b * 2] = d0;
    A.dFb[b * 2 + 1] = d1;
    if (m == 1) {
      A.Fb[b * 2] = d0;
      A.Fb[b * 2 + 1] = d1;
      A.ubs[b * 2] = acc0;
      A.ubs[b * 2 + 1] = acc1;
    } else {
      A.Fb[b * 2] += d0;
      A.Fb[b * 2 + 1] += d1;
    }
  }
}

template <int SC, int PARITY, int MODE, int ST, bool FUSED>
__global__ void __launch_bounds__(kIbmWarps * 32) ibm_interp2_kernel(IbmArgs A0, int m, Fuse FU) {
  pdl_enter();
  IBMLBM_BIND(FUSED, IbmArgs, A, A0, FU, blk);
  if constexpr (FUSED) {  // members differ in box size: run the code compiled for this one
    switch (A.box) {
      case 14: interp2_body<14, PARITY, MODE, ST, 4>(A, m, blk); return;
      case 16: interp2_body<16, PARITY, MODE, ST, 4>(A, m, blk); return;
      case 18: interp2_body<18, PARITY, MODE, ST, 4>(A, m, blk); return;
      case 20: interp2_body<20, PARITY, MODE, ST, 4>(A, m, blk); return;
      case 22: interp2_body<22, PARITY, MODE, ST, 4>(A, m, blk); return;
      default: interp2_body<0, PARITY, MODE, ST, 4>(A, m, blk); return;
    }
  }
  interp2_body<SC, PARITY, MODE, ST>(A, m, blk);
}

// Spreading (Eq. 48) without shared-memory atomics.  The point's owner lane writes a
// table row (the four weights delta_x and the four delta_y of its support, its force
// dF_b dV, the box cell of its first support node).  Then the 16 lanes of each
// half-warp take one point each, one support node per lane (its weight the product of
// its column's and its row's): half 0 point j, half 1 point j + H (H = half the
// group), about a diameter apart on the circle.  Where the two supports could share a
// node (anchors at most 3 apart on both axes) the halves take turns.  So no two lanes
// of an instruction touch one cell and plain read-add-write is exact.  Finally the warp
// adds the non-zero box cells to f_IB with one global vector atomic per cell.
template <int SC>
__device__ __forceinline__ void spread2_body(const IbmArgs& A, unsigned blk, int wf = 0) {
  extern __shared__ __align__(16) float smem2[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int slot = (int)blk * (int)(blockDim.x >> 5) + wib;  // warps per block: blockDim
  if (slot >= A.np) return;  // whole warp
  const int i = A.order[slot];
  const int S = SC ? SC : A.box, P = box_pitch(S), cells = S * P;
  __syncwarp();  // the warp's shared memory is free (a particle before may have used it)
  float* base = smem2 + (size_t)wib * (wf ? wf : spread2_warp_floats(S));
  float2* box = reinterpret_cast<float2*>(base);
  float* tw = base + 2 * cells;                                   // [32][kTw]
  float4* tp = reinterpret_cast<float4*>(tw + 32 * kTw);          // [32]
  const int ox = fix_anchor(A.Xcf[(long long)i * 2 + 0]) - A.rcell - 2;
  const int oy = fix_anchor(A.Xcf[(long long)i * 2 + 1]) - A.rcell - 2;
  const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int q = lane; q < cells / 2; q += 32) reinterpret_cast<float4*>(box)[q] = z4;
  const int h = lane >> 4, sx = lane & 3, sy = (lane >> 2) & 3;
  for (int g0 = 0; g0 < A.nl; g0 += 32) {
    const int cnt = min(32, A.nl - g0), H = (cnt + 1) >> 1;
    // owner lane: the table row of point g0 + lane
    int lbx = 0, lby = 0;
    bool valid = false;
    if (lane < cnt) {
      const long long b = (long long)i * A.nl + g0 + lane;
      const long long Xx = A.Xb[b * 2], Xy = A.Xb[b * 2 + 1];
      const float fx = A.dFb[b * 2] * A.dV, fy = A.dFb[b * 2 + 1] * A.dV;
      float rx, ry;
      const int bx = support_first(A.delta_kind, Xx, rx), by = support_first(A.delta_kind, Xy, ry);
      lbx = bx - ox;
      lby = by - oy;
      valid = lbx >= 0 && lby >= 0 && lbx + 3 < S && lby + 3 < S;
      if (!valid) atomicOr(A.status, ST_CAPACITY);
      float wx[4], wy[4];
      delta_weights(A.delta_kind, rx, wx);
      delta_weights(A.delta_kind, ry, wy);
#pragma unroll
      for (int t = 0; t < 4; ++t) {  // no weight beyond a wall
        const int gx = bx + t, gy = by + t;
        if (!A.g.per[0] && (gx < 0 || gx >= A.g.nx)) wx[t] = 0.0f;
        if (!A.g.per[1] && (gy < 0 || gy >= A.g.ny)) wy[t] = 0.0f;
      }
      float* row = tw + lane * kTw;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        row[t] = wx[t];
        row[4 + t] = wy[t];
      }
      tp[lane] = make_float4(fx, fy, __int_as_float(valid ? lby * P + lbx : 0), 0.0f);
    }
    // the two supports of a pass could share a node: anchors at most 3 apart on both axes
    const int pbx = __shfl_sync(0xffffffffu, lbx, min(lane + H, 31));
    const int pby = __shfl_sync(0xffffffffu, lby, min(lane + H, 31));
    const bool clash = lane < H && lane + H < cnt && abs(lbx - pbx) <= 3 && abs(lby - pby) <= 3;
    const unsigned cmask = __ballot_sync(0xffffffffu, clash);
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    __syncwarp();
    for (int j = 0; j < H; ++j) {
      const int p = j + h * H;
      const bool act = p < cnt && ((vmask >> p) & 1u);
      float4 pd = z4;
      float w = 0.0f;
      if (act) {
        pd = tp[p];
        w = tw[p * kTw + sx] * tw[p * kTw + 4 + sy];
      }
      const int cell = __float_as_int(pd.z) + sy * P + sx;
      if ((cmask >> j) & 1u) {
        if (h == 0 && act) {
          float2 v = box[cell];
          v.x += w * pd.x;
          v.y += w * pd.y;
          box[cell] = v;
        }
        __syncwarp();
        if (h == 1 && act) {
          float2 v = box[cell];
          v.x += w * pd.x;
          v.y += w * pd.y;
          box[cell] = v;
        }
      } else if (act) {
        float2 v = box[cell];
        v.x += w * pd.x;
        v.y += w * pd.y;
        box[cell] = v;
      }
      __syncwarp();
    }
  }
  float2* fib2 = reinterpret_cast<float2*>(A.fib);
  for (int t = lane; t < S * S; t += 32) {
    const int r = t / S, c = t - r * S;
    const float2 v = box[r * P + c];
    if (v.x == 0.0f && v.y == 0.0f) continue;
    int gx = ox + c, gy = oy + r;
    if (gx < 0 || gx >= A.g.nx) gx = ((gx % A.g.nx) + A.g.nx) % A.g.nx;  // only periodic
    if (gy < 0 || gy >= A.g.ny) gy = ((gy % A.g.ny) + A.g.ny) % A.g.ny;  // axes reach here
    const long long n = (long long)gx + (long long)A.g.nx * gy;
    if (IBMLBM_CHK(n, A.g.N)) atomicAdd(fib2 + n, v);
  }
}

template <int SC, bool FUSED>
__global__ void __launch_bounds__(kIbmWarps * 32) ibm_spread2_kernel(IbmArgs A0, Fuse FU) {
  pdl_enter();
  IBMLBM_BIND(FUSED, IbmArgs, A, A0, FU, blk);
  if constexpr (FUSED) {  // members differ in box size: run the code compiled for this one
    switch (A.box) {
      case 14: spread2_body<14>(A, blk); return;
      case 16: spread2_body<16>(A, blk); return;
      case 18: spread2_body<18>(A, blk); return;
      case 20: spread2_body<20>(A, blk); return;
      case 22: spread2_body<22>(A, blk); return;
      default: spread2_body<0>(A, blk); return;
    }
  }
  spread2_body<SC>(A, blk);
}

// ------------------------------------------------------------------ 3D
// One block per sphere, two launches per MDF iteration m (Eq. 47, 10, then 48):
// the interpolation stages u^(m-1) of the sphere's node box in shared memory and
// interpolates every point from it; the spreading accumulates dF_b dV into the box and
// adds its non-zero cells to f_IB.  Box rows are box3_pitch(S) cells apart (4 modulo
// 8), so the 16 columns of a support fall on 16 banks, and box planes box3_plane(S)
// cells apart (8 modulo 16), so the 4 z levels of a support column fall on the 4 banks
// of one residue class modulo 8.  Each point's row of the table holds its 12 weights,
// its first box cell and u_b or dF_b dV.
constexpr int kMdf3Threads = 512;
constexpr int kMdf3Warps = kMdf3Threads / 32;
constexpr int kTab3 = 17;  // table floats per point (12 weights, first cell, u_b or dF_b dV,
                            // the interpolation's residue and rank); an odd stride keeps the
                            // rows a thread-per-point loop touches on distinct banks
constexpr int kRows3 = 2;  // box rows each warp stages per round

__host__ __device__ inline int box3_pitch(int S) {
  int p = S;
  while ((p & 7) != 4) ++p;
  return p;
}
__host__ __device__ inline int box3_plane(int S) {
  int p = box3_pitch(S) * S;
  while ((p & 15) != 8) ++p;
  return p;
}
// box [3][plane][S], table [nl][kTab3], the interpolation's point order [nl] and its
// residue counts (or the spreading's reduction scratch) [32]
size_t ibm_mdf3_smem(int nl, int box) {
  const size_t plane = (size_t)box3_plane(box);
  return sizeof(float) * (3 * plane * box + (size_t)(kTab3 + 1) * nl + 32);
}

// box origin of sphere i (two nodes before its support reach) and the fixed-point
// anchor and fraction of its centre
__device__ __forceinline__ void mdf3_origin(const IbmArgs& A, int i, int (&an)[3], float (&fr)[3],
                                            int (&org)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const long long v = A.Xcf[(long long)i * 3 + k];
    an[k] = fix_anchor(v);
    fr[k] = fix_frac(v);
    org[k] = an[k] - A.rcell - 2;
  }
}

// table row of every point of sphere i: its 12 weights and first box cell (zero
// weights, and CAPACITY, for a support outside the box).  BIN: also count the points
// by the residue of the first cell modulo 8 (cnt[8]) and keep (residue, rank) in row[16].
template <bool BIN>
__device__ __forceinline__ void mdf3_table(const IbmArgs& A, int i, const int (&org)[3], int S, int Py,
                                           int Pz, float* tab, int* cnt) {
  const int nn[3] = {A.g.nx, A.g.ny, A.g.nz};
  for (int k = threadIdx.x; k < A.nl; k += kMdf3Threads) {
    const long long b = (long long)i * A.nl + k;
    float* row = tab + (size_t)k * kTab3;
    int base = 0;
    bool valid = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long X = A.Xb[b * 3 + a];
      float f, w[4];
      const int s0 = support_first(A.delta_kind, X, f);
      const int l0 = s0 - org[a];
      if (l0 < 0 || l0 + 3 >= S) valid = false;
      base += l0 * (a == 0 ? 1 : a == 1 ? Py : Pz);
      delta_weights(A.delta_kind, f, w);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int gc = s0 + t;
        row[4 * a + t] = (!A.g.per[a] && (gc < 0 || gc >= nn[a])) ? 0.0f : w[t];
      }
    }
    if (!valid) {
      atomicOr(A.status, ST_CAPACITY);
      base = 0;
#pragma unroll
      for (int t = 0; t < 12; ++t) row[t] = 0.0f;
    }
    row[12] = __int_as_float(base);
    if (BIN) {
      const int r = base & 7;
      row[16] = __int_as_float(r | (atomicAdd(&cnt[r], 1) << 3));
    }
  }
}

// Whether sphere i's node box lies inside the domain on every axis (its staging list
// then applies, with plain offsets from the box origin).
__device__ __forceinline__ bool box3_inside(const IbmArgs& A, const int (&org)[3], int S) {
  return A.slen > 0 && org[0] >= 0 && org[1] >= 0 && org[2] >= 0 && org[0] + S <= A.g.nx &&
         org[1] + S <= A.g.ny && org[2] + S <= A.g.nz;
}

// Linear offset of box cell (lx, ly, lz) from the box origin (below 2^31: the host
// builds no list otherwise)
__device__ __forceinline__ int box3_goff(const Geo& g, int lx, int ly, int lz) {
  return lx + g.nx * (ly + g.ny * lz);
}

// Staging of u^(m-1) from the staging list (box inside the domain): thread t takes
// entries t, t + kMdf3Threads, ..., kListU at a time with all their loads in flight.
// An entry is staged when the cube of half-width shell_h around the node (its offset
// from the centre is a = l - cen) meets the shell between the points' radii: every
// support node of every point passes, and the rest of the box is never read.
constexpr int kListU = 4;

template <int MODE>
__device__ __forceinline__ void stage3_from_list(const IbmArgs& A, float* box, int cells, int Py, int Pz,
                                                 long long n0, const float (&cen)[3]) {
  const float4* us4 = reinterpret_cast<const float4*>(A.ustar);
  const float4* fib4 = reinterpret_cast<const float4*>(A.fib);
  const float h = A.shell_h;
  for (int j0 = threadIdx.x; j0 < A.slen; j0 += kMdf3Threads * kListU) {
    float4 v[kListU];
    int cell[kListU];
#pragma unroll
    for (int u = 0; u < kListU; ++u) {
      const int j = j0 + u * kMdf3Threads;
      cell[u] = -1;
      v[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (j >= A.slen) continue;
      const int e = A.slist[j];
      const int lx = e & 31, ly = (e >> 5) & 31, lz = (e >> 10) & 31;
      const float ax = fabsf((float)lx - cen[0]), ay = fabsf((float)ly - cen[1]), az = fabsf((float)lz - cen[2]);
      const float ex = fmaxf(ax - h, 0.0f), ey = fmaxf(ay - h, 0.0f), ez = fmaxf(az - h, 0.0f);
      const float gx = ax + h, gy = ay + h, gz = az + h;
      if (ex * ex + ey * ey + ez * ez > A.shell_hi2 || gx * gx + gy * gy + gz * gz < A.shell_lo2) continue;
      cell[u] = lx + Py * ly + Pz * lz;
      const long long n = n0 + box3_goff(A.g, lx, ly, lz);
      if (!IBMLBM_CHK(n, A.g.N)) continue;
      v[u] = us4[n];
      if (MODE == 1) {
        const float4 f = fib4[n];
        v[u].x += 0.5f * f.x;
        v[u].y += 0.5f * f.y;
        v[u].z += 0.5f * f.z;
      }
    }
#pragma unroll
    for (int u = 0; u < kListU; ++u)
      if (cell[u] >= 0) {
        box[cell[u]] = v[u].x;
        box[cells + cell[u]] = v[u].y;
        box[2 * cells + cell[u]] = v[u].z;
      }
  }
}

// Interpolation of MDF iteration m, one block per sphere (Eq. 47, 10):
//   1. stage u^(m-1) = u* + f_IB/2 (m = 1: u*) of the box nodes that can be support
//      nodes into shared memory (u* and f_IB are [N][4]);
//   2. interpolate every point, four lanes a point (one z level each, the 16 nodes of
//      the level in a loop); dF_b = 2 (U_b - u_b), F_b += dF_b.
// The spreading of the iteration is a separate launch, so every sphere reads f_IB
// with the increments of iterations 1 .. m-1 of all spheres and none of iteration m
// (the iteration of the FP64 oracle).
template <int SC, int MODE>
__global__ void __launch_bounds__(kMdf3Threads, 2) ibm_interp3_kernel(IbmArgs A, int m) {
  extern __shared__ __align__(16) float sm3[];
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = SC ? SC : A.box, Py = box3_pitch(S), Pz = box3_plane(S), cells = Pz * S;
  float* box = sm3;                          // [3][cells]
  float* tab = sm3 + 3 * cells;              // [nl][kTab3]
  int* perm = reinterpret_cast<int*>(tab + (size_t)kTab3 * A.nl);  // [nl] points by residue
  int* cnt = perm + A.nl;                    // [8] points per residue
  const float4* us4 = reinterpret_cast<const float4*>(A.ustar);
  const float4* fib4 = reinterpret_cast<const float4*>(A.fib);
  const int nn[3] = {A.g.nx, A.g.ny, A.g.nz};
  int an[3], org[3];
  float fr[3];
  mdf3_origin(A, i, an, fr, org);
  const float Rm2 = A.mark_radius * A.mark_radius;
  const bool inside = box3_inside(A, org, S);
  // this lane's column of every box row: grid x, and whether it is inside the domain
  // (S <= 22 here: a larger box does not fit in shared memory and takes the global path)
  int gx = org[0] + lane;
  bool xok = lane < S;
  if (gx < 0 || gx >= nn[0]) {
    if (A.g.per[0]) gx = ((gx % nn[0]) + nn[0]) % nn[0]; else xok = false;
  }
  const float dx = (float)(org[0] + lane - an[0]) - fr[0];

  // 1. stage the box: from the staging list where the box lies inside the domain, else
  //    the marked ball of the box, kRows3 rows per warp and round.  The 3-point delta's
  //    fourth (zero-weight) node is staged by neither: the box starts from zero then.
  if (tid < 8) cnt[tid] = 0;
  if (A.delta_kind == 3) {
    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int q = tid; q < 3 * cells / 4; q += kMdf3Threads) reinterpret_cast<float4*>(box)[q] = z4;
  }
  __syncthreads();
  if (inside) {
    const float cen[3] = {(float)(an[0] - org[0]) + fr[0], (float)(an[1] - org[1]) + fr[1],
                          (float)(an[2] - org[2]) + fr[2]};
    const long long n0 = (long long)org[0] + (long long)nn[0] * ((long long)org[1] + (long long)nn[1] * org[2]);
    stage3_from_list<MODE>(A, box, cells, Py, Pz, n0, cen);
  }
  const int rows = inside ? 0 : S * S;  // otherwise by box rows
  for (int r0 = warp; r0 < rows; r0 += kMdf3Warps * kRows3) {
    float4 v[kRows3];
    int cell[kRows3];
#pragma unroll
    for (int u = 0; u < kRows3; ++u) {
      const int r = r0 + u * kMdf3Warps;
      cell[u] = -1;
      v[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (r >= rows || lane >= S) continue;
      const int ly = r % S, lz = r / S;
      const float dy = (float)(org[1] + ly - an[1]) - fr[1], dz = (float)(org[2] + lz - an[2]) - fr[2];
      if (dx * dx + dy * dy + dz * dz > Rm2) continue;  // outside the marked ball
      cell[u] = lane + Py * ly + Pz * lz;
      int gy = org[1] + ly, gz = org[2] + lz;
      bool ok = xok;
      if (gy < 0 || gy >= nn[1]) {
        if (A.g.per[1]) gy = ((gy % nn[1]) + nn[1]) % nn[1]; else ok = false;
      }
      if (gz < 0 || gz >= nn[2]) {
        if (A.g.per[2]) gz = ((gz % nn[2]) + nn[2]) % nn[2]; else ok = false;
      }
      if (!ok) continue;  // beyond a wall: zero
      const long long n = (long long)gx + (long long)nn[0] * ((long long)gy + (long long)nn[1] * gz);
      if (!IBMLBM_CHK(n, A.g.N)) continue;
      v[u] = us4[n];
      if (MODE == 1) {
        const float4 f = fib4[n];
        v[u].x += 0.5f * f.x;
        v[u].y += 0.5f * f.y;
        v[u].z += 0.5f * f.z;
      }
    }
#pragma unroll
    for (int u = 0; u < kRows3; ++u)
      if (cell[u] >= 0) {
        box[cell[u]] = v[u].x;
        box[cells + cell[u]] = v[u].y;
        box[2 * cells + cell[u]] = v[u].z;
      }
  }
  mdf3_table<true>(A, i, org, S, Py, Pz, tab, cnt);
  __syncthreads();

  // 2. interpolation, four lanes a point (lane sz: the 16 support nodes of z level sz)
  //    and eight points a warp.  Lanes sz of a point read the banks of one residue
  //    class modulo 8, the residue of its first cell, so the eight points of a warp come
  //    one from each residue: round j takes the j-th point of every residue's list (the
  //    lists in point order; a residue with fewer points leaves its lanes idle), and
  //    every shared-memory load of the round falls on 32 distinct banks.
  int first_r = 0, rounds = 0;  // this lane's residue list: start, and the most points of any
  const int slot = lane >> 2, sz = lane & 3;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int c = cnt[r];
    first_r += r < slot ? c : 0;
    rounds = max(rounds, c);
  }
  {
    int start[8], acc = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      start[r] = acc;
      acc += cnt[r];
    }
    for (int k = tid; k < A.nl; k += kMdf3Threads) {
      const int v = __float_as_int(tab[(size_t)k * kTab3 + 16]);
      int at = v >> 3;
#pragma unroll
      for (int r = 0; r < 8; ++r) at += (v & 7) == r ? start[r] : 0;
      perm[at] = k;
    }
  }
  const int n_r = cnt[slot];
  __syncthreads();
  for (int j = warp; j < rounds; j += kMdf3Warps) {
    const bool act = j < n_r;
    const int p = act ? perm[first_r + j] : 0;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    if (act) {
      const float* row = tab + (size_t)p * kTab3;
      const float wz = row[8 + sz];
      float wx[4], wy[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        wx[t] = row[t];
        wy[t] = row[4 + t];
      }
      const int c0 = __float_as_int(row[12]) + Pz * sz;
#pragma unroll
      for (int sy = 0; sy < 4; ++sy) {
        const float wyz = wy[sy] * wz;
        const int cr = c0 + Py * sy;
#pragma unroll
        for (int sx = 0; sx < 4; ++sx) {
          const float w = wx[sx] * wyz;
          a0 += w * box[cr + sx];
          a1 += w * box[cells + cr + sx];
          a2 += w * box[2 * cells + cr + sx];
        }
      }
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (act && sz == 0) {  // u_b into the table
      float* row = tab + (size_t)p * kTab3;  // (row[16] is not read again)
      row[13] = a0;
      row[14] = a1;
      row[15] = a2;
    }
  }
  __syncthreads();
  // dF_b = 2 (U_b - u_b) and F_b, one thread per point (coalesced); m < 0: the
  // residual U_b - u_b after the last iteration
  for (int k = tid; k < A.nl; k += kMdf3Threads) {
    const long long b = (long long)i * A.nl + k;
    const float* row = tab + (size_t)k * kTab3;
    float U[3], F[3] = {0.0f, 0.0f, 0.0f};  // all loads ahead of the stores
#pragma unroll
    for (int c = 0; c < 3; ++c) U[c] = A.Ub[b * 3 + c];
    if (m > 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] = A.Fb[b * 3 + c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float u = row[13 + c];
      if (m < 0) {
        A.res[b * 3 + c] = U[c] - u;
        continue;
      }
      const float d = 2.0f * (U[c] - u);
      A.dFb[b * 3 + c] = d;
      A.Fb[b * 3 + c] = (m == 1) ? d : F[c] + d;
      if (m == 1) A.ubs[b * 3 + c] = u;
    }
  }
}

// Spreading of an MDF iteration, one block per sphere (Eq. 48, 11):
//   1. the table of weights (as in the interpolation) and dF_b dV of every point;
//   2. spread into the sphere's box, accumulated as 32-bit fixed point with integer
//      shared-memory atomics.  The scale of the sphere is 2^30 over (max |dF_b dV|
//      times N_L times w_max), a bound on any node's sum (w_max, the largest product
//      of three one-dimensional weights: phi(0)^3 = 1/8 for the 4-point delta, 8/27
//      for the 3-point one), so no sum overflows; each addend is rounded to a step of
//      1 / scale;
//   3. add the non-zero box cells to f_IB with one vector atomic per cell.
template <int SC>
__global__ void __launch_bounds__(kMdf3Threads) ibm_spread3_kernel(IbmArgs A) {
  extern __shared__ __align__(16) float sm3[];
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = SC ? SC : A.box, Py = box3_pitch(S), Pz = box3_plane(S), cells = Pz * S;
  int* boxi = reinterpret_cast<int*>(sm3);   // [3][cells]
  float* tab = sm3 + 3 * cells;              // [nl][kTab3]
  float* red = tab + (size_t)kTab3 * A.nl;   // [32] reduction scratch
  float4* fib4 = reinterpret_cast<float4*>(A.fib);
  const int nn[3] = {A.g.nx, A.g.ny, A.g.nz};
  int an[3], org[3];
  float fr[3];
  mdf3_origin(A, i, an, fr, org);
  {
    int4* b4 = reinterpret_cast<int4*>(boxi);
    const int4 z = make_int4(0, 0, 0, 0);
    for (int q = tid; q < 3 * cells / 4; q += kMdf3Threads) b4[q] = z;
  }
  mdf3_table<false>(A, i, org, S, Py, Pz, tab, nullptr);
  float mx = 0.0f;
  for (int k = tid; k < A.nl; k += kMdf3Threads) {
    const long long b = (long long)i * A.nl + k;
    float* row = tab + (size_t)k * kTab3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float d = A.dFb[b * 3 + c] * A.dV;
      row[13 + c] = d;
      mx = fmaxf(mx, fabsf(d));
    }
  }
  // largest |dF dV| of the sphere
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  float gmax = 0.0f;
#pragma unroll
  for (int w = 0; w < kMdf3Warps; ++w) gmax = fmaxf(gmax, red[w]);
  if (!(gmax > 1e-30f) || !isfinite(gmax)) {  // below 1e-30 the spread is negligible
    if (!isfinite(gmax) && tid == 0) atomicOr(A.status, ST_NONFINITE);
    return;  // nothing to spread (the same decision in every thread of the block)
  }
  const float wmax = A.delta_kind == 3 ? 8.0f / 27.0f : 0.125f;
  const float scale = 1073741824.0f / (gmax * wmax * (float)A.nl);  // 2^30 / bound
  const float inv = 1.0f / scale;

  // 2. spreading, one point per warp: lane (sx, sy, zh) adds to the support nodes of
  //    z levels 2 zh and 2 zh + 1 (two box planes apart, 2 Pz = 16 modulo 32 for the
  //    box sides used, so the 32 lanes of an atomic touch 32 banks)
  const int zh = lane >> 4, sx = lane & 3, sy = (lane >> 2) & 3;
  const int colo = sx + Py * sy + 2 * Pz * zh;
  for (int p = warp; p < A.nl; p += kMdf3Warps) {
    const float* row = tab + (size_t)p * kTab3;
    const float wxy = row[sx] * row[4 + sy] * scale;
    const int c0 = __float_as_int(row[12]) + colo;
    const float f0 = row[13], f1 = row[14], f2 = row[15];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float w = wxy * row[8 + 2 * zh + k];
      if (w == 0.0f) continue;
      const int c = c0 + Pz * k;
      atomicAdd(&boxi[c], __float2int_rn(w * f0));
      atomicAdd(&boxi[cells + c], __float2int_rn(w * f1));
      atomicAdd(&boxi[2 * cells + c], __float2int_rn(w * f2));
    }
  }
  __syncthreads();

  // 3. flush the non-zero cells to f_IB: the staging list's cells where the box lies
  //    inside the domain (every support node is one), else one box row per warp and round
  if (box3_inside(A, org, S)) {
    const long long n0 = (long long)org[0] + (long long)nn[0] * ((long long)org[1] + (long long)nn[1] * org[2]);
    for (int j = tid; j < A.slen; j += kMdf3Threads) {
      const int e = A.slist[j];
      const int lx = e & 31, ly = (e >> 5) & 31, lz = (e >> 10) & 31;
      const int c = lx + Py * ly + Pz * lz;
      const int v0 = boxi[c], v1 = boxi[cells + c], v2 = boxi[2 * cells + c];
      if ((v0 | v1 | v2) == 0) continue;
      const long long n = n0 + box3_goff(A.g, lx, ly, lz);
      if (IBMLBM_CHK(n, A.g.N))
        atomicAdd(fib4 + n, make_float4((float)v0 * inv, (float)v1 * inv, (float)v2 * inv, 0.0f));
    }
    return;
  }
  const int rows = S * S;
  int gx = org[0] + lane;
  if (gx < 0 || gx >= nn[0]) gx = ((gx % nn[0]) + nn[0]) % nn[0];  // only periodic x reaches the add
  for (int r = warp; r < rows; r += kMdf3Warps) {
    if (lane >= S) continue;
    const int ly = r % S, lz = r / S;
    const int c = lane + Py * ly + Pz * lz;
    const int v0 = boxi[c], v1 = boxi[cells + c], v2 = boxi[2 * cells + c];
    if ((v0 | v1 | v2) == 0) continue;
    // non-zero cells lie inside the domain or across a periodic face
    int gy = org[1] + ly, gz = org[2] + lz;
    if (gy < 0 || gy >= nn[1]) gy = ((gy % nn[1]) + nn[1]) % nn[1];
    if (gz < 0 || gz >= nn[2]) gz = ((gz % nn[2]) + nn[2]) % nn[2];
    const long long n = (long long)gx + (long long)nn[0] * ((long long)gy + (long long)nn[1] * gz);
    if (IBMLBM_CHK(n, A.g.N)) atomicAdd(fib4 + n, make_float4((float)v0 * inv, (float)v1 * inv, (float)v2 * inv, 0.0f));
  }
}

// 3D spheres whose box does not fit in shared memory: the same interpolation and
// spreading, a half-warp per point (lane (sx, sy) of the 4 x 4 support columns, the
// 4 z levels in a loop), reading u* + f_IB/2 through the caches and adding each
// support node's share of dF_b dV to f_IB with a vector atomic.  Two launches per
// iteration as for the staged kernels, so the iterations stay Jacobi.
struct Support3 {
  int s0[3];     // first support node per axis
  float w[3];    // this lane's weights along x (sx) and y (sy); w[2] unused
  float wz[4];   // the 4 z weights
};

__device__ __forceinline__ Support3 support3(const IbmArgs& A, long long b, int sx, int sy) {
  Support3 S;
  const int nn[3] = {A.g.nx, A.g.ny, A.g.nz};
  const int lane_t[2] = {sx, sy};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float f;
    S.s0[a] = support_first(A.delta_kind, A.Xb[b * 3 + a], f);
    if (a < 2) {
      const int gc = S.s0[a] + lane_t[a];
      S.w[a] = (!A.g.per[a] && (gc < 0 || gc >= nn[a])) ? 0.0f : delta_w(A.delta_kind, (float)(lane_t[a] - 1) - f);
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int gc = S.s0[2] + t;
        S.wz[t] = (!A.g.per[2] && (gc < 0 || gc >= nn[2])) ? 0.0f : delta_w(A.delta_kind, (float)(t - 1) - f);
      }
    }
  }
  S.w[2] = 0.0f;
  return S;
}

// wrapped node coordinate along an axis, or -1 beyond a wall
__device__ __forceinline__ int wrap_axis(int c, int n, int per) {
  if (c >= 0 && c < n) return c;
  return per ? ((c % n) + n) % n : -1;
}

template <int MODE>
__global__ void __launch_bounds__(256) ibm_interp3g_kernel(IbmArgs A, int m) {
  const int lane = threadIdx.x & 31, sx = lane & 3, sy = (lane >> 2) & 3;
  const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;  // point
  const bool act = b < A.npts;
  float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
  if (act) {
    const Support3 S = support3(A, b, sx, sy);
    const int gx = wrap_axis(S.s0[0] + sx, A.g.nx, A.g.per[0]);
    const int gy = wrap_axis(S.s0[1] + sy, A.g.ny, A.g.per[1]);
    const float wxy = S.w[0] * S.w[1];
    if (gx >= 0 && gy >= 0 && wxy != 0.0f) {
      const float4* us4 = reinterpret_cast<const float4*>(A.ustar);
      const float4* fib4 = reinterpret_cast<const float4*>(A.fib);
#pragma unroll
      for (int sz = 0; sz < 4; ++sz) {
        const int gz = wrap_axis(S.s0[2] + sz, A.g.nz, A.g.per[2]);
        const float w = wxy * S.wz[sz];
        if (gz < 0 || w == 0.0f) continue;
        const long long n = (long long)gx + (long long)A.g.nx * ((long long)gy + (long long)A.g.ny * gz);
        if (!IBMLBM_CHK(n, A.g.N)) continue;
        float4 v = us4[n];
        if (MODE == 1) {
          const float4 f = fib4[n];
          v.x += 0.5f * f.x;
          v.y += 0.5f * f.y;
          v.z += 0.5f * f.z;
        }
        a0 += w * v.x;
        a1 += w * v.y;
        a2 += w * v.z;
      }
    }
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (act && (lane & 15) == 0) {  // dF_b = 2 (U_b - u_b), F_b; m < 0: the residual
    const float u[3] = {a0, a1, a2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (m < 0) {
        A.res[b * 3 + c] = A.Ub[b * 3 + c] - u[c];
        continue;
      }
      const float d = 2.0f * (A.Ub[b * 3 + c] - u[c]);
      A.dFb[b * 3 + c] = d;
      A.Fb[b * 3 + c] = (m == 1) ? d : A.Fb[b * 3 + c] + d;
      if (m == 1) A.ubs[b * 3 + c] = u[c];
    }
  }
}

__global__ void __launch_bounds__(256) ibm_spread3g_kernel(IbmArgs A) {
  const int lane = threadIdx.x & 31, sx = lane & 3, sy = (lane >> 2) & 3;
  const long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;  // point
  if (b >= A.npts) return;
  const Support3 S = support3(A, b, sx, sy);
  const int gx = wrap_axis(S.s0[0] + sx, A.g.nx, A.g.per[0]);
  const int gy = wrap_axis(S.s0[1] + sy, A.g.ny, A.g.per[1]);
  const float wxy = S.w[0] * S.w[1];
  if (gx < 0 || gy < 0 || wxy == 0.0f) return;
  const float f0 = A.dFb[b * 3] * A.dV, f1 = A.dFb[b * 3 + 1] * A.dV, f2 = A.dFb[b * 3 + 2] * A.dV;
  float4* fib4 = reinterpret_cast<float4*>(A.fib);
#pragma unroll
  for (int sz = 0; sz < 4; ++sz) {
    const int gz = wrap_axis(S.s0[2] + sz, A.g.nz, A.g.per[2]);
    const float w = wxy * S.wz[sz];
    if (gz < 0 || w == 0.0f) continue;
    const long long n = (long long)gx + (long long)A.g.nx * ((long long)gy + (long long)A.g.ny * gz);
    if (IBMLBM_CHK(n, A.g.N)) atomicAdd(fib4 + n, make_float4(w * f0, w * f1, w * f2, 0.0f));
  }
}

// shared memory of the staged 3D kernels; above this a sphere takes the global path
constexpr size_t kMdf3SmemMax = 227 * 1024;

// 3D interpolation of MDF iteration m >= 1 (m < 0: the residual pass after the last
// iteration), staged per sphere or, for spheres whose box exceeds shared memory, from
// global memory
cudaError_t launch_ibm_interp3(const IbmArgs& A, int m, cudaStream_t s) {
  if (A.np == 0 || m == 0) return cudaSuccess;
  const size_t sm = ibm_mdf3_smem(A.nl, A.box);
  if (sm > kMdf3SmemMax) {
    const unsigned grid = (unsigned)((A.npts * 16 + 255) / 256);
    if (m == 1) ibm_interp3g_kernel<0><<<grid, 256, 0, s>>>(A, m);
    else ibm_interp3g_kernel<1><<<grid, 256, 0, s>>>(A, m);
    return cudaGetLastError();
  }
#define IBMLBM_I3(SC)                                                          \
  do {                                                                          \
    if (m == 1) ibm_interp3_kernel<SC, 0><<<A.np, kMdf3Threads, sm, s>>>(A, m); \
    else ibm_interp3_kernel<SC, 1><<<A.np, kMdf3Threads, sm, s>>>(A, m);        \
  } while (0)
  if (A.box == 18) IBMLBM_I3(18);
  else if (A.box == 14) IBMLBM_I3(14);
  else IBMLBM_I3(0);
#undef IBMLBM_I3
  return cudaGetLastError();
}

// 3D spreading of an MDF iteration (after its interpolation launch)
cudaError_t launch_ibm_spread3(const IbmArgs& A, cudaStream_t s) {
  if (A.np == 0) return cudaSuccess;
  const size_t sm = ibm_mdf3_smem(A.nl, A.box);
  if (sm > kMdf3SmemMax)
    ibm_spread3g_kernel<<<(unsigned)((A.npts * 16 + 255) / 256), 256, 0, s>>>(A);
  else if (A.box == 18)
    ibm_spread3_kernel<18><<<A.np, kMdf3Threads, sm, s>>>(A);
  else if (A.box == 14)
    ibm_spread3_kernel<14><<<A.np, kMdf3Threads, sm, s>>>(A);
  else
    ibm_spread3_kernel<0><<<A.np, kMdf3Threads, sm, s>>>(A);
  return cudaGetLastError();
}

// F_h, T_h of particle i from its points, and the write of the warp's sums (lane 0)
// LP lanes per particle (32: a warp; 16: a half-warp, lane < 16 within the half);
// valid = false: the lane takes part in the reductions only
template <int D, int LP = 32>
__device__ __forceinline__ void forces_finish(const IbmArgs& A, int i, int lane, FF (&P)[3], FF (&L)[3],
                                              bool valid = true) {
  FF sF[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, sT[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int k = lane; valid && k < A.nl; k += LP) {
    const long long b = (long long)i * A.nl + k;
    float r[3] = {0.0f, 0.0f, 0.0f}, F[3] = {0.0f, 0.0f, 0.0f};
    for (int c = 0; c < D; ++c) {
      r[c] = A.ref_f[k * D + c];
      F[c] = A.Fb[b * D + c];
      ff_add(sF[c], F[c]);
    }
    if (D == 3) {
      ff_add(sT[0], r[1] * F[2] - r[2] * F[1]);
      ff_add(sT[1], r[2] * F[0] - r[0] * F[2]);
    }
    ff_add(sT[2], r[0] * F[1] - r[1] * F[0]);
  }
  // only the components that exist in this dimension (2D: x, y and the z rotation)
  for (int c = 0; c < D; ++c) {
    P[c] = LP == 32 ? ff_warp_sum(P[c]) : ff_half_sum(P[c]);
    sF[c] = LP == 32 ? ff_warp_sum(sF[c]) : ff_half_sum(sF[c]);
  }
  for (int c = (D == 2 ? 2 : 0); c < 3; ++c) {
    L[c] = LP == 32 ? ff_warp_sum(L[c]) : ff_half_sum(L[c]);
    sT[c] = LP == 32 ? ff_warp_sum(sT[c]) : ff_half_sum(sT[c]);
  }
  if (valid && lane == 0) {
    const double dV = (double)A.dV;
    for (int c = 0; c < D; ++c) {
      A.Pint[(long long)i * D + c] = ff_value(P[c]);
      A.FhN[(long long)i * D + c] = -dV * ff_value(sF[c]);
    }
    for (int c = 0; c < 3; ++c) {
      const bool used = !(D == 2 && c < 2);
      A.Lint[(long long)i * 3 + c] = used ? ff_value(L[c]) : 0.0;
      A.ThN[(long long)i * 3 + c] = used ? -dV * ff_value(sT[c]) : 0.0;
    }
  }
}


// Per particle (one warp), after the last MDF iteration:
//   F_h = -dV sum_b F_b, T_h = -dV sum_b r_b x F_b            (Eq. 14-15, via BTDF)
//   momentum and angular momentum about X_c of the fluid at the nodes strictly inside,
//   with the corrected velocity u* + f_IB/2 (the F_f, T_f closure of Eq. 14-15).
// Sums are compensated single precision.  The inside test |x - X_c|^2 < R^2 runs in
// single precision and falls back to the double-precision test (without fused
// multiply-add) in a thin band around R^2, so the set of interior nodes is the one
// the double-precision test gives.
template <int D>
__global__ void __launch_bounds__(256) ibm_forces_kernel(IbmArgs A) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= A.np) return;
  int an[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
  float fr[3] = {0.0f, 0.0f, 0.0f};
  const int n[3] = {A.g.nx, A.g.ny, A.g.nz};
  for (int k = 0; k < D; ++k) {
    const long long v = A.Xcf[(long long)i * D + k];
    an[k] = fix_anchor(v);
    fr[k] = fix_frac(v);
    lo[k] = an[k] - A.rcell;
    ext[k] = 2 * A.rcell + 2;
  }
  const float R2f = A.radius_f * A.radius_f;
  const float band = 1e-4f * R2f + 1e-5f;
  FF P[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, L[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const int total = ext[0] * ext[1] * ext[2];
  for (int t = lane; t < total; t += 32) {
    int gc[3] = {lo[0] + t % ext[0], lo[1] + (t / ext[0]) % ext[1], lo[2] + t / (ext[0] * ext[1])};
    float r[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < D; ++k) r[k] = (float)(gc[k] - an[k]) - fr[k];
    const float d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    bool inside = d2 < R2f;
    if (fabsf(d2 - R2f) < band) {
      double rd[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < D; ++k) rd[k] = (double)gc[k] - A.Xc[(long long)i * D + k];
      const double d2d = __dadd_rn(__dadd_rn(__dmul_rn(rd[0], rd[0]), __dmul_rn(rd[1], rd[1])),
                                   __dmul_rn(rd[2], rd[2]));
      inside = d2d < __dmul_rn(A.radius, A.radius);
    }
    if (!inside) continue;
    bool ok = true;
    for (int k = 0; k < D; ++k) {
      if (gc[k] < 0 || gc[k] >= n[k]) {
        if (A.g.per[k])
          gc[k] = ((gc[k] % n[k]) + n[k]) % n[k];
        else
          ok = false;
      }
    }
    if (!ok) continue;
    const long long nn = (long long)gc[0] + (long long)A.g.nx * ((long long)gc[1] + (long long)A.g.ny * gc[2]);
    if (!IBMLBM_CHK(nn, A.g.N)) continue;
    const float4 us = reinterpret_cast<const float4*>(A.ustar)[nn];  // 3D: [N][4]
    const float4 fv = reinterpret_cast<const float4*>(A.fib)[nn];
    const float u[3] = {us.x + 0.5f * fv.x, us.y + 0.5f * fv.y, us.z + 0.5f * fv.z};
    for (int c = 0; c < D; ++c) ff_add(P[c], u[c]);
    if (D == 3) {
      ff_add(L[0], r[1] * u[2] - r[2] * u[1]);
      ff_add(L[1], r[2] * u[0] - r[0] * u[2]);
    }
    ff_add(L[2], r[0] * u[1] - r[1] * u[0]);
  }
  forces_finish<D>(A, i, lane, P, L);
}

// 2D form of the same sums, with u* from the particle's box buffer, LP lanes per
// particle (a half-warp in a single run; a warp in the fused batch).  Each lane takes
// its candidate nodes NB at a time, so their loads are in flight together.  The common
// box sizes (16, 22) take 5 at a time within 48 registers a thread, so that 10^4
// particles fit one wave of the GPU; the general box (large particles, few of them)
// takes 9.
constexpr int kForceBatch = 6;

template <int SC, int LP = 32>
__device__ __forceinline__ void forces2_body(const IbmArgs& A, unsigned blk) {
  constexpr int NB = LP == 16 ? (SC ? 5 : 9) : kForceBatch;
  const unsigned gt = blk * blockDim.x + threadIdx.x;
  if ((int)((gt & ~31u) / LP) >= A.np) return;  // the warp's first particle: whole warp
  const int slot = (int)(gt / LP);
  const int lane = (int)(gt & (LP - 1));
  const bool valid = slot < A.np;  // (the second half-warp of the last warp may have none)
  const int S = SC ? SC : A.box, W = box_pitch(S), cells = S * W, ext = S - 4;  // ext = 2 rcell + 2
  const int i = valid ? A.order[slot] : 0, ic = i;
  const long long vx = A.Xcf[(long long)ic * 2], vy = A.Xcf[(long long)ic * 2 + 1];
  const int anx = fix_anchor(vx), any = fix_anchor(vy);
  const float frx = fix_frac(vx), fry = fix_frac(vy);
  const int lox = anx - A.rcell, loy = any - A.rcell;
  const float R2f = A.radius_f * A.radius_f;
  const float band = 1e-4f * R2f + 1e-5f;
  const float2* ub = reinterpret_cast<const float2*>(A.ubox) + (size_t)ic * cells;
  const float2* fib2 = reinterpret_cast<const float2*>(A.fib);
  FF P[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, L[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int t0 = 0; valid && t0 < ext * ext; t0 += LP * NB) {
    float rx[NB], ry[NB], u0[NB], u1[NB];
    bool in[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = t0 + lane + LP * q;
      in[q] = false;
      rx[q] = ry[q] = u0[q] = u1[q] = 0.0f;
      if (t >= ext * ext) continue;
      const int cx = t % ext, cy = t / ext;
      int gx = lox + cx, gy = loy + cy;
      rx[q] = (float)(gx - anx) - frx;
      ry[q] = (float)(gy - any) - fry;
      const float d2 = rx[q] * rx[q] + ry[q] * ry[q];
      bool inside = d2 < R2f;
      if (fabsf(d2 - R2f) < band) {
        const double dx = (double)gx - A.Xc[(long long)i * 2], dy = (double)gy - A.Xc[(long long)i * 2 + 1];
        inside = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < __dmul_rn(A.radius, A.radius);
      }
      if (!inside) continue;
      if (gx < 0 || gx >= A.g.nx) {
        if (!A.g.per[0]) continue;
        gx = ((gx % A.g.nx) + A.g.nx) % A.g.nx;
      }
      if (gy < 0 || gy >= A.g.ny) {
        if (!A.g.per[1]) continue;
        gy = ((gy % A.g.ny) + A.g.ny) % A.g.ny;
      }
      const long long nn = (long long)gx + (long long)A.g.nx * gy;
      const int o = (cy + 2) * W + (cx + 2);  // the box starts two nodes before lox, loy
      if (!IBMLBM_CHK(nn, A.g.N)) continue;
      const float2 us = ub[o], fv = fib2[nn];
      u0[q] = us.x + 0.5f * fv.x;
      u1[q] = us.y + 0.5f * fv.y;
      in[q] = true;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (!in[q]) continue;
      ff_add(P[0], u0[q]);
      ff_add(P[1], u1[q]);
      ff_add(L[2], rx[q] * u1[q] - ry[q] * u0[q]);
    }
  }
  forces_finish<2, LP>(A, i, lane, P, L, valid);
}

// Blocks per SM the registers must allow: a single run's box sizes 16 and 22 five (48
// registers), its general box three; the fused batch kernel, which holds every box
// size's body, four (64 registers, a little spilled: 0.800 -> 0.794 ms per 256-cavity
// step against three)
template <int SC, bool FUSED>
__global__ void __launch_bounds__(256, FUSED ? 4 : (SC == 0 ? 3 : 5)) ibm_forces2_kernel(IbmArgs A0, Fuse FU) {
  pdl_enter();
  IBMLBM_BIND(FUSED, IbmArgs, A, A0, FU, blk);
  if constexpr (FUSED) {  // members differ in box size: run the code compiled for this one
    switch (A.box) {
      case 14: forces2_body<14, 16>(A, blk); return;
      case 16: forces2_body<16, 16>(A, blk); return;
      case 18: forces2_body<18, 16>(A, blk); return;
      case 20: forces2_body<20, 16>(A, blk); return;
      case 22: forces2_body<22, 16>(A, blk); return;
      default: forces2_body<0, 16>(A, blk); return;
    }
  }
  forces2_body<SC, 16>(A, blk);  // a single run: half-warp per particle
}

// One warp per particle: regenerate its Lagrangian points for the next step,
//   X_b = X_c + r_b (32.32 fixed point), U_b = U_c + Omega x r_b (single precision),
// and (3D) mark the nodes within mark_radius of the centre in the next step's node mask.
// init != 0 first refreshes the fixed-point centre and the single-precision
// velocities from the double-precision state (initial state, new particle state).
template <int D>
__device__ __forceinline__ void regen_body(const RegenArgs& A, int init, unsigned blk) {
  const int i = (int)((blk * 256u + threadIdx.x) >> 5);  // 256-thread blocks
  const int lane = threadIdx.x & 31;
  if (i >= A.np) return;
  const long long pi = i;
  if (init && lane == 0) {
    for (int c = 0; c < D; ++c) {
      const double x = A.X[pi * D + c];
      A.Xcf[pi * D + c] = isfinite(x) ? __double2ll_rn(x * kFixScale) : 0;
      A.Uf[pi * D + c] = (float)A.U[pi * D + c];
    }
    for (int c = 0; c < 3; ++c) A.Omf[pi * 3 + c] = (D == 2 && c < 2) ? 0.0f : (float)A.Om[pi * 3 + c];
  }
  __syncwarp();
  long long xf[3] = {0, 0, 0};
  float uf[3] = {0.0f, 0.0f, 0.0f}, of[3] = {0.0f, 0.0f, 0.0f};
  for (int c = 0; c < D; ++c) {
    xf[c] = A.Xcf[pi * D + c];
    uf[c] = A.Uf[pi * D + c];
  }
  for (int c = 0; c < 3; ++c) of[c] = A.Omf[pi * 3 + c];
  for (int k = lane; k < A.nl; k += 32) {
    const long long b = pi * A.nl + k;
    float r[3] = {0.0f, 0.0f, 0.0f};
    for (int c = 0; c < D; ++c) r[c] = A.ref_f[k * D + c];
    const float w[3] = {of[1] * r[2] - of[2] * r[1], of[2] * r[0] - of[0] * r[2],
                        of[0] * r[1] - of[1] * r[0]};
    for (int c = 0; c < D; ++c) {
      A.Xb_out[b * D + c] = xf[c] + A.ref_fix[k * D + c];
      A.Ub_out[b * D + c] = uf[c] + w[c];
    }
  }
  // 3D: mark the nodes of the ball |x - X_c| <= mark_radius, row by row (single
  // precision relative to the centre's anchor node; the radius carries a safety
  // margin): the nodes where u* is needed and f_IB can be non-zero.  2D keeps u* per
  // particle box and reads f_IB everywhere, so it marks nothing.
  if (D == 2) return;
  int an[3] = {0, 0, 0};
  float fr[3] = {0.0f, 0.0f, 0.0f};
  for (int c = 0; c < D; ++c) {
    an[c] = fix_anchor(xf[c]);
    fr[c] = fix_frac(xf[c]);
  }
  const float Rm = A.mark_radius, Rm2 = Rm * Rm;
  const int rr = (int)ceilf(Rm) + 1;
  const int ey = 2 * rr + 1, ez = (D == 3) ? 2 * rr + 1 : 1;
  for (int t = lane; t < ey * ez; t += 32) {
    const int oy = t % ey - rr, oz = (D == 3) ? t / ey - rr : 0;
    const float dy = (float)oy - fr[1], dz = (D == 3) ? (float)oz - fr[2] : 0.0f;
    const float rem = Rm2 - dy * dy - dz * dz;
    if (rem < 0.0f) continue;
    int gy = an[1] + oy, gz = (D == 3) ? an[2] + oz : 0;
    if (gy < 0 || gy >= A.g.ny) {
      if (!A.g.per[1]) continue;
      gy = ((gy % A.g.ny) + A.g.ny) % A.g.ny;
    }
    if (D == 3 && (gz < 0 || gz >= A.g.nz)) {
      if (!A.g.per[2]) continue;
      gz = ((gz % A.g.nz) + A.g.nz) % A.g.nz;
    }
    const float h = sqrtf(rem);
    int x0 = an[0] + (int)ceilf(fr[0] - h), x1 = an[0] + (int)floorf(fr[0] + h);
    const long long ro = ((long long)gy + (long long)A.g.ny * gz) * A.g.wpr;
    if (!IBMLBM_CHK(ro + A.g.wpr - 1, (long long)A.g.rows * A.g.wpr)) continue;
    uint32_t* row = A.mask + ro;
    if (A.g.per[0] && (x0 < 0 || x1 >= A.g.nx)) {
      for (int x = x0; x <= x1; ++x) {
        const int wx = ((x % A.g.nx) + A.g.nx) % A.g.nx;
        atomicOr(row + (wx >> 5), 1u << (wx & 31));
      }
      continue;
    }
    if (x0 < 0) x0 = 0;
    if (x1 > A.g.nx - 1) x1 = A.g.nx - 1;
    for (int x = x0; x <= x1;) {
      const int wd = x >> 5;
      const int end = min(x1, wd * 32 + 31);
      const int lo = x & 31, hi = end & 31;
      const uint32_t bits = (hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u)) & ~((1u << lo) - 1u);
      atomicOr(row + wd, bits);
      x = end + 1;
    }
  }
}

template <int D, bool FUSED>
__global__ void __launch_bounds__(256) regen_kernel(RegenArgs A0, int init, Fuse FU) {
  IBMLBM_BIND(FUSED, RegenArgs, A, A0, FU, blk);
  regen_body<D>(A, init, blk);
}

// ---------------------------------------------- persistent kernel of a batched step
// The IBM phases of a batched step (2D) in one persistent kernel (cooperative launch,
// kIbmWarps warps a block, shared memory for the largest particle box of the batch):
// regenerate this step's Lagrangian points from the updated particle state, then for
// each MDF iteration the interpolation and the spreading, then the sums of the
// hydrodynamic force and interior momentum, with a bounded grid barrier after each
// phase (Jacobi across particles, as with separate launches).  Two blocks an SM: with
// every phase's code in one kernel it takes 128 registers a thread (the separate
// launches 40 to 77).
template <int PARITY, int ST>
__device__ __forceinline__ void interp2_fused(const IbmArgs& A, int m, unsigned blk, int wf) {
  if (m == 0 || m == 1) {
    switch (A.box) {
      case 14: interp2_body<14, PARITY, 0, ST>(A, m, blk, wf); return;
      case 16: interp2_body<16, PARITY, 0, ST>(A, m, blk, wf); return;
      case 18: interp2_body<18, PARITY, 0, ST>(A, m, blk, wf); return;
      case 20: interp2_body<20, PARITY, 0, ST>(A, m, blk, wf); return;
      case 22: interp2_body<22, PARITY, 0, ST>(A, m, blk, wf); return;
      default: interp2_body<0, PARITY, 0, ST>(A, m, blk, wf); return;
    }
  }
  switch (A.box) {
    case 14: interp2_body<14, 0, 1, STORE_F32>(A, m, blk, wf); return;
    case 16: interp2_body<16, 0, 1, STORE_F32>(A, m, blk, wf); return;
    case 18: interp2_body<18, 0, 1, STORE_F32>(A, m, blk, wf); return;
    case 20: interp2_body<20, 0, 1, STORE_F32>(A, m, blk, wf); return;
    case 22: interp2_body<22, 0, 1, STORE_F32>(A, m, blk, wf); return;
    default: interp2_body<0, 0, 1, STORE_F32>(A, m, blk, wf); return;
  }
}

__device__ __forceinline__ void spread2_fused(const IbmArgs& A, unsigned blk, int wf) {
  switch (A.box) {
    case 14: spread2_body<14>(A, blk, wf); return;
    case 16: spread2_body<16>(A, blk, wf); return;
    case 18: spread2_body<18>(A, blk, wf); return;
    case 20: spread2_body<20>(A, blk, wf); return;
    case 22: spread2_body<22>(A, blk, wf); return;
    default: spread2_body<0>(A, blk, wf); return;
  }
}

__device__ __forceinline__ void forces2_fused(const IbmArgs& A, unsigned blk) {
  switch (A.box) {
    case 14: forces2_body<14>(A, blk); return;
    case 16: forces2_body<16>(A, blk); return;
    case 18: forces2_body<18>(A, blk); return;
    case 20: forces2_body<20>(A, blk); return;
    case 22: forces2_body<22>(A, blk); return;
    default: forces2_body<0>(A, blk); return;
  }
}

template <int PARITY, int ST>
__global__ void __launch_bounds__(kIbmWarps * 32, 2) ibm_batch_kernel(IbmBatch P) {
  unsigned blk;
  // a barrier of an earlier launch gave up: its counts are stale until the host resets them
  if (__syncthreads_or(threadIdx.x == 0 && (*(volatile uint32_t*)P.status & ST_TIMEOUT))) return;
  for (unsigned vb = blockIdx.x; vb < P.nlane; vb += gridDim.x) {
    const RegenArgs A = fused_args<RegenArgs>(P.regen, vb, blk);
    regen_body<2>(A, 0, blk);
  }
  if (!grid_barrier(P.bar, P.limit, P.status)) return;
  for (int m = P.mdf == 0 ? 0 : 1; m <= P.mdf; ++m) {
    for (unsigned vb = blockIdx.x; vb < P.nwarp; vb += gridDim.x) {
      const IbmArgs A = fused_args<IbmArgs>(P.warp, vb, blk);
      interp2_fused<PARITY, ST>(A, m, blk, P.wfloats);
    }
    if (!grid_barrier(P.bar, P.limit, P.status)) return;
    if (m == 0) break;
    for (unsigned vb = blockIdx.x; vb < P.nwarp; vb += gridDim.x) {
      const IbmArgs A = fused_args<IbmArgs>(P.warp, vb, blk);
      spread2_fused(A, blk, P.wfloats);
    }
    if (!grid_barrier(P.bar, P.limit, P.status)) return;
  }
  for (unsigned vb = blockIdx.x; vb < P.nlane; vb += gridDim.x) {
    const IbmArgs A = fused_args<IbmArgs>(P.lane, vb, blk);
    forces2_fused(A, blk);
  }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_ibm_interp(const IbmArgs& A, int m, cudaStream_t s) {
  if (A.npts == 0) return cudaSuccess;
  if (A.D == 2) {
    const int W = ibm2_warps(A.box);
    const unsigned grid = (unsigned)((A.np + W - 1) / W);
    const int mode = (m == 0 || m == 1) ? 0 : 1;  // m < 0: residual pass (box + f_IB/2)
    const size_t sm = sizeof(float) * W * (size_t)interp2_warp_floats(mode, A.box);
    cudaError_t e = cudaSuccess;  // programmatic launches (the kernel waits on entry)
#define IBMLBM_INTERP2_ST(SC, P)                                                             \
  do {                                                                                        \
    if (A.store == STORE_F32) e = launch_pdl(ibm_interp2_kernel<SC, P, 0, STORE_F32, false>, grid, W * 32, sm, s, A, m, Fuse{}); \
    else if (A.store == STORE_F16) e = launch_pdl(ibm_interp2_kernel<SC, P, 0, STORE_F16, false>, grid, W * 32, sm, s, A, m, Fuse{}); \
    else e = launch_pdl(ibm_interp2_kernel<SC, P, 0, STORE_BF16, false>, grid, W * 32, sm, s, A, m, Fuse{}); \
  } while (0)
#define IBMLBM_INTERP2(SC)                                                                   \
  do {                                                                                        \
    if (mode == 0) {                                                                          \
      if (A.parity == 0) IBMLBM_INTERP2_ST(SC, 0);                                            \
      else IBMLBM_INTERP2_ST(SC, 1);                                                          \
    } else {                                                                                  \
      e = launch_pdl(ibm_interp2_kernel<SC, 0, 1, STORE_F32, false>, grid, W * 32, sm, s, A, m, Fuse{}); \
    }                                                                                         \
  } while (0)
    if (A.box == 16) IBMLBM_INTERP2(16);
    else if (A.box == 22) IBMLBM_INTERP2(22);
    else IBMLBM_INTERP2(0);
#undef IBMLBM_INTERP2
#undef IBMLBM_INTERP2_ST
    if (e != cudaSuccess) return e;
  } else {
    return launch_ibm_interp3(A, m, s);
  }
  return cudaGetLastError();
}

// The attribute is per kernel and process-wide, so it only ever grows: a later, smaller
// run must not lower the limit an earlier, larger run still launches with.
// shared memory of the spreading kernel used for this dimension (the 2D
// interpolation kernel uses the same amount)
size_t spread_smem(int D, int nl, int box) {
  return D == 2 ? ibm2_smem(box) : ibm_mdf3_smem(nl, box);
}

cudaError_t prepare_ibm_spread(int D, size_t smem) {
  static std::mutex mu;
  static size_t granted[2] = {0, 0};
  std::lock_guard<std::mutex> lock(mu);
  size_t& g = granted[D == 2 ? 0 : 1];
  if (smem <= g) return cudaSuccess;
  cudaError_t e;
  if (D == 2) {
#define IBMLBM_I2(SC, P, ST) (const void*)ibm_interp2_kernel<SC, P, 0, ST, false>
#define IBMLBM_I2S(SC)                                                                     \
  IBMLBM_I2(SC, 0, STORE_F32), IBMLBM_I2(SC, 1, STORE_F32), IBMLBM_I2(SC, 0, STORE_F16),    \
      IBMLBM_I2(SC, 1, STORE_F16), IBMLBM_I2(SC, 0, STORE_BF16), IBMLBM_I2(SC, 1, STORE_BF16), \
      (const void*)ibm_interp2_kernel<SC, 0, 1, STORE_F32, false>
    const void* fns[] = {(const void*)ibm_spread2_kernel<16, false>, (const void*)ibm_spread2_kernel<22, false>,
                         (const void*)ibm_spread2_kernel<0, false>, IBMLBM_I2S(16), IBMLBM_I2S(22),
                         IBMLBM_I2S(0),
                         // fused over the members of a batch (runtime box size)
                         (const void*)ibm_spread2_kernel<0, true>,
                         (const void*)ibm_interp2_kernel<0, 0, 0, STORE_F32, true>,
                         (const void*)ibm_interp2_kernel<0, 1, 0, STORE_F32, true>,
                         (const void*)ibm_interp2_kernel<0, 0, 0, STORE_F16, true>,
                         (const void*)ibm_interp2_kernel<0, 1, 0, STORE_F16, true>,
                         (const void*)ibm_interp2_kernel<0, 0, 1, STORE_F32, true>};
#undef IBMLBM_I2S
#undef IBMLBM_I2
    e = cudaSuccess;
    for (const void* fn : fns)
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  } else {
    const void* fns[] = {(const void*)ibm_interp3_kernel<18, 0>, (const void*)ibm_interp3_kernel<18, 1>,
                         (const void*)ibm_interp3_kernel<14, 0>, (const void*)ibm_interp3_kernel<14, 1>,
                         (const void*)ibm_interp3_kernel<0, 0>,  (const void*)ibm_interp3_kernel<0, 1>,
                         (const void*)ibm_spread3_kernel<18>,   (const void*)ibm_spread3_kernel<14>,
                         (const void*)ibm_spread3_kernel<0>};
    e = cudaSuccess;
    for (const void* fn : fns)
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (e == cudaSuccess) g = smem;
  return e;
}

cudaError_t launch_ibm_spread(const IbmArgs& A, cudaStream_t s) {
  if (A.np == 0) return cudaSuccess;
  if (A.D == 2) {
    const int W = ibm2_warps(A.box);
    const unsigned grid = (unsigned)((A.np + W - 1) / W);
    const size_t sm = sizeof(float) * W * (size_t)spread2_warp_floats(A.box);
    cudaError_t e;  // programmatic launches (the kernel waits on entry)
    if (A.box == 16)
      e = launch_pdl(ibm_spread2_kernel<16, false>, grid, W * 32, sm, s, A, Fuse{});
    else if (A.box == 22)
      e = launch_pdl(ibm_spread2_kernel<22, false>, grid, W * 32, sm, s, A, Fuse{});
    else
      e = launch_pdl(ibm_spread2_kernel<0, false>, grid, W * 32, sm, s, A, Fuse{});
    if (e != cudaSuccess) return e;
  } else {
    return launch_ibm_spread3(A, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_ibm_forces(const IbmArgs& A, cudaStream_t s) {
  if (A.np == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(((long long)A.np * (A.D == 2 ? 16 : 32) + 255) / 256);
  if (A.D == 2) {
    cudaError_t e;  // programmatic launches (the kernel waits on entry)
    if (A.box == 16)
      e = launch_pdl(ibm_forces2_kernel<16, false>, grid, 256, 0, s, A, Fuse{});
    else if (A.box == 22)
      e = launch_pdl(ibm_forces2_kernel<22, false>, grid, 256, 0, s, A, Fuse{});
    else
      e = launch_pdl(ibm_forces2_kernel<0, false>, grid, 256, 0, s, A, Fuse{});
    if (e != cudaSuccess) return e;
  } else {
    ibm_forces_kernel<3><<<grid, 256, 0, s>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_regen(const RegenArgs& A, int init, cudaStream_t s) {
  if (A.np == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(((long long)A.np * 32 + 255) / 256);
  if (A.D == 2)
    regen_kernel<2, false><<<grid, 256, 0, s>>>(A, init, Fuse{});
  else
    regen_kernel<3, false><<<grid, 256, 0, s>>>(A, init, Fuse{});
  return cudaGetLastError();
}

// ---------------------------------------------- fused over the members of a 2D batch
// blocks of each 2D IBM kernel for one run of np particles
unsigned ibm_warp_blocks(int np) { return (unsigned)((np + kIbmWarps - 1) / kIbmWarps); }
unsigned ibm_lane_blocks(int np) { return (unsigned)(((long long)np * 32 + 255) / 256); }
unsigned ibm_half_blocks(int np) { return (unsigned)(((long long)np * 16 + 255) / 256); }

cudaError_t launch_ibm_interp_fused(const Fuse& F, unsigned blocks, size_t smem, int m, int parity,
                                    int store, cudaStream_t s) {
  const IbmArgs none{};
  if (m <= 1) {
    if (store == STORE_F32) {
      if (parity == 0) ibm_interp2_kernel<0, 0, 0, STORE_F32, true><<<blocks, kIbmWarps * 32, smem, s>>>(none, m, F);
      else ibm_interp2_kernel<0, 1, 0, STORE_F32, true><<<blocks, kIbmWarps * 32, smem, s>>>(none, m, F);
    } else {
      if (parity == 0) ibm_interp2_kernel<0, 0, 0, STORE_F16, true><<<blocks, kIbmWarps * 32, smem, s>>>(none, m, F);
      else ibm_interp2_kernel<0, 1, 0, STORE_F16, true><<<blocks, kIbmWarps * 32, smem, s>>>(none, m, F);
    }
  } else {
    ibm_interp2_kernel<0, 0, 1, STORE_F32, true><<<blocks, kIbmWarps * 32, smem, s>>>(none, m, F);
  }
  return cudaGetLastError();
}

cudaError_t launch_ibm_spread_fused(const Fuse& F, unsigned blocks, size_t smem, cudaStream_t s) {
  ibm_spread2_kernel<0, true><<<blocks, kIbmWarps * 32, smem, s>>>(IbmArgs{}, F);
  return cudaGetLastError();
}

cudaError_t launch_ibm_forces_fused(const Fuse& F, unsigned blocks, cudaStream_t s) {
  ibm_forces2_kernel<0, true><<<blocks, 256, 0, s>>>(IbmArgs{}, F);
  return cudaGetLastError();
}

cudaError_t launch_regen_fused(const Fuse& F, unsigned blocks, cudaStream_t s) {
  regen_kernel<2, true><<<blocks, 256, 0, s>>>(RegenArgs{}, 0, F);
  return cudaGetLastError();
}

template <int PARITY, int ST>
static cudaError_t ibm_batch_go(const IbmBatch& P0, size_t smem, cudaStream_t s, bool prepare) {
  auto kern = ibm_batch_kernel<PARITY, ST>;
  if (prepare) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kIbmWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  IbmBatch P = P0;
  // one shared-memory stride per warp for every member: a block's warps move on to
  // particles of other members (other box sizes) each at its own pace
  P.wfloats = (int)(smem / (sizeof(float) * kIbmWarps));
  const unsigned need = max(max(P.nwarp, P.nlane), 1u);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(min(need, (unsigned)(per_sm * sms)));
  cfg.blockDim = dim3(kIbmWarps * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, P);
}

// prepare (once, before any capture): allow the shared memory; otherwise launch
cudaError_t launch_ibm_batch(const IbmBatch& P, int parity, int store, size_t smem, cudaStream_t s,
                             bool prepare) {
  if (store == STORE_F32)
    return parity == 0 ? ibm_batch_go<0, STORE_F32>(P, smem, s, prepare) : ibm_batch_go<1, STORE_F32>(P, smem, s, prepare);
  return parity == 0 ? ibm_batch_go<0, STORE_F16>(P, smem, s, prepare) : ibm_batch_go<1, STORE_F16>(P, smem, s, prepare);
}

}  // namespace ibmlbm

namespace ibmlbm {
unsigned long long check_fault_ibm() { return take_check_fault(); }
}  // namespace ibmlbm
