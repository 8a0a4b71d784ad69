// Reading the PDFs of a node under the AA-pattern layout (device helpers shared by
// the lattice kernels and the immersed-boundary kernels).
//
// AA pattern, one PDF array a[Q][N] (planes g.Np >= N elements apart):
//   parity 0 (before an even step): f_a(x) is stored at a[a][x];
//   parity 1 (before an odd step): f_a(x) is stored at a[opp(a)][x - e_a], or at
//     a[a][x] when x - e_a lies beyond a wall (halfway bounce-back).
//
// Storage of one PDF (the run's pdf_storage): FP32 as is, or FP16 / BF16 holding
// h_a = f_a / w_a (in the deviation gauge f = 0 at rest, so dividing by the weight
// puts every direction on one scale); all arithmetic stays FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace ibmlbm {

enum : int { STORE_F32 = 0, STORE_F16 = 1, STORE_BF16 = 2 };

template <int ST>
struct PdfType;
template <>
struct PdfType<STORE_F32> {
  using T = float;
};
template <>
struct PdfType<STORE_F16> {
  using T = __half;
};
template <>
struct PdfType<STORE_BF16> {
  using T = __nv_bfloat16;
};

// RAW: the stored variable itself (h_a for the 16-bit storages), without the weight
template <class L, int ST, bool RAW = false>
__device__ __forceinline__ float pdf_load(const void* f, long long idx, int a) {
  if constexpr (ST == STORE_F32) {
    return static_cast<const float*>(f)[idx];
  } else if constexpr (ST == STORE_F16) {
    const float h = __half2float(static_cast<const __half*>(f)[idx]);
    return RAW ? h : L::w(a) * h;
  } else {
    const float h = __bfloat162float(static_cast<const __nv_bfloat16*>(f)[idx]);
    return RAW ? h : L::w(a) * h;
  }
}

template <class L, int ST, bool RAW = false>
__device__ __forceinline__ void pdf_store(void* f, long long idx, int a, float v) {
  if constexpr (ST == STORE_F32) {
    static_cast<float*>(f)[idx] = v;
  } else if constexpr (ST == STORE_F16) {
    static_cast<__half*>(f)[idx] = __float2half_rn(RAW ? v : v * (1.0f / L::w(a)));
  } else {
    static_cast<__nv_bfloat16*>(f)[idx] = __float2bfloat16_rn(RAW ? v : v * (1.0f / L::w(a)));
  }
}

// index of the neighbour x - s*e_a (s = +1 for the pull source, -1 for the push
// target); false if it lies beyond a wall
template <class L>
__device__ __forceinline__ bool neighbour(const Geo& g, int a, int s, int x, int y, int z,
                                          long long n, long long& idx) {
  idx = n;
  const int ex = s * L::e(a, 0), ey = s * L::e(a, 1), ez = s * L::e(a, 2);
  if (ex) {
    const int t = x - ex;
    if (t < 0 || t >= g.nx) {
      if (!g.per[0]) return false;
      idx += (t < 0) ? g.nx : -g.nx;
    }
    idx -= ex;
  }
  if (ey) {
    const int t = y - ey;
    if (t < 0 || t >= g.ny) {
      if (!g.per[1]) return false;
      idx += (long long)((t < 0) ? g.ny : -g.ny) * g.nx;
    }
    idx -= (long long)ey * g.nx;
  }
  if (L::dim == 3 && ez) {
    const int t = z - ez;
    const long long plane = (long long)g.nx * g.ny;
    if (t < 0 || t >= g.nz) {
      if (!g.per[2]) return false;
      idx += ((t < 0) ? g.nz : -g.nz) * plane;
    }
    idx -= ez * plane;
  }
  return true;
}

// offset of the neighbour x - s*e_a for a node whose whole neighbourhood is inside
template <class L>
__device__ __forceinline__ long long inner_offset(const Geo& g, int a, int s) {
  return -(long long)s * ((long long)L::e(a, 0) + (long long)g.nx * L::e(a, 1) +
                          (long long)g.nx * g.ny * L::e(a, 2));
}

// pre-collision PDFs f_a(x) of the current time under the layout of the given parity;
// INNER: the node is at least one node away from every domain face; RAW: the stored
// variable (h_a = f_a / w_a for the 16-bit storages)
template <class L, int PARITY, int ST, bool INNER = false, bool RAW = false>
__device__ __forceinline__ void load_pdfs(const Geo& g, const void* __restrict__ f, int x,
                                          int y, int z, long long n, float (&fa)[L::Q]) {
  const long long N = g.Np;  // plane stride
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    long long idx;
    int s = a;  // direction whose slot is read
    if (PARITY == 0 || a == 0) {
      idx = a * N + n;
    } else if (INNER) {
      idx = opp<L>(a) * N + n + inner_offset<L>(g, a, 1);
      s = opp<L>(a);
    } else {
      long long src;
      if (neighbour<L>(g, a, 1, x, y, z, n, src)) {
        idx = opp<L>(a) * N + src;
        s = opp<L>(a);
      } else {
        idx = a * N + n;
      }
    }
    fa[a] = IBMLBM_CHK(idx, L::Q * N) ? pdf_load<L, ST, RAW>(f, idx, s) : 0.0f;
  }
}

// Eq. 5 (u* = sum e f) and the sum of the moving populations used by Eq. 6
template <class L>
__device__ __forceinline__ void moments(const float (&f)[L::Q], float (&us)[3], float& s1) {
  us[0] = us[1] = us[2] = 0.0f;
  s1 = 0.0f;
#pragma unroll
  for (int a = 1; a < L::Q; ++a) {
    s1 += f[a];
#pragma unroll
    for (int k = 0; k < L::dim; ++k) {
      if (L::e(a, k) == 1) us[k] += f[a];
      if (L::e(a, k) == -1) us[k] -= f[a];
    }
  }
}

}  // namespace ibmlbm
