// Immersed-boundary kernels (Sec. 2.2, Sec. 4) and the particle update (Sec. 2.3).
//
// Multi-direct forcing, iteration m = 1..M:
//   ibm_interp: one thread per Lagrangian point gathers the 4^D support nodes,
//     u_b = sum delta(x - X_b) (u* + dt f_IB / (2 rho_f))       (Eq. 7, 12, 47)
//     dF_b = 2 rho_f (U_b - u_b) / dt, F_b += dF_b              (Eq. 10)
//   ibm_spread: one block per particle accumulates dF_b delta dV on a shared-memory
//     box around the particle and adds the non-zero box cells to f_IB with one
//     global atomic per cell and component                      (Eq. 11, 13, 48)
// Gathering u* + f_IB/2 equals the paper's u^(m-1) = u^(m-2) + dt D_E dF/(2 rho_f)
// by linearity, so no separate velocity field is updated between iterations.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "launch.h"

namespace ibmlbm {

// 4-point regularised delta function (Fig. 2b; Peskin's form)
__device__ __forceinline__ float delta4(float r) {
  const float a = fabsf(r);
  if (a <= 1.0f) return 0.125f * (3.0f - 2.0f * a + sqrtf(fmaxf(0.0f, 1.0f + 4.0f * a - 4.0f * a * a)));
  if (a <= 2.0f) return 0.125f * (5.0f - 2.0f * a - sqrtf(fmaxf(0.0f, -7.0f + 12.0f * a - 4.0f * a * a)));
  return 0.0f;
}

struct AxisSup {
  int idx[4];
  float w[4];
  bool ok[4];
};

// support nodes floor(X)-1 .. floor(X)+2 along one axis; nodes beyond a wall are
// dropped, periodic axes wrap
__device__ __forceinline__ void axis_support(double X, int n, int per, AxisSup& s) {
  const int i0 = (int)floor(X) - 1;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int i = i0 + t;
    s.w[t] = delta4((float)((double)i - X));
    bool ok = true;
    if (i < 0 || i >= n) {
      if (per)
        i = ((i % n) + n) % n;
      else
        ok = false;
    }
    s.idx[t] = i;
    s.ok[t] = ok;
  }
}

template <int D>
__global__ void __launch_bounds__(256) ibm_interp_kernel(IbmArgs A, int m) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= A.npts) return;
  AxisSup sx, sy, sz;
  axis_support(A.Xb[b * D + 0], A.g.nx, A.g.per[0], sx);
  axis_support(A.Xb[b * D + 1], A.g.ny, A.g.per[1], sy);
  if (D == 3) {
    axis_support(A.Xb[b * D + 2], A.g.nz, A.g.per[2], sz);
  } else {
    sz.idx[0] = 0;
    sz.w[0] = 1.0f;
    sz.ok[0] = true;
  }
  float acc[3] = {0.0f, 0.0f, 0.0f};
  const long long N = A.g.N;
#pragma unroll
  for (int tz = 0; tz < (D == 3 ? 4 : 1); ++tz) {
    if (!sz.ok[tz]) continue;
#pragma unroll
    for (int ty = 0; ty < 4; ++ty) {
      if (!sy.ok[ty]) continue;
      const float wyz = sy.w[ty] * sz.w[tz];
      const long long rowbase = (long long)A.g.nx * ((long long)sy.idx[ty] + (long long)A.g.ny * sz.idx[tz]);
#pragma unroll
      for (int tx = 0; tx < 4; ++tx) {
        if (!sx.ok[tx]) continue;
        const long long n = rowbase + sx.idx[tx];
        const float w = sx.w[tx] * wyz;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          float v = A.ustar[c * N + n];
          if (m > 1) v += 0.5f * A.fib[c * N + n];
          acc[c] += w * v;
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const float dF = 2.0f * (A.Ub[b * D + c] - acc[c]);
    A.dFb[b * D + c] = dF;
    A.Fb[b * D + c] = (m == 1) ? dF : A.Fb[b * D + c] + dF;
    if (m == 1) A.ubs[b * D + c] = acc[c];
  }
}

size_t ibm_spread_smem(int D, int nl, int box) {
  size_t cells = 1;
  for (int k = 0; k < D; ++k) cells *= (size_t)box;
  return sizeof(float) * ((size_t)D * cells + (size_t)nl * D * 4) + sizeof(int) * (size_t)nl * D;
}

template <int D>
__global__ void __launch_bounds__(256) ibm_spread_kernel(IbmArgs A) {
  extern __shared__ float smem[];
  const int S = A.box;
  const int cells = (D == 3) ? S * S * S : S * S;
  float* box = smem;                                    // [D][cells]
  float* wts = box + D * cells;                         // [nl][D][4]
  int* base = reinterpret_cast<int*>(wts + A.nl * D * 4);  // [nl][D]
  const int i = blockIdx.x;
  int org[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) org[k] = (int)floor(A.Xc[(long long)i * D + k] - A.radius) - 2;

  for (int t = threadIdx.x; t < D * cells; t += blockDim.x) box[t] = 0.0f;
  for (int t = threadIdx.x; t < A.nl * D; t += blockDim.x) {
    const long long b = (long long)i * A.nl + t / D;
    const double X = A.Xb[b * D + (t % D)];
    const int i0 = (int)floor(X) - 1;
    base[t] = i0;
#pragma unroll
    for (int s = 0; s < 4; ++s) wts[t * 4 + s] = delta4((float)((double)(i0 + s) - X));
  }
  __syncthreads();

  constexpr int P = (D == 3) ? 64 : 16;
  const int n[3] = {A.g.nx, A.g.ny, A.g.nz};
  for (int q = threadIdx.x; q < A.nl * P; q += blockDim.x) {
    const int k = q / P, s = q % P;
    const int st[3] = {s & 3, (s >> 2) & 3, s >> 4};
    int loc[3] = {0, 0, 0};
    float w = A.dV;
    bool ok = true;
    for (int a = 0; a < D; ++a) {
      const int gcoord = base[k * D + a] + st[a];
      if (!A.g.per[a] && (gcoord < 0 || gcoord >= n[a])) ok = false;
      loc[a] = gcoord - org[a];
      if (loc[a] < 0 || loc[a] >= S) {
        ok = false;
        atomicOr(A.status, ST_CAPACITY);
      }
      w *= wts[(k * D + a) * 4 + st[a]];
    }
    if (!ok) continue;
    const int cell = loc[0] + S * (loc[1] + S * loc[2]);
    const long long b = (long long)i * A.nl + k;
    for (int c = 0; c < D; ++c) atomicAdd(&box[c * cells + cell], A.dFb[b * D + c] * w);
  }
  __syncthreads();

  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    int gc[3] = {org[0] + t % S, org[1] + (t / S) % S, (D == 3) ? org[2] + t / (S * S) : 0};
    bool ok = true;
    for (int a = 0; a < D; ++a) {
      if (gc[a] < 0 || gc[a] >= n[a]) {
        if (A.g.per[a])
          gc[a] = ((gc[a] % n[a]) + n[a]) % n[a];
        else
          ok = false;
      }
    }
    if (!ok) continue;
    const long long nn = (long long)gc[0] + (long long)A.g.nx * ((long long)gc[1] + (long long)A.g.ny * gc[2]);
    for (int c = 0; c < D; ++c) {
      const float v = box[c * cells + t];
      if (v != 0.0f) atomicAdd(&A.fib[c * A.g.N + nn], v);
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Momentum and angular momentum about X_c of the fluid at the nodes strictly inside
// each particle, with the corrected velocity u* + f_IB/2 after the MDF iterations;
// the inside test |x - X_c|^2 < R^2 is evaluated without fused multiply-add.
template <int D>
__global__ void __launch_bounds__(256) interior_momentum_kernel(IbmArgs A) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= A.np) return;
  double X[3] = {0.0, 0.0, 0.0};
  int lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
  const int n[3] = {A.g.nx, A.g.ny, A.g.nz};
  for (int k = 0; k < D; ++k) {
    X[k] = A.Xc[(long long)i * D + k];
    lo[k] = (int)floor(X[k] - A.radius);
    ext[k] = (int)ceil(X[k] + A.radius) - lo[k] + 1;
  }
  const double R2 = __dmul_rn(A.radius, A.radius);
  double P[3] = {0.0, 0.0, 0.0}, L[3] = {0.0, 0.0, 0.0};
  const int total = ext[0] * ext[1] * ext[2];
  for (int t = lane; t < total; t += 32) {
    int gc[3] = {lo[0] + t % ext[0], lo[1] + (t / ext[0]) % ext[1], lo[2] + t / (ext[0] * ext[1])};
    double r[3] = {0.0, 0.0, 0.0};
    bool ok = true;
    for (int k = 0; k < D; ++k) {
      r[k] = (double)gc[k] - X[k];
      if (gc[k] < 0 || gc[k] >= n[k]) {
        if (A.g.per[k])
          gc[k] = ((gc[k] % n[k]) + n[k]) % n[k];
        else
          ok = false;
      }
    }
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])), __dmul_rn(r[2], r[2]));
    if (!ok || !(d2 < R2)) continue;
    const long long nn = (long long)gc[0] + (long long)A.g.nx * ((long long)gc[1] + (long long)A.g.ny * gc[2]);
    double u[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < D; ++c) u[c] = (double)(A.ustar[c * A.g.N + nn] + 0.5f * A.fib[c * A.g.N + nn]);
    for (int c = 0; c < 3; ++c) P[c] += u[c];
    L[0] += r[1] * u[2] - r[2] * u[1];
    L[1] += r[2] * u[0] - r[0] * u[2];
    L[2] += r[0] * u[1] - r[1] * u[0];
  }
  for (int c = 0; c < 3; ++c) {
    P[c] = warp_sum(P[c]);
    L[c] = warp_sum(L[c]);
  }
  if (lane == 0) {
    for (int c = 0; c < D; ++c) A.Pint[(long long)i * D + c] = P[c];
    for (int c = 0; c < 3; ++c) A.Lint[(long long)i * 3 + c] = L[c];
  }
}

// Newton-Euler update of one particle per warp (double precision), regeneration of its
// Lagrangian points for the next step and marking of the nodes within mark_radius of
// the new centre.  mode 0 only regenerates and marks (initial state).
//   F_h = -sum_b F_b dV, T_h = -sum_b r_b x F_b dV                 (Eq. 14-15)
//   (M_p + K) a^n - K a^{n-1} = (F_h^n + F_h^{n-1})/2 + F_c + (P_int^n - P_int^{n-1})
//                              + (M_p - rho_f V_p) g
//   U^{n+1} = U^n + a^n, X^{n+1} = X^n + (U^n + U^{n+1})/2; rotation alike with I_p, K_r.
template <int D>
__global__ void __launch_bounds__(256) particle_update_kernel(PartArgs A, int mode,
                                                              int have_prev) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= A.np) return;
  const long long pi = i;
  if (mode == 1) {
    double fh[3] = {0.0, 0.0, 0.0}, th[3] = {0.0, 0.0, 0.0};
    for (int k = lane; k < A.nl; k += 32) {
      const long long b = pi * A.nl + k;
      double r[3] = {0.0, 0.0, 0.0}, F[3] = {0.0, 0.0, 0.0};
      for (int c = 0; c < D; ++c) {
        r[c] = A.ref[k * D + c];
        F[c] = (double)A.Fb[b * D + c];
        fh[c] -= F[c] * A.dV;
      }
      th[0] -= (r[1] * F[2] - r[2] * F[1]) * A.dV;
      th[1] -= (r[2] * F[0] - r[0] * F[2]) * A.dV;
      th[2] -= (r[0] * F[1] - r[1] * F[0]) * A.dV;
    }
    for (int c = 0; c < 3; ++c) {
      fh[c] = warp_sum(fh[c]);
      th[c] = warp_sum(th[c]);
    }
    if (lane == 0) {
      bool bad = false;
      for (int c = 0; c < D; ++c) {
        const long long o = pi * D + c;
        const double Fm = 0.5 * (fh[c] + A.Fhp[o]);
        const double dP = have_prev ? A.Pint[o] - A.Pprev[o] : 0.0;
        A.Fh[o] = fh[c];
        A.Fhp[o] = fh[c];
        A.Pprev[o] = A.Pint[o];
        if (!A.fixed) {
          const double F = Fm + A.Fc[o] + dP + A.meff * A.grav[c];
          const double a = (F + A.Kt * A.acc[o]) / (A.Mp + A.Kt);
          const double u0 = A.U[o], u1 = u0 + a;
          A.acc[o] = a;
          A.U[o] = u1;
          A.X[o] += 0.5 * (u0 + u1);
        }
      }
      for (int c = (D == 2 ? 2 : 0); c < 3; ++c) {
        const long long o = pi * 3 + c;
        const double Tm = 0.5 * (th[c] + A.Thp[o]);
        const double dL = have_prev ? A.Lint[o] - A.Lprev[o] : 0.0;
        A.Th[o] = th[c];
        A.Thp[o] = th[c];
        A.Lprev[o] = A.Lint[o];
        if (!A.fixed) {
          const double al = (Tm + dL + A.Kr * A.alp[o]) / (A.Ip + A.Kr);
          A.alp[o] = al;
          A.Om[o] += al;
        }
      }
      const int n[3] = {A.g.nx, A.g.ny, A.g.nz};
      for (int c = 0; c < D; ++c) {
        double& x = A.X[pi * D + c];
        if (A.g.per[c]) {
          if (x >= n[c] - 0.5)
            x -= n[c];
          else if (x < -0.5)
            x += n[c];
        } else if (!(x >= -0.5 && x < n[c] - 0.5)) {
          atomicOr(A.status, ST_OUT_OF_DOMAIN);
        }
        if (!isfinite(x) || !isfinite(A.U[pi * D + c])) bad = true;
      }
      for (int c = 0; c < 3; ++c)
        if (!isfinite(A.Om[pi * 3 + c])) bad = true;
      if (bad) atomicOr(A.status, ST_NONFINITE);
    }
    __syncwarp();
  }
  double X[3] = {0.0, 0.0, 0.0}, U[3] = {0.0, 0.0, 0.0}, Om[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < D; ++c) {
    X[c] = A.X[pi * D + c];
    U[c] = A.U[pi * D + c];
  }
  for (int c = 0; c < 3; ++c) Om[c] = A.Om[pi * 3 + c];
  if (D == 2) Om[0] = Om[1] = 0.0;
  for (int k = lane; k < A.nl; k += 32) {
    const long long b = pi * A.nl + k;
    double r[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < D; ++c) r[c] = A.ref[k * D + c];
    const double w[3] = {Om[1] * r[2] - Om[2] * r[1], Om[2] * r[0] - Om[0] * r[2],
                         Om[0] * r[1] - Om[1] * r[0]};
    for (int c = 0; c < D; ++c) {
      A.Xb_out[b * D + c] = X[c] + r[c];
      A.Ub_out[b * D + c] = (float)(U[c] + w[c]);
    }
  }
  // mark the nodes of the ball |x - X_c| <= mark_radius, row by row
  const double Rm = A.mark_radius, Rm2 = Rm * Rm;
  const int ylo = (int)ceil(X[1] - Rm), yhi = (int)floor(X[1] + Rm);
  const int zlo = (D == 3) ? (int)ceil(X[2] - Rm) : 0, zhi = (D == 3) ? (int)floor(X[2] + Rm) : 0;
  const int ey = yhi - ylo + 1, ez = zhi - zlo + 1;
  for (int t = lane; t < ey * ez; t += 32) {
    int gy = ylo + t % ey, gz = zlo + t / ey;
    const double dy = gy - X[1], dz = (D == 3) ? gz - X[2] : 0.0;
    const double rem = Rm2 - dy * dy - dz * dz;
    if (rem < 0.0) continue;
    if (gy < 0 || gy >= A.g.ny) {
      if (!A.g.per[1]) continue;
      gy = ((gy % A.g.ny) + A.g.ny) % A.g.ny;
    }
    if (D == 3 && (gz < 0 || gz >= A.g.nz)) {
      if (!A.g.per[2]) continue;
      gz = ((gz % A.g.nz) + A.g.nz) % A.g.nz;
    }
    const double h = sqrt(rem);
    int x0 = (int)ceil(X[0] - h), x1 = (int)floor(X[0] + h);
    uint32_t* row = A.mask + ((long long)gy + (long long)A.g.ny * gz) * A.g.wpr;
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

// ------------------------------------------------------------------ launchers
cudaError_t launch_ibm_interp(const IbmArgs& A, int m, cudaStream_t s) {
  if (A.npts == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((A.npts + 255) / 256);
  if (A.D == 2)
    ibm_interp_kernel<2><<<grid, 256, 0, s>>>(A, m);
  else
    ibm_interp_kernel<3><<<grid, 256, 0, s>>>(A, m);
  return cudaGetLastError();
}

// The attribute is per kernel and process-wide, so it only ever grows: a later, smaller
// run must not lower the limit an earlier, larger run still launches with.
cudaError_t prepare_ibm_spread(int D, size_t smem) {
  static std::mutex mu;
  static size_t granted[2] = {0, 0};
  std::lock_guard<std::mutex> lock(mu);
  size_t& g = granted[D == 2 ? 0 : 1];
  if (smem <= g) return cudaSuccess;
  const cudaError_t e =
      (D == 2) ? cudaFuncSetAttribute(ibm_spread_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
               : cudaFuncSetAttribute(ibm_spread_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) g = smem;
  return e;
}

cudaError_t launch_ibm_spread(const IbmArgs& A, cudaStream_t s) {
  if (A.np == 0) return cudaSuccess;
  const size_t smem = ibm_spread_smem(A.D, A.nl, A.box);
  if (A.D == 2)
    ibm_spread_kernel<2><<<A.np, 256, smem, s>>>(A);
  else
    ibm_spread_kernel<3><<<A.np, 256, smem, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_interior_momentum(const IbmArgs& A, cudaStream_t s) {
  if (A.np == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(((long long)A.np * 32 + 255) / 256);
  if (A.D == 2)
    interior_momentum_kernel<2><<<grid, 256, 0, s>>>(A);
  else
    interior_momentum_kernel<3><<<grid, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_particle_update(const PartArgs& A, int mode, int have_prev, cudaStream_t s) {
  if (A.np == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(((long long)A.np * 32 + 255) / 256);
  if (A.D == 2)
    particle_update_kernel<2><<<grid, 256, 0, s>>>(A, mode, have_prev);
  else
    particle_update_kernel<3><<<grid, 256, 0, s>>>(A, mode, have_prev);
  return cudaGetLastError();
}

}  // namespace ibmlbm
