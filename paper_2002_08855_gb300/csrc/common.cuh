// Shared device-side definitions of the IB-LBM hot path (sm_103a).
//
// Lattices D2Q9 (Eq. 2) and D3Q19 (Eq. 3; the printed z row drops one entry,
// e_9 = (-1, 0, 1) restores e_a = -e_{a-9}), weights as listed after Eq. 4.
// Units: dh = dt = 1, cs^2 = 1/3, rho_0 = rho_f = 1.
//
// Data layout in HBM (one workspace, carved by the host):
//   f      [Q][N]  float  PDFs, one copy, AA-pattern in-place streaming
//   ustar  [D][N]  float  u* = sum_a e_a f_a, written only on flagged nodes
//   fib    [D][N]  float  IB force density; zero outside the IBM phase
//   mask   [rows][wpr] u32  one bit per node: nodes within R + 2 sqrt(D) of a
//                           particle centre (support of every Lagrangian point
//                           and the particle interior)
//   particle state in double, Lagrangian point data [npts][D]; point positions as
//   32.32 fixed-point int64 (integer part = node anchor, low word = fraction), so
//   per-point work needs no double-precision arithmetic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ibmlbm {

// device status word bits
enum : uint32_t {
  ST_NONFINITE = 1u,
  ST_OUT_OF_DOMAIN = 2u,
  ST_CAPACITY = 4u,
};

// ------------------------------------------------------------------ lattices
template <int D>
struct Lat;

template <>
struct Lat<2> {
  static constexpr int dim = 2, Q = 9, H = 4;
  __host__ __device__ static constexpr int e(int a, int k) {
    return k == 0 ? ((a == 1 || a == 2 || a == 8) ? 1 : (a == 4 || a == 5 || a == 6) ? -1 : 0)
         : k == 1 ? ((a == 2 || a == 3 || a == 4) ? 1 : (a == 6 || a == 7 || a == 8) ? -1 : 0)
                  : 0;
  }
  __host__ __device__ static constexpr float w(int a) {
    return a == 0 ? 4.0f / 9.0f : (a & 1) ? 1.0f / 9.0f : 1.0f / 36.0f;
  }
};

template <>
struct Lat<3> {
  static constexpr int dim = 3, Q = 19, H = 9;
  __host__ __device__ static constexpr int e(int a, int k) {
    return k == 0 ? ((a == 1 || a == 4 || a == 8 || a == 14 || a == 18) ? 1
                     : (a == 5 || a == 9 || a == 10 || a == 13 || a == 17) ? -1 : 0)
         : k == 1 ? ((a == 2 || a == 4 || a == 5 || a == 6 || a == 16) ? 1
                     : (a == 7 || a == 11 || a == 13 || a == 14 || a == 15) ? -1 : 0)
                  : ((a == 3 || a == 6 || a == 7 || a == 8 || a == 9) ? 1
                     : (a == 12 || a == 15 || a == 16 || a == 17 || a == 18) ? -1 : 0);
  }
  __host__ __device__ static constexpr float w(int a) {
    return a == 0 ? 1.0f / 3.0f
         : ((a >= 1 && a <= 3) || (a >= 10 && a <= 12)) ? 1.0f / 18.0f : 1.0f / 36.0f;
  }
};

template <class L>
__host__ __device__ constexpr int opp(int a) {
  return a == 0 ? 0 : (a <= L::H ? a + L::H : a - L::H);
}

// ------------------------------------------------------------------ geometry
struct Geo {
  int nx, ny, nz;
  int per[3];      // periodic flags
  int rows;        // ny * nz
  int wpr;         // mask words per row = ceil(nx / 32)
  long long N;     // nx * ny * nz
};

__device__ __forceinline__ long long node_of(const Geo& g, int x, int y, int z) {
  return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
}

// Move coordinate c by s along an axis of n nodes; false if it leaves through a wall.
__device__ __forceinline__ bool step_axis(int c, int s, int n, int periodic, int& out) {
  int t = c + s;
  if (t >= 0 && t < n) {
    out = t;
    return true;
  }
  if (!periodic) return false;
  out = t < 0 ? t + n : t - n;
  return true;
}

// ------------------------------------------------------------ fixed point
// Positions as int64 with 32 fractional bits: exact integer addition of offsets,
// floor(X) = arithmetic shift, fraction exact to 2^-32 before the float conversion.
constexpr double kFixScale = 4294967296.0;  // 2^32

__host__ __device__ __forceinline__ int fix_anchor(long long v) { return (int)(v >> 32); }
__host__ __device__ __forceinline__ float fix_frac(long long v) {
  return (float)(unsigned)(v & 0xffffffffLL) * (1.0f / 4294967296.0f);
}

// compensated single-precision accumulator (Knuth's TwoSum on every addition)
struct FF {
  float hi, lo;
};
__device__ __forceinline__ void ff_add(FF& s, float x) {
  const float t = s.hi + x;
  const float bp = t - s.hi;
  s.lo += (s.hi - (t - bp)) + (x - bp);
  s.hi = t;
}
__device__ __forceinline__ FF ff_warp_sum(FF s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, s.hi, o);
    const float l = __shfl_xor_sync(0xffffffffu, s.lo, o);
    ff_add(s, h);
    s.lo += l;
  }
  return s;
}
__device__ __forceinline__ double ff_value(FF s) { return (double)s.hi + (double)s.lo; }

// ------------------------------------------------------------ kernel arguments
struct LbmArgs {
  Geo g;
  float* f;
  float* ustar;
  float* fib;
  uint32_t* mask;
  float omega;       // 1 / tau
  float kforce;      // 1 - omega / 2 (Eq. 8 prefactor)
  float body[3];     // uniform body force
};

struct IbmArgs {
  Geo g;
  int D;             // dimension
  int np, nl;
  long long npts;
  double radius;     // D_p / 2
  float radius_f;    // D_p / 2 as float
  int rcell;         // ceil(D_p / 2)
  float dV;          // point volume (Eq. 13 reading)
  int box;           // side of the spreading box (nodes)
  const float* ustar;
  float* fib;
  const long long* Xb;  // [npts][D] fixed point
  const float* Ub;   // [npts][D]
  float* Fb;         // [npts][D] sum of MDF increments
  float* dFb;        // [npts][D] increment of the current iteration
  float* ubs;        // [npts][D] D_I u*
  const double* Xc;  // [np][D]
  const long long* Xcf;  // [np][D] fixed point centres
  double* Pint;      // [np][D]
  double* Lint;      // [np][3]
  uint32_t* status;
};

struct PartArgs {
  Geo g;
  int D;
  int np, nl;
  double radius;
  float mark_radius;   // radius of the marked ball (float, already padded)
  double dV;
  double Mp, meff, Ip, Kt, Kr;
  double grav[3];
  int fixed;
  const long long* ref_fix;  // [nl][D] offsets of the points, fixed point
  const float* ref_f;        // [nl][D] offsets of the points, float
  const float* Fb;     // [npts][D]
  double* X;           // [np][D]
  double* U;           // [np][D]
  double* Om;          // [np][3]
  double* Fh;          // [np][D]
  double* Th;          // [np][3]
  double* Fhp;         // [np][D] previous step
  double* Thp;         // [np][3]
  double* acc;         // [np][D] previous linear acceleration
  double* alp;         // [np][3] previous angular acceleration
  const double* Pint;  // [np][D] interior momentum of this step
  const double* Lint;  // [np][3]
  double* Pprev;       // [np][D]
  double* Lprev;       // [np][3]
  const double* Fc;    // [np][D]
  long long* Xcf;       // [np][D] fixed-point centres (written)
  long long* Xb_out;   // [npts][D] fixed-point points for the next step
  float* Ub_out;       // [npts][D]
  uint32_t* mask;
  uint32_t* status;
};

struct PairArgs {
  Geo g;
  int D;
  int n;
  int nc[3];
  double H[3];
  double L[3];
  double diam, zeta, thr2;
  double c_ij, eps_pp, E_pp;
  int kmax;
  const double* X;      // [n][D]
  int* cell_count;      // [ncells]
  int* cell_start;      // [ncells + 1]
  int* sorted;          // [n]
  int* nbr;             // [n][kmax]
  int* nbr_count;       // [n]
  double* Fc;           // [n][D] (may be null: pair list only)
  int* gt_count;        // [n + 1] partners j > i, then their offsets
  uint32_t* status;
};

}  // namespace ibmlbm
