// Lattice-Boltzmann kernels: fused SRT-LBGK collision with Guo split forcing and
// in-place AA-pattern streaming with halfway bounce-back (Eq. 1, 4-8, 17-18), the
// macroscopic velocity on flagged nodes (Eq. 5), and layout helpers.
//
// AA pattern, one PDF array a[Q][N]:
//   even step (parity 0): node x reads f_a(x) from a[a][x] and writes the
//     post-collision f*_a to a[opp(a)][x]          (purely local);
//   odd step (parity 1): node x reads f_a(x) from a[opp(a)][x - e_a], or from a[a][x]
//     when x - e_a lies beyond a wall (halfway bounce-back of the even step), and
//     writes f*_a to a[a][x + e_a], or to a[opp(a)][x] when x + e_a lies beyond a wall.
// Each node reads and writes the same set of slots, so no two nodes race and one
// copy of the PDFs suffices (the role the swap algorithm of Sec. 3.3 plays on a CPU).
#include "common.cuh"
#include "launch.h"
#include "pdf_access.cuh"

namespace ibmlbm {

constexpr int kLbmBlock = 128;

// inverse of load_pdfs: slot of f_a(x) under the layout of the given parity
template <class L, int PARITY>
__device__ __forceinline__ void put_pdfs(const Geo& g, float* __restrict__ f, int x, int y,
                                         int z, long long n, const float (&fa)[L::Q]) {
  const long long N = g.N;
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    if (PARITY == 0 || a == 0) {
      f[a * N + n] = fa[a];
    } else {
      long long src;
      if (neighbour<L>(g, a, 1, x, y, z, n, src))
        f[opp<L>(a) * N + src] = fa[a];
      else
        f[a * N + n] = fa[a];
    }
  }
}

// post-collision store of the given parity (after which the opposite parity holds)
template <class L, int PARITY, bool INNER = false>
__device__ __forceinline__ void store_post(const Geo& g, float* __restrict__ f, int x, int y,
                                           int z, long long n, const float (&fa)[L::Q]) {
  const long long N = g.N;
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    if (a == 0) {
      f[n] = fa[0];
    } else if (PARITY == 0) {
      f[opp<L>(a) * N + n] = fa[a];
    } else if (INNER) {
      f[a * N + n + inner_offset<L>(g, a, -1)] = fa[a];
    } else {
      long long dst;
      if (neighbour<L>(g, a, -1, x, y, z, n, dst))
        f[a * N + dst] = fa[a];
      else
        f[opp<L>(a) * N + n] = fa[a];
    }
  }
}

// Eq. 6: p = cs^2/(1 - w0) (sum_{a>=1} f_a - rho0 w0 |u|^2 / (2 cs^2))
template <class L>
__device__ __forceinline__ float pressure(float s1, float uu) {
  constexpr float w0 = L::w(0);
  return s1 * (1.0f / (3.0f * (1.0f - w0))) - uu * (w0 / (2.0f * (1.0f - w0)));
}

// Eq. 4 equilibrium, Eq. 8 forcing term and the relaxation of Eq. 41-42, computed
// for each opposite pair (a, a + H) from one shared even part (Eq. 38, Eq. 40).
template <class L>
__device__ __forceinline__ void collide(float (&f)[L::Q], const float (&F)[3], float omega,
                                        float kforce) {
  float us[3], s1;
  moments<L>(f, us, s1);
  float u[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) u[k] = (k < L::dim) ? us[k] + 0.5f * F[k] : 0.0f;  // Eq. 7
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  const float p = pressure<L>(s1, uu);
  {
    constexpr float w0 = L::w(0);
    const float feq = 3.0f * (w0 - 1.0f) * p - 1.5f * w0 * uu;
    const float Fa = -3.0f * kforce * w0 * uF;
    f[0] = f[0] - omega * (f[0] - feq) + Fa;
  }
#pragma unroll
  for (int a = 1; a <= L::H; ++a) {
    const float w = L::w(a);
    float eu = 0.0f, eF = 0.0f;
#pragma unroll
    for (int k = 0; k < L::dim; ++k) {
      if (L::e(a, k) == 1) {
        eu += u[k];
        eF += F[k];
      }
      if (L::e(a, k) == -1) {
        eu -= u[k];
        eF -= F[k];
      }
    }
    const float eq_even = w * (3.0f * p + 4.5f * eu * eu - 1.5f * uu);
    const float eq_odd = 3.0f * w * eu;
    const float F_even = kforce * w * (9.0f * eu * eF - 3.0f * uF);
    const float F_odd = 3.0f * kforce * w * eF;
    const int b = a + L::H;
    f[a] = f[a] - omega * (f[a] - (eq_even + eq_odd)) + (F_even + F_odd);
    f[b] = f[b] - omega * (f[b] - (eq_even - eq_odd)) + (F_even - F_odd);
  }
}

struct NodeCoord {
  int x, y, z;
  long long row, n;
  bool valid;
};

// 32-bit index arithmetic (rows < 2^31); only the flat node index is 64-bit
__device__ __forceinline__ NodeCoord node_coord(const Geo& g, int cpr) {
  NodeCoord c;
  const unsigned b = blockIdx.x, ucpr = (unsigned)cpr, uny = (unsigned)g.ny;
  const unsigned row = b / ucpr;
  const unsigned chunk = b - row * ucpr;
  const unsigned z = row / uny;
  c.row = row;
  c.x = (int)(chunk * kLbmBlock + threadIdx.x);
  c.y = (int)(row - z * uny);
  c.z = (int)z;
  c.valid = c.x < g.nx;
  c.n = (long long)c.x + (long long)g.nx * (long long)row;
  return c;
}

// ------------------------------------------------------------------ kernels

// whole block (one row segment) at least one node away from every domain face
__device__ __forceinline__ bool block_inner(const Geo& g, int x0, int y, int z, int dim) {
  return x0 >= 1 && x0 + kLbmBlock <= g.nx - 1 && y >= 1 && y <= g.ny - 2 &&
         (dim == 2 || (z >= 1 && z <= g.nz - 2));
}

template <class L, int PARITY, bool INNER>
__device__ __forceinline__ void step_node(const LbmArgs& A, const NodeCoord& c) {
  float* __restrict__ f = A.f;
  float* __restrict__ fib = A.fib;
  float fa[L::Q];
  float fv[3] = {0.0f, 0.0f, 0.0f};
  // the IB force is read for every node together with the PDFs (one memory latency);
  // it is zero wherever no Lagrangian point spread into the node
  load_pdfs<L, PARITY, INNER>(A.g, f, c.x, c.y, c.z, c.n, fa);
  if (L::dim == 2) {  // interleaved [N][2]
    const float2 v = reinterpret_cast<const float2*>(fib)[c.n];
    fv[0] = v.x;
    fv[1] = v.y;
  } else {  // [N][4]; non-zero only on nodes the particle update marked
    if ((A.mask[c.row * A.g.wpr + (c.x >> 5)] >> (c.x & 31)) & 1u) {
      const float4 v = reinterpret_cast<const float4*>(fib)[c.n];
      fv[0] = v.x;
      fv[1] = v.y;
      fv[2] = v.z;
    }
  }
  float F[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) F[k] = A.body[k] + fv[k];
  collide<L>(fa, F, A.omega, A.kforce);
  store_post<L, PARITY, INNER>(A.g, f, c.x, c.y, c.z, c.n, fa);
  if (L::dim == 2) {
    if (fv[0] != 0.0f || fv[1] != 0.0f) reinterpret_cast<float2*>(fib)[c.n] = make_float2(0.0f, 0.0f);
  } else if (fv[0] != 0.0f || fv[1] != 0.0f || fv[2] != 0.0f) {
    reinterpret_cast<float4*>(fib)[c.n] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

// One full time step on every node: read f (AA parity) and the IB force (3D: on marked
// nodes only), collide, stream in place, clear the IB force.
template <class L, int PARITY>
__global__ void __launch_bounds__(kLbmBlock) lbm_step_kernel(LbmArgs A, int cpr) {
  const NodeCoord c = node_coord(A.g, cpr);
  if (PARITY == 1 && block_inner(A.g, c.x - (int)threadIdx.x, c.y, c.z, L::dim)) {
    step_node<L, PARITY, true>(A, c);
    return;
  }
  if (!c.valid) return;
  step_node<L, PARITY, false>(A, c);
}

// u* = sum_a e_a f_a (Eq. 5) on the flagged nodes only: one thread per node in large
// blocks; threads of unflagged nodes leave after reading their mask word.  The mask
// is cleared before the particle update marks the next step's nodes.
constexpr int kMomBlock = 512;

template <class L, int PARITY>
__global__ void __launch_bounds__(kMomBlock) lbm_moments_kernel(LbmArgs A) {
  const long long n = blockIdx.x * (long long)kMomBlock + threadIdx.x;
  if (n >= A.g.N) return;
  const unsigned nx = (unsigned)A.g.nx;
  const unsigned row = (unsigned)(n / nx);
  const int x = (int)(n - (long long)row * nx);
  const uint32_t word = A.mask[(long long)row * A.g.wpr + (x >> 5)];
  if (!((word >> (x & 31)) & 1u)) return;
  const unsigned uny = (unsigned)A.g.ny;
  const unsigned z = row / uny;
  const int y = (int)(row - z * uny);
  float fa[L::Q], us[3], s1;
  load_pdfs<L, PARITY>(A.g, A.f, x, y, (int)z, n, fa);
  moments<L>(fa, us, s1);
  if (L::dim == 3)
    reinterpret_cast<float4*>(A.ustar)[n] = make_float4(us[0], us[1], us[2], 0.0f);
  else
    reinterpret_cast<float2*>(A.ustar)[n] = make_float2(us[0], us[1]);
}

// p (Eq. 6 with u = u*) and u* (Eq. 5) on every node, as doubles.
template <class L, int PARITY>
__global__ void __launch_bounds__(kLbmBlock) lbm_fields_kernel(LbmArgs A, int cpr, double* p,
                                                              double* u) {
  const NodeCoord c = node_coord(A.g, cpr);
  if (!c.valid) return;
  float fa[L::Q], us[3], s1;
  load_pdfs<L, PARITY>(A.g, A.f, c.x, c.y, c.z, c.n, fa);
  moments<L>(fa, us, s1);
  const float uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
  if (p) p[c.n] = (double)pressure<L>(s1, uu);
  if (u) {
#pragma unroll
    for (int k = 0; k < L::dim; ++k) u[k * A.g.N + c.n] = (double)us[k];
  }
}

// canonical [Q][N] copy of the current PDFs
template <class L, int PARITY>
__global__ void __launch_bounds__(kLbmBlock) lbm_get_kernel(LbmArgs A, int cpr, float* out) {
  const NodeCoord c = node_coord(A.g, cpr);
  if (!c.valid) return;
  float fa[L::Q];
  load_pdfs<L, PARITY>(A.g, A.f, c.x, c.y, c.z, c.n, fa);
#pragma unroll
  for (int a = 0; a < L::Q; ++a) out[a * A.g.N + c.n] = fa[a];
}

// write canonical [Q][N] PDFs into the layout of the current parity
template <class L, int PARITY>
__global__ void __launch_bounds__(kLbmBlock) lbm_put_kernel(LbmArgs A, int cpr,
                                                           const float* in) {
  const NodeCoord c = node_coord(A.g, cpr);
  if (!c.valid) return;
  float fa[L::Q];
#pragma unroll
  for (int a = 0; a < L::Q; ++a) fa[a] = in[a * A.g.N + c.n];
  put_pdfs<L, PARITY>(A.g, A.f, c.x, c.y, c.z, c.n, fa);
}

// equilibrium of Eq. 4 for given p [N] and u [D][N] (doubles), current parity layout
template <class L, int PARITY>
__global__ void __launch_bounds__(kLbmBlock) lbm_equilibrium_kernel(LbmArgs A, int cpr,
                                                                   const double* p,
                                                                   const double* u) {
  const NodeCoord c = node_coord(A.g, cpr);
  if (!c.valid) return;
  float uv[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < L::dim; ++k) uv[k] = (float)u[k * A.g.N + c.n];
  const float pp = (float)p[c.n];
  const float uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
  float fa[L::Q];
  fa[0] = 3.0f * (L::w(0) - 1.0f) * pp - 1.5f * L::w(0) * uu;
#pragma unroll
  for (int a = 1; a < L::Q; ++a) {
    const float eu = L::e(a, 0) * uv[0] + L::e(a, 1) * uv[1] + L::e(a, 2) * uv[2];
    fa[a] = L::w(a) * (3.0f * pp + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
  }
  put_pdfs<L, PARITY>(A.g, A.f, c.x, c.y, c.z, c.n, fa);
}

// ------------------------------------------------------------------ launchers
static dim3 lbm_grid(const Geo& g, int& cpr) {
  cpr = (g.nx + kLbmBlock - 1) / kLbmBlock;
  return dim3((unsigned)((long long)cpr * g.rows));
}

#define IBMLBM_DISPATCH(D, PARITY, KERNEL, ...)                                     \
  do {                                                                              \
    if ((D) == 2) {                                                                 \
      if ((PARITY) == 0) KERNEL<Lat<2>, 0><<<grid, kLbmBlock, 0, s>>>(__VA_ARGS__); \
      else KERNEL<Lat<2>, 1><<<grid, kLbmBlock, 0, s>>>(__VA_ARGS__);               \
    } else {                                                                        \
      if ((PARITY) == 0) KERNEL<Lat<3>, 0><<<grid, kLbmBlock, 0, s>>>(__VA_ARGS__); \
      else KERNEL<Lat<3>, 1><<<grid, kLbmBlock, 0, s>>>(__VA_ARGS__);               \
    }                                                                               \
  } while (0)

cudaError_t launch_lbm_step(const LbmArgs& A, int D, int parity, cudaStream_t s) {
  int cpr;
  const dim3 grid = lbm_grid(A.g, cpr);
  IBMLBM_DISPATCH(D, parity, lbm_step_kernel, A, cpr);
  return cudaGetLastError();
}

cudaError_t launch_lbm_moments(const LbmArgs& A, int D, int parity, cudaStream_t s) {
  const dim3 grid((unsigned)((A.g.N + kMomBlock - 1) / kMomBlock));
  if (D == 2) {
    if (parity == 0) lbm_moments_kernel<Lat<2>, 0><<<grid, kMomBlock, 0, s>>>(A);
    else lbm_moments_kernel<Lat<2>, 1><<<grid, kMomBlock, 0, s>>>(A);
  } else {
    if (parity == 0) lbm_moments_kernel<Lat<3>, 0><<<grid, kMomBlock, 0, s>>>(A);
    else lbm_moments_kernel<Lat<3>, 1><<<grid, kMomBlock, 0, s>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_lbm_fields(const LbmArgs& A, int D, int parity, double* p, double* u,
                              cudaStream_t s) {
  int cpr;
  const dim3 grid = lbm_grid(A.g, cpr);
  IBMLBM_DISPATCH(D, parity, lbm_fields_kernel, A, cpr, p, u);
  return cudaGetLastError();
}

cudaError_t launch_lbm_get(const LbmArgs& A, int D, int parity, float* out, cudaStream_t s) {
  int cpr;
  const dim3 grid = lbm_grid(A.g, cpr);
  IBMLBM_DISPATCH(D, parity, lbm_get_kernel, A, cpr, out);
  return cudaGetLastError();
}

cudaError_t launch_lbm_put(const LbmArgs& A, int D, int parity, const float* in,
                           cudaStream_t s) {
  int cpr;
  const dim3 grid = lbm_grid(A.g, cpr);
  IBMLBM_DISPATCH(D, parity, lbm_put_kernel, A, cpr, in);
  return cudaGetLastError();
}

cudaError_t launch_lbm_equilibrium(const LbmArgs& A, int D, int parity, const double* p,
                                   const double* u, cudaStream_t s) {
  int cpr;
  const dim3 grid = lbm_grid(A.g, cpr);
  IBMLBM_DISPATCH(D, parity, lbm_equilibrium_kernel, A, cpr, p, u);
  return cudaGetLastError();
}

}  // namespace ibmlbm
