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
#include <algorithm>

#include "common.cuh"
#include "launch.h"
#include "pdf_access.cuh"

namespace ibmlbm {

constexpr int kLbmBlock = 128;

// inverse of load_pdfs: slot of f_a(x) under the layout of the given parity
template <class L, int PARITY, int ST>
__device__ __forceinline__ void put_pdfs(const Geo& g, void* __restrict__ f, int x, int y,
                                         int z, long long n, const float (&fa)[L::Q]) {
  const long long N = g.Np;  // plane stride
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    long long idx = a * N + n, src;
    if (PARITY == 1 && a != 0 && neighbour<L>(g, a, 1, x, y, z, n, src)) idx = opp<L>(a) * N + src;
    if (IBMLBM_CHK(idx, L::Q * N)) pdf_store<L, ST>(f, idx, a, fa[a]);
  }
}

// post-collision store of the given parity (after which the opposite parity holds);
// RAW: fa holds the stored variable (h_a for the 16-bit storages)
template <class L, int PARITY, int ST, bool INNER = false, bool RAW = false>
__device__ __forceinline__ void store_post(const Geo& g, void* __restrict__ f, int x, int y,
                                           int z, long long n, const float (&fa)[L::Q]) {
  const long long N = g.Np;  // plane stride
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    long long idx;
    if (a == 0) {
      idx = n;
    } else if (PARITY == 0) {
      idx = opp<L>(a) * N + n;
    } else if (INNER) {
      idx = a * N + n + inner_offset<L>(g, a, -1);
    } else {
      long long dst;
      idx = neighbour<L>(g, a, -1, x, y, z, n, dst) ? a * N + dst : opp<L>(a) * N + n;
    }
    if (IBMLBM_CHK(idx, L::Q * N)) pdf_store<L, ST, RAW>(f, idx, a, fa[a]);
  }
}

// Eq. 6: p = cs^2/(1 - w0) (sum_{a>=1} f_a - rho0 w0 |u|^2 / (2 cs^2))
template <class L>
__device__ __forceinline__ float pressure(float s1, float uu) {
  constexpr float w0 = L::w(0);
  return s1 * (1.0f / (3.0f * (1.0f - w0))) - uu * (w0 / (2.0f * (1.0f - w0)));
}

// Sums over the moving populations of a node, taken per opposite pair (a, a + H):
// s_a = v_a + v_{a+H}, d_a = v_a - v_{a+H}.  With c = 1 (v = f) or c = w (v = h = f / w):
// s1 = sum_{a>=1} c_a v_a (Eq. 6) and u*_k = sum_a e_ak c_a v_a (Eq. 5).  The pairs of
// axis directions and of diagonal ones share a weight each.
template <class L, bool HV>
__device__ __forceinline__ void pair_moments(const float (&s)[L::H], const float (&d)[L::H], float& s1,
                                             float (&us)[3]);

template <>
__device__ __forceinline__ void pair_moments<Lat<2>, false>(const float (&s)[4], const float (&d)[4],
                                                            float& s1, float (&us)[3]) {
  // pairs: 1 = (1, 0), 2 = (1, 1), 3 = (0, 1), 4 = (-1, 1)
  static_assert(Lat<2>::e(2, 0) == 1 && Lat<2>::e(2, 1) == 1 && Lat<2>::e(4, 0) == -1 && Lat<2>::e(4, 1) == 1, "");
  s1 = (s[0] + s[2]) + (s[1] + s[3]);
  us[0] = d[0] + (d[1] - d[3]);
  us[1] = d[2] + (d[1] + d[3]);
  us[2] = 0.0f;
}

template <>
__device__ __forceinline__ void pair_moments<Lat<2>, true>(const float (&s)[4], const float (&d)[4],
                                                           float& s1, float (&us)[3]) {
  constexpr float wA = Lat<2>::w(1), wD = Lat<2>::w(2);
  s1 = fmaf(wD, s[1] + s[3], wA * (s[0] + s[2]));
  us[0] = fmaf(wD, d[1] - d[3], wA * d[0]);
  us[1] = fmaf(wD, d[1] + d[3], wA * d[2]);
  us[2] = 0.0f;
}

// D3Q19 pairs: 1 = x, 2 = y, 3 = z; 4 = (1, 1, 0), 5 = (-1, 1, 0), 6 = (0, 1, 1),
// 7 = (0, -1, 1), 8 = (1, 0, 1), 9 = (-1, 0, 1)
static_assert(Lat<3>::e(5, 0) == -1 && Lat<3>::e(5, 1) == 1 && Lat<3>::e(7, 1) == -1 && Lat<3>::e(7, 2) == 1 &&
                  Lat<3>::e(9, 0) == -1 && Lat<3>::e(9, 2) == 1 && Lat<3>::e(6, 1) == 1 && Lat<3>::e(8, 2) == 1,
              "D3Q19 pair order");

template <>
__device__ __forceinline__ void pair_moments<Lat<3>, false>(const float (&s)[9], const float (&d)[9],
                                                            float& s1, float (&us)[3]) {
  s1 = ((s[0] + s[1]) + s[2]) + (((s[3] + s[4]) + (s[5] + s[6])) + (s[7] + s[8]));
  us[0] = d[0] + ((d[3] - d[4]) + (d[7] - d[8]));
  us[1] = d[1] + ((d[3] + d[4]) + (d[5] - d[6]));
  us[2] = d[2] + ((d[5] + d[6]) + (d[7] + d[8]));
}

template <>
__device__ __forceinline__ void pair_moments<Lat<3>, true>(const float (&s)[9], const float (&d)[9],
                                                           float& s1, float (&us)[3]) {
  constexpr float wA = Lat<3>::w(1), wD = Lat<3>::w(4);
  s1 = fmaf(wD, ((s[3] + s[4]) + (s[5] + s[6])) + (s[7] + s[8]), wA * ((s[0] + s[1]) + s[2]));
  us[0] = fmaf(wD, (d[3] - d[4]) + (d[7] - d[8]), wA * d[0]);
  us[1] = fmaf(wD, (d[3] + d[4]) + (d[5] - d[6]), wA * d[1]);
  us[2] = fmaf(wD, (d[5] + d[6]) + (d[7] + d[8]), wA * d[2]);
}

// Eq. 4 equilibrium, Eq. 8 forcing term and the relaxation of Eq. 41-42 on one node,
// per opposite pair (a, b = a + H) from one shared even part (Eq. 38, Eq. 40).  With
// e = e_a: v_eq = c (3 p - 1.5 u.u + 4.5 (e.u)^2 +- 3 e.u) and F_a = c k (9 (e.u)(e.F) -
// 3 u.F +- 3 e.F), k = 1 - omega / 2, so the update is
//   v_a = (1 - omega) v_a + E + O,  v_b = (1 - omega) v_b + E - O,
//   E = c (omega (3 p - 1.5 u.u) - 3 k u.F) + (e.u) c (4.5 omega (e.u) + 9 k (e.F)),
//   O = c (3 omega (e.u) + 3 k (e.F)),
// c = w_a for v = f and 1 for the 16-bit storages' v = h = f / w.  u is the
// force-corrected velocity of Eq. 7 and p follows Eq. 6.
template <class L, bool HV>
__device__ __forceinline__ void collide_pairs(float (&v)[L::Q], const float (&F)[3], float omega,
                                              float kforce) {
  float s[L::H], d[L::H];
#pragma unroll
  for (int a = 1; a <= L::H; ++a) {
    s[a - 1] = v[a] + v[a + L::H];
    d[a - 1] = v[a] - v[a + L::H];
  }
  float s1, us[3];
  pair_moments<L, HV>(s, d, s1, us);
  float u[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) u[k] = (k < L::dim) ? fmaf(0.5f, F[k], us[k]) : 0.0f;  // Eq. 7
  float uu, uF;
  if constexpr (L::dim == 2) {
    uu = fmaf(u[0], u[0], u[1] * u[1]);
    uF = fmaf(u[0], F[0], u[1] * F[1]);
  } else {
    uu = fmaf(u[0], u[0], fmaf(u[1], u[1], u[2] * u[2]));
    uF = fmaf(u[0], F[0], fmaf(u[1], F[1], u[2] * F[2]));
  }
  const float p = pressure<L>(s1, uu);
  const float om1 = 1.0f - omega, k3uF = 3.0f * kforce * uF;
  constexpr float w0 = L::w(0);
  if constexpr (HV) {
    const float eq0 = fmaf(3.0f * (1.0f - 1.0f / w0), p, -1.5f * uu);
    v[0] = fmaf(om1, v[0], fmaf(omega, eq0, -k3uF));
  } else {
    const float eq0 = fmaf(3.0f * (w0 - 1.0f), p, -1.5f * w0 * uu);
    v[0] = fmaf(om1, v[0], fmaf(omega, eq0, -w0 * k3uF));
  }
  const float A0 = fmaf(omega, fmaf(3.0f, p, -1.5f * uu), -k3uF);
  const float w45 = 4.5f * omega, k9 = 9.0f * kforce, w3 = 3.0f * omega, k3 = 3.0f * kforce;
#pragma unroll
  for (int a = 1; a <= L::H; ++a) {
    float eu = 0.0f, eF = 0.0f;
    bool any = false;
#pragma unroll
    for (int k = 0; k < L::dim; ++k) {
      const int e = L::e(a, k);
      if (e == 0) continue;
      const float uk = e > 0 ? u[k] : -u[k], Fk = e > 0 ? F[k] : -F[k];
      eu = any ? eu + uk : uk;
      eF = any ? eF + Fk : Fk;
      any = true;
    }
    constexpr float c0 = 1.0f;
    const float c = HV ? c0 : L::w(a);
    const float t = fmaf(c * k9, eF, (c * w45) * eu);
    const float E = fmaf(eu, t, c * A0);
    const float O = fmaf(c * w3, eu, (c * k3) * eF);
    const int b = a + L::H;
    v[a] = fmaf(om1, v[a], E + O);
    v[b] = fmaf(om1, v[b], E - O);
  }
}

template <class L>
__device__ __forceinline__ void collide(float (&f)[L::Q], const float (&F)[3], float omega,
                                        float kforce) {
  collide_pairs<L, false>(f, F, omega, kforce);
}

// The same collision on the stored variable h_a = f_a / w_a (16-bit storages): the
// moments weigh each h_a by w_a, and the equilibrium and force terms are divided by
// w_a, which removes w_a from them (Eq. 4, 8).
template <class L>
__device__ __forceinline__ void collide_h(float (&h)[L::Q], const float (&F)[3], float omega,
                                          float kforce) {
  collide_pairs<L, true>(h, F, omega, kforce);
}

// Eq. 4 equilibrium of every direction at (p, u)
template <class L>
__device__ __forceinline__ void equilibrium(float p, const float (&u)[3], float (&feq)[L::Q]) {
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  constexpr float w0 = L::w(0);
  feq[0] = 3.0f * (w0 - 1.0f) * p - 1.5f * w0 * uu;
#pragma unroll
  for (int a = 1; a <= L::H; ++a) {
    const float w = L::w(a);
    float eu = 0.0f;
#pragma unroll
    for (int k = 0; k < L::dim; ++k) {
      if (L::e(a, k) == 1) eu += u[k];
      if (L::e(a, k) == -1) eu -= u[k];
    }
    const float even = w * (3.0f * p + 4.5f * eu * eu - 1.5f * uu), odd = 3.0f * w * eu;
    feq[a] = even + odd;
    feq[a + L::H] = even - odd;
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

// IB force of one node.  2D [N][2], read for every node together with the PDFs (one
// memory latency; a read that first waits for the node mask was measured slower), and
// not at all in a run without particles (A.fib null); 3D [N][4], read only on nodes the
// particle update marked (where it can be non-zero)
template <class L>
__device__ __forceinline__ void ib_force(const LbmArgs& A, long long row, int x, long long n,
                                         float (&fv)[3]) {
  fv[0] = fv[1] = fv[2] = 0.0f;
  if (L::dim == 2) {
    if (!A.fib || !IBMLBM_CHK(n, A.g.N)) return;
    const float2 v = reinterpret_cast<const float2*>(A.fib)[n];
    fv[0] = v.x;
    fv[1] = v.y;
  } else if (IBMLBM_CHK(row * A.g.wpr + (x >> 5), (long long)A.g.rows * A.g.wpr) &&
             ((A.mask[row * A.g.wpr + (x >> 5)] >> (x & 31)) & 1u) && IBMLBM_CHK(n, A.g.N)) {
    const float4 v = reinterpret_cast<const float4*>(A.fib)[n];
    fv[0] = v.x;
    fv[1] = v.y;
    fv[2] = v.z;
  }
}

template <class L>
__device__ __forceinline__ void ib_force_clear(const LbmArgs& A, long long n, const float (&fv)[3]) {
  if (L::dim == 2) {
    if (fv[0] != 0.0f || fv[1] != 0.0f) reinterpret_cast<float2*>(A.fib)[n] = make_float2(0.0f, 0.0f);
  } else if (fv[0] != 0.0f || fv[1] != 0.0f || fv[2] != 0.0f) {
    reinterpret_cast<float4*>(A.fib)[n] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

// one node with the general addressing (walls and periodic wraps per direction)
template <class L, int PARITY, int ST>
__device__ __forceinline__ void step_node(const LbmArgs& A, long long row, int x, int y, int z,
                                          long long n) {
  constexpr bool H = ST != STORE_F32;  // 16-bit storages collide the stored h = f / w
  float fa[L::Q], fv[3];
  load_pdfs<L, PARITY, ST, false, H>(A.g, A.f, x, y, z, n, fa);
  ib_force<L>(A, row, x, n, fv);
  float F[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) F[k] = A.body[k] + fv[k];
  if constexpr (H) collide_h<L>(fa, F, A.omega, A.kforce);
  else collide<L>(fa, F, A.omega, A.kforce);
  store_post<L, PARITY, ST, false, H>(A.g, A.f, x, y, z, n, fa);
  ib_force_clear<L>(A, n, fv);
}

// In an odd step, rows whose nodes have neighbours across a y or z domain face (the
// first and last node of every other row also do, across an x face)
template <class L>
__device__ __forceinline__ bool odd_edge_row(const Geo& g, int y, int z) {
  return y == 0 || y == g.ny - 1 || (L::dim == 3 && (z == 0 || z == g.nz - 1));
}

// One full time step (Eq. 1, 4-8, 17-18) of the K adjacent nodes x0 .. x0 + K - 1 of a
// row: read the nodes' PDFs (AA parity) and IB force, collide, store in place.  All K
// nodes' loads are issued before any store, so a thread keeps K nodes' bytes in flight
// (K = 2 suits the 16-bit storages, whose requests are half as large).  In an odd step
// the nodes whose neighbourhood crosses a domain face (rows on a y or z face, the first
// and last node of a row) are left to lbm_step_edge_kernel, so every node here uses
// fixed neighbour offsets; the AA pattern makes the nodes independent of each other.
// The even step is local everywhere.
template <class L, int PARITY, int ST, int K>
__device__ __forceinline__ void step_row_nodes(const LbmArgs& A, long long row, int y, int z, int x0) {
  const Geo& g = A.g;
  if (PARITY == 1 && odd_edge_row<L>(g, y, z)) return;
  float fa[K][L::Q], fv[K][3];
  bool act[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int x = x0 + k;
    act[k] = x < g.nx && !(PARITY == 1 && (x == 0 || x == g.nx - 1));
    if (!act[k]) continue;
    const long long n = (long long)x + (long long)g.nx * row;
    load_pdfs<L, PARITY, ST, PARITY == 1, (ST != STORE_F32)>(g, A.f, x, y, z, n, fa[k]);
    ib_force<L>(A, row, x, n, fv[k]);  // with the PDFs: one memory latency
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!act[k]) continue;
    const int x = x0 + k;
    const long long n = (long long)x + (long long)g.nx * row;
    float F[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) F[c] = A.body[c] + fv[k][c];
    if constexpr (ST != STORE_F32) collide_h<L>(fa[k], F, A.omega, A.kforce);  // on h = f / w
    else collide<L>(fa[k], F, A.omega, A.kforce);
    store_post<L, PARITY, ST, PARITY == 1, (ST != STORE_F32)>(g, A.f, x, y, z, n, fa[k]);
    ib_force_clear<L>(A, n, fv[k]);
  }
}

// Row tiles: a block of kLbmBlock threads takes K * kLbmBlock consecutive nodes of one
// row (spr blocks per row).  Blocks per SM the registers must allow: D2Q9 10 (48
// registers a thread); D3Q19 7 (72 registers, a few bytes spilled: more PDF loads in
// flight than at the 80 registers it takes unbounded).
template <class L, int PARITY, int ST, int K>
__device__ __forceinline__ void step_tile_body(const LbmArgs& A, int spr, unsigned blk) {
  const Geo& g = A.g;
  const unsigned b = blk, uspr = (unsigned)spr, uny = (unsigned)g.ny;
  const unsigned row = b / uspr, seg = b - row * uspr;
  const unsigned uz = row / uny;
  step_row_nodes<L, PARITY, ST, K>(A, row, (int)(row - uz * uny), (int)uz,
                                   K * ((int)seg * kLbmBlock + (int)threadIdx.x));
}

template <class L, int PARITY, int ST, int K, bool FUSED>
__global__ void __launch_bounds__(kLbmBlock, L::dim == 3 ? 7 : 10) lbm_step_kernel(LbmArgs A0, int spr0, Fuse FU) {
  IBMLBM_BIND(FUSED, LbmArgs, A, A0, FU, blk);
  const int spr = FUSED ? (A.g.nx + K * kLbmBlock - 1) / (K * kLbmBlock) : spr0;
  step_tile_body<L, PARITY, ST, K>(A, spr, blk);
}

// ------------------------------------------------------------ vector row kernel
// The same step with K consecutive nodes per thread and each direction's K stored
// values moved as one vector (K x 2 bytes for the 16-bit storages, K x 4 for FP32):
// one load and one store instruction per direction and thread instead of K.  A warp
// takes 32 K consecutive nodes of one row; rows must hold a multiple of K nodes, so
// every vector is aligned (the PDF planes are 64 elements apart).  Every node of the
// lattice is stepped here, in both parities (no edge kernel):
//   - the y / z part of a neighbour is the same for the whole warp: a row beyond a
//     wall makes the direction bounce back (the node's own slot, no shift), a
//     periodic face wraps the row;
//   - an odd step's direction with e_x = +1 reads f_a(x) at x - 1, one element below
//     the thread's aligned vector: the thread loads its aligned vector and takes the
//     element below from the lane before (a warp shuffle); lane 0 loads it alone, and
//     at the row start it is the wrapped node or the bounce-back slot.  e_x = -1 is the
//     mirror image (the lane after; lane 31 and the row end alone);
//   - the post-collision values of an e_x != 0 direction go one element off as well:
//     each lane shifts its vector by one through the shuffle and stores it aligned,
//     except the one element a lane cannot know (lane 0 or the row start for e_x = +1,
//     lane 31 or the row end for e_x = -1), which its owner stores singly.
constexpr int kVecWarps = 4;

template <int ST>
struct Elem {
  static constexpr int bytes = ST == STORE_F32 ? 4 : 2;
};

// K elements of one direction in 32-bit words (two 16-bit elements per word)
template <int ST, int K>
struct PVec {
  static constexpr int EB = Elem<ST>::bytes, NW = K * EB / 4;
  uint32_t w[NW];
};

template <int ST, int K>
__device__ __forceinline__ void pvec_load(PVec<ST, K>& v, const void* base, long long idx) {
  constexpr int NW = PVec<ST, K>::NW;
  const char* p = static_cast<const char*>(base) + idx * Elem<ST>::bytes;
  if constexpr (NW == 4) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    v.w[0] = t.x, v.w[1] = t.y, v.w[2] = t.z, v.w[3] = t.w;
  } else if constexpr (NW == 2) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    v.w[0] = t.x, v.w[1] = t.y;
  } else {
    v.w[0] = *reinterpret_cast<const uint32_t*>(p);
  }
}

template <int ST, int K>
__device__ __forceinline__ void pvec_store(const PVec<ST, K>& v, void* base, long long idx) {
  constexpr int NW = PVec<ST, K>::NW;
  char* p = static_cast<char*>(base) + idx * Elem<ST>::bytes;
  if constexpr (NW == 4) *reinterpret_cast<uint4*>(p) = make_uint4(v.w[0], v.w[1], v.w[2], v.w[3]);
  else if constexpr (NW == 2) *reinterpret_cast<uint2*>(p) = make_uint2(v.w[0], v.w[1]);
  else *reinterpret_cast<uint32_t*>(p) = v.w[0];
}

// raw bits of element j (low bits of the result)
template <int ST, int K>
__device__ __forceinline__ uint32_t pvec_get(const PVec<ST, K>& v, int j) {
  if constexpr (Elem<ST>::bytes == 4) return v.w[j];
  else return (j & 1) ? (v.w[j >> 1] >> 16) : (v.w[j >> 1] & 0xffffu);
}

// element j -> j + 1, element 0 <- below
template <int ST, int K>
__device__ __forceinline__ PVec<ST, K> pvec_up(const PVec<ST, K>& v, uint32_t below) {
  PVec<ST, K> r;
  constexpr int NW = PVec<ST, K>::NW;
  if constexpr (Elem<ST>::bytes == 4) {
    r.w[0] = below;
#pragma unroll
    for (int i = 1; i < NW; ++i) r.w[i] = v.w[i - 1];
  } else {
    r.w[0] = __byte_perm(below, v.w[0], 0x5410);
#pragma unroll
    for (int i = 1; i < NW; ++i) r.w[i] = __byte_perm(v.w[i - 1], v.w[i], 0x5432);
  }
  return r;
}

// element j -> j - 1, element K - 1 <- above
template <int ST, int K>
__device__ __forceinline__ PVec<ST, K> pvec_down(const PVec<ST, K>& v, uint32_t above) {
  PVec<ST, K> r;
  constexpr int NW = PVec<ST, K>::NW;
  if constexpr (Elem<ST>::bytes == 4) {
#pragma unroll
    for (int i = 0; i + 1 < NW; ++i) r.w[i] = v.w[i + 1];
    r.w[NW - 1] = above;
  } else {
#pragma unroll
    for (int i = 0; i + 1 < NW; ++i) r.w[i] = __byte_perm(v.w[i], v.w[i + 1], 0x5432);
    r.w[NW - 1] = __byte_perm(v.w[NW - 1], above, 0x5432);
  }
  return r;
}

template <int ST>
__device__ __forceinline__ uint32_t elem_load(const void* base, long long idx) {
  if constexpr (Elem<ST>::bytes == 4) return static_cast<const uint32_t*>(base)[idx];
  else return static_cast<const uint16_t*>(base)[idx];
}

template <int ST>
__device__ __forceinline__ void elem_store(void* base, long long idx, uint32_t bits) {
  if constexpr (Elem<ST>::bytes == 4) static_cast<uint32_t*>(base)[idx] = bits;
  else static_cast<uint16_t*>(base)[idx] = (uint16_t)bits;
}

// v without its element 0 (first) or without element K - 1, in aligned pieces
template <int ST, int K>
__device__ __forceinline__ void pvec_store_skip(const PVec<ST, K>& v, void* base, long long idx, bool first) {
  constexpr int NW = PVec<ST, K>::NW;
  constexpr bool B2 = Elem<ST>::bytes == 2;
  static_assert(NW == 1 || NW == 2 || NW == 4, "vector width");
  char* p = static_cast<char*>(base) + idx * Elem<ST>::bytes;
  uint32_t* w32 = reinterpret_cast<uint32_t*>(p);
  if (first) {
    if constexpr (B2) reinterpret_cast<uint16_t*>(p)[1] = (uint16_t)(v.w[0] >> 16);
    if constexpr (NW >= 2) w32[1] = v.w[1];
    if constexpr (NW == 4) *reinterpret_cast<uint2*>(p + 8) = make_uint2(v.w[2], v.w[3]);
  } else {
    if constexpr (NW == 4) {
      *reinterpret_cast<uint2*>(p) = make_uint2(v.w[0], v.w[1]);
      w32[2] = v.w[2];
    } else if constexpr (NW == 2) {
      w32[0] = v.w[0];
    }
    if constexpr (B2) reinterpret_cast<uint16_t*>(p)[K - 2] = (uint16_t)(v.w[NW - 1] & 0xffffu);
  }
}

// the row (y + s e_y, z + s e_z) with periodic wraps, or -1 beyond a wall
template <class L>
__device__ __forceinline__ long long nb_row(const Geo& g, int a, int s, int y, int z) {
  int ty = y + s * L::e(a, 1), tz = z + s * L::e(a, 2);
  if (ty < 0 || ty >= g.ny) {
    if (!g.per[1]) return -1;
    ty += ty < 0 ? g.ny : -g.ny;
  }
  if (L::dim == 3 && (tz < 0 || tz >= g.nz)) {
    if (!g.per[2]) return -1;
    tz += tz < 0 ? g.nz : -g.nz;
  }
  return (long long)ty + (long long)g.ny * tz;
}

// nodes 2i and 2i + 1 of a word (16-bit storages) or node i (FP32)
template <int ST>
__device__ __forceinline__ void word_values(uint32_t w, float& lo, float& hi) {
  if constexpr (ST == STORE_F16) {
    const float2 t = __half22float2(*reinterpret_cast<const __half2*>(&w));
    lo = t.x, hi = t.y;
  } else if constexpr (ST == STORE_BF16) {
    lo = __uint_as_float(w << 16), hi = __uint_as_float(w & 0xffff0000u);
  } else {
    lo = __uint_as_float(w), hi = 0.0f;
  }
}

template <int ST>
__device__ __forceinline__ uint32_t word_bits(float lo, float hi) {
  if constexpr (ST == STORE_F16) {
    const __half2 t = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&t);
  } else if constexpr (ST == STORE_BF16) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&t);
  } else {
    return __float_as_uint(lo);
  }
}

template <class L, int PARITY, int ST, int K>
__global__ void __launch_bounds__(32 * kVecWarps) lbm_step_vec_kernel(LbmArgs A, int spr) {
  using V = PVec<ST, K>;
  constexpr int NW = V::NW, EPW = 4 / Elem<ST>::bytes;  // words, elements per word
  constexpr bool B2 = Elem<ST>::bytes == 2;
  constexpr unsigned FULL = 0xffffffffu;
  const Geo& g = A.g;
  const int lane = (int)(threadIdx.x & 31);
  const unsigned wg = blockIdx.x * (unsigned)kVecWarps + (threadIdx.x >> 5);
  const unsigned row = wg / (unsigned)spr, seg = wg - row * (unsigned)spr;
  if (row >= (unsigned)g.rows) return;  // whole warp
  const unsigned uz = row / (unsigned)g.ny;
  const int y = (int)(row - uz * (unsigned)g.ny), z = (int)uz;
  const int x0 = ((int)seg * 32 + lane) * K;
  const bool in = x0 < g.nx, first = x0 == 0, last = x0 + K == g.nx;
  const long long n0 = (long long)x0 + (long long)g.nx * row, N = g.Np, QN = L::Q * N;

  // loads: the PDFs of the K nodes under the layout of this parity (zero on lanes past
  // the row end, which only take part in the shuffles).  Every load, the boundary
  // elements of lanes 0 and 31 and of the row ends included, is issued before the
  // first shuffle, so a thread waits for memory once.
  V h[L::Q];
  uint32_t edge[L::Q];  // odd step, e_x != 0: the element the shuffle cannot supply
  bool shifted[L::Q];   // odd step: direction read through a shifted row (not bounced)
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
#pragma unroll
    for (int i = 0; i < NW; ++i) h[a].w[i] = 0u;
    edge[a] = 0u;
    shifted[a] = false;
    if (PARITY == 0 || a == 0) {
      if (in && IBMLBM_CHK(a * N + n0 + K - 1, QN)) pvec_load<ST, K>(h[a], A.f, a * N + n0);
      continue;
    }
    const long long rs = nb_row<L>(g, a, -1, y, z);  // row of the source x - e_a
    if (rs < 0) {  // beyond a y / z wall: bounce-back, the node's own slot
      if (in && IBMLBM_CHK(a * N + n0 + K - 1, QN)) pvec_load<ST, K>(h[a], A.f, a * N + n0);
      continue;
    }
    shifted[a] = true;
    const long long rb = opp<L>(a) * N + (long long)g.nx * rs, src = rb + x0;
    if (in && IBMLBM_CHK(src, QN) && IBMLBM_CHK(src + K - 1, QN)) pvec_load<ST, K>(h[a], A.f, src);
    const int ex = L::e(a, 0);
    if (ex == 1 && in && (first || lane == 0)) {  // f_a of node x0 sits at x0 - 1
      const long long e = !first ? src - 1 : g.per[0] ? rb + g.nx - 1 : a * N + n0;
      if (IBMLBM_CHK(e, QN)) edge[a] = elem_load<ST>(A.f, e);
    }
    if (ex == -1 && in && (last || lane == 31)) {  // f_a of node x0 + K - 1 sits at x0 + K
      const long long e = !last ? src + K : g.per[0] ? rb : a * N + n0 + K - 1;
      if (IBMLBM_CHK(e, QN)) edge[a] = elem_load<ST>(A.f, e);
    }
  }
  if (PARITY == 1) {
#pragma unroll
    for (int a = 1; a < L::Q; ++a) {
      const int ex = L::e(a, 0);
      if (ex == 0 || !shifted[a]) continue;  // uniform over the warp
      if (ex == 1) {
        const uint32_t lw = __shfl_up_sync(FULL, h[a].w[NW - 1], 1);
        const uint32_t below = (in && (first || lane == 0)) ? edge[a] : (B2 ? (lw >> 16) : lw);
        h[a] = pvec_up<ST, K>(h[a], below);
      } else {
        const uint32_t fw = __shfl_down_sync(FULL, h[a].w[0], 1);
        const uint32_t above = (in && (last || lane == 31)) ? edge[a] : (B2 ? (fw & 0xffffu) : fw);
        h[a] = pvec_down<ST, K>(h[a], above);
      }
    }
  }

  // IB force (2D every node of a run with particles, 3D the marked nodes)
  float fv[K][3];
#pragma unroll
  for (int j = 0; j < K; ++j) fv[j][0] = fv[j][1] = fv[j][2] = 0.0f;
  if (L::dim == 2) {
    if (A.fib && in && IBMLBM_CHK(n0 + K - 1, g.N)) {
      const float4* fb = reinterpret_cast<const float4*>(A.fib) + (n0 >> 1);
#pragma unroll
      for (int j = 0; j < K; j += 2) {
        const float4 t = fb[j >> 1];
        fv[j][0] = t.x, fv[j][1] = t.y, fv[j + 1][0] = t.z, fv[j + 1][1] = t.w;
      }
    }
  } else if (in && IBMLBM_CHK(row * g.wpr + (x0 >> 5), (long long)g.rows * g.wpr) && IBMLBM_CHK(n0 + K - 1, g.N)) {
    const uint32_t bits = (A.mask[row * g.wpr + (x0 >> 5)] >> (x0 & 31)) & ((1u << K) - 1);
    if (bits) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        if (!((bits >> j) & 1u)) continue;
        const float4 t = reinterpret_cast<const float4*>(A.fib)[n0 + j];
        fv[j][0] = t.x, fv[j][1] = t.y, fv[j][2] = t.z;
      }
    }
  }

  // collide in place, the EPW nodes of a word together (one conversion per word)
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    float fa[EPW][L::Q];
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
      float lo, hi;
      word_values<ST>(h[a].w[i], lo, hi);
      fa[0][a] = lo;
      if (EPW == 2) fa[EPW - 1][a] = hi;
    }
#pragma unroll
    for (int e = 0; e < EPW; ++e) {
      const int j = i * EPW + e;
      float F[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] = A.body[c] + fv[j][c];
      if constexpr (ST != STORE_F32) collide_h<L>(fa[e], F, A.omega, A.kforce);
      else collide<L>(fa[e], F, A.omega, A.kforce);
    }
#pragma unroll
    for (int a = 0; a < L::Q; ++a) h[a].w[i] = word_bits<ST>(fa[0][a], fa[EPW - 1][a]);
  }

  // stores
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    if (PARITY == 0 || a == 0) {  // even step: f*_a to a[opp(a)][x] (local)
      if (in && IBMLBM_CHK(opp<L>(a) * N + n0 + K - 1, QN)) pvec_store<ST, K>(h[a], A.f, opp<L>(a) * N + n0);
      continue;
    }
    const long long rt = nb_row<L>(g, a, 1, y, z);  // row of the target x + e_a
    if (rt < 0) {  // beyond a y / z wall: bounce-back into a[opp(a)][x]
      if (in && IBMLBM_CHK(opp<L>(a) * N + n0 + K - 1, QN)) pvec_store<ST, K>(h[a], A.f, opp<L>(a) * N + n0);
      continue;
    }
    const long long rb = a * N + (long long)g.nx * rt, dst = rb + x0;
    const bool ok = in && IBMLBM_CHK(dst, QN) && IBMLBM_CHK(dst + K - 1, QN);  // (shuffles stay warp-wide)
    const int ex = L::e(a, 0);
    if (ex == 0) {
      if (ok) pvec_store<ST, K>(h[a], A.f, dst);
    } else if (ex == 1) {  // f*_a(x) goes to x + 1: element j holds node j - 1
      const uint32_t lw = __shfl_up_sync(FULL, h[a].w[NW - 1], 1);
      const V sh = pvec_up<ST, K>(h[a], B2 ? (lw >> 16) : lw);
      if (ok) {
        if (lane == 0) pvec_store_skip<ST, K>(sh, A.f, dst, true);
        else pvec_store<ST, K>(sh, A.f, dst);
        const uint32_t mine = pvec_get<ST, K>(h[a], K - 1);  // node x0 + K - 1
        const long long e = last ? (g.per[0] ? rb : opp<L>(a) * N + n0 + K - 1) : dst + K;
        if ((last || lane == 31) && IBMLBM_CHK(e, QN)) elem_store<ST>(A.f, e, mine);
      }
    } else {  // f*_a(x) goes to x - 1: element j holds node j + 1
      const uint32_t fw = __shfl_down_sync(FULL, h[a].w[0], 1);
      const V sh = pvec_down<ST, K>(h[a], B2 ? (fw & 0xffffu) : fw);
      if (ok) {
        if (lane == 31 || last) pvec_store_skip<ST, K>(sh, A.f, dst, false);
        else pvec_store<ST, K>(sh, A.f, dst);
        const uint32_t mine = pvec_get<ST, K>(h[a], 0);  // node x0
        const long long e = first ? (g.per[0] ? rb + g.nx - 1 : opp<L>(a) * N + n0) : dst - 1;
        if ((first || lane == 0) && IBMLBM_CHK(e, QN)) elem_store<ST>(A.f, e, mine);
      }
    }
  }

  // the IB force is cleared where it was not zero
  if (!in || !IBMLBM_CHK(n0 + K - 1, g.N)) return;
  if (L::dim == 2) {
    if (A.fib) {
      float4* fb = reinterpret_cast<float4*>(A.fib) + (n0 >> 1);
#pragma unroll
      for (int j = 0; j < K; j += 2)
        if (fv[j][0] != 0.0f || fv[j][1] != 0.0f || fv[j + 1][0] != 0.0f || fv[j + 1][1] != 0.0f)
          fb[j >> 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (fv[j][0] != 0.0f || fv[j][1] != 0.0f || fv[j][2] != 0.0f)
        reinterpret_cast<float4*>(A.fib)[n0 + j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

// Warp tiles over the members of a 2D batch: the rows of a member are cut into
// segments of 32 K nodes, one per warp, and a tile is W consecutive segments of the
// member's row-major segment sequence (so a tile can span short rows).  Tile t of the
// launch belongs to the member m with first[m] <= t < first[m + 1].  PERSIST: a grid
// of as many blocks as fit on the GPU at once walks the tiles with a grid stride;
// otherwise one block per tile.
template <int PARITY, int ST, int K, int W, bool PERSIST>
__global__ void __launch_bounds__(32 * W) lbm_step_tiles_kernel(const LbmArgs* __restrict__ args,
                                                                const int* __restrict__ first, int n,
                                                                int total) {
  using L = Lat<2>;
  const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5);
  for (int t = (int)blockIdx.x; t < total; t += PERSIST ? (int)gridDim.x : total) {
    int lo = 0, hi = n - 1;  // the member: the last m with first[m] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(first + mid) <= t) lo = mid;
      else hi = mid - 1;
    }
    const LbmArgs A = args[lo];  // local copy: fields loaded once, not after every store
    const int spr = (A.g.nx + 32 * K - 1) / (32 * K);
    const long long item = (long long)(t - __ldg(first + lo)) * W + warp;
    const long long row = item / spr;
    if (row >= A.g.rows) continue;  // past the member's last row (its last tile)
    const int seg = (int)(item - row * spr);
    step_row_nodes<L, PARITY, ST, K>(A, row, (int)row, 0, K * (seg * 32 + lane));
  }
}

// The odd-step nodes lbm_step_kernel leaves: every node of the face rows, then the
// two end nodes of every other row, one thread per node, general addressing.
// face rows and inner-row end nodes of an odd step (lbm_step_edge_kernel's index space)
__host__ __device__ inline void edge_counts(const Geo& g, int dim, long long& nface, long long& nends) {
  long long inner;
  if (dim == 2) {
    nface = g.ny > 1 ? 2 : 1;
    inner = g.ny > 2 ? g.ny - 2 : 0;
  } else {
    nface = (long long)g.ny * (g.nz > 1 ? 2 : 1) + (long long)(g.nz > 2 ? g.nz - 2 : 0) * (g.ny > 1 ? 2 : 1);
    inner = (long long)(g.ny > 2 ? g.ny - 2 : 0) * (g.nz > 2 ? g.nz - 2 : 0);
  }
  nends = inner * (g.nx > 1 ? 2 : 1);
}

template <class L, int ST>
__device__ __forceinline__ void step_edge_body(const LbmArgs& A, long long nface, long long nends,
                                               unsigned blk) {
  const Geo& g = A.g;
  const long long t = blk * (long long)kLbmBlock + threadIdx.x;
  int x, y, z;
  if (t < nface * g.nx) {  // face rows
    const long long k = t / g.nx;
    x = (int)(t - k * g.nx);
    if (L::dim == 2) {
      y = k == 0 ? 0 : g.ny - 1;
      z = 0;
    } else {
      const long long plane = g.ny;                      // rows of the z = 0 face
      const long long zf = g.nz > 1 ? 2 * plane : plane;  // rows of both z faces
      if (k < plane) {
        y = (int)k;
        z = 0;
      } else if (k < zf) {
        y = (int)(k - plane);
        z = g.nz - 1;
      } else {
        const long long j = k - zf;  // y faces of the inner z planes
        const int per = g.ny > 1 ? 2 : 1;
        z = 1 + (int)(j / per);
        y = (j % per) == 0 ? 0 : g.ny - 1;
      }
    }
  } else {
    const long long j = t - nface * g.nx;
    if (j >= nends) return;
    const int ends = g.nx > 1 ? 2 : 1;
    const long long r = j / ends;  // inner row: y in 1..ny-2, z in 1..nz-2 (3D)
    x = (j % ends) == 0 ? 0 : g.nx - 1;
    y = 1 + (int)(r % (g.ny - 2));
    z = L::dim == 3 ? 1 + (int)(r / (g.ny - 2)) : 0;
  }
  const long long row = (long long)y + (long long)g.ny * z;
  step_node<L, 1, ST>(A, row, x, y, z, (long long)x + (long long)g.nx * row);
}

template <class L, int ST, bool FUSED>
__global__ void __launch_bounds__(kLbmBlock) lbm_step_edge_kernel(LbmArgs A0, long long nface0,
                                                                 long long nends0, Fuse FU) {
  IBMLBM_BIND(FUSED, LbmArgs, A, A0, FU, blk);
  long long nface = nface0, nends = nends0;
  if (FUSED) edge_counts(A.g, L::dim, nface, nends);
  step_edge_body<L, ST>(A, nface, nends, blk);
}

// An odd step of one run in one launch: the row tiles of lbm_step_kernel and the edge
// nodes (face rows, row ends), with the edge blocks spread evenly through the grid
// (one every `stride` blocks from block 0), so their scattered, latency-bound accesses
// run beside the bandwidth-bound row tiles instead of after them.  No node of one set
// reads or writes a slot of the other (an AA step swaps each node's own slots).
template <class L, int ST, int K>
__global__ void __launch_bounds__(kLbmBlock, L::dim == 3 ? 7 : 10)
    lbm_step_odd_kernel(LbmArgs A, int spr, unsigned eblocks, unsigned stride, long long nface, long long nends) {
  const unsigned b = blockIdx.x, q = b / stride;
  if (b - q * stride == 0 && q < eblocks) {
    step_edge_body<L, ST>(A, nface, nends, q);
    return;
  }
  step_tile_body<L, 1, ST, K>(A, spr, b - min(eblocks, q + 1));
}

// Flat tiles: block b takes the K kLbmBlock consecutive nodes from b K kLbmBlock on
// (row-major), a thread its nodes threadIdx.x + k kLbmBlock, so every load and store
// instruction of a warp covers consecutive nodes whatever the row length: a batch
// member's short rows leave no thread idle, and the block's copy of its member's
// arguments serves K kLbmBlock nodes.  The even step is local everywhere; an odd step
// leaves the face rows and row ends to the edge blocks and reads the other nodes' slots
// at fixed offsets, as step_row_nodes does.
constexpr int kFlatK32 = 4;  // nodes per thread, FP32 storage
constexpr int kFlatK16 = 2;  // nodes per thread, 16-bit storages
template <int ST>
__host__ __device__ constexpr int flat_k() { return ST == STORE_F32 ? kFlatK32 : kFlatK16; }

template <class L, int PARITY, int ST, int K>
__device__ __forceinline__ void step_flat_body(const LbmArgs& A, unsigned blk) {
  constexpr bool H = ST != STORE_F32;  // 16-bit storages collide the stored h = f / w
  const Geo& g = A.g;
  const long long n0 = (long long)blk * (K * kLbmBlock) + threadIdx.x;
  const bool small = g.N < (1LL << 31);  // 32-bit division where it fits
  float fa[K][L::Q], fv[K][3];
  int xs[K], ys[K], zs[K];
  long long rows[K];
  bool act[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const long long n = n0 + (long long)k * kLbmBlock;
    act[k] = n < g.N;
    xs[k] = ys[k] = zs[k] = 0;
    rows[k] = 0;
    if (!act[k]) continue;
    if (small) {
      const unsigned un = (unsigned)n, ur = un / (unsigned)g.nx;
      xs[k] = (int)(un - ur * (unsigned)g.nx);
      rows[k] = ur;
      if (L::dim == 2) {
        ys[k] = (int)ur;
      } else {
        const unsigned uz = ur / (unsigned)g.ny;
        zs[k] = (int)uz;
        ys[k] = (int)(ur - uz * (unsigned)g.ny);
      }
    } else {
      rows[k] = n / g.nx;
      xs[k] = (int)(n - rows[k] * g.nx);
      ys[k] = (int)(rows[k] % g.ny);
      zs[k] = (int)(rows[k] / g.ny);
    }
    if (PARITY == 1 && (xs[k] == 0 || xs[k] == g.nx - 1 || odd_edge_row<L>(g, ys[k], zs[k]))) {
      act[k] = false;
      continue;
    }
    load_pdfs<L, PARITY, ST, PARITY == 1, H>(g, A.f, xs[k], ys[k], zs[k], n, fa[k]);
    ib_force<L>(A, rows[k], xs[k], n, fv[k]);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!act[k]) continue;
    const long long n = n0 + (long long)k * kLbmBlock;
    float F[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) F[c] = A.body[c] + fv[k][c];
    if constexpr (H) collide_h<L>(fa[k], F, A.omega, A.kforce);
    else collide<L>(fa[k], F, A.omega, A.kforce);
    store_post<L, PARITY, ST, PARITY == 1, H>(g, A.f, xs[k], ys[k], zs[k], n, fa[k]);
    ib_force_clear<L>(A, n, fv[k]);
  }
}

// the even step of a 2D batch (or an odd step with no edge blocks), flat tiles
template <int PARITY, int ST>
__global__ void __launch_bounds__(kLbmBlock) lbm_step_flat_kernel(Fuse F) {
  unsigned blk;
  const LbmArgs A = fused_args<LbmArgs>(F, blockIdx.x, blk);
  step_flat_body<Lat<2>, PARITY, ST, flat_k<ST>()>(A, blk);
}

// A single 2D run's FP32 step on flat tiles, kFlatRun nodes a thread.  Measured on the
// 2048 x 4096 cavity (ms per collide-stream launch, mean of both parities): 0.1033 with
// particles and 0.0925 without, against 0.1094 and 0.1004 on the row tiles (K = 2: 0.1045,
// 0.0960); bit for bit the same nodes.  3D keeps the row tiles: with 19 directions four
// (two) nodes a thread take 168 (119) registers, and the 384 x 384 x 768 cavity's
// collide-stream measured 4.16 (3.75) against 3.39 ms.
constexpr int kFlatRun = 4;

template <class L, int PARITY, int K>
__global__ void __launch_bounds__(kLbmBlock) lbm_step_flat1_kernel(LbmArgs A) {
  step_flat_body<L, PARITY, STORE_F32, K>(A, blockIdx.x);
}

// the odd step of one run on flat tiles, with the edge blocks spread through the grid
// as in lbm_step_odd_kernel
template <class L, int K>
__global__ void __launch_bounds__(kLbmBlock) lbm_step_odd_flat1_kernel(LbmArgs A, unsigned eblocks, unsigned stride,
                                                                       long long nface, long long nends) {
  const unsigned b = blockIdx.x, q = b / stride;
  if (b - q * stride == 0 && q < eblocks) {
    step_edge_body<L, STORE_F32>(A, nface, nends, q);
    return;
  }
  step_flat_body<L, 1, STORE_F32, K>(A, b - min(eblocks, q + 1));
}

// An odd step of a 2D batch in one launch: blocks [0, blocks) are the members' flat
// tiles, the rest their face rows and row ends.  No node of one set reads or writes a
// slot of the other (an AA step swaps each node's own slots), so both run together.
template <int ST>
__global__ void __launch_bounds__(kLbmBlock) lbm_step_odd_batch_kernel(Fuse F, unsigned blocks, Fuse FE) {
  unsigned blk;
  if (blockIdx.x < blocks) {
    const LbmArgs A = fused_args<LbmArgs>(F, blockIdx.x, blk);
    step_flat_body<Lat<2>, 1, ST, flat_k<ST>()>(A, blk);
  } else {
    const LbmArgs A = fused_args<LbmArgs>(FE, blockIdx.x - blocks, blk);
    long long nface, nends;
    edge_counts(A.g, 2, nface, nends);
    step_edge_body<Lat<2>, ST>(A, nface, nends, blk);
  }
}

// Boundary nodes of the extrapolation boundaries: the nodes on a face of a
// non-periodic axis, enumerated as the two z faces (3D), then the two y faces of the
// inner z range, then the two x faces of the inner y and z ranges.
__host__ __device__ inline void shell_groups(const Geo& g, int dim, long long& gz, long long& gy,
                                             long long& gx) {
  const bool fz = dim == 3 && !g.per[2], fy = !g.per[1], fx = !g.per[0];
  const long long iz = dim == 3 ? (fz ? g.nz - 2 : g.nz) : 1, iy = fy ? g.ny - 2 : g.ny;
  gz = fz ? 2LL * g.nx * g.ny : 0;
  gy = fy ? 2LL * g.nx * iz : 0;
  gx = fx ? 2LL * iy * iz : 0;
}

__device__ __forceinline__ bool shell_node(const Geo& g, int dim, long long t, int (&c)[3]) {
  long long gz, gy, gx;
  shell_groups(g, dim, gz, gy, gx);
  const int oz = (dim == 3 && !g.per[2]) ? 1 : 0, oy = g.per[1] ? 0 : 1;
  if (t < gz) {
    const long long plane = (long long)g.nx * g.ny, r = t % plane;
    c[0] = (int)(r % g.nx);
    c[1] = (int)(r / g.nx);
    c[2] = t < plane ? 0 : g.nz - 1;
    return true;
  }
  t -= gz;
  if (t < gy) {
    const long long r = t >> 1;
    c[0] = (int)(r % g.nx);
    c[1] = (t & 1) ? g.ny - 1 : 0;
    c[2] = oz + (int)(r / g.nx);
    return true;
  }
  t -= gy;
  if (t < gx) {
    const long long r = t >> 1;
    const long long iy = g.per[1] ? g.ny : g.ny - 2;
    c[0] = (t & 1) ? g.nx - 1 : 0;
    c[1] = oy + (int)(r % iy);
    c[2] = oz + (int)(r / iy);
    return true;
  }
  return false;
}

// Non-equilibrium extrapolation (the method Sec. 6.1-6.2 apply; boundary 1, 2), after
// the collide-stream step, in the layout PARITY the next step reads: a boundary node
// x_b takes f_a = f_a^eq(p_b, u_b) + f_a(x_f) - f_a^eq(p_f, u_f), x_f = x_b + the sum of
// the inward normals of the faces x_b lies on, (p_f, u_f) = Eq. 6-7 at x_f with the
// body force.  Walls: u_b = 0, p_b = p_f; channel inlet (y = 0): u_b along y = the
// parabola, p_b = p_f; outlet (y = ny - 1): p_b = 0, u_b = u_f; a node on a wall face
// is a wall node.  x_f is never a boundary node (n >= 3 on those axes), and each thread
// reads only x_f's slots and writes only x_b's, so the threads are independent.
template <class L, int PARITY, int ST>
__global__ void __launch_bounds__(kLbmBlock) lbm_nee_kernel(LbmArgs A) {
  const Geo& g = A.g;
  int c[3] = {0, 0, 0};
  if (!shell_node(g, L::dim, blockIdx.x * (long long)kLbmBlock + threadIdx.x, c)) return;
  const int n3[3] = {g.nx, g.ny, g.nz};
  int cf[3] = {c[0], c[1], c[2]};
  bool wall = false, inlet = false;
#pragma unroll
  for (int k = 0; k < L::dim; ++k) {
    if (g.per[k]) continue;
    const bool lo = c[k] == 0, hi = c[k] == n3[k] - 1;
    if (!lo && !hi) continue;
    cf[k] = lo ? c[k] + 1 : c[k] - 1;
    if (A.boundary == 2 && k == 1) inlet = inlet || lo;
    else wall = true;
  }
  float fa[L::Q], eqf[L::Q], eqb[L::Q], us[3], s1, uf[3], ub[3] = {0.0f, 0.0f, 0.0f};
  load_pdfs<L, PARITY, ST>(g, A.f, cf[0], cf[1], cf[2], node_of(g, cf[0], cf[1], cf[2]), fa);
  moments<L>(fa, us, s1);
#pragma unroll
  for (int k = 0; k < 3; ++k) uf[k] = (k < L::dim) ? us[k] + 0.5f * A.body[k] : 0.0f;  // Eq. 7
  const float pf = pressure<L>(s1, uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2]);
  float pb = pf;
  if (!wall && inlet) {
    float prof = A.u_inlet;
#pragma unroll
    for (int k = 0; k < L::dim; ++k) {
      if (k == 1 || g.per[k]) continue;
      const float Lk = (float)(n3[k] - 1), ck = (float)c[k];
      prof *= 4.0f * ck * (Lk - ck) / (Lk * Lk);
    }
    ub[1] = prof;
  } else if (!wall) {  // outlet
#pragma unroll
    for (int k = 0; k < 3; ++k) ub[k] = uf[k];
    pb = 0.0f;
  }
  equilibrium<L>(pf, uf, eqf);
  equilibrium<L>(pb, ub, eqb);
#pragma unroll
  for (int a = 0; a < L::Q; ++a) fa[a] = eqb[a] + (fa[a] - eqf[a]);
  put_pdfs<L, PARITY, ST>(g, A.f, c[0], c[1], c[2], node_of(g, c[0], c[1], c[2]), fa);
}

// u* = sum_a e_a f_a (Eq. 5) on the flagged nodes only: one thread per node in large
// blocks; threads of unflagged nodes leave after reading their mask word.  The mask
// is cleared before the particle update marks the next step's nodes.
constexpr int kMomBlock = 512;

template <class L, int PARITY, int ST>
__global__ void __launch_bounds__(kMomBlock) lbm_moments_kernel(LbmArgs A) {
  const long long n = blockIdx.x * (long long)kMomBlock + threadIdx.x;
  if (n >= A.g.N) return;
  const unsigned nx = (unsigned)A.g.nx;
  const unsigned row = (unsigned)(n / nx);
  const int x = (int)(n - (long long)row * nx);
  if (!IBMLBM_CHK((long long)row * A.g.wpr + (x >> 5), (long long)A.g.rows * A.g.wpr)) return;
  const uint32_t word = A.mask[(long long)row * A.g.wpr + (x >> 5)];
  if (!((word >> (x & 31)) & 1u)) return;
  const unsigned uny = (unsigned)A.g.ny;
  const unsigned z = row / uny;
  const int y = (int)(row - z * uny);
  float fa[L::Q], us[3], s1;
  if (PARITY == 1 && x >= 1 && x <= A.g.nx - 2 && y >= 1 && y <= A.g.ny - 2 &&
      (L::dim == 2 || ((int)z >= 1 && (int)z <= A.g.nz - 2)))
    load_pdfs<L, PARITY, ST, true>(A.g, A.f, x, y, (int)z, n, fa);  // fixed neighbour offsets
  else
    load_pdfs<L, PARITY, ST>(A.g, A.f, x, y, (int)z, n, fa);
  moments<L>(fa, us, s1);
  if (L::dim == 3)
    reinterpret_cast<float4*>(A.ustar)[n] = make_float4(us[0], us[1], us[2], 0.0f);
  else
    reinterpret_cast<float2*>(A.ustar)[n] = make_float2(us[0], us[1]);
}

// p (Eq. 6 with u = u*) and u* (Eq. 5) on every node, as doubles.
template <class L, int PARITY, int ST>
__global__ void __launch_bounds__(kLbmBlock) lbm_fields_kernel(LbmArgs A, int cpr, double* p,
                                                              double* u) {
  const NodeCoord c = node_coord(A.g, cpr);
  if (!c.valid) return;
  float fa[L::Q], us[3], s1;
  load_pdfs<L, PARITY, ST>(A.g, A.f, c.x, c.y, c.z, c.n, fa);
  moments<L>(fa, us, s1);
  const float uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
  if (p) p[c.n] = (double)pressure<L>(s1, uu);
  if (u) {
#pragma unroll
    for (int k = 0; k < L::dim; ++k) u[k * A.g.N + c.n] = (double)us[k];
  }
}

// canonical [Q][N] copy of the current PDFs
template <class L, int PARITY, int ST>
__global__ void __launch_bounds__(kLbmBlock) lbm_get_kernel(LbmArgs A, int cpr, float* out) {
  const NodeCoord c = node_coord(A.g, cpr);
  if (!c.valid) return;
  float fa[L::Q];
  load_pdfs<L, PARITY, ST>(A.g, A.f, c.x, c.y, c.z, c.n, fa);
#pragma unroll
  for (int a = 0; a < L::Q; ++a) out[a * A.g.N + c.n] = fa[a];
}

// write canonical [Q][N] PDFs into the layout of the current parity
template <class L, int PARITY, int ST>
__global__ void __launch_bounds__(kLbmBlock) lbm_put_kernel(LbmArgs A, int cpr,
                                                           const float* in) {
  const NodeCoord c = node_coord(A.g, cpr);
  if (!c.valid) return;
  float fa[L::Q];
#pragma unroll
  for (int a = 0; a < L::Q; ++a) fa[a] = in[a * A.g.N + c.n];
  put_pdfs<L, PARITY, ST>(A.g, A.f, c.x, c.y, c.z, c.n, fa);
}

// equilibrium of Eq. 4 for given p [N] and u [D][N] (doubles), current parity layout
template <class L, int PARITY, int ST>
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
  put_pdfs<L, PARITY, ST>(A.g, A.f, c.x, c.y, c.z, c.n, fa);
}

// ------------------------------------------------------------------ launchers
static dim3 lbm_grid(const Geo& g, int& cpr) {
  cpr = (g.nx + kLbmBlock - 1) / kLbmBlock;
  return dim3((unsigned)((long long)cpr * g.rows));
}

#define IBMLBM_DISPATCH_ST(L, PARITY, KERNEL, GRID, BLOCK, ...)                                  \
  do {                                                                                          \
    if (A.store == STORE_F32) KERNEL<L, PARITY, STORE_F32><<<GRID, BLOCK, 0, s>>>(__VA_ARGS__);   \
    else if (A.store == STORE_F16) KERNEL<L, PARITY, STORE_F16><<<GRID, BLOCK, 0, s>>>(__VA_ARGS__); \
    else KERNEL<L, PARITY, STORE_BF16><<<GRID, BLOCK, 0, s>>>(__VA_ARGS__);                       \
  } while (0)

#define IBMLBM_DISPATCH_G(D, PARITY, KERNEL, GRID, BLOCK, ...)                               \
  do {                                                                                       \
    if ((D) == 2) {                                                                          \
      if ((PARITY) == 0) IBMLBM_DISPATCH_ST(Lat<2>, 0, KERNEL, GRID, BLOCK, __VA_ARGS__);      \
      else IBMLBM_DISPATCH_ST(Lat<2>, 1, KERNEL, GRID, BLOCK, __VA_ARGS__);                    \
    } else {                                                                                 \
      if ((PARITY) == 0) IBMLBM_DISPATCH_ST(Lat<3>, 0, KERNEL, GRID, BLOCK, __VA_ARGS__);      \
      else IBMLBM_DISPATCH_ST(Lat<3>, 1, KERNEL, GRID, BLOCK, __VA_ARGS__);                    \
    }                                                                                        \
  } while (0)

#define IBMLBM_DISPATCH(D, PARITY, KERNEL, ...) \
  IBMLBM_DISPATCH_G(D, PARITY, KERNEL, grid, kLbmBlock, __VA_ARGS__)

template <int ST>
constexpr int step_k() { return ST == STORE_F32 ? 1 : 2; }

// blocks of a batch member's flat tiles (2D) and of its odd-step edge blocks
unsigned lbm_step_blocks(const Geo& g, int store) {
  const int K = store == STORE_F32 ? flat_k<STORE_F32>() : flat_k<STORE_F16>();
  return (unsigned)((g.N + K * kLbmBlock - 1) / (K * kLbmBlock));
}
unsigned lbm_edge_blocks(const Geo& g, int D) {
  long long nface, nends;
  edge_counts(g, D, nface, nends);
  return (unsigned)((nface * g.nx + nends + kLbmBlock - 1) / kLbmBlock);
}

// The vector kernel serves D2Q9 with a 16-bit storage, eight nodes (one 16-byte
// vector per direction) per thread, on rows whose length is a multiple of 8.
// Measured on the 2048 x 4096 lattice without particles (GB300, ms per step): FP16
// 0.0616 against 0.0773 for the row kernel.  2D FP32 takes the flat tiles (0.0925;
// the row kernel 0.0985, the vector kernel with K = 4 0.104); 3D keeps the row kernel,
// which measured faster there at 384 x 384 x 768: 3.17 FP32 / 2.28 FP16 (3.74 / 3.51
// vector, K = 4): with 19 directions the vectors and their addresses take 130 to 200
// registers a thread and leave too few warps to cover the memory latency.
constexpr int kVecK = 8;
template <class L, int ST>
constexpr bool vec_form() { return L::dim == 2 && ST != STORE_F32; }

template <class L, int ST>
static bool use_vec(const Geo& g) { return vec_form<L, ST>() && g.nx % kVecK == 0; }

template <class L, int PARITY, int ST>
static void launch_step_main(const LbmArgs& A, cudaStream_t s) {
  if constexpr (vec_form<L, ST>()) {
    if (use_vec<L, ST>(A.g)) {
      const int spr = (A.g.nx + 32 * kVecK - 1) / (32 * kVecK);
      const long long warps = (long long)spr * A.g.rows;
      const dim3 grid((unsigned)((warps + kVecWarps - 1) / kVecWarps));
      lbm_step_vec_kernel<L, PARITY, ST, kVecK><<<grid, 32 * kVecWarps, 0, s>>>(A, spr);
      return;
    }
  }
  constexpr int K = step_k<ST>();
  const int spr = (A.g.nx + K * kLbmBlock - 1) / (K * kLbmBlock);
  const dim3 grid((unsigned)((long long)spr * A.g.rows));
  // an ordinary launch: programmatic blocks of this large grid would sit resident ahead
  // of the high-priority particle kernels (measured slower)
  lbm_step_kernel<L, PARITY, ST, K, false><<<grid, kLbmBlock, 0, s>>>(A, spr, Fuse{});
}

// fused over the members of a 2D batch (FP32 or FP16 storage, one for all members)
cudaError_t launch_lbm_step_fused(const Fuse& F, unsigned blocks, const Fuse& FE, unsigned eblocks,
                                  int store, int parity, cudaStream_t s) {
#define IBMLBM_STEPF(P, ST)                                                                        \
  do {                                                                                               \
    if (P == 1 && eblocks)                                                                           \
      lbm_step_odd_batch_kernel<ST><<<blocks + eblocks, kLbmBlock, 0, s>>>(F, blocks, FE);           \
    else                                                                                             \
      lbm_step_flat_kernel<P, ST><<<blocks, kLbmBlock, 0, s>>>(F);                                   \
  } while (0)
  if (store == STORE_F32) {
    if (parity == 0) IBMLBM_STEPF(0, STORE_F32); else IBMLBM_STEPF(1, STORE_F32);
  } else {
    if (parity == 0) IBMLBM_STEPF(0, STORE_F16); else IBMLBM_STEPF(1, STORE_F16);
  }
#undef IBMLBM_STEPF
  return cudaGetLastError();
}

// Tile shapes of a batch's fused lbm_step: shape 0 is the flat-tile kernel above
// (flat_k nodes per thread: 4 for FP32, 2 for FP16; kLbmBlock threads), shapes 1.. are
// warp tiles (K nodes per thread, W warps per block, persistent grid or one block per
// tile).
struct TileShape {
  int k, w, persist;
};
constexpr TileShape kTileShapes[] = {{0, 0, 0}, {1, 4, 0}, {1, 8, 0}, {2, 4, 0},
                                     {1, 4, 1}, {1, 8, 1}, {2, 4, 1}};
constexpr int kTileShapeCount = (int)(sizeof(kTileShapes) / sizeof(kTileShapes[0]));

int tile_shape_count() { return kTileShapeCount; }

void tile_shape(int s, int store, int* k, int* w, int* persist) {
  const TileShape& t = kTileShapes[s];
  *k = s == 0 ? (store == STORE_F32 ? flat_k<STORE_F32>() : flat_k<STORE_F16>()) : t.k;
  *w = s == 0 ? kLbmBlock / 32 : t.w;
  *persist = t.persist;
}

// warp tiles of one member for shape s >= 1
int tile_count(const Geo& g, int s) {
  const TileShape& t = kTileShapes[s];
  const long long spr = (g.nx + 32 * t.k - 1) / (32 * t.k);
  return (int)((spr * g.rows + t.w - 1) / t.w);
}

template <int PARITY, int ST, int K, int W, bool PERSIST>
static cudaError_t launch_tiles(const LbmArgs* args, const int* first, int n, int total, cudaStream_t s) {
  auto kern = lbm_step_tiles_kernel<PARITY, ST, K, W, PERSIST>;
  unsigned grid = (unsigned)total;
  if (PERSIST) {
    static int resident = 0;  // blocks of this kernel the GPU holds at once
    if (resident == 0) {
      int dev = 0, sms = 0, per_sm = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * W, 0);
      if (e != cudaSuccess) return e;
      resident = std::max(1, sms * per_sm);
    }
    grid = (unsigned)std::min(total, resident);
  }
  kern<<<grid, 32 * W, 0, s>>>(args, first, n, total);
  return cudaSuccess;
}

template <int PARITY, int ST>
static cudaError_t launch_tiles_shape(int shape, const LbmArgs* args, const int* first, int n, int total,
                                      cudaStream_t s) {
  switch (shape) {
    case 1: return launch_tiles<PARITY, ST, 1, 4, false>(args, first, n, total, s);
    case 2: return launch_tiles<PARITY, ST, 1, 8, false>(args, first, n, total, s);
    case 3: return launch_tiles<PARITY, ST, 2, 4, false>(args, first, n, total, s);
    case 4: return launch_tiles<PARITY, ST, 1, 4, true>(args, first, n, total, s);
    case 5: return launch_tiles<PARITY, ST, 1, 8, true>(args, first, n, total, s);
    default: return launch_tiles<PARITY, ST, 2, 4, true>(args, first, n, total, s);
  }
}

// fused lbm_step of a batch with warp-tile shape >= 1 (the edge kernel as for shape 0)
cudaError_t launch_lbm_step_tiles(int shape, const LbmArgs* args, const int* first, int n, int total,
                                  const Fuse& FE, unsigned eblocks, int store, int parity, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (total > 0) {
    if (store == STORE_F32)
      e = parity == 0 ? launch_tiles_shape<0, STORE_F32>(shape, args, first, n, total, s)
                      : launch_tiles_shape<1, STORE_F32>(shape, args, first, n, total, s);
    else
      e = parity == 0 ? launch_tiles_shape<0, STORE_F16>(shape, args, first, n, total, s)
                      : launch_tiles_shape<1, STORE_F16>(shape, args, first, n, total, s);
  }
  if (e != cudaSuccess) return e;
  const LbmArgs none{};
  if (parity == 1 && eblocks) {
    if (store == STORE_F32) lbm_step_edge_kernel<Lat<2>, STORE_F32, true><<<eblocks, kLbmBlock, 0, s>>>(none, 0, 0, FE);
    else lbm_step_edge_kernel<Lat<2>, STORE_F16, true><<<eblocks, kLbmBlock, 0, s>>>(none, 0, 0, FE);
  }
  return cudaGetLastError();
}

// extrapolation boundaries after a step of the given parity (no-op for boundary 0)
cudaError_t launch_lbm_nee(const LbmArgs& A, int D, int parity, cudaStream_t s) {
  if (A.boundary == 0) return cudaSuccess;
  long long gz, gy, gx;
  shell_groups(A.g, D, gz, gy, gx);
  const long long total = gz + gy + gx;
  if (total == 0) return cudaSuccess;
  const dim3 grid((unsigned)((total + kLbmBlock - 1) / kLbmBlock));
  const int next = 1 - parity;  // the layout the next step reads
  IBMLBM_DISPATCH_G(D, next, lbm_nee_kernel, grid, kLbmBlock, A);
  return cudaGetLastError();
}

// kernels launch_lbm_step launches: one (the vector kernel, the flat or row tiles, or in
// an odd step the tiles with the edge nodes)
int lbm_step_launches(const Geo&, int, int, int) { return 1; }

template <class L, int PARITY, int ST>
static void launch_step_one(const LbmArgs& A, cudaStream_t s) {
  if constexpr (ST == STORE_F32 && L::dim == 2) {
    constexpr int K = kFlatRun;
    const unsigned main = (unsigned)((A.g.N + K * kLbmBlock - 1) / (K * kLbmBlock));
    if (PARITY == 1) {
      long long nface, nends;
      edge_counts(A.g, L::dim, nface, nends);
      const long long total = nface * A.g.nx + nends;
      const unsigned eb = (unsigned)((total + kLbmBlock - 1) / kLbmBlock);
      const unsigned stride = eb ? (main + eb) / eb : 1;
      lbm_step_odd_flat1_kernel<L, K><<<main + eb, kLbmBlock, 0, s>>>(A, eb, stride, nface, nends);
    } else {
      lbm_step_flat1_kernel<L, 0, K><<<main, kLbmBlock, 0, s>>>(A);
    }
    return;
  }
  if (PARITY == 1 && !use_vec<L, ST>(A.g)) {
    long long nface, nends;
    edge_counts(A.g, L::dim, nface, nends);
    const long long total = nface * A.g.nx + nends;
    if (total > 0) {
      constexpr int K = step_k<ST>();
      const int spr = (A.g.nx + K * kLbmBlock - 1) / (K * kLbmBlock);
      const unsigned main = (unsigned)((long long)spr * A.g.rows);
      const unsigned eb = (unsigned)((total + kLbmBlock - 1) / kLbmBlock);
      const unsigned stride = (main + eb) / eb;
      lbm_step_odd_kernel<L, ST, K><<<main + eb, kLbmBlock, 0, s>>>(A, spr, eb, stride, nface, nends);
      return;
    }
  }
  launch_step_main<L, PARITY, ST>(A, s);
}

template <class L, int PARITY>
static void launch_step_st(const LbmArgs& A, cudaStream_t s) {
  if (A.store == STORE_F32) launch_step_one<L, PARITY, STORE_F32>(A, s);
  else if (A.store == STORE_F16) launch_step_one<L, PARITY, STORE_F16>(A, s);
  else launch_step_one<L, PARITY, STORE_BF16>(A, s);
}

// whether launch_lbm_step uses the vector kernel for this lattice and storage
bool lbm_step_vector(const Geo& g, int D, int store) {
  if (D == 2)
    return store == STORE_F32 ? use_vec<Lat<2>, STORE_F32>(g) : use_vec<Lat<2>, STORE_F16>(g);
  return store == STORE_F32 ? use_vec<Lat<3>, STORE_F32>(g) : use_vec<Lat<3>, STORE_F16>(g);
}

cudaError_t launch_lbm_step(const LbmArgs& A, int D, int parity, cudaStream_t s) {
  if (D == 2) {
    if (parity == 0) launch_step_st<Lat<2>, 0>(A, s);
    else launch_step_st<Lat<2>, 1>(A, s);
  } else {
    if (parity == 0) launch_step_st<Lat<3>, 0>(A, s);
    else launch_step_st<Lat<3>, 1>(A, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_lbm_moments(const LbmArgs& A, int D, int parity, cudaStream_t s) {
  const dim3 grid((unsigned)((A.g.N + kMomBlock - 1) / kMomBlock));
  if (D != 3) return cudaErrorInvalidValue;  // 2D computes u* per particle box
  if (parity == 0) IBMLBM_DISPATCH_ST(Lat<3>, 0, lbm_moments_kernel, grid, kMomBlock, A);
  else IBMLBM_DISPATCH_ST(Lat<3>, 1, lbm_moments_kernel, grid, kMomBlock, A);
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

namespace ibmlbm {
unsigned long long check_fault_lbm() { return take_check_fault(); }
}  // namespace ibmlbm
