// Cell-list pair search, short-range repulsive force (Sec. 5, Eq. 16) and the
// double-precision particle update (Eq. 14-15).
//
// Cells of side H_k = L_k / nc_k >= D_p + zeta (a periodic axis with fewer than three
// cells becomes one cell), so every pair closer than D_p + zeta lies in the 3^D
// neighbourhood of a cell.  Each cell is a bucket of at most cell_cap particle ids
// filled with one atomic slot per particle (overflow is reported, never dropped
// silently).  A warp per particle then scans its neighbourhood, keeps partners j with
// |X_i - X_j|^2 < (D_p + zeta)^2 -- squared distance summed in axis order in double
// precision without fused multiply-add, nearest image on periodic axes -- sorts them
// by index and sums the Eq. 16 force in that order, so the result does not depend on
// the order inside the buckets.  The canonical pair list (i < j, sorted) is compacted
// from these per-particle lists on request.  In a time step one thread per particle
// then sums the contact force and advances the particle in double precision, writing
// the new centre to the other centre buffer, so neighbours still read old centres.
#include <cmath>

#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace ibmlbm {

constexpr int kMaxNeighbors = 64;

__device__ __forceinline__ int cell_coord(double X, double H, int nc) {
  int c = (int)floor((X + 0.5) / H);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

template <int D>
__device__ __forceinline__ int cell_of(const PairArgs& A, int i) {
  int c = 0, stride = 1;
  for (int k = 0; k < D; ++k) {
    c += stride * cell_coord(A.X[(long long)i * D + k], A.H[k], A.nc[k]);
    stride *= A.nc[k];
  }
  return c;
}

// one thread per particle (thread tid of a block of nthr): its cell's next bucket slot
template <int D>
__device__ __forceinline__ void pair_insert_body(const PairArgs& A, unsigned blk, int tid, int nthr) {
  const int i = (int)(blk * nthr + tid);
  if (i >= A.n) return;
  const int c = cell_of<D>(A, i);
  if (!IBMLBM_CHK(c, (long long)A.nc[0] * A.nc[1] * A.nc[2])) return;
  const int slot = atomicAdd(&A.cell_count[c], 1);
  if (slot < A.cell_cap)
    A.cell_ids[(long long)c * A.cell_cap + slot] = i;
  else
    atomicOr(A.status, ST_CAPACITY);
}

template <int D, bool FUSED>
__global__ void pair_insert_kernel(PairArgs A0, Fuse FU) {
  IBMLBM_BIND(FUSED, PairArgs, A, A0, FU, blk);
  pair_insert_body<D>(A, blk, (int)threadIdx.x, (int)blockDim.x);
}

// X_i - X_j with the nearest image on periodic axes
template <int D>
__device__ __forceinline__ void separation(const PairArgs& A, const double* Xi, const double* Xj,
                                           double (&dx)[3]) {
  dx[0] = dx[1] = dx[2] = 0.0;
  for (int k = 0; k < D; ++k) {
    double d = Xi[k] - Xj[k];
    if (A.g.per[k]) {
      if (d > 0.5 * A.L[k])
        d -= A.L[k];
      else if (d < -0.5 * A.L[k])
        d += A.L[k];
    }
    dx[k] = d;
  }
}

__device__ __forceinline__ double dist2_nofma(const double (&dx)[3]) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx[0], dx[0]), __dmul_rn(dx[1], dx[1])),
                   __dmul_rn(dx[2], dx[2]));
}

// Eq. 16 magnitude at distance d (third case read as the sum of both printed terms)
__device__ __forceinline__ double eq16_magnitude(const PairArgs& A, double d) {
  const double D = A.diam, z = A.zeta;
  double mag = 0.0;
  if (d < D + z) {
    const double t = (d - D - z) / z;
    mag = A.c_ij / A.eps_pp * t * t;
    if (d < D) mag += A.c_ij / A.E_pp * ((D - d) / z);
  }
  return mag;
}

// Newton-Euler update of particle i (Eq. 14-15 with the interior-momentum closure):
//   (M_p + K) a^n - K a^{n-1} = (F_h^n + F_h^{n-1})/2 + F_c + (P_int^n - P_int^{n-1})
//                              + (M_p - rho_f V_p) g
//   U^{n+1} = U^n + a^n, X^{n+1} = X^n + (U^n + U^{n+1})/2; rotation alike with I_p, K_r.
// fixed = 1 holds the whole state, fixed = 2 holds centre and velocity but spins.
// The K terms telescope, so momentum is conserved; they keep the explicit coupling
// stable when the IB shell outweighs the particle.
template <int D>
__device__ void advance_particle(const PairArgs& A, int i, const double* X, const double* Fc) {
  const PartState& P = A.ps;
  const long long pi = i;
  bool bad = false;
  for (int c = 0; c < D; ++c) {
    const long long o = pi * D + c;
    const double fh = P.FhN[o];
    const double Fm = 0.5 * (fh + P.Fh[o]);
    const double dP = A.have_prev ? P.Pint[o] - P.Pprev[o] : 0.0;
    P.Fh[o] = fh;
    P.Pprev[o] = P.Pint[o];
    double x = X[c];
    if (P.fixed == 0) {
      const double F = Fm + Fc[c] + dP + P.meff * P.grav[c];
      const double a = (F + P.Kt * P.acc[o]) / (P.Mp + P.Kt);
      const double u0 = P.U[o], u1 = u0 + a;
      P.acc[o] = a;
      P.U[o] = u1;
      x += 0.5 * (u0 + u1);
    }
    const double n = A.L[c];
    if (A.g.per[c]) {
      if (x >= n - 0.5)
        x -= n;
      else if (x < -0.5)
        x += n;
    } else if (!(x >= -0.5 && x < n - 0.5)) {
      atomicOr(A.status, ST_OUT_OF_DOMAIN);
    }
    if (!isfinite(x) || !isfinite(P.U[o])) bad = true;
    P.Xnew[o] = x;
    P.Xcf[o] = isfinite(x) ? __double2ll_rn(x * kFixScale) : 0;
    P.Uf[o] = (float)P.U[o];
  }
  for (int c = (D == 2 ? 2 : 0); c < 3; ++c) {
    const long long o = pi * 3 + c;
    const double th = P.ThN[o];
    const double Tm = 0.5 * (th + P.Th[o]);
    const double dL = A.have_prev ? P.Lint[o] - P.Lprev[o] : 0.0;
    P.Th[o] = th;
    P.Lprev[o] = P.Lint[o];
    if (P.fixed != 1) {
      const double al = (Tm + dL + P.Kr * P.alp[o]) / (P.Ip + P.Kr);
      P.alp[o] = al;
      P.Om[o] += al;
    }
    if (!isfinite(P.Om[o])) bad = true;
    P.Omf[o] = (float)P.Om[o];
  }
  if (D == 2) P.Omf[pi * 3] = P.Omf[pi * 3 + 1] = 0.0f;
  if (bad) atomicOr(A.status, ST_NONFINITE);
}

// The cnt partners a warp collected for particle i (list holds the first kmax, in
// any order): sort by index, store the list, its length and the number of partners
// j > i; more than kmax partners is reported.
__device__ __forceinline__ void store_partners(const PairArgs& A, int i, int lane, int* list, int cnt) {
  __syncwarp();
  const int n_ok = min(cnt, A.kmax);
  if (lane == 0) {
    if (cnt > A.kmax) atomicOr(A.status, ST_CAPACITY);
    int gt = 0;
    for (int a = 1; a < n_ok; ++a) {  // insertion sort by partner index
      const int v = list[a];
      int b = a - 1;
      while (b >= 0 && list[b] > v) {
        list[b + 1] = list[b];
        --b;
      }
      list[b + 1] = v;
    }
    for (int a = 0; a < n_ok; ++a) gt += list[a] > i;
    A.nbr_count[i] = n_ok;
    A.gt_count[i] = gt;
  }
  __syncwarp();
  for (int a = lane; a < n_ok; a += 32) A.nbr[(long long)i * A.kmax + a] = list[a];
}

// partner test of the pair rule: j != i and |X_i - X_j|^2 < (D_p + zeta)^2
template <int D>
__device__ __forceinline__ bool is_partner(const PairArgs& A, const double (&Xi)[3], int i, int j) {
  if (j < 0 || j == i) return false;
  double Xj[3] = {0.0, 0.0, 0.0}, dx[3];
  for (int k = 0; k < D; ++k) Xj[k] = A.X[(long long)j * D + k];
  separation<D>(A, Xi, Xj, dx);
  return dist2_nofma(dx) < A.thr2;
}

// Neighbour search, one warp per particle.  Lane c < 3^D reads the count of
// neighbouring cell c; a warp scan turns the counts into offsets, and lane l then
// tests occupied slots l, l+32, ... of the concatenated buckets.  Accepted partners
// are appended in lane order and sorted by index.  Writes the sorted list, its length
// and the number of partners j > i.
// (256-thread blocks: eight warps, one particle each)
template <int D>
__device__ __forceinline__ void pair_search_body(const PairArgs& A, unsigned blk) {
  __shared__ int s_list[8][kMaxNeighbors];
  __shared__ int s_cell[8][32];
  __shared__ int s_off[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = (int)((blk * 256ll + threadIdx.x) >> 5);
  if (i >= A.n) return;  // whole warp
  __syncwarp();  // the warp's lists are free (a particle before may have used them)
  int* list = s_list[w];
  int* sc = s_cell[w];
  int* so = s_off[w];
  double Xi[3] = {0.0, 0.0, 0.0};
  int cc[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) {
    Xi[k] = A.X[(long long)i * D + k];
    cc[k] = cell_coord(Xi[k], A.H[k], A.nc[k]);
  }
  constexpr int NCELL = (D == 3) ? 27 : 9;
  int cnt_c = 0, cell = 0;
  if (lane < NCELL) {
    const int off[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
    int stride = 1;
    bool ok = true;
    for (int k = 0; k < D; ++k) {
      int c = cc[k] + off[k];
      if (A.nc[k] == 1) {
        if (off[k] != 0) ok = false;
        c = 0;
      } else if (c < 0 || c >= A.nc[k]) {
        if (A.g.per[k])
          c = (c + A.nc[k]) % A.nc[k];
        else
          ok = false;
      }
      cell += stride * c;
      stride *= A.nc[k];
    }
    if (ok && IBMLBM_CHK(cell, (long long)A.nc[0] * A.nc[1] * A.nc[2])) cnt_c = min(A.cell_count[cell], A.cell_cap);
  }
  int incl = cnt_c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  sc[lane] = cell;
  so[lane + 1] = incl;
  if (lane == 0) so[0] = 0;
  __syncwarp();
  const int total = so[32];
  int cnt = 0;
  for (int base = 0; base < total; base += 32) {
    const int q = base + lane;
    bool hit = false;
    int j = -1;
    if (q < total) {
      int c = 0;
      while (so[c + 1] <= q) ++c;
      j = A.cell_ids[(long long)sc[c] * A.cell_cap + (q - so[c])];
      if (j != i) {
        double Xj[3] = {0.0, 0.0, 0.0}, dx[3];
        for (int k = 0; k < D; ++k) Xj[k] = A.X[(long long)j * D + k];
        separation<D>(A, Xi, Xj, dx);
        hit = dist2_nofma(dx) < A.thr2;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
    if (hit && pos < A.kmax) list[pos] = j;
    cnt += __popc(m);
  }
  store_partners(A, i, lane, list, cnt);
}

template <int D, bool FUSED>
__global__ void __launch_bounds__(256) pair_search_kernel(PairArgs A0, Fuse FU) {
  IBMLBM_BIND(FUSED, PairArgs, A, A0, FU, blk);
  pair_search_body<D>(A, blk);
}

// ---------------------------------------------------------------- grid search
// The grid search of Sec. 5 (Table 5, Eq. 49-51): cells of side H_k < D_p / sqrt(D), so
// a cell can hold the centre of at most one particle when no two centres are closer
// than D_p, and the grid stores one particle index per cell (-1: empty).  Scatter: one
// thread per particle claims its cell with a compare-and-swap.  Eq. 16's contact lets
// two centres come closer than D_p, so a second centre in a claimed cell goes to an
// overflow list that every particle also scans (nothing is dropped; overflow of that
// list is reported).  Search: a warp per particle scans the cells within
// reach_k = ceil((D_p + zeta) / H_k) of its own along each axis -- 5 per axis when
// Eq. 50 holds (25 cells in 2D, 125 in 3D), wider where D_p + zeta >= 2 H_k (in 3D
// Eq. 49 and 50 only meet for zeta < 0.155 D_p) -- and keeps the partners by the same
// rule and in the same sorted order as the cell-list search, so the contact forces
// are the same.  Each particle collects its own partners (no Newton's-third-law
// pairing), so no two threads write one force.
template <int D>
__device__ __forceinline__ int grid_cell_of(const PairArgs& A, const double* X, int (&cc)[3]) {
  int c = 0, stride = 1;
  cc[0] = cc[1] = cc[2] = 0;
  for (int k = 0; k < D; ++k) {
    cc[k] = cell_coord(X[k], A.gH[k], A.gnc[k]);
    c += stride * cc[k];
    stride *= A.gnc[k];
  }
  return c;
}

template <int D>
__global__ void grid_scatter_kernel(PairArgs A) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= A.n) return;
  int cc[3];
  const int c = grid_cell_of<D>(A, A.X + (long long)i * D, cc);
  if (atomicCAS(&A.grid[c], -1, i) == -1) return;
  const int slot = atomicAdd(A.over_count, 1);
  if (slot < A.over_cap)
    A.over[slot] = i;
  else
    atomicOr(A.status, ST_CAPACITY);
}

template <int D>
__global__ void __launch_bounds__(256) grid_search_kernel(PairArgs A) {
  __shared__ int s_list[8][kMaxNeighbors];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (i >= A.n) return;  // whole warp
  int* list = s_list[w];
  double Xi[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < D; ++k) Xi[k] = A.X[(long long)i * D + k];
  int cc[3];
  grid_cell_of<D>(A, Xi, cc);
  // window per axis: 2 reach + 1 cells around the own cell, or the whole axis once
  int wk[3] = {1, 1, 1}, lo[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) {
    const int span = 2 * A.greach[k] + 1;
    if (span >= A.gnc[k]) {
      wk[k] = A.gnc[k];
    } else {
      wk[k] = span;
      lo[k] = cc[k] - A.greach[k];
    }
  }
  const int T = wk[0] * wk[1] * wk[2];
  const int n_over = min(*A.over_count, A.over_cap);
  int cnt = 0;
  for (int base = 0; base < T + n_over; base += 32) {
    const int t = base + lane;
    int j = -1;
    if (t < T) {
      int r = t, cell = 0, stride = 1;
      bool ok = true;
      for (int k = 0; k < D; ++k) {
        int c = lo[k] + r % wk[k];
        r /= wk[k];
        if (c < 0 || c >= A.gnc[k]) {
          if (A.g.per[k])
            c = (c % A.gnc[k] + A.gnc[k]) % A.gnc[k];
          else
            ok = false;
        }
        cell += stride * c;
        stride *= A.gnc[k];
      }
      if (ok) j = A.grid[cell];
    } else if (t < T + n_over) {
      j = A.over[t - T];
    }
    const bool hit = is_partner<D>(A, Xi, i, j);
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
    if (hit && pos < A.kmax) list[pos] = j;
    cnt += __popc(m);
  }
  store_partners(A, i, lane, list, cnt);
}

// Eq. 16 contact force on particle i from its sorted partner list (summed in index
// order) and from one mirror image per wall, then (in a time step) the particle update.
template <int D>
__device__ __forceinline__ void pair_force_body(const PairArgs& A, unsigned blk, int tid, int nthr) {
  const int i = (int)(blk * nthr + tid);
  if (i >= A.n) return;
  double Xi[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < D; ++k) Xi[k] = A.X[(long long)i * D + k];
  const int cnt = A.nbr_count[i];
  double F[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < cnt; ++a) {
    const int j = A.nbr[(long long)i * A.kmax + a];
    double Xj[3] = {0.0, 0.0, 0.0}, dx[3];
    for (int k = 0; k < D; ++k) Xj[k] = A.X[(long long)j * D + k];
    separation<D>(A, Xi, Xj, dx);
    const double d = sqrt(dist2_nofma(dx));
    const double mag = eq16_magnitude(A, d);
    if (d > 0.0 && mag != 0.0)
      for (int k = 0; k < D; ++k) F[k] += mag * dx[k] / d;
  }
  // walls: a mirror image through each wall (at -1/2 and L - 1/2 for halfway
  // bounce-back, on the nodes 0 and L - 1 for the extrapolation boundaries)
  for (int k = 0; k < D; ++k) {
    if (A.g.per[k]) continue;
    for (int s = 0; s < 2; ++s) {
      const double wall = (s == 0) ? A.wall_lo : A.L[k] - 1.0 - A.wall_lo;
      const double dk = 2.0 * (Xi[k] - wall);
      const double d = fabs(dk);
      const double mag = eq16_magnitude(A, d);
      if (d > 0.0 && mag != 0.0) F[k] += mag * dk / d;
    }
  }
  for (int k = 0; k < D; ++k) A.Fc[(long long)i * D + k] = F[k];
  if (A.integrate) advance_particle<D>(A, i, Xi, F);
}

template <int D, bool FUSED>
__global__ void __launch_bounds__(128) pair_force_kernel(PairArgs A0, Fuse FU) {
  IBMLBM_BIND(FUSED, PairArgs, A, A0, FU, blk);
  pair_force_body<D>(A, blk, (int)threadIdx.x, (int)blockDim.x);
}

// exclusive scan of n ints into out[0..n] (out[n] = total); one block of 1024 threads
__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ in, int* __restrict__ out,
                                                    int n) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 4096) {
    int v[4], sum = 0;
    for (int k = 0; k < 4; ++k) {
      const int idx = base + tid * 4 + k;
      v[k] = idx < n ? in[idx] : 0;
      sum += v[k];
    }
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int w = warp_tot[lane], wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      warp_tot[lane] = wi - w;  // exclusive prefix of the warp totals
    }
    __syncthreads();
    int run = carry + warp_tot[wid] + incl - sum;
    for (int k = 0; k < 4; ++k) {
      const int idx = base + tid * 4 + k;
      if (idx < n) out[idx] = run;
      run += v[k];
    }
    __syncthreads();
    if (tid == 1023) carry = run;
    __syncthreads();
  }
  if (tid == 0) out[n] = carry;
}

__global__ void pair_emit_kernel(PairArgs A, int* pairs, long long cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  long long o = A.gt_count[i];  // offsets after the scan
  const int cnt = A.nbr_count[i];
  for (int a = 0; a < cnt; ++a) {
    const int j = A.nbr[(long long)i * A.kmax + a];
    if (j <= i) continue;
    if (o < cap) {
      pairs[2 * o] = i;
      pairs[2 * o + 1] = j;
    }
    ++o;
  }
}

// ------------------------------------------------------------------ launchers
static unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_scan(const int* in, int* out, int n, cudaStream_t s) {
  scan_kernel<<<1, 1024, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_pair_cells(const PairArgs& A, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  if (A.grid_mode) {  // grid search: empty grid and overflow list, then the scatter
    const size_t gcells = (size_t)A.gnc[0] * A.gnc[1] * A.gnc[2];
    cudaError_t e = cudaMemsetAsync(A.grid, 0xff, sizeof(int) * gcells, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.over_count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const unsigned g = blocks_for(A.n, 256);
    if (A.D == 2)
      grid_scatter_kernel<2><<<g, 256, 0, s>>>(A);
    else
      grid_scatter_kernel<3><<<g, 256, 0, s>>>(A);
    return cudaGetLastError();
  }
  const size_t ncells = (size_t)A.nc[0] * A.nc[1] * A.nc[2];
  cudaError_t e = cudaMemsetAsync(A.cell_count, 0, sizeof(int) * ncells, s);
  if (e != cudaSuccess) return e;
  const unsigned g = blocks_for(A.n, 256);
  if (A.D == 2)
    pair_insert_kernel<2, false><<<g, 256, 0, s>>>(A, Fuse{});
  else
    pair_insert_kernel<3, false><<<g, 256, 0, s>>>(A, Fuse{});
  return cudaGetLastError();
}

// neighbour lists (warp per particle), then, when A.Fc is set, contact forces and the
// particle update (thread per particle)
// the partner lists alone (no force): they need only this step's centres, so a step
// can search beside its IBM kernels and leave the forces for later
cudaError_t launch_pair_search_lists(const PairArgs& A, cudaStream_t s) {
  PairArgs L = A;
  L.Fc = nullptr;
  return launch_pair_contacts(L, s);
}

// the forces of the partner lists (and, in a step, the particle update)
cudaError_t launch_pair_forces(const PairArgs& A, cudaStream_t s) {
  if (A.n == 0 || !A.Fc) return cudaSuccess;
  const unsigned g = blocks_for(A.n, 128);
  if (A.D == 2)
    pair_force_kernel<2, false><<<g, 128, 0, s>>>(A, Fuse{});
  else
    pair_force_kernel<3, false><<<g, 128, 0, s>>>(A, Fuse{});
  return cudaGetLastError();
}

cudaError_t launch_pair_contacts(const PairArgs& A, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  const unsigned gw = blocks_for((long long)A.n * 32, 256);
  if (A.grid_mode) {
    if (A.D == 2)
      grid_search_kernel<2><<<gw, 256, 0, s>>>(A);
    else
      grid_search_kernel<3><<<gw, 256, 0, s>>>(A);
  } else if (A.D == 2) {
    pair_search_kernel<2, false><<<gw, 256, 0, s>>>(A, Fuse{});
  } else {
    pair_search_kernel<3, false><<<gw, 256, 0, s>>>(A, Fuse{});
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !A.Fc) return e;
  const unsigned g = blocks_for(A.n, 128);
  if (A.D == 2)
    pair_force_kernel<2, false><<<g, 128, 0, s>>>(A, Fuse{});
  else
    pair_force_kernel<3, false><<<g, 128, 0, s>>>(A, Fuse{});
  return cudaGetLastError();
}

// ---------------------------------------------- fused over the members of a 2D batch
// zero each member's cell counts (one thread per cell)
__device__ __forceinline__ void pair_clear_body(const PairArgs& A, unsigned blk, int tid, int nthr) {
  const long long c = blk * (long long)nthr + tid;
  if (c < (long long)A.nc[0] * A.nc[1] * A.nc[2]) A.cell_count[c] = 0;
}

__global__ void pair_clear_kernel(Fuse FU) {
  IBMLBM_BIND(true, PairArgs, A, PairArgs{}, FU, blk);
  pair_clear_body(A, blk, (int)threadIdx.x, (int)blockDim.x);
}

unsigned pair_clear_blocks(const PairArgs& A) { return blocks_for((long long)A.nc[0] * A.nc[1] * A.nc[2], 256); }
unsigned pair_thread_blocks(int n, int b) { return n > 0 ? blocks_for(n, b) : 0; }
unsigned pair_warp_blocks(int n) { return n > 0 ? blocks_for((long long)n * 32, 256) : 0; }

// clear + insert + search + force for every member (the force blocks also advance the
// particles, as in a time step)
cudaError_t launch_pairs_fused(const Fuse& Fc, unsigned bc, const Fuse& Fi, unsigned bi,
                               const Fuse& Fs, unsigned bs, const Fuse& Ff, unsigned bf,
                               cudaStream_t s) {
  if (bc) pair_clear_kernel<<<bc, 256, 0, s>>>(Fc);
  if (bi) pair_insert_kernel<2, true><<<bi, 256, 0, s>>>(PairArgs{}, Fi);
  if (bs) pair_search_kernel<2, true><<<bs, 256, 0, s>>>(PairArgs{}, Fs);
  if (bf) pair_force_kernel<2, true><<<bf, 128, 0, s>>>(PairArgs{}, Ff);
  return cudaGetLastError();
}

// The contact phases of a batched step in one persistent kernel (cooperative launch,
// 256 threads a block): clear the members' cell counts, insert, search, then the
// contact force and particle update (128-thread virtual blocks, two per block), with a
// bounded grid barrier between the phases.
__global__ void __launch_bounds__(256, 2) pairs_batch_kernel(PairBatch P) {
  unsigned blk;
  // a barrier of an earlier launch gave up: its counts are stale until the host resets them
  if (__syncthreads_or(threadIdx.x == 0 && (*(volatile uint32_t*)P.status & ST_TIMEOUT))) return;
  for (unsigned vb = blockIdx.x; vb < P.nclear; vb += gridDim.x) {
    const PairArgs A = fused_args<PairArgs>(P.clear, vb, blk);
    pair_clear_body(A, blk, (int)threadIdx.x, 256);
  }
  if (!grid_barrier(P.bar, P.limit, P.status)) return;
  for (unsigned vb = blockIdx.x; vb < P.nins; vb += gridDim.x) {
    const PairArgs A = fused_args<PairArgs>(P.ins, vb, blk);
    pair_insert_body<2>(A, blk, (int)threadIdx.x, 256);
  }
  if (!grid_barrier(P.bar, P.limit, P.status)) return;
  for (unsigned vb = blockIdx.x; vb < P.nsearch; vb += gridDim.x) {
    const PairArgs A = fused_args<PairArgs>(P.search, vb, blk);
    pair_search_body<2>(A, blk);
  }
  if (!grid_barrier(P.bar, P.limit, P.status)) return;
  for (unsigned vb = blockIdx.x; 2 * vb < P.nforce; vb += gridDim.x) {
    const unsigned v = 2 * vb + (threadIdx.x >> 7);
    if (v >= P.nforce) continue;
    const PairArgs A = fused_args<PairArgs>(P.force, v, blk);
    pair_force_body<2>(A, blk, (int)(threadIdx.x & 127), 128);
  }
}

cudaError_t launch_pairs_batch(const PairBatch& P, cudaStream_t s) {
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pairs_batch_kernel, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  }
  const unsigned need = std::max({P.nclear, P.nins, P.nsearch, (P.nforce + 1) / 2, 1u});
  const unsigned grid = std::min(need, (unsigned)(per_sm * sms));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, pairs_batch_kernel, P);
}

cudaError_t launch_pair_compact(const PairArgs& A, int* pairs, long long cap, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  // gt_count[0..n) -> exclusive offsets in place via the scan (out may alias in only
  // element-wise per tile, so scan into the upper half of the same buffer first)
  cudaError_t e = launch_scan(A.gt_count, A.gt_count + (A.n + 1), A.n, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(A.gt_count, A.gt_count + (A.n + 1), sizeof(int) * (A.n + 1),
                      cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  pair_emit_kernel<<<blocks_for(A.n, 256), 256, 0, s>>>(A, pairs, cap);
  return cudaGetLastError();
}

}  // namespace ibmlbm

namespace ibmlbm {
unsigned long long check_fault_pairs() { return take_check_fault(); }
}  // namespace ibmlbm
