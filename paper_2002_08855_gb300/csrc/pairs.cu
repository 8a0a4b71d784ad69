// Cell-list pair search and short-range repulsive force (Sec. 5, Eq. 16).
//
// Cells of side H_k = L_k / nc_k >= D_p + zeta (a periodic axis with fewer than three
// cells becomes one cell), so every pair closer than D_p + zeta lies in the 3^D
// neighbourhood of a cell.  Cell lists come from a counting sort: count per cell
// (atomics), exclusive scan, scatter (atomics again, which leaves the counts at zero
// for the next step).  Each particle then scans its neighbourhood, keeps partners j
// with |X_i - X_j|^2 < (D_p + zeta)^2 -- squared distance summed in axis order in
// double precision without fused multiply-add, nearest image on periodic axes --
// sorts them by index and sums the Eq. 16 force in that order, so the result does
// not depend on the order of the cell lists.  The canonical pair list (i < j, sorted)
// is compacted from these per-particle lists on request.
#include <cmath>

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

template <int D>
__global__ void pair_count_kernel(PairArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  atomicAdd(&A.cell_count[cell_of<D>(A, i)], 1);
}

template <int D>
__global__ void pair_fill_kernel(PairArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int c = cell_of<D>(A, i);
  const int slot = A.cell_start[c] + atomicSub(&A.cell_count[c], 1) - 1;
  A.sorted[slot] = i;
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

template <int D>
__global__ void pair_contact_kernel(PairArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  double Xi[3] = {0.0, 0.0, 0.0};
  int cc[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) {
    Xi[k] = A.X[(long long)i * D + k];
    cc[k] = cell_coord(Xi[k], A.H[k], A.nc[k]);
  }
  int list[kMaxNeighbors];
  int cnt = 0;
  for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        const int off[3] = {ox, oy, oz};
        int cell = 0, stride = 1;
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
        if (!ok) continue;
        for (int s = A.cell_start[cell]; s < A.cell_start[cell + 1]; ++s) {
          const int j = A.sorted[s];
          if (j == i) continue;
          double Xj[3] = {0.0, 0.0, 0.0}, dx[3];
          for (int k = 0; k < D; ++k) Xj[k] = A.X[(long long)j * D + k];
          separation<D>(A, Xi, Xj, dx);
          if (dist2_nofma(dx) < A.thr2) {
            if (cnt < A.kmax) list[cnt] = j;
            ++cnt;
          }
        }
      }
  if (cnt > A.kmax) {
    atomicOr(A.status, ST_CAPACITY);
    cnt = A.kmax;
  }
  for (int a = 1; a < cnt; ++a) {  // insertion sort by partner index
    const int v = list[a];
    int b = a - 1;
    while (b >= 0 && list[b] > v) {
      list[b + 1] = list[b];
      --b;
    }
    list[b + 1] = v;
  }
  int gt = 0;
  for (int a = 0; a < cnt; ++a) {
    A.nbr[(long long)i * A.kmax + a] = list[a];
    gt += list[a] > i;
  }
  A.nbr_count[i] = cnt;
  A.gt_count[i] = gt;
  if (!A.Fc) return;
  double F[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < cnt; ++a) {
    const int j = list[a];
    double Xj[3] = {0.0, 0.0, 0.0}, dx[3];
    for (int k = 0; k < D; ++k) Xj[k] = A.X[(long long)j * D + k];
    separation<D>(A, Xi, Xj, dx);
    const double d = sqrt(dist2_nofma(dx));
    const double mag = eq16_magnitude(A, d);
    if (d > 0.0 && mag != 0.0)
      for (int k = 0; k < D; ++k) F[k] += mag * dx[k] / d;
  }
  // walls: a mirror image through each wall at -1/2 and L - 1/2
  for (int k = 0; k < D; ++k) {
    if (A.g.per[k]) continue;
    for (int s = 0; s < 2; ++s) {
      const double wall = (s == 0) ? -0.5 : A.L[k] - 0.5;
      const double dk = 2.0 * (Xi[k] - wall);
      const double d = fabs(dk);
      const double mag = eq16_magnitude(A, d);
      if (d > 0.0 && mag != 0.0) F[k] += mag * dk / d;
    }
  }
  for (int k = 0; k < D; ++k) A.Fc[(long long)i * D + k] = F[k];
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
  const unsigned g = blocks_for(A.n, 256);
  const int ncells = A.nc[0] * A.nc[1] * A.nc[2];
  if (A.D == 2)
    pair_count_kernel<2><<<g, 256, 0, s>>>(A);
  else
    pair_count_kernel<3><<<g, 256, 0, s>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan(A.cell_count, A.cell_start, ncells, s);
  if (e != cudaSuccess) return e;
  if (A.D == 2)
    pair_fill_kernel<2><<<g, 256, 0, s>>>(A);
  else
    pair_fill_kernel<3><<<g, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_pair_contacts(const PairArgs& A, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  const unsigned g = blocks_for(A.n, 128);
  if (A.D == 2)
    pair_contact_kernel<2><<<g, 128, 0, s>>>(A);
  else
    pair_contact_kernel<3><<<g, 128, 0, s>>>(A);
  return cudaGetLastError();
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
