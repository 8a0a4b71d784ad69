// Shared device-side definitions of the IB-LBM hot path (sm_103a).
//
// Lattices D2Q9 (Eq. 2) and D3Q19 (Eq. 3; the printed z row drops one entry,
// e_9 = (-1, 0, 1) restores e_a = -e_{a-9}), weights as listed after Eq. 4.
// Units: dh = dt = 1, cs^2 = 1/3, rho_0 = rho_f = 1.
//
// Data layout in HBM (one workspace, carved by the host):
//   f      [Q][Np] PDFs (FP32, or FP16 / BF16 holding f / w), one copy, AA-pattern
//                  in-place streaming; Np = N rounded up to 64, 64 elements of slack
//   ustar  [N][4]  float  3D: u* = sum_a e_a f_a on the marked nodes (2D keeps u* of
//                         each particle's node box instead)
//   fib    float  IB force density, zero outside the IBM phase: 2D [N][2],
//                 3D [N][4] (fourth component unused)
//   mask   [2][rows][wpr] u32  3D, one per step parity, one bit per node: the nodes
//                           within R + 2 sqrt(3) of a particle centre (support of every
//                           Lagrangian point and the particle interior)
//   particle state in double, Lagrangian point data [npts][D]; point positions as
//   32.32 fixed-point int64 (integer part = node anchor, low word = fraction), so
//   per-point work needs no double-precision arithmetic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ibmlbm {

// ------------------------------------------------------------ bounds-checked build
// Compiled with -DIBMLBM_CHECKED (libibmlbm_checked.so), every global index a kernel
// forms from the geometry or from particle positions is checked against its array's
// extent before the access; a failed check skips the access and records the source
// line and the index in this translation unit's fault word (first failure wins), which
// ibm_lbm_sync reports as IBMLBM_ERR_BOUNDS.  Nothing traps.  In the ordinary build
// the checks compile to nothing.
#ifdef IBMLBM_CHECKED
static __device__ unsigned long long g_check_fault;
__device__ __forceinline__ bool check_index(long long i, long long n, int line) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_check_fault, 0ull,
            (1ull << 63) | ((unsigned long long)(line & 0x7fffff) << 40) | ((unsigned long long)i & 0xffffffffffull));
  return false;
}
#define IBMLBM_CHK(i, n) (::ibmlbm::check_index((long long)(i), (long long)(n), __LINE__))
#else
#define IBMLBM_CHK(i, n) true
#endif

// this translation unit's fault word, cleared after reading (0: no failure, or the
// ordinary build)
static inline unsigned long long take_check_fault() {
#ifdef IBMLBM_CHECKED
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_check_fault, sizeof(v)) != cudaSuccess) return 0;
  if (v) cudaMemcpyToSymbol(g_check_fault, &z, sizeof(z));
  return v;
#else
  return 0;
#endif
}

// device status word bits
enum : uint32_t {
  ST_NONFINITE = 1u,
  ST_OUT_OF_DOMAIN = 2u,
  ST_CAPACITY = 4u,
  ST_TIMEOUT = 8u,  // a grid barrier of a persistent kernel gave up waiting
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
  long long Np;    // stride of the PDF planes: N rounded up to 64 elements
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
// the same sum over the lanes of each half-warp (every lane of the warp takes part)
__device__ __forceinline__ FF ff_half_sum(FF s) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, s.hi, o);
    const float l = __shfl_xor_sync(0xffffffffu, s.lo, o);
    ff_add(s, h);
    s.lo += l;
  }
  return s;
}
__device__ __forceinline__ double ff_value(FF s) { return (double)s.hi + (double)s.lo; }

// Row pitch (in cells) of a 2D particle box of side S: at least S, and 4 or 12 modulo
// 16, so the 16 cells of a 4 x 4 support of float2 cells use 16 different bank pairs.
__host__ __device__ inline int box_pitch(int S) {
  int p = S;
  while ((p & 15) != 4 && (p & 15) != 12) ++p;
  return p;
}

// ------------------------------------------------------------ kernel arguments
struct LbmArgs {
  Geo g;
  void* f;           // PDFs, element type by store
  int store;         // STORE_F32, STORE_F16 or STORE_BF16 (pdf_access.cuh)
  float* ustar;
  float* fib;
  uint32_t* mask;
  float omega;       // 1 / tau
  float kforce;      // 1 - omega / 2 (Eq. 8 prefactor)
  float body[3];     // uniform body force
  int boundary;      // 0 halfway bounce-back, 1 extrapolation walls, 2 extrapolation channel
  float u_inlet;     // peak inlet velocity (boundary 2)
};

struct IbmArgs {
  Geo g;
  int D;             // dimension
  int np, nl;
  long long npts;
  int delta_kind;    // 4: Peskin's 4-point delta, 3: the 3-point delta
  double radius;     // D_p / 2
  float radius_f;    // D_p / 2 as float
  int rcell;         // ceil(D_p / 2)
  float dV;          // point volume (Eq. 13 reading)
  int box;           // side of the spreading box (nodes)
  float mark_radius; // 3D: radius of the marked ball (u* is valid inside it)
  const float* ustar;    // 3D: u* on flagged nodes (lbm_moments)
  float* fib;
  const void* f;         // 2D: the PDFs, for u* of each particle's box
  int store;             // their storage (STORE_F32, STORE_F16, STORE_BF16)
  int parity;            // 2D: AA parity of the PDFs
  float* ubox;           // 2D: [np][box][box_pitch(box)] float2, u* of each particle's box
  const int* order;      // 2D: the particle each warp slot of the IBM kernels takes
  const long long* Xb;  // [npts][D] fixed point
  const float* Ub;   // [npts][D]
  float* Fb;         // [npts][D] sum of MDF increments
  float* dFb;        // [npts][D] increment of the current iteration
  float* ubs;        // [npts][D] D_I u*
  const double* Xc;  // [np][D] centres of the current step
  const long long* Xcf;  // [np][D] fixed point centres
  const float* ref_f;    // [nl][D] offsets of the points from the centre
  double* Pint;      // [np][D] interior momentum
  double* Lint;      // [np][3] interior angular momentum
  double* FhN;       // [np][D] -dV sum_b F_b of this step
  double* ThN;       // [np][3] -dV sum_b r_b x F_b of this step
  float* res;        // [npts][D] U_b - D_I u^(M) (residual pass)
  const float* frame3;  // 3D learned initializer: [nl][3][3] rows n, t1, t2 of each point
  const int* nbr3;      // 3D learned initializer: [nl][8] stencil neighbours of each point
  const int* slist;     // 3D: [slen] cells (lx | ly << 5 | lz << 10) of the node box that
  int slen;             //   can be a support node (null, 0: stage by rows)
  float shell_h;        // 3D: support half-width (2 for the 4-point delta, 1.5 for the 3-point)
  float shell_lo2, shell_hi2;  // 3D: squared radii bounding the points' distance from the centre
  uint32_t* status;
};

// Regeneration of the Lagrangian points and marking of the nodes near each particle.
struct RegenArgs {
  Geo g;
  int D;
  int np, nl;
  float mark_radius;   // radius of the marked ball (float, already padded)
  const long long* ref_fix;  // [nl][D] offsets of the points, fixed point
  const float* ref_f;        // [nl][D] offsets of the points, float
  const double* X;     // [np][D] (used to refresh the fixed-point centres when init != 0)
  const double* U;     // [np][D]
  const double* Om;    // [np][3]
  long long* Xcf;      // [np][D] fixed-point centres
  float* Uf;           // [np][D] single-precision velocity
  float* Omf;          // [np][3] single-precision angular velocity
  long long* Xb_out;   // [npts][D] fixed-point points
  float* Ub_out;       // [npts][D]
  uint32_t* mask;
};

// Per-particle double-precision state advanced by the contact kernel (Eq. 14-15).
struct PartState {
  double* Xnew;        // [np][D] centres after the step (the other buffer)
  double* U;           // [np][D]
  double* Om;          // [np][3]
  double* Fh;          // [np][D] F_h of the last step (reported)
  double* Th;          // [np][3]
  double* acc;         // [np][D] previous linear acceleration
  double* alp;         // [np][3] previous angular acceleration
  double* Pprev;       // [np][D] interior momentum of the previous step
  double* Lprev;       // [np][3]
  const double* FhN;   // [np][D] this step's F_h
  const double* ThN;   // [np][3]
  const double* Pint;  // [np][D] this step's interior momentum
  const double* Lint;  // [np][3]
  long long* Xcf;      // [np][D] fixed-point centres for the regeneration
  float* Uf;           // [np][D]
  float* Omf;          // [np][3]
  double Mp, meff, Ip, Kt, Kr;
  double grav[3];
  int fixed;
};

// ------------------------------------------------------------ fused launches
// A batch steps many independent runs (its members) together, and each kernel then
// runs once for all members: block b of the launch belongs to member cav[b] and is
// block b - first[cav[b]] of that member's own grid.  args holds the members'
// argument structs (in device memory).
// Programmatic dependent launch (sm_90 and later): a kernel launched with programmatic
// stream serialization can be scheduled while its predecessor in the stream is still
// running.  It calls pdl_enter() before its first global memory access: the wait
// returns once the predecessor grid has completed and its writes are visible, then the
// kernel lets its own successor be scheduled.  Under an ordinary launch both
// instructions return at once, so the kernels call it unconditionally.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// host: launch with programmatic stream serialization (the kernel must call pdl_enter
// before touching global memory)
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}

struct Fuse {
  const void* args;   // [members]
  const int* cav;     // [blocks]
  const int* first;   // [members]
};

// The argument struct of virtual block vb of a fused block map, and (blk) the block's
// index in its member's grid (the persistent kernels walk the virtual blocks).
template <class T>
__device__ __forceinline__ T fused_args(const Fuse& F, unsigned vb, unsigned& blk) {
  const int m = F.cav[vb];
  blk = vb - (unsigned)F.first[m];
  return static_cast<const T*>(F.args)[m];
}

// Grid-wide barrier of a persistent kernel launched cooperatively (every block of the
// grid is resident).  bar[0] counts the blocks that arrived, bar[1] is the generation;
// the host zeroes both before each launch.  The wait is bounded: after `limit` polls
// (a short sleep each) the block sets ST_TIMEOUT in *status and the barrier returns
// false, and the caller returns (every other block then gives up at the same barrier
// or the next).  Writes before the barrier are visible to every block after it.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned long long limit, uint32_t* status) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long polls = 0;
      while (*gen == g) {
        if (++polls > limit) {
          atomicOr(status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(200);
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

// In a kernel templated on bool FUSED: A = this block's argument struct (the kernel
// parameter A0 for a single run; for a member, a local copy, so the fields the kernel
// uses are loaded once instead of at every use), BLK = the block's index in its
// member's grid.
#define IBMLBM_BIND(FUSED, TYPE, A, A0, F, BLK)                                        \
  const int bind_m_ = (FUSED) ? (F).cav[blockIdx.x] : 0;                             \
  const TYPE bind_copy_ = (FUSED) ? static_cast<const TYPE*>((F).args)[bind_m_] : TYPE{}; \
  const TYPE& A = (FUSED) ? bind_copy_ : (A0);                                       \
  const unsigned BLK = (FUSED) ? blockIdx.x - (unsigned)(F).first[bind_m_] : blockIdx.x

// Capacity of one search-cell bucket: eight times the mean occupancy plus eight
// (at least 16); a bucket that overflows is reported as CAPACITY.
inline int cell_capacity(long long n, long long ncells) {
  long long mean = (n + ncells - 1) / (ncells > 0 ? ncells : 1);
  long long cap = 8 * mean + 8;
  if (cap < 16) cap = 16;
  if (cap > n && n >= 16) cap = n;
  return (int)cap;
}

struct PairArgs {
  Geo g;
  int D;
  int n;
  int nc[3];
  double H[3];
  double L[3];
  double diam, zeta, thr2;
  double c_ij, eps_pp, E_pp;
  double wall_lo;       // wall positions on a non-periodic axis: wall_lo and L - 1 - wall_lo
  int kmax;
  const double* X;      // [n][D]
  int* cell_count;      // [ncells], zero before the insertion
  int* cell_ids;        // [ncells][cell_cap]
  int cell_cap;         // bucket capacity (cell_capacity)
  int* nbr;             // [n][kmax]
  int* nbr_count;       // [n]
  double* Fc;           // [n][D] (null: pair list only)
  int* gt_count;        // [2 (n + 1)] partners j > i, then their offsets
  uint32_t* status;
  int grid_mode;        // 1: grid search (one particle per cell) instead of cell buckets
  int* grid;            // [gnc cells] particle index or -1
  int gnc[3];           // grid cells per axis (side gH < D_p / sqrt(D))
  double gH[3];
  int greach[3];        // cells scanned on each side of the own cell
  int* over;            // [over_cap] particles whose grid cell was taken
  int* over_count;
  int over_cap;
  int integrate;        // 1: advance the particles (PartState) after the contact force
  int have_prev;        // a previous step exists (history terms of the update)
  PartState ps;
};

// The persistent kernels of a batched step: the fused block maps of their phases, the
// number of virtual blocks of each, and the bounded grid barrier's state.
struct PairBatch {
  Fuse clear, ins, search, force;
  unsigned nclear, nins, nsearch, nforce;  // virtual blocks (force: 128 threads each)
  unsigned* bar;
  unsigned long long limit;
  uint32_t* status;
};

struct IbmBatch {
  Fuse regen;     // RegenArgs: this step's points (Lagrangian regeneration)
  Fuse warp;      // IbmArgs: interpolation and spreading, one warp per particle
  Fuse lane;      // IbmArgs: the sums of the hydrodynamic force and interior momentum
  unsigned nwarp, nlane;
  int mdf;
  int wfloats;    // shared-memory floats per warp (set by the launcher)
  unsigned* bar;
  unsigned long long limit;
  uint32_t* status;
};

}  // namespace ibmlbm
