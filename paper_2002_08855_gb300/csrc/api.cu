// C ABI of libibmlbm.so (declared in include/ibmlbm.h): configuration checks,
// workspace layout, the per-step kernel sequence and its CUDA-graph replay.
//
// One step (Sec. 3 step list, Sec. 6.2 part list; explicit particle coupling):
//   lbm_moments -> [ibm_interp -> ibm_spread] x M -> ibm_forces (F_h, T_h, interior
//   momentum) -> lbm_step -> pair cells (buckets) -> pair contacts + particle update
//   -> regen (points and node marks of the next step)
// All of it is enqueued on the caller's stream; after the first step each step
// parity is captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "ibmlbm.h"
#include "common.cuh"
#include "launch.h"
#include "pair_grid.h"
#include "mlp.h"

using namespace ibmlbm;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(IBMLBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Bounds-checked build: the first failed index check of any translation unit since
// the last call, reported as IBMLBM_ERR_BOUNDS (the ordinary build has none).
int report_check_faults() {
  const unsigned long long f[3] = {check_fault_lbm(), check_fault_ibm(), check_fault_pairs()};
  const char* unit[3] = {"lbm.cu", "ibm.cu", "pairs.cu"};
  for (int k = 0; k < 3; ++k) {
    if (!f[k]) continue;
    char msg[160];
    std::snprintf(msg, sizeof(msg), "index check failed in %s line %llu (index %llu)", unit[k],
                  (f[k] >> 40) & 0x7fffffull, f[k] & 0xffffffffffull);
    return fail(IBMLBM_ERR_BOUNDS, msg);
  }
  return IBMLBM_OK;
}

struct Carver {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = align_up(off + (bytes ? bytes : 1));
    return o;
  }
};

struct Derived {
  int D, Q;
  Geo g;
  long long npts;
  int kmax;
  int nc[3];
  double H[3], L[3];
  int gnc[3], greach[3];  // grid search (pair_search 1): cells per axis, cells scanned per side
  double gH[3];
  long long gcells;
  int over_cap;
  int box, rcell;
  double radius, dV, Mp, meff, Ip, Kt, Kr, c_ij, thr2;
  float mark_radius;
  int slen;  // 3D: entries of the staging list (0: none)
};

struct Layout {
  size_t f, ustar, fib, mask;
  size_t X0, X1, U, Om, Fh, Th, FhN, ThN, acc, alp, Pint, Lint, Pprev, Lprev, Fc;
  size_t Uf, Omf, ref_fix, ref_f, Xcf, Xb0, Xb1, Ub0, Ub1, Fb, dFb, ubs, ubox, res, mlp, mlp_img;
  size_t frame3, nbr3, slist, order;
  size_t cell_count, cell_ids, nbr, nbr_count, gt, pairs, status;
  size_t grid, over, over_count;
  size_t total;
};

int check_config(const ibm_lbm_config* c) {
  if (!c) return fail(IBMLBM_ERR_INVALID_ARG, "config is NULL");
  if (c->struct_size != sizeof(ibm_lbm_config))
    return fail(IBMLBM_ERR_INVALID_ARG, "config.struct_size does not match this library");
  if (c->dim != 2 && c->dim != 3) return fail(IBMLBM_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (c->nx < 1 || c->ny < 1 || c->nz < 1 || (c->dim == 2 && c->nz != 1))
    return fail(IBMLBM_ERR_INVALID_ARG, "node counts must be >= 1 (nz = 1 in 2D)");
  if ((double)c->nx * c->ny * c->nz > 4.0e9)
    return fail(IBMLBM_ERR_INVALID_ARG, "lattice larger than 4e9 nodes");
  if (!(c->tau > 0.5) || !std::isfinite(c->tau))
    return fail(IBMLBM_ERR_INVALID_ARG, "tau must be > 1/2");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(c->body_force[k]) || !std::isfinite(c->gravity[k]))
      return fail(IBMLBM_ERR_INVALID_ARG, "body force and gravity must be finite");
  if (c->n_particles < 0) return fail(IBMLBM_ERR_INVALID_ARG, "n_particles < 0");
  if (c->max_neighbors < 0 || c->max_neighbors > 64)
    return fail(IBMLBM_ERR_INVALID_ARG, "max_neighbors must be in 0..64");
  if (c->pdf_storage < IBMLBM_PDF_FP32 || c->pdf_storage > IBMLBM_PDF_BF16)
    return fail(IBMLBM_ERR_INVALID_ARG, "pdf_storage must be 0 (FP32), 1 (FP16) or 2 (BF16)");
  if (c->mlp_init != 0 && c->mlp_init != 1) return fail(IBMLBM_ERR_INVALID_ARG, "mlp_init must be 0 or 1");
  if (c->mlp_init && (c->mdf_iters < 1 || (c->dim == 2 && c->n_lag > mlp_max_points())))
    return fail(IBMLBM_ERR_UNSUPPORTED,
                "the learned initializer needs mdf_iters >= 1 (and n_lag <= 256 in 2D)");
  if (c->boundary < 0 || c->boundary > 2) return fail(IBMLBM_ERR_INVALID_ARG, "boundary must be 0, 1 or 2");
  if (c->boundary) {
    const int32_t nn[3] = {c->nx, c->ny, c->nz};
    for (int k = 0; k < c->dim; ++k)
      if (!c->periodic[k] && nn[k] < 3)
        return fail(IBMLBM_ERR_INVALID_ARG, "extrapolation boundaries need n >= 3 on every wall axis");
    if (c->boundary == 2 && c->periodic[1])
      return fail(IBMLBM_ERR_INVALID_ARG, "a channel (boundary 2) needs a non-periodic y axis");
    if (!std::isfinite(c->u_inlet)) return fail(IBMLBM_ERR_INVALID_ARG, "u_inlet must be finite");
  }
  if (c->pair_search != 0 && c->pair_search != 1)
    return fail(IBMLBM_ERR_INVALID_ARG, "pair_search must be 0 or 1");
  if (c->pair_search == 1 && c->n_particles > 0 && c->diameter > 0.0) {
    double cells = 1.0;
    const double L3[3] = {(double)c->nx, (double)c->ny, (double)c->nz};
    for (int k = 0; k < c->dim; ++k) cells *= std::ceil(L3[k] / (c->diameter / std::sqrt((double)c->dim)));
    if (cells > 1.0e9) return fail(IBMLBM_ERR_UNSUPPORTED, "grid search needs more than 1e9 cells");
  }
  if (c->n_particles > 0) {
    if (c->n_lag < 1) return fail(IBMLBM_ERR_INVALID_ARG, "n_lag must be >= 1");
    if (!(c->diameter > 0.0)) return fail(IBMLBM_ERR_INVALID_ARG, "diameter must be > 0");
    if (c->delta_kind != 4 && c->delta_kind != 3)
      return fail(IBMLBM_ERR_UNSUPPORTED, "delta_kind must be 4 or 3");
    if (!(c->drs > 0.0)) return fail(IBMLBM_ERR_INVALID_ARG, "drs must be > 0");
    if (c->mdf_iters < 0) return fail(IBMLBM_ERR_INVALID_ARG, "mdf_iters must be >= 0");
    if (!(c->density_ratio > 0.0))
      return fail(IBMLBM_ERR_INVALID_ARG, "density_ratio must be > 0");
    if (!(c->zeta > 0.0) || !(c->eps_pp > 0.0) || !(c->E_pp > 0.0))
      return fail(IBMLBM_ERR_INVALID_ARG, "zeta, eps_pp and E_pp must be > 0");
    if (c->fixed_particles < 0 || c->fixed_particles > 2)
      return fail(IBMLBM_ERR_INVALID_ARG, "fixed_particles must be 0, 1 or 2");
  }
  return IBMLBM_OK;
}

// Staging list of a 3D sphere's node box: the cells (lx | ly << 5 | lz << 10) that are
// a support node of some point of the sphere for some position of its centre within
// its anchor cell.  Cell l lies k = l - (rcell + 2) nodes from the anchor; with the
// centre at anchor + fr, fr in [0, 1)^3, the node is a support node of the surface
// point c + y (|y| = R) iff y lies in the cube of half-width h around k - fr (h = 2
// for the 4-point delta, 1.5 for the nonzero weights of the 3-point one), so over all
// fr the cube [k - 1 - h, k + h]^3 must meet the sphere.  The margin of 0.02 is wider
// than the one of the test each block makes with its own fr.  Empty where the box
// side passes 32 or the offsets of a box could pass 2^31.
std::vector<int> stage3_list(const Derived& d, int delta_kind) {
  std::vector<int> out;
  const int S = d.box;
  if (d.D != 3 || S > 32 || (double)d.g.nx * d.g.ny * S >= 2147483647.0) return out;
  const double h = delta_kind == 3 ? 1.5 : 2.0, Rlo = std::max(0.0, d.radius - 0.02), Rhi = d.radius + 0.02;
  for (int lz = 0; lz < S; ++lz)
    for (int ly = 0; ly < S; ++ly)
      for (int lx = 0; lx < S; ++lx) {
        const int l[3] = {lx, ly, lz};
        double dmin2 = 0.0, dmax2 = 0.0;
        for (int a = 0; a < 3; ++a) {
          const double k = l[a] - (d.rcell + 2), lo = k - 1.0 - h, hi = k + h;
          const double e = lo > 0.0 ? lo : (hi < 0.0 ? -hi : 0.0), g = std::max(std::fabs(lo), std::fabs(hi));
          dmin2 += e * e;
          dmax2 += g * g;
        }
        if (dmin2 <= Rhi * Rhi && dmax2 >= Rlo * Rlo) out.push_back(lx | ly << 5 | lz << 10);
      }
  return out;
}

Derived derive(const ibm_lbm_config* c) {
  Derived d{};
  d.D = c->dim;
  d.Q = c->dim == 2 ? 9 : 19;
  d.g.nx = c->nx;
  d.g.ny = c->ny;
  d.g.nz = c->dim == 2 ? 1 : c->nz;
  for (int k = 0; k < 3; ++k) d.g.per[k] = c->periodic[k] ? 1 : 0;
  if (c->dim == 2) d.g.per[2] = 0;
  d.g.rows = d.g.ny * d.g.nz;
  d.g.wpr = (d.g.nx + 31) / 32;
  d.g.N = (long long)d.g.nx * d.g.ny * d.g.nz;
  d.g.Np = (d.g.N + 63) / 64 * 64;
  d.npts = (long long)c->n_particles * c->n_lag;
  d.kmax = c->max_neighbors ? c->max_neighbors : 32;
  d.L[0] = c->nx;
  d.L[1] = c->ny;
  d.L[2] = d.g.nz;
  const double Dp = c->diameter;
  d.radius = 0.5 * Dp;
  // superset of every support node (within 2 sqrt(D) of a surface point) and of the
  // interior; the 0.05 margin absorbs single-precision rounding of the marking test
  d.mark_radius = (float)(d.radius + 2.0 * std::sqrt((double)d.D) + 0.05);
  d.rcell = (int)std::ceil(d.radius);
  d.box = 2 * d.rcell + 6;
  cell_grid(d.D, d.L, d.g.per, Dp + c->zeta, d.nc, d.H);
  // grid search (Eq. 49): the largest side below D_p / sqrt(D) that tiles each axis
  d.gcells = 0;
  if (c->pair_search == 1 && c->n_particles > 0) {
    const double hmax = Dp / std::sqrt((double)d.D) * (1.0 - 1e-12);
    d.gcells = 1;
    for (int k = 0; k < 3; ++k) {
      d.gnc[k] = 1;
      d.gH[k] = k < d.D ? d.L[k] : 1.0;
      d.greach[k] = 0;
      if (k >= d.D) continue;
      d.gnc[k] = std::max(1, (int)std::ceil(d.L[k] / hmax));
      d.gH[k] = d.L[k] / d.gnc[k];
      d.greach[k] = (int)std::ceil((Dp + c->zeta) / d.gH[k]);
      d.gcells *= d.gnc[k];
    }
    d.over_cap = std::min(c->n_particles, std::max(256, c->n_particles / 16));
  }
  // Eq. 13 point volume: 2D ds * drs with ds = pi D / N_L; 3D (pi D^2 / N_L) * drs
  if (c->n_lag > 0)
    d.dV = (d.D == 2 ? kPi * Dp / c->n_lag : kPi * Dp * Dp / c->n_lag) * c->drs;
  const double V = d.D == 2 ? kPi * Dp * Dp / 4.0 : kPi * Dp * Dp * Dp / 6.0;
  d.Mp = c->density_ratio * V;
  d.meff = d.Mp - V;
  d.Ip = d.D == 2 ? d.Mp * Dp * Dp / 8.0 : d.Mp * Dp * Dp / 10.0;
  d.Kt = c->n_lag * d.dV;
  d.Kr = d.Kt * d.radius * d.radius * (d.D == 2 ? 1.0 : 2.0 / 3.0);
  const double g2 = c->gravity[0] * c->gravity[0] + c->gravity[1] * c->gravity[1] +
                    c->gravity[2] * c->gravity[2];
  d.c_ij = std::fabs((c->density_ratio - 1.0) * V) * std::sqrt(g2);
  const double thr = Dp + c->zeta;
  d.thr2 = thr * thr;
  d.slen = c->n_particles > 0 ? (int)stage3_list(d, c->delta_kind).size() : 0;
  return d;
}

Layout carve(const ibm_lbm_config* c, const Derived& d) {
  Layout l{};
  Carver cv;
  const size_t N = (size_t)d.g.N, np = (size_t)c->n_particles, D = d.D;
  const size_t npts = (size_t)d.npts;
  l.f = cv.take((c->pdf_storage == IBMLBM_PDF_FP32 ? 4 : 2) * ((size_t)d.Q * d.g.Np + 64));
  l.ustar = cv.take(D == 3 ? sizeof(float) * 4 * N : 0);  // 3D [N][4]; 2D keeps u* per particle box
  // 2D [N][2] (none in a run without particles), 3D [N][4]
  l.fib = cv.take(D == 3 ? sizeof(float) * 4 * N : (np > 0 ? sizeof(float) * 2 * N : 0));
  l.mask = cv.take(D == 3 ? 2 * sizeof(uint32_t) * (size_t)d.g.rows * d.g.wpr : 0);  // 3D, one per parity
  l.X0 = cv.take(sizeof(double) * np * D);
  l.X1 = cv.take(sizeof(double) * np * D);
  l.U = cv.take(sizeof(double) * np * D);
  l.Om = cv.take(sizeof(double) * np * 3);
  l.Fh = cv.take(sizeof(double) * np * D);
  l.Th = cv.take(sizeof(double) * np * 3);
  l.FhN = cv.take(sizeof(double) * np * D);
  l.ThN = cv.take(sizeof(double) * np * 3);
  l.Uf = cv.take(sizeof(float) * np * D);
  l.Omf = cv.take(sizeof(float) * np * 3);
  l.acc = cv.take(sizeof(double) * np * D);
  l.alp = cv.take(sizeof(double) * np * 3);
  l.Pint = cv.take(sizeof(double) * np * D);
  l.Lint = cv.take(sizeof(double) * np * 3);
  l.Pprev = cv.take(sizeof(double) * np * D);
  l.Lprev = cv.take(sizeof(double) * np * 3);
  l.Fc = cv.take(sizeof(double) * np * D);
  l.ref_fix = cv.take(sizeof(long long) * (size_t)c->n_lag * D);
  l.ref_f = cv.take(sizeof(float) * (size_t)c->n_lag * D);
  l.Xcf = cv.take(sizeof(long long) * np * D);
  l.Xb0 = cv.take(sizeof(long long) * npts * D);
  l.Xb1 = cv.take(sizeof(long long) * npts * D);
  l.Ub0 = cv.take(sizeof(float) * npts * D);
  l.Ub1 = cv.take(sizeof(float) * npts * D);
  l.Fb = cv.take(sizeof(float) * npts * D);
  l.dFb = cv.take(sizeof(float) * npts * D);
  l.ubs = cv.take(sizeof(float) * npts * D);
  l.res = cv.take(sizeof(float) * npts * D);                 // residual pass
  l.mlp = cv.take(sizeof(float) * kMlpParams);               // learned initializer
  l.mlp_img = cv.take(mlp_image_bytes());
  // 3D stencil of the learned initializer: frames [nl][9] and neighbours [nl][8]
  l.frame3 = cv.take(D == 3 ? sizeof(float) * 9 * (size_t)c->n_lag : 0);
  l.nbr3 = cv.take(D == 3 ? sizeof(int) * 8 * (size_t)c->n_lag : 0);
  l.slist = cv.take(sizeof(int) * (size_t)d.slen);  // 3D staging list of the node box
  // 2D: u* of each particle's node box (box rows of box_pitch(box) float2 cells)
  l.ubox = cv.take(D == 2 ? sizeof(float) * np * 2 * (size_t)d.box * box_pitch(d.box) : 0);
  l.order = cv.take(D == 2 ? sizeof(int) * np : 0);  // 2D IBM processing order
  const size_t ncells = (size_t)d.nc[0] * d.nc[1] * d.nc[2];
  l.cell_count = cv.take(sizeof(int) * ncells);
  l.cell_ids = cv.take(sizeof(int) * ncells * cell_capacity(c->n_particles, (long long)ncells));
  l.nbr = cv.take(sizeof(int) * np * d.kmax);
  l.nbr_count = cv.take(sizeof(int) * np);
  l.gt = cv.take(sizeof(int) * 2 * (np + 1));
  l.pairs = cv.take(sizeof(int) * np * d.kmax);
  l.status = cv.take(sizeof(uint32_t));
  l.grid = cv.take(sizeof(int) * (size_t)d.gcells);
  l.over = cv.take(d.gcells ? sizeof(int) * (size_t)d.over_cap : 0);
  l.over_count = cv.take(d.gcells ? sizeof(int) : 0);
  l.total = cv.off;
  return l;
}

// Lagrangian point offsets from the centre: circle theta_k = 2 pi k / N_L (2D) and
// the Fibonacci sphere z_k = 1 - (2k+1)/N_L, phi_k = k pi (3 - sqrt 5) (3D), radius D/2.
std::vector<double> reference_points(int D, int nl, double R) {
  std::vector<double> r((size_t)nl * D);
  for (int k = 0; k < nl; ++k) {
    if (D == 2) {
      const double th = 2.0 * kPi * k / nl;
      r[2 * k] = R * std::cos(th);
      r[2 * k + 1] = R * std::sin(th);
    } else {
      const double zk = 1.0 - (2.0 * k + 1.0) / nl;
      const double rho = std::sqrt(1.0 - zk * zk);
      const double ph = k * kPi * (3.0 - std::sqrt(5.0));
      r[3 * k] = R * rho * std::cos(ph);
      r[3 * k + 1] = R * rho * std::sin(ph);
      r[3 * k + 2] = R * zk;
    }
  }
  return r;
}

// Stencil of the 3D learned initializer on the reference sphere (offsets ref [nl][3]).
// Per point k: the frame rows n = r_k / |r_k|, t1 = (a x n) / |a x n| (a = e_z, or e_x
// where |n_z| >= 0.9), t2 = n x t1; and its 8 nearest other points (distance |r_j - r_k|,
// ties by index) ordered by azimuth atan2((r_j - r_k).t2, (r_j - r_k).t1) in [0, 2 pi)
// (ties by index).  Distances and azimuths are compared after rounding to 1e-9, so
// the order is the same on any machine.
void sphere_stencil(const std::vector<double>& ref, int nl, std::vector<float>& frames, std::vector<int>& nbrs) {
  frames.assign((size_t)9 * nl, 0.0f);
  nbrs.assign((size_t)8 * nl, 0);
  auto rnd = [](double v) { return std::nearbyint(v * 1e9) / 1e9; };
  auto cross = [](const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
  };
  std::vector<std::pair<double, int>> cand((size_t)nl);
  for (int k = 0; k < nl; ++k) {
    const double* rk = &ref[3 * (size_t)k];
    const double len = std::sqrt(rk[0] * rk[0] + rk[1] * rk[1] + rk[2] * rk[2]);
    const double n[3] = {rk[0] / len, rk[1] / len, rk[2] / len};
    const double a[3] = {std::fabs(n[2]) < 0.9 ? 0.0 : 1.0, 0.0, std::fabs(n[2]) < 0.9 ? 1.0 : 0.0};
    double t1[3], t2[3];
    cross(a, n, t1);
    const double l1 = std::sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int c = 0; c < 3; ++c) t1[c] /= l1;
    cross(n, t1, t2);
    for (int c = 0; c < 3; ++c) {
      frames[9 * (size_t)k + c] = (float)n[c];
      frames[9 * (size_t)k + 3 + c] = (float)t1[c];
      frames[9 * (size_t)k + 6 + c] = (float)t2[c];
    }
    cand.clear();
    for (int j = 0; j < nl; ++j) {
      if (j == k) continue;
      const double* rj = &ref[3 * (size_t)j];
      const double dx = rj[0] - rk[0], dy = rj[1] - rk[1], dz = rj[2] - rk[2];
      cand.push_back({rnd(std::sqrt(dx * dx + dy * dy + dz * dz)), j});
    }
    const size_t m = std::min<size_t>(8, cand.size());
    std::partial_sort(cand.begin(), cand.begin() + m, cand.end());
    std::vector<std::pair<double, int>> az(m);
    for (size_t q = 0; q < m; ++q) {
      const int j = cand[q].second;
      const double* rj = &ref[3 * (size_t)j];
      const double d[3] = {rj[0] - rk[0], rj[1] - rk[1], rj[2] - rk[2]};
      double phi = std::atan2(d[0] * t2[0] + d[1] * t2[1] + d[2] * t2[2], d[0] * t1[0] + d[1] * t1[1] + d[2] * t1[2]);
      if (phi < 0.0) phi += 2.0 * kPi;
      az[q] = {rnd(phi), j};
    }
    std::sort(az.begin(), az.end());
    for (size_t q = 0; q < 8; ++q) nbrs[8 * (size_t)k + q] = q < m ? az[q].second : k;
  }
}

}  // namespace

struct ibm_lbm_handle {
  ibm_lbm_config cfg;
  Derived d;
  Layout l;
  char* ws;
  cudaStream_t s;
  // second stream for the particle work that runs beside lbm_step, and the events
  // that fork it from and join it back into s (fork0: at the start of a step)
  cudaStream_t side;
  cudaEvent_t fork0, fork, join;
  bool mlp_set;     // learned-initializer parameters copied in
  bool track_res;   // residual pass after the last MDF iteration
  long long res_step;  // step whose residual the buffer holds (-1: none)
  long long step;
  int have_prev;
  int64_t launches;
  bool graph_ok[2];
  bool graph_tried[2];
  cudaGraphExec_t graph[2];
  int graph_kernels[2];

  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }

  // node mask of the step of the given parity (marked by the regeneration before it)
  uint32_t* mask(int parity) const {
    return at<uint32_t>(l.mask) + (size_t)parity * d.g.rows * d.g.wpr;
  }
  LbmArgs lbm(int parity) const {
    LbmArgs a{};
    a.g = d.g;
    a.f = at<void>(l.f);
    a.store = cfg.pdf_storage;
    a.ustar = at<float>(l.ustar);
    a.fib = (d.D == 3 || cfg.n_particles > 0) ? at<float>(l.fib) : nullptr;  // 2D: null = no IB force
    a.mask = mask(parity);
    a.omega = (float)(1.0 / cfg.tau);
    a.boundary = cfg.boundary;
    a.u_inlet = (float)cfg.u_inlet;
    a.kforce = (float)(1.0 - 0.5 / cfg.tau);
    for (int k = 0; k < 3; ++k) a.body[k] = (k < d.D) ? (float)cfg.body_force[k] : 0.0f;
    return a;
  }
  double* X(int parity) const { return at<double>(parity ? l.X1 : l.X0); }

  IbmArgs ibm(int parity) const {
    IbmArgs a{};
    a.g = d.g;
    a.D = d.D;
    a.np = cfg.n_particles;
    a.nl = cfg.n_lag;
    a.npts = d.npts;
    a.delta_kind = cfg.delta_kind;
    a.radius = d.radius;
    a.radius_f = (float)d.radius;
    a.rcell = d.rcell;
    a.dV = (float)d.dV;
    a.box = d.box;
    a.mark_radius = d.mark_radius;
    a.ustar = at<float>(l.ustar);
    a.fib = at<float>(l.fib);
    a.f = at<void>(l.f);
    a.store = cfg.pdf_storage;
    a.parity = parity;
    a.ubox = at<float>(l.ubox);
    a.order = at<int>(l.order);
    a.Xb = at<long long>(parity ? l.Xb1 : l.Xb0);
    a.Ub = at<float>(parity ? l.Ub1 : l.Ub0);
    a.Fb = at<float>(l.Fb);
    a.dFb = at<float>(l.dFb);
    a.ubs = at<float>(l.ubs);
    a.res = at<float>(l.res);
    a.frame3 = at<float>(l.frame3);
    a.nbr3 = at<int>(l.nbr3);
    a.slist = d.slen ? at<int>(l.slist) : nullptr;
    a.slen = d.slen;
    a.shell_h = cfg.delta_kind == 3 ? 1.5f : 2.0f;
    a.shell_lo2 = (float)(std::max(0.0, d.radius - 0.01) * std::max(0.0, d.radius - 0.01));
    a.shell_hi2 = (float)((d.radius + 0.01) * (d.radius + 0.01));
    a.Xc = X(parity);
    a.Xcf = at<long long>(l.Xcf);
    a.ref_f = at<float>(l.ref_f);
    a.Pint = at<double>(l.Pint);
    a.Lint = at<double>(l.Lint);
    a.FhN = at<double>(l.FhN);
    a.ThN = at<double>(l.ThN);
    a.status = at<uint32_t>(l.status);
    return a;
  }
  // regeneration into the point buffer of the given parity, from the centres of
  // the same parity (init) or from the fixed-point centres the update wrote
  RegenArgs regen(int parity) const {
    RegenArgs a{};
    a.g = d.g;
    a.D = d.D;
    a.np = cfg.n_particles;
    a.nl = cfg.n_lag;
    a.mark_radius = d.mark_radius;
    a.ref_fix = at<long long>(l.ref_fix);
    a.ref_f = at<float>(l.ref_f);
    a.X = X(parity);
    a.U = at<double>(l.U);
    a.Om = at<double>(l.Om);
    a.Xcf = at<long long>(l.Xcf);
    a.Uf = at<float>(l.Uf);
    a.Omf = at<float>(l.Omf);
    a.Xb_out = at<long long>(parity ? l.Xb1 : l.Xb0);
    a.Ub_out = at<float>(parity ? l.Ub1 : l.Ub0);
    a.mask = mask(parity);
    return a;
  }
  PairArgs pairs(int parity, int have_prev) const {
    PairArgs a{};
    a.g = d.g;
    a.D = d.D;
    a.n = cfg.n_particles;
    for (int k = 0; k < 3; ++k) {
      a.nc[k] = d.nc[k];
      a.H[k] = d.H[k];
      a.L[k] = d.L[k];
    }
    a.diam = cfg.diameter;
    a.zeta = cfg.zeta;
    a.thr2 = d.thr2;
    a.c_ij = d.c_ij;
    a.eps_pp = cfg.eps_pp;
    a.E_pp = cfg.E_pp;
    a.wall_lo = cfg.boundary ? 0.0 : -0.5;
    a.kmax = d.kmax;
    a.grid_mode = d.gcells > 0 ? 1 : 0;
    a.grid = at<int>(l.grid);
    for (int k = 0; k < 3; ++k) {
      a.gnc[k] = d.gnc[k];
      a.gH[k] = d.gH[k];
      a.greach[k] = d.greach[k];
    }
    a.over = at<int>(l.over);
    a.over_count = at<int>(l.over_count);
    a.over_cap = d.over_cap;
    a.X = X(parity);
    a.cell_count = at<int>(l.cell_count);
    a.cell_ids = at<int>(l.cell_ids);
    a.cell_cap = cell_capacity(cfg.n_particles, (long long)d.nc[0] * d.nc[1] * d.nc[2]);
    a.nbr = at<int>(l.nbr);
    a.nbr_count = at<int>(l.nbr_count);
    a.Fc = at<double>(l.Fc);
    a.gt_count = at<int>(l.gt);
    a.status = at<uint32_t>(l.status);
    a.integrate = 1;
    a.have_prev = have_prev;
    PartState& p = a.ps;
    p.Xnew = X(1 - parity);
    p.U = at<double>(l.U);
    p.Om = at<double>(l.Om);
    p.Fh = at<double>(l.Fh);
    p.Th = at<double>(l.Th);
    p.acc = at<double>(l.acc);
    p.alp = at<double>(l.alp);
    p.Pprev = at<double>(l.Pprev);
    p.Lprev = at<double>(l.Lprev);
    p.FhN = at<double>(l.FhN);
    p.ThN = at<double>(l.ThN);
    p.Pint = at<double>(l.Pint);
    p.Lint = at<double>(l.Lint);
    p.Xcf = at<long long>(l.Xcf);
    p.Uf = at<float>(l.Uf);
    p.Omf = at<float>(l.Omf);
    p.Mp = d.Mp;
    p.meff = d.meff;
    p.Ip = d.Ip;
    p.Kt = d.Kt;
    p.Kr = d.Kr;
    for (int k = 0; k < 3; ++k) p.grav[k] = cfg.gravity[k];
    p.fixed = cfg.fixed_particles;
    return a;
  }
};

namespace {

// 3D node mask of a parity (lbm_moments and the f_IB read of lbm_step use it):
// cleared before the regeneration marks the nodes of the new particle positions
cudaError_t clear_mask(ibm_lbm_handle* h, int parity, cudaStream_t s) {
  if (h->d.D != 3) return cudaSuccess;  // 2D keeps no node mask
  return cudaMemsetAsync(h->mask(parity), 0, sizeof(uint32_t) * (size_t)h->d.g.rows * h->d.g.wpr, s);
}

// Enqueue one step of the given parity.  With ev != nullptr an event is recorded
// after each part (for ibm_lbm_time_parts).  Returns the number of kernels launched.
int enqueue_step(ibm_lbm_handle* h, int parity, int have_prev, cudaEvent_t* ev, int* nk) {
  const cudaStream_t s = h->s;
  const bool particles = h->cfg.n_particles > 0;
  int k = 0;
  const LbmArgs la = h->lbm(parity);
  const IbmArgs ia = h->ibm(parity);
  const PairArgs pa = h->pairs(parity, have_prev);
  if (ev) CUDA_TRY(cudaEventRecord(ev[0], s));
  if (particles && !ev) {
    // The cell lists and partner lists need only this step's centres: they are built
    // on the side stream beside the IBM kernels (all latency-bound, so they share the
    // SMs well), which leaves only the forces and the update beside lbm_step.
    CUDA_TRY(cudaEventRecord(h->fork0, s));
    CUDA_TRY(cudaStreamWaitEvent(h->side, h->fork0, 0));
    CUDA_TRY(launch_pair_cells(pa, h->side));
    CUDA_TRY(launch_pair_search_lists(pa, h->side));
    k += 2;
  }
  if (particles && h->d.D == 3) {  // 2D computes u* per particle box in the first interpolation
    CUDA_TRY(launch_lbm_moments(la, h->d.D, parity, s));
    ++k;
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], s));
  if (particles) {
    if (h->d.D == 2 && h->cfg.mdf_iters == 0) {  // the interior momentum still needs box u*
      CUDA_TRY(launch_ibm_interp(ia, 0, s));
      ++k;
    }
    for (int m = 1; m <= h->cfg.mdf_iters; ++m) {
      CUDA_TRY(launch_ibm_interp(ia, m, s));
      ++k;
      if (m == 1 && h->cfg.mlp_init) {  // learned first force
        CUDA_TRY(launch_mlp_step(ia, h->at<float>(h->l.mlp), h->at<void>(h->l.mlp_img), s));
        ++k;
      }
      CUDA_TRY(launch_ibm_spread(ia, s));
      ++k;
    }
    if (h->track_res && h->cfg.mdf_iters > 0) {
      CUDA_TRY(launch_ibm_interp(ia, -1, s));
      ++k;
    }
    CUDA_TRY(launch_ibm_forces(ia, s));
    ++k;
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[2], s));
  if (particles && !ev) {
    // The contact forces, the Newton-Euler update and the regeneration of the points
    // (into the other point buffer and the other node mask) read nothing lbm_step
    // writes and write nothing it reads, so they run on the side stream while
    // lbm_step streams the PDFs.
    CUDA_TRY(cudaEventRecord(h->fork, s));
    CUDA_TRY(cudaStreamWaitEvent(h->side, h->fork, 0));
    CUDA_TRY(launch_pair_forces(pa, h->side));
    k += 1;
    CUDA_TRY(clear_mask(h, 1 - parity, h->side));
    CUDA_TRY(launch_regen(h->regen(1 - parity), 0, h->side));
    ++k;
    CUDA_TRY(cudaEventRecord(h->join, h->side));
    CUDA_TRY(launch_lbm_step(la, h->d.D, parity, s));
    k += lbm_step_launches(h->d.g, h->d.D, parity, h->cfg.pdf_storage);
    CUDA_TRY(launch_lbm_nee(la, h->d.D, parity, s));
    k += h->cfg.boundary ? 1 : 0;
    CUDA_TRY(cudaStreamWaitEvent(s, h->join, 0));
    *nk = k;
    return IBMLBM_OK;
  }
  // one part after the other (no particles, or timed parts)
  CUDA_TRY(launch_lbm_step(la, h->d.D, parity, s));
  k += lbm_step_launches(h->d.g, h->d.D, parity, h->cfg.pdf_storage);
  CUDA_TRY(launch_lbm_nee(la, h->d.D, parity, s));
  k += h->cfg.boundary ? 1 : 0;
  if (ev) CUDA_TRY(cudaEventRecord(ev[3], s));
  if (particles) {
    CUDA_TRY(launch_pair_cells(pa, s));
    CUDA_TRY(launch_pair_contacts(pa, s));
    k += 3;
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[4], s));
  if (particles) {
    CUDA_TRY(clear_mask(h, 1 - parity, s));
    CUDA_TRY(launch_regen(h->regen(1 - parity), 0, s));
    ++k;
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[5], s));
  *nk = k;
  return IBMLBM_OK;
}

int capture_graph(ibm_lbm_handle* h, int parity) {
  cudaGraph_t graph = nullptr;
  int nk = 0;
  if (cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return IBMLBM_ERR_CUDA;
  }
  const int rc = enqueue_step(h, parity, 1, nullptr, &nk);
  const cudaError_t e = cudaStreamEndCapture(h->s, &graph);
  if (rc != IBMLBM_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return IBMLBM_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return IBMLBM_ERR_CUDA;
  }
  cudaGraphDestroy(graph);
  h->graph[parity] = exec;
  h->graph_kernels[parity] = nk;
  h->graph_ok[parity] = true;
  return IBMLBM_OK;
}

// points and node marks of the current state (after init or a new particle state)
// 2D: the order in which the IBM kernels' warps take the particles, by centre height
// from the top.  lbm_step walks the rows upwards, so the top rows are the last it
// wrote and the likeliest to be still in L2 when the next step's first interpolation
// reads the PDFs around the particles (the next lbm_step then starts on the bottom rows
// that the interpolation read last).  Set from the centres whenever they are set; the
// particles move little between settings, and any order gives the same results.
int refresh_order(ibm_lbm_handle* h) {
  const int np = h->cfg.n_particles;
  if (h->d.D != 2 || np == 0) return IBMLBM_OK;
  std::vector<double> X((size_t)np * 2);
  CUDA_TRY(cudaMemcpyAsync(X.data(), h->X((int)(h->step & 1)), sizeof(double) * X.size(),
                           cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  std::vector<int> order((size_t)np);
  for (int i = 0; i < np; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return X[2 * (size_t)a + 1] > X[2 * (size_t)b + 1]; });
  CUDA_TRY(cudaMemcpyAsync(h->at<int>(h->l.order), order.data(), sizeof(int) * order.size(),
                           cudaMemcpyHostToDevice, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return IBMLBM_OK;
}

int regenerate_points(ibm_lbm_handle* h) {
  if (h->cfg.n_particles == 0) return IBMLBM_OK;
  const int rc = refresh_order(h);
  if (rc) return rc;
  CUDA_TRY(clear_mask(h, (int)(h->step & 1), h->s));
  CUDA_TRY(launch_regen(h->regen((int)(h->step & 1)), 1, h->s));
  h->launches += 1;
  return IBMLBM_OK;
}

int check_handle(ibm_lbm_handle* h) {
  if (!h) return fail(IBMLBM_ERR_INVALID_ARG, "handle is NULL");
  return IBMLBM_OK;
}

}  // namespace

extern "C" {

int ibm_lbm_stage_list(const ibm_lbm_config* cfg, int32_t* cells, int64_t cap, int64_t* n) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!n) return fail(IBMLBM_ERR_INVALID_ARG, "n is NULL");
  const Derived d = derive(cfg);
  const std::vector<int> list = cfg->n_particles > 0 ? stage3_list(d, cfg->delta_kind) : std::vector<int>();
  *n = (int64_t)list.size();
  if (!cells) return IBMLBM_OK;
  if (*n > cap) return fail(IBMLBM_ERR_CAPACITY, "staging list longer than cap");
  for (size_t k = 0; k < list.size(); ++k) cells[k] = list[k];
  return IBMLBM_OK;
}

int ibm_lbm_workspace_size(const ibm_lbm_config* cfg, size_t* bytes) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!bytes) return fail(IBMLBM_ERR_INVALID_ARG, "bytes is NULL");
  const Derived d = derive(cfg);
  *bytes = carve(cfg, d).total;
  return IBMLBM_OK;
}

int ibm_lbm_init(const ibm_lbm_config* cfg, void* d_workspace, size_t bytes, void* stream,
                 const double* h_centres, ibm_lbm_handle** out) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!out) return fail(IBMLBM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  const Derived d = derive(cfg);
  const Layout l = carve(cfg, d);
  if (!d_workspace) return fail(IBMLBM_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign)
    return fail(IBMLBM_ERR_WORKSPACE, "workspace is not 256-byte aligned");
  if (bytes < l.total)
    return fail(IBMLBM_ERR_WORKSPACE, "workspace smaller than ibm_lbm_workspace_size");
  if (cfg->n_particles > 0 && !h_centres)
    return fail(IBMLBM_ERR_INVALID_ARG, "centres are NULL");
  for (int i = 0; i < cfg->n_particles; ++i)
    for (int k = 0; k < d.D; ++k) {
      const double x = h_centres[(size_t)i * d.D + k];
      if (!std::isfinite(x) || x < -0.5 || x >= d.L[k] - 0.5)
        return fail(IBMLBM_ERR_INVALID_ARG, "particle centre outside the domain");
    }
  // 2D: one particle's box per warp must fit (fewer warps per block for large ones);
  // 3D spheres whose box does not fit run the IBM from global memory
  if (cfg->n_particles > 0 && d.D == 2 && spread_smem(2, cfg->n_lag, d.box) > 227 * 1024)
    return fail(IBMLBM_ERR_UNSUPPORTED, "particle too large for the spreading box");
  ibm_lbm_handle* h = new ibm_lbm_handle();
  h->cfg = *cfg;
  h->d = d;
  h->l = l;
  h->ws = static_cast<char*>(d_workspace);
  h->s = static_cast<cudaStream_t>(stream);
  h->step = 0;
  h->have_prev = 0;
  h->launches = 0;
  h->graph_ok[0] = h->graph_ok[1] = false;
  h->graph_tried[0] = h->graph_tried[1] = false;
  h->side = nullptr;
  h->fork0 = h->fork = h->join = nullptr;
  h->mlp_set = false;
  h->track_res = false;
  h->res_step = -1;
  auto bail = [&](int code) {
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork0) cudaEventDestroy(h->fork0);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    delete h;
    return code;
  };
#define INIT_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bail(fail(IBMLBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  INIT_TRY(cudaMemsetAsync(h->ws, 0, l.total, h->s));
  {
    // the side stream's short particle kernels at the highest priority: the block
    // scheduler then places their blocks ahead of lbm_step's as SMs free up, so they
    // finish inside lbm_step's time instead of after it
    int lo_ = 0, hi_ = 0;
    INIT_TRY(cudaDeviceGetStreamPriorityRange(&lo_, &hi_));
    INIT_TRY(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi_));
  }
  INIT_TRY(cudaEventCreateWithFlags(&h->fork0, cudaEventDisableTiming));
  INIT_TRY(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
  INIT_TRY(cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming));
  if (cfg->n_particles > 0) {
    INIT_TRY(cudaMemcpyAsync(h->at<double>(l.X0), h_centres,
                             sizeof(double) * (size_t)cfg->n_particles * d.D,
                             cudaMemcpyHostToDevice, h->s));
    const std::vector<double> ref = reference_points(d.D, cfg->n_lag, d.radius);
    std::vector<long long> ref_fix(ref.size());
    std::vector<float> ref_f(ref.size());
    for (size_t k = 0; k < ref.size(); ++k) {
      ref_fix[k] = std::llrint(ref[k] * kFixScale);
      ref_f[k] = (float)ref[k];
    }
    INIT_TRY(cudaMemcpyAsync(h->at<long long>(l.ref_fix), ref_fix.data(),
                             sizeof(long long) * ref_fix.size(), cudaMemcpyHostToDevice, h->s));
    INIT_TRY(cudaMemcpyAsync(h->at<float>(l.ref_f), ref_f.data(), sizeof(float) * ref_f.size(),
                             cudaMemcpyHostToDevice, h->s));
    std::vector<float> frames;
    std::vector<int> nbrs;
    if (d.D == 3) {
      sphere_stencil(ref, cfg->n_lag, frames, nbrs);
      INIT_TRY(cudaMemcpyAsync(h->at<float>(l.frame3), frames.data(), sizeof(float) * frames.size(),
                               cudaMemcpyHostToDevice, h->s));
      INIT_TRY(cudaMemcpyAsync(h->at<int>(l.nbr3), nbrs.data(), sizeof(int) * nbrs.size(),
                               cudaMemcpyHostToDevice, h->s));
    }
    const std::vector<int> slist = stage3_list(d, cfg->delta_kind);
    if (!slist.empty())
      INIT_TRY(cudaMemcpyAsync(h->at<int>(l.slist), slist.data(), sizeof(int) * slist.size(),
                               cudaMemcpyHostToDevice, h->s));
    INIT_TRY(cudaStreamSynchronize(h->s));  // host vectors go out of scope
    if (spread_smem(d.D, cfg->n_lag, d.box) <= 227 * 1024)
      INIT_TRY(prepare_ibm_spread(d.D, spread_smem(d.D, cfg->n_lag, d.box)));
    if (regenerate_points(h) != IBMLBM_OK) return bail(IBMLBM_ERR_CUDA);
  }
  INIT_TRY(cudaStreamSynchronize(h->s));
#undef INIT_TRY
  *out = h;
  return IBMLBM_OK;
}

int ibm_lbm_step(ibm_lbm_handle* h, int32_t n_steps) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (n_steps < 0) return fail(IBMLBM_ERR_INVALID_ARG, "n_steps < 0");
  if (h->cfg.mlp_init && !h->mlp_set)
    return fail(IBMLBM_ERR_INVALID_ARG, "mlp_init is set but ibm_lbm_set_mlp was not called");
  for (int32_t t = 0; t < n_steps; ++t) {
    const int parity = (int)(h->step & 1);
    if (h->have_prev && !h->graph_tried[parity]) {
      h->graph_tried[parity] = true;
      capture_graph(h, parity);  // on failure the steps run as eager launches
    }
    if (h->have_prev && h->graph_ok[parity]) {
      CUDA_TRY(cudaGraphLaunch(h->graph[parity], h->s));
      h->launches += h->graph_kernels[parity];
    } else {
      int nk = 0;
      rc = enqueue_step(h, parity, h->have_prev, nullptr, &nk);
      if (rc) return rc;
      h->launches += nk;
    }
    if (h->track_res) h->res_step = h->step;
    h->step += 1;
    h->have_prev = 1;
  }
  return IBMLBM_OK;
}

int ibm_lbm_sync(ibm_lbm_handle* h) {
  int rc = check_handle(h);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(h->s));
  rc = report_check_faults();
  if (rc) return rc;
  uint32_t st = 0;
  CUDA_TRY(cudaMemcpy(&st, h->at<uint32_t>(h->l.status), sizeof(st), cudaMemcpyDeviceToHost));
  if (st) {
    CUDA_TRY(cudaMemset(h->at<uint32_t>(h->l.status), 0, sizeof(uint32_t)));
    if (st & ST_NONFINITE) return fail(IBMLBM_ERR_NONFINITE, "non-finite particle state");
    if (st & ST_OUT_OF_DOMAIN)
      return fail(IBMLBM_ERR_OUT_OF_DOMAIN, "a particle centre left the domain");
    return fail(IBMLBM_ERR_CAPACITY, "a contact list or spreading box overflowed");
  }
  return IBMLBM_OK;
}

int ibm_lbm_set_pdfs(ibm_lbm_handle* h, const float* d_f) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!d_f) return fail(IBMLBM_ERR_INVALID_ARG, "f is NULL");
  CUDA_TRY(launch_lbm_put(h->lbm((int)(h->step & 1)), h->d.D, (int)(h->step & 1), d_f, h->s));
  h->launches += 1;
  return IBMLBM_OK;
}

int ibm_lbm_get_pdfs(ibm_lbm_handle* h, float* d_f) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!d_f) return fail(IBMLBM_ERR_INVALID_ARG, "f is NULL");
  CUDA_TRY(launch_lbm_get(h->lbm((int)(h->step & 1)), h->d.D, (int)(h->step & 1), d_f, h->s));
  h->launches += 1;
  return IBMLBM_OK;
}

int ibm_lbm_set_fields(ibm_lbm_handle* h, const double* d_p, const double* d_u) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!d_p || !d_u) return fail(IBMLBM_ERR_INVALID_ARG, "p or u is NULL");
  CUDA_TRY(launch_lbm_equilibrium(h->lbm((int)(h->step & 1)), h->d.D, (int)(h->step & 1), d_p, d_u, h->s));
  h->launches += 1;
  return IBMLBM_OK;
}

int ibm_lbm_get_fields(ibm_lbm_handle* h, double* d_p, double* d_u) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!d_p && !d_u) return IBMLBM_OK;
  CUDA_TRY(launch_lbm_fields(h->lbm((int)(h->step & 1)), h->d.D, (int)(h->step & 1), d_p, d_u, h->s));
  h->launches += 1;
  return IBMLBM_OK;
}

int ibm_lbm_set_particles(ibm_lbm_handle* h, const double* X, const double* U,
                          const double* Omega) {
  int rc = check_handle(h);
  if (rc) return rc;
  const int np = h->cfg.n_particles, D = h->d.D;
  if (np == 0) return IBMLBM_OK;
  if (X) {
    for (int i = 0; i < np; ++i)
      for (int k = 0; k < D; ++k) {
        const double x = X[(size_t)i * D + k];
        if (!std::isfinite(x) || x < -0.5 || x >= h->d.L[k] - 0.5)
          return fail(IBMLBM_ERR_INVALID_ARG, "particle centre outside the domain");
      }
    CUDA_TRY(cudaMemcpyAsync(h->X((int)(h->step & 1)), X, sizeof(double) * np * D,
                             cudaMemcpyHostToDevice, h->s));
  }
  if (U)
    CUDA_TRY(cudaMemcpyAsync(h->at<double>(h->l.U), U, sizeof(double) * np * D,
                             cudaMemcpyHostToDevice, h->s));
  if (Omega) {
    if (D == 2)
      CUDA_TRY(cudaMemcpy2DAsync(h->at<double>(h->l.Om) + 2, 3 * sizeof(double), Omega,
                                 sizeof(double), sizeof(double), np, cudaMemcpyHostToDevice, h->s));
    else
      CUDA_TRY(cudaMemcpyAsync(h->at<double>(h->l.Om), Omega, sizeof(double) * np * 3,
                               cudaMemcpyHostToDevice, h->s));
  }
  rc = regenerate_points(h);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return IBMLBM_OK;
}

}  // extern "C"

namespace {

// Checkpoint blob: header, the raw PDF buffer (its layout is the AA parity of the
// stored step counter), the particle arrays the update carries from step to step, and
// the learned initializer's parameters when they are set.
struct StateHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int32_t dim, nx, ny, nz, periodic[3], n_particles, n_lag, pdf_storage, boundary, pair_search;
  int64_t step;
  int32_t have_prev, mlp_set;
  uint64_t f_bytes, part_bytes, mlp_bytes;
};
constexpr char kStateMagic[8] = {'I', 'B', 'L', 'B', 'M', 'S', 'T', '1'};

// the particle arrays of a checkpoint: (device pointer, doubles), in blob order
std::vector<std::pair<double*, size_t>> state_arrays(const ibm_lbm_handle* h) {
  const size_t np = (size_t)h->cfg.n_particles, D = (size_t)h->d.D;
  if (np == 0) return {};
  const Layout& l = h->l;
  return {{h->X((int)(h->step & 1)), np * D}, {h->at<double>(l.U), np * D}, {h->at<double>(l.Om), np * 3},
          {h->at<double>(l.Fh), np * D},      {h->at<double>(l.Th), np * 3}, {h->at<double>(l.acc), np * D},
          {h->at<double>(l.alp), np * 3},     {h->at<double>(l.Pprev), np * D},
          {h->at<double>(l.Lprev), np * 3}};
}

size_t state_f_bytes(const ibm_lbm_handle* h) {
  return (h->cfg.pdf_storage == IBMLBM_PDF_FP32 ? 4 : 2) * ((size_t)h->d.Q * h->d.g.Np + 64);
}

StateHeader state_header(const ibm_lbm_handle* h) {
  StateHeader H{};
  std::memcpy(H.magic, kStateMagic, 8);
  H.version = 1;
  H.header_bytes = sizeof(StateHeader);
  H.dim = h->cfg.dim;
  H.nx = h->cfg.nx;
  H.ny = h->cfg.ny;
  H.nz = h->cfg.nz;
  for (int k = 0; k < 3; ++k) H.periodic[k] = h->cfg.periodic[k];
  H.n_particles = h->cfg.n_particles;
  H.n_lag = h->cfg.n_lag;
  H.pdf_storage = h->cfg.pdf_storage;
  H.boundary = h->cfg.boundary;
  H.pair_search = h->cfg.pair_search;
  H.step = h->step;
  H.have_prev = h->have_prev;
  H.mlp_set = h->mlp_set ? 1 : 0;
  H.f_bytes = state_f_bytes(h);
  size_t pb = 0;
  for (const auto& a : state_arrays(h)) pb += sizeof(double) * a.second;
  H.part_bytes = pb;
  H.mlp_bytes = h->mlp_set ? sizeof(float) * kMlpParams : 0;
  return H;
}

}  // namespace

extern "C" {

int ibm_lbm_state_size(ibm_lbm_handle* h, size_t* bytes) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!bytes) return fail(IBMLBM_ERR_INVALID_ARG, "bytes is NULL");
  const StateHeader H = state_header(h);
  *bytes = sizeof(StateHeader) + H.f_bytes + H.part_bytes + H.mlp_bytes;
  return IBMLBM_OK;
}

int ibm_lbm_get_state(ibm_lbm_handle* h, void* h_buf, size_t bytes) {
  int rc = check_handle(h);
  if (rc) return rc;
  const StateHeader H = state_header(h);
  const size_t need = sizeof(StateHeader) + H.f_bytes + H.part_bytes + H.mlp_bytes;
  if (!h_buf || bytes < need) return fail(IBMLBM_ERR_INVALID_ARG, "state buffer missing or too small");
  char* p = static_cast<char*>(h_buf);
  std::memcpy(p, &H, sizeof(H));
  p += sizeof(H);
  CUDA_TRY(cudaMemcpyAsync(p, h->at<char>(h->l.f), H.f_bytes, cudaMemcpyDeviceToHost, h->s));
  p += H.f_bytes;
  for (const auto& a : state_arrays(h)) {
    CUDA_TRY(cudaMemcpyAsync(p, a.first, sizeof(double) * a.second, cudaMemcpyDeviceToHost, h->s));
    p += sizeof(double) * a.second;
  }
  if (H.mlp_bytes)
    CUDA_TRY(cudaMemcpyAsync(p, h->at<float>(h->l.mlp), H.mlp_bytes, cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return IBMLBM_OK;
}

int ibm_lbm_set_state(ibm_lbm_handle* h, const void* h_buf, size_t bytes) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h_buf || bytes < sizeof(StateHeader)) return fail(IBMLBM_ERR_INVALID_ARG, "state buffer missing or too small");
  StateHeader H;
  std::memcpy(&H, h_buf, sizeof(H));
  StateHeader mine = state_header(h);
  if (std::memcmp(H.magic, kStateMagic, 8) != 0 || H.version != 1 || H.header_bytes != sizeof(StateHeader))
    return fail(IBMLBM_ERR_INVALID_ARG, "not a state of this library version");
  if (H.dim != mine.dim || H.nx != mine.nx || H.ny != mine.ny || H.nz != mine.nz ||
      H.periodic[0] != mine.periodic[0] || H.periodic[1] != mine.periodic[1] || H.periodic[2] != mine.periodic[2] ||
      H.n_particles != mine.n_particles || H.n_lag != mine.n_lag || H.pdf_storage != mine.pdf_storage ||
      H.boundary != mine.boundary || H.pair_search != mine.pair_search || H.f_bytes != mine.f_bytes ||
      H.part_bytes != mine.part_bytes || H.step < 0 ||
      (H.mlp_bytes != 0 && H.mlp_bytes != sizeof(float) * kMlpParams))
    return fail(IBMLBM_ERR_INVALID_ARG, "state of another configuration");
  if (bytes < sizeof(StateHeader) + H.f_bytes + H.part_bytes + H.mlp_bytes)
    return fail(IBMLBM_ERR_INVALID_ARG, "state buffer too small");
  CUDA_TRY(cudaStreamSynchronize(h->s));
  h->step = H.step;  // fixes the parity of the PDF layout and of the point buffers
  h->have_prev = H.have_prev;
  h->res_step = -1;
  const char* p = static_cast<const char*>(h_buf) + sizeof(StateHeader);
  CUDA_TRY(cudaMemcpyAsync(h->at<char>(h->l.f), p, H.f_bytes, cudaMemcpyHostToDevice, h->s));
  p += H.f_bytes;
  for (const auto& a : state_arrays(h)) {
    CUDA_TRY(cudaMemcpyAsync(a.first, p, sizeof(double) * a.second, cudaMemcpyHostToDevice, h->s));
    p += sizeof(double) * a.second;
  }
  if (H.mlp_bytes) {
    CUDA_TRY(cudaMemcpyAsync(h->at<float>(h->l.mlp), p, H.mlp_bytes, cudaMemcpyHostToDevice, h->s));
    CUDA_TRY(launch_mlp_image(h->at<float>(h->l.mlp), h->at<void>(h->l.mlp_img), h->s));
    h->mlp_set = true;
  }
  // between steps f_IB is zero; the points, fixed-point centres and masks follow from
  // the restored centres and velocities
  const size_t fib_bytes = sizeof(float) * (h->d.D == 3 ? 4 : 2) * (size_t)h->d.g.N;
  if (h->cfg.n_particles > 0 || h->d.D == 3)
    CUDA_TRY(cudaMemsetAsync(h->at<float>(h->l.fib), 0, fib_bytes, h->s));
  rc = regenerate_points(h);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return IBMLBM_OK;
}

int ibm_lbm_get_particles(ibm_lbm_handle* h, double* X, double* U, double* Omega,
                          double* F_h, double* T_h, double* F_c) {
  int rc = check_handle(h);
  if (rc) return rc;
  const int np = h->cfg.n_particles, D = h->d.D;
  if (np == 0) return IBMLBM_OK;
  const size_t vb = sizeof(double) * np * D;
  if (X) CUDA_TRY(cudaMemcpyAsync(X, h->X((int)(h->step & 1)), vb, cudaMemcpyDeviceToHost, h->s));
  if (U) CUDA_TRY(cudaMemcpyAsync(U, h->at<double>(h->l.U), vb, cudaMemcpyDeviceToHost, h->s));
  if (F_h) CUDA_TRY(cudaMemcpyAsync(F_h, h->at<double>(h->l.Fh), vb, cudaMemcpyDeviceToHost, h->s));
  if (F_c) CUDA_TRY(cudaMemcpyAsync(F_c, h->at<double>(h->l.Fc), vb, cudaMemcpyDeviceToHost, h->s));
  double* ang[2] = {Omega, T_h};
  const size_t offs[2] = {h->l.Om, h->l.Th};
  for (int q = 0; q < 2; ++q) {
    if (!ang[q]) continue;
    if (D == 2)
      CUDA_TRY(cudaMemcpy2DAsync(ang[q], sizeof(double), h->at<double>(offs[q]) + 2,
                                 3 * sizeof(double), sizeof(double), np, cudaMemcpyDeviceToHost, h->s));
    else
      CUDA_TRY(cudaMemcpyAsync(ang[q], h->at<double>(offs[q]), sizeof(double) * np * 3,
                               cudaMemcpyDeviceToHost, h->s));
  }
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return IBMLBM_OK;
}

int ibm_lbm_get_lagrangian(ibm_lbm_handle* h, double* X_b, float* U_b, float* F_b,
                           float* u_b_star) {
  int rc = check_handle(h);
  if (rc) return rc;
  const size_t npts = (size_t)h->d.npts, D = h->d.D;
  if (npts == 0) return IBMLBM_OK;
  // points used by the last step (before its update regenerated them)
  const int last = h->step > 0 ? (int)((h->step - 1) & 1) : 0;
  std::vector<long long> xb_fix(X_b ? npts * D : 0);
  if (X_b)
    CUDA_TRY(cudaMemcpyAsync(xb_fix.data(), h->at<long long>(last ? h->l.Xb1 : h->l.Xb0),
                             sizeof(long long) * npts * D, cudaMemcpyDeviceToHost, h->s));
  if (U_b)
    CUDA_TRY(cudaMemcpyAsync(U_b, h->at<float>(last ? h->l.Ub1 : h->l.Ub0),
                             sizeof(float) * npts * D, cudaMemcpyDeviceToHost, h->s));
  if (F_b)
    CUDA_TRY(cudaMemcpyAsync(F_b, h->at<float>(h->l.Fb), sizeof(float) * npts * D,
                             cudaMemcpyDeviceToHost, h->s));
  if (u_b_star)
    CUDA_TRY(cudaMemcpyAsync(u_b_star, h->at<float>(h->l.ubs), sizeof(float) * npts * D,
                             cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  for (size_t k = 0; k < xb_fix.size(); ++k) X_b[k] = (double)xb_fix[k] / kFixScale;
  return IBMLBM_OK;
}

int ibm_lbm_get_interior_momentum(ibm_lbm_handle* h, double* P, double* L) {
  int rc = check_handle(h);
  if (rc) return rc;
  const int np = h->cfg.n_particles, D = h->d.D;
  if (np == 0) return IBMLBM_OK;
  if (P)
    CUDA_TRY(cudaMemcpyAsync(P, h->at<double>(h->l.Pint), sizeof(double) * np * D,
                             cudaMemcpyDeviceToHost, h->s));
  if (L) {
    if (D == 2)
      CUDA_TRY(cudaMemcpy2DAsync(L, sizeof(double), h->at<double>(h->l.Lint) + 2,
                                 3 * sizeof(double), sizeof(double), np, cudaMemcpyDeviceToHost, h->s));
    else
      CUDA_TRY(cudaMemcpyAsync(L, h->at<double>(h->l.Lint), sizeof(double) * np * 3,
                               cudaMemcpyDeviceToHost, h->s));
  }
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return IBMLBM_OK;
}

int ibm_lbm_get_pairs(ibm_lbm_handle* h, int32_t* pairs, int64_t cap, int64_t* n) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!n || (cap > 0 && !pairs)) return fail(IBMLBM_ERR_INVALID_ARG, "pairs or n is NULL");
  const int np = h->cfg.n_particles;
  *n = 0;
  if (np == 0) return IBMLBM_OK;
  const PairArgs pa = h->pairs(0, 1);
  const long long dev_cap = (long long)np * h->d.kmax / 2;
  CUDA_TRY(launch_pair_compact(pa, h->at<int>(h->l.pairs), dev_cap, h->s));
  h->launches += 2;
  int total = 0;
  CUDA_TRY(cudaMemcpyAsync(&total, h->at<int>(h->l.gt) + np, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  *n = total;
  if (total > cap) return fail(IBMLBM_ERR_CAPACITY, "more pairs than cap");
  if (total > 0)
    CUDA_TRY(cudaMemcpy(pairs, h->at<int>(h->l.pairs), sizeof(int) * 2 * (size_t)total,
                        cudaMemcpyDeviceToHost));
  return IBMLBM_OK;
}

int ibm_lbm_get_launch_count(ibm_lbm_handle* h, int64_t* n) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!n) return fail(IBMLBM_ERR_INVALID_ARG, "n is NULL");
  *n = h->launches;
  return IBMLBM_OK;
}

int ibm_lbm_time_parts(ibm_lbm_handle* h, int32_t n_steps, double* ms) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!ms || n_steps < 0) return fail(IBMLBM_ERR_INVALID_ARG, "ms is NULL or n_steps < 0");
  for (int p = 0; p < IBMLBM_PART_COUNT; ++p) ms[p] = 0.0;
  cudaEvent_t ev[6];
  for (int k = 0; k < 6; ++k) CUDA_TRY(cudaEventCreate(&ev[k]));
  int out = IBMLBM_OK;
  for (int32_t t = 0; t < n_steps && out == IBMLBM_OK; ++t) {
    int nk = 0;
    out = enqueue_step(h, (int)(h->step & 1), h->have_prev, ev, &nk);
    if (out) break;
    h->launches += nk;
    h->step += 1;
    h->have_prev = 1;
    if (cudaEventSynchronize(ev[5]) != cudaSuccess) {
      out = fail(IBMLBM_ERR_CUDA, "event synchronisation failed");
      break;
    }
    for (int p = 0; p < IBMLBM_PART_COUNT; ++p) {
      float v = 0.0f;
      cudaEventElapsedTime(&v, ev[p], ev[p + 1]);
      ms[p] += v;
    }
  }
  for (int k = 0; k < 6; ++k) cudaEventDestroy(ev[k]);
  return out;
}


int ibm_lbm_set_mlp(ibm_lbm_handle* h, const float* h_params) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h_params) return fail(IBMLBM_ERR_INVALID_ARG, "h_params is NULL");
  CUDA_TRY(cudaMemcpyAsync(h->at<float>(h->l.mlp), h_params, sizeof(float) * kMlpParams,
                           cudaMemcpyHostToDevice, h->s));
  CUDA_TRY(launch_mlp_image(h->at<float>(h->l.mlp), h->at<void>(h->l.mlp_img), h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  h->mlp_set = true;
  return IBMLBM_OK;
}

int ibm_lbm_mdf_samples(ibm_lbm_handle* h, float* d_X, float* d_Y) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!d_X || !d_Y) return fail(IBMLBM_ERR_INVALID_ARG, "sample arrays are NULL");
  if (h->step < 1) return fail(IBMLBM_ERR_INVALID_ARG, "samples need a run after its first step");
  CUDA_TRY(launch_mlp_samples(h->ibm((int)((h->step - 1) & 1)), d_X, d_Y, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  return IBMLBM_OK;
}

int ibm_lbm_set_residual_tracking(ibm_lbm_handle* h, int32_t on) {
  int rc = check_handle(h);
  if (rc) return rc;
  if ((bool)on == h->track_res) return IBMLBM_OK;
  CUDA_TRY(cudaStreamSynchronize(h->s));
  for (int p = 0; p < 2; ++p) {  // the captured steps change: capture again
    if (h->graph_ok[p]) cudaGraphExecDestroy(h->graph[p]);
    h->graph_ok[p] = h->graph_tried[p] = false;
  }
  h->track_res = on != 0;
  h->res_step = -1;
  return IBMLBM_OK;
}

int ibm_lbm_get_mdf_residual(ibm_lbm_handle* h, double* rms, double* maxabs) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->res_step < 0) return fail(IBMLBM_ERR_INVALID_ARG, "no tracked step yet");
  const size_t npts = (size_t)h->d.npts, D = (size_t)h->d.D;
  std::vector<float> r(npts * D);
  if (npts)
    CUDA_TRY(cudaMemcpyAsync(r.data(), h->at<float>(h->l.res), sizeof(float) * r.size(),
                             cudaMemcpyDeviceToHost, h->s));
  CUDA_TRY(cudaStreamSynchronize(h->s));
  double s2 = 0.0, mx = 0.0;
  for (size_t q = 0; q < npts * D; ++q) {
    s2 += (double)r[q] * r[q];
    mx = std::max(mx, std::fabs((double)r[q]));
  }
  if (rms) *rms = npts ? std::sqrt(s2 / (double)(npts * D)) : 0.0;
  if (maxabs) *maxabs = mx;
  return IBMLBM_OK;
}

void ibm_lbm_destroy(ibm_lbm_handle* h) {
  if (!h) return;
  for (int p = 0; p < 2; ++p)
    if (h->graph_ok[p]) cudaGraphExecDestroy(h->graph[p]);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  if (h->fork0) cudaEventDestroy(h->fork0);
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->join) cudaEventDestroy(h->join);
  delete h;
}

const char* ibm_lbm_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// lets other translation units report through ibm_lbm_last_error()
void ibmlbm::set_last_error(const std::string& msg) { g_err = msg; }

extern "C" {

// ------------------------------------------------------ standalone pair search
namespace {
int pair_domain(int32_t dim, const int32_t* n_nodes, const int32_t* periodic, double diameter,
                double zeta, int32_t n, int32_t max_neighbors, double* L, int* per, int* nc,
                double* H, int* kmax) {
  if (dim != 2 && dim != 3) return fail(IBMLBM_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (!n_nodes) return fail(IBMLBM_ERR_INVALID_ARG, "n_nodes is NULL");
  if (n < 0) return fail(IBMLBM_ERR_INVALID_ARG, "n < 0");
  if (!(diameter > 0.0) || !(zeta > 0.0))
    return fail(IBMLBM_ERR_INVALID_ARG, "diameter and zeta must be > 0");
  if (max_neighbors < 0 || max_neighbors > 64)
    return fail(IBMLBM_ERR_INVALID_ARG, "max_neighbors must be in 0..64");
  for (int k = 0; k < 3; ++k) {
    L[k] = k < dim ? (double)n_nodes[k] : 1.0;
    per[k] = (k < dim && periodic) ? (periodic[k] ? 1 : 0) : 0;
    if (k < dim && n_nodes[k] < 1) return fail(IBMLBM_ERR_INVALID_ARG, "n_nodes must be >= 1");
  }
  cell_grid(dim, L, per, diameter + zeta, nc, H);
  *kmax = max_neighbors ? max_neighbors : 32;
  return IBMLBM_OK;
}
}  // namespace

int ibm_lbm_pair_search_scratch_size(int32_t dim, const int32_t* n_nodes, double diameter,
                                     double zeta, int32_t n, int32_t max_neighbors,
                                     size_t* bytes) {
  double L[3], H[3];
  int per[3], nc[3], kmax;
  int rc = pair_domain(dim, n_nodes, nullptr, diameter, zeta, n, max_neighbors, L, per, nc, H, &kmax);
  if (rc) return rc;
  if (!bytes) return fail(IBMLBM_ERR_INVALID_ARG, "bytes is NULL");
  const PairScratch ps = pair_scratch(n, kmax, nc);
  if (!ps.ok) return fail(IBMLBM_ERR_CAPACITY, "pair-search scratch size does not fit in size_t");
  *bytes = ps.total;
  return IBMLBM_OK;
}

int ibm_lbm_pair_search(int32_t dim, const int32_t* n_nodes, const int32_t* periodic,
                        double diameter, double zeta, int32_t n, const double* d_X,
                        int32_t max_neighbors, void* d_scratch, size_t scratch_bytes,
                        int32_t* d_pairs, int64_t cap, int64_t* h_count, void* stream) {
  double L[3], H[3];
  int per[3], nc[3], kmax;
  int rc = pair_domain(dim, n_nodes, periodic, diameter, zeta, n, max_neighbors, L, per, nc, H, &kmax);
  if (rc) return rc;
  if (!h_count) return fail(IBMLBM_ERR_INVALID_ARG, "count is NULL");
  *h_count = 0;
  if (n == 0) return IBMLBM_OK;
  if (!d_X || (cap > 0 && !d_pairs)) return fail(IBMLBM_ERR_INVALID_ARG, "X or pairs is NULL");
  const PairScratch ps = pair_scratch(n, kmax, nc);
  if (!ps.ok) return fail(IBMLBM_ERR_CAPACITY, "pair-search scratch size does not fit in size_t");
  if (!d_scratch || scratch_bytes < ps.total || reinterpret_cast<uintptr_t>(d_scratch) % kAlign)
    return fail(IBMLBM_ERR_WORKSPACE, "scratch missing, misaligned or too small");
  char* sc = static_cast<char*>(d_scratch);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  PairArgs a{};
  a.wall_lo = -0.5;
  a.g.nx = (int)L[0];
  a.g.ny = (int)L[1];
  a.g.nz = (int)L[2];
  for (int k = 0; k < 3; ++k) {
    a.g.per[k] = per[k];
    a.nc[k] = nc[k];
    a.H[k] = H[k];
    a.L[k] = L[k];
  }
  a.D = dim;
  a.n = n;
  a.diam = diameter;
  a.zeta = zeta;
  const double thr = diameter + zeta;
  a.thr2 = thr * thr;
  a.kmax = kmax;
  a.X = d_X;
  a.cell_count = reinterpret_cast<int*>(sc + ps.cell_count);
  a.cell_ids = reinterpret_cast<int*>(sc + ps.cell_ids);
  a.cell_cap = ps.cell_cap;
  a.nbr = reinterpret_cast<int*>(sc + ps.nbr);
  a.nbr_count = reinterpret_cast<int*>(sc + ps.nbr_count);
  a.gt_count = reinterpret_cast<int*>(sc + ps.gt);
  a.status = reinterpret_cast<uint32_t*>(sc + ps.status);
  a.Fc = nullptr;
  CUDA_TRY(cudaMemsetAsync(a.status, 0, sizeof(uint32_t), s));
  CUDA_TRY(launch_pair_cells(a, s));
  CUDA_TRY(launch_pair_contacts(a, s));
  CUDA_TRY(launch_pair_compact(a, d_pairs, cap, s));
  int total = 0;
  uint32_t st = 0;
  CUDA_TRY(cudaMemcpyAsync(&total, a.gt_count + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&st, a.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  *h_count = total;
  if (st & ST_CAPACITY) return fail(IBMLBM_ERR_CAPACITY, "a particle has more than max_neighbors partners");
  if (total > cap) return fail(IBMLBM_ERR_CAPACITY, "more pairs than cap");
  return IBMLBM_OK;
}

}  // extern "C"

// ============================================================= batched ensemble
// Many independent 2D cavities stepped together (an ensemble of cavities of uneven
// size): every member is an ordinary run in its own slice of one workspace, and every
// kernel of a step runs once for all members (fused launches, see Fuse).
namespace {

struct BatchPlan {
  std::vector<size_t> off;        // member workspace offsets
  std::vector<size_t> size;       // member workspace sizes
  size_t tables = 0, total = 0;   // offset of the device tables, total bytes
};

// the launch types of a batched step, in the order of their block maps
// (BK_CW0 + c: the interpolation and spreading blocks of the members of box-size
// class c, launched with that class's shared memory)
constexpr int kMaxBoxClasses = 8;
// the batch's own device words: the grid barriers of its persistent kernels (count,
// generation) and its status word (ST_TIMEOUT), each on its own 128-byte line
constexpr int kBatchWords = 96, kBarIbm = 0, kBarPairs = 32, kBatchStatus = 64;
// polls (about 0.2 us each) before a persistent kernel's grid barrier gives up
constexpr unsigned long long kDefaultBarrierLimit = 10000000ull;
enum { BK_LBM, BK_EDGE, BK_WARP, BK_LANE, BK_HALF, BK_PCLEAR, BK_PINS, BK_PSEARCH, BK_PFORCE, BK_CW0,
       BK_COUNT = BK_CW0 + kMaxBoxClasses };

// Box-size classes of a batch: the distinct particle-box sizes of the members with
// particles, ascending (beyond kMaxBoxClasses the largest sizes share the last class).
// cls[i]: the class of member i (-1 without particles); box[c]: the largest box of c.
struct BoxClasses {
  std::vector<int> cls, box;
};

BoxClasses box_classes(const ibm_lbm_config* cfgs, int32_t n) {
  BoxClasses bc;
  std::vector<int> sizes;
  std::vector<int> mb(n, 0);
  for (int32_t i = 0; i < n; ++i)
    if (cfgs[i].n_particles > 0) {
      mb[i] = derive(&cfgs[i]).box;
      sizes.push_back(mb[i]);
    }
  std::sort(sizes.begin(), sizes.end());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  for (size_t c = 0; c < sizes.size(); ++c) {
    if (c < (size_t)kMaxBoxClasses) bc.box.push_back(sizes[c]);
    else bc.box.back() = sizes[c];
  }
  bc.cls.assign(n, -1);
  for (int32_t i = 0; i < n; ++i) {
    if (cfgs[i].n_particles == 0) continue;
    int c = 0;
    while (c + 1 < (int)bc.box.size() && bc.box[c] < mb[i]) ++c;
    bc.cls[i] = c;
  }
  return bc;
}

unsigned member_blocks(int type, const Derived& d, const ibm_lbm_config& c, int cls) {
  const int np = c.n_particles;
  if (type >= BK_CW0) return (np > 0 && cls == type - BK_CW0) ? ibm_warp_blocks(np) : 0;
  switch (type) {
    case BK_LBM: return lbm_step_blocks(d.g, c.pdf_storage);
    case BK_EDGE: return lbm_edge_blocks(d.g, 2);
    case BK_WARP: return np > 0 ? ibm_warp_blocks(np) : 0;
    case BK_LANE: return np > 0 ? ibm_lane_blocks(np) : 0;
    case BK_HALF: return np > 0 ? ibm_half_blocks(np) : 0;
    case BK_PCLEAR: {
      if (np == 0) return 0;
      PairArgs a{};
      for (int k = 0; k < 3; ++k) a.nc[k] = d.nc[k];
      return pair_clear_blocks(a);
    }
    case BK_PINS: return pair_thread_blocks(np, 256);
    case BK_PSEARCH: return pair_warp_blocks(np);
    default: return pair_thread_blocks(np, 128);
  }
}

int check_batch(const ibm_lbm_config* cfgs, int32_t n) {
  if (!cfgs || n <= 0) return fail(IBMLBM_ERR_INVALID_ARG, "a batch needs n > 0 configurations");
  for (int32_t i = 0; i < n; ++i) {
    int rc = check_config(&cfgs[i]);
    if (rc) return rc;
    if (cfgs[i].dim != 2) return fail(IBMLBM_ERR_UNSUPPORTED, "batch members must be 2D");
    if (cfgs[i].pdf_storage == IBMLBM_PDF_BF16)
      return fail(IBMLBM_ERR_UNSUPPORTED, "batch members store PDFs as FP32 or FP16");
    if (cfgs[i].mlp_init) return fail(IBMLBM_ERR_UNSUPPORTED, "batch members use the plain MDF");
    if (cfgs[i].boundary) return fail(IBMLBM_ERR_UNSUPPORTED, "batch members use halfway bounce-back walls");
    if (cfgs[i].pair_search) return fail(IBMLBM_ERR_UNSUPPORTED, "batch members use the cell-list search");
    if (cfgs[i].pdf_storage != cfgs[0].pdf_storage || cfgs[i].mdf_iters != cfgs[0].mdf_iters)
      return fail(IBMLBM_ERR_INVALID_ARG, "batch members must share pdf_storage and mdf_iters");
  }
  return IBMLBM_OK;
}

size_t batch_table_bytes(const ibm_lbm_config* cfgs, int32_t n) {
  size_t blocks = 0;
  const BoxClasses bc = box_classes(cfgs, n);
  for (int32_t i = 0; i < n; ++i) {
    const Derived d = derive(&cfgs[i]);
    for (int t = 0; t < BK_COUNT; ++t) blocks += member_blocks(t, d, cfgs[i], bc.cls[i]);
  }
  // args: Lbm x2, Ibm x2, Regen x2, Pair x4 per member; maps: first[] per type, cav[] per
  // block, and a tile prefix table [n + 1] per lbm_step tile shape (each table padded to 16 bytes)
  const size_t args = (size_t)n * (2 * sizeof(LbmArgs) + 2 * sizeof(IbmArgs) + 2 * sizeof(RegenArgs) +
                                   4 * sizeof(PairArgs));
  const size_t tiles = (size_t)tile_shape_count() * (sizeof(int) * (n + 1) + 16);
  return args + sizeof(int) * (blocks + (size_t)BK_COUNT * n) + tiles + kBatchWords * sizeof(unsigned) + 4096;
}

BatchPlan plan_batch(const ibm_lbm_config* cfgs, int32_t n) {
  BatchPlan p;
  Carver cv;
  for (int32_t i = 0; i < n; ++i) {
    const size_t b = carve(&cfgs[i], derive(&cfgs[i])).total;
    p.size.push_back(b);
    p.off.push_back(cv.take(b));
  }
  p.tables = cv.take(batch_table_bytes(cfgs, n));
  p.total = cv.off;
  return p;
}

}  // namespace

constexpr int kMaxTileShapes = 16;

struct ibm_lbm_batch {
  int n;
  std::vector<ibm_lbm_handle*> m;
  cudaStream_t s;
  cudaStream_t side;
  cudaEvent_t fork0, fork, join;
  bool mlp_set;     // learned-initializer parameters copied in
  bool track_res;   // residual pass after the last MDF iteration
  long long res_step;  // step whose residual the buffer holds (-1: none)
  int store, mdf;
  size_t smem;                   // 2D IBM shared memory for the largest box
  // box-size classes: one interpolation / spreading launch per class, with the class's
  // shared memory, on its own high-priority stream (forked and joined per phase)
  int nclass;
  size_t class_smem[kMaxBoxClasses];
  cudaStream_t cstream[kMaxBoxClasses];
  cudaEvent_t cev[kMaxBoxClasses];
  cudaEvent_t phase;
  unsigned blocks[BK_COUNT];
  // device tables
  LbmArgs* lbm_args[2];
  IbmArgs* ibm_args[2];
  RegenArgs* regen_args[2];      // [p]: regeneration into parity p
  PairArgs* pair_args[2][2];     // [parity][have_prev]
  int* first[BK_COUNT];
  int* cav[BK_COUNT];
  // lbm_step tile shape (0: row tiles through the block map; >= 1: warp tiles through
  // a per-shape prefix table of the members' tile counts)
  int shape;
  int* tile_first[kMaxTileShapes];
  int tile_total[kMaxTileShapes];
  long long step;
  int have_prev;
  int64_t launches;
  bool graph_ok[2], graph_tried[2];
  cudaGraphExec_t graph[2];
  int graph_kernels[2];
  // persistent mode: the IBM phases and the contact phases as one cooperative kernel each
  bool persistent;
  unsigned long long barrier_limit;
  unsigned* words;  // kBatchWords device words (barriers, status)
};

namespace {

Fuse fuse(const ibm_lbm_batch* b, int type, const void* args) { return Fuse{args, b->cav[type], b->first[type]}; }

// ev (or null): events recorded around the lbm_step launches (tile-shape tuning)
int enqueue_batch_step(ibm_lbm_batch* b, int parity, int have_prev, int* nk, cudaEvent_t* ev = nullptr) {
  const cudaStream_t s = b->s;
  int k = 0;
  const unsigned* B = b->blocks;
  const void* ia = b->ibm_args[parity];
  // one interpolation or spreading phase: a single launch over all members, or one
  // launch per box-size class on the class streams (forked from and joined into s)
  auto phase = [&](bool spread, int m) -> int {
    auto one = [&](int type, size_t smem, cudaStream_t st) -> cudaError_t {
      return spread ? launch_ibm_spread_fused(fuse(b, type, ia), B[type], smem, st)
                    : launch_ibm_interp_fused(fuse(b, type, ia), B[type], smem, m, parity, b->store, st);
    };
    if (b->nclass <= 1) {
      CUDA_TRY(one(BK_WARP, b->smem, s));
      ++k;
      return IBMLBM_OK;
    }
    CUDA_TRY(cudaEventRecord(b->phase, s));
    for (int c = 0; c < b->nclass; ++c) {
      if (!B[BK_CW0 + c]) continue;
      CUDA_TRY(cudaStreamWaitEvent(b->cstream[c], b->phase, 0));
      CUDA_TRY(one(BK_CW0 + c, b->class_smem[c], b->cstream[c]));
      CUDA_TRY(cudaEventRecord(b->cev[c], b->cstream[c]));
      ++k;
    }
    for (int c = 0; c < b->nclass; ++c)
      if (B[BK_CW0 + c]) CUDA_TRY(cudaStreamWaitEvent(s, b->cev[c], 0));
    return IBMLBM_OK;
  };
  if (B[BK_WARP] && b->persistent) {
    // regeneration of this step's points, the MDF iterations and the force sums in one
    // kernel; the contacts and the particle update in one kernel beside the collision
    IbmBatch P{};
    P.regen = fuse(b, BK_LANE, b->regen_args[parity]);
    P.warp = fuse(b, BK_WARP, ia);
    P.lane = fuse(b, BK_LANE, ia);
    P.nwarp = B[BK_WARP];
    P.nlane = B[BK_LANE];
    P.mdf = b->mdf;
    P.bar = b->words + kBarIbm;
    P.limit = b->barrier_limit;
    P.status = b->words + kBatchStatus;
    CUDA_TRY(launch_ibm_batch(P, parity, b->store, b->smem, s, false));
    ++k;
    CUDA_TRY(cudaEventRecord(b->fork, s));
    CUDA_TRY(cudaStreamWaitEvent(b->side, b->fork, 0));
    const void* pa = b->pair_args[parity][have_prev];
    PairBatch Q{};
    Q.clear = fuse(b, BK_PCLEAR, pa);
    Q.ins = fuse(b, BK_PINS, pa);
    Q.search = fuse(b, BK_PSEARCH, pa);
    Q.force = fuse(b, BK_PFORCE, pa);
    Q.nclear = B[BK_PCLEAR];
    Q.nins = B[BK_PINS];
    Q.nsearch = B[BK_PSEARCH];
    Q.nforce = B[BK_PFORCE];
    Q.bar = b->words + kBarPairs;
    Q.limit = b->barrier_limit;
    Q.status = b->words + kBatchStatus;
    CUDA_TRY(launch_pairs_batch(Q, b->side));
    ++k;
    CUDA_TRY(cudaEventRecord(b->join, b->side));
  } else if (B[BK_WARP]) {
    // cell and partner lists beside the IBM kernels (they need only the step's centres)
    const void* pa = b->pair_args[parity][have_prev];
    CUDA_TRY(cudaEventRecord(b->fork0, s));
    CUDA_TRY(cudaStreamWaitEvent(b->side, b->fork0, 0));
    CUDA_TRY(launch_pairs_fused(fuse(b, BK_PCLEAR, pa), B[BK_PCLEAR], fuse(b, BK_PINS, pa), B[BK_PINS],
                                fuse(b, BK_PSEARCH, pa), B[BK_PSEARCH], fuse(b, BK_PFORCE, pa), 0, b->side));
    k += 3;
    int rc;
    if (b->mdf == 0 && (rc = phase(false, 0)) != IBMLBM_OK) return rc;
    for (int m = 1; m <= b->mdf; ++m) {
      if ((rc = phase(false, m)) != IBMLBM_OK) return rc;
      if ((rc = phase(true, m)) != IBMLBM_OK) return rc;
    }
    CUDA_TRY(launch_ibm_forces_fused(fuse(b, BK_HALF, ia), B[BK_HALF], s));
    ++k;
    // contact forces, particle update and regeneration beside the collision (as in a
    // single run)
    CUDA_TRY(cudaEventRecord(b->fork, s));
    CUDA_TRY(cudaStreamWaitEvent(b->side, b->fork, 0));
    CUDA_TRY(launch_pairs_fused(fuse(b, BK_PCLEAR, pa), 0, fuse(b, BK_PINS, pa), 0, fuse(b, BK_PSEARCH, pa), 0,
                                fuse(b, BK_PFORCE, pa), B[BK_PFORCE], b->side));
    k += 1;
    CUDA_TRY(launch_regen_fused(fuse(b, BK_LANE, b->regen_args[1 - parity]), B[BK_LANE], b->side));
    ++k;
    CUDA_TRY(cudaEventRecord(b->join, b->side));
  }
  const void* la = b->lbm_args[parity];
  if (ev) CUDA_TRY(cudaEventRecord(ev[0], s));
  if (b->shape == 0)
    CUDA_TRY(launch_lbm_step_fused(fuse(b, BK_LBM, la), B[BK_LBM], fuse(b, BK_EDGE, la), B[BK_EDGE], b->store,
                                   parity, s));
  else
    CUDA_TRY(launch_lbm_step_tiles(b->shape, b->lbm_args[parity], b->tile_first[b->shape], b->n,
                                   b->tile_total[b->shape], fuse(b, BK_EDGE, la), B[BK_EDGE], b->store, parity, s));
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], s));
  k += (parity == 1 && B[BK_EDGE] && b->shape != 0) ? 2 : 1;  // shape 0: one launch
  if (B[BK_WARP]) CUDA_TRY(cudaStreamWaitEvent(s, b->join, 0));
  *nk = k;
  return IBMLBM_OK;
}

int capture_batch_graph(ibm_lbm_batch* b, int parity) {
  cudaGraph_t graph = nullptr;
  int nk = 0;
  if (cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return IBMLBM_ERR_CUDA;
  }
  const int rc = enqueue_batch_step(b, parity, 1, &nk);
  const cudaError_t e = cudaStreamEndCapture(b->s, &graph);
  if (rc != IBMLBM_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return IBMLBM_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return IBMLBM_ERR_CUDA;
  }
  cudaGraphDestroy(graph);
  b->graph[parity] = exec;
  b->graph_kernels[parity] = nk;
  b->graph_ok[parity] = true;
  return IBMLBM_OK;
}

void destroy_batch(ibm_lbm_batch* b) {
  for (ibm_lbm_handle* h : b->m) ibm_lbm_destroy(h);
  for (int p = 0; p < 2; ++p)
    if (b->graph_ok[p]) cudaGraphExecDestroy(b->graph[p]);
  if (b->side) {
    cudaStreamSynchronize(b->side);
    cudaStreamDestroy(b->side);
  }
  if (b->fork0) cudaEventDestroy(b->fork0);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  for (int c = 0; c < kMaxBoxClasses; ++c) {
    if (b->cstream[c]) {
      cudaStreamSynchronize(b->cstream[c]);
      cudaStreamDestroy(b->cstream[c]);
    }
    if (b->cev[c]) cudaEventDestroy(b->cev[c]);
  }
  if (b->phase) cudaEventDestroy(b->phase);
  delete b;
}

}  // namespace

extern "C" {

int ibm_lbm_batch_workspace_size(const ibm_lbm_config* cfgs, int32_t n, size_t* bytes) {
  int rc = check_batch(cfgs, n);
  if (rc) return rc;
  if (!bytes) return fail(IBMLBM_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = plan_batch(cfgs, n).total;
  return IBMLBM_OK;
}

int ibm_lbm_batch_init(const ibm_lbm_config* cfgs, int32_t n, void* d_workspace, size_t bytes,
                       void* stream, const double* const* h_centres, ibm_lbm_batch** out) {
  int rc = check_batch(cfgs, n);
  if (rc) return rc;
  if (!out) return fail(IBMLBM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  const BatchPlan plan = plan_batch(cfgs, n);
  if (!d_workspace || bytes < plan.total)
    return fail(IBMLBM_ERR_WORKSPACE, "batch workspace missing or too small");
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
    return fail(IBMLBM_ERR_WORKSPACE, "batch workspace must be 256-byte aligned");
  ibm_lbm_batch* b = new ibm_lbm_batch();
  b->n = n;
  b->s = static_cast<cudaStream_t>(stream);
  b->side = nullptr;
  b->fork0 = b->fork = b->join = nullptr;
  b->store = cfgs[0].pdf_storage;
  b->mdf = cfgs[0].mdf_iters;
  b->step = 0;
  b->have_prev = 0;
  b->launches = 0;
  b->graph_ok[0] = b->graph_ok[1] = b->graph_tried[0] = b->graph_tried[1] = false;
  b->persistent = false;
  b->barrier_limit = kDefaultBarrierLimit;
  b->words = nullptr;
  char* ws = static_cast<char*>(d_workspace);
  auto bail = [&](int code) {
    const std::string msg = g_err;
    destroy_batch(b);
    g_err = msg;
    return code;
  };
#define BATCH_TRY(expr)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bail(fail(IBMLBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  {
    // the side stream's short particle kernels at the highest priority: the block
    // scheduler then places their blocks ahead of lbm_step's as SMs free up, so they
    // finish inside lbm_step's time instead of after it
    int lo_ = 0, hi_ = 0;
    BATCH_TRY(cudaDeviceGetStreamPriorityRange(&lo_, &hi_));
    BATCH_TRY(cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, hi_));
  }
  BATCH_TRY(cudaEventCreateWithFlags(&b->fork0, cudaEventDisableTiming));
  BATCH_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  BATCH_TRY(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
  int maxbox = 0;
  for (int32_t i = 0; i < n; ++i) {
    ibm_lbm_handle* h = nullptr;
    rc = ibm_lbm_init(&cfgs[i], ws + plan.off[i], plan.size[i], stream,
                      h_centres ? h_centres[i] : nullptr, &h);
    if (rc) return bail(rc);
    b->m.push_back(h);
    if (cfgs[i].n_particles > 0) maxbox = std::max(maxbox, h->d.box);
  }
  b->smem = maxbox ? ibm_box2_smem(maxbox) : 0;
  if (maxbox && b->smem > 227 * 1024) return bail(fail(IBMLBM_ERR_UNSUPPORTED, "particle too large"));
  if (maxbox) BATCH_TRY(prepare_ibm_spread(2, b->smem));
  const BoxClasses bc = box_classes(cfgs, n);
  b->nclass = (int)bc.box.size();
  for (int c = 0; c < b->nclass; ++c) b->class_smem[c] = ibm_box2_smem(bc.box[c]);
  if (b->nclass > 1) {
    int lo_ = 0, hi_ = 0;
    BATCH_TRY(cudaDeviceGetStreamPriorityRange(&lo_, &hi_));
    for (int c = 0; c < b->nclass; ++c) {
      BATCH_TRY(cudaStreamCreateWithPriority(&b->cstream[c], cudaStreamNonBlocking, hi_));
      BATCH_TRY(cudaEventCreateWithFlags(&b->cev[c], cudaEventDisableTiming));
    }
    BATCH_TRY(cudaEventCreateWithFlags(&b->phase, cudaEventDisableTiming));
  }
  // host copies of the tables, then one copy to the device
  std::vector<char> host(batch_table_bytes(cfgs, n), 0);
  size_t o = 0;
  auto put = [&](const void* src, size_t len) {
    const size_t at_ = o;
    std::memcpy(host.data() + o, src, len);
    o = (o + len + 15) / 16 * 16;
    return at_;
  };
  size_t o_lbm[2], o_ibm[2], o_regen[2], o_pair[2][2], o_first[BK_COUNT], o_cav[BK_COUNT];
  for (int p = 0; p < 2; ++p) {
    std::vector<LbmArgs> la;
    std::vector<IbmArgs> ia;
    std::vector<RegenArgs> ra;
    for (ibm_lbm_handle* h : b->m) {
      la.push_back(h->lbm(p));
      ia.push_back(h->ibm(p));
      ra.push_back(h->regen(p));
    }
    o_lbm[p] = put(la.data(), sizeof(LbmArgs) * n);
    o_ibm[p] = put(ia.data(), sizeof(IbmArgs) * n);
    o_regen[p] = put(ra.data(), sizeof(RegenArgs) * n);
    for (int hp = 0; hp < 2; ++hp) {
      std::vector<PairArgs> pa;
      for (ibm_lbm_handle* h : b->m) pa.push_back(h->pairs(p, hp));
      o_pair[p][hp] = put(pa.data(), sizeof(PairArgs) * n);
    }
  }
  for (int t = 0; t < BK_COUNT; ++t) {
    std::vector<int> first(n), cav;
    for (int32_t i = 0; i < n; ++i) {
      first[i] = (int)cav.size();
      const unsigned c = member_blocks(t, b->m[i]->d, cfgs[i], bc.cls[i]);
      cav.insert(cav.end(), c, i);
    }
    b->blocks[t] = (unsigned)cav.size();
    o_first[t] = put(first.data(), sizeof(int) * n);
    o_cav[t] = cav.empty() ? o : put(cav.data(), sizeof(int) * cav.size());
  }
  std::vector<unsigned> words(kBatchWords, 0u);
  const size_t o_words = put(words.data(), sizeof(unsigned) * kBatchWords);
  size_t o_tile[kMaxTileShapes] = {};
  b->shape = 0;
  for (int sh = 1; sh < tile_shape_count(); ++sh) {
    std::vector<int> first(n + 1, 0);
    long long tot = 0;
    for (int32_t i = 0; i < n; ++i) {
      first[i] = (int)tot;
      tot += tile_count(b->m[i]->d.g, sh);
    }
    if (tot > INT32_MAX) return bail(fail(IBMLBM_ERR_UNSUPPORTED, "batch too large for the tile tables"));
    first[n] = (int)tot;
    b->tile_total[sh] = (int)tot;
    o_tile[sh] = put(first.data(), sizeof(int) * (n + 1));
  }
  if (o > host.size()) return bail(fail(IBMLBM_ERR_WORKSPACE, "batch tables overflow"));
  char* dt = ws + plan.tables;
  BATCH_TRY(cudaMemcpyAsync(dt, host.data(), o, cudaMemcpyHostToDevice, b->s));
  BATCH_TRY(cudaStreamSynchronize(b->s));
  for (int p = 0; p < 2; ++p) {
    b->lbm_args[p] = reinterpret_cast<LbmArgs*>(dt + o_lbm[p]);
    b->ibm_args[p] = reinterpret_cast<IbmArgs*>(dt + o_ibm[p]);
    b->regen_args[p] = reinterpret_cast<RegenArgs*>(dt + o_regen[p]);
    for (int hp = 0; hp < 2; ++hp) b->pair_args[p][hp] = reinterpret_cast<PairArgs*>(dt + o_pair[p][hp]);
  }
  for (int t = 0; t < BK_COUNT; ++t) {
    b->first[t] = reinterpret_cast<int*>(dt + o_first[t]);
    b->cav[t] = reinterpret_cast<int*>(dt + o_cav[t]);
  }
  for (int sh = 1; sh < tile_shape_count(); ++sh) b->tile_first[sh] = reinterpret_cast<int*>(dt + o_tile[sh]);
  b->words = reinterpret_cast<unsigned*>(dt + o_words);
#undef BATCH_TRY
  *out = b;
  return IBMLBM_OK;
}

}  // extern "C"

namespace {

void advance_batch(ibm_lbm_batch* b) {
  b->step += 1;
  b->have_prev = 1;
  for (ibm_lbm_handle* h : b->m) {  // the members' own clocks (their I/O reads by parity)
    h->step += 1;
    h->have_prev = 1;
  }
}

void drop_batch_graphs(ibm_lbm_batch* b) {
  for (int p = 0; p < 2; ++p) {
    if (b->graph_ok[p]) cudaGraphExecDestroy(b->graph[p]);
    b->graph_ok[p] = b->graph_tried[p] = false;
  }
}

}  // namespace

extern "C" {

int ibm_lbm_batch_step(ibm_lbm_batch* b, int32_t n_steps) {
  if (!b) return fail(IBMLBM_ERR_INVALID_ARG, "batch is NULL");
  if (n_steps < 0) return fail(IBMLBM_ERR_INVALID_ARG, "n_steps < 0");
  for (int32_t t = 0; t < n_steps; ++t) {
    const int parity = (int)(b->step & 1);
    if (b->have_prev && !b->graph_tried[parity]) {
      b->graph_tried[parity] = true;
      capture_batch_graph(b, parity);  // on failure the steps run as eager launches
    }
    if (b->have_prev && b->graph_ok[parity]) {
      CUDA_TRY(cudaGraphLaunch(b->graph[parity], b->s));
      b->launches += b->graph_kernels[parity];
    } else {
      int nk = 0;
      const int rc = enqueue_batch_step(b, parity, b->have_prev, &nk);
      if (rc) return rc;
      b->launches += nk;
    }
    advance_batch(b);
  }
  return IBMLBM_OK;
}

int ibm_lbm_tile_shape_count(void) { return tile_shape_count(); }

int ibm_lbm_tile_shape(int32_t shape, int32_t pdf_storage, int32_t* nodes_per_thread,
                       int32_t* warps_per_block, int32_t* persistent) {
  if (shape < 0 || shape >= tile_shape_count()) return fail(IBMLBM_ERR_INVALID_ARG, "no such tile shape");
  if (pdf_storage != IBMLBM_PDF_FP32 && pdf_storage != IBMLBM_PDF_FP16)
    return fail(IBMLBM_ERR_INVALID_ARG, "a batch stores FP32 or FP16");
  int k = 0, w = 0, p = 0;
  tile_shape(shape, pdf_storage, &k, &w, &p);
  if (nodes_per_thread) *nodes_per_thread = k;
  if (warps_per_block) *warps_per_block = w;
  if (persistent) *persistent = p;
  return IBMLBM_OK;
}

int ibm_lbm_batch_set_tile_shape(ibm_lbm_batch* b, int32_t shape) {
  if (!b) return fail(IBMLBM_ERR_INVALID_ARG, "batch is NULL");
  if (shape < 0 || shape >= tile_shape_count()) return fail(IBMLBM_ERR_INVALID_ARG, "no such tile shape");
  if (shape != b->shape) {
    b->shape = shape;
    drop_batch_graphs(b);  // captured with the old shape
  }
  return IBMLBM_OK;
}

int ibm_lbm_batch_get_tile_shape(const ibm_lbm_batch* b, int32_t* shape) {
  if (!b || !shape) return fail(IBMLBM_ERR_INVALID_ARG, "batch or shape is NULL");
  *shape = b->shape;
  return IBMLBM_OK;
}

int ibm_lbm_batch_autotune(ibm_lbm_batch* b, int32_t steps_per_shape, float* h_ms_per_shape) {
  if (!b) return fail(IBMLBM_ERR_INVALID_ARG, "batch is NULL");
  if (steps_per_shape < 2 || steps_per_shape % 2 != 0)
    return fail(IBMLBM_ERR_INVALID_ARG, "steps_per_shape must be even and >= 2");
  const int S = tile_shape_count();
  std::vector<cudaEvent_t> ev((size_t)2 * S * steps_per_shape, nullptr);
  auto done = [&](int code) {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    return code;
  };
  for (cudaEvent_t& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return done(fail(IBMLBM_ERR_CUDA, "cudaEventCreate failed"));
  drop_batch_graphs(b);
  for (int sh = 0; sh < S; ++sh) {
    b->shape = sh;
    for (int j = 0; j < steps_per_shape; ++j) {
      int nk = 0;
      const int rc = enqueue_batch_step(b, (int)(b->step & 1), b->have_prev, &nk,
                                        &ev[(size_t)2 * (sh * steps_per_shape + j)]);
      if (rc) return done(rc);
      b->launches += nk;
      advance_batch(b);
    }
  }
  if (cudaStreamSynchronize(b->s) != cudaSuccess) return done(fail(IBMLBM_ERR_CUDA, "tuning steps failed"));
  int best = 0;
  std::vector<float> ms(S, 0.0f);
  for (int sh = 0; sh < S; ++sh) {
    for (int j = 0; j < steps_per_shape; ++j) {
      float t = 0.0f;
      const size_t e = (size_t)2 * (sh * steps_per_shape + j);
      if (cudaEventElapsedTime(&t, ev[e], ev[e + 1]) != cudaSuccess)
        return done(fail(IBMLBM_ERR_CUDA, "cudaEventElapsedTime failed"));
      ms[sh] += t / steps_per_shape;
    }
    if (ms[sh] < ms[best]) best = sh;
  }
  b->shape = best;
  if (h_ms_per_shape) std::copy(ms.begin(), ms.end(), h_ms_per_shape);
  return done(IBMLBM_OK);
}

int ibm_lbm_batch_sync(ibm_lbm_batch* b) {
  if (!b) return fail(IBMLBM_ERR_INVALID_ARG, "batch is NULL");
  CUDA_TRY(cudaStreamSynchronize(b->s));
  uint32_t st = 0;
  CUDA_TRY(cudaMemcpy(&st, b->words + kBatchStatus, sizeof(st), cudaMemcpyDeviceToHost));
  if (st) {
    // a barrier gave up: its count may be left short, so both barriers start afresh
    CUDA_TRY(cudaMemset(b->words, 0, sizeof(unsigned) * kBatchWords));
  }
  int first_rc = IBMLBM_OK;
  for (ibm_lbm_handle* h : b->m) {
    const int rc = ibm_lbm_sync(h);
    if (rc && !first_rc) first_rc = rc;
  }
  if (st & ST_TIMEOUT) return fail(IBMLBM_ERR_TIMEOUT, "a grid barrier of a persistent batch kernel timed out");
  return first_rc;
}

int ibm_lbm_batch_set_persistent(ibm_lbm_batch* b, int32_t on, int64_t barrier_limit) {
  if (!b) return fail(IBMLBM_ERR_INVALID_ARG, "batch is NULL");
  if (on != 0 && on != 1) return fail(IBMLBM_ERR_INVALID_ARG, "on must be 0 or 1");
  if (barrier_limit < 0) return fail(IBMLBM_ERR_INVALID_ARG, "barrier_limit < 0");
  if (on) {
    // the shared memory of the IBM kernel is granted before any capture
    for (int p = 0; p < 2; ++p) CUDA_TRY(launch_ibm_batch(IbmBatch{}, p, b->store, b->smem, b->s, true));
  }
  b->persistent = on != 0;
  b->barrier_limit = barrier_limit ? (unsigned long long)barrier_limit : kDefaultBarrierLimit;
  drop_batch_graphs(b);  // captured in the other mode or with the old limit
  return IBMLBM_OK;
}

int ibm_lbm_batch_get_persistent(const ibm_lbm_batch* b, int32_t* on) {
  if (!b || !on) return fail(IBMLBM_ERR_INVALID_ARG, "batch or on is NULL");
  *on = b->persistent ? 1 : 0;
  return IBMLBM_OK;
}

ibm_lbm_handle* ibm_lbm_batch_member(ibm_lbm_batch* b, int32_t i) {
  if (!b || i < 0 || i >= b->n) {
    fail(IBMLBM_ERR_INVALID_ARG, "no such batch member");
    return nullptr;
  }
  return b->m[i];
}

int64_t ibm_lbm_batch_launch_count(const ibm_lbm_batch* b) { return b ? b->launches : 0; }

void ibm_lbm_batch_destroy(ibm_lbm_batch* b) {
  if (b) destroy_batch(b);
}

}  // extern "C"
