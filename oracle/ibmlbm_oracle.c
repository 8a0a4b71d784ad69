/*
 * FP64 CPU oracle for the IB-LBM hot path (Jiang, Li & Liu, Part I).
 * TEST INFRASTRUCTURE ONLY: see ibmlbm_oracle.h for scope and conventions.
 *
 * Readings of the paper used here (each is restated at the function that uses it):
 *   R1 units: dh = dt = 1, cs^2 = 1/3, rho_0 = rho_f = 1.
 *   R2 D3Q19 (Eq. 3): the printed z row has 18 entries; the rule
 *      e_a = -e_{a-9} (a >= 10) and the weight groups fix the dropped entry as
 *      e_9 = (-1, 0, 1).
 *   R3 Eq. 6, Eq. 4 and Eq. 8 use the force-corrected velocity of Eq. 7.
 *   R4 walls: halfway bounce-back at -1/2 and n-1/2 on non-periodic axes
 *      (the paper's non-equilibrium extrapolation is not used).
 *   R5 4-point delta: Peskin's function
 *        (3 - 2|r| + sqrt(1 + 4|r| - 4r^2))/8   for |r| <= 1,
 *        (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2))/8 for 1 <= |r| <= 2;
 *      3-point delta: Roma-Peskin-Berger
 *        (1 + sqrt(1 - 3r^2))/3                 for |r| <= 1/2,
 *        (5 - 3|r| - sqrt(1 - 3(1-|r|)^2))/6    for 1/2 <= |r| <= 3/2.
 *   R6 point volume: 2D dV = ds*drs with ds = pi*D/N_L; 3D dV = (pi*D^2/N_L)*drs.
 *   R7 multi-direct forcing: F_b accumulates the per-iteration increments
 *      dF_b = 2 rho_f (U_b - D_I u^(m-1)) / dt and u^(m) = u^(m-1) + dt D_E dF_b/(2 rho_f).
 *      M = 1 is the BTDF scheme of Eq. 9-11.
 *   R8 Lagrangian points: circle theta_k = 2 pi k / N_L; sphere Fibonacci lattice
 *      z_k = 1 - (2k+1)/N_L, phi_k = k*pi*(3 - sqrt 5); radius D/2.
 *   R9 particle motion (Eq. 14-15; the paper gives no closure or integrator).
 *      F_b = (M_p - rho_f V_p) g is the weight less buoyancy.  F_f, T_f (the force
 *      that keeps the interior fluid moving with the particle) are the rate of
 *      change of the momentum and angular momentum of the fluid at the nodes
 *      strictly inside the particle, with the corrected velocity u^(M) of the
 *      current step, differenced over one step (zero on the first step).
 *      F_h = -sum_b F_b dV, T_h = -sum_b r_b x F_b dV enter as the mean of the
 *      current and previous step: Guo's split (Eq. 7-8) applies half of each
 *      step's force to the velocity of either time level, so the physical force
 *      between two levels is that mean; the instantaneous value alternates sign
 *      while the fluid near the surface adjusts.  The explicit update is
 *        (M_p + K) a^n - K a^{n-1} = F_h,mean + F_c + F_f + (M_p - rho_f V_p) g,
 *        U^{n+1} = U^n + a^n, X^{n+1} = X^n + (U^n + U^{n+1})/2,
 *      and likewise for Omega with I_p and K_r.  K = rho_f N_L dV (the fluid shell
 *      the IB force moves in one step), K_r = K R^2 (2D) or 2/3 K R^2 (3D).  The
 *      K terms telescope (momentum is conserved) and change the dynamics only at
 *      O(dt); without them the explicit coupling is unstable once the shell
 *      outweighs the particle (pi D drs rho_f > M_p, rotation already earlier),
 *      which holds for every benchmark configuration.  2D per unit depth
 *      V = pi D^2/4, I = M D^2/8; 3D V = pi D^3/6, I = M D^2/10.
 *   R10 Eq. 16: c_ij = |(rho_p - rho_f) V_p g|, third case read as the sum of the
 *      two printed terms; walls act through a mirror-image particle.
 *   R11 pair rule: (i, j), i < j, is a pair iff |X_i - X_j|^2 < (D + zeta)^2,
 *      with the squared distance summed in axis order without fused multiply-add.
 *   R12 step order: macro -> IBM (MDF) -> collide -> stream -> pair force ->
 *      particle update, explicit coupling (U_b uses U_c of the current step).
 *   R13 non-equilibrium extrapolation (boundary 1, 2; Sec. 6.1-6.2 cite it as their
 *      ref. [48] without formulas): the wall lies on the outermost node x_b of every
 *      non-periodic axis.  After streaming, f_a(x_b) = f_a^eq(p_b, u_b) + f_a(x_f) -
 *      f_a^eq(p_f, u_f), with x_f = x_b + (the sum of the inward normals of the faces
 *      x_b lies on) and (p_f, u_f) the pressure and velocity of x_f (Eq. 5-7 with the
 *      fluid body force: the next step's IB force is not known yet).  Walls: u_b = 0,
 *      p_b = p_f.  Channel (boundary 2): inlet face y = 0 with u_b along y equal to
 *      u_inlet times prod_k 4 c_k (L_k - c_k) / L_k^2 over the other non-periodic axes
 *      (L_k = n_k - 1) and p_b = p_f; outlet face y = ny - 1 with p_b = 0, u_b = u_f.
 *      A node on both a wall face and an inlet or outlet face is a wall node.  The
 *      mirror images of R10 then reflect through the boundary nodes (0 and n - 1).
 */
#include "ibmlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define CS2 (1.0 / 3.0)
#define RHO0 1.0
#define PI 3.14159265358979323846

/* ---------------------------------------------------------------- lattice */

/* Eq. 2: D2Q9 columns; the ordering satisfies e_a = -e_{a-4} for a > 4. */
static const int32_t E_D2Q9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {-1, 1, 0},
    {-1, 0, 0}, {-1, -1, 0}, {0, -1, 0}, {1, -1, 0}};
/* weights stated after Eq. 4: w0 = 4/9, w_{1,3,5,7} = 1/9, w_{2,4,6,8} = 1/36 */
static const double W_D2Q9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 9, 1.0 / 36,
                                 1.0 / 9, 1.0 / 36, 1.0 / 9, 1.0 / 36};
/* Eq. 3 with reading R2; e_a = -e_{a-9} for a >= 10. */
static const int32_t E_D3Q19[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {0, 1, 0},   {0, 0, 1},  {1, 1, 0},
    {-1, 1, 0}, {0, 1, 1},   {0, -1, 1},  {1, 0, 1},  {-1, 0, 1},
    {-1, 0, 0}, {0, -1, 0},  {0, 0, -1},  {-1, -1, 0}, {1, -1, 0},
    {0, -1, -1}, {0, 1, -1}, {-1, 0, -1}, {1, 0, -1}};
/* w0 = 1/3, w_{1-3,10-12} = 1/18, w_{4-9,13-18} = 1/36 */
static const double W_D3Q19[19] = {
    1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 36, 1.0 / 36, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

typedef struct {
  int q;
  int half; /* (q-1)/2: opposite of a (1 <= a <= half) is a + half */
  int e[19][3];
  double w[19];
} lattice;

static void lattice_init(int dim, lattice* L) {
  int a, k;
  L->q = (dim == 2) ? 9 : 19;
  L->half = (L->q - 1) / 2;
  for (a = 0; a < L->q; ++a) {
    for (k = 0; k < 3; ++k) L->e[a][k] = (dim == 2) ? E_D2Q9[a][k] : E_D3Q19[a][k];
    L->w[a] = (dim == 2) ? W_D2Q9[a] : W_D3Q19[a];
  }
}

static int opposite(const lattice* L, int a) {
  if (a == 0) return 0;
  return (a <= L->half) ? a + L->half : a - L->half;
}

int or_lattice(int32_t dim, int32_t* q, int32_t* e, double* w) {
  lattice L;
  int a, k;
  if (dim != 2 && dim != 3) return -1;
  lattice_init(dim, &L);
  *q = L.q;
  for (a = 0; a < L.q; ++a) {
    for (k = 0; k < 3; ++k) e[3 * a + k] = L.e[a][k];
    w[a] = L.w[a];
  }
  return 0;
}

/* ------------------------------------------------------ node operators */

/* Eq. 4: f_eq = lambda_a p + rho0 w_a [e.u/cs2 + (e.u)^2/(2 cs4) - |u|^2/(2 cs2)],
 * lambda_0 = (w0 - 1)/cs2, lambda_a = w_a/cs2 (a > 0). */
static void feq_node(const lattice* L, double p, const double* u, double* feq) {
  int a;
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (a = 0; a < L->q; ++a) {
    double eu = L->e[a][0] * u[0] + L->e[a][1] * u[1] + L->e[a][2] * u[2];
    double lambda = (a == 0) ? (L->w[0] - 1.0) / CS2 : L->w[a] / CS2;
    feq[a] = lambda * p +
             RHO0 * L->w[a] * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
  }
}

/* Eq. 8: F_a = (1 - 1/(2 tau)) w_a [(e_a - u)/cs2 + (e_a.u)/cs4 e_a] . f */
static void force_node(const lattice* L, double tau, const double* u, const double* F,
                       double* Fa) {
  int a, k;
  for (a = 0; a < L->q; ++a) {
    double eu = L->e[a][0] * u[0] + L->e[a][1] * u[1] + L->e[a][2] * u[2];
    double s = 0.0;
    for (k = 0; k < 3; ++k)
      s += ((L->e[a][k] - u[k]) / CS2 + eu / (CS2 * CS2) * L->e[a][k]) * F[k];
    Fa[a] = (1.0 - 1.0 / (2.0 * tau)) * L->w[a] * s;
  }
}

/* Eq. 5 (u* = sum e f), Eq. 7 (u = u* + dt f / (2 rho)), Eq. 6 with the corrected u (R3). */
static void macro_node(const lattice* L, const double* fnode, const double* F, double* ustar,
                       double* u, double* p) {
  int a, k;
  double s = 0.0, uu;
  for (k = 0; k < 3; ++k) ustar[k] = 0.0;
  for (a = 0; a < L->q; ++a)
    for (k = 0; k < 3; ++k) ustar[k] += L->e[a][k] * fnode[a];
  for (k = 0; k < 3; ++k) u[k] = ustar[k] + F[k] / (2.0 * RHO0);
  for (a = 1; a < L->q; ++a) s += fnode[a];
  uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  *p = CS2 / (1.0 - L->w[0]) * (s - RHO0 * L->w[0] * uu / (2.0 * CS2));
}

void or_feq(int32_t dim, double p, const double* u, double* feq) {
  lattice L;
  lattice_init(dim, &L);
  feq_node(&L, p, u, feq);
}

void or_force_term(int32_t dim, double tau, const double* u, const double* F, double* Fa) {
  lattice L;
  lattice_init(dim, &L);
  force_node(&L, tau, u, F, Fa);
}

void or_macro(int32_t dim, const double* fnode, const double* F, double* ustar, double* u,
              double* p) {
  lattice L;
  lattice_init(dim, &L);
  macro_node(&L, fnode, F, ustar, u, p);
}

/* ------------------------------------------------------------ delta (R5) */

double or_delta(int32_t kind, double r) {
  double a = fabs(r);
  if (kind == 4) {
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
  }
  if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
  if (a <= 1.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
  return 0.0;
}

/* ------------------------------------------------------------ geometry */

static long node_index(int nx, int ny, int x, int y, int z) {
  return (long)x + (long)nx * ((long)y + (long)ny * z);
}

/* Target of a move from coordinate c by step s along an axis of n nodes:
 * returns 1 and the wrapped coordinate if it is inside, 0 if it leaves through a wall. */
static int move_axis(int c, int s, int n, int periodic, int* out) {
  int t = c + s;
  if (t >= 0 && t < n) {
    *out = t;
    return 1;
  }
  if (!periodic) return 0;
  *out = (t + n) % n;
  return 1;
}

/* Eq. 18 push streaming f_a(x + e_a) = fp_a(x); a population leaving through a wall
 * returns to its node in the opposite direction (R4). */
void or_stream_push(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const int32_t* periodic,
                    const double* fp, double* f) {
  lattice L;
  long N = (long)nx * ny * nz;
  int x, y, z, a;
  lattice_init(dim, &L);
#pragma omp parallel for collapse(2) private(x, a)
  for (z = 0; z < nz; ++z)
    for (y = 0; y < ny; ++y)
      for (x = 0; x < nx; ++x) {
        long n = node_index(nx, ny, x, y, z);
        for (a = 0; a < L.q; ++a) {
          int tx, ty, tz;
          int in = move_axis(x, L.e[a][0], nx, periodic[0], &tx) &&
                   move_axis(y, L.e[a][1], ny, periodic[1], &ty) &&
                   move_axis(z, L.e[a][2], nz, periodic[2], &tz);
          if (in)
            f[(long)a * N + node_index(nx, ny, tx, ty, tz)] = fp[(long)a * N + n];
          else
            f[(long)opposite(&L, a) * N + n] = fp[(long)a * N + n];
        }
      }
}

static void swap_d(double* a, double* b) {
  double t = *a;
  *a = *b;
  *b = t;
}

/* Sec. 3.3 swap streaming on a single post-collision array: first the local swap of
 * each a (1..half) with its opposite, then the adjacent swap of f[x][a+half] with
 * f[x+e_a][a] for every x whose neighbour x+e_a is inside the domain.  The adjacent
 * swap uses the index order of the text's second form (a = 1..half paired with
 * the node x+e_a); Table 1 prints the indices the other way round, which streams
 * backwards.  Populations with no in-domain partner stay reversed in place, which
 * is halfway bounce-back. */
void or_stream_swap(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const int32_t* periodic,
                    double* f) {
  lattice L;
  long N = (long)nx * ny * nz;
  int x, y, z, a;
  lattice_init(dim, &L);
  for (z = 0; z < nz; ++z)
    for (y = 0; y < ny; ++y)
      for (x = 0; x < nx; ++x) {
        long n = node_index(nx, ny, x, y, z);
        for (a = 1; a <= L.half; ++a) swap_d(&f[(long)a * N + n], &f[(long)(a + L.half) * N + n]);
      }
  for (z = 0; z < nz; ++z)
    for (y = 0; y < ny; ++y)
      for (x = 0; x < nx; ++x) {
        long n = node_index(nx, ny, x, y, z);
        for (a = 1; a <= L.half; ++a) {
          int tx, ty, tz;
          int in = move_axis(x, L.e[a][0], nx, periodic[0], &tx) &&
                   move_axis(y, L.e[a][1], ny, periodic[1], &ty) &&
                   move_axis(z, L.e[a][2], nz, periodic[2], &tz);
          if (in)
            swap_d(&f[(long)(a + L.half) * N + n],
                   &f[(long)a * N + node_index(nx, ny, tx, ty, tz)]);
        }
      }
}

/* ------------------------------------------------------------------ IBM */

/* Support of the delta function along one axis for point coordinate X (Eq. 47 box):
 * 4-point nodes floor(X)-1 .. floor(X)+2, 3-point nodes round(X)-1 .. round(X)+1.
 * Nodes outside a wall-bounded axis are dropped; periodic axes wrap. */
static int axis_support(int kind, double X, int n, int periodic, int* idx, double* wt) {
  int i0, s, cnt = 0, width = (kind == 4) ? 4 : 3;
  i0 = (kind == 4) ? (int)floor(X) - 1 : (int)floor(X + 0.5) - 1;
  for (s = 0; s < width; ++s) {
    int i = i0 + s;
    double w = or_delta(kind, (double)i - X);
    if (i < 0 || i >= n) {
      if (!periodic) continue;
      i = ((i % n) + n) % n;
    }
    idx[cnt] = i;
    wt[cnt] = w;
    ++cnt;
  }
  return cnt;
}

/* Eq. 47 (with Eq. 12, dh = 1): u_b = sum over the support box of g(x) delta(x-X)delta(y-Y)[delta(z-Z)]. */
void or_interp(const or_params* P, const double* g, int64_t npts, const double* X, double* ub) {
  long N = (long)P->nx * P->ny * P->nz;
  int64_t b;
#pragma omp parallel for
  for (b = 0; b < npts; ++b) {
    int ix[4], iy[4], iz[4], cx, cy, cz, i, j, k, c;
    double wx[4], wy[4], wz[4];
    cx = axis_support(P->delta_kind, X[3 * b + 0], P->nx, P->periodic[0], ix, wx);
    cy = axis_support(P->delta_kind, X[3 * b + 1], P->ny, P->periodic[1], iy, wy);
    if (P->dim == 3) {
      cz = axis_support(P->delta_kind, X[3 * b + 2], P->nz, P->periodic[2], iz, wz);
    } else {
      cz = 1;
      iz[0] = 0;
      wz[0] = 1.0;
    }
    for (c = 0; c < 3; ++c) ub[3 * b + c] = 0.0;
    for (k = 0; k < cz; ++k)
      for (j = 0; j < cy; ++j)
        for (i = 0; i < cx; ++i) {
          long n = node_index(P->nx, P->ny, ix[i], iy[j], iz[k]);
          double w = wx[i] * wy[j] * wz[k];
          for (c = 0; c < P->dim; ++c) ub[3 * b + c] += g[(long)c * N + n] * w;
        }
  }
}

/* Eq. 48 (with Eq. 13): each point adds F_b delta(x-X)delta(y-Y)[delta(z-Z)] dV to the
 * nodes of its support box; contributions of all points superpose. */
void or_spread(const or_params* P, int64_t npts, const double* X, const double* F, double dV,
               double* g) {
  long N = (long)P->nx * P->ny * P->nz;
  int64_t b;
  for (b = 0; b < npts; ++b) {
    int ix[4], iy[4], iz[4], cx, cy, cz, i, j, k, c;
    double wx[4], wy[4], wz[4];
    cx = axis_support(P->delta_kind, X[3 * b + 0], P->nx, P->periodic[0], ix, wx);
    cy = axis_support(P->delta_kind, X[3 * b + 1], P->ny, P->periodic[1], iy, wy);
    if (P->dim == 3) {
      cz = axis_support(P->delta_kind, X[3 * b + 2], P->nz, P->periodic[2], iz, wz);
    } else {
      cz = 1;
      iz[0] = 0;
      wz[0] = 1.0;
    }
    for (k = 0; k < cz; ++k)
      for (j = 0; j < cy; ++j)
        for (i = 0; i < cx; ++i) {
          long n = node_index(P->nx, P->ny, ix[i], iy[j], iz[k]);
          double w = wx[i] * wy[j] * wz[k];
          for (c = 0; c < P->dim; ++c) g[(long)c * N + n] += F[3 * b + c] * w * dV;
        }
  }
}

/* R6: volume of the solid shell owned by one Lagrangian point. */
double or_point_volume(const or_params* P) {
  if (P->n_lag <= 0) return 0.0;
  if (P->dim == 2) return (PI * P->diameter / P->n_lag) * P->drs;
  return (PI * P->diameter * P->diameter / P->n_lag) * P->drs;
}

/* ---------------------------------------------------------------- pairs */

static double axis_length(const or_params* P, int k) {
  return (double)(k == 0 ? P->nx : (k == 1 ? P->ny : P->nz));
}

/* separation X_i - X_j; on a periodic axis the nearest image is used */
static void separation(const or_params* P, const double* Xi, const double* Xj, double* dx) {
  int k;
  for (k = 0; k < 3; ++k) {
    double d = 0.0;
    if (k < P->dim) {
      double L = axis_length(P, k);
      d = Xi[k] - Xj[k];
      if (P->periodic[k]) {
        if (d > 0.5 * L)
          d -= L;
        else if (d < -0.5 * L)
          d += L;
      }
    }
    dx[k] = d;
  }
}

/* R11: squared distance summed in axis order (compiled without contraction). */
static double dist2(const double* dx) { return (dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2]; }

/* Table 4: every particle i scans the particles j > i. */
int64_t or_pairs_bruteforce(const or_params* P, int64_t n, const double* X, int32_t* pairs,
                            int64_t cap) {
  double thr = P->diameter + P->zeta, thr2 = thr * thr;
  int64_t i, j, cnt = 0;
  for (i = 0; i < n; ++i)
    for (j = i + 1; j < n; ++j) {
      double dx[3];
      separation(P, &X[3 * i], &X[3 * j], dx);
      if (dist2(dx) < thr2) {
        if (cnt < cap) {
          pairs[2 * cnt] = (int32_t)i;
          pairs[2 * cnt + 1] = (int32_t)j;
        }
        ++cnt;
      }
    }
  return cnt;
}

static int cmp_pair(const void* a, const void* b) {
  const int32_t* p = (const int32_t*)a;
  const int32_t* q = (const int32_t*)b;
  if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
  if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
  return 0;
}

/* Table 5 grid search on wall-bounded domains: square cells with
 * 0.5 (D + zeta) < H and H sqrt(dim) < D (Eq. 49-50), each cell holding at most one
 * particle centre (Eq. 51); each particle scans the 5^dim cells around its own and is
 * removed from the grid after its scan, so every pair is visited once.  Requires
 * non-overlapping particles (returns -1 when two centres share a cell) and
 * non-periodic axes (returns -2).  The list is returned sorted by (i, j). */
int64_t or_pairs_gridsearch(const or_params* P, int64_t n, const double* X, int32_t* pairs,
                            int64_t cap) {
  double thr = P->diameter + P->zeta, thr2 = thr * thr;
  double Hmin = 0.5 * thr, Hmax = P->diameter / sqrt((double)P->dim), H;
  int nc[3] = {1, 1, 1}, k;
  long ncell, c;
  int32_t* value;
  int64_t i, cnt = 0;
  for (k = 0; k < P->dim; ++k)
    if (P->periodic[k]) return -2;
  if (!(Hmin < Hmax)) return -3;
  H = 0.5 * (Hmin + Hmax);
  for (k = 0; k < P->dim; ++k) nc[k] = (int)floor(axis_length(P, k) / H) + 1;
  ncell = (long)nc[0] * nc[1] * nc[2];
  value = (int32_t*)malloc(sizeof(int32_t) * ncell);
  for (c = 0; c < ncell; ++c) value[c] = -1;
  for (i = 0; i < n; ++i) {
    int cc[3] = {0, 0, 0};
    long id;
    for (k = 0; k < P->dim; ++k) cc[k] = (int)floor((X[3 * i + k] + 0.5) / H);
    id = cc[0] + (long)nc[0] * (cc[1] + (long)nc[1] * cc[2]);
    if (value[id] != -1) {
      free(value);
      return -1;
    }
    value[id] = (int32_t)i;
  }
  for (i = 0; i < n; ++i) {
    int cc[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, gx, gy, gz;
    for (k = 0; k < P->dim; ++k) {
      cc[k] = (int)floor((X[3 * i + k] + 0.5) / H);
      lo[k] = cc[k] - 2 < 0 ? 0 : cc[k] - 2;
      hi[k] = cc[k] + 2 > nc[k] - 1 ? nc[k] - 1 : cc[k] + 2;
    }
    for (gz = lo[2]; gz <= hi[2]; ++gz)
      for (gy = lo[1]; gy <= hi[1]; ++gy)
        for (gx = lo[0]; gx <= hi[0]; ++gx) {
          int32_t j = value[gx + (long)nc[0] * (gy + (long)nc[1] * gz)];
          double dx[3];
          if (j == -1 || j == (int32_t)i) continue;
          separation(P, &X[3 * i], &X[3 * (int64_t)j], dx);
          if (dist2(dx) < thr2) {
            if (cnt < cap) {
              pairs[2 * cnt] = (int32_t)(i < j ? i : j);
              pairs[2 * cnt + 1] = (int32_t)(i < j ? j : i);
            }
            ++cnt;
          }
        }
    value[cc[0] + (long)nc[0] * (cc[1] + (long)nc[1] * cc[2])] = -1;
  }
  free(value);
  if (cnt <= cap) qsort(pairs, (size_t)cnt, 2 * sizeof(int32_t), cmp_pair);
  return cnt;
}

/* Eq. 16: force on particle i from particle j (R10 for the third case). */
void or_pair_force(const or_params* P, double c_ij, const double* Xi, const double* Xj,
                   double* F) {
  double dx[3], d, D = P->diameter, z = P->zeta, mag = 0.0;
  int k;
  separation(P, Xi, Xj, dx);
  d = sqrt(dist2(dx));
  if (d < D + z) {
    double t = (d - D - z) / z;
    mag = c_ij / P->eps_pp * t * t;
    if (d < D) mag += c_ij / P->E_pp * ((D - d) / z);
  }
  for (k = 0; k < 3; ++k) F[k] = (d > 0.0 && mag != 0.0) ? mag * dx[k] / d : 0.0;
}

static double particle_volume(const or_params* P) {
  double D = P->diameter;
  return (P->dim == 2) ? PI * D * D / 4.0 : PI * D * D * D / 6.0;
}

static double contact_scale(const or_params* P) {
  double g2 = P->gravity[0] * P->gravity[0] + P->gravity[1] * P->gravity[1] +
              P->gravity[2] * P->gravity[2];
  return fabs((P->density_ratio - 1.0) * RHO0 * particle_volume(P)) * sqrt(g2);
}

/* Collision force on every particle: half search (Table 4) with Newton's third law,
 * plus one mirror image per wall (R10). */
void or_contact_forces(const or_params* P, int64_t n, const double* X, double* Fc) {
  double c = contact_scale(P);
  int64_t i, j;
  int k;
  memset(Fc, 0, sizeof(double) * 3 * (size_t)n);
  for (i = 0; i < n; ++i)
    for (j = i + 1; j < n; ++j) {
      double F[3];
      or_pair_force(P, c, &X[3 * i], &X[3 * j], F);
      for (k = 0; k < 3; ++k) {
        Fc[3 * i + k] += F[k];
        Fc[3 * j + k] -= F[k];
      }
    }
  for (i = 0; i < n; ++i)
    for (k = 0; k < P->dim; ++k) {
      double img[3], F[3];
      int s, m;
      if (P->periodic[k]) continue;
      for (s = 0; s < 2; ++s) {
        /* wall at -1/2 (s = 0) or n - 1/2 (s = 1), on the nodes 0 and n - 1 with the
         * extrapolation boundaries (R13): image mirrored through the wall */
        double lo = P->boundary ? 0.0 : -0.5;
        double wall = (s == 0) ? lo : axis_length(P, k) - 1.0 - lo;
        for (m = 0; m < 3; ++m) img[m] = X[3 * i + m];
        img[k] = 2.0 * wall - X[3 * i + k];
        or_pair_force(P, c, &X[3 * i], img, F);
        for (m = 0; m < 3; ++m) Fc[3 * i + m] += F[m];
      }
    }
}

/* ------------------------------------------------------------ simulation */

struct or_sim {
  or_params P;
  lattice L;
  long N;
  int np, nl;
  long npts;
  double *f, *fp;                 /* [q][N] */
  double *ustar, *um, *fib, *dfib;/* [3][N] */
  double *xc, *uc, *om;           /* [np][3] */
  double *fh, *th, *fc;           /* [np][3] */
  double *ref;                    /* [nl][3] */
  double *xb, *ub, *fb, *dfb, *ubs; /* [npts][3] */
  double *pint, *lint;            /* [np][3] interior fluid momentum / angular momentum */
  double *fhp, *thp;              /* [np][3] F_h, T_h of the previous step */
  double *acc, *alp;              /* [np][3] previous linear / angular acceleration */
  int have_prev;
  double dV;
  double res_rms, res_max;
};

static void* zalloc(size_t n) { return calloc(n ? n : 1, 1); }

/* R8: reference offsets of the Lagrangian points from the particle centre. */
static void build_reference(or_sim* S) {
  int k;
  double R = 0.5 * S->P.diameter;
  for (k = 0; k < S->nl; ++k) {
    double* r = &S->ref[3 * k];
    if (S->P.dim == 2) {
      double th = 2.0 * PI * k / S->nl;
      r[0] = R * cos(th);
      r[1] = R * sin(th);
      r[2] = 0.0;
    } else {
      double zk = 1.0 - (2.0 * k + 1.0) / S->nl;
      double rho = sqrt(1.0 - zk * zk);
      double ph = k * PI * (3.0 - sqrt(5.0));
      r[0] = R * rho * cos(ph);
      r[1] = R * rho * sin(ph);
      r[2] = R * zk;
    }
  }
}

or_sim* or_create(const or_params* P, const double* xc) {
  or_sim* S = (or_sim*)zalloc(sizeof(or_sim));
  long N;
  int q;
  S->P = *P;
  if (P->dim == 2) S->P.nz = 1;
  lattice_init(S->P.dim, &S->L);
  N = (long)S->P.nx * S->P.ny * S->P.nz;
  q = S->L.q;
  S->N = N;
  S->np = P->n_particles;
  S->nl = P->n_lag;
  S->npts = (long)S->np * S->nl;
  S->f = (double*)zalloc(sizeof(double) * q * N);
  S->fp = (double*)zalloc(sizeof(double) * q * N);
  S->ustar = (double*)zalloc(sizeof(double) * 3 * N);
  S->um = (double*)zalloc(sizeof(double) * 3 * N);
  S->fib = (double*)zalloc(sizeof(double) * 3 * N);
  S->dfib = (double*)zalloc(sizeof(double) * 3 * N);
  S->xc = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->uc = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->om = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->fh = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->th = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->fc = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->ref = (double*)zalloc(sizeof(double) * 3 * S->nl);
  S->xb = (double*)zalloc(sizeof(double) * 3 * S->npts);
  S->ub = (double*)zalloc(sizeof(double) * 3 * S->npts);
  S->fb = (double*)zalloc(sizeof(double) * 3 * S->npts);
  S->dfb = (double*)zalloc(sizeof(double) * 3 * S->npts);
  S->ubs = (double*)zalloc(sizeof(double) * 3 * S->npts);
  S->pint = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->lint = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->fhp = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->thp = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->acc = (double*)zalloc(sizeof(double) * 3 * S->np);
  S->alp = (double*)zalloc(sizeof(double) * 3 * S->np);
  if (xc) memcpy(S->xc, xc, sizeof(double) * 3 * S->np);
  S->dV = or_point_volume(&S->P);
  build_reference(S);
  return S;
}

void or_destroy(or_sim* S) {
  if (!S) return;
  free(S->f); free(S->fp); free(S->ustar); free(S->um); free(S->fib); free(S->dfib);
  free(S->xc); free(S->uc); free(S->om); free(S->fh); free(S->th); free(S->fc);
  free(S->ref); free(S->xb); free(S->ub); free(S->fb); free(S->dfb); free(S->ubs);
  free(S->pint); free(S->lint); free(S->fhp); free(S->thp); free(S->acc); free(S->alp);
  free(S);
}

/* Lagrangian positions and rigid-body velocities: X_b = X_c + r_b, U_b = U_c + Omega x r_b
 * (2D: Omega is the z component). */
static void lagrangian_points(or_sim* S) {
  int i, k;
  for (i = 0; i < S->np; ++i)
    for (k = 0; k < S->nl; ++k) {
      long b = (long)i * S->nl + k;
      const double* r = &S->ref[3 * k];
      const double* O = &S->om[3 * i];
      double w[3];
      int c;
      if (S->P.dim == 2) {
        w[0] = -O[2] * r[1];
        w[1] = O[2] * r[0];
        w[2] = 0.0;
      } else {
        w[0] = O[1] * r[2] - O[2] * r[1];
        w[1] = O[2] * r[0] - O[0] * r[2];
        w[2] = O[0] * r[1] - O[1] * r[0];
      }
      for (c = 0; c < 3; ++c) {
        S->xb[3 * b + c] = S->xc[3 * i + c] + r[c];
        S->ub[3 * b + c] = S->uc[3 * i + c] + w[c];
      }
    }
}

/* Eq. 5 at every node: u* = sum_a e_a f_a. */
static void compute_ustar(or_sim* S) {
  long n;
  int a, k;
#pragma omp parallel for private(a, k)
  for (n = 0; n < S->N; ++n) {
    double u[3] = {0.0, 0.0, 0.0};
    for (a = 0; a < S->L.q; ++a)
      for (k = 0; k < 3; ++k) u[k] += S->L.e[a][k] * S->f[(long)a * S->N + n];
    for (k = 0; k < 3; ++k) S->ustar[(long)k * S->N + n] = u[k];
  }
}

/* Multi-direct forcing (R7) built from Eq. 9-11 and Eq. 47-48. */
static void ibm_mdf(or_sim* S) {
  long n, b;
  int m, c;
  size_t vbytes = sizeof(double) * 3 * (size_t)S->N;
  memcpy(S->um, S->ustar, vbytes);
  memset(S->fib, 0, vbytes);
  memset(S->fb, 0, sizeof(double) * 3 * (size_t)S->npts);
  S->res_rms = S->res_max = 0.0;
  if (S->npts == 0) return;
  for (m = 1; m <= S->P.mdf_iters; ++m) {
    or_interp(&S->P, S->um, S->npts, S->xb, S->dfb); /* dfb <- D_I u^(m-1) */
    for (b = 0; b < S->npts; ++b)
      for (c = 0; c < 3; ++c) {
        double ubm = S->dfb[3 * b + c];
        if (m == 1) S->ubs[3 * b + c] = ubm;
        S->dfb[3 * b + c] = (c < S->P.dim) ? 2.0 * RHO0 * (S->ub[3 * b + c] - ubm) : 0.0;
        S->fb[3 * b + c] += S->dfb[3 * b + c];
      }
    memset(S->dfib, 0, vbytes);
    or_spread(&S->P, S->npts, S->xb, S->dfb, S->dV, S->dfib);
#pragma omp parallel for
    for (n = 0; n < 3 * S->N; ++n) {
      S->fib[n] += S->dfib[n];
      S->um[n] += S->dfib[n] / (2.0 * RHO0);
    }
  }
  /* boundary-velocity residual after the last iteration: U_b - D_I u^(M) */
  or_interp(&S->P, S->um, S->npts, S->xb, S->dfb);
  {
    double s = 0.0, mx = 0.0;
    for (b = 0; b < S->npts; ++b)
      for (c = 0; c < S->P.dim; ++c) {
        double r = S->ub[3 * b + c] - S->dfb[3 * b + c];
        s += r * r;
        if (fabs(r) > mx) mx = fabs(r);
      }
    S->res_rms = sqrt(s / (double)(S->npts * S->P.dim));
    S->res_max = mx;
  }
}

/* Eq. 17 at every node, with the IB force plus the uniform body force. */
static void collide(or_sim* S) {
  long n;
  int a, k;
#pragma omp parallel for private(a, k)
  for (n = 0; n < S->N; ++n) {
    double fn[19], feq[19], Fa[19], F[3], us[3], u[3], p;
    for (a = 0; a < S->L.q; ++a) fn[a] = S->f[(long)a * S->N + n];
    for (k = 0; k < 3; ++k) F[k] = S->fib[(long)k * S->N + n] + S->P.body_force[k];
    macro_node(&S->L, fn, F, us, u, &p);
    feq_node(&S->L, p, u, feq);
    force_node(&S->L, S->P.tau, u, F, Fa);
    for (a = 0; a < S->L.q; ++a)
      S->fp[(long)a * S->N + n] = fn[a] - (fn[a] - feq[a]) / S->P.tau + Fa[a];
  }
}

/* centres leaving through a periodic face re-enter on the other side */
static void wrap_periodic(or_sim* S, int i) {
  int c;
  for (c = 0; c < S->P.dim; ++c) {
    double L = axis_length(&S->P, c);
    if (!S->P.periodic[c]) continue;
    if (S->xc[3 * i + c] >= L - 0.5)
      S->xc[3 * i + c] -= L;
    else if (S->xc[3 * i + c] < -0.5)
      S->xc[3 * i + c] += L;
  }
}

/* R9: momentum and angular momentum (about X_c) of the fluid at the nodes strictly
 * inside particle i, |x - X_c|^2 < R^2, with the corrected velocity u^(M). */
static void interior_momentum(const or_sim* S, int i, double* P, double* Lm) {
  const or_params* Q = &S->P;
  const double* X = &S->xc[3 * i];
  double R = 0.5 * Q->diameter;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, n[3] = {Q->nx, Q->ny, Q->nz}, k, gx, gy, gz;
  for (k = 0; k < 3; ++k) P[k] = Lm[k] = 0.0;
  for (k = 0; k < Q->dim; ++k) {
    lo[k] = (int)floor(X[k] - R);
    hi[k] = (int)ceil(X[k] + R);
  }
  for (gz = lo[2]; gz <= hi[2]; ++gz)
    for (gy = lo[1]; gy <= hi[1]; ++gy)
      for (gx = lo[0]; gx <= hi[0]; ++gx) {
        int g[3] = {gx, gy, gz}, w[3];
        double r[3];
        long nn;
        int c, inside = 1;
        for (k = 0; k < 3; ++k) {
          r[k] = (k < Q->dim) ? (double)g[k] - X[k] : 0.0;
          w[k] = g[k];
          if (k >= Q->dim) continue;
          if (g[k] < 0 || g[k] >= n[k]) {
            if (!Q->periodic[k]) inside = 0;
            w[k] = ((g[k] % n[k]) + n[k]) % n[k];
          }
        }
        if (!inside || !(dist2(r) < R * R)) continue;
        nn = node_index(Q->nx, Q->ny, w[0], w[1], w[2]);
        {
          double u[3];
          for (c = 0; c < 3; ++c) u[c] = S->um[(long)c * S->N + nn];
          for (c = 0; c < 3; ++c) P[c] += RHO0 * u[c];
          Lm[0] += RHO0 * (r[1] * u[2] - r[2] * u[1]);
          Lm[1] += RHO0 * (r[2] * u[0] - r[0] * u[2]);
          Lm[2] += RHO0 * (r[0] * u[1] - r[1] * u[0]);
        }
      }
}

/* R9: F_h = -sum_b F_b dV, T_h = -sum_b r_b x F_b dV, then Eq. 14-15. */
static void move_particles(or_sim* S) {
  const or_params* P = &S->P;
  double V = particle_volume(P), Mp = P->density_ratio * RHO0 * V;
  double meff = Mp - RHO0 * V, R = 0.5 * P->diameter;
  double Ip = (P->dim == 2) ? Mp * P->diameter * P->diameter / 8.0
                            : Mp * P->diameter * P->diameter / 10.0;
  double Kt = RHO0 * S->nl * S->dV;
  double Kr = Kt * R * R * (P->dim == 2 ? 1.0 : 2.0 / 3.0);
  int i, k, c;
  or_contact_forces(P, S->np, S->xc, S->fc);
#pragma omp parallel for private(k, c)
  for (i = 0; i < S->np; ++i) {
    double Fh[3] = {0, 0, 0}, Th[3] = {0, 0, 0}, Pn[3], Ln[3];
    for (k = 0; k < S->nl; ++k) {
      long b = (long)i * S->nl + k;
      const double* r = &S->ref[3 * k];
      const double* F = &S->fb[3 * b];
      for (c = 0; c < 3; ++c) Fh[c] -= F[c] * S->dV;
      Th[0] -= (r[1] * F[2] - r[2] * F[1]) * S->dV;
      Th[1] -= (r[2] * F[0] - r[0] * F[2]) * S->dV;
      Th[2] -= (r[0] * F[1] - r[1] * F[0]) * S->dV;
    }
    if (P->dim == 2) {
      Fh[2] = 0.0;
      Th[0] = Th[1] = 0.0;
    }
    interior_momentum(S, i, Pn, Ln);
    for (c = 0; c < 3; ++c) {
      double dP = S->have_prev ? Pn[c] - S->pint[3 * i + c] : 0.0;
      double dL = S->have_prev ? Ln[c] - S->lint[3 * i + c] : 0.0;
      double Fm = 0.5 * (Fh[c] + S->fhp[3 * i + c]);
      double Tm = 0.5 * (Th[c] + S->thp[3 * i + c]);
      S->fh[3 * i + c] = Fh[c];
      S->th[3 * i + c] = Th[c];
      S->fhp[3 * i + c] = Fh[c];
      S->thp[3 * i + c] = Th[c];
      S->pint[3 * i + c] = Pn[c];
      S->lint[3 * i + c] = Ln[c];
      if (P->fixed_particles == 1) continue;
      if (c < P->dim && P->fixed_particles == 0) {
        double F = Fm + S->fc[3 * i + c] + dP + meff * P->gravity[c];
        double a = (F + Kt * S->acc[3 * i + c]) / (Mp + Kt);
        double u0 = S->uc[3 * i + c], u1 = u0 + a;
        S->acc[3 * i + c] = a;
        S->uc[3 * i + c] = u1;
        S->xc[3 * i + c] += 0.5 * (u0 + u1);
      }
      if (P->dim == 3 || c == 2) {
        double al = (Tm + dL + Kr * S->alp[3 * i + c]) / (Ip + Kr);
        S->alp[3 * i + c] = al;
        S->om[3 * i + c] += al;
      }
    }
    if (!P->fixed_particles) wrap_periodic(S, i);
  }
  S->have_prev = 1;
}

/* R13: non-equilibrium extrapolation on the boundary nodes, after streaming. */
static void extrapolation_boundaries(or_sim* S) {
  const or_params* P = &S->P;
  const int n[3] = {P->nx, P->ny, P->nz};
  int x, y, z, k, a;
#pragma omp parallel for collapse(2) private(x, k, a)
  for (z = 0; z < n[2]; ++z)
    for (y = 0; y < n[1]; ++y)
      for (x = 0; x < n[0]; ++x) {
        int c[3], cf[3], on = 0, wall = 0, inlet = 0;
        double fn[19], eqf[19], eqb[19], us[3], uf[3], ub[3] = {0.0, 0.0, 0.0}, pf, pb;
        long nb, nf;
        c[0] = x; c[1] = y; c[2] = z;
        for (k = 0; k < 3; ++k) {
          int lo, hi;
          cf[k] = c[k];
          if (k >= P->dim || P->periodic[k]) continue;
          lo = c[k] == 0;
          hi = c[k] == n[k] - 1;
          if (!lo && !hi) continue;
          on = 1;
          cf[k] = lo ? c[k] + 1 : c[k] - 1;
          if (P->boundary == 2 && k == 1) {
            if (lo) inlet = 1;
          } else {
            wall = 1;
          }
        }
        if (!on) continue;
        nb = node_index(n[0], n[1], c[0], c[1], c[2]);
        nf = node_index(n[0], n[1], cf[0], cf[1], cf[2]);
        for (a = 0; a < S->L.q; ++a) fn[a] = S->f[(long)a * S->N + nf];
        macro_node(&S->L, fn, P->body_force, us, uf, &pf);
        feq_node(&S->L, pf, uf, eqf);
        if (wall) {
          pb = pf;
        } else if (inlet) {
          double prof = P->u_inlet;
          for (k = 0; k < P->dim; ++k) {
            double L;
            if (k == 1 || P->periodic[k]) continue;
            L = n[k] - 1.0;
            prof *= 4.0 * c[k] * (L - c[k]) / (L * L);
          }
          ub[1] = prof;
          pb = pf;
        } else { /* outlet */
          for (k = 0; k < 3; ++k) ub[k] = uf[k];
          pb = 0.0;
        }
        feq_node(&S->L, pb, ub, eqb);
        for (a = 0; a < S->L.q; ++a) S->f[(long)a * S->N + nb] = eqb[a] + fn[a] - eqf[a];
      }
}

/* One time step in the order of R12 (the step list after Eq. 18 and Sec. 6 part list). */
void or_step(or_sim* S, int32_t nsteps) {
  int32_t s;
  for (s = 0; s < nsteps; ++s) {
    compute_ustar(S);
    lagrangian_points(S);
    ibm_mdf(S);
    collide(S);
    or_stream_push(S->P.dim, S->P.nx, S->P.ny, S->P.nz, S->P.periodic, S->fp, S->f);
    if (S->P.boundary) extrapolation_boundaries(S);
    move_particles(S);
  }
}

void or_get_pdfs(const or_sim* S, double* f) {
  memcpy(f, S->f, sizeof(double) * S->L.q * (size_t)S->N);
}

void or_set_pdfs(or_sim* S, const double* f) {
  memcpy(S->f, f, sizeof(double) * S->L.q * (size_t)S->N);
}

/* f = f_eq(p, u) at every node (Eq. 4); u is [3][N]. */
void or_set_fields(or_sim* S, const double* p, const double* u) {
  long n;
  int a, k;
  for (n = 0; n < S->N; ++n) {
    double un[3], feq[19];
    for (k = 0; k < 3; ++k) un[k] = u[(long)k * S->N + n];
    feq_node(&S->L, p[n], un, feq);
    for (a = 0; a < S->L.q; ++a) S->f[(long)a * S->N + n] = feq[a];
  }
}

/* p and u of the current PDFs without any force (Eq. 5, Eq. 6 with u = u*). */
void or_get_fields(const or_sim* S, double* p, double* u) {
  long n;
  int a, k;
  for (n = 0; n < S->N; ++n) {
    double fn[19], F[3] = {0, 0, 0}, us[3], uu[3], pp;
    for (a = 0; a < S->L.q; ++a) fn[a] = S->f[(long)a * S->N + n];
    macro_node(&S->L, fn, F, us, uu, &pp);
    if (p) p[n] = pp;
    if (u)
      for (k = 0; k < 3; ++k) u[(long)k * S->N + n] = uu[k];
  }
}

void or_get_particles(const or_sim* S, double* X, double* U, double* Om, double* Fh,
                      double* Th, double* Fc) {
  size_t b = sizeof(double) * 3 * (size_t)S->np;
  if (X) memcpy(X, S->xc, b);
  if (U) memcpy(U, S->uc, b);
  if (Om) memcpy(Om, S->om, b);
  if (Fh) memcpy(Fh, S->fh, b);
  if (Th) memcpy(Th, S->th, b);
  if (Fc) memcpy(Fc, S->fc, b);
}

void or_set_particles(or_sim* S, const double* X, const double* U, const double* Om) {
  size_t b = sizeof(double) * 3 * (size_t)S->np;
  if (X) memcpy(S->xc, X, b);
  if (U) memcpy(S->uc, U, b);
  if (Om) memcpy(S->om, Om, b);
}

/* Lagrangian data of the last step: X_b, U_b, F_b = sum of MDF increments, u_b* = D_I u*. */
void or_get_lagrangian(const or_sim* S, double* Xb, double* Ub, double* Fb, double* ubstar) {
  size_t b = sizeof(double) * 3 * (size_t)S->npts;
  if (Xb) memcpy(Xb, S->xb, b);
  if (Ub) memcpy(Ub, S->ub, b);
  if (Fb) memcpy(Fb, S->fb, b);
  if (ubstar) memcpy(ubstar, S->ubs, b);
}

void or_get_mdf_residual(const or_sim* S, double* rms, double* maxabs) {
  if (rms) *rms = S->res_rms;
  if (maxabs) *maxabs = S->res_max;
}

/* interior fluid momentum and angular momentum of the last step, [np][3] */
void or_get_interior_momentum(const or_sim* S, double* P, double* L) {
  size_t b = sizeof(double) * 3 * (size_t)S->np;
  if (P) memcpy(P, S->pint, b);
  if (L) memcpy(L, S->lint, b);
}
