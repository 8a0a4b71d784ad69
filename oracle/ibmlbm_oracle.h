/*
 * FP64 CPU oracle for the IB-LBM hot path of "Efficient implementation of
 * immersed boundary-lattice Boltzmann method for massive particle-laden flows,
 * Part I" (Jiang, Li & Liu).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path: only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library; the two
 * meet only through seeded inputs produced by the input-generator module.
 *
 * Everything is plain double precision, general-alpha loops, two PDF arrays and
 * point-to-node IBM, written in the paper's order and notation:
 *   - Sec. 2.1, Eq. 1-8   incompressible SRT-LBGK with Guo split forcing
 *   - Sec. 3, Eq. 17-18   two-array push collide/stream
 *   - Sec. 3.3, Eq. 41-42 swap streaming (kept as an independent cross-check)
 *   - Sec. 2.2, Eq. 9-13  IBM interpolation / spreading, Sec. 4 Eq. 47-48
 *   - Sec. 5, Table 4     half-search pair list; Table 5 grid search (cross-check)
 *   - Sec. 2.3, Eq. 14-16 Newton-Euler particle motion and pair force
 * Readings where the paper is silent or garbled are listed at each function.
 *
 * Built with -fopenmp (liboracle_omp.so) the loops over nodes, points and particles
 * whose iterations write disjoint data run on all host cores; nothing is summed
 * across iterations, so both builds give identical bits.
 *
 * Units: dh = dt = c = 1, cs^2 = 1/3, rho_0 = rho_f = 1 (lattice units).
 * Node (x, y, z) has integer coordinates 0..n-1 on each axis; node index
 * n = x + nx*(y + ny*z).  PDF arrays are [q][N]; vector fields are [3][N]
 * (z component zero in 2D); per-particle and per-point vectors are [.][3].
 */
#ifndef IBMLBM_ORACLE_H
#define IBMLBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_params {
  int32_t dim;              /* 2 (D2Q9) or 3 (D3Q19)                             */
  int32_t nx, ny, nz;       /* fluid nodes per axis; nz = 1 for dim = 2          */
  int32_t periodic[3];      /* 1 periodic axis; 0 halfway bounce-back walls      */
  double tau;               /* relaxation time of Eq. 1                         */
  double body_force[3];     /* uniform fluid body force, added to the IB force   */
  int32_t n_particles;      /* N_p                                               */
  int32_t n_lag;            /* N_L, Lagrangian points per particle               */
  double diameter;          /* D_p                                               */
  int32_t delta_kind;       /* 4 or 3: regularised delta function (Fig. 2b)      */
  double drs;               /* solid-shell thickness of Eq. 13                   */
  int32_t mdf_iters;        /* M, multi-direct-forcing iterations                */
  double density_ratio;     /* rho_p / rho_f                                     */
  double gravity[3];        /* g acting on particles                             */
  double zeta, eps_pp, E_pp;/* Eq. 16 range and stiffness parameters             */
  int32_t fixed_particles;  /* 1: particles keep their state (static bodies);
                               2: centres and velocities held, rotation integrated */
  int32_t boundary;         /* 0: halfway bounce-back walls at -1/2, n - 1/2;
                               1: non-equilibrium extrapolation walls on the outermost
                                  nodes of every non-periodic axis;
                               2: as 1, with a velocity inlet on y = 0 and a pressure
                                  outlet on y = ny - 1 (a channel along y)           */
  double u_inlet;           /* peak inlet velocity (boundary 2)                   */
} or_params;

typedef struct or_sim or_sim;

/* lattice tables: q, e[q][3], w[q] (Eq. 2-3, weights after Eq. 4) */
int or_lattice(int32_t dim, int32_t* q, int32_t* e, double* w);

/* single-node operators (general alpha loops) */
void or_feq(int32_t dim, double p, const double* u, double* feq);                       /* Eq. 4 */
void or_force_term(int32_t dim, double tau, const double* u, const double* F, double* Fa);/* Eq. 8 */
void or_macro(int32_t dim, const double* fnode, const double* F,
              double* ustar, double* u, double* p);                                     /* Eq. 5-7 */
double or_delta(int32_t kind, double r);                                               /* Fig. 2b */

/* streaming of a post-collision field fp into f (Eq. 18 with walls) and the swap form */
void or_stream_push(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const int32_t* periodic,
                    const double* fp, double* f);
void or_stream_swap(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const int32_t* periodic,
                    double* f);

/* IBM operators on a field g[3][N] for points X[np][3] (Eq. 47, Eq. 48) */
void or_interp(const or_params* P, const double* g, int64_t npts, const double* X, double* ub);
void or_spread(const or_params* P, int64_t npts, const double* X, const double* F, double dV,
               double* g);

/* pair search: brute-force half search (Table 4) and grid search (Table 5) */
int64_t or_pairs_bruteforce(const or_params* P, int64_t n, const double* X,
                            int32_t* pairs, int64_t cap);
int64_t or_pairs_gridsearch(const or_params* P, int64_t n, const double* X,
                            int32_t* pairs, int64_t cap);
void or_pair_force(const or_params* P, double c_ij, const double* Xi, const double* Xj, double* F);
void or_contact_forces(const or_params* P, int64_t n, const double* X, double* Fc);

/* whole simulation */
or_sim* or_create(const or_params* P, const double* xc);
void or_destroy(or_sim* S);
void or_step(or_sim* S, int32_t nsteps);
void or_get_pdfs(const or_sim* S, double* f);
void or_set_pdfs(or_sim* S, const double* f);
void or_set_fields(or_sim* S, const double* p, const double* u);
void or_get_fields(const or_sim* S, double* p, double* u);
void or_get_particles(const or_sim* S, double* X, double* U, double* Om,
                      double* Fh, double* Th, double* Fc);
void or_set_particles(or_sim* S, const double* X, const double* U, const double* Om);
void or_get_lagrangian(const or_sim* S, double* Xb, double* Ub, double* Fb, double* ubstar);
void or_get_mdf_residual(const or_sim* S, double* rms, double* maxabs);
void or_get_interior_momentum(const or_sim* S, double* P, double* L);
double or_point_volume(const or_params* P);

#ifdef __cplusplus
}
#endif
#endif
