/*
 * ibmlbm.h - C ABI of the GB300 IB-LBM hot path (libibmlbm.so).
 *
 * One time step of the immersed boundary - lattice Boltzmann method for
 * particle-laden flow of Jiang, Li & Liu ("Efficient implementation of immersed
 * boundary-lattice Boltzmann method for massive particle-laden flows, Part I"):
 *   1. macroscopic velocity u* = sum_a e_a f_a on the nodes near particles (Eq. 5)
 *   2. multi-direct forcing: interpolation u_b = D_I u (Eq. 9, 12, 47), boundary
 *      force dF_b = 2 rho_f (U_b - u_b)/dt (Eq. 10), spreading f = D_E dF_b
 *      (Eq. 11, 13, 48), repeated M times
 *   3. fused SRT-LBGK collision with Guo split forcing and in-place streaming with
 *      halfway bounce-back at walls (Eq. 1, 4, 6-8, 17-18)
 *   4. cell-list pair search and the short-range repulsive force (Eq. 16, Sec. 5)
 *   5. Newton-Euler update of the particles (Eq. 14-15) in double precision.
 * Lattices: D2Q9 (Eq. 2) and D3Q19 (Eq. 3, with e_9 = (-1, 0, 1), the entry the
 * printed matrix drops).  Units are lattice units: dh = dt = 1, cs^2 = 1/3,
 * rho_0 = rho_f = 1.
 *
 * Conventions for every call
 *   - Every call returns an int status: IBMLBM_OK (0) or a negative IBMLBM_ERR_*.
 *     No call aborts, traps or exits; ibm_lbm_last_error() describes the last
 *     failure of the calling thread.
 *   - Node (x, y, z), 0 <= x < nx etc., has index n = x + nx*(y + ny*z); N = nx*ny*nz
 *     (nz = 1 in 2D).  Node x sits at coordinate x; walls of a non-periodic axis
 *     lie halfway, at -1/2 and n-1/2.
 *   - PDFs are [q][N] float; vector fields [dim][N]; per-particle vectors are
 *     [n_particles][dim]; angular quantities [n_particles][1] in 2D (the z
 *     component) and [n_particles][3] in 3D; per-point vectors [n_particles*n_lag][dim]
 *     with the points of particle i at rows i*n_lag .. i*n_lag + n_lag - 1.
 *   - Host pointers are plain CPU memory; "device" pointers are CUDA global memory
 *     on the current device.  The library never frees memory it did not allocate.
 *   - A stream argument is a cudaStream_t passed as void*; 0 is the legacy stream.
 */
#ifndef IBMLBM_H
#define IBMLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IBMLBM_OK 0
#define IBMLBM_ERR_INVALID_ARG (-1)   /* bad pointer, size or configuration value */
#define IBMLBM_ERR_UNSUPPORTED (-2)   /* valid request outside what the library supports */
#define IBMLBM_ERR_WORKSPACE (-3)     /* workspace missing, misaligned or too small */
#define IBMLBM_ERR_CUDA (-4)          /* a CUDA runtime call failed */
#define IBMLBM_ERR_NONFINITE (-5)     /* NaN/Inf in a particle state (device check) */
#define IBMLBM_ERR_OUT_OF_DOMAIN (-6) /* a particle centre left the fluid domain */
#define IBMLBM_ERR_CAPACITY (-7)      /* a fixed-capacity list overflowed */
#define IBMLBM_ERR_BOUNDS (-8)        /* bounds-checked build (libibmlbm_checked.so) only: a
                                         kernel's index check failed; the access was skipped */
#define IBMLBM_ERR_TIMEOUT (-9)       /* a grid barrier of a persistent batch kernel gave up
                                         waiting; its kernel returned early */

/* Problem statement of one run (Sec. 2, Sec. 6.2 and Table 7 of the paper). */
typedef struct ibm_lbm_config {
  uint32_t struct_size;   /* must equal sizeof(ibm_lbm_config)                           */
  int32_t dim;            /* 2: D2Q9, 3: D3Q19                                           */
  int32_t nx, ny, nz;     /* fluid nodes per axis (nz = 1 when dim = 2)                  */
  int32_t periodic[3];    /* per axis: 1 periodic, 0 walls (see boundary)                */
  double tau;             /* relaxation time of Eq. 1, tau > 1/2                         */
  double body_force[3];   /* uniform fluid body force, added to the IB force (Eq. 7-8)  */
  int32_t n_particles;    /* N_p, rigid circles (2D) or spheres (3D), >= 0               */
  int32_t n_lag;          /* N_L Lagrangian points per particle (Sec. 2.2)               */
  double diameter;        /* D_p                                                         */
  int32_t delta_kind;     /* regularised delta function of Fig. 2b: 4 (Peskin's 4-point) or
                             3 (3-point of Roma, Peskin and Berger; drs = 1.9 in Sec. 2.2) */
  double drs;             /* solid-shell thickness of Eq. 13 (2.6 for the 4-point delta) */
  int32_t mdf_iters;      /* M >= 0 multi-direct-forcing iterations; 1 is BTDF (Eq. 9-11)*/
  double density_ratio;   /* rho_p / rho_f                                               */
  double gravity[3];      /* g acting on the particles (Eq. 14, weight less buoyancy)    */
  double zeta;            /* range of the repulsive force of Eq. 16                      */
  double eps_pp, E_pp;    /* stiffness parameters of Eq. 16 (E_pp < eps_pp)              */
  int32_t fixed_particles;/* 0: free; 1: particles keep centre, velocity and spin (static
                             bodies); 2: centre and velocity held, the spin integrated  */
  int32_t max_neighbors;  /* capacity of each particle's contact list; 0 selects 32      */
  int32_t pdf_storage;    /* IBMLBM_PDF_FP32 (0), IBMLBM_PDF_FP16 (1), IBMLBM_PDF_BF16 (2):
                             element type of the stored PDFs.  FP16 and BF16 hold
                             h_a = f_a / w_a (deviations from rest divided by the lattice
                             weight); collision, IBM and particle arithmetic stay FP32 /
                             FP64.  No counterpart in the paper, which stores doubles.    */
  int32_t mlp_init;       /* 1: the first MDF iteration takes its force from the learned
                             initializer (2D; parameters from ibm_lbm_set_mlp), the
                             plain iterations 2..M follow.  No counterpart in the paper.  */
  int32_t boundary;       /* fluid boundaries of the non-periodic axes:
                             0: halfway bounce-back walls at -1/2 and n - 1/2;
                             1: walls on the outermost nodes, by non-equilibrium
                                extrapolation (Sec. 6.1-6.2: after streaming a boundary
                                node takes the equilibrium of its prescribed state plus
                                the non-equilibrium part of its inward neighbour);
                             2: as 1, with the y axis a channel: a velocity inlet on
                                y = 0 (the parabola u_inlet prod 4 c (L - c) / L^2 over the
                                other non-periodic axes, L = n - 1) and a pressure outlet
                                (p = 0) on y = ny - 1 (the Poiseuille flows of Sec. 6.1).
                             1 and 2 need n >= 3 on every non-periodic axis; 2 needs a
                             non-periodic y axis.  Particle contacts with a wall mirror
                             through the wall's position.                                */
  double u_inlet;         /* peak inlet velocity of boundary 2                           */
  int32_t pair_search;    /* particle-pair search: 0 cell lists (cells of side >= D_p +
                             zeta, buckets of particle indices); 1 the grid search of
                             Sec. 5 (Table 5, Eq. 49-51: cells of side < D_p / sqrt(dim)
                             holding one particle index each, scanned within
                             ceil((D_p + zeta) / side) cells).  Both give the same
                             sorted pair lists and forces.  Batches use 0.              */
} ibm_lbm_config;

enum { IBMLBM_PDF_FP32 = 0, IBMLBM_PDF_FP16 = 1, IBMLBM_PDF_BF16 = 2 };

typedef struct ibm_lbm_handle ibm_lbm_handle;

/* Device bytes the run needs for the configuration.  The caller allocates them
 * (any CUDA allocator, 256-byte aligned) and passes them to ibm_lbm_init.
 * Errors: IBMLBM_ERR_INVALID_ARG for a configuration ibm_lbm_init would reject. */
int ibm_lbm_workspace_size(const ibm_lbm_config* cfg, size_t* bytes);

/* The 3D staging list of the configuration (host only, no device call): the cells of
 * a sphere's node box (side S = 2 ceil(D_p / 2) + 6, the box starting rcell + 2 nodes
 * before the centre's anchor node, rcell = ceil(D_p / 2)) that can be a support node
 * of some Lagrangian point for some position of the centre within its anchor cell
 * (Eq. 47-48 with the configuration's delta function), packed lx | ly << 5 | lz << 10.
 * The interpolation stages, and the spreading flushes, only these cells of spheres
 * whose box lies inside the domain.  cells: host [cap] (may be NULL with cap = 0 to
 * query the count); n: the number of entries, 0 where no list is used (2D, no
 * particles, box side above 32).  Errors: INVALID_ARG (configuration, NULL n),
 * CAPACITY (n > cap, with cells not NULL). */
int ibm_lbm_stage_list(const ibm_lbm_config* cfg, int32_t* cells, int64_t cap, int64_t* n);

/* Create a run.  d_workspace: device memory of at least ibm_lbm_workspace_size
 * bytes, borrowed (not owned) until ibm_lbm_destroy.  stream: every kernel and
 * copy of the run is ordered on it (within a step the particle update runs on a
 * second stream the run owns, forked from and joined back into this one, so work
 * enqueued on it after a step sees the whole step).  h_centres: host [n_particles][dim] particle
 * centres (may be NULL when n_particles = 0).  The fluid starts at rest with
 * p = 0 (every PDF zero, the deviation gauge of the incompressible model) and the
 * particles with U = Omega = 0.  Copies the centres to the device and waits for
 * the stream.  Errors: INVALID_ARG (configuration, pointers, a centre outside
 * the domain), WORKSPACE, UNSUPPORTED (delta_kind other than 3 or 4), CUDA. */
int ibm_lbm_init(const ibm_lbm_config* cfg, void* d_workspace, size_t bytes, void* stream,
                 const double* h_centres, ibm_lbm_handle** out);

/* Enqueue n_steps time steps on the run's stream and return without waiting.
 * Steps after the first replay a captured CUDA graph.  Device-side failures
 * (NONFINITE, OUT_OF_DOMAIN, CAPACITY) are recorded in a status word that
 * ibm_lbm_sync reports.  Errors: INVALID_ARG (n_steps < 0), CUDA. */
int ibm_lbm_step(ibm_lbm_handle* h, int32_t n_steps);

/* Wait for the stream and report the device status word (first failure wins),
 * then clear it. */
int ibm_lbm_sync(ibm_lbm_handle* h);

/* Replace the PDFs with d_f: device [q][N] floats in canonical layout
 * (d_f[a*N + n] = f_a at node n, pre-collision at the current time).  Ordered on
 * the run's stream; returns after enqueueing. */
int ibm_lbm_set_pdfs(ibm_lbm_handle* h, const float* d_f);

/* Copy the current PDFs into device [q][N] floats d_f, canonical layout. */
int ibm_lbm_get_pdfs(ibm_lbm_handle* h, float* d_f);

/* Set every node to the equilibrium of Eq. 4 for pressure d_p [N] and velocity
 * d_u [dim][N] (device doubles). */
int ibm_lbm_set_fields(ibm_lbm_handle* h, const double* d_p, const double* d_u);

/* Pressure (Eq. 6 with u = u*) and velocity u* (Eq. 5) of the current PDFs, without
 * a force correction, into device doubles d_p [N] and d_u [dim][N]; either may be NULL. */
int ibm_lbm_get_fields(ibm_lbm_handle* h, double* d_p, double* d_u);

/* Set particle centres X [n][dim], velocities U [n][dim] and angular velocities
 * Omega (2D [n][1], 3D [n][3]); NULL leaves a quantity unchanged.  Host doubles.
 * Regenerates the Lagrangian points; synchronous. */
int ibm_lbm_set_particles(ibm_lbm_handle* h, const double* X, const double* U,
                          const double* Omega);

/* Particle state after the last step (host doubles, any pointer may be NULL;
 * synchronous):
 * X, U, Omega as above; F_h = -sum_b F_b dV and T_h = -sum_b r_b x F_b dV of the
 * last step (Eq. 14-15); F_c the contact force of Eq. 16 (walls included). */
int ibm_lbm_get_particles(ibm_lbm_handle* h, double* X, double* U, double* Omega,
                          double* F_h, double* T_h, double* F_c);

/* Lagrangian data of the last step (host, any pointer may be NULL): X_b (double),
 * U_b, F_b = sum over MDF iterations of dF_b, and u_b* = D_I u* (floats). */
int ibm_lbm_get_lagrangian(ibm_lbm_handle* h, double* X_b, float* U_b, float* F_b,
                           float* u_b_star);

/* Momentum [n][dim] and angular momentum (2D [n][1], 3D [n][3]) of the fluid at the
 * nodes strictly inside each particle, from the last step (host doubles). */
int ibm_lbm_get_interior_momentum(ibm_lbm_handle* h, double* P, double* L);

/* Contact pairs of the last step: (i, j) with i < j and
 * |X_i - X_j|^2 < (D_p + zeta)^2 (squared distance summed in axis order in double
 * precision without fused multiply-add; nearest image on periodic axes), sorted by
 * (i, j), written as pairs[2k], pairs[2k+1] (host int32).  *n receives the count;
 * IBMLBM_ERR_CAPACITY if it exceeds cap (nothing is written then). */
int ibm_lbm_get_pairs(ibm_lbm_handle* h, int32_t* pairs, int64_t cap, int64_t* n);

/* Kernels this run has launched so far (eager launches plus graph kernel nodes). */
int ibm_lbm_get_launch_count(ibm_lbm_handle* h, int64_t* n);

/* Time n_steps steps part by part with CUDA events on the run's stream (eager
 * launches, no graph) and return the total milliseconds of each part in
 * ms[IBMLBM_PART_COUNT], in the order of enum ibm_lbm_part; the parts follow the
 * per-part timing of Sec. 6.2 (Fig. 10, Fig. 16). */
enum ibm_lbm_part {
  IBMLBM_PART_MACRO = 0,      /* lbm_moments on the flagged nodes                  */
  IBMLBM_PART_IBM = 1,        /* interpolation, spreading, F_h/T_h, interior sums  */
  IBMLBM_PART_COLLIDE = 2,    /* fused collision + streaming + bounce-back         */
  IBMLBM_PART_PAIRS = 3,      /* cell buckets, contact force, Newton-Euler update  */
  IBMLBM_PART_PARTICLES = 4,  /* regeneration of the points, node marks            */
  IBMLBM_PART_COUNT = 5
};
int ibm_lbm_time_parts(ibm_lbm_handle* h, int32_t n_steps, double* ms);

/* Release the handle's host state.  The workspace stays owned by the caller.
 * Never fails; NULL is ignored. */
void ibm_lbm_destroy(ibm_lbm_handle* h);

/* Text of the calling thread's last failure ("" if none).  Valid until the next
 * call on the same thread. */
const char* ibm_lbm_last_error(void);

/* ---------------------------------------------------------------------------
 * Standalone pair search (Sec. 5): device cell lists built by a counting sort on
 * the cell key, then a scan of the 3^dim neighbouring cells of each particle.
 *   dim, n_nodes[3], periodic[3]: the domain as in ibm_lbm_config
 *   diameter, zeta: pair rule |X_i - X_j|^2 < (diameter + zeta)^2
 *   d_X: device [n][dim] double centres (inside the domain)
 *   max_neighbors: per-particle list capacity (0 selects 32)
 *   d_scratch / scratch_bytes: device scratch of ibm_lbm_pair_search_scratch_size bytes
 *   d_pairs: device int32 [cap][2] output, sorted by (i, j)
 *   h_count: host; receives the number of pairs (also when it exceeds cap, in which
 *            case IBMLBM_ERR_CAPACITY is returned and only the first cap are valid)
 * Synchronises the stream before returning.  IBMLBM_ERR_CAPACITY also reports a
 * particle with more than max_neighbors partners. */
int ibm_lbm_pair_search_scratch_size(int32_t dim, const int32_t* n_nodes, double diameter,
                                     double zeta, int32_t n, int32_t max_neighbors,
                                     size_t* bytes);
int ibm_lbm_pair_search(int32_t dim, const int32_t* n_nodes, const int32_t* periodic,
                        double diameter, double zeta, int32_t n, const double* d_X,
                        int32_t max_neighbors, void* d_scratch, size_t scratch_bytes,
                        int32_t* d_pairs, int64_t cap, int64_t* h_count, void* stream);

/* ---------------------------------------------------------------------------
 * Pair search that allocates nothing (no counterpart in the paper; it is an
 * interface for callers, not part of the method).  Same arguments and results as
 * ibm_lbm_pair_search, but the cell and neighbour lists live in a fixed 16 MiB
 * device array inside this library instead of caller-provided scratch, and the call
 * makes no cudaMalloc, cudaFree or other allocating call.  It is meant for callers
 * that cannot provide or allocate device scratch: code without access to a CUDA
 * allocator (a plug-in handed only its input and output buffers), code that must not
 * pay the implicit synchronisation of cudaMalloc/cudaFree.  It reads the pair count
 * back and synchronises the stream, so the call itself cannot be captured.
 *   - A problem whose scratch (cells, per-particle lists) exceeds 16 MiB returns
 *     IBMLBM_ERR_CAPACITY and writes nothing; use ibm_lbm_pair_search for it.
 *   - Every GPU that loads the array keeps the 16 MiB until the process exits.
 *   - All calls on a device share the array and it keeps the last call's contents
 *     (counters and the status word are cleared on the stream at each call); calls
 *     that overlap on the GPU race on it.  Order them on one stream.
 *   - The first call on a device (with that device current) looks up the array's
 *     device address and caches it; make that first call before any stream capture.
 *     After cudaDeviceReset the cached address is stale: reload the library first.
 * Synchronises the stream before returning. */
int ibm_lbm_pair_search_static(int32_t dim, const int32_t* n_nodes, const int32_t* periodic,
                               double diameter, double zeta, int32_t n, const double* d_X,
                               int32_t max_neighbors, int32_t* d_pairs, int64_t cap,
                               int64_t* h_count, void* stream);

/* Checkpoint and resume.  A state holds what the next step reads: the PDFs (as
 * stored, in the layout of the step counter's AA parity), the step counter, the
 * particle centres, velocities and angular velocities, and the history the particle
 * update carries (previous accelerations, hydrodynamic force and torque, interior
 * momenta), and the learned initializer's parameters when set.  The Lagrangian points,
 * node masks and fixed-point centres are regenerated on restore; f_IB is zero between
 * steps.  Host buffers; both calls synchronise the stream.  set_state needs a run of
 * the same lattice, particle count, points per particle, storage, boundaries and pair
 * search (INVALID_ARG otherwise, or for a buffer that is not a state of this library
 * version); tau, gravity and the other physical parameters may differ. */
int ibm_lbm_state_size(ibm_lbm_handle* h, size_t* bytes);
int ibm_lbm_get_state(ibm_lbm_handle* h, void* h_buf, size_t bytes);
int ibm_lbm_set_state(ibm_lbm_handle* h, const void* h_buf, size_t bytes);

/* ---------------------------------------------------------------------------
 * Learned MDF initializer (no counterpart in the paper, which runs the plain
 * iteration).  A perceptron 27 -> 64 -> 64 -> 3 (ReLU) maps the velocity-deficit
 * stencil of a Lagrangian point, U_b - u_b* (u_b* = D_I u*, Eq. 12), to the force of
 * the first MDF iteration, both in a frame of the point:
 *   2D: the deficits at the point and at the 4 points on either side of it on the same
 *       circle, as (normal, tangent, 0) components;
 *   3D: the deficits at the point and at its 8 nearest other points on the reference
 *       sphere, ordered by azimuth about the normal, as (n, t1, t2) components with
 *       n = r / |r|, t1 = (a x n) / |a x n| (a = e_z, or e_x where |n_z| >= 0.9),
 *       t2 = n x t1 (distances and azimuths compared after rounding to 1e-9, ties by
 *       index).
 * Parameters: ibm_lbm_mlp_param_count() floats, row-major
 * W1[27][64] b1[64] W2[64][64] b2[64] W3[64][3] b3[3] in_scale out_scale (the network
 * sees features * in_scale; its output is scaled by out_scale).
 */
int32_t ibm_lbm_mlp_param_count(void);

/* Copy host parameters into the run (used by steps when cfg.mlp_init = 1). */
int ibm_lbm_set_mlp(ibm_lbm_handle* h, const float* h_params);

/* Training samples of the last step: d_X [npts][27] features, d_Y [npts][3] the step's
 * total MDF force F_b in each point's frame (device arrays).  Synchronises the stream.
 * Errors: INVALID_ARG before the first step. */
int ibm_lbm_mdf_samples(ibm_lbm_handle* h, float* d_X, float* d_Y);

/* Record, in every later step, the boundary-velocity residual r_b = U_b - D_I u^(M)
 * after the last MDF iteration (one extra interpolation launch). */
int ibm_lbm_set_residual_tracking(ibm_lbm_handle* h, int32_t on);

/* RMS over the points and components of r_b, sqrt(sum_b sum_c r_bc^2 / (N_p N_L dim)),
 * and the largest |r_bc|, of the last tracked step (syncs). */
int ibm_lbm_get_mdf_residual(ibm_lbm_handle* h, double* rms, double* maxabs);

/* Training kernels (FP32; device pointers; loss = mean over the batch of the squared
 * error summed over the 3 outputs).  Scratch: ibm_lbm_mlp_scratch_size bytes, 16-byte
 * aligned.  mlp_grad writes d_grad (param_count floats; the two scales get none) and
 * the loss to *h_loss (syncs when h_loss is set). */
int ibm_lbm_mlp_scratch_size(int32_t batch, size_t* bytes);
int ibm_lbm_mlp_grad(const float* d_params, const float* d_X, const float* d_T, int32_t batch,
                     float* d_grad, double* h_loss, void* d_scratch, size_t scratch_bytes, void* stream);
/* One Adam step (0.9, 0.999, 1e-8) at step t >= 1 with learning rate lr. */
int ibm_lbm_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t t, float lr,
                     void* stream);
/* Tensor-core inference (FP16 operands, FP32 accumulation) of n feature rows. */
int ibm_lbm_mlp_infer(const float* d_params, const float* d_X, int64_t n, float* d_Y, void* stream);

/* ---------------------------------------------------------------------------
 * Batched ensemble: many independent 2D cavities stepped together.  Each member is an
 * ordinary run (its own cavity size, particle count, diameter, points per particle,
 * relaxation time, ...), and every kernel of a batch step runs once for all members
 * (one launch whose blocks look up their member), so a step costs about a dozen
 * launches whatever the number of members; steps after the first replay a CUDA graph.
 * All members must be 2D and share pdf_storage (FP32 or FP16) and mdf_iters.  The
 * paper runs one cavity at a time; the batch is an execution mode of the same method
 * and gives each member the results of that member run alone.
 */
typedef struct ibm_lbm_batch ibm_lbm_batch;

/* Device bytes of a batch of n members (their workspaces and the batch's tables). */
int ibm_lbm_batch_workspace_size(const ibm_lbm_config* cfgs, int32_t n, size_t* bytes);

/* Create a batch in caller-provided device memory (256-byte aligned, borrowed until
 * ibm_lbm_batch_destroy).  h_centres[i]: host [n_particles][2] centres of member i
 * (NULL for a member without particles).  Every member's kernels run on stream.
 * Errors: as ibm_lbm_init for any member; UNSUPPORTED for 3D or BF16 members;
 * INVALID_ARG when members differ in pdf_storage or mdf_iters. */
int ibm_lbm_batch_init(const ibm_lbm_config* cfgs, int32_t n, void* d_workspace, size_t bytes,
                       void* stream, const double* const* h_centres, ibm_lbm_batch** out);

/* Enqueue n_steps steps of every member; returns after enqueueing. */
int ibm_lbm_batch_step(ibm_lbm_batch* b, int32_t n_steps);

/* Wait for the stream and report the first member status (as ibm_lbm_sync), or
 * IBMLBM_ERR_TIMEOUT when a grid barrier of the persistent mode gave up (the steps from
 * that one on are not valid; the barriers are reset and the batch can be stepped again
 * after new states are set).  Clears every status it reports. */
int ibm_lbm_batch_sync(ibm_lbm_batch* b);

/* Persistent mode (on = 1; a new batch has on = 0).  A step is then three kernel
 * launches: one cooperative kernel for the immersed-boundary phases (regeneration of
 * the Lagrangian points, Eq. 9-10; the mdf_iters interpolation and spreading
 * iterations, Eq. 11-13; the sums of the hydrodynamic force and torque, Eq. 14-15), one
 * cooperative kernel for the contact phases and the particle update (Eq. 16-18, beside
 * the collision), and the collide-stream launch (Eq. 1-8; tile shape 0 steps every
 * node, edges included, in one launch; other shapes add an edge launch in odd steps).
 * The phases inside a kernel are separated by grid barriers.  Every wait is bounded:
 * a block that polls a barrier more than barrier_limit times (about 0.2 us each;
 * 0 = the default, 10^7) gives up, sets the batch's TIMEOUT status and its kernel
 * returns; so does every other block at that barrier or the next.  The kernels' blocks
 * must all be resident at once (a cooperative launch fails otherwise, reported as
 * CUDA); nothing else may wait on them.  The arithmetic is that of the ordinary mode,
 * block for block.  Takes effect from the next step (graphs are captured again).
 * Errors: INVALID_ARG for on other than 0 or 1 or a negative barrier_limit; CUDA if the
 * IBM kernel's shared memory cannot be granted. */
int ibm_lbm_batch_set_persistent(ibm_lbm_batch* b, int32_t on, int64_t barrier_limit);
int ibm_lbm_batch_get_persistent(const ibm_lbm_batch* b, int32_t* on);

/* Member i as a run handle, for the field and particle calls (get_fields,
 * get_particles, get_pdfs, ...).  Owned by the batch; do not step or destroy it. */
ibm_lbm_handle* ibm_lbm_batch_member(ibm_lbm_batch* b, int32_t i);

/* Kernels the batch has launched so far. */
int64_t ibm_lbm_batch_launch_count(const ibm_lbm_batch* b);

/* Tile shapes of a batch's fused collide-stream launch (Eq. 1, 4-8; the work items are
 * (member, tile) pairs).  Shape 0: a block of 128 threads takes 128 K consecutive nodes
 * of a member in row-major order, across row ends, thread t its nodes t + 128 k
 * (K = 4 for FP32, 2 for FP16).  Shapes >= 1: the rows of each member are
 * cut into segments of 32 K nodes, one per warp, and a block takes W consecutive
 * segments (a tile can span several short rows); a persistent shape launches as many
 * blocks as the GPU holds at once and walks the tiles with a grid stride, the others
 * one block per tile.  Every shape updates every node with the same arithmetic, so the
 * results do not depend on the shape.  ibm_lbm_tile_shape reports shape's K, W and
 * whether it is persistent for the given storage (IBMLBM_PDF_FP32 or _FP16; shape 0
 * reports W = 4).  Errors: INVALID_ARG for an unknown shape or storage. */
int ibm_lbm_tile_shape_count(void);
int ibm_lbm_tile_shape(int32_t shape, int32_t pdf_storage, int32_t* nodes_per_thread,
                       int32_t* warps_per_block, int32_t* persistent);

/* Use tile shape `shape` from the next step on (a new batch uses shape 0).  Errors:
 * INVALID_ARG for an unknown shape. */
int ibm_lbm_batch_set_tile_shape(ibm_lbm_batch* b, int32_t shape);
int ibm_lbm_batch_get_tile_shape(const ibm_lbm_batch* b, int32_t* shape);

/* Autotuner: run steps_per_shape real steps of the batch (even, >= 2, so both AA
 * parities count alike) with each tile shape in turn, timing the collide-stream launches
 * with CUDA events, and keep the shape with the least mean time per step.  The steps
 * advance the simulation like ibm_lbm_batch_step (shapes do not change results), run
 * as eager launches, and the next ibm_lbm_batch_step captures new graphs.  Blocks
 * until the tuning steps are done.  h_ms_per_shape (host, ibm_lbm_tile_shape_count()
 * floats, or NULL) receives each shape's mean milliseconds per step.  Errors:
 * INVALID_ARG for a bad steps_per_shape; CUDA when a launch or an event fails. */
int ibm_lbm_batch_autotune(ibm_lbm_batch* b, int32_t steps_per_shape, float* h_ms_per_shape);

/* Destroy the batch and its member handles (never fails). */
void ibm_lbm_batch_destroy(ibm_lbm_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* IBMLBM_H */
