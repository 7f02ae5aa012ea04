/*
 * pb.h -- C ABI of the GB300 linear Poisson-Boltzmann hot path.
 *
 * The library solves the linearised Poisson-Boltzmann equation of
 * NextGenPB (arXiv 2502.09323, Sec. 2.1, Eq. LPBE)
 *
 *     -div(eps grad phi) + eps_s k_D^2 chi_s phi = 4 pi l_B sum_i q_i delta(r - r_i)
 *
 * in reduced units (lengths in Angstrom, charges in e, phi in kT/e, energies
 * in kT, permittivities relative, l_B the vacuum Bjerrum length at the given
 * temperature) on the paper's box-method Cartesian grid (Sec. 3.1: primal-
 * mixed Q1/Nedelec elements with vertex quadrature and static condensation),
 * with the weighted-harmonic-average permittivity on surface-crossing edges
 * (Sec. 3.2, Eq. WHA), and evaluates the energy partition of Eq. energyPart
 * with the flux-based polarisation and ionic terms of Sec. 3.3.
 *
 * Discrete system, solved for the interior nodes:
 *     (G^T W G + C) phi = f
 *     W_e  = eps_e h on edge e, 1/eps_e = alpha_e/eps_in + (1-alpha_e)/eps_out,
 *            alpha_e the fraction of the edge inside the solute;
 *     C_kk = eps_out k_D^2 h^3 on solvent nodes, 0 on solute nodes;
 *     f_k  = 4 pi l_B sum_i q_i w_k(r_i) (trilinear weights, Eq. RVop)
 *            + W_e phi_b for every edge to a Dirichlet boundary node.
 *
 * Conventions of every array that crosses this boundary:
 *   - node (i,j,k), 0 <= i < nx etc., has index (k*ny + j)*nx + i (x fastest)
 *     and position origin + (i, j, k) * h;
 *   - the edge from node a along axis d (0=x,1=y,2=z) has id d*N + a,
 *     N = nx*ny*nz; it exists when that coordinate of a is < n_d - 1;
 *   - the solute is the union of the atom balls; node a is inside when
 *     |x_a - c|^2 < R^2 for some atom (a tie is solvent);
 *   - atoms are rows (x, y, z, R, q), float64, row-major, n_atoms x 5.
 *
 * General rules:
 *   - every function returns a pb_status and never aborts or exits;
 *     pb_last_error() gives a message for the last failure of this thread;
 *   - argument errors (NULL, NaN/Inf, negative radius, n < 3, a charge whose
 *     trilinear cell touches the box boundary ...) return PB_ERR_ARG before
 *     any work is queued;
 *   - stream arguments are cudaStream_t values (NULL = legacy default stream);
 *     all device work of a call is ordered on that stream;
 *   - handles own all their device memory until pb_*_free; host arrays
 *     passed in are read during the call only and never retained;
 *   - device memory comes from the allocator installed with
 *     pb_set_allocator, else from cudaMallocAsync on the call's stream;
 *   - calls on distinct handles may run concurrently from different host
 *     threads; a handle must not be used by two threads at once.
 */
#ifndef PB_H
#define PB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PB_OK = 0,
    PB_ERR_ARG = -1,     /* invalid argument; nothing was queued            */
    PB_ERR_OOM = -2,     /* the allocator refused a request                 */
    PB_ERR_CUDA = -3,    /* a CUDA call failed (message in pb_last_error)   */
    PB_ERR_NOCONV = -4,  /* solver stopped without reaching the tolerance   */
    PB_ERR_TIMEOUT = -5, /* the solve exceeded its time budget              */
    PB_ERR_STATE = -6,   /* call out of order (e.g. pb_energy before solve) */
    PB_ERR_UNIMPL = -7   /* feature not available in this build             */
} pb_status;

enum { PB_GRID_UNIFORM = 0, PB_GRID_OCTREE = 1 };
enum { PB_BC_ZERO = 0, PB_BC_COULOMB = 1, PB_BC_DH = 2 };
enum { PB_FP64 = 0, PB_MIXED = 1 };
enum { PB_HOST = 0, PB_DEVICE = 1 };
enum { PB_CT_BOUNDARY = 1, PB_CT_SURFACE = 2, PB_CT_PAIRS = 4, PB_CT_ALL = 7 };

typedef struct pb_grid pb_grid;     /* opaque: geometry, inside flags, crossing list */
typedef struct pb_system pb_system; /* opaque: coefficients, rhs, solution, energies  */

/* Device-memory hooks.  alloc(ctx, bytes, stream) returns a device pointer
 * (NULL on failure); release(ctx, ptr, stream) frees it.  Passing NULLs
 * restores the default (cudaMallocAsync / cudaFreeAsync). */
typedef void *(*pb_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*pb_free_fn)(void *ctx, void *ptr, void *stream);
pb_status pb_set_allocator(pb_alloc_fn alloc, pb_free_fn release, void *ctx);

/* Grid specification.  Uniform grid: n[3] nodes per axis (>= 3 each).
 * If h > 0 the grid is origin + (i,j,k) h.  If h == 0 the grid is placed
 * on the device (Sec. 2.3 "perfil", Sec. 3.4): a cube of side fill * extent
 * (extent = largest axis span of the union of [x_i - R_i, x_i + R_i])
 * centred on the atoms' bounding box, h = side / (max n - 1), n[0]==n[1]==n[2]
 * required.
 *
 * Octree grid (kind PB_GRID_OCTREE; Sec. 3 and Sec. 3.4 refinement near the
 * molecular surface, 2:1-balanced 8^3-cell bricks with hanging-node
 * constraints): cell sizes h_bulk / 2^l down to h_fine (h_bulk must be
 * h_fine times a power of two, at most 2^7).  A brick is split where its
 * box lies within refine_dist of an atom sphere surface; refine_dist must
 * be at least the largest radius, h_fine and 1.5 h_bulk.  If n[0] > 0 the
 * domain is n[0]^3 coarse bricks of side 8 h_bulk from `origin`; otherwise
 * n[0] = ceil(fill * extent / (8 h_bulk)) bricks centred on the atoms'
 * bounding box.  Node arrays of an octree use the slot layout: brick b (in
 * Morton order) owns slots 512 b + (8k + j) 8 + i, its low-corner nodes;
 * N = 512 * bricks.  Listed-edge ids are d * N + slot of the low end.
 *
 * De-refined octree domain (Sec. 3.4, de-refinement for efficient boundary
 * conditions): h_tight > 0 makes h_bulk the spacing of the coarse far field
 * (h_bulk = h_tight times a power of two) and also splits every brick whose
 * cells are coarser than h_tight and whose box meets the tight box, a cube of
 * side tight_fill * extent (tight_fill >= 1, e.g. 1.1 for a perfil near 90 %)
 * centred on the atoms' bounding box; fill can then be large (e.g. 1/0.15,
 * perfil 15 %), where homogeneous Dirichlet values (PB_BC_ZERO) are accurate.
 * refine_dist must then be at least 1.5 h_tight instead of 1.5 h_bulk.
 * h_tight = 0: no tight box (every unrefined brick has cells of h_bulk). */
typedef struct {
    int32_t kind;
    int32_t n[3];
    double origin[3];
    double h;
    double fill;
    double h_fine, h_bulk, refine_dist;
    double h_tight, tight_fill;
} pb_grid_spec;

/* Physical parameters (Sec. 2.1, 2.3).  eps_in/eps_out relative
 * permittivities of solute/solvent; 1:1 salt of ionic strength I (mol/L);
 * temperature in K; bc one of PB_BC_*:
 *   ZERO     phi_b = 0 (homogeneous Dirichlet);
 *   COULOMB  phi_b = (l_B/eps_out) sum_i q_i / r;
 *   DH       phi_b = (l_B/eps_out) sum_i q_i exp(-k_D r) / r. */
typedef struct {
    double eps_in, eps_out, ionic_strength_M, temperature_K;
    int32_t bc;
} pb_params;

/* Solver options.  precision PB_FP64: Jacobi-PCG entirely in FP64.
 * PB_MIXED: FP64 iterative refinement around an FP32 Jacobi-PCG (FP32
 * stencil, vectors and per-thread accumulation, FP64 global dots).
 * Stop when ||f - A phi||_2 <= rtol ||f||_2 (true residual, FP64).
 * max_iter caps the total inner iterations, max_outer the refinement
 * steps; inner_rtol (0 = default 1e-6) is the inner relative tolerance;
 * time_budget_s (0 = none) bounds the wall time of the call. */
typedef struct {
    int32_t precision;
    double rtol;
    int32_t max_iter, max_outer;
    double inner_rtol, time_budget_s;
} pb_solve_opts;

typedef struct {
    int32_t status;           /* pb_status of the solve                     */
    int32_t iters_inner;      /* PCG iterations (FP32 inner or FP64 plain)  */
    int32_t iters_outer;      /* FP64 residual evaluations                  */
    int32_t kc;               /* tuned kernel: z-chunk + 1000 * variant
                                 (+ 10000 * tile width, TMA-staged variant) */
    double true_rel_res;      /* ||f - A phi|| / ||f|| in FP64 at exit      */
    double seconds;           /* host wall time of the call                 */
    int64_t dof;              /* interior unknowns                          */
    int64_t model_bytes;      /* modelled DRAM bytes of the solve           */
} pb_solve_stats;

/* Energy terms in kT (Sec. 3.3, Eq. energyPart):
 *   e_coul      (l_B/eps_in) sum_{i<j} q_i q_j / r_ij;
 *   e_pol       1/2 (1/eps_out - 1/eps_in) sum_e F_e Phi_e / (4 pi);
 *   e_ion_flux  -1/2 (1/eps_out) sum_e F_e Phi_e / (4 pi)  (second integral
 *               of Eq. energy_ion);
 *   e_ion_surf  1/2 sum_e phi(r_e) h^2 Psi_e / (4 pi)  (first integral of
 *               Eq. energy_ion on the staircase dual faces of the flux edges,
 *               phi(r_e) from Eq. phi0) -- a quadrature of the first integral
 *               with a cheaper surface than the paper's;
 *   e_total     sum of the four;
 *   flux_charge sum_e F_e / (4 pi l_B): the enclosed charge by Gauss' law;
 *   e_ion_mc    1/2 sum_e T_e phi(r_e) Psi^n_e / (4 pi): the first integral
 *               of Eq. energy_ion as Sec. 3.3.2 takes it, on the surface
 *               re-triangulated by marching cubes through the intersection
 *               points r_e, T_e = sum of T_j/3 over the triangles with vertex
 *               r_e, Psi^n_e with the analytic ball normal at r_e, phi(r_e)
 *               from Eq. phi0 (on octree grids, the surface of the finest
 *               lattice, where every listed edge lies).  The paper's E_ion
 *               is e_ion_mc + e_ion_flux.
 * F_e = W_e (phi_in - phi_out) over flux edges (endpoints in different
 * media), Phi_e = sum_i q_i/|r_e - r_i|, Psi_e = sum_i q_i (r_e - r_i).n_e /
 * |r_e - r_i|^3, n_e the unit edge direction from the inside endpoint. */
typedef struct {
    double e_coul, e_pol, e_ion_surf, e_ion_flux, e_total, flux_charge;
    double e_ion_mc;
} pb_energy_terms;

typedef struct {
    int32_t n[3];
    double origin[3];
    double h;
    int64_t n_nodes;          /* N: nx*ny*nz (uniform) or 512*n_bricks      */
    int64_t n_atoms;
    int64_t n_cross;          /* listed edges (see PB_ARR_CROSS_ID)        */
    int64_t n_flux;           /* listed edges whose endpoints differ       */
    int64_t n_inside;         /* solute nodes                              */
    int32_t kind;             /* PB_GRID_UNIFORM or PB_GRID_OCTREE          */
    int32_t n_levels;         /* octree: levels (1 + log2(h_bulk/h_fine))   */
    int64_t n_bricks;         /* octree: leaf bricks (N = 512 n_bricks)     */
} pb_grid_info;

/* Arrays that pb_get_array copies out (element type, length). */
enum {
    PB_ARR_INSIDE = 0,   /* uint8  [N]      1 = solute node                     */
    PB_ARR_CROSS_ID,     /* int64  [n_cross] ids of listed edges, increasing:
                            edges with 0 < alpha < 1 or with endpoints in
                            different media                                   */
    PB_ARR_CROSS_ALPHA,  /* double [n_cross] inside fraction alpha             */
    PB_ARR_CROSS_RP,     /* double [3*n_cross] r_e: alpha*h from the inside
                            endpoint towards the outside one (Sec. 3.3.1);
                            edge midpoint when both endpoints share a medium  */
    PB_ARR_CROSS_SIGN,   /* int8   [n_cross] +1 / -1: inside endpoint is the
                            low / high node; 0 same medium                    */
    PB_ARR_WX,           /* double [N] W of edge (a -> a+x), 0 if none       */
    PB_ARR_WY,           /* double [N]                                       */
    PB_ARR_WZ,           /* double [N]                                       */
    PB_ARR_KAPPA,        /* double [N] C_kk = eps_out k_D^2 h^3 or 0           */
    PB_ARR_DIAG,         /* double [N] diagonal of A (0 on boundary nodes)   */
    PB_ARR_RHS,          /* double [N] f, 0 on boundary nodes                */
    PB_ARR_BC,           /* double [N] phi_b on boundary nodes, 0 inside     */
    PB_ARR_PHI,          /* double [N] solution incl. boundary values        */
    PB_ARR_PHI_SURF,     /* double [n_cross] Phi_e (0 on non-flux edges)     */
    PB_ARR_PSI_SURF,     /* double [n_cross] Psi_e (0 on non-flux edges)     */
    PB_ARR_OCT_BRICKS,   /* int32  [4*n_bricks] octree: low corner (x, y, z in
                            units of h_fine) and level of each brick           */
    PB_ARR_OCT_KIND,     /* uint8  [N] octree: 0 unknown with a 7-point row, 1
                            boundary, 2 hanging, 3 unknown next to a level
                            change (explicit row)                           */
    PB_ARR_MC_WEIGHT,    /* double [n_cross] T_e, the sum of T_j/3 over the
                            marching-cubes triangles with vertex r_e (0 on
                            edges whose endpoints share a medium); crossing
                            order of the grid (uniform or octree)             */
    PB_ARR_MC_NORMAL,    /* double [3*n_cross] analytic outward unit normal of
                            the ball surface at r_e                           */
    PB_ARR_PSI_N,        /* double [n_cross] Psi along that normal (a system
                            after pb_coulomb_terms with the surface terms)    */
    PB_ARR_COUNT
};

/* pb_build_grid -- grid placement, node classification and the list of
 * surface-crossing edges (Sec. 2.1 eps(r); Sec. 3.2 alpha and the crossing
 * points of Eq. WHA; Sec. 2.3 perfil).  atoms: n_atoms x 5 doubles at
 * atoms_loc (PB_HOST or PB_DEVICE).  On success *out owns a new grid.  The
 * call synchronises the stream once (to size the crossing list). */
pb_status pb_build_grid(const pb_grid_spec *spec, const double *atoms, int64_t n_atoms,
                        int32_t atoms_loc, void *stream, pb_grid **out);
pb_status pb_grid_info_get(const pb_grid *g, pb_grid_info *info);
void pb_grid_free(pb_grid *g);

/* pb_assemble_coeffs -- edge weights W (Sec. 3.1 vertex quadrature +
 * Sec. 3.2 WHA), the ionic diagonal C (Sec. 2.1 linearisation), boundary
 * values (Sec. 2.3) and the right-hand side (Eq. RVop + Dirichlet lift).
 * The Coulomb/DH boundary values are an N-body sum over the box faces run
 * by this call.  The system keeps a reference to g (g must outlive it). */
pb_status pb_assemble_coeffs(pb_grid *g, const pb_params *params, void *stream,
                             pb_system **out);
void pb_system_free(pb_system *s);

/* pb_coulomb_terms -- analytic N-body sums of Sec. 3.3: PB_CT_SURFACE
 * computes Phi_e and Psi_e at the crossing points of flux edges (FP32 tiled
 * kernel with split (hi+lo) coordinates and compensated sums, FP64
 * results); PB_CT_PAIRS the Coulomb energy sum_{i<j} q_i q_j / r_ij (FP64
 * kernel over pairs of 128-atom tiles, summed in a fixed order: the energy
 * is a difference of large terms of either sign; at most 1,048,576 atoms,
 * else PB_ERR_ARG); PB_CT_BOUNDARY recomputes the Coulomb / Debye-Hueckel
 * boundary values of Sec. 2.3 (FP64 kernel, so that the Dirichlet lift
 * carries no FP32 rounding).  Results stay on the device inside s. */
pb_status pb_coulomb_terms(pb_system *s, int32_t which, void *stream);

/* pb_solve -- Jacobi-preconditioned CG for (G^T W G + C) phi = f (the
 * Krylov solve of Eq. matrixequation), zero initial guess, in the
 * precision of opts.  On PB_OK or PB_ERR_NOCONV the best phi is kept in s.
 * If phi_dev is not NULL the solution (all N nodes, boundary values
 * included, double) is also copied to that device buffer. */
pb_status pb_solve(pb_system *s, const pb_solve_opts *opts, double *phi_dev, void *stream,
                   pb_solve_stats *stats);

/* pb_energy -- energy terms of Sec. 3.3 from the solved phi; needs
 * pb_solve and pb_coulomb_terms(PB_CT_SURFACE|PB_CT_PAIRS) first
 * (PB_ERR_STATE otherwise).  *out is written on the host (the call
 * synchronises the stream). */
pb_status pb_energy(pb_system *s, void *stream, pb_energy_terms *out);

/* pb_get_phi -- copy the solution (N doubles) to dst (PB_HOST/PB_DEVICE). */
pb_status pb_get_phi(pb_system *s, double *dst, int32_t dst_loc, void *stream);

/* pb_get_array -- copy one of the PB_ARR_* arrays to dst (host or device);
 * grid arrays (INSIDE, CROSS_*) may be read with s == NULL and g set.
 * bytes must be at least the array size. */
pb_status pb_get_array(const pb_grid *g, const pb_system *s, int32_t which, void *dst,
                       size_t bytes, int32_t dst_loc, void *stream);

/* pb_apply -- y = A x on interior nodes (boundary entries of x are read as
 * zero, y is zero on boundary nodes); x, y are device arrays of N elements
 * in node order: double for PB_FP64, float for PB_MIXED (the FP32 operator
 * used by the inner solver). */
pb_status pb_apply(pb_system *s, int32_t precision, const void *x, void *y, void *stream);

/* pb_solve_batch -- solve n independent systems (different molecules, grid
 * sizes, uniform or octree) together: the CG solve of Eq. matrixequation
 * (Sec. 4) with FP32 inner iterations and FP64 iterative refinement.  PB_MIXED:
 * every system holds a slot of one launch table of persistent TMA-staged PCG
 * kernels, replayed as one captured CUDA graph; each system's refinement step
 * is decided on the device as soon as its own inner solve ends (the
 * continuous-batching engine below, with capacity n).  PB_FP64: plain PCG,
 * one system after the other.  stats has n entries (each system's status;
 * the call returns the worst).  Each system's result is bit-identical to its
 * own pb_solve with the same tuning.  All systems must live on the same
 * device, and none may appear twice (PB_ERR_ARG).  time_budget_s > 0 stops
 * the batch at the budget: unfinished systems report PB_ERR_TIMEOUT. */
pb_status pb_solve_batch(pb_system *const *systems, int32_t n, const pb_solve_opts *opts,
                         void *stream, pb_solve_stats *stats);

/* ---------------------------------------------------------------------
 * Continuous-batching engine.  A serving loop submits assembled systems
 * (pb_assemble_coeffs, and pb_coulomb_terms when energies are wanted) as
 * they arrive; the engine keeps up to `capacity` of them resident in one
 * launch table that a pump thread replays as a CUDA graph of mixed-precision
 * PCG iterations (the CG solve of Eq. matrixequation, Sec. 4, with FP32
 * inner iterations and FP64 iterative refinement).  A system submitted while others run joins at the
 * next replay once a slot is free; a finished one leaves at once and is
 * reported through pb_engine_wait.  Octree systems run their brick
 * kernels beside the table, the same number of iterations per replay.  The paper solves one system at a time:
 * the engine is the serving form of the same solve, and a system's result is
 * the same (bit for bit, for the same z-chunk) alone or in any mix.
 * ------------------------------------------------------------------- */
typedef struct pb_engine pb_engine;

typedef struct {
    int64_t ticket;          /* from pb_engine_submit */
    pb_system *system;       /* the submitted system (its phi holds the solution) */
    pb_solve_stats stats;    /* status PB_OK, PB_ERR_NOCONV, PB_ERR_TIMEOUT, or the
                                engine's error; seconds = time since admission */
    double t_submit, t_admit, t_done;  /* CLOCK_MONOTONIC seconds */
} pb_engine_result;

/* pb_engine_create -- engine on `device` with `capacity` slots (1..4096);
 * opts->rtol / inner_rtol / max_iter / max_outer apply to every solve
 * (precision and time_budget_s are ignored: the engine is mixed precision).
 * Allocates a small device table (about 3.5 KB per slot) and starts the
 * pump thread. */
pb_status pb_engine_create(int32_t device, int32_t capacity, const pb_solve_opts *opts,
                           pb_engine **out);

/* pb_engine_submit -- queue s for solving.  `stream` is the stream on which
 * s was assembled (its work is waited for on the device, not on the host);
 * the solver workspace is allocated here, on that stream.  From submission
 * until its result is returned by pb_engine_wait the system belongs to the
 * engine: do not use or free it.  PB_ERR_ARG if s is already in the engine
 * or lives on another device. */
pb_status pb_engine_submit(pb_engine *e, pb_system *s, void *stream, int64_t *ticket);

/* pb_engine_wait -- move up to max_out finished solves into out (*n_out of
 * them), waiting up to timeout_s seconds for at least one (0: do not wait).
 * Returns the engine's error if it failed and nothing is left to report. */
pb_status pb_engine_wait(pb_engine *e, double timeout_s, pb_engine_result *out, int32_t max_out,
                         int32_t *n_out);

/* pb_engine_query -- systems waiting for a slot, systems in the table, and
 * graph replays so far (any pointer may be NULL); returns the engine's
 * error status. */
pb_status pb_engine_query(pb_engine *e, int32_t *n_pending, int32_t *n_active, int64_t *replays);

/* pb_engine_destroy -- stop the pump thread after the replays in flight and
 * free the engine.  Systems still waiting or running are handed back
 * unsolved (their results, with PB_ERR_STATE, are dropped). */
pb_status pb_engine_destroy(pb_engine *e);

/* pb_profile_kernels -- timing hook: run `reps` launches of the PCG kernels
 * of the given precision on s's solver state with the convergence test off
 * (iterate and state are overwritten, so call it after pb_energy).  which:
 * 0 = direction kernel (p = z + beta p, A p, p.Ap), 1 = update kernel (A p,
 * x and z update, the two dots), 2 = both (one PCG iteration per rep).
 * Needs a prior pb_solve in that precision (PB_ERR_STATE otherwise). */
pb_status pb_profile_kernels(pb_system *s, int32_t precision, int32_t which, int32_t reps,
                             void *stream);

/* pb_set_tuning -- fix the PCG kernel variant (0: register-pipelined warps,
 * 1: TMA-staged, FP32 only) and z-chunk length (planes per block) used for
 * every system with s's grid shape and this precision, instead of the
 * autotuner's choice (which times the candidates on first use of a shape).
 * For the TMA-staged variant z_chunk may add 10000 * the tile width in x
 * (128, 64 or 32 points; tiles are width x 1024/width points of a plane;
 * no addition: 128).  Other widths give PB_ERR_ARG. */
pb_status pb_set_tuning(pb_system *s, int32_t precision, int32_t variant, int32_t z_chunk);

/* pb_solve_split -- the mixed-precision solve of pb_solve (uniform grids) on
 * `ranks` z-slabs (1 .. min(64, nz - 2)): the multi-GPU decomposition of one
 * system (Sec. 4 solves on distributed memory).  Each rank holds its owned
 * planes plus one halo plane on each side in its own buffers; before the
 * direction kernels the z halos, before the update kernels the new p halos,
 * and before every FP64 residual the phi halos are copied from the
 * neighbours into each receiver's memory (cudaMemcpyPeerAsync); each
 * kernel round's partial dot products are added in rank order and the CG
 * update is written to every rank, so all ranks take the same decisions.
 * In this build every rank lives on the system's device.  ranks = 1 gives
 * pb_solve's result bit for bit (same z-chunk); more ranks change only the
 * order of the dot-product sums.  phi is gathered back into s (pb_energy
 * works as after pb_solve).  Errors: PB_ERR_ARG for a bad rank count or a
 * precision other than PB_MIXED, PB_ERR_UNIMPL for octree systems, and the
 * statuses of pb_solve. */
pb_status pb_solve_split(pb_system *s, int32_t ranks, const pb_solve_opts *opts, void *stream,
                         pb_solve_stats *stats);

/* pb_set_wait_limit -- failure-injection hook for tests: the number of polls
 * after which a ring-slot wait of the FP32 PCG kernels (one-system, batched
 * and served launches) gives up; polls < 0 restores the default (2^20).  With
 * 0 every slot wait gives up at once, so the next FP32 PCG launch stops, waits
 * for its own copies in flight and marks every system of its launch with
 * device status 3: pb_solve and pb_solve_batch then return PB_ERR_TIMEOUT, and
 * a served system finishes with that status.  The drain of a block's own
 * copies keeps the default limit, and the work counters are reset as after any
 * launch, so the system solves normally once the limit is restored.  Applies
 * to the current device; synchronises the device, so call it with no solve in
 * flight.  The paper has no counterpart (it covers failure detection). */
pb_status pb_set_wait_limit(int64_t polls);

/* pb_apply_dot_noalloc -- y = A x (FP64 operator, interior nodes; boundary
 * entries of x read as zero, y = 0 on boundary nodes) and *xAx = x.(A x),
 * computed without allocating any device memory.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory while
 * they work (an application whose device memory belongs to its own pool or to
 * another framework, or a latency-critical loop that cannot accept
 * cudaMalloc's implicit synchronisation).
 * x, y: device arrays of N doubles in node order; xAx: one device double.
 * Scratch is a fixed array inside the library (about 128 KB, held by every
 * GPU that loads the library until the process exits); grids of more than
 * 16384 * 2048 = 33,554,432 nodes are rejected with PB_ERR_ARG.  The first
 * call on a device looks up the array's device address (set-up), so make
 * that first call before any stream capture.  All calls share the array:
 * calls that overlap on the GPU race and must be serialised by the caller.
 * The system's device must be the current device. */
pb_status pb_apply_dot_noalloc(const pb_system *s, const double *x, double *y, double *xAx,
                               void *stream);

/* Number of CUDA kernels launched by this library in this process so far. */
int64_t pb_kernel_launches(void);

/* Thread-local message describing the last failure ("" if none). */
const char *pb_last_error(void);
/* Library version string. */
const char *pb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PB_H */
