/*
 * bipb.h -- C ABI of libbipb, a single-GPU (GB300, sm_103a) direct-sum
 * boundary-integral Poisson-Boltzmann solver.
 *
 * Method (Yang, Sliheet, Iriye, Reynolds, Geng, "Optimized Parallelization of
 * Boundary Integral Poisson-Boltzmann Solvers", arXiv 2312.10044):
 *   - model and units: Sec. 2.1 (linearised PB, eps_in inside, eps_out
 *     outside, inverse Debye length kappa, lengths in Angstrom, potentials
 *     times 332.0716 give kcal/mol/e);
 *   - boundary integral equations, kernels K1..K4 and source terms S1, S2:
 *     Sec. 2.2.1 (Eqs. for the well-conditioned BIE, K1..K4, S1/S2);
 *   - centroid collocation with the self term j = i omitted, and the linear
 *     system A u = b solved by GMRES: Sec. 2.2.2 (Eqs. 5-6);
 *   - solvation energy E_sol = 1/2 sum_k q_k phi_reac(y_k): Sec. 2.2.1
 *     (Eq. for E_sol);
 *   - GPU direct-sum pipeline (source, mat-vec inside GMRES, energy):
 *     Sec. 2.4 (Table "Pseudocode for DSBI-PB solver using GPU").
 *
 * Unknowns: u = [phi_1..phi_N ; psi_1..psi_N], psi = dphi/dnu on the inner
 * side of the surface, in the internal units of the paper's equations
 * (G0 = 1/(4 pi r)); entry points that return physical values say so.
 *
 * Conventions for every entry point:
 *   - Return a bipb_status; on failure bipb_last_error() (thread-local) holds
 *     a message.  No C++ exception crosses this boundary.
 *   - Host pointers ("host") are read or written synchronously and never
 *     retained; the library copies what it keeps.  Device pointers ("device")
 *     must be CUDA device memory of the current device; the library reads and
 *     writes them on the handle's stream and does not retain them.
 *   - Array layouts are row-major: an "n x 3" array holds x0 y0 z0 x1 y1 z1 ..
 *   - All work runs on the stream given at creation (NULL = legacy default
 *     stream).  Calls with host outputs synchronise that stream before they
 *     return; calls with only device outputs are asynchronous.
 *   - A handle is not thread-safe: serialise calls on one handle.
 */
#ifndef BIPB_H
#define BIPB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bipb_surface_s* bipb_surface; /* opaque; owns all its device memory */

typedef enum {
  BIPB_OK = 0,
  BIPB_ERR_INVALID_ARG = 1,   /* bad size, pointer, value; nothing launched */
  BIPB_ERR_CUDA = 2,          /* a CUDA call failed; message in bipb_last_error() */
  BIPB_ERR_OOM = 3,           /* device allocation failed */
  BIPB_ERR_NOT_CONVERGED = 4, /* solve hit max_iter; best iterate kept, info filled */
  BIPB_ERR_STATE = 5          /* call order violated (e.g. energy before solve) or stale handle */
} bipb_status;

typedef enum {
  BIPB_FP64 = 0,       /* all pair arithmetic in FP64 */
  BIPB_MIXED = 1,      /* FP32 pair arithmetic inside GMRES, FP64 refinement residual */
  BIPB_FP32 = 2,       /* mat-vec only: FP32 pair arithmetic, FP64 sums across tiles */
  BIPB_DF64 = 3,       /* pair arithmetic in double-float (two FP32 words, ~48 bits) on the FP32
                          pipe, FP64 sums across tiles; as a solve: GMRES on that mat-vec */
  BIPB_MIXED_DF64 = 4, /* FP32 pair arithmetic inside GMRES, double-float refinement residual */
  BIPB_TENSOR = 5,     /* mat-vec only, right-hand sides of one surface, A u or A^T u: kernel tiles
                          generated in FP32 and contracted against blocks of 64 right-hand sides on
                          the tensor cores (rows and columns scaled by powers of two, each operand
                          split into two FP16 parts, three products per tile, FP32 accumulation,
                          FP64 sums across tiles: about FP32 accuracy for kernel values and
                          right-hand sides within about 2^-86 .. 2^114 of their row's / column's
                          largest) */
  BIPB_MIXED_TENSOR = 6, /* tensor-core mat-vec inside GMRES (its transpose in adjoint solves),
                            double-float refinement residual */
  BIPB_TF32 = BIPB_TENSOR,             /* earlier name of BIPB_TENSOR */
  BIPB_MIXED_TF32 = BIPB_MIXED_TENSOR, /* earlier name of BIPB_MIXED_TENSOR */
  BIPB_TREE32 = 7,     /* mat-vec only, single-surface handles: the far-field (treecode) operator of
                          Sec. 2.2.3 (A u, or A^T u with the same tree, lists and proxies) in FP32 pair
                          arithmetic, FP64 sums across work items (bipb_treecode sets its parameters) */
  BIPB_MIXED_TREE = 8  /* far-field FP32 mat-vec inside GMRES (its transpose in adjoint solves),
                          double-float refinement residual (the residual stays the direct sum, so the
                          solve still reaches tol on the exact discrete system) */
} bipb_precision;

/* Dielectric medium (Sec. 2.1): eps_in > 0 inside, eps_out > 0 outside, kappa >= 0 (1/A). */
typedef struct {
  double eps_in;
  double eps_out;
  double kappa;
} bipb_medium;

typedef struct {
  bipb_medium medium;
  double tol;          /* target ||b - A u||_2 / ||b||_2, 0 < tol < 1 */
  int restart;         /* GMRES restart length m, 1..200 (10 if 0) */
  int max_iter;        /* cap on GMRES iterations summed over restarts and refinement steps (1000 if 0) */
  int precision;       /* bipb_precision: BIPB_FP64, BIPB_MIXED, BIPB_DF64, BIPB_MIXED_DF64, BIPB_MIXED_TENSOR
                          or BIPB_MIXED_TREE */
  int inner_max_iter;  /* MIXED: cap on inner iterations per refinement step (200 if 0) */
  double inner_tol;    /* MIXED: inner relative tolerance per refinement step (1e-6 if 0) */
  const double* x0;    /* optional warm start, host, n_rhs x 2N internal units, or NULL (zero) */
  int precond;         /* bipb_precond (BIPB_PRECOND_NONE if 0) */
  int reserved;        /* set to 0 */
} bipb_solve_params;

/*
 * Preconditioning of the Krylov solves by the block diagonal M of A over
 * leaves of elements (Sec. 2.2.4), applied on the right: GMRES on
 * A M^-1 y = b, u = M^-1 y, so that it minimises the true residual.
 * (The paper writes the left form M^-1 A u = M^-1 b; both have the same
 * preconditioned spectrum, and the right form keeps the residual that the
 * stopping tests and the refinement read unscaled.)
 * BIPB_PRECOND_SELF takes each element as its own leaf: with the self pair
 * omitted its 2 x 2 block is diag(1/2 (1 + eps), 1/2 (1 + 1/eps)), so M^-1
 * rescales the phi and psi rows and costs nothing per iteration (the
 * normalisation and restart kernels write the scaled input of the next
 * mat-vec, and the solution update applies it to the correction).  On
 * smooth molecular surfaces it cuts GMRES(10) to 1e-8 from about 27 to
 * about 10 iterations.  The solve still stops on the true residual
 * ||b - A u|| / ||b|| (mixed modes: the high-precision refinement
 * residual; BIPB_FP64 / BIPB_DF64: a restart on the true residual until it
 * meets tol).  The paper's GPU pipeline runs without preconditioning
 * (BIPB_PRECOND_NONE).
 */
typedef enum { BIPB_PRECOND_NONE = 0, BIPB_PRECOND_SELF = 1 } bipb_precond;

typedef struct {
  int converged;       /* 1 if rel_residual <= tol */
  int iters;           /* GMRES iterations (inner iterations for MIXED) */
  int refine_steps;    /* mixed modes: refinement steps taken (0 for FP64 and DF64) */
  int matvecs64;       /* FP64 or double-float mat-vecs applied to this right-hand side */
  int matvecs32;       /* FP32 (CUDA-core, tensor-core or far-field) mat-vecs applied to this right-hand side */
  int reserved;
  double rel_residual; /* final ||b - A u|| / ||b||: the true residual, formed with the FP64 or
                          double-float mat-vec and FP64 vector arithmetic */
  double seconds;      /* wall time of the whole bipb_solve call */
} bipb_solve_info;

/*
 * Create a surface from N flat triangles (centroid collocation, Sec. 2.2.2).
 *   centroids: host, n x 3, Angstrom.  normals: host, n x 3, unit, outward
 *   (re-normalised; |n| must be within 1e-6 of 1).  areas: host, n, > 0, A^2.
 *   cuda_stream: a cudaStream_t or NULL.
 * Validation (BIPB_ERR_INVALID_ARG, nothing allocated): n >= 2, every value
 * finite, areas > 0, no two centroids equal in FP64 or after rounding to
 * FP32 about the mean centroid.
 */
bipb_status bipb_surface_create(int64_t n, const double* centroids, const double* normals,
                                const double* areas, void* cuda_stream, bipb_surface* out);

/*
 * Create one handle for n_surf surfaces of uneven size, solved together
 * (one system per surface: every pass and every GMRES step covers all of
 * them in one launch).  Surface k: n_tri[k] triangles, centroids[k] (n x 3),
 * normals[k] (n x 3), areas[k] (n), all host, validated as in
 * bipb_surface_create.  Charges come through bipb_charges_set_batch.
 * Batched vectors (bipb_matvec with n_vec = 1, bipb_source, bipb_reaction,
 * bipb_surface_potential) hold the surfaces back to back, surface k's
 * 2 n_tri[k] unknowns [phi_k; psi_k] after those of surfaces 0 .. k-1.
 * The paper solves one molecule at a time; this batching is an extension.
 */
bipb_status bipb_surface_create_batch(int n_surf, const int64_t* n_tri, const double* const* centroids,
                                      const double* const* normals, const double* const* areas,
                                      void* cuda_stream, bipb_surface* out);

/* Free every device allocation of the handle; the handle value becomes invalid. */
bipb_status bipb_surface_destroy(bipb_surface s);

/* Number of triangles N of the handle (0 for an invalid handle). */
int64_t bipb_surface_size(bipb_surface s);

/*
 * Set n_rhs charge configurations (the point charges of Sec. 2.1, Eq. for rho).
 *   pos: host, (n_pos_sets x nc x 3) Angstrom with n_pos_sets = 1 (shared by
 *        all configurations) or n_rhs (one position set per configuration).
 *   q:   host, n_rhs x nc, units of e.
 * Charges must lie off every centroid.  Invalidates any previous solution.
 */
bipb_status bipb_charges_set(bipb_surface s, int64_t nc, const double* pos, int n_pos_sets,
                             int n_rhs, const double* q);

/*
 * bipb_charges_set with device inputs (for callers whose charges live on the
 * GPU, e.g. the autograd path): pos and q are device arrays of the current
 * device with the layouts of bipb_charges_set, read asynchronously on the
 * handle's stream (ordered after the work the creation stream has queued).
 * The checks of bipb_charges_set (finite values, no charge on a centroid)
 * run on the device; a failure is reported, as BIPB_ERR_INVALID_ARG, by the
 * next call that uses the charges (bipb_solve, bipb_source, bipb_reaction),
 * which then forgets them.  Single-surface handles.
 */
bipb_status bipb_charges_set_dev(bipb_surface s, int64_t nc, const double* pos, int n_pos_sets, int n_rhs,
                                 const double* q);

/*
 * Charges of a batch handle: surface k gets nc[k] charges at pos[k]
 * (host, nc[k] x 3, Angstrom) with values q[k] (host, nc[k], e).
 * Charge-indexed outputs (bipb_reaction, bipb_energy_grad) list them surface
 * by surface.
 */
bipb_status bipb_charges_set_batch(bipb_surface s, const int64_t* nc, const double* const* pos,
                                   const double* const* q);

/*
 * Solve A u = b for every configuration (GMRES, Sec. 2.2.2; Eqs. 5-6), where
 * b = [S1; S2] of the charges (Eq. for S1, S2).  info: host array of n_rhs
 * (may be NULL).  Returns BIPB_ERR_NOT_CONVERGED if any configuration missed
 * tol within max_iter; its best iterate is kept and can still be read.
 */
bipb_status bipb_solve(bipb_surface s, const bipb_solve_params* p, bipb_solve_info* info);

/* Solvation energy per configuration (or per surface of a batch handle),
 * kcal/mol, host array (Eq. for E_sol). */
bipb_status bipb_energy(bipb_surface s, double* e_sol);

/* bipb_energy into device memory (n_rhs doubles, kcal/mol), asynchronous on
 * the handle's stream. */
bipb_status bipb_energy_dev(bipb_surface s, double* e_sol);

/*
 * Surface potential phi (kcal/mol/e) and its inner normal derivative
 * (kcal/mol/e/A), host arrays n_rhs x N each; dphi_dn may be NULL.
 */
bipb_status bipb_surface_potential(bipb_surface s, double* phi, double* dphi_dn);

/*
 * Potential (kcal/mol/e) at points off the surface, from the last solve, for
 * every configuration: host arrays pts (n_pts x 3, A, the frame of the
 * surface's centroids) and phi (n_rhs x n_pts).  The caller states where the
 * points lie (no inside test is made):
 *   BIPB_REGION_INSIDE  (the molecule, Omega_1): Eq. eq_inside,
 *     phi(p) = sum_j ds_j [K1(p, x_j) dphi/dnu_j + K2(p, x_j) phi_j] + S1(p);
 *   BIPB_REGION_OUTSIDE (the solvent, Omega_2): the exterior representation
 *     Eq. eqbim_2, phi(p) = sum_j ds_j [-Gk(p, x_j) (eps_in/eps_out) dphi/dnu_j
 *     + dGk(p, x_j)/dnu_y phi_j] (flux continuity gives the exterior
 *     normal derivative).
 * Pair arithmetic in double-float (about 1e-14 relative), FP64 sums in a
 * fixed order.  Single-surface handles; at most 2^24 points per call.
 * Points on or very near the surface (closer than the element size) get
 * the quadrature error of the centroid rule there.
 */
typedef enum { BIPB_REGION_INSIDE = 0, BIPB_REGION_OUTSIDE = 1 } bipb_region;
bipb_status bipb_potential_at(bipb_surface s, int region, int64_t n_pts, const double* pts, double* phi);

/*
 * Electrostatic free energy (Eq. free_energy) per configuration, kcal/mol,
 * host arrays (either may be NULL):
 *   e_coul = 332.0716 / eps_in * 1/2 sum_{k != l} q_k q_l / |y_k - y_l|
 *            (the charges' Coulomb energy in the solute dielectric; the
 *            infinite self terms k = l of S1(y_k) are left out);
 *   e_free = E_sol + e_coul.
 * Requires a successful bipb_solve.  FP64, O(Nc^2) pairs, fixed order.
 * BIPB_ERR_INVALID_ARG if two charges of a configuration coincide.
 */
bipb_status bipb_energy_free(bipb_surface s, double* e_free, double* e_coul);

/*
 * Gradient of the solvation energy (kcal/mol) of every configuration with
 * respect to its charges (host, n_rhs x nc, kcal/mol/e) and charge positions
 * (host, n_rhs x nc x 3, kcal/mol/A), at fixed surface, from one adjoint
 * solve A^T lam = c per configuration (c: the energy row, E = 1/2 c.u).
 * Requires a successful bipb_solve; p gives the adjoint solve's settings.
 */
bipb_status bipb_energy_grad(bipb_surface s, const bipb_solve_params* p, double* dE_dq,
                             double* dE_dpos);

/* bipb_energy_grad with device outputs (same layouts, kcal/mol/e and
 * kcal/mol/A), written on the handle's stream; the adjoint GMRES still
 * synchronises the stream once per restart cycle to read its convergence
 * state, but no array passes through the host. */
bipb_status bipb_energy_grad_dev(bipb_surface s, const bipb_solve_params* p, double* dE_dq, double* dE_dpos);

/* ---------------------------------------------------------------------------
 * Hot-path building blocks on device memory (asynchronous on the handle's
 * stream).  They expose the passes of the paper's GPU pipeline (Sec. 2.4)
 * one by one, for parity testing, benchmarking and custom drivers.
 * ------------------------------------------------------------------------- */

/*
 * y = A u (transpose = 0) or y = A^T u (transpose = 1) for n_vec vectors.
 *   u, y: device, n_vec x 2N doubles, internal units; y must not alias u.
 *   For a batch handle n_vec must be 1 and u, y are batched vectors (the
 *   block-diagonal operator of all surfaces).
 *   precision: BIPB_FP64, BIPB_FP32 (FP32 pair arithmetic per source tile,
 *   FP64 sums across tiles and for the diagonal), BIPB_DF64, BIPB_TENSOR
 *   (single-surface handles, both directions; the tensor-core path of the
 *   multi-RHS mat-vec) or BIPB_TREE32 (single-surface handles, both
 *   directions; the far-field operator).
 */
bipb_status bipb_matvec(bipb_surface s, const bipb_medium* m, int precision, int transpose,
                        int n_vec, const double* u, double* y);

/* b = [S1; S2] for every configuration: device, n_rhs x 2N doubles (pair
 * arithmetic in double-float, about 1e-14 relative; FP64 sums). */
bipb_status bipb_source(bipb_surface s, const bipb_medium* m, double* b);

/*
 * Reaction potential at every charge of every configuration from surface
 * values u (device, n_rhs x 2N, internal units):
 *   phi_reac(y_k) = sum_j ds_j [K1(y_k, x_j) psi_j + K2(y_k, x_j) phi_j]
 * written to phi_reac (device, n_rhs x nc, internal units), and
 * e_sol (device, n_rhs, kcal/mol) = 4 pi 332.0716 * 1/2 sum_k q_k phi_reac(y_k).
 * Either output may be NULL.  Pair arithmetic in double-float (about 1e-14
 * relative), FP64 sums in a fixed order.
 */
bipb_status bipb_reaction(bipb_surface s, const bipb_medium* m, const double* u,
                          double* phi_reac, double* e_sol);

/* ---------------------------------------------------------------------------
 * Kernel timing.  The paper reports the mean time of one mat-vec per GMRES
 * iteration (Sec. 3, Eq. for the average mat-vec time); these calls expose
 * the same quantity per pair kernel, from CUDA events recorded around every
 * launch of the kind on the handle's stream (inside recorded CUDA graphs too).
 * ------------------------------------------------------------------------- */
typedef enum {
  BIPB_KERNEL_MATVEC64 = 0,   /* FP64 mat-vec pair kernel */
  BIPB_KERNEL_MATVEC32 = 1,   /* FP32 mat-vec pair kernel */
  BIPB_KERNEL_MATVEC64_T = 2, /* FP64 transposed mat-vec pair kernel */
  BIPB_KERNEL_MATVEC32_T = 3, /* FP32 transposed mat-vec pair kernel */
  BIPB_KERNEL_SOURCE = 4,     /* source-term pair kernel */
  BIPB_KERNEL_REACTION = 5,   /* reaction-potential / energy pair kernel */
  BIPB_KERNEL_ENERGY_ROW = 6, /* energy-row pair kernel (adjoint right-hand side) */
  BIPB_KERNEL_GRAD = 7,       /* energy-gradient pair kernel */
  BIPB_KERNEL_MATVECDF = 8,   /* double-float mat-vec pair kernel */
  BIPB_KERNEL_MATVECDF_T = 9, /* double-float transposed mat-vec pair kernel */
  BIPB_KERNEL_MATVEC_TC = 10, /* tensor-core multi-RHS mat-vec kernel */
  BIPB_KERNEL_POTENTIAL = 11, /* potential-at-points pair kernels */
  BIPB_KERNEL_MATVEC_TREE = 12, /* far-field (treecode) mat-vec kernel */
  BIPB_KERNEL_KINDS = 13
} bipb_kernel_kind;

/* Turn timing on (1) or off (0); turning it on clears the totals. */
bipb_status bipb_timer_enable(bipb_surface s, int on);

/* Launch count and summed duration (ms) of one kernel kind since the timer
 * was turned on (host outputs; synchronises the handle's stream). */
bipb_status bipb_timer_read(bipb_surface s, int kind, int64_t* launches, double* total_ms);

/*
 * Autotuner of the FP32 mat-vec tiling (threads per CTA, targets per thread,
 * sources per shared-memory chunk, and whether each unordered pair is
 * visited once or twice): times every compiled variant, reps launches each,
 * on this surface and medium, keeps the fastest for the handle, and returns
 * its index (host, may be NULL) and its time per mat-vec in ms (host, may be
 * NULL).  Synchronises the handle's stream.  Variants differ only in
 * summation order, not in the operator.
 */
bipb_status bipb_autotune(bipb_surface s, const bipb_medium* m, int reps, int* variant,
                          double* ms_per_matvec);

/* Select an FP32 mat-vec variant by index, 0 <= variant < BIPB_MATVEC32_VARIANTS.
 * Variants 0-6 visit every ordered pair (i, j) (one target per thread
 * gathering all sources); variants 7-9 visit every unordered pair {i, j} once
 * and apply it to both rows, sharing 1/r, exp(-kappa r), t and w between the
 * two directions of Eqs. 5-6.  A new handle starts with variant 9. */
#define BIPB_MATVEC32_VARIANTS 10
bipb_status bipb_matvec_variant(bipb_surface s, int variant);

/* How the FP64 and double-float mat-vecs (and their transposes) visit pairs:
 * symmetric = 1 (the default) evaluates every unordered pair once and applies
 * it to both rows; symmetric = 0 evaluates every ordered pair.  Both compute
 * the operator of Eqs. 5-6 and differ only in summation order.  Surfaces too
 * large for the symmetric work list use the ordered form either way. */
bipb_status bipb_symmetric_pairs(bipb_surface s, int symmetric);

/* How the double-float mat-vec applies one surface's kernel to 16 or more
 * right-hand sides (the refinement residual of batched solves; for A^T, to
 * four or more): tensor = 1 (the default) digitises the df64 kernel values
 * and right-hand sides into seven exact base-128 FP16 digits and multiplies
 * them on the tensor cores with exact FP32 accumulation, in both directions;
 * tensor = 0 runs df64 multiply-adds on the CUDA cores for A u and the
 * single-system double-float kernel for A^T.  All reach about 1e-14 of the
 * largest output. */
bipb_status bipb_exact_tensor_residual(bipb_surface s, int tensor);

/*
 * Parameters of the far-field (treecode) mat-vec, Sec. 2.2.3 (BIPB_TREE32,
 * BIPB_MIXED_TREE).  The elements form a binary tree of clusters: a cluster
 * (a box of centroids) holding more than leaf_size elements is split in two
 * at the median of its longest side.  Targets are taken leaf by leaf; for a
 * target leaf B (centre x_B, radius r_B = half its box diagonal) a cluster c
 * (x_c, r_c) is far when r_c + theta r_B <= theta |x_B - x_c|, which gives
 * the paper's acceptance criterion r_c / |x - x_c| <= theta for every target
 * x of B.  A far cluster with more elements than (degree + 1)^3 acts through
 * (degree + 1)^3 proxy sources at the Chebyshev points of its box, weighted
 * by the Lagrange interpolant of its elements' values (a polynomial of the
 * given degree per coordinate in the source position, where the paper writes
 * a Taylor series about the cluster centre); every other pair is summed
 * directly.  theta in [0, 1) (0: every pair direct), degree 4, 6 or 8,
 * leaf_size in [32, 512].  Defaults: 0.5, 6, 256 (about 1e-7 of the largest
 * output on a 81920-element molecular surface, below the FP32 mat-vec's own
 * error).  Single-surface handles only.  The tree is built on the host at the
 * first far-field mat-vec after a change (it synchronises the stream then).
 */
bipb_status bipb_treecode(bipb_surface s, double theta, int degree, int leaf_size);

/* Size of the far-field operator of the current parameters (builds it if
 * needed): pairs = (target, source or proxy) pairs one mat-vec evaluates for
 * one right-hand side, far_clusters = clusters acting through proxies,
 * leaves = target leaves.  Host outputs, each may be NULL. */
bipb_status bipb_treecode_stats(bipb_surface s, int64_t* pairs, int* far_clusters, int* leaves);

/* Number of CUDA kernels this handle has launched since creation (kernels
 * inside replayed CUDA graphs included).  Host output; no synchronisation. */
bipb_status bipb_launch_count(bipb_surface s, int64_t* launches);

/* ---------------------------------------------------------------------------
 * Allocation-free FP32 mat-vec.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- code whose host
 * framework has already reserved nearly all device memory for its own
 * allocator, or a time-critical loop that must not allocate after start-up.
 * Such callers cannot create a bipb_surface (creating one allocates).
 *
 * y = A u, the same operator as bipb_matvec with BIPB_FP32, from geometry
 * passed as device pointers:
 *   centroids: device, n x 3 doubles (Angstrom); normals: device, n x 3
 *   (unit, outward); areas: device, n (> 0); u, y: device, 2N doubles each,
 *   internal units; y must not alias u.  The geometry is not validated (the
 *   data are on the device): it must satisfy what bipb_surface_create checks.
 *   cuda_stream: a cudaStream_t or NULL; the call is asynchronous on it.
 * 2 <= n <= 32768, else BIPB_ERR_INVALID_ARG.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: its scratch (about 10 MiB) is one
 * statically sized device array that every GPU loading the library holds
 * until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current and
 * keeps it for the life of the process; make that first call before any
 * stream capture.  A cudaDeviceReset after the first call on a device is not
 * supported: the kept address would then be stale.  Every call shares the one
 * array, so calls that overlap on the GPU (concurrent streams, or several
 * host threads) race and corrupt each other's results: serialise them.
 * Errors are reported through the status and bipb_last_error().
 * ------------------------------------------------------------------------- */
bipb_status bipb_matvec32_static(int64_t n, const double* centroids, const double* normals,
                                 const double* areas, const bipb_medium* m, const double* u, double* y,
                                 void* cuda_stream);

/* Most recent error message of this thread ("" if none). */
const char* bipb_last_error(void);
const char* bipb_status_string(bipb_status st);

/* Library version string. */
const char* bipb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BIPB_H */
