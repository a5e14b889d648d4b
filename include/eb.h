/*
 * eb.h -- C ABI of the GB300 library for the explicit embedded-boundary (EB)
 * advance on a staggered mesh (Kang et al., "An Embedded Boundary Scheme for
 * Three-Dimensional Flow Over Terrain on a Staggered Mesh").
 *
 * The library computes, on one GPU:
 *   - the cut-cell geometry of the terrain z = h(x, y) on the cell-centred
 *     grid and on the x-, y- and z-face grids (Sec. 3.2), once;
 *   - the cut-cell flux divergence dU of every grid (Sec. 3.1, Eqs.
 *     update-cc and update-fc; advective fluxes of Sec. 4.1 with zero flux
 *     through the EB and the domain walls);
 *   - weighted state redistribution R on every grid (Sec. 5.1);
 *   - the step U^{n+1} = R[U^n + dt dU(U^n)] of Eq. basic_fv_srd, or the
 *     three-stage Runge-Kutta form of Algorithm 1 (Sec. 5.2).
 *
 * Conventions (all entry points):
 *   - Domain [0,Lx] x [0,Ly] x [0,Lz] with origin 0, nx x ny x nz cells,
 *     periodic in x and y, walls at z = 0 and z = Lz.  Fluid is z > h.
 *   - Every array pointer is a DEVICE pointer owned by the caller unless
 *     stated otherwise; arrays are dense, x fastest: index i + nx*(j + ny*k).
 *   - Field sizes: rho, rho*theta (cell centres), rho*u (x faces), rho*v
 *     (y faces): nx*ny*nz.  rho*w (z faces): nx*ny*(nz+1); its levels 0 and
 *     nz are the walls, are never updated and enter every flux as zero.
 *   - Element type: double for EB_F64, float for EB_MIXED.  With a reference
 *     profile (eb_geom_build), rho and rho*theta hold perturbations about it.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream).  Argument errors are found
 *     on the host before anything is launched and return
 *     EB_ERR_INVALID_ARG.  Errors raised inside kernels (non-finite values,
 *     an expired wait) latch into a device status word that eb_sync_status
 *     reports.  No C++ exception crosses this boundary.
 *   - eb_last_error() returns a thread-local message for the last non-OK
 *     status of the calling thread.
 */
#ifndef EB_H
#define EB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EB_OK = 0,
  EB_ERR_INVALID_ARG = 1, /* bad pointer, size, enum or handle            */
  EB_ERR_CUDA = 2,        /* a CUDA runtime call failed                    */
  EB_ERR_OOM = 3,         /* device allocation failed                      */
  EB_ERR_NUMERIC = 4,     /* a kernel met a non-finite value              */
  EB_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired            */
  EB_ERR_STATE = 6        /* call not valid in the handle's current state  */
} eb_status;

typedef enum {
  EB_F64 = 0,   /* state, fluxes and redistribution in double                    */
  EB_MIXED = 1  /* float state and fluxes; double geometry moments for CVs with
                   volume fraction below 1e-3 and double redistribution weights;
                   compensated sums in the neighbourhood averages               */
} eb_precision;

typedef enum { EB_GRID_C = 0, EB_GRID_U = 1, EB_GRID_V = 2, EB_GRID_W = 3 } eb_grid;

typedef enum { EB_RHO = 0, EB_RHOTHETA = 1, EB_RHOU = 2, EB_RHOV = 3, EB_RHOW = 4 } eb_field;

typedef struct {
  int nx, ny, nz;        /* cells, each >= 4; nx*ny*(nz+1) < 2^32                 */
  double Lx, Ly, Lz;     /* domain lengths, > 0                                    */
  double v_target_frac;  /* small-cell threshold V_target / (dx dy dz); the paper
                            uses 1/2 (Sec. 5.1).  Must lie in (0, 1].            */
} eb_desc;

typedef struct eb_geom_s *eb_geom; /* opaque; owns all device geometry and tables */

typedef struct {
  void *rho, *rhotheta, *rhou, *rhov, *rhow; /* caller-owned device arrays */
} eb_state;

/* Geometry exported by eb_geom_export, one dense double array of
 * nx*ny*nz_g values (nz_g = nz+1 on the w grid).  Lengths are in cell units,
 * offsets are relative to the CV (or face) centre; faces are the LOW face of
 * each CV in the named direction. */
typedef enum {
  EB_X_ALPHA = 0,                                       /* volume fraction         */
  EB_X_CENT_X = 1, EB_X_CENT_Y = 2, EB_X_CENT_Z = 3,    /* volume centroid offset  */
  EB_X_BETA_X = 4, EB_X_BETA_Y = 5, EB_X_BETA_Z = 6,    /* face area fractions     */
  EB_X_FCENT_X1 = 7, EB_X_FCENT_X2 = 8,                 /* x face centroid (y, z)  */
  EB_X_FCENT_Y1 = 9, EB_X_FCENT_Y2 = 10,                /* y face centroid (x, z)  */
  EB_X_FCENT_Z1 = 11, EB_X_FCENT_Z2 = 12,               /* z face centroid (x, y)  */
  EB_X_AEB = 13,                                        /* EB area / (dx dy)       */
  EB_X_NRM_X = 14, EB_X_NRM_Y = 15, EB_X_NRM_Z = 16,    /* unit EB normal, into fluid */
  EB_X_EBC_X = 17, EB_X_EBC_Y = 18, EB_X_EBC_Z = 19,    /* EB centroid offset      */
  EB_X_FLAG = 20,        /* 0 covered, 1 regular, 2 cut (nodal level-set test)    */
  EB_X_CODE = 21,        /* merging-neighbourhood code, 0 = not a small CV        */
  EB_X_NNB = 22,         /* N: number of neighbourhoods holding the CV            */
  EB_X_KAPPA = 23, EB_X_OMEGA = 24, EB_X_VHAT = 25,
  EB_X_XHAT_X = 26, EB_X_XHAT_Y = 27, EB_X_XHAT_Z = 28,
  EB_X_COUNT = 29
} eb_export_field;

/*
 * Neighbourhood code (EB_X_CODE) of a small CV (Sec. 5.1: merge first along
 * the EB normal, then the next-largest normal component, then to 2x2x2):
 *   axes a1, a2, a3 ordered by decreasing |n_d| of the unit EB normal, two
 *   components counting as equal when they differ by at most 1e-12, ties
 *   broken x before y before z; permutation index p over
 *   (xyz, xzy, yxz, yzx, zxy, zyx); sign bits b_d = 1 where n_d < -1e-12;
 *   growth level L = 1 (two CVs), 2 (2x2), 3 (2x2x2);
 *   code = 1 + (8 p + b_x + 2 b_y + 4 b_z) * 3 + (L - 1).
 */

/* Sizes of what a geometry handle built. */
typedef struct {
  int64_t cells;            /* nx*ny*nz                                      */
  int64_t cvs[4];           /* non-covered CVs per grid                       */
  int64_t band_records[4];  /* CVs stored with explicit geometry per grid     */
  int64_t small_cvs[4];     /* CVs with volume fraction below the threshold   */
  int64_t affected_cvs[4];  /* CVs the redistribution writes                  */
  int64_t band_cvs[4];      /* CVs updated by the general (near-EB) kernel    */
  int64_t band_faces[4];    /* near-EB faces whose provisional flux is staged */
  int64_t tiny_cvs[4];      /* cut CVs with volume fraction below 1e-3        */
  int64_t fast_cells;       /* base cells updated by the geometry-free kernel  */
  double min_alpha;         /* smallest positive volume fraction, any grid    */
  int64_t device_bytes;     /* device memory held by the handle               */
  int64_t slab_levels;      /* slab height of the bulk kernel's tiles in use
                               (0 = automatic)                                */
  int64_t bulk_high_priority; /* 1: the bulk kernel runs on a stream of the
                               highest priority beside the near-EB kernels    */
  int64_t wsrd_beside_bulk; /* 1: every CV the redistribution reads or writes
                               is a near-EB CV, so eb_step runs it right after
                               the near-EB kernels, beside the bulk kernel
                               (ensembles keep it after the bulk kernel)      */
  int64_t tile_rows;        /* rows of the bulk kernel's tiles (16, or 14)    */
} eb_geom_info_t;

/*
 * Build the geometry of all four grids and the redistribution tables
 * (Sec. 3.2: nodal level set, cut faces, cut cells, staggered CVs from two
 * half-cells; Sec. 5.1: merging neighbourhoods, kappa, omega, weighted
 * volume and centroid, all fixed at set-up).
 *   desc         grid and threshold, read during the call.
 *   h_nodes      device, (nx+1)*(ny+1) doubles, node (i, j) at i + (nx+1) j,
 *                heights at x = i Lx/nx, y = j Ly/ny; the last row and column
 *                must repeat the first (periodicity).
 *   prec         precision of every later state argument.
 *   ref_rho, ref_rhotheta
 *                device, nz doubles each, or both NULL: a reference profile
 *                at cell-centre levels; rho and rho*theta states then hold
 *                values minus ref[k].  Copied during the call.
 *   out          receives the handle; destroy it with eb_geom_destroy.
 * Synchronises the stream (sizes are read back).  EB_ERR_OOM when the device
 * has no room; nothing is leaked on failure.
 */
eb_status eb_geom_build(const eb_desc *desc, const double *h_nodes, eb_precision prec, const double *ref_rho,
                        const double *ref_rhotheta, void *stream, eb_geom *out);

/*
 * Two-level static refinement (Sec. 4.3), refinement ratio 2 in every
 * direction over the same domain.
 *
 * eb_geom_build_coarse: a handle of the coarse level (nx/2 x ny/2 x nz/2
 * cells, the fine handle's lengths, small-cell threshold and precision)
 * whose geometry is merged from the fine handle's cells, so that coarse
 * volumes, face areas and EB areas are sums of fine ones.  A coarse CV of
 * any grid is a block of 2x2x2 fine c-grid cells (cells 2I, 2I+1 along x for
 * the c grid, 2I-1, 2I for u: the right half of coarse cell I-1 and the left
 * half of cell I; likewise along y for v and z for w; fine cells outside the
 * domain hold no fluid).  Volume fraction: the mean of the 8; face fraction:
 * the mean of the 4 fine faces on the coarse face; EB area: the sum; volume,
 * face and EB centroids: weighted mean positions; EB normal: the direction of
 * sum_d (open area of the high d-face - of the low d-face) e_d; class:
 * covered / regular when all fine cells inside the domain are, else cut.  The
 * redistribution tables, lists and everything else then follow from that
 * geometry as in eb_geom_build, and the handle takes every call a handle
 * built from heights takes.
 *   fine              a handle with even nx, ny, nz (nx/2 etc. must pass the
 *                     eb_geom_build checks); it is only read, and may be
 *                     destroyed afterwards.
 *   ref_rho, ref_rhotheta  device, nz/2 doubles each, or both NULL: the coarse
 *                     level's reference profiles, as for eb_geom_build.
 * The coarse handle's nodal heights (eb_geom_export's wall values) are every
 * other fine node.  EB_ERR_INVALID_ARG for odd dimensions or another current
 * device; the eb_geom_build errors otherwise.
 *
 * eb_restrict: a fine state restricted to the coarse level: every coarse
 * cell-centred value is the mean of its 8 fine cells weighted by their volume
 * fractions (the coarse cell holds the fine cells' total), every coarse face
 * value the mean of the 4 fine values on its face weighted by their area
 * fractions (the flux integral over the coarse face is kept).  Sums in
 * double.  States hold values minus each handle's own per-level profiles,
 * which both calls account for.  Coarse CVs whose fine parts hold no fluid
 * (or no open area) keep the value Uc has.
 *
 * eb_prolong: the boundary values a refined patch takes from the coarse level
 * (Sec. 4.3): every fine CV outside the fine handle's columns [lo, hi) takes
 * the value of the coarse CV it lies in; a fine face of a face grid on a
 * coarse face takes that face's value, one halfway between two coarse faces
 * (odd fine index along the face's axis) the mean of the two.  Covered CVs
 * included (the step passes them through).
 *
 * For both: the fine handle is the coarse handle's fine level over all of y
 * and z and an x-window of it: fine column q of the handle is global fine
 * column fine_x0 + q (mod 2 nx_c); the whole level is fine_x0 = 0,
 * nx = 2 nx_c (e.g. the handle eb_geom_build_coarse was built from).
 *   lo, hi            local fine columns: eb_restrict restricts the coarse
 *                     columns over [lo, hi) (lo, hi and fine_x0 even),
 *                     eb_prolong fills every column outside [lo, hi).
 *   Uf, Uc            device states of the fine and the coarse handle.
 * Asynchronous on stream.  EB_ERR_INVALID_ARG on handles that are not two
 * levels of one grid (ny, nz halved, cells twice as large, nx_f <= 2 nx_c,
 * same precision), on a bad column range, or NULL / misaligned pointers.
 */
eb_status eb_geom_build_coarse(eb_geom fine, const double *ref_rho, const double *ref_rhotheta, void *stream,
                               eb_geom *out);
eb_status eb_restrict(eb_geom fine, eb_geom coarse, const eb_state *Uf, eb_state *Uc, int fine_x0, int lo, int hi,
                      void *stream);
eb_status eb_prolong(eb_geom coarse, const eb_state *Uc, eb_geom fine, eb_state *Uf, int fine_x0, int lo, int hi,
                     void *stream);

/*
 * Background momentum profile of the state (Sec. 2: the reference /
 * perturbation split of the governing equations, carried over to the
 * horizontal momenta of a prescribed background wind).  After this call the
 * rho*u and rho*v arguments of eb_flux_div, eb_wsrd, eb_wsrd_noalloc,
 * eb_step, eb_step_profile, eb_geom_tune and the eb_ensemble_* calls hold
 * values minus ref_rhou[k] (ref_rhov[k]) at cell-centre level k, as rho and
 * rho*theta do for ref_rho and ref_rhotheta.  The method is unchanged: every
 * flux is formed from the full values, and a profile changes only how the
 * stored numbers round (on the mixed path the float state then carries the
 * wind's deviation from the profile, not the wind itself).  dU of
 * eb_flux_div is the full derivative, with or without a profile.
 *   ref_rhou, ref_rhov  device, nz doubles each, finite; NULL means zero.
 *                       Copied during the call (the stream is synchronised
 *                       and the device drained first).
 * A profile needs the handle's reference density (eb_geom_build with
 * ref_rho; EB_ERR_STATE otherwise): the bulk kernel advects the deviations
 * of u and v from u_bg = ref_rhou / rho0 and v_bg = ref_rhov / rho0, as it
 * advects theta - theta0 (Sec. 4.1 face values of a constant are the
 * constant, so this changes rounding only).
 * The anelastic calls (eb_project, eb_anelastic_step, eb_project_sample,
 * eb_project_warm) need full momenta and return EB_ERR_STATE on a handle
 * with a nonzero profile.  Setting both to NULL (or zeros) restores full
 * values.
 */
eb_status eb_geom_set_wind_reference(eb_geom geom, const double *ref_rhou, const double *ref_rhov, void *stream);

/*
 * Sources of the compressible system (Sec. 2.1, Eq. mom-comp) that eb_step
 * adds to the flux divergence of every stage, before the redistribution:
 *   EB_SOURCE_PRESSURE  -grad p' on rho*u, rho*v, rho*w: p' = p - p0(z), p from
 *                       the equation of state p = P00 (R rho theta / P00)^gamma
 *                       and p0 from the reference rho0 theta0 of each level;
 *   EB_SOURCE_BUOYANCY  B = -rho' g on rho*w.
 * Pressure and density live at cell centres: the source of a momentum CV is
 * -(p'_b - p'_a) / dx_d across its two cells a (one step back along its
 * staggering axis d) and b (same index), on w also -g (rho'_a + rho'_b) / 2;
 * a covered cell takes the other cell's value.  Constants: P00 = 1e5 Pa (the
 * paper's), R = 287 J/(kg K), cp = 1004.5 J/(kg K), gamma = cp / (cp - R),
 * g = 9.81 m/s^2 (EB_P00, EB_RD, EB_CP, EB_GRAV).  The time step must then
 * resolve sound waves: eb_step does not check it.
 *   flags  a combination of EB_SOURCE_*; 0 switches them off (default).
 * Needs the handle's reference profiles (eb_geom_build with ref_rho and
 * ref_rhotheta): EB_ERR_STATE otherwise.  eb_flux_div, eb_wsrd and
 * eb_step_profile never add sources; the anelastic calls and
 * eb_ensemble_create return EB_ERR_STATE on a handle with sources;
 * EB_ERR_INVALID_ARG for other flag bits.
 */
#define EB_SOURCE_PRESSURE 1
#define EB_SOURCE_BUOYANCY 2
#define EB_P00 1.0e5
#define EB_RD 287.0
#define EB_CP 1004.5
#define EB_GRAV 9.81
eb_status eb_geom_set_sources(eb_geom geom, int flags);

/* Free everything the handle owns (synchronises the device).  NULL is OK. */
eb_status eb_geom_destroy(eb_geom geom);

/* Sizes and counts of the handle. */
eb_status eb_geom_info(eb_geom geom, eb_geom_info_t *info);

/* Write one geometry or redistribution field of one grid as a dense double
 * array of nx*ny*nz_g values into dst (device). */
eb_status eb_geom_export(eb_geom geom, eb_grid grid, eb_export_field field, double *dst, void *stream);

/*
 * Flux divergence of Eqs. update-cc / update-fc for every field:
 *   dU = -(1/alpha) [ sum_d (beta_+ F_+ - beta_- F_-) / delta_d ]
 * with third-order upwind face values (second-order centred where the far
 * upstream CV is covered or beyond a wall), fluxes interpolated to cut-face
 * centroids, zero flux through the EB and the walls (Sec. 4.1).  dU is zero
 * on covered CVs and on the wall levels of rho*w.  U and dU must not overlap.
 */
eb_status eb_flux_div(eb_geom geom, const eb_state *U, eb_state *dU, void *stream);

/*
 * Weighted state redistribution of one field (Sec. 5.1, Eqs. qhat_omega,
 * qrecon, final_update_omega): Unew = R[Uhat] on the field's grid.  CVs that
 * redistribution does not touch are copied.  Uhat and Unew may be the same
 * array (in-place) or must not overlap.
 */
eb_status eb_wsrd(eb_geom geom, eb_field field, const void *Uhat, void *Unew, void *stream);

/*
 * Maximum scratch, in bytes, that eb_wsrd_noalloc may use per call.
 */
#define EB_WSRD_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * eb_wsrd without device memory of its own: the same redistribution, same
 * arguments and the same results as eb_wsrd.  The paper has no counterpart;
 * this is a deployment variant.
 *
 * Who needs it: callers that may not allocate device memory at the moment
 * they redistribute -- a host loop that runs under a fixed memory budget
 * shared with other libraries, a caller that has handed all free memory to a
 * pool allocator, or one that must not synchronise the device (cudaMalloc and
 * cudaFree may).  eb_wsrd itself allocates nothing per call either, but its
 * per-small-CV scratch lives in the handle; this variant keeps that scratch in
 * one fixed block of EB_WSRD_NOALLOC_SCRATCH_BYTES bytes compiled into the
 * library (a static __device__ array), so the handle's scratch is not touched.
 *
 * Scratch needed for a field: 5 values of the handle's precision per small CV
 * of the field's grid (eb_geom_info_t.small_cvs), each of three parts rounded
 * up to 256 bytes.  A larger need is rejected with EB_ERR_INVALID_ARG and a
 * message giving both sizes; nothing is launched then.  Nothing in the
 * scratch needs to start at zero: every entry is written before it is read
 * within one call.
 *
 * Set-up: the first call on each device looks up the block's device address
 * (cudaGetSymbolAddress, which may load the library's device code) with the
 * handle's device current.  That first call therefore belongs before any
 * stream capture and outside any section that must not touch the driver;
 * later calls only launch kernels (and one device-to-device copy when Uhat
 * and Unew differ).  The address is cached per device and per CUDA context:
 * after the device's context is destroyed and created again (cudaDeviceReset)
 * the next call looks it up again, and is then a first call in the sense
 * above.  Handles themselves do not survive a device reset.  The current
 * device must be the handle's device (EB_ERR_INVALID_ARG otherwise).
 *
 * Races: there is ONE scratch block per device, shared by every handle and
 * every thread.  Two calls whose work may overlap on the device (different
 * streams without an ordering event, or calls from several host threads)
 * corrupt each other's results.  Serialise them on one stream.
 */
eb_status eb_wsrd_noalloc(eb_geom geom, eb_field field, const void *Uhat, void *Unew, void *stream);

/*
 * nsteps steps of Algorithm 1 with zero source.  stages = 1: forward Euler,
 * U^{n+1} = R[U^n + dt dU(U^n)] (Eq. basic_fv_srd); stages = 3: the
 * three-stage Runge-Kutta of Sec. 5.2 with redistribution after every stage,
 * U1 = R[U + dt/3 dU(U)], U2 = R[U + dt/2 dU(U1)], U' = R[U + dt dU(U2)].
 * Un is read only; the result lands in Unp1 (which must not overlap Un);
 * intermediate states use handle-owned scratch.  Covered CVs and the rho*w
 * wall levels of Unp1 receive Un's values.
 */
eb_status eb_step(eb_geom geom, const eb_state *Un, eb_state *Unp1, double dt, int nsteps, int stages, void *stream);

/*
 * One forward-Euler step exactly like eb_step(nsteps = 1, stages = 1), with
 * CUDA events recorded on the stream between its phases.  On return (the
 * stream is synchronised) ms[0] holds the geometry-free bulk flux/update
 * kernel, ms[1] the near-EB flux/update kernels, ms[2] the redistribution
 * passes of all five fields and ms[3] the three together, in milliseconds
 * (the pass-through of covered CVs runs before the first event).  The
 * phases run one after another here, while eb_step overlaps the first two.
 * Used by benchmarks to time the dominant kernel on its own stream.
 */
eb_status eb_step_profile(eb_geom geom, const eb_state *Un, eb_state *Unp1, double dt, void *stream, float ms[4]);

/*
 * Anelastic projection (Sec. 2.2 anelastic model; Algorithm 2 step 5): the
 * face momenta m = (rho*u, rho*v, rho*w) of U are made discretely
 * divergence-free, in place.  The divergence is the cut-cell one of the flux
 * update, D(m)_c = sum_d (beta_hi m_hi - beta_lo m_lo) / delta_d (walls and
 * closed faces carry none); the gradient on a face is
 * G(phi) = (phi_R - phi_L) / delta_d; m <- m - dt G(phi) with
 * L phi = D(G(phi)) = D(m) / dt.  L is symmetric with the constants as null
 * space, so the mean of D(m) (rounding) is removed and -L phi = -D(m)/dt is
 * solved in FP64 by Jacobi-preconditioned conjugate gradients until
 * ||rhs - L phi|| <= rtol ||rhs|| or maxit iterations.
 *   phi0     device, nx*ny*nz doubles: initial guess, or NULL for zero.
 *   phi      device, nx*ny*nz doubles: receives the solution, or NULL.
 *   iters    host: iterations used (NULL allowed).
 *   relres   host: final relative residual (NULL allowed).
 * rho and rho*theta are not touched.  Synchronises the stream every 32
 * iterations (convergence test).  The first call on a handle allocates its
 * work space (about 10 doubles per cell), so it must not be inside a stream
 * capture.
 */
eb_status eb_project(eb_geom geom, eb_state *U, double dt, double rtol, int maxit, const double *phi0, double *phi,
                     int *iters, double *relres, void *stream);

/* Preconditioner of the projection's conjugate gradients (eb_project and
 * eb_anelastic_step) for this handle.  Sec. 2.2 leaves the Poisson solver
 * open; both choices converge to the same projection.
 *   EB_PRECOND_JACOBI (default): z = r / diag(-L).
 *   EB_PRECOND_MG: one symmetric multigrid V-cycle in FP32 (the outer
 *     conjugate gradients, residuals and dot products stay FP64).  The cell grid
 *     is coarsened by 2 in every direction while all three sizes are even
 *     and at least 4, until the grid has 512 cells or fewer; a coarse face
 *     takes the mean open fraction of the four fine faces it covers and the
 *     coarse spacing; damped Jacobi sweeps (weight 0.9) before and after
 *     the coarse correction, three of each on the finest grid and two on the
 *     coarser ones; averaging restriction, injection prolongation,
 *     16 Jacobi sweeps on the coarsest grid.  Fewer iterations, each more
 *     costly; the extra device memory is about three FP64 fields.
 * Errors: EB_ERR_INVALID_ARG for another kind, or for EB_PRECOND_MG when the
 * grid cannot be coarsened at least once to a coarsest grid of at most 32768
 * cells.  The hierarchy is built on the first projection that uses it. */
typedef enum { EB_PRECOND_JACOBI = 0, EB_PRECOND_MG = 1 } eb_precond;
eb_status eb_project_set_preconditioner(eb_geom geom, int kind);

/*
 * nsteps anelastic steps (Algorithm 2) with two stages in the low-storage
 * form U* = P[R[U + dt/2 dU(U)]], U' = P[R[U + dt dU(U*)]]: the flux update
 * and redistribution of eb_step with the density held at the reference
 * profile (the rho perturbation is set to zero after each stage), then the
 * projection P above (zero initial guess).  The handle must have been built
 * with a reference profile (EB_ERR_STATE otherwise); Un holds rho*theta and
 * the face momenta rho0*u with a zero rho perturbation.  iters (host, NULL
 * allowed) receives 2*nsteps iteration counts.  Uses handle scratch; Un and
 * Unp1 must not overlap.
 */
eb_status eb_anelastic_step(eb_geom geom, const eb_state *Un, eb_state *Unp1, double dt, int nsteps, double rtol,
                            int maxit, int *iters, void *stream);

/*
 * Warm-start network of the anelastic projection (the paper has no
 * counterpart; it solves from the previous pressure or zero).  A three-level
 * 3D U-Net: channels 16 / 32 / 64, two 3x3x3 convolutions with zero padding
 * and ReLU per level, 2x2x2 average pooling down, 2x nearest upsampling up,
 * skips concatenated after the upsampled channels, a 1x1 output head.
 * Input: 2 channels (the projection's right-hand side over its RMS, and the
 * c-cell volume fraction); output: 1 channel, trained to the mean-free
 * solution over (RMS * dx^2 * scale).  BF16 weights (copied from FP32 master
 * weights), FP32 activations and accumulation.  Parameters are one flat FP32
 * vector: per layer, weights [cout][cin][k][k][k] then biases [cout].
 * Tensors are device arrays [channels][nz][ny][nx]; a network object is
 * sized for one grid (nx, ny, nz multiples of 4).  Calls on one network
 * must be serialised.
 */
typedef struct eb_unet_s *eb_unet;

/* Number of parameters (353,713). */
int64_t eb_unet_num_params(void);

/* Activation buffers for an nx x ny x nz grid; parameters start at zero. */
eb_status eb_unet_create(int nx, int ny, int nz, eb_unet *out);

/* Copy n = eb_unet_num_params() FP32 parameters from / to host memory
 * (set also resets the optimiser state). Synchronous. */
eb_status eb_unet_set_params(eb_unet net, const float *host, int64_t n);
eb_status eb_unet_get_params(eb_unet net, float *host, int64_t n);

/* out (nx*ny*nz floats) = network(in (2*nx*ny*nz floats)). */
eb_status eb_unet_forward(eb_unet net, const float *in, float *out, void *stream);

/* Masked loss 0.5 sum(mask (y - target)^2) / sum(mask > 0) and its
 * gradient with respect to every parameter.  mask: 0 / 1 floats selecting at
 * least one voxel.  loss (host, NULL allowed) and grad_host (host,
 * eb_unet_num_params() floats, NULL allowed) are filled when given (the
 * stream is then synchronised). */
eb_status eb_unet_gradient(eb_unet net, const float *in, const float *target, const float *mask, float *loss,
                           float *grad_host, void *stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on that
 * gradient; loss (host, NULL allowed) as above. */
eb_status eb_unet_train_step(eb_unet net, const float *in, const float *target, const float *mask, float lr,
                             float *loss, void *stream);

/* Waits for the device, then frees the network. */
eb_status eb_unet_destroy(eb_unet net);

/* Waits for the device; EB_ERR_TIMEOUT when a convolution's bounded wait
 * for its tensor-core products (about one second) expired since the last
 * check (eb_unet_gradient with a loss or gradient requested and
 * eb_unet_get_params check too), EB_OK otherwise.  The flag is cleared. */
eb_status eb_unet_sync_status(eb_unet net);

/* Failure test of the bounded waits (no counterpart in the paper): the next
 * convolution launch of this network issues its first products without
 * signalling their completion, so every CTA's wait runs out (about one
 * second, twice), the CTAs release their tensor memory and return, the
 * launch's output is left unwritten, and the next eb_unet_sync_status
 * reports EB_ERR_TIMEOUT.  Later launches are normal. */
eb_status eb_unet_inject_wait_fault(eb_unet net);

/* A training sample for the network from the face momenta of U (not
 * modified): in (2*N floats) = [rhs / rms, alpha] with rhs the projection's
 * mean-free right-hand side and rms its RMS over the cells in the solve;
 * target (N floats) = the mean-free solution of eb_project (zero start, rtol,
 * maxit) over (rms * dx^2 * scale); mask (N floats) = 1 on the cells in the
 * solve.  iters (host, NULL allowed): solver iterations.  EB_ERR_STATE when
 * the momenta are already divergence-free. */
eb_status eb_project_sample(eb_geom geom, const eb_state *U, double dt, double rtol, int maxit, double scale,
                            float *in, float *target, float *mask, int *iters, void *stream);

/* eb_project with the network's initial guess: phi0 = output * rms * dx^2 *
 * scale on the cells in the solve (net created for the handle's grid, scale
 * as in training).  The solve, its stopping rule and the correction are those
 * of eb_project, so the converged result is the same to the tolerance. */
eb_status eb_project_warm(eb_geom geom, eb_unet net, eb_state *U, double dt, double rtol, int maxit, double scale,
                          int *iters, double *relres, void *stream);

/*
 * Ensembles: many independent terrain instances advanced together.  The
 * paper has no counterpart (its AMReX box arrays are the closest); this is
 * the batched serving form of eb_step.
 *
 * An ensemble refers to member handles of any sizes, all of one precision
 * and on the current device; it does not own them (destroy the ensemble
 * first).  It owns two state buffers per member.  Every step of every member
 * is forward Euler (Eq. basic_fv_srd), exactly as eb_step(nsteps = 1,
 * stages = 1) computes it, bit for bit, in either of two schedules:
 *   EB_ENSEMBLE_PERSISTENT (the default): one step of the whole ensemble is
 *     ONE cooperative launch of a persistent kernel with as many CTAs as the
 *     device holds at once; they take the bulk kernel's work units of all
 *     members (longest first), then the near-EB fluxes and updates and the
 *     redistribution of all members, phase after phase, with grid-wide
 *     barriers between the phases.  A barrier wait is bounded (about a
 *     second): if a CTA never arrives, the others latch EB_DEV_TIMEOUT into
 *     every member's status word (eb_sync_status of any member reports it)
 *     and return; the step's results are then undefined.
 *   EB_ENSEMBLE_BRANCHES: each member's own kernels on a branch of their
 *     own, so that the kernels of different members run side by side.
 * Either step is captured once per step direction as a CUDA graph;
 * eb_ensemble_step replays it.  eb_ensemble_tune times both and keeps the
 * faster.  Calls on one ensemble, and on its members' handles, must be
 * serialised.  EB_ERR_STATE from eb_ensemble_create when the device cannot
 * hold one CTA of the persistent kernel.
 */
typedef struct eb_ensemble_s *eb_ensemble;

/* Schedules of an ensemble step (eb_ensemble_set_schedule). */
#define EB_ENSEMBLE_PERSISTENT 0 /* one cooperative launch of the persistent kernel per step */
#define EB_ENSEMBLE_BRANCHES 1   /* each member's kernels on a branch of their own */

/* members: n handles (copied).  Allocates the state buffers. */
eb_status eb_ensemble_create(const eb_geom *members, int n, eb_ensemble *out);

/* Load member's state from U (device arrays of that member's sizes; copied
 * on the stream).  Also fills the covered CVs of the second buffer. */
eb_status eb_ensemble_set_state(eb_ensemble e, int member, const eb_state *U, void *stream);

/* Copy member's current state into U (device arrays). */
eb_status eb_ensemble_get_state(eb_ensemble e, int member, eb_state *U, void *stream);

/* Advance every member nsteps steps; dt: host array of one time step per
 * member.  The graph is captured on the first call and again whenever dt
 * changes; capture may not already be active on the stream. */
eb_status eb_ensemble_step(eb_ensemble e, const double *dt, int nsteps, void *stream);

/* Autotuner: times 2 * reps ensemble steps for each candidate slab height
 * of the bulk kernel's tiles (automatic, 8 .. 64 levels, whole column; it
 * sets the size of the bulk work units) with the persistent schedule and
 * with the branches schedule (every member's bulk kernel at the same and at
 * a higher stream priority, eb_geom_set_bulk_priority), and keeps the
 * fastest combination; *slab_levels (if not NULL) receives the height (0 =
 * automatic).  Results depend on none of them.  The loaded states are
 * restored afterwards.  Synchronises the stream; allocates a temporary copy
 * of the states. */
eb_status eb_ensemble_tune(eb_ensemble e, const double *dt, int reps, int *slab_levels, void *stream);

/* Sets the schedule (EB_ENSEMBLE_PERSISTENT or EB_ENSEMBLE_BRANCHES) of
 * later steps; the next step captures its graphs again. */
eb_status eb_ensemble_set_schedule(eb_ensemble e, int schedule);

/* Launch figures (host array of 6): CTAs of the persistent kernel (all
 * resident at once), its bulk work units for the current split (0 before
 * the first step), its registers per thread, static shared and local
 * (spill) bytes per thread, and the schedule in use. */
eb_status eb_ensemble_info(eb_ensemble e, int out[6]);

/* Failure test of the bounded barrier (no counterpart in the paper): with
 * cta >= 0, CTA `cta` of every later step leaves before the first barrier,
 * so the other CTAs' waits expire and EB_DEV_TIMEOUT latches (the states are
 * then undefined: load them again); cta = -1 restores normal steps.  Waits
 * for the device.  No device fault is involved: the kernel only counts. */
eb_status eb_ensemble_inject_barrier_fault(eb_ensemble e, int cta);

/* Waits for the device, then frees the ensemble's buffers. */
eb_status eb_ensemble_destroy(eb_ensemble e);

/* Autotuner of one handle: times reps steps of eb_step(nsteps = 1,
 * stages = 1) from U (read only; the results go to a temporary state) for each
 * candidate slab height of the bulk kernel's tiles (automatic, 12 .. 64
 * levels, whole column), each with the bulk kernel at the same and at a
 * higher stream priority than the near-EB kernels (eb_geom_set_bulk_priority)
 * and, on the mixed path, with tiles of 16 and of 14 rows
 * (eb_geom_set_tile_rows), and keeps the fastest combination; *slab_levels
 * (NULL allowed) receives the height (0 = automatic), eb_geom_info the rest.  Results of later steps do not
 * depend on either.  Synchronises the stream; allocates and frees the
 * temporary state. */
eb_status eb_geom_tune(eb_geom geom, const eb_state *U, double dt, int reps, int *slab_levels, void *stream);

/* Stream priority of the bulk kernel within a step (scheduling only: results
 * do not depend on it).  high = 0: the bulk kernel runs on the caller's stream
 * and the near-EB kernels on the handle's side stream, at the same priority.
 * high = 1: the bulk kernel runs on a handle stream of the highest priority,
 * so that its CTAs take their SMs before the near-EB kernels' blocks; this
 * pays where the near-EB work is large (rough terrain).  Default 0;
 * eb_geom_tune chooses.  An ensemble that has already captured its step
 * graph keeps the schedule it captured until it is tuned again.
 * EB_ERR_INVALID_ARG for another value. */
eb_status eb_geom_set_bulk_priority(eb_geom geom, int high);

/* Sets the bulk kernel's slab height directly (0 = automatic; heights above
 * nz mean whole columns), e.g. to re-apply a height eb_geom_tune chose
 * earlier.  Waits for the device to be idle (the old plan may be in use). */
eb_status eb_geom_set_slab_levels(eb_geom geom, int slab_levels);

/* Rows of the bulk kernel's tiles of 32 columns: 16 (default) or, on the
 * mixed path, 14 (a 256-row domain then cuts into 19 tile rows, and two slabs
 * of its 152 tiles fill every SM with two CTAs).  Scheduling only: every
 * cell's arithmetic is the same.  eb_geom_tune tries both on the mixed path;
 * ensembles keep 16 for their members.  Waits for the device to be idle.
 * EB_ERR_INVALID_ARG for other values, or 14 on an FP64 handle. */
eb_status eb_geom_set_tile_rows(eb_geom geom, int rows);

/* Synchronise the stream, then return (and clear) the first device-side
 * error latched since the last call: EB_ERR_NUMERIC or EB_ERR_TIMEOUT. */
eb_status eb_sync_status(eb_geom geom, void *stream);

/* Thread-local message of the calling thread's last error ("" if none). */
const char *eb_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int eb_version(void);

/*
 * Benchmark instrument (no counterpart in the paper): the measured rate of
 * independent fused multiply-adds on the current device, the denominator of
 * the arithmetic roofline of a kernel bound by one arithmetic type.
 *   kind    0 FP64 (DFMA), 1 FP32 (FFMA), 2 packed FP32x2 (FFMA2)
 *   gflops  host; receives the best of three timed launches (after one
 *           untimed), an FMA counted as two flops (four for FFMA2)
 * Allocates a small device buffer, launches on the stream and synchronises
 * it.  EB_ERR_INVALID_ARG for another kind.
 */
eb_status eb_fma_peak(int kind, double *gflops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* EB_H */
