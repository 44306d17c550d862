/*
 * gff.h - C ABI of the GB300 Galerkin-FFT crystal-plasticity solver (libgff.so).
 *
 * The library solves, increment by increment, the periodic equilibrium of an
 * RVE voxel grid with the variational (Galerkin) FFT method of Lucarini &
 * Segurado, "On the accuracy of spectral solvers for micromechanics based
 * fatigue modeling" (arXiv:1806.10599):
 *   find F(x) = Fbar + F~(x) with  G(P(F, alpha)) = 0            (Eqs. linear_momentum, eql_discrete2)
 * by Newton-Raphson (Eqs. F_dif, P_dif) whose linear systems
 *   G(K : dF) = -G(P)                                            (Eqs. linequil, linequil2, newlinop)
 * are solved matrix-free by conjugate gradients (Sect. 2.1), with the
 * continuous projection G^ (Eq. G) or the discrete one G^' (Sect. 2.2), and
 * accumulates the fatigue indicator parameters of Sect. 3.3.
 *
 * Conventions (all entry points):
 *  - Every call returns a gff_status; GFF_OK is 0, errors are negative.  On
 *    error, gff_last_error(h) returns a message (valid until the next call on h).
 *  - The caller owns every pointer it passes.  Pointers are HOST pointers
 *    unless the parameter name ends in _dev, in which case they are device
 *    pointers on the GPU current at gff_create, valid on the handle's stream.
 *    No memory allocated by the library is returned to the caller.
 *  - Tensors are 3x3 row-major: component c = 3*i + j.  Voxel fields are
 *    structure-of-arrays [9][nz][ny][nx] (x fastest), N = nx*ny*nz.
 *  - A handle is one RVE; calls on one handle must not run concurrently.
 *  - Units are SI (Pa, s); lengths are those of gff_grid.L.
 *  - The GPU path requires nx, ny, nz even, between 4 and 128, with no prime
 *    factor other than 2, 3 and 5; other sizes give GFF_ERR_ARG.
 */
#ifndef GFF_H
#define GFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gff_handle gff_handle;

typedef enum {
    GFF_OK = 0,
    GFF_ERR_ARG = -1,            /* invalid argument or unsupported size            */
    GFF_ERR_OOM = -2,            /* device allocation failed                        */
    GFF_ERR_CUDA = -3,           /* CUDA runtime error (message has the detail)     */
    GFF_ERR_NO_CONVERGENCE = -4, /* Newton or CG reached its iteration cap          */
    GFF_ERR_CP_FAIL = -5,        /* crystal-plasticity local Newton failed          */
    GFF_ERR_TIMEOUT = -6,        /* a bounded device wait gave up                   */
    GFF_ERR_STATE = -7,          /* call out of order (e.g. no microstructure yet)  */
    GFF_ERR_IO = -8              /* file read/write failed                          */
} gff_status;

enum { GFF_PROJ_CONTINUOUS = 0, GFF_PROJ_DISCRETE = 1 };
enum { GFF_PREC_FP64 = 0, GFF_PREC_MIXED = 1 };
enum { GFF_WARM_OFF = 0, GFF_WARM_NET_IF_BETTER = 1, GFF_WARM_NET = 2, GFF_WARM_EXTRAPOLATE = 3 };
/* GFF_MAT_NEOHOOKE: compressible neo-Hookean solid (E, nu as Lame constants),
 * evaluated the way an FE user material is: Cauchy stress and Jaumann-rate
 * tangent per voxel, converted to P and dP/dF by the formulas of Appendix A
 * (gff_umat_tangent). */
enum { GFF_MAT_SVK_CUBIC = 0, GFF_MAT_SVK_ISO = 1, GFF_MAT_CP_FCC = 2, GFF_MAT_NEOHOOKE = 3 };
enum {
    GFF_FIELD_F = 0,      /* deformation gradient, 9 per voxel          */
    GFF_FIELD_P = 1,      /* first Piola-Kirchhoff stress, 9 per voxel  */
    GFF_FIELD_K = 2,      /* tangent dP/dF, 81 per voxel [81][N], index 9*c + d */
    GFF_FIELD_FP_INV = 3, /* inverse plastic deformation gradient, 9    */
    GFF_FIELD_CHI = 4,    /* backstress per slip system, 12             */
    GFF_FIELD_GAMMA = 5,  /* cumulative signed slip per system, 12      */
    GFF_FIELD_PCYC = 6,   /* accumulated plastic strain in the cycle, 1 */
    GFF_FIELD_WCYC = 7    /* dissipated energy per system in the cycle, 12 */
};

typedef struct {
    int nx, ny, nz;
    double L[3]; /* box lengths along x, y, z */
} gff_grid;

typedef struct {
    int kind;                /* GFF_MAT_*                                            */
    double C11, C12, C44;    /* cubic constants (SVK_CUBIC, CP_FCC), Pa             */
    double E, nu;            /* isotropic constants (SVK_ISO)                        */
    double gdot0;            /* reference slip rate, 1/s        (CP_FCC, Eq. gamma_dot) */
    double p_exp;            /* rate exponent 1/m (integer valued, CP_FCC)          */
    double tau0;             /* critical resolved shear stress, Pa (CP_FCC)         */
    double c_af, d_af;       /* Armstrong-Frederick backstress constants (CP_FCC)   */
} gff_material;

typedef struct {
    int projection;    /* GFF_PROJ_*                                               */
    int precision;     /* GFF_PREC_FP64 or GFF_PREC_MIXED (FP32 CG/FFT/projection) */
    double newton_tol; /* stop when ||b||_2 / ||P||_2 <= newton_tol; the return maps
                          converge to max(1e-14, min(1e-11, 1e-5 newton_tol))    */
    double cg_tol;     /* CG stops when ||r|| <= max(cg_tol ||b||, 0.1 newton_tol ||P||) */
    int newton_max, cg_max;
    int max_cuts;      /* increment halvings allowed after a CP or Newton failure   */
    int warm_start;    /* initial guess (gff_set_warm_start): 0 zero start, 1
                          network if its residual beats the zero start's, 2
                          network, 3 extrapolation of the last increment     */
    double fs_k, fs_sigma_y; /* Fatemi-Socie constants                             */
} gff_options;

typedef struct {
    int newton_iters;   /* Newton corrections taken                         */
    int cg_iters;       /* CG iterations summed over the increment          */
    int cuts;           /* time-step halvings used                           */
    double residual;    /* final ||b|| / ||P||                               */
    double Pmacro[9];   /* volume average of P                              */
    double Fmacro[9];   /* volume average of F                              */
    double seconds;     /* wall time of the increment                       */
    double t_constitutive; /* device time in constitutive updates, s        */
    double t_residual;     /* device time in residual evaluations, s         */
    double t_linear;       /* device time in the CG solves, s                */
    int warm_start_used;   /* 1: the Newton iteration started from the warm-start guess */
    double residual_first; /* ||b|| / ||P|| at the start the Newton iteration used     */
    int cp_fallbacks;      /* voxel return maps that needed the exact-Newton fallback */
    double cp_local_iters; /* local Newton iterations per voxel, summed over the
                              increment's constitutive evaluations                  */
    double t_tangent;      /* the part of t_constitutive spent in tangent-only launches
                              (the return maps take the rest), s                      */
} gff_step_report;

typedef struct gff_unet gff_unet;

/* Defaults: continuous projection, FP64, newton_tol 1e-8, cg_tol 1e-8,
 * newton_max 30, cg_max 2000, max_cuts 4, fs_k 0.5, fs_sigma_y 153e6. */
void gff_options_default(gff_options* opt);

/* Create one RVE on the current CUDA device: allocates its device buffers
 * (about 1.5 kB per voxel in FP64 with crystal plasticity).  F starts at the
 * identity, internal variables at zero.  Grid and equations: Sect. 2.1. */
gff_status gff_create(const gff_grid* grid, const gff_options* opt, gff_handle** out);
void gff_destroy(gff_handle* h);
const char* gff_last_error(const gff_handle* h);

/* Run all device work of h on `stream` (a cudaStream_t; NULL = legacy default stream). */
gff_status gff_set_stream(gff_handle* h, void* stream);
gff_status gff_set_options(gff_handle* h, const gff_options* opt);

/* Voxel grain map and grain orientations (Sect. 3.1 RVE).
 * grain_id: N int32 in [0, ngrains); quat: ngrains*4 unit quaternions
 * (w, x, y, z) mapping crystal axes to sample axes; grain_phase: ngrains
 * phase indices in [0, 8).  Copies the data; may be called again to change
 * the microstructure (state is reset). */
gff_status gff_set_microstructure(gff_handle* h, const int32_t* grain_id, int ngrains,
                                  const double* quat, const int32_t* grain_phase);

/* Constitutive law of one phase (Eq. constitutive; Sect. 3.2). */
gff_status gff_set_material(gff_handle* h, int phase, const gff_material* m);

/* Overwrite (set) or read (get) one voxel field of the committed state.
 * `which` = GFF_FIELD_*; host buffer of (components x N) doubles in the SoA
 * layout above.  Setting F also evaluates nothing: call gff_constitutive. */
gff_status gff_set_field(gff_handle* h, int which, const double* host);
gff_status gff_get_field(gff_handle* h, int which, double* host);

/* Evaluate P and K = dP/dF (Eq. P_dif) at the current F for a time step dt,
 * without committing internal variables. */
gff_status gff_constitutive(gff_handle* h, double dt);

/* y = G_M(K : x)  (Eq. newlinop) with the K of the last gff_constitutive.
 * gff_step computes tangents only where a Newton correction needs them, never
 * at the converged iterate, so after a step (or gff_set_field of F) an apply
 * returns GFF_ERR_STATE until gff_constitutive is called.  precision GFF_PREC_FP64: x_dev, y_dev are double[9N];
 * GFF_PREC_MIXED: float[9N] and K rounded to FP32.  mask9 (host, may be NULL)
 * marks stress-controlled components: the zero frequency of the operator is
 * diag(mask9) instead of 0.  x_dev and y_dev may not overlap. */
gff_status gff_apply_operator(gff_handle* h, int precision, const uint8_t* mask9,
                              const void* x_dev, void* y_dev);

/* Diagnostic twin of gff_apply_operator: the same three kernels, with CUDA
 * events recorded on the handle's stream around each; ms_out[3] (host)
 * receives their durations in milliseconds -- [0] the per-plane K
 * contraction with the forward x/y transforms, [1] the z transforms with the
 * projection, [2] the inverse y/x transforms.  Synchronises the stream. */
gff_status gff_apply_operator_timed(gff_handle* h, int precision, const uint8_t* mask9,
                                    const void* x_dev, void* y_dev, float* ms_out);

/* gff_apply_operator with HOST buffers, for callers without device memory of
 * their own: x_host is copied into the handle's work vector, the operator
 * applied, y copied back to y_host (double[9N] for GFF_PREC_FP64, float[9N]
 * for GFF_PREC_MIXED, the layout of gff_apply_operator).  The copies go in
 * chunks of z-planes on a second stream of the handle (made on first use):
 * a chunk's forward plane pass waits only for its own copy, a chunk's copy
 * back only for its own inverse plane pass, so with pinned host memory the
 * copies overlap the plane passes of the other chunks (pageable memory works,
 * without the overlap).  The result equals gff_apply_operator's bit for bit.
 * Returns when y_host is written, with the status of gff_sync.  It uses the
 * handle's CG work vectors as device buffers. */
gff_status gff_apply_operator_host(gff_handle* h, int precision, const uint8_t* mask9, const void* x_host,
                                   void* y_host);

/* Measurement helpers (no counterpart in the paper).
 * gff_cg_kernels_timed: durations in ms, averaged over `reps`, of the vector
 * kernels of one conjugate-gradient iteration on this handle's work vectors
 * (overwritten): ms_out[0] the dot product p.Ap with alpha, [1] x += alpha p,
 * r -= alpha Ap with the new r.r and beta, [2] p = r + beta p.  Algorithmic
 * traffic per element: 2, 6 and 3 vector accesses.
 * gff_measure_fp64_peak: FP64 FMA throughput of the current GPU (independent
 * FMA chains on every SM, best of 5 launches timed with CUDA events), in
 * GFLOP/s (2 flops per FMA); ms_out (may be NULL) the launch's duration.
 * Allocates and frees a 1.2 MB buffer. */
gff_status gff_cg_kernels_timed(gff_handle* h, int precision, int reps, float* ms_out);
gff_status gff_measure_fp64_peak(double* gflops_out, double* ms_out);

/* Choose the launch shapes of the three apply kernels (threads of the plane
 * kernels, columns per block and threads of the z kernel) by timing every
 * candidate on this grid; results are bitwise the same for every choice.
 * gff_step runs it once per handle if it has not been run.  Uses the handle's
 * work buffers (call it before setting up an apply by hand, or call
 * gff_constitutive again afterwards).  tiles_out (host, 12 ints, may be NULL):
 * {fwd threads, z columns, z threads, inv threads, inv blocks} for FP64 then
 * FP32, then the persistent TMA z pass's blocks for FP64 and FP32 (0: one
 * block per strip).  inv blocks: 0 one block per plane; > 0 the persistent
 * streamed inverse pass with that many blocks; -1 the register-staged
 * inverse pass (one block per plane) of grids with nx = ny = 64 or 128;
 * <= -2 the register-staged persistent pass (two plane buffers) with -inv
 * blocks blocks.  fwd threads < 0: the register-staged forward pass of those
 * grids with -fwd threads threads.  TMA z blocks < 0: the TMA z pass with the
 * register-staged strip (nz = 64 or 128) and -(TMA z blocks) blocks. */
gff_status gff_autotune(gff_handle* h, int* tiles_out);

/* Sets the launch shapes instead of tuning them: tiles (host, 12 ints) in the
 * layout gff_autotune writes.  Allowed: fwd threads 256/512; z columns
 * 4/8/16/32 with z threads 128/256 (one block per strip), or, with TMA z
 * blocks > 0, z columns 8/16 and z threads 192/256/384/512; inv threads 256/512, or
 * with inv blocks > 0 up to 1024 (FP32) / 512 (FP64), or with inv blocks -1
 * (nx = ny = 64 or 128 only) 256/512, or with inv blocks <= -2 512 (or 1024
 * in FP32; where two planes fit in shared memory); fwd threads also -256 /
 * -512 on those grids; with TMA z blocks < 0, z threads 256 (or 384 in
 * FP32).  Every shape performs the same
 * operations in the same order, so results do not depend on them.
 * gff_batch_run gives each size class the shapes of its first RVE and runs
 * one-block-per-strip / one-block-per-plane kernels: the other shapes are
 * mapped onto them (z threads at most 256, inv threads at most 512).  Returns
 * GFF_ERR_ARG, changing nothing, for a shape the grid cannot use (shared
 * memory, no tensor-map support for TMA, no register-staged pass). */
gff_status gff_set_tiles(gff_handle* h, const int* tiles);

/* gff_apply_operator and gff_project return once their kernels are queued on
 * the handle's stream.  gff_sync waits for the stream and reports what the
 * device recorded meanwhile: GFF_ERR_TIMEOUT if a bounded wait of an FFT pass
 * on an asynchronous (TMA) copy gave up since the last check -- the planes it
 * left uncomputed are NaN in y -- and clears that record; else GFF_OK.
 * gff_step checks the same record itself after every residual. */
gff_status gff_sync(gff_handle* h);

/* Budget, in SM clock cycles, of the first wait of each FFT pass on its
 * asynchronous (TMA) copies; cycles < 0 restores the default (about two
 * seconds).  A budget of 0 gives up at once: the pass records the timeout,
 * lets its copies land (waiting at most the default budget) and skips its
 * work, which exercises the error path of gff_sync without any fault.  For
 * tests of that path; the default is the only sensible value otherwise. */
gff_status gff_set_wait_limit(gff_handle* h, long long cycles);

/* Small-strain variant of the variational method (the paper's solver runs at
 * small and finite strains, Sect. 2.3).  GFF_STRAIN_SMALL: the unknown field
 * is the infinitesimal strain eps (stored, read and set as GFF_FIELD_F,
 * starting at 0); the phases must be linear elastic (GFF_MAT_SVK_CUBIC /
 * GFF_MAT_SVK_ISO read as sigma = C : eps, tangent C), GFF_FIELD_P is the
 * Cauchy stress; gff_step's Fbar is the prescribed average strain and Pbar
 * the prescribed average stress; the projection onto compatible fields is the
 * symmetric one, y = n (x) a + a (x) n - (n . a) n (x) n with a = sym(x^) n
 * and n the unit continuous or discrete (GFF_PROJ_*) wave vector, and the
 * zero frequency takes the mask as in the finite-strain case.  Switching
 * resets the state.  gff_batch_run rejects small-strain handles. */
enum { GFF_STRAIN_FINITE = 0, GFF_STRAIN_SMALL = 1 };
gff_status gff_set_strain_measure(gff_handle* h, int mode);

/* How the crystal-plasticity return maps are iterated (the paper leaves it
 * open; the root of the backward-Euler residual of Eq. gamma_dot is the same):
 * GFF_RETURN_MAP_FP64: Newton steps with the small-elastic-strain Jacobian
 *   from the previous iterate's slips, in FP64, then, if that fails, exact
 *   Newton from zero slip (the fallback, counted in
 *   gff_step_report.cp_fallbacks);
 * GFF_RETURN_MAP_F32_FIRST: the same FP64 iteration preceded by that
 *   iteration in FP32 (elastic state formed from the small quantities F - I
 *   and Fp^-1 - I) down to FP32 resolution; the FP64 iteration then starts
 *   from its root.  The FP64 residual still decides convergence, so the root
 *   is GFF_RETURN_MAP_FP64's to the return-map tolerance;
 * GFF_RETURN_MAP_DEFAULT (a new handle's mode): GFF_RETURN_MAP_F32_FIRST when
 *   the handle's precision is GFF_PREC_MIXED, GFF_RETURN_MAP_FP64 in
 *   GFF_PREC_FP64;
 * GFF_RETURN_MAP_EXACT: exact Newton (12x12 LU with partial pivoting) from
 *   zero slip only -- every return map counts as a fallback. */
enum {
    GFF_RETURN_MAP_DEFAULT = 0,
    GFF_RETURN_MAP_EXACT = 1,
    GFF_RETURN_MAP_F32_FIRST = 2,
    GFF_RETURN_MAP_FP64 = 3
};
gff_status gff_set_return_map(gff_handle* h, int mode);

/* y = G_M(x) = F^-1{ G^ : F(x) }  (Eq. eql_discrete3), same conventions. */
gff_status gff_project(gff_handle* h, int precision, const uint8_t* mask9,
                       const void* x_dev, void* y_dev);

/* Allocation-free twin of gff_project, for callers that may not allocate
 * device memory themselves (an application whose own allocator owns the
 * whole device-memory budget, or a loop that cannot afford the device-wide
 * synchronisation that cudaMalloc/cudaFree may cause).  No handle: the grid,
 * projection (GFF_PROJ_*) and precision (GFF_PREC_FP64: double x_dev/y_dev,
 * GFF_PREC_MIXED: float) are passed directly; mask9 as in gff_project; the
 * work is queued on `stream` (a cudaStream_t, NULL = legacy default stream).
 * The paper has no counterpart.
 * Scratch: a file-scope device array of about 3.6 MB inside libgff.so, held
 * by every GPU that loads the library until the process exits; grids are
 * limited to nx*ny*nz <= 32768 voxels (axes as for gff_create), larger ones
 * return GFF_ERR_ARG.  The first call on a device looks up that array's
 * address (make this first call before any stream capture).  No cudaMalloc,
 * cudaFree or other allocating routine is called, and no host memory is
 * copied: the grid tables are written into the array by a kernel queued on
 * `stream` ahead of the projection.  All calls share the one array per
 * device and each call overwrites it, so calls whose device work overlaps
 * (different streams, or host threads) race and corrupt each other's
 * results; serialise them.
 * The call returns once its kernels are queued, before they run, so it has
 * no status word for device-side failures: if the bounded wait on a plane's
 * asynchronous copy ever gives up (its limit is about two seconds, for a copy
 * of microseconds), that plane of y is written as NaN.
 * Returns GFF_ERR_ARG for bad arguments and GFF_ERR_CUDA on a CUDA error (no
 * handle, so no message) -- also, without clearing it, when a CUDA error left
 * by an earlier call is still pending on entry. */
gff_status gff_project_noalloc(const gff_grid* grid, int projection, int precision,
                               const uint8_t* mask9, const void* x_dev, void* y_dev, void* stream);

/* One load increment (Sect. 2.1): macroscopic Fbar[9] on components with
 * mask[c] = 0, average stress Pbar[9] on components with mask[c] = 1.
 * Newton-CG to newton_tol, then internal variables and FIP accumulators are
 * committed.  If Newton or a return map fails, the increment is halved (dt/2,
 * macroscopic targets interpolated from the committed state) and retried, up
 * to opt.max_cuts levels (report->cuts counts the halvings); on final failure
 * the committed state is unchanged.  report may be NULL. */
gff_status gff_step(gff_handle* h, double dt, const double Fbar[9], const uint8_t mask[9],
                    const double Pbar[9], gff_step_report* report);

/* nsteps increments; arrays are nsteps x 9 (mask uint8).  cycle_start
 * (nsteps, may be NULL) restarts the FIP accumulators before that increment.
 * Pmacro_out (nsteps x 9) and reports (nsteps) may be NULL.  Stops at the
 * first failing increment and returns its status. */
gff_status gff_run_history(gff_handle* h, int nsteps, const double* dt, const double* Fbar,
                           const uint8_t* mask, const double* Pbar, const uint8_t* cycle_start,
                           double* Pmacro_out, gff_step_report* reports);

/* Several RVEs through one loading history together (the statistical
 * volume element of Sect. 4.3 needs tens of RVEs; sizes may differ).
 * hs: n distinct handles (1 <= n <= 64) on one device with identical
 * precision, projection, tolerances and caps, each with microstructure and
 * materials set.  dt, Fbar, mask, Pbar, cycle_start: as in gff_run_history
 * (one history for all).  Each increment of all RVEs is one launch of a CUDA
 * graph (captured once per stress-control mask) whose Newton and CG loops run
 * on the device as conditional WHILE nodes, bounded by newton_max + 1 and
 * cg_max iterations, with per-RVE status words; RVEs of one grid size run the
 * apply kernels with the launch shapes tuned for that size, each size class
 * on its own stream inside the graph.  RVEs whose handle has warm-start mode
 * GFF_WARM_EXTRAPOLATE start from the extrapolated guess (other modes start
 * from the zero-fluctuation start).  An RVE whose increment fails in the batch
 * is redone by gff_step on its own handle, cut-backs included; if that fails
 * too, the RVE keeps its last committed state, gets the status in per_rve and
 * leaves the batch while the others go on.  An RVE that converges in the
 * batch gets bitwise the result of gff_run_history on its own handle.
 * Pmacro_out (n x nsteps x 9), reports (n x nsteps), per_rve (n): may be NULL.
 * Returns GFF_OK when all RVEs finished, else the first failing RVE's status.
 * The handles' streams are synchronised before and after the call. */
gff_status gff_batch_run(int n, gff_handle* const* hs, int nsteps, const double* dt, const double* Fbar,
                         const uint8_t* mask, const double* Pbar, const uint8_t* cycle_start,
                         double* Pmacro_out, gff_step_report* reports, gff_status* per_rve);

/* Automatic time incrementation (Sect. 2.3 names an automatic time
 * incrementation algorithm without stating it; this is the FE-style rule).
 * The macroscopic path is piecewise linear between nknots knots: at time
 * t_knots[k] the targets are Fbar_knots[9k..] (strain-controlled components)
 * and Pbar_knots[9k..] (stress-controlled ones, mask[9] for the whole path);
 * t_knots[0] is the time of the committed state.  Increments never step
 * across a knot.  The first increment takes dt_initial; after each accepted
 * increment the next size is
 *   the size that worked, if gff_step had to cut the increment;
 *   dt * grow, if it converged in at most easy_newton Newton corrections
 *     (and was not shortened by a knot);
 *   dt * shrink, if it needed hard_newton corrections or more;
 *   dt otherwise;
 * clamped to [dt_min, dt_max].  cycle_start (nknots, may be NULL) restarts
 * the FIP accumulators when the path reaches a flagged knot.  Outputs (host,
 * up to max_increments entries each; t_out, Pmacro_out, reports may be NULL):
 * *n_out increments, their end times, average P (x 9) and reports.  Stops at
 * the first failing increment (its status), or with GFF_ERR_NO_CONVERGENCE
 * if max_increments do not reach the end of the path. */
typedef struct {
    double dt_initial, dt_min, dt_max;
    double grow, shrink;
    int easy_newton, hard_newton;
} gff_auto_options;
/* dt_initial 0.05, dt_min 1e-6, dt_max 1, grow 1.5, shrink 0.75, easy 3, hard 8 */
void gff_auto_options_default(gff_auto_options* a);
gff_status gff_run_auto(gff_handle* h, int nknots, const double* t_knots, const double* Fbar_knots,
                        const uint8_t* mask, const double* Pbar_knots, const uint8_t* cycle_start,
                        const gff_auto_options* ao, int max_increments, int* n_out, double* t_out,
                        double* Pmacro_out, gff_step_report* reports);

/* ------------------------------------------------------------------------
 * Warm starts (not in the paper; Sect. 2.1 leaves the Newton initial guess
 * open).  With d_k the prescribed macroscopic increment of increment k (dFbar
 * on strain-controlled components, 0 on stress-controlled ones) and
 * y_k = (F_k - F_{k-1} - dFbar_k) / |d_k| its normalised fluctuation
 * increment, the guess for increment k is F_{k-1} + d_k + G^(|d_k| y~) with
 *   extrapolation (mode 3):  y~ = s y_{k-1},  s = (d_k . d_{k-1}) / (|d_k| |d_{k-1}|)
 *   network (modes 1, 2):    y~ = s y_{k-1} + U(x),
 * G^ projecting onto compatible zero-mean fields.  U is a 4-level periodic
 * 3D U-Net (channels 16, 32, 64, 64; leaky ReLU) whose 32 input channels per
 * voxel are the grain orientation quaternion (4), the phase (1), d_k/|d_k|
 * (9), y_{k-1} (9) and d_{k-1}/|d_{k-1}| (9) (zeros without history); it is
 * trained on y_k - s y_{k-1}.  bfloat16 weights/activations, FP32
 * accumulation on the tensor cores, FP32 master weights and Adam.  Grids
 * must be cubic with n divisible by 8.
 * ------------------------------------------------------------------------ */
/* He-uniform convolution weights from SplitMix64(seed); zero biases and head */
gff_status gff_unet_create(uint64_t seed, gff_unet** out);
void gff_unet_destroy(gff_unet* u);
const char* gff_unet_last_error(const gff_unet* u);
size_t gff_unet_num_params(const gff_unet* u);
/* Parameters as FP32 host arrays, order: for the 14 convolutions e1a e1b e2a
 * e2b e3a e3b e4a e4b d3a d3b d2a d2b d1a d1b: W[27][cout][cin] then
 * b[cout] (tap t = 9(dz+1) + 3(dy+1) + (dx+1)); then the head W[9][16], b[9]. */
gff_status gff_unet_get_params(gff_unet* u, float* host);
gff_status gff_unet_set_params(gff_unet* u, const float* host);
gff_status gff_unet_save(gff_unet* u, const char* path);
gff_status gff_unet_load(gff_unet* u, const char* path);
/* Network output y [V][9] for host inputs x [V][32] on an n^3 grid; with a
 * target [V][9] also the mean-squared-error loss and all parameter gradients
 * (order of gff_unet_get_params).  target, loss, grads may be NULL. */
gff_status gff_unet_eval_host(gff_unet* u, int n, const float* x, const float* target, float* y,
                              double* loss, float* grads);
/* Keep the last completed increment k of h (inputs from d_k, y_{k-1},
 * d_{k-1}; target y_k - s y_{k-1}) as a training sample on the device; all
 * samples share one grid.  The increment must have a prescribed strain
 * increment (|d_k| > 0). */
gff_status gff_unet_add_sample(gff_unet* u, gff_handle* h);
/* A training sample from host arrays x [V][32], target [V][9] (n^3 grid,
 * n divisible by 8, the same n as the other samples). */
gff_status gff_unet_add_sample_host(gff_unet* u, int n, const float* x, const float* target);
int gff_unet_num_samples(const gff_unet* u);
/* `steps` Adam steps (peak lr with a cosine decay to 0 over the steps, betas
 * 0.9/0.999, gradients clipped to global norm 1), one sample per step,
 * shuffled epochs; losses (host, steps, may be NULL) receives each step's
 * loss. */
gff_status gff_unet_train(gff_unet* u, int steps, double lr, double* losses);
/* How gff_unet_train picks samples: 0 (default) shuffled epochs; 1 each step
 * draws a sample with probability 1/(2 n) + e_i / (2 sum e), e_i the mean
 * square of sample i's target, so the increments the extrapolation predicts
 * worst (first increments, load reversals) are seen more often. */
gff_status gff_unet_set_sampling(gff_unet* u, int mode);
/* Initial guess of h's increments: mode 0 zero-fluctuation start; 1 network
 * guess, kept only when its first residual is below the zero start's (costs
 * one more constitutive evaluation per increment); 2 network guess always;
 * 3 extrapolation (u may be NULL).  In every mode a guess at which a return
 * map fails, or whose residual is not finite, is replaced by the zero start.
 * gff_batch_run does not use warm starts. */
gff_status gff_set_warm_start(gff_handle* h, gff_unet* u, int mode);

/* Fatigue indicator parameters (Sect. 3.3, Eqs. eqplas, strainenergy, Pmax).
 * gff_reset_fips restarts the per-cycle accumulators.  gff_get_fips returns
 * grain averages of the current accumulators: pcyc_g[ngrains],
 * wcyc_g[ngrains*12], fs_g[ngrains] (Fatemi-Socie); any may be NULL. */
gff_status gff_reset_fips(gff_handle* h);
gff_status gff_get_fips(gff_handle* h, double* pcyc_g, double* wcyc_g, double* fs_g);

/* Appendix A: what an Abaqus-style user material returns -- the Cauchy stress
 * sigma and the tangent C^ab of the Jaumann rate of the Kirchhoff stress
 * (Eq. ABAtang) -- converted into the first Piola-Kirchhoff stress
 * P = J sigma F^-T (Eq. fPK) and the tangent K = dP/dF the FFT solver needs
 * (the final expression of Appendix A), for n voxels on the device.
 * Layouts: F_dev, sigma_dev, P_dev double[9][n]; Cab_dev, K_dev double[81][n]
 * with index 9 (3i + j) + (3k + l) (C^ab with its minor symmetries).  The
 * work is queued on `stream` (a cudaStream_t, NULL = legacy default stream);
 * no handle, no allocation.  GFF_ERR_ARG for n < 0 or null pointers,
 * GFF_ERR_CUDA on a launch error. */
gff_status gff_umat_tangent(long long n, const double* F_dev, const double* sigma_dev, const double* Cab_dev,
                            double* P_dev, double* K_dev, void* stream);

/* Band-averaged dissipated energy W_cyc^b (Eq. Wmax) of the current cycle's
 * accumulators.  Each crystal-plastic grain is cut into bands of `width`
 * (a length, units of gff_grid.L) parallel to each of its four {111} slip
 * planes: a voxel's band for plane p is floor(s / width + 1/2), s = (x - x_ref).m_p,
 * x - x_ref the minimum-image offset (per axis in [-n/2, n/2) voxels) of its
 * centre from the grain's reference voxel (the grain's lowest voxel index),
 * m_p the plane's unit normal in the sample frame.  W_cyc of the plane's three
 * systems is averaged over every band; wb_g[ngrains] (may be NULL) receives
 * each grain's largest band average (0 for other phases), wb_max (may be NULL)
 * the largest over the RVE.  Allocates a temporary device buffer of about
 * 16 ngrains (sqrt(Lx^2 + Ly^2 + Lz^2) / width + 4) doubles (GFF_ERR_ARG above
 * 2 GB). */
gff_status gff_get_band_fips(gff_handle* h, double width, double* wb_g, double* wb_max);

/* Committed state to/from a raw little-endian file: header, increment
 * history (the last prescribed increments and normalised fluctuation
 * increments the warm starts use), F, internal variables, FIP accumulators
 * and the last slip increments, so that a resumed run repeats the original
 * bit for bit.  Loading requires the same grid. */
gff_status gff_save_state(gff_handle* h, const char* path);
gff_status gff_load_state(gff_handle* h, const char* path);

#ifdef __cplusplus
}
#endif
#endif /* GFF_H */
