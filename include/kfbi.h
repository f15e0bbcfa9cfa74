/*
 * kfbi.h - C ABI of the GB300 (sm_103a) kernel-free boundary integral (KFBI) library.
 *
 * The library evaluates the double-layer boundary operator K_D = 1/2 I + W of the
 * modified Helmholtz / Poisson equation  Lap u - kappa^2 u = f  on a 2-D (or 3-D, see
 * kfbi_setup) domain Omega embedded in the box B = [lo, hi]^dim, WITHOUT a Green's
 * function: the potential is the solution of the equivalent interface problem on a
 * Cartesian grid of B (paper Sec. 2.2, "Indirect evaluation of integrals"; table of F and
 * Phi there):
 *     Lap v - kappa^2 v = F in B \ Gamma,  [v] = Phi,  [d_n v] = psi on Gamma,  v = 0 on dB,
 * discretised by Alg. 1: jumps at grid-line/interface crossings, Taylor correction of the
 * right-hand side at irregular nodes (Alg. 2), a fast sine-transform box solve (Alg. 4),
 * corrected interpolation to the control points (Alg. 3).  The Dirichlet BVP is solved
 * through the BIE 1/2 phi + W phi + Y f = g (Sec. 2.1) by restarted GMRES (Alg. 5), in
 * plain FP64 or in mixed precision (FP32 box solves with FP64 iterative refinement).
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are DEVICE pointers owned by the caller (e.g. allocated through
 *     PyTorch); the library never frees them and never keeps them after the call returns.
 *     Pointers named h_* are host pointers.  All arrays are contiguous, C order, FP64.
 *   - Grid arrays are (N+1) x (N+1) with x fastest: a[j*(N+1) + i] = value at
 *     (lo + i h, lo + j h), h = (hi - lo)/N; in 3-D (N+1)^3 with x fastest, then y:
 *     a[(k*(N+1) + j)*(N+1) + i] at (lo + i h, lo + j h, lo + k h).
 *   - Interface arrays have M entries (points/normals: M x 2, interleaved x,y; 3-D as
 *     described at kfbi_setup).  2-D points are counter-clockwise samples of Gamma at
 *     equispaced parameter t_k = 2 pi k / M; normals are outward unit normals; curv is
 *     the signed curvature (> 0 where convex).
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed as void*,
 *     NULL = legacy default stream) unless documented as synchronising.
 *   - All workspace is allocated by kfbi_setup; apply and solve calls allocate nothing.
 *   - Errors are returned as kfbi_status; kfbi_last_error() gives a message for the
 *     calling thread.  No entry point aborts, exits or traps on the device.
 *   - A context may be used by one host thread at a time.
 */
#ifndef KFBI_H
#define KFBI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kfbi_ctx_s* kfbi_ctx;

typedef enum {
  KFBI_OK = 0,
  KFBI_ERR_ARG = 1,            /* bad argument (null pointer, size, option)            */
  KFBI_ERR_GEOMETRY = 2,       /* interface under-resolved, tangent to a grid line at a
                                  point with no label change, or within two cells of dB */
  KFBI_ERR_NOMEM = 3,          /* device allocation failed in kfbi_setup                 */
  KFBI_ERR_CUDA = 4,           /* a CUDA runtime call failed                             */
  KFBI_ERR_NOT_CONVERGED = 5,  /* GMRES reached its iteration limit; outputs hold the
                                  last iterate and info->rel_residual its residual      */
  KFBI_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up                     */
  KFBI_ERR_NUMERIC = 7,        /* NaN/Inf met in the iteration                           */
  KFBI_ERR_UNSUPPORTED = 8     /* valid request this build does not implement            */
} kfbi_status;

typedef enum {
  KFBI_FP64 = 0,         /* every stage in FP64                                          */
  KFBI_MIXED_FP32 = 1,   /* box solve in FP32 (apply; in 2-D the well-conditioned x-modes
                            have their tridiagonal y-systems solved directly (recursive
                            filters or elimination), the others take the sine-transform
                            pair, see kfbi_ctx_info.tri_first_mode);
                            as a solver mode: FP64 Arnoldi and Givens with relaxed-
                            precision matvecs and FP64-accurate residuals (see
                            kfbi_solve_bvp)                                              */
  KFBI_FP32_REFINED = 2, /* box solve from FP32 sine transforms corrected twice against
                            the residual of the 5-point system, formed in double-single
                            (exact FP32-pair) arithmetic at regular nodes and in FP64 at
                            irregular nodes: FP64-accurate (about 1e-13 relative) at FP32
                            cost; the mixed BVP solver uses it for its accurate steps    */
  KFBI_FP32_REFINED_ONCE = 3, /* one refinement step (about 1e-11 relative at N = 1024,
                            3e-10 at N = 4096)                                           */
  KFBI_TF32X3 = 4        /* box solve in the dense form of Alg. 4 (full diagonalisation by
                            the sine matrix) as GEMMs on the tcgen05 tensor cores (four in
                            2-D, six in 3-D), TF32 with a three-term split and FP32
                            accumulation (FP32-class accuracy); N a multiple of 128, up to
                            8192 in 2-D and 512 in 3-D (else KFBI_ERR_UNSUPPORTED); an
                            apply / box-solve / interface-solve precision, and as solver
                            precision the mixed solver with tensor-core plain applies      */
} kfbi_precision;

typedef enum {
  KFBI_DOUBLE_LAYER = 0, /* [v] = density, [d_n v] = 0: returns v^+ = (1/2 I + W) density */
  KFBI_SINGLE_LAYER = 1  /* [v] = 0, [d_n v] = density: returns v^+ on Gamma              */
} kfbi_layer;

typedef struct {
  int dim;              /* 2 or 3                                                       */
  int N;                /* cells per side, N = 2^a or 3*2^a, 32 <= N <= 8192 (2-D),
                           <= 512 (3-D)                                                */
  double lo, hi;        /* box [lo, hi]^dim                                             */
  double kappa;         /* >= 0; PDE Lap u - kappa^2 u = f                               */
  int precision;        /* kfbi_precision used by kfbi_solve_bvp: FP64 (plain FP64 GMRES)
                           or MIXED_FP32 / TF32X3 (one FP64 Arnoldi process whose matvecs
                           are twice-refined, once-refined, then plain FP32 or tensor-core
                           box solves as the residual drops; every restart cycle ends
                           with an FP64-accurate residual, see kfbi_solve_bvp)        */
  int gmres_m;          /* GMRES restart length (Alg. 5), 1..128                         */
  int max_restarts;     /* GMRES restarts (cycles - 1)                                  */
  double tol;           /* stop when ||g_hat - K_D phi||_2 <= tol ||g_hat||_2            */
  double inner_tol;     /* mixed: assumed relative accuracy of a plain FP32 apply; once
                           the residual is below tol / inner_tol the Arnoldi steps use
                           plain FP32 applies (default 1e-5)                           */
} kfbi_options;

typedef struct {
  int iterations;        /* Arnoldi steps over all cycles                                 */
  int outer_iterations;  /* GMRES restart cycles (each ends with an FP64-accurate residual) */
  int applies_fp64;      /* applies with an FP64-accurate box solve (FP64, or FP32
                            transforms refined against the FP64 residual)               */
  int applies_low;       /* K_D applies with a plain FP32 or tensor-core box solve (the
                            Arnoldi steps taken once the residual is below
                            tol / inner_tol)                                             */
  double rel_residual;   /* final ||g_hat - K_D phi|| / ||g_hat|| (FP64 apply)           */
  int converged;         /* 1 if rel_residual <= tol                                     */
} kfbi_solve_info;

typedef struct {
  int N, M;
  int n_crossings_x;     /* 2-D: crossings of Gamma with the lines x = x_i; 3-D: points on
                            x-lines (y, z on grid values)                                */
  int n_crossings_y;     /* 2-D: crossings with the lines y = y_j; 3-D: points on y-lines */
  int n_irregular;       /* interior nodes with a 5-point neighbour across Gamma          */
  int n_inside;          /* grid nodes inside Omega                                      */
  int64_t device_bytes;  /* workspace held by the context                                */
  int dst_variant[4];    /* box-solver kernel variants picked by the setup-time autotuner:
                            row pass FP32, column pass FP32, row pass FP64, column pass
                            FP64 (row: 0 = 16/24 values per thread, 1 = 8/12; column:
                            bit 0 = 256-thread blocks, bit 1 = 8/12 values per thread,
                            bit 2 = transposed pass: transpose, row-wise y-transforms,
                            transpose back; 8 = FP32 y-pass on the row layout: recursive
                            filters along y for the modes >= tri_first_mode, the transform
                            pair for the lower ones) */
  int dim;               /* 2 or 3                                                        */
  int n_crossings_z;     /* 3-D: points on z-lines; 0 in 2-D                              */
  int tri_first_mode;    /* 2-D FP32 box solves: x-modes k >= this have their tridiagonal
                            y-systems solved directly, by the recursive filters of the
                            row-layout pass (dst_variant[1] = 8; elimination coefficient
                            c <= 0.9) or by chunked elimination (c <= 0.825), the lower
                            ones by the sine-transform pair; a multiple of 32; N when every
                            mode takes the transform pair                               */
} kfbi_ctx_info;

/* Fills *opt with dim 2, N 128, box [-1,1], kappa 0, FP64, m 50, 20 restarts,
   tol 1e-10, inner_tol 1e-5. */
void kfbi_default_options(kfbi_options* opt);

/* Builds the discrete interface problem on the device (Procedure 1 of Sec. 4.4, Alg. 1
   steps 1-3): the periodic degree-5 interpolant of the control points, the crossings
   of Gamma with every grid line, the inside/outside node labels, the compacted list
   of irregular nodes with their crossed arms (Sec. 2.2, Fig. of irregular nodes), and
   the FP64 linear maps density -> corrected right-hand side (Alg. 2) and grid values
   -> v^+ at the control points (Alg. 3).  All geometry is computed in FP64 on the GPU.
   dim = 2: d_pts, d_normals: M x 2; d_curv: M signed curvatures.
   dim = 3 (N <= 512; the paper describes 3-D only by analogy with 2-D): the M control
   points are the intersections of Gamma with the grid lines, each with two coordinates
   on grid values (x-, y- and z-lines in any order); d_pts, d_normals: M x 3 (outward
   unit normals); d_curv: M x 6 packed symmetric shape operators (Sxx, Syy, Szz, Sxy,
   Sxz, Syz; dn = S dx on tangent vectors).  Points are tagged and sorted per line on
   the host; labels by line parity, irregular nodes with their arms, least-squares
   surface-derivative weights (quadratic over the points within 2.5 h, 3.5 h when fewer
   than 10) and the 10-node interpolation stencils are built on the GPU in FP64.  The
   3-D double-layer apply uses the least-squares value of the density in the jumps and
   adds half the difference to the point value (the second-kind identity part acts on
   the point values); grids are (N+1)^3 with x fastest.  3-D supports the double and
   single layers and the volume potential in every precision (the refinement residual uses the
   7-point operator).
   2-D setup times the transform variants on the context's grids and keeps the fastest
   (kfbi_ctx_info.dst_variant); the environment variable KFBI_DST_VARIANTS="r32,c32,r64,c64"
   fixes them instead (for profiling runs, whose timings would mislead the autotuner).
   Synchronises the stream (reads back counts).  Returns KFBI_ERR_GEOMETRY for an
   under-resolved interface or a point off the grid lines; *out is NULL on error. */
kfbi_status kfbi_setup(const kfbi_options* opt, int64_t M, const double* d_pts,
                       const double* d_normals, const double* d_curv, void* stream,
                       kfbi_ctx* out);

/* One layer-potential apply (the hot path, Alg. 1 steps 4-6): jumps from the density
   (Alg. 2), RHS correction at irregular nodes, sine-transform box solve (Alg. 4)
   in the given precision, corrected interpolation to the control points (Alg. 3).
   For KFBI_DOUBLE_LAYER the result is K_D density = (1/2 I + W) density (Sec. 3.3).
   d_density, d_out: M values.  Asynchronous. */
kfbi_status kfbi_apply_layer_potential(kfbi_ctx ctx, int layer, int precision,
                                       const double* d_density, double* d_out, void* stream);

/* (Y f)^+ at the control points: interface problem with F = zero extension of f to
   the box and Phi = 0 (Sec. 2.2 table).  d_f_grid: (N+1)^2, values outside Omega are
   ignored; d_f_ctrl: f at the M control points (gives the jump [F] on Gamma). */
kfbi_status kfbi_apply_volume(kfbi_ctx ctx, int precision, const double* d_f_grid,
                              const double* d_f_ctrl, double* d_out, void* stream);

/* Full interface solve with [v] = density, [d_n v] = 0, F = zero-extended f: writes the
   corrected right-hand side (d_rhs_grid, may be NULL), the grid solution v on all nodes
   (d_v_grid, may be NULL) and v^+ at the control points (d_out, may be NULL).
   d_density, d_f_grid, d_f_ctrl may each be NULL (= zero).  Exposes the stages of one
   apply for testing and post-processing. */
kfbi_status kfbi_interface_solve(kfbi_ctx ctx, int precision, const double* d_density,
                                 const double* d_f_grid, const double* d_f_ctrl,
                                 double* d_rhs_grid, double* d_v_grid, double* d_out,
                                 void* stream);

/* Box solve alone (Alg. 4): (Lap_h - kappa^2) v = b at interior nodes, v = 0 on dB,
   b and v (N+1)^2 grids (boundary entries of b ignored). */
kfbi_status kfbi_box_solve(kfbi_ctx ctx, int precision, const double* d_b_grid,
                           double* d_v_grid, void* stream);

/* ---------------------------------------------------------- allocation-free box solve
   The paper has no counterpart to this entry point.  It is the box solve above (the same
   transform kernels in their default variants) for callers that cannot allocate device
   memory when they need it: code running inside a pool that has already reserved the
   device's memory, or where the implicit device synchronisation of cudaMalloc/cudaFree
   cannot be tolerated.  kfbi_setup allocates a workspace sized by N and M, so those
   callers get no context; this call needs none.
     N, lo, hi, kappa: box [lo, hi]^2 with N cells per side (N = 2^a or 3 * 2^a,
       32 <= N <= KFBI_STATIC_MAX_N), (Lap_h - kappa^2) v = b.
     precision: KFBI_FP64 or KFBI_MIXED_FP32 (plain FP32 transforms).
     d_b_grid, d_v_grid: caller-owned device (N+1)^2 grids as for kfbi_box_solve
       (boundary entries of b ignored, v = 0 on the boundary); they may alias.
   Workspace: one static device array of KFBI_STATIC_SCRATCH_BYTES per device inside this
   library, holding the work grid and the transform tables.  No call ever allocates or
   frees device or host memory (no cudaMalloc/cudaFree, no allocating library call).
   Nothing in the array has to start at zero: each call rewrites the tables and the whole
   work grid before reading them.
   First call on each device: resolves the array's address (cudaGetSymbolAddress, with
   that device current) and sets the kernels' shared-memory limits; make this first call
   on every device before any stream capture begins.  Later calls only launch kernels.
   Calls on one device share the one array: two calls whose device work overlaps in time
   (different streams without ordering, or different host threads) race and corrupt
   each other's results; order them (one stream, or events).
   Errors: N above KFBI_STATIC_MAX_N or unsupported, null grids, hi <= lo, kappa < 0 or
   another precision -> KFBI_ERR_ARG (message names the limit), before any device work;
   a failed CUDA call -> KFBI_ERR_CUDA.  Asynchronous on `stream`: a bounded device-side
   wait of the transform kernels that gives up (a staged copy that never completed) is
   recorded in an error word at the end of the static array, not in this call's status;
   kfbi_box_solve_static_check reports it. */
#define KFBI_STATIC_MAX_N 1024
#define KFBI_STATIC_SCRATCH_BYTES (9u << 20)
kfbi_status kfbi_box_solve_static(int N, double lo, double hi, double kappa, int precision,
                                  const double* d_b_grid, double* d_v_grid, void* stream);

/* Asynchronous error report of kfbi_box_solve_static (no counterpart in the paper either):
   synchronises `stream`, then reads the static array's error word of the current device.
   Returns KFBI_ERR_TIMEOUT, and clears the word, if a bounded wait of any static box solve
   since the last check gave up (that solve's output is wrong); KFBI_OK otherwise.
   Allocates nothing. */
kfbi_status kfbi_box_solve_static_check(void* stream);

/* Dirichlet BVP (Procedures 2-3 of Sec. 4.4): g_hat = g - (Y f)^+, K_D phi = g_hat by
   GMRES(m) (Alg. 5; FP64 Arnoldi with CGS2 and Givens rotations on the device), then
   u = W phi + Y f on the grid (Sec. 2.1).  opt->precision selects plain FP64 or mixed
   precision: one FP64 Arnoldi process whose matvec precision is relaxed as the residual
   drops (inexact Krylov): twice-refined FP32 box solves while the residual is above
   tol / 1e-9, once-refined ones down to tol / inner_tol, plain FP32 below; every
   restart cycle ends with the true residual from a twice-refined (FP64-accurate) apply,
   so the GMRES residual is refined in FP64; the volume term and the final grid
   solution use the twice-refined solve as well.
   d_u_grid: (N+1)^2, written inside Omega, zero outside.  d_density_out: M or NULL.
   h_info: host struct or NULL.  Synchronising (convergence is checked on the host). */
kfbi_status kfbi_solve_bvp(kfbi_ctx ctx, const double* d_f_grid, const double* d_f_ctrl,
                           const double* d_g_ctrl, double* d_u_grid, double* d_density_out,
                           kfbi_solve_info* h_info, void* stream);

/* Neumann data of a layer potential (Procedure 2 of Sec. 4.4, "extract d_n u"): the
   interior normal derivative d_n v^+ at the control points of the interface problem of
   kfbi_apply_layer_potential (same layers and precisions), taken as n . grad of the
   quadratic fitted to the same 6 corrected grid values at each control point (outward n).
   For KFBI_SINGLE_LAYER this is the operator K_N psi of the Neumann BIE.  2-D only
   (KFBI_ERR_UNSUPPORTED in 3-D).  d_density, d_out: M values.  Asynchronous. */
kfbi_status kfbi_apply_layer_potential_dn(kfbi_ctx ctx, int layer, int precision,
                                          const double* d_density, double* d_out, void* stream);

/* d_n (Y f)^+ at the control points (the volume term of the Neumann BIE); arguments as
   kfbi_apply_volume.  2-D only.  Asynchronous. */
kfbi_status kfbi_apply_volume_dn(kfbi_ctx ctx, int precision, const double* d_f_grid,
                                 const double* d_f_ctrl, double* d_out, void* stream);

/* Neumann BVP  Lap u - kappa^2 u = f in Omega, d_n u = g_N on Gamma (Procedures 2-3 of
   Sec. 4.4 with the single-layer density psi; the single layer is the interface problem
   [v] = 0, [d_n v] = psi): u = V psi + Y f in Omega, so
   K_N psi = d_n (V psi)^+ = g_N - d_n (Y f)^+ is solved by GMRES(m) exactly as
   kfbi_solve_bvp solves K_D phi = g_hat (same solver options, FP64 or relaxed mixed
   precision), then u is the inside-node solution of the interface problem with
   [d_n v] = psi and F = zero-extended f.  kappa must be positive (for kappa = 0 the
   interior Neumann problem fixes u only up to a constant and K_N is singular):
   KFBI_ERR_ARG otherwise, before any device work.
   d_gn_ctrl: g_N at the M control points (outward normal derivative); d_density_out: psi
   (M) or NULL; other arguments as kfbi_solve_bvp.  2-D only.  Synchronising. */
kfbi_status kfbi_solve_neumann_bvp(kfbi_ctx ctx, const double* d_f_grid, const double* d_f_ctrl,
                                   const double* d_gn_ctrl, double* d_u_grid,
                                   double* d_density_out, kfbi_solve_info* h_info, void* stream);

/* Node labels: d_mask[(N+1)^2] = 1 inside Omega, 0 outside.  Asynchronous. */
kfbi_status kfbi_get_inside_mask(kfbi_ctx ctx, uint8_t* d_mask, void* stream);

/* Counts and sizes of the context (host struct).  No device work. */
kfbi_status kfbi_get_info(kfbi_ctx ctx, kfbi_ctx_info* h_info);

/* Sets the precision / restart / tolerance fields used by later kfbi_solve_bvp calls. */
kfbi_status kfbi_set_solver(kfbi_ctx ctx, int precision, int gmres_m, int max_restarts,
                            double tol, double inner_tol);

/* ---------------------------------------------------------------- stage timers
   Per-stage device time (CUDA events recorded on the context's stream around each
   launch of the apply pipeline) and launch counts of every kernel the library issues.
   Stages: 0 setup, 1 correction gather (3-D: jumps and correction), 2 DST rows FP32,
   3 DST columns FP32 (the y-transform pair with the spectral division; in 3-D the
   z-transform pair), 4 DST rows FP64, 5 DST columns FP64, 6 interpolation, 7 dense grid
   build/copy, 8 Krylov vector kernels, 9 residual refinement of FP32 box solves,
   10 tile transposes of the work grid, 11 the sparse first x-transform of the FP32 2-D
   applies (evaluated from the irregular nodes straight into the row layout; the last
   x-transform evaluated at the stencil nodes only is counted in stage 2),
   12 the tensor-core GEMMs of the dense box solve (KFBI_TF32X3), 13 the tridiagonal
   y-solves of the well-conditioned x-modes in the FP32 2-D box solve (with the row-layout
   pass: the whole y-pass, its two streams timed as one span).  Launch counts are always
   kept; times only while profiling is on (enabling clears both). */
#define KFBI_NSTAGES 16
typedef struct {
  double ms[KFBI_NSTAGES];          /* summed device time per stage (0 when not timed) */
  long long launches[KFBI_NSTAGES]; /* kernel launches per stage                      */
  int nstages;                      /* stages in use                                   */
} kfbi_stage_times;

kfbi_status kfbi_profile(kfbi_ctx ctx, int enable);
/* Synchronises the context's stream and returns the totals since the last enable. */
kfbi_status kfbi_profile_read(kfbi_ctx ctx, kfbi_stage_times* h_out);
const char* kfbi_stage_name(int stage);

/* Releases all device memory of the context.  Synchronises its stream first. */
kfbi_status kfbi_destroy(kfbi_ctx ctx);

const char* kfbi_status_string(kfbi_status s);
const char* kfbi_last_error(void);

/* ---------------------------------------------------------------- measurement helper
   No counterpart in the paper: the measured arithmetic peak used as the denominator of
   the ALU rooflines of the transform kernels.  Runs a kernel of independent fused
   multiply-add chains on every SM (FP64 if fp64 != 0, else FP32), three timed launches
   after a warm-up, and writes the best rate in TFLOP/s (2 flops per FMA) to *h_tflops.
   Synchronising on `stream`; allocates nothing. */
kfbi_status kfbi_measure_fma_peak(int fp64, double* h_tflops, void* stream);

/* ---------------------------------------------------------------- batched problems
   Many independent problems (uneven N and M, 2-D or 3-D) solved together: a pool of up
   to 16 host workers, each driving its own CUDA stream, takes problems from a shared queue
   in decreasing order of cost ((N+1)^dim log N; longest first) and solves all right-hand
   sides of a problem in turn, each with the context's own solver options, so up to 16
   problems run concurrently on the device (the environment variable KFBI_BATCH_WORKERS,
   1..64, sets another count; on one GB300, with the Arnoldi steps as CUDA graphs, 16 were
   fastest for the 256-problem workload: 729 ms against 798 ms with 8 and 778 ms with 32).
   Each context is used by one worker at a time: kfbi_batch_create refuses a context
   listed twice (KFBI_ERR_ARG).  The contexts stay owned by the caller and must outlive
   the batch. */
typedef struct kfbi_batch_s* kfbi_batch;

kfbi_status kfbi_batch_create(const kfbi_ctx* ctxs, int count, kfbi_batch* out);

/* Solves count x nrhs BVPs: problem p, right-hand side r uses d_f_grid[p*nrhs + r],
   d_f_ctrl[...], d_g_ctrl[...] and writes d_u_grid[p*nrhs + r] and, when d_density_out
   is not NULL, the boundary density into d_density_out[p*nrhs + r] (M_p values; device
   pointers, layout as in kfbi_solve_bvp; the pointer table itself is a host array).
   h_info: count*nrhs structs or NULL.  The work starts after
   everything already queued on `stream` and is finished when the call returns
   (synchronising).  The first failing solve stops the batch and its status is returned;
   KFBI_ERR_NOT_CONVERGED if some solve hit its iteration limit. */
kfbi_status kfbi_batch_solve(kfbi_batch b, int nrhs, const double* const* d_f_grid,
                             const double* const* d_f_ctrl, const double* const* d_g_ctrl,
                             double* const* d_u_grid, double* const* d_density_out,
                             kfbi_solve_info* h_info, void* stream);

kfbi_status kfbi_batch_destroy(kfbi_batch b);

#ifdef __cplusplus
}
#endif
#endif /* KFBI_H */
