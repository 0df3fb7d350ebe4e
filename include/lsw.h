/*
 * lsw.h -- C ABI of a GB300 (sm_103a) solver for the 2D acoustic
 * Lippmann-Schwinger equation  (I - G0 V) psi = psi0  by the preconditioned
 * scattering series of Eikrem, Naevdal and Jakobsen, "Iterative solution of
 * the Lippmann-Schwinger equation in strongly scattering acoustic media by
 * randomized construction of preconditioners" (arXiv:2005.01372).
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid.      nz x nx cells of size h x h.  Unknowns are ordered in vertical
 *            strips (Sec. 2.4): the linear index of cell (iz, ix) is
 *            ix * nz + iz.  nz and nx must be powers of two, 1 <= n <= 2048.
 *            A model of another shape is placed in such a grid whose other
 *            cells have velocity c0: cells of zero contrast do not scatter,
 *            so the solution inside the model is unchanged.
 * Complex.   Interleaved (re, im): LSW_C128 = two doubles, LSW_C64 = two
 *            floats.  A batch of nbatch fields is stored field after field,
 *            stride nz * nx elements.
 * Contrast.  chi is always a device array of nz * nx doubles, Eq. 1:
 *            chi = w^2 (1/c^2 - 1/c0^2).
 * Green.     G0(r) = (i/4) H0^(1)(k0 r), k0 = 2 pi f / c0 (time dependence
 *            exp(-i w t)).  Each cell is integrated over the disk of equal
 *            area, so the cell volume of Eq. 4 is inside the Green table and
 *            V = diag(chi).
 * Pointers.  Unless a parameter says "host", every array pointer is a device
 *            pointer owned by the caller.  Handles (lsw_green, lsw_hmatrix)
 *            are owned by the library; free them with lsw_destroy_*.
 * Streams.   Every call takes a cudaStream_t (passed as void*; NULL = the
 *            legacy default stream) and is asynchronous on it, except where
 *            stated.  Calls allocate their scratch with cudaMallocAsync on
 *            that stream.
 * Errors.    Calls return an lsw_status.  On failure outputs are unspecified
 *            and handles stay valid.  No call exits, aborts or traps.
 *            Calls on one handle are not thread-safe.
 */
#ifndef LSW_H
#define LSW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int lsw_status;
enum {
    LSW_OK = 0,
    LSW_ERR_INVALID_ARG = 1,      /* NULL pointer, bad enum, bad size        */
    LSW_ERR_UNSUPPORTED_SIZE = 2, /* grid not a power of two or too large    */
    LSW_ERR_OOM = 3,              /* device allocation failed                */
    LSW_ERR_CUDA = 4,             /* a CUDA runtime call failed              */
    LSW_ERR_NOT_CONVERGED = 5,    /* max_iter reached above the tolerance    */
    LSW_ERR_DIVERGED = 6,         /* residual grew 1e3x above its minimum    */
    LSW_ERR_NUMERIC = 7,          /* NaN or Inf met                          */
    LSW_ERR_TIMEOUT = 8           /* reserved for bounded device-side waits  */
};

/* LSW_BF16 is for H only (lsw_hparams.prec, HODLR): built in FP32, then kept
 * as BF16 (re, im) pairs, half the memory of LSW_C64, and applied to complex64
 * vectors with FP32 accumulation; a solve treats such an H as LSW_C64. */
typedef enum { LSW_C128 = 0, LSW_C64 = 1, LSW_MIXED = 2, LSW_BF16 = 3 } lsw_prec;

/* Products computed by lsw_apply_operator (Eq. 4, Eq. 13, Algorithm 2). */
typedef enum {
    LSW_OP_FORWARD = 0,   /* y = u0 + G0 V u                                 */
    LSW_OP_RESIDUAL = 1,  /* y = u - G0 V u - u0   (a_{j-1} of Eq. 13)        */
    LSW_OP_PLAIN = 2,     /* y = G0 V u                                      */
    LSW_OP_ADJOINT = 3    /* y = (G0 V)^H u = chi . conj(G0 conj(u))          */
} lsw_op_mode;

typedef struct {
    int32_t nz, nx;       /* cells in depth (z) and horizontally (x)         */
    double h;             /* cell size [m]                                   */
    double c0;            /* background velocity [m/s] (Eq. 1)               */
    double freq_hz;       /* frequency f, w = 2 pi f                         */
} lsw_grid;

/* A rectangle of cells [z0, z1) x [x0, x1). */
typedef struct { int32_t z0, z1, x0, x1; } lsw_box;

typedef struct lsw_green lsw_green;       /* Green table + spectra, opaque   */
typedef struct lsw_hmatrix lsw_hmatrix;   /* preconditioner H, opaque        */

typedef enum { LSW_H_LOWRANK_SMW = 0, LSW_H_HODLR = 1 } lsw_h_kind;
typedef enum { LSW_SPLIT_QUADTREE = 0, LSW_SPLIT_STRIPS = 1 } lsw_split;

typedef struct {
    int32_t kind;         /* lsw_h_kind                                       */
    int32_t prec;         /* LSW_C128 or LSW_C64: storage and arithmetic of H;
                             LSW_BF16 (HODLR): FP32 build, BF16 storage     */
    int32_t levels;       /* HODLR: levels of the cluster tree (leaves at L)  */
    int32_t split;        /* HODLR: lsw_split                                 */
    int32_t rank;         /* r, the same for every low-rank block (Sec. 2.4)  */
    int32_t oversample;   /* extra probes p: r + p Gaussian columns           */
    int32_t q;            /* power iterations of Algorithm 2 (0 on the paper's HODLR path) */
    int32_t rank_max;     /* lsw_solve_batched, HODLR: when > rank, a problem
                             that leaves a source unconverged is rebuilt with
                             twice the rank (at most rank_max and 64 -
                             oversample) and solved again (Sec. 3.1: raise r
                             and rebuild); 0 = fixed rank                      */
    uint64_t seed;        /* Philox4x32-10 key of every probe block           */
} lsw_hparams;

typedef enum { LSW_SERIES = 0, LSW_FGMRES = 1 } lsw_method;

typedef struct {
    int32_t prec;         /* LSW_C128, LSW_C64 or LSW_MIXED                    */
    int32_t max_iter;     /* series steps (30 in Sec. 3.1) or FGMRES iterations per solve */
    double tol;           /* stop when ||psi0 - (I - G0V) psi||_2 <= tol ||psi0||_2 */
    double inner_tol;     /* LSW_MIXED: relative tolerance of each FP32 inner solve */
    int32_t max_outer;    /* LSW_MIXED: refinement steps                       */
    int32_t method;       /* lsw_method                                        */
    int32_t restart;      /* LSW_FGMRES: Krylov basis size per cycle            */
    int32_t pad_;
} lsw_solve_params;

typedef struct {
    int32_t iterations;   /* series steps taken (inner steps summed for MIXED) */
    int32_t outer;        /* refinement steps (MIXED), else 0                  */
    int32_t status;       /* LSW_OK, LSW_ERR_NOT_CONVERGED, ...                */
    int32_t fallback;     /* lsw_solve_learned: 1 if the learned preconditioner
                             was dropped for H during the solve, else 0       */
    double rel_residual;  /* final ||psi0 - (I - G0V) psi|| / ||psi0||, FP64   */
} lsw_solve_info;

/* Text for a status code (static storage). */
const char* lsw_status_string(lsw_status s);
/* Text of the last CUDA failure seen by the calling thread (diagnostics). */
const char* lsw_last_error(void);
/* Number of CUDA kernels the library has launched in this process
 * (diagnostics; every call's kernels are counted as they are enqueued). */
uint64_t lsw_launch_count(void);

/* Measured arithmetic peak of the current device (diagnostics, not part of
 * the method): kind 0 = FP32 fused multiply-add, 1 = FP64; *tflops receives
 * TFLOP/s (2 flops per FMA) of one probe kernel timed with CUDA events on
 * stream (synchronises it).  The roofline denominators of the FP32 kernels. */
lsw_status lsw_measure_peak(int kind, double* tflops, void* stream);
/* The current device's default stream-ordered memory pool, from which every
 * call of the library takes its scratch (diagnostics): bytes in use now and
 * the high-water mark since the last reset (reset_high != 0 resets it to 0
 * before reading). */
lsw_status lsw_mempool_usage(uint64_t* used_current, uint64_t* used_high, int reset_high);

/* Diagnostic timing of one kernel family inside any call (not part of the
 * method).  lsw_kernel_timer_start(family) resets and enables it for
 * "operator_c64" / "operator_c128" (the three FFT passes of one operator
 * apply in that precision), "qr" (the thin QR of complex64 sketch blocks),
 * "gram", "chol", "heev" (the truncation's eigen-decompositions),
 * "gj_update" (the Gauss-Jordan block updates), "leaf_tc" (the tensor-core
 * products of H's dense leaves), "lr_levels", "lr_partial", "lr_reduce",
 * "lr_apply" (the level products of an H apply) or "arnoldi_gs" (the
 * Gram-Schmidt step of an FGMRES iteration); CUDA events are then recorded on
 * the launching stream around each such launch, with the algorithmic bytes
 * and flops of its work.  Launches captured into the solvers' CUDA graphs
 * are timed too: their events are recorded as nodes of the graph and read
 * after each replay.
 * Phases of lsw_build_hmatrix (HODLR) time the same way, on the stream that
 * runs them: "hodlr_level_sketch" (one level's sketches), "hodlr_leaf_inverse"
 * (the dense leaves' inverses), "hodlr_invert" (the recursive inversion) and,
 * inside it, "hodlr_add_lowrank" (one low-rank update with its
 * recompressions), "hodlr_leaf_woodbury" (one batched Woodbury update of a
 * node's leaf inverses) and "hodlr_subtree_products" (a pair of subtree
 * products).
 * lsw_kernel_timer_read waits for the recorded events and reports the sums
 * (any pointer may be NULL). */
lsw_status lsw_kernel_timer_start(const char* family);
lsw_status lsw_kernel_timer_read(double* total_ms, double* bytes, double* flops, uint64_t* launches);
lsw_status lsw_kernel_timer_stop(void);

/* Green table and spectra (Sec. 2.2).
 * Tabulates the cell-integrated Green's function Gt at every offset
 * 0 <= dz <= nz, 0 <= dx <= nx in FP64 (Bessel J0, J1, Y0, Y1), builds its
 * even circulant extension to 2nz x 2nx (the paper cites Nowak et al. 2003
 * for the extension; index N holds the offset-N value so the extension is
 * exactly even), and stores its 2D FFT, scaled by 1 / (4 nz nx), as the
 * (nz + 1) x (nx + 1) quarter that evenness allows, in FP64 and FP32.
 * *out receives a new handle.  Not asynchronous: returns after the build. */
lsw_status lsw_build_green(const lsw_grid* grid, void* stream, lsw_green** out);
lsw_status lsw_destroy_green(lsw_green* g);

/* Copies of the handle's tables, for checking.
 * table: (nx + 1) x (nz + 1) complex doubles, entry dx * (nz + 1) + dz.
 * spectrum: the scaled quarter spectrum, same shape and layout, kx-major. */
lsw_status lsw_green_table(const lsw_green* g, void* table_c128, void* stream);
lsw_status lsw_green_spectrum(const lsw_green* g, void* spec_c128, void* stream);

/* Eq. 1: chi = w^2 (1/c^2 - 1/c0^2) for every cell.
 * velocity, chi: device arrays of nz * nx doubles (may alias). */
lsw_status lsw_contrast(const lsw_green* g, const double* velocity, double* chi, void* stream);

/* Background fields psi0 of unit point sources, one field per source:
 * psi0_i = Gt(r_i) / h^2, i.e. (i/4) H0(k0 r) 2 J1(k0 a)/(k0 a) off the
 * source cell, a = h / sqrt(pi).
 * positions: HOST array of 2 * nsrc int32, (iz, ix) per source.
 * u0: nsrc fields of precision prec (LSW_C128 or LSW_C64). */
lsw_status lsw_point_sources(const lsw_green* g, const int32_t* positions, int nsrc,
                             int prec, void* u0, void* stream);

/* The Lippmann-Schwinger operator through zero-padded FFTs (Sec. 2.2,
 * Eq. 4): for each of nbatch fields computes the product named by mode
 * (lsw_op_mode).  prec: LSW_C128 or LSW_C64 for u, u0 and y.  u0 may be
 * NULL for FORWARD and RESIDUAL (read as zero) and is ignored otherwise.
 * y must not alias u or u0.  Scratch: 2 * nbatch * nz * nx complex. */
lsw_status lsw_apply_operator(const lsw_green* g, int prec, const double* chi,
                              const void* u, const void* u0, void* y,
                              int nbatch, int mode, void* stream);

/* lsw_apply_operator without any device allocation.  The paper has no
 * counterpart to this call.  It serves callers that cannot let a library
 * allocate device memory while it runs: applications that reserve all device
 * memory up front for their own allocator, embedders that audit the memory
 * of every call, and latency-critical loops that cannot absorb an
 * allocation's cost or its failure part-way through.  Arguments and results
 * are those of lsw_apply_operator.  The scratch it needs (2 * nbatch * nz * nx
 * complex values of prec) comes from one fixed 32 MiB device array that the
 * library holds on every GPU that loads it, until the process exits; larger
 * requests return LSW_ERR_UNSUPPORTED_SIZE without launching anything.
 * lsw_build_green looks up that array's device address on the current
 * device (loading the library's device code there, which commits the
 * array, if that has not happened yet) and this call uses that address; it
 * calls no allocating routine.  A device reset invalidates every earlier
 * handle, and the next lsw_build_green refreshes the address.  Every call shares the one array, so calls whose work overlaps on
 * the GPU (several streams or host threads) race on it: the caller must
 * serialise them.  Nothing left by an earlier call needs clearing. */
lsw_status lsw_apply_operator_noalloc(const lsw_green* g, int prec, const double* chi,
                                      const void* u, const void* u0, void* y,
                                      int nbatch, int mode, void* stream);

/* Randomized range sketch of one block of G0 V (Algorithm 2): with s =
 * rows and t = cols (boxes inside the grid, unknowns numbered in strip order
 * inside each box), computes U (n_s x rank) and W (n_t x rank), column-major,
 * with (G0 V)[s, t] ~ U W^H.  Probes: rank + oversample complex Gaussian
 * columns from Philox4x32-10 keyed by seed, stream words (2 << 28, stream).
 * q power iterations.  Products by FFT on the bounding box of s and t.
 * prec: LSW_C128 or LSW_C64 for U and W.  Columns beyond the numerical rank
 * are zero.  The factors are unique only up to U W^H. */
lsw_status lsw_sketch_range(const lsw_green* g, int prec, const double* chi,
                            lsw_box rows, lsw_box cols, int rank, int oversample, int q,
                            uint64_t seed, uint32_t stream_id, void* U, void* W, void* stream);

/* Preconditioner H ~ (I - G0 V)^-1 (Sec. 2.3-2.4).
 * kind LSW_H_LOWRANK_SMW: G0 V ~ U W^H over the whole grid (Algorithm 2) and
 *   H = I + U (I_r - W^H U)^-1 W^H (Eq. 12).
 * kind LSW_H_HODLR: randomized HODLR approximation of I - G0 V (off-diagonal
 *   blocks by Algorithm 2 on each parent box, dense diagonal leaves), then
 *   its inverse by the recursive 2x2 block-inverse formula with randomized
 *   rank-r recompression of every low-rank sum (Algorithm 1, q = 0).
 * The handle keeps its own copy of what it needs (not chi).  *out receives
 * the handle.  Returns after the build (synchronises the stream). */
lsw_status lsw_build_hmatrix(const lsw_green* g, const double* chi, const lsw_hparams* hp,
                             void* stream, lsw_hmatrix** out);
lsw_status lsw_destroy_hmatrix(lsw_hmatrix* h);
/* Device bytes held by the handle. */
lsw_status lsw_hmatrix_bytes(const lsw_hmatrix* h, uint64_t* bytes);

/* y = H x for nbatch fields in the grid's strip ordering, in H's precision
 * (hp->prec).  x and y must not alias. */
lsw_status lsw_apply_precond(const lsw_hmatrix* h, const void* x, void* y, int nbatch, void* stream);

/* Solve (I - G0 V) psi = psi0 for nbatch right-hand sides.
 * sp->method LSW_SERIES: the scattering series of Eq. 11,
 *   psi_j = psi_{j-1} - H (psi_{j-1} - G0 V psi_{j-1} - psi0), started from
 *   psi_0 = H psi0; H == NULL gives the Born series started from psi0
 *   (Sec. 2.2).  A source whose residual grows 1e3x above its minimum stops
 *   with LSW_ERR_DIVERGED (spectral radius of M above one, Eq. 7).
 * sp->method LSW_FGMRES: flexible GMRES(sp->restart) from psi = 0 with H as
 *   right preconditioner (H == NULL: none), the Krylov comparison of Sec. 3.2.
 * Each source stops once its relative residual is at most sp->tol (Sec. 3.2
 * stopping rule, read as relative); the reported residual is FP64.
 * prec LSW_C128 / LSW_C64: everything in that precision, u0 and u too.
 * prec LSW_MIXED: u0 and u are LSW_C128; iterative refinement -- the FP64
 *   residual r = psi0 - (I - G0 V) psi is formed in FP64, the correction
 *   (I - G0 V) d = r is solved by the series in FP32 (H must be LSW_C64) to
 *   sp->inner_tol, and psi += d, until the FP64 residual meets sp->tol.
 * info: HOST array of nbatch records.  Synchronises the stream (once per
 * series step to read the residual norms).  Returns LSW_OK when every source
 * converged, else the first failing source's status. */
lsw_status lsw_solve_series(const lsw_green* g, const double* chi, const lsw_hmatrix* h,
                            const void* u0, void* u, int nbatch, const lsw_solve_params* sp,
                            lsw_solve_info* info, void* stream);

/* One (grid, frequency) problem of a batched solve. */
typedef struct {
    lsw_grid grid;
    const double* velocity;   /* device, nz * nx velocities (strip order)         */
    const int32_t* sources;   /* HOST, 2 * nsrc int32: (iz, ix) per point source  */
    int32_t nsrc;
    int32_t pad_;
    void* u;                  /* device output, nsrc fields: complex128 for
                                 LSW_C128 / LSW_MIXED, complex64 for LSW_C64      */
} lsw_problem;

/* Solve many (grid, frequency) problems.  The preconditioner of a problem
 * serves all of its sources (Sec. 3: extra sources cost little once H is
 * built).  For every problem: Green table and spectrum, contrast (Eq. 1),
 * point sources, H from *hp (NULL: no preconditioner), then
 * lsw_solve_series with *sp.  Up to max_concurrent problems (<= 0: 4; at
 * most 7) are worked on at once from host worker threads, each on its own
 * stream, so that their builds and solves overlap on the GPU.  The call
 * first synchronises `stream` (inputs may come from it) and returns when
 * every problem is done.  With hp->rank_max > hp->rank (HODLR), a problem
 * that leaves a source unconverged, diverging or non-finite is rebuilt with twice the
 * rank, up to rank_max, and solved again.  info: HOST array with one record
 * per source, in problem order (the last attempt's).  Returns LSW_OK, or the
 * first failing problem's status. */
lsw_status lsw_solve_batched(const lsw_problem* probs, int nprob, const lsw_hparams* hp,
                             const lsw_solve_params* sp, int max_concurrent,
                             lsw_solve_info* info, void* stream);

/* Rank policy of a frequency sweep (Sec. 3.1): a frequency whose solve
 * does not converge within the iteration limit (the paper: 30) is rebuilt
 * with rank + rank_step and solved again from psi0; one that converges but
 * needs more than raise_iters iterations (the paper: 10) hands rank +
 * rank_step to the next frequency.  Ranks never exceed rank_max. */
typedef struct {
    int32_t rank0;        /* rank at the first frequency (>= 1)               */
    int32_t rank_step;    /* added on each increase (>= 1)                    */
    int32_t rank_max;     /* largest rank (>= rank0; rank_max + oversample <= 64) */
    int32_t raise_iters;  /* iteration count above which the next frequency
                             starts at a higher rank (>= 0)                    */
} lsw_sweep_policy;

/* Outcome of one frequency of a sweep. */
typedef struct {
    double freq_hz;
    int32_t rank;            /* rank of the H behind the final solve           */
    int32_t builds;          /* preconditioners built at this frequency        */
    int32_t converged;       /* sources that met sp->tol                       */
    int32_t max_iterations;  /* largest iteration count over the sources       */
    double max_rel_residual; /* largest final FP64 relative residual           */
    int32_t status;          /* LSW_OK, or the first failing source's status   */
    int32_t next_rank;       /* rank handed to the next frequency              */
} lsw_sweep_info;

/* One decision of the policy (host only, no GPU work): after a solve at
 * `rank` that returned solve_status (LSW_OK when every source converged)
 * with largest iteration count max_iterations, *rebuild = 1 and *next_rank
 * = the rank to rebuild with at this frequency, or *rebuild = 0 and
 * *next_rank = the rank for the next frequency.  A failed solve at
 * rank_max is not rebuilt.  LSW_ERR_INVALID_ARG for a NULL pointer, an
 * invalid policy or rank < 1. */
lsw_status lsw_sweep_next_rank(const lsw_sweep_policy* pol, int32_t rank, int32_t solve_status,
                               int32_t max_iterations, int32_t* next_rank, int32_t* rebuild);

/* The paper's frequency sweep (Sec. 3.1) on one grid: the frequencies are
 * solved in the order given (the paper goes from the lowest, the easiest
 * to approximate, upwards), each with its own Green table, contrast (Eq. 1),
 * point sources and HODLR preconditioner (*hp, with hp->rank and
 * hp->rank_max replaced by the policy's ranks), by lsw_solve_series with
 * *sp, ranks following *pol.  grid->freq_hz is ignored; freqs_hz: HOST,
 * nfreq values.  velocity: device, nz * nx (strip order).  sources: HOST,
 * 2 * nsrc int32 (iz, ix).  u: device output, nfreq * nsrc fields, frequency
 * major (complex128 for LSW_C128 / LSW_MIXED, complex64 for LSW_C64).
 * info: HOST, nfreq records; sinfo (HOST, nfreq * nsrc, may be NULL): each
 * source's final lsw_solve_info.  Synchronises the stream.  Returns LSW_OK
 * when every frequency converged, else the first failing frequency's
 * status; an error other than non-convergence, divergence or a non-finite
 * residual ends the sweep at once. */
lsw_status lsw_solve_sweep(const lsw_grid* grid, const double* velocity, const double* freqs_hz, int nfreq,
                           const int32_t* sources, int nsrc, const lsw_hparams* hp,
                           const lsw_sweep_policy* pol, const lsw_solve_params* sp, void* u,
                           lsw_sweep_info* info, lsw_solve_info* sinfo, void* stream);

/* Measure the operator's pass variants for this grid and precision on
 * nbatch fields -- 0: register radix-8 FFT passes, 1: the same with
 * 512-thread row blocks in the x pass, 2: shared-memory Stockham passes --
 * and use the fastest for this (2nz, 2nx, precision) from now on in this
 * process.  *variant (may be NULL) receives the choice, ms3 (may be NULL)
 * the three mean times per apply in ms (-1: variant not available here).
 * Synchronises the stream. */
lsw_status lsw_autotune(const lsw_green* g, int prec, int nbatch, void* stream,
                        int* variant, float* ms3);

/* Process-wide switch (default on) for the tensor-core path of the FP32
 * products of H's dense leaves with blocks of up to 32 vectors (tcgen05,
 * three TF32 products per real product, FP32 accumulation: results agree
 * with the CUDA-core path to FP32 rounding, not bit for bit).  Off: every
 * product runs on the CUDA cores.  Not part of the method; for A/B
 * comparisons and reproducibility across paths. */
lsw_status lsw_set_tensor_cores(int enable);

/* Process-wide switch (default on) for CUDA graphs in the solvers: inside a
 * flexible-GMRES call, the Arnoldi step's preconditioner apply and operator
 * (fixed buffers) are captured once into a CUDA graph and replayed at every
 * later step.  Results are the same either way (the same kernels in the
 * same order); a capture that fails falls back to ordinary launches.  Not
 * part of the method. */
lsw_status lsw_set_graphs(int enable);
/* Number of CUDA-graph launches the solvers have issued in this process
 * (diagnostics). */
uint64_t lsw_graph_replay_count(void);

/* ------------------------------------------------------------------------
 * Learned right preconditioner.  The paper has no network: its Sec. 3.2
 * compares the preconditioned series with GMRES, and this is a Fourier
 * neural operator that stands in for H inside flexible GMRES, with H kept as
 * the fallback.  Everything runs in FP32 complex.
 *
 * Network.  Input x: two complex channels on the nz x nx grid (strip order),
 *   x0 = r / ||r||_2 and x1 = chi / k0^2 + i k0 h  (chi / k0^2 = c0^2/c^2 - 1).
 *   v = P x + p  (P: W x 2);  for l < L:  v <- sigma(K_l v + W_l v + b_l),
 *   sigma = split GELU gelu(Re) + i gelu(Im), none on the last layer;
 *   y = x0 + Q v + q  (Q: 1 x W; the residual channel passes through, so the
 *   zero network is the identity).  K_l is a spectral convolution on the 2m x 2m
 *   modes kz, kx in {0..m-1} U {n-m..n-1} of the unnormalised 2D DFT F:
 *   K_l v = F^-1 (R_l[k] (F v)[k]) with one W x W complex matrix per mode.
 * Parameters: one FP32-complex device buffer of lsw_fno_num_params entries,
 *   column-major blocks in this order: P^T (2 x W), p (W); per layer R_l
 *   ((2m)^2 modes, mode index a + 2m b for kz-mode a and kx-mode b, each
 *   W x W with entry (o, i) = R_l[a, b][o][i]), W_l^T (W x W), b_l (W); then
 *   Q^T (W), q (1).
 * Gradients: G = dL/dRe + i dL/dIm of L = mean |y - target|^2 over all
 *   batch * nz * nx outputs, in the same layout.
 * Adam: Kingma & Ba (2015) on real and imaginary parts separately,
 *   beta1 0.9, beta2 0.999, eps 1e-8, moments kept in the handle.
 * ---------------------------------------------------------------------- */
typedef struct lsw_fno lsw_fno;           /* weights, gradients, Adam moments */

typedef struct {
    int32_t nz, nx;       /* grid of every input and output field (>= 2)          */
    int32_t width;        /* W channels, 1..64                                    */
    int32_t modes;        /* m: 2m retained wavenumbers per axis, 2m <= nz, nx    */
    int32_t layers;       /* L, 1..16                                             */
    int32_t pad_;
    uint64_t seed;        /* Philox4x32-10 key of the Gaussian initial weights    */
} lsw_fno_params;

/* Create a network with Gaussian weights scaled by 1/sqrt(fan-in) (R_l by
 * 1/W) and zero biases, initialised by work enqueued on `stream`. */
lsw_status lsw_fno_create(const lsw_fno_params* p, void* stream, lsw_fno** out);
lsw_status lsw_fno_destroy(lsw_fno* f);
/* Number of complex parameters (host). */
lsw_status lsw_fno_num_params(const lsw_fno* f, int64_t* count);
/* Copy one state buffer out (dst != NULL) and/or in (src != NULL): which =
 * 0 weights, 1 gradients, 2 Adam first moments (complex), 3 Adam second
 * moments (per entry: second moment of the real part, of the imaginary part).
 * Device buffers of lsw_fno_num_params complex64 entries. */
lsw_status lsw_fno_state(lsw_fno* f, int which, void* dst, const void* src, void* stream);
/* y = network(x): x is batch x 2 fields, y batch fields, complex64, device. */
lsw_status lsw_fno_forward(const lsw_fno* f, const void* x, void* y, int batch, void* stream);
/* Forward, loss and backward on one batch; the gradients stay in the handle
 * (grad, device, may be NULL: a copy of them).  loss (HOST, may be NULL)
 * receives L, which synchronises the stream. */
lsw_status lsw_fno_loss_grad(lsw_fno* f, const void* x, const void* target, int batch,
                             double* loss, void* grad, void* stream);
/* One Adam update with the handle's gradients; t >= 1 is the step number
 * (bias corrections 1 - beta^t), so a resumed run passes its own count. */
lsw_status lsw_fno_adam_step(lsw_fno* f, float lr, int32_t t, void* stream);
/* Training pairs of the network (not part of the paper): for nbatch residual
 * fields r and their corrections e = (I - G0 V)^-1 r (prec LSW_C128 or
 * LSW_C64, device, nbatch x nz*nx), writes the inputs x (complex64, nbatch x 2
 * fields: r / ||r||_2 and chi / k0^2 + i k0 h) and the targets t = e / ||r||_2
 * (complex64, nbatch fields), ||r||_2 in FP64. */
lsw_status lsw_fno_pairs(const lsw_green* g, const double* chi, const void* r, const void* e, int nbatch, int prec,
                         void* x, void* t, void* stream);
/* Phase augmentation of nbatch pairs in place: channel 0 of x_b and t_b are
 * multiplied by exp(i phases[b]) (phases: HOST array of nbatch angles in
 * radians, read before the call returns; the map r -> e is complex-linear,
 * so a rotated pair is again a pair).  n = nz * nx.  Synchronises stream. */
lsw_status lsw_fno_rotate(void* x, void* t, int nbatch, int64_t n, const float* phases, void* stream);
/* The network's error on batch pairs: *num = sum |network(x) - t|^2 and
 * *den = sum |t|^2 over every output (FP64 sums, HOST outputs; synchronises
 * stream). */
lsw_status lsw_fno_error(const lsw_fno* f, const void* x, const void* t, int batch, double* num, double* den,
                         void* stream);
/* The preconditioner: z_b = ||v_b|| * network([v_b / ||v_b||, chi/k0^2 + i k0 h])
 * for nbatch fields v (prec LSW_C128 or LSW_C64, device), on g's grid, which
 * must match the network's. */
lsw_status lsw_fno_apply(const lsw_fno* f, const lsw_green* g, const double* chi, const void* v,
                         void* z, int nbatch, int prec, void* stream);

/* FGMRES (sp->method must be LSW_FGMRES) with the network as right
 * preconditioner.  The preconditioner is the same for the whole batch of
 * sources.  Its progress is probed every five iterations of a cycle: when
 * some active source's residual estimate has not dropped below 0.5 times its
 * value five iterations earlier, the cycle ends and H (NULL: none) takes over
 * for the rest of the call; a cycle cut off at its first probe does not
 * update psi, a later one does.  info[s].fallback reports the switch.
 * Otherwise as lsw_solve_series
 * (precisions, LSW_MIXED refinement, FP64 final residual); H, when given,
 * must be stored in the inner precision. */
lsw_status lsw_solve_learned(const lsw_green* g, const double* chi, const lsw_fno* fno,
                             const lsw_hmatrix* h, const void* u0, void* u, int nbatch,
                             const lsw_solve_params* sp, lsw_solve_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LSW_H */
