/*
 * laph.h -- C ABI of the GB300 (sm_103a) LapH block-contraction library.
 *
 * The library computes the meson and baryon "blocks" of the Laplacian-
 * Heaviside (LapH) method.  Paper (arXiv:2510.26313), section "Innovations",
 * subsection "QUDA": the LapH eigenvectors are needed to form
 * quark-antiquark doublets and three-quark triplets for the Wick
 * contractions of meson and baryon sources and sinks in temporal
 * correlators; section "Current state-of-the-art" introduces LapH smearing
 * and its stochastic variant, whose smeared quark sinks are also valid
 * inputs.  For every timeslice t and integer momentum n_p (p = 2 pi n_p/L):
 *
 *   ph_p(x)        = exp(-2 pi i ((n_p . x) mod L) / L)
 *   B[t][p][i,j,k] = sum_x ph_p(x) eps_abc phi_i^a(x) phi_j^b(x) phi_k^c(x)
 *   M[t][p][i][j]  = sum_x ph_p(x) sum_a conj(phi_i^a(x)) phi_j^a(x)
 *
 * Conventions (readings where the paper is silent):
 *   - site index x = x0 + L*x1 + L*L*x2, x0 fastest, origin 0, periodic;
 *   - no 1/V normalisation; B has no conjugation; M conjugates its first index;
 *   - B is fully antisymmetric, so only i<j<k is stored, at the "colex"
 *     index C(k,3) + C(j,2) + i (independent of N);
 *   - the momentum argument is reduced mod L exactly in integers before the
 *     FP64 sine/cosine.
 *
 * Memory layouts (complex numbers interleaved re,im):
 *   phi   complex64  [T][N][L^3][3]      device, 8-byte aligned
 *   B     complex128 [T][P][C(N,3)]      device
 *   M     complex128 [T][P][N][N]        device
 *   momenta int32    [P][3]              HOST, units of 2 pi / L
 *
 * Ownership: the caller owns every buffer it passes.  Plans own the device
 * memory they allocate at creation (phase tables, tile tables, status word)
 * and free it in laph_plan_destroy.  laph_plan_execute allocates nothing.
 *
 * Errors: every function returns LAPH_OK (0) or a negative laph status; no
 * C++ exception crosses this boundary.  Argument checks happen before any
 * launch.  Faults detected on the device (a bounded wait that expired, a
 * failed index check) are recorded in the plan's status word and read with
 * laph_get_device_status.
 *
 * Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 * default stream).  All work is stream-ordered.
 */
#ifndef LAPH_H
#define LAPH_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LAPH_API __attribute__((visibility("default")))
#else
#define LAPH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define LAPH_OK 0
#define LAPH_ERR_ARG (-1)         /* invalid argument (null, size, alignment, momentum) */
#define LAPH_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define LAPH_ERR_WORKSPACE (-3)   /* workspace missing, too small or misaligned */
#define LAPH_ERR_UNSUPPORTED (-4) /* mode or shape not supported on this device */
#define LAPH_ERR_TIMEOUT (-5)     /* a bounded device wait expired (kernel returned early) */
#define LAPH_ERR_DEVICE (-6)      /* a device-side index/consistency check failed */

/* ---- precision modes of the contraction ------------------------------ */
/* FP32 CUDA-core path: FP32 products and partial sums, FP64 site reduction. */
#define LAPH_MODE_FP32_SIMT 0
/* tcgen05 tensor cores, each operand split into hi+lo FP16 after an exact
 * power-of-two rescale; products hi*hi + hi*lo + lo*hi accumulated in FP32 in
 * tensor memory, drained every 128 sites (the plan's chunk_sites) into FP32
 * running sums with round-to-nearest over a block of sites (the plan's
 * sum_sites, 8192 by default); the FP32
 * partials of the blocks are then summed in FP64, in block order, and
 * scaled back into the complex128 output. */
#define LAPH_MODE_TC_F16X3 1
/* as above with BF16 hi+lo. */
#define LAPH_MODE_TC_BF16X3 2
/* single-term FP16 / BF16 tensor-core products (hi*hi only); reduced accuracy. */
#define LAPH_MODE_TC_F16 3
#define LAPH_MODE_TC_BF16 4
#define LAPH_NUM_MODES 5

/* ---- plan flags ------------------------------------------------------ */
#define LAPH_PLAN_SKIP_B 0x1u   /* do not compute baryon blocks (out_B may be NULL) */
#define LAPH_PLAN_SKIP_M 0x2u   /* do not compute meson blocks (out_M may be NULL) */
#define LAPH_PLAN_AUTOTUNE 0x4u /* pick the tensor-core schedule by timing candidates at creation */
/* Record CUDA events around every contraction-kernel launch (see
 * laph_plan_kernel_times). */
#define LAPH_PLAN_TIMING 0x8u
/* Test hook: one producer warp of the tensor-core kernel skips an arrive, so
 * the consumer's bounded wait expires and LAPH_ERR_TIMEOUT is recorded. */
#define LAPH_PLAN_DEBUG_STALL 0x10000u
/* Test hook: every (instance, timeslice) becomes its own chunk of the
 * tensor-core path, so that small batches exercise the chunked execution. */
#define LAPH_PLAN_CHUNK_PER_TIMESLICE 0x20000u
/* Instances of several fields (stochastic-LapH quark sinks; same passage of
 * the paper: doublets and triplets of colour vectors for the sources and
 * sinks), run with laph_plan_execute_fields.  Together with exactly one of:
 *   LAPH_PLAN_SKIP_M  three-field triplets, dense, no symmetry:
 *       B3[t][p][i][j][k] = sum_x ph_p(x) eps_abc phi_i^a(x) psi_j^b(x) chi_k^c(x)
 *       out_B: device complex128 [T][P][N][N][N];
 *   LAPH_PLAN_SKIP_B  two-field doublets:
 *       M2[t][p][i][j] = sum_x ph_p(x) sum_a conj(phi_i^a(x)) psi_j^a(x)
 *       out_M: device complex128 [T][P][N][N].
 * Tensor-core modes only (LAPH_ERR_UNSUPPORTED otherwise); N >= 1. */
#define LAPH_PLAN_FIELDS 0x40000u
/* Tensor-core modes: outputs (B, M, B3, M2, device or host) are complex64
 * instead of complex128, the FP64 site sums rounded once to FP32 (half the
 * output bytes; the rounding adds a relative error of at most 2^-24 per
 * component).  LAPH_ERR_UNSUPPORTED in the FP32 mode, which accumulates in
 * its complex128 outputs. */
#define LAPH_PLAN_OUT_C64 0x80000u

/* One independent problem of a (possibly ragged) batch. */
typedef struct {
    int L;                  /* spatial extent, V = L^3 sites */
    int T;                  /* timeslices */
    int N;                  /* colour vectors per timeslice */
    int n_mom;              /* number of momenta P */
    const int32_t *momenta; /* host [n_mom][3]; copied at plan creation */
    int n_col;              /* doublet plans (LAPH_PLAN_FIELDS | LAPH_PLAN_SKIP_B): vectors of the second
                               field psi, which may differ from N (projections); 0 means N.  Must be 0 (or N)
                               for every other plan. */
} laph_instance;

typedef struct laph_plan laph_plan;

/* ---- utilities -------------------------------------------------------- */

/* Packed position of B[i,j,k], i<j<k: C(k,3) + C(j,2) + i.  -1 if not i<j<k. */
LAPH_API int64_t laph_triple_index(int i, int j, int k);

/* Static text for a status code. */
LAPH_API const char *laph_status_string(int status);

/* Text of the last failed CUDA call on this thread ("" if none). */
LAPH_API const char *laph_last_cuda_error(void);

/* Library ABI version (major*10000 + minor*100 + patch).  1.1 added the
 * fields laph_plan_options.chunk_sites_b, laph_tune_record.chunk_sites_b and
 * laph_lanczos_stats.host_steps (the structs grew at their ends), the flag
 * LAPH_PLAN_OUT_C64 and laph_plan_drain_sites; a caller built against 1.0
 * passes structs that are too small for a 1.1 library. */
LAPH_API int laph_version(void);

/* ---- K-a: momentum phase table --------------------------------------- */
/* out: device complex128 [n_mom][L^3], out[p][x] = ph_p(x) computed in FP64
 * (integer (n_p.x) mod L, then sincospi).  Momentum projection of the
 * sources/sinks (paper section "Innovations"/"QUDA").  Returns LAPH_ERR_ARG
 * for L < 1, n_mom < 1 or null pointers. */
LAPH_API int laph_phase_table(int L, const int32_t *momenta, int n_mom, void *out, void *stream);

/* ---- K-b: diquark stage, materialised -------------------------------- */
/* D[t][q][x][c] = eps_cab phi_i^a(x) phi_j^b(x) = (phi_i(x) x phi_j(x))_c
 * for every pair i<j, q = C(j,2) + i (the doublet/triplet building block of
 * section "Innovations"/"QUDA").  phi: device complex64 [T][N][L^3][3];
 * out: device complex64 [T][C(N,2)][L^3][3].  The contraction kernels fuse
 * this stage and never write D; this entry point exists for callers that
 * want D itself.  LAPH_ERR_ARG for N < 2, L < 1, T < 1, null or misaligned
 * pointers. */
LAPH_API int laph_diquarks(const void *phi, int L, int T, int N, void *out, void *stream);

/* ---- K-g: dense antisymmetric fill ------------------------------------ */
/* dense[t][p][a][b][c] = sign(sort permutation) * B[t][p][sorted(a,b,c)],
 * 0 where two indices coincide.  packed: device complex128 [T][P][C(N,3)];
 * dense: device complex128 [T][P][N][N][N]. */
LAPH_API int laph_baryon_dense(const void *packed, int T, int N, int n_mom, void *dense, void *stream);

/* ---- simple entry points ----------------------------------------------- */
/* Baryon blocks of one instance: out = B, device complex128 [T][P][C(N,3)].
 * Creates a temporary plan (device allocations), runs it on `stream`,
 * synchronises the stream and frees the plan: blocking and not graph-
 * capturable; use the plan API for that.  mode: LAPH_MODE_*.  Errors: as
 * laph_plan_create / laph_plan_execute, plus the device status. */
LAPH_API int laph_baryon_blocks(const void *phi, int L, int T, int N, const int32_t *momenta, int n_mom, void *out,
                       int mode, void *stream);

/* Meson blocks of one instance: out = M, device complex128 [T][P][N][N].
 * Same behaviour as laph_baryon_blocks. */
LAPH_API int laph_meson_blocks(const void *phi, int L, int T, int N, const int32_t *momenta, int n_mom, void *out,
                      int mode, void *stream);

/* Three-field triplets of one instance (LAPH_PLAN_FIELDS | LAPH_PLAN_SKIP_M):
 * out = B3, device complex128 [T][P][N][N][N]; phi, psi, chi device
 * complex64 [T][N][L^3][3].  Same behaviour as laph_baryon_blocks. */
LAPH_API int laph_triplet_blocks(const void *phi, const void *psi, const void *chi, int L, int T, int N,
                                 const int32_t *momenta, int n_mom, void *out, int mode, void *stream);

/* Two-field doublets of one instance (LAPH_PLAN_FIELDS | LAPH_PLAN_SKIP_B):
 * out = M2, device complex128 [T][P][N][N]. */
LAPH_API int laph_doublet_blocks(const void *phi, const void *psi, int L, int T, int N, const int32_t *momenta,
                                 int n_mom, void *out, int mode, void *stream);

/* Projection of Ns vectors s onto Nv vectors v (paper, section "Innovations",
 * subsection "Eigenvector Projection": inner products of solution vectors
 * with the LapH eigenvectors), with momentum phases:
 *   out[t][p][i][j] = sum_x ph_p(x) sum_a conj(v_i^a(x)) s_j^a(x),
 * the inner products <v_i, s_j> for the single momentum n = 0.
 * v: device complex64 [T][Nv][L^3][3]; s: device complex64 [T][Ns][L^3][3];
 * out: device complex128 [T][P][Nv][Ns].  A doublet plan with n_col = Ns;
 * same behaviour as laph_baryon_blocks.  LAPH_ERR_ARG for Nv < 1, Ns < 1,
 * Nv > 3 L^3 and the conditions of laph_plan_create. */
LAPH_API int laph_projection(const void *v, const void *s, int L, int T, int Nv, int Ns, const int32_t *momenta,
                             int n_mom, void *out, int mode, void *stream);

/* ---- LapH eigenvectors: the 3-d gauge-covariant Laplacian and a batched
 * Lanczos eigensolver (paper, section "Innovations", subsection "Scalable
 * Lanczos Eigensolver"; the timeslices are independent problems) ---------- */
/*   (-Delta f)(x) = sum_mu [ 2 f(x) - U_mu(x) f(x + mu) - U_mu(x - mu)^dagger f(x - mu) ]
 * over the three spatial directions, periodic.  U: device complex64
 * [T][3][L^3][3][3] (row-major SU(3) colour matrices per direction and site);
 * f, out: device complex64 [T][nvec][L^3][3], 8-byte aligned.  Asynchronous
 * on `stream`, no allocation.  LAPH_ERR_ARG for L < 2 or L > 1024, T or nvec
 * outside [1, 65535], null or misaligned pointers. */
LAPH_API int laph_laplacian(const void *U, const void *f, void *out, int L, int T, int nvec, void *stream);

typedef struct {
    int n_krylov;     /* Lanczos steps m, n_ev <= m <= min(4096, 3 L^3) */
    int cheb_degree;  /* 0: Lanczos on -Delta; d > 0: on the Chebyshev filter T_d((-Delta - c) / e),
                         which maps [cheb_lo, 12] onto [-1, 1] and magnifies the eigenvalues below cheb_lo */
    double cheb_lo;   /* 0 < cheb_lo < 12 when cheb_degree > 0: above the wanted eigenvalues */
    uint32_t seed;    /* start vectors (0: a fixed default) */
    int ts_group;     /* timeslices whose filter steps run back to back, so that their links and vectors stay
                         in L2 across the steps (0: as many as fill about 70% of the L2); d > 0 only */
    int pdl;          /* 1: filter steps launched as programmatic dependents of their predecessors */
    int link_rows;    /* 2: read SU(3) links as their first two rows, the third rebuilt (used only if every
                         link is SU(3) to FP32 accuracy); 3: all three rows; 0: two rows unless the filter
                         groups fit in L2 */
} laph_lanczos_params;

/* Where the time of one laph_lanczos call goes, from CUDA events recorded on
 * its stream: the whole call; the setup (workspace, start vectors); the
 * applications of -Delta (or of the filter); the orthogonalisation with the
 * norm and the Lanczos coefficients of each new basis vector; the Ritz
 * vectors, Rayleigh quotients and residuals (with the read-back of the
 * coefficients and the host tridiagonal solver).  Launches of this
 * library's kernels, of which the Laplacian launches (each over one filter
 * group of timeslices, or all T without a filter, one vector each). */
typedef struct {
    double total_ms;
    double setup_ms;
    double apply_ms;
    double orth_ms;
    double ritz_ms;
    int64_t launches;
    int64_t apply_launches;
    int links_two_rows; /* 1: the solver read its copy of the links as two rows (requested or chosen,
                           and every link SU(3) to FP32 accuracy: third row within 2e-6 of
                           conj(row0 x row1)) */
    int ts_group;       /* timeslices per filter group used (T without a filter) */
    int host_steps;     /* 1: a timeslice met an invariant subspace, so the Krylov steps ran a second time with
                           the host reading the coefficients after every step (the figures above cover both runs) */
} laph_lanczos_stats;

/* Bytes of device workspace laph_lanczos needs (about 8 T 3 L^3 (n_krylov +
 * n_ev + 15) bytes: the basis, the Ritz vectors, scratch vectors and a copy
 * of the links in the solver's layout). */
LAPH_API int laph_lanczos_workspace_size(int L, int T, int n_ev, const laph_lanczos_params *params, size_t *bytes);

/* The n_ev lowest eigenpairs of -Delta on every timeslice: Lanczos with full
 * reorthogonalisation (two Gram-Schmidt passes; FP32 vectors, inner products
 * summed in FP32 within a warp and in FP64 across warps and blocks) on -Delta
 * or its Chebyshev filter, Ritz vectors, then Rayleigh quotients and residuals
 * with -Delta.  U as for laph_laplacian.  evecs: device complex64 [T][n_ev][L^3][3], unit norm; evals, resid:
 * HOST double [T][n_ev], ascending eigenvalues and |(-Delta) v - lambda v|
 * (resid may be NULL); stats (may be NULL) receives the timings above.
 * workspace: device memory of laph_lanczos_workspace_size bytes, 256-byte
 * aligned (workspace_bytes its size), or NULL to have the call allocate it on
 * `stream` and free it before returning.  The Krylov steps run without host
 * synchronisation: the coefficients stay on the device and are read back
 * once, after the last step.  If a timeslice met an invariant subspace (its
 * new vector vanished), the steps run again from the same start vectors with
 * the stream synchronised after every step, so that the host can give that
 * timeslice a fresh vector (stats->host_steps).  Blocks until done.  LAPH_ERR_ARG for bad parameters
 * (2 <= L <= 512, 1 <= T <= 65535, n_ev <= n_krylov, the bounds on n_krylov
 * and the filter above, ts_group < 0, link_rows other than 0, 2, 3), for
 * null or misaligned (8-byte) pointers and when the host tridiagonal solver does not converge,
 * LAPH_ERR_WORKSPACE for a workspace too small or misaligned. */
LAPH_API int laph_lanczos(const void *U, int L, int T, int n_ev, const laph_lanczos_params *params, void *evecs,
                          double *evals, double *resid, void *workspace, size_t workspace_bytes,
                          laph_lanczos_stats *stats, void *stream);

/* Host utility: eigenvalues (ascending, in d) and orthonormal eigenvectors
 * (z, n x n row-major, column k for d[k]) of the symmetric tridiagonal matrix
 * with diagonal d[0..n) and off-diagonal e[0..n-1); symmetric QR with implicit Wilkinson shifts.  No
 * GPU involved.  LAPH_ERR_ARG for bad arguments or no convergence. */
LAPH_API int laph_tridiag_eigen(int n, double *d, const double *e, double *z);

/* ---- plan API (ragged batches, capture-safe execution) ----------------- */
/* Validates the instances (L >= 1; N >= 3 unless LAPH_PLAN_SKIP_B, N >= 1;
 * N <= 3 L^3; 1 <= n_mom; |n| components within +-2^20), copies the
 * momenta, builds the phase tables and the tile table on the current device
 * and picks the schedule (LAPH_PLAN_AUTOTUNE times candidates on an internal
 * stream, see laph_plan_schedule).  *plan is set only on success. */
LAPH_API int laph_plan_create(const laph_instance *inst, int n_inst, int mode, unsigned flags, laph_plan **plan);

/* Numerical parameters of a plan; 0 picks the default. */
typedef struct {
    int chunk_sites; /* tensor-core modes: sites the tensor core accumulates in FP32 before its sums are drained
                        into FP32 running sums with round-to-nearest (default 128; the error of the tensor core's
                        accumulation grows with it); FP32 mode: sites summed in FP32 before the FP64 reduction
                        (default 1024) */
    int sum_sites;   /* tensor-core modes: sites per block of the FP64 site reduction (default 8192, rounded down
                        to a multiple of 8): a tile covers one block, its running sums become one FP32 partial per
                        output, and the partials of all blocks are added in FP64 in block order */
    int tile_cols;   /* tensor-core modes: complex columns per tile: 104 (default), 96, 80 or 64 in layout 0;
                        176 (default), 192, 208 or 128 in layout 1 */
    int layout;      /* tensor-core modes: how the complex product is laid out on the real tensor cores.
                        0 (default): every complex column of the phased operand is two real rows (re, im) of the
                        MMA's B operand, 128 complex rows per tile; 1: every complex row of the diquark / meson
                        operand is two real rows of the MMA's A operand (tensor-memory lanes r, 64+r), 64 complex
                        rows per tile, and the phased operand's stage images are half as large */
    int chunk_sites_b; /* tensor-core modes: drain interval of the tiles that hold no meson rows (0: chunk_sites).
                          Baryon and triplet sums are incoherent, so their error grows more slowly with the interval
                          than that of the meson sums, whose diagonal entries add coherently */
} laph_plan_options;

/* laph_plan_create with numerical parameters (opts may be NULL).  LAPH_ERR_ARG
 * for a negative value or one above 2^24, a tile width other than 0 or one
 * listed for the layout above, a layout other than 0 or 1, plus the
 * conditions of laph_plan_create.  With LAPH_PLAN_AUTOTUNE the
 * options are the starting point of the search (see laph_plan_tuning). */
LAPH_API int laph_plan_create_opts(const laph_instance *inst, int n_inst, int mode, unsigned flags,
                                   const laph_plan_options *opts, laph_plan **plan);

/* Sites per block of the tensor-core path's FP64 site reduction and the
 * largest number of blocks (FP32 partials per output) of any instance; 0 and
 * 0 for the FP32 mode.  Either pointer may be NULL. */
LAPH_API int laph_plan_sum_sites(const laph_plan *plan, int *sum_sites, int *max_site_blocks);

/* Bytes of device workspace laph_plan_execute needs (256-byte aligned). */
LAPH_API int laph_plan_workspace_size(const laph_plan *plan, size_t *bytes);

/* Runs the whole batch on `stream`: phi[n], out_B[n], out_M[n] are device
 * pointers for instance n (layouts above; out_B/out_M ignored when skipped).
 * No allocation, no host synchronisation: safe inside stream capture.
 * The current device must be the one the plan was created on (LAPH_ERR_ARG
 * otherwise).  Returns LAPH_ERR_WORKSPACE if the workspace is NULL/misaligned
 * while workspace_size > 0. */
LAPH_API int laph_plan_execute(laph_plan *plan, const void *const *phi, void *const *out_B, void *const *out_M,
                      void *workspace, void *stream);

/* Runs a LAPH_PLAN_FIELDS plan on `stream`.  fields holds the device
 * complex64 [T][N][L^3][3] fields of every instance, three per instance
 * (phi, psi, chi) for triplets, two (phi, psi) for doublets, each 8-byte
 * aligned; out[n] is instance n's B3 or M2 (16-byte aligned).  Same
 * behaviour as laph_plan_execute (no allocation, capture-safe).
 * LAPH_ERR_ARG for a plan without LAPH_PLAN_FIELDS, null or misaligned
 * pointers. */
LAPH_API int laph_plan_execute_fields(laph_plan *plan, const void *const *fields, void *const *out, void *workspace,
                                      void *stream);

/* Same batch with HOST buffers: phi_host[n] (complex64, pinned or pageable)
 * is copied in, computed, and out_B_host[n]/out_M_host[n] (complex128, or
 * complex64 with LAPH_PLAN_OUT_C64) are copied back, timeslice chunk by chunk with copies overlapping compute.
 * Device staging comes from `workspace`, which must hold
 * laph_plan_host_workspace_size bytes (256-byte aligned), on the plan's
 * device, which must be current (LAPH_ERR_ARG otherwise).  Returns after the
 * stream is synchronised, on failure too: copies queued before a failure
 * finish before the call returns, so the host buffers are free to reuse. */
LAPH_API int laph_plan_host_workspace_size(const laph_plan *plan, size_t *bytes);
LAPH_API int laph_plan_execute_host(laph_plan *plan, const void *const *phi_host, void *const *out_B_host,
                           void *const *out_M_host, void *workspace, void *stream);

/* Reads (and clears) the plan's device status word: *status = LAPH_OK,
 * LAPH_ERR_TIMEOUT or LAPH_ERR_DEVICE.  Synchronises `stream`. */
LAPH_API int laph_get_device_status(laph_plan *plan, void *stream, int *status);

/* Kernel parameters chosen for the plan (for logs/tests): tile rows, tile
 * columns (complex), site-chunk length of the FP32 partial sums, grid size. */
LAPH_API int laph_plan_describe(const laph_plan *plan, int *mode, int *tile_rows, int *tile_cols, int *chunk_sites,
                       int *grid, int64_t *n_tiles);

/* Durations in ms of the last n contraction-kernel launches of this plan
 * (oldest first), from the events LAPH_PLAN_TIMING records on the launching
 * stream around each launch; waits for those events.  At most 256 launches
 * are kept.  Returns LAPH_ERR_ARG without LAPH_PLAN_TIMING or when fewer
 * than n were recorded. */
LAPH_API int laph_plan_kernel_times(laph_plan *plan, int n, float *ms);

/* Same for the launches that build the tensor-core path's B operand (the
 * phased vectors ph_p phi_k, split and laid out as shared-memory stage
 * images), one per chunk of timeslices.  LAPH_ERR_ARG for the FP32 mode. */
LAPH_API int laph_plan_operand_times(laph_plan *plan, int n, float *ms);

/* Same for the FP64 site reductions of the tensor-core path (one per
 * contraction launch: the FP32 partials of the chunk's site blocks summed in
 * FP64 into the outputs).  LAPH_ERR_ARG for the FP32 mode. */
LAPH_API int laph_plan_reduce_times(laph_plan *plan, int n, float *ms);

/* Contraction-kernel launches per laph_plan_execute: the tensor-core path
 * processes the batch's timeslices in chunks whose B-operand images fit its
 * workspace (at most 24 GiB), one launch per chunk. */
LAPH_API int laph_plan_contraction_launches(const laph_plan *plan, int *n);

/* Schedule of the tensor-core path.
 *   timeslices_per_chunk: timeslices per chunk of B-operand images (0: chunks
 *                         filled by bytes, for batches of several instances);
 *   tile_order:           0 = column tiles outer within a timeslice (the CTAs
 *                         that share a B stage image run together), 1 = row
 *                         tiles outer;
 *   n_chunks:             chunks (contraction launches) per execute.
 * Without LAPH_PLAN_AUTOTUNE the chunk size minimises partly filled waves of
 * persistent CTAs and the order is 0.  With it, plan creation times candidate
 * schedules (laph_plan_tuning) and keeps the fastest; *n_candidates receives
 * their number and candidate_ms (room for 8) the times of the first 8.  Any
 * pointer may be NULL. */
LAPH_API int laph_plan_schedule(const laph_plan *plan, int64_t *timeslices_per_chunk, int *tile_order, int *n_chunks,
                               int *n_candidates, float *candidate_ms);

/* Floating-point operations the tensor pipe executes per laph_plan_execute
 * on the tensor-core path: every tcgen05.mma of every tile, 2 x 128 rows x
 * the tile's real B columns x 16 K entries per k-step, all split terms, the
 * padding and the triangle waste included (0 for the FP32 mode).  Divided by
 * the contraction kernels' time it gives the executed tensor rate. */
LAPH_API int laph_plan_tensor_flops(const laph_plan *plan, double *flops);

/* One candidate schedule timed by LAPH_PLAN_AUTOTUNE. */
typedef struct {
    int tile_cols;                  /* complex columns per tile */
    int layout;                     /* laph_plan_options.layout */
    int sum_sites;                  /* sites per block of the FP64 site reduction */
    int chunk_sites;                /* drain interval of the tensor core's FP32 accumulation, in sites */
    int chunk_sites_b;              /* drain interval of the tiles without meson rows, in sites */
    int tile_order;                 /* 0: column tiles outer, 1: row tiles outer */
    int64_t timeslices_per_chunk;   /* 0: chunks filled by bytes (several instances) */
    float ms;                       /* one execute on the synthetic inputs */
    double probe_err;               /* relative error of (instance 0, timeslice 0) against the FP32 path, or -1 when
                                       not probed */
} laph_tune_record;

/* The autotuner's record.  With LAPH_PLAN_AUTOTUNE, plan creation times
 * candidate schedules on seeded synthetic inputs of the plan's shapes
 * (pseudo-random entries in [-1, 1); inputs, outputs and a workspace are
 * allocated for the duration; one warm-up and one timed execute each) by a
 * coordinate search: tile shape (layout 0 with 104, 96, 80 and 64 columns, layout 1
 * with 176, 192, 208 and 128 columns) x tile order x chunking
 * (the wave model and, for one instance, the largest chunk within the 24 GiB
 * cap); then, from the fastest, half and twice the site-block size of the
 * FP64 reduction; then half and 1.5 times the drain interval (for all
 * tiles; chunk_sites_b is kept as given); finally the three fastest accepted
 * schedules and the default schedule (the one a plan without the flag runs)
 * are timed twice more and each keeps its lowest time.  The fastest replaces
 * the default only if it is more than 1% faster.  A drain
 * interval is accepted only if the relative error of (instance 0, timeslice 0)
 * against the FP32 CUDA-core path stays within 5e-6 (half the 1e-5 bound) or
 * within the default interval's own error; plans of several fields keep the
 * default interval.  The schedule chosen so is applied (see
 * laph_plan_describe, laph_plan_schedule, laph_plan_sum_sites).
 * Writes min(cap, number of candidates) records; *n_candidates (may be NULL)
 * receives the number of candidates (0 without LAPH_PLAN_AUTOTUNE). */
LAPH_API int laph_plan_tuning(const laph_plan *plan, int cap, laph_tune_record *rec, int *n_candidates);

/* Drain intervals (sites) the plan runs: *chunk_sites for tiles with meson
 * rows, *chunk_sites_b for the others (equal unless set apart by
 * laph_plan_options.chunk_sites_b or the autotuner).  Either pointer may be
 * NULL. */
LAPH_API int laph_plan_drain_sites(const laph_plan *plan, int *chunk_sites, int *chunk_sites_b);

/* Number of kernels of this library one laph_plan_execute launches. */
LAPH_API int laph_plan_launches_per_execute(const laph_plan *plan, int *n);

/* Overrides the site-chunk length (sites summed in FP32 before the FP64
 * reduction; 0 = default).  Must be called before execute. */
LAPH_API int laph_plan_set_chunk_sites(laph_plan *plan, int chunk_sites);

LAPH_API int laph_plan_destroy(laph_plan *plan);

/* ---- allocation-free entry point -------------------------------------- */
/* The paper has no counterpart to this function: it serves callers that may
 * not allocate device memory.  It computes B and/or M of one instance with
 * the FP32 CUDA-core contraction (LAPH_MODE_FP32_SIMT) and allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.  Its
 * scratch (descriptor, momenta, tile table, FP32 phase table) lives in one
 * file-scope device array of LAPH_NOALLOC_SCRATCH_BYTES bytes, which every
 * GPU that loads the library holds until the process exits.
 *   phi    device complex64 [T][N][L^3][3], 8-byte aligned;
 *   out_B  device complex128 [T][P][C(N,3)] or NULL (baryons skipped);
 *   out_M  device complex128 [T][P][N][N] or NULL (mesons skipped);
 *          at least one of them non-NULL, each 16-byte aligned; the caller
 *          owns both and the outputs need no clearing;
 *   momenta HOST int32 [n_mom][3], read before the function returns.
 * phi, out_B and out_M must be device memory of the current device and
 * exactly the sizes listed: the function cannot check the size of a device
 * buffer, so an undersized or misplaced buffer is undefined behaviour (an
 * out-of-bounds access on the GPU), not an error code.
 * Limits: 1 <= n_mom <= 64, N >= 3 when out_B is given, N <= 3 L^3, and the
 * scratch (8 * n_mom * L^3 bytes of phase table, plus 72 bytes -- one tile
 * record -- per (64-row tile, 64-column tile, timeslice), plus the
 * descriptor and the momenta, each region rounded up to 256 bytes) must fit
 * the array: larger inputs return LAPH_ERR_WORKSPACE before any launch.
 * Asynchronous on `stream`.
 * The array's device address is looked up once per CUDA context (normally
 * once per device, in its primary context) by the first call made in that
 * context (cudaGetSymbolAddress); make that first call outside any stream
 * capture.  A context created later on the same device (after
 * cudaDeviceReset, or one made current through the driver API) gets its own
 * lookup.  Every call shares the array and leaves its contents behind; each
 * call rewrites what it reads, but calls that may overlap on the GPU
 * (different streams or threads without ordering between them) race on the
 * array. */
#define LAPH_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
LAPH_API int laph_blocks_noalloc(const void *phi, int L, int T, int N, const int32_t *momenta, int n_mom, void *out_B,
                                 void *out_M, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LAPH_H */
