/*
 * ctm.h -- C ABI of libctm: the CTMRG environment sweep of an iTPS on a 2x2
 * unit cell and the reduced density matrices used to measure one- and
 * two-site observables, on one NVIDIA GB300 (sm_103a).
 *
 * What the library computes (TeNeS, arXiv:2112.13184):
 *   Sec. 2.1  an iTPS: one tensor A[s,l,u,r,d] per unit-cell site, physical
 *             dimension d, four virtual legs of bond dimension D;
 *   Sec. 2.2  its norm network, bra and ket merged into one layer of bond
 *             dimension D^2, contracted by the corner-transfer-matrix
 *             renormalisation group: four chi x chi corners C1..C4 and four
 *             chi x D x D x chi edges T1..T4 per site, found by the
 *             directional CTMRG for arbitrary unit cells with projectors
 *             built without the QR step and a partial (randomised) SVD that
 *             never forms the half-system matrix;
 *   Sec. 5.3  the "observable" section: one-site and two-site (nearest
 *             neighbour) operators, measured from reduced density matrices;
 *   Sec. 5.2  the operator element format (before/after states, re, im).
 *
 * Conventions
 *   - Sites i = x + 2y, x,y in {0,1}; y points up, (dx,dy) = (0,1) is the top
 *     neighbour (Sec. 5.3, correlation displacement).
 *   - A is C-order [s][l][u][r][d] (left, top, right, bottom; leg order of the
 *     virtual_dim lists in Appendix A), FP64, d*D^4 doubles.
 *   - Environment of a site, clockwise from the top-left corner, C-order:
 *       which 0: C1[c_T4][c_T1]          1: T1[c_C1][k][k'][c_C2]
 *             2: C2[c_T1][c_T2]          3: T2[c_C2][k][k'][c_C3]
 *             4: C3[c_T2][c_T3]          5: T3[c_C3][k][k'][c_C4]
 *             6: C4[c_T3][c_T4]          7: T4[c_C4][k][k'][c_C1]
 *     k joins the ket tensor A, k' the bra tensor.  C: chi*chi doubles;
 *     T: chi*D*D*chi doubles.
 *   - Operators are real, row-major O[after][before]; two-site operators act
 *     on the combined index (source*d + target) (Sec. 5.2).  Reduced density
 *     matrices are rho[ket][bra] with trace 1, so <O> = Tr(O rho).
 *
 * Ownership and errors
 *   - Every buffer passed in stays owned by the caller; the library copies in
 *     and out.  Host pointers are plain host memory (pinned or not); device
 *     pointers must be device-resident FP64 arrays of the stated size.
 *   - All work of a handle is ordered on the CUDA stream given at creation.
 *     Calls that return values to host memory synchronise that stream.
 *   - Functions return a ctm_status; negative values are errors, and
 *     ctm_last_error(h) gives a message.  No C++ exception crosses the ABI.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef CTM_H
#define CTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctm_ctx* ctm_handle;

typedef enum {
    CTM_OK = 0,
    CTM_NOT_CONVERGED = 1,   /* ctm_run hit max_sweeps; results are still valid */
    CTM_ERR_ARG = -1,        /* bad argument (size, index, null pointer)          */
    CTM_ERR_OOM = -2,        /* device allocation failed                          */
    CTM_ERR_CUDA = -3,       /* a CUDA call failed                                */
    CTM_ERR_NONFINITE = -4,  /* NaN/Inf (or an all-zero tensor) in the environment */
    CTM_ERR_TIMEOUT = -5,    /* a bounded device wait gave up                     */
    CTM_ERR_STATE = -6       /* call out of order (e.g. no tensors set)           */
} ctm_status;

/* How the contractions (enlarged corners, range-finder and projector
 * applies, absorption) are computed; the QR, the SVD truncation and the
 * normalisation stay FP64 in every mode.  The tensor-core modes cut every
 * row of op(A) and column of op(B), scaled by a power of two, into digit
 * slices and multiply the slices on tcgen05. */
typedef enum {
    CTM_FP64 = 0,        /* FP64 on the CUDA cores (DFMA)                          */
    CTM_SPLIT_BF16 = 1,  /* 3 BF16 slices (base-256 digits), every product of
                            levels <= 2 accumulated in FP32 over all of K      */
    CTM_3XTF32 = 2,      /* 2 TF32 slices (base-2^11 digits), hi*hi + hi*lo +
                            lo*hi accumulated in FP32 over all of K             */
    CTM_OZAKI_INT8 = 3,  /* INT8 slices: not built (CTM_ERR_ARG)                 */
    CTM_OZAKI_BF16 = 4   /* emulated FP64: ozaki_slices BF16 slices; levels 0
                            and 1 summed exactly, levels >= 2 in FP32 per 256 of
                            K, the whole sum exact in int64                     */
} ctm_precision;

typedef struct {
    int chi;                /* corner bond dimension chi (Sec. 2.2)              */
    int max_sweeps;         /* ctm_run: sweep cap                                 */
    double tol;             /* ctm_run: stop when the corner-spectrum change < tol */
    int precision;          /* ctm_precision                                       */
    int ozaki_slices;       /* CTM_OZAKI_BF16: slices per operand, 2..6            */
    int rsvd_oversample;    /* randomised SVD: k = min(chi + p, chi*D*D)           */
    int rsvd_power_iters;   /* randomised SVD: power iterations q                  */
    double sv_cutoff_rel;   /* S^{-1/2} := 0 for s < cutoff * s_0                  */
    uint64_t seed;          /* counter-based RNG seed for the rSVD test matrices   */
    int exact_svd_max_n;    /* N = chi*D*D <= this: k = N, the range finder spans
                               everything and the truncated SVD is exact           */
    int rsvd_warm_start;    /* != 0: after the first sweep each cut's range finder
                               starts from that cut's basis of the previous sweep
                               (one subspace iteration per sweep, no extra power
                               iterations); reset by ctm_set_tensor / ctm_set_env */
    int conv_measure;       /* ctm_run's convergence measure: 0 = the normalised
                               corner spectra (ctm_spectrum_delta), 1 = the
                               gauge-invariant loop moments (ctm_loop_delta)   */
    int fp64_refine;        /* != 0 with a tensor-core mode: once ctm_run's measure
                               falls below a decade above where the mode's
                               rounding holds it (CTM_OZAKI_BF16: 1e-8 with 5+
                               slices, 2e-7 with 4, 1e-5 with 3; CTM_SPLIT_BF16
                               and CTM_3XTF32: 1e-4) the handle switches to FP64
                               contractions for the remaining sweeps and stays
                               in FP64 afterwards                               */
    int batch_cuts;         /* != 0: the two row cuts of a column step are processed
                               together -- both cuts' enlarged corners stay
                               resident (4 N^2 more doubles and, in a tensor-core
                               mode, 8 more slice caches) and their projector
                               SVDs run in one launch                          */
} ctm_options;

/* Defaults: chi=16, max_sweeps=100, tol=1e-10, FP64, 5 slices,
 * p=max(8,chi/8) (when rsvd_oversample<=0), q=2, cutoff 1e-12, seed 0,
 * exact_svd_max_n=256, rsvd_warm_start=1, conv_measure=0, fp64_refine=0,
 * batch_cuts=1. */
ctm_status ctm_default_options(ctm_options* opt);

/* Device bytes a handle of this shape allocates (workspace included): the
 * environment of Sec. 2.2 (4 corners chi x chi, 4 edges chi x D x D x chi per
 * site), the four enlarged corners of a cut (N x N, N = chi D^2) and the
 * scratch of the projector and measurement steps.  No device work. */
ctm_status ctm_footprint_bytes(int d, int D, const ctm_options* opt, size_t* bytes);

/* Create a handle for an Lx x Ly unit cell of iTPS tensors (Sec. 2.1, the
 * L_sub of Sec. 5.2) with physical dimension d and bond dimension D, on the
 * current CUDA device.  Only Lx = Ly = 2 is built; other cells return
 * CTM_ERR_ARG.  stream: a cudaStream_t, or NULL to create one owned by the
 * handle.  Allocates all device memory up front (CTM_ERR_OOM if it does not
 * fit); *out is NULL on any error, with the message in ctm_last_error(NULL). */
ctm_status ctm_create(int Lx, int Ly, int d, int D, const ctm_options* opt, void* stream, ctm_handle* out);
/* ctm_create with every device buffer of the handle carved from a
 * caller-owned arena: `arena` (device, 256-byte aligned) of arena_bytes >=
 * ctm_footprint_bytes(d, D, opt) bytes.  The handle never calls cudaMalloc
 * or cudaFree for them, so creating and destroying handles inside a running
 * server neither allocates nor waits for other streams' work; the arena
 * stays the caller's and must outlive the handle.  Per-call scratch of
 * ctm_correlation / ctm_transfer_spectrum / ctm_log_norm_per_site is still
 * allocated per call.  (No counterpart in the paper: the serving loop's
 * memory pool.) */
ctm_status ctm_create_in(int Lx, int Ly, int d, int D, const ctm_options* opt, void* stream, void* arena,
                         size_t arena_bytes, ctm_handle* out);

/* Device-memory pool of a serving loop: first-fit bookkeeping of offsets in
 * one region of `bytes` the caller reserved once (host code only; the
 * region itself is never touched).  Blocks are whole multiples of `grain`
 * (a power of two; 256 for ctm_create_in) starting at multiples of it;
 * freed blocks merge with free neighbours.  Thread-safe.  (No counterpart in
 * the paper: the serving loop's memory pool.)
 *   ctm_pool_alloc: *offset of a block of at least `bytes`, the first free
 *     one that fits; CTM_ERR_OOM when none does.
 *   ctm_pool_free: returns the block allocated at `offset` with the same
 *     `bytes`; CTM_ERR_ARG for any other (offset, bytes), e.g. a second free.
 *   ctm_pool_stats: bytes allocated, the largest free block, the number of
 *     free blocks (each pointer optional). */
typedef struct ctm_pool_s* ctm_pool;
ctm_status ctm_pool_create(size_t bytes, size_t grain, ctm_pool* out);
ctm_status ctm_pool_alloc(ctm_pool pool, size_t bytes, size_t* offset);
ctm_status ctm_pool_free(ctm_pool pool, size_t offset, size_t bytes);
ctm_status ctm_pool_stats(ctm_pool pool, size_t* used, size_t* largest_free, size_t* free_blocks);
ctm_status ctm_pool_destroy(ctm_pool pool);
ctm_status ctm_destroy(ctm_handle h);

/* Copy in the site tensor A of site i (d*D^4 doubles, C-order [s,l,u,r,d]). */
ctm_status ctm_set_tensor(ctm_handle h, int site, const double* A, int on_device);

/* Copy in / out one environment tensor (which = 0..7, see above). */
ctm_status ctm_set_env(ctm_handle h, int site, int which, const double* t, int on_device);
ctm_status ctm_get_env(ctm_handle h, int site, int which, double* t, int on_device);

/* Random initial environment (Sec. 2.2 starts CTMRG from an arbitrary
 * environment): every C and T filled with standard normal numbers from the
 * library's counter-based generator (Philox4x32-10, this seed), each T
 * symmetrised over its ket/bra legs (k, k'), one draw shared by the four
 * sites.  An alternative to ctm_set_env; the numbers differ from any host
 * generator's.  Resets the range finder's warm start. */
ctm_status ctm_init_env_random(ctm_handle h, uint64_t seed);

/* n CTMRG sweeps (left, top, right, bottom moves; Sec. 2.2).  Returns
 * CTM_NOT_CONVERGED (a status, not an error) when a projector SVD reached
 * its Jacobi sweep cap during these sweeps. */
ctm_status ctm_sweep(ctm_handle h, int n);

/* Sweeps until the convergence measure (opt.conv_measure: the normalised
 * corner spectra, max-abs over the 16 corners, or the loop moments of
 * ctm_loop_delta) changes by less than opt.tol or opt.max_sweeps is reached.  Either
 * output pointer may be NULL.  Returns CTM_NOT_CONVERGED at the cap.
 * With CTM_OZAKI_BF16 the spectrum change levels off where the emulated
 * products' rounding sits (about 1e-7 at d=3, D=8, chi=128 with 5 slices),
 * so a tol near 1e-6 is the one to use there; observables at that point
 * agree with the FP64 path to ~1e-8. */
ctm_status ctm_run(ctm_handle h, int* sweeps_done, double* last_delta);

/* Asynchronous form of ctm_sweep (sweep of Sec. 2.2; the asynchronous and
 * batched forms below serve many instances at once and have no counterpart
 * in the paper): enqueues n sweeps on the handle's stream
 * and returns without waiting.  Non-finite values or a timed-out device
 * wait are reported by the next synchronising call on the handle
 * (ctm_sync, ctm_spectrum_delta, ctm_sweep, ...).  Lets several handles,
 * each on its own stream, run at the same time on one GPU. */
ctm_status ctm_sweep_async(ctm_handle h, int n);

/* Waits for the handle's stream and reports any error its sweeps raised. */
ctm_status ctm_sync(ctm_handle h);

/* Batched sweeps: advances n independent instances by `sweeps` sweeps each.
 * Sweeps are issued round-robin over the handles (each on its own stream,
 * each steady sweep one CUDA-graph launch), so small instances overlap on
 * the GPU; then every handle is synchronised.  Returns the first error met
 * (all handles are still synchronised).  Handles must be distinct. */
ctm_status ctm_batch_sweep(const ctm_handle* hs, int n, int sweeps);

/* Convergence measure of Sec. 2.2 as ctm_run applies it: the max-abs change
 * of the normalised corner spectra since this handle's previous call
 * (+infinity on the first call).  Synchronises the handle. */
ctm_status ctm_spectrum_delta(ctm_handle h, double* delta);

/* Switches the handle's contractions to `precision` (CTM_FP64, or
 * CTM_OZAKI_BF16 for a handle created with it) for the following sweeps; the
 * environment and the range finder's warm bases are kept, the captured
 * sweep graph is rebuilt.  Lets a caller finish an emulated-FP64 run in
 * FP64 (what opt.fp64_refine does inside ctm_run).  Synchronises. */
ctm_status ctm_set_precision(ctm_handle h, int precision);

/* Gauge-invariant convergence measure (Sec. 2.2 iterates "until
 * convergence"; the measure is this library's): for each 2x2 block the
 * corner loop L = C1 C2 C3 C4 around it (the network Z_00) is a similar
 * matrix under any change of basis on the chi bonds, so its normalised
 * moments Tr(L^p) / Tr(L)^p, p = 2, 3, 4, do not move with the non-orthogonal
 * gauge the projectors leave, while single-corner singular values do (they
 * keep changing at ~1e-8 after the network has converged to 1e-12).  Returns
 * the max-abs change since this handle's previous call (+infinity on the
 * first).  FP64 products; synchronises the handle. */
ctm_status ctm_loop_delta(ctm_handle h, double* delta);

/* Normalised singular values (sum 1) of every corner: out[site][corner][chi]. */
ctm_status ctm_corner_spectra(ctm_handle h, double* out_host);

/* Reduced density matrices of the converged network (Sec. 5.3, the
 * one-site and two-site observables; the network of Sec. 2.2 with the
 * physical legs of the measured sites left open).  Host outputs, trace 1,
 * rho[ket][bra]: rdm1 is d x d; rdm2 is d^2 x d^2 over (source, target) with
 * target = site + (dx, dy), |dx| + |dy| == 1 (else CTM_ERR_ARG).
 * Synchronises the handle's stream. */
ctm_status ctm_rdm1(ctm_handle h, int site, double* rho_host);
ctm_status ctm_rdm2(ctm_handle h, int site, int dx, int dy, double* rho_host);

/* <O> = Tr(O rho) (Sec. 5.3) for a real row-major host operator O[after]
 * [before]: d x d for measure1, d^2 x d^2 on (source, target) for measure2. */
ctm_status ctm_measure1(ctm_handle h, int site, const double* op, double* value);
ctm_status ctm_measure2(ctm_handle h, int site, int dx, int dy, const double* op, double* value);

/* ln kappa per site: the logarithm of the norm-network value per site
 * (Sec. 2.2), -beta f for a classical network such as the 2D Ising model,
 * from the 2x2 block ratio kappa_block = Z_22 Z_00 / (Z_20 Z_02): Z_22 the
 * block with its full environment, Z_00 the four corners joined directly,
 * Z_20 and Z_02 the row and column strips of edge tensors without sites.
 * ln kappa = ln(kappa_block) / 4, for the site tensors as given (A -> c A
 * adds 2 ln c).  CTM_ERR_NONFINITE when the ratio is not positive and
 * finite.  Uses the handle's precision for its contractions. */
ctm_status ctm_log_norm_per_site(ctm_handle h, double* lnkappa);

/* Operator from the element format of Sec. 5.2: n lines of
 * (i_before, j_before, i_after, j_after) in idx[4n] and real parts re[n];
 * writes the (d0*d1)^2 row-major matrix O[after][before] (zeroed first).
 * A one-site operator uses d1 = 1 and j = 0. */
ctm_status ctm_op_from_elements(int d0, int d1, int n, const int* idx, const double* re,
                                double* op_out);

const char* ctm_last_error(ctm_handle h);
const char* ctm_status_string(ctm_status s);

/* Instrumentation (no counterpart in the paper).  When enabled, every
 * contraction, permutation, QR and SVD of the handle is bracketed by CUDA
 * events on its stream; ctm_profile_read returns the accumulated device
 * time per class together with the algorithmic FLOPs (2MNK per GEMM) and
 * bytes (read + write per permutation) of the calls timed.  Classes:
 * 0 GEMM (FP64 DFMA or tensor-core slice products), 1 permute, 2 QR, 3 SVD,
 * 4 operand slicing of the emulated GEMM, 5..7 unused.  reset != 0 zeroes
 * the counters. */
typedef struct {
    double ms[8];
    double flops[8];
    double bytes[8];
    long long calls[8];
} ctm_profile_data;
ctm_status ctm_profile_enable(ctm_handle h, int on);
ctm_status ctm_profile_read(ctm_handle h, ctm_profile_data* out, int reset);

/* The same timings broken down by operation (enlarged corner products X2,
 * X3, X4, range-finder and projector applies, absorption, QR, SVD) and
 * class, as a JSON object written to buf (len bytes including the NUL;
 * CTM_ERR_ARG if it does not fit). */
ctm_status ctm_profile_report(ctm_handle h, char* buf, size_t len, int reset);

/* Number of CUDA kernels libctm has launched in this process (all handles
 * and kernel-level calls); cudaMemset/cudaMemcpy are not counted. */
long long ctm_kernel_launches(void);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (no
 * counterpart in the paper; the denominator of the FP64 path's roofline):
 * 8 SM-count x 256 threads run independent FMA chains, best of three timed
 * launches after a warm-up, CUDA events.  Allocates and frees its own small
 * buffer and stream; synchronises. */
ctm_status ctm_fp64_peak(double* tflops);

/* Failure-detection check (no counterpart in the paper): launches one
 * thread that waits on an mbarrier with the same bounded wait the
 * tensor-core GEMM uses, for at most limit_cycles (1 .. 4e9) SM clock
 * cycles.  With arrive != 0 another thread arrives and the wait completes
 * (CTM_OK); with arrive == 0 nothing arrives, the wait gives up and the call
 * returns CTM_ERR_TIMEOUT with the context still usable.  flag_dev: one
 * device int of scratch, owned by the caller.  Synchronises `stream`. */
ctm_status ctm_wait_probe(long long limit_cycles, int arrive, int* flag_dev, void* stream);

/* ------------------------------------------------------------------------
 * Kernel-level entry points.  All pointers are device pointers, work is
 * ordered on `stream` (cudaStream_t, NULL = legacy default stream), nothing
 * is synchronised, and no memory is allocated unless stated.  They are the
 * building blocks of the sweep, exported for per-kernel parity tests.
 * ------------------------------------------------------------------------ */

/* C[M,N] = alpha * op(A) op(B) + beta * C, row-major, FP64.  op(X) = X or
 * X^T (trans != 0).  lda/ldb/ldc are row strides of the stored arrays. */
ctm_status ctm_dgemm(int transA, int transB, int M, int N, int K, double alpha,
                     const double* A, int lda, const double* B, int ldb, double beta,
                     double* C, int ldc, void* stream);

/* dst = src with axes permuted: dst dims are dims[perm[0..ndim-1]] and
 * dst[i_0..] = src[j] with j_{perm[a]} = i_a.  ndim <= 8, FP64. */
ctm_status ctm_permute(const double* src, double* dst, int ndim, const int* dims,
                       const int* perm, void* stream);

/* Thin Householder QR of Y (N x k row-major, N >= k): Q (N x k) with
 * orthonormal columns and upper-triangular R (k x k, diagonal >= 0), Y=QR.
 * Y is not modified.  ws: workspace of ctm_qr_workspace_bytes(N,k) bytes.
 * Runs as one persistent cooperative launch over all SMs when the row slabs
 * fit in shared memory (k columns of ~N/152 rows twice), else as two
 * launches per column; in the persistent form the first int of ws is set to
 * 1 if a bounded grid barrier gave up (Q and R then hold no result). */
size_t ctm_qr_workspace_bytes(int N, int k);
ctm_status ctm_qr(const double* Y, int N, int k, double* Q, double* R, void* ws, void* stream);

/* SVD of a small square G (k x k row-major, k <= 1024) by one-sided Jacobi:
 * G = U diag(S) V^T, S descending, U and V k x k row-major.  Columns of U
 * with S = 0 are zero.  ws: ctm_svd_workspace_bytes(k) bytes; its first int
 * is set to 1 when the rotations had not settled after the sweep cap (the
 * outputs are then the last iterate), else 0.  Not synchronised. */
size_t ctm_svd_workspace_bytes(int k);
ctm_status ctm_svd(const double* G, int k, double* U, double* S, double* V, void* ws,
                   void* stream);

/* C[M,N] = alpha op(A) op(B) + beta C like ctm_dgemm, computed on the tensor
 * cores as exact BF16 slice products (emulated FP64; see CTM_OZAKI_BF16):
 * each row of op(A) and column of op(B) is scaled by a power of two and cut
 * into `slices` (2..6) signed 8-bit digits; products of the two leading
 * digit levels are accumulated exactly, the rest in FP32 (restarted every
 * 256 of K), levels >= slices dropped, and all of it summed exactly in
 * int64.  Error per entry <= (2^(2 - 8 slices) + 2^-36) * max|row of op(A)|
 * * max|col of op(B)| * K: the first term is the slicing, the second the
 * tensor cores' FP32 rounding of the levels >= 2 (measured), so 5 slices
 * give ~1e-11 relative per unit K and 6 add nothing.  Entries whose digits
 * all fit (e.g. integers below 2^8 per row max) give exact results.
 * ws: ctm_gemm_ozaki_workspace_bytes(M,N,K,slices) bytes; its first int is
 * set non-zero if a bounded wait inside the kernel gave up (C then holds no
 * result).  Not synchronised. */
size_t ctm_gemm_ozaki_workspace_bytes(int M, int N, int K, int slices);
ctm_status ctm_gemm_ozaki(int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
                          const double* B, int ldb, double beta, double* C, int ldc, int slices, void* ws,
                          void* stream);

/* ---- correlation functions and correlation length (Sec. 5.3) -------------
 *
 * Both read the handle's current environment (a converged one: run
 * ctm_run or ctm_sweep first) and contract in the handle's precision; the
 * eigenvalue and normalisation steps are FP64.  A strip is the row (for x)
 * or column (for y) of sites through the start site, between the edge
 * tensors of that row (T1 above, T3 below; for y T4 left, T2 right) and
 * closed by the corner and edge tensors of its first and last sites. */
#define CTM_CORRELATION_MAX_R 4096
/* Correlation functions C(r, r0) = <A(r0) B(r0 + r)> (Sec. 5.3, the
 * `correlation` section's definition): out_host[dir][site][i] for the
 * displacement r = (i, 0) (dir 0) or (0, i) (dir 1), 0 <= i <= rmax, with
 * every site r0 = (x, y), site = x + 2 y, of the cell as start site.  The
 * strip with A on the ket of r0 and B on the ket of r0 + r divided by the
 * same strip without operators; i = 0 is the one-site <A B> (B acts first).
 * opA, opB: host d x d, row-major O[after, before].  out_host: 8 (rmax + 1)
 * doubles.  rmax in [0, CTM_CORRELATION_MAX_R].  Cost: 3 rmax + 2 column
 * contractions (each like one enlarged corner) per start site and
 * direction.  Allocates 9 chi^2 D^2 + 4 d D^4 + 3 d^2 doubles on first use
 * (kept until ctm_destroy) and 16 (rmax + 1) doubles per call.
 * Synchronises.  CTM_ERR_STATE when tensors or environment are not set. */
ctm_status ctm_correlation(ctm_handle h, const double* opA, const double* opB, int rmax, double* out_host);

/* Leading eigenvalues of the transfer matrix of one period of the cell
 * (Sec. 5.3, the `correlation_length` section: xi^-1 = e_1 =
 * -log(lambda_1 / lambda_0), with e_2, e_3, ... for the finite-chi
 * extrapolation 1/xi(inf) = 1/xi(chi) + k (e_2 - e_1)).  dir 0: the two
 * columns of row y = index, acting along +x; dir 1: the two rows of column
 * x = index, acting along +y.  Explicitly restarted block Arnoldi: each
 * cycle builds an orthonormal basis of the block Krylov space of `block`
 * vectors and p = min(32 / block, chi^2 D^2 / block) >= 2 powers of the
 * transfer matrix (nev <= block <= 16), takes the eigenvalues of its
 * Rayleigh-Ritz matrix, and restarts from the leading Ritz vectors, until
 * the first nev moduli |lambda_i / lambda_0| change by less than tol in one
 * cycle or max_iter cycles are done (then CTM_NOT_CONVERGED).
 * out_host: 4 nev doubles -- Re(lambda_i / lambda_0), Im(lambda_i /
 * lambda_0), |lambda_i|, e_i = -ln|lambda_i / lambda_0| / 2 per lattice
 * spacing (the period is 2 sites; +inf for lambda_i = 0) -- for i < nev
 * with |lambda_i| descending; the correlation length is 1 / e_1.  *iters,
 * *change (optional): cycles done and the last change.  Each cycle costs
 * 2 block p column contractions.  Allocates (block p + 3 block) chi^2 D^2
 * doubles plus a QR workspace per call.  Synchronises. */
ctm_status ctm_transfer_spectrum(ctm_handle h, int dir, int index, int nev, int block, int max_iter, double tol,
                                 double* out_host, int* iters, double* change);

/* Kernel-level: eigenvalues of a small real m x m matrix H (device, row
 * stride ldh, 1 <= m <= 32) -- Householder Hessenberg reduction, then the
 * complex QR algorithm with Wilkinson shifts and deflation, in one thread.
 * out (device, 4 m doubles): Re(l_i / l_0), Im(l_i / l_0), |l_i|,
 * -ln|l_i / l_0| / period, with |l_i| descending.  *status (device,
 * optional): 0; 1 when the iteration cap (60 m QR steps) was hit; 2 when
 * every eigenvalue is zero.  Not synchronised.  (The Rayleigh-Ritz step of
 * ctm_transfer_spectrum; no counterpart in the paper.) */
ctm_status ctm_small_eig(const double* H, int m, int ldh, double period, double* out, int* status, void* stream);

/* C[M,N] = alpha op(A) op(B) + beta C like ctm_dgemm, as the FP32-accumulated
 * tensor-core products of `precision` = CTM_SPLIT_BF16 (3 BF16 slices) or
 * CTM_3XTF32 (2 TF32 slices).  Error ~ 2^-24 K max|row of op(A)| max|col of
 * op(B)| from the FP32 accumulation; products whose digits fit one slice
 * and whose sums stay below 2^24 units are exact.  ws:
 * ctm_gemm_split_workspace_bytes(precision, M, N, K) bytes, its first int set
 * non-zero if a bounded wait inside the kernel gave up.  Not synchronised.
 * (No counterpart in the paper: the precision study's kernel-level entry.) */
size_t ctm_gemm_split_workspace_bytes(int precision, int M, int N, int K);
ctm_status ctm_gemm_split(int precision, int transA, int transB, int M, int N, int K, double alpha,
                          const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                          void* ws, void* stream);

/* ctm_svd without a caller workspace and without allocating (the paper has
 * no counterpart; this is a deployment aid).  For callers that cannot call
 * cudaMalloc where they need the SVD: cudaMalloc can synchronise the
 * device, which is not allowed while a CUDA graph is being captured in
 * global mode and stalls latency-bound serving loops, and callers that run
 * under a fixed device-memory budget cannot make untracked allocations.
 * The scratch (about 1 MB) lives in a static device array that every GPU
 * loading libctm holds until the process exits; k must be <= 256, larger k
 * returns CTM_ERR_ARG.  The first call on each device looks the array's
 * device address up (with that device current); make that first call
 * before any stream capture.  All calls share the one array, which keeps the
 * previous call's contents (everything that must start at zero is cleared
 * by the call itself): calls that can overlap on the GPU -- on different
 * streams without ordering -- race and must be serialised by the caller.
 * Arguments, layout and results are those of ctm_svd. */
ctm_status ctm_svd_noalloc(const double* G, int k, double* U, double* S, double* V, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CTM_H */
