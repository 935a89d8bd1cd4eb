/*
 * hisq.h -- C ABI of the GB300 library for deflated HISQ propagator solves.
 *
 * Method: "Improving HISQ propagator solves using deflation" (Hostetler, Clark,
 * DeTar, Gottlieb, Weinberg; LATTICE2024).
 *   Section 2      M = D + 2m, D the anti-Hermitian HISQ Dirac matrix (one-hop fat
 *                  links, three-hop Naik "long" links); CG on the normal equation
 *                  M^dag M psi = M^dag eta (Eq. 1), even-odd preconditioned:
 *                  y_e = (M^dag eta)_e, solve (M^dag M)_ee psi_e = y_e, then
 *                  reconstruct the odd sites.
 *   Section 2      Low eigenvectors of the squared massless operator by
 *                  thick-restart Lanczos; deflated initial guess
 *                  x = sum_i v_i lambda_i^-1 v_i^dag b (Eq. 4), with
 *                  lambda_i = eps_i + (2m)^2 (Eq. 3).
 *   Section 3      Mixed precision with reliable updates (delta_rd = 0.1) and
 *                  re-deflation whenever the residual drops by 1/delta_tr since the
 *                  last deflation (delta_tr = 1e-3), with single-precision
 *                  eigenvectors.
 *
 * Operator convention (the paper fixes neither the factor 1/2 nor the hop signs):
 *   (D psi)(x) = sum_mu eta_mu(x) [ F_mu(x) psi(x+mu) - F_mu(x-mu)^dag psi(x-mu)
 *                                 + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^dag psi(x-3mu) ]
 *   eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z);
 *   periodic in space; in time periodic or antiperiodic (a hop that wraps from
 *   t = T-1 to t = 0 carries a factor -1).  The HISQ coefficients are folded into
 *   the links the caller passes (fat = c1 * ..., long = c3 * ...).
 *   Odd reconstruction: psi_o = (eta_o - D_oe psi_e) / (2m).
 *
 * Host layouts (FP64, caller-owned, copied during the call):
 *   site index s = x + X*(y + Y*(z + Z*t)); parity (x+y+z+t) mod 2, even = 0;
 *   links  [s][mu][row][col][re,im]  (mu = x, y, z, t), V*4*18 doubles;
 *   fields [s][colour][re,im] over the full lattice, V*6 doubles.
 * Device-pointer variants (*_device) take the same layouts in device memory,
 * owned by the caller; the library never frees caller memory.
 *
 * Errors: every call returns a hisq_status; the context keeps a message for the
 * last error (hisq_last_error).  A call that fails with HISQ_ERR_CUDA leaves the
 * context in an undefined state: destroy it.  Contexts are not thread-safe; all
 * work of one context runs in order on its stream.
 */
#ifndef HISQ_H
#define HISQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hisq_ctx hisq_ctx;

typedef enum {
    HISQ_OK = 0,
    HISQ_ERR_INVALID_ARG = 1,   /* bad size, pointer, precision or parameter       */
    HISQ_ERR_CUDA = 2,          /* a CUDA runtime call failed                      */
    HISQ_ERR_OOM = 3,           /* device or pinned host allocation failed         */
    HISQ_ERR_NOT_CONVERGED = 4, /* max_iter reached; psi holds the best iterate    */
    HISQ_ERR_NUMERICAL = 5,     /* NaN/Inf in a reduction or an input              */
    HISQ_ERR_TIMEOUT = 6,       /* a bounded device wait ran out                    */
    HISQ_ERR_STATE = 7          /* call order violated (e.g. solve before links)   */
} hisq_status;

/* Storage precisions.  Arithmetic is FP64 for HISQ_PREC_DOUBLE, double-float for
 * HISQ_PREC_DF64 and FP32 otherwise. */
typedef enum {
    HISQ_PREC_DOUBLE = 64,
    HISQ_PREC_SINGLE = 32,
    HISQ_PREC_HALF = 16, /* FP16 values with one FP32 scale per site (colour vectors) */
    HISQ_PREC_BF16 = 15, /* BF16 values, 12 B per site; eigenvector storage only     */
    HISQ_PREC_HALF_EV = 14, /* FP16 values of v * 2^e with one power-of-two scale for
                               all sites and vectors (4^e >= 3 Vh, the smallest),
                               12 B per site, colour-major; eigenvector storage
                               only, read by the tensor cores as it is stored   */
    HISQ_PREC_DF64 = 48  /* double-float: each real the sum hi + lo of two FP32
                            numbers (about 48 significant bits), FP32 arithmetic
                            with exact products and error-carrying sums; the
                            reliable-update residual and the test operators only */
} hisq_precision;

/* Parameters of a propagator solve (Sections 2 and 3). */
typedef struct {
    double tol;              /* stop when |y_e - A psi_e| <= tol * min(|y_e|, 2m|eta|)
                                (FP64 true residual); 1e-10 in the benchmarks      */
    int max_iter;            /* sloppy CG iterations per right-hand side            */
    int precision_sloppy;    /* colour-vector storage of the sloppy CG: 64, 32, 16 */
    int link_precision_sloppy; /* link storage of the sloppy operator: 32 or 16
                                  (ignored, FP64, when precision_sloppy is 64)     */
    double delta_rd;         /* reliable update when |r| < delta_rd * |r_last|; 0.1 */
    int deflate;             /* 1: deflated initial guess from the stored eigenpairs */
    int n_defl;              /* eigenpairs used (<= stored); 0 = all stored         */
    double delta_tr;         /* re-deflate when |r| < delta_tr * |r_defl|; 0 = off  */
    int compute_full_residual; /* 1: also return |eta - M psi| / |eta| in FP64     */
    int batch;               /* 1: solve the right-hand sides of one call together,
                                up to 64 at a time (each keeps its own CG, reliable
                                updates and re-deflations; one batched operator
                                application per iteration reads the links once);
                                needs precision_sloppy 32|16 and FP32 links.
                                0: one right-hand side after the other            */
    int guess;               /* 1: psi holds an initial guess on entry (its even
                                sites); the solve starts from it, deflating its
                                residual when deflation is on                      */
    int precision_reliable;  /* arithmetic of the reliable-update residual
                                b - A x: 64 (FP64, Section 3) or HISQ_PREC_DF64
                                (double-float on the FP32 units; a residual that
                                meets the tolerance is recomputed in FP64 before
                                convergence is reported, and the rest of that
                                right-hand side's solve uses FP64 if it is not
                                confirmed; that FP64 check is the even part of the
                                full residual, 2m r_e = y_e - A psi_e).  The
                                double-float links are built on first use and take
                                as much device memory as the FP64 copy (2304 B per
                                site); HISQ_ERR_OOM if they do not fit.  Default 64. */
    int persistent;          /* batched solves (batch = 1, FP32 links with 18- or
                                12-real long links): 1 runs the sloppy iterations
                                between two host interventions (reliable updates,
                                re-deflations, convergence) as one cooperative
                                launch, all blocks resident, grid-wide phases
                                separated by bounded barriers, handing the batch
                                back two iterations after the first right-hand
                                side reaches its next threshold (the launch-per-
                                iteration loop also sees each residual two
                                iterations late); 0 (default) launches three kernels
                                per iteration, replayed as CUDA graphs on a
                                capturable stream.  Same arithmetic either way. */
} hisq_solve_params;

/* Per right-hand-side results of a solve. */
typedef struct {
    int iterations;          /* sloppy CG iterations                               */
    int reliable_updates;    /* true-residual recomputations (in the arithmetic of
                                precision_reliable)                                */
    int redeflations;        /* deflations after the initial guess                 */
    int converged;           /* 1 if the tolerance was met                         */
    double even_residual;    /* |y_e - A psi_e| / |y_e|, FP64                      */
    double full_residual;    /* |eta - M psi| / |eta|, FP64 (if requested, else -1) */
    double seconds_total;    /* prep + deflation + CG + reconstruction             */
    double seconds_deflate;  /* initial deflation and re-deflations                */
    /* filled only with profiling on (hisq_set_profiling): CUDA-event time of the
       two Dslash kernels of each sloppy CG iteration, summed over iterations; in
       a batched solve each launch's time is shared equally among the right-hand
       sides it served                                                           */
    double seconds_dslash_oe; /* tmp = D_oe p, |tmp|^2                          */
    double seconds_dslash_eo; /* 4m^2 p - D_eo tmp fused with the x, r update    */
    int profiled_iterations;
} hisq_solve_stats;

/* Parameters of the thick-restart Lanczos eigensolve (Section 2). */
typedef struct {
    int n_ev;                /* wanted eigenpairs (lowest of the squared operator)  */
    int n_kr;                /* Krylov basis size, > n_ev + 8                       */
    int n_keep;              /* vectors kept at a restart (0 = (n_ev + n_kr) / 2)    */
    double tol;              /* Ritz residual |A v - theta v| <= tol * a_max        */
    int max_restarts;
    int cheby_degree;        /* Chebyshev filter degree (0 = Lanczos on A itself)   */
    double a_min;            /* filter window [a_min, a_max] of the massless operator.
                                a_min > 0: given; a_min = -f < 0: placed where an
                                estimated f * n_ev eigenvalues lie below it (0: f = 2) */
    double a_max;            /* > 0: given; <= 0: 1.1 x a power-iteration estimate  */
    int storage_precision;   /* eigenvector storage: 32, 16, HISQ_PREC_BF16 (15) or
                                HISQ_PREC_HALF_EV (14)                              */
    uint64_t seed;           /* start vector                                        */
    int block_size;          /* 1: thick-restart Lanczos; b = 2..64: block thick-restart
                                Lanczos with b vectors per step, the operator applied to
                                the whole block at once (the paper's outlook, Section 4);
                                reduced to (n_kr - n_keep) / 2 when larger, so that a
                                restart adds at least two blocks; n_kr and n_keep are
                                rounded to the block grid                             */
} hisq_eig_params;

/* Fill the structs with the paper's defaults (Section 3: delta_rd = 0.1,
 * delta_tr = 1e-3; tolerance 1e-10). */
void hisq_default_solve_params(hisq_solve_params *p);
void hisq_default_eig_params(hisq_eig_params *p);

/* Create a context on CUDA device `device` for an X*Y*Z*T lattice (each extent
 * even and >= 4).  `cuda_stream` is a cudaStream_t or NULL (the context creates
 * a non-blocking stream of its own, which is NOT ordered with the legacy default
 * stream).  The special handles cudaStreamLegacy and cudaStreamPerThread are
 * accepted; pass cudaStreamLegacy to order the library's work with other work on
 * the legacy default stream.  On success *out owns all device memory of the
 * context. */
hisq_status hisq_create(const int dims[4], int t_antiperiodic, int device, void *cuda_stream,
                        hisq_ctx **out);
void hisq_destroy(hisq_ctx *ctx);
const char *hisq_last_error(const hisq_ctx *ctx);
const char *hisq_status_string(hisq_status s);

/* Load the fat (one-hop) and long (three-hop) links, FP64 host layout above,
 * coefficients folded in.  long_recon = 18 stores all 18 reals of the long links;
 * 12 stores two rows of long/long_scale (which must then be SU(3) to 1e-6;
 * otherwise HISQ_ERR_INVALID_ARG) and rebuilds the third row on the fly; 8
 * stores (a2, a3, b1, arg a1, arg c1) of the same SU(3) factor and rebuilds the
 * rest from unitarity (FP32 sloppy operator only; FP16 links need 18 or 12).  The
 * FP64 copy always holds all 18 reals.  The library folds staggered phases,
 * boundary signs and the backward adjoints into its own device copies (FP64,
 * FP32; FP16 built on first use).  Non-finite input: HISQ_ERR_NUMERICAL. */
hisq_status hisq_load_links(hisq_ctx *ctx, const double *fat, const double *lng, int long_recon,
                            double long_scale);

/* Set the bare mass m > 0 (M = D + 2m).  Stored eigenvalues follow Eq. 3. */
hisq_status hisq_set_mass(hisq_ctx *ctx, double m);

/* out_parity sites of `out` = D applied to the opposite-parity sites of `in`
 * (host full-lattice fields); the other parity of `out` is set to zero.
 * precision: colour-vector storage (64, 32, 16); link_precision: link storage
 * (64 with precision 64; 32 or 16 otherwise; arithmetic FP32).  Precision and
 * link precision HISQ_PREC_DF64 apply the double-float operator of the
 * reliable updates to the FP64 input.  Test and diagnostic entry point. */
hisq_status hisq_apply_dslash(hisq_ctx *ctx, int out_parity, int precision, int link_precision,
                              const double *in, double *out);

/* The batched operator of the multi-RHS solve (test entry point): for nrhs <= 64
 * host full-lattice fields in_j (offset j*V*6 doubles), out_parity sites of
 * out_j = D applied to the opposite-parity sites of in_j, the other parity zero,
 * through the kernel the batched CG uses for D_oe p_j (one launch for all
 * right-hand sides, reading the links once).  precision: colour-vector storage
 * 32 or 16; FP32 links.  The launch shape is the autotuned one unless
 * hisq_set_batched_kernel chose another. */
hisq_status hisq_apply_dslash_batch(hisq_ctx *ctx, int out_parity, int precision, int nrhs, const double *in,
                                    double *out);

/* Launch shape of the batched operator (testing and tuning; kind 0 = autotuned,
 * the default).  kind 1: one site per thread for rhs_per_thread (2..4)
 * right-hand sides, links loaded by each thread, with (budget 0) or without
 * (budget 1) an L2 prefetch of the next direction's links; kind 2: the same
 * work split with the links of each site group and direction bulk-copied into
 * a shared-memory ring, `budget` (2..4) blocks per SM (12-real long links only;
 * never chosen by the autotuner, slower on GB300); kind 3: as kind 1 with the
 * right-hand sides in pairs whose colour algebra runs as packed two-wide FP32
 * FMAs (rhs_per_thread 2 or 4).  A shape that does not exist for a batch size
 * makes the batched calls fail with HISQ_ERR_INVALID_ARG. */
hisq_status hisq_set_batched_kernel(hisq_ctx *ctx, int kind, int rhs_per_thread, int budget);

/* Even sites of `out` = (M^dag M)_ee applied to the even sites of `in`
 * (= 4m^2 in_e - D_eo D_oe in_e); odd sites of `out` are zero.  Precisions as
 * for hisq_apply_dslash. */
hisq_status hisq_apply_normal_op(hisq_ctx *ctx, int precision, int link_precision, const double *in,
                                 double *out);

/* Solve M psi_k = eta_k for nrhs right-hand sides (host full-lattice fields,
 * right-hand side k at offset k*V*6 doubles).  stats: nrhs entries (nullable).
 * Returns HISQ_ERR_NOT_CONVERGED if any right-hand side missed the tolerance. */
hisq_status hisq_solve(hisq_ctx *ctx, const double *eta, double *psi, int nrhs,
                       const hisq_solve_params *params, hisq_solve_stats *stats);

/* As hisq_solve, with eta and psi in caller-owned device memory, ordered on the
 * context's stream. */
hisq_status hisq_solve_device(hisq_ctx *ctx, const double *eta_dev, double *psi_dev, int nrhs,
                              const hisq_solve_params *params, hisq_solve_stats *stats);

/* Thick-restart Lanczos for the lowest n_ev eigenpairs of the massless even-site
 * operator -D_eo D_oe (Section 2), with FP32 operator and basis, FP64
 * Rayleigh-Ritz (tridiagonal QL on the host for block_size 1, a dense FP64
 * Hermitian eigensolver on the device for the block variant), and final FP64
 * Rayleigh quotients with the FP64
 * operator (Section 3, eigenvalues recomputed from the eigenvectors).  eps_out
 * (nullable, n_ev doubles) receives the massless eigenvalues eps_i in ascending
 * order; *n_conv the number that met the tolerance and whose FP64 residual
 * |A v - eps v| / |v| is at most 1e-3 a_max (a pair that passes the filtered
 * operator's test but not this one is spurious).  The eigenvectors stay on the
 * device for deflation. */
hisq_status hisq_eigensolve(hisq_ctx *ctx, const hisq_eig_params *params, int *n_conv,
                            double *eps_out);

/* Number of stored eigenpairs and their massless eigenvalues (ascending). */
hisq_status hisq_get_eigvals(hisq_ctx *ctx, int *n_ev, double *eps_out);

/* Copy stored eigenvector i to a host full-lattice field (odd sites zero). */
hisq_status hisq_get_eigvec(hisq_ctx *ctx, int i, double *out);

/* Replace the stored eigenpairs by n host fields (even sites used; orthonormal)
 * with massless eigenvalues eps (nullable: recomputed as FP64 Rayleigh
 * quotients), stored at storage_precision 32, 16, 15 (BF16) or 14
 * (HISQ_PREC_HALF_EV). */
hisq_status hisq_set_eigvecs(hisq_ctx *ctx, int n, const double *vecs, const double *eps,
                             int storage_precision);

/* x_e = sum_i v_i lambda_i^-1 v_i^dag b_e (Eq. 4) over the first n stored pairs
 * (0 = all), lambda_i = eps_i + 4m^2; host full-lattice fields, even sites. */
hisq_status hisq_deflate(hisq_ctx *ctx, int n, const double *b, double *x);

/* hisq_deflate for callers that must not allocate device memory: code that runs
 * under a device-memory budget owned by someone else (a framework allocator or
 * memory pool that must account for every byte), or in a phase of a long job
 * where allocation is not allowed because it can fail, stall the device or
 * fragment memory that the application has already laid out.  This entry point
 * makes no device allocation and calls no allocating routine; there is no
 * counterpart in the paper, it is an interface variant of hisq_deflate.
 *
 * It computes the same guess x_e = sum_i v_i lambda_i^-1 v_i^dag b_e over the
 * first n stored pairs (n <= 0 or n > stored: all), with b_dev and x_dev in
 * caller-owned device memory in the library's even-site FP64 layout: colour
 * field [colour][Vh] of complex doubles (re, im), where Vh = V/2 and the even
 * site s = x + X*(y + Y*(z + Z*t)) has index s/2.  x_dev is overwritten.
 * Work is ordered on the context's stream; the call returns without waiting.
 *
 * Scratch: one fixed array of 16 MiB in device memory.  A device reserves it
 * when the first context is created on it (hisq_create looks up the array's
 * device address with that device current, which loads the code module that
 * holds it) and keeps it until the process exits; this entry point itself
 * never reserves or allocates anything.  A call needs
 * ceil256(16 * n * ceil(Vh / 4096)) + ceil256(16 * n) bytes of it (the
 * projection's partial sums and the n coefficients, each region rounded up to
 * a multiple of 256 bytes); larger requests fail with HISQ_ERR_INVALID_ARG and
 * a message naming the sizes.  The eigenvalues are read from the device copy
 * that is written whenever eigenpairs are stored.  All calls share the array
 * and it keeps the last call's contents; every byte a call reads is first
 * written by that call, but calls that overlap on the GPU (different streams
 * or contexts on one device) race on it. */
hisq_status hisq_deflate_noalloc(hisq_ctx *ctx, int n, const double *b_dev, double *x_dev);

/* Batched deflation on the tensor cores (Eq. 4 for several right-hand sides, the
 * paper's Section 4 outlook): for nrhs <= 32 host full-lattice fields b_j,
 * x_j = sum_i v_i lambda_i^-1 v_i^dag b_j and r_j = b_j - sum_i v_i v_i^dag b_j
 * over the first n <= 512 stored pairs (0 = all), even sites.  Needs FP32, BF16
 * or HISQ_PREC_HALF_EV eigenvector storage.  The projection and the expansion
 * are complex GEMMs with FP32 accumulation: with FP32 storage both operands are
 * split into FP16 high and low parts; with 16-bit storage the stored vectors
 * are one operand as they are and only the other is split. */
hisq_status hisq_deflate_batch(hisq_ctx *ctx, int n, int nrhs, const double *b, double *x, double *r);

/* Write / read the stored eigenpairs to / from a binary file (header with
 * lattice, count, precision and checksum).  Loading recomputes the eigenvalues
 * as FP64 Rayleigh quotients (Section 3). */
hisq_status hisq_save_eigvecs(hisq_ctx *ctx, const char *path);
hisq_status hisq_load_eigvecs(hisq_ctx *ctx, const char *path);

/* Turn per-kernel CUDA-event timing of the CG iterations on (1) or off (0).
 * Events are recorded on the context's stream around the two Dslash kernels of
 * every iteration (sums returned in hisq_solve_stats) and around every FP64
 * Dslash launch (sums returned by hisq_profiled_fp64, restarted each time
 * profiling is switched on; an FP64 launch made during a stream capture is not
 * timed). */
hisq_status hisq_set_profiling(hisq_ctx *ctx, int on);

/* CUDA-event time (*seconds) and number (*launches) of the FP64 Dslash launches
 * (reliable-update residuals, source preparation, odd reconstruction, residual
 * checks) made while profiling was on, since it was last switched on.  Waits
 * for the pending launches.  HISQ_ERR_INVALID_ARG for a null argument. */
hisq_status hisq_profiled_fp64(hisq_ctx *ctx, double *seconds, unsigned long long *launches);

/* Failure injection on the host (tests of the error paths; the paper has no
 * counterpart): after `after` further successful device allocations by this
 * context, every allocation fails as if the device were out of memory, so the
 * call in progress returns HISQ_ERR_OOM with a message.  after < 0 switches the
 * injection off; the context stays usable.  Nothing is done on the device. */
hisq_status hisq_inject_alloc_failure(hisq_ctx *ctx, int after);

/* Failure injection of a bounded device wait (tests of the timeout path; the
 * paper has no counterpart): with on != 0 the next pipelined launch runs with
 * a wait that cannot be met in time.  A tensor-core deflation
 * (hisq_deflate_batch, or the batched solve's) launches its GEMM with a
 * producer that issues no copy and with waits that give up after a few
 * thousand polls, so the MMA warp's wait for its operands runs out while no
 * copy and no MMA is in flight; a persistent batched CG launch runs its grid
 * barriers with a zero time limit.  The call returns HISQ_ERR_TIMEOUT with a
 * message and the context stays usable.  One-shot: the next call runs
 * normally.  on = 0 cancels it. */
hisq_status hisq_inject_wait_timeout(hisq_ctx *ctx, int on);

/* Bounds checking (a stand-in for a memory checker): in a library built with
 * -DHISQ_BOUNDS_CHECK every neighbour and site index is range-checked in the
 * kernels; an index out of range sets a flag and is replaced by 0 (the access
 * stays inside the array).  *flag = 1 if any index was out of range since the
 * last call (the flag is then cleared).  A normal build returns
 * HISQ_ERR_STATE (its indices are not checked); *flag is still written. */
hisq_status hisq_bounds_violations(hisq_ctx *ctx, int *flag);

/* ---- learned initial guess: gauge-covariant parallel-transport layers.
 * The paper has no learned part; these entry points serve a small network that
 * predicts the CG starting vector (CG still runs to the same true residual).
 * Channel tensors are (C, V, 3) complex64 on the device, full lattice, site
 * s = x + X*(y + Y*(z + Z*t)); weights are (Cout, Cin, 9) complex64 on the device,
 * hop 0 = identity, hop 1 + 2*mu + d = one-hop fat-link transport forward (d = 0,
 * from x + mu) or backward (d = 1, from x - mu) with the Dirac operator's phases
 * and signs, so weights (0, 1, ..., 1) give the fat-link part of D.
 * out_b(x) = sum_a sum_h w[b][a][h] (T_h in_a)(x); 1 <= Cin, Cout <= 16. */

/* out = layer(in) (adjoint = 0; Cout channels) or layer^dag(in) (adjoint = 1;
 * in has Cout channels, out Cin).  w_bf16 = 1 rounds the weights to BF16 (FP32
 * accumulation).  Ordered on the context's stream. */
hisq_status hisq_net_layer(hisq_ctx *ctx, int cin, int cout, const float *w_dev, int w_bf16, int adjoint,
                           const float *in_dev, float *out_dev);

/* gw[b][a][h] = sum_x sum_c gout_b(x)_c conj((T_h in_a)(x)_c): the gradient
 * dL/dconj(w) of a real loss L, given gout = dL/dconj(out). */
hisq_status hisq_net_wgrad(hisq_ctx *ctx, int cin, int cout, const float *in_dev, const float *gout_dev,
                           float *gw_dev);

/* One Adam step (Kingma & Ba 2015) on n real parameters; step counts from 1. */
hisq_status hisq_net_adam(hisq_ctx *ctx, int n, float *w_dev, const float *g_dev, float *m1_dev, float *m2_dev,
                          float lr, float beta1, float beta2, float eps, int step);

/* Device bytes held by the context. */
size_t hisq_device_bytes(const hisq_ctx *ctx);

/* Number of CUDA kernels this context has launched so far. */
unsigned long long hisq_kernel_launches(const hisq_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HISQ_H */
