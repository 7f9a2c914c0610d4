/*
 * nspt.h -- C ABI of the B300 (sm_103a) library for the NSPT hot path of the
 * twisted Eguchi-Kawai model: the truncated product of polynomial matrices
 * (Eqs. 4-5, Sec. 2), computed naively or by FFT-CONV (Sec. 2, Steps 1-5), its
 * backward, and one NSPT Langevin step of the four links (Eqs. 1-3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A "series" is T+1 coefficient matrices, each N x N complex128 stored
 *   row-major with interleaved (re, im) doubles.  A batch of series is
 *   [batch][T+1][N][N]; entry (i, j) of order k of batch element b sits at
 *   element ((b*(T+1) + k)*N + i)*N + j.
 * - Every data pointer is a DEVICE pointer (cudaMalloc / torch CUDA memory),
 *   8-byte aligned at least; the caller owns every buffer.  The library never
 *   allocates, synchronises or reads device memory back inside a call: all
 *   work is enqueued on `stream` (a cudaStream_t passed as void*, NULL = legacy
 *   default stream), so calls can be captured into CUDA graphs once the
 *   library has been initialised on the device (see nspt_init).
 * - Scratch memory comes from the caller: opts->workspace of at least
 *   nspt_workspace_size(...) bytes, 256-byte aligned.  Too small -> NSPT_ERR_WORKSPACE.
 * - Outputs must not overlap inputs (NSPT_ERR_ALIAS), except where stated.
 * - A call returns NSPT_OK or a negative nspt_status; no exception crosses the
 *   ABI.  NSPT_ERR_CUDA: a launch failed; nspt_last_error() names it.
 */
#ifndef NSPT_H
#define NSPT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NSPT_API __attribute__((visibility("default")))
#else
#define NSPT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nspt_status {
  NSPT_OK = 0,
  NSPT_ERR_ARG = -1,          /* bad size, NULL pointer, bad option, or a buffer in the wrong
                                 kind of memory (host memory where device memory is expected,
                                 or the reverse; checked with cudaPointerGetAttributes unless the
                                 stream is being captured into a graph) */
  NSPT_ERR_ALIAS = -2,        /* an output overlaps an input */
  NSPT_ERR_UNSUPPORTED = -3,  /* valid request the library does not implement */
  NSPT_ERR_WORKSPACE = -4,    /* opts->workspace missing or too small */
  NSPT_ERR_CUDA = -5,         /* CUDA runtime error (see nspt_last_error) */
  NSPT_ERR_TIMEOUT = -6,      /* a device-side bounded wait gave up */
  NSPT_ERR_DEVICE = -7        /* the device is not an sm_103 part */
} nspt_status;

/* algorithm of the star product */
enum { NSPT_ALGO_NAIVE = 0, /* Eq. 5: C_k = sum_l A_l B_{k-l}, (T+1)(T+2)/2 GEMMs */
       NSPT_ALGO_FFT = 1,   /* Sec. 2 Steps 1-5: M-point order FFT, M mode GEMMs, inverse FFT */
       NSPT_ALGO_AUTO = 2 };/* FFT when T >= 3, else naive (split form: FFT in the entry
                               points that have no naive split form) */

/* arithmetic of the mode GEMMs */
enum { NSPT_PREC_FP64 = 0,  /* plain FP64 everywhere (the paper's ZGEMM form) */
       NSPT_PREC_SPLIT = 1  /* FP64 spectra split into BF16 slices, tensor-core GEMMs with exact
                               FP32 partial sums, double-word recombination */ };

/* which call a workspace is sized for */
enum { NSPT_OP_MUL = 0, NSPT_OP_MUL_BACKWARD = 1, NSPT_OP_LANGEVIN = 2, NSPT_OP_MD = 3,
       NSPT_OP_UNITARIZE = 4 };

#define NSPT_RESCALE_AUTO (-1000)

typedef struct nspt_opts {
  int algo;            /* NSPT_ALGO_*; default NSPT_ALGO_AUTO */
  int prec;            /* NSPT_PREC_*; default NSPT_PREC_FP64; NSPT_PREC_SPLIT needs N <= 1024,
                          and the FFT form except in nspt_polymat_mul, nspt_polymat_mul_host,
                          nspt_polymat_mul_backward, nspt_tek_unitarize and
                          nspt_tek_wilson_loops (and their workspace queries), which also take
                          the naive form (else NSPT_ERR_UNSUPPORTED) */
  int fft_len;         /* M; 0 = smallest power of two >= 2(T+1); else a power of two
                          >= 2(T+1) and <= 512 (wrap-free linear convolution, Step 1) */
  int slices;          /* split form: BF16 slices per operand, 0 = default 6, range 2..8 */
  int complex_mode;    /* split form: real products per complex product of the mode GEMMs: 4 (the
                          complex product embedded in real MMAs; every entry point), or 3 (3M:
                          A_re B_re, A_im B_im, (A_re + A_im)(B_re + B_im); nspt_polymat_mul and
                          its workspace query only, with slices <= 6 and N <= 512, else
                          NSPT_ERR_UNSUPPORTED); 0 = 4 */
  int rescale_log2r;   /* per-order rescale A_k, B_k -> r^k A_k, r^k B_k with r = 2^rescale_log2r,
                          undone exactly on C (not part of the paper): FFT-CONV products (split
                          and FP64 forms, the FP64 backward excepted); naive split products
                          (an exponent shift of the slices of order k: no rounding, it only
                          keeps the double-float accumulator within the FP32 range); split
                          and FP64 FFT forms
                          of nspt_tek_langevin_step and
                          nspt_tek_md_trajectory, where it applies to every order transform
                          of the step (the map X_k -> r^k X_k commutes with every product and
                          sum of the step, so the result is the same in exact arithmetic and
                          small high orders keep their relative precision).
                          NSPT_RESCALE_AUTO: the integer log2r (smallest |log2r| among
                          equals) minimising the spread over the nonzero orders k of
                          y_k + 2 k log2r, y_k = log2 max|A_k| + log2 max|B_k| (the worst
                          order's relative error grows with that spread; a geometric decay
                          is flattened), among those that lift no order of A or B above
                          max(1, its largest order) and, in the split form, keep the scale
                          factors 2^(k log2r) within 2^+-120; TEK step: A = B = U; MD link
                          update: A = U, B = i eps P; refitted at every step or phase.
                          The fit runs on the device (a per-order maxima kernel and a
                          one-block fit kernel on `stream`), and the transforms read the
                          fitted exponent from the workspace, so nothing is read back and
                          the call can be captured in a CUDA graph; default 0 */
  void* workspace;     /* device scratch, >= nspt_workspace_size() bytes */
  size_t workspace_bytes;
} nspt_opts;

/* Fills *o with the defaults listed above (no workspace). */
NSPT_API void nspt_opts_default(nspt_opts* o);

/* One-time per-device set-up (function attributes, device check).  Every entry
 * point calls it implicitly; call it once before capturing a CUDA graph.
 * Returns NSPT_ERR_DEVICE when the current device is not sm_103. */
NSPT_API int nspt_init(void);

/* Bytes of device workspace the call `op` (NSPT_OP_*) needs for these sizes. */
NSPT_API size_t nspt_workspace_size(int op, int N, int T, int batch, const nspt_opts* opts);

/*
 * C = A star B, truncated at order T (Eq. 5), for `batch` independent pairs.
 *   A, B : [batch][T+1][N][N] complex128 (inputs)
 *   C    : [batch][T+1][N][N] complex128 (output; must not overlap A or B)
 * NAIVE: Eq. 5 directly.  FFT: Sec. 2 Steps 1-5 -- zero-pad the order axis to
 * M, forward transform with w = exp(+2 pi i/M) (Step 2), M mode-wise complex
 * GEMMs (Step 3), inverse transform with 1/M (Step 4), keep orders 0..T
 * (Step 5).  N >= 1, T >= 0, batch >= 1.
 * Split form, NAIVE: every order of A and B is sliced once from FP64 and each
 * of the (T+1)(T+2)/2 products A_l B_{k-l} is one tensor-core GEMM with its own
 * row and column exponents, summed over l in double-float (no transforms, so
 * no order's precision depends on the others' size).
 */
NSPT_API int nspt_polymat_mul(const void* A, const void* B, void* C, int N, int T, int batch,
                     const nspt_opts* opts, void* stream);

/*
 * Backward of C = A star B for a real loss L with gC = dL/dRe C + i dL/dIm C
 * (the truncated correlations obtained by differentiating Eq. 5):
 *   gA_j = sum_{k=j}^{T} gC_k (B_{k-j})^H,   gB_j = sum_{k=j}^{T} (A_{k-j})^H gC_k.
 * FFT form: gA~_p = G~_p (B~_p)^H and gB~_p = (A~_p)^H G~_p, inverse
 * transform, keep 0..T (wrap-free for M >= 2T+1).  Split form, NAIVE: one
 * tensor-core GEMM per pair (k, k - j), every order sliced once from FP64,
 * double-float sums; a fixed rescale_log2r shifts the slices' exponents (gC_k
 * by -k log2r, A_m and B_m by m log2r) and is undone on the output.
 *   A, B, gC : [batch][T+1][N][N] inputs;  gA, gB : outputs, either may be NULL.
 */
NSPT_API int nspt_polymat_mul_backward(const void* A, const void* B, const void* gC, void* gA, void* gB,
                              int N, int T, int batch, const nspt_opts* opts, void* stream);

/*
 * One NSPT Langevin step of the TEK model for `batch` independent streams of
 * four link series (Eqs. 1-3 in the rescaled fictitious time):
 *   z_{mu nu} = exp(2 pi i flux eps_{mu nu}/L), eps = +1 (mu<nu), -1 (mu>nu), N = L^2;
 *   S_mu = U_mu star sum_{nu != mu} [z_{mu nu} U_nu U_mu^+ U_nu^+ + conj(z_{mu nu}) U_nu^+ U_mu^+ U_nu];
 *   F^(k) = i[S^(k) - S^(k)^H - Tr(S^(k) - S^(k)^H)/N];
 *   X^(0) = 0, X^(1) = eps F^(1) + sqrt(2 eps) eta, X^(k>=2) = eps F^(k);
 *   U <- exp_star(i X) star U   (order 0 of U unchanged).
 *   U   : [batch][4][T+1][N][N], updated IN PLACE
 *   eta : [batch][4][N][N] traceless Hermitian Gaussian noise (input, required)
 *   F   : [batch][4][T+1][N][N] drift of the input links (output, may be NULL)
 * N must be a perfect square L^2 with gcd(flux, L) = 1; eps > 0.
 */
NSPT_API int nspt_tek_langevin_step(void* U, const void* eta, void* F, int N, int T, int batch, int flux,
                           double eps, const nspt_opts* opts, void* stream);

/*
 * Order-by-order unitarity projection of link series, in place (Sec. 2 names a
 * unitarity projection and zero-mode subtraction among the NSPT steps and prints no
 * algorithm; this is the polar factor in the truncated ring, optionally followed by
 * the removal of the U(1) (trace) mode):
 *   V = U * (U^+ * U)^(-1/2) = U * sum_{n=0}^{T} binom(-1/2, n) D^n,  D = U^+ * U - 1,
 * with star products (Eq. 5) in the form of opts (naive or FFT, FP64 or split) and
 * the series dagger (U^+)^(k) = (U^(k))^H.  Order 0 of every series must be unitary; it
 * is left exactly unchanged (D^(0) is taken as 0).  Then V^+ * V = 1 through order T,
 * and a unitary series is its own projection (up to rounding).
 * special = 1 also removes the U(1) phase a(g) = Im Tr log(U0^+ V(g)) (a_0 = 0),
 *   V <- V * exp(-i a / N)   (a scalar series times the matrix series),
 * so that det V = det U^(0) through order T; a is taken from Jacobi's formula,
 * a_k = Im Tr(V^+ * V')_(k-1) / k with V'_j = (j+1) V_(j+1) (one more product).
 * special = 0 stops at the polar factor.  Other values: NSPT_ERR_ARG.
 *   U : [batch][T+1][N][N] complex128, updated in place (a link tensor
 *       [b][4][T+1][N][N] is batch = 4 b series)
 * T + 2 products (T + 3 with special = 1) per call.  Workspace: NSPT_OP_UNITARIZE.
 * A fixed rescale applies to every product; NSPT_RESCALE_AUTO fits one per product.
 * The projection is well conditioned for the series it is for (unitary ones with a small
 * drift); far from unitary, its high orders come out of the cancellation of much larger
 * terms and lose accuracy.
 */
NSPT_API int nspt_tek_unitarize(void* U, int N, int T, int batch, int special, const nspt_opts* opts,
                                void* stream);

/*
 * Grouped products: `count` (<= 64) independent products of uneven sizes,
 * C_i = A_i star B_i with N_i, T_i and batch_i each, by FFT-CONV with
 * M_i = smallest power of two >= 2(T_i + 1) (opts->fft_len must be 0).
 * Split form: the mode GEMMs of all products run in ONE persistent
 * tensor-core launch whose per-product tensor maps travel in the kernel
 * parameters, so the call needs no device-side table and can be captured in
 * a CUDA graph (after nspt_init).  The products' transforms and slicing (before)
 * and inverse transforms (after) run on library-owned side streams forked from
 * and joined back to `stream` by events (graph edges under capture); work
 * queued on `stream` after the call starts after all of it.  FP64 form: the products run one after
 * another.  `descs` is a HOST array; pointers inside are device pointers with
 * the layout of nspt_polymat_mul.  Workspace: nspt_workspace_size_grouped().
 */
typedef struct nspt_polymat_desc {
  const void* A;
  const void* B;
  void* C;
  int N, T, batch;
} nspt_polymat_desc;

NSPT_API size_t nspt_workspace_size_grouped(const nspt_polymat_desc* descs, int count, const nspt_opts* opts);
NSPT_API int nspt_polymat_mul_grouped(const nspt_polymat_desc* descs, int count, const nspt_opts* opts,
                                      void* stream);

/*
 * Autotuner of the split form's tensor-core tile width (128 x 32, 128 x 40 or
 * 128 x 48 output tiles, i.e. 64-, 80- or 96-column MMAs; at width 40 the left
 * operand's digit slices are held in tensor memory): times the grouped mode-GEMM
 * launch of this group signature (every product's N and M x batch, slices)
 * with each width on the caller's workspace (sized as for
 * nspt_polymat_mul_grouped, contents overwritten), keeps the fastest for
 * later calls with the same signature (a single product is a group of one),
 * and writes it to *chosen_bn.  cache_path (may be NULL): a text file of
 * "signature width" lines read before timing and appended after.  Synchronises
 * `stream`; call it before any graph capture.
 */
NSPT_API int nspt_autotune_grouped(const nspt_polymat_desc* descs, int count, const nspt_opts* opts,
                                   const char* cache_path, int* chosen_bn, void* stream);

/*
 * NSPT molecular dynamics of the TEK model, the integrator of the paper
 * (symplectic MD with periodic momentum refresh, Sec. 2; Eq. 3 with beta
 * absorbed by the rescaled time).  The momentum series P~ = sum_{k>=1} g^k P^(k)
 * has no order g^0; the drift's order 0 is dropped.  Leapfrog step of size eps:
 *   P_half = P + eps/2 F(U);  U <- exp_star(i eps P_half) star U;  P = P_half + eps/2 F(U),
 * with F and exp_star exactly as in nspt_tek_langevin_step (order 0 of U is
 * never rewritten).
 *   U   : [batch][4][T+1][N][N] link series, updated in place
 *   P   : [batch][4][T+1][N][N] momentum series, updated in place (order 0 kept 0)
 *   eta_refresh : [batch][4][N][N] traceless Hermitian Gaussian, or NULL; when given,
 *         the momentum is refreshed to P^(1) = eta, P^(k != 1) = 0 before the steps
 *   nsteps >= 0 leapfrog steps of size eps > 0.  Workspace: NSPT_OP_MD.
 */
NSPT_API int nspt_tek_md_trajectory(void* U, void* P, const void* eta_refresh, int N, int T, int batch, int flux,
                                    double eps, int nsteps, const nspt_opts* opts, void* stream);

/*
 * Seeded noise for nspt_tek_langevin_step (and the momentum refresh of
 * nspt_tek_md_trajectory): `count` traceless Hermitian N x N matrices with
 * the step's normalisation (eta = sum_a xi_a T^a, xi_a ~ N(0,1) on generators
 * with Tr(T^a T^b) = delta^ab: E|eta_ij|^2 = 1 off the diagonal), drawn from the
 * counter-based generator Philox4x32-10 (Salmon et al., SC 2011).  Every value
 * depends only on (seed, t, matrix, position), t = counter + *d_counter:
 *   key = (seed mod 2^32, seed div 2^32); block b of matrix c uses the counter
 *   (b, c, t mod 2^32, t div 2^32) and gives Gaussians 2b, 2b+1 of the matrix
 *   (row-major) by Box-Muller on two 53-bit uniforms,
 *   u1 = ((w0 >> 5) 2^26 + (w1 >> 6) + 1) 2^-53, u2 = ((w2 >> 5) 2^26 + (w3 >> 6)) 2^-53,
 *   z_2b = r cos(2 pi u2), z_2b+1 = r sin(2 pi u2), r = sqrt(-2 ln u1);
 *   eta_ij = (z_{iN+j} + i z_{jN+i})/sqrt(2) for i < j, eta_ji = conj(eta_ij),
 *   eta_ii = z_{iN+i} - mean_k z_{kN+k}.
 *   eta       : [count][N][N] complex128 (output, device)
 *   d_counter : device word or NULL; when given, t = counter + *d_counter and the
 *               call adds 1 to *d_counter after drawing, so a captured CUDA graph
 *               draws fresh noise at every replay.
 * Two launches on `stream`; no workspace.  1 <= N <= 4096, count >= 1.
 */
NSPT_API int nspt_tek_noise(void* eta, int N, int count, unsigned long long seed, unsigned long long counter,
                            unsigned long long* d_counter, void* stream);

/*
 * C = A star B (as nspt_polymat_mul, same opts) for series in HOST memory --
 * pinned (page-locked) for the copies to overlap; no counterpart in the paper.
 * The batch goes through the GPU one element at a time in two device slots:
 * the host-to-device copies of element i+1 and the device-to-host copy of
 * element i-1 run on two library-owned streams while element i is multiplied
 * on `stream`.  Work queued on `stream` after the call starts after the last
 * element of C has reached host memory (synchronise `stream` before reading
 * C; A and B must stay unchanged until then).  A call starts after the work
 * already queued on `stream`, except when it continues the previous call of
 * this device (same workspace, stream and element size): its copies in then
 * wait only for the device slot they reuse, so they overlap the end of that
 * call -- between such calls the workspace must not be used by other work.
 * Enqueues are serialised per device.
 *   A, B : host [batch][T+1][N][N] complex128;  C : host, same shape, no overlap
 * Workspace: nspt_workspace_size_host() bytes of DEVICE memory (two slots of
 * three series plus the product workspace of one element).
 * NSPT_RESCALE_AUTO fits the rescale per batch element (on the device).
 */
NSPT_API size_t nspt_workspace_size_host(int N, int T, int batch, const nspt_opts* opts);
NSPT_API int nspt_polymat_mul_host(const void* A, const void* B, void* C, int N, int T, int batch,
                                   const nspt_opts* opts, void* stream);

/*
 * Perturbative Wilson loops of the TEK links, the observable the NSPT runs of
 * the paper measure (Sec. 1; the loops are the standard TEK ones, the twist
 * factor z^(ab) making the twist-eater vacuum value 1):
 *   W(a, b)^(k) = 1/(12 N) sum_{mu != nu} z_{mu nu}^(ab) Tr[(U_mu^a U_nu^b (U_mu^a)^+ (U_nu^b)^+)^(k)]
 * for 1 <= a, b <= amax <= 8, with star products in the form of opts (FP64 or
 * split, naive or FFT).  W(b, a) = conj(W(a, b)); the real part of W(a, a) and
 * of (W(a, b) + W(b, a)) / 2 is the loop average.
 *   U : [batch][4][T+1][N][N] link series (input; N = L^2, gcd(flux, L) = 1)
 *   W : [batch][amax][amax][T+1] complex128 (output, [b][a-1][b'-1][k])
 * Workspace: nspt_workspace_size_wilson().
 */
NSPT_API size_t nspt_workspace_size_wilson(int N, int T, int batch, int amax, const nspt_opts* opts);
NSPT_API int nspt_tek_wilson_loops(const void* U, int N, int T, int batch, int flux, int amax, void* W,
                                   const nspt_opts* opts, void* stream);

/*
 * Single stages of FFT-CONV, for stage timing and per-stage tests.
 * nspt_order_fft: Steps 1-2 -- At[b][p] = sum_{k<=T} A[b][k] w^(kp), p = 0..M-1,
 *   A : [batch][T+1][N][N] -> At : [batch][M][N][N], w = exp(+2 pi i/M).
 * nspt_order_ifft: Steps 4-5 -- C[b][k] = (1/M) sum_p Ct[b][p] w^(-kp), k = 0..T,
 *   Ct : [batch][M][N][N] -> C : [batch][T+1][N][N].
 * M: power of two, 2(T+1) <= M <= 512.  FP64 arithmetic.
 */
NSPT_API int nspt_order_fft(const void* A, void* At, int N, int T, int batch, int M, void* stream);
NSPT_API int nspt_order_ifft(const void* Ct, void* C, int N, int T, int batch, int M, void* stream);

/*
 * Instrumentation (host side; no effect on results).
 * nspt_launch_count: kernel launches enqueued by this library since load.
 * nspt_profile_begin: from now on, bracket every library kernel launch with a
 *   CUDA event pair recorded on its own stream (up to max_records launches).
 * nspt_profile_end: wait for those events and sum their durations per stage
 *   (total_ms[s], launches[s] for s < nstages); returns the records used.
 * nspt_stage_name: name of stage s (fft_fwd, slice, gemm_mode, fft_inv,
 *   gemm_conv, tek_elementwise, gemm_tc, other, md_force, md_link).  The last
 *   two are phases of nspt_tek_md_trajectory (force with the momentum kicks,
 *   link update): scopes around many launches whose "launches" count is the
 *   number of scopes; their time overlaps the kernel stages inside them.
 */
NSPT_API long long nspt_launch_count(void);
NSPT_API int nspt_profile_begin(int max_records);
NSPT_API int nspt_profile_end(int nstages, double* total_ms, long long* launches);
NSPT_API const char* nspt_stage_name(int stage);

/*
 * Device-side status of the last split-precision call that used this
 * workspace: waits inside the tensor-core GEMM are bounded (2 s); a wait that
 * gives up records a code in the first word of opts->workspace and the kernel
 * drains its own copies, frees its tensor memory and returns.  This call
 * synchronises `stream`, reads the word and returns NSPT_ERR_TIMEOUT if it is
 * set, else NSPT_OK.  Not for use inside graph capture.
 */
NSPT_API int nspt_device_status(const nspt_opts* opts, void* stream);

/*
 * Test hook (no counterpart in the paper): budget in ns of the tensor-core
 * GEMMs' device-side waits that may abandon a launch (default 2 s); applies to
 * launches enqueued afterwards.  With a negative budget such a wait gives up
 * as soon as its barrier is not ready at the first try, so that the launch
 * exits cleanly -- the copies and MMAs already in flight are still drained --
 * and nspt_device_status reports NSPT_ERR_TIMEOUT: the timeout path can be
 * exercised without a hung GPU.
 * Results of a launch that gave up are undefined.
 */
NSPT_API int nspt_debug_wait_budget(long long ns);

/*
 * Test hook, host only (no GPU needed): the pair-GEMM schedule of the naive split
 * form at truncation order T (0..255) -- kind 0: the product's pairs (l, k - l);
 * 1: the backward's gA pairs; 2: its gB pairs.  Writes 7 ints per batched GEMM,
 * (launch, accumulator, left slot, right slot, first output order, count, plain),
 * for as many as fit in `cap` ints of `out`, and returns the number of GEMMs
 * (NSPT_ERR_ARG for a bad T or kind).  Within a GEMM the slots rise by 1 and the
 * output order by 2 per pair.  Product slots are orders (l, then k - l); the
 * backward's operand indexed by m = k - j sits at slot T - m, the other at slot k.
 */
NSPT_API int nspt_debug_pair_schedule(int T, int kind, int* out, int cap);

/*
 * Stage entry points of the split form, for stage tests and timing.
 *
 * nspt_split_slices (FFT-CONV Step 3 operand preparation): cuts each of the Q
 * N x N complex128 matrices X[q] into S BF16 digit planes.  Output row r is
 * row r of X[q] (trans = 0) or column r (trans = 1), conjugated if conj.
 *   slices : bf16 [Q][S][P][N][Kp], Kp = N rounded up to a multiple of 8,
 *            P = 2 for a left operand (right = 0) and P = 3 for a right
 *            operand (right = 1); plane (q, i, c) holds digit i of the real
 *            (c = 0) / imaginary (c = 1) parts, and for P = 3 plane c = 2 holds
 *            the negated real part; digits are stored as d * 2^(-8 i), |d| <= 128;
 *   exps   : int [Q][N]; row r satisfies
 *            row[k] = 2^(exps[q][r] - 7) sum_i plane(q, i, ., r, k)
 *            up to 2^(exps[q][r] - 8S).
 *
 * nspt_split_mode_gemm (FFT-CONV Step 3, Sec. 2): Ct_q = A_q B_q for q < Q
 * from the slices of A_q (trans = 0, right = 0) and of B_q (trans = 1,
 * right = 1), on the tensor cores.  Ct : [Q][N][N] float4 (re_hi, re_lo,
 * im_hi, im_lo), the double-float result; err : device int, set non-zero if a
 * bounded wait gave up.  2 <= S <= 8, N <= 1024, Q <= 65535 (slicing).
 */
NSPT_API int nspt_split_slices(const void* X, void* slices, int* exps, int N, int Q, int S, int trans, int conj,
                               int right, void* stream);
NSPT_API int nspt_split_mode_gemm(const void* slA, const void* slB, const int* expA, const int* expB, void* Ct, int N,
                                  int Q, int S, int* err, void* stream);

/*
 * Allocation-free FFT-CONV product (no counterpart in the paper): the same
 * result as nspt_polymat_mul with NSPT_ALGO_FFT, NSPT_PREC_FP64 and the default
 * M, for callers that cannot allocate device memory (code in host callbacks or
 * allocator hooks, processes whose device memory another framework owns, or
 * plug-in hosts that pass only input and output buffers).  Its scratch -- the
 * three spectra, 3 * batch * M * N^2 * 16 bytes -- lives in one fixed 32 MiB
 * device array inside the library, which every GPU that loads the library
 * holds until the process exits; larger problems return NSPT_ERR_WORKSPACE.
 *   A, B : [batch][T+1][N][N] complex128 device inputs;  C : output, no overlap.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture.  A device reset (cudaDeviceReset) between
 * calls is not supported: the kept address would no longer be valid.  All calls
 * share the one array, which keeps the last call's contents (each call
 * overwrites every entry it reads): calls that can overlap on the GPU -- on
 * different streams without ordering -- race and must not be issued.
 */
NSPT_API int nspt_polymat_mul_fft_noalloc(const void* A, const void* B, void* C, int N, int T, int batch,
                                          void* stream);

/* Static description of a status code. */
NSPT_API const char* nspt_status_string(int status);
/* Name of the last CUDA error seen by this thread ("no error" if none). */
NSPT_API const char* nspt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NSPT_H */
