/*
 * hoscf.h - C ABI of the GB300 (sm_103a) HOSCF / iHOSCF library.
 *
 * Best rank-one approximation of a dense order-d tensor A (I_1 x ... x I_d):
 * find sigma and unit vectors u^(1..d) maximising A x_1 u^(1) ... x_d u^(d)
 * (paper Sec. 2, eq. 2.3), by the higher-order self-consistent-field
 * iteration (Algorithm 1) and its Rayleigh-quotient variant (Sec. 4.4).
 *
 * Conventions used by every entry point
 *   - Tensors are dense, row-major (last index fastest), contiguous.
 *   - Factor vectors are passed concatenated: u^(1) first, u^(n) starting at
 *     offset I_1 + ... + I_{n-1}; total length n_tot = I_1 + ... + I_d.
 *   - Coupling blocks A_{m,n} (eq. 3.3) are stored for m < n only, packed in
 *     lexicographic (m, n) order, each row-major I_m x I_n; total length
 *     P = sum_{m<n} I_m I_n.  J(x) of eq. (3.2) is these blocks divided by
 *     (d - 1), placed symmetrically with zero diagonal blocks.
 *   - "device" pointers are CUDA device memory of the handle's device;
 *     "host" pointers are ordinary host memory.  Streams are cudaStream_t
 *     passed as void* (NULL = the legacy default stream).
 *   - The caller owns every buffer it passes.  The handle owns an internal
 *     workspace (grown on demand with cudaMalloc; hoscf_workspace_size
 *     reports what a problem needs).
 *   - No call aborts or prints.  Each returns an hoscf_status; on failure
 *     hoscf_last_error() gives a message.  A handle is used by one host
 *     thread and one stream at a time.
 */
#ifndef HOSCF_H
#define HOSCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HOSCF_MAX_ORDER 8

typedef enum {
    HOSCF_OK = 0,
    HOSCF_EINVAL = 1,          /* bad argument: order, dims, null or misaligned pointer, zero block */
    HOSCF_ENOMEM = 2,          /* workspace allocation failed */
    HOSCF_ECUDA = 3,           /* a CUDA call failed (message has the CUDA error string) */
    HOSCF_NOT_CONVERGED = 4,   /* max_iter reached; outputs hold the last certified iterate */
    HOSCF_NONFINITE = 5,       /* NaN/Inf met in the tensor, the factors or a solve */
    HOSCF_TIMEOUT = 6,         /* a bounded device-side wait gave up (no hang) */
    HOSCF_EUNSUPPORTED = 7     /* a valid request this build does not handle */
} hoscf_status;

typedef enum {
    HOSCF_F32 = 0,             /* IEEE float32 */
    HOSCF_BF16 = 1,            /* bfloat16, no scale */
    HOSCF_F8E4M3 = 2,          /* FP8 e4m3 (fn), one float32 scale per 128 consecutive elements */
    HOSCF_F16 = 3              /* IEEE binary16, no scale */
} hoscf_dtype;

typedef enum {
    HOSCF_VARIANT_HOSCF = 0,   /* Algorithm 1 */
    HOSCF_VARIANT_IHOSCF = 1,  /* Sec. 4.4: RQI with J built at the new point x_k (one more pass) */
    HOSCF_VARIANT_IHOSCF_PREV = 2, /* Sec. 4.4 read with J_{k-1} (tracks plain HOSCF) */
    HOSCF_VARIANT_JACOBI_HOPM = 3, /* Sec. 1 / 6.1 comparison method: every factor at once,
                                      u^(n) <- A x_{k!=n} u^(k) / ||.||, from the same blocks */
    HOSCF_VARIANT_ASVD = 4         /* Sec. 1 comparison method (orders 2 and 3): with u^(f)
                                      fixed, (u^(m), u^(n)) <- the largest singular pair of
                                      the block A_{m,n} = A x_f u^(f), f = 1, 2, 3, 1, ...
                                      (Gauss-Seidel); the pair negated together when
                                      <a, u^(m)> + <b, u^(n)> < 0; one eigen step per pair */
} hoscf_variant;

typedef struct hoscf_handle hoscf_handle;

/* A dense tensor in device memory. */
typedef struct {
    int order;                 /* d, 2 .. HOSCF_MAX_ORDER */
    const int64_t* dims;       /* host, d entries, each >= 1 */
    hoscf_dtype dtype;
    const void* data;          /* device, row-major contiguous, 16-byte aligned */
    const float* scales;       /* device, HOSCF_F8E4M3 only: ceil(N/128) float32 scales, else NULL */
} hoscf_tensor_desc;

typedef struct {
    double tol;                /* stop when r = ||g - sigma u||_2 / |sigma| <= tol (see hoscf_solve) */
    int max_iter;              /* maximum eigen steps (Alg. 1 loop trips) */
    int variant;               /* hoscf_variant */
    double eig_tol;            /* Lanczos stop: Ritz residual <= eig_tol * |theta| */
    int eig_max_steps;         /* Lanczos basis size limit (<= 128) */
    double eig_adapt;          /* hoscf_solve: eigen steps stop at the looser
                                  max(eig_tol, min(1e-3, eig_adapt * r)), r the
                                  residual just certified (inexact SCF); 0 = off */
    const hoscf_tensor_desc* refine; /* precision form: FP32 copy of the same tensor, or NULL */
    double switch_tol;         /* precision form: residual at which passes move to `refine` */
    int64_t timeout_ns;        /* bound on every device-side wait (0 = 2 s) */
    int batch_threads;         /* hoscf_solve_batched: threads per CTA (256, 512 or 1024;
                                  0 = 512); chosen by the package's autotuner */
    int batch_faces;           /* hoscf_solve_batched: at most this many faces (T[o][:][:],
                                  o over the leading modes) staged and folded per group,
                                  1 .. 32 (0 = 32); chosen by the autotuner */
    int switch_predict;        /* precision form: move to `refine` one pass early when the
                                  next residual is predicted to reach switch_tol from
                                  1 (default): the last contraction r_k / r_{k-1} - suits
                                  problems whose first steps show their rate; 2: the
                                  slower of the last two - suits a fast first step
                                  followed by a slow tail; 0: no prediction */
} hoscf_opts;

typedef struct {
    int iters;                 /* eigen steps taken */
    int passes;                /* block constructions (TTVc passes), all tensors */
    int passes_refine;         /* of which on the `refine` tensor */
    int rqi_accepts;           /* iHOSCF: RQI iterates kept */
    double resid;              /* KKT residual r at the returned point */
    double resid_4_1;          /* eq. (4.1) evaluated at the returned point */
    double sigma_raw;          /* sigma before the final sign fix */
} hoscf_info;

/* Handle lifetime.  `device` is a CUDA ordinal. */
hoscf_status hoscf_create(hoscf_handle** h, int device);
hoscf_status hoscf_destroy(hoscf_handle* h);
const char* hoscf_last_error(const hoscf_handle* h);

/* Defaults: tol 1e-6, max_iter 200, HOSCF, eig_tol 1e-10, eig_max_steps 64,
 * eig_adapt 1e-3, refine NULL, switch_tol 1e-3, timeout 2 s, switch_predict 1. */
hoscf_status hoscf_opts_default(hoscf_opts* opts);

/* Bytes of handle workspace a solve of this shape and dtype needs (host args). */
hoscf_status hoscf_workspace_size(int order, const int64_t* dims, int dtype, size_t* bytes);

/*
 * hoscf_ttvc_blocks - all coupling blocks in one read of the tensor.
 * Eq. (3.3): H[(m,n)] = A x_{k != m,n} u^(k) for every m < n (Alg. 1 line 4).
 *   T  tensor descriptor (device data).
 *   u  device, n_tot floats: the d factor vectors, used as given (the
 *      paper's blocks use unit vectors, eq. 3.4; no normalisation is done).
 *   H  device, P floats, packed as described above (overwritten).
 * Asynchronous on `stream`; FP32 accumulation.  Errors: EINVAL (order < 2
 * or > 8, a dim < 1, null pointer, F8 without scales), ENOMEM, ECUDA.  A
 * device-side wait that gives up (TIMEOUT) cannot be known when the call
 * returns: it is recorded in the handle's device status word, H is then
 * invalid, and hoscf_device_status reports it.
 */
hoscf_status hoscf_ttvc_blocks(hoscf_handle* h, const hoscf_tensor_desc* T, const float* u,
                               float* H, void* stream);

/*
 * hoscf_device_status - failures the asynchronous calls (hoscf_ttvc_blocks,
 * hoscf_eig_step, hoscf_rqi_step) recorded on the device (no counterpart in
 * the paper).  Synchronises `stream`, reads the handle's device status word
 * and clears it.  Returns OK, TIMEOUT (a bounded device wait gave up; the
 * outputs of the call that hit it, and of later calls on the handle until
 * this one, are invalid) or NONFINITE.  The synchronous calls hoscf_solve,
 * hoscf_solve_greedy and hoscf_backward report their own device failures and
 * start from a clear word, discarding an unread one.
 */
hoscf_status hoscf_device_status(hoscf_handle* h, void* stream);

/*
 * hoscf_eig_step - the largest-magnitude eigenpair of J (Alg. 1 line 5),
 * then the block normalisation of lines 6-9.
 *   order, dims   host.
 *   H             device, P floats (packed blocks; J = blocks / (d-1)).
 *   x_prev        device, n_tot doubles: warm start and sign reference
 *                 (need not be normalised; must be nonzero).
 *   x_out         device, n_tot doubles: unit eigenvector with
 *                 <x_out, x_prev> >= 0.
 *   u_out         device, n_tot floats, or NULL: x_out's blocks each scaled
 *                 to unit length (eq. 3.4; a zero block stays zero).
 *   lambda_out    device, 1 double: the eigenvalue (ties between +l and -l
 *                 resolve to +l).
 * Lanczos with full reorthogonalisation (stop: Ritz residual <= tol*|theta|
 * with tol = max(eig_tol, min(1e-3, eig_adapt * sqrt(d) * r0)), r0 the
 * relative residual ||J x - rho x|| / |rho| of the normalised x_prev, or
 * tol = eig_tol when eig_adapt = 0; at most eig_max_steps; opts may be NULL
 * for defaults).  The start-point certificate, the tridiagonal matrix, the
 * Ritz value and the final normalisation are FP64; the Lanczos vectors are
 * FP32 like the blocks.  Asynchronous on `stream`; device-side failures go to
 * the handle's status word (hoscf_device_status).
 */
hoscf_status hoscf_eig_step(hoscf_handle* h, int order, const int64_t* dims, const float* H,
                            const double* x_prev, double* x_out, float* u_out,
                            double* lambda_out, const hoscf_opts* opts, void* stream);

/*
 * hoscf_rqi_step - one Rayleigh-quotient step of iHOSCF (Sec. 4.4) from the
 * factors u: x~ = [u^(1); ...; u^(d)] / sqrt(d), rho = x~^T J x~ / x~^T x~,
 * y = (J - rho I)^{-1} x~, then the block normalisation of Alg. 1 lines 6-9.
 * The step iHOSCF's solve takes after each eigen step (the acceptance rule
 * stays in hoscf_solve).
 *   order, dims   host.
 *   H             device, P floats (packed blocks; J = blocks / (d-1)).
 *   u             device, n_tot floats: the factors (each block unit length,
 *                 as hoscf_eig_step returns them; not renormalised).
 *   x_out         device, n_tot doubles, or NULL: y / ||y|| with
 *                 <x_out, x~> >= 0.
 *   u_out         device, n_tot floats: x_out's blocks each scaled to unit
 *                 length (a zero block stays zero).
 *   rho_out       device, 1 double, or NULL: the shift rho.
 * The solve is Lanczos on the Krylov space of x~ with a shifted tridiagonal
 * solve (stop: relative Galerkin residual <= eig_tol; at most eig_max_steps
 * steps); FP32 vectors, FP64 tridiagonal and normalisation.  Asynchronous on
 * `stream`.  Errors: EINVAL (order, dims, a null H / u / u_out), NONFINITE
 * (a zero x~), ECUDA.
 */
hoscf_status hoscf_rqi_step(hoscf_handle* h, int order, const int64_t* dims, const float* H,
                            const float* u, double* x_out, float* u_out, double* rho_out,
                            const hoscf_opts* opts, void* stream);

/*
 * hoscf_solve - HOSCF / iHOSCF (Algorithm 1 and Sec. 4.4).
 *   T       tensor (device data; F32, BF16 or F8E4M3).
 *   u0      device, n_tot floats: initial guess; each block is normalised
 *           (a zero or non-finite block gives EINVAL).
 *   opts    host, or NULL for defaults.
 *   u_out   device, n_tot floats: the factors, after Alg. 1 lines 12-15
 *           and the sign gauge (for n >= 2 the largest-|.| entry of u^(n),
 *           lowest index on ties, is positive; sigma >= 0).
 *   sigma_out host double.  info host, or NULL.
 * Each iteration builds the blocks at the current factors, certifies that
 * point with r = ||g - sigma u||_2 / |sigma| (g_n = A x_{k!=n} u^(k) from the
 * blocks, sigma = mean_n <u_n, g_n>; the KKT system 2.4) and stops there when
 * r <= tol; otherwise it takes the eigen step.  With opts->refine set, passes
 * run on T until r <= switch_tol, r sets no new low for 64 iterations (or
 * half of max_iter is spent), or the next iterate is predicted to reach
 * switch_tol (opts->switch_predict), and on `refine` (FP32) afterwards.
 * Synchronous: returns when the outputs are final.  NOT_CONVERGED after
 * max_iter (outputs = last certified iterate), NONFINITE, TIMEOUT, EINVAL,
 * ENOMEM, ECUDA; EUNSUPPORTED for the ASVD variant on orders above 3.
 */
hoscf_status hoscf_solve(hoscf_handle* h, const hoscf_tensor_desc* T, const float* u0,
                         const hoscf_opts* opts, float* u_out, double* sigma_out,
                         hoscf_info* info, void* stream);

/*
 * Sharded form (tensor split over ranks, one GPU each; no paper counterpart
 * beyond its multi-node scaling runs of Sec. 6.2).  A rank holds the slab of
 * rows [row0, row0 + rows) of mode 1, itself a dense row-major tensor of
 * dims (rows, I_2, ..., I_d) because mode 1 is the slowest index.
 *
 * hoscf_ttvc_blocks_slab - this slab's contribution to every coupling block
 * of the whole tensor (eq. 3.3), in the whole tensor's packed layout:
 *   T     the slab (device data; F32, BF16 or F8E4M3 with its own scales).
 *   row0  first mode-1 row of the slab; dim0 = I_1 of the whole tensor
 *         (row0 >= 0, row0 + rows <= dim0).
 *   u     device, n_tot = dim0 + I_2 + ... + I_d floats (whole factors).
 *   H     device, P floats of the whole tensor (overwritten): A_{1,n} holds
 *         the slab's rows at rows row0.. and zeros elsewhere; A_{m,n} with
 *         m >= 2 holds the slab's partial sum over its mode-1 rows.
 * The elementwise sum of H over all slabs of a partition of mode 1 is the
 * whole tensor's blocks.  Asynchronous on `stream`.  Errors as for
 * hoscf_ttvc_blocks, plus EINVAL for rows outside mode 1.
 */
hoscf_status hoscf_ttvc_blocks_slab(hoscf_handle* h, const hoscf_tensor_desc* T, int64_t row0,
                                    int64_t dim0, const float* u, float* H, void* stream);

/* The caller's collective: sum `count` floats at device pointer H over all
 * ranks, in place, ordered on `stream` (e.g. an NCCL all-reduce); return 0 on
 * success. */
typedef int (*hoscf_reduce_fn)(float* H, int64_t count, void* stream, void* user);

typedef struct {
    int64_t row0;              /* first mode-1 row this rank's slab holds */
    int64_t dim0;              /* I_1 of the whole tensor */
    hoscf_reduce_fn reduce;    /* SUM over ranks, in place (required) */
    void* user;                /* passed to reduce */
} hoscf_shard;

/*
 * hoscf_solve_sharded - hoscf_solve on a tensor sharded by slabs of mode 1.
 * Every rank calls it with its slab T, the same u0 (whole factors, n_tot
 * floats) and the same opts; each pass is hoscf_ttvc_blocks_slab followed by
 * shard->reduce on the whole blocks, and everything after the pass (the
 * certificate, the eigen step, the final fix) runs on the whole blocks on
 * every rank, so all ranks return the same u_out and sigma.  opts->refine,
 * when set, is the FP32 slab of the same rows.  A reduce callback that
 * returns nonzero ends the call with ECUDA.  Other statuses as hoscf_solve.
 */
hoscf_status hoscf_solve_sharded(hoscf_handle* h, const hoscf_tensor_desc* T,
                                 const hoscf_shard* shard, const float* u0,
                                 const hoscf_opts* opts, float* u_out, double* sigma_out,
                                 hoscf_info* info, void* stream);

/*
 * hoscf_solve_batched - `count` independent F32 tensors of orders 3..4 and
 * small dims, solved in one persistent launch (no paper counterpart; the
 * per-tensor algorithm is hoscf_solve's HOSCF variant).
 *   T        host array of `count` descriptors (device data).
 *   u0       host array of `count` device pointers (n_tot floats each).
 *   u_out    host array of `count` device pointers (n_tot floats each).
 *   sigma_out host, count doubles.  infos host, count entries, or NULL.
 * Each tensor is solved by one CTA of a single persistent kernel (largest
 * tensors first from an atomic work queue); the launch is captured in a CUDA
 * graph on the handle's own stream and replayed for a repeated batch.
 * Synchronous (the caller's stream is synchronised first).  Returns the
 * worst per-tensor status.
 */
hoscf_status hoscf_solve_batched(hoscf_handle* h, int count, const hoscf_tensor_desc* T,
                                 const float* const* u0, const hoscf_opts* opts,
                                 float* const* u_out, double* sigma_out, hoscf_info* infos,
                                 void* stream);

/*
 * hoscf_backward - gradient of L = grad_sigma * sigma + sum_n <grad_u_n, u_n>
 * with respect to the tensor, at a converged solution (no paper
 * counterpart: envelope theorem for sigma, implicit-function adjoint of the
 * KKT system 2.4 for the factors).
 *   T        F32 tensor (device data) the solution was computed on.
 *   u        device, n_tot floats: converged unit factors.
 *   sigma    host: converged sigma (consistent with u's signs).
 *   grad_u   device, n_tot floats, or NULL (= zero).
 *   grad_T   device, N floats (overwritten):
 *            grad_sigma * u1 o ... o ud - sum_n u1 o .. o a_n o .. o ud,
 *            where [a; nu] solves [[H - sigma I, -U], [-U^T, 0]] [a; nu] = [w; 0]
 *            (H = full symmetric block matrix, U = blockdiag(u_n), w = grad_u).
 * The adjoint system is solved in FP64 on the device.  Synchronous.
 * NONFINITE if the system is singular to working precision.
 */
hoscf_status hoscf_backward(hoscf_handle* h, const hoscf_tensor_desc* T, const float* u,
                            double sigma, double grad_sigma, const float* grad_u,
                            float* grad_T, void* stream);

/*
 * hoscf_quantize - FP32 tensor to the precision-form storage (no paper
 * counterpart).  x: device, n floats.  dtype BF16 or F16: q receives n
 * uint16 (round to nearest even; F16 beyond 65504 becomes infinity as IEEE
 * rounding prescribes).  dtype F8E4M3: q receives n bytes and scales
 * ceil(n/128) floats: scale = fp32(amax/448) per 128-element group (1 for an
 * all-zero group), code = saturating round-to-nearest-even e4m3 of
 * fp32(x/scale).  Asynchronous on `stream`.
 */
hoscf_status hoscf_quantize(hoscf_handle* h, const float* x, int64_t n, int dtype, void* q,
                            float* scales, void* stream);

/*
 * hoscf_solve_greedy - rank-R approximation by the greedy rank-one update
 * (Sec. 1, Example 3): for r = 1..R, B^(r) = sigma_r u_1^(r) o ... o u_d^(r)
 * is the best rank-one approximation of A^(r) (hoscf_solve), and
 * A^(r+1) = A^(r) - B^(r), A^(1) = A.  The tensor is never rewritten: every
 * pass builds the blocks of A (eq. 3.3) and subtracts the earlier terms'
 * contributions sigma_s prod_{k != m,n} <u_k^(s), u_k> u_m^(s) u_n^(s)^T.
 *   T       as for hoscf_solve (opts->refine and the variants apply to every
 *           term).
 *   R       1 .. 32.
 *   u0      device, R x n_tot floats: initial guess of each term.
 *   u_out   device, R x n_tot floats: the terms' factors (row r is term r+1;
 *           the rows already written are read back as the deflation list).
 *   sigma_out  host, R doubles.  info host, R entries, or NULL.
 *   res_out    host, R + 1 doubles, or NULL: ||A^(r)||_F / ||A||_F for
 *           r = 1 .. R+1, from ||A^(r+1)||^2 = ||A^(r)||^2 - sigma_r^2 (the
 *           identity at a KKT point) and ||A||_F (one extra read of the tensor
 *           the certificates use).
 * Synchronous.  Returns NOT_CONVERGED if any term did not converge (all
 * terms are still computed), else the first error; EINVAL for R out of range.
 */
hoscf_status hoscf_solve_greedy(hoscf_handle* h, const hoscf_tensor_desc* T, int R,
                                const float* u0, const hoscf_opts* opts, float* u_out,
                                double* sigma_out, hoscf_info* info, double* res_out,
                                void* stream);

/*
 * hoscf_profile_enable / hoscf_profile_read - a measurement aid with no
 * counterpart in the paper: device time of single kernels for roofline
 * figures, recorded as CUDA event pairs on the launch stream.
 *   enable   nonzero: from now on record (earlier records are discarded), for
 *            at most 65536 calls of each kind: which = 0 the pass's streaming
 *            kernel of every hoscf_ttvc_blocks call (the tiled, small-face
 *            or copy kernel, without the partial-sum reductions that follow
 *            it); which = 1 the gradient write of every hoscf_backward call
 *            (its coefficient and write kernels); which = 2 its adjoint
 *            solve (the pass at the solution and the Lanczos solve);
 *            which = 3 every eigen, RQI or comparison-method step (the
 *            J-row build and the Lanczos kernel) of hoscf_eig_step,
 *            hoscf_rqi_step, the solvers' iterations and the adjoint solve
 *            of hoscf_backward;
 *            zero: stop recording (records are kept for reading).
 *   which    0 .. 3 as above.
 *   count    host: number of recorded calls of that kind.
 *   total_ms host: sum of their durations in milliseconds; the call waits
 *            for the recorded events to complete.
 * Errors: EINVAL (NULL handle or pointer, `which` out of range), ECUDA.
 */
hoscf_status hoscf_profile_enable(hoscf_handle* h, int enable);
hoscf_status hoscf_profile_read(hoscf_handle* h, int which, int* count, double* total_ms);

/*
 * hoscf_selftest_timeout - exercises the library's failure path for device
 * waits (no counterpart in the paper).  Every spin-wait in the library's
 * kernels is bounded; when a bound passes, the kernel records a timeout in
 * the handle's device status word and returns, and the host call reports
 * HOSCF_TIMEOUT.  This call runs such a wait on a condition nothing can
 * satisfy, so the bound always passes:
 *   kind 0   an mbarrier phase that no thread or copy completes (the wait
 *            the streaming kernel uses for its TMA copies);
 *   kind 1   the software grid barrier of the eigen step with one arrival
 *            missing (2 CTAs);
 *   kind 2   kind 0 launched asynchronously on `stream` like the pass, its
 *            timeout left in the status word for hoscf_device_status.
 *   timeout_ns   the bound, 1 .. 10^10.
 *   stream   kind 2 only (cudaStream_t as void*).
 * Kinds 0 and 1 are synchronous; nothing else is in flight in these
 * kernels, so the context stays usable.  Returns HOSCF_TIMEOUT when the
 * failure was detected and reported (the expected outcome of kinds 0 and 1),
 * OK for a launched kind 2, EINVAL for bad arguments, ECUDA otherwise.
 */
hoscf_status hoscf_selftest_timeout(hoscf_handle* h, int kind, int64_t timeout_ns, void* stream);

/*
 * hoscf_ttvc_blocks_static - hoscf_ttvc_blocks without any allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc - for example a plugin whose host application
 * owns the whole device-memory budget, or code that must not allocate after
 * start-up - and so cannot create an hoscf_handle (a handle allocates its
 * workspace with cudaMalloc).
 *   T, u, H  as for hoscf_ttvc_blocks (the caller still owns and passes the
 *            inputs and the output); F32, BF16 and F16 tensors.
 *   status   device, 1 int, or NULL: written in stream order after the pass
 *            with 0 (H is valid) or HOSCF_TIMEOUT's device code (a bounded
 *            wait of the pass gave up; H is invalid).  With NULL such a
 *            failure goes unreported.
 *   stream   cudaStream_t as void* (NULL = legacy default stream); the
 *            buffers must belong to the calling thread's current device.
 * Scratch comes from one file-scope device array of
 * HOSCF_STATIC_SCRATCH_BYTES (64 MiB) that every GPU loading this library
 * holds until the process exits.  Problems whose scratch would exceed it are
 * rejected with HOSCF_EINVAL (e.g. 512^3 FP32 fits, 1024^3 does not).  Each
 * call whose stream is not capturing looks up the array's device address
 * (with the device current; so a device reset between calls is harmless);
 * a call made while the stream captures uses the address an earlier call on
 * that device found, so make one call before any stream capture (EINVAL
 * otherwise).  All calls share the array and every call overwrites it:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  Asynchronous on `stream`; status codes only
 * (no message).
 */
#define HOSCF_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
hoscf_status hoscf_ttvc_blocks_static(const hoscf_tensor_desc* T, const float* u, float* H,
                                      int* status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HOSCF_H */
