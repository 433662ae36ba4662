/*
 * ef.h -- C ABI of the GB300 (sm_103a) library for the entropic Fourier method (EFM) collision
 * operator of Cai, Fan & Ying, "An entropic Fourier method for the Boltzmann equation"
 * (arXiv:1704.07369).
 *
 * The library evaluates, for every cell of a batch, the discrete collision operator
 *
 *     Q^sigma_r = sum_{p,q,s} (A^sigma)^{rs}_{pq} (F_p F_q - F_r F_s)          (eq. Qsr)
 *
 * on an N^d periodic velocity grid over [-L, L]^d, in its Fourier form (eq. Qsk) with the
 * modified-Jackson-filtered kernel modes B^sigma_N(l,m) = sigma_N(l) sigma_N(m) B_N(l,m)
 * (eq. Bsigma, eq. JacksonFilter2) and the low-rank fast algorithm of Sec. 4.1 (eq. fastAlg):
 * forward FFT of F, per-direction spectral multiplies, inverse FFTs, gain minus loss.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: per axis j in {-N/2, ..., N/2-1}, v_j = h j, h = 2L/N; array index i = j + N/2; a cell is
 *   N^d values in C order (axis 0 slowest).  Cells are stored back to back ("cell-major").
 * Even N (Sec. 4.1): kernel modes with any component -N/2 are zero; the filter uses n = N/2.  The
 *   loss term multiplies the grid value F_r (DVM form, eq. QCvr / eq. Qsr).
 * Memory: every F / Q / diag pointer is a DEVICE pointer owned by the caller, contiguous, of the
 *   plan's precision (float for EF_PREC_F32, double for EF_PREC_F64; diagnostics are always
 *   double); F and Q must start on a 16-byte boundary (EF_ERR_INVALID_ARG otherwise).  The plan
 *   owns its tables, workspaces and status word, all allocated by ef_plan_create* (and the SSP-RK3
 *   stage buffers by ef_plan_reserve).  No other entry point of a plan allocates device memory,
 *   synchronises the device or blocks the host, except ef_plan_destroy and ef_plan_status(plan, 1);
 *   so the operations can be captured into a CUDA graph.
 * Streams: operations are enqueued on the given CUDA stream (0 = legacy default stream) and return
 *   immediately.  The plan's device must be current on the calling thread.
 * Errors: every function returns an ef_status; on failure nothing is launched and
 *   ef_last_error() (thread-local) describes why.  Argument checks run before any launch.
 *   Device-side conditions (non-finite values, a positivity violation under an Euler step) are
 *   recorded in the plan's status word and read with ef_plan_status().
 * Thread safety: a plan may be used from one host thread at a time.
 */
#ifndef EF_H
#define EF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ef_plan_s *ef_plan_t;
typedef struct CUstream_st *ef_stream_t;      /* same object as cudaStream_t */

typedef enum {
    EF_OK = 0,
    EF_ERR_INVALID_ARG = 1,   /* a null pointer, bad size, mismatched cell count ... */
    EF_ERR_UNSUPPORTED = 2,   /* valid request outside what this build implements */
    EF_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in ef_last_error) */
    EF_ERR_OOM = 4,           /* device memory for the plan could not be allocated */
    EF_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    EF_ERR_POSITIVITY = 6,    /* an Euler step produced F < 0 (dt max nu > 1) */
    EF_ERR_NOT_FINITE = 7     /* a NaN or Inf reached the output */
} ef_status;

typedef enum { EF_PREC_F32 = 0, EF_PREC_F64 = 1 } ef_precision;

/* Collision kernels.  EF_KERNEL_MAXWELL: Maxwell molecules, B = 1/(2 pi) in 2D (Sec. 4.2) and
 * B = 1/(4 pi) in 3D.  EF_KERNEL_HARD_SPHERE: B = |g| / (4 pi) (3D only). */
typedef enum { EF_KERNEL_MAXWELL = 0, EF_KERNEL_HARD_SPHERE = 1 } ef_kernel;

/* Per-cell diagnostics, EF_DIAG_STRIDE doubles per cell (h = 2L/N, v = h j):
 *   [0] mass h^d sum F          [1..3] momentum h^d sum F v (unused axes 0)
 *   [4] energy h^d sum |v|^2 F / 2                [5] entropy eta = h^d sum F ln F (Sec. 4.2)
 *   [6] entropy production sum Q ln F over F > 0 (<= 0 by the discrete H-theorem, Theorem 1)
 *   [7] min F      [8] max nu (collision frequency; 0 when not computed)
 *   [9] min of the updated F (Euler), or min Q (collide / moments with Q). */
#define EF_DIAG_STRIDE 10

/* Full description of one discretisation.  Zero / negative fields take the defaults below. */
typedef struct {
    int d;                 /* 2 or 3 */
    int N;                 /* grid points per axis; even, >= 8, one of the built sizes */
    double L;              /* box half width, > 0 */
    ef_kernel kernel;
    int R;                 /* angular rank: number of (l, m) terms of the low-rank kernel (eq. fastAlg);
                              2D: even, >= 2; 3D: 2 n_mu n_phi n_c */
    ef_precision prec;
    double R_tr;           /* truncation radius R of eq. approximated_collision; default
                              4 L / (3 sqrt 2 + 1), the largest allowed by Sec. 1.2 */
    int n_mu, n_phi, n_c;  /* 3D angular quadrature; default from R (32 -> 2,4,2; 64 -> 2,4,4) */
    int J;                 /* 3D Maxwell: Gaussian terms for 1/|y+z|; default 6 */
    int sigma_enabled;     /* 1 (default, EFM) or 0: no filter (Fourier collocation method);
                              pass -1 for the default */
} ef_plan_desc;

/* Create a plan for cells of one size N.  Cells are passed at call time (ncells), cell c at
 * element offset c * N^d.  Argument meaning as in ef_plan_desc. */
ef_status ef_plan_create(int d, int N, double L, ef_kernel kernel, int R, ef_precision prec,
                         ef_plan_t *out);

/* As ef_plan_create with every field of ef_plan_desc. */
ef_status ef_plan_create_ex(const ef_plan_desc *desc, ef_plan_t *out);

/* Plan for a fixed batch of ncells cells of uneven size: N_host[c] (host array) is the size of
 * cell c; cell c starts at element offset sum_{c' < c} N_host[c']^d.  One launch per distinct
 * N, all enqueued on the caller's stream (captured once into a CUDA graph when
 * ef_plan_set_graph(plan, 1)). */
ef_status ef_plan_create_batched(int d, int64_t ncells, const int *N_host, double L, ef_kernel kernel,
                                 int R, ef_precision prec, ef_plan_t *out);

ef_status ef_plan_destroy(ef_plan_t plan);

/* Q = Q^sigma[F] for ncells cells (eq. Qsk / eq. Qsr).  F_dev and Q_dev must not overlap.
 * For a batched plan ncells must equal the plan's cell count. */
ef_status ef_collide(ef_plan_t plan, const void *F_dev, void *Q_dev, int64_t ncells, ef_stream_t stream);

/* nsteps forward Euler steps F <- F + dt Q^sigma[F], in place.  If diag_dev is not null it
 * receives nsteps * ncells * EF_DIAG_STRIDE doubles ([step][cell][k], moments of F before each
 * step, entropy production of that step, max nu and the min of the updated F); a step whose
 * updated F has a negative value sets EF_ERR_POSITIVITY in the status word (positivity holds when
 * dt max nu <= 1, proof of Theorem 1). */
ef_status ef_euler_step(ef_plan_t plan, void *F_dev, double dt, int nsteps, double *diag_dev,
                        int64_t ncells, ef_stream_t stream);

/* nsteps third-order strong-stability-preserving Runge-Kutta steps (Gottlieb, Shu and Tadmor; the
 * time integrator of Sec. 4.1), in place:
 *   F1 = F + dt Q[F],  F2 = 3/4 F + 1/4 (F1 + dt Q[F1]),  F <- 1/3 F + 2/3 (F2 + dt Q[F2]).
 * Each stage is a convex combination of forward Euler steps, so positivity carries over from the
 * Euler step under the same dt max nu <= 1.  diag_dev (nullable) receives, per step, the diagnostics
 * of the first stage ([step][cell][k] as for ef_euler_step: moments of F before the step).  The
 * two batch-sized stage buffers come from ef_plan_reserve, which must have been called for at
 * least ncells cells (EF_ERR_INVALID_ARG otherwise; nothing is launched).  F must be 16-byte
 * aligned. */
ef_status ef_rk3_step(ef_plan_t plan, void *F_dev, double dt, int nsteps, double *diag_dev, int64_t ncells,
                      ef_stream_t stream);

/* Allocate the plan's two SSP-RK3 stage buffers for batches of up to ncells cells (a batched plan:
 * its whole batch; ncells 0 or the plan's count).  A set-up call like ef_plan_create: when the
 * buffers must grow it synchronises the device, frees the old ones and allocates (EF_ERR_OOM if
 * that fails); when they are already large enough it does nothing.  Call it before capturing
 * ef_rk3_step into a CUDA graph. */
ef_status ef_plan_reserve(ef_plan_t plan, int64_t ncells);

/* ef_collide for callers that cannot allocate device memory when they evaluate the operator (a
 * host framework whose allocator owns all device memory, a real-time loop or callback where an
 * allocation may block or fail, code that must keep the device footprint fixed after start-up).
 * The paper has no counterpart: this is a deployment variant of ef_collide, same arithmetic and
 * same arguments, for a plan from ef_plan_create / ef_plan_create_ex (batched plans:
 * EF_ERR_INVALID_ARG).  It allocates nothing and calls no allocating routine: its scratch (the
 * cell-queue counter and the S/G accumulators of the clusters in flight) lives in one 16 MiB
 * static device array that every GPU loading the library holds until the process exits.
 *  - The first call on a device looks up that array's device address (cudaGetSymbolAddress);
 *    make the first call on each device before any stream capture.
 *  - All calls share the array, which keeps the last call's contents (the counter is cleared on
 *    the given stream at the start of every call): calls that can overlap on the GPU, e.g. on
 *    different streams, race and must be serialised by the caller.
 *  - If one cell's cluster needs more scratch than the array holds (very large N in FP64), the
 *    call returns EF_ERR_UNSUPPORTED with the sizes in ef_last_error(); otherwise the launch
 *    uses as many clusters as fit and any ncells is accepted.
 *  - The S/G accumulators always live in that array (global memory), with the plan's cluster
 *    size, threads per CTA and prefetch choice; where ef_collide keeps them in shared memory,
 *    this call can be slower than ef_collide. */
ef_status ef_collide_noalloc(ef_plan_t plan, const void *F_dev, void *Q_dev, int64_t ncells, ef_stream_t stream);

/* The kernel function of the plan's discretisation on the grid: G_dev[y] = G^sigma(y, z) for every
 * grid point y (flat C-order index, N^d doubles, caller-owned device memory) at the grid point z of
 * flat index z_index, where G^sigma(y, z) = sum_{i,j in K} B^sigma_fast(i, j) E_i(y) E_j(z) is the
 * weight of eq. tildeG (through eq. A_simplified) with the plan's low-rank kernel (eq. fastAlg).
 * Sec. 3.2.2: G^sigma >= 0 with the filter (every pair weight of the DVM form is non-negative);
 * without it (sigma_enabled = 0) G takes negative values (Fig. 1).  FP64 direct sums over the
 * modes; a diagnostic of the kernel decomposition, not a step of the collision operator (cost
 * N^{2d} n_e per call).  Uniform plans only (EF_ERR_INVALID_ARG for a batched plan, a null G_dev
 * or z_index outside [0, N^d)). */
ef_status ef_kernel_G(ef_plan_t plan, int64_t z_index, double *G_dev, ef_stream_t stream);

/* Low-mode features of each cell: the discrete Fourier coefficients Fh_k = N^{-d} sum F E_{-k}
 * (eq. DFT, index-origin convention of the library's FFTs) at the modes |k| <= EF_FEATURE_K in the
 * canonical half space (k_last > 0; or k_last = 0 and k_1 > 0; or k_last = k_1 = 0 and k_0 >= 0),
 * listed in lexicographic order of k.  feat_dev (FP32, caller-owned) receives EF_FEATURE_STRIDE
 * floats per cell: (re, im) of each mode, then zeros are NOT written (the caller clears the pad).
 * 3D, K = 6: 463 modes = 925 real degrees of freedom.  With log_input = 1 the transform is taken
 * of ln(max(F, 1e-30)) instead (used for the entropy-production gate of the surrogate).  Needs
 * N/2 > EF_FEATURE_K. */
#define EF_FEATURE_K 6
#define EF_FEATURE_STRIDE 928
ef_status ef_features(ef_plan_t plan, const void *F_dev, float *feat_dev, int64_t ncells, int log_input,
                      ef_stream_t stream);

/* ---------------------------------------------------------------- learned surrogate ---------
 * A multilayer perceptron with bf16 weights and activations and FP32 accumulation, trained and run
 * by the library's own tensor-core kernels.  The paper has no counterpart; it serves the
 * surrogate path that maps a cell's low Fourier modes of F to those of Q^sigma.
 *
 * Layers: x -> relu(W_0 x + b_0) -> ... -> W_{L-1} h + b_{L-1} (nlayers = L weight matrices, hidden
 * width nhidden, no activation on the output).  Feature widths are padded to multiples of 64
 * inside; batches are multiples of 64.  Parameters are FP32 master copies (Adam, beta = 0.9 /
 * 0.999, eps = 1e-8) with bf16 working copies.  All pointers are device pointers unless stated. */
typedef struct ef_mlp_s *ef_mlp_t;

/* He-normal initialisation from a seeded 64-bit Mersenne twister (host), zero biases. */
ef_status ef_mlp_create(int nin, int nhidden, int nlayers, int nout, int64_t max_batch, uint64_t seed, ef_mlp_t *out);
ef_status ef_mlp_destroy(ef_mlp_t mlp);

/* info: [0] nin, [1] nhidden, [2] nlayers, [3] nout, [4] number of FP32 parameters (padded layout:
 * per layer W[out_p][in_p] then b[out_p]), [5] padded nin, [6] padded nout, [7] max batch. */
ef_status ef_mlp_info(ef_mlp_t mlp, int64_t info[8]);

/* The MLP's device status word, as ef_plan_status does for a plan: EF_OK, or EF_ERR_TIMEOUT when a
 * tensor-core GEMM gave up one of its bounded mbarrier waits (that GEMM's outputs are then NaN and
 * the work queued after it on the stream saw them).  sync = 1 synchronises the device and reads
 * the word; sync = 0 returns the value last read.  reset = 1 clears it. */
ef_status ef_mlp_status(ef_mlp_t mlp, int sync, int reset);

/* Copy the FP32 parameters to (set = 0) or from (set = 1) a HOST buffer of info[4] floats. */
ef_status ef_mlp_params(ef_mlp_t mlp, float *host, int set);

/* Y[b][0..padded nout) = mlp(X[b][0..nin)) for b < batch; X row stride ldx >= nin, Y row stride ldy
 * >= padded nout and even.  batch a multiple of 64, <= max_batch. */
ef_status ef_mlp_forward(ef_mlp_t mlp, const float *X, int ldx, float *Y, int ldy, int64_t batch, ef_stream_t stream);

/* Mean squared error against T (row stride ldt >= nout) over the nout outputs, weighted by
 * wmask[j] (per output, nullable = 1) and rowweight[b] (per sample, nullable = 1):
 * loss_dev[0] = sum_b sum_j w_j r_b (y - t)^2 / (batch nout); gradients of the loss into the MLP's
 * gradient buffer and, if grad_dev is not null, copied there (info[4] floats). */
ef_status ef_mlp_grad(ef_mlp_t mlp, const float *X, int ldx, const float *T, int ldt, const float *wmask,
                      const float *rowweight, int64_t batch, float *loss_dev, float *grad_dev, ef_stream_t stream);

/* ef_mlp_grad followed by one Adam step with learning rate lr. */
ef_status ef_mlp_train_step(ef_mlp_t mlp, const float *X, int ldx, const float *T, int ldt, const float *wmask,
                            const float *rowweight, int64_t batch, float lr, float *loss_dev, ef_stream_t stream);

/* The surrogate path (learned map from F's low modes to Q^sigma's low modes; no counterpart in the
 * paper).  Built on a uniform plan (whose ef_features define the band) and an MLP with
 * nout = 2 x (feature modes) and nin = nout, or nout + 2 to add the two moment features below.
 * Scratch for max_batch cells (features, activations, the fallback list and a full-size Q buffer
 * for fallback cells) is allocated here, so inference allocates nothing. */
typedef struct ef_surrogate_s *ef_surrogate_t;
ef_status ef_surrogate_create(ef_plan_t plan, ef_mlp_t mlp, int64_t max_batch, ef_surrogate_t *out);
ef_status ef_surrogate_destroy(ef_surrogate_t sur);

/* Fit the normalisation from n training samples: features of F and of Q^sigma[F] (ef_features,
 * EF_FEATURE_STRIDE floats each) and the cells' moments (ef_moments_entropy, EF_DIAG_STRIDE doubles
 * each).  With m = Fh_0 and u = momentum / mass, each mode is de-translated and mass-normalised,
 * x_k = Fh_k e^{i pi k.u/L} / m and y_k = Qh_k e^{i pi k.u/L} / m^2 (the operator is quadratic in F and
 * commutes with velocity shifts up to aliasing).  If the MLP's input width is 2 x modes + 2, x also
 * carries the kinetic temperature theta = (2E/rho - |u|^2)/d and the relative entropy to the local
 * Maxwellian eta/rho - ln rho + (d/2)(ln(2 pi theta) + 1) (from the moments: mass rho, energy E,
 * eta).  Then per-column mean and std of x (the std floored
 * at 1e-4, so that columns that vary only at round-off level are not amplified), per-column mean
 * of y and one global scale of y.  Xt, Yt: caller scratch of n x EF_FEATURE_STRIDE floats.  If
 * rowweight (n floats) is not null it receives per-sample loss weights proportional to 1 / |y_b|^2
 * (mean 1), which make the training loss the per-cell relative error. */
ef_status ef_surrogate_fit_stats(ef_surrogate_t sur, const float *featF, const float *featQ, const double *mom,
                                 float *Xt, float *Yt, float *rowweight, int64_t n, ef_stream_t stream);

/* Normalised MLP inputs X (and targets Y, if featQ and Y are not null), EF_FEATURE_STRIDE per row. */
ef_status ef_surrogate_normalize(ef_surrogate_t sur, const float *featF, const float *featQ, const double *mom,
                                 float *X, float *Y, int64_t n, ef_stream_t stream);

/* Copy the statistics (4 x EF_FEATURE_STRIDE floats: mu, s, nu, t) to (set = 0) / from (set = 1) the host. */
ef_status ef_surrogate_stats(ef_surrogate_t sur, float *host, int set);

/* Audit policy (no counterpart in the paper): the whole batch falls back when more than
 * max_miss_fraction (in [0, 1]; default 0, i.e. any miss) of the audited cells miss the tolerance;
 * the input gate rejects cells with any normalised input beyond +-xmax (> 0; default 8).  Applies
 * to later ef_surrogate_infer calls; not to be changed while one is in flight on a stream. */
ef_status ef_surrogate_set_policy(ef_surrogate_t sur, float max_miss_fraction, float xmax);

/* Switches the entropy-production gate (flags bit 1 for a positive band sum Q ln F) on (default)
 * or off.  With it off the inference skips the band of ln F, about half of its feature pass; the
 * other gates stay.  Applies to later ef_surrogate_infer calls. */
ef_status ef_surrogate_set_entropy_gate(ef_surrogate_t sur, int on);

/* Band of Q^sigma for ncells cells (multiple of 64, <= max_batch): qfeat (EF_FEATURE_STRIDE per
 * cell, ef_features layout) receives the prediction, or the plain operator's band where the
 * prediction is not trusted.  flags (int per cell): 1 = a gate failed (non-finite, input outside
 * +-xmax training standard deviations, or positive band entropy production sum Q ln F, which the
 * discrete H-theorem forbids), 2 = audited (a seeded fraction audit_fraction of cells, drawn from
 * seed), 4 = audited and the prediction missed the plain band by more than tol in relative L2,
 * 8 = plain result used, 32 = the checker network disagreed (ef_surrogate_set_checker), 16 = fell
 * back because the audit failed: more than the policy's fraction
 * of the audited cells (by default none, ef_surrogate_set_policy) missed tol, and then the whole
 * batch uses the plain operator.  Everything stays on the device: no host synchronisation. */
ef_status ef_surrogate_infer(ef_surrogate_t sur, const void *F_dev, float *qfeat, int *flags, int64_t ncells,
                             float audit_fraction, uint64_t seed, float tol, ef_stream_t stream);

/* A second network (the checker: same input and output widths, max batch >= the surrogate's,
 * trained like the first from another seed).  With a checker set, the delivered band is the mean
 * of the two networks' decoded bands q and c (an ensemble of two), and the score
 * ||q - c||_2 / ||(q + c) / 2||_2 over the band (zero mode excluded) above tol (> 0) sends the cell
 * to the plain operator (flags bit 32, with 8).  The score correlates with the error of the
 * delivered band, so a threshold calibrated on held-out cells sends the cells most at risk to the
 * plain operator; it bounds no single cell's error (a few misses can score below a threshold that
 * flags a few percent of the cells).
 * Allocates the checker's output rows for max_batch cells on the first call (a set-up call);
 * checker = null switches the gate off.  The paper has no counterpart. */
ef_status ef_surrogate_set_checker(ef_surrogate_t sur, ef_mlp_t checker, float tol);

/* ef_surrogate_infer with two optional outputs: score (ncells floats, device; nullable) receives
 * each cell's checker score (0 without a checker), and Q_dev (ncells cells of N^3 floats, layout as
 * ef_collide, 16-byte aligned; nullable; FP32 3D plans) receives Q on the grid: the surrogate's band
 * mapped back to the grid (ef_features_inverse) where the prediction is delivered, and the plain
 * operator's full Q where flags has 8.  No allocation, no host synchronisation. */
ef_status ef_surrogate_infer_ex(ef_surrogate_t sur, const void *F_dev, float *qfeat, int *flags, float *score,
                                float *Q_dev, int64_t ncells, float audit_fraction, uint64_t seed, float tol,
                                ef_stream_t stream);

/* The inverse of ef_features on its band: Q_dev[c][i] = sum over the band modes k (both halves:
 * each stored mode and its conjugate) of feat[c][k] exp(2 pi i k.i / N), i the array index; so a
 * band-limited function is returned exactly and a general one is projected on the band (its
 * truncation to |k| <= EF_FEATURE_K).  FP32 3D uniform plans with a band; Q_dev 16-byte aligned,
 * ncells cells of N^3 floats.  No allocation. */
ef_status ef_features_inverse(ef_plan_t plan, const float *feat, float *Q_dev, int64_t ncells, ef_stream_t stream);

/* Moments and entropy of each cell (layout EF_DIAG_STRIDE, entries [0..7] and [9]).  Here [8] is
 * the positivity error of Sec. 4.2, Example 1: (sum |F| - sum F) / sum |F| (0 for F >= 0), in place
 * of max nu.  Q_dev may be null; then [6] = 0 and [9] = 0.  Accuracy: FP64 plans sum in FP64;
 * FP32 plans sum runs in FP32 into compensated FP32 pairs and warps in FP32, an error of at most
 * about 43 * 2^-24 of the sum of the entries' |terms|, results stored as doubles. */
ef_status ef_moments_entropy(ef_plan_t plan, const void *F_dev, const void *Q_dev, double *out_dev,
                             int64_t ncells, ef_stream_t stream);

/* Free transport between spatial cells (the spatially inhomogeneous setting that Sec. 5 leaves to
 * future work; the collision step between transport steps is ef_euler_step or ef_rk3_step on the
 * same batch, by operator splitting).  The ncells cells of a uniform plan are the points x_i of a
 * periodic 1D spatial grid of spacing dx (cell i's neighbours are i - 1 and i + 1 modulo ncells),
 * and the velocity component along the first array axis, v = h (j - N/2) with h = 2L/N, carries F
 * along x.  One first-order upwind step with the Courant number nu = v dt / dx:
 *   F_out_i = F_in_i - nu (F_in_i - F_in_{i-1})  (nu > 0),  F_in_i - nu (F_in_{i+1} - F_in_i)  (nu < 0),
 * a convex combination of F_in_i and its upwind neighbour when max |nu| = (N/2) h |dt| / dx <= 1,
 * so F >= 0 is kept then (not checked: larger steps are computed as asked).  Mass per velocity point
 * summed over the cells is conserved.  F_in and F_out: device arrays of ncells cells (layout as
 * ef_collide), 16-byte aligned, not overlapping.  Errors: EF_ERR_INVALID_ARG for a batched plan,
 * null / misaligned / overlapping arrays, ncells < 0, dx <= 0 or non-finite dt. */
ef_status ef_transport_step(ef_plan_t plan, const void *F_in_dev, void *F_out_dev, int64_t ncells, double dx,
                            double dt, ef_stream_t stream);

/* The entropic Fourier method on the classical form of the operator (the remark after eq. EFMk;
 * kernel modes of eq. classical_hatB), 3D Maxwell molecules (B = 1/(4 pi)), FP64, for the grid
 * sizes of Table 3 (Example 4).  B_hat(l, m) = 4 pi int_0^R r^2 sinc(c r |l+m|) sinc(c r |l-m|) dr
 * with c = pi / (2L) (both sphere integrals in closed form), filtered by the modified Jackson filter
 * of each axis (sigma_enabled = 0: no filter, the collocation method), and
 *   Qh_k = sum_{l + m = k mod N} (Bs(l, m) - Bs(m, m)) Fh_l Fh_m
 * is summed directly over mode pairs: the weight depends on the unaliased l + m, so the low-rank
 * transforms of ef_collide do not apply.  O(N^6) work per cell.
 * ef_classical_create: even N with 4 <= N <= 128, box half width L > 0, truncation radius R_tr
 * (<= 0: the largest the classical form allows, 4L / (3 + sqrt 2)); allocates its device table and
 * work arrays (about 8 (3N^2 + 1)^2 bytes: 75 MB at N = 32, 1.2 GB at N = 64, 19 GB at N = 128),
 * tabulates B_hat on the device and synchronises (a set-up call).  N = 64 takes about a second of
 * FP64 work per evaluation, N = 128 about a minute (N^6 pairs). 
 * ef_classical_collide: F_dev, Q_dev device arrays of ncells cells of N^3 doubles (layout as
 * ef_collide), not overlapping; cells are evaluated one after another on `stream`; calls on one
 * object share its work arrays, so they must not run concurrently.  Errors: EF_ERR_INVALID_ARG
 * for bad sizes or pointers, EF_ERR_OOM / EF_ERR_CUDA from the runtime. */
typedef struct ef_classical_s *ef_classical_t;
ef_status ef_classical_create(int N, double L, double R_tr, int sigma_enabled, ef_classical_t *out);
ef_status ef_classical_collide(ef_classical_t c, const double *F_dev, double *Q_dev, int64_t ncells,
                               ef_stream_t stream);
ef_status ef_classical_destroy(ef_classical_t c);

/* The Fourier Galerkin method (FGM), the comparison method of Fig. 2 (Sec. 1.2, eq. FGM_Q, fast form
 * eq. fastFGM): for cells of the N grid described by desc (uniform; N even with 2N a built size,
 * i.e. N <= 32), Q = the grid values of sum_{k in K} Qh^G_k E_k with
 *   Qh^G_k = sum_{l, m in K, l + m = k} (B(l,m) - B(m,m)) Fh_l Fh_m,   K = {-(N/2-1), ..., N/2-1}^d,
 * the sum NOT reduced mod N (no aliasing), Fh the DFT of the grid values F (interpolation data),
 * B the low-rank kernel of desc (its filter only if desc->sigma_enabled is 1; the FGM of the
 * literature has none: pass 0).  Evaluated by zero padding: F is interpolated to the grid of 2N
 * points, the collision kernels of ef_collide run there with multipliers restricted to K, and the
 * result is projected back onto K.  ef_galerkin_create allocates the doubled-grid plan and
 * scratch for max_cells cells (the only allocation); ef_galerkin_collide takes ncells <= max_cells
 * cells (device pointers, layout as ef_collide) and allocates nothing; calls on one object share
 * its scratch and must not overlap.  ef_galerkin_status reads the doubled-grid plan's status word
 * (as ef_plan_status).  EF_ERR_UNSUPPORTED if 2N is not a built size. */
typedef struct ef_galerkin_s *ef_galerkin_t;
ef_status ef_galerkin_create(const ef_plan_desc *desc, int64_t max_cells, ef_galerkin_t *out);
ef_status ef_galerkin_collide(ef_galerkin_t g, const void *F_dev, void *Q_dev, int64_t ncells, ef_stream_t stream);
ef_status ef_galerkin_status(ef_galerkin_t g, int sync, int reset);
ef_status ef_galerkin_destroy(ef_galerkin_t g);

/* Streaming a batch that lives in host memory (no counterpart in the paper; the paper's method
 * is per cell).  The cells (sizes N_host[c], back to back as for ef_plan_create_batched) are cut
 * into nchunks contiguous chunks of about equal work, each with its own batched plan, and a device
 * copy of the whole batch is allocated here with the plan's streams: one for the uploads, one for
 * the downloads and up to four for the steps.  ef_stream_euler_step uploads each chunk, runs nsteps
 * Euler steps on it (ef_euler_step) and downloads it, in place in F_host; the uploads run back to
 * back, a chunk's steps start when its upload is done and its download when its steps are, so
 * copies in both directions overlap the collision steps of other chunks when F_host is page-locked
 * (pageable memory works but serialises the copies).  diag_host
 * (nullable) receives nsteps * ncells * EF_DIAG_STRIDE doubles, [step][cell][k] as ef_euler_step
 * (through a one-step device buffer allocated here, copied out after each step).  All work is
 * ordered after earlier work on `stream`, and later work on `stream` waits for it; the host
 * buffers must stay untouched until then.  ef_stream_euler_step allocates nothing and does not
 * synchronise; if it fails part way, the chunks it already started are still joined into
 * `stream` before it returns the error, so the same rule holds. */
typedef struct ef_stream_plan_s *ef_stream_plan_t;
ef_status ef_stream_plan_create(int d, int64_t ncells, const int *N_host, double L, ef_kernel kernel, int R,
                                ef_precision prec, int nchunks, ef_stream_plan_t *out);
ef_status ef_stream_plan_destroy(ef_stream_plan_t sp);
/* info: [0] cells, [1] chunks, [2] values in the batch, [3] bytes per value. */
ef_status ef_stream_plan_info(ef_stream_plan_t sp, int64_t info[4]);
ef_status ef_stream_euler_step(ef_stream_plan_t sp, void *F_host, double dt, int nsteps, double *diag_host,
                               ef_stream_t stream);
/* First non-OK device status word of the chunk plans (as ef_plan_status). */
ef_status ef_stream_plan_status(ef_stream_plan_t sp, int sync, int reset);

/* Read the plan's device status word (the first error seen by a kernel, EF_OK if none).  With
 * sync = 1 the call first synchronises the plan's device; with sync = 0 it returns the value
 * copied back by the last synchronising call.  reset = 1 clears the word after reading. */
ef_status ef_plan_status(ef_plan_t plan, int sync, int reset);

/* Route ef_collide / ef_euler_step through a CUDA graph captured on first use per
 * (F, Q, ncells, stream) (1), or launch directly (0, default). */
ef_status ef_plan_set_graph(ef_plan_t plan, int enable);

/* Introspection (host values):  info[0] = d, [1] = number of distinct N, [2] = number of
 * spectral directions (inverse transforms per cell, loss included) of the first class, [3] =
 * cluster size of the first class, [4] = threads per CTA of the first class, [5] = cells (batched
 * plans; 0 otherwise), [6] = precision, [7] = kernel launches per ef_collide. */
ef_status ef_plan_info(ef_plan_t plan, int64_t info[8]);

/* Launch shape of size class i (0 <= i < info[1] of ef_plan_info), host values:
 * out[0] = N, [1] = cells (batched plans; 0 otherwise), [2] = cluster size (CTAs per cell),
 * [3] = threads per CTA, [4] = axis-0 planes per CTA, [5] = 1 if the S/G accumulators live in
 * global memory, [6] = 1 if the next multiplier slice is prefetched, [7] = autotuned time of one
 * class launch in microseconds (0 when not tuned).  EF_ERR_INVALID_ARG for a bad index. */
ef_status ef_plan_class_info(ef_plan_t plan, int i, int64_t out[8]);

const char *ef_status_string(ef_status s);
const char *ef_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EF_H */
