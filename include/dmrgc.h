/*
 * dmrgc -- circuit-DMRG compression sweep on one GB300 (sm_103a).
 *
 * C ABI of the library.  All compute runs in the library's own CUDA kernels on
 * the stream given in dmrgc_options::cuda_stream (0 = the legacy default
 * stream).  The library owns all device memory it allocates; callers own every
 * host buffer they pass.  Inputs are copied before a call returns; outputs
 * are written once the stream has been synchronised inside the call.  No
 * exception crosses this boundary and the library never aborts or traps: every
 * entry point returns a dmrgc_status and, on failure, leaves a message for
 * dmrgc_last_error().
 *
 * Method (arXiv:2207.05612, Ayral, Louvet, Zhou, Lambert, Stoudenmire,
 * Waintal): open-mode simulation (Sec. IV.C) in which every compression step
 * (Sec. IV.B) applies K gate cycles to a matrix product state and finds the
 * normalised MPS of bond dimension <= chi with the largest overlap with the
 * result, sweeping over the MPS and optimising two neighbouring tensors at a
 * time (the two-site variant named in Sec. IV.B; Eq. (scalarproduct) and
 * Eq. (optimization) with the bond constraint imposed by a truncated SVD).
 *
 * Conventions:
 *  - Qubit q sits at grid position (r, c) with q = r*cols + c.  MPS sites are
 *    ordered along the grid's chain order (dmrgc_grid.order), by default a
 *    snake down the columns (down column 0, up column 1, ...).
 *  - A gate's matrix is row-major complex128 with re/im interleaved:
 *    <s_q0 s_q1|U|t_q0 t_q1>, q0 the most significant bit (4x4, 32 doubles);
 *    a one-qubit gate (q1 = -1) uses the first 8 doubles as a 2x2 matrix.
 *  - Calls are stateful and ordered: create -> (apply_layer -> sweep)* ->
 *    fidelity / amplitude / sample.  Out-of-order calls return DMRGC_ESTATE.
 */
#ifndef DMRGC_H
#define DMRGC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrgc_ctx dmrgc_ctx;

typedef enum {
  DMRGC_OK = 0,
  DMRGC_EINVAL = 1,    /* bad argument (null pointer, size out of range) */
  DMRGC_ENOMEM = 2,    /* device or host allocation failed */
  DMRGC_ECUDA = 3,     /* a CUDA runtime call failed */
  DMRGC_ENOCONV = 4,   /* Jacobi SVD did not converge within max_jacobi_sweeps */
  DMRGC_ENUMERIC = 5,  /* NaN/Inf or a zero overlap met during a sweep */
  DMRGC_ETIMEOUT = 6,  /* a bounded device-side wait ran out */
  DMRGC_ESTATE = 7     /* call made out of order */
} dmrgc_status;

/* Arithmetic of the contractions and of the SVD. */
enum {
  DMRGC_FP64 = 0,    /* complex128 storage, FP64 arithmetic on CUDA cores */
  DMRGC_BF16X3 = 1,  /* complex64 storage, BF16 hi/lo split products (3 terms), FP32 accumulate */
  DMRGC_TF32X3 = 2,  /* complex64 storage, TF32 hi/lo split products (3 terms), FP32 accumulate */
  DMRGC_FP32 = 3     /* complex64 storage, FP32 arithmetic on CUDA cores */
};

typedef struct {
  int rows, cols; /* grid shape; n_qubits must equal rows*cols */
  int order;      /* chain order of the MPS sites: 0 = snake along the columns
                     (column 0 top to bottom, column 1 bottom to top, ...);
                     1 = snake along the rows (row 0 left to right, row 1 right
                     to left, ...); 2 = the anti-diagonals r + c = d in
                     increasing d, each in increasing r for even d and
                     decreasing r for odd d.  Runs of consecutive columns, rows
                     or anti-diagonals are then runs of consecutive sites: the
                     V, H and D qubit groupings of Sec. V.C. */
} dmrgc_grid;

typedef struct {
  int precision;              /* DMRGC_FP64 ... DMRGC_FP32 */
  int svd_mode;               /* truncated SVD of theta in the sweep:
                                 0 = one-sided Jacobi;
                                 1 = randomized range finder with a sketch of r + p columns,
                                     r = the rank that held all but 1e-6 of the weight kept
                                     at the bond's last update, tried when r + p is below
                                     half the smaller side of theta, falling back to the
                                     Jacobi SVD when the sketch fails its certificate;
                                 2 = the same with r predicted by the rank model
                                     (dmrgc_set_rank_model) */
  double sweep_rel_cutoff;    /* keep s_mu > cutoff * s_1 in the sweep SVD; <= 0: default
                                 (1e-12 for FP64, 2e-5 for the complex64 modes) */
  double zip_rel_cutoff;      /* same for the truncating steps of the zip-up guess; <= 0:
                                 default (1e-5 for FP64, 4e-3 for the complex64 modes) */
  int max_jacobi_sweeps;      /* <= 0: default 40 */
  unsigned long long seed;    /* seed of the randomized SVD sketches (SplitMix64 counter stream) */
  void* cuda_stream;          /* cudaStream_t to launch on; NULL = default stream */
  int timing;                 /* 1: record CUDA-event time per kernel class (dmrgc_stats) */
  int rsvd_oversample;        /* p, extra sketch columns; <= 0: 8 */
  int rsvd_power_iters;       /* q, power iterations (each re-orthonormalised); 0..8
                                 (dmrgc_default_options: 1) */
  double rsvd_tolerance;      /* tol of the sketch certificate: accept when the weight the
                                 optimum could hold beyond the sketch's f is <= tol * f (the
                                 result is then within tol of the optimal update); <= 0: 1e-6
                                 for FP64, 2e-5 for complex64 */
  int log_rank_records;       /* 1: log one rank-model record per full (Jacobi) SVD at a bond
                                 updated before (dmrgc_rank_records) */
  int mpo_compress;           /* 1: reduce each layer MPO's bonds to the operator Schmidt ranks
                                 (Jacobi SVD of the site tensors, two passes, cut at the
                                 sweep cutoff); 0 (default): the bond is the product of the
                                 straddling gates' Schmidt ranks */
  int svd_path;               /* complex64 modes, truncated SVDs of 128..2048 rows that keep
                                 fewer than all of them (the sweep's theta, the zip-up's Gram):
                                 0 (default) = the leading eigenvectors of the Gram matrix
                                 G G^+ (TF32x3 product, Householder tridiagonalisation,
                                 bisection and FP64 inverse iteration, back-transformation)
                                 whenever every kept eigenvalue is at least 1e-5 of the largest
                                 (the Gram's rounding then cannot move the kept subspace) and a
                                 count set by the cutoff has cutoff^2 at or above that level,
                                 the Jacobi SVD otherwise or when the eigensolver meets a
                                 non-finite value; 1 = always the Jacobi SVD.  FP64 mode
                                 always uses the Jacobi SVD. */
} dmrgc_options;

typedef struct {
  int q0, q1;        /* qubit indices; q1 = -1 for a one-qubit gate */
  double mat[32];    /* row-major complex128, re/im interleaved */
} dmrgc_gate;

/* Per-kernel-class accounting (only filled when options.timing = 1).
 * Times are CUDA-event milliseconds on the library's stream, flops are the
 * algorithmic real flops of the complex contractions (8 per complex MAC). */
typedef struct {
  double gemm_ms, gemm_flops;   /* all contractions (environments, X/Y, theta, Gram, gauge) */
  long long gemm_launches;
  double svd_ms;                /* truncated SVDs (Jacobi incl. sort/gather; Gram eigensolver
                                   without its Gram product, which counts as a contraction) */
  double svd_flops;             /* algorithmic real flops: Jacobi kernels 16 per complex element
                                   for the three dot products of every pair visited, 14 per
                                   element for every rotation applied; Gram eigensolver
                                   16/3 n^3 (tridiagonalisation) + 8 n^2 k (back-transformation) */
  long long svd_launches;
  long long jacobi_sweeps;      /* Jacobi sweeps executed (sum over SVDs) */
  double mpo_ms;                /* layer MPO build */
  double other_ms;              /* permutes, copies, norms */
  long long updates;            /* two-site updates done */
  long long kernel_launches;    /* every kernel the library launched */
  long long rsvd_attempts;      /* randomized SVDs tried (svd_mode 1, 2) */
  long long rsvd_accepted;      /* of which accepted (the rest fell back to Jacobi) */
  long long eig_svds;           /* truncated SVDs done by the Gram eigensolver (svd_path 0) */
  long long eig_fallbacks;      /* Gram eigensolver results not resolved or not finite: redone by
                                   Jacobi */
  long long eig_skipped;        /* SVDs sent straight to Jacobi: the last one at that bond was not
                                   resolvable by the eigensolver */
} dmrgc_stats;

/* Fill *opt with defaults (FP64, Jacobi, default cutoffs, default stream). */
dmrgc_status dmrgc_default_options(dmrgc_options* opt);

/* Create a context for n_qubits = grid->rows * grid->cols qubits in |0...0>
 * (the unentangled product state is an MPS with chi = 1, Sec. IV.A).
 * chi: maximum bond dimension (1 .. 4096).  *out receives the context. */
dmrgc_status dmrgc_create(int n_qubits, const dmrgc_grid* grid, int chi,
                          const dmrgc_options* opt, dmrgc_ctx** out);

/* The paper's own variant (Sec. IV.A, IV.B.1, V.C): an MPS of n_groups
 * tensors, tensor tau holding group_sizes[tau] consecutive sites of the chain
 * order (physical dimension 2^{group_sizes[tau]}, the first site the most
 * significant bit), optimised one tensor at a time: with the other tensors in
 * orthogonal form the optimum is M = F / sqrt(f) (Eq. optimization, F the
 * environment tensor of Eq. scalarproduct).  Each dmrgc_apply_layer starts
 * from a random tensor train (Sec. V.D.1): bond min(chi, 2^{sites left},
 * 2^{sites right}, old bond x layer-MPO bond) at each cut, entries
 * (2u - 1) + i (2u' - 1) with u, u' SplitMix64 uniforms of seed
 * opt->seed + (layer number - 1) at counters 2e, 2e + 1 for entry e of the
 * tensors taken in order and row-major; it is brought to orthogonal form with
 * its centre on tensor 0 by right-to-left factorisations, each remaining
 * factor carried into the left neighbour.  dmrgc_sweep(ctx, n) then runs n
 * sweeps, alternately tensors 0..n_groups-1 and back, n_groups updates each;
 * after an update the tensor is replaced by the isometry spanning the same
 * space (left or right singular vectors; values at the numerical-zero level
 * dropped, so a bond can shrink).  1 <= group_sizes[tau] <= 20, summing to
 * n_qubits; EINVAL otherwise.  Amplitudes and Metropolis sampling read the
 * grouped tensors directly; sequential sampling, overlaps and XEB are for
 * contexts with one qubit per tensor (dmrgc_create) and return EINVAL here;
 * dmrgc_get_mps returns the grouped tensors. */
dmrgc_status dmrgc_create_grouped(int n_qubits, const dmrgc_grid* grid, const int* group_sizes, int n_groups,
                                  int chi, const dmrgc_options* opt, dmrgc_ctx** out);

/* Sites per MPS tensor (*count entries: n_groups for a grouped context, else
 * n_qubits ones); sizes may be NULL. */
dmrgc_status dmrgc_group_sizes(const dmrgc_ctx* ctx, int* sizes, int* count);

/* Start one compression step (Sec. IV.B) for the gates of one layer (K
 * cycles, gates in time order).  Builds the layer MPO W_i[D,2,2,D] from the
 * gates (one-qubit gates merged into the neighbouring two-qubit gates'
 * site tensors, Sec. IV.B.2), then the initial guess by a zip-up of W.|Psi_Q>
 * from both ends towards the centre site.  The partial fidelity f_delta of
 * the previous step is committed to log F_tilde (Eq. Ftilde-sup).
 * gates: host array of n_gates records, copied before return. */
dmrgc_status dmrgc_apply_layer(dmrgc_ctx* ctx, const dmrgc_gate* gates, int n_gates);

/* Run n_sweeps * (N-1) two-site updates of the current step on the bouncing
 * schedule that starts at bond (m-1, m), m = N/2, moving left; n_sweeps = 2
 * ends at bond (m, m+1) with the orthogonality centre on site m.
 * Each update forms theta (Eq. scalarproduct), takes its truncated SVD and
 * sets the block to the constrained optimum (Eq. optimization).
 * f_last (may be NULL): partial fidelity f after the last update. */
dmrgc_status dmrgc_sweep(dmrgc_ctx* ctx, int n_sweeps, double* f_last);

/* log F_tilde = sum over steps of log f_delta (Eq. Ftilde-sup), including the
 * current step's latest f; f_delta_last: that latest f (Eq. fa-sup).
 * Either pointer may be NULL. */
dmrgc_status dmrgc_fidelity(dmrgc_ctx* ctx, double* log_F_tilde, double* f_delta_last);

/* Amplitudes <x|Psi> of count bitstrings (Sec. IV.A, the MPS definition).
 * bits: host uint8 [count][n_qubits] in qubit order (0 or 1).
 * out_re_im: host double [count][2]. */
dmrgc_status dmrgc_amplitude(dmrgc_ctx* ctx, const unsigned char* bits, long long count,
                             double* out_re_im);

/* <a|b>: inner product of the current states of two contexts (each the MPS
 * after its last sweep, or its state before the first layer), out_re_im[2].
 * With a a forward open run of the first layers from |0..0> and b a
 * backward open run from |x> under the adjoints of the remaining layers
 * (reversed, each gate U replaced by U^+), it is the closed-mode amplitude of
 * Sec. IV.C with an empty middle section.  Both contexts must have the same
 * grid and storage precision (else DMRGC_EINVAL); the contraction runs on a's
 * stream and in a's arithmetic after b's stream is synchronised. */
dmrgc_status dmrgc_overlap(dmrgc_ctx* a, dmrgc_ctx* b, double* out_re_im);

/* <a| U |b> for the gates of a middle section U (any number of cycles, in
 * time order, as for dmrgc_apply_layer): the closed-mode amplitude of
 * Sec. IV.C with the middle contracted exactly.  U becomes one exact MPO
 * (its bond, the product of the straddling gates' Schmidt ranks, must stay
 * <= 4096, else DMRGC_EINVAL) in a scratch context; a and b are not changed.
 * Same requirements and stream as dmrgc_overlap. */
dmrgc_status dmrgc_overlap_layer(dmrgc_ctx* a, dmrgc_ctx* b, const dmrgc_gate* gates, int n_gates,
                                 double* out_re_im);

/* Draw count bitstrings from |<x|Psi>|^2 by sequential conditional sampling.
 * Bit i (MPS site order) of sample j is 0 iff u < p(0 | earlier bits), with
 * u the (j*N + i + 1)-th output of SplitMix64 seeded with `seed`, mapped to
 * [0,1) with its top 53 bits.  out_bits: host uint8 [count][n_qubits], qubit order. */
dmrgc_status dmrgc_sample(dmrgc_ctx* ctx, long long count, unsigned long long seed,
                          unsigned char* out_bits);

/* Linear cross-entropy benchmark (Eq. FB-sup, estimated as in Eq. FB-estim):
 * draws `count` bit strings from `sampled` (dmrgc_sample with `seed`) and
 * returns f_b = 2^N <p(x)> - 1 with p(x) = |<x|reference>|^2 from the
 * reference context (for example an exact run at chi >= 2^(N/2)), and
 * optionally the standard error of that mean.  count in 2 .. 2^26; N <= 62. */
dmrgc_status dmrgc_xeb(dmrgc_ctx* sampled, dmrgc_ctx* reference, long long count, unsigned long long seed,
                       double* f_b, double* stderr_out);

/* Metropolis sampling of |<x|Psi>|^2 (App. C), for circuits whose
 * amplitudes are all of one order (Porter-Thomas): `chains` independent
 * Markov chains over bit strings.  Chain c starts at a uniform random string;
 * at step t = 1..steps it proposes a uniform random string x' and moves to it
 * with probability min(|<x'|Psi>|^2 / |<x|Psi>|^2, 1) (always from a string
 * of weight 0).  The random numbers are SplitMix64 uniforms of `seed` (top 53
 * bits) at counter g (N + 1) + q for bit q of the string (qubit order; the
 * bit is 1 iff u >= 1/2) and g (N + 1) + N for the acceptance test, with
 * g = c (steps + 1) + t (t = 0: the start); x' is taken iff
 * u |<x|Psi>|^2 < |<x'|Psi>|^2.  Amplitudes as dmrgc_amplitude, all chains
 * of a step in one batch.  out_bits: host uint8 [chains][steps][n_qubits],
 * the string of each chain after each step (qubit order); *accepted (may be
 * NULL): moves made at steps >= 1.  Any context, grouped ones included
 * (the amplitudes read the grouped tensors directly).  EINVAL when chains or
 * steps < 1, out_bits is NULL or chains x (steps + 1) exceeds 2^40. */
dmrgc_status dmrgc_metropolis(dmrgc_ctx* ctx, int chains, int steps, unsigned long long seed,
                              unsigned char* out_bits, long long* accepted);

/* Current bond dimensions of the MPS (tensors-1 entries: n_qubits-1, or
 * n_groups-1 for a grouped context) and of the per-site layer MPO
 * (n_qubits-1 entries); either pointer may be NULL. */
dmrgc_status dmrgc_bond_dims(const dmrgc_ctx* ctx, int* mps_bonds, int* mpo_bonds);

/* Copy the MPS tensors to the host as complex128: tensor i has shape
 * [chi_{i-1}][2^{r_i}][chi_i] (row-major; r_i = 1 unless grouped),
 * concatenated; *centre receives the orthogonality-centre tensor.  out must
 * hold dmrgc_mps_size() complex values. */
long long dmrgc_mps_size(const dmrgc_ctx* ctx);
dmrgc_status dmrgc_get_mps(const dmrgc_ctx* ctx, double* out_re_im, int* centre);

/* Load an MPS (checkpoint restore): tensor i has shape
 * [bonds[i]][2^{r_i}][bonds[i+1]] (row-major complex128, concatenated, the
 * layout of dmrgc_get_mps; N tensors, or n_groups for a grouped context),
 * bonds[0] = bonds[N] = 1 and 1 <= bonds[i] <= chi.  The tensors are converted to the
 * context's storage precision and become the state the next
 * dmrgc_apply_layer compresses (|Psi_Q> of Sec. IV.B); log_F_tilde is the
 * running Eq. (Ftilde-sup) sum to continue from.  A state saved with
 * dmrgc_get_mps after a step (centre on site N/2, the canonical form the sweep
 * leaves) and loaded here continues the run as if it had not stopped, up to
 * the rounding of a change of storage precision. */
dmrgc_status dmrgc_set_mps(dmrgc_ctx* ctx, const double* in_re_im, const int* bonds, double log_F_tilde);

/* The next n_updates two-site updates of the current step on the schedule
 * of dmrgc_sweep (which runs n_sweeps * (N-1) of them); f_last as there. */
dmrgc_status dmrgc_sweep_updates(dmrgc_ctx* ctx, long long n_updates, double* f_last);

/* Per-update partial fidelities of the current step (Sec. IV.B.1: they never
 * decrease).  Writes min(cap, count) values; *count receives the number done. */
dmrgc_status dmrgc_step_history(const dmrgc_ctx* ctx, double* f, int cap, int* count);

dmrgc_status dmrgc_get_stats(const dmrgc_ctx* ctx, dmrgc_stats* out);
dmrgc_status dmrgc_reset_stats(dmrgc_ctx* ctx);

/* Diagnostic entry points: run one kernel family of the sweep on host data,
 * synchronously on the default stream, with all device memory allocated and
 * freed inside the call.  Inputs and outputs are complex128 (re/im
 * interleaved) host arrays; the data are converted to the working precision
 * of `precision` on the device.
 *
 * dmrgc_test_gemm: C[M][N] = op(A) op(B) with the contraction engine (the
 * complex matrix products that form X, Y, theta and the environments,
 * Eq. (scalarproduct)).  op codes: 0 none, 1 transpose, 2 conjugate
 * transpose, 3 conjugate; row-major A (a_elems values, leading dim lda) and
 * B (b_elems, ldb); C row-major, N columns.
 *
 * dmrgc_test_svd: one-sided Jacobi on the columns of G (m x n, column-major)
 * followed by the truncation rule (Eq. optimization with the bond
 * constraint): s_out[n] receives the singular values in descending order,
 * *k_out the kept rank min(chi, #{s > rel_cut*s_1}), U_out[m][k] (row-major)
 * the kept left singular vectors. */
dmrgc_status dmrgc_test_gemm(int precision, int M, int N, int K, int opA, int opB, const double* A,
                             long long a_elems, long long lda, const double* B, long long b_elems,
                             long long ldb, double* C);
dmrgc_status dmrgc_test_svd(int precision, int m, int n, const double* G, int chi, double rel_cut,
                            double* s_out, int* k_out, double* U_out);

/* dmrgc_test_svd_gram: the sweep's other truncated SVD (options.svd_path 0):
 * the leading eigenvectors of H = G G^+ (m x m, TF32x3 product; FP32 for
 * precision DMRGC_FP32) by Householder tridiagonalisation, bisection, FP64
 * inverse iteration and back-transformation (the kept left singular vectors
 * of G, Eq. optimization with the bond constraint).  Complex64 precisions
 * only (1..3); 3 <= m <= 2048; 1 <= chi < m.  s_out[m]: the min(chi+1, m)
 * leading singular values, zeros after; U_out[m][k] row-major.  *k_out = k,
 * or -1 when the kept eigenvalues are not all resolved (lambda_{k-1} < 1e-5
 * lambda_0, or rel_cut set k while rel_cut^2 < 1e-5): the sweep then uses the
 * Jacobi SVD. */
dmrgc_status dmrgc_test_svd_gram(int precision, int m, int n, const double* G, int chi, double rel_cut,
                                 double* s_out, int* k_out, double* U_out);

/* Tuning: the Jacobi kernel for complex64 matrices of at most 1024 rows
 * (process-wide).  0 (default): column pairs, one warp per column, two
 * 4-column blocks per CTA; 1: 8 x 8 Gram blocks, rows spread over 512 threads,
 * one Jacobi sweep of the Gram per round.  Both compute the same
 * decomposition to working precision.  Other values: DMRGC_EINVAL. */
dmrgc_status dmrgc_set_jacobi_kernel(int variant);

/* Failure handling: the iteration limit of every spin wait of the Jacobi
 * kernels on the current device (the bounded grid barrier and the per-block
 * round counters; one poll is about 64 ns).  A wait that runs out sets the
 * launch's error flag, every CTA leaves at its next wait, and the calling
 * entry point returns DMRGC_ETIMEOUT; the context stays usable.  0 restores
 * the default (2e7 polls, about 1.3 s).  Process-wide per device. */
dmrgc_status dmrgc_set_wait_limit(unsigned long long spins);

/* ---- Rank model (svd_mode 2)
 *
 * Not in the paper: a multilayer perceptron that predicts, for the next update
 * at a bond, r = the smallest rank whose leading singular values hold all but
 * 1e-6 of the weight the update keeps (its log2).  The randomized SVD then
 * sketches r + p columns; the acceptance test above judges the result.
 *
 * Input (DMRGC_MLP_IN floats): 32 samples of log10(s_mu^2 / sum_{nu<k} s_nu^2)
 * at mu_j = round(j (k-1) / 31), j = 0..31, of the spectrum the last update at
 * the bond kept (k values); log2 k; log2 of the layer MPO's bond dimension at
 * the bond (the operator rank of the gates crossing it); log2 of the smaller
 * side of theta; 1 if the bond was already updated in this layer, else 0.
 * Network: x -> relu(W1 x + b1) -> relu(W2 h + b2) -> w3 . h + b3, hidden width
 * DMRGC_MLP_HIDDEN.  Parameters, FP32, in this order: W1 [H][IN] row-major,
 * b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1] (DMRGC_MLP_PARAMS floats). */
#define DMRGC_MLP_IN 36
#define DMRGC_MLP_HIDDEN 128
#define DMRGC_MLP_PARAMS (DMRGC_MLP_HIDDEN * DMRGC_MLP_IN + DMRGC_MLP_HIDDEN + \
                          DMRGC_MLP_HIDDEN * DMRGC_MLP_HIDDEN + DMRGC_MLP_HIDDEN + DMRGC_MLP_HIDDEN + 1)

/* Load a rank model into the context (host FP32 parameters, copied; inference
 * runs with BF16 weights and FP32 accumulation). */
dmrgc_status dmrgc_set_rank_model(dmrgc_ctx* ctx, const float* params);

/* Move the records logged since the last call (options.log_rank_records) to
 * the caller: features [count][DMRGC_MLP_IN], labels [count] (log2 r judged by
 * the full Jacobi SVD).  At most max records are returned; *count is set. */
dmrgc_status dmrgc_rank_records(dmrgc_ctx* ctx, float* features, float* labels, int max, int* count);

/* Train a rank model on the GPU (hand-written FP32 kernels): mean squared error
 * on the labels, Adam (beta 0.9, 0.999), mini-batches of `batch` rows drawn
 * without replacement per epoch from a SplitMix64-seeded shuffle; inputs and
 * labels are standardised internally and the returned parameters act on raw
 * inputs.  x: host [n][DMRGC_MLP_IN], y: host [n]; params_out: host
 * DMRGC_MLP_PARAMS floats; epoch_loss (optional): host [epochs], the mean
 * standardised loss of each epoch. */
dmrgc_status dmrgc_mlp_train(const float* x, const float* y, int n, int epochs, int batch, float lr,
                             unsigned long long seed, float* params_out, float* epoch_loss);

/* Loss (1/n) sum (f(x) - y)^2 and its gradient with respect to every
 * parameter, in the parameter order above, FP32 on the GPU (host buffers). */
dmrgc_status dmrgc_mlp_loss_grad(const float* params, const float* x, const float* y, int n, float* loss,
                                 float* grad);

/* y_out[n] = f(x) on the GPU; bf16 = 1 uses the BF16 inference kernel. */
dmrgc_status dmrgc_mlp_predict(const float* params, const float* x, int n, int bf16, float* y_out);

/* Batched open-mode runs of independent circuits (the compression step of
 * Sec. IV.B applied layer after layer, Sec. IV.C) on one GPU.  n_workers host
 * threads each own a CUDA stream and one context that is re-initialised for
 * every instance it takes from the shared queue (its device buffers are kept,
 * so allocation stops once a worker has seen its largest instance); instances
 * of different size and bond dimension run concurrently on the streams.
 * Options (precision, cutoffs) apply to all; options.cuda_stream is ignored.
 * rank_model (host, DMRGC_MLP_PARAMS floats, or NULL) is loaded into every
 * worker's context; svd_mode 2 without it returns DMRGC_EINVAL.
 * For each item the caller fills the inputs; the call fills the outputs. */
typedef struct {
  int rows, cols;            /* grid of this instance (n_qubits = rows*cols) */
  dmrgc_grid grid_view;      /* must equal {rows, cols, 0} */
  int chi;                   /* bond dimension */
  int n_layers;              /* compression steps */
  int n_sweeps;              /* dmrgc_sweep argument per step (2 = n_s of the paper's schedule) */
  const dmrgc_gate* gates;   /* all layers' gates, concatenated in order (host) */
  const int* layer_sizes;    /* n_layers gate counts (host) */
  double log_F_tilde;        /* out: Eq. (Ftilde-sup) */
  double seconds;            /* out: wall time of this instance */
  long long updates;         /* out: two-site updates done */
  int status;                /* out: dmrgc_status of this instance */
  int worker;                /* out: worker that ran it */
} dmrgc_batch_item;

dmrgc_status dmrgc_batch_run(dmrgc_batch_item* items, int count, int n_workers, const dmrgc_options* opt,
                             const float* rank_model, double* wall_seconds);

/* Truncated SVD of a device matrix that allocates no memory at all.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc -- for example code whose device memory is already fully
 * claimed by its own caching allocator (an extra cudaMalloc would fail or
 * break that allocator's budget), or latency-critical loops that must not
 * pay the device-wide synchronisation cudaMalloc and cudaFree can cause.
 * It runs the same one-sided Jacobi, truncation and gather kernels as the
 * sweep, but its scratch -- the barrier block, |G|_F^2, the sorted spectrum
 * and its permutation -- lives in a fixed 64 KiB array compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * G: device, complex (double2 for precision DMRGC_FP64, float2 otherwise),
 *    m x n column-major; it is overwritten (on return its columns are G V).
 * n: 2 .. 4096 columns (the array's limit); larger n returns DMRGC_EINVAL.
 * s_out: device double[n], the singular values in descending order.
 * U_out: device, m x k row-major in the same complex type (capacity m*min(chi,n)),
 *        the kept left singular vectors; *k_out (host) = k = min(chi,
 *        #{s > max(rel_cut*s_1, numerical zero)}).
 * stream: cudaStream_t (NULL = default stream); the call synchronises it
 *        before returning.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (the device must be current); make that first call
 * before any stream capture.  All calls share the one array and leave their
 * contents in it; the parts that must start at zero are cleared by each call.
 * Calls that overlap on the GPU (several host threads, or several streams)
 * race on the array: serialise them. */
dmrgc_status dmrgc_svd_noalloc(int precision, int m, int n, void* G, int chi, double rel_cut,
                               double* s_out, int* k_out, void* U_out, void* stream);

/* Message of the context's most recent failure (empty if no call has failed
 * yet; a later success does not clear it); the string is owned by the context
 * and valid until its next call.  A NULL context gives "null context". */
const char* dmrgc_last_error(const dmrgc_ctx* ctx);

/* Synchronise the context's stream and free every device and host buffer it
 * owns; ctx may be NULL.  The context must not be used afterwards. */
void dmrgc_destroy(dmrgc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DMRGC_H */
