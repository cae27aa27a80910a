/* qfs.h -- C-ABI of libqfs: QFactor-Sample circuit instantiation on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Kukliansky et al., "Leveraging Quantum Machine Learning
 * Generalization to Significantly Speed-up Quantum Compilation",
 * arXiv 2405.12866.  Instantiation (Section 2.1): given a target unitary U on
 * n qubits and a circuit structure C of 2-qubit gates, find gate unitaries
 * minimising the sample cost (Section 3, Eq. qfactor_sample_cost_function)
 *     c = (1/M) sum_j || U psi_j - C psi_j ||^2
 *       = 2 - (2/M) Re sum_j <psi_j| U^dagger C |psi_j>
 * over M orthonormal training states psi_j, by sweeps that replace each
 * gate with Y X^dagger from the SVD E = X D Y^dagger of its environment
 * (Eq. 2), right to left (Section 3), until c <= dist_tol or max_sweeps
 * (Appendix A).
 *
 * Conventions used by every entry point:
 *   - Complex numbers are interleaved (re, im) doubles, i.e. C99
 *     double complex / numpy complex128.
 *   - n qubits, N = 2^n.  Qubit q is bit (n-1-q) of a row index (qubit 0
 *     is the most significant bit).
 *   - pairs[2k], pairs[2k+1] = (a, b) are the qubits of gate k; the gate is
 *     a row-major 4x4 matrix indexed by 2*bit_a + bit_b.  Gates act in list
 *     order: gate 0 acts first, C = g_{L-1} ... g_1 g_0.
 *   - A target is N x N row-major; samples are N x M row-major (column j is
 *     psi_j); gates are L x 16 complex per start, starts contiguous.
 *   - "host" pointers are ordinary CPU memory (pinned memory makes the
 *     copies faster); "device" pointers are CUDA global memory on the
 *     context's device, e.g. torch tensor data pointers.  The caller owns
 *     every buffer passed in; the library never frees or keeps them.
 *   - Every int-returning call returns QFS_OK (0) or a negative QFS_E*
 *     code, and then qfs_last_error() describes the failure.  Reaching
 *     max_sweeps without converging is not an error (converged = 0).
 *   - A context is used by one host thread at a time.  Calls are
 *     synchronous with respect to the host unless noted.
 */
#ifndef QFS_H
#define QFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QFS_OK 0
#define QFS_EINVAL (-1)       /* bad argument (message says which) */
#define QFS_ENOMEM (-2)       /* device workspace allocation failed */
#define QFS_ECUDA (-3)        /* a CUDA call failed */
#define QFS_ETIMEOUT (-4)     /* a bounded device wait ran out */
#define QFS_EUNSUPPORTED (-5) /* valid but not supported (e.g. n > 14) */
#define QFS_ENONFINITE (-6)   /* NaN or Inf in an input */
#define QFS_EINTERNAL (-7)    /* an internal consistency check failed before any launch */

#define QFS_FP64 0  /* every step in complex128 */
#define QFS_MIXED 1 /* complex64 sweeps; FP64 SVD, master gates, refinement, cost check */

#define QFS_MAX_QUBITS 14

typedef struct qfs_ctx qfs_ctx;

typedef struct {
  int32_t n;             /* qubits, 2 <= n <= QFS_MAX_QUBITS */
  int32_t L;             /* gates, >= 1 */
  const int32_t* pairs;  /* host, 2*L qubit indices, a != b, both < n */
} qfs_circuit;

/* Hyperparameters (Appendix A of the paper).  qfs_default_params() fills
 * the values of the paper's evaluation where they apply. */
typedef struct {
  int32_t M;                 /* training states, 1 <= M <= 2^n (number_of_training_states) */
  int32_t multistarts;       /* independent random initial gate sets, >= 1 */
  int32_t max_sweeps;        /* max_iter: sweeps per run, >= 1 */
  int32_t min_sweeps;        /* min_iter before a plateau may stop a start */
  int32_t plateau_window;    /* plateau_windows_size; 0 disables plateau detection */
  int32_t precision;         /* QFS_FP64 or QFS_MIXED */
  int32_t refine_sweeps_max; /* QFS_MIXED: FP64 refinement sweeps allowed per start */
  int32_t start_groups;      /* starts are swept in this many concurrent groups (0 = auto);
                                results are bitwise the same for any value */
  uint64_t seed;             /* draws the training states and the initial gates */
  double dist_tol;           /* stop when a start's cost <= dist_tol */
  double diff_tol_r;         /* plateau: relative improvement threshold */
  double beta;               /* update damping, 0 <= beta < 1 (0 = full update) */
  int32_t restart_doubling;  /* 1: double-and-restart (Sec. 3, App. A): after every sweep from
                                min_sweeps on, the start with the lowest training cost is also
                                evaluated on M fresh validation states; when c_val / c_train - 1 >
                                overtrain_ratio the run halts, M doubles (up to 2^n), new training
                                and validation states are drawn, every start keeps its gates and
                                the run restarts (max_sweeps per attempt).  Success needs
                                c_train <= dist_tol and c_val <= (1 + overtrain_ratio) c_train.
                                Needs library-drawn training states (qfs_instantiate). */
  double overtrain_ratio;    /* overtrain_ratio of the generalisation check */
  int32_t training_distribution; /* distribution of library-drawn training and validation states
                                    (Appendix D): QFS_STATES_HAAR (columns of a Haar-random
                                    unitary) or QFS_STATES_BASIS (distinct computational-basis
                                    states, uniform without replacement) */
  int32_t concurrent_targets;    /* qfs_instantiate_many: target slots swept together (0 = 4); a slot
                                    whose target finishes takes the next one */
  double refine_switch_tol;      /* QFS_MIXED: a start whose complex64 cost is <= max(dist_tol, this) is
                                    checked in FP64 and, if that cost is above dist_tol, continued with
                                    up to refine_sweeps_max FP64 sweeps (0: switch at dist_tol) */
} qfs_params;

typedef struct {
  double cost;         /* sample cost of the returned gates (FP64) */
  int32_t sweeps;      /* sweeps run (all starts in lock step) */
  int32_t converged;   /* 1 if cost <= dist_tol */
  int32_t best_start;  /* index of the returned start */
  int32_t fp64_sweeps; /* QFS_MIXED: FP64 refinement sweeps run */
  int32_t training_states; /* M of the (last) attempt */
} qfs_result;

#define QFS_STATES_HAAR 0
#define QFS_STATES_BASIS 1

/* Fill *p with defaults: M = 2, multistarts = 16, max_sweeps = 10000,
 * min_sweeps = 6, plateau_window = 0, precision = QFS_FP64,
 * refine_sweeps_max = 50, start_groups = 0, seed = 0, dist_tol = 1e-8,
 * diff_tol_r = 1e-5, beta = 0, restart_doubling = 0, overtrain_ratio = 0.1,
 * training_distribution = QFS_STATES_HAAR, concurrent_targets = 0,
 * refine_switch_tol = 0 (the paper's
 * suggested values, with plateau detection and double-and-restart off).  With restart_doubling, attempt a > 0 draws its
 * training states (stream 1) and validation states (stream 5) from seed
 * XOR (a * 0x9E3779B97F4A7C15); attempt 0 validates with stream 5 of seed. */
void qfs_default_params(qfs_params* p);

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to run on (e.g. torch.cuda.current_stream().cuda_stream), or
 * NULL for a stream the context creates and owns.  The context owns its
 * device workspace, grown on demand and freed by qfs_destroy. */
int qfs_create(qfs_ctx** out, int device, void* cuda_stream);
void qfs_destroy(qfs_ctx* ctx);

/* Message of the last failed call on this host thread ("" if none).  The
 * pointer stays valid until the thread's next qfs_* call. */
const char* qfs_last_error(void);

/* Number of SMs of the context's device (host query, no kernel). */
int qfs_device_sms(const qfs_ctx* ctx);

/* Context options (none of them is in the paper; defaults in brackets).
 *   QFS_OPT_WAIT_LIMIT [2^25]: polls (each >= 32 ns) a dependency wait of
 *     the dataflow sweep makes before it gives up; the kernel then sets the
 *     run's error word, every CTA stops taking work and returns, and the call
 *     returns QFS_ETIMEOUT.  The context stays usable; the next call clears
 *     the error word.  Must be >= 1.
 *   QFS_OPT_WORKSPACE_CAP [0 = none]: largest device workspace, in bytes, a
 *     call may use; a call that needs more returns QFS_ENOMEM before it
 *     allocates (the paper's runs instead halve their multistarts on an
 *     out-of-memory error, Appendix A).
 *   QFS_OPT_FUSED_UPDATE [1]: per-step sweeps run each gate update in the
 *     backward launch (0: a separate update launch).
 *   QFS_OPT_DATAFLOW [1]: a sweep of all starts is one persistent launch
 *     (0: per-step launches).
 *   QFS_OPT_TWO_GATE_FORWARD [1]: the dataflow sweep applies consecutive
 *     forward gates on four distinct qubits in one step (0: one per step).
 *   QFS_OPT_FP64_TARGET_PRODUCT [0]: QFS_MIXED runs form U Psi in FP64
 *     instead of FP32 pair arithmetic.
 *   QFS_OPT_BATCH_LANES_PER_START [0 = tuned]: the batched form runs every
 *     problem class with this many lanes per start (4, 8, 16 or 32) instead
 *     of the autotuner's choice.
 * Every setting gives the same results up to the order of reduction sums.
 * QFS_EINVAL for an unknown option or a value out of range. */
#define QFS_OPT_WAIT_LIMIT 0
#define QFS_OPT_WORKSPACE_CAP 1
#define QFS_OPT_FUSED_UPDATE 2
#define QFS_OPT_DATAFLOW 3
#define QFS_OPT_TWO_GATE_FORWARD 4
#define QFS_OPT_FP64_TARGET_PRODUCT 5
#define QFS_OPT_BATCH_LANES_PER_START 6
int qfs_set_option(qfs_ctx* ctx, int32_t option, int64_t value);
int qfs_get_option(qfs_ctx* ctx, int32_t option, int64_t* value);

/* Kernel accounting.  Launches of every kind are always counted; with
 * profiling enabled each launch is also bracketed by CUDA events on the
 * context's stream, and qfs_profile_read returns, for one kind (or -1 for
 * all), the launches, the timed launches, their total device time in ms and
 * their total algorithmic traffic (bytes read + written by the definition
 * of the step; FLOPs for QFS_PROF_GEMM).  The counters are per context. */
#define QFS_PROF_BACKWARD 0 /* fused Phi update + environment partials */
#define QFS_PROF_FORWARD 1  /* B_k = g_k B_{k-1} */
#define QFS_PROF_UPDATE 2   /* warp SVD/polar update */
#define QFS_PROF_GEMM 3     /* Phi_L = U Psi */
#define QFS_PROF_RESIDUAL 4 /* complex64 residual cost pass */
#define QFS_PROF_CHECK 5    /* FP64 cost check of a candidate start */
#define QFS_PROF_OTHER 6    /* casts, input checks, finishing reductions */
#define QFS_PROF_BATCH 7    /* persistent batched sweep kernel */
#define QFS_PROF_MLP 8      /* tensor-core GEMMs of the learned warm start (FLOPs) */
#define QFS_PROF_DATAFLOW 9 /* one whole sweep of all starts as one persistent launch */
#define QFS_PROF_KINDS 10
int qfs_profile_enable(qfs_ctx* ctx, int enable);
int qfs_profile_reset(qfs_ctx* ctx);
int qfs_profile_read(qfs_ctx* ctx, int32_t kind, int64_t* launches, int64_t* timed,
                     double* total_ms, double* total_bytes);

/* Step time stamps of the dataflow sweep (a measurement aid; the paper has
 * no counterpart).  qfs_dataflow_trace_enable allocates room for `capacity`
 * stamps on the device (0 frees it and turns tracing off); while enabled,
 * every dataflow sweep whose steps x multistarts x 4 stamps fit records, per
 * (step, start), the device global timer (ns) when its first chunk started,
 * when its last chunk finished, when the environment partials were summed
 * (gate updates only; 0 otherwise) and when the step was published; when
 * the capacity also covers them, every work item (step, start, chunk, in
 * the order they are handed out) gets 4 more entries: dequeued, ready
 * (after its wait), processed (ns) and (CTA << 40) | (step << 20) | start.
 * qfs_dataflow_trace_read copies the stamps of the last traced sweep, laid
 * out [step][start][4] then [item][4], to out (host, capacity entries; may
 * be NULL to query *steps, *S and *items only; items may be NULL). */
int qfs_dataflow_trace_enable(qfs_ctx* ctx, int64_t capacity);
int qfs_dataflow_trace_read(qfs_ctx* ctx, uint64_t* out, int64_t capacity, int32_t* steps, int32_t* S,
                            int64_t* items);

/* Unit time stamps of the batched form's persistent sweep (a measurement aid;
 * the paper has no counterpart).  qfs_batch_trace_enable allocates room for
 * `capacity` stamps on the device (0 frees it and turns tracing off); while
 * enabled, every batched run whose units x 4 stamps fit records, per unit
 * (one problem and the starts that one warp sweeps to the end), the device
 * global timer (ns) when a warp took the unit and when it finished it, the
 * problem index, and (SM << 32) | (first start << 16) | (starts << 8) |
 * lanes per start.  Units are laid out launch by launch (one persistent
 * launch per lanes-per-start shape), each launch's units largest problem
 * first; the whole-batch plan check of a new class mix traces each plan it
 * times, and the last run is the one kept.  qfs_batch_trace_read copies the
 * stamps of the last traced run, [unit][4], to out (host, capacity entries;
 * may be NULL to query *units only). */
int qfs_batch_trace_enable(qfs_ctx* ctx, int64_t capacity);
int qfs_batch_trace_read(qfs_ctx* ctx, uint64_t* out, int64_t capacity, int64_t* units);

/* The method's own random draws (host only, no GPU): the M training states
 * (Section 3 and Appendix A: columns of a Haar-random unitary, here the Q
 * factor with positive R diagonal of a complex Gaussian N x M matrix) and
 * S x L Haar-random initial gates, from Philox4x32-10 (Salmon et al. 2011)
 * with key = seed, counter = (index, stream, 0); stream 1 = samples,
 * stream 2 = initial gates.  samples_out: host N x M; gates_out: host
 * S x L x 16 (either may be NULL). */
int qfs_generate_inputs(uint64_t seed, int32_t n, int32_t M, int32_t S, int32_t L,
                        double* samples_out, double* gates_out);

/* The library's draw of M states of either training distribution (host
 * only, no GPU), as qfs_instantiate makes it for training_distribution =
 * distribution: QFS_STATES_HAAR as in qfs_generate_inputs on the given
 * stream; QFS_STATES_BASIS the computational-basis states e_{p_0} ..
 * e_{p_{M-1}}, p the first M entries of a partial Fisher-Yates shuffle of
 * 0..N-1 whose step j swaps positions j and j + floor(w_j (N - j) / 2^32),
 * w_j = word 0 of Philox block (j, stream) under key = seed.  Streams: 1 =
 * training states, 5 = validation states.  out: host N x M complex128,
 * row-major.  QFS_EINVAL for n, M or distribution out of range. */
int qfs_generate_states(uint64_t seed, int32_t distribution, uint32_t stream, int32_t n, int32_t M,
                        double* out);

/* Instantiate `target` (host, N x N) on `circuit`: draws samples and
 * initial gates from p->seed, runs the multistart sweeps and writes the
 * selected start's gates to gates_out (host, L x 16).  Multistarts run in
 * lock step; the run stops at the first sweep after which some start has
 * cost <= dist_tol and returns the start with the lowest cost then (lowest
 * index on ties); otherwise the lowest final cost.  start_costs (host,
 * multistarts doubles, may be NULL) receives every start's last cost. */
int qfs_instantiate(qfs_ctx* ctx, const qfs_circuit* circuit, const double* target,
                    const qfs_params* p, double* gates_out, qfs_result* result,
                    double* start_costs);

/* As qfs_instantiate, with the training states (host, N x M, orthonormal
 * columns) and initial gates (host, multistarts x L x 16) given instead of
 * drawn from the seed. */
int qfs_instantiate_ex(qfs_ctx* ctx, const qfs_circuit* circuit, const double* target,
                       const double* samples, const double* init_gates, const qfs_params* p,
                       double* gates_out, qfs_result* result, double* start_costs);

/* As qfs_instantiate_ex with every array in device memory (result stays a
 * host struct).  Runs on the context's stream and returns when done. */
int qfs_instantiate_dev(qfs_ctx* ctx, const qfs_circuit* circuit, const double* target_dev,
                        const double* samples_dev, const double* init_gates_dev,
                        const qfs_params* p, double* gates_out_dev, qfs_result* result,
                        double* start_costs);

/* T independent instantiations of one circuit structure in one call: every
 * target's starts sweep together in the same dataflow launches, so the
 * per-start dependency chain of one target is hidden behind the work of the
 * others (throughput mode).  Each target follows exactly the rules of
 * qfs_instantiate (its own first converged sweep, its own selection) and
 * gets the result it would get alone: a target's work items and sums do not
 * depend on the other targets.  Arrays are target-major: targets T x N x N,
 * samples T x N x M and init_gates T x multistarts x L x 16 (either may be
 * NULL on the host entry: target t then draws from p->seed + t), gates_out
 * T x L x 16, results[T], start_costs T x multistarts (may be NULL).
 * QFS_EUNSUPPORTED with restart_doubling, without a cooperative launch, or
 * for odd M in QFS_MIXED. */
int qfs_instantiate_many(qfs_ctx* ctx, const qfs_circuit* circuit, int32_t T, const double* targets,
                         const double* samples, const double* init_gates, const qfs_params* p,
                         double* gates_out, qfs_result* results, double* start_costs);
/* As qfs_instantiate_many with targets, samples, init_gates and gates_out in
 * device memory (samples and init_gates required). */
int qfs_instantiate_many_dev(qfs_ctx* ctx, const qfs_circuit* circuit, int32_t T, const double* targets_dev,
                             const double* samples_dev, const double* init_gates_dev, const qfs_params* p,
                             double* gates_out_dev, qfs_result* results, double* start_costs);

/* Exactly one sweep (Section 3) for S starts, for parity checks: from
 * gates_in (host, S x L x 16) with target (host N x N) and samples (host
 * N x M), write the swept gates (host, S x L x 16), optionally every
 * gate's environment as used (envs_out, host, S x L x 16, row-major
 * E[x][y] = sum_{r,j} B_{k-1}[(x,r),j] conj(Phi_k[(y,r),j])) and each
 * start's cost after the sweep (costs_out, host, S).  QFS_FP64 reports
 * 2 - (2/M) Re Tr(g_1 E_1); QFS_MIXED runs the sweep in complex64 and
 * reports the residual form (1/M) sum_j ||U psi_j - C psi_j||^2 of the
 * swept gates accumulated from complex64 states. */
int qfs_sweep_once(qfs_ctx* ctx, const qfs_circuit* circuit, const double* target,
                   const double* samples, int32_t M, int32_t S, const double* gates_in,
                   int32_t precision, double beta, double* gates_out, double* envs_out,
                   double* costs_out);

/* The update step alone (Eq. 2 with the damping of Appendix A) for `count`
 * independent environments (host, count x 16): gates_out = polar factor of
 * ((1-beta) E + beta g_old^dagger)^dagger.  gates_old may be NULL when
 * beta = 0.  For a rank-deficient E any unitary completion is returned. */
int qfs_gate_update(qfs_ctx* ctx, int32_t count, const double* envs, const double* gates_old,
                    double beta, double* gates_out);

/* Phi_L = U Psi, the A tensor of Section 3 (the product every instantiation
 * starts from), on device buffers: target_dev N x N and samples_dev N x M
 * complex128 row-major, out_dev N x M (N = 2^n).  precision = QFS_FP64:
 * FP64 arithmetic.  QFS_MIXED: FP32 pair arithmetic (each FP64 operand
 * split into two floats, exact products through FMA, error-tracked sums),
 * about 48 significant bits, the product the mixed-precision runs use.
 * Synchronous; uses the context's workspace.  QFS_EINVAL for bad sizes. */
int qfs_target_product_dev(qfs_ctx* ctx, int32_t n, int32_t M, const double* target_dev,
                           const double* samples_dev, int32_t precision, double* out_dev);

/* Batched instantiation of P small problems (e.g. thousands of uneven 3-5
 * qubit partition blocks) in one persistent launch.  Problem i has ns[i] qubits
 * (2..6) and Ls[i] gates (1..32); pairs (host) holds 2*Ls[i] qubit indices
 * per problem, concatenated.  targets (host) holds the N_i x N_i targets
 * concatenated.  M_i = p->M if p->M > 0 (capped at N_i), else N_i / 2, with
 * N_i * M_i <= 1024.  samples (host, the N_i x M_i matrices concatenated)
 * and init_gates (host, multistarts x L_i x 16 per problem, concatenated)
 * may be NULL: then problem i draws them as qfs_generate_inputs does with
 * seed p->seed + i.  Every start sweeps in complex64 (FP32 polar update)
 * until its residual cost is <= p->dist_tol, p->max_sweeps, or a plateau
 * (p->plateau_window > 0: no relative improvement > p->diff_tol_r over that
 * many sweeps once p->min_sweeps have run, as in qfs_instantiate); the problem's
 * answer is the lowest-cost start among those that converged at its
 * earliest converged sweep (the lock-step rule of qfs_instantiate), made
 * unitary in FP64, checked in FP64 and refined with up to
 * p->refine_sweeps_max FP64 sweeps if the check is above tol.  gates_out
 * (host) receives L_i x 16 complex per problem, concatenated; results
 * (host) one qfs_result per problem (fp64_sweeps = refinement sweeps).
 * Problems are grouped in classes (n, L, M); for each class an autotuner
 * times the launch shapes that fit (G = 4, 8, 16 or 32 lanes per start, i.e.
 * 8, 4, 2 or 1 starts of a problem per warp, the block shape with the most
 * resident warps) on 4 sweeps of that class's problems at full occupancy the
 * first time the context sees the class, and keeps the fastest per
 * start-sweep (G = 32 unless another is 5% faster).  A unit of several
 * starts lives longer than a warp-per-start unit, so the first call of a
 * batch shape also times the whole batch with the per-class shapes and
 * with one start per warp everywhere, and keeps the faster plan.  The batch
 * runs as one captured graph with one persistent launch per shape,
 * replayed by later calls of the same shape.  Results do not depend on the shapes chosen beyond the order of
 * FP32 sums.  beta must be 0; multistarts 1..64. */
int qfs_instantiate_batch(qfs_ctx* ctx, int32_t P, const int32_t* ns, const int32_t* Ls,
                          const int32_t* pairs, const double* targets, const double* samples,
                          const double* init_gates, const qfs_params* p, double* gates_out,
                          qfs_result* results);

/* As qfs_instantiate_batch with targets, samples, init_gates (all required)
 * and gates_out in device memory; ns, Ls, pairs and results stay host. */
int qfs_instantiate_batch_dev(qfs_ctx* ctx, int32_t P, const int32_t* ns, const int32_t* Ls,
                              const int32_t* pairs, const double* targets_dev,
                              const double* samples_dev, const double* init_gates_dev,
                              const qfs_params* p, double* gates_out_dev, qfs_result* results);

/* The batched form's autotuner state on this context (a measurement aid;
 * the paper has no counterpart).  tuned (host, cap x 6 int32, may be NULL):
 * per problem class, n, L, M, multistarts, the chosen lanes per start G and
 * warps per block; *n_tuned: the classes tuned so far.  trials (cap x 6,
 * may be NULL) and trial_ns (cap doubles, may be NULL): every timed trial
 * (n, L, M, multistarts, G, warps) and its time per start-sweep in ns;
 * *n_trials: the trials so far.  plan_choice (cap int32, may be NULL) and
 * plan_ms (cap x 3 doubles, may be NULL): per class mix whose per-class
 * shapes were not all warp-per-start, the plan kept (0: per-class shapes,
 * 1: one start per warp everywhere, 2: 16 lanes per start wherever a class
 * admits it) and each plan's median ms over three interleaved timed runs
 * (-1: not timed, when plan 2 is plan 0); *n_plans: their number.  At most
 * cap rows are written. */
int qfs_batch_schedules(qfs_ctx* ctx, int32_t cap, int32_t* tuned, int32_t* n_tuned, int32_t* trials,
                        double* trial_ns, int32_t* n_trials, int32_t* plan_choice, double* plan_ms,
                        int32_t* n_plans);

/* Exactly one complex64 sweep of the batched form for every start of P
 * problems (parity checks): inputs as qfs_instantiate_batch (host; samples
 * N_i x M_i with M_i = M if M > 0 (capped at N_i) else N_i / 2, gates_in S x
 * L_i x 16 per problem, concatenated), lanes_per_start = 4, 8, 16 or 32
 * forces that launch shape for every class (0: the tuned shapes).  Every
 * start runs one sweep from its gates_in with the Jacobi started from the
 * identity; gates_out (host, same layout as gates_in, complex128 values of
 * the complex64 gates) and costs_out (host, P x S, may be NULL) receive the
 * swept gates and each start's complex64 residual cost
 * (1/M) sum_j ||U psi_j - C psi_j||^2. */
int qfs_batch_sweep_once(qfs_ctx* ctx, int32_t P, const int32_t* ns, const int32_t* Ls, const int32_t* pairs,
                         const double* targets, const double* samples, int32_t M, int32_t S,
                         const double* gates_in, int32_t lanes_per_start, double* gates_out, double* costs_out);

/* BF16 GEMM on the tcgen05 tensor cores (the learned warm start's layers):
 * C = A B^T (+ bias, optional GELU), A (M x K, leading dimension lda) and B
 * (N x K, ldb) bf16 row-major in device memory, accumulation in FP32; C32
 * (fp32) and/or C16 (bf16, GELU applied when gelu != 0) receive M_valid
 * (<= M, 0 = M) rows with leading dimension ldc.  M and N multiples of 128,
 * K of 64, lda and ldb multiples of 8, ldc of 8, and A, B, C32, C16, bias
 * 16-byte aligned.  A product with only C32 (no bias, no GELU) whose tiles
 * would leave most SMs idle is split along K; the partial tiles are added
 * into C32 (zeroed first) with atomics, so the summation order, and the
 * last bits of C32, can vary from call to call. */
int qfs_gemm_bf16_dev(qfs_ctx* ctx, int32_t M, int32_t N, int32_t K, const void* A, int32_t lda,
                      const void* B, int32_t ldb, float* C32, void* C16, int32_t ldc,
                      const float* bias, int32_t gelu, int32_t M_valid);

/* Learned warm start.  A multilayer perceptron maps the target of a 4-qubit
 * block applied to 8 fixed states (16 x 8 complex = 256 reals) through three
 * hidden layers of 1024 (GELU, tanh form) to 6 gates (192 reals: gate g,
 * entry 4r + c, re/im), projected onto U(4) by their polar factors.  It is
 * trained on (target, converged gates) pairs that the method produces,
 * with mean squared error on the 192 reals and Adam; all products run on
 * the tcgen05 GEMM (BF16 operands, FP32 accumulation, FP32 master weights).
 * The paper has no learned part; the sweep judges every proposal.
 *
 * qfs_ws_create: weights N(0, 2/fan_in) from Philox (seed), biases zero;
 *   batch_cap (multiple of 128) bounds the rows of one pass.
 * qfs_ws_params: copy the FP32 parameters out (out) and/or in (in), layer
 *   by layer W[out x in] then b[out], dims 256->1024->1024->1024->256 (the
 *   last 64 outputs are padding); *count receives the number of floats.
 * qfs_ws_loss_grad: loss and gradients (same layout) on one batch of
 *   targets (host, count x 16 x 16 complex) and labels (host, count x 192).
 * qfs_ws_train: epochs of shuffled mini-batches with Adam (beta1 0.9,
 *   beta2 0.999, eps 1e-8), the step size decaying from lr to lr_final on a
 *   cosine over the call's steps (lr_final = lr: constant); the training set
 *   stays on the device for the call; epoch_loss (may be NULL) gets each
 *   epoch's mean loss.  Features are 4 U Phi_fix (unit variance).
 * qfs_ws_predict: gates_out (host, count x 6 x 16 complex, unitary). */
typedef struct qfs_ws qfs_ws;
int qfs_ws_create(qfs_ctx* ctx, uint64_t seed, int32_t batch_cap, qfs_ws** out);
void qfs_ws_destroy(qfs_ws* ws);
int qfs_ws_params(qfs_ws* ws, float* out, const float* in, int64_t* count);
int qfs_ws_loss_grad(qfs_ws* ws, int32_t count, const double* targets, const double* labels, double* loss,
                     float* grads_out);
int qfs_ws_train(qfs_ws* ws, int32_t count, const double* targets, const double* labels, int32_t epochs,
                 int32_t batch, double lr, double lr_final, uint64_t shuffle_seed, double* epoch_loss);
int qfs_ws_predict(qfs_ws* ws, int32_t count, const double* targets, double* gates_out);

/* The learned warm start as an instantiation policy for P targets of the
 * learned structure (host, P x 16 x 16): the first start of target i is the
 * network's prediction projected onto U(4) (or first_gates, host P x 6 x 16,
 * when given: the same policy with other first starts), run alone in the
 * batched form for at most first_sweeps sweeps (training states drawn from
 * p->seed + i); every target left unconverged falls back to
 * p->multistarts random starts and p->max_sweeps sweeps, with training
 * states and starts drawn from p->seed + 2^30 + i.  The prediction stays on
 * the device.  gates_out (host, P x 6 x 16) and results[P] receive each
 * target's answer (best_start 0: the first start; j + 1: fallback start j;
 * sweeps: both stages).  stats (host, 4 int64, may be NULL): targets the
 * first start converged, its start-sweeps, the fallback's start-sweeps,
 * targets that fell back.  p->M = 0 takes N / 2 = 8 training states. */
int qfs_ws_instantiate(qfs_ws* ws, int32_t P, const double* targets, const double* first_gates,
                       const qfs_params* p, int32_t first_sweeps, double* gates_out, qfs_result* results,
                       int64_t* stats);

/* One FP64 sweep (as qfs_sweep_once with QFS_FP64) that allocates no
 * memory, for callers that cannot call cudaMalloc: code running inside a
 * host framework that owns every device byte through its own allocator or a
 * fixed memory budget, and code that must not reach cudaMalloc/cudaFree
 * because those calls can synchronise the whole device.  The paper has no
 * counterpart; this is a deployment variant of the sweep.
 *
 * Every array is device memory supplied by the caller, on the current CUDA
 * device: target_dev (N x N), samples_dev (N x M), gates_in_dev and
 * gates_out_dev (S x L x 16; they may be the same buffer), costs_out_dev
 * (S doubles, may be NULL: 2 - (2/M) Re Tr(g_1 E_1) per start) and
 * envs_out_dev (S x L x 16, may be NULL).  The call is enqueued on
 * `cuda_stream` (a cudaStream_t, NULL = the legacy default stream) and
 * returns without waiting for it.
 *
 * The sweep's scratch (U Psi, the B list, Phi, reduction partials) is one
 * statically sized device array of QFS_NOALLOC_SCRATCH_BYTES, which every
 * GPU that loads the library holds until the process exits.  A problem
 * whose scratch, N*M*16 * (1 + S*max(L-1,1) + S) bytes plus the partials,
 * exceeds it is rejected with QFS_EUNSUPPORTED and a message giving the
 * size it needs.  All calls on a device share the array and it keeps the
 * last call's contents; every scratch word a sweep reads is written earlier
 * in the same call, so nothing has to be cleared between calls, but calls
 * that overlap on the GPU (two streams, or two host threads) race on it.
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current) and caches it for the
 * rest of the process, which assumes the device's primary context lives as
 * long (after a cudaDeviceReset the cached address is stale); make that
 * first call before any stream capture. */
#define QFS_NOALLOC_SCRATCH_BYTES (16u << 20)
int qfs_sweep_once_noalloc(void* cuda_stream, const qfs_circuit* circuit, const double* target_dev,
                           const double* samples_dev, int32_t M, int32_t S, double beta,
                           const double* gates_in_dev, double* gates_out_dev,
                           double* costs_out_dev, double* envs_out_dev);

#ifdef __cplusplus
}
#endif

#endif /* QFS_H */
