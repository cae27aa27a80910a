// Internal launcher interface between the engine (host C++) and the kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qfs {

enum Real { R32 = 0, R64 = 1 };

// Geometry of one gate step on one state shape.
struct Geom {
  int n;          // qubits
  int M;          // samples (columns)
  int pos_a;      // bit position of qubit a: n-1-a
  int pos_b;      // bit position of qubit b
  int lo, hi;     // min/max of the two positions
  long long sN;   // N*M complex elements per state
};
Geom make_geom(int n, int M, int a, int b);

// Geometry of a fused backward step: the union of the qubits of the gate
// carried into Phi (ua, ub) and of the gate whose environment is reduced
// (qa, qb).  Local bits U-1, U-2 are (ua, ub); EA, EB are the local bits of
// (qa, qb).  pos[i] is the row-bit position of local bit i; ins[] the same
// positions sorted ascending (for inserting zero bits into a unit index).
struct BwdGeom {
  int n, M;
  long long sN;
  int U;
  int pos[4];
  int ins[4];
  int ea, eb;
};
BwdGeom make_bwd_geom(int n, int M, int ua, int ub, int qa, int qb);

// Launch shape of the streaming kernels for one (n, M, S, precision).
struct Shape {
  int vec;              // complex samples per thread unit (2 for fp32, 1 for fp64)
  int units_per_start;  // (N/4) * (M/vec)
  int chunk;            // units per block
  int nblk;             // blocks per start
  int threads;          // block size
};
Shape make_shape(int n, int M, int S, Real r, int num_sms);
// Shape of a backward step whose unit spans 2^U rows.
Shape make_bwd_shape(int n, int M, int S, Real r, int num_sms, int U);

// B_out[s] = g[s] B_in[s] for each start s (B_in shared when in_stride = 0).
void launch_forward(Real r, const Geom& g, const Shape& sh, int S,
                    const void* in, long long in_stride, void* out,
                    const void* gates, long long gate_stride, const int* active,
                    cudaStream_t st);

// One warp per start: sum the partials, form (1-beta) E + beta g_old^dagger,
// take the unitary polar factor of its adjoint (the SVD update of Eq. 2),
// write it to g64 (and to g32 as complex64 when non-null).  When cost_out is
// non-null it receives 2 - (2/M) Re Tr(g_new E).  When env_out is non-null
// the environment itself is stored there (16 complex128 per start).
struct UpdateArgs {
  const void* partials; int nblk;
  int partials_f32;                      // partials are float (complex64 steps) or double
  double2* g64; long long g_stride;     // gate to replace, per start
  float2* g32;                           // complex64 copy (nullable)
  double beta;
  double* cost_out; double inv_M;        // nullable
  double2* env_out; long long env_stride;  // nullable
  int S;
  const int* active;                     // nullable: all starts active
  double2* vprev;                        // nullable: per-start right singular vectors of the
                                         // gate's previous update (same strides as g64)
};
void launch_update(const UpdateArgs& a, cudaStream_t st);

// Dataflow sweep (sweep_df.cu): one cooperative launch runs every step of a
// sweep for every start as (step, start, chunk) work items.
enum DfKind {
  DF_FWD = 0,      // B_k = g_k B_{k-1} on the pair of fg
  DF_BWD4 = 1,     // backward step, gates k+1 and k on four distinct qubits (16-row units)
  DF_BWD2_10 = 2,  // backward step on one pair (no gate, or gate k+1 on the same pair)
  DF_BWD2_01 = 3,  //   ... with the pair of gate k in the other order
  DF_BWD3_20 = 4,  // backward step, gates k+1 and k sharing one qubit (ea, eb)
  DF_BWD3_02 = 5,
  DF_BWD3_10 = 6,
  DF_BWD3_01 = 7,
  DF_RESID = 8,    // residual cost (1/M) sum |g_1^dagger Phi_1 - Psi|^2
  DF_FWD2 = 9,     // B_k = g_k B_{k-1} and B_{k+1} = g_{k+1} B_k, gates on four distinct qubits
};
struct DfStep {
  int kind;
  int units, chunk, nchunk;             // units per start, units per chunk, chunks per start
  long long item0;                      // first work item of this step
  const void* in; long long in_stride;  // forward input / backward B_{k-1} / residual Psi
  long long in_gstride;                 // per target (start s belongs to target s / spt): Psi of each target
  long long phi_in_gstride;             // per target: Phi_L = U Psi of each target
  int spt;                              // starts per target (targets swept together share one launch)
  void* out;                            // forward output B_k (start stride fg.sN)
  void* out2;                           // DF_FWD2: B_{k+1} (start stride bg.sN)
  const void* gate2;                    // DF_FWD2: gate k+1 (start stride gate_stride)
  const void* phi_in; long long phi_in_stride;
  void* phi_out;                        // start stride bg.sN; null: not stored
  const void* gate; long long gate_stride;  // gate applied (null: none)
  Geom fg;
  BwdGeom bg;
  UpdateArgs upd;                       // backward steps: the update of gate k
};
struct DfArgs {
  const DfStep* steps; int nsteps; int S;
  long long total_items;
  const int* active;                    // nullable
  unsigned* queue;                      // 1: next work item
  unsigned* chunk_cnt;                  // nsteps x S finished chunks
  unsigned* done;                       // S: steps finished per start
  int* err;                             // bit 0: a bounded wait ran out
  long long wait_limit;                 // polls of a dependency wait before it gives up
  void* partials;                       // S x part_stride x 32 environment partials (float or double)
  double* resid_partials;               // S x part_stride x 32, residual step only
  int part_stride;                      // slots per start: the most chunks of any step
  double* resid_cost; double inv_M;     // residual step output
  double* cost_row;                     // nullable: this sweep's costs are also written here
  unsigned* zero_next; int zero_count;  // nullable: the next sweep's control words, zeroed at entry
  double resid_skip;                    // > 0: a start whose update-time cost estimate exceeds it skips the
                                        //   residual pass (the estimate stands as its cost)
  int stop_from_update;                 // the update's cost (FP64 sweeps) may set the stop flag
  int* stop;                            // nullable: set when an active start's cost <= stop_tol; a launch
  double stop_tol;                      //   that finds it set returns at once (batched sweeps)
  unsigned long long* item_trace;       // nullable: per work item (dequeued, ready, processed, CTA)
  unsigned long long* trace;            // nullable: per (step, start) 4 global-timer stamps (first
                                        // chunk started, last chunk done, partials summed, published)
};
int df_blocks_per_sm(Real r);
cudaError_t launch_sweep_df(Real r, const DfArgs& a, int num_sms, cudaStream_t st);
void df_chunking(DfStep& st, double bytes_per_unit, double target);

// Set `count` 4x4 complex128 matrices to the identity.
void launch_set_identity4(double2* v, long long count, cudaStream_t st);

// Environment partials of one backward step.  Phi_k = g^dagger Phi_in on
// the pair (ua, ub) of the geometry when `gate` is non-null (else Phi_k =
// Phi_in); Phi_k is stored to phi_out when non-null; per-block partial sums
// of E[x][y] += Bprev[x] conj(Phi_k[y]) over the pair (qa, qb) go to
// partials[(s*nblk + blk)*32 + 2*(4x+y) + {0: re, 1: im}].
// mode 1: instead of E, slot 0 gets sum |Phi_k - Bprev|^2 (needs U = 2).
// Partials are float for complex64 steps in mode 0, double otherwise.
// With `fuse`, the last block of each start to finish performs that start's
// update (as launch_update would); `counters` (one per start) must be zero
// before the launch and are zero again after it.
void launch_backward(Real r, int mode, const BwdGeom& g, const Shape& sh, int S,
                     const void* bprev, long long bprev_stride,
                     const void* phi_in, long long phi_in_stride, void* phi_out,
                     const void* gates, long long gate_stride,
                     void* partials, int stream_b, const int* active, cudaStream_t st,
                     const UpdateArgs* fuse = nullptr, unsigned* counters = nullptr);

// Arguments of the backward kernels.
struct BwdArgs {
  const void* bprev; long long bprev_stride;
  const void* phi_in; long long phi_in_stride;
  void* phi_out;
  const void* gates; long long gate_stride;
  void* partials; int nblk;   // T per slot in MODE 0, double in MODE 1
  BwdGeom g; int units_per_start; int chunk;
  int stream_b;   // B_{k-1} is read once per sweep: load it evict-first
  const int* active;
  // Fused update (MODE 0): the last block of start s to finish updates gate
  // k of start s from all blocks' partials.
  int fuse;
  unsigned* counters;  // per start, zero between launches
  UpdateArgs upd;
};

// Residual cost: cost[s] = sum_blk partial[s][blk][0] * inv_M.
void launch_residual_finish(const double* partials, int nblk, int S, double inv_M,
                            double* cost_out, cudaStream_t st);

// Batched polar update of independent environments (the a4 step alone).
void launch_gate_update_batch(int count, const double2* envs, const double2* g_old,
                              double beta, double2* g_out, cudaStream_t st);

// out (N x M, complex128) = U (N x N) * Psi (N x M), all row-major.
void launch_gemm_upsi(const double2* U, const double2* Psi, double2* out, int N, int M,
                      cudaStream_t st);

// U Psi in FP32 pair arithmetic (FP64-class accuracy, about 48 bits).
// psi_split: N x M float4 scratch; scratch: splits x N x M double2 (unused
// when splits == 1).  upsi_pair_splits picks the number of K slabs that
// fills num_sms and fits scratch_bytes.
int upsi_pair_splits(int N, int M, int num_sms, size_t scratch_bytes);
void launch_gemm_upsi_pair(const double2* U, const double2* Psi, double2* out, int N, int M, float4* psi_split,
                           double2* scratch, int splits, int num_sms, cudaStream_t st);
void launch_cast_c128_to_c64(const double2* in, float2* out, long long count, cudaStream_t st);

// flag[0] |= 1 when any of the `count` doubles is NaN or infinite.
void launch_nonfinite_check(const double* x, long long count, int* flag, cudaStream_t st);

// ---------------------------------------------------------------- batches

constexpr int kBatchMaxWarps = 8;

// One instantiation problem of a batch; offsets are in complex elements
// (pairs: in ints) into the packed arrays of BatchArgs.
struct BatchProblem {
  int n, L, M;
  int pair_off;
  long long state_off;   // psi/phil (N x M)
  long long target_off;  // targets (N x N)
  long long gate_off;    // init_gates/gates32 (S x L x 16)
  long long gate_out_off;  // gates_out (L x 16)
};

struct BatchArgs {
  const BatchProblem* probs;
  int P, S;
  const double2* targets;
  double2* psi64;
  double2* phil64;
  float2* psi32;
  float2* phil32;
  const int* pairs;
  const double2* init_gates;
  float2* gates32;        // each start's gates after its sweeps
  int* conv_sweep;        // P x S: sweep at which the start converged (INT_MAX if not)
  double* final_cost;     // P x S: complex64 residual cost after its last sweep
  int* sweeps_run;        // P x S
  int* s_star;            // P: earliest converged sweep of each problem
  int* queue;             // work counter, zero before the sweep launch
  const int* order;       // problem indices, largest work first
  int max_sweeps;
  double tol;
  int plateau_window;     // > 0: a start stops after this many sweeps without relative
  double diff_tol_r;      //   improvement > diff_tol_r (App. A), once min_sweeps have run
  int min_sweeps;
  int max_elems, max_L;   // largest N*M and L in the batch (shared-memory slices)
  double2* gates_out;     // selected gates, FP64 (L x 16 per problem)
  double* res_cost;
  int* res_sweeps;
  int* res_best;
  int* res_refine;
  int refine_max;
  int refine_unconverged;  // also refine problems whose starts never reached tol
  // Non-null: 4 stamps per unit of this launch, indexed as its units are
  // (taken, finished (global timer, ns), problem, (SM << 32) | (first start
  // << 16) | (starts << 8) | lanes per start).
  unsigned long long* unit_trace;
};

// A unit of the batched sweep: problem p and its starts s0 .. s0 + ns - 1,
// swept by one warp with G lanes per start (ns <= 32 / G).
struct BatchUnit {
  int p, s0, ns;
};

void launch_batch_prep(const BatchArgs& a, cudaStream_t st);
// A warp's shared memory (float2) with G lanes per start, for problems of
// at most max_elems = N * M amplitudes and max_L gates.
int batch_region_f2(int G, int max_elems, int max_L);
// Shared memory of a block of `warps` warps of that shape.
size_t batch_sweep_smem(int G, int warps, int max_elems, int max_L);
// Resident blocks per SM of a launch of `warps` warps and `smem` bytes (0:
// it does not fit).
int batch_sweep_blocks_per_sm(int G, int warps, size_t smem);
// The persistent sweep over `units` (queue: a zeroed counter), G in
// {4, 8, 16, 32}; region_f2: each warp's shared memory in float2.
void launch_batch_sweep(int G, const BatchArgs& a, const BatchUnit* units, int nunits, int* queue, int blocks,
                        int warps, int region_f2, cudaStream_t st);
void launch_batch_finalize(const BatchArgs& a, cudaStream_t st);

// ---------------------------------------------------------- learned part

// C[M x N] = A[M x K] B[N x K]^T (+ bias) with tcgen05 tensor cores.  M, N
// multiples of 128, K of 64; lda, ldb multiples of 8; rows >= M_valid are
// computed but not stored.  C32 (fp32) and/or C16 (bf16, after GELU if
// gelu) receive the result with leading dimension ldc.
struct GemmArgs {
  const __nv_bfloat16* A;
  int lda;
  const __nv_bfloat16* B;
  int ldb;
  float* C32;
  __nv_bfloat16* C16;
  int ldc;
  const float* bias;
  int gelu;
  int M, N, K, M_valid;
  int* err;
  int splitk = 1;  // > 1: K split over grid z, partial tiles added into C32 (C32 only)
  int sms = 0;     // SMs of the device (> 0: products with fewer 128 x 256 tiles than SMs take
                   // 128 x 128 tiles, two CTAs per SM)
};
cudaError_t launch_gemm_bf16_tc(const GemmArgs& g, cudaStream_t st);
// Split-K factor that fills the GPU for a C32-only product (1 otherwise).
int gemm_splitk_for(const GemmArgs& g, int num_sms);
// Tile width of a product: 256 when N allows it and the 128 x 256 tiles fill
// every SM (or the SM count is unknown), else 128.
int gemm_bn_for(const GemmArgs& g);

void launch_ws_features(const double2* U, const double2* phif, int count, int rows, __nv_bfloat16* X,
                        cudaStream_t st);
void launch_transpose_bf16(const __nv_bfloat16* src, int R, int C, __nv_bfloat16* dst, cudaStream_t st);
void launch_ws_gates_adjoint(const float* Y, int ldy, int count, double2* E, cudaStream_t st);
void launch_loss_accumulate(const double* parts, int n, double scale, double* acc, cudaStream_t st);
// jstep (nullable, device): the step within the epoch; the rows taken
// start at idx + *jstep * batch.
void launch_ws_gather(const __nv_bfloat16* Xall, const float* Tall, const int* idx, int bv, int B,
                      __nv_bfloat16* X, float* T, cudaStream_t st, const int* jstep = nullptr, int batch = 0);
// *jstep += 1 and *gstep += 1 on the device (the end of a training step).
void launch_ws_step_advance(int* jstep, int* gstep, cudaStream_t st);
void launch_cast_f32_bf16(const float* a, __nv_bfloat16* b, long long n, cudaStream_t st);
// Returns the number of loss partial sums written.
int launch_ws_loss_grad(const float* Y, int ldy, const float* T, int n_out, int rows, int B_valid, float* dY32,
                        __nv_bfloat16* dY16, double* loss_part, cudaStream_t st);
void launch_gelu_back(const float* dH, const float* Z, long long n, int ld, int B_valid, float* dZ32,
                      __nv_bfloat16* dZ16, cudaStream_t st);
void launch_colsum(const float* G, int rows, int cols, float* db, cudaStream_t st);
// sched (nullable, device): lr, bc1, bc2 of step *sched_step (3 floats per
// step), in place of the lr, bc1, bc2 arguments.
void launch_adam(float* w, float* m, float* v, const float* g, long long n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, __nv_bfloat16* w16, cudaStream_t st, const float* sched = nullptr,
                 const int* sched_step = nullptr);

}  // namespace qfs
