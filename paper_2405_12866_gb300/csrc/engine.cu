// Host engine and C-ABI of libqfs: argument checks, workspace, the sweep
// sequence of QFactor-Sample (Section 3 of the paper) and the multistart run
// with its stopping rules (Appendix A).  Every arithmetic step of the sweep
// runs in the CUDA kernels; the host orders launches and reads back one cost
// per start after each sweep.
#include "../../include/qfs.h"
#include "qfs_kernels.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <future>
#include <functional>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace qfs {
void generate_samples(uint64_t seed, int n, int M, std::complex<double>* out);
void generate_states(uint64_t seed, uint32_t stream, int n, int M, std::complex<double>* out);
void draw_states(int kind, uint64_t seed, uint32_t stream, int n, int M, std::complex<double>* out);
void generate_gates(uint64_t seed, int count, std::complex<double>* out);
}  // namespace qfs

using namespace qfs;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? QFS_ENOMEM : QFS_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
  } while (0)

#define TRY(expr)              \
  do {                         \
    int r_ = (expr);           \
    if (r_ != QFS_OK) return r_; \
  } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

// Per-kernel timing with CUDA events on the context's stream (off unless
// enabled); launches are counted always.
struct ProfRec {
  cudaEvent_t a, b;
  int id;
  double bytes;
};
struct Prof {
  bool on = false;
  bool capturing = false;        // launches are being captured into a graph
  std::vector<cudaEvent_t> pool;
  std::vector<ProfRec> pending;
  std::vector<ProfRec> graph;    // event pairs recorded by graph nodes
  long long launches[QFS_PROF_KINDS] = {};
  long long timed[QFS_PROF_KINDS] = {};
  double ms[QFS_PROF_KINDS] = {};
  double bytes[QFS_PROF_KINDS] = {};
};

constexpr int kMaxGroups = 8;

struct qfs_ctx {
  Prof prof;
  // Streams for groups of starts swept concurrently, forked from and joined
  // back to `stream` with events (created on first use).
  cudaStream_t gstream[kMaxGroups] = {};
  cudaEvent_t gevent[kMaxGroups] = {};
  cudaEvent_t fork_event = nullptr;
  cudaStream_t cap_stream = nullptr;  // stream used only to capture sweep graphs
  bool fuse_update = true;  // gate update inside the backward launch (QFS_OPT_FUSED_UPDATE)
  bool dataflow = true;     // whole sweeps as one cooperative persistent launch (QFS_OPT_DATAFLOW)
  bool df_fwd2 = true;      // forward gates on four distinct qubits two per step (QFS_OPT_TWO_GATE_FORWARD)
  bool upsi_fp64 = false;   // mixed runs: U Psi in FP64 instead of FP32 pair arithmetic (QFS_OPT_FP64_TARGET_PRODUCT)
  unsigned long long* df_trace = nullptr;  // device buffer for step time stamps (qfs_dataflow_trace_*)
  size_t df_trace_n = 0;
  int df_trace_steps = 0, df_trace_S = 0;  // shape of the last traced sweep
  long long df_trace_items = 0;            // work items with stamps in that sweep (0: none)
  unsigned long long* bt_trace = nullptr;  // device buffer for batched unit stamps (qfs_batch_trace_*)
  size_t bt_trace_n = 0;
  long long bt_units = 0;                  // units with stamps in the last traced batched run
  double df_item_bytes = 1024.0 * 1024.0;  // largest streaming bytes of one dataflow work item (QFS_DF_ITEM_KB)
  double df_items_per_cta = 1.5;           // work items per CTA and backward step (QFS_DF_ITEMS_PER_CTA)
  double df_items_per_cta_fwd = 1.0;       // ... and forward step (QFS_DF_ITEMS_PER_CTA_FWD)
  long long df_wait_limit = 1LL << 25;     // polls before a dataflow dependency wait gives up (QFS_OPT_WAIT_LIMIT)
  // Batched form: the tuned launch shape per problem class (n, L, M) and the
  // captured graphs of recent batch shapes (replayed when a call repeats one).
  std::vector<std::pair<long long, std::pair<int, int>>> batch_tuned;  // class key -> (G, warps)
  // Every autotuner trial: n, L, M, S, G, warps, and the measured time per
  // start-sweep in ns (qfs_batch_schedules reads them back).
  std::vector<std::array<int, 6>> batch_trial_shape;
  std::vector<double> batch_trial_ns;
  // Whole-batch plan decisions: batch shape key -> 0 (per-class shapes), 1
  // (one start per warp everywhere) or 2 (16 lanes per start wherever a class
  // admits it), with the three timings in ms.
  std::vector<std::pair<uint64_t, int>> batch_plans;
  std::vector<std::array<float, 3>> batch_plan_ms;
  struct BatchGraph {
    uint64_t key = 0;
    cudaGraphExec_t exec = nullptr;
    long long launches[QFS_PROF_KINDS] = {};
  };
  std::vector<BatchGraph> batch_graphs;
  int batch_force_G = 0;                   // > 0: every class runs with G lanes per start (tests)
  size_t ws_cap = 0;                       // largest device workspace a call may use, 0 = no cap
  int coop = 0;             // device supports cooperative launches
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  size_t l2_bytes = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  std::complex<double>* h_draw = nullptr;  // pinned: the batched form's host draws (grown on demand)
  size_t h_draw_cap = 0;
  std::complex<double>* h_half[2] = {};    // pinned: the draws of each half of a large seeded batch
  size_t h_half_cap[2] = {};
  double* h_pinned = nullptr;  // cost read-back
  size_t h_pinned_n = 0;
};

namespace {

cudaEvent_t prof_event(qfs_ctx* ctx) {
  if (!ctx->prof.pool.empty()) {
    cudaEvent_t e = ctx->prof.pool.back();
    ctx->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Bracket one kernel launch; `bytes` is its algorithmic traffic.
struct ProfScope {
  qfs_ctx* ctx;
  int id;
  double bytes;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  // n: the launches the scope brackets (consecutive launches of one kind
  // can share one pair of events).
  ProfScope(qfs_ctx* c, int i, double b, cudaStream_t s = nullptr, int n = 1)
      : ctx(c), id(i), bytes(b), st(s ? s : c->stream) {
    ctx->prof.launches[id] += n;
    if (ctx->prof.on) {
      a = prof_event(ctx);
      record(a);
    }
  }
  // Inside stream capture only externally visible event records can be timed.
  void record(cudaEvent_t e) {
    if (ctx->prof.capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = prof_event(ctx);
      record(b);
      (ctx->prof.capturing ? ctx->prof.graph : ctx->prof.pending).push_back({a, b, id, bytes});
    }
  }
};

// After a synchronised replay of a captured graph: fold its timings in.
void prof_harvest_graph(qfs_ctx* ctx) {
  for (auto& r : ctx->prof.graph) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ctx->prof.ms[r.id] += ms;
      ctx->prof.timed[r.id] += 1;
      ctx->prof.bytes[r.id] += r.bytes;
    } else {
      cudaGetLastError();  // an untimed pair must not surface as a later error
    }
  }
}

void prof_release_graph(qfs_ctx* ctx) {
  for (auto& r : ctx->prof.graph) {
    ctx->prof.pool.push_back(r.a);
    ctx->prof.pool.push_back(r.b);
  }
  ctx->prof.graph.clear();
}

// After a stream synchronisation: fold finished timings into the totals.
void prof_harvest(qfs_ctx* ctx) {
  for (auto& r : ctx->prof.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ctx->prof.ms[r.id] += ms;
      ctx->prof.timed[r.id] += 1;
      ctx->prof.bytes[r.id] += r.bytes;
    } else {
      cudaGetLastError();
    }
    ctx->prof.pool.push_back(r.a);
    ctx->prof.pool.push_back(r.b);
  }
  ctx->prof.pending.clear();
}

// Sweeps queued per host round trip while no per-sweep host decision
// (plateau, validation) is needed: a launch behind a sweep that met the
// tolerance returns at once (device stop flag), so the run ends at the same
// sweep as with one launch per round trip.
constexpr int kSweepBatch = 4;

// Device buffers of one run, carved from the context's workspace.
struct Run {
  int n = 0, L = 0, M = 0, S = 0;
  int T = 1, spt = 1;      // target slots swept together and starts per slot (S = T * spt); start s
                           // belongs to slot s / spt, and U, Psi, Phi_L hold one copy per slot
  std::vector<const double2*> Uslot;  // the target of each slot (N x N, device)
  long long N = 0, sN = 0;
  std::vector<int> pairs;
  int prec = QFS_FP64;
  double beta = 0.0;
  Shape sh, sh64;          // sweep shape (prec) and the FP64 shape for S = 1
  int nblk_max = 1, nblk64_max = 1;  // largest backward block count (partials size)
  int groups = 1, group_size = 0;    // starts swept concurrently in `groups` slices
  // inputs (device)
  const double2* U = nullptr;  // N x N
  double2* U_copy = nullptr;   // used by the host-pointer entry points
  double2* psi64 = nullptr;
  double2* phil64 = nullptr;
  float2* psi32 = nullptr;
  float2* phil32 = nullptr;
  // state of the sweeps
  void* B = nullptr;    // (L-1) x S x N x M in the sweep precision
  void* phi = nullptr;  // S x N x M in the sweep precision
  double2* g64 = nullptr;
  float2* g32 = nullptr;
  double2* vprev = nullptr;  // right singular vectors of each gate's last update
  double* partials = nullptr;
  double* costs = nullptr;
  double* cost_rows = nullptr;   // kSweepBatch x S: the costs of each sweep of a batch
  int* active = nullptr;
  int* flag = nullptr;
  unsigned* counters = nullptr;  // S + 1 "last block done" counters (fused update)
  int* err = nullptr;            // device error word: bit 0 = a bounded device wait ran out
  double2* envs = nullptr;
  // FP64 single-start buffers (mixed precision: cost check and refinement)
  double2* B64r = nullptr;
  double2* phi64r = nullptr;
  double* partials64r = nullptr;
  double* cost64r = nullptr;
  // Validation states and U times them (double-and-restart), FP64.
  bool validate = false;
  double2* psi_val64 = nullptr;
  double2* phil_val64 = nullptr;
  int stream_b = 0;
  int stream_b64 = 0;
  // Dataflow sweep: step table (device), control words, partial sums.
  DfStep* df_steps = nullptr;
  unsigned* df_ctrl = nullptr;
  size_t df_ctrl_cap = 0;
  int df_slot = 0;              // control slot of the next sweep
  bool df_slot_zero = false;    // that slot is known to be zero (the previous sweep cleared it)
  double* df_partials = nullptr;
  double* df_resid = nullptr;
  int df_cap = 0;           // steps the table holds
  int df_max_nchunk = 0;    // largest chunks per start of any step
  int df_nsteps = 0;
  long long df_items = 0;
  double df_bytes = 0.0;    // algorithmic bytes of one dataflow sweep (all starts)
  const void* df_key[4] = {};  // what the uploaded table was built for
  int df_key_r = -1;
};

size_t elem_bytes(Real r) { return r == R32 ? sizeof(float2) : sizeof(double2); }

// Start count the launch shapes are computed for (see sweep()).
int shape_starts(int S_total) { return S_total >= 4 ? (S_total + 3) / 4 : S_total; }

// Lays out (or, with base == nullptr, only measures) the buffers of a run.
size_t carve(Run& R, char* base, bool need_U, bool need_envs) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const Real rs = R.prec == QFS_MIXED ? R32 : R64;
  const size_t es = elem_bytes(rs);
  const size_t state64 = (size_t)R.sN * sizeof(double2);
  R.U_copy = need_U ? (double2*)take((size_t)R.T * R.N * R.N * sizeof(double2)) : nullptr;
  R.psi64 = (double2*)take(R.T * state64);
  R.phil64 = (double2*)take(R.T * state64);
  if (R.prec == QFS_MIXED) {
    R.psi32 = (float2*)take((size_t)R.T * R.sN * sizeof(float2));
    R.phil32 = (float2*)take((size_t)R.T * R.sN * sizeof(float2));
  }
  R.B = take((size_t)std::max(R.L - 1, 1) * R.S * R.sN * es);
  R.phi = take((size_t)R.S * R.sN * es);
  R.g64 = (double2*)take((size_t)R.S * R.L * 16 * sizeof(double2));
  R.g32 = R.prec == QFS_MIXED ? (float2*)take((size_t)R.S * R.L * 16 * sizeof(float2)) : nullptr;
  R.vprev = (double2*)take((size_t)R.S * R.L * 16 * sizeof(double2));
  R.partials = (double*)take((size_t)R.S * R.nblk_max * 32 * sizeof(double));
  R.costs = (double*)take((size_t)R.S * sizeof(double));
  R.cost_rows = (double*)take((size_t)kSweepBatch * R.S * sizeof(double));
  R.active = (int*)take((size_t)R.S * sizeof(int));
  R.counters = (unsigned*)take((size_t)(R.S + 1) * sizeof(unsigned));
  R.flag = (int*)take(sizeof(int) * 4);
  R.err = R.flag ? R.flag + 1 : nullptr;
  R.envs = need_envs ? (double2*)take((size_t)R.S * R.L * 16 * sizeof(double2)) : nullptr;
  R.df_steps = (DfStep*)take((size_t)std::max(R.df_cap, 1) * sizeof(DfStep));
  R.df_ctrl_cap = 1 + ((size_t)R.df_cap + 1) * R.S;
  R.df_ctrl = (unsigned*)take(sizeof(unsigned) * 2 * R.df_ctrl_cap);  // two slots: this sweep's, the next's
  R.df_partials = (double*)take(sizeof(double) * 32 * (size_t)R.S * std::max(R.df_max_nchunk, 1));
  // The residual pass keeps its double partials apart: in complex64 the
  // environment partials are floats, and one start's residual slots would
  // overlap another start's environment slots while that start still sweeps.
  R.df_resid = (double*)take(sizeof(double) * 32 * (size_t)R.S * std::max(R.df_max_nchunk, 1));
  if (R.prec == QFS_MIXED || R.validate) {
    R.B64r = (double2*)take((size_t)std::max(R.L - 1, 2) * state64);
    R.phi64r = (double2*)take(state64);
    R.partials64r = (double*)take((size_t)R.nblk64_max * 32 * sizeof(double));
    R.cost64r = (double*)take(sizeof(double) * 2);
  }
  if (R.validate) {
    R.psi_val64 = (double2*)take(state64);
    R.phil_val64 = (double2*)take(state64);
  }
  return off;
}

int check_circuit(const qfs_circuit* c) {
  if (!c) return fail(QFS_EINVAL, "circuit is NULL");
  if (c->n < 2) return fail(QFS_EINVAL, "n = %d: need at least 2 qubits", c->n);
  if (c->n > QFS_MAX_QUBITS) return fail(QFS_EUNSUPPORTED, "n = %d > %d", c->n, QFS_MAX_QUBITS);
  if (c->L < 1) return fail(QFS_EINVAL, "L = %d: need at least one gate", c->L);
  if (!c->pairs) return fail(QFS_EINVAL, "pairs is NULL");
  for (int k = 0; k < c->L; ++k) {
    const int a = c->pairs[2 * k], b = c->pairs[2 * k + 1];
    if (a < 0 || b < 0 || a >= c->n || b >= c->n)
      return fail(QFS_EINVAL, "gate %d: qubit out of range (%d, %d) for n = %d", k, a, b, c->n);
    if (a == b) return fail(QFS_EINVAL, "gate %d: both qubits are %d", k, a);
  }
  return QFS_OK;
}

int check_run_params(int n, int M, int S, int max_sweeps, int precision, double beta, double tol) {
  if (M < 1 || (long long)M > (1LL << n))
    return fail(QFS_EINVAL, "M = %d: need 1 <= M <= 2^n = %lld", M, 1LL << n);
  if (S < 1) return fail(QFS_EINVAL, "multistarts = %d: need >= 1", S);
  if (S > 65535) return fail(QFS_EUNSUPPORTED, "multistarts = %d > 65535", S);
  if (max_sweeps < 1) return fail(QFS_EINVAL, "max_sweeps = %d: need >= 1", max_sweeps);
  if (precision != QFS_FP64 && precision != QFS_MIXED)
    return fail(QFS_EINVAL, "precision = %d: need QFS_FP64 or QFS_MIXED", precision);
  if (!(beta >= 0.0 && beta < 1.0)) return fail(QFS_EINVAL, "beta = %g: need 0 <= beta < 1", beta);
  if (!(tol >= 0.0) || std::isinf(tol)) return fail(QFS_EINVAL, "dist_tol = %g: need a finite value >= 0", tol);
  return QFS_OK;
}

int ensure_ws(qfs_ctx* ctx, size_t bytes) {
  if (ctx->ws_cap && bytes > ctx->ws_cap)
    return fail(QFS_ENOMEM, "this call needs %.3f GiB of device workspace, above the context's cap of %.3f GiB",
                bytes / 1073741824.0, ctx->ws_cap / 1073741824.0);
  if (ctx->ws_bytes >= bytes) return QFS_OK;
  if (ctx->ws) {
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaFree(ctx->ws));
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return fail(QFS_ENOMEM, "cannot allocate %.3f GiB of device workspace: %s",
                bytes / 1073741824.0, cudaGetErrorString(e));
  }
  ctx->ws_bytes = bytes;
  return QFS_OK;
}

int ensure_pinned(qfs_ctx* ctx, size_t n) {
  if (ctx->h_pinned_n >= n) return QFS_OK;
  if (ctx->h_pinned) CK(cudaFreeHost(ctx->h_pinned));
  ctx->h_pinned = nullptr;
  ctx->h_pinned_n = 0;
  CK(cudaMallocHost(&ctx->h_pinned, n * sizeof(double)));
  ctx->h_pinned_n = n;
  return QFS_OK;
}

// ---------------------------------------------------------------- dataflow

// Whether one sweep in precision r can run as a single dataflow launch.
bool df_usable(const qfs_ctx* ctx, const Run& R, Real r) {
  return ctx->dataflow && ctx->coop && (r == R64 || R.M % 2 == 0) && df_blocks_per_sm(r) > 0;
}

// The step table of one sweep (the same steps, in the same order, as
// sweep()), chunked so that each step offers about two items per resident
// CTA.  With null buffers in R it only sizes the table.
void df_build(const qfs_ctx* ctx, const Run& R, Real r, const void* psi, const void* phil, double2* envs,
              const int* active, double2* vprev, std::vector<DfStep>& steps, double* bytes) {
  steps.clear();
  *bytes = 0.0;
  const size_t es = elem_bytes(r);
  const int vec = r == R32 ? 2 : 1;
  const long long sN = R.sN;
  const int L = R.L, S = R.S, n = R.n, M = R.M;
  const long long gstride = (long long)L * 16;
  const char* gT = r == R32 ? reinterpret_cast<const char*>(R.g32) : reinterpret_cast<const char*>(R.g64);
  auto gate_ptr = [&](int idx) -> const void* { return gT ? gT + (size_t)idx * 16 * es : nullptr; };
  auto B_ptr = [&](int k) -> void* {
    return R.B ? (void*)((char*)R.B + (size_t)(k - 1) * S * sN * es) : nullptr;
  };
  const double resident = (double)std::max(1, df_blocks_per_sm(r)) * std::max(1, ctx->num_sms);
  // Items per CTA and step: forward steps have no update on the chain, so
  // fewer, larger items pay off; backward steps keep more, smaller items so
  // that a start's chunks finish sooner and its update starts earlier.
  // Chunks are sized from one target's starts, so a start's items (and its
  // sums) are the same whether it sweeps alone or beside other targets.
  auto chunk_it = [&](DfStep& st, double bytes_per_unit) {
    const double step_bytes = bytes_per_unit * st.units * R.spt;
    const bool fwd = st.kind == DF_FWD || st.kind == DF_FWD2;
    const double per_cta = fwd ? ctx->df_items_per_cta_fwd : ctx->df_items_per_cta;
    const double target = std::min(ctx->df_item_bytes, std::max(16.0 * 1024.0, step_bytes / (per_cta * resident)));
    df_chunking(st, bytes_per_unit, target);
    *bytes += bytes_per_unit * st.units * S;
  };
  // Forward: gates k and k+1 on four distinct qubits go in one step (B_k is
  // then written but not read back), others one at a time.
  for (int k = 1; k <= L - 1;) {
    DfStep st{};
    st.in = k == 1 ? psi : B_ptr(k - 1);
    st.in_stride = k == 1 ? 0 : sN;
    st.in_gstride = k == 1 ? sN : 0;
    st.out = B_ptr(k);
    st.gate = gate_ptr(k - 1);
    st.gate_stride = gstride;
    const int a1 = R.pairs[2 * (k - 1)], b1 = R.pairs[2 * (k - 1) + 1];
    bool two = ctx->df_fwd2 && k + 1 <= L - 1;
    if (two) {
      const int a2 = R.pairs[2 * k], b2 = R.pairs[2 * k + 1];
      two = a2 != a1 && a2 != b1 && b2 != a1 && b2 != b1;
      if (two) st.bg = make_bwd_geom(n, M, a1, b1, a2, b2);
    }
    if (two) {
      st.kind = DF_FWD2;
      st.out2 = B_ptr(k + 1);
      st.gate2 = gate_ptr(k);
      st.units = (1 << (n - 4)) * (M / vec);
      chunk_it(st, 16.0 * vec * es * 3.0);
      k += 2;
    } else {
      st.kind = DF_FWD;
      st.fg = make_geom(n, M, a1, b1);
      st.units = (1 << (n - 2)) * (M / vec);
      chunk_it(st, 4.0 * vec * es * 2.0);
      k += 1;
    }
    steps.push_back(st);
  }
  for (int k = L; k >= 1; --k) {
    DfStep st{};
    const int qa = R.pairs[2 * (k - 1)], qb = R.pairs[2 * (k - 1) + 1];
    int ua = qa, ub = qb;
    st.in = k == 1 ? psi : B_ptr(k - 1);
    st.in_stride = k == 1 ? 0 : sN;
    st.in_gstride = k == 1 ? sN : 0;
    if (k == L) {
      st.phi_in = phil;
      st.phi_in_stride = 0;
      st.phi_in_gstride = sN;
      st.phi_out = nullptr;
      st.gate = nullptr;
    } else {
      st.phi_in = k == L - 1 ? phil : R.phi;
      st.phi_in_stride = k == L - 1 ? 0 : sN;
      st.phi_in_gstride = k == L - 1 ? sN : 0;
      st.phi_out = R.phi;
      st.gate = gate_ptr(k);
      ua = R.pairs[2 * k];
      ub = R.pairs[2 * k + 1];
    }
    st.gate_stride = gstride;
    st.bg = make_bwd_geom(n, M, ua, ub, qa, qb);
    const int U = st.bg.U, ea = st.bg.ea, eb = st.bg.eb;
    int v = vec;
    if (U == 4) st.kind = DF_BWD4;
    else if (U == 2) st.kind = ea == 1 ? DF_BWD2_10 : DF_BWD2_01;
    else {
      v = 1;
      st.kind = ea == 2 ? DF_BWD3_20 : eb == 2 ? DF_BWD3_02 : ea == 1 ? DF_BWD3_10 : DF_BWD3_01;
    }
    st.units = (1 << (n - U)) * (M / v);
    // Phi_k is stored by every backward step but the first (k = L).
    chunk_it(st, (double)(1 << U) * v * es * (k < L ? 3.0 : 2.0));
    UpdateArgs& u = st.upd;
    u.partials = R.df_partials;
    u.nblk = st.nchunk;  // (the dataflow kernel sums the chunk slots itself)
    u.partials_f32 = r == R32;
    u.g64 = R.g64 ? R.g64 + (size_t)(k - 1) * 16 : nullptr;
    u.g_stride = gstride;
    u.g32 = R.g32 ? R.g32 + (size_t)(k - 1) * 16 : nullptr;
    u.beta = R.beta;
    // Gate 1's update leaves 2 - (2/M) Re Tr(g_1 E_1): the cost of FP64
    // sweeps, and the estimate that lets complex64 sweeps skip the residual.
    u.cost_out = k == 1 ? R.costs : nullptr;
    u.inv_M = 1.0 / M;
    u.env_out = envs ? envs + (size_t)(k - 1) * 16 : nullptr;
    u.env_stride = gstride;
    u.S = S;
    u.active = active;
    u.vprev = vprev ? vprev + (size_t)(k - 1) * 16 : nullptr;
    steps.push_back(st);
  }
  if (r == R32) {
    DfStep st{};
    st.kind = DF_RESID;
    st.in = psi;
    st.in_stride = 0;
    st.in_gstride = sN;
    st.phi_in = L == 1 ? phil : R.phi;
    st.phi_in_stride = L == 1 ? 0 : sN;
    st.phi_in_gstride = L == 1 ? sN : 0;
    st.phi_out = nullptr;
    st.gate = gate_ptr(0);
    st.gate_stride = gstride;
    st.bg = make_bwd_geom(n, M, R.pairs[0], R.pairs[1], R.pairs[0], R.pairs[1]);
    st.units = (1 << (n - 2)) * (M / vec);
    chunk_it(st, 4.0 * vec * es * 2.0);
    steps.push_back(st);
  }
  long long item = 0;
  for (DfStep& st : steps) {
    st.spt = std::max(R.spt, 1);
    st.item0 = item;
    item += (long long)S * st.nchunk;
  }
}

int prepare(qfs_ctx* ctx, Run& R, const qfs_circuit* c, int M, int S_target, int prec, double beta,
            bool need_U, bool need_envs, int groups = 1, bool validate = false, int T = 1) {
  R.validate = validate;
  R.n = c->n;
  R.L = c->L;
  R.M = M;
  R.T = T;
  R.spt = S_target;
  const int S = T * S_target;
  R.S = S;
  R.N = 1LL << c->n;
  R.sN = (long long)M << c->n;
  R.pairs.assign(c->pairs, c->pairs + 2 * c->L);
  R.prec = prec;
  R.beta = beta;
  R.sh = make_shape(R.n, M, S, prec == QFS_MIXED ? R32 : R64, ctx->num_sms);
  R.sh64 = make_shape(R.n, M, 1, R64, ctx->num_sms);
  R.groups = std::max(1, std::min({groups, S, kMaxGroups}));
  R.group_size = (S + R.groups - 1) / R.groups;
  R.groups = (S + R.group_size - 1) / R.group_size;
  R.nblk_max = R.nblk64_max = 1;
  for (int U = 2; U <= std::min(4, R.n); ++U) {
    const Real rs = prec == QFS_MIXED ? R32 : R64;
    R.nblk_max = std::max(R.nblk_max, make_bwd_shape(R.n, M, shape_starts(S), rs, ctx->num_sms, U).nblk);
    R.nblk64_max = std::max(R.nblk64_max, make_bwd_shape(R.n, M, 1, R64, ctx->num_sms, U).nblk);
  }
  R.df_cap = 0;
  R.df_max_nchunk = 0;
  R.df_key_r = -1;
  {
    const Real rs = prec == QFS_MIXED ? R32 : R64;
    if (df_usable(ctx, R, rs)) {
      std::vector<DfStep> steps;
      double b = 0.0;
      df_build(ctx, R, rs, nullptr, nullptr, nullptr, nullptr, nullptr, steps, &b);
      R.df_cap = (int)steps.size();
      for (const DfStep& st : steps) R.df_max_nchunk = std::max(R.df_max_nchunk, st.nchunk);
    }
  }
  const size_t bytes = carve(R, nullptr, need_U, need_envs);
  TRY(ensure_ws(ctx, bytes));
  carve(R, ctx->ws, need_U, need_envs);
  const size_t blist = (size_t)std::max(R.L - 1, 1) * S * R.sN * elem_bytes(prec == QFS_MIXED ? R32 : R64);
  R.stream_b = blist > ctx->l2_bytes / 2;
  R.stream_b64 = (size_t)std::max(R.L - 1, 1) * R.sN * sizeof(double2) > ctx->l2_bytes / 2;
  TRY(ensure_pinned(ctx, (size_t)kSweepBatch * S + 8));
  return QFS_OK;
}

// Phi_L = U Psi (Sec. 3, the A tensor).  QFS_FP64 runs take the FP64
// product; mixed runs the FP32 pair-arithmetic product (about 48 bits, far
// below what the FP64 cost check at dist_tol resolves), with the B list,
// not in use before the first sweep, as its scratch.  Returns the launches.
int target_product(qfs_ctx* ctx, Run& R, const double2* U, const double2* psi, double2* out) {
  cudaStream_t st = ctx->stream;
  const size_t bbytes = (size_t)std::max(R.L - 1, 1) * R.S * R.sN * elem_bytes(R.prec == QFS_MIXED ? R32 : R64);
  const size_t split_bytes = align_up((size_t)R.sN * sizeof(float4));
  if (R.prec == QFS_MIXED && !ctx->upsi_fp64 && bbytes >= 2 * split_bytes) {
    const int splits = upsi_pair_splits((int)R.N, R.M, ctx->num_sms, bbytes - split_bytes);
    float4* ps = reinterpret_cast<float4*>(R.B);
    double2* scratch = reinterpret_cast<double2*>(static_cast<char*>(R.B) + split_bytes);
    launch_gemm_upsi_pair(U, psi, out, (int)R.N, R.M, ps, scratch, splits, ctx->num_sms, st);
    return splits > 1 ? 3 : 2;
  }
  launch_gemm_upsi(U, psi, out, (int)R.N, R.M, st);
  return 1;
}

// Phi_L = U Psi, complex64 copies for the mixed sweeps, gate copies.
// Inputs of slot t, whose target U (R.Uslot[t]), training states
// (R.psi64 + t sN) and initial gates (its starts' rows of R.g64) are in
// place: input checks, Phi_L = U Psi, the complex64 copies, the warm starts
// and the slot's starts active.
int setup_slot(qfs_ctx* ctx, Run& R, int t) {
  cudaStream_t st = ctx->stream;
  const size_t so = (size_t)t * R.sN, go = (size_t)t * R.spt * R.L * 16;
  CK(cudaMemsetAsync(R.flag, 0, sizeof(int), st));
  {
    ProfScope ps(ctx, QFS_PROF_OTHER, 0.0);
    launch_nonfinite_check(reinterpret_cast<const double*>(R.Uslot[t]), 2 * R.N * R.N, R.flag, st);
  }
  {
    ProfScope ps(ctx, QFS_PROF_OTHER, 0.0);
    launch_nonfinite_check(reinterpret_cast<const double*>(R.psi64 + so), 2 * R.sN, R.flag, st);
  }
  {
    ProfScope ps(ctx, QFS_PROF_OTHER, 0.0);
    launch_nonfinite_check(reinterpret_cast<const double*>(R.g64 + go), 2LL * R.spt * R.L * 16, R.flag, st);
  }
  {
    ProfScope ps(ctx, QFS_PROF_GEMM, 8.0 * R.N * R.N * R.M);  // flops, not bytes
    ctx->prof.launches[QFS_PROF_GEMM] += target_product(ctx, R, R.Uslot[t], R.psi64 + so, R.phil64 + so) - 1;
  }
  if (R.prec == QFS_MIXED) {
    ProfScope ps(ctx, QFS_PROF_OTHER, 0.0);
    launch_cast_c128_to_c64(R.psi64 + so, R.psi32 + so, R.sN, st);
    launch_cast_c128_to_c64(R.phil64 + so, R.phil32 + so, R.sN, st);
    launch_cast_c128_to_c64(R.g64 + go, R.g32 + go, (long long)R.spt * R.L * 16, st);
    ctx->prof.launches[QFS_PROF_OTHER] += 2;
  }
  std::vector<int> ones(R.spt, 1);
  CK(cudaMemcpyAsync(R.active + (size_t)t * R.spt, ones.data(), sizeof(int) * R.spt, cudaMemcpyHostToDevice, st));
  {
    ProfScope ps(ctx, QFS_PROF_OTHER, 0.0);
    launch_set_identity4(R.vprev + go, (long long)R.spt * R.L, st);
  }
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, R.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  prof_harvest(ctx);
  if (flag) return fail(QFS_ENONFINITE, "NaN or Inf in the target, samples or initial gates");
  return QFS_OK;
}

int setup_inputs(qfs_ctx* ctx, Run& R) {
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(R.flag, 0, sizeof(int) * 4, st));
  CK(cudaMemsetAsync(R.counters, 0, sizeof(unsigned) * (R.S + 1), st));
  if ((int)R.Uslot.size() != R.T) R.Uslot.assign(R.T, R.U);
  for (int t = 0; t < R.T; ++t) TRY(setup_slot(ctx, R, t));
  return QFS_OK;
}

// One sweep (Section 3) for S starts in precision r.  Forward: B_k = g_k
// B_{k-1}, k = 1..L-1, with the current gates.  Backward, k = L..1: Phi_k =
// g_{k+1}^dagger Phi_{k+1} fused with the environment partials of gate k
// from B_{k-1} and Phi_k, then the warp update of gate k.  FP64 writes
// cost = 2 - (2/M) Re Tr(g_1 E_1); complex64 adds a residual pass
// (1/M) sum |g_1^dagger Phi_1 - Psi|^2 = (1/M) sum_j ||U psi_j - C psi_j||^2.
// A group of starts swept together on one stream: starts s0 .. s0+S-1 of a
// run with S_total starts (the B list is laid out [k][S_total][N*M]).
struct Slice {
  int s0 = 0;
  int S = 0;
  int S_total = 0;
  cudaStream_t st = nullptr;
};

// Returns QFS_EINTERNAL, before any launch, if a backward step's blocks
// would outnumber the nblk_stride partial-sum slots each start owns.
int sweep(qfs_ctx* ctx, Run& R, Real r, const Slice& sl, double2* g64, float2* g32,
          const void* psi, const void* phil, void* B, void* phi, double* partials,
          int nblk_stride, double* cost_out, double2* envs, const int* active, int stream_b,
          double2* vprev, unsigned* counters) {
  cudaStream_t st = sl.st ? sl.st : ctx->stream;
  const int S = sl.S, s0 = sl.s0;
  const size_t es = elem_bytes(r);
  const long long sN = R.sN;
  const long long gstride = (long long)R.L * 16;
  const size_t goff = (size_t)s0 * R.L * 16;
  g64 += goff;
  if (g32) g32 += goff;
  if (vprev) vprev += goff;
  if (envs) envs += goff;
  if (cost_out) cost_out += s0;
  if (active) active += s0;
  counters += s0;
  phi = (char*)phi + (size_t)s0 * sN * es;
  partials += (size_t)s0 * nblk_stride * 32;
  // Shapes follow a fixed share of the run's starts (a quarter, the size of
  // the library's largest concurrent group) so that the reduction order, and
  // hence every result bit, does not depend on the grouping, while a group
  // of that size still fills a wave.
  const int S_shape = shape_starts(sl.S_total);
  const Shape sh = make_shape(R.n, R.M, S_shape, r, ctx->num_sms);
  const char* gT = r == R32 ? reinterpret_cast<const char*>(g32) : reinterpret_cast<const char*>(g64);
  auto gate_ptr = [&](int idx) { return (const void*)(gT + (size_t)idx * 16 * es); };
  auto B_ptr = [&](int k) {  // B_k, k >= 1
    return (void*)((char*)B + ((size_t)(k - 1) * sl.S_total + s0) * sN * es);
  };
  const int L = R.L;
  for (int k = L; k >= 1; --k) {
    const int ua = k == L ? R.pairs[2 * (k - 1)] : R.pairs[2 * k];
    const int ub = k == L ? R.pairs[2 * (k - 1) + 1] : R.pairs[2 * k + 1];
    const BwdGeom bg = make_bwd_geom(R.n, R.M, ua, ub, R.pairs[2 * (k - 1)], R.pairs[2 * (k - 1) + 1]);
    const int nb = make_bwd_shape(R.n, R.M, S_shape, r, ctx->num_sms, bg.U).nblk;
    if (nb > nblk_stride)
      return fail(QFS_EINTERNAL, "backward step %d needs %d partial-sum slots per start, %d allocated", k, nb,
                  nblk_stride);
  }
  if (r == R32 && make_bwd_shape(R.n, R.M, S_shape, r, ctx->num_sms, 2).nblk > nblk_stride)
    return fail(QFS_EINTERNAL, "the residual pass needs more partial-sum slots than allocated");
  for (int k = 1; k <= L - 1; ++k) {
    const Geom gm = make_geom(R.n, R.M, R.pairs[2 * (k - 1)], R.pairs[2 * (k - 1) + 1]);
    const void* in = k == 1 ? psi : B_ptr(k - 1);
    ProfScope ps(ctx, QFS_PROF_FORWARD, 2.0 * S * sN * es, st);
    launch_forward(r, gm, sh, S, in, k == 1 ? 0 : sN, B_ptr(k), gate_ptr(k - 1), gstride, active, st);
  }
  for (int k = L; k >= 1; --k) {
    const int qa = R.pairs[2 * (k - 1)], qb = R.pairs[2 * (k - 1) + 1];
    const void* bprev = k == 1 ? psi : B_ptr(k - 1);
    const long long bstride = k == 1 ? 0 : sN;
    const void* pin;
    long long pstride;
    void* pout;
    const void* gate;
    int ua = qa, ub = qb;  // pair of the gate carried into Phi (gate k+1)
    if (k == L) {
      pin = phil; pstride = 0; pout = nullptr; gate = nullptr;
    } else {
      pin = k == L - 1 ? phil : phi;
      pstride = k == L - 1 ? 0 : sN;
      pout = phi;
      gate = gate_ptr(k);
      ua = R.pairs[2 * k];
      ub = R.pairs[2 * k + 1];
    }
    const BwdGeom bg = make_bwd_geom(R.n, R.M, ua, ub, qa, qb);
    const Shape bsh = make_bwd_shape(R.n, R.M, S_shape, r, ctx->num_sms, bg.U);
    UpdateArgs ua_{};
    ua_.partials = partials;
    ua_.nblk = bsh.nblk;
    ua_.partials_f32 = r == R32;
    ua_.g64 = g64 + (size_t)(k - 1) * 16;
    ua_.g_stride = gstride;
    ua_.g32 = g32 ? g32 + (size_t)(k - 1) * 16 : nullptr;
    ua_.beta = R.beta;
    ua_.cost_out = (k == 1 && r == R64) ? cost_out : nullptr;
    ua_.inv_M = 1.0 / R.M;
    ua_.env_out = envs ? envs + (size_t)(k - 1) * 16 : nullptr;
    ua_.env_stride = gstride;
    ua_.S = S;
    ua_.active = active;
    ua_.vprev = vprev ? vprev + (size_t)(k - 1) * 16 : nullptr;
    // By default the backward step and the update of gate k run as one
    // launch: the last block of each start to finish performs its update.
    {
      ProfScope ps(ctx, QFS_PROF_BACKWARD, (double)S * sN * es * (pout ? 3.0 : 2.0), st);
      launch_backward(r, 0, bg, bsh, S, bprev, bstride, pin, pstride, pout, gate, gstride, partials, stream_b,
                      active, st, ctx->fuse_update ? &ua_ : nullptr, counters);
    }
    if (!ctx->fuse_update) {
      ProfScope ps(ctx, QFS_PROF_UPDATE, (double)S * bsh.nblk * 32 * sizeof(double), st);
      launch_update(ua_, st);
    }
  }
  if (r == R32) {
    const BwdGeom bg = make_bwd_geom(R.n, R.M, R.pairs[0], R.pairs[1], R.pairs[0], R.pairs[1]);
    const Shape bsh = make_bwd_shape(R.n, R.M, S_shape, r, ctx->num_sms, 2);
    const void* pin = L == 1 ? phil : phi;
    {
      ProfScope ps(ctx, QFS_PROF_RESIDUAL, 2.0 * S * sN * es, st);
      launch_backward(r, 1, bg, bsh, S, psi, 0, pin, L == 1 ? 0 : sN, nullptr, gate_ptr(0), gstride,
                      partials, 0, active, st);
    }
    ProfScope ps(ctx, QFS_PROF_OTHER, 0.0, st);
    launch_residual_finish(partials, bsh.nblk, S, 1.0 / R.M, cost_out, st);
  }
  return QFS_OK;
}

// One sweep of all starts of R as one dataflow launch (same results as
// sweep() up to the order of the reduction sums).  The step table is built
// and uploaded once per (precision, outputs) and reused by later sweeps.
int df_sweep(qfs_ctx* ctx, Run& R, Real r, const void* psi, const void* phil, double2* envs, const int* active,
             double2* vprev, cudaStream_t st, int* stop = nullptr, double stop_tol = 0.0,
             double* cost_row = nullptr, double resid_skip = 0.0) {
  const void* key[4] = {psi, envs, active, vprev};
  if (R.df_key_r != (int)r || std::memcmp(key, R.df_key, sizeof(key)) != 0) {
    std::vector<DfStep> steps;
    double bytes = 0.0;
    df_build(ctx, R, r, psi, phil, envs, active, vprev, steps, &bytes);
    int mx = 0;
    for (const DfStep& s : steps) mx = std::max(mx, s.nchunk);
    if ((int)steps.size() > R.df_cap || mx > R.df_max_nchunk)
      return fail(QFS_EUNSUPPORTED, "dataflow table does not fit its buffers (%d steps, %d chunks)",
                  (int)steps.size(), mx);
    CK(cudaMemcpyAsync(R.df_steps, steps.data(), sizeof(DfStep) * steps.size(), cudaMemcpyHostToDevice, st));
    R.df_nsteps = (int)steps.size();
    R.df_items = steps.back().item0 + (long long)R.S * steps.back().nchunk;
    R.df_bytes = bytes;
    std::memcpy(R.df_key, key, sizeof(key));
    R.df_key_r = (int)r;
  }
  // Control words (queue, chunk counts, published steps) alternate between
  // two slots; each sweep clears the slot of the next one at its entry.
  unsigned* ctrl = R.df_ctrl + (size_t)R.df_slot * R.df_ctrl_cap;
  unsigned* next = R.df_ctrl + (size_t)(R.df_slot ^ 1) * R.df_ctrl_cap;
  if (!R.df_slot_zero) CK(cudaMemsetAsync(ctrl, 0, sizeof(unsigned) * R.df_ctrl_cap, st));
  DfArgs a{};
  a.steps = R.df_steps;
  a.nsteps = R.df_nsteps;
  a.S = R.S;
  a.total_items = R.df_items;
  a.active = active;
  a.queue = ctrl;
  a.chunk_cnt = ctrl + 1;
  a.done = ctrl + 1 + (size_t)R.df_nsteps * R.S;
  a.zero_next = next;
  a.zero_count = (int)R.df_ctrl_cap;
  a.cost_row = cost_row;
  a.err = R.err;
  a.wait_limit = ctx->df_wait_limit;
  a.partials = R.df_partials;
  a.resid_partials = R.df_resid;
  a.part_stride = R.df_max_nchunk;
  a.resid_cost = R.costs;
  a.inv_M = 1.0 / R.M;
  a.stop = stop;
  a.stop_tol = stop_tol;
  a.stop_from_update = r == R64 ? 1 : 0;
  a.resid_skip = r == R32 ? resid_skip : 0.0;
  const size_t nstep_stamps = (size_t)R.df_nsteps * R.S * 4;
  a.trace = ctx->df_trace && ctx->df_trace_n >= nstep_stamps ? ctx->df_trace : nullptr;
  a.item_trace = a.trace && ctx->df_trace_n >= nstep_stamps + (size_t)R.df_items * 4 ? a.trace + nstep_stamps : nullptr;
  if (a.trace) {
    ctx->df_trace_steps = R.df_nsteps;
    ctx->df_trace_S = R.S;
    ctx->df_trace_items = a.item_trace ? R.df_items : 0;
  }
  ProfScope ps(ctx, QFS_PROF_DATAFLOW, R.df_bytes, st);
  R.df_slot_zero = false;
  CK(launch_sweep_df(r, a, ctx->num_sms, st));
  R.df_slot ^= 1;
  R.df_slot_zero = true;
  return QFS_OK;
}

// FP64 sample cost of start s's master gates on states psi with
// phil = U psi: (1/M) ||phil - C psi||^2 (the training states by default).
int check64(qfs_ctx* ctx, Run& R, int s, double* out, const double2* psi = nullptr,
            const double2* phil = nullptr) {
  cudaStream_t st = ctx->stream;
  const double2* g = R.g64 + (size_t)s * R.L * 16;
  if (!psi) psi = R.psi64 + (size_t)(s / R.spt) * R.sN;
  if (!phil) phil = R.phil64 + (size_t)(s / R.spt) * R.sN;
  const void* in = psi;
  for (int k = 1; k <= R.L; ++k) {
    const Geom gm = make_geom(R.n, R.M, R.pairs[2 * (k - 1)], R.pairs[2 * (k - 1) + 1]);
    double2* out_buf = R.B64r + (size_t)(k & 1) * R.sN;
    ProfScope ps(ctx, QFS_PROF_CHECK, 2.0 * R.sN * sizeof(double2));
    launch_forward(R64, gm, R.sh64, 1, in, 0, out_buf, g + (size_t)(k - 1) * 16, 16, nullptr, st);
    in = out_buf;
  }
  const BwdGeom bg = make_bwd_geom(R.n, R.M, R.pairs[0], R.pairs[1], R.pairs[0], R.pairs[1]);
  {
    ProfScope ps(ctx, QFS_PROF_CHECK, 2.0 * R.sN * sizeof(double2));
    launch_backward(R64, 1, bg, R.sh64, 1, in, 0, phil, 0, nullptr, nullptr, 16, R.partials64r,
                    0, nullptr, st);
  }
  {
    ProfScope ps(ctx, QFS_PROF_OTHER, 0.0);
    launch_residual_finish(R.partials64r, R.sh64.nblk, 1, 1.0 / R.M, R.cost64r, st);
  }
  CK(cudaMemcpyAsync(ctx->h_pinned, R.cost64r, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  prof_harvest(ctx);
  *out = ctx->h_pinned[0];
  return QFS_OK;
}

int read_costs(qfs_ctx* ctx, const double* dev, int S, std::vector<double>& out,
               const int* err = nullptr) {
  CK(cudaMemcpyAsync(ctx->h_pinned, dev, sizeof(double) * S, cudaMemcpyDeviceToHost, ctx->stream));
  if (err)
    CK(cudaMemcpyAsync(ctx->h_pinned + S, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  prof_harvest(ctx);
  out.assign(ctx->h_pinned, ctx->h_pinned + S);
  if (err) {
    int e;
    std::memcpy(&e, ctx->h_pinned + S, sizeof(int));
    if (e) return fail(QFS_ETIMEOUT, "a bounded device wait ran out (error word %d)", e);
  }
  return QFS_OK;
}

// The cost rows of a batch of B sweeps and the error word, without folding
// the profile (the caller first drops the launches that found the stop flag).
int read_rows(qfs_ctx* ctx, const double* dev, int S, int B, std::vector<std::vector<double>>& rows,
              const int* err) {
  CK(cudaMemcpyAsync(ctx->h_pinned, dev, sizeof(double) * S * B, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_pinned + (size_t)S * B, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  rows.assign(B, std::vector<double>());
  for (int b = 0; b < B; ++b) rows[b].assign(ctx->h_pinned + (size_t)b * S, ctx->h_pinned + (size_t)(b + 1) * S);
  int e;
  std::memcpy(&e, ctx->h_pinned + (size_t)S * B, sizeof(int));
  if (e) return fail(QFS_ETIMEOUT, "a bounded device wait ran out (error word %d)", e);
  return QFS_OK;
}

// Forget the last k dataflow launches of the profile (launches that
// returned at once on the stop flag did no work).
void prof_drop_dataflow(qfs_ctx* ctx, int k) {
  ctx->prof.launches[QFS_PROF_DATAFLOW] -= k;
  for (int i = (int)ctx->prof.pending.size() - 1; i >= 0 && k > 0; --i) {
    if (ctx->prof.pending[i].id != QFS_PROF_DATAFLOW) continue;
    ctx->prof.pool.push_back(ctx->prof.pending[i].a);
    ctx->prof.pool.push_back(ctx->prof.pending[i].b);
    ctx->prof.pending.erase(ctx->prof.pending.begin() + i);
    --k;
  }
}

int ensure_group_streams(qfs_ctx* ctx, int groups) {
  if (!ctx->fork_event) CK(cudaEventCreateWithFlags(&ctx->fork_event, cudaEventDisableTiming));
  for (int g = 0; g < groups; ++g) {
    if (!ctx->gstream[g]) CK(cudaStreamCreateWithFlags(&ctx->gstream[g], cudaStreamNonBlocking));
    if (!ctx->gevent[g]) CK(cudaEventCreateWithFlags(&ctx->gevent[g], cudaEventDisableTiming));
  }
  return QFS_OK;
}

// One sweep of every start: the run's starts are split into R.groups slices
// swept concurrently on their own streams (one slice's SVD updates overlap
// the others' streaming), forked from and joined back to ctx->stream.
int sweep_all(qfs_ctx* ctx, Run& R, Real rs, const void* psi, const void* phil, cudaStream_t origin) {
  if (R.groups <= 1)
    return sweep(ctx, R, rs, Slice{0, R.S, R.S, origin}, R.g64, R.g32, psi, phil, R.B, R.phi, R.partials,
                 R.nblk_max, R.costs, nullptr, R.active, R.stream_b, R.vprev, R.counters);
  TRY(ensure_group_streams(ctx, R.groups));
  CK(cudaEventRecord(ctx->fork_event, origin));
  for (int g = 0; g < R.groups; ++g) {
    const int s0 = g * R.group_size;
    const int Sg = std::min(R.group_size, R.S - s0);
    CK(cudaStreamWaitEvent(ctx->gstream[g], ctx->fork_event, 0));
    TRY(sweep(ctx, R, rs, Slice{s0, Sg, R.S, ctx->gstream[g]}, R.g64, R.g32, psi, phil, R.B, R.phi,
              R.partials, R.nblk_max, R.costs, nullptr, R.active, R.stream_b, R.vprev, R.counters));
    CK(cudaEventRecord(ctx->gevent[g], ctx->gstream[g]));
    CK(cudaStreamWaitEvent(origin, ctx->gevent[g], 0));
  }
  return QFS_OK;
}

// One sweep of all starts as a CUDA graph (captured once per run, replayed
// every sweep): a single launch per sweep instead of ~3L per group.
struct SweepGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  qfs_ctx* ctx = nullptr;
  long long launches[QFS_PROF_KINDS] = {};  // kernel launches per replay
  ~SweepGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ctx) prof_release_graph(ctx);
  }
};

int capture_sweep(qfs_ctx* ctx, Run& R, Real rs, const void* psi, const void* phil, SweepGraph& g) {
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  g.ctx = ctx;
  long long before[QFS_PROF_KINDS];
  for (int i = 0; i < QFS_PROF_KINDS; ++i) before[i] = ctx->prof.launches[i];
  CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
  ctx->prof.capturing = true;
  const int rc = sweep_all(ctx, R, rs, psi, phil, ctx->cap_stream);
  ctx->prof.capturing = false;
  // Captured launches run at each replay, not now.
  for (int i = 0; i < QFS_PROF_KINDS; ++i) {
    g.launches[i] = ctx->prof.launches[i] - before[i];
    ctx->prof.launches[i] = before[i];
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
  if (rc != QFS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  CK(e);
  g.graph = graph;
  CK(cudaGraphInstantiate(&g.exec, graph, 0));
  return QFS_OK;
}

struct Outcome {
  int best = 0;
  double cost = std::numeric_limits<double>::infinity();
  int sweeps = 0;
  int converged = 0;
  int fp64_sweeps = 0;
  std::vector<double> start_costs;
  bool overtrained = false;  // the validation check halted the run (double-and-restart)
  double c_val = std::numeric_limits<double>::quiet_NaN();
};

// The multistart run.  Starts sweep in lock step; the run stops at the first
// sweep after which some start's cost is <= tol and returns the lowest-cost
// start of that sweep (lowest index on ties).  With plateau_window > 0 a
// start stops once its cost failed plateau_window times in a row to improve
// by diff_tol_r relative to the newer cost (Appendix A) after min_sweeps.
// The multistart run of every slot.  A slot's starts sweep in lock step with
// every other slot's; the slot's target is finished at the first sweep after
// which one of its starts has cost <= tol (FP64-confirmed), when all its
// starts stopped on a plateau, when the validation check halts it, or after
// max_sweeps of its own sweeps.  finish(slot, outcome) then receives the
// lowest-cost start (lowest index on ties) and returns true when it loaded a
// new target into the slot (its starts begin afresh) or false to leave the
// slot idle.  The run ends when every slot is idle.
int run_multistart(qfs_ctx* ctx, Run& R, const qfs_params* p,
                   const std::function<int(int, const Outcome&, bool&)>& finish) {
  cudaStream_t st = ctx->stream;
  const int S = R.S, T = R.T, spt = R.spt;
  const double tol = p->dist_tol;
  // Complex64 cost at which a start is handed to FP64 (checked, and refined
  // if the check is above tol): tol, or the larger refine_switch_tol.
  const double ctol = R.prec == QFS_MIXED ? std::max(tol, p->refine_switch_tol) : tol;
  const double inf = std::numeric_limits<double>::infinity(), nan = std::numeric_limits<double>::quiet_NaN();
  std::vector<double> c, prev(S, inf);
  std::vector<int> stall(S, 0), act(S, 1);
  std::vector<double> c64(S, nan);
  const Real rs = R.prec == QFS_MIXED ? R32 : R64;
  const void* psi = rs == R32 ? (const void*)R.psi32 : (const void*)R.psi64;
  const void* phil = rs == R32 ? (const void*)R.phil32 : (const void*)R.phil64;
  // Per slot: busy (a target is sweeping), its sweeps, FP64 refinement
  // sweeps, validation outcome.
  std::vector<char> busy(T, 1);
  std::vector<int> tsweeps(T, 0), tfp64(T, 0);
  std::vector<Outcome> cur(T);
  int left = T;
  SweepGraph graph;
  const bool df = df_usable(ctx, R, rs);
  if (!df) TRY(capture_sweep(ctx, R, rs, psi, phil, graph));
  // Without plateau detection or validation the host decides nothing until
  // some start meets the tolerance, so sweeps go out in batches.
  const bool batch = df && p->plateau_window == 0 && !R.validate;
  int* stop = R.flag + 2;
  // Complex64 sweeps skip the residual pass of starts whose update-time
  // estimate (error ~1e-7) is far above tol; plateau detection needs every
  // sweep's residual, so it keeps them all.
  const double skip = p->plateau_window == 0 ? std::max(1e3 * ctol, 1e-5) : 0.0;
  std::vector<std::vector<double>> rows;
  int row = 0, nrows = 0;
  while (left > 0) {
    if (row == nrows) {  // launch the next batch (or single sweep)
      int room = p->max_sweeps;
      for (int t = 0; t < T; ++t)
        if (busy[t]) room = std::min(room, p->max_sweeps - tsweeps[t]);
      const int B = batch ? std::max(1, std::min(kSweepBatch, room)) : 1;
      if (df && B > 1) {
        CK(cudaMemsetAsync(stop, 0, sizeof(int), st));
        for (int b = 0; b < B; ++b)
          TRY(df_sweep(ctx, R, rs, psi, phil, nullptr, R.active, R.vprev, st, stop, ctol,
                       R.cost_rows + (size_t)b * S, skip));
        TRY(read_rows(ctx, R.cost_rows, S, B, rows, R.err));
        // The sweep whose cost met the tolerance ends the batch; the
        // launches behind it returned at once.
        nrows = B;
        for (int b = 0; b < B; ++b) {
          bool met = false;
          for (int s = 0; s < S; ++s) met |= act[s] && rows[b][s] <= ctol;
          if (met) {
            nrows = b + 1;
            break;
          }
        }
        prof_drop_dataflow(ctx, B - nrows);
        prof_harvest(ctx);
      } else {
        if (df) {
          TRY(df_sweep(ctx, R, rs, psi, phil, nullptr, R.active, R.vprev, st, nullptr, 0.0, nullptr, skip));
        } else {
          CK(cudaGraphLaunch(graph.exec, st));
          for (int i = 0; i < QFS_PROF_KINDS; ++i) ctx->prof.launches[i] += graph.launches[i];
        }
        rows.assign(1, std::vector<double>());
        TRY(read_costs(ctx, R.costs, S, rows[0], R.err));
        if (ctx->prof.on && !df) prof_harvest_graph(ctx);
        nrows = 1;
      }
      row = 0;
    }
    c = rows[row++];
    for (int t = 0; t < T; ++t)
      if (busy[t]) ++tsweeps[t];
    for (int s = 0; s < S; ++s)
      if (!act[s]) c[s] = prev[s];
    std::vector<char> fin(T, 0);  // slots whose target finishes at this sweep
    for (int t = 0; t < T; ++t) {
      if (!busy[t]) continue;
      const int s0 = t * spt, s1 = s0 + spt;
      if (R.prec == QFS_FP64) {
        for (int s = s0; s < s1; ++s)
          if (act[s] && c[s] <= tol) fin[t] = 1;
        continue;
      }
      // Candidates by their complex64 cost; each is confirmed in FP64.
      std::vector<int> cand;
      for (int s = s0; s < s1; ++s)
        if (act[s] && c[s] <= ctol) cand.push_back(s);
      for (int s : cand) {
        TRY(check64(ctx, R, s, &c64[s]));
        if (c64[s] <= tol) fin[t] = 1;
      }
      if (!fin[t]) {
        // complex64 reached the switch cost but FP64 is above tol: refine
        // that start in FP64.
        for (int s : cand) {
          const size_t toff = (size_t)t * R.sN;
          for (int it = 0; it < p->refine_sweeps_max && !fin[t]; ++it) {
            TRY(sweep(ctx, R, R64, Slice{0, 1, 1, ctx->stream}, R.g64 + (size_t)s * R.L * 16,
                      R.g32 + (size_t)s * R.L * 16, R.psi64 + toff, R.phil64 + toff, R.B64r, R.phi64r,
                      R.partials64r, R.nblk64_max, R.cost64r, nullptr, nullptr, R.stream_b64,
                      R.vprev + (size_t)s * R.L * 16, R.counters + R.S));
            ++tfp64[t];
            std::vector<double> cr;
            TRY(read_costs(ctx, R.cost64r, 1, cr));
            if (cr[0] <= tol) {
              TRY(check64(ctx, R, s, &c64[s]));
              if (c64[s] <= tol) fin[t] = 1;
            }
          }
          if (fin[t]) break;
        }
      }
      for (int s = s0; s < s1; ++s)
        if (!std::isnan(c64[s])) c[s] = c64[s];
    }
    if (R.validate && busy[0] && (fin[0] || tsweeps[0] >= p->min_sweeps)) {
      // Generalisation check (Sec. 3): the start with the lowest training
      // cost, evaluated in FP64 on the validation states (one target).
      int b = -1;
      for (int s = 0; s < S; ++s)
        if (act[s] && (b < 0 || c[s] < c[b])) b = s;
      if (b >= 0) {
        double cv = 0.0;
        TRY(check64(ctx, R, b, &cv, R.psi_val64, R.phil_val64));
        cur[0].c_val = cv;
        const double gen = c[b] > 0.0 ? cv / c[b] - 1.0 : (cv > 0.0 ? inf : 0.0);
        if (gen > p->overtrain_ratio) {
          cur[0].overtrained = true;
          fin[0] = 1;
        }
      }
    }
    bool act_changed = false;
    if (p->plateau_window > 0) {
      for (int s = 0; s < S; ++s) {
        const int t = s / spt;
        if (!act[s] || !busy[t] || fin[t]) continue;
        if (std::isfinite(prev[s])) {
          const bool improved = std::fabs(prev[s]) - std::fabs(c[s]) > p->diff_tol_r * std::fabs(c[s]);
          stall[s] = improved ? 0 : stall[s] + 1;
          if (stall[s] >= p->plateau_window && tsweeps[t] >= p->min_sweeps) {
            act[s] = 0;
            act_changed = true;
          }
        }
      }
      for (int t = 0; t < T; ++t) {
        if (!busy[t] || fin[t]) continue;
        bool any = false;
        for (int s = t * spt; s < (t + 1) * spt; ++s) any |= act[s] != 0;
        if (!any) fin[t] = 1;
      }
    }
    for (int t = 0; t < T; ++t)
      if (busy[t] && !fin[t] && tsweeps[t] >= p->max_sweeps) fin[t] = 1;
    prev = c;
    for (int t = 0; t < T; ++t) {
      if (!fin[t]) continue;
      // Selection: lowest cost (FP64-confirmed where available), lowest
      // index on ties.
      Outcome& out = cur[t];
      const int s0 = t * spt;
      int best = s0;
      for (int s = s0 + 1; s < s0 + spt; ++s)
        if (prev[s] < prev[best]) best = s;
      double cost = prev[best];
      if (R.prec == QFS_MIXED) TRY(check64(ctx, R, best, &cost));
      out.best = best - s0;
      out.cost = cost;
      out.sweeps = tsweeps[t];
      out.converged = cost <= tol && !out.overtrained;
      out.fp64_sweeps = tfp64[t];
      out.start_costs.assign(prev.begin() + s0, prev.begin() + s0 + spt);
      out.start_costs[best - s0] = cost;
      bool refilled = false;
      TRY(finish(t, out, refilled));
      for (int s = s0; s < s0 + spt; ++s) {
        prev[s] = inf;
        stall[s] = 0;
        c64[s] = nan;
        if ((act[s] != 0) != refilled) act_changed = true;
        act[s] = refilled ? 1 : 0;
      }
      cur[t] = Outcome();
      tsweeps[t] = 0;
      tfp64[t] = 0;
      if (!refilled) {
        busy[t] = 0;
        --left;
      }
    }
    if (act_changed && left > 0)
      CK(cudaMemcpyAsync(R.active, act.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
    if (R.prec == QFS_MIXED)
      for (int s = 0; s < S; ++s)
        if (!std::isnan(c64[s])) c64[s] = nan;
  }
  return QFS_OK;
}

// One target (slot 0): run and report its outcome.
int run_multistart(qfs_ctx* ctx, Run& R, const qfs_params* p, Outcome& out) {
  return run_multistart(ctx, R, p, [&](int, const Outcome& o, bool& refilled) {
    out = o;
    refilled = false;
    return (int)QFS_OK;
  });
}

int ctx_check(const qfs_ctx* ctx) {
  if (!ctx) return fail(QFS_EINVAL, "context is NULL");
  return QFS_OK;
}

int set_device(qfs_ctx* ctx) {
  CK(cudaSetDevice(ctx->device));
  return QFS_OK;
}

// Seed of attempt a's training and validation states (attempt 0: the seed).
uint64_t attempt_seed(uint64_t seed, int a) { return a == 0 ? seed : seed ^ ((uint64_t)a * 0x9E3779B97F4A7C15ULL); }

// Double-and-restart (Sec. 3, App. A): multistart runs on M training
// states with the validation check; when it halts a run, M doubles (up to
// 2^n), fresh states are drawn, every start keeps its gates, and the run
// restarts.
int instantiate_restarting(qfs_ctx* ctx, const qfs_circuit* c, const double* target, bool target_dev,
                           const double* gates0, bool gates_dev, uint64_t seed, const qfs_params* p,
                           double* gates_out, bool out_dev, qfs_result* result, double* start_costs) {
  cudaStream_t st = ctx->stream;
  const int S = p->multistarts, L = c->L, n = c->n;
  const long long N = 1LL << n;
  int groups = p->start_groups;
  if (groups <= 0) groups = S >= 8 ? 2 : 1;
  // Every start's gates, carried from attempt to attempt (host).
  std::vector<std::complex<double>> G((size_t)S * L * 16);
  if (gates0) {
    CK(cudaMemcpy(G.data(), gates0, G.size() * sizeof(double2), gates_dev ? cudaMemcpyDeviceToHost
                                                                           : cudaMemcpyHostToHost));
  } else {
    generate_gates(seed, S * L, G.data());
  }
  int M = p->M, total = 0, fp64 = 0;
  for (int attempt = 0;; ++attempt) {
    const bool validate = M < N;
    Run R;
    TRY(prepare(ctx, R, c, M, S, p->precision, p->beta, !target_dev, false, groups, validate));
    if (target_dev) {
      R.U = reinterpret_cast<const double2*>(target);
    } else {
      CK(cudaMemcpyAsync(R.U_copy, target, (size_t)R.N * R.N * sizeof(double2), cudaMemcpyHostToDevice, st));
      R.U = R.U_copy;
    }
    const uint64_t sa = attempt_seed(seed, attempt);
    std::vector<std::complex<double>> h((size_t)R.sN);
    draw_states(p->training_distribution, sa, 1u, n, M, h.data());
    CK(cudaMemcpyAsync(R.psi64, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (validate) {
      draw_states(p->training_distribution, sa, 5u, n, M, h.data());
      CK(cudaMemcpyAsync(R.psi_val64, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
      ctx->prof.launches[QFS_PROF_GEMM] += target_product(ctx, R, R.U, R.psi_val64, R.phil_val64);
      CK(cudaStreamSynchronize(st));
    }
    CK(cudaMemcpyAsync(R.g64, G.data(), G.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    TRY(setup_inputs(ctx, R));
    Outcome o;
    TRY(run_multistart(ctx, R, p, o));
    total += o.sweeps;
    fp64 += o.fp64_sweeps;
    CK(cudaMemcpyAsync(G.data(), R.g64, G.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (o.overtrained && 2LL * M <= N) {
      M *= 2;
      continue;
    }
    CK(cudaMemcpyAsync(gates_out, G.data() + (size_t)o.best * L * 16, (size_t)L * 16 * sizeof(double2),
                       out_dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
    CK(cudaStreamSynchronize(st));
    result->cost = o.cost;
    result->sweeps = total;
    result->converged = o.converged;
    result->best_start = o.best;
    result->fp64_sweeps = fp64;
    result->training_states = M;
    if (start_costs) std::copy(o.start_costs.begin(), o.start_costs.end(), start_costs);
    return QFS_OK;
  }
}

// T targets of one structure swept together (several targets per dataflow
// launch; T = 1: one instantiation).  Arrays are target-major: targets
// T x N x N, samples T x N x M, initial gates T x multistarts x L x 16,
// gates_out T x L x 16, result[T], start_costs T x multistarts.  Drawn
// inputs of target t come from seed + t.
int instantiate_common(qfs_ctx* ctx, const qfs_circuit* c, const double* target, bool target_dev,
                       const double* samples, bool samples_dev, const double* gates0,
                       bool gates_dev, uint64_t seed, const qfs_params* p, double* gates_out,
                       bool out_dev, qfs_result* result, double* start_costs, int T = 1) {
  TRY(check_circuit(c));
  if (!p) return fail(QFS_EINVAL, "params is NULL");
  if (!target) return fail(QFS_EINVAL, "target is NULL");
  if (!gates_out) return fail(QFS_EINVAL, "gates_out is NULL");
  if (!result) return fail(QFS_EINVAL, "result is NULL");
  TRY(check_run_params(c->n, p->M, p->multistarts, p->max_sweeps, p->precision, p->beta, p->dist_tol));
  if (p->plateau_window < 0 || p->min_sweeps < 0 || !(p->diff_tol_r >= 0.0))
    return fail(QFS_EINVAL, "plateau_window, min_sweeps and diff_tol_r must be >= 0");
  if (p->precision == QFS_MIXED && p->refine_sweeps_max < 0)
    return fail(QFS_EINVAL, "refine_sweeps_max must be >= 0");
  if (!(p->refine_switch_tol >= 0.0) || std::isinf(p->refine_switch_tol))
    return fail(QFS_EINVAL, "refine_switch_tol = %g: need a finite value >= 0", p->refine_switch_tol);
  if (p->start_groups < 0) return fail(QFS_EINVAL, "start_groups = %d: need >= 0", p->start_groups);
  if (p->training_distribution != QFS_STATES_HAAR && p->training_distribution != QFS_STATES_BASIS)
    return fail(QFS_EINVAL, "training_distribution = %d: need QFS_STATES_HAAR or QFS_STATES_BASIS",
                p->training_distribution);
  if (p->restart_doubling && (samples || !(p->overtrain_ratio >= 0.0)))
    return fail(QFS_EINVAL, "restart_doubling needs library-drawn training states and overtrain_ratio >= 0");
  if (T < 1) return fail(QFS_EINVAL, "T = %d: need >= 1 targets", T);
  if (p->concurrent_targets < 0) return fail(QFS_EINVAL, "concurrent_targets = %d: need >= 0", p->concurrent_targets);
  if (T > 1 && p->restart_doubling)
    return fail(QFS_EUNSUPPORTED, "double-and-restart takes one target per call");
  // Targets sweep in `slots` concurrent slots; a slot whose target finishes
  // takes the next target (continuous batching).
  const int slots = T == 1 ? 1 : std::max(1, std::min(T, p->concurrent_targets > 0 ? p->concurrent_targets : 4));
  if ((long long)slots * p->multistarts > 65535)
    return fail(QFS_EUNSUPPORTED, "concurrent targets x multistarts = %lld > 65535",
                (long long)slots * p->multistarts);
  TRY(ctx_check(ctx));
  TRY(set_device(ctx));
  if (p->restart_doubling) return instantiate_restarting(ctx, c, target, target_dev, gates0, gates_dev, seed, p,
                                                         gates_out, out_dev, result, start_costs);
  Run R;
  int groups = p->start_groups;
  if (groups <= 0) groups = p->multistarts >= 8 ? 2 : 1;
  TRY(prepare(ctx, R, c, p->M, p->multistarts, p->precision, p->beta, !target_dev, false, groups, false, slots));
  if (slots > 1 && !df_usable(ctx, R, p->precision == QFS_MIXED ? R32 : R64))
    return fail(QFS_EUNSUPPORTED, "several targets per call need the dataflow sweep (cooperative launch%s)",
                p->precision == QFS_MIXED ? ", even M" : "");
  cudaStream_t st = ctx->stream;
  const size_t NN = (size_t)R.N * R.N, gsz = (size_t)R.spt * R.L * 16;
  R.Uslot.assign(slots, nullptr);
  std::vector<int> slot_target(slots, -1);
  // Target i's inputs into slot t.
  auto load = [&](int t, int i) -> int {
    if (target_dev) {
      R.Uslot[t] = reinterpret_cast<const double2*>(target) + (size_t)i * NN;
    } else {
      CK(cudaMemcpyAsync(R.U_copy + (size_t)t * NN, target + (size_t)i * NN * 2, NN * sizeof(double2),
                         cudaMemcpyHostToDevice, st));
      R.Uslot[t] = R.U_copy + (size_t)t * NN;
    }
    if (samples) {
      CK(cudaMemcpyAsync(R.psi64 + (size_t)t * R.sN, samples + (size_t)i * R.sN * 2, (size_t)R.sN * sizeof(double2),
                         samples_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
      std::vector<std::complex<double>> h((size_t)R.sN);
      draw_states(p->training_distribution, seed + (uint64_t)i, 1u, R.n, R.M, h.data());
      CK(cudaMemcpyAsync(R.psi64 + (size_t)t * R.sN, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice,
                         st));
      CK(cudaStreamSynchronize(st));
    }
    if (gates0) {
      CK(cudaMemcpyAsync(R.g64 + (size_t)t * gsz, gates0 + (size_t)i * gsz * 2, gsz * sizeof(double2),
                         gates_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
      std::vector<std::complex<double>> h(gsz);
      generate_gates(seed + (uint64_t)i, R.spt * R.L, h.data());
      CK(cudaMemcpyAsync(R.g64 + (size_t)t * gsz, h.data(), gsz * sizeof(double2), cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
    }
    slot_target[t] = i;
    return QFS_OK;
  };
  for (int t = 0; t < slots; ++t) TRY(load(t, t));
  TRY(setup_inputs(ctx, R));
  int next = slots;
  auto finish = [&](int t, const Outcome& o, bool& refilled) -> int {
    const int i = slot_target[t];
    CK(cudaMemcpyAsync(gates_out + (size_t)i * R.L * 32, R.g64 + ((size_t)t * R.spt + o.best) * R.L * 16,
                       (size_t)R.L * 16 * sizeof(double2), out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
    qfs_result& r = result[i];
    r.cost = o.cost;
    r.sweeps = o.sweeps;
    r.converged = o.converged;
    r.best_start = o.best;
    r.fp64_sweeps = o.fp64_sweeps;
    r.training_states = R.M;
    if (start_costs) std::copy(o.start_costs.begin(), o.start_costs.end(), start_costs + (size_t)i * R.spt);
    refilled = next < T;
    if (refilled) {
      TRY(load(t, next++));
      TRY(setup_slot(ctx, R, t));
    }
    return QFS_OK;
  };
  TRY(run_multistart(ctx, R, p, finish));
  return QFS_OK;
}

}  // namespace

extern "C" {

void qfs_default_params(qfs_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->M = 2;
  p->multistarts = 16;
  p->max_sweeps = 10000;
  p->min_sweeps = 6;
  p->plateau_window = 0;
  p->precision = QFS_FP64;
  p->refine_sweeps_max = 50;
  p->start_groups = 0;
  p->restart_doubling = 0;
  p->overtrain_ratio = 0.1;
  p->training_distribution = QFS_STATES_HAAR;
  p->concurrent_targets = 0;
  p->refine_switch_tol = 0.0;
  p->seed = 0;
  p->dist_tol = 1e-8;
  p->diff_tol_r = 1e-5;
  p->beta = 0.0;
}

const char* qfs_last_error(void) { return g_err.c_str(); }

int qfs_create(qfs_ctx** out, int device, void* cuda_stream) {
  g_err.clear();
  if (!out) return fail(QFS_EINVAL, "out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0)
    return fail(QFS_ECUDA, "no CUDA device: %s", e != cudaSuccess ? cudaGetErrorString(e) : "count = 0");
  if (device < 0 || device >= count) return fail(QFS_EINVAL, "device %d of %d", device, count);
  qfs_ctx* ctx = new qfs_ctx();
  ctx->device = device;
  if (const char* f = std::getenv("QFS_DF_ITEM_KB")) ctx->df_item_bytes = std::max(16, std::atoi(f)) * 1024.0;
  if (const char* f = std::getenv("QFS_DF_ITEMS_PER_CTA")) ctx->df_items_per_cta = std::max(0.25, std::atof(f));
  if (const char* f = std::getenv("QFS_DF_ITEMS_PER_CTA_FWD"))
    ctx->df_items_per_cta_fwd = std::max(0.25, std::atof(f));
  e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->coop, cudaDevAttrCooperativeLaunch, device);
  int l2 = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
  ctx->l2_bytes = (size_t)l2;
  if (e == cudaSuccess) {
    if (cuda_stream) {
      ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = e == cudaSuccess;
    }
  }
  if (e != cudaSuccess) {
    delete ctx;
    return fail(QFS_ECUDA, "context set-up on device %d: %s", device, cudaGetErrorString(e));
  }
  *out = ctx;
  return QFS_OK;
}

int qfs_dataflow_trace_enable(qfs_ctx* ctx, int64_t capacity) {
  g_err.clear();
  TRY(ctx_check(ctx));
  if (capacity < 0) return fail(QFS_EINVAL, "capacity = %lld", (long long)capacity);
  TRY(set_device(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->df_trace) CK(cudaFree(ctx->df_trace));
  ctx->df_trace = nullptr;
  ctx->df_trace_n = 0;
  ctx->df_trace_steps = ctx->df_trace_S = 0;
  ctx->df_trace_items = 0;
  if (capacity > 0) {
    CK(cudaMalloc(&ctx->df_trace, sizeof(unsigned long long) * (size_t)capacity));
    CK(cudaMemset(ctx->df_trace, 0, sizeof(unsigned long long) * (size_t)capacity));
    ctx->df_trace_n = (size_t)capacity;
  }
  return QFS_OK;
}

int qfs_dataflow_trace_read(qfs_ctx* ctx, uint64_t* out, int64_t capacity, int32_t* steps, int32_t* S,
                            int64_t* items) {
  g_err.clear();
  TRY(ctx_check(ctx));
  if (!steps || !S) return fail(QFS_EINVAL, "steps and S must be given");
  *steps = ctx->df_trace_steps;
  *S = ctx->df_trace_S;
  if (items) *items = ctx->df_trace_items;
  const size_t n = (size_t)ctx->df_trace_steps * ctx->df_trace_S * 4 + (size_t)ctx->df_trace_items * 4;
  if (!out || n == 0) return QFS_OK;
  if ((size_t)capacity < n) return fail(QFS_EINVAL, "capacity %lld < %zu stamps", (long long)capacity, n);
  TRY(set_device(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(out, ctx->df_trace, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
  return QFS_OK;
}

int qfs_batch_trace_enable(qfs_ctx* ctx, int64_t capacity) {
  g_err.clear();
  TRY(ctx_check(ctx));
  if (capacity < 0) return fail(QFS_EINVAL, "capacity = %lld", (long long)capacity);
  TRY(set_device(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->bt_trace) CK(cudaFree(ctx->bt_trace));
  ctx->bt_trace = nullptr;
  ctx->bt_trace_n = 0;
  ctx->bt_units = 0;
  if (capacity > 0) {
    CK(cudaMalloc(&ctx->bt_trace, sizeof(unsigned long long) * (size_t)capacity));
    CK(cudaMemset(ctx->bt_trace, 0, sizeof(unsigned long long) * (size_t)capacity));
    ctx->bt_trace_n = (size_t)capacity;
  }
  return QFS_OK;
}

int qfs_batch_trace_read(qfs_ctx* ctx, uint64_t* out, int64_t capacity, int64_t* units) {
  g_err.clear();
  TRY(ctx_check(ctx));
  if (!units) return fail(QFS_EINVAL, "units must be given");
  *units = ctx->bt_units;
  const size_t n = (size_t)ctx->bt_units * 4;
  if (!out || n == 0) return QFS_OK;
  if ((size_t)capacity < n) return fail(QFS_EINVAL, "capacity %lld < %zu stamps", (long long)capacity, n);
  TRY(set_device(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(out, ctx->bt_trace, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
  return QFS_OK;
}

void qfs_destroy(qfs_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->df_trace) cudaFree(ctx->df_trace);
  if (ctx->bt_trace) cudaFree(ctx->bt_trace);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->h_draw) cudaFreeHost(ctx->h_draw);
  for (int k = 0; k < 2; ++k)
    if (ctx->h_half[k]) cudaFreeHost(ctx->h_half[k]);
  prof_harvest(ctx);
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  for (int g = 0; g < kMaxGroups; ++g) {
    if (ctx->gstream[g]) cudaStreamDestroy(ctx->gstream[g]);
    if (ctx->gevent[g]) cudaEventDestroy(ctx->gevent[g]);
  }
  if (ctx->fork_event) cudaEventDestroy(ctx->fork_event);
  for (auto& g : ctx->batch_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

int qfs_device_sms(const qfs_ctx* ctx) { return ctx ? ctx->num_sms : 0; }

int qfs_set_option(qfs_ctx* ctx, int32_t option, int64_t value) {
  g_err.clear();
  if (!ctx) return fail(QFS_EINVAL, "ctx is NULL");
  switch (option) {
    case QFS_OPT_WAIT_LIMIT:
      if (value < 1) return fail(QFS_EINVAL, "wait limit %lld < 1", (long long)value);
      ctx->df_wait_limit = value;
      return QFS_OK;
    case QFS_OPT_WORKSPACE_CAP:
      if (value < 0) return fail(QFS_EINVAL, "workspace cap %lld < 0", (long long)value);
      ctx->ws_cap = (size_t)value;
      return QFS_OK;
    case QFS_OPT_FUSED_UPDATE: ctx->fuse_update = value != 0; return QFS_OK;
    case QFS_OPT_DATAFLOW: ctx->dataflow = value != 0; return QFS_OK;
    case QFS_OPT_TWO_GATE_FORWARD: ctx->df_fwd2 = value != 0; return QFS_OK;
    case QFS_OPT_FP64_TARGET_PRODUCT: ctx->upsi_fp64 = value != 0; return QFS_OK;
    case QFS_OPT_BATCH_LANES_PER_START:
      if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32)
        return fail(QFS_EINVAL, "lanes per start %lld: need 0, 4, 8, 16 or 32", (long long)value);
      ctx->batch_force_G = (int)value;
      return QFS_OK;
    default: return fail(QFS_EINVAL, "unknown option %d", option);
  }
}

int qfs_get_option(qfs_ctx* ctx, int32_t option, int64_t* value) {
  g_err.clear();
  if (!ctx || !value) return fail(QFS_EINVAL, "ctx and value must be given");
  switch (option) {
    case QFS_OPT_WAIT_LIMIT: *value = ctx->df_wait_limit; return QFS_OK;
    case QFS_OPT_WORKSPACE_CAP: *value = (int64_t)ctx->ws_cap; return QFS_OK;
    case QFS_OPT_FUSED_UPDATE: *value = ctx->fuse_update; return QFS_OK;
    case QFS_OPT_DATAFLOW: *value = ctx->dataflow; return QFS_OK;
    case QFS_OPT_TWO_GATE_FORWARD: *value = ctx->df_fwd2; return QFS_OK;
    case QFS_OPT_FP64_TARGET_PRODUCT: *value = ctx->upsi_fp64; return QFS_OK;
    case QFS_OPT_BATCH_LANES_PER_START: *value = ctx->batch_force_G; return QFS_OK;
    default: return fail(QFS_EINVAL, "unknown option %d", option);
  }
}

int qfs_profile_enable(qfs_ctx* ctx, int enable) {
  g_err.clear();
  TRY(ctx_check(ctx));
  if (ctx->prof.on && !enable) {
    CK(cudaStreamSynchronize(ctx->stream));
    prof_harvest(ctx);
  }
  ctx->prof.on = enable != 0;
  return QFS_OK;
}

int qfs_profile_reset(qfs_ctx* ctx) {
  g_err.clear();
  TRY(ctx_check(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  prof_harvest(ctx);
  for (int i = 0; i < QFS_PROF_KINDS; ++i) {
    ctx->prof.launches[i] = ctx->prof.timed[i] = 0;
    ctx->prof.ms[i] = ctx->prof.bytes[i] = 0.0;
  }
  return QFS_OK;
}

int qfs_profile_read(qfs_ctx* ctx, int32_t kind, int64_t* launches, int64_t* timed,
                     double* total_ms, double* total_bytes) {
  g_err.clear();
  TRY(ctx_check(ctx));
  if (kind < -1 || kind >= QFS_PROF_KINDS) return fail(QFS_EINVAL, "kind = %d", kind);
  CK(cudaStreamSynchronize(ctx->stream));
  prof_harvest(ctx);
  long long l = 0, t = 0;
  double ms = 0.0, by = 0.0;
  for (int i = 0; i < QFS_PROF_KINDS; ++i) {
    if (kind != -1 && kind != i) continue;
    l += ctx->prof.launches[i];
    t += ctx->prof.timed[i];
    ms += ctx->prof.ms[i];
    by += ctx->prof.bytes[i];
  }
  if (launches) *launches = l;
  if (timed) *timed = t;
  if (total_ms) *total_ms = ms;
  if (total_bytes) *total_bytes = by;
  return QFS_OK;
}

int qfs_generate_inputs(uint64_t seed, int32_t n, int32_t M, int32_t S, int32_t L,
                        double* samples_out, double* gates_out) {
  g_err.clear();
  if (n < 2 || n > QFS_MAX_QUBITS) return fail(QFS_EINVAL, "n = %d out of [2, %d]", n, QFS_MAX_QUBITS);
  if (samples_out) {
    if (M < 1 || (long long)M > (1LL << n)) return fail(QFS_EINVAL, "M = %d out of [1, 2^n]", M);
    qfs::generate_samples(seed, n, M, reinterpret_cast<std::complex<double>*>(samples_out));
  }
  if (gates_out) {
    if (S < 1 || L < 1) return fail(QFS_EINVAL, "S = %d, L = %d: need >= 1", S, L);
    qfs::generate_gates(seed, S * L, reinterpret_cast<std::complex<double>*>(gates_out));
  }
  return QFS_OK;
}

int qfs_generate_states(uint64_t seed, int32_t distribution, uint32_t stream, int32_t n, int32_t M,
                        double* out) {
  g_err.clear();
  if (n < 2 || n > QFS_MAX_QUBITS) return fail(QFS_EINVAL, "n = %d out of [2, %d]", n, QFS_MAX_QUBITS);
  if (M < 1 || (long long)M > (1LL << n)) return fail(QFS_EINVAL, "M = %d out of [1, 2^n]", M);
  if (distribution != QFS_STATES_HAAR && distribution != QFS_STATES_BASIS)
    return fail(QFS_EINVAL, "distribution = %d: need QFS_STATES_HAAR or QFS_STATES_BASIS", distribution);
  if (!out) return fail(QFS_EINVAL, "out is NULL");
  qfs::draw_states(distribution, seed, stream, n, M, reinterpret_cast<std::complex<double>*>(out));
  return QFS_OK;
}

int qfs_instantiate(qfs_ctx* ctx, const qfs_circuit* circuit, const double* target,
                    const qfs_params* p, double* gates_out, qfs_result* result,
                    double* start_costs) {
  g_err.clear();
  return instantiate_common(ctx, circuit, target, false, nullptr, false, nullptr, false,
                            p ? p->seed : 0, p, gates_out, false, result, start_costs);
}

int qfs_instantiate_ex(qfs_ctx* ctx, const qfs_circuit* circuit, const double* target,
                       const double* samples, const double* init_gates, const qfs_params* p,
                       double* gates_out, qfs_result* result, double* start_costs) {
  g_err.clear();
  if (!samples || !init_gates) return fail(QFS_EINVAL, "samples and init_gates must be given");
  return instantiate_common(ctx, circuit, target, false, samples, false, init_gates, false,
                            0, p, gates_out, false, result, start_costs);
}

int qfs_instantiate_dev(qfs_ctx* ctx, const qfs_circuit* circuit, const double* target_dev,
                        const double* samples_dev, const double* init_gates_dev,
                        const qfs_params* p, double* gates_out_dev, qfs_result* result,
                        double* start_costs) {
  g_err.clear();
  if (!samples_dev || !init_gates_dev) return fail(QFS_EINVAL, "samples and init_gates must be given");
  return instantiate_common(ctx, circuit, target_dev, true, samples_dev, true, init_gates_dev, true,
                            0, p, gates_out_dev, true, result, start_costs);
}

int qfs_instantiate_many(qfs_ctx* ctx, const qfs_circuit* circuit, int32_t T, const double* targets,
                         const double* samples, const double* init_gates, const qfs_params* p,
                         double* gates_out, qfs_result* results, double* start_costs) {
  g_err.clear();
  return instantiate_common(ctx, circuit, targets, false, samples, false, init_gates, false, p ? p->seed : 0, p,
                            gates_out, false, results, start_costs, T);
}

int qfs_instantiate_many_dev(qfs_ctx* ctx, const qfs_circuit* circuit, int32_t T, const double* targets_dev,
                             const double* samples_dev, const double* init_gates_dev, const qfs_params* p,
                             double* gates_out_dev, qfs_result* results, double* start_costs) {
  g_err.clear();
  if (!samples_dev || !init_gates_dev) return fail(QFS_EINVAL, "samples and init_gates must be given");
  return instantiate_common(ctx, circuit, targets_dev, true, samples_dev, true, init_gates_dev, true, 0, p,
                            gates_out_dev, true, results, start_costs, T);
}

int qfs_sweep_once(qfs_ctx* ctx, const qfs_circuit* circuit, const double* target,
                   const double* samples, int32_t M, int32_t S, const double* gates_in,
                   int32_t precision, double beta, double* gates_out, double* envs_out,
                   double* costs_out) {
  g_err.clear();
  TRY(check_circuit(circuit));
  TRY(check_run_params(circuit->n, M, S, 1, precision, beta, 0.0));
  if (!target || !samples || !gates_in || !gates_out)
    return fail(QFS_EINVAL, "target, samples, gates_in and gates_out must be given");
  TRY(ctx_check(ctx));
  TRY(set_device(ctx));
  Run R;
  TRY(prepare(ctx, R, circuit, M, S, precision, beta, true, envs_out != nullptr));
  cudaStream_t st = ctx->stream;
  const size_t gbytes = (size_t)S * R.L * 16 * sizeof(double2);
  CK(cudaMemcpyAsync(R.U_copy, target, (size_t)R.N * R.N * sizeof(double2), cudaMemcpyHostToDevice, st));
  R.U = R.U_copy;
  CK(cudaMemcpyAsync(R.psi64, samples, (size_t)R.sN * sizeof(double2), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(R.g64, gates_in, gbytes, cudaMemcpyHostToDevice, st));
  TRY(setup_inputs(ctx, R));
  const Real rs = precision == QFS_MIXED ? R32 : R64;
  const void* psi = rs == R32 ? (const void*)R.psi32 : (const void*)R.psi64;
  const void* phil = rs == R32 ? (const void*)R.phil32 : (const void*)R.phil64;
  if (df_usable(ctx, R, rs))
    TRY(df_sweep(ctx, R, rs, psi, phil, R.envs, nullptr, nullptr, st));
  else
    TRY(sweep(ctx, R, rs, Slice{0, S, S, ctx->stream}, R.g64, R.g32, psi, phil, R.B, R.phi, R.partials,
              R.nblk_max, R.costs, R.envs, nullptr, R.stream_b, nullptr, R.counters));
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(gates_out, R.g64, gbytes, cudaMemcpyDeviceToHost, st));
  if (envs_out) CK(cudaMemcpyAsync(envs_out, R.envs, gbytes, cudaMemcpyDeviceToHost, st));
  if (costs_out) CK(cudaMemcpyAsync(costs_out, R.costs, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
  int err = 0;
  CK(cudaMemcpyAsync(&err, R.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err) return fail(QFS_ETIMEOUT, "a bounded device wait ran out (error word %d)", err);
  return QFS_OK;
}

int qfs_gate_update(qfs_ctx* ctx, int32_t count, const double* envs, const double* gates_old,
                    double beta, double* gates_out) {
  g_err.clear();
  if (count < 0) return fail(QFS_EINVAL, "count = %d", count);
  if (count == 0) return QFS_OK;
  if (!envs || !gates_out) return fail(QFS_EINVAL, "envs and gates_out must be given");
  if (!(beta >= 0.0 && beta < 1.0)) return fail(QFS_EINVAL, "beta = %g: need 0 <= beta < 1", beta);
  if (beta != 0.0 && !gates_old) return fail(QFS_EINVAL, "beta != 0 needs gates_old");
  TRY(ctx_check(ctx));
  TRY(set_device(ctx));
  const size_t bytes = (size_t)count * 16 * sizeof(double2);
  TRY(ensure_ws(ctx, 3 * align_up(bytes)));
  double2* dE = reinterpret_cast<double2*>(ctx->ws);
  double2* dG = reinterpret_cast<double2*>(ctx->ws + align_up(bytes));
  double2* dO = reinterpret_cast<double2*>(ctx->ws + 2 * align_up(bytes));
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(dE, envs, bytes, cudaMemcpyHostToDevice, st));
  if (gates_old) CK(cudaMemcpyAsync(dG, gates_old, bytes, cudaMemcpyHostToDevice, st));
  ctx->prof.launches[QFS_PROF_UPDATE] += 1;
  launch_gate_update_batch(count, dE, gates_old ? dG : nullptr, beta, dO, st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(gates_out, dO, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return QFS_OK;
}

int qfs_target_product_dev(qfs_ctx* ctx, int32_t n, int32_t M, const double* target_dev,
                           const double* samples_dev, int32_t precision, double* out_dev) {
  g_err.clear();
  if (n < 2 || n > QFS_MAX_QUBITS) return fail(QFS_EINVAL, "n = %d out of [2, %d]", n, QFS_MAX_QUBITS);
  if (M < 1 || (long long)M > (1LL << n)) return fail(QFS_EINVAL, "M = %d out of [1, 2^n]", M);
  if (precision != QFS_FP64 && precision != QFS_MIXED)
    return fail(QFS_EINVAL, "precision = %d: need QFS_FP64 or QFS_MIXED", precision);
  if (!target_dev || !samples_dev || !out_dev) return fail(QFS_EINVAL, "target, samples and out must be given");
  TRY(ctx_check(ctx));
  TRY(set_device(ctx));
  const int N = 1 << n;
  const double2* U = reinterpret_cast<const double2*>(target_dev);
  const double2* P = reinterpret_cast<const double2*>(samples_dev);
  double2* O = reinterpret_cast<double2*>(out_dev);
  cudaStream_t st = ctx->stream;
  if (precision == QFS_FP64) {
    ctx->prof.launches[QFS_PROF_GEMM] += 1;
    launch_gemm_upsi(U, P, O, N, M, st);
  } else {
    const size_t split_bytes = align_up((size_t)N * M * sizeof(float4));
    const int splits = upsi_pair_splits(N, M, ctx->num_sms, (size_t)16 * N * M * sizeof(double2));
    TRY(ensure_ws(ctx, split_bytes + align_up((size_t)splits * N * M * sizeof(double2))));
    ctx->prof.launches[QFS_PROF_GEMM] += splits > 1 ? 3 : 2;
    launch_gemm_upsi_pair(U, P, O, N, M, reinterpret_cast<float4*>(ctx->ws),
                          reinterpret_cast<double2*>(ctx->ws + split_bytes), splits, ctx->num_sms, st);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return QFS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free single sweep.  The scratch of the sweep (U Psi, the B list,
// Phi and the reduction partials) lives in one statically sized device array
// instead of the context's cudaMalloc'd workspace, for callers that may not
// allocate device memory.  The paper has no counterpart.

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[QFS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
int g_noalloc_sms[kMaxDevices] = {};
int g_noalloc_l2[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array (host code cannot use the symbol itself) and the SM count.
int noalloc_setup(int dev, void** ptr, int* sms, int* l2) {
  if (dev < 0 || dev >= kMaxDevices) return fail(QFS_EUNSUPPORTED, "device %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    int s = 0, l = 0;
    CK(cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&l, cudaDevAttrL2CacheSize, dev));
    g_noalloc_sms[dev] = s;
    g_noalloc_l2[dev] = l;
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  *sms = g_noalloc_sms[dev];
  *l2 = g_noalloc_l2[dev];
  return QFS_OK;
}

}  // namespace

extern "C" int qfs_sweep_once_noalloc(void* cuda_stream, const qfs_circuit* circuit,
                                      const double* target_dev, const double* samples_dev,
                                      int32_t M, int32_t S, double beta, const double* gates_in_dev,
                                      double* gates_out_dev, double* costs_out_dev,
                                      double* envs_out_dev) {
  g_err.clear();
  TRY(check_circuit(circuit));
  TRY(check_run_params(circuit->n, M, S, 1, QFS_FP64, beta, 0.0));
  if (!target_dev || !samples_dev || !gates_in_dev || !gates_out_dev)
    return fail(QFS_EINVAL, "target, samples, gates_in and gates_out must be given");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  void* scratch = nullptr;
  int sms = 0, l2 = 0;
  TRY(noalloc_setup(dev, &scratch, &sms, &l2));

  // A context on the stack: no workspace, no pinned buffer, no events.
  qfs_ctx tmp;
  tmp.device = dev;
  tmp.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  tmp.num_sms = sms;
  tmp.l2_bytes = (size_t)l2;

  Run R;
  R.n = circuit->n;
  R.L = circuit->L;
  R.M = M;
  R.S = S;
  R.N = 1LL << circuit->n;
  R.sN = (long long)M << circuit->n;
  R.pairs.assign(circuit->pairs, circuit->pairs + 2 * circuit->L);
  R.prec = QFS_FP64;
  R.beta = beta;
  R.sh = make_shape(R.n, M, S, R64, sms);
  // sweep() shapes every backward launch for shape_starts(S) starts (fewer
  // starts per shape, smaller chunks, more blocks), so the partial-sum slots
  // per start are sized for that shape, as prepare() sizes them.
  R.nblk_max = 1;
  for (int U = 2; U <= std::min(4, R.n); ++U)
    R.nblk_max = std::max(R.nblk_max, make_bwd_shape(R.n, M, shape_starts(S), R64, sms, U).nblk);

  const size_t state = (size_t)R.sN * sizeof(double2);
  const size_t need = align_up(state) + align_up((size_t)std::max(R.L - 1, 1) * S * state) +
                      align_up((size_t)S * state) + align_up((size_t)S * R.nblk_max * 32 * sizeof(double)) +
                      align_up((size_t)S * sizeof(unsigned));
  if (need > (size_t)QFS_NOALLOC_SCRATCH_BYTES)
    return fail(QFS_EUNSUPPORTED, "this sweep needs %zu bytes of scratch; the static scratch holds %u bytes",
                need, (unsigned)QFS_NOALLOC_SCRATCH_BYTES);
  char* base = static_cast<char*>(scratch);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base + off;
    off += align_up(bytes);
    return p;
  };
  R.phil64 = reinterpret_cast<double2*>(take(state));
  R.B = take((size_t)std::max(R.L - 1, 1) * S * state);
  R.phi = take((size_t)S * state);
  R.partials = reinterpret_cast<double*>(take((size_t)S * R.nblk_max * 32 * sizeof(double)));
  R.counters = reinterpret_cast<unsigned*>(take((size_t)S * sizeof(unsigned)));
  R.U = reinterpret_cast<const double2*>(target_dev);
  R.psi64 = const_cast<double2*>(reinterpret_cast<const double2*>(samples_dev));
  R.g64 = reinterpret_cast<double2*>(gates_out_dev);
  const int stream_b = (size_t)std::max(R.L - 1, 1) * S * state > tmp.l2_bytes / 2;

  cudaStream_t st = tmp.stream;
  // The fused update's counters must start at zero; a call that stopped
  // part-way could have left them otherwise.
  CK(cudaMemsetAsync(R.counters, 0, (size_t)S * sizeof(unsigned), st));
  if (gates_out_dev != gates_in_dev)
    CK(cudaMemcpyAsync(gates_out_dev, gates_in_dev, (size_t)S * R.L * 16 * sizeof(double2),
                       cudaMemcpyDeviceToDevice, st));
  launch_gemm_upsi(R.U, R.psi64, R.phil64, (int)R.N, M, st);
  TRY(sweep(&tmp, R, R64, Slice{0, S, S, st}, R.g64, nullptr, R.psi64, R.phil64, R.B, R.phi, R.partials,
            R.nblk_max, costs_out_dev, reinterpret_cast<double2*>(envs_out_dev), nullptr, stream_b,
            nullptr, R.counters));
  CK(cudaGetLastError());
  return QFS_OK;
}

// ---------------------------------------------------------------------------
// Batched instantiation of many small problems (one persistent launch per
// launch shape, all in one captured graph).

namespace {

// Where the arrays of a batched call live, and how drawn inputs are seeded.
struct BatchInputs {
  const double* targets = nullptr;
  bool targets_dev = false;
  const double* samples = nullptr;  // nullable: drawn
  bool samples_dev = false;
  const double* init_gates = nullptr;  // nullable: drawn
  bool gates_dev = false;
  double* gates_out = nullptr;  // nullable with sweep_once
  bool out_dev = false;
  const int32_t* draw_index = nullptr;  // nullable: problem i draws from seed + draw_index[i] (else seed + i)
  // One complex64 sweep of every start, no selection or FP64 finish: the
  // swept gates of every start (host, complex128) and their residual costs.
  bool sweep_once = false;
  double* start_gates_out = nullptr;
  double* start_costs_out = nullptr;
};

long long batch_class_key(int n, int L, int M, int S, bool lane_groups) {
  return ((((long long)n * 64 + L) * 4096 + M) * 128 + S) * 2 + (lane_groups ? 1 : 0);
}

// Warps per block (2, 4 or 8) for a launch whose warps each take region_f2
// float2 of shared memory: the most resident warps per SM (4 on ties, then
// 2, then 8; the kernel has no block-wide barrier, so this only sets the
// shared-memory granularity); 0 if none fits.
int batch_warps_region(int G, int region_f2) {
  int best = 0, best_res = 0;
  for (int w : {4, 2, 8}) {
    const size_t smem = (size_t)w * region_f2 * sizeof(float2);
    if (smem > 200 * 1024) continue;
    const int res = w * batch_sweep_blocks_per_sm(G, w, smem);
    if (res > best_res) {
      best_res = res;
      best = w;
    }
  }
  return best;
}

// The same for problems of at most max_elems amplitudes and max_L gates.
int batch_warps_for(int G, int max_elems, int max_L) {
  return batch_warps_region(G, batch_region_f2(G, max_elems, max_L));
}

// Schedules worth trying for a class: G lanes per start no larger than the
// state's 4-row groups (a lane with no group would idle in every state
// step), at most S starts per warp (a unit holds starts of one problem), and
// a block shape that fits.
std::vector<std::pair<int, int>> batch_candidates(int n, int M, int L, int S, bool lane_groups) {
  std::vector<std::pair<int, int>> c;
  const int groups = (1 << (n - 2)) * M;
  for (int G : {4, 8, 16, 32}) {
    if (G < 32 && !lane_groups) continue;
    if (32 / G > S) continue;
    if (G > groups * 2 && G != 32) continue;
    if (G < 32 && groups / G > 8) continue;  // many groups per lane: the warp-per-start form is as lane-efficient
    const int w = batch_warps_for(G, M << n, L);
    if (w) c.push_back({G, w});
  }
  return c;
}

struct BatchClass {
  int n, L, M;
  std::vector<int> problems;  // indices into the batch
  int G = 32, warps = 4;
};

// A unit's cost per sweep, for ordering the queue: per gate, a fixed update
// cost (about that of one gate step on 1024 amplitudes) plus the state's
// N M amplitudes.  Longer circuits also run more sweeps before they
// converge or give up, so the queue starts with them.
long long batch_unit_weight(const BatchProblem& b) { return (long long)b.L * (1024 + ((long long)b.M << b.n)); }

// Units of the given problems, heaviest first (ties by position): a
// problem's starts in runs of 32 / G.
void batch_units(const std::vector<BatchProblem>& probs, std::vector<int> idx, int S, int G,
                 std::vector<BatchUnit>& out) {
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int x, int y) { return batch_unit_weight(probs[x]) > batch_unit_weight(probs[y]); });
  const int per = 32 / G;
  for (int i : idx)
    for (int s0 = 0; s0 < S; s0 += per) out.push_back(BatchUnit{i, s0, std::min(per, S - s0)});
}

// The autotuner: for each class not yet tuned, time every candidate schedule
// on that class's problems for a few sweeps with the tolerance out of reach
// (every start runs them all) and keep the fastest per start-sweep.  The
// choice is cached per (n, L, M) on the context.  `a` points at the batch's
// prepared buffers; units and the queue go to the scratch at `scratch`.
int autotune_batch(qfs_ctx* ctx, BatchArgs a, const std::vector<BatchProblem>& probs,
                   std::vector<BatchClass>& classes, BatchUnit* units_dev, int* queue_dev, long long max_units_trial) {
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  for (BatchClass& c : classes) {
    const long long key = batch_class_key(c.n, c.L, c.M, a.S, true);
    bool found = false;
    for (auto& kv : ctx->batch_tuned)
      if (kv.first == key) {
        c.G = kv.second.first;
        c.warps = kv.second.second;
        found = true;
      }
    if (found) continue;
    const auto cand = batch_candidates(c.n, c.M, c.L, a.S, true);
    if (cand.empty()) return fail(QFS_EUNSUPPORTED, "no batched launch shape fits n = %d, L = %d, M = %d", c.n, c.L, c.M);
    if (cand.size() == 1) {
      c.G = cand[0].first;
      c.warps = cand[0].second;
      ctx->batch_tuned.push_back({key, cand[0]});
      continue;
    }
    if (!e0) {
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
    }
    // A trial of the class at full occupancy: its problems (up to 512,
    // repeated until the units fill every resident warp four times over),
    // 4 sweeps of every start, timed twice after a warm-up run; the time per
    // start-sweep decides.  The warp-per-start shape is kept unless another
    // is at least 5% faster.
    std::vector<int> sample(c.problems.begin(), c.problems.begin() + std::min<size_t>(c.problems.size(), 512));
    BatchArgs t = a;
    t.max_sweeps = 4;
    t.tol = -1.0;
    t.plateau_window = 0;
    float best = 1e30f;
    float best32 = 1e30f;
    int w32 = 0;
    for (auto [G, w] : cand) {
      std::vector<BatchUnit> u;
      const size_t smem0 = batch_sweep_smem(G, w, c.M << c.n, c.L);
      const long long slots = 4LL * ctx->num_sms * w * std::max(1, batch_sweep_blocks_per_sm(G, w, smem0));
      while ((long long)u.size() < slots && (long long)u.size() < max_units_trial) batch_units(probs, sample, a.S, G, u);
      if ((long long)u.size() > max_units_trial) u.resize((size_t)max_units_trial);
      const double start_sweeps = (double)u.size() * std::min(a.S, 32 / G) * t.max_sweeps;
      CK(cudaMemcpyAsync(units_dev, u.data(), sizeof(BatchUnit) * u.size(), cudaMemcpyHostToDevice, st));
      const size_t smem = batch_sweep_smem(G, w, c.M << c.n, c.L);
      const int bps = batch_sweep_blocks_per_sm(G, w, smem);
      const int blocks = std::max(1, std::min(ctx->num_sms * bps, (int)((u.size() + w - 1) / w)));
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {  // the first run warms up
        CK(cudaMemsetAsync(queue_dev, 0, sizeof(int), st));
        CK(cudaEventRecord(e0, st));
        launch_batch_sweep(G, t, units_dev, (int)u.size(), queue_dev, blocks, w, batch_region_f2(G, c.M << c.n, c.L),
                           st);
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        CK(cudaGetLastError());
        float r = 0.f;
        CK(cudaEventElapsedTime(&r, e0, e1));
        if (rep) ms = std::min(ms, r);
      }
      const float per = (float)(1e6 * ms / start_sweeps);  // ns per start-sweep
      ctx->batch_trial_shape.push_back({c.n, c.L, c.M, a.S, G, w});
      ctx->batch_trial_ns.push_back(per);
      if (G == 32 && per < best32) {
        best32 = per;
        w32 = w;
      }
      if (per < best) {
        best = per;
        c.G = G;
        c.warps = w;
      }
    }
    if (w32 && c.G != 32 && best > 0.95f * best32) {
      c.G = 32;
      c.warps = w32;
    }
    ctx->batch_tuned.push_back({key, {c.G, c.warps}});
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return QFS_OK;
}

uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ULL;
  }
  return h;
}

// fn(0 .. n-1) over the host cores (at most 16 threads); the draws it runs
// are pure functions of their index writing disjoint ranges.
template <class F>
void host_parallel_for(int n, F fn) {
  const int hw = (int)std::thread::hardware_concurrency();
  const int T = std::max(1, std::min({hw > 0 ? hw : 1, 16, n / 64}));
  if (T <= 1) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t)
    th.emplace_back([&, t] {
      for (int i = t; i < n; i += T) fn(i);
    });
  for (auto& x : th) x.join();
}

int batch_common(qfs_ctx* ctx, int32_t P, const int32_t* ns, const int32_t* Ls, const int32_t* pairs,
                 const BatchInputs& in, const qfs_params* p, qfs_result* results) {
  const bool any_dev = in.targets_dev || in.samples_dev || in.gates_dev || in.out_dev;
  if (P < 1) return fail(QFS_EINVAL, "P = %d: need >= 1", P);
  if (!ns || !Ls || !pairs || !in.targets || !p || (!in.sweep_once && (!in.gates_out || !results)))
    return fail(QFS_EINVAL, "ns, Ls, pairs, targets, params, gates_out and results must be given");
  if (in.sweep_once && (!in.samples || !in.init_gates || !in.start_gates_out))
    return fail(QFS_EINVAL, "one batched sweep needs samples, init_gates and gates_out");
  const int S = p->multistarts;
  if (S < 1 || S > 64) return fail(QFS_EUNSUPPORTED, "multistarts = %d: the batched form takes 1..64", S);
  if (p->max_sweeps < 1) return fail(QFS_EINVAL, "max_sweeps = %d: need >= 1", p->max_sweeps);
  if (!(p->dist_tol >= 0.0)) return fail(QFS_EINVAL, "dist_tol = %g", p->dist_tol);
  if (p->beta != 0.0) return fail(QFS_EUNSUPPORTED, "the batched form runs beta = 0 only");
  if (p->training_distribution != QFS_STATES_HAAR && p->training_distribution != QFS_STATES_BASIS)
    return fail(QFS_EINVAL, "training_distribution = %d: need QFS_STATES_HAAR or QFS_STATES_BASIS",
                p->training_distribution);
  std::vector<BatchProblem> probs(P);
  long long pair_off = 0, state_off = 0, target_off = 0, gate_off = 0, gout_off = 0;
  int max_elems = 0, max_L = 0;
  for (int i = 0; i < P; ++i) {
    const int n = ns[i], L = Ls[i];
    if (n < 2 || n > 6) return fail(QFS_EUNSUPPORTED, "problem %d: n = %d (batched form: 2..6)", i, n);
    if (L < 1 || L > 32) return fail(QFS_EUNSUPPORTED, "problem %d: L = %d (batched form: 1..32)", i, L);
    const int N = 1 << n;
    int M = p->M > 0 ? std::min(p->M, N) : N / 2;
    if (M * N > 1024) return fail(QFS_EUNSUPPORTED, "problem %d: N*M = %d > 1024", i, M * N);
    qfs_circuit c{n, L, pairs + pair_off};
    TRY(check_circuit(&c));
    probs[i] = BatchProblem{n, L, M, (int)pair_off, state_off, target_off, gate_off, gout_off};
    pair_off += 2 * L;
    state_off += (long long)N * M;
    target_off += (long long)N * N;
    gate_off += (long long)S * L * 16;
    gout_off += (long long)L * 16;
    max_elems = std::max(max_elems, N * M);
    max_L = std::max(max_L, L);
  }
  TRY(ctx_check(ctx));
  TRY(set_device(ctx));
  // Problem classes (n, L, M) in order of first appearance.
  std::vector<BatchClass> classes;
  {
    std::vector<std::pair<long long, int>> seen;
    for (int i = 0; i < P; ++i) {
      const long long key = batch_class_key(probs[i].n, probs[i].L, probs[i].M, S, false);
      int ci = -1;
      for (auto& kv : seen)
        if (kv.first == key) ci = kv.second;
      if (ci < 0) {
        ci = (int)classes.size();
        seen.push_back({key, ci});
        classes.push_back(BatchClass{probs[i].n, probs[i].L, probs[i].M, {}});
      }
      classes[ci].problems.push_back(i);
    }
  }
  // Workspace.
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align_up(bytes);
    return o;
  };
  // Unit lists: a batch needs at most P * S; the autotuner's trials up to 16384.
  const long long max_units = std::max<long long>((long long)P * S, 16384);
  const size_t o_probs = take(sizeof(BatchProblem) * P), o_units = take(sizeof(BatchUnit) * max_units),
               o_pairs = take(sizeof(int) * pair_off), o_tgt = take(sizeof(double2) * target_off),
               o_psi64 = take(sizeof(double2) * state_off), o_phil64 = take(sizeof(double2) * state_off),
               o_psi32 = take(sizeof(float2) * state_off), o_phil32 = take(sizeof(float2) * state_off),
               o_g0 = take(sizeof(double2) * gate_off), o_g32 = take(sizeof(float2) * gate_off),
               o_conv = take(sizeof(int) * P * S), o_cost = take(sizeof(double) * P * S),
               o_swr = take(sizeof(int) * P * S), o_sstar = take(sizeof(int) * P), o_q = take(sizeof(int) * 64),
               o_gout = take(sizeof(double2) * gout_off), o_rc = take(sizeof(double) * P),
               o_rs = take(sizeof(int) * P), o_rb = take(sizeof(int) * P), o_rr = take(sizeof(int) * P);
  TRY(ensure_ws(ctx, off));
  char* w = ctx->ws;
  cudaStream_t st = ctx->stream;
  BatchArgs a{};
  a.probs = reinterpret_cast<BatchProblem*>(w + o_probs);
  a.P = P;
  a.S = S;
  a.targets = reinterpret_cast<double2*>(w + o_tgt);
  a.psi64 = reinterpret_cast<double2*>(w + o_psi64);
  a.phil64 = reinterpret_cast<double2*>(w + o_phil64);
  a.psi32 = reinterpret_cast<float2*>(w + o_psi32);
  a.phil32 = reinterpret_cast<float2*>(w + o_phil32);
  a.pairs = reinterpret_cast<int*>(w + o_pairs);
  a.init_gates = reinterpret_cast<double2*>(w + o_g0);
  a.gates32 = reinterpret_cast<float2*>(w + o_g32);
  a.conv_sweep = reinterpret_cast<int*>(w + o_conv);
  a.final_cost = reinterpret_cast<double*>(w + o_cost);
  a.sweeps_run = reinterpret_cast<int*>(w + o_swr);
  a.s_star = reinterpret_cast<int*>(w + o_sstar);
  a.queue = reinterpret_cast<int*>(w + o_q);
  a.order = nullptr;
  a.max_sweeps = in.sweep_once ? 1 : p->max_sweeps;
  a.tol = in.sweep_once ? -1.0 : p->dist_tol;
  a.plateau_window = in.sweep_once ? 0 : p->plateau_window;
  a.diff_tol_r = p->diff_tol_r;
  a.min_sweeps = p->min_sweeps;
  a.max_elems = max_elems;
  a.max_L = max_L;
  a.gates_out = reinterpret_cast<double2*>(w + o_gout);
  a.res_cost = reinterpret_cast<double*>(w + o_rc);
  a.res_sweeps = reinterpret_cast<int*>(w + o_rs);
  a.res_best = reinterpret_cast<int*>(w + o_rb);
  a.res_refine = reinterpret_cast<int*>(w + o_rr);
  a.refine_max = std::max(0, p->refine_sweeps_max);
  a.refine_unconverged = 0;
  BatchUnit* units_dev = reinterpret_cast<BatchUnit*>(w + o_units);
  const cudaMemcpyKind t_kind = in.targets_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind s_kind = in.samples_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind g_kind = in.gates_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(w + o_probs, probs.data(), sizeof(BatchProblem) * P, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(w + o_pairs, pairs, sizeof(int) * pair_off, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(w + o_tgt, in.targets, sizeof(double2) * target_off, t_kind, st));
  // Training states and initial gates: given, or drawn per problem from
  // seed + problem index (or seed + draw_index[i]; the library's Philox draws).
  auto draw_seed = [&](int i) { return p->seed + (uint64_t)(in.draw_index ? in.draw_index[i] : i); };
  // Draws go into the context's pinned buffer (reused across calls; any
  // copy still reading it has finished once the stream is idle).
  const size_t need = (in.samples ? 0 : (size_t)state_off) + (in.init_gates ? 0 : (size_t)gate_off);
  std::complex<double>* hbuf = nullptr;
  if (need) {
    CK(cudaStreamSynchronize(st));
    if (ctx->h_draw_cap < need) {
      if (ctx->h_draw) CK(cudaFreeHost(ctx->h_draw));
      ctx->h_draw = nullptr;
      ctx->h_draw_cap = 0;
      void* ptr = nullptr;
      if (cudaMallocHost(&ptr, need * sizeof(std::complex<double>)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QFS_ENOMEM, "pinned host memory for %zu drawn complex values", need);
      }
      ctx->h_draw = static_cast<std::complex<double>*>(ptr);
      ctx->h_draw_cap = need;
    }
    hbuf = ctx->h_draw;
  }
  if (in.samples) {
    CK(cudaMemcpyAsync(w + o_psi64, in.samples, sizeof(double2) * state_off, s_kind, st));
  } else {
    std::complex<double>* hs = hbuf;
    host_parallel_for(P, [&](int i) {
      draw_states(p->training_distribution, draw_seed(i), 1u, probs[i].n, probs[i].M, hs + probs[i].state_off);
    });
    CK(cudaMemcpyAsync(w + o_psi64, hs, sizeof(double2) * state_off, cudaMemcpyHostToDevice, st));
  }
  if (in.init_gates) {
    CK(cudaMemcpyAsync(w + o_g0, in.init_gates, sizeof(double2) * gate_off, g_kind, st));
  } else {
    std::complex<double>* hg = hbuf + (in.samples ? 0 : state_off);
    host_parallel_for(P, [&](int i) { generate_gates(draw_seed(i), S * probs[i].L, hg + probs[i].gate_off); });
    CK(cudaMemcpyAsync(w + o_g0, hg, sizeof(double2) * gate_off, cudaMemcpyHostToDevice, st));
  }
  (void)any_dev;
  // Schedules: forced (tests) or tuned per class.
  if (ctx->batch_force_G > 0) {
    for (BatchClass& c : classes) {
      c.G = ctx->batch_force_G;
      c.warps = 0;
      for (int wv : {4, 2, 8}) {
        const size_t smem = batch_sweep_smem(c.G, wv, c.M << c.n, c.L);
        if (smem <= 200 * 1024 && batch_sweep_blocks_per_sm(c.G, wv, smem) >= 1) {
          c.warps = wv;
          break;
        }
      }
      if (!c.warps) return fail(QFS_EUNSUPPORTED, "G = %d does not fit n = %d, L = %d", c.G, c.n, c.L);
    }
  } else {
    bool untuned = false;
    for (const BatchClass& c : classes) {
      bool f = false;
      for (auto& kv : ctx->batch_tuned) f |= kv.first == batch_class_key(c.n, c.L, c.M, S, true);
      untuned |= !f;
    }
    if (untuned) launch_batch_prep(a, st);
    TRY(autotune_batch(ctx, a, probs, classes, units_dev, a.queue, max_units));
  }
  // Builds (or finds in the cache) and launches the graph of one plan: the
  // classes with the same G share one persistent launch over their units,
  // heaviest first.
  auto launch_plan = [&](const std::vector<BatchClass>& classes) -> int {
    struct Launch {
      int G, warps, unit0, nunits, region;
    };
    std::vector<Launch> launches;
    std::vector<BatchUnit> units;
    {
      std::vector<int> shapes;
      for (const BatchClass& c : classes)
        if (std::find(shapes.begin(), shapes.end(), c.G) == shapes.end()) shapes.push_back(c.G);
      for (int G : shapes) {
        std::vector<int> idx;
        int region = 0;
        for (const BatchClass& c : classes)
          if (c.G == G) {
            idx.insert(idx.end(), c.problems.begin(), c.problems.end());
            region = std::max(region, batch_region_f2(G, c.M << c.n, c.L));
          }
        const int wv = batch_warps_region(G, region);
        if (!wv) return fail(QFS_EUNSUPPORTED, "no block shape fits G = %d with %d float2 per warp", G, region);
        const int u0 = (int)units.size();
        batch_units(probs, idx, S, G, units);
        launches.push_back(Launch{G, wv, u0, (int)units.size() - u0, region});
      }
    }
    // Launches start in order of their heaviest unit, heaviest first (the
    // persistent launches overlap; the heaviest units should not come last).
    {
      std::vector<int> ord(launches.size());
      for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
      auto work = [&](const Launch& L) { return batch_unit_weight(probs[units[L.unit0].p]); };
      std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return work(launches[x]) > work(launches[y]); });
      std::vector<Launch> sorted;
      for (int i : ord) sorted.push_back(launches[i]);
      launches.swap(sorted);
    }
    if ((int)launches.size() > 60) return fail(QFS_EUNSUPPORTED, "too many launch shapes (%d)", (int)launches.size());
    unsigned long long* trace = ctx->bt_trace && ctx->bt_trace_n >= 4 * units.size() ? ctx->bt_trace : nullptr;
    if (ctx->bt_trace) ctx->bt_units = trace ? (long long)units.size() : 0;
    CK(cudaMemcpyAsync(units_dev, units.data(), sizeof(BatchUnit) * units.size(), cudaMemcpyHostToDevice, st));
    // The graph: queue reset, set-up, one persistent launch per shape (on
    // parallel branches), the finishing kernel.  Replayed while the batch's
    // shape, parameters and workspace stay the same.
    uint64_t key = 1469598103934665603ULL;
    {
      const int sc[] = {P, S, a.max_sweeps, a.plateau_window, a.min_sweeps, a.refine_max, (int)in.sweep_once,
                        (int)launches.size()};
      key = fnv1a(key, sc, sizeof(sc));
      const double sd[] = {a.tol, a.diff_tol_r};
      key = fnv1a(key, sd, sizeof(sd));
      key = fnv1a(key, &w, sizeof(w));
      key = fnv1a(key, ns, sizeof(int32_t) * P);
      key = fnv1a(key, Ls, sizeof(int32_t) * P);
      key = fnv1a(key, launches.data(), sizeof(Launch) * launches.size());
      const int mm[] = {p->M, max_elems, max_L};
      key = fnv1a(key, mm, sizeof(mm));
      key = fnv1a(key, &trace, sizeof(trace));
    }
    // With per-launch timing on, the graph carries this call's event records:
    // it is captured, replayed once, harvested and dropped.
    const bool cache = !ctx->prof.on;
    qfs_ctx::BatchGraph* bg = nullptr;
    qfs_ctx::BatchGraph once;
    if (cache)
      for (auto& g : ctx->batch_graphs)
        if (g.key == key && g.exec) bg = &g;
    if (!bg) {
      if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
      TRY(ensure_group_streams(ctx, std::min<int>(kMaxGroups, (int)launches.size())));
      long long before[QFS_PROF_KINDS];
      for (int i = 0; i < QFS_PROF_KINDS; ++i) before[i] = ctx->prof.launches[i];
      cudaStream_t cs = ctx->cap_stream;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
      ctx->prof.capturing = true;
      cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int) * 64, cs);
      {
        ProfScope ps(ctx, QFS_PROF_OTHER, 0.0, cs);
        launch_batch_prep(a, cs);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ctx->fork_event, cs);
      for (size_t li = 0; li < launches.size() && e == cudaSuccess; ++li) {
        const Launch& L = launches[li];
        const size_t smem = (size_t)L.warps * L.region * sizeof(float2);
        const int bps = std::max(1, batch_sweep_blocks_per_sm(L.G, L.warps, smem));
        const int blocks = std::max(1, std::min(ctx->num_sms * bps, (L.nunits + L.warps - 1) / L.warps));
        const int gs = (int)(li % kMaxGroups);
        cudaStream_t ls = li == 0 ? cs : ctx->gstream[gs];
        if (li > 0) e = cudaStreamWaitEvent(ls, ctx->fork_event, 0);
        if (e != cudaSuccess) break;
        {
          ProfScope ps(ctx, QFS_PROF_BATCH, 0.0, ls);
          BatchArgs al = a;
          al.unit_trace = trace ? trace + 4 * (size_t)L.unit0 : nullptr;
          launch_batch_sweep(L.G, al, units_dev + L.unit0, L.nunits, a.queue + li, blocks, L.warps, L.region, ls);
        }
        if (li > 0) {
          e = cudaEventRecord(ctx->gevent[gs], ls);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->gevent[gs], 0);
        }
      }
      if (!in.sweep_once) {
        ProfScope ps(ctx, QFS_PROF_CHECK, 0.0, cs);
        launch_batch_finalize(a, cs);
      }
      ctx->prof.capturing = false;
      cudaGraph_t graph = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = e2;
      qfs_ctx::BatchGraph ng;
      ng.key = key;
      for (int i = 0; i < QFS_PROF_KINDS; ++i) {
        ng.launches[i] = ctx->prof.launches[i] - before[i];
        ctx->prof.launches[i] = before[i];
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ng.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        if (ng.exec) cudaGraphExecDestroy(ng.exec);
        prof_release_graph(ctx);
        CK(e);
      }
      if (cache) {
        if (ctx->batch_graphs.size() >= 4) {
          cudaGraphExecDestroy(ctx->batch_graphs.front().exec);
          ctx->batch_graphs.erase(ctx->batch_graphs.begin());
        }
        ctx->batch_graphs.push_back(ng);
        bg = &ctx->batch_graphs.back();
      } else {
        once = ng;
        bg = &once;
      }
    }
    const cudaError_t el = cudaGraphLaunch(bg->exec, st);
    for (int i = 0; i < QFS_PROF_KINDS; ++i) ctx->prof.launches[i] += bg->launches[i];
    if (!cache) {
      const cudaError_t es = cudaStreamSynchronize(st);
      if (el == cudaSuccess && es == cudaSuccess) prof_harvest_graph(ctx);
      prof_release_graph(ctx);
      cudaGraphExecDestroy(once.exec);
      CK(el);
      CK(es);
    }
    CK(el);
    return QFS_OK;
  };

  // Plans: the per-class shapes; every class with one start per warp; every
  // class that admits it with 16 lanes per start.  The autotuner's per-class
  // trials measure throughput at full occupancy over a few sweeps, but a
  // batch's makespan is set by the starts that run long (a problem that does
  // not converge runs all of them to max_sweeps), and their latency per
  // sweep depends on the schedule and on what shares the SM with them.  So
  // the first call of a class mix times the plans on the batch itself and
  // keeps the fastest (cached per class mix).
  bool mixed = false;
  for (const BatchClass& c : classes) mixed |= c.G != 32;
  if (mixed && ctx->batch_force_G == 0) {
    std::vector<BatchClass> plans[3] = {classes, classes, classes};
    for (BatchClass& c : plans[1]) c.G = 32;
    bool all16_differs = false;
    for (BatchClass& c : plans[2]) {
      c.G = 32;
      for (auto [G, wv] : batch_candidates(c.n, c.M, c.L, S, true))
        if (G == 16) c.G = 16;
    }
    for (size_t i = 0; i < classes.size(); ++i) all16_differs |= plans[2][i].G != classes[i].G;
    // The decision is kept per class mix (the set of classes and their
    // shares of the batch, in tenths) and run parameters, so batches of the
    // same composition but another size reuse it.
    uint64_t pk = 1469598103934665603ULL;
    {
      const int sc[] = {S, a.max_sweeps, a.plateau_window, a.min_sweeps};
      pk = fnv1a(pk, sc, sizeof(sc));
      std::vector<std::pair<long long, int>> mix;
      for (const BatchClass& c : classes)
        mix.push_back({batch_class_key(c.n, c.L, c.M, S, true), (int)(10 * c.problems.size() / P)});
      std::sort(mix.begin(), mix.end());
      for (auto& m : mix) {  // field by field: a pair's padding bytes are indeterminate
        pk = fnv1a(pk, &m.first, sizeof(m.first));
        pk = fnv1a(pk, &m.second, sizeof(m.second));
      }
      const double sd[] = {a.tol, a.diff_tol_r};
      pk = fnv1a(pk, sd, sizeof(sd));
    }
    int choice = -1;
    for (auto& kv : ctx->batch_plans)
      if (kv.first == pk) choice = kv.second;
    if (choice < 0) {
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      // A batch's makespan varies by a few percent from run to run (which
      // warp takes a long-running unit when), so each plan is timed three
      // times, interleaved, and its median decides.
      std::array<float, 3> ms = {-1.f, -1.f, -1.f};
      float runs[3][3] = {};
      for (int rep = 0; rep < 3; ++rep)
        for (int k = 0; k < 3; ++k) {
          if (k == 2 && !all16_differs) continue;
          CK(cudaEventRecord(e0, st));
          const int rc = launch_plan(plans[k]);
          if (rc != QFS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc;
          }
          CK(cudaEventRecord(e1, st));
          CK(cudaEventSynchronize(e1));
          CK(cudaEventElapsedTime(&runs[k][rep], e0, e1));
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      for (int k = 0; k < 3; ++k) {
        if (k == 2 && !all16_differs) continue;
        std::sort(runs[k], runs[k] + 3);
        ms[k] = runs[k][1];
      }
      choice = 0;
      for (int k = 1; k < 3; ++k)
        if (ms[k] >= 0.f && ms[k] < ms[choice]) choice = k;
      ctx->batch_plans.push_back({pk, choice});
      ctx->batch_plan_ms.push_back(ms);
    }
    classes = plans[choice];
  }
  TRY(launch_plan(classes));
  if (in.sweep_once) {
    std::vector<float2> g32(gate_off);
    std::vector<double> fc((size_t)P * S);
    CK(cudaMemcpyAsync(g32.data(), a.gates32, sizeof(float2) * gate_off, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(fc.data(), a.final_cost, sizeof(double) * P * S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (long long i = 0; i < gate_off; ++i) {
      in.start_gates_out[2 * i] = g32[i].x;
      in.start_gates_out[2 * i + 1] = g32[i].y;
    }
    if (in.start_costs_out) std::copy(fc.begin(), fc.end(), in.start_costs_out);
    return QFS_OK;
  }
  std::vector<double> rc(P);
  std::vector<int> rs(P), rb(P), rr(P);
  CK(cudaMemcpyAsync(in.gates_out, a.gates_out, sizeof(double2) * gout_off,
                     in.out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rc.data(), a.res_cost, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rs.data(), a.res_sweeps, sizeof(int) * P, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rb.data(), a.res_best, sizeof(int) * P, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rr.data(), a.res_refine, sizeof(int) * P, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < P; ++i) {
    results[i].cost = rc[i];
    results[i].sweeps = rs[i];
    results[i].converged = rc[i] <= p->dist_tol;
    results[i].best_start = rb[i];
    results[i].fp64_sweeps = rr[i];
    results[i].training_states = probs[i].M;
  }
  return QFS_OK;
}

}  // namespace

// A large batch with library-drawn inputs in two halves: the host draws of
// the second half (training states from seed + i, stream 1; initial gates
// from seed + i, into pinned buffers of the context) run on a helper thread
// while the first half sweeps.  The draws are those batch_common would make,
// so each problem's inputs are unchanged.
int batch_seeded_halves(qfs_ctx* ctx, int32_t P, const int32_t* ns, const int32_t* Ls, const int32_t* pairs,
                        const double* targets, const qfs_params* p, double* gates_out, qfs_result* results) {
  const int S = p->multistarts;
  std::vector<long long> toff(P + 1, 0), poff(P + 1, 0), goff(P + 1, 0), soff(P + 1, 0), ioff(P + 1, 0);
  for (int i = 0; i < P; ++i) {
    const int n = ns[i], L = Ls[i];
    const long long N = 1LL << n;
    const long long M = p->M > 0 ? std::min<long long>(p->M, N) : N / 2;
    toff[i + 1] = toff[i] + N * N;
    poff[i + 1] = poff[i] + 2LL * L;
    goff[i + 1] = goff[i] + 16LL * L;
    soff[i + 1] = soff[i] + N * M;
    ioff[i + 1] = ioff[i] + 16LL * S * L;
  }
  auto lo = [&](int k) { return k == 0 ? 0 : k == 1 ? P / 2 : P; };
  TRY(ctx_check(ctx));
  TRY(set_device(ctx));
  CK(cudaStreamSynchronize(ctx->stream));  // no copy of an earlier call still reads the buffers
  for (int k = 0; k < 2; ++k) {
    const size_t need = (size_t)(soff[lo(k + 1)] - soff[lo(k)] + ioff[lo(k + 1)] - ioff[lo(k)]);
    if (ctx->h_half_cap[k] < need) {
      if (ctx->h_half[k]) CK(cudaFreeHost(ctx->h_half[k]));
      ctx->h_half[k] = nullptr;
      ctx->h_half_cap[k] = 0;
      void* ptr = nullptr;
      if (cudaMallocHost(&ptr, need * sizeof(std::complex<double>)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QFS_ENOMEM, "pinned host memory for %zu drawn complex values", need);
      }
      ctx->h_half[k] = static_cast<std::complex<double>*>(ptr);
      ctx->h_half_cap[k] = need;
    }
  }
  // Half k's states, then its gates, in h_half[k].
  auto draw = [&](int k) {
    const int a = lo(k), b = lo(k + 1);
    std::complex<double>* states = ctx->h_half[k];
    std::complex<double>* gates = states + (soff[b] - soff[a]);
    host_parallel_for(b - a, [&](int j) {
      const int i = a + j;
      const int n = ns[i];
      const int N = 1 << n;
      const int M = p->M > 0 ? std::min(p->M, N) : N / 2;
      draw_states(p->training_distribution, p->seed + (uint64_t)i, 1u, n, M, states + (soff[i] - soff[a]));
      generate_gates(p->seed + (uint64_t)i, S * Ls[i], gates + (ioff[i] - ioff[a]));
    });
  };
  auto run = [&](int k) {
    const int a = lo(k), b = lo(k + 1);
    BatchInputs in;
    in.targets = targets + 2 * toff[a];
    in.samples = reinterpret_cast<const double*>(ctx->h_half[k]);
    in.init_gates = reinterpret_cast<const double*>(ctx->h_half[k] + (soff[b] - soff[a]));
    in.gates_out = gates_out + 2 * goff[a];
    return batch_common(ctx, b - a, ns + a, Ls + a, pairs + poff[a], in, p, results + a);
  };
  try {
    draw(0);
    std::future<void> f1 = std::async(std::launch::async, draw, 1);
    const int r0 = run(0);
    f1.get();  // joined before any return
    TRY(r0);
    return run(1);
  } catch (const std::exception& e) {
    return fail(QFS_EINTERNAL, "host draw threads: %s", e.what());
  }
}

extern "C" int qfs_instantiate_batch(qfs_ctx* ctx, int32_t P, const int32_t* ns, const int32_t* Ls,
                                     const int32_t* pairs, const double* targets,
                                     const double* samples, const double* init_gates,
                                     const qfs_params* p, double* gates_out, qfs_result* results) {
  g_err.clear();
  if (!samples && !init_gates && P >= 16384 && ns && Ls && pairs && targets && p && gates_out && results) {
    bool sized = p->multistarts >= 1 && p->multistarts <= 64 &&
                 (p->training_distribution == QFS_STATES_HAAR || p->training_distribution == QFS_STATES_BASIS);
    for (int i = 0; i < P && sized; ++i) sized = ns[i] >= 2 && ns[i] <= 6 && Ls[i] >= 1 && Ls[i] <= 32;
    if (sized) return batch_seeded_halves(ctx, P, ns, Ls, pairs, targets, p, gates_out, results);
  }
  BatchInputs in;
  in.targets = targets;
  in.samples = samples;
  in.init_gates = init_gates;
  in.gates_out = gates_out;
  return batch_common(ctx, P, ns, Ls, pairs, in, p, results);
}

extern "C" int qfs_instantiate_batch_dev(qfs_ctx* ctx, int32_t P, const int32_t* ns, const int32_t* Ls,
                                         const int32_t* pairs, const double* targets_dev,
                                         const double* samples_dev, const double* init_gates_dev,
                                         const qfs_params* p, double* gates_out_dev, qfs_result* results) {
  g_err.clear();
  if (!samples_dev || !init_gates_dev) return fail(QFS_EINVAL, "the device-pointer batch needs samples and init_gates");
  BatchInputs in;
  in.targets = targets_dev;
  in.targets_dev = true;
  in.samples = samples_dev;
  in.samples_dev = true;
  in.init_gates = init_gates_dev;
  in.gates_dev = true;
  in.gates_out = gates_out_dev;
  in.out_dev = true;
  return batch_common(ctx, P, ns, Ls, pairs, in, p, results);
}

extern "C" int qfs_batch_schedules(qfs_ctx* ctx, int32_t cap, int32_t* tuned, int32_t* n_tuned, int32_t* trials,
                                   double* trial_ns, int32_t* n_trials, int32_t* plan_choice, double* plan_ms,
                                   int32_t* n_plans) {
  g_err.clear();
  TRY(ctx_check(ctx));
  if (n_plans) *n_plans = (int32_t)ctx->batch_plans.size();
  for (int i = 0; i < cap && i < (int)ctx->batch_plans.size(); ++i) {
    if (plan_choice) plan_choice[i] = ctx->batch_plans[i].second;
    if (plan_ms)
      for (int k = 0; k < 3; ++k) plan_ms[3 * i + k] = ctx->batch_plan_ms[i][k];
  }
  if (n_tuned) *n_tuned = (int32_t)ctx->batch_tuned.size();
  if (n_trials) *n_trials = (int32_t)ctx->batch_trial_ns.size();
  for (int i = 0; tuned && i < cap && i < (int)ctx->batch_tuned.size(); ++i) {
    const long long k = ctx->batch_tuned[i].first / 2;
    const int S = (int)(k % 128), M = (int)((k / 128) % 4096), L = (int)((k / 128 / 4096) % 64),
              n = (int)(k / 128 / 4096 / 64);
    const int v[6] = {n, L, M, S, ctx->batch_tuned[i].second.first, ctx->batch_tuned[i].second.second};
    std::copy(v, v + 6, tuned + 6 * i);
  }
  for (int i = 0; trials && i < cap && i < (int)ctx->batch_trial_ns.size(); ++i) {
    std::copy(ctx->batch_trial_shape[i].begin(), ctx->batch_trial_shape[i].end(), trials + 6 * i);
    if (trial_ns) trial_ns[i] = ctx->batch_trial_ns[i];
  }
  return QFS_OK;
}

extern "C" int qfs_batch_sweep_once(qfs_ctx* ctx, int32_t P, const int32_t* ns, const int32_t* Ls,
                                    const int32_t* pairs, const double* targets, const double* samples,
                                    int32_t M, int32_t S, const double* gates_in, int32_t lanes_per_start,
                                    double* gates_out, double* costs_out) {
  g_err.clear();
  TRY(ctx_check(ctx));
  if (lanes_per_start != 0 && lanes_per_start != 4 && lanes_per_start != 8 && lanes_per_start != 16 &&
      lanes_per_start != 32)
    return fail(QFS_EINVAL, "lanes_per_start = %d: need 0, 4, 8, 16 or 32", lanes_per_start);
  qfs_params prm;
  qfs_default_params(&prm);
  prm.M = M;
  prm.multistarts = S;
  prm.max_sweeps = 1;
  BatchInputs in;
  in.targets = targets;
  in.samples = samples;
  in.init_gates = gates_in;
  in.sweep_once = true;
  in.start_gates_out = gates_out;
  in.start_costs_out = costs_out;
  const int old = ctx->batch_force_G;
  ctx->batch_force_G = lanes_per_start;
  const int rc = batch_common(ctx, P, ns, Ls, pairs, in, &prm, nullptr);
  ctx->batch_force_G = old;
  return rc;
}

// ---------------------------------------------------------------------------
// Learned warm start: tensor-core GEMM entry point.

extern "C" int qfs_gemm_bf16_dev(qfs_ctx* ctx, int32_t M, int32_t N, int32_t K, const void* A, int32_t lda,
                                 const void* B, int32_t ldb, float* C32, void* C16, int32_t ldc,
                                 const float* bias, int32_t gelu, int32_t M_valid) {
  g_err.clear();
  if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64)
    return fail(QFS_EINVAL, "M, N multiples of 128 and K of 64 needed (M=%d N=%d K=%d)", M, N, K);
  if (lda % 8 || ldb % 8 || lda < K || ldb < K || ldc < N)
    return fail(QFS_EINVAL, "lda, ldb >= K and multiples of 8, ldc >= N needed");
  if (!A || !B || (!C32 && !C16)) return fail(QFS_EINVAL, "A, B and an output must be given");
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C32) |
       reinterpret_cast<uintptr_t>(C16) | reinterpret_cast<uintptr_t>(bias)) & 15)
    return fail(QFS_EINVAL, "A, B, C32, C16 and bias must be 16-byte aligned");
  if (ldc % 8) return fail(QFS_EINVAL, "ldc must be a multiple of 8");
  TRY(ctx_check(ctx));
  TRY(set_device(ctx));
  TRY(ensure_ws(ctx, 256));
  int* err = reinterpret_cast<int*>(ctx->ws);
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  GemmArgs g{reinterpret_cast<const __nv_bfloat16*>(A), lda, reinterpret_cast<const __nv_bfloat16*>(B), ldb,
             C32, reinterpret_cast<__nv_bfloat16*>(C16), ldc, bias, gelu, M, N, K,
             M_valid > 0 ? M_valid : M, err};
  g.splitk = gemm_splitk_for(g, ctx->num_sms > 0 ? ctx->num_sms : 148);
  {
    ProfScope ps(ctx, QFS_PROF_MLP, 2.0 * M * N * K, st);
    CK(launch_gemm_bf16_tc(g, st));
  }
  CK(cudaGetLastError());
  int h = 0;
  CK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  prof_harvest(ctx);
  if (h) return fail(QFS_ETIMEOUT, "a bounded tensor-core wait ran out");
  return QFS_OK;
}

// ---------------------------------------------------------------------------
// Learned warm start: a multilayer perceptron mapping the target applied to
// eight fixed states of a 4-qubit block (16 x 8 complex = 256 reals) through
// three hidden layers of 1024 (GELU) to 6 gates (192 reals), trained on
// (target, converged gates) pairs that the method itself produces.  All
// products run on the tcgen05 GEMM; weights are FP32 masters with BF16
// copies, activations BF16, accumulation FP32, Adam on the masters.

namespace qfs {
void generate_samples(uint64_t seed, int n, int M, std::complex<double>* out);
std::complex<double> complex_normal(uint64_t seed, uint32_t stream, uint64_t index);
}

namespace {
// A normal draw with variance 1/2 (the real part of a standard complex normal).
inline double qfs_normal_re(uint64_t seed, uint32_t stream, uint64_t index) {
  return qfs::complex_normal(seed, stream, index).real();
}
}  // namespace

struct qfs_ws {
  qfs_ctx* ctx = nullptr;
  static constexpr int kLayers = 4;
  int din[kLayers] = {256, 1024, 1024, 1024};
  int dout[kLayers] = {1024, 1024, 1024, 256};  // the last 64 outputs are padding
  int n_out = 192;
  int B_cap = 0;
  long long step = 0;
  char* mem = nullptr;
  float *W[kLayers], *b[kLayers], *mW[kLayers], *vW[kLayers], *mb[kLayers], *vb[kLayers], *gW[kLayers], *gb[kLayers];
  __nv_bfloat16 *W16[kLayers], *WT16[kLayers];
  double2* phif = nullptr;      // 16 x 8 fixed states
  __nv_bfloat16* X16 = nullptr;  // B_cap x 256
  __nv_bfloat16* H16[kLayers];   // B_cap x dout
  float* Z32[kLayers];           // B_cap x dout
  float *dA32, *dB32;            // B_cap x 1024 scratch (fp32 gradients)
  __nv_bfloat16 *dA16, *dB16, *T1, *T2;  // bf16 gradient and transposes (1024 x B_cap)
  float* Tlab = nullptr;         // B_cap x 192 labels
  double* loss_part = nullptr;   // 1024
  double2* tgt = nullptr;        // B_cap x 256 complex (targets of a batch)
  double2* envs = nullptr;       // B_cap x 6 x 16 (projection scratch)
  int* err = nullptr;
  double2* pred = nullptr;       // predicted gates of a policy call (grown on demand)
  size_t pred_cap = 0;           // in problems
  // Pinned host buffers the policy draws its inputs into (grown on demand,
  // reused by later calls): stage-1 states of each half, and states and
  // random starts of each half's unconverged targets.
  static constexpr int kPinSlots = 6;
  std::complex<double>* pin[kPinSlots] = {};
  size_t pin_cap[kPinSlots] = {};
};

namespace {

long long ws_param_count(const qfs_ws* m) {
  long long c = 0;
  for (int l = 0; l < qfs_ws::kLayers; ++l) c += (long long)m->dout[l] * m->din[l] + m->dout[l];
  return c;
}

// One GEMM launch; its timing (when profiling) comes from the ProfScope the
// caller opens around the consecutive GEMMs of one pass or layer.
int ws_gemm(qfs_ws* m, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
            float* C32, __nv_bfloat16* C16, int ldc, const float* bias, int gelu, int M_valid) {
  GemmArgs g{A, lda, B, ldb, C32, C16, ldc, bias, gelu, M, N, K, M_valid, m->err};
  g.splitk = gemm_splitk_for(g, m->ctx->num_sms > 0 ? m->ctx->num_sms : 148);
  CK(launch_gemm_bf16_tc(g, m->ctx->stream));
  return QFS_OK;
}

// Forward pass on B rows (multiple of 128) of m->X16: Z32[l], H16[l].
void ws_forward(qfs_ws* m, int B) {
  const __nv_bfloat16* in = m->X16;
  double flops = 0.0;
  for (int l = 0; l < qfs_ws::kLayers; ++l) flops += 2.0 * B * m->dout[l] * m->din[l];
  ProfScope ps(m->ctx, QFS_PROF_MLP, flops, nullptr, qfs_ws::kLayers);  // four GEMMs back to back
  for (int l = 0; l < qfs_ws::kLayers; ++l) {
    const bool last = l == qfs_ws::kLayers - 1;
    ws_gemm(m, in, m->din[l], m->W16[l], m->din[l], B, m->dout[l], m->din[l], m->Z32[l], last ? nullptr : m->H16[l],
            m->dout[l], m->b[l], last ? 0 : 1, B);
    in = m->H16[l];
  }
}

// Loss and gradients for B rows (B_valid real) with labels in m->Tlab.  The
// mean loss goes to *loss (host, synchronising) and/or is added to
// *loss_acc_dev (device, asynchronous).
int ws_backward(qfs_ws* m, int B, int B_valid, double* loss, double* loss_acc_dev = nullptr) {
  cudaStream_t st = m->ctx->stream;
  const int L = qfs_ws::kLayers;
  const int nparts = launch_ws_loss_grad(m->Z32[L - 1], m->dout[L - 1], m->Tlab, m->n_out, B, B_valid, m->dA32,
                                         m->dA16, m->loss_part, st);
  float* g32 = m->dA32;
  __nv_bfloat16* g16 = m->dA16;
  for (int l = L - 1; l >= 0; --l) {
    const int N = m->dout[l], K = m->din[l];
    launch_colsum(g32, B, N, m->gb[l], st);
    launch_transpose_bf16(g16, B, N, m->T1, st);  // N x B
    const __nv_bfloat16* hin = l == 0 ? m->X16 : m->H16[l - 1];
    launch_transpose_bf16(hin, B, K, m->T2, st);  // K x B
    float* o32 = g32 == m->dA32 ? m->dB32 : m->dA32;
    __nv_bfloat16* o16 = g16 == m->dA16 ? m->dB16 : m->dA16;
    {
      // The layer's weight gradient and (below the first layer) dH = g W
      // (B x K), back to back under one pair of events.
      ProfScope ps(m->ctx, QFS_PROF_MLP, (l > 0 ? 4.0 : 2.0) * N * K * B, nullptr, l > 0 ? 2 : 1);
      TRY(ws_gemm(m, m->T1, B, m->T2, B, N, K, B, m->gW[l], nullptr, K, nullptr, 0, N));
      if (l > 0) TRY(ws_gemm(m, g16, N, m->WT16[l], N, B, K, N, o32, nullptr, K, nullptr, 0, B));
    }
    if (l > 0) {
      // dZ = dH * gelu'(Z_{l-1}).
      launch_gelu_back(o32, m->Z32[l - 1], (long long)B * K, K, B_valid, o32, o16, st);
      g32 = o32;
      g16 = o16;
    }
  }
  if (loss_acc_dev) launch_loss_accumulate(m->loss_part, nparts, 1.0 / ((double)B_valid * m->n_out), loss_acc_dev, st);
  if (loss) {
    std::vector<double> parts(nparts);
    CK(cudaMemcpyAsync(parts.data(), m->loss_part, sizeof(double) * nparts, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double x : parts) s += x;
    *loss = s / ((double)B_valid * m->n_out);
  }
  return QFS_OK;
}

void ws_refresh_bf16(qfs_ws* m) {
  cudaStream_t st = m->ctx->stream;
  for (int l = 0; l < qfs_ws::kLayers; ++l) {
    launch_cast_f32_bf16(m->W[l], m->W16[l], (long long)m->dout[l] * m->din[l], st);
    launch_transpose_bf16(m->W16[l], m->dout[l], m->din[l], m->WT16[l], st);
  }
}

// Features of `count` host targets (16 x 16 each) into m->X16 rows (B_pad).
int ws_load_features(qfs_ws* m, const double* targets, int count, int B_pad) {
  cudaStream_t st = m->ctx->stream;
  CK(cudaMemcpyAsync(m->tgt, targets, sizeof(double2) * 256 * (size_t)count, cudaMemcpyHostToDevice, st));
  launch_ws_features(m->tgt, m->phif, count, B_pad, m->X16, st);
  return QFS_OK;
}

int check_err_word(qfs_ws* m) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->ctx->stream));
  CK(cudaStreamSynchronize(m->ctx->stream));
  if (h) return fail(QFS_ETIMEOUT, "a bounded tensor-core wait ran out");
  return QFS_OK;
}

}  // namespace

extern "C" int qfs_ws_create(qfs_ctx* ctx, uint64_t seed, int32_t batch_cap, qfs_ws** out) {
  g_err.clear();
  if (!out) return fail(QFS_EINVAL, "out is NULL");
  *out = nullptr;
  if (batch_cap < 128 || batch_cap % 128) return fail(QFS_EINVAL, "batch_cap = %d: a multiple of 128 needed", batch_cap);
  TRY(ctx_check(ctx));
  TRY(set_device(ctx));
  qfs_ws* m = new qfs_ws();
  m->ctx = ctx;
  m->B_cap = batch_cap;
  const int L = qfs_ws::kLayers;
  size_t off = 0;
  std::vector<size_t> o;
  auto take = [&](size_t bytes) {
    o.push_back(off);
    off += align_up(bytes);
    return o.back();
  };
  size_t oW[L], ob[L], omW[L], ovW[L], omb[L], ovb[L], ogW[L], ogb[L], oW16[L], oWT[L], oH[L], oZ[L];
  for (int l = 0; l < L; ++l) {
    const size_t nw = (size_t)m->dout[l] * m->din[l], nb = m->dout[l];
    oW[l] = take(nw * 4); ob[l] = take(nb * 4); omW[l] = take(nw * 4); ovW[l] = take(nw * 4);
    omb[l] = take(nb * 4); ovb[l] = take(nb * 4); ogW[l] = take(nw * 4); ogb[l] = take(nb * 4);
    oW16[l] = take(nw * 2); oWT[l] = take(nw * 2);
    oH[l] = take((size_t)batch_cap * m->dout[l] * 2); oZ[l] = take((size_t)batch_cap * m->dout[l] * 4);
  }
  const size_t ophif = take(sizeof(double2) * 128), oX = take((size_t)batch_cap * 256 * 2),
               odA32 = take((size_t)batch_cap * 1024 * 4), odB32 = take((size_t)batch_cap * 1024 * 4),
               odA16 = take((size_t)batch_cap * 1024 * 2), odB16 = take((size_t)batch_cap * 1024 * 2),
               oT1 = take((size_t)batch_cap * 1024 * 2), oT2 = take((size_t)batch_cap * 1024 * 2),
               oT = take((size_t)batch_cap * 192 * 4), olp = take(1040 * sizeof(double)),
               otg = take(sizeof(double2) * 256 * (size_t)batch_cap), oenv = take(sizeof(double2) * 96 * (size_t)batch_cap),
               oerr = take(sizeof(int) * 4);
  cudaError_t e = cudaMalloc(&m->mem, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return fail(QFS_ENOMEM, "warm-start model: cannot allocate %.2f GiB", off / 1073741824.0);
  }
  char* b = m->mem;
  for (int l = 0; l < L; ++l) {
    m->W[l] = (float*)(b + oW[l]); m->b[l] = (float*)(b + ob[l]); m->mW[l] = (float*)(b + omW[l]);
    m->vW[l] = (float*)(b + ovW[l]); m->mb[l] = (float*)(b + omb[l]); m->vb[l] = (float*)(b + ovb[l]);
    m->gW[l] = (float*)(b + ogW[l]); m->gb[l] = (float*)(b + ogb[l]);
    m->W16[l] = (__nv_bfloat16*)(b + oW16[l]); m->WT16[l] = (__nv_bfloat16*)(b + oWT[l]);
    m->H16[l] = (__nv_bfloat16*)(b + oH[l]); m->Z32[l] = (float*)(b + oZ[l]);
  }
  m->phif = (double2*)(b + ophif);
  m->X16 = (__nv_bfloat16*)(b + oX);
  m->dA32 = (float*)(b + odA32); m->dB32 = (float*)(b + odB32);
  m->dA16 = (__nv_bfloat16*)(b + odA16); m->dB16 = (__nv_bfloat16*)(b + odB16);
  m->T1 = (__nv_bfloat16*)(b + oT1); m->T2 = (__nv_bfloat16*)(b + oT2);
  m->Tlab = (float*)(b + oT); m->loss_part = (double*)(b + olp);
  m->tgt = (double2*)(b + otg); m->envs = (double2*)(b + oenv); m->err = (int*)(b + oerr);
  cudaStream_t st = ctx->stream;
  // Initial weights: normal with variance 1/fan_in from Philox (stream 6);
  // the padded output rows and all biases start at zero; Adam moments zero.
  std::vector<float> h;
  for (int l = 0; l < L; ++l) {
    const size_t nw = (size_t)m->dout[l] * m->din[l];
    h.assign(nw, 0.f);
    const double sd = 1.0 / std::sqrt((double)m->din[l]);
    const int rows = l == L - 1 ? m->n_out : m->dout[l];
    for (size_t i = 0; i < (size_t)rows * m->din[l]; ++i)
      h[i] = (float)(sd * std::sqrt(2.0) * qfs_normal_re(seed, 6u, ((uint64_t)l << 40) + i));
    CK(cudaMemcpyAsync(m->W[l], h.data(), nw * 4, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(m->b[l], 0, (size_t)m->dout[l] * 4, st));
    CK(cudaMemsetAsync(m->mW[l], 0, nw * 4, st));
    CK(cudaMemsetAsync(m->vW[l], 0, nw * 4, st));
    CK(cudaMemsetAsync(m->mb[l], 0, (size_t)m->dout[l] * 4, st));
    CK(cudaMemsetAsync(m->vb[l], 0, (size_t)m->dout[l] * 4, st));
  }
  // Fixed feature states: 8 orthonormal states of 4 qubits drawn from the seed.
  std::vector<std::complex<double>> pf(128);
  qfs::generate_samples(seed ^ 0x5eedf1c5ULL, 4, 8, pf.data());
  CK(cudaMemcpyAsync(m->phif, pf.data(), sizeof(double2) * 128, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(m->err, 0, sizeof(int) * 4, st));
  ws_refresh_bf16(m);
  CK(cudaStreamSynchronize(st));
  *out = m;
  return QFS_OK;
}

extern "C" void qfs_ws_destroy(qfs_ws* m) {
  if (!m) return;
  cudaSetDevice(m->ctx->device);
  cudaStreamSynchronize(m->ctx->stream);
  cudaFree(m->mem);
  if (m->pred) cudaFree(m->pred);
  for (int i = 0; i < qfs_ws::kPinSlots; ++i)
    if (m->pin[i]) cudaFreeHost(m->pin[i]);
  delete m;
}

extern "C" int qfs_ws_params(qfs_ws* m, float* out, const float* in, int64_t* count) {
  g_err.clear();
  if (!m) return fail(QFS_EINVAL, "model is NULL");
  const long long n = ws_param_count(m);
  if (count) *count = n;
  TRY(set_device(m->ctx));
  cudaStream_t st = m->ctx->stream;
  long long off = 0;
  for (int l = 0; l < qfs_ws::kLayers; ++l) {
    const size_t nw = (size_t)m->dout[l] * m->din[l], nb = m->dout[l];
    if (out) {
      CK(cudaMemcpyAsync(out + off, m->W[l], nw * 4, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(out + off + nw, m->b[l], nb * 4, cudaMemcpyDeviceToHost, st));
    }
    if (in) {
      CK(cudaMemcpyAsync(m->W[l], in + off, nw * 4, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(m->b[l], in + off + nw, nb * 4, cudaMemcpyHostToDevice, st));
    }
    off += nw + nb;
  }
  if (in) ws_refresh_bf16(m);
  CK(cudaStreamSynchronize(st));
  return QFS_OK;
}

extern "C" int qfs_ws_loss_grad(qfs_ws* m, int32_t count, const double* targets, const double* labels,
                                double* loss, float* grads_out) {
  g_err.clear();
  if (!m || !targets || !labels) return fail(QFS_EINVAL, "model, targets and labels must be given");
  if (count < 1 || count > m->B_cap) return fail(QFS_EINVAL, "count = %d: 1..%d", count, m->B_cap);
  TRY(set_device(m->ctx));
  cudaStream_t st = m->ctx->stream;
  const int B = (count + 127) / 128 * 128;
  TRY(ws_load_features(m, targets, count, B));
  std::vector<float> t((size_t)count * 192);
  for (size_t i = 0; i < t.size(); ++i) t[i] = (float)labels[i];
  CK(cudaMemcpyAsync(m->Tlab, t.data(), t.size() * 4, cudaMemcpyHostToDevice, st));
  ws_forward(m, B);
  TRY(ws_backward(m, B, count, loss));
  if (grads_out) {
    long long off = 0;
    for (int l = 0; l < qfs_ws::kLayers; ++l) {
      const size_t nw = (size_t)m->dout[l] * m->din[l], nb = m->dout[l];
      CK(cudaMemcpyAsync(grads_out + off, m->gW[l], nw * 4, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(grads_out + off + nw, m->gb[l], nb * 4, cudaMemcpyDeviceToHost, st));
      off += nw + nb;
    }
  }
  CK(cudaStreamSynchronize(st));
  return check_err_word(m);
}

extern "C" int qfs_ws_train(qfs_ws* m, int32_t count, const double* targets, const double* labels, int32_t epochs,
                            int32_t batch, double lr, double lr_final, uint64_t shuffle_seed, double* epoch_loss) {
  g_err.clear();
  if (!m || !targets || !labels) return fail(QFS_EINVAL, "model, targets and labels must be given");
  if (count < 1 || epochs < 1) return fail(QFS_EINVAL, "count and epochs must be >= 1");
  if (batch < 128 || batch % 128 || batch > m->B_cap)
    return fail(QFS_EINVAL, "batch = %d: a multiple of 128 up to %d", batch, m->B_cap);
  if (!(lr > 0.0) || !(lr_final >= 0.0)) return fail(QFS_EINVAL, "lr must be > 0 and lr_final >= 0");
  TRY(set_device(m->ctx));
  cudaStream_t st = m->ctx->stream;
  const long long steps_total = (long long)epochs * ((count + batch - 1) / batch);
  // The whole training set stays on the device: features (bf16, count x
  // 256) computed once, labels (fp32, count x 192), and the shuffled order.
  __nv_bfloat16* Xall = nullptr;
  float* Tall = nullptr;
  int* didx = nullptr;
  auto release = [&]() {
    if (Xall) cudaFree(Xall);
    if (Tall) cudaFree(Tall);
    if (didx) cudaFree(didx);
  };
  if (cudaMalloc(&Xall, (size_t)count * 256 * 2) != cudaSuccess ||
      cudaMalloc(&Tall, (size_t)count * 192 * 4) != cudaSuccess ||
      cudaMalloc(&didx, (size_t)count * 4) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(QFS_ENOMEM, "training set of %d samples does not fit on the device", count);
  }
  int rc = QFS_OK;
  {
    std::vector<float> lb((size_t)m->B_cap * 192);
    for (int s0 = 0; s0 < count && rc == QFS_OK; s0 += m->B_cap) {
      const int bv = std::min(m->B_cap, count - s0);
      if (cudaMemcpyAsync(m->tgt, targets + (size_t)s0 * 512, sizeof(double2) * 256 * (size_t)bv,
                          cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = fail(QFS_ECUDA, "copy of targets failed");
      launch_ws_features(m->tgt, m->phif, bv, bv, Xall + (size_t)s0 * 256, st);
      for (size_t i = 0; i < (size_t)bv * 192; ++i) lb[i] = (float)labels[(size_t)s0 * 192 + i];
      if (cudaMemcpyAsync(Tall + (size_t)s0 * 192, lb.data(), sizeof(float) * 192 * (size_t)bv,
                          cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = fail(QFS_ECUDA, "copy of labels failed");
      cudaStreamSynchronize(st);
    }
  }
  std::vector<int> idx(count);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  // The step's Adam values (lr with cosine decay from lr to lr_final over
  // this call's steps, bias corrections) for every step of the call, and two
  // device counters (step within the epoch, step of the call): every
  // full-batch step is then the same work, captured once as a graph and
  // replayed (no host launch work per step).
  float* sched = nullptr;
  int* counters = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long graph_launches[QFS_PROF_KINDS] = {};
  auto release_train = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (sched) cudaFree(sched);
    if (counters) cudaFree(counters);
    prof_release_graph(m->ctx);
  };
  if (rc == QFS_OK) {
    std::vector<float> hs((size_t)steps_total * 3);
    for (long long k = 0; k < steps_total; ++k) {
      const float t = (float)(m->step + 1 + k);
      const double frac = steps_total > 1 ? (double)k / (double)(steps_total - 1) : 0.0;
      hs[3 * k] = (float)(lr_final + 0.5 * (lr - lr_final) * (1.0 + std::cos(3.141592653589793 * frac)));
      hs[3 * k + 1] = 1.f - std::pow(b1, t);
      hs[3 * k + 2] = 1.f - std::pow(b2, t);
    }
    if (cudaMalloc(&sched, sizeof(float) * hs.size()) != cudaSuccess ||
        cudaMalloc(&counters, 2 * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(QFS_ENOMEM, "training schedule does not fit on the device");
    } else if (cudaMemcpyAsync(sched, hs.data(), sizeof(float) * hs.size(), cudaMemcpyHostToDevice, st) !=
                   cudaSuccess ||
               cudaMemsetAsync(counters, 0, 2 * sizeof(int), st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess) {
      rc = fail(QFS_ECUDA, "upload of the training schedule failed");
    }
  }
  int* jstep = counters;
  int* gstep = counters ? counters + 1 : nullptr;
  double* ep_acc = m->loss_part + 1032;  // the epoch's loss, summed on the device
  // One training step on the context's stream: gather, forward, backward,
  // Adam with the device schedule, refreshed bf16 weights, counters advanced.
  auto run_step = [&](int bv, int B) -> int {
    cudaStream_t s = m->ctx->stream;
    launch_ws_gather(Xall, Tall, didx, bv, B, m->X16, m->Tlab, s, jstep, batch);
    ws_forward(m, B);
    TRY(ws_backward(m, B, bv, nullptr, ep_acc));
    for (int k = 0; k < qfs_ws::kLayers; ++k) {
      launch_adam(m->W[k], m->mW[k], m->vW[k], m->gW[k], (long long)m->dout[k] * m->din[k], 0.f, b1, b2, eps, 1.f,
                  1.f, m->W16[k], s, sched, gstep);
      launch_adam(m->b[k], m->mb[k], m->vb[k], m->gb[k], m->dout[k], 0.f, b1, b2, eps, 1.f, 1.f, nullptr, s, sched,
                  gstep);
      launch_transpose_bf16(m->W16[k], m->dout[k], m->din[k], m->WT16[k], s);
    }
    launch_ws_step_advance(jstep, gstep, s);
    return QFS_OK;
  };
  // The captured full-batch step, made on first use.
  auto capture_step = [&]() -> int {
    qfs_ctx* c = m->ctx;
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    long long before[QFS_PROF_KINDS];
    for (int i = 0; i < QFS_PROF_KINDS; ++i) before[i] = c->prof.launches[i];
    cudaStream_t saved = c->stream;
    c->stream = c->cap_stream;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
    c->prof.capturing = true;
    const int r = run_step(batch, batch);
    c->prof.capturing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->stream = saved;
    for (int i = 0; i < QFS_PROF_KINDS; ++i) {
      graph_launches[i] = c->prof.launches[i] - before[i];
      c->prof.launches[i] = before[i];
    }
    if (r != QFS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return r;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    CK(e);
    return QFS_OK;
  };
  for (int ep = 0; ep < epochs && rc == QFS_OK; ++ep) {
    for (int i = 0; i < count; ++i) idx[i] = i;
    // Fisher-Yates with Philox draws (deterministic per seed and epoch).
    for (int i = count - 1; i > 0; --i) {
      const double u = 0.5 + 0.5 * std::erf(qfs_normal_re(shuffle_seed, 7u, ((uint64_t)ep << 32) + i) * std::sqrt(2.0));
      int j = (int)(u * (i + 1));
      if (j > i) j = i;
      std::swap(idx[i], idx[j]);
    }
    if (cudaMemcpyAsync(didx, idx.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(ep_acc, 0, sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(jstep, 0, sizeof(int), st) != cudaSuccess) {
      rc = fail(QFS_ECUDA, "epoch set-up failed");
      break;
    }
    int nb = 0;
    for (int s0 = 0; s0 < count; s0 += batch) {
      const int bv = std::min(batch, count - s0);
      if (bv == batch) {
        if (!exec) {
          rc = capture_step();
          if (rc != QFS_OK) break;
        }
        if (cudaGraphLaunch(exec, st) != cudaSuccess) {
          rc = fail(QFS_ECUDA, "training step launch failed");
          break;
        }
        for (int i = 0; i < QFS_PROF_KINDS; ++i) m->ctx->prof.launches[i] += graph_launches[i];
        if (m->ctx->prof.on) {  // per-launch timings: harvested after each replay
          if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(QFS_ECUDA, "training step failed");
            break;
          }
          prof_harvest_graph(m->ctx);
        }
      } else {
        rc = run_step(bv, (bv + 127) / 128 * 128);
        if (rc != QFS_OK) break;
      }
      ++nb;
      ++m->step;
    }
    if (rc != QFS_OK) break;
    double ep_loss = 0.0;
    if (cudaMemcpyAsync(&ep_loss, ep_acc, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = fail(QFS_ECUDA, "reading the epoch loss failed");
      break;
    }
    if (epoch_loss) epoch_loss[ep] = ep_loss / std::max(nb, 1);
  }
  cudaStreamSynchronize(st);
  release_train();
  release();
  if (rc != QFS_OK) return rc;
  CK(cudaGetLastError());
  return check_err_word(m);
}

extern "C" int qfs_ws_predict(qfs_ws* m, int32_t count, const double* targets, double* gates_out) {
  g_err.clear();
  if (!m || !targets || !gates_out) return fail(QFS_EINVAL, "model, targets and gates_out must be given");
  if (count < 1) return fail(QFS_EINVAL, "count must be >= 1");
  TRY(set_device(m->ctx));
  cudaStream_t st = m->ctx->stream;
  for (int s0 = 0; s0 < count; s0 += m->B_cap) {
    const int bv = std::min(m->B_cap, count - s0);
    const int B = (bv + 127) / 128 * 128;
    TRY(ws_load_features(m, targets + (size_t)s0 * 512, bv, B));
    ws_forward(m, B);
    // Output rows -> 6 gates each; project each onto U(4) by its polar
    // factor (the update routine returns polar(E^dagger), so pass G^dagger).
    launch_ws_gates_adjoint(m->Z32[qfs_ws::kLayers - 1], m->dout[qfs_ws::kLayers - 1], bv, m->envs, st);
    launch_gate_update_batch(bv * 6, m->envs, nullptr, 0.0, m->envs, st);
    CK(cudaMemcpyAsync(gates_out + (size_t)s0 * 192, m->envs, sizeof(double2) * 96 * (size_t)bv,
                       cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  return check_err_word(m);
}

// ---------------------------------------------------------------------------
// Learned warm start as a policy: the network's prediction is the only start
// of a short first batched run; the targets it leaves unconverged fall back
// to random multistarts.  The paper has no learned part; the sweep judges
// every proposal, so a bad prediction costs sweeps, never correctness.

extern "C" int qfs_ws_instantiate(qfs_ws* m, int32_t P, const double* targets, const double* first_gates,
                                  const qfs_params* p, int32_t first_sweeps, double* gates_out,
                                  qfs_result* results, int64_t* stats) {
  g_err.clear();
  if (!m || !targets || !p || !gates_out || !results)
    return fail(QFS_EINVAL, "model, targets, params, gates_out and results must be given");
  if (P < 1) return fail(QFS_EINVAL, "P = %d: need >= 1", P);
  if (first_sweeps < 1) return fail(QFS_EINVAL, "first_sweeps = %d: need >= 1", first_sweeps);
  TRY(set_device(m->ctx));
  qfs_ctx* ctx = m->ctx;
  cudaStream_t st = ctx->stream;
  constexpr int kL = 6, kN = 4;
  const int32_t pairs1[2 * kL] = {0, 1, 2, 3, 1, 2, 0, 1, 2, 3, 1, 2};
  std::vector<int32_t> ns(P, kN), Ls(P, kL), pairs((size_t)P * 2 * kL);
  for (int i = 0; i < P; ++i) std::copy(pairs1, pairs1 + 2 * kL, pairs.begin() + (size_t)i * 2 * kL);
  // First start: the prediction (on the device) or the given gates.
  BatchInputs in1;
  in1.targets = targets;
  in1.gates_out = gates_out;
  if (first_gates) {
    in1.init_gates = first_gates;
  } else {
    if (m->pred_cap < (size_t)P) {
      if (m->pred) CK(cudaFree(m->pred));
      m->pred = nullptr;
      m->pred_cap = 0;
      if (cudaMalloc(&m->pred, sizeof(double2) * 96 * (size_t)P) != cudaSuccess) {
        cudaGetLastError();
        m->pred = nullptr;
        return fail(QFS_ENOMEM, "cannot allocate the predictions of %d targets", P);
      }
      m->pred_cap = (size_t)P;
    }
    for (int s0 = 0; s0 < P; s0 += m->B_cap) {
      const int bv = std::min(m->B_cap, P - s0);
      const int B = (bv + 127) / 128 * 128;
      TRY(ws_load_features(m, targets + (size_t)s0 * 512, bv, B));
      ws_forward(m, B);
      // Output rows -> 6 gates each, projected onto U(4) by their polar
      // factors (the update returns polar(E^dagger), so pass G^dagger).
      double2* out = m->pred + (size_t)s0 * 96;
      launch_ws_gates_adjoint(m->Z32[qfs_ws::kLayers - 1], m->dout[qfs_ws::kLayers - 1], bv, out, st);
      launch_gate_update_batch(bv * 6, out, nullptr, 0.0, out, st);
    }
    TRY(check_err_word(m));
    in1.init_gates = reinterpret_cast<const double*>(m->pred);
    in1.gates_dev = true;
  }
  qfs_params p1 = *p;
  p1.multistarts = 1;
  p1.max_sweeps = first_sweeps;
  qfs_params p2 = *p;
  p2.seed = p->seed + (1ULL << 30);
  const int S2 = p->multistarts;
  const int M = p->M > 0 ? std::min(p->M, 1 << kN) : (1 << kN) / 2;
  const size_t sN = (size_t)M << kN;
  // Large calls run in two halves so that the host draws of one half's
  // inputs (training states of stage 1; states and random starts of the
  // unconverged targets for stage 2) overlap the other half's sweeps: the
  // draws are those batch_common would make itself (state stream 1 from
  // seed + i, gates from the same seed), so the answers do not change.
  const int K = P >= 16384 ? 2 : 1;
  auto lo = [&](int k) { return (int)((long long)P * k / K); };
  // Pinned slot `slot` with room for n complex values (grown when needed;
  // nullptr if the host allocation fails).
  auto pinned = [&](int slot, size_t n) -> std::complex<double>* {
    if (m->pin_cap[slot] < n) {
      if (m->pin[slot]) cudaFreeHost(m->pin[slot]);
      m->pin[slot] = nullptr;
      m->pin_cap[slot] = 0;
      void* ptr = nullptr;
      if (cudaMallocHost(&ptr, std::max<size_t>(n, 1) * sizeof(std::complex<double>)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      m->pin[slot] = static_cast<std::complex<double>*>(ptr);
      m->pin_cap[slot] = n;
    }
    return m->pin[slot];
  };
  for (int k = 0; k < K; ++k) {
    if (!pinned(k, (size_t)(lo(k + 1) - lo(k)) * sN))
      return fail(QFS_ENOMEM, "pinned host memory for the drawn training states");
  }
  // Stage-1 states of half k into slot k.
  auto draw1 = [&](int k) {
    const int c0 = lo(k), n = lo(k + 1) - c0;
    std::complex<double>* st1 = m->pin[k];
    host_parallel_for(n, [&](int j) { draw_states(p->training_distribution, p1.seed + (uint64_t)(c0 + j), 1u, kN, M,
                                                  st1 + (size_t)j * sN); });
  };
  // States and starts of the unconverged targets idx of half k into slots
  // 2 + 2k and 3 + 2k (sized by the caller).
  auto draw2 = [&](int k, const std::vector<int32_t>& idx) {
    const int F = (int)idx.size();
    std::complex<double>* states = m->pin[2 + 2 * k];
    std::complex<double>* gates = m->pin[3 + 2 * k];
    host_parallel_for(F, [&](int j) {
      const uint64_t sd = p2.seed + (uint64_t)idx[j];
      draw_states(p->training_distribution, sd, 1u, kN, M, states + (size_t)j * sN);
      generate_gates(sd, S2 * kL, gates + (size_t)j * S2 * kL * 16);
    });
  };
  auto room2 = [&](int k, size_t F) {
    return pinned(2 + 2 * k, F * sN) != nullptr && pinned(3 + 2 * k, F * S2 * kL * 16) != nullptr;
  };
  auto stage1 = [&](int k) -> int {
    const int c0 = lo(k), n = lo(k + 1) - c0;
    BatchInputs in = in1;
    in.targets = targets + (size_t)c0 * 512;
    in.gates_out = gates_out + (size_t)c0 * 192;
    in.init_gates = in1.init_gates + (size_t)c0 * 192;  // one start of six gates per target
    in.samples = reinterpret_cast<const double*>(m->pin[k]);
    return batch_common(ctx, n, ns.data(), Ls.data(), pairs.data(), in, &p1, results + c0);
  };
  int64_t conv1 = 0, work1 = 0, work2 = 0, nfail = 0;
  auto failures = [&](int k) {
    std::vector<int32_t> f;
    for (int i = lo(k); i < lo(k + 1); ++i) {
      conv1 += results[i].converged;
      work1 += results[i].sweeps;
      if (!results[i].converged) f.push_back(i);
    }
    nfail += (int64_t)f.size();
    return f;
  };
  auto stage2 = [&](int k, const std::vector<int32_t>& idx) -> int {
    const int F = (int)idx.size();
    if (F == 0) return QFS_OK;
    std::vector<double> tf((size_t)F * 512), gf((size_t)F * 192);
    for (int j = 0; j < F; ++j)
      std::copy(targets + (size_t)idx[j] * 512, targets + (size_t)(idx[j] + 1) * 512, tf.begin() + (size_t)j * 512);
    std::vector<qfs_result> rf(F);
    BatchInputs in2;
    in2.targets = tf.data();
    in2.gates_out = gf.data();
    in2.samples = reinterpret_cast<const double*>(m->pin[2 + 2 * k]);
    in2.init_gates = reinterpret_cast<const double*>(m->pin[3 + 2 * k]);
    TRY(batch_common(ctx, F, ns.data(), Ls.data(), pairs.data(), in2, &p2, rf.data()));
    for (int j = 0; j < F; ++j) {
      const int i = idx[j];
      work2 += (int64_t)rf[j].sweeps * S2;
      std::copy(gf.begin() + (size_t)j * 192, gf.begin() + (size_t)(j + 1) * 192, gates_out + (size_t)i * 192);
      qfs_result r = rf[j];
      r.sweeps += results[i].sweeps;
      r.fp64_sweeps += results[i].fp64_sweeps;
      r.best_start += 1;  // 0 is the first start; fallback start j is j + 1
      results[i] = r;
    }
    return QFS_OK;
  };
  if (K == 1) {
    draw1(0);
    TRY(stage1(0));
    const std::vector<int32_t> f = failures(0);
    if (!room2(0, f.size())) return fail(QFS_ENOMEM, "pinned host memory for the fallback inputs");
    draw2(0, f);
    TRY(stage2(0, f));
  } else try {
    // draw1(1) || stage 1 of half 0; draw2(half 0) || stage 1 of half 1;
    // draw2(half 1) || stage 2 of half 0.  Every future is joined before a
    // return, so no helper outlives the buffers it writes.
    draw1(0);
    std::future<void> d1 = std::async(std::launch::async, draw1, 1);
    const int r0 = stage1(0);
    d1.get();
    TRY(r0);
    const std::vector<int32_t> f0 = failures(0);
    if (!room2(0, f0.size())) return fail(QFS_ENOMEM, "pinned host memory for the fallback inputs");
    std::future<void> d20 = std::async(std::launch::async, draw2, 0, std::cref(f0));
    const int r1 = stage1(1);
    d20.get();
    TRY(r1);
    const std::vector<int32_t> f1 = failures(1);
    if (!room2(1, f1.size())) return fail(QFS_ENOMEM, "pinned host memory for the fallback inputs");
    std::future<void> d21 = std::async(std::launch::async, draw2, 1, std::cref(f1));
    const int r2 = stage2(0, f0);
    d21.get();
    TRY(r2);
    TRY(stage2(1, f1));
  } catch (const std::exception& e) {
    return fail(QFS_EINTERNAL, "host draw threads: %s", e.what());
  }
  if (stats) {
    stats[0] = conv1;
    stats[1] = work1;
    stats[2] = work2;
    stats[3] = nfail;
  }
  return QFS_OK;
}
