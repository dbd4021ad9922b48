// Host runtime and C ABI: handles, solve plans (workspaces, tile maps, captured CUDA graphs)
// and the FP64 refinement / inner-CG driver.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "sylv_internal.cuh"

using namespace sylv;

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
namespace {
// Text of the last error of this thread, in a fixed buffer: setting it never allocates (the
// allocation-free solve reports its errors through it too); longer messages are cut.
constexpr size_t LAST_ERROR_BYTES = 512;
thread_local char g_last_error[LAST_ERROR_BYTES] = "";

void store_error(const char* msg) {
  std::snprintf(g_last_error, LAST_ERROR_BYTES, "%s", msg ? msg : "");
}

int fail(int code, const char* msg) {
  store_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_last_error, LAST_ERROR_BYTES, "%s: %s (%s)", what, cudaGetErrorName(e),
                cudaGetErrorString(e));
  (void)cudaGetLastError();  // clear a sticky-free error so later calls are not confused
  return e == cudaErrorMemoryAllocation ? SYLV_E_NOMEM : SYLV_E_CUDA;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return cuda_fail(_e, #call);   \
  } while (0)

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
  }
  ~DeviceGuard() {
    if (prev_ != dev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = 0, dev_ = 0;
};

template <typename P>
cudaError_t dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  return cudaMalloc((void**)p, bytes);
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

// ------------------------------------------------------------------------------------------
// plan: everything needed to run one list of systems
// ------------------------------------------------------------------------------------------
struct Group {
  int k = 0, m = 0, e = 0;  // shape shared by the group's systems
  int has_w = 0;
  std::vector<int> sys;     // systems of the group
  int block = TILE_PX;      // pixels per tile = threads per CTA
  int mult = 1;             // CTA slots = mult x resident CTAs
  int va = 0, vu = 0;       // kernel variant of inner_apply / inner_update (0: direct, 1: staged
                            // per (tile, column) unit, 2: multi-column, a tile's operator data
                            // staged once for all its columns)
  int csum = 0;             // staged pair with consumer-side sums (variants 2/3, chunks end
                            // with launch_inner_close): both staged and at most 2 columns
  int rs_ok = 0;             // the staged FP64 residual serves this group's shape and tiles
  // Four CTA lists: [0] for operator (inner_apply) launches, [1] for update launches, [2] for
  // residual and update_x launches, [3] for staged residual launches (their kernels keep
  // different numbers of CTAs resident).
  int ncta[4] = {0, 0, 0, 0};  // CTAs of every launch of that kind (fixed per configuration)
  int cta_cap = 0;
  CtaRef* d_ctas[4] = {nullptr, nullptr, nullptr, nullptr};
  CtaRef* h_ctas[4] = {nullptr, nullptr, nullptr, nullptr};  // pinned staging for reassignments
  std::vector<int> cur_set;  // systems the CTA lists currently cover
};

struct SysWork {
  int slot_cap = 0;          // partial-sum capacity in CTA slots
  void* vec = nullptr;       // 5 inner vectors
  ColState* st = nullptr;
  ColState* st2 = nullptr;
  double* partial = nullptr;
  double* partial2 = nullptr;
  unsigned int* counter = nullptr;
};

struct Plan {
  int device = 0, nsm = 1;
  std::vector<sylv_handle> hs;
  std::vector<int> R;
  int inner_double = 0;
  int ncols = 0;
  std::vector<Group> groups;
  std::vector<SysWork> work;
  SysDesc* d_desc = nullptr;
  SysDesc* h_desc = nullptr;    // pinned
  Control* d_ctl = nullptr;
  Control* h_ctl = nullptr;     // pinned
  unsigned int* h_poll = nullptr;  // pinned: n_active, n_unfinished, error
  ColState* h_states = nullptr;    // pinned, ncols
  ColState* d_states = nullptr;    // ncols, contiguous; system s starts at col_off[s]
  std::vector<int> col_off;
  int* d_col_sys = nullptr;
  int* d_col_rhs = nullptr;
  std::vector<int> col_sys, col_rhs;
  cudaStream_t cap_stream = nullptr;
  // several shape groups: one stream per group while a chunk graph is captured, so the
  // groups' iteration chains become parallel branches of the graph (their kernels never wait
  // on one another; the GPU fills one group's kernel tails with another's CTAs)
  std::vector<cudaStream_t> gstreams;
  std::vector<cudaEvent_t> gjoin;
  cudaEvent_t gfork = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  int graph_profile = 0;
  std::vector<cudaEvent_t> chunk_events;  // 2 * graph_iters + 1 when profiling
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evr0 = nullptr, evr1 = nullptr;

  ~Plan();
};

struct sylv_ctx {
  int device = 0;
  OpData op{};
  int explicit_A = 0;
  double nu0 = 100.0;
  int32_t* ell_col = nullptr;
  float* ell_val32 = nullptr;
  double* ell_val64 = nullptr;
  float* diag32 = nullptr;
  double* diag64 = nullptr;
  float* D32 = nullptr;
  double* D64 = nullptr;
  float* w32 = nullptr;
  double* w64 = nullptr;
  double* blk64 = nullptr;
  double* fac64 = nullptr;
  unsigned int* apply_err = nullptr;  // staged stand-alone apply: timeout flag, tile counter,
                                      // CTAs done
  float* fs32 = nullptr;
  __half2* fl16 = nullptr;
  float* blk_hl = nullptr;    // pixel blocks as FP32 pairs (double-float residual)
  float* val_hl = nullptr;    // ELL values as FP32 pairs
  int val_df_bad = 0;         // an ELL value lies outside the double-float range
  std::unique_ptr<Plan> plan[2];  // single-system plans, [inner_double]
  double* lam = nullptr;
  size_t lam_bytes = 0;
  double* grad_ws = nullptr;
  size_t grad_bytes = 0;
  double* var_ws = nullptr;   // sylv_variance: solves of one chunk of probes, num, den
  size_t var_bytes = 0;
  double* host_ws = nullptr;  // sylv_solve_host: device Yobs, B, X
  size_t host_bytes = 0;
  cudaStream_t copy_stream = nullptr, copy_stream2 = nullptr;
  cudaEvent_t ev_host[12] = {};   // slices of Yobs copied, start, X updated, X copied (x2)
};

Plan::~Plan() {
  for (auto& g : groups) {
    for (int k = 0; k < 4; ++k) {
      cudaFree(g.d_ctas[k]);
      cudaFreeHost(g.h_ctas[k]);
    }
  }
  cudaFree(d_states);
  for (auto& w : work) {
    cudaFree(w.vec);
    cudaFree(w.partial);
    cudaFree(w.partial2);
    cudaFree(w.counter);
  }
  cudaFree(d_desc);
  cudaFree(d_ctl);
  cudaFree(d_col_sys);
  cudaFree(d_col_rhs);
  cudaFreeHost(h_desc);
  cudaFreeHost(h_ctl);
  cudaFreeHost(h_poll);
  cudaFreeHost(h_states);
  if (graph) cudaGraphExecDestroy(graph);
  for (auto e : chunk_events) cudaEventDestroy(e);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (evr0) cudaEventDestroy(evr0);
  if (evr1) cudaEventDestroy(evr1);
  for (auto e : gjoin) cudaEventDestroy(e);
  if (gfork) cudaEventDestroy(gfork);
  for (auto gs : gstreams) cudaStreamDestroy(gs);
  if (cap_stream) cudaStreamDestroy(cap_stream);
}

namespace {

// The mixed solve's true residual: double-float (default), SYLV_RESIDUAL=f64 the FP64 kernels,
// SYLV_RESIDUAL=plain the double-float kernel without staging; read at every solve.
int residual_mode() {
  const char* v = std::getenv("SYLV_RESIDUAL");
  if (v && std::strcmp(v, "f64") == 0) return 0;
  if (v && std::strcmp(v, "plain") == 0) return 2;
  return 1;
}

// SYLV_STAGED_APPLY=0 keeps the stand-alone FP32 apply on the direct kernel.
const bool g_staged_apply = [] {
  const char* v = std::getenv("SYLV_STAGED_APPLY");
  return !(v && v[0] == '0');
}();

// Batched plans, keyed by the list of (handle, nrhs) and the inner type.
std::mutex g_plan_mu;
std::map<std::vector<uintptr_t>, std::unique_ptr<Plan>> g_plans;

// ------------------------------------------------------------------------------------------
// tiling of a group and the autotuner
// ------------------------------------------------------------------------------------------
// A configuration: tile size (threads per CTA), CTA slots as a multiple of what stays
// resident, and the variant of each inner kernel.  configure_group computes every system's
// tile and slot counts, uploads the group's CTA list and records them in the host descriptors
// (uploaded before each solve).
template <typename T>
int configure_group(Plan& P, Group& g, int block, int mult, int va, int vu) {
  const int occ[4] = {occupancy<T>(0, g.k, g.m, g.e, va, block),
                      occupancy<T>(1, g.k, g.m, g.e, vu, block),
                      occupancy<T>(2, g.k, g.m, g.e, 0, block),
                      occupancy<T>(3, g.k, g.m, g.e, 0, block)};
  int64_t total = 0;
  for (int s : g.sys) total += ceil_div(P.hs[s]->op.n, block);
  for (int kind = 0; kind < 4; ++kind) {
    const int64_t budget = (int64_t)P.nsm * occ[kind] * mult;
    int used = 0;
    for (int s : g.sys) {
      const int nt = (int)ceil_div(P.hs[s]->op.n, block);
      int64_t ns = total <= budget ? nt : (budget * nt) / total;
      ns = std::max<int64_t>(1, std::min<int64_t>(ns, nt));
      ns = std::min<int64_t>(ns, P.work[s].slot_cap);
      P.h_desc[s].ntiles = nt;
      P.h_desc[s].nslots[kind] = (int)ns;
      for (int t = 0; t < ns; ++t) {
        if (used >= g.cta_cap) return fail(SYLV_E_CUDA, "internal: CTA list overflow");
        g.h_ctas[kind][used++] = CtaRef{s, t};
      }
    }
    CK(cudaMemcpy(g.d_ctas[kind], g.h_ctas[kind], (size_t)used * sizeof(CtaRef),
                  cudaMemcpyHostToDevice));
    g.ncta[kind] = used;
  }
  g.cur_set = g.sys;
  g.block = block;
  g.mult = mult;
  g.va = va;
  g.vu = vu;
  int rmax = 0;
  for (int s : g.sys) rmax = std::max(rmax, P.R[s]);
  g.csum = (!P.inner_double && va == 1 && vu == 1 && rmax <= 2) ? 1 : 0;
  g.rs_ok = (!P.inner_double && !g.has_w && block == TILE_PX && tma_available(g.k, g.m, g.e)) ? 1 : 0;
  return SYLV_OK;
}

// Spreads the group's fixed number of CTAs over the systems in `set` only (in proportion to
// their tiles), padding with idle entries; called between kernels when systems finish, so
// that the remaining ones get the whole GPU.  Asynchronous on s (pinned staging).
int reassign_group(Plan& P, Group& g, const std::vector<int>& set, cudaStream_t s) {
  if (set == g.cur_set) return SYLV_OK;
  int64_t total = 0;
  for (int sy : set) total += P.h_desc[sy].ntiles;
  for (int kind = 0; kind < 4; ++kind) {
    const int ncta = g.ncta[kind];
    std::vector<int64_t> ns(set.size());
    int64_t sum = 0;
    for (size_t t = 0; t < set.size(); ++t) {
      const int sy = set[t];
      const int64_t nt = P.h_desc[sy].ntiles;
      int64_t v = total <= ncta ? nt : ((int64_t)ncta * nt) / total;
      v = std::max<int64_t>(1, std::min<int64_t>({v, nt, (int64_t)P.work[sy].slot_cap}));
      ns[t] = v;
      sum += v;
    }
    while (sum > ncta) {  // the launch grid is fixed (captured graphs): trim the largest shares
      size_t big = 0;
      for (size_t t = 1; t < ns.size(); ++t)
        if (ns[t] > ns[big]) big = t;
      if (ns[big] <= 1) return fail(SYLV_E_CUDA, "internal: more systems than CTAs");
      --ns[big];
      --sum;
    }
    int used = 0;
    for (size_t t = 0; t < set.size(); ++t) {
      P.h_desc[set[t]].nslots[kind] = (int)ns[t];
      for (int q = 0; q < ns[t]; ++q) g.h_ctas[kind][used++] = CtaRef{set[t], q};
    }
    for (int t = used; t < ncta; ++t) g.h_ctas[kind][t] = CtaRef{-1, 0};
    CK(cudaMemcpyAsync(g.d_ctas[kind], g.h_ctas[kind], (size_t)ncta * sizeof(CtaRef),
                       cudaMemcpyHostToDevice, s));
  }
  g.cur_set = set;
  return SYLV_OK;
}

// Systems of group g with a column in one of the given phases (from the last state read).
std::vector<int> systems_in_phase(const Plan& P, const Group& g, int ph_a, int ph_b) {
  std::vector<int> out;
  for (int sy : g.sys) {
    for (int r = 0; r < P.R[sy]; ++r) {
      const int ph = P.h_states[P.col_off[sy] + r].phase;
      if (ph == ph_a || ph == ph_b) {
        out.push_back(sy);
        break;
      }
    }
  }
  return out;
}

// Before the residual of a refinement step (want_inner false) or before a chunk of inner
// iterations (true): cover only the systems that have work in that phase, and upload the
// descriptors whose slot counts changed.
int rebalance(Plan& P, bool want_inner, cudaStream_t s) {
  if (P.hs.size() <= 1) return SYLV_OK;
  bool changed = false;
  for (auto& g : P.groups) {
    std::vector<int> set = want_inner ? systems_in_phase(P, g, PH_INNER, PH_INNER)
                                      : systems_in_phase(P, g, PH_START, PH_INNER_DONE);
    if (set != g.cur_set) {
      int rc = reassign_group(P, g, set, s);
      if (rc != SYLV_OK) return rc;
      changed = true;
    }
  }
  if (changed)
    CK(cudaMemcpyAsync(P.d_desc, P.h_desc, P.hs.size() * sizeof(SysDesc),
                       cudaMemcpyHostToDevice, s));
  return SYLV_OK;
}

const char* const kVariantName[3] = {"direct", "staged", "multi-column"};

struct TuneChoice {
  int block, mult, va, vu;
  float ms;
};
std::mutex g_tune_mu;
std::map<std::vector<int>, TuneChoice> g_tune;
// SYLV_AUTOTUNE=0 skips timing and takes the default configuration.
const bool g_autotune = [] {
  const char* v = std::getenv("SYLV_AUTOTUNE");
  return !(v && v[0] == '0');
}();

// Times one inner kernel over the group with every column forced into the inner phase.
template <typename T>
int time_inner(Plan& P, Group& g, int kind, int reps, float* ms_out) {
  cudaStream_t s = P.cap_stream;
  int rmax = 1;
  for (int sidx : g.sys) rmax = std::max(rmax, P.R[sidx]);
  std::vector<ColState> st(rmax, ColState{});
  {
    for (auto& c : st) {
      c.phase = PH_INNER;
      c.gamma = 1.0;
      c.alpha = 0.25;
      c.beta = 0.25;
      c.rr_in = 1.0;
      c.thr_in = 0.0;
      c.first = 0;
    }
  }
  float best = 1e30f;
  for (int rep = 0; rep < reps + 1; ++rep) {
    for (int sidx : g.sys) {
      CK(cudaMemcpyAsync(P.work[sidx].st, st.data(), P.R[sidx] * sizeof(ColState),
                         cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(P.work[sidx].st2, st.data(), P.R[sidx] * sizeof(ColState),
                         cudaMemcpyHostToDevice, s));
    }
    CK(cudaEventRecord(P.evr0, s));
    // consumer-side pair: launch variant 2 (the column states as stored, no sums at the start)
    const int v = g.csum ? 2 : ((kind == 0 ? g.va : g.vu) == 2 ? 4 : (kind == 0 ? g.va : g.vu));
    if (kind == 0)
      CK(launch_inner_apply<T>(g.k, g.m, g.e, v, g.ncta[0], g.block, P.d_desc, g.d_ctas[0],
                               P.d_ctl, s));
    else
      CK(launch_inner_update<T>(g.k, g.m, g.e, v, g.ncta[1], g.block, P.d_desc, g.d_ctas[1],
                                P.d_ctl, s));
    CK(cudaEventRecord(P.evr1, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, P.evr0, P.evr1));
    if (rep > 0) best = std::min(best, ms);
  }
  *ms_out = best;
  return SYLV_OK;
}

// Chooses the group's configuration: cached per (device, inner type, shape, right-hand sides,
// size bucket); otherwise every candidate is timed on the plan's own buffers (the inner
// vectors hold a finite filler; the solve rewrites them before use).
template <typename T>
int tune_group(Plan& P, Group& g) {
  const bool dbl = sizeof(T) == 8;
  const bool can_tma = !dbl && !g.has_w && tma_available(g.k, g.m, g.e);
  int64_t ntot = 0;
  int rmax = 0;
  for (int s : g.sys) {
    ntot += P.hs[s]->op.n;
    rmax = std::max(rmax, P.R[s]);
  }
  int lg = 0;
  while ((int64_t(1) << (lg + 1)) <= ntot) ++lg;
  const TuneChoice dflt{TILE_PX, 1, 0, can_tma ? 1 : 0, 0.f};
  // SYLV_TUNE_FORCE="tile,mult,apply_variant,update_variant" pins a configuration (used to
  // profile exactly the configuration a timed run chose, and by tests of one kernel variant);
  // it takes precedence over the cache of earlier choices
  if (const char* f = std::getenv("SYLV_TUNE_FORCE")) {
    TuneChoice c = dflt;
    if (std::sscanf(f, "%d,%d,%d,%d", &c.block, &c.mult, &c.va, &c.vu) == 4 &&
        (c.block == 128 || c.block == TILE_PX) && c.mult >= 1 && c.mult <= 4) {
      if (!can_tma || c.block != TILE_PX) c.va = c.vu = 0;
      c.va = std::min(std::max(c.va, 0), 2);
      c.vu = std::min(std::max(c.vu, 0), 2);
      return configure_group<T>(P, g, c.block, c.mult, c.va, c.vu);
    }
  }
  const std::vector<int> key = {P.device, (int)dbl, g.k, g.m, g.e, g.has_w, rmax, lg,
                                (int)g.sys.size()};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      const TuneChoice& c = it->second;
      return configure_group<T>(P, g, c.block, c.mult, c.va, c.vu);
    }
  }
  if (!g_autotune) return configure_group<T>(P, g, dflt.block, dflt.mult, dflt.va, dflt.vu);
  // finite filler in the inner vectors and a permissive control word
  for (int s : g.sys) {
    const size_t vb = (size_t)P.R[s] * P.hs[s]->op.k * P.hs[s]->op.ld * sizeof(T);
    CK(cudaMemsetAsync(P.work[s].vec, 0x3C, 5 * vb, P.cap_stream));
  }
  Control c{};
  c.maxit = 1 << 30;
  c.max_outer = 1 << 30;
  c.precond = SYLV_PRECOND_BLOCK_JACOBI;
  *P.h_ctl = c;
  CK(cudaMemcpyAsync(P.d_ctl, P.h_ctl, sizeof(Control), cudaMemcpyHostToDevice, P.cap_stream));
  std::vector<TuneChoice> cands;
  for (int mult = 1; mult <= 2; ++mult) {
    cands.push_back({128, mult, 0, 0, 0.f});
    cands.push_back({TILE_PX, mult, 0, 0, 0.f});
    if (can_tma) {
      cands.push_back({TILE_PX, mult, 1, 0, 0.f});
      cands.push_back({TILE_PX, mult, 0, 1, 0.f});
      cands.push_back({TILE_PX, mult, 1, 1, 0.f});
      if (rmax >= 2) {   // multi-column kernels: operator data once per tile for all columns
        cands.push_back({TILE_PX, mult, 2, 2, 0.f});
        cands.push_back({TILE_PX, mult, 2, 1, 0.f});
        cands.push_back({TILE_PX, mult, 1, 2, 0.f});
      }
    }
  }
  TuneChoice best = dflt;
  best.ms = 1e30f;
  for (auto& cnd : cands) {
    int rc = configure_group<T>(P, g, cnd.block, cnd.mult, cnd.va, cnd.vu);
    if (rc != SYLV_OK) return rc;
    CK(cudaMemcpyAsync(P.d_desc, P.h_desc, P.hs.size() * sizeof(SysDesc),
                       cudaMemcpyHostToDevice, P.cap_stream));
    float ta = 0, tu = 0;
    if ((rc = time_inner<T>(P, g, 0, 3, &ta)) != SYLV_OK) return rc;
    if ((rc = time_inner<T>(P, g, 1, 3, &tu)) != SYLV_OK) return rc;
    cnd.ms = ta + tu;
    if (cnd.ms < best.ms) best = cnd;
  }
  CK(cudaStreamSynchronize(P.cap_stream));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  if (const char* v = std::getenv("SYLV_TUNE_LOG")) {
    if (v[0] == '1')
      std::fprintf(stderr,
                   "sylv autotune: %s k=%d m=%d E=%d systems=%zu nrhs<=%d n=%lld -> tile %d, "
                   "slots x%d, apply %s, update %s (%.3f ms per iteration)\n",
                   dbl ? "fp64" : "fp32", g.k, g.m, g.e, g.sys.size(), rmax, (long long)ntot,
                   best.block, best.mult, kVariantName[best.va], kVariantName[best.vu], best.ms);
  }
  return configure_group<T>(P, g, best.block, best.mult, best.va, best.vu);
}

int build_plan(Plan& P, int nsys, const sylv_handle* hs, const int* R, int inner_double) {
  P.hs.assign(hs, hs + nsys);
  P.R.assign(R, R + nsys);
  P.inner_double = inner_double;
  const size_t tsz = inner_double ? sizeof(double) : sizeof(float);
  P.work.resize(nsys);
  // groups by shape (k, m, ELL width); each system of a group gets CTA slots in proportion to its tiles, and the
  // launch is sized to what the device keeps resident (nothing relies on residency: no CTA
  // ever waits for another)
  int dev = 0, nsm = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  P.device = dev;
  P.nsm = nsm;
  std::map<std::vector<int>, std::vector<int>> byshape;
  for (int s = 0; s < nsys; ++s)
    byshape[{hs[s]->op.k, hs[s]->op.m, hs[s]->op.E}].push_back(s);
  for (int s = 0; s < nsys; ++s)
    P.work[s].slot_cap = (int)std::min<int64_t>(ceil_div(hs[s]->op.n, 128), (int64_t)nsm * 32);
  for (auto& kv : byshape) {
    Group g;
    g.k = kv.first[0];
    g.m = kv.first[1];
    g.e = kv.first[2];
    g.sys = kv.second;
    for (int s : kv.second) {
      g.has_w = g.has_w || hs[s]->op.has_w;
      g.cta_cap += P.work[s].slot_cap;
    }
    g.cta_cap += 1;
    P.groups.push_back(g);  // owned by the plan before its lists are allocated
    Group& gp = P.groups.back();
    for (int k = 0; k < 4; ++k) {
      CK(dalloc(&gp.d_ctas[k], (size_t)gp.cta_cap * sizeof(CtaRef)));
      CK(cudaMallocHost((void**)&gp.h_ctas[k], (size_t)gp.cta_cap * sizeof(CtaRef)));
    }
  }
  for (int s = 0; s < nsys; ++s) {
    const OpData& op = hs[s]->op;
    SysWork& w = P.work[s];
    const size_t vbytes = (size_t)R[s] * op.k * op.ld * tsz;
    CK(dalloc(&w.vec, 5 * vbytes));
    CK(cudaMemset(w.vec, 0, 5 * vbytes));
    P.col_off.push_back(P.ncols);
    P.ncols += R[s];
    CK(dalloc(&w.partial, (size_t)w.slot_cap * R[s] * NPART * sizeof(double)));
    CK(dalloc(&w.partial2, (size_t)w.slot_cap * R[s] * NPART * sizeof(double)));
    CK(dalloc(&w.counter, sizeof(unsigned int)));
    CK(cudaMemset(w.counter, 0, sizeof(unsigned int)));
    for (int r = 0; r < R[s]; ++r) {
      P.col_sys.push_back(s);
      P.col_rhs.push_back(r);
    }
  }
  CK(dalloc(&P.d_states, (size_t)2 * P.ncols * sizeof(ColState)));
  for (int s = 0; s < nsys; ++s) {
    P.work[s].st = P.d_states + P.col_off[s];
    P.work[s].st2 = P.d_states + P.ncols + P.col_off[s];
  }
  CK(dalloc(&P.d_desc, nsys * sizeof(SysDesc)));
  CK(cudaMallocHost((void**)&P.h_desc, nsys * sizeof(SysDesc)));
  CK(dalloc(&P.d_ctl, sizeof(Control)));
  CK(cudaMallocHost((void**)&P.h_ctl, sizeof(Control)));
  CK(cudaMallocHost((void**)&P.h_poll, 4 * sizeof(unsigned int)));
  CK(cudaMallocHost((void**)&P.h_states, P.ncols * sizeof(ColState)));
  CK(dalloc(&P.d_col_sys, P.ncols * sizeof(int)));
  CK(dalloc(&P.d_col_rhs, P.ncols * sizeof(int)));
  CK(cudaMemcpy(P.d_col_sys, P.col_sys.data(), P.ncols * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P.d_col_rhs, P.col_rhs.data(), P.ncols * sizeof(int), cudaMemcpyHostToDevice));
  // static part of the descriptors
  for (int s = 0; s < nsys; ++s) {
    SysDesc& d = P.h_desc[s];
    std::memset(&d, 0, sizeof(SysDesc));
    d.op = hs[s]->op;
    d.R = R[s];
    d.ntiles = 0;  // set by configure_group
    d.nslots[0] = d.nslots[1] = d.nslots[2] = 0;
    const size_t vbytes = (size_t)R[s] * d.op.k * d.op.ld * tsz;
    char* base = (char*)P.work[s].vec;
    d.vd = base;
    d.vr = base + vbytes;
    d.vz = base + 2 * vbytes;
    d.vp = base + 3 * vbytes;
    d.vq = base + 4 * vbytes;
    d.st = P.work[s].st;
    d.st2 = P.work[s].st2;
    d.partial = P.work[s].partial;
    d.partial2 = P.work[s].partial2;
    d.counter = P.work[s].counter;
  }
  CK(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
  if (P.groups.size() > 1) {
    P.gstreams.assign(P.groups.size(), nullptr);
    P.gjoin.assign(P.groups.size(), nullptr);
    for (size_t gi = 0; gi < P.groups.size(); ++gi) {
      CK(cudaStreamCreateWithFlags(&P.gstreams[gi], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&P.gjoin[gi], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&P.gfork, cudaEventDisableTiming));
  }
  CK(cudaEventCreate(&P.ev0));
  CK(cudaEventCreate(&P.ev1));
  CK(cudaEventCreate(&P.evr0));
  CK(cudaEventCreate(&P.evr1));
  for (auto& g : P.groups) {
    int rc = inner_double ? tune_group<double>(P, g) : tune_group<float>(P, g);
    if (rc != SYLV_OK) return rc;
  }
  return SYLV_OK;
}

// Launch variant of the group's operator (kind 0) or update (kind 1) kernel at iteration `it`
// of a chunk (see launch_inner_apply): consumer-side sums 2/3, multi-column 4, else 0/1.
int kernel_variant(const Group& g, int kind, int it) {
  if (g.csum) return kind == 0 ? (it == 0 ? 2 : 3) : 3;
  const int v = kind == 0 ? g.va : g.vu;
  return v == 2 ? 4 : v;
}

// Iteration `it` of a chunk of `iters`.  Groups with consumer-side sums: the chunk's first
// operator kernel reads the stored states, every other kernel first sums its predecessor's
// partials, and the chunk ends with the state change of its last update (launch_inner_close).
template <typename T>
int launch_inner_iteration(Plan& P, cudaStream_t s, cudaEvent_t e_mid, cudaEvent_t e_end,
                           bool capture_events, int it, int iters) {
  for (auto& g : P.groups)
    CK(launch_inner_apply<T>(g.k, g.m, g.e, kernel_variant(g, 0, it), g.ncta[0], g.block,
                             P.d_desc, g.d_ctas[0], P.d_ctl, s));
  if (e_mid)
    CK(capture_events ? cudaEventRecordWithFlags(e_mid, s, cudaEventRecordExternal)
                      : cudaEventRecord(e_mid, s));
  for (auto& g : P.groups)
    CK(launch_inner_update<T>(g.k, g.m, g.e, kernel_variant(g, 1, it), g.ncta[1], g.block,
                              P.d_desc, g.d_ctas[1], P.d_ctl, s));
  if (it == iters - 1)
    for (auto& g : P.groups)
      if (g.csum) CK(launch_inner_close(g.ncta[1], P.d_desc, g.d_ctas[1], P.d_ctl, s));
  if (e_end)
    CK(capture_events ? cudaEventRecordWithFlags(e_end, s, cudaEventRecordExternal)
                      : cudaEventRecord(e_end, s));
  return SYLV_OK;
}

// Iteration `it` of a chunk for one group only (the branch of that group in a chunk graph).
template <typename T>
int launch_group_iteration(Plan& P, const Group& g, cudaStream_t s, int it, int iters) {
  CK(launch_inner_apply<T>(g.k, g.m, g.e, kernel_variant(g, 0, it), g.ncta[0], g.block,
                           P.d_desc, g.d_ctas[0], P.d_ctl, s));
  CK(launch_inner_update<T>(g.k, g.m, g.e, kernel_variant(g, 1, it), g.ncta[1], g.block,
                            P.d_desc, g.d_ctas[1], P.d_ctl, s));
  if (it == iters - 1 && g.csum)
    CK(launch_inner_close(g.ncta[1], P.d_desc, g.d_ctas[1], P.d_ctl, s));
  return SYLV_OK;
}

// The chunk as one branch per group: fork from the capturing stream, each group's `iters`
// iterations on its own stream, join back.
template <typename T>
int capture_group_branches(Plan& P, int iters) {
  CK(cudaEventRecord(P.gfork, P.cap_stream));
  for (size_t gi = 0; gi < P.groups.size(); ++gi) {
    CK(cudaStreamWaitEvent(P.gstreams[gi], P.gfork, 0));
    for (int it = 0; it < iters; ++it) {
      const int rc = launch_group_iteration<T>(P, P.groups[gi], P.gstreams[gi], it, iters);
      if (rc != SYLV_OK) return rc;
    }
    CK(cudaEventRecord(P.gjoin[gi], P.gstreams[gi]));
    CK(cudaStreamWaitEvent(P.cap_stream, P.gjoin[gi], 0));
  }
  return SYLV_OK;
}

template <typename T>
int ensure_graph(Plan& P, int iters, int profile) {
  if (P.graph && P.graph_iters == iters && P.graph_profile == profile) return SYLV_OK;
  if (P.graph) {
    cudaGraphExecDestroy(P.graph);
    P.graph = nullptr;
  }
  for (auto e : P.chunk_events) cudaEventDestroy(e);
  P.chunk_events.clear();
  if (profile) {
    P.chunk_events.resize(2 * iters + 1);
    for (auto& e : P.chunk_events) CK(cudaEventCreate(&e));
  }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = SYLV_OK;
  if (profile) {
    cudaError_t e = cudaEventRecordWithFlags(P.chunk_events[0], P.cap_stream,
                                             cudaEventRecordExternal);
    if (e != cudaSuccess) rc = cuda_fail(e, "event record in capture");
  }
  if (!profile && !P.gstreams.empty() && rc == SYLV_OK) {
    rc = capture_group_branches<T>(P, iters);
  } else {
    // (one stream when profiling: the per-launch events time the kernels one after another)
    for (int it = 0; it < iters && rc == SYLV_OK; ++it)
      rc = launch_inner_iteration<T>(P, P.cap_stream,
                                     profile ? P.chunk_events[2 * it + 1] : nullptr,
                                     profile ? P.chunk_events[2 * it + 2] : nullptr, true, it,
                                     iters);
  }
  cudaError_t e = cudaStreamEndCapture(P.cap_stream, &graph);
  if (rc != SYLV_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&P.graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  P.graph_iters = iters;
  P.graph_profile = profile;
  return SYLV_OK;
}

int poll(Plan& P, cudaStream_t s) {
  CK(cudaMemcpyAsync(P.h_poll, &P.d_ctl->n_active, 3 * sizeof(unsigned int),
                     cudaMemcpyDeviceToHost, s));
  if (P.hs.size() > 1)
    CK(cudaMemcpyAsync(P.h_states, P.d_states, (size_t)P.ncols * sizeof(ColState),
                       cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (P.h_poll[2]) return fail(SYLV_E_TIMEOUT, "a bounded device-side wait expired");
  return SYLV_OK;
}

// Copies of the solution to the host for sylv_solve_host: after every refinement step's update
// X += d (not the first, which leaves the start unchanged) the solution is copied on its own
// stream while the FP64 residual that decides convergence runs, and the next update waits for
// that copy; the last copy is the result.
struct HostSink {
  cudaStream_t cs[2] = {nullptr, nullptr};    // the two halves go to two copy engines
  cudaEvent_t ev_x = nullptr;                 // X updated
  cudaEvent_t ev_done[2] = {nullptr, nullptr};   // copies finished
  double* host = nullptr;
  const double* dev = nullptr;
  size_t bytes = 0;
  int copies = 0;
};

template <typename T>
int run_plan(Plan& P, const double* const* B, double* const* X, const sylv_opts& o,
             sylv_info* infos, cudaStream_t s, HostSink* sink = nullptr) {
  const int nsys = (int)P.hs.size();
  for (int t = 0; t < nsys; ++t) {
    P.h_desc[t].op = P.hs[t]->op;  // operator scalars may have changed since the plan was built
    P.h_desc[t].B = B[t];
    P.h_desc[t].X = X[t];
  }
  Control& c = *P.h_ctl;
  std::memset(&c, 0, sizeof(Control));
  c.tol2 = o.tol * o.tol;
  c.tol_in2 = o.precision == SYLV_PREC_MIXED ? o.inner_tol * o.inner_tol : 0.0;
  c.safety2 = 0.25;
  c.maxit = o.maxit;
  c.max_outer = o.max_outer;
  c.precond = o.precond;
  c.x0_zero = o.use_x0 ? 0 : 1;
  // SYLV_WAIT_BUDGET_CYCLES shortens the staged kernels' pipeline waits (tests of the timeout
  // path; the waits that drain copies in flight keep the default)
  if (const char* wb = std::getenv("SYLV_WAIT_BUDGET_CYCLES")) c.wait_budget = std::atoll(wb);
  // SYLV_INJECT_STALL=bits makes the named staged kernels' producers issue nothing (tests of
  // the timeout path: a wait that nothing completes runs out; no copy is ever in flight)
  if (const char* is = std::getenv("SYLV_INJECT_STALL")) c.inject_stall = std::atoi(is);
  const int iters = o.check_every > 0 ? o.check_every : 16;
  const bool prof = o.profile != 0;
  double ms_apply = 0, ms_update = 0, ms_res = 0;
  int n_apply = 0, n_update = 0, n_res = 0, polls = 0;
  long launches = 0;
  const int ng = (int)P.groups.size();

  CK(cudaEventRecord(P.ev0, s));
  CK(cudaMemcpyAsync(P.d_desc, P.h_desc, nsys * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(P.d_ctl, P.h_ctl, sizeof(Control), cudaMemcpyHostToDevice, s));
  if (!o.use_x0) {
    for (int t = 0; t < nsys; ++t) {
      const OpData& op = P.hs[t]->op;
      CK(cudaMemsetAsync(X[t], 0, (size_t)P.R[t] * op.k * op.ldu * sizeof(double), s));
    }
  }
  CK(launch_init_states(P.ncols, P.d_col_sys, P.d_col_rhs, P.d_desc, P.d_ctl, s));
  launches += 1;
  // the staged FP64 residual copies the caller's rows of X and B whole: every system of the
  // group needs whole tiles, an even leading dimension and 16-byte aligned X and B; its units
  // are (tile, column) pairs that re-stage the tile's pixel blocks for every column, so with
  // more than two columns the direct kernel is faster (8 columns, 50M pixels: 292 against
  // 325 ms per solve)
  // In mixed precision the residual is formed in double-float on the FP32 pipe when every
  // system of the group allows it (operator entries in its range): staged (k_residual_tma_df)
  // where the caller's rows can be copied whole, else k_residual_df; the FP64 kernels are bound
  // by the FP64 unit.  rs_staged: 0 direct FP64, 1 staged FP64, 2 double-float, 3 staged
  // double-float.
  const int rmode = residual_mode();
  std::vector<char> rs_staged(P.groups.size(), 0);
  for (size_t gi = 0; gi < P.groups.size(); ++gi) {
    const Group& g = P.groups[gi];
    bool df = !P.inner_double && rmode != 0;
    bool ok = g.rs_ok != 0;
    int rmax = 0;
    for (int t : g.sys) {
      const OpData& op = P.hs[t]->op;
      df = df && op.df_ok;
      rmax = std::max(rmax, P.R[t]);
      ok = ok && op.n % TILE_PX == 0 && op.ldu % 2 == 0 &&
           ((uintptr_t)B[t] & 15u) == 0 && ((uintptr_t)X[t] & 15u) == 0;
    }
    if (df) rs_staged[gi] = (ok && rmode == 1) ? 3 : 2;
    else rs_staged[gi] = (ok && rmax <= 2) ? 1 : 0;
  }
  if (o.use_graph) {
    int rc = ensure_graph<T>(P, iters, prof ? 1 : 0);
    if (rc != SYLV_OK) return rc;
  }
  const long max_polls = (long)o.maxit / iters + 4L * (o.max_outer + 2) + 16;
  bool gave_up = false;
  struct Events {  // destroyed on every return
    std::vector<cudaEvent_t> v;
    ~Events() {
      for (auto e : v)
        if (e) cudaEventDestroy(e);
    }
  } direct;
  std::vector<cudaEvent_t>& direct_events = direct.v;
  if (prof && !o.use_graph) {
    direct_events.assign(2 * iters + 1, nullptr);
    for (auto& e : direct_events) CK(cudaEventCreate(&e));
  }
  int rc = SYLV_OK;
  // every system starts in the residual phase: cover all of them
  for (auto& g : P.groups) {
    if ((rc = reassign_group(P, g, g.sys, s)) != SYLV_OK) return rc;
  }
  CK(cudaMemcpyAsync(P.d_desc, P.h_desc, nsys * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
  bool first_outer = true;
  while (true) {
    if (!first_outer && (rc = rebalance(P, false, s)) != SYLV_OK) return rc;
    const bool at_start = first_outer;
    first_outer = false;
    if (sink && sink->copies > 0) {
      CK(cudaStreamWaitEvent(s, sink->ev_done[0], 0));
      CK(cudaStreamWaitEvent(s, sink->ev_done[1], 0));
    }
    for (auto& g : P.groups)
      CK(launch_update_x<T>(g.k, g.ncta[2], g.block, P.d_desc, g.d_ctas[2], s));
    if (sink && !at_start) {
      CK(cudaEventRecord(sink->ev_x, s));
      const size_t half = (sink->bytes / 2) & ~(size_t)255;
      for (int c = 0; c < 2; ++c) {
        const size_t off = c == 0 ? 0 : half, len = c == 0 ? half : sink->bytes - half;
        CK(cudaStreamWaitEvent(sink->cs[c], sink->ev_x, 0));
        CK(cudaMemcpyAsync((char*)sink->host + off, (const char*)sink->dev + off, len,
                           cudaMemcpyDeviceToHost, sink->cs[c]));
        CK(cudaEventRecord(sink->ev_done[c], sink->cs[c]));
      }
      ++sink->copies;
    }
    if (prof) CK(cudaEventRecord(P.evr0, s));
    for (size_t gi = 0; gi < P.groups.size(); ++gi) {
      Group& g = P.groups[gi];
      if (rs_staged[gi] == 3)
        CK(launch_residual_staged_df(g.k, g.m, g.e, g.ncta[3], P.d_desc, g.d_ctas[3], P.d_ctl,
                                     s));
      else if (rs_staged[gi] == 2)
        CK(launch_residual_df(g.k, g.m, g.e, g.ncta[2], g.block, P.d_desc, g.d_ctas[2], P.d_ctl,
                              s));
      else if (rs_staged[gi] == 1)
        CK(launch_residual_staged(g.k, g.m, g.e, g.ncta[3], P.d_desc, g.d_ctas[3], P.d_ctl, s));
      else
        CK(launch_residual<T>(g.k, g.m, g.e, g.ncta[2], g.block, P.d_desc, g.d_ctas[2], P.d_ctl,
                              s));
    }
    if (prof) CK(cudaEventRecord(P.evr1, s));
    launches += 2 * ng;
    if ((rc = poll(P, s)) != SYLV_OK) break;
    ++polls;
    if (prof) {
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, P.evr0, P.evr1));
      ms_res += ms;
      ++n_res;
    }
    if (P.h_poll[1] == 0u) break;
    while (P.h_poll[0] > 0u) {
      if (polls > max_polls) {
        gave_up = true;
        break;
      }
      if ((rc = rebalance(P, true, s)) != SYLV_OK) return rc;
      if (o.use_graph) {
        CK(cudaGraphLaunch(P.graph, s));
      } else {
        if (prof) CK(cudaEventRecord(direct_events[0], s));
        for (int it = 0; it < iters; ++it) {
          rc = launch_inner_iteration<T>(P, s, prof ? direct_events[2 * it + 1] : nullptr,
                                         prof ? direct_events[2 * it + 2] : nullptr, false, it,
                                         iters);
          if (rc != SYLV_OK) return rc;
        }
      }
      launches += 2L * iters * ng;
      for (auto& g : P.groups) launches += g.csum;
      if ((rc = poll(P, s)) != SYLV_OK) return rc;
      ++polls;
      if (prof) {
        auto& ev = o.use_graph ? P.chunk_events : direct_events;
        for (int it = 0; it < iters; ++it) {
          float a = 0, b = 0;
          CK(cudaEventElapsedTime(&a, ev[2 * it], ev[2 * it + 1]));
          CK(cudaEventElapsedTime(&b, ev[2 * it + 1], ev[2 * it + 2]));
          ms_apply += a;
          ms_update += b;
        }
        n_apply += iters * (int)P.groups.size();
        n_update += iters * (int)P.groups.size();
      }
    }
    if (gave_up || polls > max_polls) {
      gave_up = true;
      break;
    }
  }
  if (rc != SYLV_OK) return rc;
  CK(cudaEventRecord(P.ev1, s));
  // read back per-column states
  int off = 0;
  for (int t = 0; t < nsys; ++t) {
    CK(cudaMemcpyAsync(P.h_states + off, P.work[t].st, P.R[t] * sizeof(ColState),
                       cudaMemcpyDeviceToHost, s));
    off += P.R[t];
  }
  CK(cudaStreamSynchronize(s));
  float ms_total = 0;
  CK(cudaEventElapsedTime(&ms_total, P.ev0, P.ev1));
  int worst = SYLV_OK;
  off = 0;
  for (int t = 0; t < nsys; ++t) {
    sylv_info inf;
    std::memset(&inf, 0, sizeof(inf));
    inf.status = SYLV_OK;
    for (int r = 0; r < P.R[t]; ++r) {
      const ColState& cs = P.h_states[off + r];
      int st = cs.status;
      if (cs.phase != PH_CONVERGED && cs.phase != PH_FAILED) st = SYLV_E_NOT_CONVERGED;
      if (cs.phase == PH_CONVERGED) st = SYLV_OK;
      if (st != SYLV_OK && (inf.status == SYLV_OK || st == SYLV_E_BREAKDOWN)) inf.status = st;
      inf.iterations = std::max(inf.iterations, cs.it);
      inf.outer = std::max(inf.outer, cs.outer);
      inf.relres = std::max(inf.relres, cs.relres);
    }
    off += P.R[t];
    inf.polls = polls;
    inf.ms_total = ms_total;
    inf.ms_apply = ms_apply;
    inf.ms_update = ms_update;
    inf.ms_residual = ms_res;
    inf.n_apply = n_apply;
    inf.n_update = n_update;
    inf.n_residual = n_res;
    inf.launches = (int32_t)std::min<long>(launches, INT32_MAX);
    if (!P.groups.empty()) {
      inf.tile = P.groups[0].block;
      inf.slots_mult = P.groups[0].mult;
      inf.apply_staged = P.groups[0].va;
      inf.update_staged = P.groups[0].vu;
      inf.residual_staged = rs_staged.empty() ? 0 : rs_staged[0];
    }
    if (infos) infos[t] = inf;
    if (inf.status != SYLV_OK && (worst == SYLV_OK || inf.status == SYLV_E_BREAKDOWN))
      worst = inf.status;
  }
  if (worst == SYLV_E_NOT_CONVERGED)
    store_error(gave_up ? "solve stopped: poll limit reached" : "tolerance not reached");
  if (worst == SYLV_E_BREAKDOWN) store_error("CG breakdown (non-positive or non-finite scalar)");
  return worst;
}

int check_opts(const sylv_opts& o) {
  if (!(o.tol > 0.0) || !(o.tol < 1.0)) return fail(SYLV_E_INVALID, "opts.tol must be in (0,1)");
  if (o.precision == SYLV_PREC_MIXED && (!(o.inner_tol > 0.0) || !(o.inner_tol < 1.0)))
    return fail(SYLV_E_INVALID, "opts.inner_tol must be in (0,1)");
  if (o.precision != SYLV_PREC_MIXED && o.precision != SYLV_PREC_F64)
    return fail(SYLV_E_INVALID, "opts.precision");
  if (o.precond != SYLV_PRECOND_NONE && o.precond != SYLV_PRECOND_BLOCK_JACOBI)
    return fail(SYLV_E_INVALID, "opts.precond");
  if (o.maxit < 1 || o.max_outer < 1) return fail(SYLV_E_INVALID, "opts.maxit/max_outer");
  if (o.check_every < 0 || o.check_every > 4096) return fail(SYLV_E_INVALID, "opts.check_every");
  return SYLV_OK;
}

}  // namespace

namespace sylv {
// Read-only view of a handle for other translation units of the library.
int handle_view(sylv_handle h, OpData* op, int* device) {
  if (!h) return SYLV_E_INVALID;
  *op = h->op;
  *device = h->device;
  return SYLV_OK;
}
void set_last_error(const char* msg) { store_error(msg); }
}  // namespace sylv

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" {

int sylv_opts_default(sylv_opts* o) {
  if (!o) return fail(SYLV_E_INVALID, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->inner_tol = 1e-4;
  o->maxit = 20000;
  o->max_outer = 30;
  o->precision = SYLV_PREC_MIXED;
  o->precond = SYLV_PRECOND_BLOCK_JACOBI;
  o->use_graph = 1;
  o->check_every = 0;
  o->profile = 0;
  o->use_x0 = 0;
  return SYLV_OK;
}

const char* sylv_strerror(int code) {
  switch (code) {
    case SYLV_OK: return "ok";
    case SYLV_E_INVALID: return "invalid argument";
    case SYLV_E_CUDA: return "CUDA error";
    case SYLV_E_NOMEM: return "out of device memory";
    case SYLV_E_NOT_CONVERGED: return "not converged";
    case SYLV_E_BREAKDOWN: return "CG breakdown";
    case SYLV_E_TIMEOUT: return "device wait timed out";
    case SYLV_E_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* sylv_last_error(void) { return g_last_error; }

static void free_handle(sylv_ctx* h) {
  if (!h) return;
  lanczos_release(h);
  h->plan[0].reset();
  h->plan[1].reset();
  cudaFree(h->ell_col);
  cudaFree(h->ell_val32);
  cudaFree(h->ell_val64);
  cudaFree(h->diag32);
  cudaFree(h->diag64);
  cudaFree(h->D32);
  cudaFree(h->D64);
  cudaFree(h->w32);
  cudaFree(h->w64);
  cudaFree(h->blk64);
  cudaFree(h->fac64);
  cudaFree(h->fs32);
  cudaFree(h->fl16);
  cudaFree(h->blk_hl);
  cudaFree(h->val_hl);
  cudaFree(h->apply_err);
  cudaFree(h->lam);
  cudaFree(h->grad_ws);
  cudaFree(h->var_ws);
  cudaFree(h->host_ws);
  for (auto e : h->ev_host)
    if (e) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->copy_stream2) cudaStreamDestroy(h->copy_stream2);
  delete h;
}

// Mixing matrix (explicit, or a_cj = (nu_c / nu0)^beta_j) and prior scalars into op.
static int set_scalars(OpData& op, const double* tau, const double* kappa, const double* nu,
                       const double* beta, const double* A, double nu0) {
  const int k = op.k, m = op.m;
  for (int j = 0; j < k; ++j) {
    if (!(tau[j] > 0.0) || !std::isfinite(tau[j]))
      return fail(SYLV_E_INVALID, "tau_j must be finite and > 0");
    if (!(kappa[j] >= 0.0) || !std::isfinite(kappa[j]))
      return fail(SYLV_E_INVALID, "kappa_j must be finite and >= 0");
  }
  double A64[MMAX * KMAX], logf[MMAX];
  for (int c = 0; c < m; ++c) {
    if (!A && !(nu[c] > 0.0)) return fail(SYLV_E_INVALID, "nu_c must be > 0");
    for (int j = 0; j < k; ++j) {
      const double a = A ? A[c * k + j] : std::pow(nu[c] / nu0, beta[j]);
      if (!std::isfinite(a)) return fail(SYLV_E_INVALID, "mixing matrix entry is not finite");
      A64[c * k + j] = a;
    }
    logf[c] = A ? 0.0 : std::log(nu[c] / nu0);
  }
  for (int c = 0; c < m; ++c) {
    for (int j = 0; j < k; ++j) {
      op.A64[c * k + j] = A64[c * k + j];
      op.A32[c * k + j] = (float)A64[c * k + j];
    }
    op.logf64[c] = logf[c];
  }
  for (int j = 0; j < k; ++j) {
    op.tau64[j] = tau[j];
    op.kappa64[j] = kappa[j];
    op.tk2_64[j] = tau[j] * kappa[j] * kappa[j];
    op.tau32[j] = (float)op.tau64[j];
    op.tk2_32[j] = (float)op.tk2_64[j];
    op.tau_hl[0][j] = (float)tau[j];
    op.tau_hl[1][j] = (float)(tau[j] - (double)op.tau_hl[0][j]);
  }
  return SYLV_OK;
}

// tau within the double-float residual's range (every nonzero operator entry in [2^-40, 2^40])
static bool tau_in_df_range(const OpData& op) {
  for (int j = 0; j < op.k; ++j)
    if (!(op.tau64[j] >= 0x1p-40 && op.tau64[j] <= 0x1p40)) return false;
  return true;
}

// FP32 pairs of the pixel blocks (and, with `vals`, of the ELL values) for the double-float
// residual; sets op.df_ok.  Synchronises s.
static int split_operator(sylv_ctx* h, OpData& op, bool vals, cudaStream_t s) {
  const size_t ld = (size_t)op.ld, nb = (size_t)op.k * (op.k + 1) / 2;
  const size_t ne = (size_t)std::max(op.E, 1);
  unsigned int* dflag = nullptr;
  unsigned int hflag[2] = {0, 0};
  cudaError_t e = cudaSuccess;
  if (!h->blk_hl) e = dalloc(&h->blk_hl, 2 * nb * ld * sizeof(float));
  if (e == cudaSuccess && !h->val_hl) e = dalloc(&h->val_hl, 2 * ne * ld * sizeof(float));
  if (e == cudaSuccess) e = dalloc(&dflag, 2 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, 2 * sizeof(unsigned int), s);
  if (e == cudaSuccess) e = launch_split_hl(op.blk64, nb, ld, h->blk_hl, dflag, s);
  if (e == cudaSuccess && vals) {
    e = cudaMemsetAsync(h->val_hl, 0, 2 * ne * ld * sizeof(float), s);
    if (e == cudaSuccess && op.E > 0)
      e = launch_split_hl(op.ell_val64, op.E, ld, h->val_hl, dflag + 1, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hflag, dflag, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dflag);
  if (e != cudaSuccess) return cuda_fail(e, "double-float operator copies");
  if (vals) h->val_df_bad = hflag[1] != 0;
  op.blk_hl = h->blk_hl;
  op.val_hl = h->val_hl;
  op.df_ok = (hflag[0] == 0 && !h->val_df_bad && tau_in_df_range(op)) ? 1 : 0;
  return SYLV_OK;
}

int sylv_create(sylv_handle* out, const sylv_problem* p, sylv_stream stream) {
  if (!out) return fail(SYLV_E_INVALID, "handle pointer is NULL");
  *out = nullptr;
  if (!p) return fail(SYLV_E_INVALID, "problem is NULL");
  if (p->n < 1) return fail(SYLV_E_INVALID, "n must be >= 1");
  if (p->n > (int64_t)INT32_MAX) return fail(SYLV_E_UNSUPPORTED, "n exceeds 2^31-1");
  if (p->k < 1 || p->m < 1) return fail(SYLV_E_INVALID, "k and m must be >= 1");
  if (p->k > KMAX) return fail(SYLV_E_UNSUPPORTED, "k exceeds SYLV_MAX_K");
  if (p->m > MMAX) return fail(SYLV_E_UNSUPPORTED, "m exceeds SYLV_MAX_M");
  if (p->ld < p->n) return fail(SYLV_E_INVALID, "ld must be >= n");
  if (!p->L_rowptr || !p->L_col || !p->L_val || !p->D || !p->tau || !p->kappa)
    return fail(SYLV_E_INVALID, "required pointer is NULL");
  if (p->nnz < 0 || p->nnz > (int64_t)INT32_MAX) return fail(SYLV_E_INVALID, "nnz out of range");
  if (!p->A && (!p->nu || !p->beta))
    return fail(SYLV_E_INVALID, "give A, or nu and beta for the power-law mixing");
  const double nu0 = p->nu0 > 0.0 ? p->nu0 : 100.0;
  cudaStream_t s = (cudaStream_t)stream;
  sylv_ctx* h = new sylv_ctx();
  cudaGetDevice(&h->device);
  OpData& op = h->op;
  op.n = p->n;
  op.ld = ceil_div(p->n, TILE_PX) * TILE_PX;
  op.ldu = p->ld;
  op.k = p->k;
  op.m = p->m;
  op.has_w = p->w != nullptr;
  h->nu0 = nu0;
  {
    const int rc0 = set_scalars(op, p->tau, p->kappa, p->nu, p->beta, p->A, nu0);
    if (rc0 != SYLV_OK) {
      free_handle(h);
      return rc0;
    }
  }
  h->explicit_A = p->A != nullptr;
  // validate the CSR and find the ELL width
  unsigned int* dflags = nullptr;
  auto bail = [&](int code) {
    cudaFree(dflags);
    free_handle(h);
    return code;
  };
  cudaError_t e = dalloc(&dflags, 2 * sizeof(unsigned int));
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
  unsigned int hflags[2] = {0, 0};
  if ((e = cudaMemsetAsync(dflags, 0, 2 * sizeof(unsigned int), s)) != cudaSuccess ||
      (e = launch_csr_check(op, p->L_rowptr, p->L_col, p->nnz, dflags, dflags + 1, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(hflags, dflags, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return bail(cuda_fail(e, "CSR validation"));
  if (hflags[0]) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "invalid Laplacian CSR (flags 0x%x: 1 rowptr, 2 column, "
                  "4 rowptr[0]/rowptr[n]/nnz, 16 more than %d off-diagonals in a row)",
                  hflags[0], EMAX);
    return bail(fail((hflags[0] & 16u) && !(hflags[0] & 15u) ? SYLV_E_UNSUPPORTED
                                                             : SYLV_E_INVALID, msg));
  }
  const int E = (int)hflags[1];
  op.E = E;
  const size_t ld = (size_t)op.ld;
  if ((e = dalloc(&h->ell_col, std::max<size_t>(E, 1) * ld * sizeof(int32_t))) != cudaSuccess ||
      (e = dalloc(&h->ell_val32, std::max<size_t>(E, 1) * ld * sizeof(float))) != cudaSuccess ||
      (e = dalloc(&h->ell_val64, std::max<size_t>(E, 1) * ld * sizeof(double))) != cudaSuccess ||
      (e = dalloc(&h->diag32, ld * sizeof(float))) != cudaSuccess ||
      (e = dalloc(&h->diag64, ld * sizeof(double))) != cudaSuccess ||
      (e = dalloc(&h->D32, (size_t)p->m * ld * sizeof(float))) != cudaSuccess ||
      (e = dalloc(&h->D64, (size_t)p->m * ld * sizeof(double))) != cudaSuccess)
    return bail(cuda_fail(e, "cudaMalloc (operator data)"));
  if (p->w) {
    if ((e = dalloc(&h->w32, ld * sizeof(float))) != cudaSuccess ||
        (e = dalloc(&h->w64, ld * sizeof(double))) != cudaSuccess)
      return bail(cuda_fail(e, "cudaMalloc (mass diagonal)"));
  }
  // zero the padding so every buffer is defined
  if ((e = cudaMemsetAsync(h->diag32, 0, ld * sizeof(float), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->diag64, 0, ld * sizeof(double), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->D32, 0, (size_t)p->m * ld * sizeof(float), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->D64, 0, (size_t)p->m * ld * sizeof(double), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->ell_col, 0, std::max<size_t>(E, 1) * ld * sizeof(int32_t), s)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(h->ell_val32, 0, std::max<size_t>(E, 1) * ld * sizeof(float), s)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(h->ell_val64, 0, std::max<size_t>(E, 1) * ld * sizeof(double), s)) !=
          cudaSuccess)
    return bail(cuda_fail(e, "cudaMemsetAsync"));
  op.ell_col = h->ell_col;
  op.ell_val32 = h->ell_val32;
  op.ell_val64 = h->ell_val64;
  op.diag32 = h->diag32;
  op.diag64 = h->diag64;
  op.D32 = h->D32;
  op.D64 = h->D64;
  op.w32 = h->w32;
  op.w64 = h->w64;
  if ((e = cudaMemsetAsync(dflags, 0, sizeof(unsigned int), s)) != cudaSuccess ||
      (e = launch_ell_build(op, p->L_rowptr, p->L_col, p->L_val, h->ell_col, h->ell_val32,
                            h->ell_val64, h->diag32, h->diag64, E, s)) != cudaSuccess ||
      (e = launch_convert_check(p->D, p->m, p->n, p->ld, op.ld, h->D32, h->D64, 0, dflags, s)) !=
          cudaSuccess)
    return bail(cuda_fail(e, "operator set-up"));
  if (p->w) {
    if ((e = cudaMemsetAsync(h->w32, 0, ld * sizeof(float), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->w64, 0, ld * sizeof(double), s)) != cudaSuccess ||
        (e = launch_convert_check(p->w, 1, p->n, p->ld, op.ld, h->w32, h->w64, 1, dflags, s)) !=
            cudaSuccess)
      return bail(cuda_fail(e, "mass diagonal set-up"));
  }
  if ((e = cudaMemcpyAsync(hflags, dflags, sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return bail(cuda_fail(e, "operator set-up"));
  if (hflags[0]) return bail(fail(SYLV_E_INVALID, "D (>= 0) or w (> 0) has invalid entries"));
  if (p->prior == SYLV_PRIOR_IGMRF) {
    // intrinsic GMRF prior shape: replace L by L^2 (formed from the ELL copy of L)
    unsigned int width = 0;
    if ((e = cudaMemsetAsync(dflags, 0, sizeof(unsigned int), s)) != cudaSuccess ||
        (e = launch_square_count(op, dflags, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&width, dflags, sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return bail(cuda_fail(e, "prior L^2 (width)"));
    if (width > (unsigned)SYLV_MAX_PRIOR_DEGREE)
      return bail(fail(SYLV_E_UNSUPPORTED, "L^2 has more than SYLV_MAX_PRIOR_DEGREE "
                                           "off-diagonals in a row"));
    const int E2 = (int)width;
    int32_t* sq_col = nullptr;
    float *sq_val32 = nullptr, *sq_diag32 = nullptr;
    double *sq_val64 = nullptr, *sq_diag64 = nullptr;
    auto drop = [&]() {
      cudaFree(sq_col);
      cudaFree(sq_val32);
      cudaFree(sq_val64);
      cudaFree(sq_diag32);
      cudaFree(sq_diag64);
    };
    const size_t w2 = std::max<size_t>(E2, 1);
    if ((e = dalloc(&sq_col, w2 * ld * sizeof(int32_t))) != cudaSuccess ||
        (e = dalloc(&sq_val32, w2 * ld * sizeof(float))) != cudaSuccess ||
        (e = dalloc(&sq_val64, w2 * ld * sizeof(double))) != cudaSuccess ||
        (e = dalloc(&sq_diag32, ld * sizeof(float))) != cudaSuccess ||
        (e = dalloc(&sq_diag64, ld * sizeof(double))) != cudaSuccess ||
        (e = cudaMemsetAsync(sq_col, 0, w2 * ld * sizeof(int32_t), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(sq_val32, 0, w2 * ld * sizeof(float), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(sq_val64, 0, w2 * ld * sizeof(double), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(sq_diag32, 0, ld * sizeof(float), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(sq_diag64, 0, ld * sizeof(double), s)) != cudaSuccess ||
        (e = launch_square_fill(op, E2, sq_col, sq_val32, sq_val64, sq_diag32, sq_diag64, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      drop();
      return bail(cuda_fail(e, "prior L^2"));
    }
    cudaFree(h->ell_col);
    cudaFree(h->ell_val32);
    cudaFree(h->ell_val64);
    cudaFree(h->diag32);
    cudaFree(h->diag64);
    h->ell_col = sq_col;
    h->ell_val32 = sq_val32;
    h->ell_val64 = sq_val64;
    h->diag32 = sq_diag32;
    h->diag64 = sq_diag64;
    op.E = E2;
    op.ell_col = sq_col;
    op.ell_val32 = sq_val32;
    op.ell_val64 = sq_val64;
    op.diag32 = sq_diag32;
    op.diag64 = sq_diag64;
  } else if (p->prior != SYLV_PRIOR_GMRF) {
    return bail(fail(SYLV_E_INVALID, "prior must be SYLV_PRIOR_GMRF or SYLV_PRIOR_IGMRF"));
  }
  // FP64 pixel blocks and their factors (FP64 operator and preconditioner)
  const size_t nb = (size_t)p->k * (p->k + 1) / 2;
  if ((e = dalloc(&h->blk64, nb * ld * sizeof(double))) != cudaSuccess ||
      (e = dalloc(&h->fac64, (nb + p->k) * ld * sizeof(double))) != cudaSuccess ||
      (e = cudaMemsetAsync(h->blk64, 0, nb * ld * sizeof(double), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->fac64, 0, (nb + p->k) * ld * sizeof(double), s)) != cudaSuccess ||
      (e = dalloc(&h->fs32, (size_t)p->k * ld * sizeof(float))) != cudaSuccess ||
      (e = dalloc(&h->fl16, ((nb + 1) / 2) * ld * sizeof(__half2))) != cudaSuccess ||
      (e = cudaMemsetAsync(h->fs32, 0, (size_t)p->k * ld * sizeof(float), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->fl16, 0, ((nb + 1) / 2) * ld * sizeof(__half2), s)) !=
          cudaSuccess)
    return bail(cuda_fail(e, "cudaMalloc (pixel blocks)"));
  op.blk64 = h->blk64;
  op.fac64 = h->fac64;
  op.fs32 = h->fs32;
  op.fl16 = h->fl16;
  if ((e = launch_block_setup(op, h->blk64, h->fac64, h->fs32, h->fl16, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return bail(cuda_fail(e, "pixel-block set-up"));
  {
    const int rc2 = split_operator(h, op, true, s);
    if (rc2 != SYLV_OK) return bail(rc2);
  }
  cudaFree(dflags);
  *out = h;
  return SYLV_OK;
}

int sylv_set_params(sylv_handle h, const double* tau, const double* kappa, const double* nu,
                    const double* beta, const double* A, sylv_stream stream) {
  if (!h || !tau || !kappa) return fail(SYLV_E_INVALID, "NULL argument");
  if (!A && (!nu || !beta)) return fail(SYLV_E_INVALID, "give A, or nu and beta");
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  OpData op = h->op;
  int rc = set_scalars(op, tau, kappa, nu, beta, A, h->nu0);
  if (rc != SYLV_OK) return rc;
  // the pixel blocks and their factors depend on tau, kappa and A
  CK(launch_block_setup(op, h->blk64, h->fac64, h->fs32, h->fl16, s));
  CK(cudaStreamSynchronize(s));
  rc = split_operator(h, op, false, s);
  if (rc != SYLV_OK) return rc;
  h->op = op;
  h->explicit_A = A != nullptr;
  lanczos_release(h);   // separability and Lhat were derived from the old scalars
  return SYLV_OK;
}

void sylv_destroy(sylv_handle h) {
  if (!h) return;
  DeviceGuard g(h->device);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
      bool uses = std::find(it->second->hs.begin(), it->second->hs.end(), h) !=
                  it->second->hs.end();
      it = uses ? g_plans.erase(it) : std::next(it);
    }
  }
  free_handle(h);
}

int sylv_rhs(sylv_handle h, const double* Yobs, double* B, int nrhs, sylv_stream s) {
  if (!h || !Yobs || !B) return fail(SYLV_E_INVALID, "NULL argument");
  if (nrhs < 1) return fail(SYLV_E_INVALID, "nrhs must be >= 1");
  DeviceGuard g(h->device);
  CK(launch_rhs(h->op, Yobs, B, nrhs, (cudaStream_t)s));
  return SYLV_OK;
}

int sylv_apply(sylv_handle h, const void* X, void* Y, int nrhs, int dtype, sylv_stream s) {
  if (!h || !X || !Y) return fail(SYLV_E_INVALID, "NULL argument");
  if (nrhs < 1) return fail(SYLV_E_INVALID, "nrhs must be >= 1");
  DeviceGuard g(h->device);
  if (dtype == SYLV_F32) {
    if (!h->apply_err) {
      CK(dalloc(&h->apply_err, 3 * sizeof(unsigned int)));
      CK(cudaMemset(h->apply_err, 0, 3 * sizeof(unsigned int)));
    }
    cudaError_t e = g_staged_apply ? launch_apply_staged(h->op, (const float*)X, (float*)Y, nrhs,
                                                         h->apply_err, (cudaStream_t)s)
                                   : cudaErrorNotSupported;
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      CK(launch_apply<float>(h->op, (const float*)X, (float*)Y, nrhs, (cudaStream_t)s));
    } else if (e != cudaSuccess) {
      return cuda_fail(e, "staged apply");
    }
  } else if (dtype == SYLV_F64) {
    CK(launch_apply<double>(h->op, (const double*)X, (double*)Y, nrhs, (cudaStream_t)s));
  } else {
    return fail(SYLV_E_INVALID, "dtype must be SYLV_F32 or SYLV_F64");
  }
  return SYLV_OK;
}

int sylv_residual(sylv_handle h, const double* B, const double* X, int nrhs, double* R,
                  sylv_stream s) {
  if (!h || !B || !X || !R) return fail(SYLV_E_INVALID, "NULL argument");
  if (nrhs < 1) return fail(SYLV_E_INVALID, "nrhs must be >= 1");
  DeviceGuard g(h->device);
  CK(launch_residual_out(h->op, B, X, nrhs, R, h->op.df_ok, (cudaStream_t)s));
  return SYLV_OK;
}

static int solve_impl(int nsys, const sylv_handle* hs, const double* const* B, double* const* X,
                      const int* nrhs, const sylv_opts* o_in, sylv_info* infos,
                      cudaStream_t s, bool single, HostSink* sink = nullptr) {
  sylv_opts o;
  if (o_in) o = *o_in;
  else sylv_opts_default(&o);
  int rc = check_opts(o);
  if (rc != SYLV_OK) return rc;
  if (nsys < 1 || !hs || !B || !X || !nrhs) return fail(SYLV_E_INVALID, "NULL or empty arrays");
  for (int t = 0; t < nsys; ++t) {
    if (!hs[t] || !B[t] || !X[t]) return fail(SYLV_E_INVALID, "NULL handle or buffer");
    if (nrhs[t] < 1 || nrhs[t] > RMAX) return fail(SYLV_E_INVALID, "nrhs out of 1..SYLV_MAX_RHS");
    if (hs[t]->device != hs[0]->device)
      return fail(SYLV_E_INVALID, "all handles must live on one device");
  }
  DeviceGuard g(hs[0]->device);
  const int inner_double = o.precision == SYLV_PREC_F64 ? 1 : 0;
  Plan* P = nullptr;
  std::unique_lock<std::mutex> lk(g_plan_mu, std::defer_lock);
  if (single) {
    auto& slot = hs[0]->plan[inner_double];
    if (!slot || slot->R[0] != nrhs[0]) {
      slot.reset(new Plan());
      rc = build_plan(*slot, 1, hs, nrhs, inner_double);
      if (rc != SYLV_OK) {
        slot.reset();
        return rc;
      }
    }
    P = slot.get();
  } else {
    std::vector<uintptr_t> key;
    key.push_back((uintptr_t)inner_double);
    for (int t = 0; t < nsys; ++t) {
      key.push_back((uintptr_t)hs[t]);
      key.push_back((uintptr_t)nrhs[t]);
    }
    lk.lock();
    auto it = g_plans.find(key);
    if (it == g_plans.end()) {
      std::unique_ptr<Plan> np(new Plan());
      rc = build_plan(*np, nsys, hs, nrhs, inner_double);
      if (rc != SYLV_OK) return rc;
      it = g_plans.emplace(key, std::move(np)).first;
    }
    P = it->second.get();
  }
  return inner_double ? run_plan<double>(*P, B, X, o, infos, s, sink)
                      : run_plan<float>(*P, B, X, o, infos, s, sink);
}

int sylv_solve(sylv_handle h, const double* B, double* X, int nrhs, const sylv_opts* o,
               sylv_info* info, sylv_stream s) {
  if (!h) return fail(SYLV_E_INVALID, "NULL handle");
  const double* Bs[1] = {B};
  double* Xs[1] = {X};
  int R[1] = {nrhs};
  return solve_impl(1, &h, Bs, Xs, R, o, info, (cudaStream_t)s, true);
}

int sylv_solve_host(sylv_handle h, const double* Yobs, double* X, int nrhs, const sylv_opts* o_in,
                    sylv_info* info, sylv_stream stream) {
  if (!h || !Yobs || !X) return fail(SYLV_E_INVALID, "NULL argument");
  if (nrhs < 1 || nrhs > RMAX) return fail(SYLV_E_INVALID, "nrhs out of 1..SYLV_MAX_RHS");
  sylv_opts o;
  if (o_in) o = *o_in;
  else sylv_opts_default(&o);
  int rc = check_opts(o);
  if (rc != SYLV_OK) return rc;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const OpData& op = h->op;
  const size_t ye = (size_t)nrhs * op.m * op.ldu, xe = (size_t)nrhs * op.k * op.ldu;
  const size_t bytes = (ye + 2 * xe) * sizeof(double);
  if (h->host_bytes < bytes) {
    cudaFree(h->host_ws);
    h->host_ws = nullptr;
    h->host_bytes = 0;
    CK(dalloc(&h->host_ws, bytes));
    h->host_bytes = bytes;
  }
  // created on first use; each is kept only once it exists, so a failed call is retried whole
  for (cudaStream_t* cs : {&h->copy_stream, &h->copy_stream2}) {
    if (*cs) continue;
    cudaStream_t t = nullptr;
    CK(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
    *cs = t;
  }
  for (auto& e : h->ev_host) {
    if (e) continue;
    cudaEvent_t t = nullptr;
    CK(cudaEventCreateWithFlags(&t, cudaEventDisableTiming));
    e = t;
  }
  constexpr int NSLICE = 8;
  // [0, NSLICE): slices, NSLICE: start, +1: X updated, +2, +3: copies back finished
  cudaEvent_t* ev = h->ev_host;
  double* Yd = h->host_ws;
  double* Bd = Yd + ye;
  double* Xd = Bd + xe;
  cudaStream_t cs = h->copy_stream;
  // the copy stream follows the work already queued on s
  CK(cudaEventRecord(ev[NSLICE], s));
  CK(cudaStreamWaitEvent(cs, ev[NSLICE], 0));
  if (o.use_x0) CK(cudaMemcpyAsync(Xd, X, xe * sizeof(double), cudaMemcpyHostToDevice, cs));
  const int64_t n = op.n;
  // page-locked maps: the right-hand-side kernel reads them where they are, through their
  // device alias (no staging copy); pageable ones go to the device in pixel slices, the
  // right-hand side of a slice being formed while the next one is copied
  cudaPointerAttributes pa{};
  const bool direct = cudaPointerGetAttributes(&pa, Yobs) == cudaSuccess &&
                      pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr;
  (void)cudaGetLastError();
  if (direct) {
    if (o.use_x0) {
      CK(cudaEventRecord(ev[0], cs));
      CK(cudaStreamWaitEvent(s, ev[0], 0));
    }
    CK(launch_rhs(op, (const double*)pa.devicePointer, Bd, nrhs, s));
  } else {
    const int nsl = n >= (int64_t)NSLICE * 4096 ? NSLICE : 1;
    const size_t pitch = (size_t)op.ldu * sizeof(double);
    for (int q = 0; q < nsl; ++q) {
      const int64_t i0 = n * q / nsl, i1 = n * (q + 1) / nsl;
      CK(cudaMemcpy2DAsync(Yd + i0, pitch, Yobs + i0, pitch, (size_t)(i1 - i0) * sizeof(double),
                           (size_t)nrhs * op.m, cudaMemcpyHostToDevice, cs));
      CK(cudaEventRecord(ev[q], cs));
      CK(cudaStreamWaitEvent(s, ev[q], 0));
      CK(launch_rhs_range(op, Yd, Bd, nrhs, i0, i1, s));
    }
  }
  HostSink sink;
  sink.cs[0] = cs;
  sink.cs[1] = h->copy_stream2;
  sink.ev_x = ev[NSLICE + 1];
  sink.ev_done[0] = ev[NSLICE + 2];
  sink.ev_done[1] = ev[NSLICE + 3];
  sink.host = X;
  sink.dev = Xd;
  sink.bytes = xe * sizeof(double);
  const double* Bs[1] = {Bd};
  double* Xs[1] = {Xd};
  int R[1] = {nrhs};
  rc = solve_impl(1, &h, Bs, Xs, R, &o, info, s, true, &sink);
  cudaError_t e = cudaSuccess;
  if (sink.copies == 0) {   // the start was already the answer (or the solve stopped early)
    e = cudaMemcpyAsync(X, Xd, xe * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaError_t e2 = cudaStreamSynchronize(cs);
  const cudaError_t e3 = cudaStreamSynchronize(h->copy_stream2);
  if (e2 == cudaSuccess) e2 = e3;
  if (rc != SYLV_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "copy of the solution to the host");
  if (e2 != cudaSuccess) return cuda_fail(e2, "copy of the solution to the host");
  return SYLV_OK;
}

int sylv_solve_batched(int nsys, const sylv_handle* hs, const double* const* B,
                       double* const* X, const int* nrhs, const sylv_opts* o,
                       sylv_info* infos, sylv_stream s) {
  return solve_impl(nsys, hs, B, X, nrhs, o, infos, (cudaStream_t)s, false);
}

// The probe loop of sylv_variance and sylv_variance_probing: nprobe probes, SYLV_MAX_RHS at a
// time, each chunk's probes either the caller's (Z) or generated from a colouring (colour).
static int variance_impl(sylv_handle h, const double* Z, const int32_t* colour, int ncol,
                         int nprobe, double* var, const sylv_opts* o_in, sylv_info* info,
                         sylv_stream stream) {
  sylv_opts o;
  if (o_in) o = *o_in;
  else sylv_opts_default(&o);
  o.use_x0 = 0;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const OpData& op = h->op;
  const int chunk = std::min(nprobe, RMAX);
  const size_t xelems = (size_t)chunk * op.k * op.ldu, kelems = (size_t)op.k * op.ld;
  // X of a chunk, num, den, a flag word (and the chunk's generated probes)
  const size_t bytes = ((colour ? 2 : 1) * xelems + 2 * kelems + 1) * sizeof(double);
  if (h->var_bytes < bytes) {
    cudaFree(h->var_ws);
    h->var_ws = nullptr;
    h->var_bytes = 0;
    CK(dalloc(&h->var_ws, bytes));
    h->var_bytes = bytes;
  }
  double* X = h->var_ws;
  double* num = X + xelems;
  double* den = num + kelems;
  unsigned int* flag = (unsigned int*)(den + kelems);
  double* Zg = colour ? (double*)(flag + 2) : nullptr;
  CK(cudaMemsetAsync(num, 0, 2 * kelems * sizeof(double) + sizeof(double), s));
  sylv_info tot;
  std::memset(&tot, 0, sizeof(tot));
  int worst = SYLV_OK;
  for (int s0 = 0; s0 < nprobe; s0 += chunk) {
    const int r = std::min(chunk, nprobe - s0);
    const double* Zc = Z ? Z + (size_t)s0 * op.k * op.ldu : Zg;
    if (colour) CK(launch_probe_fill(op, colour, ncol, s0, r, Zg, flag, s));
    sylv_info inf;
    int rc = sylv_solve(h, Zc, X, r, &o, &inf, stream);
    if (rc != SYLV_OK && rc != SYLV_E_NOT_CONVERGED) return rc;
    if (rc != SYLV_OK) worst = rc;
    CK(launch_var_accum(op, Zc, X, r, num, den, s));
    tot.iterations = std::max(tot.iterations, inf.iterations);
    tot.outer = std::max(tot.outer, inf.outer);
    tot.polls += inf.polls;
    tot.relres = std::max(tot.relres, inf.relres);
    tot.ms_total += inf.ms_total;
    tot.ms_apply += inf.ms_apply;
    tot.ms_update += inf.ms_update;
    tot.ms_residual += inf.ms_residual;
    tot.launches += inf.launches + (colour ? 2 : 1);
    tot.tile = inf.tile;
    tot.slots_mult = inf.slots_mult;
    tot.apply_staged = inf.apply_staged;
    tot.update_staged = inf.update_staged;
    tot.residual_staged = inf.residual_staged;
  }
  CK(launch_var_finish(op, num, den, var, s));
  unsigned int hflag = 0;
  CK(cudaMemcpyAsync(&hflag, flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hflag) return fail(SYLV_E_INVALID, "a pixel's colour lies outside [0, ncolours)");
  tot.launches += 1;
  tot.status = worst;
  if (info) *info = tot;
  if (worst != SYLV_OK) store_error("a probe solve did not reach the tolerance");
  return worst;
}

int sylv_variance(sylv_handle h, const double* Z, int nprobe, double* var, const sylv_opts* o_in,
                  sylv_info* info, sylv_stream stream) {
  if (!h || !Z || !var) return fail(SYLV_E_INVALID, "NULL argument");
  if (nprobe < 1) return fail(SYLV_E_INVALID, "nprobe must be >= 1");
  return variance_impl(h, Z, nullptr, 0, nprobe, var, o_in, info, stream);
}

int sylv_variance_probing(sylv_handle h, const int32_t* colour, int ncolours, double* var,
                          const sylv_opts* o_in, sylv_info* info, sylv_stream stream) {
  if (!h || !colour || !var) return fail(SYLV_E_INVALID, "NULL argument");
  if (ncolours < 1) return fail(SYLV_E_INVALID, "ncolours must be >= 1");
  if ((int64_t)ncolours * h->op.k > INT32_MAX)
    return fail(SYLV_E_INVALID, "ncolours * k too large");
  return variance_impl(h, nullptr, colour, ncolours, ncolours * h->op.k, var, o_in, info,
                       stream);
}

int sylv_backward(sylv_handle h, const double* Xhat, const double* dLdX, const double* Yobs,
                  int nrhs, double* lambda, double* g_tau, double* g_kappa, double* g_beta,
                  const sylv_opts* o, sylv_info* info, sylv_stream stream) {
  if (!h || !Xhat || !dLdX) return fail(SYLV_E_INVALID, "NULL argument");
  if (nrhs < 1 || nrhs > RMAX) return fail(SYLV_E_INVALID, "nrhs out of range");
  if (g_beta && h->explicit_A)
    return fail(SYLV_E_INVALID, "g_beta needs the power-law mixing (handle has explicit A)");
  if (g_beta && !Yobs) return fail(SYLV_E_INVALID, "g_beta needs Yobs");
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const OpData& op = h->op;
  const size_t vbytes = (size_t)nrhs * op.k * op.ldu * sizeof(double);
  double* lam = lambda;
  if (!lam) {
    if (h->lam_bytes < vbytes) {
      cudaFree(h->lam);
      h->lam = nullptr;
      h->lam_bytes = 0;
      CK(dalloc(&h->lam, vbytes));
      h->lam_bytes = vbytes;
    }
    lam = h->lam;
  }
  // adjoint solve: G lambda = dl/dX (G is symmetric)
  int rc = sylv_solve(h, dLdX, lam, nrhs, o, info, stream);
  if (rc != SYLV_OK) return rc;
  const int ntiles = (int)ceil_div(op.n, 256);
  const size_t gbytes = ((size_t)ntiles * 3 * op.k + 3 * op.k) * sizeof(double);
  if (h->grad_bytes < gbytes) {
    cudaFree(h->grad_ws);
    h->grad_ws = nullptr;
    h->grad_bytes = 0;
    CK(dalloc(&h->grad_ws, gbytes));
    h->grad_bytes = gbytes;
  }
  double* out = h->grad_ws + (size_t)ntiles * 3 * op.k;
  CK(launch_grad(op, Xhat, lam, Yobs, nrhs, g_beta ? 1 : 0, h->grad_ws, ntiles, out, s));
  double host[3 * KMAX];
  CK(cudaMemcpyAsync(host, out, 3 * op.k * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int j = 0; j < op.k; ++j) {
    if (g_tau) g_tau[j] = host[j];
    if (g_kappa) g_kappa[j] = host[op.k + j];
    if (g_beta) g_beta[j] = host[2 * op.k + j];
  }
  return SYLV_OK;
}

}  // extern "C"
