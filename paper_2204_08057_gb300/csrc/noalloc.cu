// sylv_solve_noalloc: the solve of sylv_solve for callers that must not allocate memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where they
// solve: a real-time or embedded pipeline whose memory is reserved once at start-up, a host
// process running under a fixed device-memory budget shared with other work, or code that
// must not trigger an allocator's implicit device synchronisation or pool growth in the middle
// of a latency-sensitive loop.  For them this entry point runs the same preconditioned CG
// iteration inside FP64 iterative refinement as sylv_solve, but every byte of its workspace
// (descriptor, CTA list, control word, per-column CG state, partial sums and the five inner
// vectors) lives in one file-scope device array, g_scratch, of SOLVE_SCRATCH_BYTES.
//
// Properties (also stated in include/sylv.h):
// * Nothing is allocated: no cudaMalloc/cudaFree, no pinned host buffers, no events, no CUDA
//   graphs, no heap memory on the host (error messages go to a fixed per-thread buffer);
//   control data travels through stack variables.
// * The array exists once per device for the life of the process (every GPU that loads the
//   library holds it).  Its device address is looked up with cudaGetSymbolAddress the first
//   time the entry point runs on a device (with that device current); that first call should
//   therefore come before any stream capture.  The address is kept for the process: after a
//   cudaDeviceReset (which also invalidates every handle) the module may load elsewhere, so
//   neither handles nor this entry point may be used after one.
// * Every return leaves the stream idle: on an error after the first launch the call waits
//   for the work it queued before it returns.
// * Every call shares the array, so calls that overlap on the GPU (two streams, two threads)
//   race and corrupt each other; serialise them.  Each call rewrites everything it reads
//   before reading it (the kernels that start a solve clear the counters and CG state).
// * Problems whose workspace does not fit are rejected with SYLV_E_UNSUPPORTED.
#include <chrono>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sylv_internal.cuh"

namespace sylv {
namespace {

constexpr size_t SOLVE_SCRATCH_BYTES = size_t(16) << 20;  // 16 MiB per device
constexpr int MAX_DEVICES = 64;
constexpr int MAX_NOALLOC_CTAS = 4096;

static __device__ __align__(256) unsigned char g_scratch[SOLVE_SCRATCH_BYTES];

std::mutex g_scratch_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int fail_msg(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

int cuda_msg(cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  set_last_error(buf);
  (void)cudaGetLastError();
  return SYLV_E_CUDA;
}

#define NA_CK(call)                                        \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return cuda_msg(_e, #call);     \
  } while (0)

// The same inside the solve loop, where kernels may already be queued on s: before returning,
// wait (ignoring the result) until they have finished, so that no return leaves work running
// on the shared array, which the caller's next call would race with.
#define NA_CK_DRAIN(call)                                  \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) {                               \
      const int _rc = cuda_msg(_e, #call);                 \
      (void)cudaStreamSynchronize(s);                      \
      (void)cudaGetLastError();                            \
      return _rc;                                          \
    }                                                      \
  } while (0)

struct Poll {
  unsigned int n_active, n_unfinished, error, pad;
};

template <typename T>
int solve_in_scratch(const OpData& op, int device, const double* B, double* X, int R,
                     const sylv_opts& o, sylv_info* info, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const int K = op.k;
  const int ntiles = (int)((op.n + TILE_PX - 1) / TILE_PX);
  int nsm = 1;
  NA_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
  const int oa = occupancy<T>(0, op.k, op.m, op.E, 0, TILE_PX);
  const int ou = occupancy<T>(1, op.k, op.m, op.E, 0, TILE_PX);
  const int occ = oa < ou ? oa : ou;
  int nslots = ntiles < nsm * occ ? ntiles : nsm * occ;
  if (nslots > MAX_NOALLOC_CTAS) nslots = MAX_NOALLOC_CTAS;
  if (nslots < 1) nslots = 1;

  // scratch layout, every section 256-byte aligned
  const size_t vbytes = (size_t)R * K * op.ld * sizeof(T);
  size_t off = 0;
  const size_t o_ctl = off;     off = align256(off + sizeof(Control));
  const size_t o_desc = off;    off = align256(off + sizeof(SysDesc));
  const size_t o_cta = off;     off = align256(off + nslots * sizeof(CtaRef));
  const size_t o_st = off;      off = align256(off + R * sizeof(ColState));
  const size_t o_cnt = off;     off = align256(off + sizeof(unsigned int));
  const size_t o_cols = off;    off = align256(off + 2 * R * sizeof(int));
  const size_t o_part = off;    off = align256(off + (size_t)nslots * R * NPART * sizeof(double));
  const size_t o_vec = off;     off = align256(off + 5 * vbytes);
  if (off > SOLVE_SCRATCH_BYTES) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "sylv_solve_noalloc: workspace of %zu bytes exceeds the %zu-byte scratch array "
                  "(nrhs * k * n too large; use sylv_solve)", off, SOLVE_SCRATCH_BYTES);
    return fail_msg(SYLV_E_UNSUPPORTED, buf);
  }
  void* base_v = nullptr;
  NA_CK(scratch_address(device, &base_v));
  unsigned char* base = (unsigned char*)base_v;

  Control ctl;
  std::memset(&ctl, 0, sizeof ctl);
  ctl.tol2 = o.tol * o.tol;
  ctl.tol_in2 = o.precision == SYLV_PREC_MIXED ? o.inner_tol * o.inner_tol : 0.0;
  ctl.safety2 = 0.25;
  ctl.maxit = o.maxit;
  ctl.max_outer = o.max_outer;
  ctl.precond = o.precond;
  ctl.x0_zero = o.use_x0 ? 0 : 1;

  SysDesc sd;
  std::memset(&sd, 0, sizeof sd);
  sd.op = op;
  sd.R = R;
  sd.ntiles = ntiles;
  sd.nslots[0] = nslots;
  sd.nslots[1] = nslots;
  sd.nslots[2] = nslots;
  sd.B = B;
  sd.X = X;
  unsigned char* vec = base + o_vec;
  sd.vd = vec;
  sd.vr = vec + vbytes;
  sd.vz = vec + 2 * vbytes;
  sd.vp = vec + 3 * vbytes;
  sd.vq = vec + 4 * vbytes;
  sd.st = (ColState*)(base + o_st);
  sd.partial = (double*)(base + o_part);
  sd.counter = (unsigned int*)(base + o_cnt);

  CtaRef ctas[MAX_NOALLOC_CTAS];
  for (int t = 0; t < nslots; ++t) ctas[t] = CtaRef{0, t};
  int cols[2 * RMAX];
  for (int r = 0; r < R; ++r) {
    cols[r] = 0;       // system of column r
    cols[R + r] = r;   // right-hand side of column r
  }
  Control* d_ctl = (Control*)(base + o_ctl);
  SysDesc* d_desc = (SysDesc*)(base + o_desc);
  CtaRef* d_cta = (CtaRef*)(base + o_cta);
  int* d_cols = (int*)(base + o_cols);
  // host -> device from stack memory; the copies are staged before each call returns
  NA_CK(cudaMemcpyAsync(d_ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_desc, &sd, sizeof sd, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_cta, ctas, nslots * sizeof(CtaRef), cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_cols, cols, 2 * R * sizeof(int), cudaMemcpyHostToDevice, s));
  if (!o.use_x0)
    NA_CK(cudaMemsetAsync(X, 0, (size_t)R * K * op.ldu * sizeof(double), s));
  NA_CK_DRAIN(launch_init_states(R, d_cols, d_cols + R, d_desc, d_ctl, s));
  long launches = 1;

  const int iters = o.check_every > 0 ? o.check_every : 16;
  const long max_polls = (long)o.maxit / iters + 4L * (o.max_outer + 2) + 16;
  long polls = 0;
  Poll pl;
  auto poll = [&]() -> int {
    NA_CK_DRAIN(cudaMemcpyAsync(&pl, d_ctl, sizeof pl, cudaMemcpyDeviceToHost, s));
    NA_CK_DRAIN(cudaStreamSynchronize(s));
    ++polls;
    if (pl.error) return fail_msg(SYLV_E_TIMEOUT, "a bounded device-side wait expired");
    return SYLV_OK;
  };
  int rc = SYLV_OK;
  bool gave_up = false;
  while (true) {
    NA_CK_DRAIN(launch_update_x<T>(K, nslots, TILE_PX, d_desc, d_cta, s));
    NA_CK_DRAIN(launch_residual<T>(K, op.m, op.E, nslots, TILE_PX, d_desc, d_cta, d_ctl, s));
    launches += 2;
    if ((rc = poll()) != SYLV_OK) return rc;
    if (pl.n_unfinished == 0u) break;
    while (pl.n_active > 0u) {
      if (polls > max_polls) {
        gave_up = true;
        break;
      }
      for (int it = 0; it < iters; ++it) {
        NA_CK_DRAIN(launch_inner_apply<T>(K, op.m, op.E, 0, nslots, TILE_PX, d_desc, d_cta,
                                          d_ctl, s));
        NA_CK_DRAIN(launch_inner_update<T>(K, op.m, op.E, 0, nslots, TILE_PX, d_desc, d_cta, d_ctl,
                                     s));
      }
      launches += 2L * iters;
      if ((rc = poll()) != SYLV_OK) return rc;
    }
    if (gave_up || polls > max_polls) {
      gave_up = true;
      break;
    }
  }
  ColState st[RMAX];
  NA_CK_DRAIN(cudaMemcpyAsync(st, sd.st, R * sizeof(ColState), cudaMemcpyDeviceToHost, s));
  NA_CK_DRAIN(cudaStreamSynchronize(s));
  sylv_info inf;
  std::memset(&inf, 0, sizeof inf);
  for (int r = 0; r < R; ++r) {
    int code = st[r].status;
    if (st[r].phase == PH_CONVERGED) code = SYLV_OK;
    else if (st[r].phase != PH_FAILED) code = SYLV_E_NOT_CONVERGED;
    if (code != SYLV_OK && (inf.status == SYLV_OK || code == SYLV_E_BREAKDOWN)) inf.status = code;
    inf.iterations = inf.iterations > st[r].it ? inf.iterations : st[r].it;
    inf.outer = inf.outer > st[r].outer ? inf.outer : st[r].outer;
    inf.relres = inf.relres > st[r].relres ? inf.relres : st[r].relres;
  }
  inf.polls = (int32_t)polls;
  inf.launches = (int32_t)launches;
  inf.tile = TILE_PX;
  inf.slots_mult = 1;
  inf.ms_total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (inf.status == SYLV_E_NOT_CONVERGED)
    set_last_error(gave_up ? "solve stopped: poll limit reached" : "tolerance not reached");
  if (inf.status == SYLV_E_BREAKDOWN) set_last_error("CG breakdown");
  return inf.status;
}

}  // namespace
}  // namespace sylv

extern "C" int sylv_solve_noalloc(sylv_handle h, const double* B, double* X, int nrhs,
                                  const sylv_opts* o_in, sylv_info* info, sylv_stream stream) {
  using namespace sylv;
  if (!h || !B || !X) return fail_msg(SYLV_E_INVALID, "NULL argument");
  if (nrhs < 1 || nrhs > RMAX) return fail_msg(SYLV_E_INVALID, "nrhs out of 1..SYLV_MAX_RHS");
  sylv_opts o;
  if (o_in) {
    o = *o_in;
  } else {
    sylv_opts_default(&o);
  }
  if (!(o.tol > 0.0) || !(o.tol < 1.0)) return fail_msg(SYLV_E_INVALID, "opts.tol must be in (0,1)");
  if (o.precision != SYLV_PREC_MIXED && o.precision != SYLV_PREC_F64)
    return fail_msg(SYLV_E_INVALID, "opts.precision");
  if (o.precision == SYLV_PREC_MIXED && (!(o.inner_tol > 0.0) || !(o.inner_tol < 1.0)))
    return fail_msg(SYLV_E_INVALID, "opts.inner_tol must be in (0,1)");
  if (o.precond != SYLV_PRECOND_NONE && o.precond != SYLV_PRECOND_BLOCK_JACOBI)
    return fail_msg(SYLV_E_INVALID, "opts.precond");
  if (o.maxit < 1 || o.max_outer < 1) return fail_msg(SYLV_E_INVALID, "opts.maxit/max_outer");
  if (o.check_every < 0 || o.check_every > 4096)
    return fail_msg(SYLV_E_INVALID, "opts.check_every");
  OpData op;
  int device = 0;
  if (handle_view(h, &op, &device) != SYLV_OK) return fail_msg(SYLV_E_INVALID, "bad handle");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  const cudaStream_t s = (cudaStream_t)stream;
  const int rc = o.precision == SYLV_PREC_F64
                     ? solve_in_scratch<double>(op, device, B, X, nrhs, o, info, s)
                     : solve_in_scratch<float>(op, device, B, X, nrhs, o, info, s);
  if (prev != device) cudaSetDevice(prev);
  return rc;
}
