// Internal device/host data structures of the solver library.
//
// One "system" is one handle (operator) together with nrhs right-hand sides.  A solve runs a
// list of systems at once (sylv_solve is the one-system case).  Systems are cut into tiles of
// blockDim.x consecutive pixels.  Every kernel of the iteration is one launch over all systems
// that share a number of sources k: each system owns `nslots` CTAs (the launch is sized to be
// resident at once) and CTA `slot` walks the system's tiles slot, slot + nslots, ...  Each
// right-hand side of each system ("column") carries its own CG scalars and state (ColState).
//
// Scalar reductions (dot products) are deterministic: each CTA writes one partial sum per
// column, and the last CTA of a system to finish (detected with an atomic counter, no
// waiting) adds the partials in a fixed order and updates the system's scalars.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "sylv.h"

namespace sylv {

constexpr int KMAX = SYLV_MAX_K;
constexpr int MMAX = SYLV_MAX_M;
constexpr int EMAX = SYLV_MAX_DEGREE;
constexpr int RMAX = SYLV_MAX_RHS;
constexpr int NPART = 4;          // partial sums per (tile, column)
constexpr int MAX_BLOCK = 256;
constexpr int MAX_WARPS = 9;      // warps per CTA, producer warp included
constexpr int TILE_PX = 256;      // pixels per tile = threads per CTA of the iteration kernels

enum Phase : int {
  PH_START = 0,       // before the first FP64 residual
  PH_INNER = 1,       // inner CG running
  PH_INNER_DONE = 2,  // inner CG finished: X += d and a new FP64 residual are due
  PH_CONVERGED = 3,   // final: tolerance reached
  PH_FAILED = 4       // final: see status
};

struct ColState {
  double bnorm2;   // ||b||^2
  double rr64;     // ||b - G X||^2 at the last FP64 residual
  double gamma;    // r . z of the inner iteration
  double alpha;
  double beta;
  double rr_in0;   // ||r||^2 at the start of the inner solve
  double rr_in;    // current inner ||r||^2 (recursive)
  double thr_in;   // inner stop threshold on ||r||^2
  double relres;   // last true relative residual
  int phase;
  int it;          // inner iterations so far
  int outer;       // FP64 residual evaluations so far
  int status;      // SYLV_* status once final
  int first;       // next inner apply is the first of this inner solve
  int stop_after;  // inner solve stopped on the iteration cap
  int dpend;       // d still lacks alpha p of the last iteration (the operator kernel of the
                   // next iteration adds it; k_update_x when the inner solve ended there)
  int pad1;
};

// Operator data of one handle, in the device layouts the kernels read.
struct OpData {
  int64_t n;
  int64_t ld;                // leading dimension of every library-owned buffer: n rounded up
                             // to whole tiles (TILE_PX), so tile rows are 16-byte aligned
  int64_t ldu;               // leading dimension of the caller's vectors (X, B, Y, Yobs)
  int k, m, E, has_w;
  const int32_t* ell_col;    // E x ld: off-diagonal columns of L (padding: own row, value 0)
  const float* ell_val32;    // E x ld
  const double* ell_val64;   // E x ld
  const float* diag32;       // ld: diagonal of L
  const double* diag64;
  const float* D32;          // m x ld
  const double* D64;
  const float* w32;          // ld or null
  const double* w64;
  const double* blk64;       // K(K+1)/2 x ld: packed lower triangle of the pixel block
                             // P_i = diag_j(tau_j (kappa_j^2 w_i + L_ii)) + sum_c d_ci a_c a_c^T
  const double* fac64;       // (K + K(K+1)/2) x ld: scaling and factor of P_i (block_chol)
  const float* fs32;         // K x ld: the scaling of that factor in FP32
  const __half2* fl16;       // ceil(K(K+1)/2 / 2) x ld: its triangular factor in FP16, two
                             // entries per pixel and row (entry a in row a/2, lane a%2); the
                             // FP32 inner preconditioner; entries lie in [-1, 1e3]
  const float* blk_hl;       // 2 K(K+1)/2 x ld: blk64 as FP32 pairs, hi rows then lo rows
                             // (blk64 = hi + lo to 2^-48), for the double-float residual
  const float* val_hl;       // 2 E x ld: ell_val64 the same way
  int df_ok;                 // every nonzero entry of blk64, ell_val64 and tau lies in
                             // [2^-40, 2^40]: the double-float residual applies
  int pad_df;
  float tau_hl[2][KMAX];     // tau as an FP32 pair
  float A32[MMAX * KMAX];    // A[c * k + j]
  double A64[MMAX * KMAX];
  float tau32[KMAX];
  float tk2_32[KMAX];        // tau_j kappa_j^2
  double tau64[KMAX];
  double tk2_64[KMAX];
  double kappa64[KMAX];
  double logf64[MMAX];       // ln(nu_c / nu0), power-law mixing only
};

struct SysDesc {
  OpData op;
  int R;                 // right-hand sides
  int ntiles;            // tiles of blockDim.x pixels
  int nslots[4];         // CTAs working on this system: [0] in operator (inner_apply) launches,
                         // [1] in update launches, [2] in residual and update_x launches,
                         // [3] in staged residual launches
  const double* B;       // R x k x ld
  double* X;             // R x k x ld
  void* vd;              // inner vectors, R x k x ld of the inner type
  void* vr;
  void* vz;
  void* vp;
  void* vq;
  ColState* st;          // R
  ColState* st2;         // R: the staged pair's second copy (written by its operator kernel)
  double* partial;       // nslots x R x NPART
  double* partial2;      // nslots x R x NPART: the staged update kernel's partials
  unsigned int* counter; // one per system, zero between kernels
};

struct Control {
  unsigned int n_active;      // columns in PH_INNER
  unsigned int n_unfinished;  // columns not final
  unsigned int error;         // nonzero: a bounded device wait expired (SYLV_E_TIMEOUT)
  unsigned int pad0;
  double tol2;                // tol^2
  double tol_in2;             // inner_tol^2 (0 in FP64 mode)
  double safety2;             // squared safety factor on the inner target
  int maxit;
  int max_outer;
  int precond;
  int x0_zero;                // X starts at zero: the first residual is B itself
  long long wait_budget;      // SM clock cycles a staged kernel's pipeline wait may take before
                              // it records SYLV_E_TIMEOUT; 0: the default (about a second)
  int inject_stall;           // tests of the timeout path: the producer warps of the staged
                              // kernels named by the bits (1 residual, 2 operator, 4 update)
                              // issue no copies, so their consumers' first wait runs out
  int pad_ctl;
};
enum : int { STALL_RESIDUAL = 1, STALL_APPLY = 2, STALL_UPDATE = 4 };

struct CtaRef {
  int sys;   // system of this CTA (-1: idle, the CTA returns at once)
  int slot;  // 0..nslots-1 within the system
};

// ------------------------------------------------------------------------------------------
// launchers (defined in the kernel translation units)
// ------------------------------------------------------------------------------------------
// Iteration kernels for a group of systems of one shape (k sources, m channels, ELL width e).
// variant 0: the direct kernels; 1-3: the bulk-copy staged FP32 kernels (shapes with
// compile-time instances, no mass diagonal; tma_available() says whether a shape has them)
// with 1 the last-CTA protocol, 2 and 3 the consumer-side protocol (3: the kernel first sums
// the previous kernel's partials; a chunk of such iterations ends with launch_inner_close).
template <typename T>
cudaError_t launch_inner_apply(int k, int m, int e, int variant, int ncta, int block,
                               const SysDesc* d, const CtaRef* c, Control* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_inner_update(int k, int m, int e, int variant, int ncta, int block,
                                const SysDesc* d, const CtaRef* c, Control* ctl,
                                cudaStream_t s);
bool tma_available(int k, int m, int e);
cudaError_t launch_inner_close(int ncta, const SysDesc* d, const CtaRef* c, Control* ctl,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_residual(int k, int m, int e, int ncta, int block, const SysDesc* d,
                            const CtaRef* c, Control* ctl, cudaStream_t s);
// Staged FP64 residual of the mixed solve (FP32 inner vectors, shapes with staged instances,
// no mass diagonal, TILE_PX tiles, caller rows copied whole); cudaErrorNotSupported otherwise.
cudaError_t launch_residual_staged(int k, int m, int e, int ncta, const SysDesc* d,
                                   const CtaRef* c, Control* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_update_x(int k, int ncta, int block, const SysDesc* d, const CtaRef* c,
                            cudaStream_t s);
// Resident CTAs per SM of one kernel (kind 0: inner apply, 1: inner update, 2: residual,
// 3: staged residual) for a shape.
template <typename T>
int occupancy(int kind, int k, int m, int e, int variant, int block);
cudaError_t launch_init_states(int ncols, const int* col_sys, const int* col_rhs,
                               const SysDesc* d, Control* c, cudaStream_t s);

cudaError_t launch_csr_check(const OpData& op, const int32_t* rowptr, const int32_t* col,
                             int64_t nnz, unsigned int* flags, unsigned int* maxdeg,
                             cudaStream_t s);
cudaError_t launch_ell_build(const OpData& op, const int32_t* rowptr, const int32_t* col,
                             const double* val, int32_t* ell_col, float* ell_val32,
                             double* ell_val64, float* diag32, double* diag64, int E,
                             cudaStream_t s);
// Probe estimator of the posterior variances (sylv_variance).
cudaError_t launch_var_accum(const OpData& op, const double* Z, const double* X, int R,
                             double* num, double* den, cudaStream_t s);
cudaError_t launch_var_finish(const OpData& op, const double* num, const double* den,
                              double* var, cudaStream_t s);
// R probing vectors of a colouring (probes p0 .. p0 + R - 1; probe t is colour t / k in
// source t % k) into Z (R x k x ldu); *flag set if a colour lies outside [0, ncol).
cudaError_t launch_probe_fill(const OpData& op, const int32_t* colour, int ncol, int p0, int R,
                              double* Z, unsigned int* flag, cudaStream_t s);
// Intrinsic GMRF prior shape: the ELL width of L^2 (atomic max into *width), then L^2 itself
// into new ELL arrays of that width and a new diagonal.
cudaError_t launch_square_count(const OpData& op, unsigned int* width, cudaStream_t s);
cudaError_t launch_square_fill(const OpData& op, int E2, int32_t* sq_col, float* sq_val32,
                               double* sq_val64, float* sq_diag32, double* sq_diag64,
                               cudaStream_t s);
cudaError_t launch_convert_check(const double* src, int64_t rows, int64_t n, int64_t ld_src,
                                 int64_t ld_dst, float* dst32, double* dst64, int positive,
                                 unsigned int* flags, cudaStream_t s);
cudaError_t launch_rhs(const OpData& op, const double* Y, double* B, int R, cudaStream_t s);
// The same for pixels i0 .. i1 - 1 only.
cudaError_t launch_rhs_range(const OpData& op, const double* Y, double* B, int R, int64_t i0,
                             int64_t i1, cudaStream_t s);
cudaError_t launch_block_setup(const OpData& op, double* blk64, double* fac64, float* fs32,
                               __half2* fl16, cudaStream_t s);
// dst[q][i] = hi, dst[rows + q][i] = lo of src[q][i] (q < rows, i < ld); sets *flag if a
// nonzero entry lies outside [2^-40, 2^40] or is not finite.
cudaError_t launch_split_hl(const double* src, int64_t rows, int64_t ld, float* dst,
                            unsigned int* flag, cudaStream_t s);
// Stand-alone residual Rout = B - G X (FP64 caller vectors, nrhs columns), double-float when
// use_df (else FP64).
cudaError_t launch_residual_out(const OpData& op, const double* B, const double* X, int R,
                                double* Rout, int use_df, cudaStream_t s);
// The same with bulk-copy staging (the conditions and CTA list of launch_residual_staged).
cudaError_t launch_residual_staged_df(int k, int m, int e, int ncta, const SysDesc* d,
                                      const CtaRef* c, Control* ctl, cudaStream_t s);
// Mixed-precision residual of the refinement loop in double-float (handles with df_ok), over
// the residual CTA list with tiles of `block` pixels.
cudaError_t launch_residual_df(int k, int m, int e, int ncta, int block, const SysDesc* d,
                               const CtaRef* c, Control* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_apply(const OpData& op, const T* X, T* Y, int R, cudaStream_t s);
cudaError_t launch_apply_staged(const OpData& op, const float* X, float* Y, int R,
                                unsigned int* err, cudaStream_t s);
cudaError_t launch_grad(const OpData& op, const double* X, const double* lam, const double* Y,
                        int R, int want_beta, double* partial, int ntiles, double* out,
                        cudaStream_t s);

// Handle internals for other translation units (runtime.cu).
int handle_view(sylv_handle h, OpData* op, int* device);
void set_last_error(const char* msg);
// Frees what the Sylvester solver cached for a handle (lanczos.cu).
void lanczos_release(sylv_handle h);

}  // namespace sylv
