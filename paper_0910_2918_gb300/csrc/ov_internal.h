// Internal declarations shared by the libov translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <complex>
#include <vector>

#include "../../include/ov.h"

namespace ov {

constexpr int kBlockDefault = 128;  // threads per block of the site kernels unless tuned (64 / 128 / 256)
constexpr int kMaxL = 120;        // largest inner dimension (Roberts-Higham fits one CTA's shared memory)
constexpr int kMaxInnerK = 1024;  // largest outer dimension the inner level accepts (H_k factors in shared memory)

// status codes kept on the device per right-hand side
constexpr int kStOK = 0;
constexpr int kStLucky = 1;      // Lanczos found an invariant subspace at step kbreak
constexpr int kStBreakdown = 2;  // serious two-sided breakdown at step kbreak
constexpr int kStZero = 3;       // the source is zero: y = 0

// Device coefficient arrays, each [nrhs][ld] (index j = 1..k is the step).
struct Coefs {
  double2* alp;  // alpha_j (complex; imaginary part 0 for Lanczos)
  double2* bet;  // beta_j  (recurrence coefficient of the w_{j-1} / v_{j-1} terms)
  double2* gam;  // gamma_j
  double* nv;    // v_j = tv_j / nv_j
  double2* nw;   // w_j = tw_j / conj(nw_j)
  int* status;   // [nrhs]
  int* kbreak;   // [nrhs]
  int ld;
};

// Modes of the stencil step kernel.
enum StepMode { kModeLanczos = 0, kModeTwoSided = 1, kModeRegen = 2, kModeApply = 3 };
// step precision of the relaxed double-float steps (float hopping, double-float vectors);
// launch_step accepts it besides OV_PREC_*, every other launcher treats it as OV_PREC_DF64
constexpr int kPrecDF64Relaxed = 3;

struct Geometry {
  int V, Lx, Ly, Lz, Lt;
};

// One lattice problem of a launch: its geometry, links and operator constants, the
// offset of its vectors in every vector pool (and of its x / y in the canonical
// buffers; both hold 12 V complex entries per problem), and its range of site blocks
// in the one-dimensional grid. A handle with n right-hand sides on one gauge field is n
// problems sharing geometry and links; a batch of lattices is one problem per lattice.
struct ProbDesc {
  Geometry g;
  const void* links;
  double mass;       // m_w + 4
  double emu, emui;  // e^{mu}, e^{-mu}
  float mass_hl[2], emu_hl[2], emui_hl[2];  // the same constants as float pairs (hi + lo)
  size_t voff;
  int block0, nblk;
};
struct Batch {
  const ProbDesc* desc;  // device [nprob]
  const int2* blk_map;   // device [nblocks]: (problem, site block within the problem) of each block
  int nblocks, nprob;
  int block;             // threads per site block (64, 128 or 256)
};

// Arguments of one outer step (vector pointers are pools; problem r's vectors start at
// desc[r].voff and are laid out [12][V] of the precision's storage type).
//
// The Krylov vectors are kept unnormalised: t_j = nv_j v_j on the v side and
// tw_j = conj(nw_j) w_j on the w side, where nv_j, nw_j are the normalisations of the
// recurrence (Sec. 2). The stored basis holds t_1 .. t_k, and 1/nv_j is folded into the
// recurrence scalars and into the recombination coefficients, so no kernel writes the
// normalised vectors.
struct StepArgs {
  Batch b;
  // per-problem step scalars in the arithmetic type of the precision (vec_t slots, [nprob][8]),
  // written once per step by the block that finalises the coefficient (the site kernels do
  // no double-precision work):
  //   0: 1/nv_j                      1: c_v = gamma_j / nv_{j-1} (Lanczos: beta_j / nv_{j-1})
  //   2: 1/conj(nw_j)                3: c_w = beta_j / conj(nw_{j-1})
  //   4: alpha_j / nv_j              5: conj(alpha_j) / conj(nw_j)
  void* scal;
  const void* tv;  // apply mode: the source
  void* p;         // A v_j - ..., and the apply mode's output
  void* r;         // A^dag w_j - ...
  // vectors of step j when jdev is NULL (the regeneration pass): t_j, t_{j-1} and the
  // destination of t_{j+1} (which may alias t_{j-1})
  const void* tc;
  const void* tp;
  void* tn;
  void* yacc;        // regeneration pass: y accumulator (accumulator type)
  const void* cacc;  // regeneration pass: c_j / nv_j in accumulator type, [nprob][ld]
  Coefs c;
  int j;
  // Device-side step state, so that a run of steps can be captured once in a CUDA graph
  // and replayed: when jdev is set the kernels take j from *jdev (the update kernel's last
  // block advances it) and their vectors from the basis slot table (slot i holds t_{i+1};
  // t_0 is the zeroed ring slot 0) or, without a table, from the two-slot ring vring
  // (t_j in slot j & 1; t_{j+1} overwrites t_{j-1}); the w side always uses the ring wring.
  int* jdev;
  unsigned* gticket;       // finished blocks of an update launch (global ticket)
  void* const* slot_tab;   // device [k + 1]: address of basis slot i (t_{i+1} of every problem)
  void* vring;
  void* wring;
  size_t pool_bytes;       // bytes of one vector of every problem (a slot)
  int dagger;  // apply mode: 1 = A^dag
  double breakdown_tol;
  double* partials;     // [nblocks][4]
  unsigned* counters;   // [nprob]
};

void fill_consts(ProbDesc& d, double m_w, double mu);

// outer-level launchers (ov_outer.cu); prec = OV_PREC_*. Canonical buffers hold, per
// problem r, 12 V complex doubles at offset desc[r].voff (layout [V][12]).
// x -> xint (and a copy to xint2 if not NULL); with want_norm the norms set nv_1 = nw_1 and
// the step-1 scalars
cudaError_t launch_pack(int prec, const Batch& b, const double2* xcanon, void* xint, void* xint2, Coefs c,
                        double* partials, unsigned* counters, int want_norm, void* scal, cudaStream_t st);
cudaError_t launch_unpack(int prec, const Batch& b, const void* xint, double2* ycanon, cudaStream_t st);
cudaError_t launch_step(int prec, int mode, const StepArgs& a, cudaStream_t st);
cudaError_t launch_update(int prec, int mode, const StepArgs& a, cudaStream_t st);
// y_r = scale_r * sum_{j<k_r} c[r][j+1] v_{r,j+1} (+ x_r and gamma5 if add_x); slots[j] is
// the device address of basis slot j (a vector pool)
cudaError_t launch_recombine(int prec, const Batch& b, const void* const* slots, const void* cacc, int ldc,
                             const int* k_dev, const double* scale, const double2* xcanon, int add_x,
                             double2* ycanon, cudaStream_t st);
// y_r = scale_r * yacc_r (+ x_r, gamma5)
cudaError_t launch_finish_acc(int prec, const Batch& b, const void* yacc, const double* scale,
                              const double2* xcanon, int add_x, double2* ycanon, cudaStream_t st);
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);
void split_const(double d, float hl[2]);
size_t vec_elem_bytes(int prec);  // bytes per complex vector element
size_t acc_elem_bytes(int prec);  // bytes per complex accumulator element
int num_site_blocks(const Geometry& g, int bs);

// inner level (ov_inner.cu)
struct InnerWork {
  // per problem i (batch of count problems):
  double2* Q;       // [count][ld][kMaxL]  (row-major k x l_eff, leading dim kMaxL)
  double2* T;       // [count][kMaxL][3]  inner alpha, beta, gamma
  int* leff;        // [count]
  double2* S;       // [2*count][kMaxL*kMaxL] Roberts-Higham scratch (global copy of S_n)
  double2* s;       // [2*count][kMaxL]  first column of sgn(T)
  int* rh_its;      // [2*count]
  int* rh_ok;       // [2*count]
  int* perm;        // [2*count][kMaxL]
  int* fail;        // [count] singular H_k
  int ld;
  int arith;        // OV_INNER_DF64 / OV_INNER_FP64: arithmetic of the serial solves and inversions
  int rh_scale;     // 1: determinant-scaled Roberts-Higham steps in the inner level (DF64 arithmetic)
};
// Inner level for `count` problems whose tridiagonal coefficients live in device
// arrays alp/bet/gam with leading dimension ldc (index j = 1..k as in Coefs, so the
// diagonal is alp[j], the subdiagonal H_{j,j-1} = bet[j] and the superdiagonal
// H_{j-1,j} = gam[j] for j >= 2). Results, index 1..k: c (double2 [count][ldo]) and, if
// cacc is not NULL, c_j / nv[j] (nv: the normalisations of the unnormalised basis vectors,
// leading dimension ldc; NULL: 1) in the accumulator type of `prec`; est_inner[i]; est_outer[i]
// against cprev (rows of length kprev[i], NULL: infinite); rh_status[i] (0 ok, 1 RH not
// converged, 2 singular H); rh_iters[i]. phase 0: everything; phase 1: no inner estimate
// (est_inner = NaN); phase 2: the inner estimate for the problems of a preceding phase-1
// call (re-runs only the smaller Roberts-Higham set and the combination).
cudaError_t run_inner(int count, const int* k_dev, const int* l_dev, int hermitian, const double2* alp,
                      const double2* bet, const double2* gam, const double* nv, int ldc, InnerWork& w,
                      double rh_tol, int rh_maxit, int inner_dl, double2* c, int ldo, void* cacc, int prec,
                      double* est_inner, const double2* cprev, int ldp, const int* kprev_dev,
                      double* est_outer, int* rh_status, int* rh_iters, int phase, cudaStream_t st);
cudaError_t run_rh_dense(int count, int m, const double2* T, double2* S, int* iters, int* ok,
                         double rh_tol, int rh_maxit, InnerWork& w, cudaStream_t st);

// Roberts-Higham on large dense matrices and the non-nested stopping check (ov_rhbig.cu)
size_t rh_big_scratch_bytes(int count, int k);
// sgn of `count` dense k x k matrices T (device) into S (device); iters / ok: host arrays
cudaError_t run_rh_big(int count, int k, const double2* T, double2* S, int* iters, int* ok, double rh_tol,
                       int rh_maxit, void* scratch, cudaStream_t st);
size_t nonnested_scratch_bytes(int count, int kmax);
// the stopping check of the non-nested method: c = sgn(H_k) e_1 by Roberts-Higham on the
// full H_k of each problem (k_host: host array of the problems' k); outputs as run_inner's
// phase 0 (est_inner = 0: nothing is nested)
cudaError_t run_nonnested(int count, const int* k_host, const double2* alp, const double2* bet, const double2* gam,
                          const double* nv, int ldc, double rh_tol, int rh_maxit, double2* c, int ldo, void* cacc,
                          int prec, double* est_inner, const double2* cprev, int ldp, const int* kprev_dev,
                          double* est_outer, int* rh_status, int* rh_iters, void* scratch, cudaStream_t st);

// host orchestration used by the solver (defined in ov_api.cu)
int sign_apply_device(ov_handle* h, int nrhs, const double2* x, double2* y, double tol, int k_max, int l,
                      ov_info* info, int neg_mu);
cudaStream_t handle_stream(const ov_handle* h);
int handle_device(const ov_handle* h);
size_t handle_pool(const ov_handle* h, int nrhs);  // complex entries of nrhs vectors (0: not allowed)

// block operations of the eigensolver and the deflated apply (ov_eig.cu); blocks are
// bx (or by) canonical complex-double n-vectors with strides ldx (ldy)
size_t lattice_size(const ov_handle* h, int q);  // 12 V of lattice q
double lattice_mu(const ov_handle* h, int q);
double lattice_mass(const ov_handle* h, int q);  // m_w + 4
// Fixed sets of matvecs in the handle's arithmetic: item r computes Y[voff..] = A X[voff..]
// for 12 V entries of lattice q at mu (neg = 0) or at -mu (neg = 1: A(-mu) = A^dag); X and Y
// are canonical complex-double buffers of `pool` entries. One run = three launches.
struct ApplyItem {
  int q, neg;
  size_t voff;
};
struct ApplySet;
int apply_set_create(ov_handle* h, const std::vector<ApplyItem>& items, size_t pool, ApplySet** out);
int apply_set_run(ov_handle* h, const ApplySet* s, const double2* X, double2* Y);
void apply_set_destroy(ApplySet* s);
size_t block_gram_part_bytes(int bx, int by);
cudaError_t block_gram(size_t n, const double2* X, size_t ldx, int bx, const double2* Y, size_t ldy, int by,
                       double2* part, double2* G, cudaStream_t st);  // G = X^dag Y (bx x by, row-major)
cudaError_t block_mul(size_t n, const double2* X, size_t ldx, int bx, const double2* C, double2* Y, size_t ldy, int by,
                      double alpha, double beta, cudaStream_t st);  // Y = beta Y + alpha X C
cudaError_t add_x_gamma5(size_t n, const double2* x, double2* y, cudaStream_t st);  // y = x + gamma5 y
// the m eigenpairs of smallest |lambda| of A(+-mu) on each job's lattice, all jobs in the
// same launches (ov_eig.cu)
struct EigJob {
  int q = 0, neg = 0;  // lattice; 1: eigenvectors of A(-mu) = A^dag
  double2* Rout = nullptr;  // [m][n] device: right eigenvectors (unit norm)
  std::vector<std::complex<double>> lam;  // eigenvalues, by increasing magnitude
  std::vector<double> res;                // ||A x - lambda x|| / ||A|| per pair
  int its = 0;
  int status = 0;  // OV_OK, OV_NOT_CONVERGED (best vectors returned) or OV_ERR_BREAKDOWN
};
int eig_smallest(ov_handle* h, std::vector<EigJob>& jobs, int m, int b, int deg, double tol, int maxit, int verbose);
// small dense complex matrices, row-major, on the host (ov_small.cpp)
bool small_eig(int n, const double2* A, double2* w, double2* V);
bool small_eigh(int n, const double2* A, double* w, double2* V);
bool small_chol_inv(int n, const double2* A, double2* Rinv);
bool small_inv(int n, const double2* A, double2* X);
bool small_qr_q(int n, const double2* A, double2* Q);  // unitary Q of A = Q R

// learned sizing (ov_mlp.cu)
cudaError_t mlp_predict_device(const float* theta_dev, int n, const float* X_dev, float* Y_dev, cudaStream_t st);
int mlp_num_params();

}  // namespace ov
