// The overlap operator inside an iterative solver (Sec. 1: D_ov is what iterative solvers
// for the overlap Dirac operator need; each solver iteration applies it).
//
//   D(m) = (1 - m/2) D_ov(mu) + m,   D_ov(mu) = 1 + gamma5 sgn(A),   A = gamma5 D_w(mu)
//   D(m) v   = (1 - m/2) (v + gamma5 sgn(A) v) + m v
//   D(m)^dag v = (1 - m/2) (v + sgn(A^dag) gamma5 v) + m v,   A^dag = gamma5 D_w(-mu)
//
// x = D(m)^{-1} b by conjugate gradients on the normal equations D^dag D x = D^dag b
// (CGNR; Hestenes and Stiefel 1952): every iteration applies D once and D^dag once, each a
// nested sign apply of the handle. The vector algebra (canonical layout, double) runs in
// the kernels below, with per-right-hand-side reductions summed in a fixed order.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "ov_internal.h"

namespace ov {
namespace {

constexpr int kSolveThreads = 256;
constexpr int kSolveBlocksPerRhs = 152;  // one wave of the SMs per right-hand side

__device__ __forceinline__ bool lower_spin(size_t e) { return (e % 12) >= 6; }  // gamma5 = diag(1, 1, -1, -1)

// out = c (v + gamma5 s) + m v   (D applied: s = sgn(A) v)
// out = c (v + s) + m v          (D^dag applied: s = sgn(A^dag) gamma5 v), g5 = 0
__global__ void k_combine_d(size_t n, const double2* __restrict__ v, const double2* __restrict__ sg, double c,
                            double m, int g5, double2* out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double2 a = v[e];
    double2 b = sg[e];
    if (g5 && lower_spin(e)) b = make_double2(-b.x, -b.y);
    out[e] = make_double2(c * (a.x + b.x) + m * a.x, c * (a.y + b.y) + m * a.y);
  }
}

__global__ void k_gamma5(size_t n, const double2* __restrict__ v, double2* out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double2 a = v[e];
    out[e] = lower_spin(e) ? make_double2(-a.x, -a.y) : a;
  }
}

// y_r += a_r x_r (a: real, one per right-hand side of length nr)
__global__ void k_axpy(size_t nr, int nrhs, const double* __restrict__ a, const double2* __restrict__ x, double2* y) {
  const size_t n = nr * nrhs;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double s = a[e / nr];
    const double2 xv = x[e];
    double2 yv = y[e];
    yv.x = fma(s, xv.x, yv.x);
    yv.y = fma(s, xv.y, yv.y);
    y[e] = yv;
  }
}

// p_r = z_r + b_r p_r
__global__ void k_xpby(size_t nr, int nrhs, const double* __restrict__ b, const double2* __restrict__ z, double2* p) {
  const size_t n = nr * nrhs;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double s = b[e / nr];
    const double2 zv = z[e];
    double2 pv = p[e];
    p[e] = make_double2(fma(s, pv.x, zv.x), fma(s, pv.y, zv.y));
  }
}

// partial sums of ||x_r||^2: block (q, r) sums its grid-stride share of right-hand side r
__global__ void k_norm2_part(size_t nr, const double2* __restrict__ x, double* part) {
  __shared__ double red[kSolveThreads / 32];
  const int r = blockIdx.y, q = blockIdx.x;
  const double2* xr = x + (size_t)r * nr;
  double acc = 0.0;
  for (size_t e = (size_t)q * blockDim.x + threadIdx.x; e < nr; e += (size_t)gridDim.x * blockDim.x) {
    const double2 a = xr[e];
    acc = fma(a.x, a.x, fma(a.y, a.y, acc));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kSolveThreads / 32; ++w) s += red[w];
    part[(size_t)r * gridDim.x + q] = s;
  }
}

// fixed-order total of each right-hand side's partial sums (one thread per right-hand side)
__global__ void k_norm2_fin(int nrhs, int nparts, const double* __restrict__ part, double* out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += part[(size_t)r * nparts + q];
  out[r] = s;
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + kSolveThreads - 1) / kSolveThreads, 152 * 16); }

struct SolveBufs {
  void* p[8] = {};
  bool alloc(size_t vec_bytes, size_t small_bytes) {
    for (int i = 0; i < 7; ++i)
      if (cudaMalloc(&p[i], vec_bytes) != cudaSuccess) return false;
    return cudaMalloc(&p[7], small_bytes) == cudaSuccess;
  }
  ~SolveBufs() {
    for (void* q : p)
      if (q) cudaFree(q);
  }
};

}  // namespace
}  // namespace ov

using namespace ov;

extern "C" int ov_solve(ov_handle* h, int nrhs, const void* b, void* x, int mem, double mass, double tol, int maxit,
                        double sign_tol, int k_max, int l, int* iters, double* resid) {
  if (!h || !b || !x || nrhs < 1 || maxit < 1 || !(tol > 0.0) || !(sign_tol >= 0.0) || !(mass >= 0.0) ||
      !(mass < 2.0))
    return OV_ERR_ARG;
  if (mem != OV_MEM_HOST && mem != OV_MEM_DEVICE) return OV_ERR_ARG;
  const size_t nall = handle_pool(h, nrhs);
  if (nall == 0) return OV_ERR_ARG;
  if (cudaSetDevice(handle_device(h)) != cudaSuccess) return OV_ERR_CUDA;
  cudaStream_t st = handle_stream(h);
  const size_t nr = nall / nrhs;
  const size_t vb = sizeof(double2) * nall;
  SolveBufs B;
  const size_t small = sizeof(double) * ((size_t)nrhs * (kSolveBlocksPerRhs + 8));
  if (!B.alloc(vb, small)) return OV_ERR_NOMEM;
  double2 *bd = (double2*)B.p[0], *xd = (double2*)B.p[1], *r = (double2*)B.p[2], *z = (double2*)B.p[3],
          *p = (double2*)B.p[4], *q = (double2*)B.p[5], *t = (double2*)B.p[6];
  double* part = (double*)B.p[7];
  double* nrm = part + (size_t)nrhs * kSolveBlocksPerRhs;  // [nrhs]
  double* sc = nrm + nrhs;                                  // [nrhs] step scalars
  const int gr = grid_for(nall);
  const double c1 = 1.0 - 0.5 * mass;
  std::vector<ov_info> info(nrhs);
  int worst = OV_OK;
  auto note = [&](int rc) {
    if (rc < 0) return rc;
    if (rc > 0 && worst == OV_OK) worst = rc;
    return OV_OK;
  };
#define SCK(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      fprintf(stderr, "libov: ov_solve: %s\n", cudaGetErrorString(e_)); \
      return OV_ERR_CUDA;                           \
    }                                               \
  } while (0)
  auto norms = [&](const double2* v, std::vector<double>& out) -> int {
    k_norm2_part<<<dim3(kSolveBlocksPerRhs, nrhs), kSolveThreads, 0, st>>>(nr, v, part);
    k_norm2_fin<<<(nrhs + 127) / 128, 128, 0, st>>>(nrhs, kSolveBlocksPerRhs, part, nrm);
    SCK(cudaGetLastError());
    SCK(cudaMemcpyAsync(out.data(), nrm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    return OV_OK;
  };
  // out = D v
  auto applyD = [&](const double2* v, double2* out) -> int {
    int rc = note(sign_apply_device(h, nrhs, v, t, sign_tol, k_max, l, info.data(), 0));
    if (rc != OV_OK) return rc;
    k_combine_d<<<gr, kSolveThreads, 0, st>>>(nall, v, t, c1, mass, 1, out);
    SCK(cudaGetLastError());
    return OV_OK;
  };
  // out = D^dag v (q serves as the gamma5 v scratch: it is free whenever D^dag is applied)
  auto applyDH = [&](const double2* v, double2* out) -> int {
    k_gamma5<<<gr, kSolveThreads, 0, st>>>(nall, v, q);
    SCK(cudaGetLastError());
    int rc = note(sign_apply_device(h, nrhs, q, t, sign_tol, k_max, l, info.data(), 1));
    if (rc != OV_OK) return rc;
    k_combine_d<<<gr, kSolveThreads, 0, st>>>(nall, v, t, c1, mass, 0, out);
    SCK(cudaGetLastError());
    return OV_OK;
  };
  const cudaMemcpyKind kin = mem == OV_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  SCK(cudaMemcpyAsync(bd, b, vb, kin, st));
  SCK(cudaMemsetAsync(xd, 0, vb, st));
  SCK(cudaMemcpyAsync(r, bd, vb, cudaMemcpyDeviceToDevice, st));  // r = b - D 0
  std::vector<double> bn(nrhs), gam(nrhs), gnew(nrhs), qq(nrhs), rr(nrhs), a(nrhs), bb(nrhs);
  int rc = norms(bd, bn);
  if (rc != OV_OK) return rc;
  std::vector<int> it_done(nrhs, -1);
  std::vector<double> res(nrhs, 1.0);
  for (int i = 0; i < nrhs; ++i)
    if (bn[i] == 0.0) {
      it_done[i] = 0;  // b = 0: x = 0
      res[i] = 0.0;
    }
  if ((rc = applyDH(r, z)) != OV_OK) return rc;
  SCK(cudaMemcpyAsync(p, z, vb, cudaMemcpyDeviceToDevice, st));
  if ((rc = norms(z, gam)) != OV_OK) return rc;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    if (std::all_of(it_done.begin(), it_done.end(), [](int v) { return v >= 0; })) break;
    if ((rc = applyD(p, q)) != OV_OK) return rc;
    if ((rc = norms(q, qq)) != OV_OK) return rc;
    for (int i = 0; i < nrhs; ++i) a[i] = (it_done[i] < 0 && qq[i] > 0.0) ? gam[i] / qq[i] : 0.0;
    SCK(cudaMemcpyAsync(sc, a.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    k_axpy<<<gr, kSolveThreads, 0, st>>>(nr, nrhs, sc, p, xd);  // x += a p
    for (int i = 0; i < nrhs; ++i) a[i] = -a[i];
    SCK(cudaMemcpyAsync(sc, a.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    k_axpy<<<gr, kSolveThreads, 0, st>>>(nr, nrhs, sc, q, r);  // r -= a q
    SCK(cudaGetLastError());
    if ((rc = norms(r, rr)) != OV_OK) return rc;
    for (int i = 0; i < nrhs; ++i) {
      if (it_done[i] >= 0) continue;
      res[i] = sqrt(rr[i]) / bn[i];
      if (res[i] <= tol) it_done[i] = it;
    }
    if (std::all_of(it_done.begin(), it_done.end(), [](int v) { return v >= 0; })) break;
    if ((rc = applyDH(r, z)) != OV_OK) return rc;
    if ((rc = norms(z, gnew)) != OV_OK) return rc;
    for (int i = 0; i < nrhs; ++i) {
      bb[i] = gam[i] > 0.0 ? gnew[i] / gam[i] : 0.0;
      gam[i] = gnew[i];
    }
    SCK(cudaMemcpyAsync(sc, bb.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    k_xpby<<<gr, kSolveThreads, 0, st>>>(nr, nrhs, sc, z, p);  // p = z + b p
    SCK(cudaGetLastError());
  }
  const cudaMemcpyKind kout = mem == OV_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  SCK(cudaMemcpyAsync(x, xd, vb, kout, st));
  SCK(cudaStreamSynchronize(st));
  bool all = true;
  for (int i = 0; i < nrhs; ++i) {
    if (iters) iters[i] = it_done[i] >= 0 ? it_done[i] : std::min(it, maxit);
    if (resid) resid[i] = res[i];
    all = all && it_done[i] >= 0;
  }
#undef SCK
  return all ? worst : OV_NOT_CONVERGED;
}
