// Roberts-Higham sign of large dense matrices (Sec. 2, Eq. (Roberts)): the non-nested
// method's sgn(H_k) for k up to 1024, batched over `count` matrices.
//
//   S_0 = H,  S_{n+1} = (S_n + S_n^{-1}) / 2,  stop when ||S_{n+1} - S_n||_F <= tol ||S_{n+1}||_F
//
// The inverse is taken by Gauss-Jordan elimination with partial pivoting over global memory
// (a 1024 x 1024 complex matrix is 16 MB, L2-resident for a few matrices at a time), one
// launch per pivot column for all matrices of the batch:
//   - the pivot of column j is the unused row of largest |W_ij|; every block of launch j-1
//     wrote the largest candidate among its rows, so each block of launch j reduces those
//     few partial maxima itself (no grid-wide synchronisation inside a launch);
//   - rows are not swapped: row p_j is marked used and the elimination reads from one
//     buffer and writes the other (ping-pong), so no block reads an element another block
//     of the same launch writes;
//   - at the end, with pivot rows p_0 .. p_{k-1}, (H^{-1})_{i, p_m} = W_{p_i, m}.
// FP64 arithmetic throughout (the oracle's LAPACK inversion is FP64 too).
#include <math.h>

#include <algorithm>
#include <vector>

#include "ov_internal.h"

namespace ov {
namespace {

constexpr int kRows = 8;        // rows of one block's tile (all columns)
constexpr int kThreads = 256;

__device__ __forceinline__ double2 bz_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double bz_abs2(double2 a) { return a.x * a.x + a.y * a.y; }
// 1/b with scaling against overflow
__device__ __forceinline__ double2 bz_inv(double2 b) {
  const double s = fmax(fabs(b.x), fabs(b.y));
  const double2 bs = make_double2(b.x / s, b.y / s);
  const double d = bs.x * bs.x + bs.y * bs.y;
  return make_double2(bs.x / (d * s), -bs.y / (d * s));
}

// the largest (value, row) of the block's candidates: value -1 means none
__device__ __forceinline__ void block_argmax(double v, int i, double* sv, int* si, double* out_v, int* out_i) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
  if (lane == 0) { sv[warp] = v; si[warp] = i; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
    *out_v = bv;
    *out_i = bi;
  }
  __syncthreads();
}

struct BigWork {
  double2* S;      // [count][k][k] the iterate
  double2* W0;     // [count][k][k] elimination buffers (ping-pong)
  double2* W1;
  // partial maxima of a pivot column and their rows, [2][count][nparts]: launch j reads
  // half j & 1 (written by launch j - 1, or the start for j = 0) and writes half
  // (j + 1) & 1, so no block reads a value another block of its own launch writes
  double* pv;
  int* pi;
  int* used;       // [count][k] row already a pivot
  int* piv;        // [count][k] pivot row of column j
  int* status;     // [count] 0 running, 1 converged, 2 singular or not finite
  double* norms;   // [count][nparts][2] partial sums of ||S_{n+1} - S_n||^2, ||S_{n+1}||^2
  int k, count, nparts;
};

// W = S (start of an inversion), clear the pivot marks, partial maxima of column 0
__global__ void __launch_bounds__(kThreads) k_big_start(BigWork w) {
  __shared__ double sv[kThreads / 32];
  __shared__ int si[kThreads / 32];
  const int mat = blockIdx.y, part = blockIdx.x, k = w.k;
  if (w.status[mat] != 0) return;
  const size_t base = (size_t)mat * k * k;
  const int r0 = part * kRows;
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int e = threadIdx.x; e < kRows * k; e += kThreads) {
    const int i = r0 + e / k, c = e % k;
    if (i >= k) break;
    const double2 v = w.S[base + (size_t)i * k + c];
    w.W0[base + (size_t)i * k + c] = v;
    if (c == 0) {
      w.used[(size_t)mat * k + i] = 0;
      const double a = bz_abs2(v);
      if (a > bv) { bv = a; bi = i; }
    }
  }
  block_argmax(bv, bi, sv, si, &w.pv[(size_t)mat * w.nparts + part], &w.pi[(size_t)mat * w.nparts + part]);
}

// elimination of column j: Win -> Wout; partial maxima of column j + 1 for the next launch
__global__ void __launch_bounds__(kThreads) k_big_col(BigWork w, int j, const double2* __restrict__ Win,
                                                      double2* __restrict__ Wout) {
  __shared__ double sv[kThreads / 32];
  __shared__ int si[kThreads / 32];
  __shared__ int s_p;
  __shared__ double2 s_inv;
  __shared__ double2 s_f[kRows];  // column j of the block's rows
  const int mat = blockIdx.y, part = blockIdx.x, k = w.k;
  if (w.status[mat] != 0) return;
  const size_t base = (size_t)mat * k * k;
  // the pivot: reduce the partial maxima of the previous launch (same order in every block)
  const size_t half_in = (size_t)(j & 1) * w.count * w.nparts;
  const size_t half_out = (size_t)((j + 1) & 1) * w.count * w.nparts;
  if (threadIdx.x < 32) {
    double v = -1.0;
    int i = 0x7fffffff;
    for (int q = threadIdx.x; q < w.nparts; q += 32) {
      const double qv = w.pv[half_in + (size_t)mat * w.nparts + q];
      const int qi = w.pi[half_in + (size_t)mat * w.nparts + q];
      if (qv > v || (qv == v && qi < i)) { v = qv; i = qi; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
    if (threadIdx.x == 0) {
      s_p = (v > 0.0 && i < k) ? i : -1;
      if (s_p >= 0) s_inv = bz_inv(Win[base + (size_t)s_p * k + j]);
    }
  }
  __syncthreads();
  const int p = s_p;
  if (p < 0) {
    // no nonzero candidate: singular to working precision
    if (part == 0 && threadIdx.x == 0) w.status[mat] = 2;
    return;
  }
  if (part == 0 && threadIdx.x == 0) {
    w.used[(size_t)mat * k + p] = 1;
    w.piv[(size_t)mat * k + j] = p;
  }
  const double2 inv = s_inv;
  const int r0 = part * kRows;
  if (threadIdx.x < kRows && r0 + threadIdx.x < k) s_f[threadIdx.x] = Win[base + (size_t)(r0 + threadIdx.x) * k + j];
  __syncthreads();
  const double2* prow = Win + base + (size_t)p * k;
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int e = threadIdx.x; e < kRows * k; e += kThreads) {
    const int li = e / k, c = e % k, i = r0 + li;
    if (i >= k) break;
    double2 out;
    if (i == p) {
      out = c == j ? inv : bz_mul(prow[c], inv);
    } else {
      const double2 fi = bz_mul(s_f[li], inv);  // W_ij / W_pj
      if (c == j) {
        out = make_double2(-fi.x, -fi.y);
      } else {
        const double2 t = bz_mul(fi, prow[c]);
        const double2 a = Win[base + (size_t)i * k + c];
        out = make_double2(a.x - t.x, a.y - t.y);
      }
    }
    Wout[base + (size_t)i * k + c] = out;
    // candidates for the pivot of column j + 1: rows not yet used (p is used from now on)
    if (c == j + 1 && i != p && !w.used[(size_t)mat * k + i]) {
      const double a = bz_abs2(out);
      if (a > bv) { bv = a; bi = i; }
    }
  }
  block_argmax(bv, bi, sv, si, &w.pv[half_out + (size_t)mat * w.nparts + part],
               &w.pi[half_out + (size_t)mat * w.nparts + part]);
}

// S_{n+1} = (S_n + S_n^{-1}) / 2 with (S_n^{-1})_{i, p_m} = W_{p_i, m}; partial norms
__global__ void __launch_bounds__(kThreads) k_big_update(BigWork w, const double2* __restrict__ Wf,
                                                         const int* __restrict__ pinv) {
  __shared__ double red[2][kThreads / 32];
  const int mat = blockIdx.y, part = blockIdx.x, k = w.k;
  if (w.status[mat] != 0) return;
  const size_t base = (size_t)mat * k * k;
  const int* piv = w.piv + (size_t)mat * k;
  const int* pinvm = pinv + (size_t)mat * k;
  const int r0 = part * kRows;
  double d2 = 0.0, n2 = 0.0;
  bool fin = true;
  for (int e = threadIdx.x; e < kRows * k; e += kThreads) {
    const int i = r0 + e / k, c = e % k;
    if (i >= k) break;
    const double2 inv = Wf[base + (size_t)piv[i] * k + pinvm[c]];
    const double2 s = w.S[base + (size_t)i * k + c];
    const double2 sn = make_double2(0.5 * (s.x + inv.x), 0.5 * (s.y + inv.y));
    fin = fin && isfinite(sn.x) && isfinite(sn.y);
    d2 += bz_abs2(make_double2(sn.x - s.x, sn.y - s.y));
    n2 += bz_abs2(sn);
    w.S[base + (size_t)i * k + c] = sn;
  }
  if (!fin) d2 = NAN;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  }
  if (lane == 0) { red[0][warp] = d2; red[1][warp] = n2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double D = 0.0, N = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) { D += red[0][q]; N += red[1][q]; }
    w.norms[((size_t)mat * w.nparts + part) * 2] = D;
    w.norms[((size_t)mat * w.nparts + part) * 2 + 1] = N;
  }
}

// the inverse permutation of the pivot rows (one block per matrix)
__global__ void k_big_pinv(BigWork w, int* pinv) {
  const int mat = blockIdx.x, k = w.k;
  if (w.status[mat] != 0) return;
  for (int m = threadIdx.x; m < k; m += blockDim.x) pinv[(size_t)mat * k + w.piv[(size_t)mat * k + m]] = m;
}

// convergence of each matrix from the partial norms, in a fixed order (one thread per matrix)
__global__ void k_big_conv(BigWork w, double tol, int* its, int it) {
  const int mat = blockIdx.x * blockDim.x + threadIdx.x;
  if (mat >= w.count || w.status[mat] != 0) return;
  double D = 0.0, N = 0.0;
  for (int q = 0; q < w.nparts; ++q) {
    D += w.norms[((size_t)mat * w.nparts + q) * 2];
    N += w.norms[((size_t)mat * w.nparts + q) * 2 + 1];
  }
  its[mat] = it;
  if (!isfinite(D) || !isfinite(N)) w.status[mat] = 2;
  else if (sqrt(D) <= tol * sqrt(N)) w.status[mat] = 1;
}

}  // namespace

// sgn of `count` dense k x k matrices (device, row-major, complex double) into S (device);
// scratch from the caller (bytes: rh_big_scratch_bytes); per matrix the iterations and
// ok (1 converged, 0 not or singular). The host waits once per iteration (to stop when
// every matrix has converged).
size_t rh_big_scratch_bytes(int count, int k) {
  const int nparts = (k + kRows - 1) / kRows;
  const size_t mk = (size_t)count * k * k * sizeof(double2);
  return 2 * mk + (size_t)count * nparts * (sizeof(double) * 4 + sizeof(int) * 2) + (size_t)count * k * sizeof(int) * 3 +
         (size_t)count * sizeof(int) * 2 + 256 * 16;
}

cudaError_t run_rh_big(int count, int k, const double2* T, double2* S, int* iters, int* ok, double rh_tol,
                       int rh_maxit, void* scratch, cudaStream_t st) {
  BigWork w;
  const int nparts = (k + kRows - 1) / kRows;
  char* p = (char*)scratch;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 255) / 256 * 256;
    return (void*)q;
  };
  const size_t mk = (size_t)count * k * k * sizeof(double2);
  w.S = S;
  w.W0 = (double2*)take(mk);
  w.W1 = (double2*)take(mk);
  w.pv = (double*)take(sizeof(double) * 2 * count * nparts);
  w.pi = (int*)take(sizeof(int) * 2 * count * nparts);
  w.norms = (double*)take(sizeof(double) * 2 * count * nparts);
  w.used = (int*)take(sizeof(int) * count * k);
  w.piv = (int*)take(sizeof(int) * count * k);
  int* pinv = (int*)take(sizeof(int) * count * k);
  w.status = (int*)take(sizeof(int) * count);
  int* its = (int*)take(sizeof(int) * count);
  w.k = k;
  w.count = count;
  w.nparts = nparts;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(S, T, mk, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.status, 0, sizeof(int) * count, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(its, 0, sizeof(int) * count, st)) != cudaSuccess) return e;
  const dim3 grid(nparts, count);
  std::vector<int> stat(count);
  for (int it = 1; it <= rh_maxit; ++it) {
    k_big_start<<<grid, kThreads, 0, st>>>(w);
    for (int j = 0; j < k; ++j) {
      const double2* in = (j & 1) ? w.W1 : w.W0;
      double2* out = (j & 1) ? w.W0 : w.W1;
      k_big_col<<<grid, kThreads, 0, st>>>(w, j, in, out);
    }
    const double2* Wf = (k & 1) ? w.W1 : w.W0;
    k_big_pinv<<<count, 256, 0, st>>>(w, pinv);
    k_big_update<<<grid, kThreads, 0, st>>>(w, Wf, pinv);
    k_big_conv<<<(count + 127) / 128, 128, 0, st>>>(w, rh_tol, its, it);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(stat.data(), w.status, sizeof(int) * count, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (std::all_of(stat.begin(), stat.end(), [](int s) { return s != 0; })) break;
  }
  std::vector<int> itv(count);
  if ((e = cudaMemcpyAsync(itv.data(), its, sizeof(int) * count, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  for (int i = 0; i < count; ++i) {
    if (iters) iters[i] = itv[i];
    if (ok) ok[i] = stat[i] == 1;
  }
  return cudaSuccess;
}

namespace {

// dense H_k of problem list[g] from its tridiagonal coefficients (index j = 1..k): diagonal
// alp[j], subdiagonal H_{j,j-1} = bet[j], superdiagonal H_{j-1,j} = gam[j]
__global__ void k_nn_dense(int k, const int* __restrict__ list, const double2* __restrict__ alp,
                           const double2* __restrict__ bet, const double2* __restrict__ gam, int ldc, double2* H) {
  const int g = blockIdx.y;
  const size_t co = (size_t)list[g] * ldc;
  double2* Hg = H + (size_t)g * k * k;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)k * k; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), c = (int)(e % k);
    double2 v = make_double2(0.0, 0.0);
    if (i == c) v = alp[co + i + 1];
    else if (i == c + 1) v = bet[co + i + 1];
    else if (c == i + 1) v = gam[co + c + 1];
    Hg[e] = v;
  }
}

// c = first column of sgn(H_k) for problem list[g] (one block each), with the stopping
// estimates as the nested level reports them (the inner estimate is 0: nothing is nested)
__global__ void k_nn_combine(int k, const int* __restrict__ list, const double2* __restrict__ S,
                             const int* __restrict__ ok, const int* __restrict__ its, const double* __restrict__ nv,
                             int ldc, double2* c, int ldo, void* cacc, int prec, double* est_inner,
                             const double2* cprev, int ldp, const int* kprev_dev, double* est_outer, int* rh_status,
                             int* rh_iters) {
  __shared__ double red[2][32];
  const int g = blockIdx.x, prob = list[g];
  const double2* Sg = S + (size_t)g * k * k;
  const int kp = kprev_dev ? kprev_dev[prob] : 0;
  double nc = 0.0, no = 0.0;
  for (int m = threadIdx.x; m < ldo - 1; m += blockDim.x) {
    const double2 v = m < k && ok[g] ? Sg[(size_t)m * k] : make_double2(0.0, 0.0);
    c[(size_t)prob * ldo + m + 1] = v;
    if (cacc) {
      const double sc = m < k ? 1.0 / nv[(size_t)prob * ldc + m + 1] : 0.0;
      const double2 vs = make_double2(v.x * sc, v.y * sc);
      if (prec == OV_PREC_FP64) {
        ((double2*)cacc)[(size_t)prob * ldo + m + 1] = vs;
      } else {
        const float rh = __double2float_rn(vs.x), ih = __double2float_rn(vs.y);
        ((float4*)cacc)[(size_t)prob * ldo + m + 1] =
            make_float4(rh, __double2float_rn(vs.x - (double)rh), ih, __double2float_rn(vs.y - (double)ih));
      }
    }
    if (m < k) {
      nc += v.x * v.x + v.y * v.y;
      if (kp > 0 && cprev) {
        const double2 pv = m < kp ? cprev[(size_t)prob * ldp + m + 1] : make_double2(0.0, 0.0);
        no += (v.x - pv.x) * (v.x - pv.x) + (v.y - pv.y) * (v.y - pv.y);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nc += __shfl_xor_sync(0xffffffffu, nc, o);
    no += __shfl_xor_sync(0xffffffffu, no, o);
  }
  if (lane == 0) { red[0][warp] = nc; red[1][warp] = no; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double C = 0.0, O = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { C += red[0][q]; O += red[1][q]; }
    est_inner[prob] = ok[g] ? 0.0 : INFINITY;
    if (est_outer) est_outer[prob] = (kp > 0 && cprev && ok[g]) ? sqrt(O) / sqrt(C) : INFINITY;
    rh_status[prob] = ok[g] ? 0 : 1;
    rh_iters[prob] = its[g];
  }
}

}  // namespace

size_t nonnested_scratch_bytes(int count, int kmax) {
  const size_t mk = (size_t)count * kmax * kmax * sizeof(double2);
  return 2 * mk + rh_big_scratch_bytes(count, kmax) + (size_t)count * sizeof(int) * 3 + 1024;
}

cudaError_t run_nonnested(int count, const int* k_host, const double2* alp, const double2* bet, const double2* gam,
                          const double* nv, int ldc, double rh_tol, int rh_maxit, double2* c, int ldo, void* cacc,
                          int prec, double* est_inner, const double2* cprev, int ldp, const int* kprev_dev,
                          double* est_outer, int* rh_status, int* rh_iters, void* scratch, cudaStream_t st) {
  int kmax = 0;
  for (int i = 0; i < count; ++i) kmax = std::max(kmax, k_host[i]);
  char* p = (char*)scratch;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 255) / 256 * 256;
    return (void*)q;
  };
  const size_t mk = (size_t)count * kmax * kmax * sizeof(double2);
  double2* H = (double2*)take(mk);
  double2* S = (double2*)take(mk);
  int* list = (int*)take(sizeof(int) * count);
  int* okd = (int*)take(sizeof(int) * count);
  int* itsd = (int*)take(sizeof(int) * count);
  void* big = take(rh_big_scratch_bytes(count, kmax));
  cudaError_t e;
  // one Roberts-Higham batch per distinct k
  std::vector<int> done(count, 0);
  for (int i0 = 0; i0 < count; ++i0) {
    if (done[i0]) continue;
    const int k = k_host[i0];
    std::vector<int> grp;
    for (int i = i0; i < count; ++i)
      if (!done[i] && k_host[i] == k) {
        grp.push_back(i);
        done[i] = 1;
      }
    const int ng = (int)grp.size();
    if ((e = cudaMemcpyAsync(list, grp.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    k_nn_dense<<<dim3(std::max(1, std::min(64, (k * k + 255) / 256)), ng), 256, 0, st>>>(k, list, alp, bet, gam, ldc, H);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<int> its(ng), ok(ng);
    if ((e = run_rh_big(ng, k, H, S, its.data(), ok.data(), rh_tol, rh_maxit, big, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(okd, ok.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(itsd, its.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    k_nn_combine<<<ng, 256, 0, st>>>(k, list, S, okd, itsd, nv, ldc, c, ldo, cacc, prec, est_inner, cprev, ldp, kprev_dev,
                                     est_outer, rh_status, rh_iters);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the host vectors above are read by the copies: wait before they go out of scope
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ov
