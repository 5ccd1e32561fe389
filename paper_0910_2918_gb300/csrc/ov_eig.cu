// Critical eigenpairs of A = gamma5 D_w(mu) and the deflated sign function (Sec. 2, the
// deflation paragraph):
//
//   f(A) x = R_m f(Lambda_m) (L_m^dag x) + f(A) (I - R_m L_m^dag) x
//
// with the m eigenvalues of smallest magnitude, their right eigenvectors R_m and left
// eigenvectors L_m (L_m^dag R_m = 1).
//
// Eigensolver: subspace iteration with a Chebyshev polynomial filter in A^2 (Zhou and Saad,
// "Chebyshev-filtered subspace iteration", J. Comput. Phys. 219 (2006)) on a block of
// b > m vectors: the polynomial T_d(l(A^2)), l mapping [a, b_max] onto [-1, 1], damps the
// eigenvectors whose lambda^2 lies in that interval (the bulk) and amplifies those of small
// |lambda|; a polynomial in A keeps A's eigenvectors, so the same iteration serves the
// non-Hermitian case (mu != 0). Each iteration: filter, orthonormalise (Cholesky QR twice),
// Rayleigh-Ritz with A^2 on the block (the wanted eigenvalues are the smallest of A^2, an
// end of its spectrum; Rayleigh-Ritz with A itself on a subspace aimed at the interior of
// A's spectrum gives spurious Ritz values near 0) with the Ritz vectors kept orthonormal
// through the QR factorisation of their coefficients, then Rayleigh-Ritz with A on the
// leading m of them (the projected b x b and m x m problems are solved on the host,
// ov_small.cpp), residuals ||A x - lambda x||. At mu != 0 the left eigenvectors are the right eigenvectors of
// A^dag = gamma5 D_w(-mu) for conj(lambda): a second job on A(-mu), matched by eigenvalue and
// biorthonormalised (L <- L (L^dag R)^{-dag}).
//
// All n-vectors are canonical complex doubles on the device; the matvecs run in the handle's
// arithmetic (ov_api.cu: ApplySet, one launch over every job of an iteration).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <complex>
#include <thread>
#include <vector>

#include "ov_internal.h"

namespace ov {
namespace {

constexpr int kEigThreads = 256;
constexpr int kGramChunk = 32;
constexpr int kGramBlocks = 304;  // two blocks per SM, grid-stride over the vector length

__device__ __forceinline__ double2 e_cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) b
__device__ __forceinline__ double2 e_cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// partial sums of G_ij = X_i^dag Y_j over a grid-stride share of the n entries
// (X: bx vectors, Y: by vectors, each of length n with stride ldx / ldy entries)
__global__ void __launch_bounds__(kEigThreads) k_gram_part(size_t n, const double2* __restrict__ X, size_t ldx, int bx,
                                                          const double2* __restrict__ Y, size_t ldy, int by,
                                                          double2* part) {
  extern __shared__ double2 sm[];
  double2* xs = sm;                        // [bx][kGramChunk]
  double2* ys = sm + (size_t)bx * kGramChunk;  // [by][kGramChunk]
  const int npairs = bx * by;
  constexpr int kMaxPairs = 16;            // pairs a thread owns: bx * by <= kEigThreads * kMaxPairs
  double2 acc[kMaxPairs];
#pragma unroll
  for (int q = 0; q < kMaxPairs; ++q) acc[q] = make_double2(0.0, 0.0);
  for (size_t c0 = (size_t)blockIdx.x * kGramChunk; c0 < n; c0 += (size_t)gridDim.x * kGramChunk) {
    for (int t = threadIdx.x; t < (bx + by) * kGramChunk; t += blockDim.x) {
      const int v = t / kGramChunk, e = t % kGramChunk;
      const size_t g = c0 + e;
      double2 val = make_double2(0.0, 0.0);
      if (g < n) val = v < bx ? X[(size_t)v * ldx + g] : Y[(size_t)(v - bx) * ldy + g];
      sm[(size_t)v * kGramChunk + e] = val;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxPairs; ++q) {
      const int p = threadIdx.x + q * kEigThreads;
      if (p < npairs) {
        const int i = p / by, j = p % by;
        double2 a = acc[q];
        for (int e = 0; e < kGramChunk; ++e) {
          const double2 t = e_cmulc(xs[(size_t)i * kGramChunk + e], ys[(size_t)j * kGramChunk + e]);
          a.x += t.x;
          a.y += t.y;
        }
        acc[q] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kMaxPairs; ++q) {
    const int p = threadIdx.x + q * kEigThreads;
    if (p < npairs) part[(size_t)blockIdx.x * npairs + p] = acc[q];
  }
}

// G = sum over blocks of the partial sums, in block order (one thread per pair)
__global__ void k_gram_fin(int nblocks, int npairs, const double2* __restrict__ part, double2* G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblocks; ++b) {
    const double2 v = part[(size_t)b * npairs + p];
    s.x += v.x;
    s.y += v.y;
  }
  G[p] = s;
}

// Y_j = beta Y_j + alpha sum_i X_i C_ij   (C: bx x by row-major; Y must not alias X)
__global__ void __launch_bounds__(kEigThreads) k_block_mul(size_t n, const double2* __restrict__ X, size_t ldx, int bx,
                                                          const double2* __restrict__ C, double2* __restrict__ Y,
                                                          size_t ldy, int by, double alpha, double beta) {
  extern __shared__ double2 cs[];
  for (int t = threadIdx.x; t < bx * by; t += blockDim.x) cs[t] = C[t];
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    for (int j = 0; j < by; ++j) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = 0; i < bx; ++i) {
        const double2 t = e_cmul(X[(size_t)i * ldx + e], cs[i * by + j]);
        s.x += t.x;
        s.y += t.y;
      }
      double2 y = beta == 0.0 ? make_double2(0.0, 0.0) : Y[(size_t)j * ldy + e];
      y.x = beta * y.x + alpha * s.x;
      y.y = beta * y.y + alpha * s.y;
      Y[(size_t)j * ldy + e] = y;
    }
  }
}

// Chebyshev recurrence on A^2 with l(z) = s z + t:
//   first step: out = s W + t T    (W = A^2 T)
//   later:      out = 2 (s W + t T) - P
__global__ void k_cheb(size_t n, const double2* __restrict__ W, const double2* __restrict__ T,
                       const double2* __restrict__ P, double s, double t, int first, double2* out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double2 w = W[e], v = T[e];
    double2 o = make_double2(s * w.x + t * v.x, s * w.y + t * v.y);
    if (!first) {
      const double2 p = P[e];
      o = make_double2(2.0 * o.x - p.x, 2.0 * o.y - p.y);
    }
    out[e] = o;
  }
}

// per-vector partial sums of ||Z_i - theta_i V_i||^2 (one block row per vector)
__global__ void __launch_bounds__(kEigThreads) k_resid_part(size_t n, const double2* __restrict__ Z,
                                                            const double2* __restrict__ V, size_t ld,
                                                            const double2* __restrict__ theta, double* part) {
  __shared__ double red[kEigThreads / 32];
  const int i = blockIdx.y;
  const double2 th = theta[i];
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double2 z = Z[(size_t)i * ld + e], v = V[(size_t)i * ld + e];
    const double2 tv = e_cmul(th, v);
    const double dx = z.x - tv.x, dy = z.y - tv.y;
    acc += dx * dx + dy * dy;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kEigThreads / 32; ++w) s += red[w];
    part[(size_t)i * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_resid_fin(int b, int nparts, const double* __restrict__ part, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += part[(size_t)i * nparts + q];
  out[i] = sqrt(s);
}

// y = x + gamma5 y (the overlap operator's epilogue, canonical layout)
__global__ void k_add_x_g5(size_t n, const double2* __restrict__ x, double2* y) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double2 v = y[e];
    if ((e % 12) >= 6) v = make_double2(-v.x, -v.y);
    const double2 a = x[e];
    y[e] = make_double2(a.x + v.x, a.y + v.y);
  }
}

// the Chebyshev recurrence of k_cheb over several jobs' blocks at once: segment i covers
// entries [start_i, start_{i+1}) of the concatenation of the active blocks and maps them to
// the buffers at off_i, with the job's own interval (s_i, t_i)
struct ChebSeg {
  size_t start, off;
  double s, t;
};
__global__ void k_cheb_seg(int nseg, const ChebSeg* __restrict__ seg, size_t total, const double2* __restrict__ W,
                           const double2* __restrict__ T, const double2* __restrict__ P, int first, double2* out) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (size_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg[mid].start <= v) lo = mid;
      else hi = mid - 1;
    }
    const ChebSeg sg = seg[lo];
    const size_t e = sg.off + (v - sg.start);
    const double2 w = W[e], x = T[e];
    double2 o = make_double2(sg.s * w.x + sg.t * x.x, sg.s * w.y + sg.t * x.y);
    if (!first) {
      const double2 p = P[e];
      o = make_double2(2.0 * o.x - p.x, 2.0 * o.y - p.y);
    }
    out[e] = o;
  }
}

// start vectors: entries uniform in [-1/2, 1/2) + i [-1/2, 1/2) from a counter-based hash
// (SplitMix64 finaliser, Steele, Lea and Flood 2014) of (seed, index)
__device__ __forceinline__ unsigned long long e_mix(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void k_fill_random(size_t n, unsigned long long seed, double2* x) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long r = e_mix(seed * 0x100000001b3ull + e);
    x[e] = make_double2((double)(r >> 40) / 16777216.0 - 0.5, (double)((r >> 16) & 0xffffffull) / 16777216.0 - 0.5);
  }
}

int grid_n(size_t n) { return (int)std::min<size_t>((n + kEigThreads - 1) / kEigThreads, 152 * 8); }

}  // namespace

// ---------------------------------------------------------------------------------------
// block linear algebra used by the eigensolver and the deflated apply

cudaError_t block_gram(size_t n, const double2* X, size_t ldx, int bx, const double2* Y, size_t ldy, int by,
                       double2* part, double2* G, cudaStream_t st) {
  if (bx * by > kEigThreads * 16) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double2) * (size_t)(bx + by) * kGramChunk;
  cudaError_t e = cudaFuncSetAttribute(k_gram_part, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (e != cudaSuccess) return e;
  k_gram_part<<<kGramBlocks, kEigThreads, smem, st>>>(n, X, ldx, bx, Y, ldy, by, part);
  k_gram_fin<<<(bx * by + 127) / 128, 128, 0, st>>>(kGramBlocks, bx * by, part, G);
  return cudaGetLastError();
}
size_t block_gram_part_bytes(int bx, int by) { return sizeof(double2) * (size_t)kGramBlocks * bx * by; }

cudaError_t block_mul(size_t n, const double2* X, size_t ldx, int bx, const double2* C, double2* Y, size_t ldy, int by,
                      double alpha, double beta, cudaStream_t st) {
  if (bx * by > 4096) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_block_mul, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (e != cudaSuccess) return e;
  k_block_mul<<<grid_n(n), kEigThreads, sizeof(double2) * (size_t)bx * by, st>>>(n, X, ldx, bx, C, Y, ldy, by, alpha,
                                                                                 beta);
  return cudaGetLastError();
}

cudaError_t add_x_gamma5(size_t n, const double2* x, double2* y, cudaStream_t st) {
  k_add_x_g5<<<grid_n(n), kEigThreads, 0, st>>>(n, x, y);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------
// the eigensolver, all jobs together: every matvec of an iteration is one stencil launch over
// all active jobs' blocks (ov_api.cu: ApplySet), the block kernels are queued per job on the
// handle's stream, and the projected problems of all jobs are solved on the host between two
// synchronisations (in parallel over jobs). A job leaves the active set when its m residuals
// are below tol (its vectors are copied out then) or after maxit iterations.
int eig_smallest(ov_handle* h, std::vector<EigJob>& jobs, int m, int b, int deg, double tol, int maxit, int verbose) {
  using cd = std::complex<double>;
  cudaStream_t st = handle_stream(h);
  const int nj = (int)jobs.size();
  if (nj == 0) return OV_OK;
  std::vector<size_t> n(nj), off(nj);
  std::vector<char> herm(nj);
  size_t S = 0;
  for (int e = 0; e < nj; ++e) {
    n[e] = lattice_size(h, jobs[e].q);
    off[e] = S;
    S += n[e] * (size_t)b;
    herm[e] = lattice_mu(h, jobs[e].q) == 0.0;
    jobs[e].lam.assign(m, cd(0.0));
    jobs[e].res.assign(m, INFINITY);
    jobs[e].its = 0;
    jobs[e].status = OV_NOT_CONVERGED;
  }
  const size_t bb = (size_t)b * b;
  const int rgrid = 64;
  // work: V, T0, T1, W, Z (all jobs' blocks), gram partials, small matrices
  double2 *V = nullptr, *T0 = nullptr, *T1 = nullptr, *W = nullptr, *Z = nullptr, *part = nullptr, *G = nullptr,
          *Cd = nullptr, *thd = nullptr;
  double *rpart = nullptr, *rn = nullptr;
  ChebSeg* segd = nullptr;
  ApplySet *setB = nullptr, *setM = nullptr;
  auto cleanup = [&]() {
    for (void* p : {(void*)V, (void*)T0, (void*)T1, (void*)W, (void*)Z, (void*)part, (void*)G, (void*)Cd, (void*)thd,
                    (void*)rpart, (void*)rn, (void*)segd})
      if (p) cudaFree(p);
    apply_set_destroy(setB);
    apply_set_destroy(setM);
    setB = setM = nullptr;
  };
  if (cudaMalloc(&V, sizeof(double2) * S) != cudaSuccess || cudaMalloc(&T0, sizeof(double2) * S) != cudaSuccess ||
      cudaMalloc(&T1, sizeof(double2) * S) != cudaSuccess || cudaMalloc(&W, sizeof(double2) * S) != cudaSuccess ||
      cudaMalloc(&Z, sizeof(double2) * S) != cudaSuccess ||
      cudaMalloc(&part, block_gram_part_bytes(b, b)) != cudaSuccess ||
      cudaMalloc(&G, sizeof(double2) * bb * nj) != cudaSuccess || cudaMalloc(&Cd, sizeof(double2) * bb * nj) != cudaSuccess ||
      cudaMalloc(&thd, sizeof(double2) * (size_t)m * nj) != cudaSuccess ||
      cudaMalloc(&rpart, sizeof(double) * (size_t)m * rgrid * nj) != cudaSuccess ||
      cudaMalloc(&rn, sizeof(double) * (size_t)m * nj) != cudaSuccess ||
      cudaMalloc(&segd, sizeof(ChebSeg) * nj) != cudaSuccess) {
    cleanup();
    return OV_ERR_NOMEM;
  }
#define ECK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      fprintf(stderr, "libov: eigensolver: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      cleanup();                                                                    \
      return OV_ERR_CUDA;                                                           \
    }                                                                               \
  } while (0)
#define RCK(call)          \
  do {                     \
    int r_ = (call);       \
    if (r_ != OV_OK) {     \
      cleanup();           \
      return r_;           \
    }                      \
  } while (0)
  // the host's share: the projected problems of the active jobs, in parallel over jobs
  auto par_for = [](const std::vector<int>& act, const auto& fn) {
    const int na = (int)act.size();
    const int nt = std::min<int>(na, std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    if (nt <= 1) {
      for (int e : act) fn(e);
      return;
    }
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
      th.emplace_back([&]() {
        for (int i; (i = next.fetch_add(1)) < na;) fn(act[i]);
      });
    for (auto& t : th) t.join();
  };
  std::vector<int> act(nj);
  for (int e = 0; e < nj; ++e) act[e] = e;
  bool act_changed = true;
  // apply sets over the active jobs: b vectors each (setB), the leading m (setM)
  auto make_set = [&](int nvec, int flip, const std::vector<int>& which, ApplySet** out) -> int {
    std::vector<ApplyItem> items;
    for (int e : which)
      for (int i = 0; i < nvec; ++i) items.push_back({jobs[e].q, jobs[e].neg ^ flip, off[e] + (size_t)i * n[e]});
    return apply_set_create(h, items, S, out);
  };
  auto refresh_sets = [&]() -> int {
    if (!act_changed) return OV_OK;
    apply_set_destroy(setB);
    apply_set_destroy(setM);
    setB = setM = nullptr;
    if (act.empty()) return OV_OK;
    int rc = make_set(b, 0, act, &setB);
    if (rc == OV_OK) rc = make_set(m, 0, act, &setM);
    act_changed = false;
    return rc;
  };
  auto drop = [&](const std::vector<char>& gone) {
    std::vector<int> keep;
    for (int e : act)
      if (!gone[e]) keep.push_back(e);
    if (keep.size() != act.size()) act_changed = true;
    act.swap(keep);
  };
  // a job whose projected problem breaks down leaves with no usable pair
  auto fail = [&](int e) {
    jobs[e].status = OV_ERR_BREAKDOWN;
    jobs[e].res.assign(m, INFINITY);
  };
  std::vector<double2> Gh(bb * nj), Ch(bb * nj), Sv(bb * nj), wv((size_t)b * nj), th((size_t)m * nj);
  std::vector<double> wr((size_t)b * nj), t2(nj, 0.0), rh((size_t)m * nj);
  // orthonormalise every active job's block X in place (Cholesky QR twice); Tmp: scratch
  auto orth = [&](double2*& X, double2*& Tmp) -> int {
    for (int pass = 0; pass < 2; ++pass) {
      for (int e : act)
        if (block_gram(n[e], X + off[e], n[e], b, X + off[e], n[e], b, part, G + e * bb, st) != cudaSuccess)
          return OV_ERR_CUDA;
      if (cudaMemcpyAsync(Gh.data(), G, sizeof(double2) * bb * nj, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return OV_ERR_CUDA;
      std::vector<char> bad(nj, 0);
      par_for(act, [&](int e) {
        double2* g = Gh.data() + e * bb;
        double tr = 0.0;
        for (int i = 0; i < b; ++i) tr += g[(size_t)i * b + i].x;
        if (pass == 0)  // a tiny shift keeps the factorisation defined for a nearly dependent block
          for (int i = 0; i < b; ++i) g[(size_t)i * b + i].x += 1e-14 * tr;
        if (!small_chol_inv(b, g, Ch.data() + e * bb)) bad[e] = 1;
      });
      for (int e : act)
        if (bad[e]) fail(e);
      drop(bad);
      if (act.empty()) return OV_OK;
      if (cudaMemcpyAsync(Cd, Ch.data(), sizeof(double2) * bb * nj, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return OV_ERR_CUDA;
      for (int e : act)
        if (block_mul(n[e], X + off[e], n[e], b, Cd + e * bb, Tmp + off[e], n[e], b, 1.0, 0.0, st) != cudaSuccess)
          return OV_ERR_CUDA;
      std::swap(X, Tmp);
    }
    return OV_OK;
  };
  {
    k_fill_random<<<grid_n(S), kEigThreads, 0, st>>>(S, 0x6f76ull, V);  // one stream of entries over all jobs
    ECK(cudaGetLastError());
  }
  RCK(orth(V, T0));
  RCK(refresh_sets());
  // The filter needs an upper bound of |lambda|^2 over the whole spectrum: beyond it the
  // Chebyshev polynomial grows as fast as below the cut and would amplify the largest
  // eigenvectors. ||A||^2 from power steps on A^dag A (a lower estimate) with a 25% margin,
  // capped by the bound of the operator's form, ||A|| <= |m_w + 4| + 6 + 2 cosh(mu); a block
  // whose largest Ritz value comes near the bound enlarges it (safeguard below).
  std::vector<double> amax2(nj, 0.0), a_cut(nj), anorm(nj);
  {
    ApplySet *P0 = nullptr, *P1 = nullptr;
    int rc = make_set(1, 0, act, &P0);
    if (rc == OV_OK) rc = make_set(1, 1, act, &P1);  // the adjoint: A(-mu) of A(mu) and back
    std::vector<double2> g2(2 * (size_t)nj), sc(nj);
    for (int e : act) {
      cudaError_t ce = cudaMemcpyAsync(T1 + off[e], V + off[e], sizeof(double2) * n[e], cudaMemcpyDeviceToDevice, st);
      if (ce != cudaSuccess) rc = OV_ERR_CUDA;
    }
    for (int it = 0; it < 60 && rc == OV_OK; ++it) {
      rc = apply_set_run(h, P0, T1, W);
      if (rc == OV_OK) rc = apply_set_run(h, P1, W, Z);
      cudaError_t ce = cudaSuccess;
      for (int e : act) {
        if (ce == cudaSuccess) ce = block_gram(n[e], Z + off[e], n[e], 1, Z + off[e], n[e], 1, part, G + 2 * e, st);
        if (ce == cudaSuccess) ce = block_gram(n[e], T1 + off[e], n[e], 1, Z + off[e], n[e], 1, part, G + 2 * e + 1, st);
      }
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(g2.data(), G, sizeof(double2) * 2 * nj, cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
      for (int e : act) {
        amax2[e] = std::max(amax2[e], g2[2 * e + 1].x);  // Rayleigh quotient of A^dag A (T1 has unit norm)
        sc[e] = make_double2(1.0 / sqrt(g2[2 * e].x), 0.0);
      }
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(Cd, sc.data(), sizeof(double2) * nj, cudaMemcpyHostToDevice, st);
      for (int e : act)
        if (ce == cudaSuccess) ce = block_mul(n[e], Z + off[e], n[e], 1, Cd + e, T1 + off[e], n[e], 1, 1.0, 0.0, st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);  // sc is read by the copy
      if (ce != cudaSuccess && rc == OV_OK) rc = OV_ERR_CUDA;
    }
    apply_set_destroy(P0);
    apply_set_destroy(P1);
    RCK(rc);
    for (int e : act) {
      const double form = fabs(lattice_mass(h, jobs[e].q)) + 6.0 + 2.0 * cosh(lattice_mu(h, jobs[e].q));
      if (verbose && e == act[0])
        fprintf(stderr, "{\"ov_eig_bound\": %d, \"power\": %.6g, \"form\": %.6g}\n", e, amax2[e], form * form);
      amax2[e] = std::min(1.25 * amax2[e], form * form);
      anorm[e] = sqrt(amax2[e]);
      a_cut[e] = 0.05 * amax2[e];
    }
  }
  auto mag2 = [](double2 z) { return z.x * z.x + z.y * z.y; };
  int it = 0;
  using clk = std::chrono::steady_clock;
  auto secs = [](clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); };
  for (it = 1; it <= maxit && !act.empty(); ++it) {
    const clk::time_point t_start = clk::now();
    RCK(refresh_sets());
    // filter: T_d(l(A^2)) V, l(z) = s z + t mapping [a_cut, amax2] onto [-1, 1] per job. The
    // degree d (<= deg, >= 8) keeps the largest amplification, T_d(|l(0)|) = cosh(d acosh|t|),
    // within kAmp for every active job: a larger spread of the block's column norms would leave
    // the filtered block too ill-conditioned for the Cholesky QR that follows.
    constexpr double kAmp = 1e6;
    std::vector<ChebSeg> sg;
    size_t tot = 0;
    int dgo = deg;
    for (int e : act) {
      const double s = 2.0 / (amax2[e] - a_cut[e]), t = -(amax2[e] + a_cut[e]) / (amax2[e] - a_cut[e]);
      sg.push_back({tot, off[e], s, t});
      tot += n[e] * (size_t)b;
      const double x = acosh(fabs(t));
      if (x > 0.0) dgo = std::min<int>(dgo, std::max(8, (int)(acosh(kAmp) / x)));
    }
    const int nseg = (int)sg.size();
    ECK(cudaMemcpyAsync(segd, sg.data(), sizeof(ChebSeg) * nseg, cudaMemcpyHostToDevice, st));
    // T0 = V, T1 = l(A^2) V, then T_{k+1} = 2 l(A^2) T_k - T_{k-1} (kept in V / T0 / T1)
    RCK(apply_set_run(h, setB, V, Z));
    RCK(apply_set_run(h, setB, Z, W));
    k_cheb_seg<<<grid_n(tot), kEigThreads, 0, st>>>(nseg, segd, tot, W, V, nullptr, 1, T1);
    ECK(cudaGetLastError());
    double2* Tm = V;   // T_{k-1}
    double2* Tc = T1;  // T_k
    double2* Tn = T0;  // T_{k+1}
    for (int k = 1; k < dgo; ++k) {
      RCK(apply_set_run(h, setB, Tc, Z));
      RCK(apply_set_run(h, setB, Z, W));
      k_cheb_seg<<<grid_n(tot), kEigThreads, 0, st>>>(nseg, segd, tot, W, Tc, Tm, 0, Tn);
      ECK(cudaGetLastError());
      double2* o = Tm;
      Tm = Tc;
      Tc = Tn;
      Tn = o;
    }
    ECK(cudaStreamSynchronize(st));  // sg is read by the copy before it goes out of scope
    const clk::time_point t_filter = clk::now();
    {
      double2* bufs[3] = {V, T0, T1};
      double2* others[2];
      int k2 = 0;
      for (double2* bp : bufs)
        if (bp != Tc) others[k2++] = bp;
      V = Tc;
      T0 = others[0];
      T1 = others[1];
    }
    RCK(orth(V, T0));
    if (act.empty()) break;
    RCK(refresh_sets());
    // Rayleigh-Ritz with A^2 on the block (its wanted eigenvalues are at the bottom of the
    // spectrum of A^2, so no spurious Ritz values; Rayleigh-Ritz with A on a subspace aimed
    // at the interior of A's spectrum gives spurious values near 0 from mixed +-lambda
    // vectors): Z = A V, W = A Z, H2 = V^dag W
    RCK(apply_set_run(h, setB, V, Z));
    RCK(apply_set_run(h, setB, Z, W));
    for (int e : act) ECK(block_gram(n[e], V + off[e], n[e], b, W + off[e], n[e], b, part, G + e * bb, st));
    ECK(cudaMemcpyAsync(Gh.data(), G, sizeof(double2) * bb * nj, cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    {
      std::vector<char> bad(nj, 0);
      par_for(act, [&](int e) {
        double2* g = Gh.data() + e * bb;
        double2* w = wv.data() + (size_t)e * b;
        double2* sv = Sv.data() + e * bb;
        bool ok;
        if (herm[e]) {
          for (int i = 0; i < b; ++i)
            for (int j = 0; j < i; ++j) {  // symmetrise the projection (roundoff)
              const double2 u = g[(size_t)i * b + j], v = g[(size_t)j * b + i];
              const double2 avg = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
              g[(size_t)i * b + j] = avg;
              g[(size_t)j * b + i] = make_double2(avg.x, -avg.y);
            }
          double* r = wr.data() + (size_t)e * b;
          ok = small_eigh(b, g, r, sv);
          for (int i = 0; i < b; ++i) w[i] = make_double2(r[i], 0.0);
        } else {
          ok = small_eig(b, g, w, sv);
        }
        if (!ok) {
          bad[e] = 1;
          return;
        }
        std::vector<int> idx(b);
        for (int i = 0; i < b; ++i) idx[i] = i;
        std::sort(idx.begin(), idx.end(), [&](int x, int y) { return mag2(w[x]) < mag2(w[y]); });
        // the eigenvectors by increasing |theta^2| (into Gh's slot, no longer needed), then the
        // unitary factor of their QR factorisation: its leading m columns span the leading m
        // Ritz vectors, and V Q stays orthonormal (the eigenvectors of a non-Hermitian H2 are
        // not orthogonal)
        for (int i = 0; i < b; ++i)
          for (int j = 0; j < b; ++j) g[(size_t)i * b + j] = sv[(size_t)i * b + idx[j]];
        if (!small_qr_q(b, g, Ch.data() + e * bb)) {
          bad[e] = 1;
          return;
        }
        t2[e] = sqrt(mag2(w[idx[b - 1]]));  // largest |theta^2| of the block
      });
      for (int e : act)
        if (bad[e]) fail(e);
      drop(bad);
      if (act.empty()) break;
    }
    // the orthonormal basis V Q of the Ritz vectors of A^2
    ECK(cudaMemcpyAsync(Cd, Ch.data(), sizeof(double2) * bb * nj, cudaMemcpyHostToDevice, st));
    for (int e : act) ECK(block_mul(n[e], V + off[e], n[e], b, Cd + e * bb, T0 + off[e], n[e], b, 1.0, 0.0, st));
    std::swap(V, T0);
    RCK(refresh_sets());
    const clk::time_point t_rr2 = clk::now();
    // Rayleigh-Ritz with A on the leading m vectors: H1 = V_m^dag A V_m
    RCK(apply_set_run(h, setM, V, Z));
    for (int e : act) ECK(block_gram(n[e], V + off[e], n[e], m, Z + off[e], n[e], m, part, G + e * bb, st));
    ECK(cudaMemcpyAsync(Gh.data(), G, sizeof(double2) * bb * nj, cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    {
      std::vector<char> bad(nj, 0);
      par_for(act, [&](int e) {
        double2* H1 = Gh.data() + e * bb;  // m x m, row-major
        std::vector<double2> S1((size_t)m * m), w1(m);
        std::vector<double> w1r(m);
        bool ok;
        if (herm[e]) {
          for (int i = 0; i < m; ++i)
            for (int j = 0; j < i; ++j) {
              const double2 u = H1[(size_t)i * m + j], v = H1[(size_t)j * m + i];
              const double2 avg = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
              H1[(size_t)i * m + j] = avg;
              H1[(size_t)j * m + i] = make_double2(avg.x, -avg.y);
            }
          ok = small_eigh(m, H1, w1r.data(), S1.data());
          for (int i = 0; i < m; ++i) w1[i] = make_double2(w1r[i], 0.0);
        } else {
          ok = small_eig(m, H1, w1.data(), S1.data());
        }
        if (!ok) {
          bad[e] = 1;
          return;
        }
        std::vector<int> o1(m);
        for (int i = 0; i < m; ++i) o1[i] = i;
        std::sort(o1.begin(), o1.end(), [&](int x, int y) { return mag2(w1[x]) < mag2(w1[y]); });
        double2* c = Ch.data() + e * bb;  // m x m
        for (int i = 0; i < m; ++i)
          for (int j = 0; j < m; ++j) c[(size_t)i * m + j] = S1[(size_t)i * m + o1[j]];
        for (int j = 0; j < m; ++j) th[(size_t)e * m + j] = w1[o1[j]];
      });
      for (int e : act)
        if (bad[e]) fail(e);
      drop(bad);
      if (act.empty()) break;
    }
    // eigenvector estimates X = V_m C1 (in T1), A X = Z_m C1 (in W); residuals ||A x - lambda x||
    ECK(cudaMemcpyAsync(Cd, Ch.data(), sizeof(double2) * bb * nj, cudaMemcpyHostToDevice, st));
    ECK(cudaMemcpyAsync(thd, th.data(), sizeof(double2) * (size_t)m * nj, cudaMemcpyHostToDevice, st));
    for (int e : act) {
      ECK(block_mul(n[e], V + off[e], n[e], m, Cd + e * bb, T1 + off[e], n[e], m, 1.0, 0.0, st));
      ECK(block_mul(n[e], Z + off[e], n[e], m, Cd + e * bb, W + off[e], n[e], m, 1.0, 0.0, st));
      k_resid_part<<<dim3(rgrid, m), kEigThreads, 0, st>>>(n[e], W + off[e], T1 + off[e], n[e], thd + (size_t)e * m,
                                                           rpart + (size_t)e * m * rgrid);
      k_resid_fin<<<(m + 127) / 128, 128, 0, st>>>(m, rgrid, rpart + (size_t)e * m * rgrid, rn + (size_t)e * m);
      ECK(cudaGetLastError());
    }
    ECK(cudaMemcpyAsync(rh.data(), rn, sizeof(double) * (size_t)m * nj, cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    std::vector<char> fin(nj, 0);
    double worst_all = 0.0;
    for (int e : act) {
      double worst = 0.0;
      for (int i = 0; i < m; ++i) {
        const double2 z = th[(size_t)e * m + i];
        jobs[e].lam[i] = cd(z.x, z.y);
        jobs[e].res[i] = rh[(size_t)e * m + i] / anorm[e];
        worst = std::max(worst, jobs[e].res[i]);
      }
      worst_all = std::max(worst_all, worst);
      jobs[e].its = it;
      if (worst <= tol) {
        jobs[e].status = OV_OK;
        fin[e] = 1;
        ECK(cudaMemcpyAsync(jobs[e].Rout, T1 + off[e], sizeof(double2) * n[e] * m, cudaMemcpyDeviceToDevice, st));
      }
      // next filter interval: damp everything beyond the block's largest Ritz value of A^2;
      // one in the upper half of [0, bound] means vectors from the top of the spectrum were
      // amplified: widen the bound and start the interval afresh
      if (t2[e] > 0.5 * amax2[e]) {
        amax2[e] = std::max(2.0 * amax2[e], 1.25 * t2[e]);
        anorm[e] = sqrt(amax2[e]);
        a_cut[e] = 0.05 * amax2[e];
      } else {
        a_cut[e] = std::min(std::max(t2[e], 1e-6 * amax2[e]), 0.9 * amax2[e]);
      }
    }
    if (verbose) {
      const int e0 = act[0];  // the first active job in detail, with the interval for the next iteration
      fprintf(stderr,
              "{\"ov_eig\": %d, \"degree\": %d, \"active\": %d, \"worst_residual\": %.3e, \"job\": %d, "
              "\"amax2\": %.4g, \"t2\": %.4g, \"cut\": %.4g, \"abs_lambda\": [%.6g, %.6g, %.6g], "
              "\"res\": [%.3e, %.3e, %.3e], \"s_filter\": %.4f, \"s_orth_rr2\": %.4f, \"s_rr1\": %.4f}\n",
              it, dgo, (int)act.size(), worst_all, e0, amax2[e0], t2[e0], a_cut[e0], std::abs(jobs[e0].lam[0]),
              std::abs(jobs[e0].lam[m / 2]), std::abs(jobs[e0].lam[m - 1]), jobs[e0].res[0], jobs[e0].res[m / 2],
              jobs[e0].res[m - 1], secs(t_start, t_filter), secs(t_filter, t_rr2), secs(t_rr2, clk::now()));
    }
    drop(fin);
  }
  // jobs still active: the best vectors of the last iteration (in T1)
  for (int e : act)
    ECK(cudaMemcpyAsync(jobs[e].Rout, T1 + off[e], sizeof(double2) * n[e] * m, cudaMemcpyDeviceToDevice, st));
  ECK(cudaStreamSynchronize(st));
  cleanup();
#undef ECK
#undef RCK
  return OV_OK;
}

}  // namespace ov
